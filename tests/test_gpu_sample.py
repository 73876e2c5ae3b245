"""GPU shot sampling against the oracle's sampler on the same state and the
same uniforms: every sample is the oracle's, except where the uniform falls
within rounding of a cumulative-probability boundary (then it must be one
of the two neighbouring outcomes); counts equal the histogram of samples."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch  # noqa: F401
    import paper_2406_03466_gb300 as m
    return m


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [3, 10, 15])
def test_sampling_matches_oracle(sv, dtype, n):
    import torch
    w = wl.ddcl(n, 1, seed=n)
    circ = sv.Circuit(n, w.gates, w.n_params, 0)
    st = sv.sv_alloc(n, 2, dtype)
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda").reshape(1, -1)
    sv.sv_apply_circuit_batch(st, [circ], sv.make_slots([(0, 0, -1, -1, 0, 0.0),
                                                         (0, 0, 0, -1, 0, 0.7)]), th)
    u = np.random.default_rng(n).random(5000)
    ud = torch.as_tensor(u, device="cuda")
    for row in (0, 1):
        samples, counts = sv.sv_sample(st, row, ud, counts=True)
        got = samples.cpu().numpy()
        psi = st.tensor[row].cpu().numpy()
        want, cdf = oracle.sample_shots(psi, u)
        diff = np.nonzero(got != want)[0]
        x = u * cdf[-1]
        for i in diff:  # only at a rounding boundary, and a neighbour
            assert abs(got[i] - want[i]) == 1
            assert abs(cdf[min(got[i], want[i])] - x[i]) < 1e-12 * cdf[-1]
        assert len(diff) <= 2
        assert np.array_equal(counts.cpu().numpy(), np.bincount(got, minlength=1 << n))
        vals, cnt = sv.bitstring_counts(samples)
        assert int(cnt.sum()) == len(u) and np.all(np.diff(vals.cpu().numpy()) > 0)


def test_sampling_basis_state_and_no_shots(sv):
    import torch
    n = 12
    st = sv.sv_alloc(n, 1, "c64")
    st.tensor.zero_()
    st.tensor[0, 1234] = 1.0
    u = torch.rand(1000, dtype=torch.float64, device="cuda")
    samples, counts = sv.sv_sample(st, 0, u, counts=True)
    assert bool((samples == 1234).all()) and int(counts[1234]) == 1000
    s0, _ = sv.sv_sample(st, 0, u[:0])
    assert s0.numel() == 0
