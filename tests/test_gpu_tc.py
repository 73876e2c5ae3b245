"""GPU parity of the tensor-core forward passes (sv_plan_opts.tensor_blocks)
and the bounded-wait error path.

With tensor_blocks every register stage of a forward tile pass runs as one
dense 16 x 16 complex block on the tensor cores (tcgen05, 3xTF32 split, FP32
accumulation).  States, energies and gradients (whose forward sweep runs on
the tensor cores) are compared with the oracle at the complex64 tolerances of
the other GPU tests, on complex Rx-Rz-Rx layers (circuit learning) and real
Ry layers (MC-VQE), with tiles of 2^11 and 2^12 amplitudes, and with the
register path on the same plan.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = dict(E=1e-5, G=1e-4, A=2e-5)


@pytest.fixture(scope="module")
def sv():
    import torch  # noqa: F401
    import paper_2406_03466_gb300 as m
    return m


def close(got, want, tol):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(1.0, float(np.max(np.abs(want))))
    err = float(np.max(np.abs(got - want)))
    assert err <= tol * scale, f"max err {err:.3e} > {tol:.1e} x {scale:.3g}"


def theta_of(w):
    import torch
    return torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")


def states_of(sv, w, opts, rows):
    import torch
    d = 0 if w.inputs is None else 1
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    st = sv.sv_alloc(w.n_qubits, len(rows), "c64")
    xin = None if w.inputs is None else torch.as_tensor(w.inputs, device="cuda")
    sv.sv_apply_circuit_batch(st, [circ], sv.make_slots(rows), theta_of(w).reshape(1, -1), xin,
                              opts)
    sv.sv_sync_status()
    return st.tensor.cpu().numpy()


CASES = {
    "qcl14": lambda: wl.qcl(14, 3, 3),
    "mcvqe15": lambda: wl.mcvqe(15, 3, "nn+nnn", n_refs=3),
    "rand14_enc": lambda: wl.random_workload(14, 120, 6, 3, seed=61, with_encoding=True),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tile_bits", [11, 12])
def test_tensor_block_states_match_oracle(sv, name, tile_bits):
    w = CASES[name]()
    d = 0 if w.inputs is None else 1
    rows = [(0, 0, (3 * i) % w.n_params, i if d else -1, int(w.refs[i]), 0.2 * (i + 1))
            for i in range(w.n_instances)]
    tc = sv.plan_opts(reg_bits=4, tile_bits=tile_bits, tensor_blocks=True)
    amps = states_of(sv, w, tc, rows)
    for i, r in enumerate(rows):
        want = oracle.state(w, instance=i, shift_param=r[2], shift=r[5])
        close(amps[i], want, TOL["A"])
        assert abs(np.linalg.norm(amps[i]) - 1.0) < 1e-5
    reg = states_of(sv, w, sv.plan_opts(reg_bits=4, tile_bits=tile_bits), rows)
    close(amps, reg, TOL["A"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_tensor_block_gradients_match_oracle(sv, name):
    """Energies by tile passes and the adjoint gradient (forward sweep on the
    tensor cores, reverse sweep on registers) against the oracle."""
    w = CASES[name]()
    prob = sv.Problem.from_spec(w, "c64",
                                opts=sv.plan_opts(reg_bits=4, tile_bits=11, tensor_blocks=True))
    L, E, g = oracle.grad_param_shift(w)
    l_, e_ = sv.sv_energies(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL["E"])
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w))
    sv.sv_sync_status()
    close(e_.cpu().numpy(), E, TOL["E"])
    close(l_.cpu().numpy()[0], L, TOL["E"])
    close(g_.cpu().numpy()[: w.n_params], g, TOL["G"])


def test_tensor_blocks_circuit_learning_20_qubits(sv):
    """The 20-qubit circuit-learning family at full depth (10 layers of
    Rx-Rz-Rx, the benchmark's gate application) on 2 inputs: tensor-core
    states against the register path, and the instance energies against
    the oracle."""
    w = wl.qcl(20, 10, 2)
    rows = [(0, 0, -1, i, 0, 0.0) for i in range(2)]
    a_tc = states_of(sv, w, sv.plan_opts(reg_bits=4, tile_bits=12, tensor_blocks=True), rows)
    a_reg = states_of(sv, w, sv.plan_opts(reg_bits=4, tile_bits=12), rows)
    close(a_tc, a_reg, TOL["A"])
    prob = sv.Problem.from_spec(w, "c64",
                                opts=sv.plan_opts(reg_bits=4, tile_bits=12, tensor_blocks=True))
    l_, e_ = sv.sv_energies(prob, theta_of(w))
    close(e_.cpu().numpy(), oracle.instance_energies(w), TOL["E"])


def test_tensor_blocks_rejected_where_unsupported(sv):
    import torch
    w = wl.mcvqe(14, 1, "nn+nnn", n_refs=1)
    for dtype, opts in (("c128", sv.plan_opts(reg_bits=3, tile_bits=11, tensor_blocks=True)),
                        ("c64", sv.plan_opts(reg_bits=3, tile_bits=11, tensor_blocks=True)),
                        ("c64", sv.plan_opts(reg_bits=4, tile_bits=10, tensor_blocks=True))):
        prob = sv.Problem.from_spec(w, dtype, opts=opts)
        with pytest.raises(sv.SvError) as ei:
            sv.sv_energies(prob, torch.as_tensor(w.theta, device="cuda"))
        assert ei.value.status == sv.SV_ERR_UNSUPPORTED


def test_bounded_wait_expiry_reports_timeout_and_context_survives(sv):
    """A wait that nothing completes gives up after its limit, the next
    sv_sync_status reports SV_ERR_TIMEOUT once, and the context keeps
    working (a gradient afterwards matches the oracle)."""
    sv.sv_sync_status()
    sv.sv_debug_wait_expiry(1000)
    with pytest.raises(sv.SvError) as ei:
        sv.sv_sync_status()
    assert ei.value.status == sv.SV_ERR_TIMEOUT
    sv.sv_sync_status()  # cleared
    w = wl.vqe_random_pauli(4, 2, 10)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_, g_ = sv.sv_grad_param_shift(prob, theta_of(w))
    close(g_.cpu().numpy()[: w.n_params], oracle.grad_param_shift(w)[2], TOL["G"])


def test_autotuner_may_pick_tensor_blocks(sv):
    """sv_autotune times tensor-core candidates beside the register shapes
    for complex64 states in device memory; whatever it picks matches the
    oracle."""
    w = wl.qcl(16, 2, 2)
    prob = sv.Problem.from_spec(w, "c64")
    sv.sv_autotune(prob, theta_of(w), 3)
    for kind in (1, 2):
        t, R, tc, us = sv.sv_tuned_tile(prob, kind)
        assert 10 <= t <= 12 and 3 <= R <= 4 and us > 0
        if tc:
            assert R == 4 and t in (11, 12)
    L, E, g = oracle.grad_param_shift(w, params=[0, 17, 40])
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL["E"])
    close(g_.cpu().numpy()[[0, 17, 40]], g, TOL["G"])
