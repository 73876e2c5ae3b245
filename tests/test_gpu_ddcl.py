"""GPU parity of data-driven circuit learning (Sec. 4.2, Eq. 3) against the
oracle: the JS divergence of the output distribution and its adjoint
gradient (through the C ABI), complex64 and complex128."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"c128": dict(E=1e-12, G=1e-12), "c64": dict(E=1e-5, G=1e-4)}


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


def run(sv, w, dtype, opts=None):
    import torch
    prob = sv.Problem.from_spec(w, dtype, opts=opts)
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    tg = torch.as_tensor(w.target_dist, dtype=torch.float64, device="cuda")
    js, g = sv.sv_grad_ddcl(prob, th, tg)
    return float(js.cpu()[0]), g.cpu().numpy()[: w.n_params]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,layers", [(8, 2), (9, 1), (10, 2)])
def test_ddcl_matches_oracle(sv, dtype, n, layers):
    w = wl.ddcl(n, layers, seed=n)
    js_o, g_o = oracle.ddcl_grad_param_shift(w)
    js, g = run(sv, w, dtype)
    close(js, js_o, TOL[dtype]["E"])
    close(g, g_o, TOL[dtype]["G"])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_ddcl_forced_small_tiles(sv, dtype):
    w = wl.ddcl(10, 2, seed=3)
    js_o, g_o = oracle.ddcl_grad_param_shift(w)
    js, g = run(sv, w, dtype, opts=sv.plan_opts(tile_bits=8, reg_bits=3 if dtype == "c64" else 2))
    close(js, js_o, TOL[dtype]["E"])
    close(g, g_o, TOL[dtype]["G"])


def test_ddcl_fourteen_qubits_sampled(sv):
    w = wl.ddcl(14, 1, seed=14)
    ks = [0, 13, 40, 83]
    js_o, g_o = oracle.ddcl_grad_param_shift(w, params=ks)
    js, g = run(sv, w, "c64")
    close(js, js_o, 1e-5)
    close(g[ks], g_o, 1e-4)


def test_ddcl_zero_gradient_at_its_own_output(sv):
    w0 = wl.ddcl(9, 2, seed=6)
    w = wl.ddcl(9, 2, seed=6, target=oracle.output_distribution(w0))
    js, g = run(sv, w, "c128")
    assert abs(js) < 1e-12 and np.max(np.abs(g)) < 1e-10


def run_ps(sv, w, dtype, opts=None):
    import torch
    prob = sv.Problem.from_spec(w, dtype, opts=opts)
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    tg = torch.as_tensor(w.target_dist, dtype=torch.float64, device="cuda")
    js, g = sv.sv_grad_ddcl_param_shift(prob, th, tg)
    return float(js.cpu()[0]), g.cpu().numpy()[: w.n_params]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,layers,opts", [(8, 2, None), (10, 2, (8, 2)), (9, 1, None)])
def test_ddcl_param_shift_form(sv, dtype, n, layers, opts):
    """The paper's form of the gradient (2 N_theta shifted circuits and the
    derivative table of the unshifted one) against the oracle's parameter
    shift, and against the adjoint form on the device."""
    w = wl.ddcl(n, layers, seed=n)
    o = None if opts is None else sv.plan_opts(tile_bits=opts[0], reg_bits=opts[1])
    js_o, g_o = oracle.ddcl_grad_param_shift(w)
    js, g = run_ps(sv, w, dtype, o)
    close(js, js_o, TOL[dtype]["E"])
    close(g, g_o, TOL[dtype]["G"])
    js_a, g_a = run(sv, w, dtype, o)
    close(g, g_a, TOL[dtype]["G"])
