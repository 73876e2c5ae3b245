"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: complex128 paths <= 1e-12 relative to max(1, |reference|);
complex64 paths <= 1e-5 on energies and losses, <= 1e-4 on gradients,
2e-5 on amplitudes (products in FP32, reductions in FP64).
"""
import ctypes
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"c128": dict(E=1e-12, G=1e-12, A=1e-12), "c64": dict(E=1e-5, G=1e-4, A=2e-5)}


@pytest.fixture(scope="module")
def sv():
    import torch  # noqa: F401
    import paper_2406_03466_gb300 as m
    return m


def close(got, want, tol):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(1.0, float(np.max(np.abs(want)))) if want.size else 1.0
    err = float(np.max(np.abs(got - want))) if want.size else 0.0
    assert err <= tol * scale, f"max err {err:.3e} > {tol:.1e} x {scale:.3g}"


def theta_of(w):
    import torch
    return torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")


SMALL = {
    "vqe4": lambda: wl.vqe_random_pauli(4, 2, 10),
    "mcvqe8": lambda: wl.mcvqe(8, 4),
    "mcvqe6_nn": lambda: wl.mcvqe(6, 3, "nn+nnn", n_refs=4),
    "qcl6": lambda: wl.qcl(6, 2, 7),
    "qcl10": lambda: wl.qcl(10, 2, 5),
    "rand5": lambda: wl.random_workload(5, 70, 9, 3, seed=11, with_encoding=True),
    "rand7_mse": lambda: wl.random_workload(7, 90, 6, 4, seed=12, cost="mse"),
    "rand1": lambda: wl.random_workload(1, 12, 3, 2, seed=13),
    "rand2": lambda: wl.random_workload(2, 25, 5, 3, seed=14),
    "rand12": lambda: wl.random_workload(12, 40, 4, 2, seed=15),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_param_shift_gradient(sv, name, dtype):
    w = SMALL[name]()
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    l_, e_, g_ = sv.sv_grad_param_shift(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL[dtype]["E"])
    close(l_.cpu().numpy()[0], L, TOL[dtype]["E"])
    close(g_.cpu().numpy()[: w.n_params], g, TOL[dtype]["G"])


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_gradient(sv, name, dtype):
    w = SMALL[name]()
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL[dtype]["E"])
    close(l_.cpu().numpy()[0], L, TOL[dtype]["E"])
    close(g_.cpu().numpy()[: w.n_params], g, TOL[dtype]["G"])


@pytest.mark.parametrize("name", ["vqe4", "rand5", "rand2", "qcl6"])
def test_plain_form(sv, name):
    w = SMALL[name]()
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, "c128")
    l_, e_, g_ = sv.sv_grad_param_shift_plain(prob, theta_of(w))
    close(e_.cpu().numpy(), E, 1e-12)
    close(g_.cpu().numpy()[: w.n_params], g, 1e-12)


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_and_expect(sv, name, dtype):
    import torch
    w = SMALL[name]()
    d = 0 if w.inputs is None else w.inputs.shape[1]
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    obs = sv.PauliSum(w.n_qubits, w.pauli_letters, w.pauli_coeffs)
    I = w.n_instances
    rows = []
    for i in range(I):
        sp = (3 * i) % w.n_params if w.n_params else -1
        rows.append((0, 0, sp, i if d else -1, int(w.refs[i]), 0.25 * (i + 1)))
    slots = sv.make_slots(rows)
    st = sv.sv_alloc(w.n_qubits, I, dtype)
    th = theta_of(w).reshape(1, -1) if w.n_params else torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    xin = None if w.inputs is None else torch.as_tensor(w.inputs, device="cuda")
    sv.sv_apply_circuit_batch(st, [circ], slots, th, xin)
    out = sv.sv_expect_pauli_sum(st, obs)
    amps = st.tensor.cpu().numpy()
    for i, (c, tr, sp, ir, ref, sh) in enumerate(rows):
        psi = oracle.state(w, instance=i, shift_param=sp, shift=sh)
        close(amps[i], psi, TOL[dtype]["A"])
        e_ref = oracle.expect_state(psi, w.pauli_letters, w.pauli_coeffs).real
        close(out.cpu().numpy()[i], e_ref, TOL[dtype]["E"])


@pytest.mark.parametrize("reg_bits", [1, 2, 3, 4])
@pytest.mark.parametrize("tpb", [0, 512])
@pytest.mark.parametrize("no_fusion", [False, True])
def test_plan_invariance(sv, reg_bits, tpb, no_fusion):
    """The same gradient under every register width, block size and fusion mode."""
    w = wl.mcvqe(8, 3)
    L, E, g = oracle.grad_param_shift(w)
    opts = sv.plan_opts(reg_bits, tpb, no_fusion)
    for dtype in ("c64", "c128"):
        if dtype == "c128" and reg_bits > 3:
            continue
        prob = sv.Problem.from_spec(w, dtype, opts=opts)
        for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint):
            l_, e_, g_ = fn(prob, theta_of(w))
            close(g_.cpu().numpy(), g, TOL[dtype]["G"])
            close(e_.cpu().numpy(), E, TOL[dtype]["E"])


def test_autograd_function(sv):
    import torch
    from paper_2406_03466_gb300.autograd import energies
    w = wl.qcl(6, 2, 9)
    prob = sv.Problem.from_spec(w, "c64")
    th = theta_of(w).clone().requires_grad_(True)
    y = torch.as_tensor(w.targets, device="cuda")
    E = energies(th, prob)
    loss = ((E - y) ** 2).mean()
    loss.backward()
    L, _, g = oracle.grad_param_shift(w)
    close(loss.item(), L, 1e-5)
    close(th.grad.cpu().numpy(), g, 1e-4)


def test_full_config1(sv):
    """Plain parameter-shift gradient, 4 qubits, complex128: all paths."""
    w = wl.config(0)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, "c128")
    for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint, sv.sv_grad_param_shift_plain):
        l_, e_, g_ = fn(prob, theta_of(w))
        close(g_.cpu().numpy(), g, 1e-12)
        close(l_.cpu().numpy()[0], L, 1e-12)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_full_config2(sv, dtype):
    """Multi-contracted VQE, 8 qubits, 585 circuits in one batched launch."""
    w = wl.config(1)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint):
        l_, e_, g_ = fn(prob, theta_of(w))
        close(g_.cpu().numpy(), g, TOL[dtype]["G"])
        close(e_.cpu().numpy(), E, TOL[dtype]["E"])


def test_full_config3_sampled(sv):
    """Circuit learning, 12 qubits, 256 x 433 circuits: the full batch on the
    GPU, sampled gradient entries from the oracle, adjoint vs parameter shift."""
    w = wl.config(2)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_, g_ = sv.sv_grad_param_shift(prob, theta_of(w))
    la, ea, ga = sv.sv_grad_adjoint(prob, theta_of(w))
    E = oracle.instance_energies(w)
    close(e_.cpu().numpy(), E, 1e-5)
    close(ea.cpu().numpy(), E, 1e-5)
    close(l_.cpu().numpy()[0], oracle.cost_from_energies(w, E), 1e-5)
    ks = [0, 1, 37, 108, 215]
    _, _, g_sub = oracle.grad_param_shift(w, params=ks)
    close(g_.cpu().numpy()[ks], g_sub, 1e-4)
    close(ga.cpu().numpy()[ks], g_sub, 1e-4)
    close(ga.cpu().numpy(), g_.cpu().numpy(), 1e-4)


def test_errors_are_reported(sv):
    import torch
    w = wl.vqe_random_pauli(4, 2, 10)
    prob = sv.Problem.from_spec(w, "c64")
    grad = torch.empty(w.n_params, dtype=torch.float64, device="cuda")
    st = sv.library().sv_grad_param_shift(ctypes.byref(prob.struct), None, None, None,
                                          ctypes.c_void_p(grad.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sv.SV_ERR_ARG and "theta" in sv.sv_last_error()
    bad = wl.vqe_random_pauli(4, 2, 10)
    bad.refs = np.array([1 << 4])
    with pytest.raises(sv.SvError):
        sv.sv_grad_adjoint(sv.Problem.from_spec(bad, "c64"), theta_of(w))
    big = wl.random_workload(16, 10, 2, 1, seed=1)
    with pytest.raises(sv.SvError):  # tiles larger than 2^12 amplitudes are not offered
        sv.sv_grad_adjoint(sv.Problem.from_spec(big, "c64", opts=sv.plan_opts(tile_bits=13)),
                           theta_of(big))
    sv.sv_sync_status()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotune_keeps_results(sv, dtype):
    """The autotuner picks a launch shape; results under it still match."""
    w = wl.mcvqe(8, 4)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    sv.sv_autotune(prob, theta_of(w))
    for kind in (1, 2):
        R, tpb, us = sv.sv_tuned_shape(prob, kind)
        assert 1 <= R <= 4 and 32 <= tpb <= 512 and us > 0
    for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint):
        l_, e_, g_ = fn(prob, theta_of(w))
        close(g_.cpu().numpy(), g, TOL[dtype]["G"])
        close(e_.cpu().numpy(), E, TOL[dtype]["E"])


def test_energies_entry(sv):
    w = wl.qcl(8, 2, 11)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_ = sv.sv_energies(prob, theta_of(w))
    E = oracle.instance_energies(w)
    close(e_.cpu().numpy(), E, 1e-5)
    close(l_.cpu().numpy()[0], oracle.cost_from_energies(w, E), 1e-5)
    B = sv.sv_param_shift_energies(prob, theta_of(w)).cpu().numpy()
    inst, sp, sh = oracle.param_shift_slots(w)
    close(B, oracle.energies(w, None, inst, sp, sh), 1e-5)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [8, 14])
def test_param_shift_host_buffers(sv, dtype, n):
    """The host-buffer entry point against the oracle, on chip (8 qubits) and
    as tile passes (14 qubits); bitwise equal to the device-buffer call on
    chip (the tile passes sum energies with FP64 atomics, in any order)."""
    import torch
    w = wl.mcvqe(n, 2) if n == 8 else wl.mcvqe(n, 2, "nn+nnn", n_refs=2)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    th = torch.as_tensor(w.theta, dtype=torch.float64)
    l_, e_, g_ = sv.sv_grad_param_shift_host(prob, th)
    assert l_.device.type == "cpu" and g_.device.type == "cpu"
    close(e_.numpy(), E, TOL[dtype]["E"])
    close(l_.numpy()[0], L, TOL[dtype]["E"])
    close(g_.numpy()[: w.n_params], g, TOL[dtype]["G"])
    ld, ed, gd = sv.sv_grad_param_shift(prob, theta_of(w))
    if n == 8:
        assert np.array_equal(gd.cpu().numpy(), g_.numpy())
        assert np.array_equal(ed.cpu().numpy(), e_.numpy())
    else:
        close(gd.cpu().numpy(), g_.numpy(), 1e-12 if dtype == "c128" else 1e-6)
    # outputs may be left out, and the call repeats with new theta
    th2 = th + 0.25
    g2 = torch.empty(w.n_params, dtype=torch.float64)
    sv.sv_grad_param_shift_host(prob, th2, None, None, g2)
    w2 = dataclasses.replace(w, theta=th2.numpy())
    close(g2.numpy(), oracle.grad_param_shift(w2)[2], TOL[dtype]["G"])
    with pytest.raises(ValueError):
        sv.sv_grad_param_shift_host(prob, theta_of(w))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [8, 15])
def test_adjoint_host_buffers(sv, dtype, n):
    """The host-buffer adjoint entry point against the oracle, on chip (8
    qubits) and as tile passes (15 qubits), and against the device-buffer
    call; outputs may be left out and the call repeats with a new theta."""
    import torch
    w = wl.mcvqe(n, 2) if n == 8 else wl.mcvqe(n, 2, "nn+nnn", n_refs=2)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    th = torch.as_tensor(w.theta, dtype=torch.float64)
    l_, e_, g_ = sv.sv_grad_adjoint_host(prob, th)
    assert l_.device.type == "cpu" and g_.device.type == "cpu"
    close(e_.numpy(), E, TOL[dtype]["E"])
    close(l_.numpy()[0], L, TOL[dtype]["E"])
    close(g_.numpy()[: w.n_params], g, TOL[dtype]["G"])
    ld, ed, gd = sv.sv_grad_adjoint(prob, theta_of(w))
    close(gd.cpu().numpy(), g_.numpy(), 1e-12 if dtype == "c128" else 1e-6)
    th2 = th - 0.4
    g2 = torch.empty(w.n_params, dtype=torch.float64)
    sv.sv_grad_adjoint_host(prob, th2, None, None, g2)
    w2 = dataclasses.replace(w, theta=th2.numpy())
    close(g2.numpy(), oracle.grad_param_shift(w2)[2], TOL[dtype]["G"])
    with pytest.raises(ValueError):
        sv.sv_grad_adjoint_host(prob, theta_of(w))


def test_whole_warp_blocks(sv):
    """A batch whose default launch would put 3 circuits of 16 threads in a
    block (48 threads) runs in whole warps and matches the oracle; a
    threads_per_block that is not a multiple of 32 is rejected."""
    w = wl.random_workload(6, 200, 6, 5, seed=7)
    assert 609 <= w.n_slots_param_shift <= 912  # ceil(B / 304) == 3
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_, g_ = sv.sv_grad_param_shift(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL["c64"]["E"])
    close(g_.cpu().numpy()[: w.n_params], g, TOL["c64"]["G"])
    bad = sv.Problem.from_spec(w, "c64", opts=sv.plan_opts(reg_bits=2, threads_per_block=48))
    with pytest.raises(sv.SvError):
        sv.sv_grad_param_shift(bad, theta_of(w))


def test_repeatable(sv):
    """A fixed plan gives bitwise identical results run to run."""
    w = wl.mcvqe(8, 4)
    prob = sv.Problem.from_spec(w, "c64")
    a = [sv.sv_grad_param_shift(prob, theta_of(w))[2].cpu().numpy() for _ in range(3)]
    assert all(np.array_equal(a[0], x) for x in a[1:])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("cfg", [1, 3])
def test_param_shift_segments_and_combine(sv, dtype, cfg):
    """Segments of the parameter-shift batch (one per virtual QPU) assembled
    and combined give sv_grad_param_shift's result."""
    import torch
    from paper_2406_03466_gb300 import vqpu
    w = wl.config(cfg) if cfg != 3 else wl.mcvqe(14, 1, "nn+nnn", n_refs=2)
    prob = sv.Problem.from_spec(w, dtype)
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    B = (2 * w.n_params + 1) * w.n_instances
    parts = [sv.sv_param_shift_energies_range(prob, th, *(lambda lo, hi: (lo, hi - lo))(
        *vqpu.segment(B, 3, r))) for r in range(3)]
    E = torch.cat(parts).contiguous()
    l1, e1, g1 = sv.sv_param_shift_combine(prob, E)
    l2, e2, g2 = sv.sv_grad_param_shift(prob, th)
    tol = 1e-12 if dtype == "c128" else 1e-5
    np.testing.assert_allclose(g1.cpu().numpy(), g2.cpu().numpy(), atol=tol * 10)
    np.testing.assert_allclose(e1.cpu().numpy(), e2.cpu().numpy(), atol=tol)
    np.testing.assert_allclose(l1.cpu().numpy(), l2.cpu().numpy(), atol=tol)
    l3, e3, g3 = vqpu.param_shift_gradient(prob, th)  # single process: the whole batch
    np.testing.assert_allclose(g3.cpu().numpy(), g2.cpu().numpy(), atol=tol * 10)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_paper_mcvqe_circuit(sv, dtype):
    """The paper's MC-VQE circuit (CIS references as per-instance inputs,
    merged entanglers): parameter shift and adjoint against the oracle."""
    import torch
    w = wl.mcvqe_paper(8, n_refs=3, seed=2)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    tol = {"c128": (1e-12, 1e-12), "c64": (1e-5, 1e-4)}[dtype]
    for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint):
        l_, e_, g_ = fn(prob, th)
        close(e_.cpu().numpy(), E, tol[0])
        close(g_.cpu().numpy()[: w.n_params], g, tol[1])


def test_paper_mcvqe_circuit_tiles(sv):
    import torch
    w = wl.mcvqe_paper(16, n_refs=2, seed=4)
    prob = sv.Problem.from_spec(w, "c64")
    th = torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")
    l_, e_, g_ = sv.sv_grad_adjoint(prob, th)
    ks = [0, 11, 40, 75]
    _, E, gs = oracle.grad_param_shift(w, params=ks)
    close(e_.cpu().numpy(), E, 1e-5)
    close(g_.cpu().numpy()[ks], gs, 1e-4)
