"""GPU parity of the tile-pass path (states in device memory) against the oracle.

Small states are forced through tile passes with `tile_bits` so that every
tile size, register width and checkpoint interval is compared with the CPU
oracle; 14-qubit states take the path on their own; reduced circuit-learning
and multi-contracted VQE workloads at 16-20 qubits check sampled gradient
entries; the benchmark's 28-qubit workload itself is checked at full size
through properties that hold at any size (the closed form at theta = 0, and
the complex64 adjoint against complex128 parameter shift on a subsample) and
against the sparse-state oracle at angles where few qubits rotate; the
20-qubit circuit-learning workload at full depth against the dense oracle on
sampled instances and parameters.
Tolerances as in test_gpu_parity.
"""
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
    scale = max(1.0, float(np.max(np.abs(want))))
    err = float(np.max(np.abs(got - want)))
    assert err <= tol * scale, f"max err {err:.3e} > {tol:.1e} x {scale:.3g}"


def theta_of(w):
    import torch
    return torch.as_tensor(w.theta, dtype=torch.float64, device="cuda")


FORCED = {
    "qcl9": lambda: wl.qcl(9, 3, 3),
    "mcvqe9_nn": lambda: wl.mcvqe(9, 3, "nn+nnn", n_refs=3),
    "rand8_enc": lambda: wl.random_workload(8, 90, 7, 3, seed=31, with_encoding=True),
    "rand10_mse": lambda: wl.random_workload(10, 70, 5, 2, seed=32, cost="mse"),
}


@pytest.mark.parametrize("name", sorted(FORCED))
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("tile_bits,reg_bits", [(7, 2), (8, 3), (8, 2), (9, 3)])
def test_forced_tiles_gradients(sv, name, dtype, tile_bits, reg_bits):
    w = FORCED[name]()
    L, E, g = oracle.grad_param_shift(w)
    opts = sv.plan_opts(reg_bits=reg_bits, tile_bits=tile_bits)
    prob = sv.Problem.from_spec(w, dtype, opts=opts)
    l_, e_, g_ = sv.sv_grad_param_shift(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL[dtype]["E"])
    close(g_.cpu().numpy()[: w.n_params], g, TOL[dtype]["G"])
    for every in (1, 2, 0):
        l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w), checkpoint_every=every)
        close(e_.cpu().numpy(), E, TOL[dtype]["E"])
        close(l_.cpu().numpy()[0], L, TOL[dtype]["E"])
        close(g_.cpu().numpy()[: w.n_params], g, TOL[dtype]["G"])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_forced_tiles_states_and_energies(sv, dtype):
    import torch
    w = wl.random_workload(9, 60, 6, 3, seed=33, with_encoding=True)
    opts = sv.plan_opts(tile_bits=7)
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, 1)
    rows = [(0, 0, (2 * i) % w.n_params, i, int(w.refs[i]), 0.3 * (i + 1)) for i in range(3)]
    st = sv.sv_alloc(w.n_qubits, 3, dtype)
    xin = torch.as_tensor(w.inputs, device="cuda")
    sv.sv_apply_circuit_batch(st, [circ], sv.make_slots(rows), theta_of(w).reshape(1, -1), xin, opts)
    amps = st.tensor.cpu().numpy()
    for i, r in enumerate(rows):
        close(amps[i], oracle.state(w, instance=i, shift_param=r[2], shift=r[5]), TOL[dtype]["A"])
    prob = sv.Problem.from_spec(w, dtype, opts=opts)
    l_, e_ = sv.sv_energies(prob, theta_of(w))
    close(e_.cpu().numpy(), oracle.instance_energies(w), TOL[dtype]["E"])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_fourteen_qubits_take_tiles(sv, dtype):
    """Just beyond the on-chip limit: the default tile path, full gradient."""
    w = wl.mcvqe(14, 2, "nn+nnn", n_refs=2)
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, dtype)
    for fn in (sv.sv_grad_param_shift, sv.sv_grad_adjoint):
        l_, e_, g_ = fn(prob, theta_of(w))
        close(e_.cpu().numpy(), E, TOL[dtype]["E"])
        close(g_.cpu().numpy(), g, TOL[dtype]["G"])


def test_expect_pauli_sum_large_state(sv):
    import torch
    w = wl.mcvqe(15, 1, "nn+nnn", n_refs=2)
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, 0)
    obs = sv.PauliSum(w.n_qubits, w.pauli_letters, w.pauli_coeffs)
    st = sv.sv_alloc(w.n_qubits, 2, "c64")
    rows = [(0, 0, -1, -1, int(w.refs[i]), 0.0) for i in range(2)]
    sv.sv_apply_circuit_batch(st, [circ], sv.make_slots(rows), theta_of(w).reshape(1, -1))
    out = sv.sv_expect_pauli_sum(st, obs)
    close(out.cpu().numpy(), oracle.instance_energies(w), 1e-5)


def test_circuit_learning_20_qubits_sampled(sv):
    """Reduced circuit learning at 20 qubits (2 layers, 3 inputs): the adjoint
    gradient against oracle parameter-shift entries."""
    w = wl.qcl(20, 2, 3)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w), checkpoint_every=2)
    E = oracle.instance_energies(w)
    close(e_.cpu().numpy(), E, 1e-5)
    ks = [0, 17, 60, 119]
    _, _, gs = oracle.grad_param_shift(w, params=ks)
    close(g_.cpu().numpy()[ks], gs, 1e-4)


def test_mcvqe_16_qubits_adjoint_vs_param_shift(sv):
    w = wl.mcvqe(16, 2, "nn+nnn", n_refs=3)
    prob = sv.Problem.from_spec(w, "c64")
    la, ea, ga = sv.sv_grad_adjoint(prob, theta_of(w))
    lp, ep, gp = sv.sv_grad_param_shift(prob, theta_of(w))
    close(ga.cpu().numpy(), gp.cpu().numpy(), 1e-4)
    close(ea.cpu().numpy(), oracle.instance_energies(w), 1e-5)
    ks = [0, 9, 31]
    _, _, gs = oracle.grad_param_shift(w, params=ks)
    close(ga.cpu().numpy()[ks], gs, 1e-4)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotuned_tile_shape(sv, dtype):
    """sv_autotune picks a tile shape for device-memory states; later calls
    use it and still match the oracle."""
    w = wl.mcvqe(14, 2, "nn+nnn", n_refs=2)
    prob = sv.Problem.from_spec(w, dtype)
    sv.sv_autotune(prob, theta_of(w), 3)
    for kind in (1, 2):
        R, tpb, us = sv.sv_tuned_shape(prob, kind)
        t = R + tpb.bit_length() - 1
        assert tpb == 1 << (t - R) and t - R >= 5 and 9 <= t <= 12 and us > 0
    L, E, g = oracle.grad_param_shift(w)
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL[dtype]["E"])
    close(g_.cpu().numpy(), g, TOL[dtype]["G"])
    l_, e_ = sv.sv_energies(prob, theta_of(w))
    close(e_.cpu().numpy(), E, TOL[dtype]["E"])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_uneven_batch_adjoint(sv, dtype):
    """Circuits of different qubit counts, depths and observables in one
    pass-major sequence; the second call replays the captured graph."""
    ws = [wl.qcl(14, 2, 3), wl.mcvqe(15, 3, "nn+nnn", n_refs=2), wl.qcl(16, 1, 2),
          wl.random_workload(14, 80, 6, 2, seed=51, with_encoding=True)]
    probs = [sv.Problem.from_spec(w, dtype) for w in ws]
    thetas = [theta_of(w) for w in ws]
    outs = sv.sv_grad_adjoint_multi(probs, thetas)
    for rep in range(2):
        for w, pr, th, (l_, e_, g_) in zip(ws, probs, thetas, outs):
            ls, es, gs = sv.sv_grad_adjoint(pr, th, checkpoint_every=1000)
            close(e_.cpu().numpy(), es.cpu().numpy(), TOL[dtype]["E"])
            close(g_.cpu().numpy(), gs.cpu().numpy(), TOL[dtype]["G"])
            close(l_.cpu().numpy(), ls.cpu().numpy(), TOL[dtype]["E"])
        for o in outs:  # the replay must rewrite every output
            for x in o:
                x.fill_(float("nan"))
        outs = sv.sv_grad_adjoint_multi(probs, thetas, outputs=outs)
    # every problem of the batch against the oracle: all instance energies,
    # the cost and sampled gradient entries (parameter shift on the CPU)
    for w, (l_, e_, g_) in zip(ws, outs):
        ks = sorted({0, w.n_params // 3, w.n_params // 2, w.n_params - 1})
        L, E, g = oracle.grad_param_shift(w, params=ks)
        close(e_.cpu().numpy(), E, TOL[dtype]["E"])
        close(l_.cpu().numpy()[0], L, TOL[dtype]["E"])
        close(g_.cpu().numpy()[ks], g, TOL[dtype]["G"])


# ------------------------------------------------ the 28-qubit workload itself

def _basis_state_at_zero_angles(w, ref):
    """The index of the basis state the circuit maps |ref> to when every
    rotation angle is 0 (rotations are then identities, CNOTs permute)."""
    b = [(int(ref) >> q) & 1 for q in range(w.n_qubits)]
    for g in w.gates:
        if g.op in ("RX", "RY", "RZ"):
            continue
        assert g.op == "CNOT", g.op
        b[g.target] ^= b[g.control]
    return sum(bit << q for q, bit in enumerate(b))


def _closed_form_energy(w, j):
    """<j|H|j> for a basis state: only terms without X or Y letters count,
    each with sign (-1)^(number of its Z letters on 1-bits of j)."""
    letters = np.asarray(w.pauli_letters)
    e = 0.0
    for row, c in zip(letters, w.pauli_coeffs):
        if np.any((row == 1) | (row == 2)):
            continue
        zs = [q for q in range(w.n_qubits) if row[q] == 3]
        e += c * (-1) ** sum((j >> q) & 1 for q in zs)
    return e


def test_mcvqe28_full_size_closed_form(sv):
    """The benchmark's 28-qubit multi-contracted VQE (8 states of 2 GiB), in
    the launch configuration the benchmark uses (autotuned tile passes): at
    theta = 0 every instance energy equals the closed form of its basis
    state."""
    import torch
    w = wl.config(4)
    prob = sv.Problem.from_spec(w, "c64")
    th = torch.zeros(w.n_params, dtype=torch.float64, device="cuda")
    l_, e_ = sv.sv_energies(prob, th)
    want = [_closed_form_energy(w, _basis_state_at_zero_angles(w, r)) for r in w.refs]
    close(e_.cpu().numpy(), want, TOL["c64"]["E"])


def test_mcvqe28_full_size_adjoint_vs_param_shift_c128(sv):
    """The 28-qubit adjoint gradient (complex64, relabeling passes, stored
    forward states) on a 16-parameter subsample against parameter shift in
    complex128 on the GPU (segments of the parameter-shift batch).  Two of
    the eight reference states keep the complex128 side (FP64 arithmetic,
    scarce on this GPU) to about 40 s; every state is a full 2^28 one."""
    import dataclasses
    import torch
    w8 = wl.config(4)
    w = dataclasses.replace(w8, refs=w8.refs[:2], weights=w8.weights[:2])
    th = theta_of(w)
    prob64 = sv.Problem.from_spec(w, "c64")
    g64 = sv.sv_grad_adjoint(prob64, th)[2].cpu().numpy()
    prob128 = sv.Problem.from_spec(w, "c128")
    I = w.n_instances
    wts = np.asarray(w.weights)
    ks = list(range(0, w.n_params, w.n_params // 16))[:16]
    for k in ks:
        seg = torch.empty(2 * I, dtype=torch.float64, device="cuda")
        sv.sv_param_shift_energies_range(prob128, th, I + 2 * k * I, 2 * I, seg)
        e = seg.cpu().numpy()
        g128 = float(np.dot(wts, 0.5 * (e[:I] - e[I:])))
        assert abs(g64[k] - g128) <= TOL["c64"]["G"] * max(1.0, abs(g128)), (k, g64[k], g128)


# Angles of the 28-qubit workload at which the sparse-state oracle is exact:
# qubit 0 rotates in every layer, qubit 17 in layers 2 and 5, qubit 27 in
# layer 3, every other angle is 0.  Sampled parameters: those rotations, and
# others on the same and neighbouring qubits (their derivatives at angle 0).
MCVQE28_ROTATING = [l * 28 for l in range(8)] + [2 * 28 + 17, 5 * 28 + 17, 3 * 28 + 27]
MCVQE28_SAMPLED = [0, 5, 10, 21, 27, 28, 33, 45, 50, 56, 73, 84, 87, 101, 111, 117, 140, 144, 157,
                   168, 172, 196, 222]


def test_mcvqe28_full_size_gradient_against_sparse_oracle(sv):
    """The benchmark's 28-qubit multi-contracted VQE at full size (8 states of
    2^28, 8 layers, 224 parameters, 268 terms) in the launch configuration
    the benchmark times (autotuned tile passes, relabeling plan, stored
    forward states): its complex64 adjoint energies, cost and sampled
    gradient entries against the sparse-state oracle's exact values."""
    import torch
    from oracle import sparse
    w = wl.config(4)
    th = np.zeros(w.n_params)
    th[MCVQE28_ROTATING] = w.theta[MCVQE28_ROTATING]
    th_dev = torch.as_tensor(th, dtype=torch.float64, device="cuda")
    prob = sv.Problem.from_spec(w, "c64")
    sv.sv_autotune(prob, th_dev, 2)
    l_, e_, g_ = sv.sv_grad_adjoint(prob, th_dev)
    L, E, g = sparse.grad_param_shift(w, th, params=MCVQE28_SAMPLED, workers=16)
    close(e_.cpu().numpy(), E, TOL["c64"]["E"])
    close(l_.cpu().numpy()[0], L, TOL["c64"]["E"])
    close(g_.cpu().numpy()[MCVQE28_SAMPLED], g, TOL["c64"]["G"])


def test_qcl20_full_depth_against_oracle(sv):
    """The benchmark's 20-qubit circuit learning at full depth (10 layers of
    Rx-Rz-Rx + ring, 600 parameters, 64 inputs) in the launch configuration
    the benchmark times: with dL/dE weights on two of the 64 inputs, the
    adjoint gradient is a weighted sum of those inputs' derivatives, which
    the dense oracle computes by parameter shift on sampled parameters; every
    instance energy of a sample of inputs is checked too."""
    import torch
    w = wl.config(3)
    th = theta_of(w)
    prob = sv.Problem.from_spec(w, "c64")
    sv.sv_autotune(prob, th, 2)
    wts = np.zeros(w.n_instances)
    wts[0], wts[37] = 1.0, -0.5
    l_, e_, g_ = sv.sv_grad_adjoint(prob, th, weights=torch.as_tensor(wts, device="cuda"))
    ks = [0, 1, 2, 151, 305, 598, 599]
    inst, sp, sh = [], [], []
    for k in ks:
        for sign in (1.0, -1.0):
            for i in (0, 37):
                inst.append(i)
                sp.append(k)
                sh.append(sign * np.pi / 2)
    checked = [0, 11, 37, 63]
    E = oracle.energies(w, None, np.array(checked + inst), np.array([-1] * 4 + sp),
                        np.array([0.0] * 4 + sh))
    close(e_.cpu().numpy()[checked], E[:4], TOL["c64"]["E"])
    Es = E[4:].reshape(len(ks), 2, 2)
    g = 0.5 * (Es[:, 0, :] - Es[:, 1, :]) @ np.array([1.0, -0.5])
    close(g_.cpu().numpy()[ks], g, TOL["c64"]["G"])


def test_mcvqe22_full_depth_against_oracle(sv):
    """The 28-qubit workload's generator at 22 qubits with all 8 layers and
    general angles (every rotation non-trivial), 2 references: the adjoint
    against the dense oracle's energies and sampled parameter-shift
    gradient entries."""
    w = wl.mcvqe(22, 8, "nn+nnn", n_refs=2)
    prob = sv.Problem.from_spec(w, "c64")
    l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w))
    ks = [0, 21, 88, 130, 175]
    L, E, g = oracle.grad_param_shift(w, params=ks)
    close(e_.cpu().numpy(), E, TOL["c64"]["E"])
    close(l_.cpu().numpy()[0], L, TOL["c64"]["E"])
    close(g_.cpu().numpy()[ks], g, TOL["c64"]["G"])


@pytest.mark.parametrize("tile_bits", [9, 10])
def test_stage_paths_with_mixed_rotation_forms(sv, tile_bits):
    """Tile passes take a branch-free path for stages whose register bits
    0..M-1 all carry real rotations in shear form (cos(angle/2) > 0) and the
    generic path otherwise.  Angles beyond pi (cos < 0), exactly 0 and
    exactly pi put both kinds of stages, and stages with fewer ops, into the
    same passes; the adjoint at every checkpoint interval and the energies
    must still match the oracle."""
    w = wl.mcvqe(12, 4, "nn+nnn", n_refs=3)
    theta = np.array(w.theta)
    rng = np.random.default_rng(5)
    theta[rng.choice(w.n_params, 12, replace=False)] += 2 * np.pi  # cos(angle / 2) < 0
    theta[rng.choice(w.n_params, 4, replace=False)] = 0.0
    theta[rng.choice(w.n_params, 3, replace=False)] = np.pi
    w.theta = theta
    L, E, g = oracle.grad_param_shift(w)
    prob = sv.Problem.from_spec(w, "c64", opts=sv.plan_opts(reg_bits=4, tile_bits=tile_bits))
    for every in (1, 2, 0):
        l_, e_, g_ = sv.sv_grad_adjoint(prob, theta_of(w), checkpoint_every=every)
        close(e_.cpu().numpy(), E, TOL["c64"]["E"])
        close(l_.cpu().numpy()[0], L, TOL["c64"]["E"])
        close(g_.cpu().numpy()[: w.n_params], g, TOL["c64"]["G"])


def test_last_adjoint_info_counts_reverse_bytes(sv):
    """sv_last_adjoint_info reports the checkpoint interval the tile adjoint
    used and the algorithmic bytes of its reverse passes: per pass psi (or
    its stored state) and lambda read and lambda written, psi written unless
    the next pass restarts from a stored state; zeros after an on-chip
    adjoint."""
    w = wl.mcvqe(12, 8, "nn+nnn", n_refs=3)
    opts = sv.plan_opts(reg_bits=4, tile_bits=9)
    prob = sv.Problem.from_spec(w, "c64", opts=opts)
    d = 0 if w.inputs is None else 1
    npass = sv.sv_plan_info(sv.Circuit(w.n_qubits, w.gates, w.n_params, d), "c64",
                            opts)["n_passes"]
    assert npass >= 5
    state = w.n_instances * (8 << w.n_qubits)
    for every in (1, 2, 4):
        sv.sv_grad_adjoint(prob, theta_of(w), checkpoint_every=every)
        got = sv.sv_last_adjoint_info()
        writes = sum(1 for i in range(npass) if i > 0 and not (i % every == 0 and i < npass))
        assert got["checkpoint_every"] == every
        assert got["reverse_bytes"] == state * (3 * npass + writes)
    small = sv.Problem.from_spec(wl.vqe_random_pauli(4, 2, 10), "c64")
    sv.sv_grad_adjoint(small, theta_of(wl.vqe_random_pauli(4, 2, 10)))
    assert sv.sv_last_adjoint_info() == {"checkpoint_every": 0, "reverse_bytes": 0}
