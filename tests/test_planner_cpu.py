"""Host-logic tests of the planner, on CPU.

The compiled stage program (fused groups, register stages, deferred CNOT
permutations, swizzled shared-memory address vectors, thread-bit order) is
exported from libsv.so and executed here thread by thread, the way the
kernels execute it, in numpy; the final states must equal the oracle's.  The
library also has to load and export every symbol its headers declare.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import workloads as wl

sv = pytest.importorskip("paper_2406_03466_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
I32, U32 = ctypes.c_int32, ctypes.c_uint32


class Stage(ctypes.Structure):
    _fields_ = [("op_begin", I32), ("op_end", I32), ("n_thr", I32), ("n_u1", I32),
                ("q", I32 * 5), ("tpos", I32 * 30), ("ldq", U32 * 5), ("stq", U32 * 5),
                ("ldt", U32 * 30), ("stt", U32 * 30), ("sorted", I32), ("bit_begin", I32 * 6)]


class Op(ctypes.Structure):
    _fields_ = [("kind", I32), ("a", I32), ("b", I32), ("group", I32)]


class Group(ctypes.Structure):
    _fields_ = [("m_begin", I32), ("m_end", I32), ("qubit", I32), ("has_param", I32),
                ("real", I32)]


class Member(ctypes.Structure):
    _fields_ = [("kind", I32), ("param", I32), ("angle", ctypes.c_double)]


class PassDesc(ctypes.Structure):
    _fields_ = [("stage_begin", I32), ("stage_end", I32), ("t", I32), ("n_tile_bits", I32),
                ("n_u1", I32), ("local_mask", U32), ("gl", U32 * 30), ("gt", U32 * 30),
                ("ldperm", U32 * 30)]


def lib():
    L = sv.library()
    L.sv_debug_plan.argtypes = [ctypes.c_void_p, I32, I32, I32, ctypes.POINTER(I32)] + [ctypes.c_void_p] * 4
    L.sv_debug_plan.restype = I32
    return L


def test_header_symbols_exported():
    L = sv.library()
    declared = set()
    for h in ("sv.h", "sv_debug.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        declared |= set(re.findall(r"\b(sv_[a-z_0-9]+)\s*\(", text))
    assert "sv_grad_adjoint" in declared and "sv_alloc" in declared
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared but not exported"


def test_struct_sizes_match():
    sizes = (I32 * 8)()
    lib().sv_debug_sizes(sizes)
    assert list(sizes)[:4] == [ctypes.sizeof(Stage), ctypes.sizeof(Op), ctypes.sizeof(Group),
                               ctypes.sizeof(Member)]
    assert sizes[6] == ctypes.sizeof(PassDesc)


def export_plan(circ, R, fuse, w):
    L = lib()
    counts = (I32 * 4)()
    st = L.sv_debug_plan(ctypes.byref(circ.struct), R, int(fuse), w, counts, None, None, None, None)
    assert st == 0, sv.sv_status_string(st)
    arrays = [(Stage * max(1, counts[0]))(), (Op * max(1, counts[1]))(),
              (Group * max(1, counts[2]))(), (Member * max(1, counts[3]))()]
    st = L.sv_debug_plan(ctypes.byref(circ.struct), R, int(fuse), w, counts, *arrays)
    assert st == 0
    return [a[:c] for a, c in zip(arrays, counts)]


def swz(a, w):
    f, h = 0, a >> w
    while h:
        f ^= h
        h >>= w
    return a ^ (f & ((1 << w) - 1))


def rot(axis, a):
    c, s = np.cos(a / 2), np.sin(a / 2)
    if axis == 0:
        return np.array([[c, -1j * s], [-1j * s, c]])
    if axis == 1:
        return np.array([[c, -s], [s, c]], dtype=complex)
    return np.array([[np.exp(-0.5j * a), 0], [0, np.exp(0.5j * a)]])


def member_matrix(m, theta, x, sp, sh):
    if m.kind <= 2:
        a = m.angle if m.param < 0 else theta[m.param] + (sh if m.param == sp else 0.0)
        return rot(m.kind, a)
    if m.kind == 3:
        return np.array([[0, 1], [1, 0]], dtype=complex)
    if m.kind == 4:
        return np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
    if m.kind == 5:
        return rot(1, np.arcsin(x[m.param]))
    return rot(2, np.arccos(x[m.param] ** 2))


def group_mats(groups, members, theta, x, sp, sh):
    mats = []
    for g in groups:
        M = np.eye(2, dtype=complex)
        for m in members[g.m_begin:g.m_end]:
            M = member_matrix(m, theta, x, sp, sh) @ M
        mats.append(M)
    return mats


def run_stages(smem, stages, ops, mats, t, R, ref=None):
    """Executes register stages thread by thread on a 2^t shared-memory image
    (swizzled addresses); stage 0 builds |ref> when ref is given."""
    R = min(R, t)
    T = 1 << (t - R)
    tid = np.arange(T)
    for s, sg in enumerate(stages):
        lb = np.zeros(T, np.int64); sb = np.zeros(T, np.int64); lg = np.zeros(T, np.int64)
        for k in range(sg.n_thr):
            bit = (tid >> k) & 1
            lb ^= bit * sg.ldt[k]; sb ^= bit * sg.stt[k]; lg |= bit << sg.tpos[k]
        lo = [0] * (1 << R); so = [0] * (1 << R); lj = [0] * (1 << R)
        for r in range(1 << R):
            for i in range(R):
                if r >> i & 1:
                    lo[r] ^= sg.ldq[i]; so[r] ^= sg.stq[i]; lj[r] |= 1 << sg.q[i]
        a = np.zeros((T, 1 << R), dtype=complex)
        for r in range(1 << R):
            if s == 0 and ref is not None:
                a[:, r] = ((lg | lj[r]) == ref).astype(float)
            else:
                a[:, r] = smem[lb ^ lo[r]]
        for op in ops[sg.op_begin:sg.op_end]:
            if op.kind == 0:
                M = mats[op.group]
                for r in range(1 << R):
                    if r >> op.a & 1:
                        continue
                    r1 = r | 1 << op.a
                    x0, x1 = a[:, r].copy(), a[:, r1].copy()
                    a[:, r] = M[0, 0] * x0 + M[0, 1] * x1
                    a[:, r1] = M[1, 0] * x0 + M[1, 1] * x1
            else:
                for r in range(1 << R):
                    j = lg | lj[r]
                    flip = ((j >> op.a) & 1) & ((j >> op.b) & 1)
                    a[:, r] = np.where(flip == 1, -a[:, r], a[:, r])
        new = np.full(1 << t, np.nan, dtype=complex)
        addrs = []
        for r in range(1 << R):
            new[sb ^ so[r]] = a[:, r]
            addrs.append(sb ^ so[r])
        addrs = np.concatenate(addrs)
        assert len(np.unique(addrs)) == 1 << t, "stage store is not a bijection"
        smem = new
    return smem


def run_plan(plan, n, R, w, theta, x, ref, sp=-1, sh=0.0):
    stages, ops, groups, members = plan
    mats = group_mats(groups, members, theta, x, sp, sh)
    smem = run_stages(np.zeros(1 << n, dtype=complex), stages, ops, mats, n, R, ref)
    return np.array([smem[swz(j, w)] for j in range(1 << n)])


def export_passes(circ, t, c, R, fuse, w):
    L = sv.library()
    L.sv_debug_passes.argtypes = [ctypes.c_void_p, I32, I32, I32, I32, I32, ctypes.POINTER(I32)] + [ctypes.c_void_p] * 5
    L.sv_debug_passes.restype = I32
    counts = (I32 * 5)()
    st = L.sv_debug_passes(ctypes.byref(circ.struct), t, c, R, int(fuse), w, counts, None, None, None, None, None)
    assert st == 0, sv.sv_status_string(st)
    arrays = [(Stage * max(1, counts[0]))(), (Op * max(1, counts[1]))(), (Group * max(1, counts[2]))(),
              (Member * max(1, counts[3]))(), (PassDesc * max(1, counts[4]))()]
    assert L.sv_debug_passes(ctypes.byref(circ.struct), t, c, R, int(fuse), w, counts, *arrays) == 0
    return [a[:k] for a, k in zip(arrays, counts)]


def run_passes(plan, n, R, w, theta, x, ref, sp=-1, sh=0.0):
    stages, ops, groups, members, passes = plan
    mats = group_mats(groups, members, theta, x, sp, sh)
    state = np.zeros(1 << n, dtype=complex)
    state[ref] = 1.0
    for pd in passes:
        t = pd.t
        loc = np.zeros(1 << t, np.int64)
        for i in range(1 << t):
            for b in range(t):
                if i >> b & 1:
                    loc[i] ^= pd.gl[b]
        sw = np.array([swz(i, w) for i in range(1 << t)])
        lp = np.zeros(1 << t, np.int64)  # load through the pass's leading permutation
        for i in range(1 << t):
            for b in range(t):
                if i >> b & 1:
                    lp[i] ^= pd.ldperm[b]
        covered = np.zeros(1 << n, bool)
        for tile in range(1 << pd.n_tile_bits):
            tb = 0
            for k in range(pd.n_tile_bits):
                if tile >> k & 1:
                    tb ^= pd.gt[k]
            gidx = tb ^ loc
            assert not covered[gidx].any(), "tiles overlap"
            covered[gidx] = True
            smem = np.full(1 << t, np.nan, dtype=complex)
            smem[lp] = state[gidx]
            assert not np.isnan(smem).any(), "load permutation is not a bijection"
            smem = run_stages(smem, stages[pd.stage_begin:pd.stage_end], ops, mats, t, R)
            state[gidx] = smem[sw]
        assert covered.all(), "tiles do not cover the state"
    return state


CASES = [
    lambda: wl.vqe_random_pauli(4, 2, 10),
    lambda: wl.mcvqe(8, 4),
    lambda: wl.qcl(6, 2, 3),
    lambda: wl.qcl(9, 2, 2),
    lambda: wl.random_workload(5, 60, 3, 2, seed=3, with_encoding=True),
    lambda: wl.random_workload(7, 90, 3, 2, seed=4),
    lambda: wl.random_workload(1, 10, 2, 2, seed=5),
    lambda: wl.random_workload(2, 20, 2, 2, seed=6),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("R", [1, 2, 3, 4])
@pytest.mark.parametrize("fuse", [True, False])
def test_plan_matches_oracle(case, R, fuse):
    w = CASES[case]()
    d = 0 if w.inputs is None else w.inputs.shape[1]
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    for swz_bits in (3, 4):
        plan = export_plan(circ, R, fuse, swz_bits)
        for i in range(min(2, w.n_instances)):
            x = None if w.inputs is None else w.inputs[i]
            sp = (i * 7) % w.n_params if w.n_params else -1
            got = run_plan(plan, w.n_qubits, R, swz_bits, w.theta, x, int(w.refs[i]), sp, 0.3)
            want = oracle.state(w, instance=i, shift_param=sp, shift=0.3)
            assert np.allclose(got, want, atol=1e-12), (case, R, fuse, swz_bits, i)


def test_stage_limits():
    w = wl.qcl(12, 6, 2)
    circ = sv.Circuit(12, w.gates, w.n_params, 1)
    stages, ops, groups, members = export_plan(circ, 4, True, 4)
    assert all(s.n_u1 <= 8 for s in stages)
    # fused groups: encoding + first layer per qubit, then one group per layer per qubit
    assert len(groups) == 12 * 6
    # 12 rotations per layer with 4 register bits -> 3 stages per layer
    assert len(stages) == 18


PASS_CASES = [
    (lambda: wl.qcl(9, 3, 2), 7, 3),
    (lambda: wl.mcvqe(9, 3, "nn+nnn", n_refs=3), 6, 3),
    (lambda: wl.random_workload(8, 80, 3, 2, seed=21, with_encoding=True), 6, 3),
    (lambda: wl.mcvqe(7, 2), 7, 3),
]


@pytest.mark.parametrize("case", range(len(PASS_CASES)))
@pytest.mark.parametrize("R", [2, 3])
def test_tile_passes_match_oracle(case, R):
    make, t, c = PASS_CASES[case]
    w = make()
    d = 0 if w.inputs is None else w.inputs.shape[1]
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    for swz_bits in (3, 4):
        plan = export_passes(circ, t, c, R, True, swz_bits)
        passes = plan[4]
        assert all(((p.local_mask & ((1 << c) - 1)) == (1 << c) - 1) for p in passes)
        for i in range(min(2, w.n_instances)):
            x = None if w.inputs is None else w.inputs[i]
            sp = (5 * i + 1) % w.n_params
            got = run_passes(plan, w.n_qubits, R, swz_bits, w.theta, x, int(w.refs[i]), sp, -0.4)
            want = oracle.state(w, instance=i, shift_param=sp, shift=-0.4)
            assert np.allclose(got, want, atol=1e-12), (case, R, swz_bits, i)


def test_pass_counts_at_scale():
    # 20-qubit circuit learning: encoding + 10 layers of Rx-Rz-Rx + CNOT ring
    w = wl.qcl(20, 10, 1)
    circ = sv.Circuit(20, w.gates, w.n_params, 1)
    stages, ops, groups, members, passes = export_passes(circ, 12, 4, 4, True, 4)
    assert 10 <= len(passes) <= 40
    assert sum(p.n_u1 for p in passes) == len(groups)


@pytest.mark.parametrize("name,R", [("mcvqe8", 3), ("mcvqe8", 2), ("qcl8", 3), ("rand8", 2)])
def test_straight_line_stage_flag(name, R):
    """The planner marks a stage sorted = 2 (the kernels' straight-line path)
    exactly when every register bit carries one fused group and all of them
    are real; other sorted stages stay 1."""
    w = {"mcvqe8": lambda: wl.mcvqe(8, 4, "all"), "qcl8": lambda: wl.qcl(8, 3, 2),
         "rand8": lambda: wl.random_workload(8, 60, 4, 2, seed=3, with_encoding=True)}[name]()
    d = 0 if w.inputs is None else 1
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    stages, ops, groups, members = export_plan(circ, R, True, 4)
    flagged = 0
    for st in stages:
        if not st.sorted:
            continue
        counts = [st.bit_begin[i + 1] - st.bit_begin[i] for i in range(R)]
        one_real = all(c == 1 for c in counts) and all(
            groups[ops[st.op_begin + st.bit_begin[i]].group].real for i in range(R))
        assert st.sorted == (2 if one_real else 1)
        flagged += st.sorted == 2
    if name == "mcvqe8":
        assert flagged > 0  # single Ry groups on every register bit
    if name == "qcl8":
        assert flagged == 0  # Rx Rz Rx groups are complex
