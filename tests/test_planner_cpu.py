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
                ("ldt", U32 * 30), ("stt", U32 * 30)]


class Op(ctypes.Structure):
    _fields_ = [("kind", I32), ("a", I32), ("b", I32), ("group", I32)]


class Group(ctypes.Structure):
    _fields_ = [("m_begin", I32), ("m_end", I32), ("qubit", I32), ("has_param", I32)]


class Member(ctypes.Structure):
    _fields_ = [("kind", I32), ("param", I32), ("angle", ctypes.c_double)]


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
    sizes = (I32 * 6)()
    lib().sv_debug_sizes(sizes)
    assert list(sizes)[:4] == [ctypes.sizeof(Stage), ctypes.sizeof(Op), ctypes.sizeof(Group),
                               ctypes.sizeof(Member)]


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


def run_plan(plan, n, R, w, theta, x, ref, sp=-1, sh=0.0):
    stages, ops, groups, members = plan
    mats = []
    for g in groups:
        M = np.eye(2, dtype=complex)
        for m in members[g.m_begin:g.m_end]:
            M = member_matrix(m, theta, x, sp, sh) @ M
        mats.append(M)
    R = min(R, n)
    T = 1 << (n - R)
    tid = np.arange(T)
    smem = np.zeros(1 << n, dtype=complex)
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
            if s == 0:
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
        new = np.full(1 << n, np.nan, dtype=complex)
        addrs = []
        for r in range(1 << R):
            new[sb ^ so[r]] = a[:, r]
            addrs.append(sb ^ so[r])
        addrs = np.concatenate(addrs)
        assert len(np.unique(addrs)) == 1 << n, "stage store is not a bijection"
        smem = new
    return np.array([smem[swz(j, w)] for j in range(1 << n)])


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
