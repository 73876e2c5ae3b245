"""Host-side checks of the tile-pass kernel descriptors, on CPU.

libsv.so exports the TilePass descriptors exactly as the GPU entry points
build them.  Here they drive a numpy model of the two pass kernels, thread
by thread and tile by tile, with the kernels' byte addresses, tile walk
(per-block contiguous tile ranges, incremental tile bases) and op order:
the forward passes must reproduce the oracle's states, and the reverse
passes (adjoint sweep with per-group reduced matrices, then the member walk
that turns them into derivatives) the oracle's parameter-shift gradient.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import dense
import workloads as wl

sv = pytest.importorskip("paper_2406_03466_gb300")

I32, U32, U64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
KT = 13  # largest tile bits


class Group(ctypes.Structure):
    _fields_ = [("m_begin", I32), ("m_end", I32), ("qubit", I32), ("has_param", I32),
                ("real", I32)]


class Member(ctypes.Structure):
    _fields_ = [("kind", I32), ("param", I32), ("angle", ctypes.c_double)]


class TileStage(ctypes.Structure):
    _fields_ = [("ldq", U32 * 5), ("stq", U32 * 5), ("ldt", U32 * KT), ("stt", U32 * KT),
                ("op", I32 * 5)]


class TilePass(ctypes.Structure):
    _fields_ = [("t", I32), ("R", I32), ("n_stages", I32), ("n_ops", I32), ("n_tile_bits", I32),
                ("all_single", I32), ("real_mask", U64), ("param_mask", U64), ("gl", U32 * KT),
                ("gpre", U32 * 30), ("ldperm", U32 * KT), ("nat", U32 * KT), ("grp", I32 * 48),
                ("st", TileStage * 16), ("fmode", ctypes.c_int8 * 48)]


def _debug_tile_passes():
    L = sv.library()
    L.sv_debug_tile_passes.argtypes = [ctypes.c_void_p, I32, I32, I32, I32, I32,
                                       ctypes.POINTER(I32), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.sv_debug_tile_passes.restype = I32
    return L.sv_debug_tile_passes


def export(circ, t, R, fuse=True, dtype=0, relabel=False):
    """(groups, members, tile passes, layout): layout[q] = the index bit that
    holds qubit q after the last pass."""
    f = _debug_tile_passes()
    counts = (I32 * 3)()
    st = f(ctypes.byref(circ.struct), t, R, int(fuse), dtype, int(relabel), counts,
           None, None, None, None)
    assert st == 0, sv.sv_status_string(st)
    arrs = [(Group * max(1, counts[0]))(), (Member * max(1, counts[1]))(),
            (TilePass * max(1, counts[2]))()]
    lay = (I32 * circ.n_qubits)()
    assert f(ctypes.byref(circ.struct), t, R, int(fuse), dtype, int(relabel), counts,
             *arrs, lay) == 0
    return [a[:k] for a, k in zip(arrs, counts)] + [list(lay)]


def test_descriptor_size_matches():
    sizes = (I32 * 8)()
    sv.library().sv_debug_sizes(sizes)
    assert sizes[7] == ctypes.sizeof(TilePass)


# --------------------------------------------------------------- numpy model

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


def group_mats(groups, members, theta, x, sp=-1, sh=0.0):
    out = []
    for g in groups:
        M = np.eye(2, dtype=complex)
        for m in members[g.m_begin:g.m_end]:
            M = member_matrix(m, theta, x, sp, sh) @ M
        out.append(M)
    return out


def xsel(r, v):
    a = 0
    for i, x in enumerate(v):
        if r >> i & 1:
            a ^= x
    return a


def thread_vectors(v, t, R, tid):
    g = np.zeros(len(tid), np.int64)
    for b in range(t - R):
        g ^= ((tid >> b) & 1) * int(v[b])
    return g, [int(v[t - R + j]) for j in range(R)]


def tile_walk(P, n_slots, n_blocks):
    """The (slot, base) sequence of every block, walked as the kernels do."""
    ntb = P.n_tile_bits
    tiles = n_slots << ntb
    per = -(-tiles // n_blocks)
    gt = [P.gpre[k] ^ (P.gpre[k - 1] if k else 0) for k in range(ntb)]
    out = []
    for blk in range(n_blocks):
        t0, t1 = per * blk, min(tiles, per * (blk + 1))
        if t0 >= t1:
            continue
        slot, local = t0 >> ntb, t0 & ((1 << ntb) - 1)
        base = 0
        for k in range(ntb):
            if local >> k & 1:
                base ^= gt[k]
        for _ in range(t0, t1):
            out.append((slot, base))
            local += 1
            if local >> ntb:
                slot, local, base = slot + 1, 0, 0
            else:
                base ^= P.gpre[(local & -local).bit_length() - 1]
    return out


def apply_bit(a, I, M):
    """2x2 matrix M on register bit I of a[thread, r]."""
    for r in range(a.shape[1]):
        if r >> I & 1:
            continue
        x, y = a[:, r].copy(), a[:, r | 1 << I].copy()
        a[:, r] = M[0, 0] * x + M[0, 1] * y
        a[:, r | 1 << I] = M[1, 0] * x + M[1, 1] * y


def stage_bases(sg, t, R, tid):
    lb = np.zeros(len(tid), np.int64)
    sb = np.zeros(len(tid), np.int64)
    for k in range(t - R):
        bit = (tid >> k) & 1
        lb ^= bit * int(sg.ldt[k])
        sb ^= bit * int(sg.stt[k])
    return lb, sb


def run_fwd(P, states, mats, csz, n_blocks=3):
    t, R = P.t, P.R
    tid = np.arange(1 << (t - R))
    g0, gk = thread_vectors(P.gl, t, R, tid)
    p0, pk = thread_vectors(P.ldperm, t, R, tid)
    n0, nk = thread_vectors(P.nat, t, R, tid)
    NA = 1 << R
    for slot, base in tile_walk(P, states.shape[0], n_blocks):
        S = states[slot]
        sm = np.full(1 << t, np.nan, dtype=complex)
        for k in range(NA):
            sm[(p0 ^ xsel(k, pk)) // csz] = S[base + (g0 ^ xsel(k, gk))]
        assert not np.isnan(sm).any(), "tile load misses shared-memory words"
        for s in range(P.n_stages):
            sg = P.st[s]
            lb, sb = stage_bases(sg, t, R, tid)
            a = np.stack([sm[(lb ^ xsel(r, sg.ldq[:R])) // csz] for r in range(NA)], axis=1)
            for I in range(R):
                u = sg.op[I]
                if u >= 0:
                    M = mats[slot][P.grp[u]]
                    if P.real_mask >> u & 1:
                        assert np.all(M.imag == 0)
                    apply_bit(a, I, M)
            new = np.full(1 << t, np.nan, dtype=complex)
            for r in range(NA):
                new[(sb ^ xsel(r, sg.stq[:R])) // csz] = a[:, r]
            assert not np.isnan(new).any(), "stage store misses shared-memory words"
            sm = new
        for k in range(NA):
            S[base + (g0 ^ xsel(k, gk))] = sm[(n0 ^ xsel(k, nk)) // csz]


def run_rev(P, psi, lam, mats, rho, csz, n_blocks=2):
    t, R = P.t, P.R
    tid = np.arange(1 << (t - R))
    g0, gk = thread_vectors(P.gl, t, R, tid)
    p0, pk = thread_vectors(P.ldperm, t, R, tid)
    n0, nk = thread_vectors(P.nat, t, R, tid)
    NA = 1 << R
    for slot, base in tile_walk(P, psi.shape[0], n_blocks):
        sp = np.zeros(1 << t, complex)
        sl = np.zeros(1 << t, complex)
        for k in range(NA):
            so, go = (n0 ^ xsel(k, nk)) // csz, base + (g0 ^ xsel(k, gk))
            sp[so] = psi[slot][go]
            sl[so] = lam[slot][go]
        for s in range(P.n_stages - 1, -1, -1):
            sg = P.st[s]
            lb, sb = stage_bases(sg, t, R, tid)
            ad = [(sb ^ xsel(r, sg.stq[:R])) // csz for r in range(NA)]
            a = np.stack([sp[x] for x in ad], axis=1)
            al = np.stack([sl[x] for x in ad], axis=1)
            for I in range(R - 1, -1, -1):
                u = sg.op[I]
                if u < 0:
                    continue
                g = P.grp[u]
                if P.param_mask >> u & 1:
                    # the kernel keeps K = (rho - rho^dag) / 2i as four sums
                    # and stores i K in place of rho
                    k = np.zeros(4)
                    for r in range(NA):
                        if r >> I & 1:
                            continue
                        x0, x1 = a[:, r], a[:, r | 1 << I]
                        y0, y1 = al[:, r], al[:, r | 1 << I]
                        k[0] += np.sum(x0 * np.conj(y0)).imag
                        k[1] += np.sum(x1 * np.conj(y1)).imag
                        k[2] += np.sum(x0 * np.conj(y1) + x1 * np.conj(y0)).imag
                        k[3] += np.sum(x0 * np.conj(y1) - x1 * np.conj(y0)).real
                    if P.all_single:
                        # one sum per op, stored as the component its fmode needs
                        md = P.fmode[u]
                        assert md in (1, 2, 3)
                        k = {1: [0, 0, 0, k[3]], 2: [0, 0, k[2], 0], 3: [k[0] - k[1], 0, 0, 0]}[md]
                    rho[slot][g] += np.array([[1j * k[0], 0.5 * (k[3] + 1j * k[2])],
                                              [0.5 * (-k[3] + 1j * k[2]), 1j * k[1]]])
                Md = mats[slot][g].conj().T
                apply_bit(a, I, Md)
                apply_bit(al, I, Md)
            for r in range(NA):
                x = (lb ^ xsel(r, sg.ldq[:R])) // csz
                sp[x] = a[:, r]
                sl[x] = al[:, r]
        for k in range(NA):
            so, go = (p0 ^ xsel(k, pk)) // csz, base + (g0 ^ xsel(k, gk))
            psi[slot][go] = sp[so]
            lam[slot][go] = sl[so]


def group_gradients(groups, members, rho, theta, x, grad, weight):
    """dE/dtheta = Im tr(P rho) member by member, rho <- G^dag rho G between."""
    for gi, g in enumerate(groups):
        if not g.has_param:
            continue
        r = rho[gi].copy() * weight
        ms = list(members[g.m_begin:g.m_end])
        first = next(i for i, m in enumerate(ms) if m.kind <= 2 and m.param >= 0)
        for i in range(len(ms) - 1, first - 1, -1):
            m = ms[i]
            if m.kind <= 2 and m.param >= 0:
                Pm = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
                      np.diag([1, -1])][m.kind]
                grad[m.param] += np.imag(np.trace(Pm @ r))
            if i > first:
                G = member_matrix(m, theta, x, -1, 0.0)
                r = G.conj().T @ r @ G


def init_states(w, n_inst):
    S = np.zeros((n_inst, 1 << w.n_qubits), complex)
    for i in range(n_inst):
        S[i, int(w.refs[i])] = 1.0
    return S


CASES = {
    "qcl8": lambda: wl.qcl(8, 2, 2),
    "mcvqe8": lambda: wl.mcvqe(8, 2, "nn+nnn", n_refs=2),
    "rand8_cz": lambda: wl.random_workload(8, 70, 5, 2, seed=41, with_encoding=True),
    "rand9": lambda: wl.random_workload(9, 60, 4, 2, seed=42, cost="mse"),
}


def circuit_of(w):
    d = 0 if w.inputs is None else w.inputs.shape[1]
    return sv.Circuit(w.n_qubits, w.gates, w.n_params, d)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t,R,dtype", [(7, 2, 0), (8, 3, 0), (7, 2, 1), (8, 3, 1), (6, 1, 0)])
def test_forward_passes_match_oracle(name, t, R, dtype):
    w = CASES[name]()
    circ = circuit_of(w)
    groups, members, passes, _ = export(circ, t, R, dtype=dtype)
    csz = 16 if dtype else 8
    I = min(2, w.n_instances)
    xs = [None if w.inputs is None else w.inputs[i] for i in range(I)]
    mats = [group_mats(groups, members, w.theta, xs[i]) for i in range(I)]
    S = init_states(w, I)
    for P in passes:
        assert P.n_stages >= 1 and P.t == t and P.R == R
        run_fwd(P, S, mats, csz)
    for i in range(I):
        np.testing.assert_allclose(S[i], oracle.state(w, instance=i), atol=1e-12)


def test_tile_walk_covers_every_tile_once():
    w = wl.qcl(12, 1, 1)
    groups, members, passes, _ = export(circuit_of(w), 8, 3)
    for P in passes[:4]:
        for nb in (1, 3, 7, 40):
            seen = tile_walk(P, 3, nb)
            assert len(seen) == 3 << P.n_tile_bits
            assert len(set(seen)) == len(seen)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t,R,dtype", [(7, 2, 0), (8, 3, 1)])
def test_reverse_passes_give_oracle_gradient(name, t, R, dtype):
    w = CASES[name]()
    circ = circuit_of(w)
    groups, members, passes, _ = export(circ, t, R, dtype=dtype)
    csz = 16 if dtype else 8
    I = w.n_instances
    xs = [None if w.inputs is None else w.inputs[i] for i in range(I)]
    mats = [group_mats(groups, members, w.theta, xs[i]) for i in range(I)]
    psi = init_states(w, I)
    for P in passes:
        run_fwd(P, psi, mats, csz)
    H = dense.hamiltonian(w.n_qubits, w.pauli_letters, w.pauli_coeffs)
    lam = np.stack([H @ psi[i] for i in range(I)])
    E = np.array([np.vdot(psi[i], lam[i]).real for i in range(I)])
    rho = [[np.zeros((2, 2), complex) for _ in groups] for _ in range(I)]
    for P in reversed(passes):
        run_rev(P, psi, lam, mats, rho, csz)
    for i in range(I):  # the reverse sweep returns psi to |ref>
        np.testing.assert_allclose(psi[i], init_states(w, I)[i], atol=1e-12)
    wts = oracle.cost_weights(w, E)
    grad = np.zeros(w.n_params)
    for i in range(I):
        group_gradients(groups, members, rho[i], w.theta, xs[i], grad, wts[i])
    L, E_o, g_o = oracle.grad_param_shift(w)
    np.testing.assert_allclose(E, E_o, atol=1e-12)
    np.testing.assert_allclose(grad, g_o, atol=1e-11)


def to_layout(vec, layout):
    """A state in qubit order, rearranged so that qubit q sits in index bit
    layout[q]."""
    n = len(layout)
    j = np.arange(1 << n)
    jp = np.zeros_like(j)
    for q in range(n):
        jp |= ((j >> q) & 1) << layout[q]
    out = np.empty_like(vec)
    out[jp] = vec
    return out


def moved_letters(letters, layout):
    out = np.zeros_like(letters)  # identity letters (code 0)
    for q in range(letters.shape[1]):
        out[:, layout[q]] = letters[:, q]
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("t,R,dtype", [(7, 2, 0), (6, 1, 0), (7, 2, 1)])
def test_relabeling_passes_forward_and_reverse(name, t, R, dtype):
    """Passes that move qubits into the low index bits: the forward sweep
    leaves the oracle's state in the exported layout, and the reverse sweep
    with lambda = H psi in that layout gives the oracle's gradient and
    returns psi to |ref>."""
    w = CASES[name]()
    circ = circuit_of(w)
    groups, members, passes, lay = export(circ, t, R, dtype=dtype, relabel=True)
    assert sorted(lay) == list(range(w.n_qubits))
    csz = 16 if dtype else 8
    I = w.n_instances
    xs = [None if w.inputs is None else w.inputs[i] for i in range(I)]
    mats = [group_mats(groups, members, w.theta, xs[i]) for i in range(I)]
    psi = init_states(w, I)
    for P in passes:
        run_fwd(P, psi, mats, csz)
    for i in range(I):
        np.testing.assert_allclose(psi[i], to_layout(oracle.state(w, instance=i), lay), atol=1e-12)
    H = dense.hamiltonian(w.n_qubits, moved_letters(np.asarray(w.pauli_letters), lay),
                          w.pauli_coeffs)
    lam = np.stack([H @ psi[i] for i in range(I)])
    E = np.array([np.vdot(psi[i], lam[i]).real for i in range(I)])
    rho = [[np.zeros((2, 2), complex) for _ in groups] for _ in range(I)]
    for P in reversed(passes):
        run_rev(P, psi, lam, mats, rho, csz)
    for i in range(I):
        np.testing.assert_allclose(psi[i], init_states(w, I)[i], atol=1e-12)
    wts = oracle.cost_weights(w, E)
    grad = np.zeros(w.n_params)
    for i in range(I):
        group_gradients(groups, members, rho[i], w.theta, xs[i], grad, wts[i])
    L, E_o, g_o = oracle.grad_param_shift(w)
    np.testing.assert_allclose(E, E_o, atol=1e-12)
    np.testing.assert_allclose(grad, g_o, atol=1e-11)


def test_relabeling_saves_passes():
    """On a wide layered circuit the low (contiguous) index bits carry qubits
    that the next pass needs, instead of the same four qubits in every pass."""
    w = wl.mcvqe(16, 4, "nn+nnn", n_refs=1)
    plain = export(circuit_of(w), 10, 3)[2]
    moved, lay = export(circuit_of(w), 10, 3, relabel=True)[2:]
    assert len(moved) < len(plain)
    assert lay != list(range(16))


def test_cz_is_planned_as_h_cnot_h():
    w = wl.random_workload(8, 70, 5, 2, seed=41, with_encoding=True)
    assert any(g.op == "CZ" for g in w.gates)
    groups, members, passes, _ = export(circuit_of(w), 7, 2)
    assert any(m.kind == 4 for m in members)  # H members absorbed into groups


def test_rejects_tiles_narrower_than_a_warp():
    w = wl.qcl(8, 1, 1)
    counts = (I32 * 3)()
    assert _debug_tile_passes()(ctypes.byref(circuit_of(w).struct), 7, 3, 1, 0, 0, counts,
                                None, None, None, None) != 0


# ------------------------------------------------------------ lambda = H psi

class HPassRec(ctypes.Structure):
    _fields_ = [("t", I32), ("n_tile_bits", I32), ("n_groups", I32), ("n_classes", I32),
                ("n_terms", I32), ("first", I32), ("real", I32), ("R", I32), ("gl", U32 * KT),
                ("gpre", U32 * 30), ("n_rows", I32), ("pad", I32),
                ("groups", ctypes.c_void_p), ("classes", ctypes.c_void_p),
                ("terms", ctypes.c_void_p), ("rows", ctypes.c_void_p)]


class HGroup(ctypes.Structure):
    _fields_ = [("xl", U32), ("c_begin", I32), ("c_end", I32), ("xfar", U32), ("kact", U32),
                ("r_begin", I32), ("r_end", I32), ("pad", U32)]


class HRow(ctypes.Structure):
    _fields_ = [("zt", U32), ("c_begin", I32), ("c_end", I32), ("pad", I32)]


class HClass(ctypes.Structure):
    _fields_ = [("zl", U32), ("t_begin", I32), ("t_end", I32), ("xnl", U32), ("xl", U32),
                ("pad", I32)]


class HTerm(ctypes.Structure):
    _fields_ = [("z", U32), ("phase", I32), ("coeff", ctypes.c_double)]


def export_h(obs, t, c):
    """(passes, groups, classes, terms, rows) of the H tile plan."""
    L = sv.library()
    L.sv_debug_h_passes.argtypes = [ctypes.c_void_p, I32, I32, ctypes.POINTER(I32)] + [ctypes.c_void_p] * 5
    L.sv_debug_h_passes.restype = I32
    counts = (I32 * 5)()
    assert L.sv_debug_h_passes(ctypes.byref(obs.struct), t, c, counts, None, None, None, None,
                               None) == 0
    arrs = [(HPassRec * counts[0])(), (HGroup * max(1, counts[1]))(),
            (HClass * max(1, counts[2]))(), (HTerm * max(1, counts[3]))(),
            (HRow * max(1, counts[4]))()]
    assert L.sv_debug_h_passes(ctypes.byref(obs.struct), t, c, counts, *arrs) == 0
    return [a[:k] for a, k in zip(arrs, counts)]


def run_h(plan, psi, n):
    """The tile H kernel, tile by tile: returns lambda = H psi and <psi|H|psi>.
    Like the kernel, thread tid holds amplitudes j = tid + k 2^(t - R).  A
    group without a Z on a register bit takes one value per thread (its
    signed class coefficients); the others take, per row (a run of classes
    with one Z mask zt on the thread bits), the per-tile row values
    E[k] = sum_c coef_c (-1)^|k & kz_c| times the thread's sign (-1)^|tid & zt|."""
    passes, groups, classes, terms, rows = plan
    lam = np.zeros_like(psi)
    E = 0.0
    for P in passes:
        t, ntb = P.t, P.n_tile_bits
        g0, c0, t0, r0 = P.groups or 0, P.classes or 0, P.terms or 0, P.rows or 0
        loc = np.zeros(1 << t, np.int64)
        for i in range(1 << t):
            for b in range(t):
                if i >> b & 1:
                    loc[i] ^= P.gl[b]
        j = np.arange(1 << t)
        R = P.R
        T = 1 << (t - R)
        tid = np.arange(T)
        kk = np.arange(1 << R)
        par = lambda a: np.array([bin(int(v)).count("1") & 1 for v in a])
        for slot, base in tile_walk(P, 1, 3):
            tile = psi[base + loc]
            coef = []
            for cl in classes[c0:c0 + P.n_classes]:
                v = 0j
                for tm in terms[t0 + cl.t_begin:t0 + cl.t_end]:
                    sgn = -1.0 if bin((base ^ cl.xnl) & tm.z).count("1") & 1 else 1.0
                    v += sgn * tm.coeff * 1j ** tm.phase
                # the class's sign on the flip bits: D(j ^ xl) = D(j) x that
                sx = -1.0 if bin(cl.xl & cl.zl).count("1") & 1 else 1.0
                coef.append(sx * v)
            # the kernel's row table of this tile
            etab = []
            for rw in rows[r0:r0 + P.n_rows]:
                e = np.zeros(1 << R, complex)
                for c in range(rw.c_begin, rw.c_end):
                    zl = classes[c0 + c].zl
                    assert zl & (T - 1) == rw.zt
                    e += np.where(par(kk & (zl >> (t - R))) == 1, -coef[c], coef[c])
                etab.append(e)
            part = np.zeros(1 << t, complex)
            for gr in groups[g0:g0 + P.n_groups]:
                jx = j ^ gr.xl
                kact = 0
                for c in range(gr.c_begin, gr.c_end):
                    kact |= classes[c0 + c].zl >> (t - R)
                assert gr.kact == kact
                Dk = np.zeros((T, 1 << R), complex)
                if kact == 0:
                    assert gr.r_begin == gr.r_end
                    for c in range(gr.c_begin, gr.c_end):
                        zt = classes[c0 + c].zl & (T - 1)
                        Dk += np.where(par(tid & zt) == 1, -coef[c], coef[c])[:, None]
                else:
                    # the rows cover the group's classes, in order
                    covered = [c for r in range(gr.r_begin, gr.r_end)
                               for c in range(rows[r0 + r].c_begin, rows[r0 + r].c_end)]
                    assert covered == list(range(gr.c_begin, gr.c_end))
                    for r in range(gr.r_begin, gr.r_end):
                        sg = np.where(par(tid & rows[r0 + r].zt) == 1, -1.0, 1.0)
                        Dk += sg[:, None] * etab[r][None, :]
                # amplitude j = tid + k T holds D(j ^ xl) at [tid, k]
                D = Dk.T.reshape(-1)
                part += D * (psi[(base + loc) ^ gr.xfar] if gr.xfar else tile[jx])
            E += float(np.sum(np.conj(tile) * part).real)
            if P.first:
                lam[base + loc] = part
            else:
                lam[base + loc] += part
    return lam, E


@pytest.mark.parametrize("n,t,c,kind", [(9, 7, 4, "mcvqe"), (10, 8, 4, "mcvqe"), (8, 7, 3, "random"),
                                        (9, 9, 4, "random"), (10, 7, 4, "mcvqe")])
def test_h_passes_match_dense(n, t, c, kind):
    if kind == "mcvqe":
        w = wl.mcvqe(n, 1, "nn+nnn", n_refs=1)
    else:
        w = wl.vqe_random_pauli(n, 1, 40)
    obs = sv.PauliSum(n, w.pauli_letters, w.pauli_coeffs)
    plan = export_h(obs, t, c)
    passes = plan[0]
    assert passes[0].first == 1 and all(p.first == 0 for p in passes[1:])
    # every X-mask group is covered by exactly one pass
    xs = {}
    for row in np.asarray(w.pauli_letters).reshape(-1, n):
        x = sum(1 << q for q in range(n) if row[q] in (1, 2))
        xs[x] = 1
    assert len(plan[1]) == len(xs)
    rng = np.random.default_rng(n + t)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    H = dense.hamiltonian(n, w.pauli_letters, w.pauli_coeffs)
    lam, E = run_h(plan, psi, n)
    np.testing.assert_allclose(lam, H @ psi, atol=1e-12)
    assert abs(E - np.vdot(psi, H @ psi).real) < 1e-12


def test_single_sum_mode_chosen_for_one_rotation_groups():
    w = wl.mcvqe(8, 2, "nn+nnn", n_refs=2)  # one Ry per group
    groups, members, passes, _ = export(circuit_of(w), 8, 3)
    assert all(P.all_single for P in passes)
    assert all(P.fmode[u] == 1 for P in passes for u in range(P.n_ops) if P.param_mask >> u & 1)
    w = wl.qcl(8, 2, 2)  # Rx Rz Rx groups
    groups, members, passes, _ = export(circuit_of(w), 8, 3)
    assert not any(P.all_single for P in passes)


def _low_rank(vecs, w):
    """GF(2) rank of the low w bits of the given address vectors."""
    basis = [0] * w
    r = 0
    for v in vecs:
        x = int(v) & ((1 << w) - 1)
        for h in range(w - 1, -1, -1):
            if not (x >> h) & 1:
                continue
            if basis[h]:
                x ^= basis[h]
            else:
                basis[h] = x
                r += 1
                break
    return r


@pytest.mark.parametrize("name,t,R", [("mcvqe", 10, 4), ("mcvqe", 11, 4), ("qcl", 12, 4)])
def test_relabeled_lanes_hit_distinct_banks(name, t, R):
    """The planner's shared-memory positions: in every relabeling pass the
    lanes of one wavefront (tile bits 0-3) store from four distinct banks
    pairs, and in every stage the lane bits' load and store vectors stay as
    independent as the stage's positions allow (here: full rank for at
    least 90 % of the stages)."""
    w = wl.mcvqe(22, 8, "nn+nnn", n_refs=2) if name == "mcvqe" else wl.qcl(19, 10, 2)
    passes = export(circuit_of(w), t, R, relabel=True)[2]
    csz, sw = 8, 4
    full = total = 0
    for P in passes:
        assert _low_rank([P.nat[b] // csz for b in range(sw)], sw) == sw
        for s in range(P.n_stages):
            sg = P.st[s]
            total += 2
            full += _low_rank([sg.ldt[k] // csz for k in range(sw)], sw) == sw
            full += _low_rank([sg.stt[k] // csz for k in range(sw)], sw) == sw
    assert full >= 0.9 * total


def test_plan_info_reports_the_relabeling_plan_and_no_relabel():
    """sv_plan_info gives the pass count of the plan the energy and gradient
    paths run (relabeling), and of the identity layout with no_relabel."""
    w = wl.mcvqe(22, 8, "nn+nnn", n_refs=2)
    c = circuit_of(w)
    moved = sv.sv_plan_info(c, "c64", sv.plan_opts(reg_bits=4, tile_bits=10))
    ident = sv.sv_plan_info(c, "c64", sv.plan_opts(reg_bits=4, tile_bits=10, no_relabel=True))
    assert moved["n_passes"] == len(export(c, 10, 4, relabel=True)[2])
    assert ident["n_passes"] == len(export(c, 10, 4)[2])
    assert moved["n_passes"] < ident["n_passes"]


@pytest.mark.parametrize("seed", [3, 4, 5, 6])
@pytest.mark.parametrize("dtype", [0, 1])
def test_relabeling_random_circuits(seed, dtype):
    """Random circuits with CZ, encodings and long-range CNOTs at 10-11
    qubits through narrow tiles (many passes, many relabelings), both
    amplitude sizes: the forward model leaves the oracle's state in the
    exported layout."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 12))
    t, R = [(7, 2), (8, 3), (7, 1)][seed % 3]
    if dtype == 1 and R > 3:
        R = 3
    w = wl.random_workload(n, 90, 4, 1, seed=100 + seed, with_encoding=bool(seed % 2))
    groups, members, passes, lay = export(circuit_of(w), t, R, dtype=dtype, relabel=True)
    assert sorted(lay) == list(range(n))
    xs = [None if w.inputs is None else w.inputs[0]]
    mats = [group_mats(groups, members, w.theta, xs[0])]
    psi = init_states(w, 1)
    for P in passes:
        run_fwd(P, psi, mats, 16 if dtype else 8)
    np.testing.assert_allclose(psi[0], to_layout(oracle.state(w, instance=0), lay), atol=1e-12)


@pytest.mark.parametrize("name", ["mcvqe8", "rand8_cz"])
def test_relabeled_sweep_with_moved_hamiltonian(name):
    """A full relabeled sweep: forward passes, then lambda = H psi by the H
    passes of the Hamiltonian moved to the final layout (the same plan the
    library builds), then the reverse passes: energies and gradient equal the
    oracle's."""
    w = CASES[name]()
    n = w.n_qubits
    groups, members, passes, lay = export(circuit_of(w), 7, 2, relabel=True)
    I = w.n_instances
    xs = [None if w.inputs is None else w.inputs[i] for i in range(I)]
    mats = [group_mats(groups, members, w.theta, xs[i]) for i in range(I)]
    psi = init_states(w, I)
    for P in passes:
        run_fwd(P, psi, mats, 8)
    obs = sv.PauliSum(n, moved_letters(np.asarray(w.pauli_letters), lay), w.pauli_coeffs)
    plan = export_h(obs, 7, 4)
    lam = np.zeros_like(psi)
    E = np.zeros(I)
    for i in range(I):
        lam[i], E[i] = run_h(plan, psi[i], n)
    rho = [[np.zeros((2, 2), complex) for _ in groups] for _ in range(I)]
    for P in reversed(passes):
        run_rev(P, psi, lam, mats, rho, 8)
    wts = oracle.cost_weights(w, E)
    grad = np.zeros(w.n_params)
    for i in range(I):
        group_gradients(groups, members, rho[i], w.theta, xs[i], grad, wts[i])
    L, E_o, g_o = oracle.grad_param_shift(w)
    np.testing.assert_allclose(E, E_o, atol=1e-12)
    np.testing.assert_allclose(grad, g_o, atol=1e-11)


def test_three_shears_equal_the_rotation():
    """The tile passes apply a real rotation [[c, -s], [s, c]] with c > 0 as
    x += a y; y += b x; x += a y with a = -s / (1 + c), b = s: the product of
    the three shears is the rotation, for every angle with |angle| < pi/2,
    and the staged coefficients stay in [-1, 1]."""
    rng = np.random.default_rng(3)
    for phi in np.concatenate([rng.uniform(-np.pi / 2, np.pi / 2, 200), [0.0, 1e-8, -1.5707]]):
        c, s = np.cos(phi), np.sin(phi)
        a, b = -s / (1 + c), s
        assert abs(a) <= 1 and abs(b) <= 1
        shear_x = np.array([[1.0, a], [0.0, 1.0]])
        shear_y = np.array([[1.0, 0.0], [b, 1.0]])
        np.testing.assert_allclose(shear_x @ shear_y @ shear_x, [[c, -s], [s, c]], atol=1e-14)
        # applied in place to a complex pair, in the kernel's order
        x, y = rng.normal(size=2) + 1j * rng.normal(size=2)
        x1 = x + a * y
        y1 = y + b * x1
        x1 = x1 + a * y1
        np.testing.assert_allclose([x1, y1], [c * x - s * y, s * x + c * y], atol=1e-14)
