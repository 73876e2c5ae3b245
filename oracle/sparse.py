"""Exact simulation of states with few nonzero amplitudes, at any qubit count.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): the test suite may
use it; the product library never imports it and shares no code with it.

A state is kept as the list of its nonzero amplitudes: sorted basis indices
and their complex128 values.  Gates act on that list directly -- a
one-qubit gate U on qubit q sends amplitude a at index j to U[b', b] a at
index j with bit q set to b' (b the bit of j), a CNOT relabels indices, a
CZ flips signs -- so circuits whose rotations are mostly identities (angle
0) stay small however many qubits they have.  This gives exact oracle
values for the full-size 28-qubit multi-contracted VQE (Sec. 4.1, Eq. 1 and
Eq. 2) at angles where only a few qubits rotate: every state the circuit
passes through is a superposition of at most 2^(number of non-identity
rotations) basis states.

Conventions are those of the dense oracle: qubit q is bit q of a basis
index, R_P(a) = exp(-i a P / 2) = cos(a/2) I - i sin(a/2) P, and
E = sum_t c_t <psi| P_t psi> with P_t psi built by applying the Pauli
letters of the string one qubit at a time.  Energies, the cost and the
parameter-shift gradient (Sec. 4.1: g_k = 1/2 [E(theta + pi/2 e_k) -
E(theta - pi/2 e_k)]) follow the definitions in ``oracle/__init__.py``.
"""
from __future__ import annotations

import numpy as np

# single-qubit matrices written from their definitions
_PAULI = {
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),        # X
    2: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),     # Y
    3: np.array([[1, 0], [0, -1]], dtype=np.complex128),       # Z
}
_LETTER_OF = {"RX": 1, "RY": 2, "RZ": 3}


def rotation(letter: int, a: float) -> np.ndarray:
    """R_P(a) = cos(a/2) I - i sin(a/2) P."""
    return np.cos(a / 2) * np.eye(2, dtype=np.complex128) - 1j * np.sin(a / 2) * _PAULI[letter]


def _combine(idx: np.ndarray, amp: np.ndarray):
    """Adds amplitudes of equal indices; drops exact zeros; sorted by index."""
    keep = amp != 0
    idx, amp = idx[keep], amp[keep]
    u, inv = np.unique(idx, return_inverse=True)
    out = np.zeros(len(u), dtype=np.complex128)
    np.add.at(out, inv, amp)
    keep = out != 0
    return u[keep], out[keep]


def apply_1q(idx, amp, q: int, m: np.ndarray):
    """psi <- (m on qubit q) psi for a state given by its nonzero entries."""
    bit = np.int64(1) << np.int64(q)
    b = (idx >> q) & 1
    base = idx & ~bit
    # entry (j, a) with bit b contributes m[0, b] a at base and m[1, b] a at base | bit
    new_idx = np.concatenate([base, base | bit])
    new_amp = np.concatenate([m[0, b] * amp, m[1, b] * amp])
    return _combine(new_idx, new_amp)


def apply_gate(idx, amp, gate, theta, x=None, shift_param=-1, shift=0.0):
    op = gate.op
    if op in _LETTER_OF:
        a = theta[gate.param] if gate.param >= 0 else gate.angle
        if gate.param >= 0 and gate.param == shift_param:
            a = a + shift
        return apply_1q(idx, amp, gate.target, rotation(_LETTER_OF[op], a))
    if op == "X":
        return apply_1q(idx, amp, gate.target, _PAULI[1])
    if op == "H":
        return apply_1q(idx, amp, gate.target, (_PAULI[1] + _PAULI[3]) / np.sqrt(2.0))
    if op == "ENC_RY_ASIN":
        return apply_1q(idx, amp, gate.target, rotation(2, np.arcsin(x[gate.param])))
    if op == "ENC_RZ_ACOS_SQ":
        return apply_1q(idx, amp, gate.target, rotation(3, np.arccos(x[gate.param] ** 2)))
    if op == "CNOT":
        # flips the target bit of every index whose control bit is 1
        c = (idx >> gate.control) & 1
        idx = idx ^ (c << gate.target)
        order = np.argsort(idx, kind="stable")
        return idx[order], amp[order]
    if op == "CZ":
        both = ((idx >> gate.control) & 1) & ((idx >> gate.target) & 1)
        return idx, np.where(both == 1, -amp, amp)
    raise ValueError(f"unknown gate {op!r}")


def state(w, theta=None, instance: int = 0, shift_param: int = -1, shift: float = 0.0):
    """(indices, amplitudes) of psi = U |ref_instance>, nonzero entries only."""
    th = np.asarray(w.theta if theta is None else theta, dtype=np.float64)
    x = None if w.inputs is None else np.asarray(w.inputs[instance], dtype=np.float64)
    idx = np.array([int(w.refs[instance])], dtype=np.int64)
    amp = np.array([1.0 + 0j])
    for g in w.gates:
        idx, amp = apply_gate(idx, amp, g, th, x, shift_param, shift)
    return idx, amp


def apply_pauli_string(idx, amp, row):
    """P psi for a Pauli row (0=I, 1=X, 2=Y, 3=Z), one letter at a time.  A
    Pauli matrix has one nonzero entry per column, so the entry (j, a) with
    bit b on the letter's qubit goes to the row r with m[r, b] != 0, times
    m[r, b]; no two entries meet, and the list is sorted once at the end."""
    idx, amp = idx.copy(), amp.copy()
    for q, letter in enumerate(row):
        if letter == 0:
            continue
        m = _PAULI[int(letter)]
        b = (idx >> q) & 1
        r = np.where(m[0, b] != 0, 0, 1)
        amp = m[r, b] * amp
        idx = (idx & ~(np.int64(1) << np.int64(q))) | (r.astype(np.int64) << q)
    order = np.argsort(idx)
    return idx[order], amp[order]


def inner(idx_a, amp_a, idx_b, amp_b) -> complex:
    """<a|b> over the common indices of two sorted entry lists."""
    common, ia, ib = np.intersect1d(idx_a, idx_b, assume_unique=True, return_indices=True)
    return complex(np.sum(np.conj(amp_a[ia]) * amp_b[ib]))


def expect(idx, amp, letters, coeffs) -> float:
    """E = sum_t c_t <psi| P_t psi>."""
    e = 0.0 + 0j
    for row, c in zip(np.asarray(letters), np.asarray(coeffs)):
        pi, pa = apply_pauli_string(idx, amp, row)
        e += c * inner(idx, amp, pi, pa)
    return float(e.real)


def _slot_energies(args):
    w, theta, slots = args
    return [expect(*state(w, theta, i, k, s), w.pauli_letters, w.pauli_coeffs)
            for i, k, s in slots]


def energies(w, theta, slot_instance, slot_shift_param=None, slot_shift=None, workers: int = 1):
    """Energy of every slot (instance, shifted parameter or -1, shift).
    workers > 1 spreads whole circuits over that many processes (started
    with spawn, so that it is safe after CUDA has been initialised)."""
    n = len(slot_instance)
    sp = np.full(n, -1) if slot_shift_param is None else np.asarray(slot_shift_param)
    sh = np.zeros(n) if slot_shift is None else np.asarray(slot_shift)
    th = np.asarray(w.theta if theta is None else theta, dtype=np.float64)
    slots = [(int(slot_instance[s]), int(sp[s]), float(sh[s])) for s in range(n)]
    if workers <= 1 or n < 2:
        return np.array(_slot_energies((w, th, slots)))
    import multiprocessing as mp
    chunks = [slots[c::workers] for c in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_slot_energies, [(w, th, c) for c in chunks])
    out = np.empty(n)
    for c, part in enumerate(parts):
        out[c::workers] = part
    return out


def grad_param_shift(w, theta=None, params=None, workers: int = 1):
    """(cost, instance energies, gradient entries of `params`) by the
    parameter-shift rule, with the cost definitions of the dense oracle."""
    import oracle
    inst, sp, sh = oracle.param_shift_slots(w, params)
    E = energies(w, theta, inst, sp, sh, workers)
    I = w.n_instances
    E0 = E[:I]
    Es = E[I:].reshape(-1, 2, I)
    dE = 0.5 * (Es[:, 0, :] - Es[:, 1, :])
    return oracle.cost_from_energies(w, E0), E0, dE @ oracle.cost_weights(w, E0)
