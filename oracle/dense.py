"""Dense 2^n brute force, an independent check of the C oracle (n <= ~8).

TEST INFRASTRUCTURE ONLY.  Builds every gate as a full 2^n x 2^n matrix by
Kronecker products, with rotation matrices taken from the matrix exponential
exp(-i a P / 2) (scipy.linalg.expm) instead of the closed cos/sin form the C
oracle uses, and builds H as a dense sum of Kronecker-product Pauli strings.
Qubit q is bit q of the basis index, so in a Kronecker product the factor for
qubit n-1 comes first.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

_PAULI = {
    0: np.eye(2, dtype=np.complex128),
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),
    2: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    3: np.array([[1, 0], [0, -1]], dtype=np.complex128),
}
_HAD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def embed(n: int, q: int, m: np.ndarray) -> np.ndarray:
    """m acting on qubit q of n, identity elsewhere."""
    out = np.array([[1.0 + 0j]])
    for k in reversed(range(n)):
        out = np.kron(out, m if k == q else np.eye(2))
    return out


def controlled(n: int, c: int, t: int, m: np.ndarray) -> np.ndarray:
    """|0><0|_c (x) I + |1><1|_c (x) m_t."""
    p0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    p1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
    a = np.array([[1.0 + 0j]])
    b = np.array([[1.0 + 0j]])
    for k in reversed(range(n)):
        a = np.kron(a, p0 if k == c else np.eye(2))
        b = np.kron(b, p1 if k == c else (m if k == t else np.eye(2)))
    return a + b


def rotation(letter: int, a: float) -> np.ndarray:
    return expm(-0.5j * a * _PAULI[letter])


def gate_matrix(n, g, theta, x=None, shift_param=-1, shift=0.0):
    if g.op in ("RX", "RY", "RZ"):
        a = g.angle if g.param < 0 else theta[g.param] + (shift if g.param == shift_param else 0.0)
        return embed(n, g.target, rotation("_XYZ".index(g.op[1]), a))
    if g.op == "X":
        return embed(n, g.target, _PAULI[1])
    if g.op == "H":
        return embed(n, g.target, _HAD)
    if g.op == "CNOT":
        return controlled(n, g.control, g.target, _PAULI[1])
    if g.op == "CZ":
        return controlled(n, g.control, g.target, _PAULI[3])
    if g.op == "ENC_RY_ASIN":
        return embed(n, g.target, rotation(2, np.arcsin(x[g.param])))
    if g.op == "ENC_RZ_ACOS_SQ":
        return embed(n, g.target, rotation(3, np.arccos(x[g.param] ** 2)))
    raise ValueError(g.op)


def unitary(w, theta=None, instance=0, shift_param=-1, shift=0.0):
    n = w.n_qubits
    th = w.theta if theta is None else theta
    x = None if w.inputs is None else np.asarray(w.inputs)[instance]
    U = np.eye(1 << n, dtype=np.complex128)
    for g in w.gates:
        U = gate_matrix(n, g, th, x, shift_param, shift) @ U
    return U


def state(w, theta=None, instance=0, shift_param=-1, shift=0.0):
    U = unitary(w, theta, instance, shift_param, shift)
    return U[:, int(w.refs[instance])].copy()


def pauli_string(n: int, row) -> np.ndarray:
    out = np.array([[1.0 + 0j]])
    for k in reversed(range(n)):
        out = np.kron(out, _PAULI[int(row[k])])
    return out


def hamiltonian(n: int, letters, coeffs) -> np.ndarray:
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for row, c in zip(letters, coeffs):
        H += c * pauli_string(n, row)
    return H


def energy(w, theta=None, instance=0, shift_param=-1, shift=0.0) -> complex:
    psi = state(w, theta, instance, shift_param, shift)
    H = hamiltonian(w.n_qubits, w.pauli_letters, w.pauli_coeffs)
    return complex(np.vdot(psi, H @ psi))
