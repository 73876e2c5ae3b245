"""Pins of the sparse-state oracle (oracle/sparse.py), on the CPU.

The sparse simulation must agree with the dense oracle wherever both run
(every gate type, random angles, n <= 8), keep states normalised, and
reproduce the closed forms that hold at any size: at theta = 0 the 28-qubit
multi-contracted VQE state is a basis state whose energy is the sum of its
diagonal terms, and with Ry only on qubit 0 the value of Z_0 is the product
of the cosines (CNOT ladders never target qubit 0).  Its parameter-shift
gradient must match central differences of its own energies.
"""
import numpy as np
import pytest

import oracle
from oracle import sparse
import workloads as wl


def _dense(idx, amp, n):
    v = np.zeros(1 << n, dtype=np.complex128)
    v[idx] = amp
    return v


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_states_match_dense_oracle(seed):
    w = wl.random_workload(7, 80, 9, 3, seed=seed, with_encoding=(seed == 2))
    for i in range(w.n_instances):
        idx, amp = sparse.state(w, instance=i, shift_param=3, shift=0.7)
        want = oracle.state(w, instance=i, shift_param=3, shift=0.7)
        assert np.max(np.abs(_dense(idx, amp, w.n_qubits) - want)) < 1e-13
        assert np.sum(np.abs(amp) ** 2) == pytest.approx(1.0, abs=1e-13)


def test_energies_and_gradient_match_dense_oracle():
    w = wl.mcvqe(6, 3, "nn+nnn", n_refs=3)
    L, E, g = oracle.grad_param_shift(w)
    Ls, Es, gs = sparse.grad_param_shift(w)
    assert Ls == pytest.approx(L, abs=1e-13)
    assert np.max(np.abs(Es - E)) < 1e-13
    assert np.max(np.abs(gs - g)) < 1e-13


def test_bell_and_ghz():
    n = 5
    gates = [wl.Gate("H", 0)] + wl.cnot_ladder(n)
    w = wl.Workload("ghz", n, gates, 0, np.zeros(0), np.zeros((0, n), np.int8), np.zeros(0),
                    np.zeros(1, np.int64))
    idx, amp = sparse.state(w)
    assert list(idx) == [0, (1 << n) - 1]
    assert np.allclose(amp, [2 ** -0.5, 2 ** -0.5], atol=1e-15)


def _basis_after_ladders(w, ref):
    b = [(int(ref) >> q) & 1 for q in range(w.n_qubits)]
    for g in w.gates:
        if g.op == "CNOT":
            b[g.target] ^= b[g.control]
    return sum(bit << q for q, bit in enumerate(b))


def _diagonal_energy(w, j):
    e = 0.0
    for row, c in zip(np.asarray(w.pauli_letters), w.pauli_coeffs):
        if np.any((row == 1) | (row == 2)):
            continue
        e += c * (-1) ** sum((j >> q) & 1 for q in range(w.n_qubits) if row[q] == 3)
    return e


def test_28_qubit_closed_form_at_zero_angles():
    w = wl.config(4)
    th = np.zeros(w.n_params)
    E = sparse.energies(w, th, np.arange(w.n_instances))
    want = [_diagonal_energy(w, _basis_after_ladders(w, r)) for r in w.refs]
    assert np.max(np.abs(E - want)) < 1e-13


def test_28_qubit_product_of_cosines():
    n, layers = 28, 8
    gates = wl.layered_ansatz(n, layers, ("RY",), "ladder")
    rng = np.random.default_rng(9)
    th = np.zeros(n * layers)
    th[::n] = rng.uniform(-np.pi, np.pi, layers)
    letters = wl.letters_from_terms(n, [[(0, "Z")]])
    w = wl.Workload("z0", n, gates, n * layers, th, letters, np.ones(1), np.zeros(1, np.int64))
    idx, amp = sparse.state(w)
    assert len(idx) <= 1 << layers
    assert sparse.expect(idx, amp, letters, [1.0]) == pytest.approx(np.prod(np.cos(th[::n])),
                                                                     abs=1e-13)


def test_gradient_against_central_differences_at_28_qubits():
    w = wl.config(4)
    th = np.zeros(w.n_params)
    th[0::28] = w.theta[0::28]          # qubit 0 rotates in every layer
    ks = [0, 28, 5, 200]
    _, _, g = sparse.grad_param_shift(w, th, params=ks)
    h = 1e-5
    for k, gk in zip(ks, g):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        Lp = oracle.cost_from_energies(w, sparse.energies(w, tp, np.arange(w.n_instances)))
        Lm = oracle.cost_from_energies(w, sparse.energies(w, tm, np.arange(w.n_instances)))
        assert gk == pytest.approx((Lp - Lm) / (2 * h), abs=1e-8)
