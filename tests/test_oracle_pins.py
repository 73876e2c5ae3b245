"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Closed forms of single-qubit rotations, Bell/GHZ amplitudes, CNOT ladders on
basis states, the encoding's Bloch vector, norm preservation, an independent
dense brute force (matrix exponentials + Kronecker products), Hermiticity and
the variational bound of Eq. 1, parameter shift against finite differences,
the closed-form energy of the MC-VQE ansatz at theta = 0, and the circuit
counts printed in Tables 1 and 2.
"""
import dataclasses
import os

import numpy as np
import pytest

import oracle
from oracle import counts, dense
import workloads as wl
from workloads import Gate, Workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def single_term(n, term):
    return wl.letters_from_terms(n, [term]), np.ones(1)


def make(n, gates, letters, coeffs, n_params=0, theta=None, refs=(0,), inputs=None):
    return Workload(name="t", n_qubits=n, gates=gates, n_params=n_params,
                    theta=np.zeros(n_params) if theta is None else np.asarray(theta, float),
                    pauli_letters=letters, pauli_coeffs=coeffs,
                    refs=np.asarray(refs, dtype=np.int64), inputs=inputs,
                    weights=np.ones(len(refs)) / len(refs))


def expval(n, gates, term, theta=None, n_params=0, ref=0, inputs=None):
    letters, coeffs = single_term(n, term)
    w = make(n, gates, letters, coeffs, n_params, theta, refs=(ref,), inputs=inputs)
    return oracle.instance_energies(w)[0]


ANGLES = np.linspace(-3.0, 3.0, 13)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_ry_closed_form(q):
    # <Z> = cos a, <X> = sin a, <Y> = 0 after Ry(a)|0>, on any qubit of three.
    for a in ANGLES:
        g = [Gate("RY", q, param=0)]
        assert expval(3, g, [(q, "Z")], [a], 1) == pytest.approx(np.cos(a), abs=1e-14)
        assert expval(3, g, [(q, "X")], [a], 1) == pytest.approx(np.sin(a), abs=1e-14)
        assert expval(3, g, [(q, "Y")], [a], 1) == pytest.approx(0.0, abs=1e-14)
        other = (q + 1) % 3
        assert expval(3, g, [(other, "Z")], [a], 1) == pytest.approx(1.0, abs=1e-14)


def test_rx_rz_closed_form():
    for a in ANGLES:
        g = [Gate("RX", 1, param=0)]
        assert expval(2, g, [(1, "Z")], [a], 1) == pytest.approx(np.cos(a), abs=1e-14)
        assert expval(2, g, [(1, "Y")], [a], 1) == pytest.approx(-np.sin(a), abs=1e-14)
        assert expval(2, g, [(1, "X")], [a], 1) == pytest.approx(0.0, abs=1e-14)
        # Rz on |0> changes nothing observable; on |+> it turns X towards Y.
        assert expval(1, [Gate("RZ", 0, param=0)], [(0, "Z")], [a], 1) == pytest.approx(1.0)
        gz = [Gate("H", 0), Gate("RZ", 0, param=0)]
        assert expval(1, gz, [(0, "X")], [a], 1) == pytest.approx(np.cos(a), abs=1e-14)
        assert expval(1, gz, [(0, "Y")], [a], 1) == pytest.approx(np.sin(a), abs=1e-14)


def test_ry_merging_amplitudes():
    # Sec. 4.1: Ry(a) Ry(b) = Ry(a + b), used to merge adjacent Ry gates.
    rng = np.random.default_rng(1)
    for _ in range(10):
        a, b = rng.uniform(-4, 4, 2)
        pre = [Gate("H", 0), Gate("H", 1), Gate("CNOT", 1, 0)]
        w2 = make(2, pre + [Gate("RY", 1, param=0), Gate("RY", 1, param=1)],
                  *single_term(2, [(0, "Z")]), 2, [a, b])
        w1 = make(2, pre + [Gate("RY", 1, param=0)], *single_term(2, [(0, "Z")]), 1, [a + b])
        assert np.allclose(oracle.state(w2), oracle.state(w1), atol=1e-15, rtol=0)


def test_bell_and_ghz_amplitudes():
    h = 1 / np.sqrt(2)
    w = make(2, [Gate("RY", 0, angle=np.pi / 2), Gate("CNOT", 1, 0)], *single_term(2, [(0, "Z")]))
    assert np.allclose(oracle.state(w), [h, 0, 0, h], atol=1e-15)
    w = make(2, [Gate("H", 0), Gate("CNOT", 1, 0)], *single_term(2, [(0, "Z")]))
    assert np.allclose(oracle.state(w), [h, 0, 0, h], atol=1e-15)
    for n in (3, 5, 7):
        w = make(n, [Gate("H", 0)] + wl.cnot_ladder(n), *single_term(n, [(0, "Z")]))
        psi = oracle.state(w)
        expect = np.zeros(1 << n, complex)
        expect[0] = expect[-1] = h
        assert np.allclose(psi, expect, atol=1e-15)


def test_ladder_and_ring_on_basis_states():
    n = 6
    for ref in range(1 << n):
        bits = [(ref >> i) & 1 for i in range(n)]
        prefix = np.cumsum(bits) % 2             # bit i <- b_0 ^ ... ^ b_i
        lad = sum(int(prefix[i]) << i for i in range(n))
        ring = lad & ~1 | (int(sum(bits[1:]) % 2))  # bit 0 <- b_1 ^ ... ^ b_{n-1}
        for gates, target in ((wl.cnot_ladder(n), lad), (wl.cnot_ring(n), ring)):
            w = make(n, gates, *single_term(n, [(0, "Z")]), refs=(ref,))
            psi = oracle.state(w)
            assert abs(psi[target]) == pytest.approx(1.0, abs=1e-15)


def test_encoding_bloch_vector():
    # Ry(arcsin x) then Rz(arccos x^2) on |0>: Bloch vector (x^3, x sqrt(1-x^4), sqrt(1-x^2)).
    for x in np.linspace(-1, 1, 11):
        g = wl.encoding_gates(1)
        inp = np.array([[x]])
        assert expval(1, g, [(0, "Z")], inputs=inp) == pytest.approx(np.sqrt(1 - x * x), abs=1e-14)
        assert expval(1, g, [(0, "X")], inputs=inp) == pytest.approx(x ** 3, abs=1e-14)
        assert expval(1, g, [(0, "Y")], inputs=inp) == pytest.approx(x * np.sqrt(1 - x ** 4), abs=1e-14)


@pytest.mark.parametrize("n", [1, 2, 5, 10])
def test_norm_preserved(n):
    w = wl.random_workload(n, 60, 3, seed=n, with_encoding=True)
    for i in range(w.n_instances):
        assert np.linalg.norm(oracle.state(w, instance=i)) == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_dense_brute_force(n):
    for seed in range(3):
        w = wl.random_workload(n, 40, 6, n_instances=2, seed=10 * n + seed, with_encoding=seed == 2)
        for i in range(w.n_instances):
            assert np.allclose(oracle.state(w, instance=i), dense.state(w, instance=i),
                               atol=1e-12, rtol=0)
            assert oracle.instance_energies(w)[i] == pytest.approx(dense.energy(w, instance=i).real,
                                                                  abs=1e-12)
        k = int(seed % w.n_params) if w.n_params else -1
        if k >= 0:
            assert np.allclose(oracle.state(w, shift_param=k, shift=0.7),
                               dense.state(w, shift_param=k, shift=0.7), atol=1e-12)


def test_dense_brute_force_workload_shapes():
    for w in (wl.vqe_random_pauli(4, 2, 10), wl.mcvqe(5, 2), wl.qcl(4, 2, 3)):
        E = oracle.instance_energies(w)
        for i in range(w.n_instances):
            assert E[i] == pytest.approx(dense.energy(w, instance=i).real, abs=1e-12)


def test_energy_is_real():
    # Eq. 2 coefficients are real and every Pauli string is Hermitian.
    w = wl.random_workload(5, 50, 20, n_instances=3, seed=4)
    re, im = oracle.energies(w, None, np.arange(3), return_imag=True)
    assert np.max(np.abs(im)) < 1e-13


@pytest.mark.parametrize("make_w", [lambda: wl.mcvqe(6, 3), lambda: wl.vqe_random_pauli(5, 2, 12),
                                    lambda: wl.random_workload(7, 80, 15, 3, seed=7)])
def test_variational_bound(make_w):
    # Eq. 1: E_0 <= <H>(theta) for every theta.
    w = make_w()
    lam = np.linalg.eigvalsh(dense.hamiltonian(w.n_qubits, w.pauli_letters, w.pauli_coeffs))[0]
    rng = np.random.default_rng(3)
    for _ in range(5):
        th = rng.uniform(-np.pi, np.pi, w.n_params)
        assert np.all(oracle.instance_energies(w, th) >= lam - 1e-12)


@pytest.mark.parametrize("make_w", [
    lambda: wl.vqe_random_pauli(4, 2, 10),
    lambda: wl.mcvqe(4, 2),
    lambda: wl.qcl(3, 2, 5),
    lambda: wl.random_workload(4, 30, 8, 3, seed=2, cost="mse", with_encoding=True),
])
def test_param_shift_matches_finite_difference(make_w):
    w = make_w()
    L, E, g = oracle.grad_param_shift(w)
    assert L == pytest.approx(oracle.loss(w), abs=1e-14)
    g_fd = oracle.grad_finite_difference(w, h=1e-5)
    assert np.allclose(g, g_fd, atol=2e-8, rtol=0)


def test_single_gate_derivative():
    for a in ANGLES:
        w = make(1, [Gate("RY", 0, param=0)], *single_term(1, [(0, "Z")]), 1, [a])
        _, _, g = oracle.grad_param_shift(w)
        assert g[0] == pytest.approx(-np.sin(a), abs=1e-14)


@pytest.mark.parametrize("n,layers", [(8, 4), (12, 3)])
def test_mcvqe_energy_at_zero_angles(n, layers):
    # theta = 0: the ansatz is the CNOT ladders alone, the state is a basis
    # state and only Z / ZZ terms of Eq. 2 survive.
    w = wl.mcvqe(n, layers)
    E = oracle.instance_energies(w, np.zeros(w.n_params))
    a = w.pauli_coeffs[:n]
    pairs = wl.all_pairs(n)
    f = w.pauli_coeffs[2 * n:].reshape(-1, 4)[:, 3]
    for i, ref in enumerate(w.refs):
        b = np.array([(int(ref) >> q) & 1 for q in range(n)])
        for _ in range(layers):
            b = np.cumsum(b) % 2
        s = 1 - 2 * b
        closed = float(np.dot(a, s) + sum(fc * s[p] * s[q] for fc, (p, q) in zip(f, pairs)))
        assert E[i] == pytest.approx(closed, abs=1e-13)


@pytest.mark.parametrize("n", [5, 9])
def test_z0_product_of_cosines(n):
    # Ry only on qubit 0 (other angles 0) + CNOT ladders: a ladder never
    # targets qubit 0, so Z_0 commutes with it.  The X_0 part made by a
    # rotation spreads, after k ladders, onto the qubits of row k of Pascal's
    # triangle mod 2; with fewer ladders than qubits that set always holds a
    # qubit other than 0 that starts in |0>, so the part averages to zero and
    # <Z_0> = prod_l cos(theta_{l,0}).
    layers = 5
    gates = wl.layered_ansatz(n, layers, ("RY",), "ladder")
    rng = np.random.default_rng(5)
    th = np.zeros(n * layers)
    th[::n] = rng.uniform(-np.pi, np.pi, layers)
    e = expval(n, gates, [(0, "Z")], th, n * layers)
    assert e == pytest.approx(np.prod(np.cos(th[::n])), abs=1e-13)


def _golden(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return [tuple(int(v) for v in r) for r in rows]


def test_table1_counts():
    for nq, nh, nth, circ in _golden("mcvqe_table1_counts.txt"):
        assert counts.mcvqe_paper_counts(nq) == (nh, nth, circ)


def test_table2_counts():
    for nq, nth, circ in _golden("ddcl_table2_counts.txt"):
        assert counts.ddcl_paper_counts(nq) == (nth, circ)


def test_config_shapes():
    sizes = [(4, 22, 16, 10, 1), (8, 60, 32, 128, 9), (12, 24 + 6 * 48, 216, 1, 256),
             (20, 40 + 10 * 80, 600, 1, 64), (28, 8 * 55, 224, 268, 8)]
    for idx, (n, ng, P, T, I) in enumerate(sizes):
        w = wl.config(idx)
        assert (w.n_qubits, len(w.gates), w.n_params, w.n_terms, w.n_instances) == (n, ng, P, T, I)
    assert wl.config(1).n_slots_param_shift == 585
    assert counts.batched_param_shift_slots(216, 256) == 110848


def test_sample_shots_pins():
    """The shot sampler against fixed cases: a two-outcome distribution at
    known uniforms, a basis state, and frequencies of a Bell state."""
    psi = np.array([0.5, np.sqrt(0.75)], dtype=complex)  # P = (0.25, 0.75)
    s, _ = oracle.sample_shots(psi, [0.0, 0.1, 0.2499, 0.2501, 0.9, 0.999999])
    assert list(s) == [0, 0, 0, 1, 1, 1]
    e5 = np.zeros(16, dtype=complex); e5[5] = 1.0
    s, _ = oracle.sample_shots(e5, np.random.default_rng(0).random(100))
    assert np.all(s == 5)
    bell = np.zeros(4, dtype=complex); bell[0] = bell[3] = 2 ** -0.5
    s, _ = oracle.sample_shots(bell, np.random.default_rng(1).random(20000))
    assert set(np.unique(s)) == {0, 3}
    assert abs(np.mean(s == 0) - 0.5) < 0.02


def test_paper_mcvqe_circuit_reproduces_table1():
    """The paper-exact MC-VQE circuit (CIS references, 6-Ry/2-CNOT entanglers
    with merged rotations) has Table 1's N_H and N_theta; each parameter sits
    in exactly one gate."""
    rows = np.loadtxt(os.path.join(GOLDEN, "mcvqe_table1_counts.txt"), dtype=np.int64)
    for nq, nh, nth, circ in rows:
        w = wl.mcvqe_paper(int(nq))
        assert (w.n_terms, w.n_params, 2 * w.n_terms * w.n_params) == (nh, nth, circ)
        params = [g.param for g in w.gates if g.op in ("RX", "RY", "RZ")]
        assert sorted(params) == list(range(w.n_params))


def test_cis_preparation_closed_form():
    """The CIS preparation alone gives sum_i c_i |e_i> with the closed-form c."""
    n = 6
    w = wl.mcvqe_paper(n, n_refs=3, seed=7)
    prep = dataclasses.replace(w, gates=wl.cis_prep_gates(n), n_params=0, theta=np.zeros(0))
    for r in range(3):
        psi = oracle.state(prep, instance=r)
        c = wl.cis_coefficients(w.meta["beta"][r])
        want = np.zeros(1 << n); want[[1 << i for i in range(n)]] = c
        np.testing.assert_allclose(psi, want, atol=1e-14)
        assert abs(np.sum(c ** 2) - 1) < 1e-14


def test_paper_mcvqe_gradient_finite_differences():
    w = wl.mcvqe_paper(5, n_refs=2, seed=3)
    L, E, g = oracle.grad_param_shift(w)
    np.testing.assert_allclose(g, oracle.grad_finite_difference(w, h=1e-5), atol=1e-8)
