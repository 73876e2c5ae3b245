"""Pins of the data-driven circuit learning oracle (Sec. 4.2, Eq. 3), on CPU.

The Jensen-Shannon divergence against facts that do not restate its
formula (zero for equal distributions, log 2 for disjoint supports,
symmetry, bounds), the Bell-pair start of the circuit, and the chain-rule
parameter-shift gradient against central differences and against a target
equal to the circuit's own output distribution (a minimum: zero gradient).
"""
import numpy as np
import pytest

import oracle
import workloads as wl


def test_js_zero_for_equal_distributions():
    rng = np.random.default_rng(1)
    P = rng.random(64); P /= P.sum()
    assert abs(oracle.js_divergence(P, P)) < 1e-15


def test_js_log2_for_disjoint_supports():
    P = np.array([0.5, 0.5, 0.0, 0.0])
    Q = np.array([0.0, 0.0, 0.25, 0.75])
    assert oracle.js_divergence(P, Q) == pytest.approx(np.log(2.0), abs=1e-15)


def test_js_symmetric_and_bounded():
    rng = np.random.default_rng(2)
    for _ in range(20):
        P = rng.random(32) ** 3; P /= P.sum()
        Q = rng.random(32) ** 3; Q /= Q.sum()
        a, b = oracle.js_divergence(P, Q), oracle.js_divergence(Q, P)
        assert a == pytest.approx(b, abs=1e-15)
        assert 0.0 < a < np.log(2.0)


def test_js_is_half_the_kl_sum_to_the_mixture():
    # JS = (KL(P|M) + KL(Q|M)) / 2 with scipy's relative entropy
    from scipy.special import rel_entr
    rng = np.random.default_rng(3)
    P = rng.random(16); P /= P.sum()
    Q = rng.random(16); Q /= Q.sum()
    M = 0.5 * (P + Q)
    ref = 0.5 * (rel_entr(P, M).sum() + rel_entr(Q, M).sum())
    assert oracle.js_divergence(P, Q) == pytest.approx(ref, abs=1e-15)


def test_bell_pairs_distribution():
    w = wl.ddcl(6, 0)  # no layers: only the Bell pairs
    Q = oracle.output_distribution(w)
    # each pair (2i, 2i+1) is (|00> + |11>)/sqrt2: 8 equally likely bitstrings
    support = [b for b in range(64) if all(((b >> (2 * i)) & 1) == ((b >> (2 * i + 1)) & 1)
                                            for i in range(3))]
    assert np.allclose(Q[support], 1 / 8) and abs(Q.sum() - 1) < 1e-14
    assert len(support) == 8


def test_table2_parameter_count():
    for n in (20, 22, 24, 26):
        w = wl.ddcl(n, 10)
        assert w.n_params == 60 * n and 2 * w.n_params == [2400, 2640, 2880, 3120][(n - 20) // 2]


def test_param_shift_matches_finite_differences():
    w = wl.ddcl(5, 2, seed=4)
    js, g = oracle.ddcl_grad_param_shift(w)
    g_fd = oracle.ddcl_grad_finite_difference(w, h=1e-5)
    assert js == pytest.approx(oracle.ddcl_cost(w))
    assert np.max(np.abs(g - g_fd)) < 1e-8


def test_zero_gradient_when_target_is_the_output():
    w0 = wl.ddcl(6, 2, seed=5)
    target = oracle.output_distribution(w0)
    w = wl.ddcl(6, 2, seed=5, target=target)
    js, g = oracle.ddcl_grad_param_shift(w)
    assert abs(js) < 1e-14 and np.max(np.abs(g)) < 1e-12
