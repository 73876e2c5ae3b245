"""CPU oracle for the batched state-vector gradient path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product library
(``paper_2406_03466_gb300``) never imports, links or runs it, and the two
share no code: the only common input is the seeded generator module
``workloads``.

The heavy lifting is the plain complex128 C simulator in ``sv_oracle.c``
(exact state-vector simulation and direct Pauli-sum expectation values, paper
Sec. 4.1).  This module adds, in plain numpy:

* the cost of a workload: the weighted (state-averaged) energy of the
  multi-contracted VQE (Sec. 4.1, the paragraph on averaging the energy over
  all monomers) or the mean squared error of circuit learning;
* the parameter-shift gradient, g_k = 1/2 [E(theta + pi/2 e_k) -
  E(theta - pi/2 e_k)] for generators with P^2 = I (Sec. 4.1, the
  O(2 N_H N_theta) parameter-shift count), chained through the cost;
* central finite differences of the cost, as an independent check.

A dense 2^n brute force lives in ``oracle.dense``; circuit counting of the
paper's Tables 1 and 2 in ``oracle.counts``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP over circuits)."""
    src = os.path.join(_HERE, "sv_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "sv_oracle.h"))):
        return _LIB_PATH
    os.makedirs(_BUILD_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Circuit(ctypes.Structure):
    _fields_ = [
        ("n_qubits", ctypes.c_int), ("n_gates", ctypes.c_int), ("n_params", ctypes.c_int),
        ("input_dim", ctypes.c_int), ("op", ctypes.c_void_p), ("target", ctypes.c_void_p),
        ("control", ctypes.c_void_p), ("param", ctypes.c_void_p), ("angle", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_state.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, P, P]
            lib.orc_expect_state.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P]
            lib.orc_energies.argtypes = [P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P,
                                         P, P, ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class _CircuitArgs:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, w):
        ops, tgt, ctl, par, ang = w.gate_array()
        self.arrays = [np.ascontiguousarray(a) for a in (ops, tgt, ctl, par, ang)]
        d = 0 if w.inputs is None else int(np.asarray(w.inputs).shape[1])
        self.struct = _Circuit(w.n_qubits, len(w.gates), w.n_params, d,
                               *[a.ctypes.data for a in self.arrays])


def _check(status):
    if status != 0:
        raise RuntimeError(f"oracle error status {status}")


def _theta(w, theta):
    return np.ascontiguousarray(w.theta if theta is None else theta, dtype=np.float64)


def _instance_inputs(w, i):
    if w.inputs is None:
        return None
    return np.ascontiguousarray(np.asarray(w.inputs, dtype=np.float64)[i])


def state(w, theta=None, instance: int = 0, shift_param: int = -1, shift: float = 0.0):
    """Final complex128 state of one instance's circuit."""
    lib = _load()
    c = _CircuitArgs(w)
    th = _theta(w, theta)
    x = _instance_inputs(w, instance)
    out = np.zeros(2 << w.n_qubits, dtype=np.float64)
    _check(lib.orc_state(ctypes.byref(c.struct), _ptr(th), shift_param, shift,
                         int(w.refs[instance]), _ptr(x), _ptr(out)))
    return out.view(np.complex128)


def expect_state(psi, letters, coeffs):
    """Complex sum_t c_t <psi|P_t|psi> of an explicit state."""
    lib = _load()
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(round(np.log2(psi.size)))
    letters = np.ascontiguousarray(letters, dtype=np.int8)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib.orc_expect_state(_ptr(psi.view(np.float64)), n, len(coeffs), _ptr(letters),
                                _ptr(coeffs), ctypes.byref(re), ctypes.byref(im)))
    return complex(re.value, im.value)


def energies(w, theta, slot_instance, slot_shift_param=None, slot_shift=None,
             n_threads: int = 0, return_imag: bool = False):
    """Energies of a list of circuit slots (instance, shifted param, shift)."""
    lib = _load()
    c = _CircuitArgs(w)
    th = _theta(w, theta)
    slot_instance = np.asarray(slot_instance, dtype=np.int64)
    S = len(slot_instance)
    refs = np.ascontiguousarray(np.asarray(w.refs, dtype=np.int64)[slot_instance])
    xs = None
    if w.inputs is not None:
        xs = np.ascontiguousarray(np.asarray(w.inputs, dtype=np.float64)[slot_instance])
    sp = np.ascontiguousarray(np.full(S, -1, np.int32) if slot_shift_param is None
                              else np.asarray(slot_shift_param, dtype=np.int32))
    sh = np.ascontiguousarray(np.zeros(S) if slot_shift is None
                              else np.asarray(slot_shift, dtype=np.float64))
    letters = np.ascontiguousarray(w.pauli_letters, dtype=np.int8)
    coeffs = np.ascontiguousarray(w.pauli_coeffs, dtype=np.float64)
    re = np.zeros(S)
    im = np.zeros(S)
    _check(lib.orc_energies(ctypes.byref(c.struct), _ptr(th), len(coeffs), _ptr(letters),
                            _ptr(coeffs), S, _ptr(refs), _ptr(xs), _ptr(sp), _ptr(sh),
                            _ptr(re), _ptr(im), int(n_threads)))
    return (re, im) if return_imag else re


def instance_energies(w, theta=None, n_threads: int = 0):
    return energies(w, theta, np.arange(w.n_instances), n_threads=n_threads)


def cost_from_energies(w, E):
    """Scalar cost: sum_i w_i E_i (state averaging) or mean_i (E_i - y_i)^2."""
    E = np.asarray(E, dtype=np.float64)
    if w.cost == "linear":
        return float(np.dot(np.asarray(w.weights, dtype=np.float64), E))
    if w.cost == "mse":
        return float(np.mean((E - np.asarray(w.targets)) ** 2))
    raise ValueError(w.cost)


def cost_weights(w, E):
    """dL/dE_i for every instance."""
    E = np.asarray(E, dtype=np.float64)
    if w.cost == "linear":
        return np.asarray(w.weights, dtype=np.float64).copy()
    if w.cost == "mse":
        return 2.0 * (E - np.asarray(w.targets)) / len(E)
    raise ValueError(w.cost)


def loss(w, theta=None, n_threads: int = 0):
    return cost_from_energies(w, instance_energies(w, theta, n_threads))


def param_shift_slots(w, params=None):
    """The parameter-shift batch: every instance unshifted, then for each k,
    +pi/2 for every instance, then -pi/2 for every instance."""
    I = w.n_instances
    ks = np.arange(w.n_params) if params is None else np.asarray(params)
    inst = [np.arange(I)]
    sp = [np.full(I, -1)]
    sh = [np.zeros(I)]
    for k in ks:
        for sign in (+1.0, -1.0):
            inst.append(np.arange(I))
            sp.append(np.full(I, k))
            sh.append(np.full(I, sign * np.pi / 2))
    return np.concatenate(inst), np.concatenate(sp), np.concatenate(sh)


def grad_param_shift(w, theta=None, params=None, n_threads: int = 0):
    """(cost, instance energies, gradient) by the parameter-shift rule."""
    inst, sp, sh = param_shift_slots(w, params)
    E = energies(w, theta, inst, sp, sh, n_threads=n_threads)
    I = w.n_instances
    E0 = E[:I]
    Es = E[I:].reshape(-1, 2, I)
    dE = 0.5 * (Es[:, 0, :] - Es[:, 1, :])        # (K, I) dE_i/dtheta_k
    g = dE @ cost_weights(w, E0)
    return cost_from_energies(w, E0), E0, g


def grad_finite_difference(w, theta=None, h: float = 1e-5, n_threads: int = 0):
    """Central differences of the cost, [L(theta+h e_k) - L(theta-h e_k)] / 2h."""
    th = _theta(w, theta)
    g = np.zeros(w.n_params)
    for k in range(w.n_params):
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        g[k] = (loss(w, tp, n_threads) - loss(w, tm, n_threads)) / (2 * h)
    return g


# ---------------------------------------------- data-driven circuit learning

def js_divergence(P, Q):
    """Jensen-Shannon divergence of Sec. 4.2 Eq. 3 with natural logarithms:
    JS = 1/2 sum_b (P log(P/M) + Q log(Q/M)), M = (P + Q)/2, 0 log 0 = 0."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    M = 0.5 * (P + Q)
    total = 0.0
    for X in (P, Q):
        nz = X > 0
        total += float(np.sum(X[nz] * np.log(X[nz] / M[nz])))
    return 0.5 * total


def output_distribution(w, theta=None, shift_param: int = -1, shift: float = 0.0):
    """P_theta(b) = |<b|psi>|^2: all qubits measured in the Z basis (Sec. 4.2)."""
    psi = state(w, theta, 0, shift_param, shift)
    return (psi.real ** 2 + psi.imag ** 2)


def ddcl_cost(w, theta=None):
    """JS(P | P_theta) of the workload's target distribution P."""
    return js_divergence(w.target_dist, output_distribution(w, theta))


def ddcl_grad_param_shift(w, theta=None, params=None):
    """(JS, gradient): each P_theta(b) is the expectation of the projector on
    |b>, so its derivative is the parameter-shift difference of the shifted
    distributions; the chain rule weights it with dJS/dP_theta(b) =
    1/2 log(P_theta(b) / M(b)) (0 where P_theta(b) = 0)."""
    P = np.asarray(w.target_dist, dtype=np.float64)
    Q = output_distribution(w, theta)
    M = 0.5 * (P + Q)
    wb = np.zeros_like(Q)
    nz = Q > 0
    wb[nz] = 0.5 * np.log(Q[nz] / M[nz])
    ks = np.arange(w.n_params) if params is None else np.asarray(params)
    g = np.zeros(len(ks))
    for i, k in enumerate(ks):
        Qp = output_distribution(w, theta, int(k), np.pi / 2)
        Qm = output_distribution(w, theta, int(k), -np.pi / 2)
        g[i] = float(np.dot(wb, 0.5 * (Qp - Qm)))
    return js_divergence(P, Q), g


def ddcl_grad_finite_difference(w, theta=None, params=None, h: float = 1e-5):
    """Central differences of JS(P | P_theta)."""
    th = _theta(w, theta)
    ks = np.arange(w.n_params) if params is None else np.asarray(params)
    g = np.zeros(len(ks))
    for i, k in enumerate(ks):
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        g[i] = (ddcl_cost(w, tp) - ddcl_cost(w, tm)) / (2 * h)
    return g


# ------------------------------------------------------------ shot sampling

def sample_shots(psi, uniforms):
    """Shots of a state measured in the Z basis with the caller's uniforms:
    shot s is the first basis index whose cumulative probability exceeds
    u_s times the total (FP64 probabilities |psi_b|^2)."""
    psi = np.asarray(psi)
    P = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    cdf = np.cumsum(P)
    x = np.asarray(uniforms, dtype=np.float64) * cdf[-1]
    return np.minimum(np.searchsorted(cdf, x, side="right"), P.size - 1), cdf


def max_threads() -> int:
    return int(_load().orc_max_threads())
