"""Seeded synthetic inputs for the batched state-vector gradient path.

This module is the one thing the CPU oracle and the CUDA path both read. It
holds no simulation arithmetic at all: only circuit *structure* (ordered gate
lists), random circuit parameters, Pauli strings with coefficients, reference
basis states, training inputs and training targets.

Conventions shared by every consumer (the paper fixes none of them):

* qubit ``q`` is bit ``q`` of a basis index (little-endian);
* a gate is ``Gate(op, target, control, param, angle)``.  For the parametric
  rotations ``RX``/``RY``/``RZ`` the angle is ``theta[param]`` when
  ``param >= 0`` and the literal ``angle`` otherwise.  For the two encoding
  gates ``ENC_RY_ASIN`` / ``ENC_RZ_ACOS_SQ`` ``param`` is a column of the
  instance's input row.  ``control`` is ``-1`` for one-qubit gates;
* Pauli strings are int8 rows over qubits with 0=I, 1=X, 2=Y, 3=Z;
* an *instance* is one term of the cost: a reference state (multi-contracted
  VQE, paper Sec. 4.1) or a training sample (circuit learning, Sec. 4.2).

Workload shapes follow the paper's two use cases (Eq. 2 spin Hamiltonian with
state averaging over references; a data-encoding circuit learning model) with
synthetic coefficients, since the paper's ab-initio coefficients and target
distribution are not published.  Every generator draws from
``numpy.random.default_rng(seed)`` in a fixed order: Hamiltonian coefficients,
then circuit parameters, then inputs, then target noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

GATE_OPS = ("RX", "RY", "RZ", "CNOT", "X", "H", "CZ", "ENC_RY_ASIN", "ENC_RZ_ACOS_SQ")
PAULI_LETTERS = "IXYZ"


@dataclass(frozen=True)
class Gate:
    op: str
    target: int
    control: int = -1
    param: int = -1
    angle: float = 0.0

    def __post_init__(self):
        if self.op not in GATE_OPS:
            raise ValueError(f"unknown gate op {self.op!r}")


@dataclass
class Workload:
    """One gradient problem: a parametrised circuit, an observable and instances."""

    name: str
    n_qubits: int
    gates: List[Gate]
    n_params: int
    theta: np.ndarray                  # (P,) float64
    pauli_letters: np.ndarray          # (T, n) int8
    pauli_coeffs: np.ndarray           # (T,) float64
    refs: np.ndarray                   # (I,) int64 reference basis index per instance
    inputs: Optional[np.ndarray] = None   # (I, D) float64 encoding inputs per instance
    targets: Optional[np.ndarray] = None  # (I,) float64 training targets (cost "mse")
    weights: Optional[np.ndarray] = None  # (I,) float64 instance weights (cost "linear")
    cost: str = "linear"               # "linear": sum_i w_i E_i ; "mse": mean_i (E_i - y_i)^2
    meta: dict = field(default_factory=dict)
    # cost "js": target distribution over the 2^n bitstrings (data-driven
    # circuit learning, Sec. 4.2 Eq. 3); the observable is unused
    target_dist: Optional[np.ndarray] = None

    @property
    def n_instances(self) -> int:
        return int(len(self.refs))

    @property
    def n_terms(self) -> int:
        return int(len(self.pauli_coeffs))

    @property
    def n_slots_param_shift(self) -> int:
        """Circuits in one parameter-shift gradient: (2P + 1) per instance."""
        return (2 * self.n_params + 1) * self.n_instances

    def gate_array(self):
        """Gate list as parallel numpy arrays (op index, target, control, param, angle)."""
        ops = np.array([GATE_OPS.index(g.op) for g in self.gates], dtype=np.int32)
        tgt = np.array([g.target for g in self.gates], dtype=np.int32)
        ctl = np.array([g.control for g in self.gates], dtype=np.int32)
        par = np.array([g.param for g in self.gates], dtype=np.int32)
        ang = np.array([g.angle for g in self.gates], dtype=np.float64)
        return ops, tgt, ctl, par, ang


# --------------------------------------------------------------------------
# circuit structure helpers
# --------------------------------------------------------------------------

def cnot_ladder(n: int) -> List[Gate]:
    """CNOT(i -> i+1) for i = 0..n-2, in that order."""
    return [Gate("CNOT", target=i + 1, control=i) for i in range(n - 1)]


def cnot_ring(n: int) -> List[Gate]:
    """CNOT(i -> i+1 mod n) for i = 0..n-1; the wrap-around gate comes last."""
    if n < 2:
        return []
    return [Gate("CNOT", target=(i + 1) % n, control=i) for i in range(n)]


def layered_ansatz(n: int, layers: int, rot_ops: Sequence[str], entangler: str,
                   first_param: int = 0) -> List[Gate]:
    """Layers of per-qubit rotations followed by a CNOT ladder or ring.

    Parameter index layout is layer-major, then qubit, then gate-within-qubit.
    """
    gates: List[Gate] = []
    p = first_param
    for _ in range(layers):
        for q in range(n):
            for op in rot_ops:
                gates.append(Gate(op, target=q, param=p))
                p += 1
        if entangler == "ladder":
            gates.extend(cnot_ladder(n))
        elif entangler == "ring":
            gates.extend(cnot_ring(n))
        elif entangler != "none":
            raise ValueError(entangler)
    return gates


def encoding_gates(n: int) -> List[Gate]:
    """Per-qubit data encoding Ry(arcsin x) then Rz(arccos x^2), input column 0."""
    out: List[Gate] = []
    for q in range(n):
        out.append(Gate("ENC_RY_ASIN", target=q, param=0))
        out.append(Gate("ENC_RZ_ACOS_SQ", target=q, param=0))
    return out


def letters_from_terms(n: int, terms: Sequence[Sequence[tuple]]) -> np.ndarray:
    """Pauli rows from sparse terms [(qubit, 'X'|'Y'|'Z'), ...]."""
    rows = np.zeros((len(terms), n), dtype=np.int8)
    for t, term in enumerate(terms):
        for q, letter in term:
            rows[t, q] = PAULI_LETTERS.index(letter)
    return rows


def spin_hamiltonian_terms(n: int, pairs: Sequence[tuple]):
    """Term list of the Eq. 2 exciton Hamiltonian over the given monomer pairs.

    Order: Z_A for every A, X_A for every A, then per pair (A, B):
    XX, XZ, ZX, ZZ.  The constant term is omitted.
    """
    terms = [[(a, "Z")] for a in range(n)] + [[(a, "X")] for a in range(n)]
    for a, b in pairs:
        terms += [[(a, "X"), (b, "X")], [(a, "X"), (b, "Z")],
                  [(a, "Z"), (b, "X")], [(a, "Z"), (b, "Z")]]
    return terms


def spin_hamiltonian_coeffs(rng, n: int, n_pairs: int, sd_one=0.5, sd_two=0.05):
    a = rng.normal(0.0, sd_one, n)      # Z_A
    b = rng.normal(0.0, sd_one, n)      # X_A
    c = rng.normal(0.0, sd_two, n_pairs)  # X_A X_B
    d = rng.normal(0.0, sd_two, n_pairs)  # X_A Z_B
    e = rng.normal(0.0, sd_two, n_pairs)  # Z_A X_B
    f = rng.normal(0.0, sd_two, n_pairs)  # Z_A Z_B
    pair_part = np.stack([c, d, e, f], axis=1).reshape(-1)
    return np.concatenate([a, b, pair_part])


def all_pairs(n: int):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def nn_nnn_pairs(n: int):
    return [(a, a + 1) for a in range(n - 1)] + [(a, a + 2) for a in range(n - 2)]


# --------------------------------------------------------------------------
# the five workloads (and their reduced-size variants)
# --------------------------------------------------------------------------

def vqe_random_pauli(n: int = 4, layers: int = 2, n_terms: int = 10, seed: int = 0) -> Workload:
    """Plain VQE gradient: Ry-Rz layers + CNOT ladder, random Pauli-string H."""
    rng = np.random.default_rng(seed)
    letters = rng.integers(0, 4, size=(n_terms, n)).astype(np.int8)
    coeffs = rng.normal(0.0, 1.0, n_terms)
    gates = layered_ansatz(n, layers, ("RY", "RZ"), "ladder")
    P = layers * n * 2
    theta = rng.uniform(-np.pi, np.pi, P)
    return Workload(name=f"vqe{n}", n_qubits=n, gates=gates, n_params=P, theta=theta,
                    pauli_letters=letters, pauli_coeffs=coeffs,
                    refs=np.zeros(1, dtype=np.int64), weights=np.ones(1), cost="linear")


def mcvqe(n: int = 8, layers: int = 4, pairs: str = "all", n_refs: Optional[int] = None,
          seed: int = 0) -> Workload:
    """Multi-contracted VQE gradient (paper Sec. 4.1, Eq. 2) with basis references.

    References are |0...0> followed by single bit flips |e_0>, |e_1>, ...;
    the cost is the plain average of the reference energies.
    """
    rng = np.random.default_rng(seed)
    pair_list = all_pairs(n) if pairs == "all" else nn_nnn_pairs(n)
    terms = spin_hamiltonian_terms(n, pair_list)
    coeffs = spin_hamiltonian_coeffs(rng, n, len(pair_list))
    letters = letters_from_terms(n, terms)
    gates = layered_ansatz(n, layers, ("RY",), "ladder")
    P = layers * n
    theta = rng.uniform(-np.pi, np.pi, P)
    R = n + 1 if n_refs is None else n_refs
    refs = np.array([0] + [1 << i for i in range(R - 1)], dtype=np.int64)
    return Workload(name=f"mcvqe{n}", n_qubits=n, gates=gates, n_params=P, theta=theta,
                    pauli_letters=letters, pauli_coeffs=coeffs, refs=refs,
                    weights=np.full(R, 1.0 / R), cost="linear",
                    meta={"pairs": pairs, "layers": layers})


def cis_prep_gates(n: int) -> List[Gate]:
    """Preparation of a CIS-like state sum_i c_i |e_i> (a generalised W
    state, Sec. 4.1) from |e_0>: for i = 0..n-2 a controlled Ry(beta_i) from
    qubit i to qubit i+1, written as Ry(beta_i/2) CNOT Ry(-beta_i/2) CNOT on
    the target, then CNOT(i+1 -> i), which moves the excitation on.  The
    angles are per instance: Ry(arcsin x) gates read x = +-sin(beta_i/2) from
    input columns 2i and 2i+1, so beta_i is in [-pi, pi] and
    c_i = prod_{j<i} sin(beta_j/2) cos(beta_i/2), c_{n-1} = prod_j sin(beta_j/2)."""
    out: List[Gate] = []
    for i in range(n - 1):
        out.append(Gate("ENC_RY_ASIN", target=i + 1, param=2 * i))
        out.append(Gate("CNOT", target=i + 1, control=i))
        out.append(Gate("ENC_RY_ASIN", target=i + 1, param=2 * i + 1))
        out.append(Gate("CNOT", target=i + 1, control=i))
        out.append(Gate("CNOT", target=i, control=i + 1))
    return out


def cis_coefficients(beta: np.ndarray) -> np.ndarray:
    """The c_i that cis_prep_gates prepares from angles beta (closed form)."""
    n = len(beta) + 1
    c = np.zeros(n)
    run = 1.0
    for i in range(n - 1):
        c[i] = run * np.cos(beta[i] / 2)
        run *= np.sin(beta[i] / 2)
    c[n - 1] = run
    return c


def mcvqe_entanglers(n: int) -> List[Gate]:
    """Entanglers U_AB of Sec. 4.1 on adjacent monomers (A, A+1), in order:
    Ry Ry, CNOT(A -> B), Ry Ry, CNOT(A -> B), Ry Ry (6 Ry, 2 CNOT; the
    layout figure is lost, this is a reading).  The last Ry of qubit B in
    U_(A,B) and the first of B in U_(B,C) act back to back, so they merge
    (Ry(a)Ry(b) = Ry(a+b), Sec. 4.1) into one parameter: N_theta = 5N - 4
    (Table 1)."""
    out: List[Gate] = []
    p = 0
    last_on = {}
    for a in range(n - 1):
        b = a + 1
        # first pair of rotations: qubit a's merges into the previous
        # entangler's last rotation of a (already in place), so it is omitted
        if a not in last_on:
            out.append(Gate("RY", target=a, param=p)); p += 1
        out.append(Gate("RY", target=b, param=p)); p += 1
        out.append(Gate("CNOT", target=b, control=a))
        out.append(Gate("RY", target=a, param=p)); p += 1
        out.append(Gate("RY", target=b, param=p)); p += 1
        out.append(Gate("CNOT", target=b, control=a))
        out.append(Gate("RY", target=a, param=p)); p += 1
        last_on[b] = True
        out.append(Gate("RY", target=b, param=p)); p += 1
    return out


def mcvqe_paper(n: int = 16, n_refs: int = 4, seed: int = 0) -> Workload:
    """The paper's MC-VQE circuit (Sec. 4.1, Table 1): per reference a CIS
    state prepared from |e_0> (angles beta ~ U(-pi, pi) per reference, as
    inputs), then the shared entanglers over adjacent monomers; the Eq. 2
    Hamiltonian over nearest neighbours (N_H = 6N - 4); cost: the average of
    the reference energies.  The CIS coefficients of the paper come from
    quantum-chemistry runs and are not published: these stand in for them."""
    rng = np.random.default_rng(seed)
    pairs = [(a, a + 1) for a in range(n - 1)]
    terms = spin_hamiltonian_terms(n, pairs)
    coeffs = spin_hamiltonian_coeffs(rng, n, len(pairs))
    letters = letters_from_terms(n, terms)
    ent = mcvqe_entanglers(n)
    P = 1 + max(g.param for g in ent if g.param >= 0)
    theta = rng.uniform(-np.pi, np.pi, P)
    beta = rng.uniform(-np.pi, np.pi, (n_refs, n - 1))
    x = np.zeros((n_refs, 2 * (n - 1)))
    x[:, 0::2] = np.sin(beta / 2)
    x[:, 1::2] = -np.sin(beta / 2)
    return Workload(name=f"mcvqe_paper{n}", n_qubits=n, gates=cis_prep_gates(n) + ent, n_params=P,
                    theta=theta, pauli_letters=letters, pauli_coeffs=coeffs,
                    refs=np.full(n_refs, 1, dtype=np.int64), inputs=x,
                    weights=np.full(n_refs, 1.0 / n_refs), cost="linear",
                    meta={"beta": beta, "pairs": "nn"})


def qcl(n: int = 12, layers: int = 6, n_samples: int = 256, seed: int = 0,
        noise_sd: float = 0.05) -> Workload:
    """Quantum circuit learning regression (paper Sec. 4.2 use-case family).

    Encoding Ry(arcsin x) Rz(arccos x^2) on every qubit, then layers of
    Rx-Rz-Rx on every qubit + CNOT ring; model output <Z_0>; MSE loss on
    targets y = sin(pi x) + N(0, noise_sd).
    """
    rng = np.random.default_rng(seed)
    gates = encoding_gates(n) + layered_ansatz(n, layers, ("RX", "RZ", "RX"), "ring")
    P = layers * n * 3
    theta = rng.uniform(0.0, 2.0 * np.pi, P)
    x = rng.uniform(-1.0, 1.0, n_samples)
    y = np.sin(np.pi * x) + rng.normal(0.0, noise_sd, n_samples)
    letters = letters_from_terms(n, [[(0, "Z")]])
    return Workload(name=f"qcl{n}", n_qubits=n, gates=gates, n_params=P, theta=theta,
                    pauli_letters=letters, pauli_coeffs=np.ones(1),
                    refs=np.zeros(n_samples, dtype=np.int64), inputs=x.reshape(-1, 1),
                    targets=y, cost="mse", meta={"layers": layers})


def qcl_uneven(n_circuits: int = 8, n_samples: int = 16, n_range=(20, 24), depth_range=(4, 12),
               seed: int = 0) -> List[Workload]:
    """The uneven-batch variant of the 20-qubit circuit-learning configuration:
    circuits with n ~ U{n_range} qubits and depth ~ U{depth_range} layers
    (drawn in that order per circuit from default_rng(seed)), each a `qcl`
    workload with its own theta, inputs and targets (seed + 1 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_circuits):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        layers = int(rng.integers(depth_range[0], depth_range[1] + 1))
        out.append(qcl(n, layers, n_samples, seed=seed + 1 + i))
    return out


def bell_pairs(n: int) -> List[Gate]:
    """Neighbouring qubits (0,1), (2,3), ... entangled as Bell pairs: H then CNOT
    (Sec. 4.2: the DDCL circuit starts with each pair of neighbouring qubits
    entangled as a Bell pair; an odd last qubit stays |0>)."""
    out: List[Gate] = []
    for q in range(0, n - 1, 2):
        out.append(Gate("H", target=q))
        out.append(Gate("CNOT", target=q + 1, control=q))
    return out


def ddcl_target(n: int) -> np.ndarray:
    """Synthetic target distribution over the 2^n bitstrings b (read as
    integers): two discretised Gaussians at 2^n/4 and 3*2^n/4 with width
    2^n/16, normalised; it stands in for the paper's unpublished target."""
    b = np.arange(1 << n, dtype=np.float64)
    N = float(1 << n)
    sig = N / 16.0
    p = np.exp(-0.5 * ((b - N / 4) / sig) ** 2) + np.exp(-0.5 * ((b - 3 * N / 4) / sig) ** 2)
    return p / p.sum()


def ddcl(n: int = 20, layers: int = 10, seed: int = 0, target: Optional[np.ndarray] = None) -> Workload:
    """Data-driven circuit learning (Sec. 4.2, Eq. 3, Table 2): Bell pairs, then
    `layers` layers of Rz-Ry-Rz on every qubit, CNOT ladder, Rz-Ry-Rz on every
    qubit (6 parameters per qubit per layer, N_theta = 60 N_q at 10 layers;
    the paper's layer figure is lost, this layout is a reading); cost: the JS
    divergence of the output distribution from `target` (default ddcl_target)."""
    rng = np.random.default_rng(seed)
    gates = bell_pairs(n)
    p = 0
    for _ in range(layers):
        for half in range(2):
            for q in range(n):
                for op in ("RZ", "RY", "RZ"):
                    gates.append(Gate(op, target=q, param=p))
                    p += 1
            if half == 0:
                gates.extend(cnot_ladder(n))
    theta = rng.uniform(-np.pi, np.pi, p)
    letters = letters_from_terms(n, [[(0, "Z")]])
    return Workload(name=f"ddcl{n}", n_qubits=n, gates=gates, n_params=p, theta=theta,
                    pauli_letters=letters, pauli_coeffs=np.ones(1), refs=np.zeros(1, dtype=np.int64),
                    cost="js", meta={"layers": layers},
                    target_dist=ddcl_target(n) if target is None else np.asarray(target, np.float64))


def config(idx: int) -> Workload:
    """The five workload configurations at full size (0-based index)."""
    if idx == 0:
        return vqe_random_pauli(4, 2, 10)
    if idx == 1:
        return mcvqe(8, 4, "all")
    if idx == 2:
        return qcl(12, 6, 256)
    if idx == 3:
        return qcl(20, 10, 64)
    if idx == 4:
        return mcvqe(28, 8, "nn+nnn", n_refs=8)
    raise IndexError(idx)


def random_circuit(n: int, n_gates: int, seed: int = 0, n_params: Optional[int] = None,
                   ops: Sequence[str] = ("RX", "RY", "RZ", "CNOT", "X", "H", "CZ")):
    """Random gate list over the given ops; every parametric gate gets its own param."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    p = 0
    for _ in range(n_gates):
        op = ops[rng.integers(0, len(ops))]
        if op in ("CNOT", "CZ"):
            if n < 2:
                continue
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(Gate(op, target=int(b), control=int(a)))
        elif op in ("RX", "RY", "RZ"):
            gates.append(Gate(op, target=int(rng.integers(0, n)), param=p))
            p += 1
        else:
            gates.append(Gate(op, target=int(rng.integers(0, n))))
    P = p if n_params is None else n_params
    theta = rng.uniform(-np.pi, np.pi, P)
    return gates, P, theta


def random_pauli_sum(n: int, n_terms: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    letters = rng.integers(0, 4, size=(n_terms, n)).astype(np.int8)
    coeffs = rng.normal(0.0, 1.0, n_terms)
    return letters, coeffs


def random_workload(n: int, n_gates: int, n_terms: int, n_instances: int = 2, seed: int = 0,
                    cost: str = "linear", with_encoding: bool = False) -> Workload:
    """Random circuit + random Pauli sum, for parity tests of arbitrary gate mixes."""
    gates, P, theta = random_circuit(n, n_gates, seed)
    letters, coeffs = random_pauli_sum(n, n_terms, seed + 1)
    rng = np.random.default_rng(seed + 2)
    refs = rng.integers(0, 1 << n, size=n_instances).astype(np.int64)
    inputs = targets = weights = None
    if with_encoding:
        gates = encoding_gates(n) + gates
        inputs = rng.uniform(-1.0, 1.0, (n_instances, 1))
    if cost == "mse":
        targets = rng.normal(0.0, 0.5, n_instances)
    else:
        weights = rng.uniform(0.2, 1.0, n_instances)
    return Workload(name=f"random{n}", n_qubits=n, gates=gates, n_params=P, theta=theta,
                    pauli_letters=letters, pauli_coeffs=coeffs, refs=refs, inputs=inputs,
                    targets=targets, weights=weights, cost=cost)
