"""Circuit counting of the paper's workloads (TEST INFRASTRUCTURE ONLY).

Parameter-shift circuit counts, as used to size a gradient batch:

* multi-contracted VQE (Sec. 4.1, Table 1): one circuit per Hamiltonian term
  and per shifted parameter, 2 N_H N_theta per update.  N_H counts the
  Eq. 2 terms of a nearest-neighbour monomer chain without the constant:
  X_A and Z_A per monomer plus XX, XZ, ZX, ZZ per adjacent pair.  N_theta
  counts 6 Ry per entangler over the N_q - 1 adjacent pairs, minus one merged
  Ry pair (Ry(a)Ry(b) = Ry(a+b)) on every qubit shared by two consecutive
  entanglers; the entangler layout itself is only in a figure, so this
  merge count is a reading of the text.
* data-driven circuit learning (Sec. 4.2, Table 2): a single Pauli string, so
  2 N_theta circuits, with N_theta = 6 per qubit per layer.
* the batched form used here runs every reference (or training sample) with
  the full <H> per circuit: (2 P + 1) circuits per instance.
"""
from __future__ import annotations

from workloads import spin_hamiltonian_terms


def mcvqe_paper_counts(n_qubits: int):
    pairs = [(a, a + 1) for a in range(n_qubits - 1)]
    n_h = len(spin_hamiltonian_terms(n_qubits, pairs))
    n_entanglers = n_qubits - 1
    n_theta = 6 * n_entanglers - (n_entanglers - 1)
    return n_h, n_theta, 2 * n_h * n_theta


def ddcl_paper_counts(n_qubits: int, layers: int = 10, per_qubit_per_layer: int = 6):
    n_theta = per_qubit_per_layer * layers * n_qubits
    return n_theta, 2 * n_theta


def batched_param_shift_slots(n_params: int, n_instances: int) -> int:
    return (2 * n_params + 1) * n_instances
