// Host planner: compiles a circuit (gate list) into the stage program run by
// the on-chip kernels, and a Pauli sum into X-mask term groups.
#pragma once
#include <string>
#include <vector>

#include "sv.h"
#include "svk_types.h"

namespace svk {

struct HostProgram {
    int n = 0, R = 0, n_params = 0, input_dim = 0, swz_bits = 4;
    std::vector<Member> members;
    std::vector<Group> groups;
    std::vector<Op> ops;
    std::vector<Stage> stages;
    std::vector<std::vector<uint32_t>> perm_cols;  // per stage: f(e_b), b < n
};

struct HostObservable {
    int n = 0;
    std::vector<TermGroup> tgroups;
    std::vector<Term> terms;
};

// Returns "" on success, otherwise the reason the circuit was rejected.
std::string plan_circuit(const sv_circuit &c, int reg_bits, bool fuse, int swz_bits,
                         HostProgram *out);
std::string plan_observable(const sv_pauli_sum &h, int n, int swz_bits, HostObservable *out);

// Structural hash of a circuit (gates, sizes) for plan caching.
uint64_t hash_circuit(const sv_circuit &c);
uint64_t hash_observable(const sv_pauli_sum &h);

}  // namespace svk
