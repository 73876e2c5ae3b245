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
    std::vector<PassDesc> passes;                  // tile passes (device-memory states)
    // Per tile pass: shared-memory address vector (swizzled, in amplitudes)
    // of the tile-local bit stored at global tile bit b; differs from
    // swizzle(e_b) where the pass relabels qubits on its way out.
    std::vector<std::vector<uint32_t>> stperm;
    // Layout after the last tile pass: qubit q lives in bit layout[q] of the
    // amplitude index (the identity unless the passes relabel).
    std::vector<int> layout;
    std::vector<ThreadBase> tbase;                 // [stages][2^(t-R)] thread bases
};

// Fills P->tbase for stages whose thread count is 2^(t - R).
void build_thread_bases(HostProgram *P, int t);

// Logical op stream after single-qubit fusion.
struct LOp {
    int kind;  // 0 = fused group on qubit a, 1 = CNOT a -> b, 2 = CZ(a, b)
    int a, b, group;
};

struct FusedCircuit {
    std::vector<LOp> lops;
    std::vector<Group> groups;
    std::vector<Member> members;
};

std::string fuse_circuit(const sv_circuit &c, bool fuse, FusedCircuit *out);
// Appends the register stages of `lops` (qubit q at tile position pos[q] < t).
// one_per_bit: close a stage rather than put a second op on a register bit.
void stage_lops(const std::vector<LOp> &lops, const std::vector<int> &pos, int t, int R, int w,
                HostProgram *P, bool one_per_bit);
// Cuts a circuit into tile passes of 2^tile_bits amplitudes whose local
// qubits always include the qubits in the lowest coalesce_bits bits of the
// amplitude index (so that tiles move in contiguous runs).  relabel: a pass
// may store its tile with its qubits in other bits of the same tile, moving
// into the low bits qubits that the next pass needs (P->layout gives the
// final bit of every qubit); otherwise every qubit keeps its own bit.
std::string plan_passes(const sv_circuit &c, int tile_bits, int coalesce_bits, int reg_bits,
                        bool fuse, int swz_bits, HostProgram *P, bool relabel = false);

// Kernel descriptors of every pass of a tile plan (amplitudes of csz bytes).
std::string build_tile_passes(const HostProgram &P, int csz, std::vector<TilePass> *out);

struct HostObservable {
    int n = 0;
    std::vector<TermGroup> tgroups;
    std::vector<Term> terms;
};

// Tile passes of lambda = H psi: pass i uses groups[g_begin[i]..g_begin[i+1])
// etc.  Device pointers of HPass are left null (set after upload).
struct HostHPlan {
    std::vector<HPass> passes;
    std::vector<int> g_begin, c_begin, t_begin, r_begin;  // per pass, plus an end entry
    std::vector<HGroup> groups;
    std::vector<HClass> classes;
    std::vector<HTerm> terms;
    std::vector<HRow> rows;
};
std::string plan_h_passes(const HostObservable &h, int tile_bits, int coalesce_bits,
                          HostHPlan *out);

// Returns "" on success, otherwise the reason the circuit was rejected.
std::string plan_circuit(const sv_circuit &c, int reg_bits, bool fuse, int swz_bits,
                         HostProgram *out);
std::string plan_observable(const sv_pauli_sum &h, int n, int swz_bits, HostObservable *out);

// Structural hash of a circuit (gates, sizes) for plan caching.
uint64_t hash_circuit(const sv_circuit &c);
uint64_t hash_observable(const sv_pauli_sum &h);

}  // namespace svk
