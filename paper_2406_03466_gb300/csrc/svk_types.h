// Plain-old-data structures shared by the host planner and the CUDA kernels.
//
// A circuit is compiled into a *program* for the on-chip engine:
//  * consecutive single-qubit gates on one qubit are fused into a *group*
//    whose 2x2 matrix is built per circuit slot (shifted parameters and
//    per-instance encoding inputs differ between slots);
//  * the op stream is cut into *stages*.  In a stage every thread holds
//    2^R amplitudes in registers; the R qubits in registers are the stage's
//    register bits, the other index bits come from the thread index.  A
//    stage applies its fused 2x2 groups in registers, then writes the
//    amplitudes back to shared memory through the stage's GF(2)-linear
//    index permutation (the CNOTs deferred to the end of the stage);
//  * shared-memory addresses are XOR-swizzled so that the lanes of a warp
//    hit distinct banks; the swizzle is GF(2)-linear, so every address is
//    an XOR of per-bit address vectors, precomputed here for each stage.
#pragma once
#include <cstdint>

namespace svk {

constexpr int kRMax = 5;    // largest register-bit count
constexpr int kNMax = 30;   // largest qubit count
constexpr int kMaxGroupOpsPerStage = 8;

// Members of a fused single-qubit group.
enum MemberKind : int32_t {
    M_RX = 0, M_RY = 1, M_RZ = 2, M_X = 3, M_H = 4, M_ENC_RY_ASIN = 5, M_ENC_RZ_ACOS_SQ = 6
};

struct Member {
    int32_t kind;
    int32_t param;   // theta index (rotations), input column (encodings), -1 otherwise
    double angle;    // fixed angle of a rotation with param < 0
};

struct Group {
    int32_t m_begin, m_end;  // members [m_begin, m_end) in time order
    int32_t qubit;
    int32_t has_param;       // 1 if some member reads theta (needs a gradient)
    int32_t real;            // 1 if the fused matrix is real (Ry, X, H, Ry encodings only)
};

enum OpKind : int32_t { OP_U1 = 0, OP_CZ = 1 };

struct Op {
    int32_t kind;
    int32_t a;      // OP_U1: register index; OP_CZ: first qubit position
    int32_t b;      // OP_CZ: second qubit position
    int32_t group;  // OP_U1: group index
};

struct Stage {
    int32_t op_begin, op_end;
    int32_t n_thr;              // thread bits = n - R
    int32_t n_u1;               // OP_U1 ops in this stage (<= kMaxGroupOpsPerStage)
    int32_t q[kRMax];           // register bit i -> qubit
    int32_t tpos[kNMax];        // thread bit k -> qubit
    uint32_t ldq[kRMax];        // swizzled address vector of register bit i, load layout
    uint32_t stq[kRMax];        // swizzled address vector of register bit i, store layout
    uint32_t ldt[kNMax];        // same for thread bit k
    uint32_t stt[kNMax];
    // sorted = 1: the stage's ops are all fused groups, ordered by register
    // bit (ops on different bits commute), and bit i owns the ops
    // [op_begin + bit_begin[i], op_begin + bit_begin[i + 1]); sorted = 2:
    // moreover every register bit owns exactly one group, and all are real.
    int32_t sorted;
    int32_t bit_begin[kRMax + 1];
};

// One tile pass over states in device memory: a tile is the 2^t amplitudes
// whose non-local index bits are fixed.  Local bit b of a tile index sits at
// global address bit vector gl[b]; tile-number bit k at gt[k].
struct PassDesc {
    int32_t stage_begin, stage_end;  // the pass's stages (tile-local positions)
    int32_t t;                       // local qubits
    int32_t n_tile_bits;             // n - t
    int32_t n_u1;                    // fused-group ops in the pass
    uint32_t local_mask;             // qubits local to the pass
    uint32_t gl[kNMax];
    uint32_t gt[kNMax];
    // Shared-memory address vector of tile-local bit b when the tile is
    // loaded (forward) or stored back (reverse): swizzle(f(e_b)) for the
    // pass's leading CNOT permutation f (identity if it has none).
    uint32_t ldperm[kNMax];
};

// Device descriptor of one tile pass, passed to the pass kernels as a
// __grid_constant__ parameter.  Shared-memory addresses are byte offsets
// within one tile buffer (swizzled, times the amplitude size); global
// offsets are amplitude indices within one state.
constexpr int kTileBitsMax = 13;  // largest tile: 2^13 amplitudes
constexpr int kPassStages = 16;   // register stages per pass
constexpr int kPassOps = 48;      // fused-group ops per pass (< 63: kernels pack u + 1 in 6 bits)

struct TileStage {
    uint32_t ldq[kRMax], stq[kRMax];                // register bit i: load / store vector
    uint32_t ldt[kTileBitsMax], stt[kTileBitsMax];  // thread bit k: load / store vector
    int32_t op[kRMax];                              // pass-local op on register bit i, or -1
};

struct TilePass {
    int32_t t, R, n_stages, n_ops, n_tile_bits;
    int32_t all_single;             // every parametrised op has fmode > 0
    uint64_t real_mask;             // bit u: op u has a real matrix
    uint64_t param_mask;            // bit u: op u's group has parameters
    uint32_t gl[kTileBitsMax];      // tile-local bit b -> global offset bit
    uint32_t gpre[kNMax];           // gt[0] ^ ... ^ gt[k] for tile-number bit k
    uint32_t ldperm[kTileBitsMax];  // tile-local bit b -> shared address at load (forward)
    uint32_t nat[kTileBitsMax];     // tile-local bit b -> natural shared address
    int32_t grp[kPassOps];          // pass-local op u -> fused group
    TileStage st[kPassStages];
    // The derivative of op u's group needs one sum of the reduced matrix
    // when its only rotation is the group's last member: fmode 1 = RY (k3),
    // 2 = RX (k2), 3 = RZ (k0 - k1); 0 = all four.
    int8_t fmode[kPassOps];
};

// Pauli terms grouped by X-mask: <psi|P|psi> = Re(i^phase sum_j (-1)^{|j & z|}
// conj(psi_{j^x}) psi_j) with phase = (#Y) mod 4.
struct TermGroup {
    uint32_t x;
    uint32_t sx;        // swizzled x (address vector of the partner offset)
    int32_t t_begin, t_end;
};

struct Term {
    uint32_t z;
    int32_t phase;
    double coeff;
};

// Device view of a compiled circuit (all pointers are device memory).
// Per-thread address bases of one stage: x = load base (swizzled), y = store
// base (swizzled, after the stage's permutation), z = logical index base.
struct ThreadBase {
    uint32_t lb, sb, lg, pad;
};

struct Program {
    int32_t n, R, n_stages, n_groups, n_params, input_dim, swz_bits;
    int32_t pad;
    const Stage *stages;
    const Op *ops;
    const Group *groups;
    const Member *members;
    const ThreadBase *tbase;  // [n_stages][2^(n-R)] (NULL: computed in the kernel)
};

struct Observable {
    int32_t n_tgroups, n_terms;
    int32_t real, pad;  // real: every c_t i^phase_t is real (no Y-parity imaginary parts)
    const TermGroup *tgroups;
    const Term *terms;
};

// One pass of one problem in a persistent multi-problem sweep: its tiles
// are cut into chunks of chunk_tiles, which take the tickets
// [chunk_begin, chunk_begin + n_chunks) of the sweep; a chunk may run once
// task `dep` (the problem's previous pass, or -1) has completed every chunk.
struct SweepTask {
    const TilePass *P;  // device descriptor
    int32_t n, n_slots, G, dep;
    int64_t tiles, chunk_begin, n_chunks;
    int32_t chunk_tiles, pad;
    const void *mats;   // [slots][G][4]
    void *psi, *lam;    // the problem's states
    double *rho;        // reverse: [slots][G][8]
};

// lambda = H psi (and <H>) over tiles of 2^t amplitudes.  A pass covers the
// X-mask groups whose flip mask lies inside its local qubits; inside a
// group, terms with the same Z mask on the local qubits form a class whose
// coefficient is summed once per tile (the Z mask's tile-number bits only
// give each term a sign per tile).
// The H kernel's threads hold 2^R amplitudes j = tid + k 2^(t - R) (k over
// the R register bits, the top R tile-local bits).  A class's Z mask splits
// into its thread bits zt = zl & (2^(t-R) - 1) and its register bits
// kz = zl >> (t - R), so the group's diagonal factor at thread tid and
// register index k is D(tid, k) = sum over its rows of (-1)^|tid & zt| E[k],
// one row per distinct zt, E[k] = sum of the row's class coefficients times
// (-1)^|k & kz| (per tile, shared by all threads).  Groups whose classes put
// no Z on a register bit (kact = 0) take one value per thread instead.
constexpr int kHRegBitsMax = 4;
struct HGroup {
    uint32_t xl;              // flip mask on tile-local bits
    int32_t c_begin, c_end;   // its classes, sorted by (zt, kz)
    uint32_t xfar;            // whole flip mask when it leaves the tile (partner read from
                              // global memory), else 0
    uint32_t kact;            // register bits in some class's Z mask (0: one value per thread)
    int32_t r_begin, r_end;   // its rows (kact != 0), else empty
    uint32_t pad;
};

// A run of a group's classes with the same Z mask on the thread bits.
struct HRow {
    uint32_t zt;              // Z mask on the thread bits
    int32_t c_begin, c_end;   // its classes (pass-relative)
    int32_t pad;
};

struct HClass {
    uint32_t zl;              // Z mask on tile-local bits
    int32_t t_begin, t_end;   // its terms
    uint32_t xnl;             // the group's flip bits outside the tile (sign of the partner)
    uint32_t xl;              // the group's flip bits on tile-local bits
    int32_t pad;
};

struct HTerm {
    uint32_t z;               // Z mask (global index bits)
    int32_t phase;            // i^phase, phase = #Y mod 4
    double coeff;
};

struct HPass {
    int32_t t, n_tile_bits, n_groups, n_classes, n_terms, first;  // first: writes lambda
    int32_t real;               // every coefficient c_t i^phase_t is real
    int32_t R;                  // register bits of the kernel's threads (h_reg_bits(t))
    uint32_t gl[kTileBitsMax];  // tile-local bit b -> global offset bit
    uint32_t gpre[kNMax];       // gt[0] ^ ... ^ gt[k] for tile-number bit k
    int32_t n_rows, pad;
    const HGroup *groups;       // device arrays of this pass
    const HClass *classes;
    const HTerm *terms;
    const HRow *rows;
};

// Register bits of the H-pass kernel for tiles of 2^t amplitudes: 256
// threads for t >= 12 (R = 4), fewer below (at least 32 threads).
inline int h_reg_bits(int t) { return t >= 12 ? 4 : (t == 11 ? 3 : 2); }

// GF(2)-linear swizzle of a shared-memory amplitude index: the low `w` bits
// are XORed with the fold of all higher w-bit chunks.  w = 4 for 8-byte
// amplitudes (16 per 128-byte wavefront), 3 for 16-byte amplitudes.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t swizzle(uint32_t a, int w) {
    uint32_t f = 0;
    for (uint32_t h = a >> w; h; h >>= w) f ^= h;
    return a ^ (f & ((1u << w) - 1u));
}

}  // namespace svk
