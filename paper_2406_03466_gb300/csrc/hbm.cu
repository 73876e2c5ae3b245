// Tile passes over states in device memory (states too large for one
// block's shared memory: 14..30 qubits).
//
// A circuit is cut into passes (planner: plan_passes).  In a pass every block
// loads tiles of 2^t amplitudes whose non-local index bits are fixed, runs
// the pass's register stages on the tile in shared memory (the same stage
// engine as the on-chip kernels, with tile-local qubit positions), and
// stores the tile back in place.  The lowest qubits are always local, so
// every load and store moves whole 128-byte segments.  Blocks are persistent:
// each walks (slot, tile) pairs with a grid stride.
//
// Kernels: per-slot fused group matrices, |ref> initialisation, forward
// pass, reverse (adjoint) pass with per-group reduced matrices accumulated
// per block and added to global FP64 sums, <H> and lambda = H psi over whole
// states, and the per-slot gradient assembly.
#include <cuda_runtime.h>

#include "engine.cuh"
#include "hbm.h"

namespace svk {
namespace {

// Fused 2x2 matrices of every group for every slot: out[slot][group][4].
template <typename Real>
__global__ void k_group_mats(Program p, SlotSource src, typename CT<Real>::T *out) {
    const int G = p.n_groups;
    const int64_t total = (int64_t)src.n_slots * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / G), g = (int)(i % G);
        const SlotInfo si = resolve(src, b);
        group_matrix<Real, typename CT<Real>::T>(p, g, si, out + (size_t)i * 4);
    }
}

// Sets amplitude |ref_b> of every (zeroed) slot state to 1.
template <typename C>
__global__ void k_set_ref(C *states, int n, SlotSource src) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < src.n_slots; b += gridDim.x * blockDim.x) {
        const SlotInfo si = resolve(src, b);
        C one;
        one.x = 1;
        one.y = 0;
        states[((int64_t)b << n) + si.ref] = one;
    }
}

// Shared-memory addresses of this thread's tile amplitudes through the
// pass's load permutation: returns the tid part, fills the k part.
template <int R>
__device__ __forceinline__ uint32_t perm_vectors(const PassDesc &pd, int tid, uint32_t (&pk)[R]) {
    const int tb = pd.t - R;
    uint32_t g = 0;
    for (int b = 0; b < tb; ++b)
        if ((tid >> b) & 1) g ^= pd.ldperm[b];
#pragma unroll
    for (int j = 0; j < R; ++j) pk[j] = pd.ldperm[tb + j];
    return g;
}

// Global offsets (within one state) of this thread's 2^R tile amplitudes:
// local index i = tid + k * 2^(t-R); returns the tid part, fills the k part.
template <int R>
__device__ __forceinline__ uint32_t tile_vectors(const PassDesc &pd, int tid, uint32_t (&gk)[R]) {
    const int tb = pd.t - R;
    uint32_t g = 0;
    for (int b = 0; b < tb; ++b)
        if ((tid >> b) & 1) g ^= pd.gl[b];
#pragma unroll
    for (int j = 0; j < R; ++j) gk[j] = pd.gl[tb + j];
    return g;
}

__device__ __forceinline__ uint32_t tile_base(const PassDesc &pd, uint32_t tile) {
    uint32_t g = 0;
    for (int k = 0; k < pd.n_tile_bits; ++k)
        if ((tile >> k) & 1) g ^= pd.gt[k];
    return g;
}

// One forward pass over every tile of every slot.  `pv` is the pass's view
// of the program (n = t, its own stages); `mats` holds [slots][G][4].
// Asynchronous global -> shared copies (bypass registers) so that the next
// tile is in flight while the current one is computed.
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The pass's program in shared memory: stage records, its op range, the
// thread bases of its stages and every group record.  `pv` must carry thread
// bases (tile plans always do).  Byte offsets follow `base`.
struct PassSmem {
    uint32_t stages, ops, tbase, groups, end;
};

__host__ __device__ inline PassSmem pass_smem_layout(uint32_t base, int n_st, int n_ops, int T,
                                                     int G) {
    PassSmem L{};
    auto up = [](uint32_t x) { return (x + 15u) & ~15u; };
    L.stages = up(base);
    L.ops = up(L.stages + (uint32_t)n_st * (uint32_t)sizeof(Stage));
    L.tbase = up(L.ops + (uint32_t)n_ops * (uint32_t)sizeof(Op));
    L.groups = up(L.tbase + (uint32_t)n_st * T * (uint32_t)sizeof(ThreadBase));
    L.end = up(L.groups + (uint32_t)G * (uint32_t)sizeof(Group));
    return L;
}

template <typename T>
__device__ __forceinline__ void copy_words(T *dst, const T *src, int count) {
    const int words = (int)(count * sizeof(T) / 4);
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
}

// Copies the pass program into shared memory and returns a view whose
// pointers all derive from the shared array (so reads compile to shared loads).
__device__ __forceinline__ Program stage_pass_program(const Program &pv, int op0, int n_ops, int G,
                                                      unsigned char *smem, const PassSmem &L) {
    const int T = 1 << (pv.n - pv.R);
    Stage *st = reinterpret_cast<Stage *>(smem + L.stages);
    Op *ops = reinterpret_cast<Op *>(smem + L.ops);
    ThreadBase *tb = reinterpret_cast<ThreadBase *>(smem + L.tbase);
    Group *gr = reinterpret_cast<Group *>(smem + L.groups);
    copy_words(st, pv.stages, pv.n_stages);
    copy_words(ops, pv.ops + op0, n_ops);
    copy_words(tb, pv.tbase, pv.n_stages * T);
    copy_words(gr, pv.groups, G);
    __syncthreads();
    Program ps = pv;
    ps.stages = st;
    ps.ops = ops - op0;
    ps.tbase = tb;
    ps.groups = gr;
    return ps;
}

// Copies slot b's fused group matrices ([G][4] complex) into shared memory.
template <typename C>
__device__ __forceinline__ void load_mats(C *dst, const C *mats, int b, int G) {
    __syncthreads();
    const C *src = mats + (size_t)b * G * 4;
    for (int i = threadIdx.x; i < 4 * G; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

template <typename Real, int R>
__global__ void __launch_bounds__(256, 3) k_pass_fwd(PassDesc pd, Program pv, int op0, int n_ops,
                                                     int n, int n_slots,
                                                     const typename CT<Real>::T *mats, int G,
                                                     typename CT<Real>::T *states) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t tbytes = (size_t)sizeof(C) << pd.t;
    C *buf[2] = {reinterpret_cast<C *>(smem), reinterpret_cast<C *>(smem + tbytes)};
    C *smats = reinterpret_cast<C *>(smem + 2 * tbytes);
    const PassSmem PL = pass_smem_layout((uint32_t)(2 * tbytes + (size_t)G * 4 * sizeof(C)),
                                         pv.n_stages, n_ops, 1 << (pd.t - R), G);
    const Program ps = stage_pass_program(pv, op0, n_ops, G, smem, PL);
    const int tid = threadIdx.x, t = pd.t, w = pv.swz_bits;
    uint32_t gk[R], sv[R], pk[R];
    const uint32_t g0 = tile_vectors<R>(pd, tid, gk);
    const uint32_t s0 = natural_vectors<R>(tid, t - R, w, sv);
    const uint32_t p0 = perm_vectors<R>(pd, tid, pk);
    // contiguous tile ranges per block: the slot (and its matrices) rarely changes
    const int64_t tiles = (int64_t)n_slots << pd.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = per * blockIdx.x, t_end = min(tiles, t0 + per);
    const int64_t tmask = (int64_t(1) << pd.n_tile_bits) - 1;
    auto fetch = [&](int64_t tix, C *dst) {
        const C *S = states + ((tix >> pd.n_tile_bits) << n);
        const uint32_t tb = tile_base(pd, (uint32_t)(tix & tmask));
#pragma unroll
        for (int k = 0; k < NA; ++k)
            cp_async(dst + (p0 ^ xsel<R>(k, pk)), S + (tb ^ g0 ^ xsel<R>(k, gk)), (int)sizeof(C));
        cp_async_commit();
    };
    if (t0 < t_end) fetch(t0, buf[0]);
    int cur = -1;
    for (int64_t tix = t0, i = 0; tix < t_end; ++tix, ++i) {
        const int b = (int)(tix >> pd.n_tile_bits);
        if (b != cur) {
            load_mats(smats, mats, b, G);
            cur = b;
        }
        C *tile = buf[i & 1];
        cp_async_wait_all();
        __syncthreads();
        if (tix + 1 < t_end) fetch(tix + 1, buf[(i + 1) & 1]);
        forward_stages<Real, R, 2>(ps, tile, smats, tid, -1);
        C *S = states + ((int64_t)b << n);
        const uint32_t tb = tile_base(pd, (uint32_t)(tix & tmask));
#pragma unroll
        for (int k = 0; k < NA; ++k) S[tb ^ g0 ^ xsel<R>(k, gk)] = tile[s0 ^ xsel<R>(k, sv)];
    }
}

// Shared-memory layout of the reverse pass: psi tile, lambda tile, per-warp
// rho partials (two buffers), per-block FP64 rho sums by group, group ids of
// the pass's fused ops.
struct RevLayout {
    uint32_t tile, rhow, rho, u2g, total;
};

__host__ __device__ inline RevLayout rev_layout(int t, int R, int csz, int rsz, int G, int n_u1) {
    RevLayout L{};
    const uint32_t tile = (uint32_t)(csz << t);
    const int T = 1 << (t - R), wps = T >= 32 ? T / 32 : 1;
    L.tile = tile;
    L.rhow = 2 * tile;
    L.rho = L.rhow + (uint32_t)((2 * kMaxGroupOpsPerStage * wps * 8 * rsz + 15) & ~15);
    L.u2g = L.rho + (uint32_t)(G * 64);
    L.total = L.u2g + (uint32_t)((n_u1 * 4 + 15) & ~15);
    return L;
}

// Adds the block's rho sums of slot b for the pass's groups to rho_g and clears them.
__device__ void flush_rho(const Program &pv, const int *u2g, int n_u1, double *rho_blk,
                          double *rho_g, int b, int G) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < n_u1 * 8; idx += blockDim.x) {
        const int gi = u2g[idx >> 3], v = idx & 7;
        if (!pv.groups[gi].has_param) continue;
        const double x = rho_blk[gi * 8 + v];
        if (x != 0.0) atomicAdd(&rho_g[((size_t)b * G + gi) * 8 + v], x);
        rho_blk[gi * 8 + v] = 0.0;
    }
    __syncthreads();
}

// One reverse pass: un-applies the pass on psi and lambda tiles and sums the
// reduced matrices of its groups (FP64) into rho_g[slot][group][8].
template <typename Real, int R>
__global__ void __launch_bounds__(256, 2) k_pass_rev(PassDesc pd, Program pv_g, int op0, int n_ops,
                                                  int n, int n_slots,
                                                  const typename CT<Real>::T *mats, int G,
                                                  typename CT<Real>::T *psi,
                                                  typename CT<Real>::T *lam, double *rho_g) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, t = pd.t, w = pv_g.swz_bits, T = blockDim.x;
    const RevLayout L = rev_layout(t, R, (int)sizeof(C), (int)sizeof(Real), G, pd.n_u1);
    C *smats = reinterpret_cast<C *>(smem + L.total);
    const PassSmem PL = pass_smem_layout(L.total + (uint32_t)(G * 4 * sizeof(C)), pv_g.n_stages,
                                         n_ops, 1 << (pd.t - R), G);
    const Program pv = stage_pass_program(pv_g, op0, n_ops, G, smem, PL);
    C *tp = reinterpret_cast<C *>(smem);
    C *tl = reinterpret_cast<C *>(smem + L.tile);
    Real *rhow = reinterpret_cast<Real *>(smem + L.rhow);
    double *rho_blk = reinterpret_cast<double *>(smem + L.rho);
    int *u2g = reinterpret_cast<int *>(smem + L.u2g);
    for (int i = tid; i < G * 8; i += T) rho_blk[i] = 0.0;
    if (tid == 0) {
        int u = 0;
        for (int s = 0; s < pv.n_stages; ++s)
            for (int oi = pv.stages[s].op_begin; oi < pv.stages[s].op_end; ++oi)
                if (pv.ops[oi].kind == OP_U1 && u < pd.n_u1) u2g[u++] = pv.ops[oi].group;
    }
    __syncthreads();
    uint32_t gk[R], sv[R], pk[R];
    const uint32_t g0 = tile_vectors<R>(pd, tid, gk);
    const uint32_t s0 = natural_vectors<R>(tid, t - R, w, sv);
    const uint32_t p0 = perm_vectors<R>(pd, tid, pk);
    // Each block walks one contiguous range of tiles (few slot changes, so
    // few flushes of its rho sums).
    const int64_t tiles = (int64_t)n_slots << pd.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t_end = min(tiles, per * (blockIdx.x + 1));
    int cur = -1;
    for (int64_t tix = per * blockIdx.x; tix < t_end; ++tix) {
        const int b = (int)(tix >> pd.n_tile_bits);
        if (b != cur) {
            if (cur >= 0) flush_rho(pv, u2g, pd.n_u1, rho_blk, rho_g, cur, G);
            load_mats(smats, mats, b, G);
            cur = b;
        }
        const uint32_t tb = tile_base(pd, (uint32_t)(tix & ((int64_t(1) << pd.n_tile_bits) - 1)));
        C *P = psi + ((int64_t)b << n), *Lm = lam + ((int64_t)b << n);
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t ga = tb ^ g0 ^ xsel<R>(k, gk), sa = s0 ^ xsel<R>(k, sv);
            tp[sa] = P[ga];
            tl[sa] = Lm[ga];
        }
        __syncthreads();
        reverse_stages<Real, R, 2>(pv, tp, tl, smats, tid, T, rhow, rho_blk);
#pragma unroll
        for (int k = 0; k < NA; ++k) {  // back through the pass's load permutation
            const uint32_t ga = tb ^ g0 ^ xsel<R>(k, gk), sa = p0 ^ xsel<R>(k, pk);
            P[ga] = tp[sa];
            Lm[ga] = tl[sa];
        }
        __syncthreads();
    }
    if (cur >= 0) flush_rho(pv, u2g, pd.n_u1, rho_blk, rho_g, cur, G);
}

// D_g(j) = sum_{t in g} c_t i^{phase_t} (-1)^{|j & z_t|} for one amplitude.
template <typename Real>
__device__ __forceinline__ void diag_of(const Observable &o, const TermGroup &tg, uint32_t j,
                                        Real &dre, Real &dim) {
    dre = 0;
    dim = 0;
    for (int t = tg.t_begin; t < tg.t_end; ++t) {
        const Term tm = o.terms[t];
        const Real c = (__popc(j & tm.z) & 1u) ? (Real)-tm.coeff : (Real)tm.coeff;
        if (tm.phase == 0) dre += c;
        else if (tm.phase == 1) dim += c;
        else if (tm.phase == 2) dre -= c;
        else dim -= c;
    }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// out[b] += sum_j sum_g Re(conj(psi_{j^x_g}) psi_j D_g(j)); grid.y = slot.
// Products in the state's precision over 8 amplitudes, sums in FP64.
template <typename Real>
__global__ void k_expect_big(Observable o, int n, const typename CT<Real>::T *states, double *out) {
    using C = typename CT<Real>::T;
    __shared__ double red[32];
    const int b = blockIdx.y;
    const C *S = states + ((int64_t)b << n);
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    for (int64_t j0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 8; j0 < dim;
         j0 += (int64_t)gridDim.x * blockDim.x * 8) {
        Real part = 0;
        for (int u = 0; u < 8 && j0 + u < dim; ++u) {
            const uint32_t j = (uint32_t)(j0 + u);
            const C pj = S[j];
            for (int g = 0; g < o.n_tgroups; ++g) {
                const TermGroup tg = o.tgroups[g];
                const C px = S[j ^ tg.x];
                Real dr, di;
                diag_of<Real>(o, tg, j, dr, di);
                const Real wr = fmaR(px.x, pj.x, px.y * pj.y);
                const Real wi = fmaR(px.x, pj.y, -px.y * pj.x);
                part = fmaR(wr, dr, fmaR(-wi, di, part));
            }
        }
        acc += (double)part;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&out[b], s);
}

// lambda = H psi over whole states; E[b] += sum_j Re(conj(psi_j) lambda_j).
template <typename Real>
__global__ void k_apply_h_big(Observable o, int n, const typename CT<Real>::T *psi,
                              typename CT<Real>::T *lam, double *E) {
    using C = typename CT<Real>::T;
    __shared__ double red[32];
    const int b = blockIdx.y;
    const C *S = psi + ((int64_t)b << n);
    C *Lm = lam + ((int64_t)b << n);
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    for (int64_t j0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 8; j0 < dim;
         j0 += (int64_t)gridDim.x * blockDim.x * 8) {
        Real part = 0;
        for (int u = 0; u < 8 && j0 + u < dim; ++u) {
            const uint32_t j = (uint32_t)(j0 + u);
            C l;
            l.x = 0;
            l.y = 0;
            for (int g = 0; g < o.n_tgroups; ++g) {
                const TermGroup tg = o.tgroups[g];
                const uint32_t jx = j ^ tg.x;
                const C px = S[jx];
                Real dr, di;
                diag_of<Real>(o, tg, jx, dr, di);
                l.x = fmaR(dr, px.x, fmaR(-di, px.y, l.x));
                l.y = fmaR(dr, px.y, fmaR(di, px.x, l.y));
            }
            Lm[j] = l;
            const C pj = S[j];
            part = fmaR(pj.x, l.x, fmaR(pj.y, l.y, part));
        }
        acc += (double)part;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&E[b], s);
}

// Per-slot gradients from the summed reduced matrices: one thread per
// (slot, group); slot_grads[b][param] += weight_b * dE_b/dtheta.
template <typename Real>
__global__ void k_group_grads(Program p, SlotSource src, const double *rho_g, CostSource cs,
                              const double *E, double *slot_grads) {
    const int G = p.n_groups, P = p.n_params;
    const int64_t total = (int64_t)src.n_slots * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / G), g = (int)(i % G);
        if (!p.groups[g].has_param) continue;
        const SlotInfo si = resolve(src, b);
        const double wgt = cost_weight(cs, si.instance, E[b]);
        double r8[8];
        for (int v = 0; v < 8; ++v) r8[v] = wgt * rho_g[(size_t)i * 8 + v];
        group_gradients<Real>(p, g, r8, si, slot_grads + (size_t)b * P);
    }
}

template <typename K> cudaError_t allow_smem(K kernel, uint32_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int grid_1d(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b > 8192) b = 8192;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

// ----------------------------------------------------------- launchers

#define HBM_DISPATCH_R(c128, R_, ...)                                      \
    do {                                                                    \
        if (c128) {                                                         \
            using Real = double;                                            \
            switch (R_) {                                                   \
            case 2: { constexpr int RR = 2; __VA_ARGS__; } break;                  \
            case 3: { constexpr int RR = 3; __VA_ARGS__; } break;                  \
            default: return cudaErrorInvalidValue;                          \
            }                                                               \
        } else {                                                            \
            using Real = float;                                             \
            switch (R_) {                                                   \
            case 2: { constexpr int RR = 2; __VA_ARGS__; } break;                  \
            case 3: { constexpr int RR = 3; __VA_ARGS__; } break;                  \
            case 4: { constexpr int RR = 4; __VA_ARGS__; } break;                  \
            default: return cudaErrorInvalidValue;                          \
            }                                                               \
        }                                                                   \
    } while (0)

cudaError_t launch_group_mats(int c128, const Program &p, const SlotSource &src, void *mats,
                              cudaStream_t st) {
    const int g = grid_1d((int64_t)src.n_slots * p.n_groups, 128);
    if (c128) k_group_mats<double><<<g, 128, 0, st>>>(p, src, (double2 *)mats);
    else k_group_mats<float><<<g, 128, 0, st>>>(p, src, (float2 *)mats);
    return cudaGetLastError();
}

cudaError_t launch_init_states(int c128, void *states, int n, const SlotSource &src,
                               cudaStream_t st) {
    const size_t bytes = ((size_t)src.n_slots << n) * (c128 ? 16 : 8);
    cudaError_t e = cudaMemsetAsync(states, 0, bytes, st);
    if (e != cudaSuccess) return e;
    const int g = grid_1d(src.n_slots, 128);
    if (c128) k_set_ref<double2><<<g, 128, 0, st>>>((double2 *)states, n, src);
    else k_set_ref<float2><<<g, 128, 0, st>>>((float2 *)states, n, src);
    return cudaGetLastError();
}

uint32_t pass_fwd_smem(int c128, int t, int R, int G, int n_st, int n_ops) {
    const uint32_t base = 2u * (uint32_t)((c128 ? 16 : 8) << t) + (uint32_t)(G * 4 * (c128 ? 16 : 8));
    return pass_smem_layout(base, n_st, n_ops, 1 << (t - R), G).end;
}

uint32_t pass_rev_smem(int c128, int t, int R, int G, int n_u1, int n_st, int n_ops) {
    const uint32_t base = rev_layout(t, R, c128 ? 16 : 8, c128 ? 8 : 4, G, n_u1).total +
                          (uint32_t)(G * 4 * (c128 ? 16 : 8));
    return pass_smem_layout(base, n_st, n_ops, 1 << (t - R), G).end;
}

cudaError_t launch_pass_fwd(int c128, int R, const PassDesc &pd, const Program &pv, int op0,
                            int n_ops, int n, int n_slots, const void *mats, int G, void *states,
                            int blocks, cudaStream_t st) {
    const uint32_t smem = pass_fwd_smem(c128, pd.t, R, G, pv.n_stages, n_ops);
    const int threads = 1 << (pd.t - R);
    HBM_DISPATCH_R(c128, R, {
        using C = typename CT<Real>::T;
        auto k = k_pass_fwd<Real, RR>;
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<blocks, threads, smem, st>>>(pd, pv, op0, n_ops, n, n_slots, (const C *)mats, G,
                                         (C *)states);
    });
    return cudaGetLastError();
}

cudaError_t launch_pass_rev(int c128, int R, const PassDesc &pd, const Program &pv, int op0,
                            int n_ops, int n, int n_slots, const void *mats, int G, void *psi,
                            void *lam, double *rho_g, int blocks, cudaStream_t st) {
    const uint32_t smem = pass_rev_smem(c128, pd.t, R, G, pd.n_u1, pv.n_stages, n_ops);
    const int threads = 1 << (pd.t - R);
    HBM_DISPATCH_R(c128, R, {
        using C = typename CT<Real>::T;
        auto k = k_pass_rev<Real, RR>;
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<blocks, threads, smem, st>>>(pd, pv, op0, n_ops, n, n_slots, (const C *)mats, G,
                                         (C *)psi, (C *)lam, rho_g);
    });
    return cudaGetLastError();
}

static dim3 whole_state_grid(int n, int rows) {
    const int64_t per = ((int64_t(1) << n) + 2047) / 2048;  // 256 threads x 8 amplitudes
    int64_t x = per;
    const int64_t cap = rows >= 1024 ? 1 : (int64_t)2048 / rows;
    if (x > cap) x = cap < 1 ? 1 : cap;
    return dim3((unsigned)x, (unsigned)rows, 1);
}

cudaError_t launch_expect_big(int c128, const Observable &o, int n, int n_rows,
                              const void *states, double *out, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * n_rows, st);
    if (e != cudaSuccess) return e;
    const dim3 g = whole_state_grid(n, n_rows);
    if (c128) k_expect_big<double><<<g, 256, 0, st>>>(o, n, (const double2 *)states, out);
    else k_expect_big<float><<<g, 256, 0, st>>>(o, n, (const float2 *)states, out);
    return cudaGetLastError();
}

cudaError_t launch_apply_h_big(int c128, const Observable &o, int n, int n_rows, const void *psi,
                               void *lam, double *E, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(E, 0, sizeof(double) * n_rows, st);
    if (e != cudaSuccess) return e;
    const dim3 g = whole_state_grid(n, n_rows);
    if (c128) k_apply_h_big<double><<<g, 256, 0, st>>>(o, n, (const double2 *)psi, (double2 *)lam, E);
    else k_apply_h_big<float><<<g, 256, 0, st>>>(o, n, (const float2 *)psi, (float2 *)lam, E);
    return cudaGetLastError();
}

cudaError_t launch_group_grads(int c128, const Program &p, const SlotSource &src,
                               const double *rho_g, const CostSource &cs, const double *E,
                               double *slot_grads, cudaStream_t st) {
    const int g = grid_1d((int64_t)src.n_slots * p.n_groups, 128);
    if (c128) k_group_grads<double><<<g, 128, 0, st>>>(p, src, rho_g, cs, E, slot_grads);
    else k_group_grads<float><<<g, 128, 0, st>>>(p, src, rho_g, cs, E, slot_grads);
    return cudaGetLastError();
}

}  // namespace svk
