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

// ------------------------------------------------------------ tile passes
//
// A block owns one contiguous range of (slot, tile) pairs.  Tiles arrive by
// cp.async in one of two buffers, so the next tile is in flight while the
// current one is computed.  Every register stage loads the thread's 2^R
// amplitudes from shared memory, applies the fused 2x2 group of each of its
// register bits (at most one per bit) and stores them back in place.  The
// pass descriptor is a __grid_constant__ parameter: its stage vectors are
// read with warp-uniform indices through the constant cache.  Each thread
// computes its per-stage address bases once per launch.

__device__ __forceinline__ void cp_async_amp(uint32_t sdst, const float2 *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sdst), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_amp(uint32_t sdst, const double2 *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Offsets of this thread's amplitudes (tile-local index tid + k 2^(t-R))
// through the per-bit vector table v: returns the tid part and fills the
// parts of the R register bits.
template <int R>
__device__ __forceinline__ uint32_t bit_vectors(const uint32_t *v, int t, int tid,
                                                uint32_t (&k)[R]) {
    const int tb = t - R;
    uint32_t g = 0;
    for (int b = 0; b < tb; ++b)
        if ((tid >> b) & 1) g ^= v[b];
#pragma unroll
    for (int j = 0; j < R; ++j) k[j] = v[tb + j];
    return g;
}

// Position of one tile in the walk over (slot, tile): global offset of the
// tile's first amplitude within its state.
struct TileCursor {
    int slot;
    uint32_t local, base;
};

__device__ __forceinline__ TileCursor tile_cursor(const TilePass &P, int64_t tix) {
    TileCursor c;
    c.slot = (int)(tix >> P.n_tile_bits);
    c.local = (uint32_t)(tix & ((int64_t(1) << P.n_tile_bits) - 1));
    c.base = 0;
    for (int k = 0; k < P.n_tile_bits; ++k)
        if ((c.local >> k) & 1u) c.base ^= P.gpre[k] ^ (k ? P.gpre[k - 1] : 0u);
    return c;
}

// Next tile: counting up flips tile-number bits 0..ctz(local + 1).
__device__ __forceinline__ TileCursor tile_next(const TilePass &P, TileCursor c) {
    ++c.local;
    if ((c.local >> P.n_tile_bits) != 0u) {
        c.local = 0;
        c.base = 0;
        ++c.slot;
    } else {
        c.base ^= P.gpre[__ffs((int)c.local) - 1];
    }
    return c;
}

// The group ops of one stage, register bits I..R-1 in order.
template <typename C, int R, int I>
__device__ __forceinline__ void tile_ops_fwd(const TilePass &P, const TileStage &sg, const C *sm,
                                             C (&a)[1 << R]) {
    if constexpr (I < R) {
        const int u = sg.op[I];
        if (u >= 0) {
            const C m0 = sm[4 * u], m1 = sm[4 * u + 1], m2 = sm[4 * u + 2], m3 = sm[4 * u + 3];
            if ((P.real_mask >> u) & 1ull)
                u1r_bit<C, decltype(m0.x), R, I>(a, m0.x, m1.x, m2.x, m3.x);
            else
                u1_bit<C, R, I>(a, m0, m1, m2, m3);
        }
        tile_ops_fwd<C, R, I + 1>(P, sg, sm, a);
    }
}

// One forward pass over every tile of every slot.  mats: [slots][G][4].
template <typename Real, int R>
__global__ void __launch_bounds__(256, 3)
k_tile_fwd(const __grid_constant__ TilePass P, int n, int n_slots,
           const typename CT<Real>::T *mats, int G, typename CT<Real>::T *states) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, T = blockDim.x, t = P.t, S = P.n_stages;
    const uint32_t tbytes = (uint32_t)sizeof(C) << t;
    uint2 *tb = reinterpret_cast<uint2 *>(smem + 2 * tbytes);
    C *sm = reinterpret_cast<C *>(smem + 2 * tbytes + (uint32_t)S * T * 8u);
    for (int s = 0; s < S; ++s) {
        const TileStage &sg = P.st[s];
        uint32_t lb = 0, sb = 0;
        for (int k = 0; k < t - R; ++k)
            if ((tid >> k) & 1) {
                lb ^= sg.ldt[k];
                sb ^= sg.stt[k];
            }
        tb[s * T + tid] = make_uint2(lb, sb);
    }
    uint32_t gk[R], pk[R], nk[R];
    const uint32_t g0 = bit_vectors<R>(P.gl, t, tid, gk);
    const uint32_t p0 = bit_vectors<R>(P.ldperm, t, tid, pk);
    const uint32_t n0 = bit_vectors<R>(P.nat, t, tid, nk);
    const uint32_t sh = (uint32_t)__cvta_generic_to_shared(smem);
    const int64_t tiles = (int64_t)n_slots << P.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = per * blockIdx.x, t_end = min(tiles, t0 + per);
    if (t0 >= t_end) return;
    auto fetch = [&](const TileCursor &c, int buf) {
        const C *src = states + ((int64_t)c.slot << n) + c.base;
        const uint32_t d = sh + (uint32_t)buf * tbytes;
#pragma unroll
        for (int k = 0; k < NA; ++k) cp_async_amp(d + (p0 ^ xsel<R>(k, pk)), src + (g0 ^ xsel<R>(k, gk)));
        cp_async_commit();
    };
    TileCursor cur = tile_cursor(P, t0);
    fetch(cur, 0);
    TileCursor nxt = tile_next(P, cur);
    int mslot = -1;
    for (int64_t tix = t0, i = 0; tix < t_end; ++tix, ++i) {
        const int buf = (int)(i & 1);
        if (cur.slot != mslot) {  // the previous tile's stages are past their last barrier
            for (int x = tid; x < 4 * P.n_ops; x += T)
                sm[x] = mats[((size_t)cur.slot * G + P.grp[x >> 2]) * 4 + (x & 3)];
            mslot = cur.slot;
        }
        cp_async_wait_all();
        __syncthreads();
        if (tix + 1 < t_end) fetch(nxt, buf ^ 1);
        unsigned char *tile = smem + (uint32_t)buf * tbytes;
        for (int s = 0; s < S; ++s) {
            const TileStage &sg = P.st[s];
            const uint2 bb = tb[s * T + tid];
            uint32_t lq[R], sq[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                lq[j] = sg.ldq[j];
                sq[j] = sg.stq[j];
            }
            C a[NA];
#pragma unroll
            for (int r = 0; r < NA; ++r) a[r] = *reinterpret_cast<const C *>(tile + (bb.x ^ xsel<R>(r, lq)));
            tile_ops_fwd<C, R, 0>(P, sg, sm, a);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < NA; ++r) *reinterpret_cast<C *>(tile + (bb.y ^ xsel<R>(r, sq))) = a[r];
            __syncthreads();
        }
        C *dst = states + ((int64_t)cur.slot << n) + cur.base;
#pragma unroll
        for (int k = 0; k < NA; ++k)
            dst[g0 ^ xsel<R>(k, gk)] = *reinterpret_cast<const C *>(tile + (n0 ^ xsel<R>(k, nk)));
        cur = nxt;
        nxt = tile_next(P, nxt);
    }
}

// Sum over the 32 lanes of the 8 values rh[0..7]: lane l ends with the total
// of value l & 7 (reduce-scatter over lane bits 0-2, then lane bits 3-4).
template <typename Real>
__device__ __forceinline__ Real warp_reduce8(const Real (&rh)[8], int lane) {
    constexpr unsigned full = 0xffffffffu;
    Real y[4], z[2];
    const bool b0 = lane & 1, b1 = lane & 2, b2 = lane & 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const Real keep = b0 ? rh[2 * j + 1] : rh[2 * j], give = b0 ? rh[2 * j] : rh[2 * j + 1];
        y[j] = keep + __shfl_xor_sync(full, give, 1);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const Real keep = b1 ? y[2 * m + 1] : y[2 * m], give = b1 ? y[2 * m] : y[2 * m + 1];
        z[m] = keep + __shfl_xor_sync(full, give, 2);
    }
    const Real keep = b2 ? z[1] : z[0], give = b2 ? z[0] : z[1];
    Real v = keep + __shfl_xor_sync(full, give, 4);
    v += __shfl_xor_sync(full, v, 8);
    v += __shfl_xor_sync(full, v, 16);
    return v;
}

// Reverse of tile_ops_fwd, register bits I, I-1, ..., 0: per op, first the
// reduced matrix rho_ab = sum psi_a conj(lambda_b) of its bit (at the point
// after the group) into the warp's accumulator acc[u][warp][8], then the
// inverse group (sm holds the adjoint matrices) on psi and lambda.
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void tile_ops_rev(const TilePass &P, const TileStage &sg, const C *sm,
                                             C (&a)[1 << R], C (&al)[1 << R], Real *accw,
                                             int wps, int lane) {
    if constexpr (I >= 0) {
        const int u = sg.op[I];
        if (u >= 0) {
            if ((P.param_mask >> u) & 1ull) {
                Real rh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                rho_bit<C, Real, R, I>(a, al, rh);
                const Real v = warp_reduce8<Real>(rh, lane);
                if (lane < 8) accw[u * wps * 8 + lane] += v;
            }
            const C m0 = sm[4 * u], m1 = sm[4 * u + 1], m2 = sm[4 * u + 2], m3 = sm[4 * u + 3];
            if ((P.real_mask >> u) & 1ull) {
                u1r_bit<C, Real, R, I>(a, m0.x, m1.x, m2.x, m3.x);
                u1r_bit<C, Real, R, I>(al, m0.x, m1.x, m2.x, m3.x);
            } else {
                u1_bit<C, R, I>(a, m0, m1, m2, m3);
                u1_bit<C, R, I>(al, m0, m1, m2, m3);
            }
        }
        tile_ops_rev<C, Real, R, I - 1>(P, sg, sm, a, al, accw, wps, lane);
    }
}

// Adds the block's reduced-matrix sums of slot b (FP64 over warps) to
// rho_g[b][group][8] and clears them.  Called by every thread.
template <typename Real>
__device__ void flush_acc(const TilePass &P, Real *acc, int wps, double *rho_g, int b, int G) {
    __syncthreads();
    for (int x = threadIdx.x; x < P.n_ops * 8; x += blockDim.x) {
        const int u = x >> 3, v = x & 7;
        if (!((P.param_mask >> u) & 1ull)) continue;
        double s = 0.0;
        for (int w = 0; w < wps; ++w) {
            Real &r = acc[(u * wps + w) * 8 + v];
            s += (double)r;
            r = 0;
        }
        if (s != 0.0) atomicAdd(&rho_g[((size_t)b * G + P.grp[u]) * 8 + v], s);
    }
    __syncthreads();
}

// One reverse pass: un-applies the pass on psi and lambda tiles and sums the
// reduced matrices of its parametrised groups into rho_g[slot][group][8].
// Reduced-matrix partials are summed in the state's precision over one
// warp and at most 64 tiles, then in FP64.
template <typename Real, int R>
__global__ void __launch_bounds__(256, 2)
k_tile_rev(const __grid_constant__ TilePass P, int n, int n_slots,
           const typename CT<Real>::T *mats, int G, typename CT<Real>::T *psi,
           typename CT<Real>::T *lam, double *rho_g) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    constexpr int kFlushTiles = 64;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, T = blockDim.x, t = P.t, S = P.n_stages;
    const int lane = tid & 31, wps = T >> 5;
    const uint32_t tbytes = (uint32_t)sizeof(C) << t;
    uint2 *tb = reinterpret_cast<uint2 *>(smem + 4 * tbytes);
    C *sm = reinterpret_cast<C *>(smem + 4 * tbytes + (uint32_t)S * T * 8u);
    Real *acc = reinterpret_cast<Real *>(sm + 4 * P.n_ops);
    for (int s = 0; s < S; ++s) {
        const TileStage &sg = P.st[s];
        uint32_t lb = 0, sb = 0;
        for (int k = 0; k < t - R; ++k)
            if ((tid >> k) & 1) {
                lb ^= sg.ldt[k];
                sb ^= sg.stt[k];
            }
        tb[s * T + tid] = make_uint2(lb, sb);
    }
    for (int x = tid; x < P.n_ops * wps * 8; x += T) acc[x] = 0;
    Real *accw = acc + (tid >> 5) * 8;
    uint32_t gk[R], pk[R], nk[R];
    const uint32_t g0 = bit_vectors<R>(P.gl, t, tid, gk);
    const uint32_t p0 = bit_vectors<R>(P.ldperm, t, tid, pk);
    const uint32_t n0 = bit_vectors<R>(P.nat, t, tid, nk);
    const uint32_t sh = (uint32_t)__cvta_generic_to_shared(smem);
    const int64_t tiles = (int64_t)n_slots << P.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = per * blockIdx.x, t_end = min(tiles, t0 + per);
    if (t0 >= t_end) return;
    // psi tile of buffer j at [j tbytes], lambda tile at [(2 + j) tbytes]
    auto fetch = [&](const TileCursor &c, int buf) {
        const int64_t off = ((int64_t)c.slot << n) + c.base;
        const C *sp = psi + off, *sl = lam + off;
        const uint32_t dp = sh + (uint32_t)buf * tbytes, dl = dp + 2 * tbytes;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t so = n0 ^ xsel<R>(k, nk), go = g0 ^ xsel<R>(k, gk);
            cp_async_amp(dp + so, sp + go);
            cp_async_amp(dl + so, sl + go);
        }
        cp_async_commit();
    };
    TileCursor cur = tile_cursor(P, t0);
    fetch(cur, 0);
    TileCursor nxt = tile_next(P, cur);
    int mslot = -1, since = 0;
    for (int64_t tix = t0, i = 0; tix < t_end; ++tix, ++i) {
        const int buf = (int)(i & 1);
        if (cur.slot != mslot || since == kFlushTiles) {
            if (mslot >= 0) flush_acc<Real>(P, acc, wps, rho_g, mslot, G);
            since = 0;
        }
        if (cur.slot != mslot) {  // adjoint matrices of this slot's groups
            for (int x = tid; x < 4 * P.n_ops; x += T) {
                const C *m = mats + ((size_t)cur.slot * G + P.grp[x >> 2]) * 4;
                const int e = x & 3, te = e == 1 ? 2 : (e == 2 ? 1 : e);
                C d = m[te];
                d.y = -d.y;
                sm[x] = d;
            }
            mslot = cur.slot;
        }
        cp_async_wait_all();
        __syncthreads();
        if (tix + 1 < t_end) fetch(nxt, buf ^ 1);
        unsigned char *tp = smem + (uint32_t)buf * tbytes, *tl = tp + 2 * tbytes;
        for (int s = S - 1; s >= 0; --s) {
            const TileStage &sg = P.st[s];
            const uint2 bb = tb[s * T + tid];
            uint32_t lq[R], sq[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                lq[j] = sg.ldq[j];
                sq[j] = sg.stq[j];
            }
            C a[NA], al[NA];
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                const uint32_t ad = bb.y ^ xsel<R>(r, sq);
                a[r] = *reinterpret_cast<const C *>(tp + ad);
                al[r] = *reinterpret_cast<const C *>(tl + ad);
            }
            tile_ops_rev<C, Real, R, R - 1>(P, sg, sm, a, al, accw, wps, lane);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                const uint32_t ad = bb.x ^ xsel<R>(r, lq);
                *reinterpret_cast<C *>(tp + ad) = a[r];
                *reinterpret_cast<C *>(tl + ad) = al[r];
            }
            __syncthreads();
        }
        const int64_t off = ((int64_t)cur.slot << n) + cur.base;
        C *dp = psi + off, *dl = lam + off;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t so = p0 ^ xsel<R>(k, pk), go = g0 ^ xsel<R>(k, gk);
            dp[go] = *reinterpret_cast<const C *>(tp + so);
            dl[go] = *reinterpret_cast<const C *>(tl + so);
        }
        ++since;
        cur = nxt;
        nxt = tile_next(P, nxt);
    }
    flush_acc<Real>(P, acc, wps, rho_g, mslot, G);
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

// Resident blocks of kernel k on the whole GPU, at most max_blocks.
template <typename K> int fill_blocks(K kernel, int threads, uint32_t smem, int64_t max_blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess ||
        per < 1)
        per = 1;
    int64_t b = (int64_t)sms * per;
    if (b > max_blocks) b = max_blocks;
    return b < 1 ? 1 : (int)b;
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

uint32_t tile_fwd_smem(int c128, const TilePass &P) {
    const uint32_t csz = c128 ? 16u : 8u, T = 1u << (P.t - P.R);
    return 2u * (csz << P.t) + (uint32_t)P.n_stages * T * 8u + (uint32_t)P.n_ops * 4u * csz;
}

uint32_t tile_rev_smem(int c128, const TilePass &P) {
    const uint32_t csz = c128 ? 16u : 8u, rsz = c128 ? 8u : 4u, T = 1u << (P.t - P.R);
    return 4u * (csz << P.t) + (uint32_t)P.n_stages * T * 8u + (uint32_t)P.n_ops * 4u * csz +
           (uint32_t)P.n_ops * (T / 32u) * 8u * rsz;
}

cudaError_t launch_tile_fwd(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *states, int64_t max_blocks, cudaStream_t st) {
    const uint32_t smem = tile_fwd_smem(c128, P);
    const int threads = 1 << (P.t - P.R);
    HBM_DISPATCH_R(c128, P.R, {
        using C = typename CT<Real>::T;
        auto k = k_tile_fwd<Real, RR>;
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        const int blocks = fill_blocks(k, threads, smem, max_blocks);
        k<<<blocks, threads, smem, st>>>(P, n, n_slots, (const C *)mats, G, (C *)states);
    });
    return cudaGetLastError();
}

cudaError_t launch_tile_rev(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *psi, void *lam, double *rho_g, int64_t max_blocks,
                            cudaStream_t st) {
    const uint32_t smem = tile_rev_smem(c128, P);
    const int threads = 1 << (P.t - P.R);
    HBM_DISPATCH_R(c128, P.R, {
        using C = typename CT<Real>::T;
        auto k = k_tile_rev<Real, RR>;
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        const int blocks = fill_blocks(k, threads, smem, max_blocks);
        k<<<blocks, threads, smem, st>>>(P, n, n_slots, (const C *)mats, G, (C *)psi, (C *)lam,
                                         rho_g);
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
