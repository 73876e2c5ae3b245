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

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "engine.cuh"
#include "hbm.h"
#include "tile_common.cuh"

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

// One forward pass over every tile of every slot.  mats: [slots][G][4].
// One forward stage: a branch-free path when register bits 0..M-1 carry
// real rotations in shear form or complex matrices (M from the stage
// flags), tile_ops_fwd otherwise.
template <typename C, int R, bool kReal>
__device__ __forceinline__ void stage_ops_fwd(uint32_t ops, uint32_t flags, const C *sm,
                                              C (&a)[1 << R]) {
    const uint32_t m = flags & 15u;
    if constexpr (R >= 4) {
        if (m == 4) return tile_ops_fwd_rot<C, R, 0, 4>(ops, sm, a);
    }
    if constexpr (R >= 3) {
        if (m == 3) return tile_ops_fwd_rot<C, R, 0, 3>(ops, sm, a);
    }
    if (m == 2) return tile_ops_fwd_rot<C, R, 0, 2>(ops, sm, a);
    if (m == 1) return tile_ops_fwd_rot<C, R, 0, 1>(ops, sm, a);
    if constexpr (!kReal) {
        const uint32_t mc = (flags >> 8) & 15u;
        if constexpr (R >= 4) {
            if (mc == 4) return tile_ops_fwd_cplx<C, R, 0, 4>(ops, sm, a);
        }
        if constexpr (R >= 3) {
            if (mc == 3) return tile_ops_fwd_cplx<C, R, 0, 3>(ops, sm, a);
        }
        if (mc == 2) return tile_ops_fwd_cplx<C, R, 0, 2>(ops, sm, a);
        if (mc == 1) return tile_ops_fwd_cplx<C, R, 0, 1>(ops, sm, a);
    }
    tile_ops_fwd<C, R, 0, kReal>(ops, sm, a);
}

template <typename Real, int R, bool kReal>
__device__ __forceinline__ void tile_fwd_body(const TilePass &P, int n, int n_slots,
                                              const typename CT<Real>::T *mats, int G,
                                              const typename CT<Real>::T *src_states,
                                              typename CT<Real>::T *states, int64_t t0,
                                              int64_t t_end, unsigned char *smem) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    constexpr uint32_t kBufs = 2u;
    const int tid = threadIdx.x, T = blockDim.x, t = P.t, S = P.n_stages;
    const uint32_t tbytes = (uint32_t)sizeof(C) << t;
    uint2 *tb = reinterpret_cast<uint2 *>(smem + kBufs * tbytes);
    uint4 *rec = reinterpret_cast<uint4 *>(smem + kBufs * tbytes + (uint32_t)S * T * 8u);
    C *sm = reinterpret_cast<C *>(rec + 2 * S);
    build_stage_recs(P, rec);
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
    if (t0 >= t_end) return;
    auto fetch = [&](const TileCursor &c, int buf) {
        const C *src = src_states + ((int64_t)c.slot << n) + c.base;
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
            __syncthreads();
            for (int u = tid; u < P.n_ops; u += T)
                if ((P.real_mask >> u) & 1ull) stage_shears(sm + 4 * u);
            if constexpr (std::is_same<C, float2>::value) {
                __syncthreads();  // the branch-free paths' stage flags
                set_stage_flags(P, rec, sm);
            }
            mslot = cur.slot;
        }
        cp_async_wait_all();
        __syncthreads();
        if (tix + 1 < t_end) fetch(nxt, buf ^ 1);
        unsigned char *tile = smem + (uint32_t)buf * tbytes;
        for (int s = 0; s < S; ++s) {
            const uint2 bb = tb[s * T + tid];
            uint32_t lq[R], sq[R];
            const uint32_t ops = read_stage_rec<R>(rec, s, lq, sq);
            C a[NA];
#pragma unroll
            for (int r = 0; r < NA; ++r) a[r] = *reinterpret_cast<const C *>(tile + (bb.x ^ xsel<R>(r, lq)));
            // complex64: the branch-free paths where the stage allows
            if constexpr (std::is_same<C, float2>::value) {
                stage_ops_fwd<C, R, kReal>(ops, rec[2 * s + 1].w, sm, a);
            } else {
                tile_ops_fwd<C, R, 0, kReal>(ops, sm, a);
            }
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

// src: the states the pass reads; states: where it writes them (the same
// buffer, or another one when the pass's output is also kept as a stored
// forward state).
template <typename Real, int R, bool kReal>
__global__ void __launch_bounds__(256, R >= 4 ? 2 : 3)
k_tile_fwd(const __grid_constant__ TilePass P, int n, int n_slots,
           const typename CT<Real>::T *mats, int G, const typename CT<Real>::T *src,
           typename CT<Real>::T *states) {
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t t0, t_end;
    block_range((int64_t)n_slots << P.n_tile_bits, gridDim.x, blockIdx.x, t0, t_end);
    tile_fwd_body<Real, R, kReal>(P, n, n_slots, mats, G, src, states, t0, t_end, smem);
}

// The derivative of a rotation exp(-i theta P / 2) inside a fused group is
// Im tr(Q rho) for a Hermitian Q, with rho_ab = sum psi_a conj(lambda_b) over
// the amplitude pairs of the group's qubit.  Only the Hermitian matrix
// K = (rho - rho^dag) / 2i enters (Im tr(Q rho) = tr(Q K)), and i K gives
// the same derivatives as rho, also after conjugation by the group's
// members.  Four sums fix K:
//   k0 = Im rho_00, k1 = Im rho_11, k2 = Im rho_01 + Im rho_10,
//   k3 = Re rho_01 - Re rho_10,
// and i K = [[i k0, (k3 + i k2) / 2], [(-k3 + i k2) / 2, i k1]].
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void kmat_bit(const C (&a)[1 << R], const C (&l)[1 << R], Real *k) {
#pragma unroll
    for (int r = 0; r < (1 << R); ++r) {
        if (r & (1 << I)) continue;
        const C p0 = a[r], p1 = a[r | (1 << I)], l0 = l[r], l1 = l[r | (1 << I)];
        k[0] = fmaR(p0.y, l0.x, fmaR(-p0.x, l0.y, k[0]));
        k[1] = fmaR(p1.y, l1.x, fmaR(-p1.x, l1.y, k[1]));
        k[2] = fmaR(p0.y, l1.x, fmaR(-p0.x, l1.y, fmaR(p1.y, l0.x, fmaR(-p1.x, l0.y, k[2]))));
        k[3] = fmaR(p0.x, l1.x, fmaR(p0.y, l1.y, fmaR(-p1.x, l0.x, fmaR(-p1.y, l0.y, k[3]))));
    }
}

// Partial sum over the lanes of NV values x[0..NV-1] (NV = 8 or 16):
// afterwards x[m] (m < NV / 4) holds value 4 m + (lane & 3) summed over the
// four lanes that differ in lane bits 0-1 (a reduce-scatter of two levels;
// the kept half follows the lane bit).
template <typename Real, int NV>
__device__ __forceinline__ void warp_reduce_quad(Real (&x)[NV], int lane) {
    constexpr unsigned full = 0xffffffffu;
#pragma unroll
    for (int j = 0, M = NV; j < 2; ++j, M >>= 1) {
        const bool b = (lane >> j) & 1;
#pragma unroll
        for (int m = 0; m < M / 2; ++m) {
            const Real keep = b ? x[2 * m + 1] : x[2 * m], give = b ? x[2 * m] : x[2 * m + 1];
            x[m] = keep + __shfl_xor_sync(full, give, 1 << j);
        }
    }
}

// The one sum a group needs when its only rotation is its last member
// (fmode md): 1: k3 (RY), 2: k2 (RX), 3: k0 - k1 (RZ), over the pairs of
// register bit I.
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ Real single_sum(const C (&a)[1 << R], const C (&l)[1 << R],
                                           uint32_t md) {
    Real v = 0;
    if (md == 1) {
        if constexpr (std::is_same<C, float2>::value) {
            // k3 = sum x0 . y1 - x1 . y0 (as real 2-vectors): packed FMA
            // chains (two per product when there are four or more pairs, so
            // that the chains are half as long), their halves added at the end
            constexpr int NC = (1 << R) >= 8 ? 2 : 1;
            uint64_t pa[NC], pb[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) pa[c] = pb[c] = 0;
            int m = 0;
#pragma unroll
            for (int r = 0; r < (1 << R); ++r) {
                if (r & (1 << I)) continue;
                pa[m % NC] = f2fma(f2of(a[r]), f2of(l[r | (1 << I)]), pa[m % NC]);
                pb[m % NC] = f2fma(f2of(a[r | (1 << I)]), f2of(l[r]), pb[m % NC]);
                ++m;
            }
            float2 A = f2unpack(pa[0]), B = f2unpack(pb[0]);
            if constexpr (NC > 1) {
                const float2 A1 = f2unpack(pa[1]), B1 = f2unpack(pb[1]);
                A.x += A1.x;
                A.y += A1.y;
                B.x += B1.x;
                B.y += B1.y;
            }
            v = (A.x + A.y) - (B.x + B.y);
        } else {
#pragma unroll
            for (int r = 0; r < (1 << R); ++r) {
                if (r & (1 << I)) continue;
                const C x0 = a[r], x1 = a[r | (1 << I)], y0 = l[r], y1 = l[r | (1 << I)];
                v = fmaR(x0.x, y1.x, fmaR(x0.y, y1.y, fmaR(-x1.x, y0.x, fmaR(-x1.y, y0.y, v))));
            }
        }
    } else if (md == 2) {
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            const C x0 = a[r], x1 = a[r | (1 << I)], y0 = l[r], y1 = l[r | (1 << I)];
            v = fmaR(x0.y, y1.x, fmaR(-x0.x, y1.y, fmaR(x1.y, y0.x, fmaR(-x1.x, y0.y, v))));
        }
    } else {
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            const C x0 = a[r], x1 = a[r | (1 << I)], y0 = l[r], y1 = l[r | (1 << I)];
            v = fmaR(x0.y, y0.x, fmaR(-x0.x, y0.y, fmaR(-x1.y, y1.x, fmaR(x1.x, y1.y, v))));
        }
    }
    return v;
}

// Reverse of tile_ops_fwd, register bits I, I-1, ..., 0: per op, first its
// sums (at the point after the group) into k — k0..k3 at k[4 I ..], or with
// kSingle the one sum of its fmode at k[I] — then the inverse group (sm
// holds the adjoint matrices) on psi and lambda.
template <typename C, typename Real, int R, int I, int NV, bool kSingle, bool kReal>
__device__ __forceinline__ void tile_ops_rev(uint32_t ops, uint32_t modes, const C *sm,
                                             C (&a)[1 << R], C (&al)[1 << R], Real (&k)[NV]) {
    if constexpr (I >= 0) {
        const uint32_t ob = (ops >> (8 * I)) & 0xffu;
        if (ob) {
            if (ob & 128u) {
                if constexpr (kSingle)
                    k[I] = single_sum<C, Real, R, I>(a, al, (modes >> (8 * I)) & 3u);
                else
                    kmat_bit<C, Real, R, I>(a, al, &k[4 * I]);
            }
            C m0, m1, m2, m3;
            load_mat(sm, (int)(ob & 63u) - 1, m0, m1, m2, m3);
            if (kReal || (ob & 64u)) {
                if (m2.y != 0) {
                    rot3_bit<C, Real, R, I>(a, m0.y, m1.y);
                    rot3_bit<C, Real, R, I>(al, m0.y, m1.y);
                } else {
                    u1r_bit<C, Real, R, I>(a, m0.x, m1.x, m2.x, m3.x);
                    u1r_bit<C, Real, R, I>(al, m0.x, m1.x, m2.x, m3.x);
                }
            } else {
                u1_bit<C, R, I>(a, m0, m1, m2, m3);
                u1_bit<C, R, I>(al, m0, m1, m2, m3);
            }
        }
        tile_ops_rev<C, Real, R, I - 1, NV, kSingle, kReal>(ops, modes, sm, a, al, k);
    }
}

// tile_ops_rev for register bits I..0 that all carry parametrised real
// rotations in shear form with the single Ry sum (stage flags, bits 4-7):
// the same arithmetic without its per-op branches, so the compiler can
// overlap one op's dependent FMA chains with the next op's.
template <typename C, typename Real, int R, int I, int NV>
__device__ __forceinline__ void tile_ops_rev_rot(uint32_t ops, const C *sm, C (&a)[1 << R],
                                                 C (&al)[1 << R], Real (&k)[NV]) {
    if constexpr (I >= 0) {
        k[I] = single_sum<C, Real, R, I>(a, al, 1u);
        C m0, m1, m2, m3;
        load_mat(sm, (int)((ops >> (8 * I)) & 63u) - 1, m0, m1, m2, m3);
        rot3_bit<C, Real, R, I>(a, m0.y, m1.y);
        rot3_bit<C, Real, R, I>(al, m0.y, m1.y);
        tile_ops_rev_rot<C, Real, R, I - 1, NV>(ops, sm, a, al, k);
    }
}

// One reverse stage of single-sum ops: the branch-free path when register
// bits 0..M-1 carry parametrised real rotations (M from the stage flags),
// tile_ops_rev otherwise.
template <typename C, typename Real, int R, int NV, bool kReal>
__device__ __forceinline__ void stage_ops_rev(uint32_t ops, uint32_t modes, uint32_t m,
                                              const C *sm, C (&a)[1 << R], C (&al)[1 << R],
                                              Real (&k)[NV]) {
    if constexpr (R >= 4) {
        if (m == 4) return tile_ops_rev_rot<C, Real, R, 3, NV>(ops, sm, a, al, k);
    }
    if constexpr (R >= 3) {
        if (m == 3) return tile_ops_rev_rot<C, Real, R, 2, NV>(ops, sm, a, al, k);
    }
    if (m == 2) return tile_ops_rev_rot<C, Real, R, 1, NV>(ops, sm, a, al, k);
    if (m == 1) return tile_ops_rev_rot<C, Real, R, 0, NV>(ops, sm, a, al, k);
    tile_ops_rev<C, Real, R, R - 1, NV, true, kReal>(ops, modes, sm, a, al, k);
}

// tile_ops_rev's four-sum complex path when register bits 0..M-1 all carry
// parametrised complex matrices (stage flags, bits 12-15), without its
// per-op branches.
template <typename C, typename Real, int R, int I, int NV>
__device__ __forceinline__ void tile_ops_rev_cplx(uint32_t ops, const C *sm, C (&a)[1 << R],
                                                  C (&al)[1 << R], Real (&k)[NV]) {
    if constexpr (I >= 0) {
        kmat_bit<C, Real, R, I>(a, al, &k[4 * I]);
        C m0, m1, m2, m3;
        load_mat(sm, (int)((ops >> (8 * I)) & 63u) - 1, m0, m1, m2, m3);
        u1_bit<C, R, I>(a, m0, m1, m2, m3);
        u1_bit<C, R, I>(al, m0, m1, m2, m3);
        tile_ops_rev_cplx<C, Real, R, I - 1, NV>(ops, sm, a, al, k);
    }
}

// One reverse stage of four-sum ops: the branch-free complex path when
// register bits 0..M-1 carry parametrised complex matrices, tile_ops_rev
// otherwise.
template <typename C, typename Real, int R, int NV, bool kReal>
__device__ __forceinline__ void stage_ops_rev4(uint32_t ops, uint32_t modes, uint32_t m,
                                               const C *sm, C (&a)[1 << R], C (&al)[1 << R],
                                               Real (&k)[NV]) {
    if constexpr (R >= 4) {
        if (m == 4) return tile_ops_rev_cplx<C, Real, R, 3, NV>(ops, sm, a, al, k);
    }
    if constexpr (R >= 3) {
        if (m == 3) return tile_ops_rev_cplx<C, Real, R, 2, NV>(ops, sm, a, al, k);
    }
    if (m == 2) return tile_ops_rev_cplx<C, Real, R, 1, NV>(ops, sm, a, al, k);
    if (m == 1) return tile_ops_rev_cplx<C, Real, R, 0, NV>(ops, sm, a, al, k);
    tile_ops_rev<C, Real, R, R - 1, NV, false, kReal>(ops, modes, sm, a, al, k);
}

// Adds the block's sums of slot b (FP64 over warps and lane quads), as i K
// in reduced-matrix form, to rho_g[b][group][8] and clears them.  Called by
// every thread.
template <typename Real, bool kSingle>
__device__ void flush_acc(const TilePass &P, Real *acc, int wps, double *rho_g, int b, int G) {
    __syncthreads();
    for (int x = threadIdx.x; x < P.n_ops * 4; x += blockDim.x) {
        const int u = x >> 2;
        if (!((P.param_mask >> u) & 1ull)) continue;
        // kSingle: one sum per op in all lanes, stored as the component of
        // its fmode; otherwise lane q holds component q & 3.
        const int c = kSingle ? (P.fmode[u] == 1 ? 3 : (P.fmode[u] == 2 ? 2 : 0)) : (x & 3);
        if (kSingle && (x & 3)) continue;
        double k = 0.0;
        for (int w = 0; w < wps; ++w)
            for (int q = kSingle ? 0 : c; q < 32; q += kSingle ? 1 : 4) {
                Real &r = acc[(u * wps + w) * 32 + q];
                k += (double)r;
                r = 0;
            }
        if (k == 0.0) continue;
        // i K = [[i k0, (k3 + i k2) / 2], [(-k3 + i k2) / 2, i k1]]
        double *dst = rho_g + ((size_t)b * G + P.grp[u]) * 8;
        if (c == 0) {
            atomicAdd(dst + 1, k);
        } else if (c == 1) {
            atomicAdd(dst + 7, k);
        } else if (c == 2) {
            atomicAdd(dst + 3, 0.5 * k);
            atomicAdd(dst + 5, 0.5 * k);
        } else {
            atomicAdd(dst + 2, 0.5 * k);
            atomicAdd(dst + 4, -0.5 * k);
        }
    }
    __syncthreads();
}

// One reverse pass: un-applies the pass on psi and lambda tiles and sums the
// reduced matrices of its parametrised groups (as i K) into
// rho_g[slot][group][8].  The sums run in the state's precision over one
// warp and at most 64 tiles, then in FP64.
template <typename Real, int R, bool kSingle, bool kReal, int NB = 2>
__device__ __forceinline__ void tile_rev_body(const TilePass &P, int n, int n_slots,
                                              const typename CT<Real>::T *mats, int G,
                                              const typename CT<Real>::T *psi_src,
                                              typename CT<Real>::T *psi, typename CT<Real>::T *lam,
                                              double *rho_g, int64_t t0, int64_t t_end,
                                              unsigned char *smem, bool write_psi = true) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    constexpr int kFlushTiles = 64;
    const int tid = threadIdx.x, T = blockDim.x, t = P.t, S = P.n_stages;
    const int lane = tid & 31, wps = T >> 5;
    const uint32_t tbytes = (uint32_t)sizeof(C) << t;
    // NB tile buffers (2: the next tile's copy overlaps this one's stages;
    // 1: more blocks per SM, the copy after the tile is written back)
    uint2 *tb = reinterpret_cast<uint2 *>(smem + 2 * NB * tbytes);
    uint4 *rec = reinterpret_cast<uint4 *>(smem + 2 * NB * tbytes + (uint32_t)S * T * 8u);
    C *sm = reinterpret_cast<C *>(rec + 2 * S);
    Real *acc = reinterpret_cast<Real *>(sm + 4 * P.n_ops);
    build_stage_recs(P, rec);
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
    for (int x = tid; x < P.n_ops * wps * 32; x += T) acc[x] = 0;
    Real *accw = acc + (tid >> 5) * 32 + lane;  // [op][warp][lane]: sum k_(lane & 3)
    uint32_t gk[R], pk[R], nk[R];
    const uint32_t g0 = bit_vectors<R>(P.gl, t, tid, gk);
    const uint32_t p0 = bit_vectors<R>(P.ldperm, t, tid, pk);
    const uint32_t n0 = bit_vectors<R>(P.nat, t, tid, nk);
    const uint32_t sh = (uint32_t)__cvta_generic_to_shared(smem);
    if (t0 >= t_end) return;
    // psi tile of buffer j at [j tbytes], lambda tile at [(NB + j) tbytes]
    auto fetch = [&](const TileCursor &c, int buf) {
        const int64_t off = ((int64_t)c.slot << n) + c.base;
        const C *sp = psi_src + off, *sl = lam + off;
        const uint32_t dp = sh + (uint32_t)buf * tbytes, dl = dp + NB * tbytes;
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
        const int buf = NB == 2 ? (int)(i & 1) : 0;
        if (cur.slot != mslot || since == kFlushTiles) {
            if (mslot >= 0) flush_acc<Real, kSingle>(P, acc, wps, rho_g, mslot, G);
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
            __syncthreads();
            for (int u = tid; u < P.n_ops; u += T)
                if ((P.real_mask >> u) & 1ull) stage_shears(sm + 4 * u);
            if constexpr (std::is_same<C, float2>::value && kSingle == kReal) {
                __syncthreads();  // the branch-free paths' stage flags
                set_stage_flags(P, rec, sm);
            }
            mslot = cur.slot;
        }
        cp_async_wait_all();
        __syncthreads();
        if (NB == 2 && tix + 1 < t_end) fetch(nxt, buf ^ 1);
        unsigned char *tp = smem + (uint32_t)buf * tbytes, *tl = tp + NB * tbytes;
        for (int s = S - 1; s >= 0; --s) {
            const uint2 bb = tb[s * T + tid];
            uint32_t lq[R], sq[R];
            const uint32_t ops = read_stage_rec<R>(rec, s, lq, sq);
            const uint32_t modes = kSingle ? rec[2 * s + 1].y : 0u;
            C a[NA], al[NA];
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                const uint32_t ad = bb.y ^ xsel<R>(r, sq);
                a[r] = *reinterpret_cast<const C *>(tp + ad);
                al[r] = *reinterpret_cast<const C *>(tl + ad);
            }
            // the stage's sums: over lane quads in registers, then per lane
            // into the warp's accumulators
            constexpr int NV = kSingle ? 4 : (4 * R <= 8 ? 8 : 16);
            Real kk[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) kk[v] = 0;
            if constexpr (kSingle && kReal && std::is_same<C, float2>::value) {
                stage_ops_rev<C, Real, R, NV, kReal>(ops, modes, (rec[2 * s + 1].w >> 4) & 15u, sm, a,
                                                     al, kk);
            } else if constexpr (!kSingle && !kReal && std::is_same<C, float2>::value) {
                stage_ops_rev4<C, Real, R, NV, kReal>(ops, modes, (rec[2 * s + 1].w >> 12) & 15u, sm,
                                                      a, al, kk);
            } else {
                tile_ops_rev<C, Real, R, R - 1, NV, kSingle, kReal>(ops, modes, sm, a, al, kk);
            }
            warp_reduce_quad<Real, NV>(kk, lane);
            if constexpr (kSingle) {  // lane: the sum of register bit lane & 3
                const int m = lane & 3;
                const uint32_t ob = m < R ? (ops >> (8 * m)) & 0xffu : 0u;
                if (ob & 128u) accw[((int)(ob & 63u) - 1) * wps * 32] += kk[0];
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const uint32_t ob = (ops >> (8 * m)) & 0xffu;
                    if (ob & 128u) accw[((int)(ob & 63u) - 1) * wps * 32] += kk[m];
                }
            }
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
        if (write_psi) {
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const uint32_t so = p0 ^ xsel<R>(k, pk), go = g0 ^ xsel<R>(k, gk);
                dp[go] = *reinterpret_cast<const C *>(tp + so);
                dl[go] = *reinterpret_cast<const C *>(tl + so);
            }
        } else {  // the next reverse pass restarts psi from a stored state
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const uint32_t so = p0 ^ xsel<R>(k, pk), go = g0 ^ xsel<R>(k, gk);
                dl[go] = *reinterpret_cast<const C *>(tl + so);
            }
        }
        ++since;
        if (NB == 1 && tix + 1 < t_end) {
            __syncthreads();  // every thread has read its part of the tile
            fetch(nxt, 0);
        }
        cur = nxt;
        nxt = tile_next(P, nxt);
    }
    flush_acc<Real, kSingle>(P, acc, wps, rho_g, mslot, G);
}

// NB = 1: launched with 64 threads only (at least five blocks per SM).
template <typename Real, int R, bool kSingle, bool kReal, int NB = 2>
__global__ void __launch_bounds__(NB == 1 ? 64 : 256, NB == 1 ? 5 : (R >= 4 ? 1 : 2))
k_tile_rev(const __grid_constant__ TilePass P, int n, int n_slots,
           const typename CT<Real>::T *mats, int G, const typename CT<Real>::T *psi_src,
           typename CT<Real>::T *psi, typename CT<Real>::T *lam, double *rho_g, int write_psi) {
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t t0, t_end;
    block_range((int64_t)n_slots << P.n_tile_bits, gridDim.x, blockIdx.x, t0, t_end);
    tile_rev_body<Real, R, kSingle, kReal, NB>(P, n, n_slots, mats, G, psi_src, psi, lam, rho_g,
                                               t0, t_end, smem, write_psi != 0);
}

// Sum of v over the block (every thread gets it); red: one double per warp.
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

// ------------------------------------- several problems, one persistent launch
//
// The forward (or reverse) sweeps of several problems of any qubit count and
// depth (one tile shape) run as one launch of resident blocks.  Each pass of
// each problem is a task cut into chunks of tiles; the chunks of all tasks
// form one ticket sequence, level by level (pass 0 of every problem, then
// pass 1, ...).  A block takes the next ticket, waits until the task its
// chunk depends on (the same problem's previous pass) has completed all of
// its chunks, runs the chunk with the ordinary pass body and counts it done.
// Every ticket before a waited-on chunk was taken by a running block, so the
// wait always ends; it is bounded anyway (kSweepWaitNs of wall time), after
// which the block records SV_DEVERR_SWEEP_WAIT and stops.

constexpr unsigned long long kSweepWaitNs = 20ull * 1000 * 1000 * 1000;  // 20 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename Real, int R, bool kRev>
__global__ void __launch_bounds__(256, (R >= 4 && kRev) ? 1 : 2)
k_tile_sweep(const SweepTask *tasks, int n_tasks, long long n_tickets,
             unsigned long long *ticket, unsigned int *done, int *err) {
    using C = typename CT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_tk;
    __shared__ int s_task, s_fail;
    TilePass &P = *reinterpret_cast<TilePass *>(smem);
    unsigned char *rest = smem + ((sizeof(TilePass) + 255) & ~size_t(255));
    int hint = 0, cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long tk = (long long)atomicAdd(ticket, 1ull);
            int j = hint;
            if (tk < n_tickets)
                while (j + 1 < n_tasks && tasks[j + 1].chunk_begin <= tk) ++j;
            s_tk = tk;
            s_task = j;
            s_fail = 0;
            if (tk < n_tickets && tasks[j].dep >= 0) {
                const SweepTask &d = tasks[tasks[j].dep];
                const unsigned int need = (unsigned int)d.n_chunks;
                unsigned long long t_start = 0;
                while (ld_acquire(done + tasks[j].dep) < need) {
                    const unsigned long long now = global_ns();
                    if (!t_start) t_start = now;
                    if (now - t_start > kSweepWaitNs) {
                        s_fail = 1;
                        if (err) atomicCAS(err, 0, SV_DEVERR_SWEEP_WAIT);
                        break;
                    }
                    __nanosleep(256);
                }
            }
        }
        __syncthreads();
        const long long tk = s_tk;
        const int j = s_task;
        if (tk >= n_tickets || s_fail) break;
        hint = j;
        const SweepTask T = tasks[j];
        // every thread acquires the dependency's writes for its own loads
        if (T.dep >= 0) (void)ld_acquire(done + T.dep);
        if (j != cur) {  // this pass's descriptor into shared memory
            const uint32_t *src = reinterpret_cast<const uint32_t *>(T.P);
            uint32_t *dst = reinterpret_cast<uint32_t *>(smem);
            for (int i = threadIdx.x; i < (int)(sizeof(TilePass) / 4); i += blockDim.x) dst[i] = src[i];
            cur = j;
        }
        __syncthreads();
        const long long c = tk - T.chunk_begin;
        const int64_t t0 = c * (int64_t)T.chunk_tiles;
        const int64_t t1 = min(T.tiles, t0 + (int64_t)T.chunk_tiles);
        if constexpr (kRev)
            tile_rev_body<Real, R, false, false>(P, T.n, T.n_slots, (const C *)T.mats, T.G,
                                                 (const C *)T.psi, (C *)T.psi, (C *)T.lam, T.rho,
                                                 t0, t1, rest);
        else
            tile_fwd_body<Real, R, false>(P, T.n, T.n_slots, (const C *)T.mats, T.G,
                                          (const C *)T.psi, (C *)T.psi, t0, t1, rest);
        __syncthreads();  // every store of the chunk issued
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + j, 1u);
        }
    }
}

// ------------------------------------------------------ H over tile passes

// Tile walk of an H pass (the same counting as TileCursor).
__device__ __forceinline__ TileCursor h_cursor(const HPass &P, int64_t tix) {
    TileCursor c;
    c.slot = (int)(tix >> P.n_tile_bits);
    c.local = (uint32_t)(tix & ((int64_t(1) << P.n_tile_bits) - 1));
    c.base = 0;
    for (int k = 0; k < P.n_tile_bits; ++k)
        if ((c.local >> k) & 1u) c.base ^= P.gpre[k] ^ (k ? P.gpre[k - 1] : 0u);
    return c;
}

__device__ __forceinline__ TileCursor h_next(const HPass &P, TileCursor c) {
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

// Per-tile record of one class of terms: its coefficient sum_t c_t i^phase_t
// times the term's sign on the tile's non-local bits and the class's sign
// on the group's flip bits, and its Z mask on the thread bits.
template <typename Real> struct HCoef {
    uint32_t zt, pad;
    Real re, im;
};

// One H pass: for the pass's X-mask groups g,
//   lambda_j (+)= sum_g D_g(j ^ x_g) psi_(j ^ x_g),
//   D_g(k) = sum_(t in g) c_t i^phase_t (-1)^|k & z_t|,
// and E[slot] += sum_j Re(conj(psi_j) lambda_j) over this pass's part of
// lambda.  psi tiles arrive by cp.async (double-buffered) in natural order;
// the thread's amplitudes are j = tid + k 2^(t-R).  A group whose classes
// put no Z on a register bit takes one value per thread (its signed class
// coefficients summed).  The others read D_g at the thread's 2^R amplitudes
// from a per-tile table: one row of 2^R values per distinct Z mask on the
// thread bits (the row's class coefficients times their register-bit signs,
// built once per tile by the whole block), each row added with the sign of
// its thread-bit mask.  Products in the state's precision, sums over the
// block's amplitudes in FP64.  kLam = false: energies only.
template <typename Real, int R, bool kLam, bool kRealH>
__global__ void __launch_bounds__(256)
k_tile_h(const __grid_constant__ HPass P, int n, int n_slots, const typename CT<Real>::T *psi,
         typename CT<Real>::T *lam, double *E) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    static_assert(R <= kHRegBitsMax, "H kernel register bits");
    extern __shared__ __align__(16) unsigned char smem[];
    // 256 threads whenever R >= 3 (tiles of 2^11 and 2^12 amplitudes)
    const int tid = threadIdx.x, T = R >= 3 ? 256 : (int)blockDim.x, t = P.t;
    const uint32_t tbytes = (uint32_t)sizeof(C) << t;
    // psi tiles at [0, 2 tbytes), the lambda tile being added to at [2 tbytes,
    // 3 tbytes), then this tile's row table (NA values per row, real parts,
    // then imaginary parts unless kRealH)
    constexpr int kRowVals = kRealH ? NA : 2 * NA;
    Real *etab = reinterpret_cast<Real *>(smem + 3 * tbytes);
    HGroup *grp = reinterpret_cast<HGroup *>(etab + P.n_rows * kRowVals);
    HCoef<Real> *coef = reinterpret_cast<HCoef<Real> *>(grp + P.n_groups);
    HTerm *trm = reinterpret_cast<HTerm *>(coef + P.n_classes);
    HClass *cls = reinterpret_cast<HClass *>(trm + P.n_terms);
    HRow *rows = reinterpret_cast<HRow *>(cls + P.n_classes);
    double *red = reinterpret_cast<double *>(rows + P.n_rows);
    for (int i = tid; i < P.n_terms; i += T) trm[i] = P.terms[i];
    for (int i = tid; i < P.n_groups; i += T) grp[i] = P.groups[i];
    for (int i = tid; i < P.n_classes; i += T) cls[i] = P.classes[i];
    for (int i = tid; i < P.n_rows; i += T) rows[i] = P.rows[i];
    __syncthreads();
    const bool add = kLam && !P.first;
    uint32_t gk[R];
    const uint32_t g0 = bit_vectors<R>(P.gl, t, tid, gk);
    const uint32_t sh = (uint32_t)__cvta_generic_to_shared(smem);
    const int64_t tiles = (int64_t)n_slots << P.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = per * blockIdx.x, t_end = min(tiles, t0 + per);
    if (t0 >= t_end) return;
    auto fetch = [&](const TileCursor &c, int buf) {
        const C *src = psi + ((int64_t)c.slot << n) + c.base;
        const uint32_t d = sh + (uint32_t)buf * tbytes;
#pragma unroll
        for (int k = 0; k < NA; ++k)
            cp_async_amp(d + (uint32_t)(tid + k * T) * (uint32_t)sizeof(C), src + (g0 ^ xsel<R>(k, gk)));
        cp_async_commit();
    };
    TileCursor cur = h_cursor(P, t0);
    fetch(cur, 0);
    TileCursor nxt = h_next(P, cur);
    double e_acc = 0.0;
    int eslot = cur.slot;
    for (int64_t tix = t0, i = 0; tix < t_end; ++tix, ++i) {
        const int buf = (int)(i & 1);
        if (cur.slot != eslot) {  // the slot's energy so far
            const double s = block_sum(e_acc, red);
            if (tid == 0) atomicAdd(&E[eslot], s);
            e_acc = 0.0;
            eslot = cur.slot;
        }
        for (int c = tid; c < P.n_classes; c += T) {  // this tile's class records
            const HClass cl = cls[c];
            Real re = 0, im = 0;
            for (int ti = cl.t_begin; ti < cl.t_end; ++ti) {
                const HTerm tm = trm[ti];
                const Real v =
                    (__popc((cur.base ^ cl.xnl) & tm.z) & 1u) ? (Real)-tm.coeff : (Real)tm.coeff;
                if (tm.phase == 0) re += v;
                else if (tm.phase == 1) im += v;
                else if (tm.phase == 2) re -= v;
                else im -= v;
            }
            if (__popc(cl.xl & cl.zl) & 1u) {
                re = -re;
                im = -im;
            }
            HCoef<Real> h;
            h.zt = cl.zl & (uint32_t)(T - 1);
            h.pad = 0;
            h.re = re;
            h.im = im;
            coef[c] = h;
        }
        if (P.n_rows) {  // the row table: E[k] = sum_c coef_c (-1)^|k & kz_c|
            __syncthreads();
            for (int x = tid; x < P.n_rows * NA; x += T) {
                const HRow rw = rows[x / NA];
                const int k = x & (NA - 1);
                Real er = 0, ei = 0;
                for (int c = rw.c_begin; c < rw.c_end; ++c) {
                    const bool neg = __popc((uint32_t)k & (cls[c].zl >> (t - R))) & 1u;
                    er += neg ? -coef[c].re : coef[c].re;
                    if constexpr (!kRealH) ei += neg ? -coef[c].im : coef[c].im;
                }
                Real *e = etab + (x / NA) * kRowVals;
                e[k] = er;
                if constexpr (!kRealH) e[NA + k] = ei;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        C *L = lam + ((int64_t)cur.slot << n) + cur.base;
        C *lt = reinterpret_cast<C *>(smem + 2 * tbytes);
        if (add) {  // this tile's lambda so far, in flight during the sums
            const uint32_t d = sh + 2 * tbytes;
#pragma unroll
            for (int k = 0; k < NA; ++k)
                cp_async_amp(d + (uint32_t)(tid + k * T) * (uint32_t)sizeof(C), L + (g0 ^ xsel<R>(k, gk)));
            cp_async_commit();
        }
        if (tix + 1 < t_end) fetch(nxt, buf ^ 1);
        else cp_async_commit();  // keeps "all but the newest group" meaning the lambda tile
        const C *tile = reinterpret_cast<const C *>(smem + (uint32_t)buf * tbytes);
        const C *Sg = psi + ((int64_t)cur.slot << n);
        // lambda_k = acc[k] (real part .x, imaginary part .y)
        C acc[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k].x = acc[k].y = 0;
        auto add_real = [&](int k, Real d, const C &pk) {
            acc[k].x = fmaR(d, pk.x, acc[k].x);
            acc[k].y = fmaR(d, pk.y, acc[k].y);
        };
        // byte offset in shared memory of partner j ^ x (j = tid + k T) is
        // gb ^ (k T sizeof(C)): thread and register bits are disjoint, and
        // the buffer offset is above every in-tile offset
        const uint32_t bufb = (uint32_t)buf * tbytes;
        for (int g = 0; g < P.n_groups; ++g) {
            const HGroup &gr = grp[g];
            const uint32_t xl = gr.xl, xfar = gr.xfar, kact = gr.kact;
            const uint32_t gb = ((uint32_t)(tid ^ (int)xl) * (uint32_t)sizeof(C)) ^ bufb;
            auto partner = [&](int k) -> C {
                return xfar ? Sg[(cur.base ^ g0 ^ xsel<R>(k, gk)) ^ xfar]
                            : *reinterpret_cast<const C *>(
                                  smem + (gb ^ ((uint32_t)(k * T) * (uint32_t)sizeof(C))));
            };
            if (kact == 0) {
                // no class has a Z on a register bit: one value per thread
                Real vr = 0, vi = 0;
                for (int c = gr.c_begin; c < gr.c_end; ++c) {
                    const HCoef<Real> h = coef[c];
                    const bool nt = __popc((uint32_t)tid & h.zt) & 1u;
                    vr += nt ? -h.re : h.re;
                    if constexpr (!kRealH) vi += nt ? -h.im : h.im;
                }
                if constexpr (kRealH && std::is_same<C, float2>::value) {
                    // one packed FP32-pair FMA per amplitude
                    const uint64_t d2 = f2pack(vr, vr);
#pragma unroll
                    for (int k = 0; k < NA; ++k) acc[k] = f2unpack(f2fma(d2, f2of(partner(k)), f2of(acc[k])));
                } else {
#pragma unroll
                    for (int k = 0; k < NA; ++k) {
                        const C pk = partner(k);
                        if constexpr (kRealH) {
                            add_real(k, vr, pk);
                        } else {
                            acc[k].x = fmaR(vr, pk.x, fmaR(-vi, pk.y, acc[k].x));
                            acc[k].y = fmaR(vr, pk.y, fmaR(vi, pk.x, acc[k].y));
                        }
                    }
                }
                continue;
            }
            // D(tid, k) = sum over the group's rows of (-1)^|tid & zt| E_row[k]
            Real vr[NA], vi[NA];
#pragma unroll
            for (int k = 0; k < NA; ++k) vr[k] = vi[k] = 0;
            for (int r = gr.r_begin; r < gr.r_end; ++r) {
                const Real sg = (__popc((uint32_t)tid & rows[r].zt) & 1u) ? (Real)-1 : (Real)1;
                const Real *e = etab + r * kRowVals;
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    vr[k] = fmaR(sg, e[k], vr[k]);
                    if constexpr (!kRealH) vi[k] = fmaR(sg, e[NA + k], vi[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const C pk = partner(k);
                if constexpr (kRealH) {
                    add_real(k, vr[k], pk);
                } else {
                    acc[k].x = fmaR(vr[k], pk.x, fmaR(-vi[k], pk.y, acc[k].x));
                    acc[k].y = fmaR(vr[k], pk.y, fmaR(vi[k], pk.x, acc[k].y));
                }
            }
        }
        if (add) cp_async_wait_prior();  // own copies of the lambda tile have landed
        Real part = 0;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const C pj = tile[tid + k * T];
            part = fmaR(pj.x, acc[k].x, fmaR(pj.y, acc[k].y, part));
            if constexpr (kLam) {
                const uint32_t go = g0 ^ xsel<R>(k, gk);
                C out = acc[k];
                if (add) {  // each thread reads back only its own copies
                    const C old = lt[tid + k * T];
                    out.x += old.x;
                    out.y += old.y;
                }
                L[go] = out;
            }
        }
        e_acc += (double)part;
        __syncthreads();  // coef and this buffer are rewritten next
        cur = nxt;
        nxt = h_next(P, nxt);
    }
    const double s = block_sum(e_acc, red);
    if (tid == 0) atomicAdd(&E[eslot], s);
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

// Data-driven circuit learning (Sec. 4.2, Eq. 3): with Q(b) = |psi_b|^2 and
// the target P, M = (P + Q)/2, adds JS = 1/2 sum_b (P log(P/M) + Q log(Q/M))
// to js[slot] and writes lambda_b = w_b psi_b with w_b = dJS/dQ(b) =
// 1/2 log(Q(b)/M(b)) (0 where Q(b) = 0), so that the reverse sweep with
// lambda gives dJS/dtheta.  Per amplitude the arithmetic is in the state's
// precision (FP32 for complex64, whose states carry FP32 rounding anyway;
// FP64 for complex128); the sums over amplitudes are FP64.  grid.y = slot.
template <typename Real>
__global__ void k_ddcl_lambda(int n, const typename CT<Real>::T *psi, const double *target,
                              typename CT<Real>::T *lam, double *js) {
    using C = typename CT<Real>::T;
    __shared__ double red[32];
    const int b = blockIdx.y;
    const C *S = psi + ((int64_t)b << n);
    C *Lm = lam + ((int64_t)b << n);
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x) {
        const C a = S[j];
        const Real q = fmaR(a.x, a.x, a.y * a.y), p = (Real)target[j];
        const Real m = (Real)0.5 * (p + q);
        Real w = 0, term = 0;
        if (p > (Real)0) term = p * log(p / m);
        if (q > (Real)0) {
            const Real l = log(q / m);
            term = fmaR(q, l, term);
            w = (Real)0.5 * l;
        }
        acc += (double)term;
        C out;
        out.x = w * a.x;
        out.y = w * a.y;
        Lm[j] = out;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&js[b], 0.5 * s);
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

// A kernel's dynamic shared-memory limit only ever grows (per device and
// kernel), so a launch sequence that ran once has every limit it needs.
// While a sequence is captured into a CUDA graph no attribute is changed: a
// launch that would need a larger limit fails instead.
thread_local bool t_capturing = false;
std::mutex g_smem_mu;
std::map<std::pair<int, const void *>, uint32_t> g_smem_limit;

template <typename K> cudaError_t allow_smem(K kernel, uint32_t bytes);

}  // namespace

cudaError_t allow_smem_attr(const void *kernel, uint32_t bytes) { return allow_smem(kernel, bytes); }

namespace {

template <typename K> cudaError_t allow_smem(K kernel, uint32_t bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_smem_mu);
    uint32_t &have = g_smem_limit[{dev, (const void *)kernel}];
    if (bytes <= have) return cudaSuccess;
    if (t_capturing) return cudaErrorInvalidValue;
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
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
    return 2u * (csz << P.t) + (uint32_t)P.n_stages * (T * 8u + 32u) + (uint32_t)P.n_ops * 4u * csz;
}

// Reverse passes with at least this many register stages run single-buffered.
constexpr int kOneBufStages = 6;

uint32_t tile_rev_smem(int c128, const TilePass &P, int bufs) {
    const uint32_t csz = c128 ? 16u : 8u, rsz = c128 ? 8u : 4u, T = 1u << (P.t - P.R);
    return 2u * (uint32_t)bufs * (csz << P.t) + (uint32_t)P.n_stages * (T * 8u + 32u) + (uint32_t)P.n_ops * 4u * csz +
           (uint32_t)P.n_ops * T * rsz;
}

cudaError_t launch_tile_fwd(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *states, int64_t max_blocks, cudaStream_t st,
                            const void *src) {
    const uint32_t smem = tile_fwd_smem(c128, P);
    const int threads = 1 << (P.t - P.R);
    if (!src) src = states;
    HBM_DISPATCH_R(c128, P.R, {
        using C = typename CT<Real>::T;
        auto k = pass_all_real(P) ? k_tile_fwd<Real, RR, true> : k_tile_fwd<Real, RR, false>;
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        const int blocks = fill_blocks(k, threads, smem, max_blocks);
        k<<<blocks, threads, smem, st>>>(P, n, n_slots, (const C *)mats, G, (const C *)src,
                                         (C *)states);
    });
    return cudaGetLastError();
}

cudaError_t launch_tile_rev(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *psi, void *lam, double *rho_g, int64_t max_blocks,
                            cudaStream_t st, const void *psi_src, bool write_psi) {
    // passes of many stages are arithmetic-bound: one tile buffer, more
    // blocks per SM (complex64 real single-sum passes, tiles of 2^10 at 16
    // amplitudes per thread: 64 threads)
    const bool one_buf = !c128 && P.R == 4 && P.t == 10 && P.all_single && pass_all_real(P) &&
                         P.n_stages >= kOneBufStages;
    const uint32_t smem = tile_rev_smem(c128, P, one_buf ? 1 : 2);
    const int threads = 1 << (P.t - P.R);
    HBM_DISPATCH_R(c128, P.R, {
        using C = typename CT<Real>::T;
        auto k = P.all_single ? (pass_all_real(P) ? k_tile_rev<Real, RR, true, true>
                                                  : k_tile_rev<Real, RR, true, false>)
                              : (pass_all_real(P) ? k_tile_rev<Real, RR, false, true>
                                                  : k_tile_rev<Real, RR, false, false>);
        if constexpr (std::is_same<Real, float>::value && RR == 4) {
            if (one_buf) k = k_tile_rev<Real, RR, true, true, 1>;
        }
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        const int blocks = fill_blocks(k, threads, smem, max_blocks);
        k<<<blocks, threads, smem, st>>>(P, n, n_slots, (const C *)mats, G,
                                         (const C *)(psi_src ? psi_src : psi), (C *)psi, (C *)lam,
                                         rho_g, write_psi ? 1 : 0);
    });
    return cudaGetLastError();
}

uint32_t tile_h_smem(int c128, const HPass &P) {
    const uint32_t csz = c128 ? 16u : 8u;
    const uint32_t row_vals = (1u << h_reg_bits(P.t)) * (P.real ? 1u : 2u);
    return 3u * (csz << P.t) + (uint32_t)P.n_rows * (row_vals * (csz / 2u) + (uint32_t)sizeof(HRow)) +
           (uint32_t)P.n_groups * (uint32_t)sizeof(HGroup) +
           (uint32_t)P.n_classes * (csz + 8u + (uint32_t)sizeof(HClass)) +
           (uint32_t)P.n_terms * (uint32_t)sizeof(HTerm) + 32u * 8u + 16u;
}

cudaError_t launch_tile_h(int c128, const HPass &P, int n, int n_slots, const void *psi, void *lam,
                          double *E, int64_t max_blocks, cudaStream_t st) {
    const uint32_t smem = tile_h_smem(c128, P);
    // 2^R amplitudes per thread (R = h_reg_bits(t), the planner's bucketing)
    const int R = h_reg_bits(P.t);
    const int threads = 1 << (P.t - R);
    if (P.t < 7 || P.t > 12 || P.R != R) return cudaErrorInvalidValue;
    auto go = [&](auto k, auto *psi_t, auto *lam_t) -> cudaError_t {
        cudaError_t e = allow_smem(k, smem);
        if (e != cudaSuccess) return e;
        const int blocks = fill_blocks(k, threads, smem, max_blocks);
        k<<<blocks, threads, smem, st>>>(P, n, n_slots, psi_t, lam_t, E);
        return cudaGetLastError();
    };
    auto pick2 = [&](auto rr, auto re) -> cudaError_t {
        constexpr int RR = decltype(rr)::value;
        constexpr bool RE = decltype(re)::value;
        if (c128) {
            if (lam) return go(k_tile_h<double, RR, true, RE>, (const double2 *)psi, (double2 *)lam);
            return go(k_tile_h<double, RR, false, RE>, (const double2 *)psi, (double2 *)nullptr);
        }
        if (lam) return go(k_tile_h<float, RR, true, RE>, (const float2 *)psi, (float2 *)lam);
        return go(k_tile_h<float, RR, false, RE>, (const float2 *)psi, (float2 *)nullptr);
    };
    auto pick = [&](auto rr) -> cudaError_t {
        if (P.real) return pick2(rr, std::true_type());
        return pick2(rr, std::false_type());
    };
    if (R == 4) return pick(std::integral_constant<int, 4>());
    if (R == 3) return pick(std::integral_constant<int, 3>());
    return pick(std::integral_constant<int, 2>());
}

void set_capturing(bool on) { t_capturing = on; }

uint32_t tile_sweep_smem(int c128, bool rev, const TilePass &P) {
    return (uint32_t)((sizeof(TilePass) + 255) & ~size_t(255)) +
           (rev ? tile_rev_smem(c128, P) : tile_fwd_smem(c128, P));
}

int tile_sweep_blocks_per_sm(int c128, int R, bool rev, uint32_t smem, int threads) {
    int per = 0;
    HBM_DISPATCH_R(c128, R, {
        cudaError_t e;
        if (rev) {
            auto k = k_tile_sweep<Real, RR, true>;
            e = allow_smem(k, smem);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem);
        } else {
            auto k = k_tile_sweep<Real, RR, false>;
            e = allow_smem(k, smem);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem);
        }
        if (e != cudaSuccess) return 0;
    });
    return per;
}

cudaError_t launch_tile_sweep(int c128, int R, bool rev, const SweepTask *tasks, int n_tasks,
                              long long n_tickets, unsigned long long *ticket, unsigned int *done,
                              int *err, int blocks, int threads, uint32_t smem, cudaStream_t st) {
    HBM_DISPATCH_R(c128, R, {
        if (rev) {
            auto k = k_tile_sweep<Real, RR, true>;
            cudaError_t e = allow_smem(k, smem);
            if (e != cudaSuccess) return e;
            k<<<blocks, threads, smem, st>>>(tasks, n_tasks, n_tickets, ticket, done, err);
        } else {
            auto k = k_tile_sweep<Real, RR, false>;
            cudaError_t e = allow_smem(k, smem);
            if (e != cudaSuccess) return e;
            k<<<blocks, threads, smem, st>>>(tasks, n_tasks, n_tickets, ticket, done, err);
        }
    });
    return cudaGetLastError();
}

static dim3 whole_state_grid(int n, int rows);

// The JS divergence of one state's output distribution from the target and
// its derivative table D[j] = dJS/dP_theta(j) = 1/2 log(P_theta(j) / M(j)),
// M = (P + P_theta) / 2 (0 where P_theta(j) = 0); per-amplitude arithmetic
// in Real, the sum in FP64 (js zeroed by the launcher).
template <typename Real>
__global__ void k_ddcl_diag(int n, const typename CT<Real>::T *psi, const double *target,
                            double *D, double *js) {
    using C = typename CT<Real>::T;
    __shared__ double red[32];
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x) {
        const C a = psi[j];
        const Real q = fmaR(a.x, a.x, a.y * a.y), p = (Real)target[j];
        const Real m = (Real)0.5 * (p + q);
        Real w = 0, term = 0;
        if (p > (Real)0) term = p * log(p / m);
        if (q > (Real)0) {
            const Real l = log(q / m);
            term = fmaR(q, l, term);
            w = (Real)0.5 * l;
        }
        acc += (double)term;
        D[j] = (double)w;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(js, 0.5 * s);
}

// out[r] = sum_j D[j] |psi_r(j)|^2 for n_rows states (grid.y = row; out
// zeroed by the launcher); products in Real, sums in FP64.
template <typename Real>
__global__ void k_diag_expect(int n, const typename CT<Real>::T *states, const double *D,
                              double *out) {
    using C = typename CT<Real>::T;
    __shared__ double red[32];
    const int r = blockIdx.y;
    const C *S = states + ((int64_t)r << n);
    const int64_t dim = int64_t(1) << n;
    double acc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x) {
        const C a = S[j];
        acc += (double)((Real)D[j] * fmaR(a.x, a.x, a.y * a.y));
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(&out[r], s);
}

// out[j] = in[j'] where j' moves bit b of j to bit who.q[b]: a table indexed
// by qubit values rewritten in a relabeled bit layout (who.q[b] = the qubit
// held by bit b).  Grid-stride, one entry per thread step.
struct QubitOfBit {
    int32_t q[30];
};
__global__ void k_relayout(int n, QubitOfBit who, const double *in, double *out) {
    const int64_t dim = int64_t(1) << n;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < dim;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t src = 0;
        for (int b = 0; b < n; ++b) src |= ((j >> b) & 1) << who.q[b];
        out[j] = in[src];
    }
}

cudaError_t launch_relayout(int n, const int32_t *qubit_of_bit, const double *in, double *out,
                            cudaStream_t st) {
    if (n < 1 || n > 30) return cudaErrorInvalidValue;
    QubitOfBit w{};
    for (int b = 0; b < n; ++b) w.q[b] = qubit_of_bit[b];
    const int64_t dim = int64_t(1) << n;
    const int64_t blocks = std::min<int64_t>((dim + 255) / 256, 152 * 16);
    k_relayout<<<(unsigned)blocks, 256, 0, st>>>(n, w, in, out);
    return cudaGetLastError();
}

cudaError_t launch_ddcl_diag(int c128, int n, const void *psi, const double *target, double *D,
                             double *js, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(js, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const dim3 g = whole_state_grid(n, 1);
    if (c128) k_ddcl_diag<double><<<g, 256, 0, st>>>(n, (const double2 *)psi, target, D, js);
    else k_ddcl_diag<float><<<g, 256, 0, st>>>(n, (const float2 *)psi, target, D, js);
    return cudaGetLastError();
}

cudaError_t launch_diag_expect(int c128, int n, int n_rows, const void *states, const double *D,
                               double *out, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * n_rows, st);
    if (e != cudaSuccess) return e;
    const dim3 g = whole_state_grid(n, n_rows);
    if (c128) k_diag_expect<double><<<g, 256, 0, st>>>(n, (const double2 *)states, D, out);
    else k_diag_expect<float><<<g, 256, 0, st>>>(n, (const float2 *)states, D, out);
    return cudaGetLastError();
}

cudaError_t launch_ddcl_lambda(int c128, int n, int n_rows, const void *psi, const double *target,
                               void *lam, double *js, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(js, 0, sizeof(double) * n_rows, st);
    if (e != cudaSuccess) return e;
    const dim3 g = whole_state_grid(n, n_rows);
    if (c128) k_ddcl_lambda<double><<<g, 256, 0, st>>>(n, (const double2 *)psi, target, (double2 *)lam, js);
    else k_ddcl_lambda<float><<<g, 256, 0, st>>>(n, (const float2 *)psi, target, (float2 *)lam, js);
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
