// Device helpers shared by the tile-pass kernels (register stages in
// hbm.cu, tensor-core blocks in tc.cu): asynchronous tile copies, the walk
// over (slot, tile) pairs, per-thread address vectors and the packed stage
// records of a pass descriptor.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "engine.cuh"

namespace svk {
namespace {

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
// Waits for all but the most recently committed group.
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

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

// Block blk's contiguous share [t0, t_end) of `tiles` (slot, tile) pairs.
__device__ __forceinline__ void block_range(int64_t tiles, int nblk, int blk, int64_t &t0,
                                            int64_t &t_end) {
    const int64_t per = (tiles + nblk - 1) / nblk;
    t0 = per * blk;
    t_end = min(tiles, t0 + per);
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

// Shared-memory record of one stage (32 bytes, read with warp-uniform
// addresses): word 0 holds one op byte per register bit, (u + 1) | real << 6
// | parametrised << 7 for pass-local op u (0: no op); word 1 + i holds
// ldq[i] | stq[i] << 16 (byte offsets, < 2^16 for every supported tile);
// word 5 holds the ops' fmode bytes.
__device__ __forceinline__ void build_stage_recs(const TilePass &P, uint4 *rec) {
    for (int s = threadIdx.x; s < P.n_stages; s += blockDim.x) {
        const TileStage &sg = P.st[s];
        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < P.R && i < 4; ++i) {
            const int u = sg.op[i];
            if (u >= 0) {
                const uint32_t ob = (uint32_t)(u + 1) | (((P.real_mask >> u) & 1ull) ? 64u : 0u) |
                                    (((P.param_mask >> u) & 1ull) ? 128u : 0u);
                w[0] |= ob << (8 * i);
            }
            w[1 + i] = sg.ldq[i] | (sg.stq[i] << 16);
            if (u >= 0) w[5] |= (uint32_t)(P.fmode[u] & 3) << (8 * i);
        }
        rec[2 * s] = make_uint4(w[0], w[1], w[2], w[3]);
        rec[2 * s + 1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

template <int R>
__device__ __forceinline__ uint32_t read_stage_rec(const uint4 *rec, int s, uint32_t (&lq)[R],
                                                   uint32_t (&sq)[R]) {
    static_assert(R <= 4, "stage records hold four register bits");
    const uint4 a = rec[2 * s];
    uint32_t w[4] = {a.y, a.z, a.w, 0u};
    if constexpr (R > 3) w[3] = rec[2 * s + 1].x;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        lq[j] = w[j] & 0xffffu;
        sq[j] = w[j] >> 16;
    }
    return a.x;
}

// The four entries of matrix u (32-byte aligned records) as two 16-byte loads.
__device__ __forceinline__ void load_mat(const float2 *sm, int u, float2 &m0, float2 &m1,
                                         float2 &m2, float2 &m3) {
    const float4 *p = reinterpret_cast<const float4 *>(sm) + 2 * u;
    const float4 x = p[0], y = p[1];
    m0 = make_float2(x.x, x.y);
    m1 = make_float2(x.z, x.w);
    m2 = make_float2(y.x, y.y);
    m3 = make_float2(y.z, y.w);
}
__device__ __forceinline__ void load_mat(const double2 *sm, int u, double2 &m0, double2 &m1,
                                         double2 &m2, double2 &m3) {
    m0 = sm[4 * u];
    m1 = sm[4 * u + 1];
    m2 = sm[4 * u + 2];
    m3 = sm[4 * u + 3];
}

// A real rotation [[c, -s], [s, c]] with c > 0 (|angle| < pi/2) as three
// shears: x += alpha y; y += beta x; x += alpha y, with alpha = -s / (1 + c)
// = -tan(angle / 2) and beta = s (both in [-1, 1]): three fused
// multiply-adds per amplitude pair and component instead of four.
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void rot3_bit(C (&a)[1 << R], const Real alpha, const Real beta) {
    if constexpr (std::is_same<C, float2>::value) {
        const uint64_t pa = f2pack(alpha, alpha), pb = f2pack(beta, beta);
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            uint64_t x = f2of(a[r]), y = f2of(a[r | (1 << I)]);
            x = f2fma(pa, y, x);
            y = f2fma(pb, x, y);
            x = f2fma(pa, y, x);
            a[r] = f2unpack(x);
            a[r | (1 << I)] = f2unpack(y);
        }
    } else {
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            C x = a[r], y = a[r | (1 << I)];
            x.x = fmaR(alpha, y.x, x.x);
            x.y = fmaR(alpha, y.y, x.y);
            y.x = fmaR(beta, x.x, y.x);
            y.y = fmaR(beta, x.y, y.y);
            x.x = fmaR(alpha, y.x, x.x);
            x.y = fmaR(alpha, y.y, x.y);
            a[r] = x;
            a[r | (1 << I)] = y;
        }
    }
}

// The imaginary parts of a staged real matrix are unused: for a real
// rotation with c > 0 they carry the shear form (m0.y = alpha, m1.y = beta,
// m2.y = 1); otherwise m2.y = 0.  Called once per staged matrix.
template <typename C>
__device__ __forceinline__ void stage_shears(C *m) {
    using Real = decltype(m[0].x);
    const Real c = m[0].x, s = m[2].x;
    const bool rot = m[3].x == c && m[1].x == -s && c > (Real)0;
    m[0].y = rot ? -s / ((Real)1 + c) : (Real)0;
    m[1].y = rot ? s : (Real)0;
    m[2].y = rot ? (Real)1 : (Real)0;
    m[3].y = (Real)0;
}

// The group ops of one stage (op bytes `ops`), register bits I..R-1 in order.
// kReal: every op of the pass has a real matrix (no complex path compiled).
template <typename C, int R, int I, bool kReal>
__device__ __forceinline__ void tile_ops_fwd(uint32_t ops, const C *sm, C (&a)[1 << R]) {
    if constexpr (I < R) {
        const uint32_t ob = (ops >> (8 * I)) & 0xffu;
        if (ob) {
            C m0, m1, m2, m3;
            load_mat(sm, (int)(ob & 63u) - 1, m0, m1, m2, m3);
            if (kReal || (ob & 64u)) {
                if (m2.y != 0)
                    rot3_bit<C, decltype(m0.x), R, I>(a, m0.y, m1.y);
                else
                    u1r_bit<C, decltype(m0.x), R, I>(a, m0.x, m1.x, m2.x, m3.x);
            } else {
                u1_bit<C, R, I>(a, m0, m1, m2, m3);
            }
        }
        tile_ops_fwd<C, R, I + 1, kReal>(ops, sm, a);
    }
}

// The forward stage ops when register bits 0..M-1 carry real rotations in
// shear form and the others carry no op (stage flags): the arithmetic of
// tile_ops_fwd without its per-op branches, so the compiler can overlap one
// op's dependent FMA chains with the next op's.
template <typename C, int R, int I, int M>
__device__ __forceinline__ void tile_ops_fwd_rot(uint32_t ops, const C *sm, C (&a)[1 << R]) {
    if constexpr (I < M) {
        C m0, m1, m2, m3;
        load_mat(sm, (int)((ops >> (8 * I)) & 63u) - 1, m0, m1, m2, m3);
        rot3_bit<C, decltype(m0.x), R, I>(a, m0.y, m1.y);
        tile_ops_fwd_rot<C, R, I + 1, M>(ops, sm, a);
    }
}

// The forward stage ops when register bits 0..M-1 carry complex matrices
// and the others carry no op (stage flags, bits 8-11): tile_ops_fwd's
// complex arithmetic without its per-op branches.
template <typename C, int R, int I, int M>
__device__ __forceinline__ void tile_ops_fwd_cplx(uint32_t ops, const C *sm, C (&a)[1 << R]) {
    if constexpr (I < M) {
        C m0, m1, m2, m3;
        load_mat(sm, (int)((ops >> (8 * I)) & 63u) - 1, m0, m1, m2, m3);
        u1_bit<C, R, I>(a, m0, m1, m2, m3);
        tile_ops_fwd_cplx<C, R, I + 1, M>(ops, sm, a);
    }
}

// Stage flags, the w word of a stage's second record, set for the staged
// matrices of the current slot.  Bits 0-3: M > 0 when register bits
// 0..M-1 carry ops with real matrices in shear form (rotations with c > 0)
// and the other bits none (the forward's branch-free path); bits 4-7: the
// same M when those ops are moreover parametrised with the single Ry sum
// (fmode 1; the reverse's); bits 8-11: M when register bits 0..M-1 carry
// ops with complex matrices and the other bits none; bits 12-15: that M
// when those complex ops are moreover all parametrised (the reverse's
// four-sum path); 0 otherwise.  Called by every thread once the slot's
// shear forms are in shared memory; visible after the next barrier.
template <typename C>
__device__ __forceinline__ void set_stage_flags(const TilePass &P, uint4 *rec, const C *sm) {
    for (int s = threadIdx.x; s < P.n_stages; s += blockDim.x) {
        const uint32_t ops = rec[2 * s].x, modes = rec[2 * s + 1].y;
        int m = 0, mc = 0;
        bool single = true, rot = true, cplx = true, cpar = true;
        for (int i = 0; i < P.R; ++i) {
            const uint32_t ob = (ops >> (8 * i)) & 0xffu;
            if (!ob) break;
            rot = rot && (ob & 64u) && sm[4 * ((int)(ob & 63u) - 1) + 2].y != 0;
            cplx = cplx && !(ob & 64u);
            if (rot) {
                single = single && (ob & 128u) && ((modes >> (8 * i)) & 3u) == 1u;
                m = i + 1;
            }
            if (cplx) {
                cpar = cpar && (ob & 128u);
                mc = i + 1;
            }
        }
        // the bits above M must carry no op
        if (m > 0 && m < 4 && (ops >> (8 * m)) != 0u) m = 0;
        if (mc > 0 && mc < 4 && (ops >> (8 * mc)) != 0u) mc = 0;
        rec[2 * s + 1].w = (uint32_t)m | (single ? (uint32_t)m << 4 : 0u) | ((uint32_t)mc << 8) |
                           (cpar ? (uint32_t)mc << 12 : 0u);
    }
}

// Every op of pass P has a real matrix.
__host__ __device__ inline bool pass_all_real(const TilePass &P) {
    const uint64_t all = P.n_ops >= 64 ? ~0ull : ((1ull << P.n_ops) - 1ull);
    return (P.real_mask & all) == all;
}

}  // namespace
}  // namespace svk
