// Forward tile passes on the tensor cores.
//
// The register-stage forward pass (hbm.cu) applies, in every stage, the
// fused 2x2 group of each of the stage's four register bits with FP32 FMAs.
// Those four groups act on four different qubits, so together they are one
// dense 16 x 16 complex block: the Kronecker product of the four 2x2
// matrices (identity on a bit without a group).  This kernel applies that
// block with tcgen05.mma: the 16 amplitudes a thread gathers in a stage are
// one row of a real 128 x 32 matrix A (re, im interleaved), the block is a
// real 32 x 32 matrix B, and D = A B^T lands in tensor memory, one lane per
// thread, from where the thread reads its 16 new amplitudes and stores them
// through the stage's (CNOT-permuted) store addresses exactly as the
// register path does.  The plan, the tile walk and every address are the
// register path's; only the arithmetic moves to the tensor cores.
//
// Precision: kind::tf32 operands carry 11 significant bits, so every
// operand is split into hi (its top 11 bits, exactly a tf32 value) and lo =
// x - hi, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the "3xTF32" split,
// about 22 significant bits per product), accumulated in FP32 in tensor
// memory.  Complex64 states only.
//
// Operands sit in shared memory in the K-major 128-byte-swizzle layout:
// row r of 32 fp32 (128 bytes) at r * 128, its 16-byte chunk c stored at
// chunk position c ^ (r mod 8), 8-row groups 1024 bytes apart; one MMA
// instruction covers K = 8 (32 bytes), the next starts 32 bytes further.
//
// Waits: the one wait (MMA completion, an mbarrier) spins at most
// kWaitLimit times; on expiry the block records SV_DEVERR_MMA_WAIT in the
// caller's error word, stops working, waits once more (bounded) for the
// MMAs it issued, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include "engine.cuh"
#include "hbm.h"
#include "tile_common.cuh"

namespace svk {
namespace {

constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kOpBytes = 128u * 128u;  // one A operand: 128 rows x 128 bytes
constexpr uint32_t kBBytes = 32u * 128u;    // one B operand: 32 rows x 128 bytes

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One bounded test of the barrier's phase `parity`: true once it completed.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Spins at most `limit` times; false if the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy writes to shared memory made visible to the tensor cores.
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A B^T, kind::tf32, one CTA; acc = 0 overwrites D.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 32 consecutive 32-bit columns of the warp's 32 tensor-memory lanes: thread
// i of the warp gets lane (lane base + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the leading offset is unused in this layout).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3ffffu) >> 4);  // start address / 16, bits 0-13
    d |= (uint64_t)1 << 16;                    // leading byte offset / 16 (unused)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset / 16, bits 32-45
    d |= (uint64_t)1 << 46;                    // descriptor version, bits 46-47
    d |= (uint64_t)2 << 61;                    // layout: 128-byte swizzle, bits 61-63
    return d;
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands
// K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(uint32_t M, uint32_t N) {
    return (1u << 4)             // D format: F32
           | (2u << 7)           // A format: TF32
           | (2u << 10)          // B format: TF32
           | ((N >> 3) << 17)    // N / 8, bits 17-22
           | ((M >> 4) << 24);   // M / 16, bits 24-28
}

// Byte offset of element (row, k), k < 32, in the swizzled operand layout.
__device__ __forceinline__ uint32_t sw128_off(uint32_t row, uint32_t k) {
    return row * 128u + ((((k >> 2) ^ row) & 7u) << 4) + ((k & 3u) << 2);
}

// hi = the top 11 significant bits of x (a tf32 value), lo = x - hi (exact).
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Device error word: the first bounded wait that gave up in a launch.
__device__ __forceinline__ void record_device_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// One forward pass over every tile of every slot with the register stages
// applied as dense blocks.  Threads T = 2^(t - 4) = 128 or 256 (one or two
// 128-row MMA tiles); mats: [slots][G][4] complex64.
__global__ void __launch_bounds__(256, 1)
k_tile_fwd_tc(const __grid_constant__ TilePass P, int n, int n_slots, const float2 *mats, int G,
              const float2 *src_states, float2 *states, int *err) {
    constexpr int R = 4, NA = 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, T = blockDim.x, t = P.t, S = P.n_stages;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t tiles = (int64_t)n_slots << P.n_tile_bits;
    const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = per * blockIdx.x, t_end = min(tiles, t0 + per);
    if (t0 >= t_end) return;

    // shared memory (1024-aligned base): A_hi[MT], A_lo[MT], B_hi, B_lo,
    // two tile buffers, per-thread stage bases, stage records, the slot's
    // group matrices and the per-stage 4x4 Kronecker factors, the mbarrier
    // and the tensor-memory address
    const int MT = T >> 7;
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sb = smem_addr(base);
    const uint32_t o_alo = MT * kOpBytes, o_bhi = 2 * MT * kOpBytes, o_blo = o_bhi + kBBytes;
    const uint32_t o_tile = o_blo + kBBytes;
    const uint32_t tbytes = 8u << t;
    uint2 *tb = reinterpret_cast<uint2 *>(base + o_tile + 2 * tbytes);
    uint4 *rec = reinterpret_cast<uint4 *>(tb + (size_t)S * T);
    float2 *sm = reinterpret_cast<float2 *>(rec + 2 * S);
    float2 *kf = sm + 4 * P.n_ops;  // [S][2][16]: low pair (bits 0, 1), high pair (bits 2, 3)
    uint64_t *bar = reinterpret_cast<uint64_t *>(kf + 32 * S);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const uint32_t bar_a = smem_addr(bar);

    build_stage_recs(P, rec);
    for (int s = 0; s < S; ++s) {
        const TileStage &sg = P.st[s];
        uint32_t lb = 0, sbv = 0;
        for (int k = 0; k < t - R; ++k)
            if ((tid >> k) & 1) {
                lb ^= sg.ldt[k];
                sbv ^= sg.stt[k];
            }
        tb[s * T + tid] = make_uint2(lb, sbv);
    }
    if (tid == 0) {
        mbar_init(bar_a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t ncols = MT == 1 ? 32u : 64u;
    if (warp == 0) tmem_alloc(smem_addr(tslot), ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    uint32_t gk[R], pk[R], nk[R];
    const uint32_t g0 = bit_vectors<R>(P.gl, t, tid, gk);
    const uint32_t p0 = bit_vectors<R>(P.ldperm, t, tid, pk);
    const uint32_t n0 = bit_vectors<R>(P.nat, t, tid, nk);
    const uint32_t sh_tile = sb + o_tile;
    auto fetch = [&](const TileCursor &c, int buf) {
        const float2 *src = src_states + ((int64_t)c.slot << n) + c.base;
        const uint32_t d = sh_tile + (uint32_t)buf * tbytes;
#pragma unroll
        for (int k = 0; k < NA; ++k) cp_async_amp(d + (p0 ^ xsel<R>(k, pk)), src + (g0 ^ xsel<R>(k, gk)));
        cp_async_commit();
    };
    constexpr uint32_t idesc = tf32_idesc(128, 32);
    const int mt = tid >> 7, row = tid & 127;                // MMA tile and row of this thread
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32u * (uint32_t)mt;
    uint32_t phase = 0;
    bool failed = false;
    TileCursor cur = tile_cursor(P, t0);
    fetch(cur, 0);
    TileCursor nxt = tile_next(P, cur);
    int mslot = -1;
    for (int64_t tix = t0, i = 0; tix < t_end && !failed; ++tix, ++i) {
        const int buf = (int)(i & 1);
        if (cur.slot != mslot) {
            // the slot's group matrices, then per stage the Kronecker
            // factors of its register bits 0-1 and 2-3 (identity on a bit
            // without a group)
            for (int x = tid; x < 4 * P.n_ops; x += T)
                sm[x] = mats[((size_t)cur.slot * G + P.grp[x >> 2]) * 4 + (x & 3)];
            __syncthreads();
            for (int x = tid; x < 32 * S; x += T) {
                const int s = x >> 5, half = (x >> 4) & 1, e = x & 15;
                const int ao = e >> 2, bi = e & 3;  // 2-bit output / input index of the pair
                const uint32_t ops = rec[2 * s].x;
                float2 v = make_float2(1.f, 0.f);
                for (int j = 0; j < 2; ++j) {
                    const int bit = 2 * half + j;
                    const uint32_t ob = (ops >> (8 * bit)) & 0xffu;
                    const int o = (ao >> j) & 1, in = (bi >> j) & 1;
                    float2 m;
                    if (ob) m = sm[4 * ((int)(ob & 63u) - 1) + 2 * o + in];
                    else m = make_float2(o == in ? 1.f : 0.f, 0.f);
                    v = cmul(v, m);
                }
                kf[x] = v;
            }
            mslot = cur.slot;
        }
        cp_async_wait_all();
        __syncthreads();
        if (tix + 1 < t_end) fetch(nxt, buf ^ 1);
        unsigned char *tile = base + o_tile + (uint32_t)buf * tbytes;
        for (int s = 0; s < S; ++s) {
            const uint2 bb = tb[s * T + tid];
            uint32_t lq[R], sq[R];
            const uint32_t ops = read_stage_rec<R>(rec, s, lq, sq);
            float2 a[NA];
#pragma unroll
            for (int r = 0; r < NA; ++r) a[r] = *reinterpret_cast<const float2 *>(tile + (bb.x ^ xsel<R>(r, lq)));
            if (ops) {
                // B = the stage's block, real 32 x 32: B[2o + c][2i + c'] from
                // U[o][i] = K_high[o >> 2][i >> 2] K_low[o & 3][i & 3]
                for (int e = tid; e < 256; e += T) {
                    const int o = e >> 4, in = e & 15;
                    const float2 u = cmul(kf[32 * s + 16 + ((o >> 2) << 2) + (in >> 2)],
                                          kf[32 * s + ((o & 3) << 2) + (in & 3)]);
                    float h0, l0, h1, l1;
                    split_tf32(u.x, h0, l0);
                    split_tf32(u.y, h1, l1);
                    // row 2o (real part out): ( Re U, -Im U ) at k = 2i, 2i + 1
                    // row 2o + 1 (imaginary part out): ( Im U, Re U )
                    const uint32_t r0 = sw128_off(2 * o, 2 * in), r1 = sw128_off(2 * o + 1, 2 * in);
                    *reinterpret_cast<float2 *>(base + o_bhi + r0) = make_float2(h0, -h1);
                    *reinterpret_cast<float2 *>(base + o_bhi + r1) = make_float2(h1, h0);
                    *reinterpret_cast<float2 *>(base + o_blo + r0) = make_float2(l0, -l1);
                    *reinterpret_cast<float2 *>(base + o_blo + r1) = make_float2(l1, l0);
                }
                // A: this thread's row, 16 amplitudes as 32 reals, hi and lo
                unsigned char *ahi = base + (uint32_t)mt * kOpBytes;
                unsigned char *alo = base + o_alo + (uint32_t)mt * kOpBytes;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float4 h, l;
                    split_tf32(a[2 * c].x, h.x, l.x);
                    split_tf32(a[2 * c].y, h.y, l.y);
                    split_tf32(a[2 * c + 1].x, h.z, l.z);
                    split_tf32(a[2 * c + 1].y, h.w, l.w);
                    const uint32_t off = sw128_off((uint32_t)row, 4u * c);
                    *reinterpret_cast<float4 *>(ahi + off) = h;
                    *reinterpret_cast<float4 *>(alo + off) = l;
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    for (int m = 0; m < MT; ++m) {
                        const uint32_t d = tmem + 32u * (uint32_t)m;
                        const uint32_t ah = sb + (uint32_t)m * kOpBytes, al = sb + o_alo + (uint32_t)m * kOpBytes;
#pragma unroll
                        for (int kc = 0; kc < 4; ++kc) {
                            const uint32_t ko = 32u * kc;
                            mma_tf32(d, sw128_desc(ah + ko), sw128_desc(sb + o_bhi + ko), idesc, kc > 0);
                            mma_tf32(d, sw128_desc(ah + ko), sw128_desc(sb + o_blo + ko), idesc, 1);
                            mma_tf32(d, sw128_desc(al + ko), sw128_desc(sb + o_bhi + ko), idesc, 1);
                        }
                    }
                    mma_commit(bar_a);
                }
                bool ok = mbar_wait_bounded(bar_a, phase, kWaitLimit);
                if (!ok) record_device_error(err, SV_DEVERR_MMA_WAIT);
                phase ^= 1u;
                // one decision for the whole block: tcgen05.ld is warp-collective
                failed = __syncthreads_or(!ok) != 0;
                tc_fence_after();
                if (!failed) {
                    uint32_t v[32];
                    tmem_ld32(t_lane, v);
#pragma unroll
                    for (int r = 0; r < NA; ++r)
                        a[r] = make_float2(__uint_as_float(v[2 * r]), __uint_as_float(v[2 * r + 1]));
                }
                tc_fence_before();
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < NA; ++r) *reinterpret_cast<float2 *>(tile + (bb.y ^ xsel<R>(r, sq))) = a[r];
            __syncthreads();
            if (failed) break;
        }
        if (failed) break;
        float2 *dst = states + ((int64_t)cur.slot << n) + cur.base;
#pragma unroll
        for (int k = 0; k < NA; ++k)
            dst[g0 ^ xsel<R>(k, gk)] = *reinterpret_cast<const float2 *>(tile + (n0 ^ xsel<R>(k, nk)));
        cur = nxt;
        nxt = tile_next(P, nxt);
    }
    cp_async_wait_all();
    if (failed) mbar_wait_bounded(bar_a, phase ^ 1u, kWaitLimit);  // the MMAs still in flight
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tmem, ncols);
}

// A launch that only waits on an mbarrier nobody arrives on, `limit` times:
// the bounded-wait path end to end (records SV_DEVERR_MMA_WAIT and returns).
__global__ void k_wait_expiry(int *err, uint32_t limit) {
    __shared__ uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(b, 0, limit)) record_device_error(err, SV_DEVERR_MMA_WAIT);
}

}  // namespace

uint32_t tile_fwd_tc_smem(const TilePass &P) {
    const uint32_t T = 1u << (P.t - P.R), MT = T >> 7;
    return 1024u + 2u * MT * kOpBytes + 2u * kBBytes + 2u * (8u << P.t) +
           (uint32_t)P.n_stages * (T * 8u + 32u) + (uint32_t)P.n_ops * 4u * 8u +
           (uint32_t)P.n_stages * 32u * 8u + 16u;
}

bool tile_fwd_tc_supported(int c128, const TilePass &P) {
    return !c128 && P.R == 4 && (P.t == 11 || P.t == 12) && tile_fwd_tc_smem(P) <= 227u * 1024u;
}

cudaError_t launch_tile_fwd_tc(const TilePass &P, int n, int n_slots, const void *mats, int G,
                               void *states, int64_t max_blocks, cudaStream_t st, int *err,
                               const void *src) {
    if (!tile_fwd_tc_supported(0, P)) return cudaErrorInvalidValue;
    const uint32_t smem = tile_fwd_tc_smem(P);
    const int threads = 1 << (P.t - P.R);
    cudaError_t e = allow_smem_attr((const void *)k_tile_fwd_tc, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tile_fwd_tc, threads, smem) !=
            cudaSuccess ||
        per < 1)
        per = 1;
    int64_t blocks = (int64_t)sms * per;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    k_tile_fwd_tc<<<(unsigned)blocks, threads, smem, st>>>(P, n, n_slots, (const float2 *)mats, G,
                                                           (const float2 *)(src ? src : states),
                                                           (float2 *)states, err);
    return cudaGetLastError();
}

cudaError_t launch_wait_expiry(int *err, uint32_t limit, cudaStream_t st) {
    k_wait_expiry<<<1, 32, 0, st>>>(err, limit);
    return cudaGetLastError();
}

}  // namespace svk
