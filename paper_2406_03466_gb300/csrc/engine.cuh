// Device engine shared by the on-chip kernels (onchip.cu) and the tile-pass
// kernels (hbm.cu): complex helpers, slot resolution, fused 2x2 group
// matrices, register-stage execution forwards and backwards, reductions and
// the <H> epilogues.  Everything is inline/template device code.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.h"

namespace svk {
namespace {

template <typename Real> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__device__ __forceinline__ float fmaR(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ void sincosR(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincosR(double a, double *s, double *c) { sincos(a, s, c); }
__device__ __forceinline__ float asinR(float x) { return asinf(x); }
__device__ __forceinline__ double asinR(double x) { return asin(x); }
__device__ __forceinline__ float acosR(float x) { return acosf(x); }
__device__ __forceinline__ double acosR(double x) { return acos(x); }

template <typename C> __device__ __forceinline__ C cmk(double re, double im) {
    C r;
    r.x = (decltype(r.x))re;
    r.y = (decltype(r.y))im;
    return r;
}
template <typename C> __device__ __forceinline__ C cmul(const C a, const C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(const C a, const C b) {
    C r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C cconj(const C a) {
    C r;
    r.x = a.x;
    r.y = -a.y;
    return r;
}
// Packed FP32 pairs (sm_100 and later): one instruction does the same
// IEEE operation on both halves of a 64-bit register pair, so complex64
// arithmetic written as pairs rounds exactly as the scalar form does.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ uint64_t f2of(const float2 v) { return f2pack(v.x, v.y); }
__device__ __forceinline__ float2 f2unpack(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// m*x + k*y with 4 fused operations per component.  (Scalar: in packed
// pairs the swapped operands (x.y, x.x) cost register moves, and the packed
// form measured slower on the complex tile passes.)
template <typename C>
__device__ __forceinline__ C mad2(const C m, const C x, const C k, const C y) {
    C r;
    r.x = fmaR(m.x, x.x, fmaR(-m.y, x.y, fmaR(k.x, y.x, -k.y * y.y)));
    r.y = fmaR(m.x, x.y, fmaR(m.y, x.x, fmaR(k.x, y.y, k.y * y.x)));
    return r;
}

// ------------------------------------------------------------------ slots

struct SlotInfo {
    int64_t ref;
    int32_t shift_param;
    int32_t instance;
    double shift;
    const double *theta;
    const double *x;
};

__device__ SlotInfo resolve(const SlotSource &s, int b) {
    b += s.slot_base;
    SlotInfo si;
    si.shift_param = -1;
    si.shift = 0.0;
    if (s.mode == SLOTS_EXPLICIT) {
        const sv_slot sl = s.slots[b];
        si.instance = b;
        si.ref = sl.ref;
        si.shift_param = sl.shift_param;
        si.shift = sl.shift;
        si.theta = s.theta + (int64_t)sl.theta_row * s.theta_stride;
        si.x = (s.inputs && sl.input_row >= 0) ? s.inputs + (int64_t)sl.input_row * s.input_stride
                                                : nullptr;
        return si;
    }
    const int I = s.n_instances;
    int inst = b;
    if (s.mode == SLOTS_PARAM_SHIFT && b >= I) {
        const int bb = b - I;
        const int k = bb / (2 * I), r = bb % (2 * I);
        inst = r % I;
        si.shift_param = k;
        si.shift = r < I ? 1.5707963267948966 : -1.5707963267948966;
    }
    si.instance = inst;
    si.ref = s.refs[inst];
    si.theta = s.theta;
    si.x = s.inputs ? s.inputs + (int64_t)inst * s.input_stride : nullptr;
    return si;
}

// ------------------------------------------------------- gate matrices

// exp(-i a P / 2) for P = X (0), Y (1), Z (2), row-major [m00 m01 m10 m11].
template <typename Real, typename C>
__device__ __forceinline__ void rotation(int axis, Real a, C g[4]) {
    Real s, c;
    sincosR(a * Real(0.5), &s, &c);
    if (axis == 0) {
        g[0] = cmk<C>(c, 0); g[1] = cmk<C>(0, -s); g[2] = cmk<C>(0, -s); g[3] = cmk<C>(c, 0);
    } else if (axis == 1) {
        g[0] = cmk<C>(c, 0); g[1] = cmk<C>(-s, 0); g[2] = cmk<C>(s, 0); g[3] = cmk<C>(c, 0);
    } else {
        g[0] = cmk<C>(c, -s); g[1] = cmk<C>(0, 0); g[2] = cmk<C>(0, 0); g[3] = cmk<C>(c, s);
    }
}

template <typename Real, typename C>
__device__ void member_matrix(const Member &m, const SlotInfo &si, C g[4]) {
    switch (m.kind) {
    case M_RX:
    case M_RY:
    case M_RZ: {
        double a = m.angle;
        if (m.param >= 0) a = si.theta[m.param] + (m.param == si.shift_param ? si.shift : 0.0);
        rotation<Real, C>(m.kind - M_RX, (Real)a, g);
        break;
    }
    case M_X:
        g[0] = cmk<C>(0, 0); g[1] = cmk<C>(1, 0); g[2] = cmk<C>(1, 0); g[3] = cmk<C>(0, 0);
        break;
    case M_H: {
        const double h = 0.70710678118654752440;
        g[0] = cmk<C>(h, 0); g[1] = cmk<C>(h, 0); g[2] = cmk<C>(h, 0); g[3] = cmk<C>(-h, 0);
        break;
    }
    case M_ENC_RY_ASIN: {
        const Real x = (Real)si.x[m.param];
        rotation<Real, C>(1, asinR(x), g);
        break;
    }
    default: {  // M_ENC_RZ_ACOS_SQ
        const Real x = (Real)si.x[m.param];
        rotation<Real, C>(2, acosR(x * x), g);
        break;
    }
    }
}

template <typename C> __device__ __forceinline__ void matmul2(const C A[4], const C B[4], C out[4]) {
    out[0] = cadd(cmul(A[0], B[0]), cmul(A[1], B[2]));
    out[1] = cadd(cmul(A[0], B[1]), cmul(A[1], B[3]));
    out[2] = cadd(cmul(A[2], B[0]), cmul(A[3], B[2]));
    out[3] = cadd(cmul(A[2], B[1]), cmul(A[3], B[3]));
}

// Fused matrix of group g for this slot: M = G_last ... G_first.
template <typename Real, typename C>
__device__ void group_matrix(const Program &p, int g, const SlotInfo &si, C *out) {
    const Group grp = p.groups[g];
    C M[4] = {cmk<C>(1, 0), cmk<C>(0, 0), cmk<C>(0, 0), cmk<C>(1, 0)};
    for (int m = grp.m_begin; m < grp.m_end; ++m) {
        C G[4], T[4];
        member_matrix<Real, C>(p.members[m], si, G);
        matmul2(G, M, T);
        M[0] = T[0]; M[1] = T[1]; M[2] = T[2]; M[3] = T[3];
    }
    out[0] = M[0]; out[1] = M[1]; out[2] = M[2]; out[3] = M[3];
}

// --------------------------------------------------- register operations

template <int R>
__device__ __forceinline__ uint32_t xsel(int r, const uint32_t (&v)[R]) {
    uint32_t a = 0;
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (r & (1 << i)) a ^= v[i];
    return a;
}

template <typename C, int R, int I>
__device__ __forceinline__ void u1_bit(C (&a)[1 << R], const C m0, const C m1, const C m2,
                                       const C m3) {
#pragma unroll
    for (int r = 0; r < (1 << R); ++r) {
        if (r & (1 << I)) continue;
        const C x = a[r], y = a[r | (1 << I)];
        a[r] = mad2(m0, x, m1, y);
        a[r | (1 << I)] = mad2(m2, x, m3, y);
    }
}

// Real 2x2 matrix [[m0, m1], [m2, m3]] on register bit I: 4 FMAs per amplitude.
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void u1r_bit(C (&a)[1 << R], const Real m0, const Real m1,
                                        const Real m2, const Real m3) {
    if constexpr (std::is_same<C, float2>::value) {
        const uint64_t p0 = f2pack(m0, m0), p1 = f2pack(m1, m1), p2 = f2pack(m2, m2),
                       p3 = f2pack(m3, m3);
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            const uint64_t x = f2of(a[r]), y = f2of(a[r | (1 << I)]);
            a[r] = f2unpack(f2fma(p0, x, f2mul(p1, y)));
            a[r | (1 << I)] = f2unpack(f2fma(p2, x, f2mul(p3, y)));
        }
    } else {
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) {
            if (r & (1 << I)) continue;
            const C x = a[r], y = a[r | (1 << I)];
            a[r].x = fmaR(m0, x.x, m1 * y.x);
            a[r].y = fmaR(m0, x.y, m1 * y.y);
            a[r | (1 << I)].x = fmaR(m2, x.x, m3 * y.x);
            a[r | (1 << I)].y = fmaR(m2, x.y, m3 * y.y);
        }
    }
}

template <typename C, int R>
__device__ __forceinline__ void u1_reg(C (&a)[1 << R], int i, const C m0, const C m1, const C m2,
                                       const C m3) {
    switch (i) {
    case 0: u1_bit<C, R, 0>(a, m0, m1, m2, m3); break;
    case 1: if constexpr (R > 1) u1_bit<C, R, 1>(a, m0, m1, m2, m3); break;
    case 2: if constexpr (R > 2) u1_bit<C, R, 2>(a, m0, m1, m2, m3); break;
    case 3: if constexpr (R > 3) u1_bit<C, R, 3>(a, m0, m1, m2, m3); break;
    case 4: if constexpr (R > 4) u1_bit<C, R, 4>(a, m0, m1, m2, m3); break;
    default: break;
    }
}

template <typename C, int R>
__device__ __forceinline__ void cz_regs(C (&a)[1 << R], uint32_t lg, const int (&qq)[R], int qa,
                                        int qb) {
#pragma unroll
    for (int r = 0; r < (1 << R); ++r) {
        uint32_t j = lg;
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (r & (1 << i)) j |= 1u << qq[i];
        if (((j >> qa) & 1u) && ((j >> qb) & 1u)) {
            a[r].x = -a[r].x;
            a[r].y = -a[r].y;
        }
    }
}

// Partial reduced matrix rho_ab = sum psi_a conj(lambda_b) over the register
// pairs of bit I, as [re00 im00 re01 im01 re10 im10 re11 im11].
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void rho_bit(const C (&a)[1 << R], const C (&l)[1 << R], Real rh[8]) {
#pragma unroll
    for (int r = 0; r < (1 << R); ++r) {
        if (r & (1 << I)) continue;
        const C p0 = a[r], p1 = a[r | (1 << I)], l0 = l[r], l1 = l[r | (1 << I)];
        rh[0] = fmaR(p0.x, l0.x, fmaR(p0.y, l0.y, rh[0]));
        rh[1] = fmaR(p0.y, l0.x, fmaR(-p0.x, l0.y, rh[1]));
        rh[2] = fmaR(p0.x, l1.x, fmaR(p0.y, l1.y, rh[2]));
        rh[3] = fmaR(p0.y, l1.x, fmaR(-p0.x, l1.y, rh[3]));
        rh[4] = fmaR(p1.x, l0.x, fmaR(p1.y, l0.y, rh[4]));
        rh[5] = fmaR(p1.y, l0.x, fmaR(-p1.x, l0.y, rh[5]));
        rh[6] = fmaR(p1.x, l1.x, fmaR(p1.y, l1.y, rh[6]));
        rh[7] = fmaR(p1.y, l1.x, fmaR(-p1.x, l1.y, rh[7]));
    }
}

template <typename C, typename Real, int R>
__device__ __forceinline__ void rho_reg(const C (&a)[1 << R], const C (&l)[1 << R], int i,
                                        Real rh[8]) {
    switch (i) {
    case 0: rho_bit<C, Real, R, 0>(a, l, rh); break;
    case 1: if constexpr (R > 1) rho_bit<C, Real, R, 1>(a, l, rh); break;
    case 2: if constexpr (R > 2) rho_bit<C, Real, R, 2>(a, l, rh); break;
    case 3: if constexpr (R > 3) rho_bit<C, Real, R, 3>(a, l, rh); break;
    case 4: if constexpr (R > 4) rho_bit<C, Real, R, 4>(a, l, rh); break;
    default: break;
    }
}

struct Bases {
    uint32_t lb, sb, lg;
};

__device__ __forceinline__ Bases stage_bases(const Stage *sg, int tid);

// Thread bases of stage s.  kMode 0: program in global memory (precomputed
// table when the plan has one); 1: program staged in shared memory, bases
// computed from the stage record; 2: table staged in shared memory.
template <int kMode>
__device__ __forceinline__ Bases bases_of(const Program &p, int s, int tid, int Ts) {
    if constexpr (kMode == 2) {
        const uint4 v = reinterpret_cast<const uint4 *>(p.tbase)[(size_t)s * Ts + tid];
        return Bases{v.x, v.y, v.z};
    } else if constexpr (kMode == 0) {
        if (p.tbase) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.tbase) + (size_t)s * Ts + tid);
            return Bases{v.x, v.y, v.z};
        }
    }
    return stage_bases(p.stages + s, tid);
}

__device__ __forceinline__ Bases stage_bases(const Stage *sg, int tid) {
    Bases b{0u, 0u, 0u};
    const int nt = sg->n_thr;
    for (int k = 0; k < nt; ++k) {
        if ((tid >> k) & 1) {
            b.lb ^= sg->ldt[k];
            b.sb ^= sg->stt[k];
            b.lg |= 1u << sg->tpos[k];
        }
    }
    return b;
}

// The ops of register bit I (sorted stages): compile-time register indices,
// no dispatch; real matrices take the half-cost path.
template <typename C, int R, int I>
__device__ __forceinline__ void bit_ops_fwd(const Program &p, const Stage *sg, const C *mats,
                                            C (&a)[1 << R]) {
    if constexpr (I < R) {
        const int e = sg->op_begin + sg->bit_begin[I + 1];
        for (int o = sg->op_begin + sg->bit_begin[I]; o < e; ++o) {
            const Op op = p.ops[o];
            const C *m = mats + 4 * op.group;
            if (p.groups[op.group].real)
                u1r_bit<C, decltype(m[0].x), R, I>(a, m[0].x, m[1].x, m[2].x, m[3].x);
            else
                u1_bit<C, R, I>(a, m[0], m[1], m[2], m[3]);
        }
        bit_ops_fwd<C, R, I + 1>(p, sg, mats, a);
    }
}

// bit_ops_fwd for a stage whose register bits each carry exactly one real
// group (sorted = 2): no loops or branches between the ops, so one op's FMA
// chains can overlap the next op's.
template <typename C, int R, int I>
__device__ __forceinline__ void bit_ops_fwd_one_real(const Program &p, const Stage *sg,
                                                     const C *mats, C (&a)[1 << R]) {
    if constexpr (I < R) {
        const C *m = mats + 4 * p.ops[sg->op_begin + sg->bit_begin[I]].group;
        u1r_bit<C, decltype(m[0].x), R, I>(a, m[0].x, m[1].x, m[2].x, m[3].x);
        bit_ops_fwd_one_real<C, R, I + 1>(p, sg, mats, a);
    }
}

template <typename C, int R>
__device__ __forceinline__ void apply_stage_ops(const Program &p, const Stage *sg, const C *mats,
                                                C (&a)[1 << R], uint32_t lg, const int (&qq)[R]) {
    if (sg->sorted == 2) {
        bit_ops_fwd_one_real<C, R, 0>(p, sg, mats, a);
        return;
    }
    if (sg->sorted) {
        bit_ops_fwd<C, R, 0>(p, sg, mats, a);
        return;
    }
    for (int o = sg->op_begin; o < sg->op_end; ++o) {
        const Op op = p.ops[o];
        if (op.kind == OP_U1) {
            const C *m = mats + 4 * op.group;
            u1_reg<C, R>(a, op.a, m[0], m[1], m[2], m[3]);
        } else {
            cz_regs<C, R>(a, lg, qq, op.a, op.b);
        }
    }
}

// Runs every stage; the final state is left in shared memory `st` (natural
// index order, swizzled).  Stage 0 builds |ref> in registers, or (ref < 0)
// loads the state already in `st`.
template <typename Real, int R, int kMode>
__device__ void forward_stages(const Program &p, typename CT<Real>::T *st,
                               const typename CT<Real>::T *mats, int tid, int64_t ref) {
    using C = typename CT<Real>::T;
    C a[1 << R];
    const int Ts = 1 << (p.n - R);
    Bases nxt = bases_of<kMode>(p, 0, tid, Ts);
    for (int s = 0; s < p.n_stages; ++s) {
        const Stage *sg = p.stages + s;
        const Bases bs = nxt;
        if (s + 1 < p.n_stages) nxt = bases_of<kMode>(p, s + 1, tid, Ts);
        uint32_t lq[R], sq[R];
        int qq[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            lq[i] = sg->ldq[i];
            sq[i] = sg->stq[i];
            qq[i] = sg->q[i];
        }
        if (s == 0 && ref >= 0) {
#pragma unroll
            for (int r = 0; r < (1 << R); ++r) {
                uint32_t j = bs.lg;
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (r & (1 << i)) j |= 1u << qq[i];
                a[r] = cmk<C>((int64_t)j == ref ? 1.0 : 0.0, 0.0);
            }
        } else {
#pragma unroll
            for (int r = 0; r < (1 << R); ++r) a[r] = st[bs.lb ^ xsel<R>(r, lq)];
        }
        apply_stage_ops<C, R>(p, sg, mats, a, bs.lg, qq);
        if (s > 0 || ref < 0) __syncthreads();
#pragma unroll
        for (int r = 0; r < (1 << R); ++r) st[bs.sb ^ xsel<R>(r, sq)] = a[r];
        __syncthreads();
    }
}

// Sum of v over the Ts threads of a slot; every thread of the slot gets it.
// `red` holds one double per warp of the block.  Called uniformly.
__device__ double slot_sum(double v, int Ts, double *red) {
    const int width = Ts < 32 ? Ts : 32;
    for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (Ts <= 32) return v;
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    const int wps = Ts >> 5, first = (threadIdx.x / Ts) * wps;
    double s = 0.0;
    for (int i = 0; i < wps; ++i) s += red[first + i];
    return s;
}

// Amplitude index vectors of this thread's 2^R amplitudes in natural order:
// j_k = tid + k * Ts.  Returns the swizzled base and per-bit vectors.
template <int R>
__device__ __forceinline__ uint32_t natural_vectors(int tid, int sh, int w, uint32_t (&v)[R]) {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = swizzle(1u << (sh + i), w);
    return swizzle((uint32_t)tid, w);
}

// sum_t c_t <psi|P_t|psi> over this thread's amplitudes (FP64 across terms).
template <typename Real, int R>
__device__ double expect_partial(const Observable &o, const typename CT<Real>::T *st, int tid,
                                 int sh, int w) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    uint32_t v[R];
    const uint32_t s0 = natural_vectors<R>(tid, sh, w, v);
    constexpr int kRun = 8;  // groups per FP32 run, as in expect_table
    double e = 0.0;
    Real run = 0;
    for (int g = 0; g < o.n_tgroups; ++g) {
        const TermGroup tg = o.tgroups[g];
        C wv[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t sj = s0 ^ xsel<R>(k, v);
            const C pj = st[sj], px = st[sj ^ tg.sx];
            // conj(psi_{j^x}) psi_j
            wv[k].x = fmaR(px.x, pj.x, px.y * pj.y);
            wv[k].y = fmaR(px.x, pj.y, -px.y * pj.x);
        }
        Real gacc = 0;
        for (int t = tg.t_begin; t < tg.t_end; ++t) {
            const Term tm = o.terms[t];
            const bool im = tm.phase & 1;
            const uint32_t p0 = __popc((uint32_t)tid & tm.z) & 1u;
            const uint32_t zh = tm.z >> sh;
            Real acc = 0;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const Real val = im ? wv[k].y : wv[k].x;
                const uint32_t par = p0 ^ (__popc((uint32_t)k & zh) & 1u);
                acc += par ? -val : val;
            }
            const Real c = (Real)((tm.phase == 1 || tm.phase == 2) ? -tm.coeff : tm.coeff);
            gacc = fmaR(c, acc, gacc);
        }
        run += gacc;
        if ((g + 1) % kRun == 0) {
            e += (double)run;
            run = 0;
        }
    }
    return e + (double)run;
}

// Same sum from precomputed diagonals: for each X-mask group g,
// D_g(j) = sum_{t in g} c_t i^{phase_t} (-1)^{|j & z_t|} (table `dtab`,
// [groups][2^n] complex in natural index order), E = sum_g sum_j
// Re(conj(psi_{j^x}) psi_j D_g(j)).
// kRealD: every D_g is real (a real observable): the imaginary parts are
// skipped.
template <typename Real, int R, bool kRealD = false>
__device__ double expect_table(const Observable &o, const typename CT<Real>::T *dtab,
                               const typename CT<Real>::T *st, int tid, int sh, int w, int dim) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    uint32_t v[R];
    const uint32_t s0 = natural_vectors<R>(tid, sh, w, v);
    C pj[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) pj[k] = st[s0 ^ xsel<R>(k, v)];
    // runs of kRun groups are summed in the state's precision (at most
    // kRun * NA products), the runs in FP64: FP64 adds are scarce on this GPU
    // One accumulator per amplitude slot k: NA independent FMA chains
    // instead of one chain through every group (the epilogue runs with few
    // warps per SM, so the chain's latency is exposed).
    constexpr int kRun = 8;
    double e = 0.0;
    Real run[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) run[k] = 0;
    auto fold = [&]() {
        Real r = 0;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            r += run[k];
            run[k] = 0;
        }
        e += (double)r;
    };
    for (int g = 0; g < o.n_tgroups; ++g) {
        const uint32_t sx = o.tgroups[g].sx;
        const C *D = dtab + (size_t)g * dim + tid;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const C px = st[s0 ^ xsel<R>(k, v) ^ sx];
            const C d = D[(size_t)k << sh];  // shared memory when staged, else global
            const Real wr = fmaR(px.x, pj[k].x, px.y * pj[k].y);
            if constexpr (kRealD) {
                run[k] = fmaR(wr, d.x, run[k]);
            } else {
                const Real wi = fmaR(px.x, pj[k].y, -px.y * pj[k].x);
                run[k] = fmaR(wr, d.x, fmaR(-wi, d.y, run[k]));
            }
        }
        if ((g + 1) % kRun == 0) fold();
    }
    fold();
    return e;
}

// lambda = H psi for this thread's amplitudes; returns sum Re(conj(psi_j) lambda_j).
template <typename Real, int R>
__device__ double apply_h(const Observable &o, const typename CT<Real>::T *psi,
                          typename CT<Real>::T *lam, int tid, int sh, int w) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    uint32_t v[R];
    const uint32_t s0 = natural_vectors<R>(tid, sh, w, v);
    C acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = cmk<C>(0, 0);
    for (int g = 0; g < o.n_tgroups; ++g) {
        const TermGroup tg = o.tgroups[g];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t j = (uint32_t)tid | ((uint32_t)k << sh);
            const uint32_t jx = j ^ tg.x;
            Real dre = 0, dim = 0;
            for (int t = tg.t_begin; t < tg.t_end; ++t) {
                const Term tm = o.terms[t];
                const Real c = (__popc(jx & tm.z) & 1u) ? (Real)-tm.coeff : (Real)tm.coeff;
                if (tm.phase == 0) dre += c;
                else if (tm.phase == 1) dim += c;
                else if (tm.phase == 2) dre -= c;
                else dim -= c;
            }
            const C px = psi[s0 ^ xsel<R>(k, v) ^ tg.sx];
            acc[k].x = fmaR(dre, px.x, fmaR(-dim, px.y, acc[k].x));
            acc[k].y = fmaR(dre, px.y, fmaR(dim, px.x, acc[k].y));
        }
    }
    double e = 0.0;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        const uint32_t sj = s0 ^ xsel<R>(k, v);
        const C pj = psi[sj];
        lam[sj] = acc[k];
        e += (double)fmaR(pj.x, acc[k].x, pj.y * acc[k].y);
    }
    return e;
}

// apply_h from the observable's diagonal tables `dtab` ([groups][2^n]
// complex, natural index order; device memory, read through the cache):
// lambda_j = sum_g D_g(j ^ x_g) psi_(j ^ x_g).  kRealD: every D_g is real.
template <typename Real, int R, bool kRealD>
__device__ double apply_h_table(const Observable &o, const typename CT<Real>::T *dtab,
                                const typename CT<Real>::T *psi, typename CT<Real>::T *lam,
                                int tid, int sh, int w, int dim) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    uint32_t v[R];
    const uint32_t s0 = natural_vectors<R>(tid, sh, w, v);
    C acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = cmk<C>(0, 0);
    for (int g = 0; g < o.n_tgroups; ++g) {
        const TermGroup tg = o.tgroups[g];
        const C *D = dtab + (size_t)g * dim;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const uint32_t jx = ((uint32_t)tid | ((uint32_t)k << sh)) ^ tg.x;
            const C d = __ldg(D + jx);
            const C px = psi[s0 ^ xsel<R>(k, v) ^ tg.sx];
            if constexpr (kRealD) {
                acc[k].x = fmaR(d.x, px.x, acc[k].x);
                acc[k].y = fmaR(d.x, px.y, acc[k].y);
            } else {
                acc[k].x = fmaR(d.x, px.x, fmaR(-d.y, px.y, acc[k].x));
                acc[k].y = fmaR(d.x, px.y, fmaR(d.y, px.x, acc[k].y));
            }
        }
    }
    double e = 0.0;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        const uint32_t sj = s0 ^ xsel<R>(k, v);
        const C pj = psi[sj];
        lam[sj] = acc[k];
        e += (double)fmaR(pj.x, acc[k].x, pj.y * acc[k].y);
    }
    return e;
}

// Parameter-shift combination by one block: dL/dtheta_k = sum_i L'_i
// (E_{k+,i} - E_{k-,i}) / 2, the energies and the cost.  `red`: 32 doubles.
__device__ void ps_combine_block(const double *E, int I, int P, const CostSource &c, double *lp,
                                 double *energy_out, double *loss_out, double *grad_out,
                                 double *red, double *stage = nullptr, int stage_cap = 0) {
    // With room in `stage` (shared memory the block no longer needs), every
    // thread first copies a share of the (2P + 1) I energies, so the sums
    // below wait for one round of device-memory loads instead of one per
    // unrolled batch; the arithmetic and its order are the same.
    const int64_t B = (int64_t)(2 * P + 1) * I;
    const bool staged = stage && B + I <= (int64_t)stage_cap;
    if (staged) {
        for (int64_t i = threadIdx.x; i < B; i += blockDim.x) stage[i] = __ldcg(E + i);
        __syncthreads();
        lp = stage + B;
    }
    auto ld = [&](int64_t i) { return staged ? stage[i] : __ldcg(E + i); };
    double part = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double e = ld(i);
        if (energy_out) energy_out[i] = e;
        if (c.cost == SV_COST_MSE) {
            const double d = e - c.targets[i];
            part += d * d / I;
        } else {
            part += c.weights[i] * e;
        }
        lp[i] = c.ext_weights ? c.ext_weights[i]
                              : (c.cost == SV_COST_MSE ? 2.0 * (e - c.targets[i]) / I : c.weights[i]);
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0 && loss_out) {
        double s = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi];
        loss_out[0] = s;
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int64_t ep = I + (int64_t)2 * k * I, em = ep + I;
        double g = 0.0;
#pragma unroll 8
        for (int i = 0; i < I; ++i) g += lp[i] * 0.5 * (ld(ep + i) - ld(em + i));
        grad_out[k] = g;
    }
}

// Copies the block-constant arrays into shared memory (independent 16-byte
// loads from every thread) and points the program/observable views at them.
// (kMode >= 1) Copies the block-constant arrays into shared memory with
// independent 16-byte loads from every thread and points the program and
// observable views at the copies.  The pointers are derived from the shared
// array unconditionally, so every later read compiles to a shared load.
__device__ __forceinline__ void bc_cp16(void *sdst, const void *gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void bc_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// The copies are asynchronous (cp.async, all in flight at once): the
// program, observable and thread bases form the first group and are waited
// for here; the diagonal tables (piece 6) form a second group, which
// finish_block_const waits for before the epilogue reads them.
template <int kMode>
__device__ __forceinline__ void stage_block_const(const BlockConst &bc, unsigned char *smem,
                                                  Program &p, Observable &o) {
    if constexpr (kMode == 0) return;
    unsigned char *base = smem + bc.base;
#pragma unroll
    for (int k = 0; k < kBlockConst; ++k) {
        if (k == 6) continue;
        uint4 *dst = reinterpret_cast<uint4 *>(base + bc.off[k]);
        const uint4 *src = bc.src[k];
        for (uint32_t i = threadIdx.x; i < bc.n16[k]; i += blockDim.x) bc_cp16(dst + i, src + i);
    }
    bc_commit();
    {
        uint4 *dst = reinterpret_cast<uint4 *>(base + bc.off[6]);
        const uint4 *src = bc.src[6];
        for (uint32_t i = threadIdx.x; i < bc.n16[6]; i += blockDim.x) bc_cp16(dst + i, src + i);
    }
    bc_commit();
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    p.stages = reinterpret_cast<const Stage *>(base + bc.off[0]);
    p.ops = reinterpret_cast<const Op *>(base + bc.off[1]);
    p.groups = reinterpret_cast<const Group *>(base + bc.off[2]);
    p.members = reinterpret_cast<const Member *>(base + bc.off[3]);
    o.tgroups = reinterpret_cast<const TermGroup *>(base + bc.off[4]);
    o.terms = reinterpret_cast<const Term *>(base + bc.off[5]);
    if constexpr (kMode == 2) p.tbase = reinterpret_cast<const ThreadBase *>(base + bc.off[7]);
}

// Waits for the diagonal tables staged by stage_block_const (all threads).
template <int kMode> __device__ __forceinline__ void finish_block_const() {
    if constexpr (kMode == 0) return;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

__device__ double cost_weight(const CostSource &c, int inst, double E) {
    if (c.ext_weights) return c.ext_weights[inst];
    if (c.cost == SV_COST_MSE) return 2.0 * (E - c.targets[inst]) / (double)c.n_instances;
    return c.weights[inst];
}

// rho <- G^dag rho G for the 2x2 reduced matrix of one qubit.
template <typename C> __device__ void sandwich(const C G[4], C r[4]) {
    C T[4], Gd[4], out[4];
    matmul2(r, G, T);
    Gd[0] = cconj(G[0]); Gd[1] = cconj(G[2]); Gd[2] = cconj(G[1]); Gd[3] = cconj(G[3]);
    matmul2(Gd, T, out);
    r[0] = out[0]; r[1] = out[1]; r[2] = out[2]; r[3] = out[3];
}

// Derivatives of every rotation in group g from the reduced matrix after the
// group: d E / d theta = Im tr(P rho), walking back member by member.
template <typename Real>
__device__ void group_gradients(const Program &p, int g, const double *rho8, const SlotInfo &si,
                                double *grad) {
    using C = typename CT<Real>::T;
    const Group grp = p.groups[g];
    int first = -1;
    for (int m = grp.m_begin; m < grp.m_end; ++m) {
        const Member mb = p.members[m];
        if (mb.kind <= M_RZ && mb.param >= 0) {
            first = m;
            break;
        }
    }
    if (first < 0) return;
    C r[4] = {cmk<C>(rho8[0], rho8[1]), cmk<C>(rho8[2], rho8[3]), cmk<C>(rho8[4], rho8[5]),
              cmk<C>(rho8[6], rho8[7])};
    for (int m = grp.m_end - 1; m >= first; --m) {
        const Member mb = p.members[m];
        if (mb.kind <= M_RZ && mb.param >= 0) {
            Real d;
            if (mb.kind == M_RX) d = r[1].y + r[2].y;
            else if (mb.kind == M_RY) d = r[1].x - r[2].x;
            else d = r[0].y - r[3].y;
            atomicAdd(&grad[mb.param], (double)d);
        }
        if (m > first) {
            C G[4];
            member_matrix<Real, C>(mb, si, G);
            sandwich(G, r);
        }
    }
}

// Stores the sums of the 8 values x over the slot's `width` lanes (a power
// of two) to dst[0..8).  From 8 lanes up: a reduce-scatter over lane bits
// 0-2 (the kept half follows the lane bit; afterwards x[0] holds value
// lane & 7), then butterfly adds over the remaining lane bits, and lanes
// 0..7 store one value each: 8 + log2(width / 8) shuffles instead of
// 8 log2(width).  Below 8 lanes, plain butterflies and lane 0 stores.
template <typename Real>
__device__ __forceinline__ void store_rho8(Real (&x)[8], int tid, int width, Real *dst) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = tid & 31;
    if (width >= 8) {
#pragma unroll
        for (int j = 0, M = 8; j < 3; ++j, M >>= 1) {
            const bool b = (lane >> j) & 1;
#pragma unroll
            for (int m = 0; m < M / 2; ++m) {
                const Real keep = b ? x[2 * m + 1] : x[2 * m], give = b ? x[2 * m] : x[2 * m + 1];
                x[m] = keep + __shfl_xor_sync(full, give, 1 << j);
            }
        }
        for (int off = 8; off < width; off <<= 1) x[0] += __shfl_xor_sync(full, x[0], off);
        if ((lane & (width - 1)) < 8) dst[lane & 7] = x[0];
    } else {
#pragma unroll
        for (int v = 0; v < 8; ++v)
            for (int off = width >> 1; off > 0; off >>= 1) x[v] += __shfl_xor_sync(full, x[v], off);
        if ((lane & (width - 1)) == 0) {
#pragma unroll
            for (int v = 0; v < 8; ++v) dst[v] = x[v];
        }
    }
}

// Reverse of bit_ops_fwd for bits I, I-1, ..., 0: per op, the partial reduced
// matrix of bit I (reduced over the warp, written to rw[group][warp]) then
// the inverse gate on psi and lambda.
template <typename C, typename Real, int R, int I>
__device__ __forceinline__ void bit_ops_rev(const Program &p, const Stage *sg, const C *mats,
                                            C (&a)[1 << R], C (&al)[1 << R], int width,
                                            int tid, int wps, Real *rw) {
    if constexpr (I >= 0) {
        const int b0 = sg->op_begin + sg->bit_begin[I];
        for (int o = sg->op_begin + sg->bit_begin[I + 1] - 1; o >= b0; --o) {
            const Op op = p.ops[o];
            const Group grp = p.groups[op.group];
            if (grp.has_param) {
                Real rh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                rho_bit<C, Real, R, I>(a, al, rh);
                store_rho8<Real>(rh, tid, width, rw + (op.group * wps + (tid >> 5)) * 8);
            }
            const C *m = mats + 4 * op.group;
            if (grp.real) {
                u1r_bit<C, Real, R, I>(a, m[0].x, m[2].x, m[1].x, m[3].x);
                u1r_bit<C, Real, R, I>(al, m[0].x, m[2].x, m[1].x, m[3].x);
            } else {
                const C d0 = cconj(m[0]), d1 = cconj(m[2]), d2 = cconj(m[1]), d3 = cconj(m[3]);
                u1_bit<C, R, I>(a, d0, d1, d2, d3);
                u1_bit<C, R, I>(al, d0, d1, d2, d3);
            }
        }
        bit_ops_rev<C, Real, R, I - 1>(p, sg, mats, a, al, width, tid, wps, rw);
    }
}

// Reverse sweep over every stage of `p` on psi and lambda (both in shared
// memory, natural order, swizzled): un-applies each stage, and for every
// fused group with parameters writes the warp sums of its reduced matrix
// rho_ab = sum psi_a conj(lambda_b) at the point after the group to
// rw[group][warp][8] (each group occurs once); fold_rho then sums the warps
// in FP64.  Called by all threads of the slot.
template <typename Real, int R, int kMode>
__device__ void reverse_stages(const Program &p, typename CT<Real>::T *psi,
                               typename CT<Real>::T *lam, const typename CT<Real>::T *mats,
                               int tid, int Ts, Real *rw) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    const int wps = Ts >= 32 ? (Ts >> 5) : 1;
    C a[NA], al[NA];
    const int width = Ts < 32 ? Ts : 32;
    Bases nxt = bases_of<kMode>(p, p.n_stages - 1, tid, Ts);
    for (int s = p.n_stages - 1; s >= 0; --s) {
        const Stage *sg = p.stages + s;
        const Bases bs = nxt;
        if (s > 0) nxt = bases_of<kMode>(p, s - 1, tid, Ts);
        uint32_t lq[R], sq[R];
        int qq[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            lq[i] = sg->ldq[i];
            sq[i] = sg->stq[i];
            qq[i] = sg->q[i];
        }
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const uint32_t ad = bs.sb ^ xsel<R>(r, sq);
            a[r] = psi[ad];
            al[r] = lam[ad];
        }
        if (sg->sorted)
            bit_ops_rev<C, Real, R, R - 1>(p, sg, mats, a, al, width, tid, wps, rw);
        else
        for (int oi = sg->op_end - 1; oi >= sg->op_begin; --oi) {
            const Op op = p.ops[oi];
            if (op.kind == OP_U1) {
                if (p.groups[op.group].has_param) {
                    Real rh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    rho_reg<C, Real, R>(a, al, op.a, rh);
                    store_rho8<Real>(rh, tid, width, rw + (op.group * wps + (tid >> 5)) * 8);
                }
                const C *m = mats + 4 * op.group;
                const C d0 = cconj(m[0]), d1 = cconj(m[2]), d2 = cconj(m[1]), d3 = cconj(m[3]);
                u1_reg<C, R>(a, op.a, d0, d1, d2, d3);
                u1_reg<C, R>(al, op.a, d0, d1, d2, d3);
            } else {
                cz_regs<C, R>(a, bs.lg, qq, op.a, op.b);
                cz_regs<C, R>(al, bs.lg, qq, op.a, op.b);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const uint32_t ad = bs.lb ^ xsel<R>(r, lq);
            psi[ad] = a[r];
            lam[ad] = al[r];
        }
        __syncthreads();
    }
}

// rho[g][v] = sum over the warps of rw[g][warp][v] in FP64, for the groups
// with parameters.  Called by all threads of the slot after reverse_stages.
template <typename Real>
__device__ void fold_rho(const Program &p, const Real *rw, int tid, int Ts, double *rho) {
    const int wps = Ts >= 32 ? (Ts >> 5) : 1;
    for (int q = tid; q < 8 * p.n_groups; q += Ts) {
        const int g = q >> 3, v = q & 7;
        double acc = 0.0;
        if (p.groups[g].has_param)
            for (int w = 0; w < wps; ++w) acc += (double)rw[(g * wps + w) * 8 + v];
        rho[q] = acc;
    }
}

}  // namespace
}  // namespace svk
