// On-chip engine: one circuit slot per group of 2^(n-R) threads, the whole
// 2^n-amplitude state in shared memory, 2^R amplitudes per thread in
// registers.  Kernels:
//   k_energy   - build |ref>, apply the circuit, <H> epilogue (one launch for
//                every parameter-shift copy x instance of a gradient);
//   k_store    - same, but write the final states to device memory;
//   k_expect   - <H> of states already in device memory;
//   k_adjoint  - forward pass, lambda = H psi, reverse sweep with the
//                derivative of every rotation (paper's method evaluates
//                gradients by parameter shift, Sec. 4.1; the adjoint sweep
//                gives the same numbers from 2 states per circuit).
// Products run in the state's precision (FP32 for complex64); every
// reduction across amplitudes, threads or terms is accumulated in FP64.
#include <cuda_runtime.h>

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
// m*x + k*y with 4 fused operations per component.
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

template <typename C, int R>
__device__ __forceinline__ void apply_stage_ops(const Program &p, const Stage *sg, const C *mats,
                                                C (&a)[1 << R], uint32_t lg, const int (&qq)[R]) {
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
// index order, swizzled).  Stage 0 builds |ref> in registers.
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
        if (s == 0) {
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
        if (s > 0) __syncthreads();
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
    double e = 0.0;
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
        e += (double)gacc;
    }
    return e;
}

// Same sum from precomputed diagonals: for each X-mask group g,
// D_g(j) = sum_{t in g} c_t i^{phase_t} (-1)^{|j & z_t|} (table `dtab`,
// [groups][2^n] complex in natural index order), E = sum_g sum_j
// Re(conj(psi_{j^x}) psi_j D_g(j)).
template <typename Real, int R>
__device__ double expect_table(const Observable &o, const typename CT<Real>::T *dtab,
                               const typename CT<Real>::T *st, int tid, int sh, int w, int dim) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    uint32_t v[R];
    const uint32_t s0 = natural_vectors<R>(tid, sh, w, v);
    C pj[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) pj[k] = st[s0 ^ xsel<R>(k, v)];
    double e = 0.0;
    for (int g = 0; g < o.n_tgroups; ++g) {
        const uint32_t sx = o.tgroups[g].sx;
        const C *D = dtab + (size_t)g * dim + tid;
        Real acc = 0;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const C px = st[s0 ^ xsel<R>(k, v) ^ sx];
            const C d = D[(size_t)k << sh];  // shared memory when staged, else global
            const Real wr = fmaR(px.x, pj[k].x, px.y * pj[k].y);
            const Real wi = fmaR(px.x, pj[k].y, -px.y * pj[k].x);
            acc = fmaR(wr, d.x, fmaR(-wi, d.y, acc));
        }
        e += (double)acc;
    }
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

// Parameter-shift combination by one block: dL/dtheta_k = sum_i L'_i
// (E_{k+,i} - E_{k-,i}) / 2, the energies and the cost.  `red`: 32 doubles.
__device__ void ps_combine_block(const double *E, int I, int P, const CostSource &c, double *lp,
                                 double *energy_out, double *loss_out, double *grad_out,
                                 double *red) {
    double part = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double e = __ldcg(E + i);
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
        const double *ep = E + I + (int64_t)2 * k * I, *em = ep + I;
        double g = 0.0;
#pragma unroll 8
        for (int i = 0; i < I; ++i) g += lp[i] * 0.5 * (__ldcg(ep + i) - __ldcg(em + i));
        grad_out[k] = g;
    }
}

// Copies the block-constant arrays into shared memory (independent 16-byte
// loads from every thread) and points the program/observable views at them.
// (kMode >= 1) Copies the block-constant arrays into shared memory with
// independent 16-byte loads from every thread and points the program and
// observable views at the copies.  The pointers are derived from the shared
// array unconditionally, so every later read compiles to a shared load.
template <int kMode>
__device__ __forceinline__ void stage_block_const(const BlockConst &bc, unsigned char *smem,
                                                  Program &p, Observable &o) {
    if constexpr (kMode == 0) return;
    unsigned char *base = smem + bc.base;
#pragma unroll
    for (int k = 0; k < kBlockConst; ++k) {
        uint4 *dst = reinterpret_cast<uint4 *>(base + bc.off[k]);
        const uint4 *src = bc.src[k];
        for (uint32_t i = threadIdx.x; i < bc.n16[k]; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    p.stages = reinterpret_cast<const Stage *>(base + bc.off[0]);
    p.ops = reinterpret_cast<const Op *>(base + bc.off[1]);
    p.groups = reinterpret_cast<const Group *>(base + bc.off[2]);
    p.members = reinterpret_cast<const Member *>(base + bc.off[3]);
    o.tgroups = reinterpret_cast<const TermGroup *>(base + bc.off[4]);
    o.terms = reinterpret_cast<const Term *>(base + bc.off[5]);
    if constexpr (kMode == 2) p.tbase = reinterpret_cast<const ThreadBase *>(base + bc.off[7]);
}

// ---------------------------------------------------------------- kernels

template <typename Real, int R, int kMode>
__global__ void __launch_bounds__(512) k_energy(Program p, Observable o, SlotSource src,
                                                OnchipShape sh, double *energies,
                                                const typename CT<Real>::T *dtab,
                                                FusedCombine fc, BlockConst bc) {
    using C = typename CT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    stage_block_const<kMode>(bc, smem, p, o);
    const int n = p.n, shb = n - R, Ts = 1 << shb;
    const int ls = threadIdx.x >> shb, tid = threadIdx.x & (Ts - 1);
    const int b = blockIdx.x * sh.S + ls;
    const bool live = b < src.n_slots;
    C *st = reinterpret_cast<C *>(smem + (size_t)ls * sh.st_state);
    C *mats = reinterpret_cast<C *>(smem + sh.off_mats + (size_t)ls * sh.st_mats);
    double *red = reinterpret_cast<double *>(smem + sh.off_red);

    const SlotInfo si = resolve(src, live ? b : 0);
    for (int g = tid; g < p.n_groups; g += Ts) group_matrix<Real, C>(p, g, si, mats + 4 * g);
    __syncthreads();
    forward_stages<Real, R, kMode>(p, st, mats, tid, si.ref);
    double e;
    if (kMode > 0 && bc.n16[6]) {  // diagonal tables staged in shared memory
        const C *tab = reinterpret_cast<const C *>(smem + bc.base + bc.off[6]);
        e = expect_table<Real, R>(o, tab, st, tid, shb, p.swz_bits, 1 << n);
    } else if (dtab) {
        e = expect_table<Real, R>(o, dtab, st, tid, shb, p.swz_bits, 1 << n);
    } else {
        e = expect_partial<Real, R>(o, st, tid, shb, p.swz_bits);
    }
    e = slot_sum(e, Ts, red);
    if (live && tid == 0) energies[b] = e;
    if (!fc.counter) return;
    // The last block to finish assembles the gradient (no second launch).
    __shared__ unsigned last;
    __shared__ double cred[32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(fc.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    ps_combine_block(energies, fc.I, fc.P, fc.cost, fc.lp, fc.energy_out, fc.loss_out,
                     fc.grad_out, cred);
    if (threadIdx.x == 0) *fc.counter = 0u;
}

template <typename Real, int R>
__global__ void __launch_bounds__(512) k_store(Program p, SlotSource src, OnchipShape sh,
                                               typename CT<Real>::T *states) {
    using C = typename CT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = p.n, shb = n - R, Ts = 1 << shb;
    const int ls = threadIdx.x >> shb, tid = threadIdx.x & (Ts - 1);
    const int b = blockIdx.x * sh.S + ls;
    const bool live = b < src.n_slots;
    C *st = reinterpret_cast<C *>(smem + (size_t)ls * sh.st_state);
    C *mats = reinterpret_cast<C *>(smem + sh.off_mats + (size_t)ls * sh.st_mats);

    const SlotInfo si = resolve(src, live ? b : 0);
    for (int g = tid; g < p.n_groups; g += Ts) group_matrix<Real, C>(p, g, si, mats + 4 * g);
    __syncthreads();
    forward_stages<Real, R, 0>(p, st, mats, tid, si.ref);
    if (!live) return;
    const int row = src.rows ? src.rows[b] : b;
    C *out = states + ((int64_t)row << n);
    const int w = p.swz_bits;
    for (int k = 0; k < (1 << R); ++k) {
        const uint32_t j = (uint32_t)tid + ((uint32_t)k << shb);
        out[j] = st[swizzle(j, w)];
    }
}

template <typename Real, int R>
__global__ void __launch_bounds__(512) k_expect(int n, int swz_bits, Observable o,
                                                const typename CT<Real>::T *states, int n_rows,
                                                OnchipShape sh, double *out) {
    using C = typename CT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int shb = n - R, Ts = 1 << shb;
    const int ls = threadIdx.x >> shb, tid = threadIdx.x & (Ts - 1);
    const int b = blockIdx.x * sh.S + ls;
    const bool live = b < n_rows;
    C *st = reinterpret_cast<C *>(smem + (size_t)ls * sh.st_state);
    double *red = reinterpret_cast<double *>(smem + sh.off_red);
    const C *in = states + ((int64_t)(live ? b : 0) << n);
    for (int k = 0; k < (1 << R); ++k) {
        const uint32_t j = (uint32_t)tid + ((uint32_t)k << shb);
        st[swizzle(j, swz_bits)] = in[j];
    }
    __syncthreads();
    double e = expect_partial<Real, R>(o, st, tid, shb, swz_bits);
    e = slot_sum(e, Ts, red);
    if (live && tid == 0) out[b] = e;
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

template <typename Real, int R, int kMode>
__global__ void __launch_bounds__(512) k_adjoint(Program p, Observable o, SlotSource src,
                                                 CostSource cs, OnchipShape sh,
                                                 double *slot_grads, double *slot_E,
                                                 BlockConst bc) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    stage_block_const<kMode>(bc, smem, p, o);
    const int n = p.n, shb = n - R, Ts = 1 << shb;
    const int ls = threadIdx.x >> shb, tid = threadIdx.x & (Ts - 1);
    const int b = blockIdx.x * sh.S + ls;
    const bool live = b < src.n_slots;
    const int G = p.n_groups, P = p.n_params;
    const int wps = Ts >= 32 ? (Ts >> 5) : 1;
    C *psi = reinterpret_cast<C *>(smem + (size_t)ls * sh.st_state);
    C *lam = reinterpret_cast<C *>(smem + sh.off_lam + (size_t)ls * sh.st_state);
    C *mats = reinterpret_cast<C *>(smem + sh.off_mats + (size_t)ls * sh.st_mats);
    double *rho = reinterpret_cast<double *>(smem + sh.off_rho + (size_t)ls * sh.st_rho);
    double *grad = reinterpret_cast<double *>(smem + sh.off_grad + (size_t)ls * sh.st_grad);
    Real *rhow = reinterpret_cast<Real *>(smem + sh.off_rhow + (size_t)ls * sh.st_rhow);
    double *red = reinterpret_cast<double *>(smem + sh.off_red);

    const SlotInfo si = resolve(src, live ? b : 0);
    for (int g = tid; g < G; g += Ts) group_matrix<Real, C>(p, g, si, mats + 4 * g);
    for (int q = tid; q < P; q += Ts) grad[q] = 0.0;
    __syncthreads();
    forward_stages<Real, R, kMode>(p, psi, mats, tid, si.ref);
    double e = apply_h<Real, R>(o, psi, lam, tid, shb, p.swz_bits);
    e = slot_sum(e, Ts, red);
    __syncthreads();

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
        Real *rw = rhow + (s & 1) * (kMaxGroupOpsPerStage * wps * 8);
        int u = sg->n_u1;
        for (int oi = sg->op_end - 1; oi >= sg->op_begin; --oi) {
            const Op op = p.ops[oi];
            if (op.kind == OP_U1) {
                --u;
                if (p.groups[op.group].has_param) {
                    Real rh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    rho_reg<C, Real, R>(a, al, op.a, rh);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        for (int off = width >> 1; off > 0; off >>= 1)
                            rh[v] += __shfl_xor_sync(0xffffffffu, rh[v], off);
                    if ((tid & 31) == 0) {
                        Real *dst = rw + (u * wps + (tid >> 5)) * 8;
#pragma unroll
                        for (int v = 0; v < 8; ++v) dst[v] = rh[v];
                    }
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
        // Fold the per-warp partials of every group op of this stage (a slot
        // may have fewer threads than the stage has group ops).
        for (int uu = tid; uu < sg->n_u1; uu += Ts) {
            int cnt = 0, gi = -1;
            for (int oi = sg->op_begin; oi < sg->op_end; ++oi) {
                const Op op = p.ops[oi];
                if (op.kind != OP_U1) continue;
                if (cnt == uu) {
                    gi = op.group;
                    break;
                }
                ++cnt;
            }
            if (gi >= 0 && p.groups[gi].has_param) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    double acc = 0.0;
                    for (int wi = 0; wi < wps; ++wi) acc += (double)rw[(uu * wps + wi) * 8 + v];
                    rho[gi * 8 + v] = acc;
                }
            }
        }
    }
    __syncthreads();
    for (int g = tid; g < G; g += Ts)
        if (p.groups[g].has_param) group_gradients<Real>(p, g, rho + 8 * g, si, grad);
    __syncthreads();
    if (!live) return;
    const double wgt = cost_weight(cs, si.instance, e);
    for (int q = tid; q < P; q += Ts) slot_grads[(int64_t)b * P + q] = wgt * grad[q];
    if (tid == 0) slot_E[b] = e;
}

// --------------------------------------------------------- combinations

// Parameter-shift combination as its own launch.
__global__ void k_ps_combine(const double *E, int I, int P, CostSource c, double *lp,
                             double *energy_out, double *loss_out, double *grad_out) {
    __shared__ double red[32];
    ps_combine_block(E, I, P, c, lp, energy_out, loss_out, grad_out, red);
}

// Adjoint combination: dL/dtheta = sum_i (weighted per-instance gradients).
__global__ void k_adjoint_combine(const double *Gs, const double *E, int I, int P, CostSource c,
                                  double *energy_out, double *loss_out, double *grad_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        double g = 0.0;
        for (int i = 0; i < I; ++i) g += Gs[(int64_t)i * P + k];
        grad_out[k] = g;
    }
    if (blockIdx.x == 0) {
        __shared__ double red[32];
        double part = 0.0;
        for (int i = threadIdx.x; i < I; i += blockDim.x) {
            const double e = E[i];
            if (energy_out) energy_out[i] = e;
            if (c.cost == SV_COST_MSE) {
                const double d = e - c.targets[i];
                part += d * d / I;
            } else {
                part += c.weights ? c.weights[i] * e : 0.0;
            }
        }
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0 && loss_out) {
            double s = 0.0;
            for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi];
            loss_out[0] = s;
        }
    }
}

template <typename T> T *kptr(void *p) { return reinterpret_cast<T *>(p); }

uint32_t up16(size_t x) { return (uint32_t)((x + 15) & ~size_t(15)); }

template <typename K> cudaError_t prep(K kernel, uint32_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

// ----------------------------------------------------------- host side

const char *onchip_shape(int kind, int n, int n_groups, int n_params, int c128, int n_slots,
                         int reg_bits, int threads_per_block, OnchipShape *out, int num_sms,
                         uint32_t const_bytes) {
    OnchipShape s{};
    const size_t csz = c128 ? 16 : 8, rsz = c128 ? 8 : 4;
    if (num_sms < 1) num_sms = 1;
    // Register bits: at most 4 (3 for complex128), at most 512 threads per
    // slot.  By default fewer register bits (more threads per circuit) when
    // the batch would otherwise leave the schedulers with < 2 warps each.
    const int rmax = c128 ? 3 : 4;
    int R = reg_bits;
    if (R <= 0) {
        R = kind == ONCHIP_ADJOINT ? 3 : rmax;
        const int64_t want = (int64_t)num_sms * 4 * 32 * 2;
        while (R > 2 && (int64_t)n_slots * (int64_t(1) << (n > R ? n - R : 0)) < want) --R;
    }
    if (R < 1 || R > rmax) return "reg_bits out of range for this kernel";
    if (R > n) R = n;
    if (n - R > 9) R = n - 9;
    if (R > rmax) return "state too large for the on-chip engine";
    const int Ts = 1 << (n - R);
    if (threads_per_block > 512) return "threads_per_block must be <= 512";
    int S;
    if (threads_per_block > 0) {
        S = threads_per_block / Ts;
        if (threads_per_block % Ts != 0 || S < 1)
            return "threads_per_block must be a multiple of the threads per slot";
    } else {
        // Enough blocks for two per SM where the batch allows, at least one
        // warp and at most 256 threads per block.
        S = (int)((n_slots + 2 * num_sms - 1) / (2 * num_sms));
        if (S * Ts > 256) S = 256 / Ts;
        if (S < 1) S = 1;
    }
    if (S * Ts < 32) S = 32 / Ts;
    const size_t dim = size_t(1) << n;
    const int wps = Ts >= 32 ? Ts / 32 : 1;
    const uint32_t kLimit = 200 * 1024;
    for (;;) {
        s.st_state = up16(dim * csz);
        s.st_mats = up16((size_t)n_groups * 4 * csz);
        s.st_rho = 0;
        s.st_grad = 0;
        s.st_rhow = 0;
        size_t off = (size_t)S * s.st_state;
        s.off_lam = 0;
        if (kind == ONCHIP_ADJOINT) {
            s.off_lam = (uint32_t)off;
            off += (size_t)S * s.st_state;
        }
        s.off_mats = (uint32_t)off;
        if (kind != ONCHIP_EXPECT) off += (size_t)S * s.st_mats;
        if (kind == ONCHIP_ADJOINT) {
            s.st_rho = up16((size_t)n_groups * 8 * 8);
            s.st_grad = up16((size_t)n_params * 8);
            s.st_rhow = up16((size_t)2 * kMaxGroupOpsPerStage * wps * 8 * rsz);
            s.off_rho = (uint32_t)off;
            off += (size_t)S * s.st_rho;
            s.off_grad = (uint32_t)off;
            off += (size_t)S * s.st_grad;
            s.off_rhow = (uint32_t)off;
            off += (size_t)S * s.st_rhow;
        }
        s.off_red = (uint32_t)off;
        off += up16((size_t)((S * Ts + 31) / 32) * 8);
        s.off_const = (uint32_t)off;
        s.const_bytes = 0;
        if (const_bytes && off + const_bytes <= kLimit) {
            s.const_bytes = const_bytes;
            off += const_bytes;
        }
        if (off <= kLimit) {
            s.smem = (uint32_t)off;
            break;
        }
        if (S == 1) return "state too large for the on-chip engine";
        S = S / 2;
    }
    s.R = R;
    s.Ts = Ts;
    s.S = S;
    s.blocks = (n_slots + S - 1) / S;
    *out = s;
    return nullptr;
}

#define SVK_DISPATCH_R(R_, CALL)                                                 \
    switch (R_) {                                                                \
    case 1: { constexpr int RR = 1; CALL; } break;                               \
    case 2: { constexpr int RR = 2; CALL; } break;                               \
    case 3: { constexpr int RR = 3; CALL; } break;                               \
    case 4: { constexpr int RR = 4; CALL; } break;                               \
    default: return cudaErrorInvalidValue;                                       \
    }
// complex128 kernels stop at 3 register bits (8 amplitudes = 32 registers).
#define SVK_DISPATCH_R_C128(R_, CALL)                                            \
    switch (R_) {                                                                \
    case 1: { constexpr int RR = 1; CALL; } break;                               \
    case 2: { constexpr int RR = 2; CALL; } break;                               \
    case 3: { constexpr int RR = 3; CALL; } break;                               \
    default: return cudaErrorInvalidValue;                                       \
    }

template <typename Real, int R>
static cudaError_t run_energy(const OnchipShape &sh, const Program &p, const Observable &o,
                              const SlotSource &s, double *E, const void *dtab,
                              const FusedCombine &fc, const BlockConst &bc, cudaStream_t st) {
    auto k = !bc.bytes ? k_energy<Real, R, 0> : (bc.n16[7] ? k_energy<Real, R, 2>
                                                           : k_energy<Real, R, 1>);
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(
        p, o, s, sh, E, reinterpret_cast<const typename CT<Real>::T *>(dtab), fc, bc);
    return cudaGetLastError();
}

// The staged block constants live at the end of the shape's layout; a
// BlockConst without a region in `sh` is ignored (global reads).
static BlockConst fit_const(const OnchipShape &sh, const BlockConst *bc) {
    BlockConst b{};
    if (bc && sh.const_bytes >= bc->bytes && bc->bytes) {
        b = *bc;
        b.base = sh.off_const;
    }
    return b;
}

cudaError_t launch_onchip_energy(int c128, const OnchipShape &sh, const Program &p,
                                 const Observable &o, const SlotSource &s, double *E,
                                 cudaStream_t st, const void *dtab, const FusedCombine *fc,
                                 const BlockConst *bc) {
    if (sh.blocks == 0) return cudaSuccess;
    FusedCombine none{};
    const FusedCombine &f = fc ? *fc : none;
    BlockConst b = fit_const(sh, bc);
    if (!dtab) b.n16[6] = 0;
    if (c128) {
        SVK_DISPATCH_R_C128(sh.R, return (run_energy<double, RR>(sh, p, o, s, E, dtab, f, b, st)));
    }
    SVK_DISPATCH_R(sh.R, return (run_energy<float, RR>(sh, p, o, s, E, dtab, f, b, st)));
    return cudaSuccess;
}

// Diagonal tables D_g(j) of an observable, [groups][2^n] complex (Real).
template <typename Real>
__global__ void k_build_dtable(Observable o, int n, typename CT<Real>::T *out) {
    using C = typename CT<Real>::T;
    const int64_t dim = int64_t(1) << n;
    const int64_t total = dim * o.n_tgroups;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(i >> n);
        const uint32_t j = (uint32_t)(i & (dim - 1));
        const TermGroup tg = o.tgroups[g];
        double re = 0.0, im = 0.0;
        for (int t = tg.t_begin; t < tg.t_end; ++t) {
            const Term tm = o.terms[t];
            const double c = (__popc(j & tm.z) & 1u) ? -tm.coeff : tm.coeff;
            if (tm.phase == 0) re += c;
            else if (tm.phase == 1) im += c;
            else if (tm.phase == 2) re -= c;
            else im -= c;
        }
        C d;
        d.x = (Real)re;
        d.y = (Real)im;
        out[i] = d;
    }
}

cudaError_t launch_build_dtable(int c128, const Observable &o, int n, void *out, cudaStream_t st) {
    const int64_t total = (int64_t(1) << n) * o.n_tgroups;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (c128) k_build_dtable<double><<<blocks, 256, 0, st>>>(o, n, (double2 *)out);
    else k_build_dtable<float><<<blocks, 256, 0, st>>>(o, n, (float2 *)out);
    return cudaGetLastError();
}

template <typename Real, int R>
static cudaError_t run_store(const OnchipShape &sh, const Program &p, const SlotSource &s,
                             void *states, cudaStream_t st) {
    auto k = k_store<Real, R>;
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(p, s, sh,
                                               kptr<typename CT<Real>::T>(states));
    return cudaGetLastError();
}

cudaError_t launch_onchip_store(int c128, const OnchipShape &sh, const Program &p,
                                const SlotSource &s, void *states, cudaStream_t st) {
    if (sh.blocks == 0) return cudaSuccess;
    if (c128) { SVK_DISPATCH_R_C128(sh.R, return (run_store<double, RR>(sh, p, s, states, st))); }
    SVK_DISPATCH_R(sh.R, return (run_store<float, RR>(sh, p, s, states, st)));
    return cudaSuccess;
}

template <typename Real, int R>
static cudaError_t run_expect(const OnchipShape &sh, int n, int w, const Observable &o,
                              const void *states, int rows, double *out, cudaStream_t st) {
    auto k = k_expect<Real, R>;
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(
        n, w, o, reinterpret_cast<const typename CT<Real>::T *>(states), rows, sh, out);
    return cudaGetLastError();
}

cudaError_t launch_onchip_expect(int c128, const OnchipShape &sh, int n, int swz_bits,
                                 const Observable &o, const void *states, int n_rows,
                                 double *out, cudaStream_t st) {
    if (sh.blocks == 0) return cudaSuccess;
    if (c128) { SVK_DISPATCH_R_C128(sh.R, return (run_expect<double, RR>(sh, n, swz_bits, o, states, n_rows,
                                                            out, st)));
    }
    SVK_DISPATCH_R(sh.R,
                   return (run_expect<float, RR>(sh, n, swz_bits, o, states, n_rows, out, st)));
    return cudaSuccess;
}

template <typename Real, int R>
static cudaError_t run_adjoint(const OnchipShape &sh, const Program &p, const Observable &o,
                               const SlotSource &s, const CostSource &c, double *G, double *E,
                               const BlockConst &b, cudaStream_t st) {
    auto k = !b.bytes ? k_adjoint<Real, R, 0> : (b.n16[7] ? k_adjoint<Real, R, 2>
                                                         : k_adjoint<Real, R, 1>);
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(p, o, s, c, sh, G, E, b);
    return cudaGetLastError();
}

cudaError_t launch_onchip_adjoint(int c128, const OnchipShape &sh, const Program &p,
                                  const Observable &o, const SlotSource &s, const CostSource &c,
                                  double *G, double *E, cudaStream_t st, const BlockConst *bc) {
    if (sh.blocks == 0) return cudaSuccess;
    BlockConst b = fit_const(sh, bc);
    b.n16[6] = 0;
    if (c128) {
        SVK_DISPATCH_R_C128(sh.R, return (run_adjoint<double, RR>(sh, p, o, s, c, G, E, b, st)));
    }
    SVK_DISPATCH_R(sh.R, return (run_adjoint<float, RR>(sh, p, o, s, c, G, E, b, st)));
    return cudaSuccess;
}

cudaError_t launch_ps_combine(const double *E, int I, int P, const CostSource &c, double *lp,
                              double *energy_out, double *loss_out, double *grad_out,
                              cudaStream_t st) {
    k_ps_combine<<<1, 256, 0, st>>>(E, I, P, c, lp, energy_out, loss_out, grad_out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_combine(const double *G, const double *E, int I, int P,
                                   const CostSource &c, double *energy_out, double *loss_out,
                                   double *grad_out, cudaStream_t st) {
    const int threads = 256;
    int blocks = (P + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    k_adjoint_combine<<<blocks, threads, 0, st>>>(G, E, I, P, c, energy_out, loss_out, grad_out);
    return cudaGetLastError();
}

}  // namespace svk
