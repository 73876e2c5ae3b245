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

#include <algorithm>

#include "engine.cuh"
#include "kernels.h"

namespace svk {
namespace {

// ---------------------------------------------------------------- kernels

template <typename Real, int R, int kMode>
__global__ void __launch_bounds__(512) k_energy(Program p, Observable o, SlotSource src,
                                                OnchipShape sh, double *energies,
                                                const typename CT<Real>::T *dtab,
                                                BlockConst bc) {
    using C = typename CT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    // a combination kernel launched behind this one may be scheduled now (it
    // waits for this grid's completion before reading the energies)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
    finish_block_const<kMode>();  // the diagonal tables, copied during the stages
    double e;
    if (kMode > 0 && bc.n16[6]) {  // diagonal tables staged in shared memory
        const C *tab = reinterpret_cast<const C *>(smem + bc.base + bc.off[6]);
        e = o.real ? expect_table<Real, R, true>(o, tab, st, tid, shb, p.swz_bits, 1 << n)
                   : expect_table<Real, R>(o, tab, st, tid, shb, p.swz_bits, 1 << n);
    } else if (dtab) {
        e = expect_table<Real, R>(o, dtab, st, tid, shb, p.swz_bits, 1 << n);
    } else {
        e = expect_partial<Real, R>(o, st, tid, shb, p.swz_bits);
    }
    e = slot_sum(e, Ts, red);
    if (live && tid == 0) energies[b] = e;
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

template <typename Real, int R, int kMode>
__global__ void __launch_bounds__(512) k_adjoint(Program p, Observable o, SlotSource src,
                                                 CostSource cs, OnchipShape sh,
                                                 double *slot_grads, double *slot_E,
                                                 BlockConst bc,
                                                 const typename CT<Real>::T *dtab) {
    using C = typename CT<Real>::T;
    constexpr int NA = 1 << R;
    extern __shared__ __align__(16) unsigned char smem[];
    stage_block_const<kMode>(bc, smem, p, o);
    finish_block_const<kMode>();
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
    double e = !dtab ? apply_h<Real, R>(o, psi, lam, tid, shb, p.swz_bits)
                     : (o.real ? apply_h_table<Real, R, true>(o, dtab, psi, lam, tid, shb, p.swz_bits, 1 << n)
                               : apply_h_table<Real, R, false>(o, dtab, psi, lam, tid, shb, p.swz_bits,
                                                               1 << n));
    e = slot_sum(e, Ts, red);
    __syncthreads();

    reverse_stages<Real, R, kMode>(p, psi, lam, mats, tid, Ts, rhow);
    fold_rho<Real>(p, rhow, tid, Ts, rho);
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

// The same, launched as a programmatic dependent of the energy kernel: it
// is scheduled while the energies are computed and waits for that grid to
// complete (its writes visible) before it reads them.  `stage`: dynamic
// shared memory of stage_cap doubles for the energies.
__global__ void k_ps_combine_dep(const double *E, int I, int P, CostSource c, double *lp,
                                 double *energy_out, double *loss_out, double *grad_out,
                                 int stage_cap) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double red[32];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    ps_combine_block(E, I, P, c, lp, energy_out, loss_out, grad_out, red,
                     reinterpret_cast<double *>(dsm), stage_cap);
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
        if (threads_per_block % 32 != 0) return "threads_per_block must be a multiple of 32";
    } else {
        // Enough blocks for two per SM where the batch allows, at least one
        // warp and at most 256 threads per block.
        S = (int)((n_slots + 2 * num_sms - 1) / (2 * num_sms));
        if (S * Ts > 256) S = 256 / Ts;
        if (S < 1) S = 1;
    }
    // whole warps: the reductions shuffle over full warps
    const int sm = Ts < 32 ? 32 / Ts : 1;
    S = (S + sm - 1) / sm * sm;
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
            s.st_rhow = up16((size_t)n_groups * wps * 8 * rsz);  // [group][warp][8]
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
        if (S <= sm) return "state too large for the on-chip engine";
        S = std::max(sm, S / 2 / sm * sm);
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
                              const BlockConst &bc, cudaStream_t st) {
    auto k = !bc.bytes ? k_energy<Real, R, 0> : (bc.n16[7] ? k_energy<Real, R, 2>
                                                           : k_energy<Real, R, 1>);
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(
        p, o, s, sh, E, reinterpret_cast<const typename CT<Real>::T *>(dtab), bc);
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

static cudaError_t energy_kernel(int c128, const OnchipShape &sh, const Program &p,
                                 const Observable &o, const SlotSource &s, double *E,
                                 cudaStream_t st, const void *dtab, const BlockConst &b) {
    if (c128) {
        SVK_DISPATCH_R_C128(sh.R, return (run_energy<double, RR>(sh, p, o, s, E, dtab, b, st)));
    }
    SVK_DISPATCH_R(sh.R, return (run_energy<float, RR>(sh, p, o, s, E, dtab, b, st)));
    return cudaSuccess;
}

cudaError_t launch_onchip_energy(int c128, const OnchipShape &sh, const Program &p,
                                 const Observable &o, const SlotSource &s, double *E,
                                 cudaStream_t st, const void *dtab, const FusedCombine *fc,
                                 const BlockConst *bc) {
    if (sh.blocks == 0) return cudaSuccess;
    BlockConst b = fit_const(sh, bc);
    if (!dtab) b.n16[6] = 0;
    if (!fc) return energy_kernel(c128, sh, p, o, s, E, st, dtab, b);
    // The gradient combination follows as a programmatic dependent launch:
    // its launch overlaps the energy kernel, no block of which waits for the
    // others (a last-block tail in the energy kernel measured slower).
    cudaError_t e = energy_kernel(c128, sh, p, o, s, E, st, dtab, b);
    if (e != cudaSuccess) return e;
    const int64_t B = (int64_t)(2 * fc->P + 1) * fc->I;
    const int cap = B + fc->I <= 6144 ? (int)(B + fc->I) : 0;  // <= 48 KiB of staging
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sizeof(double) * (size_t)cap;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_ps_combine_dep, (const double *)E, fc->I, fc->P, fc->cost,
                           fc->lp, fc->energy_out, fc->loss_out, fc->grad_out, cap);
    return e == cudaSuccess ? cudaGetLastError() : e;
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
                               const BlockConst &b, cudaStream_t st, const void *dtab) {
    auto k = !b.bytes ? k_adjoint<Real, R, 0> : (b.n16[7] ? k_adjoint<Real, R, 2>
                                                         : k_adjoint<Real, R, 1>);
    cudaError_t e = prep(k, sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.blocks, sh.S * sh.Ts, sh.smem, st>>>(
        p, o, s, c, sh, G, E, b, reinterpret_cast<const typename CT<Real>::T *>(dtab));
    return cudaGetLastError();
}

cudaError_t launch_onchip_adjoint(int c128, const OnchipShape &sh, const Program &p,
                                  const Observable &o, const SlotSource &s, const CostSource &c,
                                  double *G, double *E, cudaStream_t st, const BlockConst *bc,
                                  const void *dtab) {
    if (sh.blocks == 0) return cudaSuccess;
    BlockConst b = fit_const(sh, bc);
    b.n16[6] = 0;
    if (c128) {
        SVK_DISPATCH_R_C128(sh.R,
                            return (run_adjoint<double, RR>(sh, p, o, s, c, G, E, b, st, dtab)));
    }
    SVK_DISPATCH_R(sh.R, return (run_adjoint<float, RR>(sh, p, o, s, c, G, E, b, st, dtab)));
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
