// Launch wrappers of the CUDA kernels (host-callable, C++ linkage).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sv.h"
#include "svk_types.h"

namespace svk {

// Where each circuit slot takes its reference, parameters, shift and inputs.
enum SlotMode : int32_t {
    SLOTS_PARAM_SHIFT = 0,  // slot b < I: instance b unshifted; then per k: +pi/2 (all I), -pi/2 (all I)
    SLOTS_EXPLICIT = 1,     // sv_slot array
    SLOTS_INSTANCES = 2     // slot b = instance b, unshifted
};

struct SlotSource {
    int32_t mode;
    int32_t n_slots;
    int32_t n_instances;
    int32_t theta_stride;
    int32_t input_stride;
    int32_t slot_base;       // slot b of a launch is slot slot_base + b of the batch
    const int64_t *refs;     // per instance (modes 0, 2)
    const double *theta;     // [P] (modes 0, 2) or [rows][theta_stride] (mode 1)
    const double *inputs;    // per instance (modes 0, 2) or per row (mode 1)
    const sv_slot *slots;    // mode 1 (device copy)
    const int32_t *rows;     // mode 1: output row of each slot (NULL = slot index)
};

struct CostSource {
    int32_t cost;              // sv_cost
    int32_t n_instances;
    const double *ext_weights; // dL/dE_i supplied by the caller, or NULL
    const double *weights;     // SV_COST_LINEAR
    const double *targets;     // SV_COST_MSE
};

// Launch shape of an on-chip kernel and the carve-up of its dynamic shared
// memory: region base offsets per block and per-slot strides, in bytes.
struct OnchipShape {
    int32_t R;       // register bits (amplitudes per thread = 2^R)
    int32_t Ts;      // threads per slot = 2^(n-R)
    int32_t S;       // slots per block
    int32_t blocks;
    uint32_t smem;   // dynamic shared memory per block
    uint32_t off_lam, off_mats, off_rho, off_grad, off_rhow, off_red;
    uint32_t st_state, st_mats, st_rho, st_grad, st_rhow;
    uint32_t off_const, const_bytes;  // block-constant region (0 bytes = not staged)
};

// Block-constant arrays (program, observable, diagonal tables) that a block
// copies into its shared memory before it starts, so that the stage loop
// and the epilogue never wait on global memory.  Slot k: 0 stages, 1 ops,
// 2 groups, 3 members, 4 term groups, 5 terms, 6 diagonal tables, 7 thread
// bases of every stage.  Sizes are
// in 16-byte units; the global arrays are padded to whole 16-byte units.
constexpr int kBlockConst = 8;  // slot 7: per-thread stage bases
struct BlockConst {
    const uint4 *src[kBlockConst];
    uint32_t n16[kBlockConst];
    uint32_t off[kBlockConst];  // byte offset inside the block-constant region
    uint32_t base;              // byte offset of the region in dynamic shared memory
    uint32_t bytes;             // region size (0 = read everything from global memory)
};

// Shapes (or an error string) for the on-chip kernels; `const_bytes` of
// block-constant data are appended to the shared-memory layout when they fit.
const char *onchip_shape(int kind, int n, int n_groups, int n_params, int c128, int n_slots,
                         int reg_bits, int threads_per_block, OnchipShape *out,
                         int num_sms = 152, uint32_t const_bytes = 0);
enum OnchipKind { ONCHIP_ENERGY = 0, ONCHIP_STORE = 1, ONCHIP_EXPECT = 2, ONCHIP_ADJOINT = 3 };

// Gradient assembly launched behind the energy kernel (a programmatic
// dependent launch that waits for the energies).
struct FusedCombine {
    int32_t I, P;
    CostSource cost;
    double *lp;         // [I] scratch
    double *energy_out, *loss_out, *grad_out;
};

// dtab: diagonal tables of the observable ([groups][2^n] complex of the
// state's precision) or NULL for the per-term epilogue; fc: NULL or the
// gradient assembly that follows the energies.
cudaError_t launch_onchip_energy(int c128, const OnchipShape &sh, const Program &p,
                                 const Observable &o, const SlotSource &s, double *energies,
                                 cudaStream_t st, const void *dtab = nullptr,
                                 const FusedCombine *fc = nullptr, const BlockConst *bc = nullptr);
cudaError_t launch_build_dtable(int c128, const Observable &o, int n, void *out, cudaStream_t st);
cudaError_t launch_onchip_store(int c128, const OnchipShape &sh, const Program &p,
                                const SlotSource &s, void *states, cudaStream_t st);
cudaError_t launch_onchip_expect(int c128, const OnchipShape &sh, int n, int swz_bits,
                                 const Observable &o, const void *states, int n_rows,
                                 double *out, cudaStream_t st);
// dtab: the observable's diagonal tables (launch_build_dtable) in device
// memory, or null (lambda = H psi then sums each group's terms per amplitude).
cudaError_t launch_onchip_adjoint(int c128, const OnchipShape &sh, const Program &p,
                                  const Observable &o, const SlotSource &s, const CostSource &c,
                                  double *slot_grads, double *slot_energies, cudaStream_t st,
                                  const BlockConst *bc = nullptr, const void *dtab = nullptr);

cudaError_t launch_ps_combine(const double *E, int I, int P, const CostSource &c,
                              double *lprime_scratch, double *energy_out, double *loss_out,
                              double *grad_out, cudaStream_t st);
cudaError_t launch_adjoint_combine(const double *G, const double *E, int I, int P,
                                   const CostSource &c, double *energy_out, double *loss_out,
                                   double *grad_out, cudaStream_t st);

// Plain one-circuit-at-a-time complex128 kernels.
cudaError_t launch_plain_init(double2 *psi, int n, int64_t ref, cudaStream_t st);
cudaError_t launch_plain_u1(double2 *psi, int n, int q, const double2 m[4], cudaStream_t st);
cudaError_t launch_plain_cx(double2 *psi, int n, int c, int t, cudaStream_t st);
cudaError_t launch_plain_cz(double2 *psi, int n, int a, int b, cudaStream_t st);
cudaError_t launch_plain_term(const double2 *psi, int n, uint32_t x, uint32_t z, int phase,
                              double coeff, double *acc, cudaStream_t st);

}  // namespace svk
