// Launchers of the tile-pass kernels (hbm.cu): states in device memory.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "svk_types.h"

namespace svk {

// mats: [slots][groups][4] complex of the state's precision.
cudaError_t launch_group_mats(int c128, const Program &p, const SlotSource &src, void *mats,
                              cudaStream_t st);
// Zeroes the slot states and sets amplitude |ref> of each to 1.
cudaError_t launch_init_states(int c128, void *states, int n, const SlotSource &src,
                               cudaStream_t st);
uint32_t pass_fwd_smem(int c128, int t, int R, int G, int n_st, int n_ops);
uint32_t pass_rev_smem(int c128, int t, int R, int G, int n_u1, int n_st, int n_ops);
// pv: the program view of one pass (n = t, the pass's stages and thread bases);
// its ops are [op0, op0 + n_ops) of the plan's op array.
cudaError_t launch_pass_fwd(int c128, int R, const PassDesc &pd, const Program &pv, int op0,
                            int n_ops, int n, int n_slots, const void *mats, int G, void *states,
                            int blocks, cudaStream_t st);
cudaError_t launch_pass_rev(int c128, int R, const PassDesc &pd, const Program &pv, int op0,
                            int n_ops, int n, int n_slots, const void *mats, int G, void *psi,
                            void *lam, double *rho_g, int blocks, cudaStream_t st);
// out[r] = <psi_r|H|psi_r> (zeroed here first).
cudaError_t launch_expect_big(int c128, const Observable &o, int n, int n_rows,
                              const void *states, double *out, cudaStream_t st);
// lam = H psi and E[r] = <psi_r|H|psi_r> (E zeroed here first).
cudaError_t launch_apply_h_big(int c128, const Observable &o, int n, int n_rows, const void *psi,
                               void *lam, double *E, cudaStream_t st);
// slot_grads[b][param] += weight_b * gradient from rho_g[b][group][8] (zero it first).
cudaError_t launch_group_grads(int c128, const Program &p, const SlotSource &src,
                               const double *rho_g, const CostSource &cs, const double *E,
                               double *slot_grads, cudaStream_t st);

}  // namespace svk
