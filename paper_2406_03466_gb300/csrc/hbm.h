// Launchers of the tile-pass kernels (hbm.cu): states in device memory.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "svk_types.h"

namespace svk {

// mats: [slots][groups][4] complex of the state's precision.
cudaError_t launch_group_mats(int c128, const Program &p, const SlotSource &src, void *mats,
                              cudaStream_t st);
// Zeroes the slot states and sets amplitude |ref> of each to 1.
cudaError_t launch_init_states(int c128, void *states, int n, const SlotSource &src,
                               cudaStream_t st);
// Shared memory of one block of the forward / reverse kernels of pass P.
uint32_t tile_fwd_smem(int c128, const TilePass &P);
uint32_t tile_rev_smem(int c128, const TilePass &P, int bufs = 2);
// Forward pass P over n_slots states of n qubits (mats: [slots][G][4]).
// src (null: states) holds the pass's input; the output goes to states.
cudaError_t launch_tile_fwd(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *states, int64_t max_blocks, cudaStream_t st,
                            const void *src = nullptr);
// Reverse pass P on psi and lambda; adds the reduced matrices of its
// parametrised groups to rho_g[slot][G][8].  psi_src (null: psi) holds the
// psi the pass reads (a stored forward state); its output psi goes to psi
// unless write_psi is false (the next reverse pass restarts psi from a
// stored state, or this is the last one).
cudaError_t launch_tile_rev(int c128, const TilePass &P, int n, int n_slots, const void *mats,
                            int G, void *psi, void *lam, double *rho_g, int64_t max_blocks,
                            cudaStream_t st, const void *psi_src = nullptr,
                            bool write_psi = true);
// Codes a kernel writes to the library's device error word when a bounded
// device-side wait gives up (reported as SV_ERR_TIMEOUT by sv_sync_status).
constexpr int SV_DEVERR_MMA_WAIT = 1;
constexpr int SV_DEVERR_SWEEP_WAIT = 2;
// Raises kernel's dynamic shared-memory limit to `bytes` (limits only grow;
// no attribute change while a graph capture runs: fails instead).
cudaError_t allow_smem_attr(const void *kernel, uint32_t bytes);
// Forward pass P with every register stage applied as one dense 16 x 16
// complex block on the tensor cores (tc.cu; complex64, R = 4, t = 11 or 12).
// err: the device error word (bounded waits), or null.
uint32_t tile_fwd_tc_smem(const TilePass &P);
bool tile_fwd_tc_supported(int c128, const TilePass &P);
cudaError_t launch_tile_fwd_tc(const TilePass &P, int n, int n_slots, const void *mats, int G,
                               void *states, int64_t max_blocks, cudaStream_t st, int *err,
                               const void *src = nullptr);
// One block that waits `limit` times on an mbarrier nothing arrives on and
// records SV_DEVERR_MMA_WAIT: the bounded-wait path, for tests.
cudaError_t launch_wait_expiry(int *err, uint32_t limit, cudaStream_t st);
// Persistent sweeps of several problems (forward, or reverse with rev):
// tasks (device) in ticket order; ticket (device, zero) and done[n_tasks]
// (device, zero) are the scheduler's counters; every task uses the same tile
// shape (threads = 2^(t - R)); smem: the largest tile_sweep_smem over the
// tasks; blocks: at most the resident blocks (tile_sweep_blocks_per_sm x SMs).
// Launchers skip kernel attribute calls while a graph capture runs.
void set_capturing(bool on);
uint32_t tile_sweep_smem(int c128, bool rev, const TilePass &P);
int tile_sweep_blocks_per_sm(int c128, int R, bool rev, uint32_t smem, int threads);
cudaError_t launch_tile_sweep(int c128, int R, bool rev, const SweepTask *tasks, int n_tasks,
                              long long n_tickets, unsigned long long *ticket, unsigned int *done,
                              int *err, int blocks, int threads, uint32_t smem, cudaStream_t st);
// One tile pass of lambda = H psi (lam may be null: energies only); adds this
// pass's part of <psi|H|psi> to E[slot] (zero E before the first pass).
uint32_t tile_h_smem(int c128, const HPass &P);
cudaError_t launch_tile_h(int c128, const HPass &P, int n, int n_slots, const void *psi, void *lam,
                          double *E, int64_t max_blocks, cudaStream_t st);
// Data-driven circuit learning: js[r] = JS(target | |psi_r|^2) (zeroed here
// first) and lam_r = dJS/d|psi_r|^2 * psi_r elementwise.
cudaError_t launch_ddcl_lambda(int c128, int n, int n_rows, const void *psi, const double *target,
                               void *lam, double *js, cudaStream_t st);
// js[0] = JS divergence of one state's output distribution from `target`;
// D[j] = dJS/dP_theta(j) (device [2^n] doubles).
cudaError_t launch_ddcl_diag(int c128, int n, const void *psi, const double *target, double *D,
                             double *js, cudaStream_t st);
// out[r] = sum_j D[j] |psi_r(j)|^2 for n_rows states of 2^n amplitudes.
cudaError_t launch_diag_expect(int c128, int n, int n_rows, const void *states, const double *D,
                               double *out, cudaStream_t st);
// out[j] = in[j with bit b moved to bit qubit_of_bit[b]]: a 2^n table indexed
// by qubit values, rewritten for states whose bit b holds qubit qubit_of_bit[b].
cudaError_t launch_relayout(int n, const int32_t *qubit_of_bit, const double *in, double *out,
                            cudaStream_t st);
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
