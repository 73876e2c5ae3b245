/*
 * sv_debug.h -- test hooks of libsv.so (not part of the computational API).
 *
 * sv_debug_plan compiles a circuit exactly as the GPU entry points do and
 * copies the resulting stage program to host buffers, so that the planner's
 * fusion, staging, index permutations and shared-memory address vectors can
 * be checked on a machine without a GPU.  Call it once with NULL buffers to
 * read the four counts (stages, ops, groups, members), then again with
 * buffers of counts[i] * sizes[i] bytes (sizes from sv_debug_sizes).
 */
#ifndef SV_DEBUG_H
#define SV_DEBUG_H

#include "sv.h"

#ifdef __cplusplus
extern "C" {
#endif

/* sizes[0..7] = sizeof of Stage, Op, Group, Member, TermGroup, Term, PassDesc, TilePass. */
void sv_debug_sizes(int32_t *sizes);

sv_status sv_debug_plan(const sv_circuit *circuit, int32_t reg_bits, int32_t fuse,
                        int32_t swz_bits, int32_t *counts, void *stages, void *ops,
                        void *groups, void *members);

/* The same for the tile passes of states in device memory: counts[4] also
 * receives the number of passes; `passes` gets counts[4] pass descriptors
 * (sizes[6] bytes each). */
sv_status sv_debug_passes(const sv_circuit *circuit, int32_t tile_bits, int32_t coalesce_bits,
                          int32_t reg_bits, int32_t fuse, int32_t swz_bits, int32_t *counts,
                          void *stages, void *ops, void *groups, void *members, void *passes);

/* The kernel descriptors of the tile passes exactly as the GPU entry points
 * build them for `dtype` (SV_C64 / SV_C128): counts[0..2] = groups, members,
 * passes; `tile_passes` gets counts[2] descriptors of sizes[7] bytes.
 * relabel: plan as the gradient and energy paths do (passes move qubits
 * into the low index bits); `layout` (int32 [n_qubits] or NULL) gets the bit
 * of the amplitude index that holds each qubit after the last pass. */
sv_status sv_debug_tile_passes(const sv_circuit *circuit, int32_t tile_bits, int32_t reg_bits,
                               int32_t fuse, int32_t dtype, int32_t relabel, int32_t *counts,
                               void *groups, void *members, void *tile_passes, int32_t *layout);

/* The tile passes of lambda = H psi: counts[0..4] = passes, groups, classes,
 * terms, rows.  In the exported pass records the four array pointers hold
 * the pass's first index into `groups`, `classes`, `terms` and `rows`. */
sv_status sv_debug_h_passes(const sv_pauli_sum *h, int32_t tile_bits, int32_t coalesce_bits,
                            int32_t *counts, void *passes, void *groups, void *classes,
                            void *terms, void *rows);

/* The bounded-wait path end to end: launches one block on `stream` that
 * waits `limit` times on an mbarrier nothing arrives on and then records the
 * expiry in the library's device error word, as a tensor-core pass whose
 * MMAs never completed would (the next sv_sync_status returns
 * SV_ERR_TIMEOUT).  limit: 1..2^20. */
sv_status sv_debug_wait_expiry(int32_t limit, sv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
