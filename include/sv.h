/*
 * sv.h -- C ABI of the batched state-vector gradient library (libsv.so).
 *
 * The library simulates, as one batch on one GPU, the many slightly different
 * circuits a gradient needs: parameter-shift copies of a parametrised circuit,
 * taken over several reference states (multi-contracted VQE, paper Sec. 4.1)
 * or over many training inputs (data-driven circuit learning, Sec. 4.2), each
 * ending in the expectation value of a Pauli sum (Sec. 4.1, the paragraph
 * casting Eq. 2 as generic terms P_i weighed by c_i).  The paper spreads these
 * independent circuits over virtual QPUs (Sec. 3); here the same partition
 * runs over thread blocks of one GPU.
 *
 * Conventions (the paper fixes none of them):
 *   - qubit q is bit q of a basis index;
 *   - RX/RY/RZ(a) = exp(-i a P / 2);
 *   - CNOT(control -> target) flips the target bit when the control bit is 1;
 *   - amplitudes are interleaved (re, im); SV_C64 = 2 x float, SV_C128 = 2 x double;
 *   - a state batch is row-major [batch][2^n] amplitudes.
 *
 * Memory: pointers documented as "device" must be device memory of the
 * current CUDA device (e.g. from torch); pointers documented as "host" are
 * read during the call only and may be freed when it returns.  The library
 * never frees caller memory.  It owns only its plan cache and its per-stream
 * scratch buffers, released by sv_shutdown().
 *
 * Asynchrony: every call that takes a stream only enqueues work on it
 * (except where noted) and returns; outputs are valid once the stream has
 * reached that point.  Argument errors are reported synchronously; errors
 * of the CUDA runtime as SV_ERR_CUDA.  First use of a new circuit
 * structure builds and uploads its plan (synchronous, not capturable), so
 * make that first call before any CUDA graph capture.
 *
 * Errors: functions return sv_status; sv_last_error() gives a thread-local
 * text of the last failure.  Arguments are never silently clamped.
 *
 * Limits: n_qubits <= 30 (SV_C64) or <= 29 (SV_C128).
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *sv_stream_t;

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,         /* invalid argument: null pointer, size, gate, qubit index */
    SV_ERR_OOM = 2,         /* device memory for state or scratch could not be allocated */
    SV_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SV_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    SV_ERR_UNSUPPORTED = 5  /* well-formed request outside this build's limits */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Gate set.  ENC_* are the circuit-learning data encodings
 * Ry(arcsin x) and Rz(arccos x^2) with x read from the instance's input row. */
typedef enum {
    SV_GATE_RX = 0,
    SV_GATE_RY = 1,
    SV_GATE_RZ = 2,
    SV_GATE_CNOT = 3,
    SV_GATE_X = 4,
    SV_GATE_H = 5,
    SV_GATE_CZ = 6,
    SV_GATE_ENC_RY_ASIN = 7,
    SV_GATE_ENC_RZ_ACOS_SQ = 8
} sv_gate_op;

typedef struct {
    int32_t op;       /* sv_gate_op */
    int32_t target;   /* qubit the gate acts on (CZ: second qubit) */
    int32_t control;  /* CNOT / CZ control qubit; -1 otherwise */
    int32_t param;    /* RX/RY/RZ: index into theta, or -1 to use `angle`;
                         ENC_*: column of the instance's input row */
    double angle;     /* fixed rotation angle when param < 0 */
} sv_gate;

/* A circuit: gates in time order (host array). */
typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    int32_t n_params;    /* length of a theta row */
    int32_t input_dim;   /* length of an input row (0 if no ENC_* gates) */
    const sv_gate *gates;
} sv_circuit;

/* Pauli sum H = sum_t coeff[t] P_t (host arrays).  P_t has X on the qubits set
 * only in x_mask, Z on those set only in z_mask, Y on those set in both. */
typedef struct {
    int32_t n_qubits;
    int32_t n_terms;
    const uint64_t *x_mask;
    const uint64_t *z_mask;
    const double *coeff;
} sv_pauli_sum;

/* Planning knobs; all-zero (or a NULL pointer) selects the defaults. */
typedef struct {
    int32_t reg_bits;        /* amplitudes held per thread = 2^reg_bits (1..5); 0 = default */
    int32_t threads_per_block; /* 0 = default; else a multiple of 32 (whole warps) and of
                                  the threads per circuit, at most 512 */
    int32_t no_fusion;       /* 1 = apply every gate on its own (no 1-qubit gate fusion) */
    int32_t epilogue;        /* <H> epilogue: 0 = default, 1 = per Pauli term, 2 = per-X-group
                                diagonal tables (states of at most 13 qubits) */
    int32_t tile_bits;       /* 0 = states of at most 13 (complex64) / 12 (complex128) qubits
                                stay on chip, larger ones run as tile passes over device
                                memory with the default tile; > 0 forces tile passes of
                                2^tile_bits amplitudes (6..12) */
    int32_t coalesce_bits;   /* tile passes: the lowest qubits kept in every tile, so that
                                tiles are read and written in contiguous runs of
                                2^coalesce_bits amplitudes (1..tile_bits - 2); 0 = default
                                (4 complex64 / 3 complex128: 128-byte runs) */
    int32_t no_relabel;      /* tile passes of energies and gradients: 1 = every qubit keeps
                                its own index bit (by default a pass may move the qubits the
                                next pass needs into the low bits); states returned to the
                                caller always keep qubit order */
    int32_t tensor_blocks;   /* forward tile passes (complex64, reg_bits 4, tile_bits 11 or
                                12): 1 = apply every register stage's four fused groups as
                                one dense 16 x 16 complex block on the tensor cores
                                (tcgen05, 3xTF32 split, FP32 accumulation); 0 = FP32 FMAs
                                in registers.  sv_autotune may pick either. */
} sv_plan_opts;

/* ---------------------------------------------------------------- states */

typedef struct sv_state_s *sv_state;

/* Create a batch of `batch` states of n_qubits.  If dev_buf is non-NULL it
 * must hold dev_bytes >= batch * 2^n * sizeof(amplitude) bytes of device
 * memory, 256-byte aligned; it stays owned by the caller.  Otherwise the
 * library allocates (and sv_free releases) the buffer.  Contents are
 * undefined until written. */
sv_status sv_alloc(sv_state *out, int32_t n_qubits, int32_t batch, sv_dtype dtype,
                   void *dev_buf, size_t dev_bytes, sv_stream_t stream);
sv_status sv_free(sv_state state);
/* Device pointer, sizes and dtype of a state batch (any out-pointer may be NULL). */
sv_status sv_state_info(sv_state state, void **dev_ptr, int32_t *n_qubits, int32_t *batch,
                        sv_dtype *dtype);

/* --------------------------------------------------- forward simulation */

/* One row of a batch: which circuit, parameters, shift, inputs and reference. */
typedef struct {
    int32_t circuit;      /* index into the circuits array */
    int32_t theta_row;    /* row of theta used by the slot */
    int32_t shift_param;  /* parameter to shift, or -1 */
    int32_t input_row;    /* row of inputs used by ENC_* gates, or -1 */
    int64_t ref;          /* initial basis state |ref> */
    double shift;         /* added to theta[theta_row][shift_param] */
} sv_slot;

/* State-vector simulation (paper Sec. 4; Eq. 1's U(theta)|ref>) of n_slots
 * circuits into rows 0..n_slots-1 of `state`: row s = U_{circuit(s)}(theta
 * row + shift) |ref_s>.  circuits/slots: host.  theta: device
 * [rows][theta_stride] doubles; inputs: device [rows][input_stride] doubles
 * (NULL if no ENC_* gates).  Every circuit must have the state's n_qubits. */
sv_status sv_apply_circuit_batch(sv_state state, const sv_circuit *circuits, int32_t n_circuits,
                                 const sv_slot *slots, int32_t n_slots, const double *theta,
                                 int32_t theta_stride, const double *inputs,
                                 int32_t input_stride, const sv_plan_opts *opts,
                                 sv_stream_t stream);

/* Direct expectation values (Sec. 4.1: a simulator evaluates
 * <psi|P_i|psi> exactly): out[s] = sum_t c_t <psi_s|P_t|psi_s> for the first
 * n_rows rows of the batch.  out: device [n_rows] doubles.  Products are
 * taken in the state's precision, sums in FP64. */
sv_status sv_expect_pauli_sum(sv_state state, const sv_pauli_sum *h, int32_t n_rows,
                              double *out, sv_stream_t stream);

/* Shots of row `row` of a state: every qubit measured in the Z basis (the
 * bitstring counts a quantum backend returns, Sec. 3 and Sec. 4.2).  Shot s
 * is the first basis index b whose cumulative probability
 * sum_{b' <= b} |psi_b'|^2 (FP64) exceeds uniforms[s] times the total, so
 * the draw is fixed by the caller's uniforms (device [n_shots] in [0, 1)).
 * samples_out: device [n_shots] int64 basis indices (bit q = qubit q);
 * counts_out: device [2^n] int64 histogram of the samples, or NULL.  Uses
 * library scratch of 2^n / 1024 + 1 doubles. */
sv_status sv_sample(sv_state state, int32_t row, const double *uniforms, int64_t n_shots,
                    int64_t *samples_out, int64_t *counts_out, sv_stream_t stream);

/* ------------------------------------------------------------ gradients */

typedef enum {
    SV_COST_LINEAR = 0,  /* L = sum_i w_i E_i  (state averaging, Sec. 4.1: w_i = 1/R) */
    SV_COST_MSE = 1      /* L = (1/I) sum_i (E_i - y_i)^2  (circuit learning) */
} sv_cost;

/* A gradient problem: one circuit, one observable, n_instances instances.
 * Instance i starts from |refs[i]> and reads input row i. */
typedef struct {
    sv_dtype dtype;
    const sv_circuit *circuit;       /* host */
    const sv_pauli_sum *observable;  /* host */
    int32_t n_instances;
    const int64_t *refs;             /* host [n_instances] */
    const double *inputs;            /* device [n_instances][input_stride], or NULL */
    int32_t input_stride;
    sv_cost cost;
    const double *weights;           /* device [n_instances] (SV_COST_LINEAR) */
    const double *targets;           /* device [n_instances] (SV_COST_MSE) */
    const sv_plan_opts *opts;        /* may be NULL */
} sv_problem;

/* Energies of every instance, E_i = <ref_i| U^dag H U |ref_i> (Eq. 1 per
 * instance), and the cost, in one batched launch.  energy_out: device
 * [n_instances]; loss_out: device [1] or NULL.  Uses library scratch of
 * I doubles when loss_out is set. */
sv_status sv_energies(const sv_problem *problem, const double *theta, double *energy_out,
                      double *loss_out, sv_stream_t stream);

/* Every circuit of the parameter-shift batch, one expectation value each
 * (the per-circuit results the paper's execute() returns, Sec. 4.1): slot b
 * < I is instance b unshifted; slot I + 2kI + i is instance i with
 * theta_k + pi/2, slot I + (2k+1)I + i with theta_k - pi/2.  out: device
 * [(2P + 1) I] doubles.  One kernel launch. */
sv_status sv_param_shift_energies(const sv_problem *problem, const double *theta, double *out,
                                  sv_stream_t stream);

/* Parameter-shift gradient (Sec. 4.1: O(2 N_H N_theta) shifted circuits per
 * update; here the whole <H> per circuit, so (2P + 1) circuits per instance,
 * all in one batched launch for states on chip, followed by the assembly as a
 * programmatic dependent launch): dE_i/dtheta_k = 1/2 [E_i(theta + pi/2 e_k)
 * - E_i(theta - pi/2 e_k)], chained through the cost.  theta: device [P].
 * energy_out: device [n_instances] or NULL; loss_out: device [1] or NULL;
 * grad_out: device [P].  Uses library scratch of (2P+1) I doubles. */
sv_status sv_grad_param_shift(const sv_problem *problem, const double *theta,
                              double *energy_out, double *loss_out, double *grad_out,
                              sv_stream_t stream);

/* sv_grad_param_shift with host buffers, synchronous: copies theta (host
 * [P], any host memory) through library-owned pinned staging to the device,
 * runs the same fused launch, copies loss, gradient and instance energies
 * back in one transfer and waits for `stream` before returning.  For states
 * on chip the three steps are recorded once as a CUDA graph (keyed by every
 * pointer and launch argument they use) and later calls launch that graph;
 * the first call records it after running the steps, so make it outside any
 * stream capture of the caller's.
 * energy_host: [n_instances] or NULL; loss_host: [1] or NULL; grad_host: [P].
 * Uses (2P + 1 + I) doubles of pinned host and device staging per stream
 * besides the scratch of sv_grad_param_shift. */
sv_status sv_grad_param_shift_host(const sv_problem *problem, const double *theta_host,
                                   double *energy_host, double *loss_host, double *grad_host,
                                   sv_stream_t stream);

/* Adjoint (reverse-sweep) gradient, same result as sv_grad_param_shift:
 * lambda = H psi, then for each gate in reverse order the derivative
 * Im <lambda| G psi> of its generator G, psi <- U^dag psi, lambda <- U^dag lambda.
 * weights: device [n_instances] dL/dE_i; NULL derives them from the
 * problem's cost.  States that do not fit on chip run as tile passes over
 * device memory; their forward states are stored every `checkpoint_every`
 * passes and the reverse sweep restarts psi from each stored state instead
 * of carrying the rounding of the un-computation further (a reverse pass
 * followed by such a restart writes only lambda).  0 = every pass, else
 * every 2nd, if that many stored states still let all instances run at
 * once in free device memory, else every 4th.
 * Uses library scratch of I * P doubles, plus for device-memory states
 * (2 + checkpoints) states per instance processed at once (instances are
 * processed in groups that fit in free device memory). */
sv_status sv_grad_adjoint(const sv_problem *problem, const double *theta, const double *weights,
                          double *energy_out, double *loss_out, double *grad_out,
                          int32_t checkpoint_every, sv_stream_t stream);

/* sv_grad_adjoint with host buffers, synchronous (the adjoint counterpart of
 * sv_grad_param_shift_host): copies theta (host [P], any host memory)
 * through library-owned pinned staging to the device, runs the adjoint
 * gradient with the problem's cost (no external weights), copies loss,
 * gradient and instance energies back in one transfer and waits for
 * `stream` before returning.  energy_host: [n_instances] or NULL;
 * loss_host: [1] or NULL; grad_host: [P].  checkpoint_every as for
 * sv_grad_adjoint.  Uses (2P + 1 + I) doubles of pinned host and device
 * staging per stream besides the scratch of sv_grad_adjoint. */
sv_status sv_grad_adjoint_host(const sv_problem *problem, const double *theta_host,
                               double *energy_host, double *loss_host, double *grad_host,
                               int32_t checkpoint_every, sv_stream_t stream);

/* The plain form, for comparison only: one circuit at a time, one kernel
 * launch per gate and per Pauli term, complex128 state in device memory,
 * parameter shift as above.  Host-synchronous per circuit batch. */
sv_status sv_grad_param_shift_plain(const sv_problem *problem, const double *theta,
                                    double *energy_out, double *loss_out, double *grad_out,
                                    sv_stream_t stream);

/* Bytes of the fixed device array used by sv_grad_param_shift_noalloc. */
#define SV_NOALLOC_SCRATCH_BYTES (8u << 20)

/* The same result as sv_grad_param_shift, without allocating anything.  (The
 * paper has no counterpart: this is a deployment variant of the library.)
 *
 * For callers that cannot let a library call cudaMalloc: their device memory
 * belongs to another allocator that must account for every byte (a
 * framework's caching allocator), or their running loop must never hit
 * cudaMalloc's implicit device-wide synchronisation.  Instead of the
 * library's allocated caches and scratch, the call keeps its compiled plan,
 * observable, references and per-circuit energies in one file-scope device
 * array of SV_NOALLOC_SCRATCH_BYTES (8 MiB), which every GPU that loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it; make that
 * first call before any stream capture.  After cudaDeviceReset, call
 * sv_shutdown() before the next call, which then looks the address up again
 * in the new context.  Every call re-plans on the host and copies the plan
 * from pageable host memory into the array, so the call waits for work
 * already queued on `stream`, and it cannot be captured into a CUDA graph:
 * on a capturing stream it returns SV_ERR_UNSUPPORTED and enqueues nothing.
 * It runs the on-chip engine only: at most 13 qubits for SV_C64 and 12 for
 * SV_C128 (larger problems return SV_ERR_UNSUPPORTED naming this limit).  All calls share the one array and it keeps
 * the last call's contents; nothing in it needs to start at zero (every
 * value is written before it is read).  Calls that overlap on the GPU
 * (different streams, or other threads) race on the array: serialise them.
 * Problems whose plan, references and (2P + 1) I + I doubles do not fit are
 * rejected with SV_ERR_UNSUPPORTED and a message giving both sizes.
 * Arguments and outputs as for sv_grad_param_shift. */
sv_status sv_grad_param_shift_noalloc(const sv_problem *problem, const double *theta,
                                      double *energy_out, double *loss_out, double *grad_out,
                                      sv_stream_t stream);

/* A contiguous segment of the parameter-shift batch: the energies of slots
 * [slot_begin, slot_begin + n_slots) in the order sv_param_shift_energies
 * uses (every instance unshifted, then per parameter k: +pi/2 for every
 * instance, -pi/2 for every instance).  This is the paper's split of the
 * vector of circuits into one segment per virtual QPU (Sec. 4.1): each
 * rank computes its segment, an allgather assembles the batch, and
 * sv_param_shift_combine finishes the gradient.  out: device [n_slots]. */
sv_status sv_param_shift_energies_range(const sv_problem *problem, const double *theta,
                                        int32_t slot_begin, int32_t n_slots, double *out,
                                        sv_stream_t stream);
/* The parameter-shift combination of a whole batch of energies (device
 * [(2P+1) I], the order above): instance energies, cost and gradient, as
 * sv_grad_param_shift returns them.  Any output but grad_out may be NULL. */
sv_status sv_param_shift_combine(const sv_problem *problem, const double *energies,
                                 double *energy_out, double *loss_out, double *grad_out,
                                 sv_stream_t stream);

/* Data-driven circuit learning (Sec. 4.2, Eq. 3): the Jensen-Shannon
 * divergence JS(P | P_theta) of the circuit's output distribution
 * P_theta(b) = |<b|psi>|^2 (all qubits measured in the Z basis) from the
 * target P, and its gradient by the adjoint sweep: dJS/dP_theta(b) =
 * 1/2 log(P_theta(b)/M(b)), M = (P + P_theta)/2, so dJS/dtheta is the
 * gradient of <psi| diag(dJS/dP_theta) |psi> with the diagonal held fixed.
 * The problem's circuit, dtype, refs (one instance), inputs and opts are
 * used; its observable and cost are ignored.  Runs as tile passes at every
 * size (n >= 7).  target: device [2^n] doubles (normalised); js_out: device
 * [1]; grad_out: device [P]; theta: device [P]. */
sv_status sv_grad_ddcl(const sv_problem *problem, const double *theta, const double *target,
                       double *js_out, double *grad_out, sv_stream_t stream);

/* The same gradient by the paper's parameter-shift rule (Sec. 4.2: 2 N_theta
 * circuits per update): P_theta(b) is the expectation of the projector
 * |b><b|, so dP_theta(b)/dtheta_k = 1/2 [P_{theta+pi/2 e_k}(b) -
 * P_{theta-pi/2 e_k}(b)] and dJS/dtheta_k = 1/2 [<D>_{k+} - <D>_{k-}] with
 * D = diag(dJS/dP_theta) taken from the unshifted circuit.  Runs the 2P + 1
 * circuits as tile passes over device memory in chunks that fit; arguments
 * and outputs as for sv_grad_ddcl.  Uses library scratch of (2P + 2 + 2^n)
 * doubles. */
sv_status sv_grad_ddcl_param_shift(const sv_problem *problem, const double *theta,
                                   const double *target, double *js_out, double *grad_out,
                                   sv_stream_t stream);

/* Adjoint gradients of several problems at once: circuits of different qubit
 * counts and depths whose states take the tile path (14..30 qubits; all
 * problems share the dtype and the tile shape), each with its own
 * observable, instances, theta and outputs.  The forward sweeps of all
 * problems run as one persistent launch, and so do the reverse sweeps: every
 * pass of every problem is cut into chunks of tiles that take tickets level
 * by level (pass k of every problem before pass k + 1), and a block runs a
 * chunk once the same problem's previous pass has completed every chunk
 * (a bounded wait: on expiry the launch records a device error that
 * sv_sync_status reports as SV_ERR_TIMEOUT), so problems of different depth
 * never wait for one another at a pass boundary.  The whole sequence (group
 * matrices, |ref>, forward sweep, lambda = H psi, reverse sweep, gradients)
 * is captured into one CUDA graph per configuration (the problems'
 * structures and every pointer), replayed by a single graph launch on
 * `stream`.  The first call
 * for a configuration plans, allocates, runs eagerly and captures
 * (host-synchronous); later calls only launch the graph.  No checkpoints.
 * theta[j]: device [P_j]; energy_out[j]: device [I_j] or NULL; loss_out[j]:
 * device [1] or NULL; grad_out[j]: device [P_j].  Arrays of n_problems host
 * pointers.  SV_ERR_OOM when the states of all problems do not fit. */
sv_status sv_grad_adjoint_multi(const sv_problem *problems, int32_t n_problems,
                                const double *const *theta, double *const *energy_out,
                                double *const *loss_out, double *const *grad_out,
                                sv_stream_t stream);

/* How a circuit will run for a state precision and options: on_chip = 1 when
 * the whole state stays in one block's shared memory, else the number of tile
 * passes over device memory and their tile size (2^tile_bits amplitudes), as
 * the energy and gradient entry points plan them (relabeling passes unless
 * opts->no_relabel; sv_apply_circuit_batch plans with no_relabel set);
 * n_stages: register stages of the program; n_groups: fused single-qubit
 * groups.  Host-only (plans the circuit, launches nothing).  Any out-pointer
 * may be NULL. */
sv_status sv_plan_info(const sv_circuit *circuit, sv_dtype dtype, const sv_plan_opts *opts,
                       int32_t *on_chip, int32_t *n_passes, int32_t *tile_bits,
                       int32_t *n_stages, int32_t *n_groups);

/* How lambda = H psi and <H> run for states that take the tile path: the
 * number of tile passes over device memory and their tile size (2^tile_bits
 * amplitudes).  Host-only.  Any out-pointer may be NULL. */
sv_status sv_h_plan_info(const sv_pauli_sum *observable, sv_dtype dtype, int32_t *n_passes,
                         int32_t *tile_bits);

/* Phase timing of the adjoint gradient of states in device memory (the
 * forward tile passes, lambda = H psi, the reverse tile passes), taken with
 * CUDA events on the call's stream.  sv_phase_timing(1) turns it on for the
 * current device (it adds event records to every such call); after a call,
 * sv_last_phase_ms synchronizes on its events and returns the milliseconds
 * of each phase summed over the call's chunks of instances, or
 * SV_ERR_ARG when no timed call has run since timing was turned on. */
sv_status sv_phase_timing(int32_t on);
sv_status sv_last_phase_ms(float *forward_ms, float *h_ms, float *reverse_ms);

/* What the last adjoint gradient of states in device memory (sv_grad_adjoint,
 * sv_grad_adjoint_host or sv_grad_ddcl on the tile path of the current
 * device) did: the checkpoint interval it used (1, 2 or 4) and the
 * algorithmic bytes of its reverse tile passes (per pass psi, or its stored
 * state, and lambda read, lambda written, and psi written unless the next
 * reverse pass restarts from a stored state; summed over the call's chunks
 * of instances).  Both are 0 after an adjoint that ran on chip.  Host-only:
 * reads values the host recorded when it launched the passes.  Any
 * out-pointer may be NULL. */
sv_status sv_last_adjoint_info(int32_t *checkpoint_every, int64_t *reverse_bytes);

/* ------------------------------------------------------------- autotune */

/* Times the launch shapes (register bits 1..4, 32..512 threads per block) of
 * the batched parameter-shift energy kernel (kinds bit 1) and of the adjoint
 * kernel (kinds bit 2) on this problem and remembers the fastest per problem
 * structure; later calls whose opts leave reg_bits and threads_per_block at
 * zero use it.  For states in device memory (tile passes) it times tile
 * shapes instead — 2^t-amplitude tiles with R register bits, t in 9..12 —
 * for the instance energies (bit 1) and the adjoint gradient (bit 2), and
 * later calls whose opts leave tile_bits and reg_bits at zero use them.
 * Host-synchronous: launches and times kernels on `stream`, so do not call
 * it during stream capture.  theta: device [P]. */
sv_status sv_autotune(const sv_problem *problem, const double *theta, int32_t kinds,
                      sv_stream_t stream);
/* The remembered shape for kind 1 (parameter-shift energies; instance
 * energies for tile passes) or 2 (adjoint).  For tile passes
 * threads_per_block is 2^(tile_bits - reg_bits). */
sv_status sv_tuned_shape(const sv_problem *problem, int32_t kind, int32_t *reg_bits,
                         int32_t *threads_per_block, float *microseconds);
/* The tile shape sv_autotune chose for a problem whose states live in device
 * memory (kind 1 = energies, 2 = adjoint): tile bits, register bits, whether
 * the forward passes run as tensor-core blocks (sv_plan_opts.tensor_blocks),
 * and the time of the best call.  Any out-pointer may be NULL. */
sv_status sv_tuned_tile(const sv_problem *problem, int32_t kind, int32_t *tile_bits,
                        int32_t *reg_bits, int32_t *tensor_blocks, float *microseconds);

/* ----------------------------------------------------------------- misc */

const char *sv_status_string(sv_status status);
/* Thread-local description of the last failed call (empty if none). */
const char *sv_last_error(void);
/* Synchronize `stream` and report any pending CUDA error as a status.  A
 * kernel whose bounded device-side wait gave up (the tensor-core passes wait
 * for their MMAs at most about 2^22 times) records that in the library's
 * device error word; this call reports it as SV_ERR_TIMEOUT (and clears
 * it): the results of the calls since the last check are then invalid,
 * while the CUDA context stays usable. */
sv_status sv_sync_status(sv_stream_t stream);
/* Release plan caches and scratch on every device, and forget the device
 * addresses that sv_grad_param_shift_noalloc looked up. */
sv_status sv_shutdown(void);
int32_t sv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_H */
