/*
 * qsgb.h -- C ABI of the GB300 (sm_103a) Schroedinger-style state-vector
 * simulator: fused k-qubit gates applied to a dense 2^n complex state.
 *
 * Source of the operations: Fatima & Markov, "Faster Schroedinger-style
 * simulation of quantum circuits" (arXiv:2008.00216).
 *   - state: 2^n complex amplitudes alpha_j, computation starts from
 *     |0...0> (Section 2); all amplitudes are kept (strong simulation).
 *   - gate: a 2^q x 2^q unitary on qubits i_0..i_{q-1}, applied in place to
 *     the 2^(n-q) disjoint sets of 2^q amplitudes (Section 3).
 *   - clustering / reordering of commuting gates before simulation into a
 *     simulation plan (Sections 4.2 and 4.5, Eq. 2).
 *   - norm check with robust accumulation (Section 4.1).
 *
 * Conventions (every entry point):
 *   - qubit q is bit q of the amplitude index (qubit 0 = least significant).
 *   - a k-qubit matrix is 2^k x 2^k, row-major, complex entries interleaved
 *     (re, im) as doubles, in Kronecker order with qubits[0] the MOST
 *     significant local bit (Section 2's CNOT lists the control first).
 *     So kron(A, B) on {a, b} equals A on a followed by B on b.
 *   - matrices are always FP64 host memory and are copied before return.
 *   - device state: interleaved complex64 (QS_C64: float re, im) or
 *     complex128 (QS_C128), the layout of torch.complex64/complex128.
 *   - every call returns a status and never aborts, traps or asserts;
 *     arguments are checked on the host before any launch.  On failure,
 *     qs_last_error() returns a message for the calling thread.
 *   - work is enqueued on the state's CUDA stream and is asynchronous,
 *     except calls that return host values (qs_amplitudes, qs_norm,
 *     qs_expectation, qs_adjoint_gradient, qs_batch_run's results), which
 *     synchronise that stream.
 *   - objects are not thread-safe; use one object per thread or lock.
 */
#ifndef QSGB_H
#define QSGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qs_status {
    QS_OK = 0,
    QS_ERR_ARG = 1,          /* invalid argument (null, range, shape, alignment) */
    QS_ERR_OOM = 2,          /* device or host allocation failed / would not fit */
    QS_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has details) */
    QS_ERR_UNSUPPORTED = 4,  /* valid request this build does not implement */
    QS_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    QS_ERR_STATE = 6         /* object in the wrong state for this call */
} qs_status;

typedef enum qs_dtype { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Arithmetic of dense fused gates with k >= 5 on a complex64 state.  FP32 is
 * plain FP32 on the CUDA cores; the others run the 2^k x 2^k complex
 * product on the tensor cores (tcgen05) with FP32 accumulation: TF32
 * operands, split 3xTF32 (hi*hi + hi*lo + lo*hi), split 3xBF16, or split
 * 3xFP16 (IEEE half parts, 11-bit significands like TF32, at the 16-bit
 * MMA rate; every set of amplitudes and the gate are scaled by powers of
 * two into FP16's range first, so any finite state is accepted).
 * Ignored for complex128 states (always FP64-accurate arithmetic). */
typedef enum qs_precision {
    QS_PREC_FP32 = 0,
    QS_PREC_TF32 = 1,
    QS_PREC_3XTF32 = 2,
    QS_PREC_3XBF16 = 3,
    QS_PREC_3XFP16 = 4
} qs_precision;

/* Kind of a (fused) gate, from its exact FP64 entries. */
typedef enum qs_gate_kind {
    QS_GATE_DENSE = 0,
    QS_GATE_DIAGONAL = 1,   /* only the diagonal is nonzero */
    QS_GATE_MONOMIAL = 2    /* one nonzero per row and column (permutation with phases) */
} qs_gate_kind;

typedef struct qs_state qs_state;
typedef struct qs_circuit qs_circuit;
typedef struct qs_plan qs_plan;
typedef struct qs_pauli_sum qs_pauli_sum;

/* Planner and kernel options (qs_options_default fills the defaults).
 *   k_max       : largest fused gate, 1..6 (qs_fuse's bound).
 *   tile_qubits : qubits held per shared-memory tile, 0 = automatic;
 *                 otherwise 6..13 (c64) / 6..12 (c128).
 *   use_tile    : 1 = group consecutive gates on tile qubits into one pass.
 *   precision   : qs_precision for dense k >= 5 gates on complex64.
 *   fuse        : 1 = run qs_fuse(k_max) inside qs_plan_create.
 *   inject_wait_timeout : testing only, batches: 1 = the last pass of the
 *                 last wide circuit waits for a count that is never reached,
 *                 so its bounded device wait runs out (~2 s) and
 *                 qs_batch_sync reports QS_ERR_TIMEOUT.  0 in normal use.
 *   diag_clusters : 1 = cluster gates of a kind (Sections 4.2, 4.5):
 *                 diagonal gates with diagonal gates, in clusters of any
 *                 width (one wide diagonal pass each, pass kind 6), the
 *                 other gates with each other up to k_max.  0 (default) =
 *                 fuse any gates while their qubits fit k_max.
 *   fusion_effort : search behind each fused block (Section 4.5's scan,
 *                 best-first).  1 (default): each candidate qubit set is
 *                 scored by its completion with a one-level lookahead at
 *                 the first step (fewer blocks; tens of ms for ~1000 gates);
 *                 0: greedy completion only (a few ms).
 *   inject_mma_timeout : testing only, tensor-core passes of a plan: 1 = in
 *                 the first thread block, one producer warp withholds its
 *                 "operand ready" arrival for the first tile, so the MMA
 *                 issuer's bounded wait runs out (~2 s); the block stops
 *                 its other roles, frees its tensor memory and exits, and
 *                 qs_state_sync reports QS_ERR_TIMEOUT.  0 in normal use.
 *   tensor_tiles : 3xFP16 plans: 1 = group consecutive 6-qubit blocks whose
 *                 qubits (with qubits 0 and 1) fit 12 into tensor tile
 *                 passes of up to two blocks each (one HBM round trip for
 *                 both).  0 (default) = one round trip per block.  */
typedef struct qs_options {
    int k_max;
    int tile_qubits;
    int use_tile;
    int precision;
    int fuse;
    int inject_wait_timeout;
    int diag_clusters;
    int fusion_effort;
    int inject_mma_timeout;
    int tensor_tiles;
    int reserved[3];
} qs_options;

const char* qs_version(void);
const char* qs_status_string(qs_status s);
/* Message of the last failed call on this thread ("" if none). */
const char* qs_last_error(void);
qs_status qs_options_default(qs_options* opt);

/* ------------------------------------------------------------------ state */

/* Allocate a library-owned device state of 2^n amplitudes (1 <= n <= 36)
 * on the current device, initialised to |0...0> (Section 2).  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  QS_ERR_OOM if the free
 * device memory cannot hold it. */
qs_status qs_state_create(int n, qs_dtype dt, void* stream, qs_state** out);

/* Wrap caller-owned device memory (e.g. a torch tensor) of 2^n amplitudes.
 * `device_ptr` must be 16-byte aligned; the caller keeps it alive until
 * qs_state_destroy.  The contents are left as they are. */
qs_status qs_state_wrap(void* device_ptr, int n, qs_dtype dt, void* stream, qs_state** out);

/* Free the handle (and the amplitudes if library-owned).  NULL is a no-op. */
qs_status qs_state_destroy(qs_state* s);

qs_status qs_state_set_stream(qs_state* s, void* stream);
qs_status qs_state_info(const qs_state* s, int* n, qs_dtype* dt, void** device_ptr);

/* |index> (all amplitudes 0 except alpha_index = 1). */
qs_status qs_state_init_basis(qs_state* s, uint64_t index);

/* H on every qubit of |0...0>: every amplitude 2^(-n/2).  Section 4.5 notes
 * that the initial Hadamard layer can be replaced by this initialisation. */
qs_status qs_state_init_uniform(qs_state* s);

/* Wait for the state's stream; QS_ERR_TIMEOUT if a bounded device-side wait
 * (tensor-core pipeline) gave up since the last check (the flag is then
 * cleared).  qs_norm and qs_amplitudes perform the same check. */
qs_status qs_state_sync(qs_state* s);

/* Device-to-device copy of all amplitudes; n and dtype must match. */
qs_status qs_state_copy(qs_state* dst, const qs_state* src);

/* ------------------------------------------------------------------ gates */

/* Apply one k-qubit gate (1 <= k <= 6, distinct qubits < n) in place
 * (Section 3).  m: 2^k x 2^k FP64 complex, interleaved, Kronecker order. */
qs_status qs_apply_gate(qs_state* s, const int* qubits, int k, const double* m);

/* --------------------------------------------------------------- circuits */

qs_status qs_circuit_create(int n, qs_circuit** out);
qs_status qs_circuit_destroy(qs_circuit* c);

/* Append a fixed gate (copied). */
qs_status qs_circuit_add(qs_circuit* c, const int* qubits, int k, const double* m);

/* Append `count` fixed gates at once (copied), in order: gate i has ks[i]
 * qubits, the next ks[i] entries of `qubits`, and the next 2 * 4^ks[i]
 * doubles of `mats` (its matrix as for qs_circuit_add).  Every gate is
 * checked first; on an error nothing is appended (QS_ERR_ARG). */
qs_status qs_circuit_add_gates(qs_circuit* c, int count, const int* ks, const int* qubits, const double* mats);

/* Append a parametrised gate exp(-i theta P / 2) with P the Pauli string
 * `paulis` ("X", "ZZ", "XY", ... ; paulis[i] acts on qubits[i]), parameter
 * index `param` >= 0 and current value `theta`. */
qs_status qs_circuit_add_rotation(qs_circuit* c, const int* qubits, int k,
                                  const char* paulis, int param, double theta);

/* Set every parameter (theta[p] for p < num) and rebuild rotation matrices. */
qs_status qs_circuit_set_params(qs_circuit* c, const double* theta, int num);

qs_status qs_circuit_size(const qs_circuit* c, int* n, int* num_gates, int* num_params);

/* Read back gate `index`: k, qubits (up to 6 ints), matrix (up to
 * 2*4^k doubles) and its qs_gate_kind.  Any output pointer may be NULL. */
qs_status qs_circuit_gate(const qs_circuit* c, int index, int* k, int* qubits,
                          double* m, int* kind);

/* Gate fusion with commuting reorder (Sections 4.2 and 4.5, Eq. 2): scan the
 * gates in order; start a block at the first unplaced gate and pull each
 * later gate into it when every gate skipped so far commutes with it
 * (disjoint qubits, or both diagonal) and the block's qubit set stays
 * within k_max (1..6).  Block matrices are the FP64 products, each block is
 * classified dense / diagonal / monomial.  Rotation parameters are dropped:
 * the result is a fixed circuit.  *out is a new circuit owned by the caller. */
qs_status qs_fuse(const qs_circuit* in, int k_max, qs_circuit** out);

/* ------------------------------------------------------------------ plans */

/* Build an execution plan for circuits on states of c's n and dtype dt:
 * optional fusion, grouping into passes (shared-memory tile passes, strided
 * dense passes, diagonal / monomial passes, tensor-core passes), matrices
 * converted to the state's precision and uploaded to the device.  Uses the
 * current device; `opt` may be NULL for defaults (qs_options_default, with
 * k_max 3 for complex128: blocks its float-float register tile applies). */
qs_status qs_plan_create(const qs_circuit* c, qs_dtype dt, const qs_options* opt, qs_plan** out);
qs_status qs_plan_destroy(qs_plan* p);

/* Number of passes (full HBM round trips) and kernel launches of the plan,
 * and the passes of each kind (array of 8: tile, dense, diagonal, monomial,
 * tensor-core, dense-smem, wide diagonal, tensor tile; may be NULL).  A
 * tensor tile pass (3xFP16 plans) applies up to two 6-qubit blocks to
 * 12-qubit tiles held in shared memory, one HBM round trip for all. */
qs_status qs_plan_info(const qs_plan* p, int* num_passes, int* num_launches, int* per_kind);

/* Enqueue the plan on the state's stream.  n and dtype must match. */
qs_status qs_plan_execute(qs_state* s, const qs_plan* p);

/* Enqueue passes [first, first+count) only (count < 0: to the end); used to
 * time passes one by one.  Running every range in order equals execute.
 * Between passes the state may be stored with the index bits of qubit 0 and
 * one other qubit exchanged (runs of 6-qubit tensor-core passes keep qubit 0
 * out of their targets that way); each run, and so the plan, ends in the
 * standard order. */
qs_status qs_plan_execute_range(qs_state* s, const qs_plan* p, int first, int count);

/* Describe pass i: its kind (index as in qs_plan_info), qubits touched per
 * amplitude pass (k, or the tile's L), and gates applied in it. */
qs_status qs_plan_pass(const qs_plan* p, int i, int* kind, int* width, int* num_gates);

/* Fuse and run a circuit with the default options and the given precision.
 * A tensor-core mode on a complex64 state (n >= 12): 6-qubit blocks, fused
 * and run together -- a host thread runs the block search while this call
 * launches each block's pass (its own pass: no tile grouping) as soon as the
 * block is found, so the search overlaps the device passes (passes wait in
 * a window of up to 3 so that qubit 0 can be kept out of their targets); the
 * call returns after the last launch.  Otherwise: plan (k_max 4 for
 * complex64, 3 for complex128), execute, free the plan.
 * Asynchronous like qs_plan_execute: matrices are allocated and freed in the
 * state's stream order. */
qs_status qs_apply_circuit(qs_state* s, const qs_circuit* c, qs_precision prec);

/* ------------------------------------------------------------ read back */

/* Copy amplitudes [first, first+count) to host `out` as interleaved FP64
 * (2*count doubles).  Synchronises the state's stream. */
qs_status qs_amplitudes(const qs_state* s, uint64_t first, uint64_t count, double* out);

/* sum_j |alpha_j|^2 with per-thread compensated (two-float) accumulation
 * and FP64 cross-block sums (Section 4.1).  Synchronises the stream. */
qs_status qs_norm(const qs_state* s, double* out);

/* Allocation-free norm: sum_j |alpha_j|^2 of 2^n amplitudes at a raw device
 * pointer, for callers that cannot allocate device memory -- a process whose
 * GPU memory another allocator has reserved up front, an application with a
 * device-memory budget fixed at start-up, or code that must keep off the
 * driver's allocation path because cudaMalloc/cudaFree can synchronise the
 * device.  qs_norm needs a qs_state, whose creation allocates scratch; this
 * call allocates nothing.  The paper has no counterpart: it is an interface
 * addition, computing what qs_norm computes with the same kernels.
 *   device_amplitudes: 16-byte aligned, 2^n complex64/complex128 (dt).
 *   stream: cudaStream_t to run on; the call synchronises it.
 *   out: host double receiving the sum.
 * Scratch: a fixed device array of 4096 partial sums (plus a result slot,
 * about 32 KB) inside the library, held by every GPU that loads it until the
 * process exits.  A GPU that needs more partial sums than that (more than
 * 1024 SMs) gets QS_ERR_UNSUPPORTED.  Each call outside stream capture looks
 * up the array's device address (cudaGetSymbolAddress) with the current
 * device, so the address stays valid across a device reset; a call during a
 * capture reuses the address of the last uncaptured call on that device, so
 * make one call before any stream capture (a first call made during a
 * capture returns QS_ERR_STATE).  The amplitudes must be on the current
 * device.  All calls share the one
 * array and it keeps the last call's contents (each call overwrites every
 * entry it reads, so nothing needs clearing): calls whose work overlaps on
 * the GPU -- on different streams, or from several host threads -- race and
 * must be serialised by the caller. */
qs_status qs_norm_noalloc(const void* device_amplitudes, int n, qs_dtype dt, void* stream, double* out);

/* ------------------------------------------------- Schroedinger-Feynman */

/* Amplitudes <x|U|0...0> of circuit c by the paper's Schroedinger-Feynman
 * mode (Sections 1 and 6): the qubits in the bit mask part_a form half A,
 * the others half B; each gate across the cut (it must act on two qubits,
 * one in each half) is written as a sum of r <= 4 products X_k (x) Y_k
 * (elimination with full pivoting on the gate's realigned 4 x 4 matrix:
 * r = 2 for CZ, 4 for fSim), and every choice of one term per crossing gate
 * is a path.  Both halves of every path are simulated from |0...0> by the
 * batched kernel (one launch per half); then
 *   out[i] = sum over paths psi_A(path)[x_A] psi_B(path)[x_B],
 * x = indices[i], x_A / x_B its bits in each half, summed in FP64.
 *   dt: state precision of the half simulations.
 *   indices: count amplitude indices (host), each < 2^n.
 *   out: 2 * count doubles (host), interleaved (re, im).
 *   num_paths: if not NULL, receives the number of paths (also when
 *   count == 0: a way to cost a cut without simulating).
 * Each half has at most 30 qubits; at most 65536 paths (QS_ERR_UNSUPPORTED
 * otherwise).  Device memory: every path's two half states, allocated and
 * freed in `stream`'s order; the call synchronises `stream`. */
qs_status qs_sf_amplitudes(const qs_circuit* c, uint64_t part_a, qs_dtype dt, const uint64_t* indices,
                           uint64_t count, void* stream, double* out, uint64_t* num_paths);

/* ------------------------------------------------------------ observables */

qs_status qs_pauli_sum_create(int n, qs_pauli_sum** out);
qs_status qs_pauli_sum_destroy(qs_pauli_sum* h);
/* Add coeff * P with P = paulis[i] on qubits[i] ('I','X','Y','Z'), len <= n. */
qs_status qs_pauli_sum_add(qs_pauli_sum* h, double coeff, const int* qubits,
                           const char* paulis, int len);

/* <psi|H|psi> (real part), FP64 accumulation.  Synchronises the stream. */
qs_status qs_expectation(const qs_state* s, const qs_pauli_sum* h, double* out);

/* out = H psi (states of equal n and dtype, distinct memory). Asynchronous. */
qs_status qs_apply_pauli_sum(const qs_state* psi, const qs_pauli_sum* h, qs_state* out);

/* ------------------------------------------------------------ gradients */

/* Adjoint (reverse state-vector) gradient of E(theta) = <0|U^dag H U|0> for a
 * circuit whose parametrised gates are exp(-i theta_p P / 2) (each
 * parameter used by one gate).  Sets the circuit's parameters to theta,
 * runs U on `psi` from |0...0>, forms lambda = H psi in `lam`, E = <psi|lam>,
 * then walks the gates backwards: at each parametrised gate
 * dE/dtheta = Im <lambda|P|psi>, then psi <- U_l^dag psi and
 * lambda <- U_l^dag lambda (no intermediate states stored).  Gates that
 * commute pairwise are taken as one stage: all their gradients from the same
 * (psi, lambda), then their inverse as fused passes.  Complex64 states of 12
 * or more qubits undo whole fused 6-qubit blocks instead: every gradient of
 * a block follows from the 64 x 64 matrix sum_s psi_s lambda_s^dag over its
 * qubits (tensor cores) and the block's gates; its scratch (up to 64 KB per
 * SM for each block with parameters) comes from a memory pool of the library
 * that keeps its reservation until the process exits.  `psi` and `lam` are
 * work states with the circuit's n and a common dtype and stream (their
 * contents on return are unspecified); grad has num_params entries (host).
 * Synchronises the states' stream only. */
qs_status qs_adjoint_gradient(qs_circuit* c, const double* theta, int num_params,
                              const qs_pauli_sum* h, qs_state* psi, qs_state* lam,
                              double* energy, double* grad);

/* Many adjoint gradients at once (the differentiation workload's batched
 * form): gradient i is qs_adjoint_gradient(circuits[i], thetas[i],
 * num_params[i], hams[i], psi[i], lam[i], &energies[i], grads[i]).  Host
 * threads plan the gradients concurrently and each gradient's work runs on
 * the stream of its own states, so gradients whose states have distinct
 * streams overlap on the GPU.  Every circuit and every state must be a
 * distinct object (QS_ERR_ARG otherwise); all host arrays have `count`
 * entries.  Returns the first failing gradient's status (message names its
 * index); the others still run.  Synchronises every stream used. */
qs_status qs_adjoint_gradient_batch(int count, qs_circuit* const* circuits, const double* const* thetas,
                                    const int* num_params, const qs_pauli_sum* const* hams,
                                    qs_state* const* psi, qs_state* const* lam, double* energies,
                                    double* const* grads);

/* ------------------------------------------------------------ batches */

typedef struct qs_batch qs_batch;

/* Plan many circuits (any mix of 1..30 qubits) for one persistent launch.
 * Each circuit starts from |0...0>.  Circuits with n <= tile_qubits (13 for
 * complex64, 12 for complex128 by default) run entirely inside one thread
 * block's shared memory; wider ones run as shared-memory tile passes whose
 * work items are claimed from a device queue (pass p of a circuit waits,
 * bounded, for its passes < p).  `opt` may be NULL (k_max 3); k_max <= 4.
 * The circuits are copied; they may be destroyed afterwards.  Extends the
 * paper's Section 3 simulation to many circuits at once (its introduction
 * cites VQE-style workloads that run numerous circuits in sequence). */
qs_status qs_batch_create(const qs_circuit* const* circuits, int count, qs_dtype dt,
                          const qs_options* opt, qs_batch** out);

/* offsets[0..count]: amplitude offset of each circuit's state in the state
 * buffer; offsets[count] = total amplitudes the buffer must hold. */
qs_status qs_batch_layout(const qs_batch* b, uint64_t* offsets);

qs_status qs_batch_info(const qs_batch* b, int* items, int* passes, int* gates, int* grid);

/* Run the whole batch on `stream` into `device_states` (16-byte aligned,
 * offsets from qs_batch_layout): one CUDA-graph launch (counter reset +
 * persistent kernel), captured on first use for that buffer.  Async. */
qs_status qs_batch_run(qs_batch* b, void* device_states, void* stream);

/* Wait for the last run; QS_ERR_TIMEOUT if a device-side wait gave up. */
qs_status qs_batch_sync(qs_batch* b);
qs_status qs_batch_destroy(qs_batch* b);

/* Time k_max in {2,3,4} x two tile widths on this batch (runs it 2x each)
 * and return the fastest options in *best. */
qs_status qs_batch_autotune(const qs_circuit* const* circuits, int count, qs_dtype dt,
                            void* device_states, void* stream, qs_options* best);

#ifdef __cplusplus
}
#endif

#endif /* QSGB_H */
