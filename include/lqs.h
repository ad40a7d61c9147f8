/*
 * lqs.h -- C ABI of the GB300 state-vector gate engine.
 *
 * The engine applies quantum gates to a 2^n-amplitude state vector held in one
 * GPU's HBM, with kernels chosen by gate class and qubit index, after the
 * index-dependent, gate-specific strategy of arxiv 2508.13615 (Sec. 2):
 * every gate uses only the nonzero entries of its matrix, and how a gate runs
 * depends on which qubit indices it touches.  On one GPU the paper's
 * local/non-local split becomes "inside a shared-memory tile" versus "strided
 * HBM passes".
 *
 * Conventions
 *   - Qubit q is bit q of the amplitude index (stride 2^q).  The paper numbers
 *     qubits from 0 and pairs a gate on target q_T with the amplitude 2^q_T
 *     away (rank distance 2^(q_T-L), Sec. 2, Fig. 1a/1b), so qubit 0 is the
 *     least significant bit.
 *   - Amplitudes are interleaved complex numbers (re, im): complex64 is two
 *     float32, complex128 two float64.  The state is one contiguous array of
 *     2^n amplitudes, 256-byte aligned.
 *   - A gate's wires are listed control(s) first, target last (CNOT = {c, t},
 *     Toffoli = {c1, c2, t}).  A user matrix (U2: 2x2, U4: 4x4) is row-major
 *     interleaved complex128 on the host; its first listed wire is the most
 *     significant bit of the row/column index.
 *   - Gate definitions follow the public PennyLane operator definitions, which
 *     the paper's simulator extends (Sec. 1): RX/RY/RZ(t) = exp(-i t P / 2),
 *     PhaseShift(p) = diag(1, e^{ip}), Rot(a, b, c) = RZ(c) RY(b) RZ(a),
 *     ControlledPhaseShift(p) = diag(1, 1, 1, e^{ip}).
 *
 * Errors: every call returns LQS_OK (0) or a negative LQS_ERR_* code and never
 * throws across the ABI; lqs_last_error() returns a message for the calling
 * thread.  Arguments are validated before any work is enqueued: a call that
 * fails validation leaves the state untouched.
 *
 * Streams: every call on a state is enqueued on the CUDA stream given to
 * lqs_sv_alloc (a cudaStream_t; NULL = the legacy default stream) and is
 * asynchronous unless it returns host values (lqs_expval, lqs_norm2,
 * lqs_adjoint_grad, lqs_batch_run, lqs_sv_copy_to_host, lqs_sv_sync).
 *
 * Arithmetic: complex64 states use float32 gate arithmetic; complex128 states
 * use double-float arithmetic on the float32 pipes (two float32 per double,
 * about 2^-46 relative error per operation for magnitudes in [2^-80, 2^127),
 * absolute error below 2^-125 under it), because GB300's float64 units run at
 * a small fraction of its float32 rate.  In that mode amplitudes with
 * magnitude below 2^-103 are treated as zero and magnitudes must stay below
 * 2^127; LQS_ARITH_F64 selects native float64 instead.  Norms, expectation
 * values and gradient inner products accumulate in float64 for both dtypes.
 */
#ifndef LQS_ABI_H_INCLUDED
#define LQS_ABI_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LQS_API __attribute__((visibility("default")))
#else
#define LQS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define LQS_OK 0
#define LQS_ERR_ARG (-1)          /* invalid argument: wires, counts, sizes, null pointers      */
#define LQS_ERR_OOM (-2)          /* device memory could not be allocated                        */
#define LQS_ERR_CUDA (-3)         /* a CUDA call or kernel launch failed                         */
#define LQS_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up (the kernel returned)    */
#define LQS_ERR_UNSUPPORTED (-5)  /* the request is valid but not supported (no GPU, dtype ...)  */

typedef enum { LQS_C64 = 0, LQS_C128 = 1 } lqs_dtype;

/* Gate set: Pauli-X/Z and CNOT (Sec. 2, Sec. 3.1), Hadamard and controlled
 * phase / R_k (Sec. 3.2, Fig. 5a, Fig. 6a), parametrised rotations and
 * DoubleExcitation for variational circuits (Listing 1), Toffoli and CSWAP
 * (the 8x8 cases of Sec. 2), and generic 2x2 / 4x4 unitaries (the "general
 * approach" of Sec. 3.1).
 *   CSWAP: wires {c, a, b}: swaps a and b where c = 1.
 *   DoubleExcitation(theta): wires {w0, w1, w2, w3} (w0 the most significant
 *     bit of the 16x16 matrix); rotates the pair |0011>, |1100>:
 *     |0011> -> cos(theta/2)|0011> + sin(theta/2)|1100>,
 *     |1100> -> cos(theta/2)|1100> - sin(theta/2)|0011>; every other basis
 *     state is unchanged.  It runs as CNOTs from w0 to w1, w2, w3, X on w1,
 *     an RY(theta) on w0 controlled by w1, w2, w3, and the same CNOTs and X
 *     undone, so it takes the dense, permutation and fused kernels as they
 *     are; its gradient is that controlled RY's. */
typedef enum {
  LQS_X = 0, LQS_Y = 1, LQS_Z = 2, LQS_H = 3, LQS_S = 4, LQS_T = 5,
  LQS_RX = 6, LQS_RY = 7, LQS_RZ = 8, LQS_PHASE = 9, LQS_ROT = 10,
  LQS_CNOT = 11, LQS_CZ = 12, LQS_SWAP = 13, LQS_CPHASE = 14, LQS_CRY = 15,
  LQS_TOFFOLI = 16, LQS_U2 = 17, LQS_U4 = 18, LQS_CSWAP = 19, LQS_DOUBLE_EXCITATION = 20,
  LQS_NUM_GATES = 21
} lqs_gate;

/* c128 arithmetic selection (lqs_fuse_cfg.arith and lqs_set_arith). */
typedef enum { LQS_ARITH_AUTO = 0, LQS_ARITH_F64 = 1, LQS_ARITH_DF = 2 } lqs_arith;

typedef struct lqs_sv lqs_sv; /* opaque state-vector handle */

/* One gate of a circuit.  param_idx indexes the caller's parameter array
 * (first of the gate's parameters; -1 when the gate has none).  matrix: U2/U4
 * only, host pointer, row-major interleaved complex128, read during the call. */
typedef struct {
  int32_t gate;
  int32_t wires[4]; /* the gate's wires in order (unused entries ignored) */
  int32_t param_idx;
  int32_t inverse; /* nonzero: apply the adjoint U^dagger */
  const double* matrix;
} lqs_op;

/* coeff * prod_q sigma_q with sigma_q chosen by bit q of (x_mask, z_mask):
 * I = (0,0), X = (1,0), Z = (0,1), Y = (1,1). */
typedef struct {
  double coeff;
  uint64_t x_mask;
  uint64_t z_mask;
} lqs_pauli;

/* Fusion / tiling controls; all zero = automatic (autotuned per n and dtype). */
typedef struct {
  int32_t tile_qubits; /* k: qubits per shared-memory tile (2^k amplitudes), 0 = auto */
  int32_t low_qubits;  /* b: contiguous low qubits always in a tile (coalescing), 0 = auto */
  int32_t arith;       /* lqs_arith, c128 only */
  int32_t max_ops;     /* cap on gates per fused segment, 0 = no cap beyond the program size */
  int32_t tc_blocks;   /* complex64, n >= 12: a run of gates confined to qubits 0..4 whose dense weight
                          (4 per two-qubit dense gate, 1 per one-qubit dense gate, 1/4 per other gate)
                          reaches this value is applied as one 32x32 block on the tensor cores
                          (lqs_apply_block); gates on other qubits that commute with the run move past
                          it.  0 = default (16), negative = never. */
} lqs_fuse_cfg;

/* ---- state vectors ----------------------------------------------------------- */

/* Create a handle for an n-qubit state (1 <= n <= 36).
 * device_ptr: caller-owned device memory of at least 2^n amplitudes, 256-byte
 *   aligned (for example a torch tensor's data_ptr()); the caller keeps
 *   ownership and must keep it alive until lqs_sv_free.  NULL: the library
 *   allocates it with cudaMalloc (LQS_ERR_OOM on failure) and owns it.
 * cuda_stream: the cudaStream_t every call on this state is ordered on.
 * The contents are not initialised.  *out receives the handle. */
LQS_API int lqs_sv_alloc(int n_qubits, int dtype, void* device_ptr, void* cuda_stream, lqs_sv** out);

/* Release the handle, its scratch buffers and, when the library allocated the
 * state, the state itself (after the stream drains).  NULL is accepted. */
LQS_API int lqs_sv_free(lqs_sv* sv);

/* Device pointer, qubit count and dtype of a handle. */
LQS_API int lqs_sv_info(const lqs_sv* sv, void** device_ptr, int* n_qubits, int* dtype);

/* |x>: amplitude x = 1, all others 0 (x < 2^n).  Asynchronous. */
LQS_API int lqs_sv_set_basis(lqs_sv* sv, uint64_t x);

/* Copy 2^n amplitudes (the state's dtype, interleaved) from host memory.
 * Enqueued on the stream; pinned host memory makes it asynchronous, so the
 * host buffer must stay unchanged until the stream passes the copy. */
LQS_API int lqs_sv_copy_from_host(lqs_sv* sv, const void* host);

/* Copy the state to host memory; returns when the data is in `host`. */
LQS_API int lqs_sv_copy_to_host(const lqs_sv* sv, void* host);

/* The same copy, only enqueued on the state's stream: `host` (pinned memory
 * for the copy to overlap other work) holds the state once the stream has
 * passed the copy, e.g. after lqs_sv_sync.  Lets a caller read a result back
 * while other states are being computed on other streams. */
LQS_API int lqs_sv_copy_to_host_async(const lqs_sv* sv, void* host);

/* Wait for all work enqueued on the state's stream; reports deferred kernel
 * errors (LQS_ERR_CUDA) and device-side wait timeouts (LQS_ERR_TIMEOUT). */
LQS_API int lqs_sv_sync(lqs_sv* sv);

/* Exercises the device-side timeout path: enqueues one kernel that waits, with
 * the bounded wait every tile-loading kernel uses, on a shared-memory barrier
 * that nothing completes.  Each such wait gives up after 2^22 polls or 2 s of
 * the GPU's global timer, whichever comes first, flags the handle's status and
 * returns, so the next lqs_sv_sync returns LQS_ERR_TIMEOUT (and clears the
 * flag); the context and the state stay usable.  No amplitude is read or
 * written. */
LQS_API int lqs_check_bounded_wait(lqs_sv* sv);

/* ---- gates --------------------------------------------------------------------- */

/* Plain per-gate path: one kernel for one gate, chosen by gate class
 * (diagonal / permutation / dense one-qubit / dense two-qubit) and by qubit
 * index (Sec. 2).  wires: n_wires distinct qubits < n (controls first).
 * params: the gate's parameters (RX..CRY: 1, Rot: 3), or for U2/U4 the
 * matrix as exactly 8 / 32 doubles (row-major interleaved complex128).
 * U2/U4 matrices are inspected: a diagonal or anti-diagonal matrix takes the
 * diagonal or permutation kernels (only nonzero entries are used, Sec. 2). */
LQS_API int lqs_apply_gate(lqs_sv* sv, int gate, const int* wires, int n_wires, const double* params, int n_params,
                   int inverse);

/* The "general approach" of Sec. 3.1: apply a dense 2^m x 2^m matrix
 * (m = n_wires = 1 or 2; row-major interleaved complex128, host) with the
 * dense kernels and no inspection of its structure. */
LQS_API int lqs_apply_matrix(lqs_sv* sv, const int* wires, int n_wires, const double* matrix);

/* Dense block on the tensor cores: the general approach of Sec. 3.1 applied
 * to a set of qubits.  psi <- U psi for a 2^m x 2^m complex matrix U acting on
 * qubits 0..m-1: U[j][k] maps the amplitude whose low m index bits read k to
 * the one that reads j (qubit q is bit q of k).  `matrix` is row-major
 * interleaved complex128 on the host (read during the call).
 *
 * Complex64 states only, m = 5, n >= m + 7 (LQS_ERR_UNSUPPORTED otherwise).
 * The product runs as float32 matrix multiplies on the tensor cores with
 * each operand split into a TF32 leading part and a residual (three
 * products), about float32 accuracy; one pass over the state.  Asynchronous;
 * a device-side timeout is reported by lqs_sv_sync (LQS_ERR_TIMEOUT). */
LQS_API int lqs_apply_block(lqs_sv* sv, int m, const double* matrix);

/* The 32x32 matrix of a run of gates on qubits 0..4 (every wire < 5), as
 * lqs_apply_fused composes the runs it sends to the tensor cores: the ops
 * applied in order to each of the 32 basis states of five qubits.  Written to
 * `matrix` (row-major interleaved complex128, 2 * 32 * 32 doubles, host) in
 * the layout lqs_apply_block takes.  Host only; LQS_ERR_ARG on a bad op or a
 * wire >= 5. */
LQS_API int lqs_block_matrix(const lqs_op* ops, int n_ops, const double* params, int n_params, double* matrix);

/* Fused path: the host planner groups the circuit into segments whose
 * non-diagonal targets fit one tile of 2^k amplitudes (low contiguous qubits
 * plus chosen high qubits); each segment is one HBM pass in which the tile is
 * staged in shared memory by bulk asynchronous copies and all of its gates are
 * applied on chip.  Gates on disjoint wires may be reordered; the result equals
 * applying ops[0..n_ops) in order.  params: the circuit's parameter array.
 * Between consecutive compiled complex128 segments of one call the state is
 * held as pairs of float32 (the double-float working format); the call's
 * last segment writes complex128 again, so the state is complex128 whenever
 * work queued after the call (or on another stream after synchronising) reads
 * it.  If the call returns an error after launching, the state is
 * unspecified. */
LQS_API int lqs_apply_fused(lqs_sv* sv, const lqs_op* ops, int n_ops, const double* params, int n_params,
                    const lqs_fuse_cfg* cfg_or_null);

/* Autotuner (the tuner of the batched driver, Sec. 4 / Listing 1's repeated circuits): times
 * lqs_apply_fused on this state with candidate configurations (low contiguous tile qubits b = 3..5
 * for c128, 4..6 for c64; no segment cap or 48 gates), each applied twice untimed (compiled kernels
 * are built then) and `repeats` (1..100) times under CUDA events on the state's stream.  *best
 * receives the fastest, which is also remembered for this qubit count, dtype and circuit structure
 * (gates and wires; not angles or matrices): later lqs_apply_fused calls with cfg_or_null = NULL on
 * that structure use it.  The state serves as scratch: its contents are undefined on return.  States
 * of one tile have nothing to tune (*best = all zero).  Synchronous. */
LQS_API int lqs_autotune_fused(lqs_sv* sv, const lqs_op* ops, int n_ops, const double* params, int n_params,
                               int repeats, lqs_fuse_cfg* best);

/* Host-only view of the fused plan (no GPU work, usable without a device):
 * *n_segments receives the number of HBM passes; when seg_qubit_mask is
 * non-null it receives each segment's tile qubit set (capacity `cap`), and
 * op_segment (n_ops entries, optional) each op's segment.  Ops executed
 * segment by segment in their original relative order reproduce the circuit.
 * A gate that runs as several kernel ops (DoubleExcitation) is reported with
 * the segment of its last one; its ops may sit in several segments. */
LQS_API int lqs_plan_fused(int n_qubits, int dtype, const lqs_op* ops, int n_ops, const lqs_fuse_cfg* cfg_or_null,
                   int* n_segments, uint64_t* seg_qubit_mask, int cap, int* op_segment);

/* ---- measurement -------------------------------------------------------------- */

/* <psi|psi> accumulated in float64. */
LQS_API int lqs_norm2(lqs_sv* sv, double* out_host);

/* Distance between two states of the same qubit count (any dtypes):
 * *diff2 = sum_i |a_i - b_i|^2 and *norm2_b = sum_i |b_i|^2, accumulated in
 * float64 (double-float per thread, fixed-order reduction).  Used to report
 * the complex64 error against a complex128 run of the same circuit.  Both
 * handles' streams are synchronised.  Synchronous. */
LQS_API int lqs_sv_distance(lqs_sv* a, lqs_sv* b, double* diff2_host, double* norm2_b_host);

/* Expectation value of H = sum_w coeff_w P_w (Listing 1: qml.expval(H)),
 * accumulated in float64 with deterministic two-stage reductions (no float
 * atomics).  *out_host = sum_w coeff_w <P_w>; per_term_host (optional,
 * n_terms entries) receives each <P_w>.  Synchronous. */
LQS_API int lqs_expval(lqs_sv* sv, const lqs_pauli* terms, int n_terms, double* out_host, double* per_term_host);

/* ---- gradients --------------------------------------------------------------- */

/* Adjoint-method gradient of E(theta) = <psi(theta)|H|psi(theta)> for every
 * parameter slot, in one reverse sweep.  psi must hold the state AFTER the
 * circuit (ops, params) was applied; the sweep computes lambda = H psi and,
 * for gates l = L..1, g += Im-part inner products of lambda with the gate's
 * generator applied to psi, then un-applies the gate from both.  On return psi
 * holds the circuit's input state again (up to rounding).  Two extra state
 * buffers are used, allocated once per handle and reused.  grads_host has
 * n_params entries (slots used by several gates receive the sum);
 * energy_host (optional) receives E.  Synchronous. */
LQS_API int lqs_adjoint_grad(lqs_sv* psi, const lqs_op* ops, int n_ops, const double* params, int n_params,
                     const lqs_pauli* terms, int n_terms, double* grads_host, double* energy_host);

/* ---- batches of small circuits ---------------------------------------------- */

/* One circuit of a batch: its own qubit count, gates, parameters and
 * observable; starts from |0..0>.  grads (host, n_params entries) and
 * energy are written by lqs_batch_run. */
typedef struct {
  int32_t n_qubits;
  int32_t n_ops;
  const lqs_op* ops;
  int32_t n_params;
  const double* params;
  int32_t n_terms;
  const lqs_pauli* terms;
  double* grads;  /* host, n_params entries, or NULL for energy only */
  double* energy; /* host, 1 entry */
} lqs_batch_item;

/* Forward + expectation + adjoint gradient of many independent circuits
 * (Listing 1's loop of small circuits) in one persistent launch on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  Every
 * circuit is a chain of passes over its own state (forward segments, Pauli
 * passes forming lambda = H psi and the energy, reverse segments with the
 * gradient partials), one task per tile of the state; resident thread blocks
 * claim the tasks of all circuits level by level from a shared counter, and a
 * task waits (bounded: 2 s, LQS_ERR_TIMEOUT) until the tiles of its circuit's
 * previous pass are done, so the tiles of many circuits run at once on every
 * SM.  Energies and gradients are summed in a fixed order (deterministic).
 * Plans are cached by circuit structure; device buffers are kept by the
 * library between calls (they only grow, and calls are serialised).  The
 * tile shape of each qubit count is the one lqs_batch_autotune chose, if it
 * ran, else 2^12 amplitudes (complex64) / 2^11 (complex128) with 32 / 16
 * contiguous amplitudes per row.  1 <= n_qubits <= 26 per circuit; every
 * Pauli word's X/Y qubits must fit one tile (LQS_ERR_UNSUPPORTED otherwise).
 * Synchronous: energies and gradients are in host memory on return. */
LQS_API int lqs_batch_run(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream);

/* Autotuner of the batched driver: for each qubit count of the batch that
 * spans more than one tile, times lqs_batch_run on that count's circuits with
 * each candidate tile shape (tile qubits k in {12, 11} for complex64, {11, 10}
 * for complex128; contiguous low qubits b in {5, 4} / {4, 3}), each candidate
 * run once untimed and `repeats` (1..100) times under CUDA events, and keeps
 * the fastest per (qubit count, dtype) for later lqs_batch_run calls.  The
 * items' outputs are written as by lqs_batch_run.  *n_tuned (optional)
 * receives the number of qubit counts tuned.  Synchronous. */
LQS_API int lqs_batch_autotune(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream, int repeats,
                               int* n_tuned);

/* ---- measurement without device allocation ------------------------------------- */

/* <psi|H|psi> like lqs_expval, for callers that must not allocate device
 * memory when they measure: hosts whose memory pool owns all device memory,
 * or loops that cannot pay for the synchronisation cudaMalloc/cudaFree bring.
 * The paper has no counterpart; this is a property of this library's
 * interface.
 * It needs no state handle: psi_device points to 2^n_qubits amplitudes of
 * `dtype` in device memory (read only), work is ordered on cuda_stream, which
 * must belong to the current device (LQS_ERR_ARG otherwise), and the call is
 * synchronous: it copies the results to *out_host (and per_term_host[0..n_terms),
 * if given) and waits for the stream, so it cannot run on a stream that is
 * being captured into a CUDA graph: there it returns LQS_ERR_ARG before
 * enqueuing any work, and the capture stays valid.  n_terms = 0 gives 0.  It calls no
 * cudaMalloc/cudaFree and no allocating library routine: partial sums live in
 * a fixed scratch array compiled into the library (64 terms x 1024 blocks of
 * float64, about 513 KiB), which every GPU that loads the library keeps until
 * the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress).  At most 64 terms (LQS_ERR_ARG beyond).
 * All calls share the array, so calls that overlap on the GPU race on it:
 * serialise them.  One float64-accumulated pass over the state per term.
 * Accuracy: complex128 amplitudes are split into double-float pairs (about 47
 * significant bits) before the products, so each <P_w> is within about 1e-14
 * relative of the exact value rather than float64's 1e-16. */
LQS_API int lqs_expval_static(const void* psi_device, int n_qubits, int dtype, void* cuda_stream,
                              const lqs_pauli* terms, int n_terms, double* out_host, double* per_term_host);

/* ---- misc ------------------------------------------------------------------------ */

/* Message describing the calling thread's most recent error ("" if none). */
LQS_API const char* lqs_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
LQS_API int lqs_version(void);

/* Default c128 arithmetic for subsequent calls on this process (lqs_arith). */
LQS_API int lqs_set_arith(int arith);

/* Number of kernels this library has launched since load (for accounting). */
LQS_API uint64_t lqs_kernel_launches(void);

/* ---- compiled segments ----------------------------------------------------------- *
 * The fused path applies each segment of a circuit (the gates that share one pass of
 * tiles through on-chip memory; Sec. 2's "local" gates, see lqs_apply_fused) with a
 * register-tile kernel.  That kernel can run in two forms with the same arithmetic:
 *   - the interpreter: one precompiled kernel reads the segment's op list at run time;
 *   - a compiled segment: the op list written out as straight-line CUDA C++ (register
 *     slots, control patterns and coefficient offsets constant) and compiled at run
 *     time for sm_103a with NVRTC (libnvrtc.so.13, found by dlopen; the environment
 *     variable LQS_NVRTC may name it).
 * Compiled segments are cached per structure (not per angle: coefficients stay kernel
 * parameters) and device for the life of the process.
 * Modes: LQS_JIT_OFF never compiles; LQS_JIT_ON compiles every segment at its first use;
 * LQS_JIT_AUTO (default, or the environment variable LQS_JIT=0/1/2 at load) compiles a
 * structure at its second use on states of 20 or more qubits, running the interpreter
 * before that.  A call compiles the structures it needs on up to 8 host threads before
 * its first launch.  When NVRTC is missing, LQS_JIT_ON makes lqs_apply_fused fail with
 * LQS_ERR_UNSUPPORTED and LQS_JIT_AUTO keeps the interpreter (lqs_jit_info reports it). */
typedef enum { LQS_JIT_OFF = 0, LQS_JIT_ON = 1, LQS_JIT_AUTO = 2 } lqs_jit_mode;
LQS_API int lqs_set_jit(int mode);
typedef struct {
  int mode;                /* current lqs_jit_mode */
  int compiled;            /* structures compiled since load */
  int failed;              /* structures NVRTC rejected (the interpreter runs them) */
  int cached;              /* structures seen (compiled or not) */
  uint64_t launches;       /* compiled-segment launches since load */
  double compile_seconds;  /* host time spent in NVRTC, summed over threads */
  char last_error[256];    /* last compile or load failure ("" if none) */
} lqs_jit_stats;
LQS_API int lqs_jit_info(lqs_jit_stats* out);
/* Compiles, without a GPU, every segment structure lqs_apply_fused would launch for this
 * circuit on an n-qubit state of `dtype` with arithmetic `arith` (lqs_arith) and `cfg`
 * (may be NULL), whatever the mode; *n_compiled (may be NULL) gets the number of
 * structures compiled by this call.  Lets a caller pay the compile cost ahead of a timed
 * or latency-critical loop.  Errors as lqs_apply_fused, plus LQS_ERR_UNSUPPORTED when
 * NVRTC cannot be loaded or rejects a segment (lqs_last_error has its log). */
LQS_API int lqs_jit_precompile(int n_qubits, int dtype, int arith, const lqs_op* ops, int n_ops,
                               const double* params, int n_params, const lqs_fuse_cfg* cfg, int* n_compiled);
/* The same for the reverse sweep of lqs_adjoint_grad on this circuit: its compiled kernels hold psi and
 * lambda in registers (tiles one qubit smaller than lqs_apply_fused's, 128 threads) and add each
 * parameter's Im<lambda|G|psi> as they un-apply the gates.  lqs_adjoint_grad uses them whenever compiled
 * segments are enabled for the state's size (LQS_JIT_ON, or LQS_JIT_AUTO on 20 or more qubits),
 * compiling missing ones at that call; states of at most 10 (c128) / 11 (c64) qubits use the
 * shared-memory sweep and compile nothing here. */
LQS_API int lqs_jit_precompile_adjoint(int n_qubits, int dtype, int arith, const lqs_op* ops, int n_ops,
                                       const double* params, int n_params, int* n_compiled);
/* The same for the expectation-value passes of lqs_expval on these terms (lambda = 0), or for the passes
 * that also form lambda = H psi in lqs_adjoint_grad (lambda != 0).  Each pass covers the words whose X/Y
 * qubits fit one tile (2^11 amplitudes for c128, 2^12 for c64, up to 32 words): thread registers hold the
 * tile, diagonal words are evaluated together through one Walsh butterfly per warp and register-bit sign
 * pattern, X/Y words pair amplitudes.  Words wider than a tile, and states of one tile, use the
 * interpreter passes and compile nothing here. */
LQS_API int lqs_jit_precompile_expval(int n_qubits, int dtype, int arith, const lqs_pauli* terms, int n_terms,
                                      int lambda, int* n_compiled);

/* Per-launch profile records (tracing).  Between lqs_profile_start and
 * lqs_profile_stop every kernel the library launches is bracketed by CUDA
 * events on its stream; stop synchronises those streams and returns, per
 * launch, the kernel family, its device time, and the algorithmic HBM bytes
 * and float64-equivalent flops the launch had to process (what the method
 * must move and compute, not what the hardware counters report). */
typedef struct {
  char kernel[48];
  float ms;
  double bytes;
  double flops;
} lqs_launch_record;
LQS_API int lqs_profile_start(void);
/* Copies up to `cap` records into `out` (may be NULL), the total into *count. */
LQS_API int lqs_profile_stop(lqs_launch_record* out, int cap, int* count);

/* Host-only check of the double-float conversions used for complex128
 * arithmetic (no device needed).  For each in[i]: out[2i] = hi + lo of its
 * double-float split widened exactly, out[2i+1] = the double the store path
 * rounds the split back to.  LQS_ERR_ARG on NULL pointers or count < 0. */
LQS_API int lqs_debug_df_roundtrip(const double* in, double* out, int64_t count);

#ifdef __cplusplus
}
#endif
#endif /* LQS_ABI_H_INCLUDED */
