// Internal types shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lqs.h"

namespace lqs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);
#define LQS_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::lqs::cuda_error(e_, #call); \
  } while (0)
#define LQS_TRY(expr)          \
  do {                         \
    int r_ = (expr);           \
    if (r_ != LQS_OK) return r_; \
  } while (0)

void count_launch(uint64_t n = 1);

// Launch profiling: when enabled, record CUDA events around each launch.
struct ProfScope {
  int idx = -1;
  ProfScope(cudaStream_t st, const char* name, double bytes, double flops);
  ~ProfScope();
  cudaStream_t st;
};
const char* arith_tag(int dtype, int arith);

// ---------------------------------------------------------------------------
// kernel ops: a gate after classification (Sec. 2: use only the nonzero
// entries of the gate matrix; the kernel depends on the gate's class)
// ---------------------------------------------------------------------------
enum KKind : int {
  K_PHASE = 0,   // psi[i] *= f   where all cmask bits of i are 1   (Z S T PhaseShift CZ CPhase)
  K_DIAG1 = 1,   // psi[i] *= d[bit t of i]   (RZ, diagonal 2x2), controls allowed
  K_ANTI1 = 2,   // (a0, a1) <- (f0 a1, f1 a0) on bit t   (X CNOT Toffoli Y)
  K_SWAP = 3,    // swap amplitudes ..1..0.. <-> ..0..1.. on bits (t0, t1)   (SWAP)
  K_DENSE1 = 4,  // complex 2x2 on bit t (RX Rot U2), controls allowed
  K_DENSE1R = 5, // real 2x2 on bit t (H RY CRY)
  K_DENSE2 = 6,  // complex 4x4 on bits (t0 = most significant local bit, t1)
  K_DIAG2 = 7,   // diagonal 4x4 on bits (t0, t1)
  K_LAYOUT = 8,  // register-tile kernel: move amplitudes to a new register/thread bit layout
  K_DPROD = 9,   // register-tile kernel: merged diagonal run, C * prod_q f_q^bit_q on amplitudes whose cond bits are 1
  K_GRAD = 10,   // compiled adjoint: gradient partial of a merged run's member (no state change)
};

// Generators for the adjoint method: a parametrised gate U(theta) with
// dU/dtheta = -i K U contributes dE/dtheta = 2 Im <lambda|K|psi>.  K is
// `scale`/2 times one of these operators on target t (with controls cmask).
enum KGen : int { G_NONE = 0, G_X = 1, G_Y = 2, G_Z = 3, G_P1 = 4 };

struct KOp {
  int kind = K_PHASE;
  int special = 0;      // K_PHASE: 1 = factor -1, 2 = +i, 3 = -i (no arithmetic); K_ANTI1: 1 = plain swap
  int t0 = -1, t1 = -1; // target qubits
  uint64_t cmask = 0;   // control qubits (all must be 1)
  double m[32] = {0};   // coefficients (interleaved complex or reals, per kind)
  // adjoint bookkeeping
  int param_slot = -1;
  int gen = G_NONE;
  double gen_scale = 0; // dE/dtheta = gen_scale * Im<lambda|G|psi> with G in {X,Y,Z,P1}
  bool diagonal() const { return kind == K_PHASE || kind == K_DIAG1 || kind == K_DIAG2; }
  uint64_t target_mask() const {
    uint64_t m_ = 0;
    if (t0 >= 0) m_ |= 1ull << t0;
    if (t1 >= 0) m_ |= 1ull << t1;
    return m_;
  }
  uint64_t wire_mask() const { return target_mask() | cmask; }
  // qubits whose value the op must see inside a tile (non-diagonal targets)
  uint64_t tile_mask() const { return diagonal() ? 0 : target_mask(); }
};

// Validate one gate and lower it to kernel ops.  `decompose` splits Rot into
// RZ RY RZ so every parametrised op has a single-parameter generator (adjoint).
// `general` forces the dense kernels (no class specialisation).
int lower_gate(int n_qubits, int gate, const int* wires, int n_wires, const double* params, int n_params,
               const double* matrix, int inverse, int param_slot, bool decompose, bool general,
               std::vector<KOp>& out);
int lower_ops(int n_qubits, const lqs_op* ops, int n_ops, const double* params, int n_params, bool decompose,
              std::vector<KOp>& out);
// Algorithmic work of a lowered op: fraction of amplitudes it touches and
// float64-equivalent flops per touched amplitude (for profile records).
double kop_touched_fraction(const KOp& op);
double kop_flops_per_amp(const KOp& op);

// ---------------------------------------------------------------------------
// state handle
// ---------------------------------------------------------------------------
struct SV {
  int n = 0;
  int dtype = LQS_C128;
  void* d = nullptr;        // amplitudes
  bool owns = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  // scratch, grown on demand and kept for the handle's lifetime
  void* scratch[3] = {nullptr, nullptr, nullptr};
  size_t scratch_bytes[3] = {0, 0, 0};
  int* d_status = nullptr;  // device-side error flags (bounded waits)
  size_t amp_bytes() const { return dtype == LQS_C64 ? 8 : 16; }
  uint64_t N() const { return 1ull << n; }
  size_t bytes() const { return amp_bytes() * N(); }
};

int sv_scratch(SV* sv, int slot, size_t bytes, void** out);
int current_arith(int requested);  // resolves LQS_ARITH_AUTO

// ---------------------------------------------------------------------------
// per-gate kernels (plain path)
// ---------------------------------------------------------------------------
int launch_gate(SV* sv, const KOp& op, int arith);

// ---------------------------------------------------------------------------
// fused tiles
// ---------------------------------------------------------------------------
struct Segment {
  uint64_t qmask = 0;           // tile qubits
  std::vector<int> ops;         // indices into the lowered op list, in execution order
};
struct PlanCfg {
  int k = 0;          // tile qubits
  int b = 0;          // low contiguous qubits
  int max_ops = 0;    // per-segment cap
  int dense_cap = 0;  // cap on a segment's dense weight (compiled segments; 0 = none)
};
int resolve_cfg(int n, int dtype, const lqs_fuse_cfg* cfg, PlanCfg& pc, int* arith);
// Tensor-core dense blocks (block_tc.cu): lowered ops confined to qubits
// 0..kBlockQubits-1 composed into one 32x32 complex matrix (row-major
// interleaved, qubit q = bit q of the local index), applied to a complex64
// state in one pass; block_weight is an op's share of a run's dense work (a
// run goes to the tensor cores when its weights reach the threshold).
constexpr int kBlockQubits = 5;
void block_matrix(const std::vector<KOp>& ops, const std::vector<int>& idx, double* U);
int apply_block(SV* sv, const double* U);
double block_weight(const KOp& op);
// The configuration lqs_autotune_fused chose for this circuit structure, if any.
bool tuned_cfg(int n, int dtype, const lqs_op* ops, int n_ops, lqs_fuse_cfg* out);
int plan_segments(int n, const std::vector<KOp>& ops, const PlanCfg& pc, std::vector<Segment>& segs);
// fmt != 0 only for a segment that seg_split_capable accepted (see jit_launch).
int launch_segment(SV* sv, const std::vector<KOp>& ops, const Segment& seg, const PlanCfg& pc, int arith,
                   unsigned fmt = 0);
// Register-resident tile kernel (k = reg_tile_qubits(dtype)); returns
// LQS_ERR_UNSUPPORTED when the segment's program does not fit (split it).
int reg_tile_qubits(int dtype);
int launch_fused_reg(SV* sv, const std::vector<KOp>& ops, const Segment& seg, int k, int b, int arith,
                     unsigned fmt = 0);
// True when launch_segment runs this complex128 double-float segment as one
// compiled kernel, which can read and leave hi/lo float pairs.
bool seg_split_capable(const SV* sv, const std::vector<KOp>& ops, const Segment& seg, int k, int b, int arith);
// Compiled adjoint: the reverse sweep's segments as register-tile programs
// over psi and lambda.  reg_adjoint_available tells whether this state takes
// it (mode, size); run_adjoint_compiled launches all segments, writing the
// per-slot partial sums of Im<lambda|G|psi> (slot_op: the op of each slot;
// slot_scale: the factor each slot's summed partials take).  Returns
// LQS_ERR_UNSUPPORTED, having launched nothing, when the interpreter must run.
bool reg_adjoint_available(const SV* sv, int arith);
int adjoint_tile_qubits(int dtype);  // tile of the compiled reverse sweep
int run_adjoint_compiled(SV* sv, const std::vector<KOp>& rev, void* lam, int arith, std::vector<int>& slot_op,
                         std::vector<double>& slot_scale, double** partial, int* grid);
// Host only: compile the reverse sweep's kernels (rev = inverse ops, reversed).
int adjoint_precompile(int n, int dtype, int arith, const std::vector<KOp>& rev, int* compiled);
// Segment compiler hooks: note_reg_prog builds a segment's register-tile
// program (LQS_ERR_UNSUPPORTED when it must be split) and notes it;
// jit_collect walks a segment the way launch_segment routes and splits it.
int note_reg_prog(int n, int dtype, int arith, const std::vector<KOp>& ops, const Segment& seg, int k, int b,
                  bool force, std::vector<void*>& todo);
int jit_collect(int n, int dtype, int arith, const std::vector<KOp>& ops, const Segment& seg, const PlanCfg& pc,
                bool force, std::vector<void*>& todo);

// ---------------------------------------------------------------------------
// reductions / expectation values / adjoint
// ---------------------------------------------------------------------------
int run_norm2(SV* sv, int arith, double* out);
// Fixed-order sums of per-block partials: sums[s] = sum_b partial[s * grid + b].
int k_sum_partials_launch(double* partial, int grid, double* sums, int slots, cudaStream_t st);
// Compiled Pauli passes (<P_w> per word into vals; lambda = H psi when lam is
// non-null).  LQS_ERR_UNSUPPORTED when this state or word set does not take
// them (the interpreter passes run instead); nothing is launched then.
int pauli_compiled(SV* sv, const lqs_pauli* terms, int n_terms, void* lam, int arith, double* vals);
int pauli_precompile(int n, int dtype, int arith, const lqs_pauli* terms, int n_terms, bool lambda, int* compiled);
int run_expval(SV* sv, const lqs_pauli* terms, int n_terms, const PlanCfg& pc, int arith, double* out,
               double* per_term, const void* lambda_out);
int run_adjoint(SV* sv, const std::vector<KOp>& ops, int n_params, const lqs_pauli* terms, int n_terms,
                const PlanCfg& pc, int arith, double* grads, double* energy);

}  // namespace lqs
