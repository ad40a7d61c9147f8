// Fusion planner (host) and the fused-segment tile kernel.
//
// The planner groups a circuit into segments; all gates of a segment are
// applied to each tile while it sits in shared memory, so a segment costs
// one HBM read and one HBM write of the state however many gates it holds.
// This is the single-GPU counterpart of the paper's observation that gates
// on local qubits need no data exchange (Sec. 2): a segment's tile qubits
// play the role of the local qubits, and choosing them per segment lets the
// "non-local" gates become local too.
#include <algorithm>
#include <string>
#include <type_traits>

#include "arith.cuh"
#include "jit.h"
#include "lqs_internal.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"

// Dense work per segment: a compiled segment is straight-line code, and one
// whose dense updates add up past this weight (4 per two-qubit dense op, 1
// per one-qubit dense op; diagonal and permutation ops are free) spends more
// in instruction fetch than a further pass costs.
#ifndef LQS_SEGMENT_DENSE_CAP
#define LQS_SEGMENT_DENSE_CAP 16
#endif
// complex64 segments carry float32 arithmetic, several times less code per op
#ifndef LQS_SEGMENT_DENSE_CAP_C64
#define LQS_SEGMENT_DENSE_CAP_C64 64
#endif

namespace lqs {

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------
int resolve_cfg(int n, int dtype, const lqs_fuse_cfg* cfg, PlanCfg& pc, int* arith) {
  const int kmax = dtype == LQS_C64 ? 14 : 13;  // tile <= 128 KiB of shared memory
  pc.k = reg_tile_qubits(dtype);                  // the register-tile kernel's shape
  pc.b = dtype == LQS_C64 ? 5 : 4;
  pc.max_ops = kMaxTileOps;
  // multi-tile states whose segments run as compiled code
  pc.dense_cap = n > reg_tile_qubits(dtype) && jit_enabled_for(n)
                     ? (dtype == LQS_C64 ? LQS_SEGMENT_DENSE_CAP_C64 : LQS_SEGMENT_DENSE_CAP)
                     : 0;
  int ar = LQS_ARITH_AUTO;
  if (cfg) {
    if (cfg->tile_qubits) pc.k = cfg->tile_qubits;
    if (cfg->low_qubits) pc.b = cfg->low_qubits;
    if (cfg->max_ops) pc.max_ops = std::min<int>(cfg->max_ops, kMaxTileOps);
    ar = cfg->arith;
    if (ar != LQS_ARITH_AUTO && ar != LQS_ARITH_F64 && ar != LQS_ARITH_DF)
      return set_error(LQS_ERR_ARG, "cfg.arith must be LQS_ARITH_AUTO, LQS_ARITH_F64 or LQS_ARITH_DF");
  }
  if (pc.k < 3 || pc.k > kmax)
    return set_error(LQS_ERR_ARG, "tile_qubits must be in [3, " + std::to_string(kmax) + "]");
  const int bmin = dtype == LQS_C64 ? 1 : 0;  // bulk copies move multiples of 16 bytes
  if (pc.b < std::max(bmin, 1) || pc.b > pc.k - 2)
    return set_error(LQS_ERR_ARG, "low_qubits must be in [1, tile_qubits - 2]");
  if (pc.max_ops < 1) return set_error(LQS_ERR_ARG, "max_ops must be positive");
  if (n <= pc.k) {  // the whole state is one tile
    pc.k = n;
    pc.b = n;
  }
  if (arith) *arith = current_arith(ar);
  return LQS_OK;
}

static int coef_count(const KOp& o) {
  switch (o.kind) {
    case K_PHASE: return 1;
    case K_DIAG1: return 2;
    case K_ANTI1: return 2;
    case K_SWAP: return 0;
    case K_DENSE1: return 4;
    case K_DENSE1R: return 4;
    case K_DENSE2: return 16;
    case K_DIAG2: return 4;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------
//
// Greedy in program order.  A segment starts with the low b qubits in its
// tile.  Each not-yet-scheduled op is taken if (1) no earlier unscheduled op
// shares a wire with it ("blocked" wires), so moving it ahead of those ops
// only passes gates on disjoint wires, which commute, and (2) its
// non-diagonal targets fit the tile, adding qubits while fewer than k are
// used.  Diagonal ops and controls need no tile qubit.  An op that is not
// taken blocks its wires for the rest of the segment.
static int dense_weight(const KOp& o) {
  return o.kind == K_DENSE2 ? 4 : (o.kind == K_DENSE1 || o.kind == K_DENSE1R) ? 1 : 0;
}

int plan_segments(int n, const std::vector<KOp>& ops, const PlanCfg& pc, std::vector<Segment>& segs) {
  const int k = std::min(pc.k, n), b = std::min(pc.b, k);
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
  const uint64_t low = b >= 64 ? ~0ull : ((1ull << b) - 1);
  std::vector<char> done(ops.size(), 0);
  size_t remaining = ops.size(), first = 0;
  segs.clear();
  while (remaining) {
    while (done[first]) ++first;
    Segment seg;
    uint64_t Q = low, blocked = 0;
    int ncoef = 0, dense = 0;
    for (size_t i = first; i < ops.size() && blocked != all; ++i) {
      if (done[i]) continue;
      const KOp& o = ops[i];
      const uint64_t wires = o.wire_mask();
      if (wires & blocked) {
        blocked |= wires;
        continue;
      }
      const uint64_t need = o.tile_mask() & ~Q;
      const int nc = coef_count(o);
      const int dw = dense_weight(o);
      const bool fits = __builtin_popcountll(Q | need) <= k && (int)seg.ops.size() < pc.max_ops &&
                        ncoef + nc <= kMaxTileCoef &&
                        (pc.dense_cap <= 0 || dense + dw <= pc.dense_cap || seg.ops.empty());
      if (fits) {
        Q |= need;
        seg.ops.push_back((int)i);
        done[i] = 1;
        --remaining;
        ncoef += nc;
        dense += dw;
      } else {
        blocked |= wires;
      }
    }
    if (seg.ops.empty()) return set_error(LQS_ERR_ARG, "internal: planner made no progress");
    for (int q = b; q < n && __builtin_popcountll(Q) < k; ++q) Q |= 1ull << q;  // pad to exactly k qubits
    seg.qmask = Q;
    segs.push_back(std::move(seg));
  }
  return LQS_OK;
}

// ---------------------------------------------------------------------------
// tile program construction
// ---------------------------------------------------------------------------
static TileGeom make_tile_geom(int n, uint64_t Q, int k, int b, size_t amp_bytes) {
  TileGeom G{};
  G.n = n;
  G.k = k;
  G.b = b;
  G.r = 0;
  for (int q = b; q < n; ++q)
    if ((Q >> q) & 1) G.h[G.r++] = q;
  G.ntiles = 1ull << (n - k);
  G.row_bytes = (uint32_t)(amp_bytes << b);
  return G;
}

static int local_pos(const TileGeom& G, int q) {
  if (q < 0) return -1;
  if (q < G.b) return q;
  for (int m = 0; m < G.r; ++m)
    if (G.h[m] == q) return G.b + m;
  return -1;
}

template <class A>
static typename A::C cc(const KOp& op, int i) { return A::cconst(op.m[2 * i], op.m[2 * i + 1]); }

template <class A>
int add_tile_op(TileProg<A>& P, const KOp& o, int gslot) {
  if (P.nops >= kMaxTileOps) return set_error(LQS_ERR_ARG, "internal: tile program full");
  const TileGeom& G = P.g;
  TOp t{};
  t.kind = (uint8_t)o.kind;
  t.special = (uint8_t)o.special;
  t.gen = (uint8_t)o.gen;
  t.gslot = (int16_t)gslot;
  t.l0 = (int8_t)local_pos(G, o.t0);
  t.l1 = (int8_t)local_pos(G, o.t1);
  if (!o.diagonal() && ((o.t0 >= 0 && t.l0 < 0) || (o.t1 >= 0 && t.l1 < 0)))
    return set_error(LQS_ERR_ARG, "internal: non-diagonal target outside the tile");
  if (o.t0 >= 0 && t.l0 < 0) t.e0 = 1ull << o.t0;
  if (o.t1 >= 0 && t.l1 < 0) t.e1 = 1ull << o.t1;
  int fix[6], nfix = 0;
  for (int q = 0; q < G.n; ++q) {
    if (!((o.cmask >> q) & 1)) continue;
    const int lp = local_pos(G, q);
    if (lp >= 0) {
      t.lcmask |= 1u << lp;
      fix[nfix++] = lp;
    } else {
      t.ecmask |= 1ull << q;
    }
  }
  // diagonal ops with a local target enumerate pairs (K_DIAG1) over it; K_DIAG2
  // and K_PHASE enumerate single amplitudes
  const bool pair_target = o.kind != K_PHASE && o.kind != K_DIAG2 && !(o.kind == K_DIAG1 && t.l0 < 0);
  if (pair_target) {
    if (t.l0 >= 0) fix[nfix++] = t.l0;
    if (t.l1 >= 0 && o.kind != K_DIAG1) fix[nfix++] = t.l1;
  }
  if (nfix > 4) return set_error(LQS_ERR_ARG, "internal: more than 4 fixed tile bits");
  std::sort(fix, fix + nfix);
  t.nfix = (uint8_t)nfix;
  for (int i = 0; i < nfix; ++i) t.fix[i] = (uint8_t)fix[i];
  const int nc = coef_count(o);
  if (P.ncoef + nc > kMaxTileCoef) return set_error(LQS_ERR_ARG, "internal: tile coefficient pool full");
  t.coef = (int16_t)P.ncoef;
  for (int i = 0; i < nc; ++i) P.coef[P.ncoef + i] = (o.kind == K_DENSE1R) ? A::cconst(o.m[i], 0.0) : cc<A>(o, i);
  P.ncoef += nc;
  // an uncontrolled real 2x2 with m11 = s m00 and m10 = -s m01 (s = +1:
  // rotations such as RY, special 1; s = -1: reflections such as H, special 2)
  // is g times an orthogonal matrix: compiled segments apply it in a cheaper
  // form (the interpreter ignores the mark).  Special 3: the Hadamard pattern
  // m00 = m01 = m10 = -m11 > 0, sums and differences only.
  if (o.kind == K_DENSE1R && o.cmask == 0) {
    if (o.m[3] == o.m[0] && o.m[2] == -o.m[1]) t.special = 1;
    else if (o.m[0] > 0.0 && o.m[1] == o.m[0] && o.m[2] == o.m[0] && o.m[3] == -o.m[0]) t.special = 3;
    else if (o.m[3] == -o.m[0] && o.m[2] == o.m[1]) t.special = 2;
  }
  P.op[P.nops++] = t;
  return LQS_OK;
}

template <class A>
void init_prog(TileProg<A>& P, int n, uint64_t Q, int k, int b) {
  P.g = make_tile_geom(n, Q, k, b, (size_t)A::kAmpBytes);
  P.nops = 0;
  P.ncoef = 0;
  P.ngrad = 0;
  P.nfold = 0;
}

// ---------------------------------------------------------------------------
// the fused kernel: persistent CTAs, one tile in shared memory per CTA
// ---------------------------------------------------------------------------
template <class A>
__global__ void __launch_bounds__(kTileThreads) k_fused(typename A::S* __restrict__ psi,
                                                        const __grid_constant__ TileProg<A> P, int* status) {
  using S = typename A::S;
  using W = typename A::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TileGeom& G = P.g;
  const uint32_t nt = 1u << G.k;
  S* buf = reinterpret_cast<S*>(smem_raw);
  W* T = reinterpret_cast<W*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)nt * sizeof(S));
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  bool ok = true;
  for (uint64_t t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(G, t);
    if (threadIdx.x < 32) tile_load_issue(G, buf, psi, base, bar);
    ok = __syncthreads_and(mbar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    if constexpr (!std::is_same<S, W>::value) {
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        const S s = buf[j];
        T[j] = A::load(s);
      }
      __syncthreads();
    }
    for (int i = 0; i < P.nops; ++i) {
      tile_apply<A>(T, P.op[i], P.coef, base, G.k);
      __syncthreads();
    }
    if constexpr (!std::is_same<S, W>::value) {
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        const W w = T[j];
        buf[j] = A::store(w);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x < 32) tile_store_issue(G, psi, buf, base);
  }
  if (threadIdx.x < 32) bulk_wait0();
  if (!ok) {
    if (threadIdx.x == 0) {
      flag_timeout(status, 1);
      mbar_wait(bar, phase ^ 1u);  // let the load in flight land before the CTA exits (bounded)
    }
  }
}

template <class A>
static int launch_fused_t(SV* sv, const std::vector<KOp>& ops, const Segment& seg, const PlanCfg& pc, int arith) {
  const int n = sv->n, k = std::min(pc.k, n), b = std::min(pc.b, k);
  static thread_local TileProg<A> P;  // ~14 KB: keep it off the stack
  init_prog(P, n, seg.qmask, k, b);
  for (int i : seg.ops) LQS_TRY(add_tile_op(P, ops[i], -1));
  const size_t smem = ((size_t)sizeof(typename A::S) << k) + 16;
  static bool attr_done = false;
  if (!attr_done) {
    LQS_CUDA_TRY(cudaFuncSetAttribute(k_fused<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done = true;
  }
  int per_sm = 0;
  LQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<A>, kTileThreads, smem));
  per_sm = std::max(per_sm, 1);
  const uint64_t grid = std::min<uint64_t>(P.g.ntiles, (uint64_t)std::max(sv->sms, 1) * per_sm);
  double flops = 0.0;
  for (int i : seg.ops) flops += kop_touched_fraction(ops[i]) * kop_flops_per_amp(ops[i]);
  const std::string pname = std::string("k_fused/") + arith_tag(sv->dtype, arith);
  ProfScope ps(sv->stream, pname.c_str(), 2.0 * (double)sv->bytes(), flops * (double)sv->N());
  k_fused<A><<<(unsigned)grid, kTileThreads, smem, sv->stream>>>(static_cast<typename A::S*>(sv->d), P, sv->d_status);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

int launch_segment(SV* sv, const std::vector<KOp>& ops, const Segment& seg, const PlanCfg& pc, int arith,
                   unsigned fmt) {
  const int k = std::min(pc.k, sv->n), b = std::min(pc.b, k);
  if (fmt) return launch_fused_reg(sv, ops, seg, k, b, arith, fmt);  // checked by seg_split_capable
  // A lone gate is cheaper as a plain pass: it only touches the amplitudes it changes.
  if (seg.ops.size() == 1) return launch_gate(sv, ops[seg.ops[0]], arith);
  if (k == reg_tile_qubits(sv->dtype)) {
    const int rc = launch_fused_reg(sv, ops, seg, k, b, arith);
    if (rc != LQS_ERR_UNSUPPORTED) return rc;
    // the register program (gates plus layout changes) overflowed: split the
    // segment in two, keeping the order of its gates
    Segment lo, hi;
    lo.qmask = hi.qmask = seg.qmask;
    lo.ops.assign(seg.ops.begin(), seg.ops.begin() + seg.ops.size() / 2);
    hi.ops.assign(seg.ops.begin() + seg.ops.size() / 2, seg.ops.end());
    LQS_TRY(launch_segment(sv, ops, lo, pc, arith));
    return launch_segment(sv, ops, hi, pc, arith);
  }
  if (sv->dtype == LQS_C64) return launch_fused_t<ArF32>(sv, ops, seg, pc, arith);
  if (arith == LQS_ARITH_F64) return launch_fused_t<ArF64>(sv, ops, seg, pc, arith);
  return launch_fused_t<ArDF>(sv, ops, seg, pc, arith);
}

// Mirrors launch_segment's routing and splitting without launching: each
// register-tile program the segment will run is noted for the segment
// compiler (and queued for compilation when the mode asks, or `force`).
int jit_collect(int n, int dtype, int arith, const std::vector<KOp>& ops, const Segment& seg, const PlanCfg& pc,
                bool force, std::vector<void*>& todo) {
  if (seg.ops.size() == 1) return LQS_OK;
  const int k = std::min(pc.k, n), b = std::min(pc.b, k);
  if (k != reg_tile_qubits(dtype)) return LQS_OK;
  const int rc = note_reg_prog(n, dtype, arith, ops, seg, k, b, force, todo);
  if (rc != LQS_ERR_UNSUPPORTED) return rc;
  Segment lo, hi;
  lo.qmask = hi.qmask = seg.qmask;
  lo.ops.assign(seg.ops.begin(), seg.ops.begin() + seg.ops.size() / 2);
  hi.ops.assign(seg.ops.begin() + seg.ops.size() / 2, seg.ops.end());
  LQS_TRY(jit_collect(n, dtype, arith, ops, lo, pc, force, todo));
  return jit_collect(n, dtype, arith, ops, hi, pc, force, todo);
}

// explicit instantiations used by the measurement kernels
template int add_tile_op<ArF32>(TileProg<ArF32>&, const KOp&, int);
template int add_tile_op<ArF64>(TileProg<ArF64>&, const KOp&, int);
template int add_tile_op<ArDF>(TileProg<ArDF>&, const KOp&, int);
template void init_prog<ArF32>(TileProg<ArF32>&, int, uint64_t, int, int);
template void init_prog<ArF64>(TileProg<ArF64>&, int, uint64_t, int, int);
template void init_prog<ArDF>(TileProg<ArDF>&, int, uint64_t, int, int);

}  // namespace lqs

namespace lqs {

// One thread waits, with the kernels' bounded wait, on a shared-memory barrier
// that expects one arrival and never gets it; the wait gives up and flags the
// status exactly as a tile load that never landed would.  No copy is issued.
__global__ void k_wait_for_nothing(int* status) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait(&bar, 0)) flag_timeout(status, 16);
}

}  // namespace lqs

extern "C" int lqs_check_bounded_wait(lqs_sv* h) {
  void* dptr = nullptr;
  int n = 0, dtype = 0;
  LQS_TRY(lqs_sv_info(h, &dptr, &n, &dtype));  // validates the handle
  lqs::SV* sv = reinterpret_cast<lqs::SV*>(h);
  lqs::k_wait_for_nothing<<<1, 1, 0, sv->stream>>>(sv->d_status);
  LQS_CUDA_TRY(cudaGetLastError());
  lqs::count_launch();
  return LQS_OK;
}
