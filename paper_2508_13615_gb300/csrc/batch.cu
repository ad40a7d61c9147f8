// Batches of small independent circuits in one persistent launch.
//
// Variational workloads (Listing 1 of arxiv 2508.13615 is one such loop)
// evaluate many small circuits: each needs a forward pass, an expectation
// value and a gradient.  Run one at a time, a circuit of 10-20 qubits leaves
// most of the GPU idle and the host spends more time launching and
// synchronising than the GPU spends computing.
//
// Here the whole batch is one task graph executed by one persistent kernel.
// Every circuit is a chain of stages -- the forward segments, the Pauli
// passes that form lambda = H psi and the energy, and the adjoint reverse
// segments -- and every stage is a pass over the circuit's state, one task
// per tile of 2^k amplitudes.  Tasks are numbered level by level (the first
// stage of every circuit, then the second stage of every circuit, ...), and
// resident CTAs claim them in that order from a global counter.  A task may
// start once every tile of its circuit's previous stage is done (a
// per-stage completion counter).  Since those tiles carry smaller numbers,
// they were claimed earlier by CTAs that are running, so the waits always
// end; each wait is bounded all the same (2 s of the global timer), and a
// wait that gives up flags the batch and every CTA leaves.  Tiles of many
// circuits are in flight at once, so all SMs work on the batch whatever the
// sizes of its circuits.
//
// Energies and gradients are reduced without float atomics: each task writes
// its per-word or per-generator partial sums to its own slot, and a second
// kernel adds them per circuit in a fixed order (deterministic results).
//
// Host side: the plans (segments and passes) depend only on a circuit's
// structure, so they are cached by structure and built for new structures on
// several host threads; device buffers are kept between calls and only grow.
// The tile shape (tile qubits k, contiguous low qubits b) of each qubit count
// comes from lqs_batch_autotune when it has timed one, else from defaults.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "arith.cuh"
#include "lqs_internal.cuh"
#include "measure_common.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"

namespace lqs {

template <class A> int add_tile_op(TileProg<A>& P, const KOp& o, int gslot);
template <class A> void init_prog(TileProg<A>& P, int n, uint64_t Q, int k, int b);

enum { QS_FWD = 0, QS_PAULI = 1, QS_REV = 2 };

// One pass over one circuit's state; its tiles are tasks task0 .. task0 + ntiles - 1.
struct QStage {
  TileGeom g;
  int kind, circ;
  int op0, nops, coef0;  // forward / reverse segments: ops and coefficients
  int w0, nw;            // Pauli pass: words
  int ngrad, gen0;       // reverse segment: generator slots and their parameters
  int init;              // 1: the circuit's first stage, psi starts as |0..0> (and is written)
  int lam0;              // Pauli pass: 1 = lambda starts at zero
  int dep;               // the stage that must be complete first (-1: none)
  uint32_t task0;
  uint64_t part0;        // first partial sum of this stage (ntiles x nw or ntiles x ngrad)
};
struct QCirc {
  uint64_t psi;       // offset of psi in the state pool (amplitudes); lambda follows 2^n later
  int n;
  int pas0, npas;     // its Pauli stages: circ_stages[pas0 .. pas0 + npas) are their stage indices
  int rev0, nrev;     // its reverse stages, likewise
  int grad0;          // first of its gradients in the output
  int out;            // its energy in the output
};
struct BGen {
  int param;
  double scale;
};

template <class A>
struct QArgs {
  const QStage* stages;
  int nstages;
  const int* task_stage;   // per task: its stage
  const int* circ_stages;  // per circuit: the stage indices of its Pauli passes, then of its reverse segments
  const QCirc* circ;
  int ncirc;
  const TOp* ops;
  const typename A::C* coef;
  const PWord* words;
  const double* wcoef;
  const BGen* gens;
  typename A::S* pool;
  double* part;
  int* done;     // per stage: tiles finished
  int* counter;  // next task
  int* abort;    // a wait gave up: every CTA leaves
  int* status;   // status[0] = code, status[1] = block
  uint32_t ntasks;
  int kmax;
  double* grads;     // reduction outputs
  double* energies;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait of one thread until *cnt reaches `need` (true) or the batch is
// aborted / 2 s of the global timer pass / 2^26 polls pass (false).
__device__ bool wait_count(const int* cnt, int need, const int* abort) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (ld_acquire(cnt) >= need) return true;
    if ((it & 31u) == 31u) {
      if (ld_acquire(abort)) return false;
      const uint64_t now = globaltimer_ns();
      if (it == 31u) t0 = now;
      else if (now - t0 > kWaitLimitNs) return false;
    }
    __nanosleep(128);
  }
  return false;
}

template <class A>
__device__ __forceinline__ uint64_t tile_elem(const TileGeom& G, uint64_t base, uint32_t j) {
  return base + row_offset(G, j >> G.b) + (j & ((1u << G.b) - 1u));
}

// Loads of state written by other CTAs go through L2 (ld.global.cg).
template <class S> __device__ __forceinline__ S ldcg(const S* p);
template <> __device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }

template <class A>
__device__ __forceinline__ typename A::W basis0(uint64_t tile, uint32_t j) {
  typename A::W w = A::zero();
  if (tile == 0 && j == 0) {
    if constexpr (sizeof(typename A::S) == 8) w = A::load(make_float2(1.f, 0.f));
    else w = A::load(make_double2(1.0, 0.0));
  }
  return w;
}

template <class A>
__global__ void __launch_bounds__(kTileThreads) k_batch(const QArgs<A> a) {
  using S = typename A::S;
  using W = typename A::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t tmax = 1u << a.kmax;
  W* Pt = reinterpret_cast<W*>(smem_raw);
  W* Lt = Pt + tmax;
  double* wacc = reinterpret_cast<double*>(Lt + tmax);  // [warp][slot]
  __shared__ uint32_t s_task;
  __shared__ int s_stage;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nth = blockDim.x;
  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(a.counter, 1);
      int st = -1;
      if (t < a.ntasks && !ld_acquire(a.abort)) {
        st = a.task_stage[t];
        const int dep = a.stages[st].dep;
        if (dep >= 0 && !wait_count(a.done + dep, (int)a.stages[dep].g.ntiles, a.abort)) {
          if (atomicCAS(a.status, 0, 4) == 0) a.status[1] = (int)blockIdx.x;
          atomicExch(a.abort, 1);
          st = -1;
        }
        __threadfence();
      }
      s_task = t;
      s_stage = st;
    }
    __syncthreads();
    const int st = s_stage;
    const uint32_t t = s_task;
    __syncthreads();  // s_* are rewritten only after every thread has read them
    if (st < 0) break;
    const QStage& Sg = a.stages[st];
    const QCirc C = a.circ[Sg.circ];
    const TileGeom G = Sg.g;
    const uint64_t tile = t - Sg.task0;
    const uint64_t base = tile_base(G, tile);
    const uint32_t nt = 1u << G.k;
    S* psi = a.pool + C.psi;
    S* lam = psi + (1ull << C.n);
    const typename A::C* coef = a.coef + Sg.coef0;
    if (Sg.kind == QS_FWD) {
      for (uint32_t j = tid; j < nt; j += nth)
        Pt[j] = Sg.init ? basis0<A>(tile, j) : A::load(ldcg(psi + tile_elem<A>(G, base, j)));
      __syncthreads();
      for (int i = 0; i < Sg.nops; ++i) {
        tile_apply<A>(Pt, a.ops[Sg.op0 + i], coef, base, G.k);
        __syncthreads();
      }
      for (uint32_t j = tid; j < nt; j += nth) psi[tile_elem<A>(G, base, j)] = A::store(Pt[j]);
    } else if (Sg.kind == QS_PAULI) {
      for (uint32_t i = tid; i < (uint32_t)(kTileWarps * kPassWords); i += nth) wacc[i] = 0.0;
      for (uint32_t j = tid; j < nt; j += nth) {
        const uint64_t g = tile_elem<A>(G, base, j);
        Pt[j] = Sg.init ? basis0<A>(tile, j) : A::load(ldcg(psi + g));
        Lt[j] = Sg.lam0 ? A::zero() : A::load(ldcg(lam + g));
      }
      __syncthreads();
      for (int w = 0; w < Sg.nw; ++w) {
        const PWord Wd = a.words[Sg.w0 + w];
        const bool tneg = __popcll(base & Wd.ze) & 1;
        DAcc acc{0.f, 0.f};
        if (Wd.lowbit < 0) {
          for (uint32_t j = tid; j < nt; j += nth) {
            const DFC v = to_dfc(Pt[j]);
            acc_re_conj(acc, v, v, tneg ^ (__popc(j & Wd.zl) & 1));
          }
        } else {
          const uint8_t fx[1] = {(uint8_t)Wd.lowbit};
          for (uint32_t g = tid; g < nt / 2; g += nth) {
            const uint32_t j = ins0(g, fx, 1);
            const DFC b = to_dfc(Pt[j]), c = to_dfc(Pt[j ^ Wd.xl]);
            const bool neg = tneg ^ (__popc(j & Wd.zl) & 1);
            switch (Wd.ph) {
              case 0: acc_re_conj(acc, c, b, neg); break;
              case 1: acc_im_conj(acc, c, b, !neg); break;
              case 2: acc_re_conj(acc, c, b, !neg); break;
              default: acc_im_conj(acc, c, b, neg); break;
            }
          }
          acc.s = fmul(acc.s, 2.f);
          acc.e = fmul(acc.e, 2.f);
        }
        const DF sum = warp_sum(acc);
        if (lane == 0) wacc[warp * kPassWords + w] = df2d(sum);
      }
      // lambda_j += sum_w c_w i^ph (-1)^popc((j^x) & z) psi_{j^x}
      for (uint32_t j = tid; j < nt; j += nth) {
        const DFC l0 = to_dfc(Lt[j]);
        DAcc re{l0.re.h, l0.re.l}, im{l0.im.h, l0.im.l};
        for (int w = 0; w < Sg.nw; ++w) {
          const PWord Wd = a.words[Sg.w0 + w];
          const uint32_t src = j ^ Wd.xl;
          const DFC v = to_dfc(Pt[src]);
          const bool neg = ((__popcll(base & Wd.ze) + __popc(src & Wd.zl)) & 1) != 0;
          DF vr = v.re, vi = v.im;
          if (Wd.ph & 1) {
            const DF t_ = vr;
            vr = df_neg(vi);
            vi = t_;
          }
          if (Wd.ph & 2) {
            vr = df_neg(vr);
            vi = df_neg(vi);
          }
          if (neg) {
            vr = df_neg(vr);
            vi = df_neg(vi);
          }
          df_mac(re, vr, Wd.c);
          df_mac(im, vi, Wd.c);
        }
        const DFC o{df_norm(re), df_norm(im)};
        const uint64_t g = tile_elem<A>(G, base, j);
        if constexpr (sizeof(S) == 16) lam[g] = make_double2(df2d(o.re), df2d(o.im));
        else lam[g] = make_float2(o.re.h + o.re.l, o.im.h + o.im.l);
        if (Sg.init) psi[g] = A::store(Pt[j]);
      }
      __syncthreads();
      for (int w = (int)tid; w < Sg.nw; w += (int)nth) {
        double v = 0.0;
        for (int q = 0; q < kTileWarps; ++q) v += wacc[q * kPassWords + w];
        a.part[Sg.part0 + tile * (uint64_t)Sg.nw + (uint64_t)w] = v;
      }
    } else {  // QS_REV
      for (uint32_t i = tid; i < (uint32_t)(kTileWarps * kMaxGradSlots); i += nth) wacc[i] = 0.0;
      for (uint32_t j = tid; j < nt; j += nth) {
        const uint64_t g = tile_elem<A>(G, base, j);
        Pt[j] = A::load(ldcg(psi + g));
        Lt[j] = A::load(ldcg(lam + g));
      }
      __syncthreads();
      for (int i = 0; i < Sg.nops; ++i) {
        const TOp& o = a.ops[Sg.op0 + i];
        if (o.gslot >= 0 && (base & o.ecmask) == o.ecmask) {
          const DF v = warp_sum(gen_partial<A>(Pt, Lt, o, base, G.k));
          if (lane == 0) wacc[warp * kMaxGradSlots + o.gslot] = df2d(v);
        }
        tile_apply2<A>(Pt, Lt, o, coef, base, G.k);
        __syncthreads();
      }
      for (uint32_t j = tid; j < nt; j += nth) {
        const uint64_t g = tile_elem<A>(G, base, j);
        psi[g] = A::store(Pt[j]);
        lam[g] = A::store(Lt[j]);
      }
      for (int q = (int)tid; q < Sg.ngrad; q += (int)nth) {
        double v = 0.0;
        for (int w = 0; w < kTileWarps; ++w) v += wacc[w * kMaxGradSlots + q];
        a.part[Sg.part0 + tile * (uint64_t)Sg.ngrad + (uint64_t)q] = v;
      }
    }
    __syncthreads();  // this tile's results are written
    if (tid == 0) {
      __threadfence();  // ... and visible to the CTAs that wait for this stage
      atomicAdd(a.done + st, 1);
    }
  }
}

// Per circuit (one CTA each): energy = sum over its Pauli passes and words of
// coefficient x (partials summed over tiles), gradient of each parameter =
// sum over its reverse segments' generator slots of scale x (partials summed
// over tiles); every sum in a fixed order.
template <class A>
__global__ void __launch_bounds__(256) k_batch_reduce(const QArgs<A> a) {
  __shared__ double red[kMaxGradSlots];
  const QCirc C = a.circ[blockIdx.x];
  const int tid = threadIdx.x;
  double energy = 0.0;
  for (int p = 0; p < C.npas; ++p) {
    const QStage& Sg = a.stages[a.circ_stages[C.pas0 + p]];
    for (int w = tid; w < Sg.nw; w += blockDim.x) {
      double v = 0.0;
      for (uint64_t t = 0; t < Sg.g.ntiles; ++t) v += a.part[Sg.part0 + t * (uint64_t)Sg.nw + (uint64_t)w];
      red[w] = v;
    }
    __syncthreads();
    if (tid == 0)
      for (int w = 0; w < Sg.nw; ++w) energy += a.wcoef[Sg.w0 + w] * red[w];
    __syncthreads();
  }
  if (tid == 0) a.energies[C.out] = energy;
  for (int r = 0; r < C.nrev; ++r) {
    const QStage& Sg = a.stages[a.circ_stages[C.rev0 + r]];
    for (int q = tid; q < Sg.ngrad; q += blockDim.x) {
      double v = 0.0;
      for (uint64_t t = 0; t < Sg.g.ntiles; ++t) v += a.part[Sg.part0 + t * (uint64_t)Sg.ngrad + (uint64_t)q];
      red[q] = v;
    }
    __syncthreads();
    if (tid == 0)
      for (int q = 0; q < Sg.ngrad; ++q) {
        const BGen gn = a.gens[Sg.gen0 + q];
        a.grads[C.grad0 + gn.param] += gn.scale * red[q];
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side: plans
// ---------------------------------------------------------------------------
// Tile shape of the batch kernel: k tile qubits (the shared-memory tile),
// b contiguous low qubits per tile row.
struct QShape {
  int k, b;
};
static std::mutex g_shape_mu;
static std::map<std::pair<int, int>, QShape> g_shape;  // (n, dtype) -> tuned shape

static QShape default_shape(int n, int dtype) {
  const int kb = dtype == LQS_C64 ? 12 : 11, bb = dtype == LQS_C64 ? 5 : 4;
  if (n <= kb) return QShape{n, n};
  return QShape{kb, bb};
}
static QShape shape_for(int n, int dtype) {
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shape.find({n, dtype});
    if (it != g_shape.end()) return it->second;
  }
  return default_shape(n, dtype);
}

// The structural plan of one circuit: its lowered ops' segment partition for
// the forward and the reverse sweep, and its Pauli passes.  Independent of
// parameter values, so it is cached by structure.
struct QPlan {
  std::vector<Segment> fwd, rev;  // rev: at most kMaxGradSlots generator slots per segment
  std::vector<PassPlan> passes;
};
static std::mutex g_plan_mu;
static std::map<std::string, std::shared_ptr<const QPlan>> g_plans;
constexpr size_t kMaxCachedPlans = 4096;

static std::string plan_key(const lqs_batch_item& it, int dtype, QShape sh) {
  std::string k;
  const int hdr[7] = {it.n_qubits, dtype, sh.k, sh.b, it.n_ops, it.n_terms, it.grads ? 1 : 0};
  k.append(reinterpret_cast<const char*>(hdr), sizeof hdr);
  for (int i = 0; i < it.n_ops; ++i) {
    const lqs_op& o = it.ops[i];
    const int32_t rec[6] = {o.gate, o.wires[0], o.wires[1], o.wires[2], o.wires[3], o.inverse};
    k.append(reinterpret_cast<const char*>(rec), sizeof rec);
    if (o.gate == LQS_U2 || o.gate == LQS_U4) {  // a user matrix's structure picks the kernel class
      const int m = o.gate == LQS_U2 ? 8 : 32;
      for (int j = 0; j < m; ++j) k.push_back(o.matrix && o.matrix[j] != 0.0 ? '1' : '0');
    }
  }
  for (int i = 0; i < it.n_terms; ++i) {
    const uint64_t m[2] = {it.terms[i].x_mask, it.terms[i].z_mask};
    k.append(reinterpret_cast<const char*>(m), sizeof m);
  }
  return k;
}

static int make_plan(const lqs_batch_item& it, const std::vector<KOp>& kops, const std::vector<KOp>& rev, QShape sh,
                     QPlan& P, int index) {
  const int n = it.n_qubits;
  PlanCfg pc;
  pc.k = sh.k;
  pc.b = sh.b;
  pc.max_ops = kMaxTileOps;
  LQS_TRY(plan_segments(n, kops, pc, P.fwd));
  std::vector<int> wide;
  LQS_TRY(plan_passes(n, it.terms, it.n_terms, sh.k, sh.b, P.passes, wide));
  if (!wide.empty())
    return set_error(LQS_ERR_UNSUPPORTED, "batch item " + std::to_string(index) +
                                              ": a Pauli word's X/Y qubits do not fit a tile (use lqs_adjoint_grad)");
  if (it.grads && !rev.empty() && !P.passes.empty()) {
    std::vector<Segment> rs;
    LQS_TRY(plan_segments(n, rev, pc, rs));
    for (auto& s : rs) {
      Segment cur;
      cur.qmask = s.qmask;
      int ng = 0;
      for (int i : s.ops) {
        const bool g = rev[i].param_slot >= 0 && rev[i].gen != G_NONE;
        if (g && ng == kMaxGradSlots) {
          P.rev.push_back(cur);
          cur.ops.clear();
          ng = 0;
        }
        cur.ops.push_back(i);
        ng += g;
      }
      if (!cur.ops.empty()) P.rev.push_back(cur);
    }
  }
  return LQS_OK;
}

// Everything one circuit contributes, built on a host thread.
template <class A>
struct QPart {
  std::vector<QStage> stages;  // in chain order; op0 / coef0 / w0 / gen0 relative to the vectors below
  std::vector<TOp> ops;
  std::vector<typename A::C> coef;
  std::vector<PWord> words;
  std::vector<double> wcoef;
  std::vector<BGen> gens;
  int npas = 0, nrev = 0;
  double cost = 0.0;
  int rc = LQS_OK;
  std::string err;
};

template <class A>
static int append_segs(QPart<A>& Q, int n, QShape sh, const std::vector<KOp>& kops, const std::vector<Segment>& segs,
                       int kind) {
  static thread_local TileProg<A> P;
  for (const Segment& s : segs) {
    init_prog(P, n, s.qmask, sh.k, sh.b);
    QStage st{};
    st.kind = kind;
    st.gen0 = (int)Q.gens.size();
    int ng = 0;
    for (int i : s.ops) {
      const KOp& o = kops[i];
      const bool g = kind == QS_REV && o.param_slot >= 0 && o.gen != G_NONE;
      LQS_TRY(add_tile_op(P, o, g ? ng : -1));
      if (g) {
        Q.gens.push_back(BGen{o.param_slot, o.gen_scale});
        ++ng;
      }
    }
    st.g = P.g;
    st.op0 = (int)Q.ops.size();
    st.nops = P.nops;
    st.coef0 = (int)Q.coef.size();
    st.ngrad = ng;
    Q.ops.insert(Q.ops.end(), P.op, P.op + P.nops);
    Q.coef.insert(Q.coef.end(), P.coef, P.coef + P.ncoef);
    Q.stages.push_back(st);
  }
  return LQS_OK;
}

template <class A>
static int build_part(const lqs_batch_item& it, int dtype, int index, QPart<A>& Q) {
  const int n = it.n_qubits;
  const QShape sh = shape_for(n, dtype);
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(n, it.ops, it.n_ops, it.params, it.n_params, true, kops));
  std::vector<KOp> rev;
  if (it.grads)
    for (size_t i = kops.size(); i-- > 0;) rev.push_back(inverse_op(kops[i]));
  const std::string key = plan_key(it, dtype, sh);
  std::shared_ptr<const QPlan> plan;
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto f = g_plans.find(key);
    if (f != g_plans.end()) plan = f->second;
  }
  if (!plan) {
    auto p = std::make_shared<QPlan>();
    LQS_TRY(make_plan(it, kops, rev, sh, *p, index));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (g_plans.size() >= kMaxCachedPlans) g_plans.clear();
    g_plans.emplace(key, p);
    plan = p;
  }
  LQS_TRY(append_segs(Q, n, sh, kops, plan->fwd, QS_FWD));
  for (const PassPlan& pp : plan->passes) {
    QStage st{};
    st.kind = QS_PAULI;
    st.g = geom_for(n, pp.Q, sh.k, sh.b, sizeof(typename A::S));
    st.w0 = (int)Q.words.size();
    st.nw = (int)pp.words.size();
    st.lam0 = Q.npas == 0;
    for (int w : pp.words) {
      Q.words.push_back(make_pword(st.g, it.terms[w]));
      Q.wcoef.push_back(it.terms[w].coeff);
    }
    Q.stages.push_back(st);
    ++Q.npas;
  }
  const size_t r0 = Q.stages.size();
  LQS_TRY(append_segs(Q, n, sh, rev, plan->rev, QS_REV));
  Q.nrev = (int)(Q.stages.size() - r0);
  if (!Q.stages.empty()) Q.stages[0].init = 1;
  Q.cost = std::ldexp((double)Q.stages.size() + 1.0, n);
  return LQS_OK;
}

// ---------------------------------------------------------------------------
// host side: device buffers kept between calls (grow only)
// ---------------------------------------------------------------------------
struct QArena {
  void* buf[4] = {nullptr, nullptr, nullptr, nullptr};  // descriptors, state pool, partials, counters+outputs
  size_t cap[4] = {0, 0, 0, 0};
  void* host = nullptr;  // pinned staging for descriptors and outputs
  size_t host_cap = 0;
};
static std::mutex g_arena_mu;  // one batch at a time per process: the arena is shared
static QArena g_arena[64];

static int arena_grow(QArena& A, int slot, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  if (A.cap[slot] >= bytes) return LQS_OK;
  if (A.buf[slot]) {
    cudaFree(A.buf[slot]);
    A.buf[slot] = nullptr;
    A.cap[slot] = 0;
  }
  const size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&A.buf[slot], want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQS_ERR_OOM, std::string("batch buffers: ") + cudaGetErrorString(e));
  }
  A.cap[slot] = want;
  return LQS_OK;
}
static int arena_host(QArena& A, size_t bytes) {
  if (A.host_cap >= bytes) return LQS_OK;
  if (A.host) cudaFreeHost(A.host);
  A.host = nullptr;
  A.host_cap = 0;
  const size_t want = bytes + bytes / 4 + 4096;
  cudaError_t e = cudaMallocHost(&A.host, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQS_ERR_OOM, std::string("batch host staging: ") + cudaGetErrorString(e));
  }
  A.host_cap = want;
  return LQS_OK;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class A>
static int batch_run_t(const lqs_batch_item* items, int n_items, int dtype, cudaStream_t st, int dev) {
  // 1. per-circuit parts, on up to 8 host threads
  std::vector<QPart<A>> parts((size_t)n_items);
  {
    std::atomic<int> next{0};
    auto work = [&]() {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n_items) break;
        parts[i].rc = build_part(items[i], dtype, i, parts[i]);
        if (parts[i].rc != LQS_OK) parts[i].err = lqs_last_error();
      }
    };
    const int nth = std::max(1, std::min<int>(8, (n_items + 15) / 16));
    std::vector<std::thread> th;
    for (int i = 1; i < nth; ++i) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
    for (int i = 0; i < n_items; ++i)
      if (parts[i].rc != LQS_OK) return set_error(parts[i].rc, parts[i].err);
  }
  // 2. merge: stages level by level, circuits largest first within a level
  std::vector<int> order(n_items);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return parts[x].cost > parts[y].cost; });
  std::vector<QStage> stages;
  std::vector<TOp> ops;
  std::vector<typename A::C> coef;
  std::vector<PWord> words;
  std::vector<double> wcoef;
  std::vector<BGen> gens;
  std::vector<QCirc> circ((size_t)n_items);
  std::vector<int> op0(n_items), coef0(n_items), w0(n_items), gen0(n_items);
  uint64_t pool = 0;
  int ngrads = 0, kmax = 1;
  size_t maxlev = 0;
  for (int i = 0; i < n_items; ++i) {
    const QPart<A>& Q = parts[i];
    op0[i] = (int)ops.size();
    coef0[i] = (int)coef.size();
    w0[i] = (int)words.size();
    gen0[i] = (int)gens.size();
    ops.insert(ops.end(), Q.ops.begin(), Q.ops.end());
    coef.insert(coef.end(), Q.coef.begin(), Q.coef.end());
    words.insert(words.end(), Q.words.begin(), Q.words.end());
    wcoef.insert(wcoef.end(), Q.wcoef.begin(), Q.wcoef.end());
    gens.insert(gens.end(), Q.gens.begin(), Q.gens.end());
    QCirc& C = circ[i];
    C.n = items[i].n_qubits;
    C.psi = pool;
    pool += 2ull << C.n;  // psi and lambda
    pool = align_up(pool, 32);
    C.out = i;
    C.grad0 = ngrads;
    ngrads += std::max(items[i].n_params, 0);
    maxlev = std::max(maxlev, Q.stages.size());
    for (const QStage& s : Q.stages) kmax = std::max(kmax, s.g.k);
  }
  std::vector<int> sidx(n_items, -1);  // global index of each circuit's latest stage
  std::vector<std::vector<int>> cst((size_t)n_items);  // each circuit's stage indices, chain order
  uint32_t ntasks = 0;
  uint64_t nparts = 0;
  for (size_t lev = 0; lev < maxlev; ++lev)
    for (int i : order) {
      const QPart<A>& Q = parts[i];
      if (lev >= Q.stages.size()) continue;
      QStage s = Q.stages[lev];
      s.circ = i;
      s.op0 += op0[i];
      s.coef0 += coef0[i];
      s.w0 += w0[i];
      s.gen0 += gen0[i];
      s.dep = sidx[i];
      s.task0 = ntasks;
      if (s.g.ntiles > (1ull << 30) || ntasks + s.g.ntiles > (1ull << 31))
        return set_error(LQS_ERR_UNSUPPORTED, "batch has too many tiles");
      ntasks += (uint32_t)s.g.ntiles;
      s.part0 = nparts;
      if (s.kind == QS_PAULI) nparts += s.g.ntiles * (uint64_t)s.nw;
      if (s.kind == QS_REV) nparts += s.g.ntiles * (uint64_t)s.ngrad;
      sidx[i] = (int)stages.size();
      cst[i].push_back((int)stages.size());
      stages.push_back(s);
    }
  std::vector<int> circ_stages;  // per circuit: Pauli stage indices, then reverse stage indices
  for (int i = 0; i < n_items; ++i) {
    QCirc& C = circ[i];
    const QPart<A>& Q = parts[i];
    const int nf = (int)Q.stages.size() - Q.npas - Q.nrev;
    C.pas0 = (int)circ_stages.size();
    C.npas = Q.npas;
    for (int p = 0; p < Q.npas; ++p) circ_stages.push_back(cst[i][nf + p]);
    C.rev0 = (int)circ_stages.size();
    C.nrev = Q.nrev;
    for (int r = 0; r < Q.nrev; ++r) circ_stages.push_back(cst[i][nf + Q.npas + r]);
  }
  const size_t nout = (size_t)ngrads + (size_t)n_items;
  // 3. buffers and upload (one packed copy of every descriptor)
  std::lock_guard<std::mutex> lk(g_arena_mu);
  QArena& AR = g_arena[dev];
  size_t off = 0;
  auto place = [&](size_t bytes) {
    off = align_up(off, 256);
    const size_t at = off;
    off += bytes;
    return at;
  };
  std::vector<int> task_stage(ntasks);
  for (size_t si = 0; si < stages.size(); ++si)
    std::fill(task_stage.begin() + stages[si].task0, task_stage.begin() + stages[si].task0 + stages[si].g.ntiles,
              (int)si);
  const size_t o_st = place(sizeof(QStage) * stages.size());
  const size_t o_ts = place(sizeof(int) * std::max<size_t>(ntasks, 1));
  const size_t o_cs = place(sizeof(int) * std::max<size_t>(circ_stages.size(), 1));
  const size_t o_ci = place(sizeof(QCirc) * circ.size());
  const size_t o_op = place(sizeof(TOp) * std::max<size_t>(ops.size(), 1));
  const size_t o_co = place(sizeof(typename A::C) * std::max<size_t>(coef.size(), 1));
  const size_t o_wd = place(sizeof(PWord) * std::max<size_t>(words.size(), 1));
  const size_t o_wc = place(sizeof(double) * std::max<size_t>(wcoef.size(), 1));
  const size_t o_gn = place(sizeof(BGen) * std::max<size_t>(gens.size(), 1));
  const size_t desc_bytes = align_up(off, 256);
  const size_t n_ctr = align_up(stages.size() + 8, 64);  // done[], counter, abort, status
  const size_t ctr_bytes = sizeof(int) * n_ctr;
  LQS_TRY(arena_grow(AR, 0, desc_bytes));
  LQS_TRY(arena_grow(AR, 1, sizeof(typename A::S) * std::max<uint64_t>(pool, 1)));
  LQS_TRY(arena_grow(AR, 2, sizeof(double) * std::max<uint64_t>(nparts, 1)));
  LQS_TRY(arena_grow(AR, 3, ctr_bytes + sizeof(double) * nout));
  LQS_TRY(arena_host(AR, std::max(desc_bytes, sizeof(double) * nout)));
  unsigned char* h = static_cast<unsigned char*>(AR.host);
  auto put = [&](size_t at, const void* src, size_t bytes) {
    if (bytes) std::memcpy(h + at, src, bytes);
  };
  put(o_st, stages.data(), sizeof(QStage) * stages.size());
  put(o_ts, task_stage.data(), sizeof(int) * task_stage.size());
  put(o_cs, circ_stages.data(), sizeof(int) * circ_stages.size());
  put(o_ci, circ.data(), sizeof(QCirc) * circ.size());
  put(o_op, ops.data(), sizeof(TOp) * ops.size());
  put(o_co, coef.data(), sizeof(typename A::C) * coef.size());
  put(o_wd, words.data(), sizeof(PWord) * words.size());
  put(o_wc, wcoef.data(), sizeof(double) * wcoef.size());
  put(o_gn, gens.data(), sizeof(BGen) * gens.size());
  unsigned char* d = static_cast<unsigned char*>(AR.buf[0]);
  LQS_CUDA_TRY(cudaMemcpyAsync(d, h, desc_bytes, cudaMemcpyHostToDevice, st));
  int* ctr = static_cast<int*>(AR.buf[3]);
  double* outs = reinterpret_cast<double*>(static_cast<unsigned char*>(AR.buf[3]) + ctr_bytes);
  LQS_CUDA_TRY(cudaMemsetAsync(AR.buf[3], 0, ctr_bytes + sizeof(double) * nout, st));
  QArgs<A> a{};
  a.stages = reinterpret_cast<const QStage*>(d + o_st);
  a.nstages = (int)stages.size();
  a.task_stage = reinterpret_cast<const int*>(d + o_ts);
  a.circ_stages = reinterpret_cast<const int*>(d + o_cs);
  a.circ = reinterpret_cast<const QCirc*>(d + o_ci);
  a.ncirc = n_items;
  a.ops = reinterpret_cast<const TOp*>(d + o_op);
  a.coef = reinterpret_cast<const typename A::C*>(d + o_co);
  a.words = reinterpret_cast<const PWord*>(d + o_wd);
  a.wcoef = reinterpret_cast<const double*>(d + o_wc);
  a.gens = reinterpret_cast<const BGen*>(d + o_gn);
  a.pool = static_cast<typename A::S*>(AR.buf[1]);
  a.part = static_cast<double*>(AR.buf[2]);
  a.done = ctr;
  a.counter = ctr + stages.size();
  a.abort = ctr + stages.size() + 1;
  a.status = ctr + stages.size() + 2;
  a.ntasks = ntasks;
  a.kmax = kmax;
  a.grads = outs;
  a.energies = outs + ngrads;
  // 4. the task kernel on every SM, then the per-circuit reduction
  const size_t smem = 2 * ((size_t)sizeof(typename A::W) << kmax) + sizeof(double) * kTileWarps * kMaxGradSlots;
  static std::once_flag attr_once;
  cudaError_t ae = cudaSuccess;
  std::call_once(attr_once, [&] {
    ae = cudaFuncSetAttribute(k_batch<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  LQS_CUDA_TRY(ae);
  int sms = 1, per_sm = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  LQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<A>, kTileThreads, smem));
  // every CTA must be resident (a waiting task relies on the CTAs running earlier tasks)
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ntasks, (uint64_t)std::max(per_sm, 1) * sms));
  if (ntasks) {
    const std::string pname = std::string("k_batch/") + arith_tag(dtype, std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF);
    ProfScope ps(st, pname.c_str(), 0.0, 0.0);
    k_batch<A><<<grid, kTileThreads, smem, st>>>(a);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
  }
  {
    ProfScope ps(st, "k_batch_reduce", 0.0, 0.0);
    k_batch_reduce<A><<<(unsigned)n_items, 256, 0, st>>>(a);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
  }
  int status[4] = {0, 0, 0, 0};
  LQS_CUDA_TRY(cudaMemcpyAsync(h, outs, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
  LQS_CUDA_TRY(cudaMemcpyAsync(status, a.status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  LQS_CUDA_TRY(cudaStreamSynchronize(st));
  if (status[0])
    return set_error(LQS_ERR_TIMEOUT, "batch: a device-side wait gave up (block " + std::to_string(status[1]) + ")");
  const double* ho = reinterpret_cast<const double*>(h);
  for (int i = 0; i < n_items; ++i) {
    const lqs_batch_item& it = items[i];
    *it.energy = ho[ngrads + i];
    if (it.grads)
      for (int q = 0; q < it.n_params; ++q) it.grads[q] = ho[circ[i].grad0 + q];
  }
  return LQS_OK;
}

static int validate_batch(const lqs_batch_item* items, int n_items, int dtype) {
  if (n_items < 0 || (n_items > 0 && !items)) return set_error(LQS_ERR_ARG, "bad batch");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  for (int i = 0; i < n_items; ++i) {
    const lqs_batch_item& it = items[i];
    if (it.n_qubits < 1 || it.n_qubits > 26)
      return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": qubit count outside [1, 26]");
    if (!it.energy) return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": energy pointer is NULL");
    if (it.n_ops < 0 || (it.n_ops > 0 && !it.ops))
      return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": bad ops");
    if (it.n_terms < 0 || (it.n_terms > 0 && !it.terms))
      return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": bad terms");
    const uint64_t lim = (1ull << it.n_qubits) - 1;
    for (int w = 0; w < it.n_terms; ++w)
      if ((it.terms[w].x_mask | it.terms[w].z_mask) & ~lim)
        return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": term acts on a qubit >= n");
  }
  return LQS_OK;
}

static int batch_dispatch(const lqs_batch_item* items, int n_items, int dtype, cudaStream_t st) {
  int dev = 0;
  LQS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  if (dtype == LQS_C64) return batch_run_t<ArF32>(items, n_items, dtype, st, dev);
  if (current_arith(LQS_ARITH_AUTO) == LQS_ARITH_F64) return batch_run_t<ArF64>(items, n_items, dtype, st, dev);
  return batch_run_t<ArDF>(items, n_items, dtype, st, dev);
}

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_batch_run(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream) {
  LQS_TRY(validate_batch(items, n_items, dtype));
  if (n_items == 0) return LQS_OK;
  return batch_dispatch(items, n_items, dtype, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" int lqs_batch_autotune(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream, int repeats,
                                  int* n_tuned) {
  if (n_tuned) *n_tuned = 0;
  LQS_TRY(validate_batch(items, n_items, dtype));
  if (repeats < 1 || repeats > 100) return set_error(LQS_ERR_ARG, "repeats must be in [1, 100]");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int kb = dtype == LQS_C64 ? 12 : 11, bb = dtype == LQS_C64 ? 5 : 4;
  std::map<int, std::vector<lqs_batch_item>> by_n;
  for (int i = 0; i < n_items; ++i)
    if (items[i].n_qubits > kb - 1) by_n[items[i].n_qubits].push_back(items[i]);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LQS_CUDA_TRY(cudaEventCreate(&e0));
  LQS_CUDA_TRY(cudaEventCreate(&e1));
  int rc = LQS_OK, tuned = 0;
  for (auto& kv : by_n) {
    const int n = kv.first;
    std::vector<QShape> cand;
    for (int k : {kb, kb - 1})
      for (int b : {bb, bb - 1})
        if (k <= n && b >= 1 && b <= k - 2) cand.push_back(QShape{k, b});
    if (n <= kb) cand.push_back(QShape{n, n});
    QShape best{0, 0};
    float best_ms = 0.f;
    for (const QShape& c : cand) {
      {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        g_shape[{n, dtype}] = c;
      }
      rc = batch_dispatch(kv.second.data(), (int)kv.second.size(), dtype, st);  // builds plans, warms up
      if (rc != LQS_OK) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < repeats && rc == LQS_OK; ++r)
        rc = batch_dispatch(kv.second.data(), (int)kv.second.size(), dtype, st);
      cudaEventRecord(e1, st);
      if (rc != LQS_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "batch autotune timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best.k == 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
    std::lock_guard<std::mutex> lk(g_shape_mu);
    if (rc != LQS_OK || best.k == 0) {
      g_shape.erase({n, dtype});
      break;
    }
    g_shape[{n, dtype}] = best;
    ++tuned;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_tuned) *n_tuned = tuned;
  return rc;
}
