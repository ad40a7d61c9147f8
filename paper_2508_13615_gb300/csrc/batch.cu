// Batches of small independent circuits in one persistent launch.
//
// Variational workloads (Listing 1 of arxiv 2508.13615 is one such loop)
// evaluate many small circuits: each needs a forward pass, an expectation
// value and a gradient.  Launching every step of every circuit separately is
// bound by launch and synchronisation latency, not by the GPU.  Here one
// persistent kernel processes the whole batch: each CTA claims a circuit from
// a work counter (largest first, for load balance) and runs all of it --
// |0..0>, the forward segments, the Pauli passes that build lambda = H psi and
// the energy, and the adjoint reverse sweep -- on its own scratch copy of the
// state, staging tiles in shared memory.  Nothing crosses CTAs, so there is no
// grid-wide synchronisation, and the per-circuit gradient sums are reduced
// inside the CTA in a fixed order (deterministic).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <thread>
#include <string>
#include <vector>

#include "arith.cuh"
#include "lqs_internal.cuh"
#include "measure_common.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"

namespace lqs {

template <class A> int add_tile_op(TileProg<A>& P, const KOp& o, int gslot);
template <class A> void init_prog(TileProg<A>& P, int n, uint64_t Q, int k, int b);

struct BCirc {
  int n;
  int fwd0, nfwd;  // forward segments
  int pas0, npas;  // Pauli passes (lambda and energy)
  int rev0, nrev;  // reverse (adjoint) segments
  int grad0;       // offset of this circuit's gradients in the output
  int out;         // index of this circuit in the outputs
};
struct BSeg {
  TileGeom g;
  int op0, nops, coef0, ngrad, gen0;
};
struct BPass {
  TileGeom g;
  int w0, nw;
};
struct BGen {
  int param;
  double scale;
};

template <class A>
struct BatchArgs {
  const BCirc* circ;
  const int* order;
  int ncirc;
  const BSeg* segs;
  const TOp* ops;
  const typename A::C* coef;
  const BPass* passes;
  const PWord* words;
  const double* wcoef;
  const BGen* gens;
  typename A::S* scratch;
  uint64_t per_cta;  // amplitudes of scratch per CTA (psi then lambda)
  int* counter;
  double* grads;
  double* energies;
  int kmax;
};

template <class A>
__device__ __forceinline__ uint64_t tile_elem(const TileGeom& G, uint64_t base, uint32_t j) {
  return base + row_offset(G, j >> G.b) + (j & ((1u << G.b) - 1u));
}

template <class A>
__global__ void __launch_bounds__(kTileThreads) k_batch(const BatchArgs<A> a) {
  using S = typename A::S;
  using W = typename A::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t tmax = 1u << a.kmax;
  W* Pt = reinterpret_cast<W*>(smem_raw);
  W* Lt = Pt + tmax;
  double* wacc = reinterpret_cast<double*>(Lt + tmax);  // [warp][slot]
  __shared__ int s_ci;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nth = blockDim.x;
  S* psi = a.scratch + (uint64_t)blockIdx.x * a.per_cta;
  S* lam = psi + a.per_cta / 2;
  for (;;) {
    if (tid == 0) s_ci = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ci = s_ci;
    __syncthreads();
    if (ci >= a.ncirc) break;
    const BCirc C = a.circ[a.order[ci]];
    const uint64_t N = 1ull << C.n;
    for (uint64_t i = tid; i < N; i += nth) psi[i] = A::store(A::zero());
    __syncthreads();
    if (tid == 0) {
      W one = A::zero();
      if constexpr (sizeof(S) == 8) one = make_float2(1.f, 0.f);
      psi[0] = A::store(one);
      if constexpr (sizeof(S) == 16) psi[0] = make_double2(1.0, 0.0);
    }
    __syncthreads();
    // ---- forward segments ----
    for (int s = 0; s < C.nfwd; ++s) {
      const BSeg sg = a.segs[C.fwd0 + s];
      const uint32_t nt = 1u << sg.g.k;
      for (uint64_t t = 0; t < sg.g.ntiles; ++t) {
        const uint64_t base = tile_base(sg.g, t);
        for (uint32_t j = tid; j < nt; j += nth) Pt[j] = A::load(psi[tile_elem<A>(sg.g, base, j)]);
        __syncthreads();
        for (int i = 0; i < sg.nops; ++i) {
          tile_apply<A>(Pt, a.ops[sg.op0 + i], a.coef + sg.coef0, base, sg.g.k);
          __syncthreads();
        }
        for (uint32_t j = tid; j < nt; j += nth) psi[tile_elem<A>(sg.g, base, j)] = A::store(Pt[j]);
        __syncthreads();
      }
    }
    // ---- lambda = H psi and the energy ----
    double energy = 0.0;
    for (int p = 0; p < C.npas; ++p) {
      const BPass ps = a.passes[C.pas0 + p];
      const uint32_t nt = 1u << ps.g.k;
      for (int i = tid; i < kTileWarps * kPassWords; i += nth) wacc[i] = 0.0;
      __syncthreads();
      for (uint64_t t = 0; t < ps.g.ntiles; ++t) {
        const uint64_t base = tile_base(ps.g, t);
        for (uint32_t j = tid; j < nt; j += nth) {
          const uint64_t g = tile_elem<A>(ps.g, base, j);
          Pt[j] = A::load(psi[g]);
          Lt[j] = p == 0 ? A::zero() : A::load(lam[g]);
        }
        __syncthreads();
        for (int w = 0; w < ps.nw; ++w) {
          const PWord Wd = a.words[ps.w0 + w];
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
          if (lane == 0) wacc[warp * kPassWords + w] += df2d(sum);
        }
        // lambda_j += sum_w c_w i^ph (-1)^popc((j^x) & z) psi_{j^x}
        for (uint32_t j = tid; j < nt; j += nth) {
          const DFC l0 = to_dfc(Lt[j]);
          DAcc re{l0.re.h, l0.re.l}, im{l0.im.h, l0.im.l};
          for (int w = 0; w < ps.nw; ++w) {
            const PWord Wd = a.words[ps.w0 + w];
            const uint32_t src = j ^ Wd.xl;
            const DFC v = to_dfc(Pt[src]);
            const bool neg = ((__popcll(base & Wd.ze) + __popc(src & Wd.zl)) & 1) != 0;
            DF vr = v.re, vi = v.im;
            if (Wd.ph & 1) { const DF t_ = vr; vr = df_neg(vi); vi = t_; }
            if (Wd.ph & 2) { vr = df_neg(vr); vi = df_neg(vi); }
            if (neg) { vr = df_neg(vr); vi = df_neg(vi); }
            df_mac(re, vr, Wd.c);
            df_mac(im, vi, Wd.c);
          }
          const DFC out{df_norm(re), df_norm(im)};
          if constexpr (sizeof(S) == 16) lam[tile_elem<A>(ps.g, base, j)] = make_double2(df2d(out.re), df2d(out.im));
          else lam[tile_elem<A>(ps.g, base, j)] = make_float2(out.re.h + out.re.l, out.im.h + out.im.l);
        }
        __syncthreads();
      }
      if (tid == 0)
        for (int w = 0; w < ps.nw; ++w) {
          double v = 0.0;
          for (int q = 0; q < kTileWarps; ++q) v += wacc[q * kPassWords + w];
          energy += a.wcoef[ps.w0 + w] * v;
        }
      __syncthreads();
    }
    if (tid == 0) a.energies[C.out] = energy;
    // ---- adjoint reverse sweep ----
    for (int s = 0; s < C.nrev; ++s) {
      const BSeg sg = a.segs[C.rev0 + s];
      const uint32_t nt = 1u << sg.g.k;
      for (int i = tid; i < kTileWarps * kMaxGradSlots; i += nth) wacc[i] = 0.0;
      __syncthreads();
      for (uint64_t t = 0; t < sg.g.ntiles; ++t) {
        const uint64_t base = tile_base(sg.g, t);
        for (uint32_t j = tid; j < nt; j += nth) {
          const uint64_t g = tile_elem<A>(sg.g, base, j);
          Pt[j] = A::load(psi[g]);
          Lt[j] = A::load(lam[g]);
        }
        __syncthreads();
        for (int i = 0; i < sg.nops; ++i) {
          const TOp& o = a.ops[sg.op0 + i];
          if (o.gslot >= 0 && (base & o.ecmask) == o.ecmask) {
            const DF v = warp_sum(gen_partial<A>(Pt, Lt, o, base, sg.g.k));
            if (lane == 0) wacc[warp * kMaxGradSlots + o.gslot] += df2d(v);
          }
          tile_apply<A>(Pt, o, a.coef + sg.coef0, base, sg.g.k);
          tile_apply<A>(Lt, o, a.coef + sg.coef0, base, sg.g.k);
          __syncthreads();
        }
        for (uint32_t j = tid; j < nt; j += nth) {
          const uint64_t g = tile_elem<A>(sg.g, base, j);
          psi[g] = A::store(Pt[j]);
          lam[g] = A::store(Lt[j]);
        }
        __syncthreads();
      }
      if (tid == 0)
        for (int q = 0; q < sg.ngrad; ++q) {
          double v = 0.0;
          for (int w = 0; w < kTileWarps; ++w) v += wacc[w * kMaxGradSlots + q];
          const BGen gn = a.gens[sg.gen0 + q];
          a.grads[C.grad0 + gn.param] += gn.scale * v;
        }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <class A>
struct BatchBuild {
  std::vector<BCirc> circ;
  std::vector<BSeg> segs;
  std::vector<TOp> ops;
  std::vector<typename A::C> coef;
  std::vector<BPass> passes;
  std::vector<PWord> words;
  std::vector<double> wcoef;
  std::vector<BGen> gens;
  std::vector<double> cost;
  int nmax = 1, kmax = 1, ngrads = 0;
};

template <class A>
static int append_segments(BatchBuild<A>& B, int n, int k, int b, const std::vector<KOp>& kops,
                           const std::vector<Segment>& segs, bool adjoint) {
  static thread_local TileProg<A> P;
  for (const Segment& s : segs) {
    init_prog(P, n, s.qmask, k, b);
    BSeg bs{};
    bs.gen0 = (int)B.gens.size();
    int ng = 0;
    for (int i : s.ops) {
      const KOp& o = kops[i];
      const bool g = adjoint && o.param_slot >= 0 && o.gen != G_NONE;
      LQS_TRY(add_tile_op(P, o, g ? ng : -1));
      if (g) {
        B.gens.push_back(BGen{o.param_slot, o.gen_scale});
        ++ng;
      }
    }
    bs.g = P.g;
    bs.op0 = (int)B.ops.size();
    bs.nops = P.nops;
    bs.coef0 = (int)B.coef.size();
    bs.ngrad = ng;
    B.ops.insert(B.ops.end(), P.op, P.op + P.nops);
    B.coef.insert(B.coef.end(), P.coef, P.coef + P.ncoef);
    B.segs.push_back(bs);
  }
  return LQS_OK;
}

template <class A>
static int build_batch(const lqs_batch_item* items, int n_items, int dtype, BatchBuild<A>& B) {
  const int kb = dtype == LQS_C64 ? 12 : 11, bb = dtype == LQS_C64 ? 5 : 4;
  for (int ci = 0; ci < n_items; ++ci) {
    const lqs_batch_item& it = items[ci];
    const int n = it.n_qubits;
    std::vector<KOp> kops;
    LQS_TRY(lower_ops(n, it.ops, it.n_ops, it.params, it.n_params, true, kops));
    const int k = std::min(n, kb), b = n <= kb ? n : bb;
    PlanCfg pc;
    pc.k = k;
    pc.b = b;
    pc.max_ops = kMaxTileOps;
    BCirc C{};
    C.n = n;
    C.out = ci;
    C.grad0 = B.ngrads;
    B.ngrads += std::max(it.n_params, 0);
    // forward
    std::vector<Segment> segs;
    LQS_TRY(plan_segments(n, kops, pc, segs));
    C.fwd0 = (int)B.segs.size();
    LQS_TRY(append_segments(B, n, k, b, kops, segs, false));
    C.nfwd = (int)B.segs.size() - C.fwd0;
    // passes
    std::vector<PassPlan> pp;
    std::vector<int> wide;
    LQS_TRY(plan_passes(n, it.terms, it.n_terms, k, b, pp, wide));
    if (!wide.empty())
      return set_error(LQS_ERR_UNSUPPORTED, "batch item " + std::to_string(ci) +
                                                ": a Pauli word's X/Y qubits do not fit a tile (use lqs_adjoint_grad)");
    C.pas0 = (int)B.passes.size();
    for (auto& p : pp) {
      BPass bp{};
      bp.g = geom_for(n, p.Q, k, b, sizeof(typename A::S));
      bp.w0 = (int)B.words.size();
      bp.nw = (int)p.words.size();
      for (int w : p.words) {
        B.words.push_back(make_pword(bp.g, it.terms[w]));
        B.wcoef.push_back(it.terms[w].coeff);
      }
      B.passes.push_back(bp);
    }
    C.npas = (int)B.passes.size() - C.pas0;
    // reverse sweep (only when gradients are wanted)
    C.rev0 = (int)B.segs.size();
    if (it.grads && !kops.empty()) {
      std::vector<KOp> rev;
      for (size_t i = kops.size(); i-- > 0;) rev.push_back(inverse_op(kops[i]));
      std::vector<Segment> rs;
      LQS_TRY(plan_segments(n, rev, pc, rs));
      std::vector<Segment> rs2;  // at most kMaxGradSlots generator slots per segment
      for (auto& s : rs) {
        Segment cur;
        cur.qmask = s.qmask;
        int ng = 0;
        for (int i : s.ops) {
          const bool g = rev[i].param_slot >= 0 && rev[i].gen != G_NONE;
          if (g && ng == kMaxGradSlots) {
            rs2.push_back(cur);
            cur.ops.clear();
            ng = 0;
          }
          cur.ops.push_back(i);
          ng += g;
        }
        if (!cur.ops.empty()) rs2.push_back(cur);
      }
      LQS_TRY(append_segments(B, n, k, b, rev, rs2, true));
    }
    C.nrev = (int)B.segs.size() - C.rev0;
    B.circ.push_back(C);
    B.cost.push_back(std::ldexp((double)(C.nfwd + C.npas + 2 * C.nrev + 1), n));
    B.nmax = std::max(B.nmax, n);
    B.kmax = std::max(B.kmax, k);
  }
  return LQS_OK;
}

template <class T>
static int upload(const std::vector<T>& v, T** d, cudaStream_t st) {
  *d = nullptr;
  if (v.empty()) return LQS_OK;
  LQS_CUDA_TRY(cudaMalloc(d, sizeof(T) * v.size()));
  LQS_CUDA_TRY(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return LQS_OK;
}

template <class A>
static int batch_run_t(const lqs_batch_item* items, const std::vector<int>& sel, int dtype, cudaStream_t st,
                       int max_grid) {
  const int n_sel = (int)sel.size();
  if (n_sel == 0) return LQS_OK;
  std::vector<lqs_batch_item> sub(n_sel);
  for (int i = 0; i < n_sel; ++i) sub[i] = items[sel[i]];
  BatchBuild<A> B;
  LQS_TRY(build_batch(sub.data(), n_sel, dtype, B));
  std::vector<int> order(n_sel);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return B.cost[x] > B.cost[y]; });
  int dev = 0, sms = 1;
  LQS_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 2 * ((size_t)sizeof(typename A::W) << B.kmax) + sizeof(double) * kTileWarps * kMaxGradSlots;
  LQS_CUDA_TRY(cudaFuncSetAttribute(k_batch<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 1;
  LQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<A>, kTileThreads, smem));
  const int grid = std::max(1, std::min({n_sel, std::max(per_sm, 1) * sms, std::max(max_grid, 1)}));
  std::vector<void*> owned;
  auto fail = [&](int rc) {
    cudaStreamSynchronize(st);
    for (void* q : owned) cudaFree(q);
    return rc;
  };
  BatchArgs<A> a{};
  BCirc* dc;
  int* dorder;
  BSeg* dsegs;
  TOp* dops;
  typename A::C* dcoef;
  BPass* dpass;
  PWord* dwords;
  double* dwcoef;
  BGen* dgens;
  int rc;
#define UP(vec, ptr)                                           \
  if ((rc = upload(vec, &ptr, st)) != LQS_OK) return fail(rc); \
  owned.push_back(ptr);
  UP(B.circ, dc);
  UP(order, dorder);
  UP(B.segs, dsegs);
  UP(B.ops, dops);
  UP(B.coef, dcoef);
  UP(B.passes, dpass);
  UP(B.words, dwords);
  UP(B.wcoef, dwcoef);
  UP(B.gens, dgens);
#undef UP
  const uint64_t per_cta = 2ull << B.nmax;
  void *scratch = nullptr, *counter = nullptr, *outs = nullptr;
  cudaError_t e = cudaMalloc(&scratch, sizeof(typename A::S) * per_cta * grid);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc(batch scratch)"));
  owned.push_back(scratch);
  e = cudaMalloc(&counter, 16);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc(batch counter)"));
  owned.push_back(counter);
  const size_t nout = (size_t)B.ngrads + n_sel;
  e = cudaMalloc(&outs, sizeof(double) * std::max<size_t>(nout, 1));
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc(batch outputs)"));
  owned.push_back(outs);
  if ((e = cudaMemsetAsync(counter, 0, 16, st)) != cudaSuccess) return fail(cuda_error(e, "cudaMemsetAsync"));
  if ((e = cudaMemsetAsync(outs, 0, sizeof(double) * std::max<size_t>(nout, 1), st)) != cudaSuccess)
    return fail(cuda_error(e, "cudaMemsetAsync"));
  a.circ = dc;
  a.order = dorder;
  a.ncirc = n_sel;
  a.segs = dsegs;
  a.ops = dops;
  a.coef = dcoef;
  a.passes = dpass;
  a.words = dwords;
  a.wcoef = dwcoef;
  a.gens = dgens;
  a.scratch = static_cast<typename A::S*>(scratch);
  a.per_cta = per_cta;
  a.counter = static_cast<int*>(counter);
  a.grads = static_cast<double*>(outs);
  a.energies = static_cast<double*>(outs) + B.ngrads;
  a.kmax = B.kmax;
  {
    const std::string pname = std::string("k_batch/") + arith_tag(dtype, std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF);
    ProfScope ps(st, pname.c_str(), 0.0, 0.0);
    k_batch<A><<<grid, kTileThreads, smem, st>>>(a);
    count_launch();
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(e, "k_batch launch"));
  std::vector<double> h(nout);
  if (nout && (e = cudaMemcpyAsync(h.data(), outs, sizeof(double) * nout, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(cuda_error(e, "cudaMemcpyAsync(batch outputs)"));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_error(e, "k_batch"));
  for (void* q : owned) cudaFree(q);
  for (int ci = 0; ci < n_sel; ++ci) {
    const lqs_batch_item& it = sub[ci];
    *it.energy = h[B.ngrads + ci];
    if (it.grads)
      for (int q = 0; q < it.n_params; ++q) it.grads[q] = h[B.circ[ci].grad0 + q];
  }
  return LQS_OK;
}

// Larger circuits: the full-GPU fused and adjoint kernels, driven by a few
// host threads with their own streams and reusable buffers (no allocation
// per circuit), so host-side planning and synchronisation of one circuit
// overlap with GPU work of the others.
struct Worker {
  cudaStream_t st = nullptr;
  void* state = nullptr;
  int* status = nullptr;
  void* scratch[3] = {nullptr, nullptr, nullptr};
  size_t scratch_bytes[3] = {0, 0, 0};
};

static int run_large(const lqs_batch_item* items, const std::vector<int>& large, int dtype, int dev, int nworkers,
                     std::string& err) {
  if (large.empty()) return LQS_OK;
  int nmax = 1;
  for (int i : large) nmax = std::max(nmax, items[i].n_qubits);
  const size_t amp = dtype == LQS_C64 ? 8 : 16;
  std::vector<Worker> W((size_t)std::max(1, std::min<int>(nworkers, (int)large.size())));
  int rc = LQS_OK;
  for (auto& w : W) {
    cudaError_t e = cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&w.state, amp << nmax);
    if (e == cudaSuccess) e = cudaMalloc(&w.status, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, 64, w.st);
    if (e == cudaSuccess) e = cudaMalloc(&w.scratch[0], amp << nmax);  // lambda
    if (e != cudaSuccess) {
      rc = cuda_error(e, "batch worker buffers");
      break;
    }
    w.scratch_bytes[0] = amp << nmax;
  }
  std::atomic<int> next{0}, first_rc{LQS_OK};
  std::mutex emu;
  auto body = [&](Worker* w) {
    cudaSetDevice(dev);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (;;) {
      const int idx = next.fetch_add(1);
      if (idx >= (int)large.size() || first_rc.load() != LQS_OK) break;
      const lqs_batch_item& it = items[large[idx]];
      SV sv;
      sv.n = it.n_qubits;
      sv.dtype = dtype;
      sv.d = w->state;
      sv.owns = false;
      sv.stream = w->st;
      sv.device = dev;
      sv.sms = sms;
      sv.d_status = w->status;
      for (int q = 0; q < 3; ++q) {
        sv.scratch[q] = w->scratch[q];
        sv.scratch_bytes[q] = w->scratch_bytes[q];
      }
      lqs_sv* h = reinterpret_cast<lqs_sv*>(&sv);
      int r = lqs_sv_set_basis(h, 0);
      if (r == LQS_OK) r = lqs_apply_fused(h, it.ops, it.n_ops, it.params, it.n_params, nullptr);
      if (r == LQS_OK) {
        if (it.grads)
          r = lqs_adjoint_grad(h, it.ops, it.n_ops, it.params, it.n_params, it.terms, it.n_terms, it.grads,
                               it.energy);
        else
          r = lqs_expval(h, it.terms, it.n_terms, it.energy, nullptr);
      }
      for (int q = 0; q < 3; ++q) {  // keep buffers the calls grew
        w->scratch[q] = sv.scratch[q];
        w->scratch_bytes[q] = sv.scratch_bytes[q];
      }
      if (r != LQS_OK) {
        std::lock_guard<std::mutex> lk(emu);
        if (first_rc.load() == LQS_OK) err = lqs_last_error();
        first_rc.store(r);
      }
    }
  };
  if (rc == LQS_OK) {
    std::vector<std::thread> th;
    for (auto& w : W) th.emplace_back(body, &w);
    for (auto& t : th) t.join();
    rc = first_rc.load();
  }
  for (auto& w : W) {
    if (w.st) cudaStreamSynchronize(w.st);
    for (int q = 0; q < 3; ++q)
      if (w.scratch[q]) cudaFree(w.scratch[q]);
    if (w.state) cudaFree(w.state);
    if (w.status) cudaFree(w.status);
    if (w.st) cudaStreamDestroy(w.st);
  }
  return rc;
}

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_batch_run(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream) {
  if (n_items < 0 || (n_items > 0 && !items)) return set_error(LQS_ERR_ARG, "bad batch");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  if (n_items == 0) return LQS_OK;
  for (int i = 0; i < n_items; ++i) {
    const lqs_batch_item& it = items[i];
    if (it.n_qubits < 1 || it.n_qubits > 26)
      return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": qubit count outside [1, 26]");
    if (!it.energy) return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": energy pointer is NULL");
    if (it.n_terms < 0 || (it.n_terms > 0 && !it.terms))
      return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": bad terms");
    const uint64_t lim = (1ull << it.n_qubits) - 1;
    for (int w = 0; w < it.n_terms; ++w)
      if ((it.terms[w].x_mask | it.terms[w].z_mask) & ~lim)
        return set_error(LQS_ERR_ARG, "batch item " + std::to_string(i) + ": term acts on a qubit >= n");
  }
  // Circuits whose state is one tile run whole inside one CTA of the
  // persistent kernel; larger ones go to the full-GPU kernels (worker threads).
  const int single_tile = dtype == LQS_C64 ? 12 : 11;
  std::vector<int> small, large;
  for (int i = 0; i < n_items; ++i) (items[i].n_qubits <= single_tile ? small : large).push_back(i);
  cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
  LQS_CUDA_TRY(cudaStreamSynchronize(user));
  int dev = 0, sms = 1;
  LQS_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = nullptr;
  LQS_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int rc_small = LQS_OK;
  std::string err_small, err_large;
  // the persistent kernel (launched from its own thread: it synchronises at the end)
  std::thread ts([&] {
    cudaSetDevice(dev);
    const int cap = large.empty() ? 4 * sms : sms / 2;  // leave SMs to the large circuits
    if (dtype == LQS_C64) rc_small = batch_run_t<ArF32>(items, small, dtype, st, cap);
    else if (current_arith(LQS_ARITH_AUTO) == LQS_ARITH_F64) rc_small = batch_run_t<ArF64>(items, small, dtype, st, cap);
    else rc_small = batch_run_t<ArDF>(items, small, dtype, st, cap);
    if (rc_small != LQS_OK) err_small = lqs_last_error();
  });
  const int rc_large = run_large(items, large, dtype, dev, 4, err_large);
  ts.join();
  cudaStreamDestroy(st);
  if (rc_small != LQS_OK) return set_error(rc_small, err_small);
  if (rc_large != LQS_OK) return set_error(rc_large, err_large);
  return LQS_OK;
}
