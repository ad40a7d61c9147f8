// Expectation values, lambda = H psi, and the adjoint-method gradient sweep.
//
// Listing 1 of arxiv 2508.13615 drives a variational loop through
// qml.expval(H) of a Hamiltonian that is a sum of Pauli words, and through
// gradients of that expectation.  Here:
//   * <P_w> for each word: a tile pass sums Re[i^ny (-1)^popc(j & z)
//     conj(psi_{j^x}) psi_j] over amplitude pairs that lie in one tile (the
//     word's X/Y qubits are tile qubits).  Sums are double-float per thread,
//     reduced per warp every tile, and accumulated in float64 per warp; a
//     second kernel adds the per-block partials in a fixed order, so results
//     are deterministic (no floating-point atomics).
//   * lambda = H psi is built by the same passes, adding c_w P_w psi into a
//     second state buffer.
//   * The adjoint sweep (Jones & Gacon 2020, "Efficient calculation of
//     gradients in classical simulations of variational quantum algorithms")
//     runs the circuit backwards over tiles holding psi and lambda together:
//     for a gate U(theta) with dU/dtheta = -i K U, dE/dtheta = 2 Im<lambda|K|psi>
//     is accumulated before U^dagger is applied to both states.
#include <algorithm>
#include <string>
#include <cstring>
#include <type_traits>

#include "arith.cuh"
#include "jit.h"
#include "lqs_internal.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"
#include "measure_common.cuh"

namespace lqs {

template <class A> int add_tile_op(TileProg<A>& P, const KOp& o, int gslot);
template <class A> void init_prog(TileProg<A>& P, int n, uint64_t Q, int k, int b);

// ---------------------------------------------------------------------------
// Pauli-word passes
// ---------------------------------------------------------------------------
// Per-thread double-float partial sums (one per word, in shared memory) are
// flushed every kFlushTiles tiles: warp sum in double-float, then float64
// per warp.  A chain holds at most kFlushTiles * (tile amplitudes / threads)
// = 64 (complex128) or 128 (complex64) terms, which keeps the double-float
// rounding near 2^-41 relative or better.
constexpr int kFlushTiles = 8;

template <class S> struct PauliTile { static constexpr int k = 11, ept = 8; };     // complex128: 2^11
template <> struct PauliTile<float2> { static constexpr int k = 12, ept = 16; };  // complex64: 2^12

// mode bit 1: accumulate <P_w>; bit 2: add c_w P_w psi to lambda; bit 4: lambda starts at zero
template <class A, int MODE>
__global__ void __launch_bounds__(kTileThreads) k_pauli(const typename A::S* __restrict__ psi,
                                                        typename A::S* __restrict__ lam,
                                                        const __grid_constant__ PauliProg P, double* partial,
                                                        int pstride, int* status) {
  using S = typename A::S;
  // working view of a tile: complex128 tiles are converted in place to
  // double-float once per tile; complex64 amplitudes are widened on the fly
  using V = typename std::conditional<sizeof(S) == 16, DFC, float2>::type;
  constexpr int EPT = PauliTile<S>::ept;  // amplitudes per thread in a full tile
  constexpr bool kExp = MODE & 1, kLam = MODE & 2, kFresh = MODE & 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TileGeom& G = P.g;
  const uint32_t nt = 1u << G.k;
  S* buf = reinterpret_cast<S*>(smem_raw);
  S* lbuf = buf + nt;  // lambda tile (kLam)
  V* T = reinterpret_cast<V*>(buf);
  V* LT = reinterpret_cast<V*>(lbuf);
  double* wacc = reinterpret_cast<double*>(smem_raw + (size_t)nt * sizeof(S) * (kLam ? 2 : 1));
  DAcc* sacc = reinterpret_cast<DAcc*>(wacc + kTileWarps * kPassWords);  // [word][thread]
  PWord* words = reinterpret_cast<PWord*>(sacc + kPassWords * kTileThreads);  // staged copy of P.w
  uint64_t* bar = reinterpret_cast<uint64_t*>(words + kPassWords);
  for (int w = threadIdx.x; w < P.nw; w += blockDim.x) words[w] = P.w[w];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kTileWarps * kPassWords; i += blockDim.x) wacc[i] = 0.0;
  for (int w = 0; w < kPassWords; ++w) sacc[w * kTileThreads + threadIdx.x] = DAcc{0.f, 0.f};
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto flush = [&]() {
    for (int w = 0; w < P.nw; ++w) {
      const DF s = warp_sum(sacc[w * kTileThreads + threadIdx.x]);
      if (lane == 0) wacc[warp * kPassWords + w] += (words[w].lowbit >= 0 ? 2.0 : 1.0) * df2d(s);
      sacc[w * kTileThreads + threadIdx.x] = DAcc{0.f, 0.f};
    }
  };
  uint32_t phase = 0;
  bool ok = true;
  int since_flush = 0;
  for (uint64_t t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(G, t);
    if (threadIdx.x < 32) {
      // one arrival per phase: the expected bytes cover the lambda tile too
      tile_expect(G, bar, (kLam && !kFresh) ? 2u : 1u);
      tile_load_rows(G, buf, psi, base, bar);
      if (kLam && !kFresh) tile_load_rows(G, lbuf, lam, base, bar);
    }
    ok = __syncthreads_and(mbar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    if constexpr (sizeof(S) == 16) {
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        const S a = buf[j];
        T[j] = to_dfc(a);
        if (kLam && !kFresh) {
          const S c = lbuf[j];
          LT[j] = to_dfc(c);
        }
      }
      __syncthreads();
    }
    if (kExp) {
      // |psi_j|^2 of this thread's amplitudes, shared by every diagonal word
      DF p[EPT];
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const uint32_t j = threadIdx.x + i * kTileThreads;
        p[i] = DF{0.f, 0.f};
        if (j < nt) {
          const DFC v = to_dfc(T[j]);
          DAcc pa = df_prod(v.re, v.re);
          df_mac(pa, v.im, v.im);
          p[i] = df_norm(pa);
        }
      }
      for (int w = 0; w < P.nw; ++w) {
        const PWord& Wd = words[w];
        DAcc a = sacc[w * kTileThreads + threadIdx.x];
        const bool tneg = __popcll(base & Wd.ze) & 1;
        if (Wd.lowbit < 0) {
#pragma unroll
          for (int i = 0; i < EPT; ++i) {
            const uint32_t j = threadIdx.x + i * kTileThreads;
            const bool neg = tneg ^ (__popc(j & Wd.zl) & 1);
            df_acc(a, neg ? df_neg(p[i]) : p[i]);
          }
        } else {
          // pairs {j, j^x}; the two orders are conjugates, so one is counted
          // (doubled at the flush)
          const uint8_t fx[1] = {(uint8_t)Wd.lowbit};
          for (uint32_t g = threadIdx.x; g < nt / 2; g += blockDim.x) {
            const uint32_t j = ins0(g, fx, 1);
            const DFC b = to_dfc(T[j]), c = to_dfc(T[j ^ Wd.xl]);
            const bool neg = tneg ^ (__popc(j & Wd.zl) & 1);
            switch (Wd.ph) {
              case 0: acc_re_conj(a, c, b, neg); break;
              case 1: acc_im_conj(a, c, b, !neg); break;
              case 2: acc_re_conj(a, c, b, !neg); break;
              default: acc_im_conj(a, c, b, neg); break;
            }
          }
        }
        sacc[w * kTileThreads + threadIdx.x] = a;
      }
      if (++since_flush == kFlushTiles) {
        flush();
        since_flush = 0;
      }
    }
    if (kLam) {
      // lambda_j += sum_w c_w i^ph (-1)^popc((j^x) & z) psi_{j^x}
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        DAcc re{0.f, 0.f}, im{0.f, 0.f};
        if (!kFresh) {
          const DFC l0 = to_dfc(LT[j]);
          re = DAcc{l0.re.h, l0.re.l};
          im = DAcc{l0.im.h, l0.im.l};
        }
#pragma unroll 1
        for (int w = 0; w < P.nw; ++w) {
          const PWord& Wd = words[w];
          const uint32_t src = j ^ Wd.xl;
          const DFC v = to_dfc(T[src]);
          const bool neg = ((__popcll(base & Wd.ze) + __popc(src & Wd.zl)) & 1) != 0;
          DF vr = v.re, vi = v.im;  // i^ph * v
          if (Wd.ph & 1) { const DF t_ = vr; vr = df_neg(vi); vi = t_; }
          if (Wd.ph & 2) { vr = df_neg(vr); vi = df_neg(vi); }
          if (neg) { vr = df_neg(vr); vi = df_neg(vi); }
          df_mac(re, vr, Wd.c);
          df_mac(im, vi, Wd.c);
        }
        const DFC out{df_norm(re), df_norm(im)};
        // every thread reads psi from T only; lambda j is written by its own thread
        if constexpr (sizeof(S) == 16) lbuf[j] = make_double2(df2d(out.re), df2d(out.im));
        else lbuf[j] = make_float2(out.re.h + out.re.l, out.im.h + out.im.l);
      }
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x < 32) tile_store_issue(G, lam, lbuf, base);
    }
    __syncthreads();  // every thread is done with the tile before it is refilled
  }
  if (kExp && since_flush) flush();
  if (kLam && threadIdx.x < 32) bulk_wait0();
  if (!ok && threadIdx.x == 0) {
    flag_timeout(status, 2);
    mbar_wait(bar, phase ^ 1u);
  }
  __syncthreads();
  if (kExp)
    for (int w = threadIdx.x; w < P.nw; w += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < kTileWarps; ++q) s += wacc[q * kPassWords + w];
      partial[(size_t)w * pstride + blockIdx.x] = s;
    }
}

// One Pauli word whose X/Y qubits do not fit a tile: a global pair pass over
// (j, j^x) with j's lowest X bit clear.  Expectation partials per block
// (deterministic), and optionally lambda += c P psi for both members of the
// pair (each pair belongs to exactly one thread, so there are no races).
template <class A, bool kLam>
__global__ void __launch_bounds__(256) k_pauli_wide(const typename A::S* __restrict__ psi,
                                                    typename A::S* __restrict__ lam, uint64_t npairs, int lowbit,
                                                    uint64_t x, uint64_t z, int ph, DF c, double* partial) {
  using S = typename A::S;
  __shared__ double red[256];
  DAcc acc{0.f, 0.f};
  double dacc = 0.0;
  int cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < npairs; g += stride) {
    const uint64_t j = ((g >> lowbit) << (lowbit + 1)) | (g & ((1ull << lowbit) - 1));
    const uint64_t jp = j ^ x;
    const DFC b = to_dfc(A::load(psi[j])), a = to_dfc(A::load(psi[jp]));
    const bool neg = __popcll(j & z) & 1;
    switch (ph) {
      case 0: acc_re_conj(acc, a, b, neg); break;
      case 1: acc_im_conj(acc, a, b, !neg); break;
      case 2: acc_re_conj(acc, a, b, !neg); break;
      default: acc_im_conj(acc, a, b, neg); break;
    }
    if (++cnt == 64) {
      dacc += df2d(df_norm(acc));
      acc = DAcc{0.f, 0.f};
      cnt = 0;
    }
    if (kLam) {
      // lambda_jp += c i^ph (-1)^popc(j&z) psi_j ; lambda_j += c i^ph (-1)^popc(jp&z) psi_jp
      const uint64_t dst[2] = {jp, j};
      const DFC src[2] = {b, a};
      const bool sg[2] = {neg, (__popcll(jp & z) & 1) != 0};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const DFC l0 = to_dfc(A::load(lam[dst[q]]));
        DAcc re{l0.re.h, l0.re.l}, im{l0.im.h, l0.im.l};
        DF vr = src[q].re, vi = src[q].im;
        if (ph & 1) { const DF t_ = vr; vr = df_neg(vi); vi = t_; }
        if (ph & 2) { vr = df_neg(vr); vi = df_neg(vi); }
        if (sg[q]) { vr = df_neg(vr); vi = df_neg(vi); }
        df_mac(re, vr, c);
        df_mac(im, vi, c);
        const DFC out{df_norm(re), df_norm(im)};
        if constexpr (sizeof(S) == 16) lam[dst[q]] = make_double2(df2d(out.re), df2d(out.im));
        else lam[dst[q]] = make_float2(out.re.h + out.re.l, out.im.h + out.im.l);
      }
    }
  }
  dacc += df2d(df_norm(acc));
  red[threadIdx.x] = 2.0 * dacc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[i] = sum_b partial[i * nb + b], in a fixed order (one block per slot).
__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double sh[256];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(size_t)i * nb + b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = sh[0];
}

int k_sum_partials_launch(double* partial, int grid, double* sums, int slots, cudaStream_t st) {
  if (slots <= 0) return LQS_OK;
  k_sum_partials<<<(unsigned)slots, 256, 0, st>>>(partial, grid, sums);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

// Tile size for measurement passes: smaller than the fused default so that
// two tiles (psi and lambda) plus accumulators leave room for 2-3 CTAs per SM.
static void measure_kb(int n, int dtype, int& k, int& b) {
  k = dtype == LQS_C64 ? PauliTile<float2>::k : PauliTile<double2>::k;
  b = dtype == LQS_C64 ? 5 : 4;
  if (n <= k) { k = n; b = n; }
}

static size_t pauli_smem(size_t amp, int k, bool lam) {
  return (amp << k) * (lam ? 2 : 1) + sizeof(double) * kTileWarps * kPassWords +
         sizeof(DAcc) * kPassWords * kTileThreads + sizeof(PWord) * kPassWords + 16;
}

template <class A, int MODE>
static int launch_pauli(SV* sv, const PauliProg& P, void* lam, double* partial, int grid, int pstride) {
  const size_t amp = sizeof(typename A::S);
  // bytes: psi read, plus lambda written (and read unless fresh); flops: 8 per
  // amplitude per word (an amplitude pair product and accumulation)
  const double S = (double)sv->bytes();
  const double bytes = S * (1.0 + ((MODE & 2) ? ((MODE & 4) ? 1.0 : 2.0) : 0.0));
  const std::string pname = std::string((MODE & 2) ? "k_pauli_lambda/" : "k_pauli/") + arith_tag(sv->dtype, std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF);
  ProfScope ps(sv->stream, pname.c_str(), bytes, 8.0 * P.nw * (double)sv->N());
  const size_t smem = pauli_smem(amp, P.g.k, (MODE & 2) != 0);
  static bool attr = false;
  if (!attr) {
    LQS_CUDA_TRY(cudaFuncSetAttribute(k_pauli<A, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  k_pauli<A, MODE><<<grid, kTileThreads, smem, sv->stream>>>(static_cast<const typename A::S*>(sv->d),
                                                              static_cast<typename A::S*>(lam), P, partial,
                                                              pstride, sv->d_status);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

template <class A>
static int occupancy_grid(SV* sv, const void* fn, size_t smem, uint64_t ntiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileThreads, smem) != cudaSuccess) per_sm = 1;
  per_sm = std::max(per_sm, 1);
  return (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sv->sms, 1) * per_sm);
}

// Runs the passes; per-word <P_w> into `vals`; lambda (optional) receives H psi.
template <class A>
static int pauli_passes(SV* sv, const lqs_pauli* terms, int n_terms, void* lam, double* vals) {
  int k, b;
  measure_kb(sv->n, sv->dtype, k, b);
  if (n_terms > 0 && sv->n > k && jit_enabled_for(sv->n)) {  // compiled passes when this state takes them
    const int ar = std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF;
    const int rc = pauli_compiled(sv, terms, n_terms, lam, ar, vals);
    if (rc != LQS_ERR_UNSUPPORTED) return rc;
  }
  std::vector<PassPlan> passes;
  std::vector<int> wide;
  LQS_TRY(plan_passes(sv->n, terms, n_terms, k, b, passes, wide));
  if (passes.empty() && wide.empty()) {
    for (int i = 0; i < n_terms; ++i) vals[i] = 0.0;
    if (lam) LQS_CUDA_TRY(cudaMemsetAsync(lam, 0, sv->bytes(), sv->stream));
    return LQS_OK;
  }
  // wide words accumulate into lambda, so it must start at zero
  const bool lam_zeroed = lam && !wide.empty();
  if (lam_zeroed) LQS_CUDA_TRY(cudaMemsetAsync(lam, 0, sv->bytes(), sv->stream));
  // partial sums: one slot per word per block, laid out pass by pass
  const uint64_t ntiles = 1ull << (sv->n - k);
  const size_t amp = sizeof(typename A::S);
  for (const void* fn : {(const void*)k_pauli<A, 1>, (const void*)k_pauli<A, 3>, (const void*)k_pauli<A, 7>})
    LQS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  const int grid = lam ? occupancy_grid<A>(sv, (const void*)k_pauli<A, 3>, pauli_smem(amp, k, true), ntiles)
                       : occupancy_grid<A>(sv, (const void*)k_pauli<A, 1>, pauli_smem(amp, k, false), ntiles);
  const int wgrid = (int)std::min<uint64_t>(std::max<uint64_t>(sv->N() / 2 / 256, 1), (uint64_t)std::max(sv->sms, 1) * 8);
  size_t slots = 0;
  for (auto& p : passes) slots += p.words.size();
  const size_t tiled_slots = slots;
  slots += wide.size();
  void* scratch = nullptr;
  const int pgrid = wide.empty() ? grid : std::max(grid, wgrid);  // partial rows are pgrid wide
  LQS_TRY(sv_scratch(sv, 2, sizeof(double) * (slots * pgrid + slots), &scratch));
  double* partial = static_cast<double*>(scratch);
  double* sums = partial + slots * pgrid;
  if (pgrid != grid || pgrid != wgrid)
    LQS_CUDA_TRY(cudaMemsetAsync(partial, 0, sizeof(double) * slots * pgrid, sv->stream));
  size_t off = 0;
  for (size_t pi = 0; pi < passes.size(); ++pi) {
    const PassPlan& pp = passes[pi];
    PauliProg P{};
    P.g = geom_for(sv->n, pp.Q, k, b, amp);
    P.nw = (int)pp.words.size();
    for (int w = 0; w < P.nw; ++w) {
      const lqs_pauli& t = terms[pp.words[w]];
      PWord& W = P.w[w];
      W.xl = 0;
      W.zl = 0;
      W.ze = 0;
      W.lowbit = -1;
      for (int q = 0; q < sv->n; ++q) {
        const int lp = lpos(P.g, q);
        if ((t.x_mask >> q) & 1) {
          W.xl |= 1u << lp;  // planned: every X/Y qubit is a tile qubit
          if (W.lowbit < 0 || lp < W.lowbit) W.lowbit = lp;
        }
        if ((t.z_mask >> q) & 1) {
          if (lp >= 0) W.zl |= 1u << lp;
          else W.ze |= 1ull << q;
        }
      }
      W.ph = (uint32_t)(__builtin_popcountll(t.x_mask & t.z_mask) & 3);
      W.c = split_const(t.coeff);
    }
    // each word's partial row is pgrid wide; a tiled pass writes `grid` of it
    double* part = partial + off * pgrid;
    if (!lam) LQS_TRY((launch_pauli<A, 1>(sv, P, nullptr, part, grid, pgrid)));
    else if (pi == 0 && !lam_zeroed) LQS_TRY((launch_pauli<A, 7>(sv, P, lam, part, grid, pgrid)));
    else LQS_TRY((launch_pauli<A, 3>(sv, P, lam, part, grid, pgrid)));
    off += pp.words.size();
  }
  for (size_t i = 0; i < wide.size(); ++i) {
    const lqs_pauli& t = terms[wide[i]];
    int lowbit = 0;
    while (!((t.x_mask >> lowbit) & 1)) ++lowbit;
    const int ph = __builtin_popcountll(t.x_mask & t.z_mask) & 3;
    double* pw = partial + (tiled_slots + i) * pgrid;
    const std::string pname = std::string(lam ? "k_pauli_wide_lambda/" : "k_pauli_wide/") +
                              arith_tag(sv->dtype, std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF);
    ProfScope ps(sv->stream, pname.c_str(), (double)sv->bytes() * (lam ? 3.0 : 1.0), 8.0 * (double)sv->N());
    if (lam)
      k_pauli_wide<A, true><<<wgrid, 256, 0, sv->stream>>>(static_cast<const typename A::S*>(sv->d),
                                                            static_cast<typename A::S*>(lam), sv->N() / 2, lowbit,
                                                            t.x_mask, t.z_mask, ph, split_const(t.coeff), pw);
    else
      k_pauli_wide<A, false><<<wgrid, 256, 0, sv->stream>>>(static_cast<const typename A::S*>(sv->d), nullptr,
                                                             sv->N() / 2, lowbit, t.x_mask, t.z_mask, ph,
                                                             split_const(t.coeff), pw);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
  }
  k_sum_partials<<<(unsigned)slots, 256, 0, sv->stream>>>(partial, pgrid, sums);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  std::vector<double> h(slots);
  LQS_CUDA_TRY(cudaMemcpyAsync(h.data(), sums, sizeof(double) * slots, cudaMemcpyDeviceToHost, sv->stream));
  LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
  off = 0;
  for (auto& p : passes)
    for (int w : p.words) vals[w] = h[off++];
  for (int w : wide) vals[w] = h[off++];
  int status[2] = {0, 0};
  LQS_CUDA_TRY(cudaMemcpy(status, sv->d_status, sizeof status, cudaMemcpyDeviceToHost));
  if (status[0]) {
    cudaMemset(sv->d_status, 0, 64);
    return set_error(LQS_ERR_TIMEOUT, "a tile load did not complete (bounded wait expired)");
  }
  return LQS_OK;
}

static int dispatch_pauli(SV* sv, int arith, const lqs_pauli* terms, int n_terms, void* lam, double* vals) {
  if (sv->dtype == LQS_C64) return pauli_passes<ArF32>(sv, terms, n_terms, lam, vals);
  if (arith == LQS_ARITH_F64) return pauli_passes<ArF64>(sv, terms, n_terms, lam, vals);
  return pauli_passes<ArDF>(sv, terms, n_terms, lam, vals);
}

int run_expval(SV* sv, const lqs_pauli* terms, int n_terms, const PlanCfg&, int arith, double* out,
               double* per_term, const void* lambda_out) {
  std::vector<double> vals(std::max(n_terms, 1), 0.0);
  LQS_TRY(dispatch_pauli(sv, arith, terms, n_terms, const_cast<void*>(lambda_out), vals.data()));
  double e = 0.0;
  for (int i = 0; i < n_terms; ++i) e += terms[i].coeff * vals[i];
  *out = e;
  if (per_term)
    for (int i = 0; i < n_terms; ++i) per_term[i] = vals[i];
  return LQS_OK;
}

int run_norm2(SV* sv, int arith, double* out) {
  lqs_pauli id{1.0, 0, 0};
  double v = 0.0;
  LQS_TRY(dispatch_pauli(sv, arith, &id, 1, nullptr, &v));
  *out = v;
  return LQS_OK;
}

// ---------------------------------------------------------------------------
// adjoint sweep
// ---------------------------------------------------------------------------
template <class A>
__global__ void __launch_bounds__(kTileThreads) k_adjoint(typename A::S* __restrict__ psi,
                                                          typename A::S* __restrict__ lam,
                                                          const __grid_constant__ TileProg<A> P, double* partial,
                                                          int* status) {
  using S = typename A::S;
  using W = typename A::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TileGeom& G = P.g;
  const uint32_t nt = 1u << G.k;
  S* pb = reinterpret_cast<S*>(smem_raw);
  S* lb = pb + nt;
  W* Pt = reinterpret_cast<W*>(pb);
  W* Lt = reinterpret_cast<W*>(lb);
  double* wacc = reinterpret_cast<double*>(smem_raw + 2 * (size_t)nt * sizeof(S));
  uint64_t* bar = reinterpret_cast<uint64_t*>(wacc + kTileWarps * kMaxGradSlots);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kTileWarps * kMaxGradSlots; i += blockDim.x) wacc[i] = 0.0;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  bool ok = true;
  for (uint64_t t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(G, t);
    if (threadIdx.x < 32) {
      tile_expect(G, bar, 2u);
      tile_load_rows(G, pb, psi, base, bar);
      tile_load_rows(G, lb, lam, base, bar);
    }
    ok = __syncthreads_and(mbar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    if constexpr (!std::is_same<S, W>::value) {
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        const S a = pb[j], c = lb[j];
        Pt[j] = A::load(a);
        Lt[j] = A::load(c);
      }
      __syncthreads();
    }
    for (int i = 0; i < P.nops; ++i) {
      const TOp& o = P.op[i];
      if (o.gslot >= 0 && (base & o.ecmask) == o.ecmask) {
        const DF s = warp_sum(gen_partial<A>(Pt, Lt, o, base, G.k));
        if (lane == 0) wacc[warp * kMaxGradSlots + o.gslot] += df2d(s);
      }
      tile_apply2<A>(Pt, Lt, o, P.coef, base, G.k);
      __syncthreads();
    }
    if constexpr (!std::is_same<S, W>::value) {
      for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) {
        const W a = Pt[j], c = Lt[j];
        pb[j] = A::store(a);
        lb[j] = A::store(c);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t nrows = 1u << G.r, per_row = 1u << G.b;
      for (uint32_t row = lane; row < nrows; row += 32) {
        const uint64_t go = base + row_offset(G, row);
        bulk_s2g(psi + go, pb + (size_t)row * per_row, G.row_bytes);
        bulk_s2g(lam + go, lb + (size_t)row * per_row, G.row_bytes);
      }
      bulk_commit();
      bulk_wait_read0();
      __syncwarp();
    }
  }
  if (threadIdx.x < 32) bulk_wait0();
  if (!ok && threadIdx.x == 0) {
    flag_timeout(status, 3);
    mbar_wait(bar, phase ^ 1u);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < P.ngrad; s += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < kTileWarps; ++q) v += wacc[q * kMaxGradSlots + s];
    partial[(size_t)s * gridDim.x + blockIdx.x] = v;
  }
}

// Sums the per-block partials of every gradient slot in a fixed order (one
// block per slot), brings them to the host and adds gen_scale * sum to the
// gradient of each slot's parameter.
static int adjoint_finish(SV* sv, const std::vector<KOp>& rev, double* partial, int grid,
                          const std::vector<int>& slot_owner, int n_params, double* grads,
                          const std::vector<double>* slot_scale = nullptr) {
  const size_t nslots = slot_owner.size();
  double* sums = partial + nslots * (size_t)grid;
  if (nslots) {
    k_sum_partials<<<(unsigned)nslots, 256, 0, sv->stream>>>(partial, grid, sums);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
  }
  std::vector<double> h(nslots);
  if (nslots)
    LQS_CUDA_TRY(cudaMemcpyAsync(h.data(), sums, sizeof(double) * nslots, cudaMemcpyDeviceToHost, sv->stream));
  LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
  int status[2] = {0, 0};
  LQS_CUDA_TRY(cudaMemcpy(status, sv->d_status, sizeof status, cudaMemcpyDeviceToHost));
  if (status[0]) {
    cudaMemset(sv->d_status, 0, 64);
    return set_error(LQS_ERR_TIMEOUT, "a tile load did not complete (bounded wait expired)");
  }
  for (size_t s = 0; s < nslots; ++s) {
    const KOp& o = rev[slot_owner[s]];
    const double sc = slot_scale && s < slot_scale->size() ? (*slot_scale)[s] : 1.0;
    if (o.param_slot < n_params) grads[o.param_slot] += o.gen_scale * sc * h[s];
  }
  return LQS_OK;
}

template <class A>
static int adjoint_t(SV* sv, const std::vector<KOp>& ops, int n_params, const lqs_pauli* terms, int n_terms,
                     double* grads, double* energy) {
  const int n = sv->n;
  int k, b;
  measure_kb(n, sv->dtype, k, b);
  if (n > k && k - b < 2) b = k - 2;
  void* lam = nullptr;
  LQS_TRY(sv_scratch(sv, 0, sv->bytes(), &lam));
  // 1. lambda = H psi and the energy
  std::vector<double> vals(std::max(n_terms, 1), 0.0);
  if (n_terms > 0) {
    LQS_TRY(pauli_passes<A>(sv, terms, n_terms, lam, vals.data()));
  } else {
    LQS_CUDA_TRY(cudaMemsetAsync(lam, 0, sv->bytes(), sv->stream));
  }
  double e = 0.0;
  for (int i = 0; i < n_terms; ++i) e += terms[i].coeff * vals[i];
  if (energy) *energy = e;
  for (int i = 0; i < n_params; ++i) grads[i] = 0.0;
  if (ops.empty()) return LQS_OK;
  // 2. reversed circuit of inverse ops, planned into tile segments
  std::vector<KOp> rev;
  rev.reserve(ops.size());
  for (size_t i = ops.size(); i-- > 0;) rev.push_back(inverse_op(ops[i]));
  if (reg_adjoint_available(sv, 0)) {
    // compiled reverse sweep: register-tile programs over psi and lambda
    std::vector<int> slot_op;
    std::vector<double> slot_scale;
    double* partial = nullptr;
    int grid = 0;
    const int ar = std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF;
    const int rc = run_adjoint_compiled(sv, rev, lam, ar, slot_op, slot_scale, &partial, &grid);
    if (rc == LQS_OK) return adjoint_finish(sv, rev, partial, grid, slot_op, n_params, grads, &slot_scale);
    if (rc != LQS_ERR_UNSUPPORTED) return rc;  // nothing was launched when it is unsupported
  }
  PlanCfg pc;
  pc.k = k;
  pc.b = b;
  pc.max_ops = kMaxTileOps;
  std::vector<Segment> segs;
  LQS_TRY(plan_segments(n, rev, pc, segs));
  // split segments whose gradient slots exceed the per-CTA accumulator space
  std::vector<Segment> segs2;
  for (auto& s : segs) {
    Segment cur;
    cur.qmask = s.qmask;
    int ng = 0;
    for (int i : s.ops) {
      const bool g = rev[i].param_slot >= 0 && rev[i].gen != G_NONE;
      if (g && ng == kMaxGradSlots) {
        segs2.push_back(cur);
        cur.ops.clear();
        ng = 0;
      }
      cur.ops.push_back(i);
      ng += g;
    }
    if (!cur.ops.empty()) segs2.push_back(cur);
  }
  const size_t amp = sizeof(typename A::S);
  const size_t smem = (amp << k) * 2 + sizeof(double) * kTileWarps * kMaxGradSlots + 16;
  static bool attr = false;
  if (!attr) {
    LQS_CUDA_TRY(cudaFuncSetAttribute(k_adjoint<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const uint64_t ntiles = 1ull << (n - k);
  const int grid = occupancy_grid<A>(sv, (const void*)k_adjoint<A>, smem, ntiles);
  std::vector<int> slot_owner;  // gradient slot -> op index in rev
  size_t nslots = 0;
  for (auto& s : segs2)
    for (int i : s.ops)
      if (rev[i].param_slot >= 0 && rev[i].gen != G_NONE) ++nslots;
  void* scratch = nullptr;
  LQS_TRY(sv_scratch(sv, 1, sizeof(double) * (std::max<size_t>(nslots, 1) * (grid + 1)), &scratch));
  double* partial = static_cast<double*>(scratch);
  static thread_local TileProg<A> P;
  size_t off = 0;
  for (auto& s : segs2) {
    init_prog(P, n, s.qmask, k, b);
    int ng = 0;
    for (int i : s.ops) {
      const bool g = rev[i].param_slot >= 0 && rev[i].gen != G_NONE;
      LQS_TRY(add_tile_op(P, rev[i], g ? ng : -1));
      if (g) {
        slot_owner.push_back(i);
        ++ng;
      }
    }
    P.ngrad = ng;
    double fl = 0.0;
    for (int i : s.ops) fl += kop_touched_fraction(rev[i]) * kop_flops_per_amp(rev[i]);
    const std::string pname = std::string("k_adjoint/") + arith_tag(sv->dtype, std::is_same<A, ArF64>::value ? LQS_ARITH_F64 : LQS_ARITH_DF);
    ProfScope ps(sv->stream, pname.c_str(), 4.0 * (double)sv->bytes(), (2.0 * fl + 8.0 * ng) * (double)sv->N());
    k_adjoint<A><<<grid, kTileThreads, smem, sv->stream>>>(static_cast<typename A::S*>(sv->d),
                                                            static_cast<typename A::S*>(lam), P,
                                                            partial + off * grid, sv->d_status);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
    off += ng;
  }
  return adjoint_finish(sv, rev, partial, grid, slot_owner, n_params, grads);
}

int run_adjoint(SV* sv, const std::vector<KOp>& ops, int n_params, const lqs_pauli* terms, int n_terms,
                const PlanCfg&, int arith, double* grads, double* energy) {
  if (sv->dtype == LQS_C64) return adjoint_t<ArF32>(sv, ops, n_params, terms, n_terms, grads, energy);
  if (arith == LQS_ARITH_F64) return adjoint_t<ArF64>(sv, ops, n_params, terms, n_terms, grads, energy);
  return adjoint_t<ArDF>(sv, ops, n_params, terms, n_terms, grads, energy);
}

}  // namespace lqs
