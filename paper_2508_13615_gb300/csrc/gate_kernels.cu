// Plain per-gate path: one streaming kernel per gate, chosen by gate class.
//
// Index structure (Sec. 2, Fig. 1): a gate on target q_T pairs amplitude i
// with i ^ 2^q_T; a control bit never moves data, it only selects which
// groups are touched (Fig. 1c).  Here every kernel enumerates exactly the
// touched index groups: group g's base index is g with zero bits inserted at
// the gate's fixed positions (targets and controls, ascending) and the
// control bits then set.  Consecutive threads take consecutive g, so each of
// the group's 1, 2 or 4 amplitude streams is contiguous and coalesced
// whatever the target index; a high target only changes the distance
// between the streams.
#include <algorithm>
#include <string>

#include "arith.cuh"
#include "lqs_internal.cuh"

namespace lqs {

struct Geom {
  uint64_t ngroups;
  int nfix;
  int fix[5];
  uint64_t cmask;
  uint64_t b0, b1;  // target bits
};

__device__ __forceinline__ uint64_t group_base(const Geom& G, uint64_t g) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k < G.nfix) {
      const int p = G.fix[k];
      g = ((g >> p) << (p + 1)) | (g & ((1ull << p) - 1));
    }
  }
  return g | G.cmask;
}

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

// Grid-stride loop that issues kUnroll independent groups per thread before
// using any of them, so each thread keeps several loads in flight.
#define GROUP_LOOP_BEGIN                                                                  \
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;                               \
  for (uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < G.ngroups;     \
       g0 += stride * kUnroll) {
#define GROUP_LOOP_END }

template <class A>
__global__ void __launch_bounds__(kThreads) k_phase(typename A::S* __restrict__ psi, Geom G, typename A::C f,
                                                    int special) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S v[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); v[u] = psi[idx[u]]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    S r;
    if (special == 1) r = A::sneg(v[u]);
    else if (special == 2) r = A::smul_i(v[u]);
    else if (special == 3) r = A::sneg(A::smul_i(v[u]));
    else r = A::store(A::cmul(f, A::load(v[u])));
    psi[idx[u]] = r;
  }
  GROUP_LOOP_END
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_diag1(typename A::S* __restrict__ psi, Geom G, typename A::C d0,
                                                    typename A::C d1) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S a[kUnroll], b[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); a[u] = psi[idx[u]]; b[u] = psi[idx[u] | G.b0]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    psi[idx[u]] = A::store(A::cmul(d0, A::load(a[u])));
    psi[idx[u] | G.b0] = A::store(A::cmul(d1, A::load(b[u])));
  }
  GROUP_LOOP_END
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_anti1(typename A::S* __restrict__ psi, Geom G, typename A::C f0,
                                                    typename A::C f1, int plain) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S a[kUnroll], b[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); a[u] = psi[idx[u]]; b[u] = psi[idx[u] | G.b0]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    if (plain) {  // a pure permutation: move the stored bits, no arithmetic
      psi[idx[u]] = b[u];
      psi[idx[u] | G.b0] = a[u];
    } else {
      psi[idx[u]] = A::store(A::cmul(f0, A::load(b[u])));
      psi[idx[u] | G.b0] = A::store(A::cmul(f1, A::load(a[u])));
    }
  }
  GROUP_LOOP_END
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_swap(typename A::S* __restrict__ psi, Geom G) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S a[kUnroll], b[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); a[u] = psi[idx[u] | G.b0]; b[u] = psi[idx[u] | G.b1]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    psi[idx[u] | G.b0] = b[u];
    psi[idx[u] | G.b1] = a[u];
  }
  GROUP_LOOP_END
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_dense1(typename A::S* __restrict__ psi, Geom G, typename A::C u00,
                                                     typename A::C u01, typename A::C u10, typename A::C u11) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S a[kUnroll], b[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); a[u] = psi[idx[u]]; b[u] = psi[idx[u] | G.b0]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    const auto x = A::load(a[u]), y = A::load(b[u]);
    psi[idx[u]] = A::store(A::cmac2(u00, x, u01, y));
    psi[idx[u] | G.b0] = A::store(A::cmac2(u10, x, u11, y));
  }
  GROUP_LOOP_END
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_dense1r(typename A::S* __restrict__ psi, Geom G, typename A::R u00,
                                                      typename A::R u01, typename A::R u10, typename A::R u11) {
  using S = typename A::S;
  GROUP_LOOP_BEGIN
  S a[kUnroll], b[kUnroll];
  uint64_t idx[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g < G.ngroups) { idx[u] = group_base(G, g); a[u] = psi[idx[u]]; b[u] = psi[idx[u] | G.b0]; }
  }
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const uint64_t g = g0 + u * stride;
    if (g >= G.ngroups) continue;
    const auto x = A::load(a[u]), y = A::load(b[u]);
    psi[idx[u]] = A::store(A::rmac2(u00, x, u01, y));
    psi[idx[u] | G.b0] = A::store(A::rmac2(u10, x, u11, y));
  }
  GROUP_LOOP_END
}

// 4x4 coefficients travel by value in a struct (kernel parameter space).
template <class C>
struct Mat4 { C c[16]; };

template <class A>
__global__ void __launch_bounds__(kThreads) k_dense2(typename A::S* __restrict__ psi, Geom G,
                                                     Mat4<typename A::C> M) {
  using S = typename A::S;
  using W = typename A::W;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G.ngroups; g += stride) {
    const uint64_t base = group_base(G, g);
    // local index r = 2*bit(t0) + bit(t1): t0 is the matrix's most significant wire
    const uint64_t id[4] = {base, base | G.b1, base | G.b0, base | G.b0 | G.b1};
    S s[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) s[r] = psi[id[r]];
    W x[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) x[r] = A::load(s[r]);
#pragma unroll
    for (int r = 0; r < 4; ++r) psi[id[r]] = A::store(A::cmac4_raw(&M.c[4 * r], x));
  }
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_diag2(typename A::S* __restrict__ psi, Geom G, typename A::C d0,
                                                    typename A::C d1, typename A::C d2, typename A::C d3) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G.ngroups; g += stride) {
    const uint64_t base = group_base(G, g);
    psi[base] = A::store(A::cmul(d0, A::load(psi[base])));
    psi[base | G.b1] = A::store(A::cmul(d1, A::load(psi[base | G.b1])));
    psi[base | G.b0] = A::store(A::cmul(d2, A::load(psi[base | G.b0])));
    psi[base | G.b0 | G.b1] = A::store(A::cmul(d3, A::load(psi[base | G.b0 | G.b1])));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static Geom make_geom(int n, const KOp& op, bool targets_fixed) {
  Geom G{};
  uint64_t fixmask = op.cmask;
  if (targets_fixed) fixmask |= op.target_mask();
  G.nfix = 0;
  for (int q = 0; q < n; ++q)
    if ((fixmask >> q) & 1) G.fix[G.nfix++] = q;
  G.ngroups = 1ull << (n - G.nfix);
  G.cmask = op.cmask;
  G.b0 = op.t0 >= 0 ? 1ull << op.t0 : 0;
  G.b1 = op.t1 >= 0 ? 1ull << op.t1 : 0;
  return G;
}

static unsigned grid_for(const SV* sv, uint64_t work) {
  const uint64_t per_block = (uint64_t)kThreads * kUnroll;
  const uint64_t want = (work + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)std::max(sv->sms, 1) * 8;  // 8 resident blocks of 256 per SM
  return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

template <class A>
static typename A::C cc(const KOp& op, int i) { return A::cconst(op.m[2 * i], op.m[2 * i + 1]); }

static const char* gate_kernel_name(int kind) {
  static const char* names[] = {"k_phase", "k_diag1", "k_anti1", "k_swap", "k_dense1", "k_dense1r", "k_dense2",
                                "k_diag2"};
  return (kind >= 0 && kind < 8) ? names[kind] : "k_gate";
}

template <class A>
static int launch_gate_t(SV* sv, const KOp& op, int arith) {
  using S = typename A::S;
  S* psi = static_cast<S*>(sv->d);
  cudaStream_t st = sv->stream;
  const int n = sv->n;
  const double touched = kop_touched_fraction(op) * (double)sv->N();
  const std::string pname = std::string(gate_kernel_name(op.kind)) + "/" + arith_tag(sv->dtype, arith);
  ProfScope ps(st, pname.c_str(), 2.0 * touched * (double)sv->amp_bytes(), touched * kop_flops_per_amp(op));
  switch (op.kind) {
    case K_PHASE: {
      Geom G = make_geom(n, op, false);
      k_phase<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G, cc<A>(op, 0), op.special);
      break;
    }
    case K_DIAG1: {
      Geom G = make_geom(n, op, true);
      k_diag1<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G, cc<A>(op, 0), cc<A>(op, 1));
      break;
    }
    case K_ANTI1: {
      Geom G = make_geom(n, op, true);
      k_anti1<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G, cc<A>(op, 0), cc<A>(op, 1), op.special);
      break;
    }
    case K_SWAP: {
      Geom G = make_geom(n, op, true);
      k_swap<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G);
      break;
    }
    case K_DENSE1: {
      Geom G = make_geom(n, op, true);
      k_dense1<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G, cc<A>(op, 0), cc<A>(op, 1), cc<A>(op, 2),
                                                                  cc<A>(op, 3));
      break;
    }
    case K_DENSE1R: {
      Geom G = make_geom(n, op, true);
      k_dense1r<A><<<grid_for(sv, G.ngroups), kThreads, 0, st>>>(psi, G, A::rconst(op.m[0]), A::rconst(op.m[1]),
                                                                   A::rconst(op.m[2]), A::rconst(op.m[3]));
      break;
    }
    case K_DENSE2: {
      Geom G = make_geom(n, op, true);
      Mat4<typename A::C> M;
      for (int i = 0; i < 16; ++i) M.c[i] = cc<A>(op, i);
      unsigned grid = (unsigned)std::max<uint64_t>(
          1, std::min<uint64_t>((G.ngroups + kThreads - 1) / kThreads, (uint64_t)std::max(sv->sms, 1) * 8));
      k_dense2<A><<<grid, kThreads, 0, st>>>(psi, G, M);
      break;
    }
    case K_DIAG2: {
      Geom G = make_geom(n, op, true);
      unsigned grid = (unsigned)std::max<uint64_t>(
          1, std::min<uint64_t>((G.ngroups + kThreads - 1) / kThreads, (uint64_t)std::max(sv->sms, 1) * 8));
      k_diag2<A><<<grid, kThreads, 0, st>>>(psi, G, cc<A>(op, 0), cc<A>(op, 1), cc<A>(op, 2), cc<A>(op, 3));
      break;
    }
    default:
      return set_error(LQS_ERR_ARG, "internal: unknown kernel op kind");
  }
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

int launch_gate(SV* sv, const KOp& op, int arith) {
  if (sv->dtype == LQS_C64) return launch_gate_t<ArF32>(sv, op, arith);
  if (arith == LQS_ARITH_F64) return launch_gate_t<ArF64>(sv, op, arith);
  return launch_gate_t<ArDF>(sv, op, arith);
}

}  // namespace lqs
