// Pieces shared by the measurement, adjoint and batched kernels: double-float
// inner products, Pauli-word descriptions and their pass planning, adjoint
// generator partials, and inverse ops.  The measured quantity is the
// expectation of a Hamiltonian given as a sum of Pauli words, and the
// differentiated one its gradient in the gate parameters (Listing 1).
#pragma once
#include <algorithm>
#include <vector>

#include "arith.cuh"
#include "lqs_internal.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"

namespace lqs {

// ---------------------------------------------------------------------------
// double-float views of the working amplitudes
// ---------------------------------------------------------------------------
LQS_HD DFC to_dfc(const float2& w) { return DFC{DF{w.x, 0.f}, DF{w.y, 0.f}}; }
LQS_HD DFC to_dfc(const double2& w) { return DFC{d2df(w.x), d2df(w.y)}; }
LQS_HD DFC to_dfc(const DFC& w) { return w; }

// Re(conj(a) b) and Im(conj(a) b) accumulated with a sign.
__device__ __forceinline__ void acc_re_conj(DAcc& A, const DFC& a, const DFC& b, bool neg) {
  const DF ar = neg ? df_neg(a.re) : a.re, ai = neg ? df_neg(a.im) : a.im;
  df_mac(A, ar, b.re);
  df_mac(A, ai, b.im);
}
__device__ __forceinline__ void acc_im_conj(DAcc& A, const DFC& a, const DFC& b, bool neg) {
  const DF ar = neg ? df_neg(a.re) : a.re, ai = neg ? a.im : df_neg(a.im);
  df_mac(A, ar, b.im);
  df_mac(A, ai, b.re);
}

__device__ __forceinline__ DF shfl_df(DF v, int off) {
  return DF{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
}
// Warp sum of a double-float accumulator; the result is valid in every lane.
__device__ __forceinline__ DF warp_sum(DAcc a) {
  DF v = df_norm(a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = df_add(v, shfl_df(v, off));
  return v;
}

constexpr int kPassWords = 24;

struct PWord {
  uint32_t xl, zl;   // local X and Z masks
  uint64_t ze;       // Z bits outside the tile (a per-tile sign)
  uint32_t ph;       // number of Y factors mod 4 (phase i^ph)
  int lowbit;        // lowest local bit of xl (-1: diagonal word)
  DF c;              // coefficient (for lambda)
};

struct PauliProg {
  TileGeom g;
  int nw;
  PWord w[kPassWords];
};

// Build the tile-local description of Pauli word t for tile geometry G
// (every X/Y qubit of t must be a tile qubit).
inline int tile_lpos(const TileGeom& G, int q) {
  if (q < G.b) return q;
  for (int m = 0; m < G.r; ++m)
    if (G.h[m] == q) return G.b + m;
  return -1;
}
inline PWord make_pword(const TileGeom& G, const lqs_pauli& t) {
  PWord W{};
  W.lowbit = -1;
  for (int q = 0; q < G.n; ++q) {
    const int lp = tile_lpos(G, q);
    if ((t.x_mask >> q) & 1) {
      W.xl |= 1u << lp;
      if (W.lowbit < 0 || lp < W.lowbit) W.lowbit = lp;
    }
    if ((t.z_mask >> q) & 1) {
      if (lp >= 0) W.zl |= 1u << lp;
      else W.ze |= 1ull << q;
    }
  }
  W.ph = (uint32_t)(__builtin_popcountll(t.x_mask & t.z_mask) & 3);
  W.c = split_const(t.coeff);
  return W;
}

// Group words into passes: X masks must fit a tile of k qubits (low b qubits
// plus chosen high qubits); at most kPassWords words per pass.  Words whose
// X/Y qubits cannot fit any tile go to `wide` (global pair passes).
struct PassPlan {
  uint64_t Q;
  std::vector<int> words;
};
inline int plan_passes(int n, const lqs_pauli* terms, int n_terms, int k, int b, std::vector<PassPlan>& out,
                       std::vector<int>& wide, int max_words = kPassWords) {
  std::vector<char> done(n_terms, 0);
  int left = n_terms;
  const uint64_t low = (b >= 64) ? ~0ull : ((1ull << b) - 1);
  for (int i = 0; i < n_terms; ++i)
    if (__builtin_popcountll(terms[i].x_mask | low) > k) {
      wide.push_back(i);
      done[i] = 1;
      --left;
    }
  while (left) {
    PassPlan p;
    p.Q = low;
    for (int i = 0; i < n_terms && (int)p.words.size() < max_words; ++i) {
      if (done[i]) continue;
      const uint64_t need = terms[i].x_mask & ~p.Q;
      if (__builtin_popcountll(p.Q | need) <= k) {
        p.Q |= need;
        p.words.push_back(i);
        done[i] = 1;
        --left;
      }
    }
    if (p.words.empty()) return set_error(LQS_ERR_ARG, "internal: Pauli pass planner made no progress");
    for (int q = b; q < n && __builtin_popcountll(p.Q) < k; ++q) p.Q |= 1ull << q;
    out.push_back(std::move(p));
  }
  return LQS_OK;
}

inline TileGeom geom_for(int n, uint64_t Q, int k, int b, size_t amp) {
  TileGeom G{};
  G.n = n;
  G.k = k;
  G.b = b;
  for (int q = b; q < n; ++q)
    if ((Q >> q) & 1) G.h[G.r++] = q;
  G.ntiles = 1ull << (n - k);
  G.row_bytes = (uint32_t)(amp << b);
  return G;
}
inline int lpos(const TileGeom& G, int q) {
  if (q < G.b) return q;
  for (int m = 0; m < G.r; ++m)
    if (G.h[m] == q) return G.b + m;
  return -1;
}

constexpr int kMaxGradSlots = 128;

// Im <lambda|G|psi> over the tile for generator G of op o (before U^dagger).
template <class A, int NF>
__device__ __forceinline__ DAcc gen_partial_n(const typename A::W* Ps, const typename A::W* Ls, const TOp& o,
                                              uint64_t base, int k, const uint32_t (&mk)[5]) {
  DAcc acc{0.f, 0.f};
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const uint32_t lc = o.lcmask;
  if (o.gen == G_P1 || (o.gen == G_Z && o.l0 < 0)) {
    // single amplitudes: P1 on the op's control set, or Z on a qubit outside
    // the tile (a per-tile sign)
    const bool neg = (o.gen == G_Z) && (base & o.e0);
    const uint32_t ng = 1u << (k - o.nfix);
    for (uint32_t g = tid; g < ng; g += nth) {
      const uint32_t j = ins_m<NF>(g, mk) | lc;
      acc_im_conj(acc, to_dfc(Ls[j]), to_dfc(Ps[j]), neg);
    }
    return acc;
  }
  const uint32_t tb = 1u << o.l0;
  const uint32_t ng = 1u << (k - o.nfix);
  for (uint32_t g = tid; g < ng; g += nth) {
    const uint32_t j0 = ins_m<NF>(g, mk) | lc, j1 = j0 | tb;
    const DFC p0 = to_dfc(Ps[j0]), p1 = to_dfc(Ps[j1]), l0 = to_dfc(Ls[j0]), l1 = to_dfc(Ls[j1]);
    if (o.gen == G_X) {  // conj(l0) p1 + conj(l1) p0
      acc_im_conj(acc, l0, p1, false);
      acc_im_conj(acc, l1, p0, false);
    } else if (o.gen == G_Y) {  // conj(l0)(-i p1) + conj(l1)(i p0)
      acc_re_conj(acc, l0, p1, true);
      acc_re_conj(acc, l1, p0, false);
    } else {  // G_Z: conj(l0) p0 - conj(l1) p1
      acc_im_conj(acc, l0, p0, false);
      acc_im_conj(acc, l1, p1, true);
    }
  }
  return acc;
}

template <class A>
__device__ __forceinline__ DAcc gen_partial(const typename A::W* Ps, const typename A::W* Ls, const TOp& o,
                                            uint64_t base, int k) {
  uint32_t mk[5];
  ins_masks(o, mk);
  switch (o.nfix) {
    case 0: return gen_partial_n<A, 0>(Ps, Ls, o, base, k, mk);
    case 1: return gen_partial_n<A, 1>(Ps, Ls, o, base, k, mk);
    case 2: return gen_partial_n<A, 2>(Ps, Ls, o, base, k, mk);
    case 3: return gen_partial_n<A, 3>(Ps, Ls, o, base, k, mk);
    default: return gen_partial_n<A, 4>(Ps, Ls, o, base, k, mk);
  }
}

// U^dagger of a lowered op (same kernel class, conjugate-transposed entries).
inline KOp inverse_op(const KOp& o) {
  KOp r = o;
  auto conj_at = [&](int i) { r.m[2 * i + 1] = -r.m[2 * i + 1]; };
  switch (o.kind) {
    case K_PHASE:
      conj_at(0);
      if (o.special == 2) r.special = 3;
      else if (o.special == 3) r.special = 2;
      break;
    case K_DIAG1: conj_at(0); conj_at(1); break;
    case K_DIAG2: for (int i = 0; i < 4; ++i) conj_at(i); break;
    case K_ANTI1:  // [[0, f0], [f1, 0]]^dagger = [[0, conj f1], [conj f0, 0]]
      r.m[0] = o.m[2]; r.m[1] = -o.m[3];
      r.m[2] = o.m[0]; r.m[3] = -o.m[1];
      break;
    case K_SWAP: break;
    case K_DENSE1:
      for (int rr = 0; rr < 2; ++rr)
        for (int c = 0; c < 2; ++c) {
          r.m[2 * (2 * rr + c)] = o.m[2 * (2 * c + rr)];
          r.m[2 * (2 * rr + c) + 1] = -o.m[2 * (2 * c + rr) + 1];
        }
      break;
    case K_DENSE1R:
      r.m[1] = o.m[2];
      r.m[2] = o.m[1];
      break;
    case K_DENSE2:
      for (int rr = 0; rr < 4; ++rr)
        for (int c = 0; c < 4; ++c) {
          r.m[2 * (4 * rr + c)] = o.m[2 * (4 * c + rr)];
          r.m[2 * (4 * rr + c) + 1] = -o.m[2 * (4 * c + rr) + 1];
        }
      break;
  }
  return r;
}


}  // namespace lqs
