// Applying one kernel op to a tile held in shared memory.
//
// Each op enumerates exactly the index groups it touches inside the tile
// (local fixed bits = its local targets and local controls, zero bits
// inserted, control bits set).  Controls on qubits outside the tile are
// decided once per tile from the tile's base index (the paper's observation
// that a non-local control qubit only selects which processes act, Sec. 2 /
// Fig. 1c); diagonal ops on qubits outside the tile become per-tile factors.
#pragma once
#include "lqs_internal.cuh"
#include "tile.cuh"

namespace lqs {

template <class A> struct CRe;
template <> struct CRe<ArF32> { static LQS_HD float get(const float2& c) { return c.x; } };
template <> struct CRe<ArF64> { static LQS_HD double get(const double2& c) { return c.x; } };
template <> struct CRe<ArDF> { static LQS_HD DF get(const DFK& c) { return c.re; } };

template <class A>
__device__ __forceinline__ typename A::W phase_apply(const typename A::C& f, int special, typename A::W w) {
  if (special == 1) return A::neg(w);
  if (special == 2) return A::mul_i(w);
  if (special == 3) return A::neg(A::mul_i(w));
  return A::cmul(f, w);
}

// Index group g -> its base index: zero bits inserted at the op's fixed
// positions p_0 < .. < p_{NF-1}.  Bits [p_{i-1} - (i-1), p_i - i) of g move up
// by i; the masks are formed once per op (ins_masks), so a group costs
// 2 NF + 1 instructions with no branch.
template <int NF>
__device__ __forceinline__ uint32_t ins_m(uint32_t g, const uint32_t (&m)[5]) {
  uint32_t r = g & m[0];
#pragma unroll
  for (int i = 1; i <= NF; ++i) r |= (g & m[i]) << i;
  return r;
}
__device__ __forceinline__ void ins_masks(const TOp& o, uint32_t (&m)[5]) {
  uint32_t lo = 0;  // first bit of g in segment i
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint32_t hi = i < o.nfix ? (uint32_t)o.fix[i] - (uint32_t)i : 32u;  // end of segment i
    const uint32_t below_hi = hi >= 32u ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    const uint32_t below_lo = lo >= 32u ? 0xFFFFFFFFu : ((1u << lo) - 1u);
    m[i] = below_hi & ~below_lo;
    lo = hi;
  }
}

// Applies op `o` (with NF = o.nfix fixed bits) to tile T, and with NT = 2 the
// same op to tile T2 in the same loop (the adjoint sweep's two states share
// every index); see tile_apply.
template <class A, int NF, int NT>
__device__ __forceinline__ void tile_apply_n(typename A::W* T, typename A::W* T2, const TOp& o,
                                             const typename A::C* coef, uint64_t base, int k, const uint32_t (&mk)[5]) {
  using W = typename A::W;
  using C = typename A::C;
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const uint32_t ng = 1u << (k - o.nfix);
  const uint32_t lc = o.lcmask;
  W* const tiles[2] = {T, T2};
  switch (o.kind) {
    case K_PHASE: {
      const C f = coef[o.coef];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins_m<NF>(g, mk) | lc;
#pragma unroll
        for (int s = 0; s < NT; ++s) tiles[s][j] = phase_apply<A>(f, o.special, tiles[s][j]);
      }
      break;
    }
    case K_DIAG1: {
      if (o.l0 >= 0) {
        const C d0 = coef[o.coef], d1 = coef[o.coef + 1];
        const uint32_t tb = 1u << o.l0;
        for (uint32_t g = tid; g < ng; g += nth) {
          const uint32_t j = ins_m<NF>(g, mk) | lc;
#pragma unroll
          for (int s = 0; s < NT; ++s) {
            W* X = tiles[s];
            X[j] = A::cmul(d0, X[j]);
            X[j | tb] = A::cmul(d1, X[j | tb]);
          }
        }
      } else {
        const C d = coef[o.coef + ((base & o.e0) ? 1 : 0)];
        for (uint32_t g = tid; g < ng; g += nth) {
          const uint32_t j = ins_m<NF>(g, mk) | lc;
#pragma unroll
          for (int s = 0; s < NT; ++s) tiles[s][j] = A::cmul(d, tiles[s][j]);
        }
      }
      break;
    }
    case K_DIAG2: {
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins_m<NF>(g, mk) | lc;
        const int b0 = o.l0 >= 0 ? (int)((j >> o.l0) & 1u) : ((base & o.e0) ? 1 : 0);
        const int b1 = o.l1 >= 0 ? (int)((j >> o.l1) & 1u) : ((base & o.e1) ? 1 : 0);
        const C f = coef[o.coef + 2 * b0 + b1];
#pragma unroll
        for (int s = 0; s < NT; ++s) tiles[s][j] = A::cmul(f, tiles[s][j]);
      }
      break;
    }
    case K_ANTI1: {
      const uint32_t tb = 1u << o.l0;
      const C f0 = coef[o.coef], f1 = coef[o.coef + 1];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins_m<NF>(g, mk) | lc, j1 = j0 | tb;
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          W* X = tiles[s];
          const W a = X[j0], b = X[j1];
          if (o.special == 1) {
            X[j0] = b;
            X[j1] = a;
          } else {
            X[j0] = A::cmul(f0, b);
            X[j1] = A::cmul(f1, a);
          }
        }
      }
      break;
    }
    case K_SWAP: {
      const uint32_t ba = 1u << o.l0, bb = 1u << o.l1;
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins_m<NF>(g, mk) | lc;
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          W* X = tiles[s];
          const W a = X[j | ba];
          X[j | ba] = X[j | bb];
          X[j | bb] = a;
        }
      }
      break;
    }
    case K_DENSE1: {
      const uint32_t tb = 1u << o.l0;
      const C u00 = coef[o.coef], u01 = coef[o.coef + 1], u10 = coef[o.coef + 2], u11 = coef[o.coef + 3];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins_m<NF>(g, mk) | lc, j1 = j0 | tb;
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          W* X = tiles[s];
          const W a = X[j0], b = X[j1];
          X[j0] = A::cmac2(u00, a, u01, b);
          X[j1] = A::cmac2(u10, a, u11, b);
        }
      }
      break;
    }
    case K_DENSE1R: {
      const uint32_t tb = 1u << o.l0;
      const typename A::R u00 = CRe<A>::get(coef[o.coef]), u01 = CRe<A>::get(coef[o.coef + 1]),
                          u10 = CRe<A>::get(coef[o.coef + 2]), u11 = CRe<A>::get(coef[o.coef + 3]);
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins_m<NF>(g, mk) | lc, j1 = j0 | tb;
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          W* X = tiles[s];
          const W a = X[j0], b = X[j1];
          X[j0] = A::rmac2(u00, a, u01, b);
          X[j1] = A::rmac2(u10, a, u11, b);
        }
      }
      break;
    }
    case K_DENSE2: {
      const uint32_t b0 = 1u << o.l0, b1 = 1u << o.l1;
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins_m<NF>(g, mk) | lc;
        const uint32_t id[4] = {j, j | b1, j | b0, j | b0 | b1};
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          W* X = tiles[s];
          W x[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) x[r] = X[id[r]];
#pragma unroll
          for (int r = 0; r < 4; ++r) X[id[r]] = A::cmac4(&coef[o.coef + 4 * r], x);
        }
      }
      break;
    }
    default:
      break;
  }
}

// Applies op `o` to tile T (2^k working amplitudes) whose base index is `base`.
// All threads of the block call it; the caller synchronises afterwards.
template <class A>
__device__ __forceinline__ void tile_apply(typename A::W* T, const TOp& o, const typename A::C* coef, uint64_t base,
                                           int k) {
  if ((base & o.ecmask) != o.ecmask) return;  // an outside control is 0 on this tile
  uint32_t mk[5];
  ins_masks(o, mk);
  switch (o.nfix) {
    case 0: tile_apply_n<A, 0, 1>(T, nullptr, o, coef, base, k, mk); break;
    case 1: tile_apply_n<A, 1, 1>(T, nullptr, o, coef, base, k, mk); break;
    case 2: tile_apply_n<A, 2, 1>(T, nullptr, o, coef, base, k, mk); break;
    case 3: tile_apply_n<A, 3, 1>(T, nullptr, o, coef, base, k, mk); break;
    default: tile_apply_n<A, 4, 1>(T, nullptr, o, coef, base, k, mk); break;
  }
}

// The same op applied to two tiles (psi and lambda of the adjoint sweep) in one loop.
template <class A>
__device__ __forceinline__ void tile_apply2(typename A::W* T, typename A::W* T2, const TOp& o,
                                            const typename A::C* coef, uint64_t base, int k) {
  if ((base & o.ecmask) != o.ecmask) return;
  uint32_t mk[5];
  ins_masks(o, mk);
  switch (o.nfix) {
    case 0: tile_apply_n<A, 0, 2>(T, T2, o, coef, base, k, mk); break;
    case 1: tile_apply_n<A, 1, 2>(T, T2, o, coef, base, k, mk); break;
    case 2: tile_apply_n<A, 2, 2>(T, T2, o, coef, base, k, mk); break;
    case 3: tile_apply_n<A, 3, 2>(T, T2, o, coef, base, k, mk); break;
    default: tile_apply_n<A, 4, 2>(T, T2, o, coef, base, k, mk); break;
  }
}

}  // namespace lqs
