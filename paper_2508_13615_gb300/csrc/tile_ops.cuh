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

// Applies op `o` to tile T (2^k working amplitudes) whose base index is `base`.
// All threads of the block call it; the caller synchronises afterwards.
template <class A>
__device__ __forceinline__ void tile_apply(typename A::W* T, const TOp& o, const typename A::C* coef, uint64_t base,
                                           int k) {
  using W = typename A::W;
  if ((base & o.ecmask) != o.ecmask) return;  // an outside control is 0 on this tile
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const uint32_t ng = 1u << (k - o.nfix);
  const uint32_t lc = o.lcmask;
  switch (o.kind) {
    case K_PHASE: {
      const typename A::C f = coef[o.coef];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
        T[j] = phase_apply<A>(f, o.special, T[j]);
      }
      break;
    }
    case K_DIAG1: {
      if (o.l0 >= 0) {
        const typename A::C d0 = coef[o.coef], d1 = coef[o.coef + 1];
        const uint32_t tb = 1u << o.l0;
        for (uint32_t g = tid; g < ng; g += nth) {
          const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
          T[j] = A::cmul(d0, T[j]);
          T[j | tb] = A::cmul(d1, T[j | tb]);
        }
      } else {
        const typename A::C d = coef[o.coef + ((base & o.e0) ? 1 : 0)];
        for (uint32_t g = tid; g < ng; g += nth) {
          const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
          T[j] = A::cmul(d, T[j]);
        }
      }
      break;
    }
    case K_DIAG2: {
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
        const int b0 = o.l0 >= 0 ? (int)((j >> o.l0) & 1u) : ((base & o.e0) ? 1 : 0);
        const int b1 = o.l1 >= 0 ? (int)((j >> o.l1) & 1u) : ((base & o.e1) ? 1 : 0);
        T[j] = A::cmul(coef[o.coef + 2 * b0 + b1], T[j]);
      }
      break;
    }
    case K_ANTI1: {
      const uint32_t tb = 1u << o.l0;
      const typename A::C f0 = coef[o.coef], f1 = coef[o.coef + 1];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins0(g, o.fix, o.nfix) | lc, j1 = j0 | tb;
        const W a = T[j0], b = T[j1];
        if (o.special == 1) {
          T[j0] = b;
          T[j1] = a;
        } else {
          T[j0] = A::cmul(f0, b);
          T[j1] = A::cmul(f1, a);
        }
      }
      break;
    }
    case K_SWAP: {
      const uint32_t ba = 1u << o.l0, bb = 1u << o.l1;
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
        const W a = T[j | ba];
        T[j | ba] = T[j | bb];
        T[j | bb] = a;
      }
      break;
    }
    case K_DENSE1: {
      const uint32_t tb = 1u << o.l0;
      const typename A::C u00 = coef[o.coef], u01 = coef[o.coef + 1], u10 = coef[o.coef + 2],
                          u11 = coef[o.coef + 3];
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins0(g, o.fix, o.nfix) | lc, j1 = j0 | tb;
        const W a = T[j0], b = T[j1];
        T[j0] = A::cmac2(u00, a, u01, b);
        T[j1] = A::cmac2(u10, a, u11, b);
      }
      break;
    }
    case K_DENSE1R: {
      const uint32_t tb = 1u << o.l0;
      const typename A::R u00 = CRe<A>::get(coef[o.coef]), u01 = CRe<A>::get(coef[o.coef + 1]),
                          u10 = CRe<A>::get(coef[o.coef + 2]), u11 = CRe<A>::get(coef[o.coef + 3]);
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j0 = ins0(g, o.fix, o.nfix) | lc, j1 = j0 | tb;
        const W a = T[j0], b = T[j1];
        T[j0] = A::rmac2(u00, a, u01, b);
        T[j1] = A::rmac2(u10, a, u11, b);
      }
      break;
    }
    case K_DENSE2: {
      const uint32_t b0 = 1u << o.l0, b1 = 1u << o.l1;
      for (uint32_t g = tid; g < ng; g += nth) {
        const uint32_t j = ins0(g, o.fix, o.nfix) | lc;
        const uint32_t id[4] = {j, j | b1, j | b0, j | b0 | b1};
        W x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = T[id[r]];
#pragma unroll
        for (int r = 0; r < 4; ++r) T[id[r]] = A::cmac4(&coef[o.coef + 4 * r], x);
      }
      break;
    }
    default:
      break;
  }
}

}  // namespace lqs
