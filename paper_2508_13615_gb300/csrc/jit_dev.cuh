// Device helpers for runtime-compiled segment kernels: the pair and quad
// updates of gates on local qubits (Sec. 2, Fig. 1a) written for a tile held
// in registers.
//
// A compiled segment is straight-line code: every register index, layout,
// control pattern and coefficient offset is a constant of its source, so the
// kernel carries none of the register-tile interpreter's per-op dispatch.
// The helpers here are the pair and quad updates it is written in; they use
// the same arithmetic policies (arith.cuh) as every other kernel of the
// library, so a compiled segment and the interpreter compute the same
// products and sums.
#pragma once
#include "arith.cuh"
#include "tile.cuh"

namespace lqs {
namespace jit {

// Amplitude updates of a compiled segment.  For double-float they return the
// accumulator pair (leading sum, collected errors) without renormalising it:
// that pair stands for the same value, and the next product, sum or float64
// conversion takes it as it is (3 fewer float32 instructions per real
// output).  The low parts then grow with every update, so the segment
// renormalises every register after a bounded number of updates (renorm).
// The other policies have no renormalisation to skip.
template <class A> struct Lz {
  using W = typename A::W;
  using C = typename A::C;
  using R = typename A::R;
  static __device__ __forceinline__ W cmul(const C& c, const W& a) { return A::cmul(c, a); }
  static __device__ __forceinline__ W cmac2(const C& c0, const W& a, const C& c1, const W& b) {
    return A::cmac2(c0, a, c1, b);
  }
  static __device__ __forceinline__ W cmac4(const C* c, const W* a) { return A::cmac4(c, a); }
  static __device__ __forceinline__ W rmac2(const R& c0, const W& a, const R& c1, const W& b) {
    return A::rmac2(c0, a, c1, b);
  }
  static __device__ __forceinline__ C kmul(const C& a, const C& b) { return A::kmul(a, b); }
  static __device__ __forceinline__ void renorm(W&) {}
  // SX x + k y for a real k
  template <int SX>
  static __device__ __forceinline__ W uma(const W& x, const R& k, const W& y) {
    W r;
    r.x = k * y.x + (SX > 0 ? x.x : -x.x);
    r.y = k * y.y + (SX > 0 ? x.y : -x.y);
    return r;
  }
  static __device__ __forceinline__ W rscale(const R& g, const W& x) {
    W r;
    r.x = g * x.x;
    r.y = g * x.y;
    return r;
  }
  // x + SY y
  template <int SY>
  static __device__ __forceinline__ W uadd(const W& x, const W& y) {
    W r;
    r.x = SY > 0 ? x.x + y.x : x.x - y.x;
    r.y = SY > 0 ? x.y + y.y : x.y - y.y;
    return r;
  }
};
template <> struct Lz<ArDF> {
  using W = DFC;
  using C = DFK;
  static __device__ __forceinline__ DF raw(const DAcc& a) { return DF{a.s, a.e}; }
  static __device__ __forceinline__ W cmul(const C& c, const W& a) {
    DAcc re = df_prod(a.re, c.re);
    df_mac(re, df_neg(a.im), c.im);
    DAcc im = df_prod(a.im, c.re);
    df_mac(im, a.re, c.im);
    return W{raw(re), raw(im)};
  }
  static __device__ __forceinline__ W cmac2(const C& c0, const W& a, const C& c1, const W& b) {
    DAcc re = df_prod(a.re, c0.re);
    df_mac(re, df_neg(a.im), c0.im);
    df_mac(re, b.re, c1.re);
    df_mac(re, df_neg(b.im), c1.im);
    DAcc im = df_prod(a.im, c0.re);
    df_mac(im, a.re, c0.im);
    df_mac(im, b.im, c1.re);
    df_mac(im, b.re, c1.im);
    return W{raw(re), raw(im)};
  }
  static __device__ __forceinline__ W cmac4(const C* c, const W* a) {
    DAcc re = df_prod(a[0].re, c[0].re);
    df_mac(re, df_neg(a[0].im), c[0].im);
    DAcc im = df_prod(a[0].im, c[0].re);
    df_mac(im, a[0].re, c[0].im);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      df_mac(re, a[k].re, c[k].re);
      df_mac(re, df_neg(a[k].im), c[k].im);
      df_mac(im, a[k].im, c[k].re);
      df_mac(im, a[k].re, c[k].im);
    }
    return W{raw(re), raw(im)};
  }
  static __device__ __forceinline__ W rmac2(const DF& c0, const W& a, const DF& c1, const W& b) {
    DAcc re = df_prod(a.re, c0);
    df_mac(re, b.re, c1);
    DAcc im = df_prod(a.im, c0);
    df_mac(im, b.im, c1);
    return W{raw(re), raw(im)};
  }
  static __device__ __forceinline__ C kmul(const C& a, const C& b) {
    const W r = cmul(a, W{b.re, b.im});
    return C{r.re, r.im};
  }
  static __device__ __forceinline__ void renorm(W& w) {
    w.re = df_norm(DAcc{w.re.h, w.re.l});
    w.im = df_norm(DAcc{w.im.h, w.im.l});
  }
  // SX x + k y for a real k: one exact product, one TwoSum and the error terms
  template <int SX>
  static __device__ __forceinline__ DF uma1(const DF& x, const DF& k, const DF& y) {
    const DAcc q = df_prod(y, k);
    const float xh = SX > 0 ? x.h : -x.h, xl = SX > 0 ? x.l : -x.l;
    const float s = fadd(q.s, xh);
    const float bp = fsub(s, q.s);
    const float err = fadd(fsub(q.s, fsub(s, bp)), fsub(xh, bp));
    return DF{s, fadd(q.e, fadd(err, xl))};
  }
  template <int SX>
  static __device__ __forceinline__ W uma(const W& x, const DF& k, const W& y) {
    return W{uma1<SX>(x.re, k, y.re), uma1<SX>(x.im, k, y.im)};
  }
  static __device__ __forceinline__ W rscale(const DF& g, const W& x) {
    return W{raw(df_prod(x.re, g)), raw(df_prod(x.im, g))};
  }
  // x + SY y: one TwoSum of the leading parts, the low parts and the error added
  template <int SY>
  static __device__ __forceinline__ DF uadd1(const DF& x, const DF& y) {
    const float yh = SY > 0 ? y.h : -y.h, yl = SY > 0 ? y.l : -y.l;
    const float s = fadd(x.h, yh);
    const float bp = fsub(s, x.h);
    const float err = fadd(fsub(x.h, fsub(s, bp)), fsub(yh, bp));
    return DF{s, fadd(fadd(x.l, yl), err)};
  }
  template <int SY>
  static __device__ __forceinline__ W uadd(const W& x, const W& y) {
    return W{uadd1<SY>(x.re, y.re), uadd1<SY>(x.im, y.im)};
  }
};

template <class A>
__device__ __forceinline__ void renorm(typename A::W& a) { Lz<A>::renorm(a); }

template <class A> struct Re;
template <> struct Re<ArF32> { static __device__ __forceinline__ float get(const float2& c) { return c.x; } };
template <> struct Re<ArF64> { static __device__ __forceinline__ double get(const double2& c) { return c.x; } };
template <> struct Re<ArDF> { static __device__ __forceinline__ DF get(const DFK& c) { return c.re; } };

// (a, b) <- (u00 a + u01 b, u10 a + u11 b)
template <class A>
__device__ __forceinline__ void d1(typename A::W& a, typename A::W& b, const typename A::C& u00,
                                   const typename A::C& u01, const typename A::C& u10, const typename A::C& u11) {
  const typename A::W x = a, y = b;
  a = Lz<A>::cmac2(u00, x, u01, y);
  b = Lz<A>::cmac2(u10, x, u11, y);
}

// the same with a real matrix (real parts of the coefficients)
template <class A>
__device__ __forceinline__ void d1r(typename A::W& a, typename A::W& b, const typename A::C& u00,
                                    const typename A::C& u01, const typename A::C& u10, const typename A::C& u11) {
  const typename A::W x = a, y = b;
  a = Lz<A>::rmac2(Re<A>::get(u00), x, Re<A>::get(u01), y);
  b = Lz<A>::rmac2(Re<A>::get(u10), x, Re<A>::get(u11), y);
}

// A real 2x2 that is g times an orthogonal matrix, m11 = SG m00 and
// m10 = -SG m01 with SG = +-1 (rotations such as RY, reflections such as H).
// Divided by m00 or m10, whichever has the larger modulus, each row keeps one
// entry of modulus 1, so each output costs one product and one sum:
//   form A (g = m00, |m00| >= |m01|): a' = a + k0 b,     b' = SG b + k1 a
//   form B (g = m10, |m01| >  |m00|): a' = -SG b + k0 a,  b' = a + k1 b
// with |k0|, |k1| <= 1 for orthogonal matrices.  The caller multiplies the
// amplitudes by the product of the g's afterwards (rscale).
template <class A, int SG>
__device__ __forceinline__ void u1a(typename A::W& a, typename A::W& b, const typename A::C& k0,
                                    const typename A::C& k1) {
  const typename A::W x = a, y = b;
  a = Lz<A>::template uma<1>(x, Re<A>::get(k0), y);
  b = Lz<A>::template uma<SG>(y, Re<A>::get(k1), x);
}
template <class A, int SG>
__device__ __forceinline__ void u1b(typename A::W& a, typename A::W& b, const typename A::C& k0,
                                    const typename A::C& k1) {
  const typename A::W x = a, y = b;
  a = Lz<A>::template uma<-SG>(y, Re<A>::get(k0), x);
  b = Lz<A>::template uma<1>(x, Re<A>::get(k1), y);
}

// The Hadamard pattern (m00 = m01 = m10 = -m11 = g): form A with k0 = k1 = 1,
// a' = a + b and b' = a - b, sums only; g joins the product of the g's.
template <class A>
__device__ __forceinline__ void u1h(typename A::W& a, typename A::W& b) {
  const typename A::W x = a, y = b;
  a = Lz<A>::template uadd<1>(x, y);
  b = Lz<A>::template uadd<-1>(x, y);
}

// (x0..x3) <- U x with U row-major at u[0..15]
template <class A>
__device__ __forceinline__ void d2(typename A::W& x0, typename A::W& x1, typename A::W& x2, typename A::W& x3,
                                   const typename A::C* u) {
  const typename A::W x[4] = {x0, x1, x2, x3};
  x0 = Lz<A>::cmac4(u, x);
  x1 = Lz<A>::cmac4(u + 4, x);
  x2 = Lz<A>::cmac4(u + 8, x);
  x3 = Lz<A>::cmac4(u + 12, x);
}

// (a, b) <- (f0 b, f1 a)
template <class A>
__device__ __forceinline__ void anti(typename A::W& a, typename A::W& b, const typename A::C& f0,
                                     const typename A::C& f1) {
  const typename A::W x = a;
  a = Lz<A>::cmul(f0, b);
  b = Lz<A>::cmul(f1, x);
}

// exchange a and b where p holds (a per-thread predicate)
template <class W>
__device__ __forceinline__ void swap_if(bool p, W& a, W& b) {
  const W x = a, y = b;
  a = p ? y : x;
  b = p ? x : y;
}

// Exchange-buffer position of a local amplitude index (same fold as the
// interpreter's buffer, so bank spread is unchanged).  It is linear over XOR,
// so for a thread part jt and a register part c with disjoint bits,
// swz(jt | c) = swz(jt) ^ swz(c): the thread part is folded once per layout
// and the register parts are constants.
template <int SZ>
__device__ __forceinline__ uint32_t swz(uint32_t j) {
  if (SZ == 16) return j ^ (((j >> 3) ^ (j >> 6) ^ (j >> 9)) & 7u);
  return j ^ (((j >> 4) ^ (j >> 8)) & 15u);
}

// Bit q of a tile's base index (an outside qubit's value on that tile), as
// the 0 / 1 that selects a folded permutation's outside-controlled flips.
__device__ __forceinline__ uint32_t obit(uint64_t base, int q) { return (uint32_t)(base >> q) & 1u; }

// Bank bits an exchange's swizzle changes relative to swz: bit b is the
// parity of the position bits in m_b (the masks are literal constants, so
// unused ones vanish at compile time).
__device__ __forceinline__ uint32_t pfold(uint32_t j, uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
  uint32_t f = 0;
  if (m0) f |= (uint32_t)__popc(j & m0) & 1u;
  if (m1) f |= ((uint32_t)__popc(j & m1) & 1u) << 1;
  if (m2) f |= ((uint32_t)__popc(j & m2) & 1u) << 2;
  if (m3) f |= ((uint32_t)__popc(j & m3) & 1u) << 3;
  return f;
}

// Issues the bulk copies of one tile into `buf`, one row per thread (rows
// beyond the block size wrap): the work is spread over the block instead of
// one warp, so no warp falls behind the others before the next barrier.
// `my_roff` is row_offset(G, tid), formed once per launch.  The phase's
// expected byte count (its only arrival) must already be posted by thread 0
// (seg_expect) before any thread issues a copy of that phase.
template <class S>
__device__ __forceinline__ void seg_copy(const TileGeom& G, S* buf, const S* psi, uint64_t base, uint64_t* bar,
                                         uint64_t my_roff) {
  const uint32_t tid = threadIdx.x;
  const uint32_t nrows = 1u << G.r;
  const uint32_t per_row = 1u << G.b;
  for (uint32_t row = tid; row < nrows; row += blockDim.x)
    bulk_g2s(buf + (size_t)row * per_row, psi + base + (row == tid ? my_roff : row_offset(G, row)), G.row_bytes, bar);
}
__device__ __forceinline__ void seg_expect(const TileGeom& G, uint64_t* bar, uint32_t ntiles = 1) {
  mbar_expect_tx(bar, ntiles * (1u << G.r) * G.row_bytes);
}

// ---------------------------------------------------------------------------
// compiled adjoint: gradient partials Im <lambda|G|psi>
// ---------------------------------------------------------------------------
template <class A> struct Dfc;
template <> struct Dfc<ArF32> {
  static __device__ __forceinline__ DFC get(const float2& w) { return DFC{DF{w.x, 0.f}, DF{w.y, 0.f}}; }
};
template <> struct Dfc<ArF64> {
  static __device__ __forceinline__ DFC get(const double2& w) { return DFC{d2df(w.x), d2df(w.y)}; }
};
template <> struct Dfc<ArDF> {
  static __device__ __forceinline__ DFC get(const DFC& w) { return w; }
};

// Per-tile partial sums: double-float for complex128 (the products must keep
// about 2^-46 relative accuracy), float32 for complex64 states.  Either is
// added in float64 across tiles.
template <class A> struct GAcc {
  using T = DAcc;  // running sum (leading part, accumulated errors)
  using V = DF;    // one term
  static __device__ __forceinline__ T zero() { return DAcc{0.f, 0.f}; }
};
template <> struct GAcc<ArF32> {
  using T = float;
  using V = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
};

// acc += sign * Im(conj(l) p) = sign * (l.re p.im - l.im p.re)
__device__ __forceinline__ void gim_t(DAcc& acc, const DFC& l, const DFC& p, bool neg) {
  df_mac(acc, neg ? df_neg(l.re) : l.re, p.im);
  df_mac(acc, neg ? l.im : df_neg(l.im), p.re);
}
__device__ __forceinline__ void gim_t(float& acc, const float2& l, const float2& p, bool neg) {
  const float s = neg ? -1.f : 1.f;
  acc = __fmaf_rn(s * l.x, p.y, acc);
  acc = __fmaf_rn(-s * l.y, p.x, acc);
}
// acc += sign * Re(conj(l) p) = sign * (l.re p.re + l.im p.im)
__device__ __forceinline__ void gre_t(DAcc& acc, const DFC& l, const DFC& p, bool neg) {
  df_mac(acc, neg ? df_neg(l.re) : l.re, p.re);
  df_mac(acc, neg ? df_neg(l.im) : l.im, p.im);
}
__device__ __forceinline__ void gre_t(float& acc, const float2& l, const float2& p, bool neg) {
  const float s = neg ? -1.f : 1.f;
  acc = __fmaf_rn(s * l.x, p.x, acc);
  acc = __fmaf_rn(s * l.y, p.y, acc);
}
template <class A>
__device__ __forceinline__ void gim(typename GAcc<A>::T& acc, const typename A::W& l, const typename A::W& p, bool neg) {
  if constexpr (sizeof(typename GAcc<A>::T) == sizeof(float)) gim_t(acc, l, p, neg);
  else gim_t(acc, Dfc<A>::get(l), Dfc<A>::get(p), neg);
}
template <class A>
__device__ __forceinline__ void gre(typename GAcc<A>::T& acc, const typename A::W& l, const typename A::W& p, bool neg) {
  if constexpr (sizeof(typename GAcc<A>::T) == sizeof(float)) gre_t(acc, l, p, neg);
  else gre_t(acc, Dfc<A>::get(l), Dfc<A>::get(p), neg);
}

// One term w = Im(conj(l) p), shared by every Z / P1 partial of a merged
// diagonal run (those partials are signed sums of the same w_j).
template <class A>
__device__ __forceinline__ typename GAcc<A>::V wim(const typename A::W& l, const typename A::W& p) {
  typename GAcc<A>::T a = GAcc<A>::zero();
  gim<A>(a, l, p, false);
  if constexpr (sizeof(typename GAcc<A>::T) == sizeof(float)) return a;
  else return df_norm(a);
}
__device__ __forceinline__ void wadd(DAcc& acc, const DF& w, bool neg) { df_acc(acc, neg ? df_neg(w) : w); }
__device__ __forceinline__ void wadd(float& acc, float w, bool neg) { acc = neg ? acc - w : acc + w; }
__device__ __forceinline__ DAcc gneg(const DAcc& a, bool neg) { return neg ? DAcc{-a.s, -a.e} : a; }
__device__ __forceinline__ float gneg(float a, bool neg) { return neg ? -a : a; }

// Per-warp partial-sum slots.  Double-float kernels keep each 8-byte slot as
// a double-float pair and add to it with float32 operations (float64 adds run
// on a far narrower pipe); the slot is read as a float64 once, after the tile
// loop.  Float32 kernels add in float64.
__device__ __forceinline__ void slot_add(double* slot, const DF& v) {
  DF* d = reinterpret_cast<DF*>(slot);
  *d = df_add(*d, v);
}
template <class A>
__device__ __forceinline__ double slot_get(const double* slot) {
  if constexpr (sizeof(typename GAcc<A>::T) == sizeof(float)) return *slot;
  else return df2d(*reinterpret_cast<const DF*>(slot));
}

// Warp sum of a partial, added by lane 0 to the warp's slot.  All 32 lanes
// must call it.
__device__ __forceinline__ void gflush(DAcc a, double* slot) {
  DF v = df_norm(a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    v = df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)});
  if ((threadIdx.x & 31u) == 0) slot_add(slot, v);
}
__device__ __forceinline__ void gflush(float a, double* slot) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if ((threadIdx.x & 31u) == 0) *slot += (double)a;
}

// Four per-lane partials summed over the warp at once (a reduce-scatter):
// two halving exchanges leave each lane with one of the four (lanes with bit
// 4 take slots 2-3, with bit 3 the odd one), three butterfly steps complete
// the sums, and lanes 0, 8, 16, 24 add them to slots s0..s3 (null: unused).
// All 32 lanes must call it.
__device__ __forceinline__ DF shfl_df(const DF& v, int off) {
  return DF{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
}
__device__ __forceinline__ void gflush4(const DAcc& a0, const DAcc& a1, const DAcc& a2, const DAcc& a3, double* s0,
                                        double* s1, double* s2, double* s3) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool u16 = lane & 16u, u8 = lane & 8u;
  const DF v0 = df_norm(a0), v1 = df_norm(a1), v2 = df_norm(a2), v3 = df_norm(a3);
  DF k0 = u16 ? v2 : v0, k1 = u16 ? v3 : v1;
  const DF t0 = u16 ? v0 : v2, t1 = u16 ? v1 : v3;
  k0 = df_add(k0, shfl_df(t0, 16));
  k1 = df_add(k1, shfl_df(t1, 16));
  DF k = u8 ? k1 : k0;
  k = df_add(k, shfl_df(u8 ? k0 : k1, 8));
  k = df_add(k, shfl_df(k, 4));
  k = df_add(k, shfl_df(k, 2));
  k = df_add(k, shfl_df(k, 1));
  double* s = u16 ? (u8 ? s3 : s2) : (u8 ? s1 : s0);
  if ((lane & 7u) == 0 && s) slot_add(s, k);
}
__device__ __forceinline__ void gflush4(float a0, float a1, float a2, float a3, double* s0, double* s1, double* s2,
                                        double* s3) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool u16 = lane & 16u, u8 = lane & 8u;
  float k0 = u16 ? a2 : a0, k1 = u16 ? a3 : a1;
  const float t0 = u16 ? a0 : a2, t1 = u16 ? a1 : a3;
  k0 += __shfl_xor_sync(0xffffffffu, t0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, t1, 16);
  float k = u8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, u8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  double* s = u16 ? (u8 ? s3 : s2) : (u8 ? s1 : s0);
  if ((lane & 7u) == 0 && s) *s += (double)k;
}

// A running sum held by one lane across the tile loop and stored in its
// slot once: double-float for complex128 kernels, float64 for complex64.
template <class A> struct LaneAcc {
  DF s;
  __device__ __forceinline__ void zero() { s = DF{0.f, 0.f}; }
  __device__ __forceinline__ void add(const DF& x, bool neg) { s = df_add(s, neg ? df_neg(x) : x); }
  __device__ __forceinline__ void put(double* slot) const { *reinterpret_cast<DF*>(slot) = s; }
};
template <> struct LaneAcc<ArF32> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(float x, bool neg) { s += neg ? -(double)x : (double)x; }
  __device__ __forceinline__ void put(double* slot) const { *slot = s; }
};
__device__ __forceinline__ DF shfl_idx(const DF& v, uint32_t src) {
  return DF{__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}
__device__ __forceinline__ float shfl_idx(float v, uint32_t src) { return __shfl_sync(0xffffffffu, v, src); }

// Walsh butterfly over the warp: lane l ends with sum_i (-1)^popc(i & l) v_i,
// so lane 0 holds the plain sum and lane 2^m the sum signed by lane bit m.
// All 32 lanes must call it.
__device__ __forceinline__ DF wht(DAcc a) {
  DF v = df_norm(a);
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const DF o{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
    v = (lane & (uint32_t)off) ? df_sub(o, v) : df_add(v, o);
  }
  return v;
}
__device__ __forceinline__ float wht(float v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float o = __shfl_xor_sync(0xffffffffu, v, off);
    v = (lane & (uint32_t)off) ? o - v : v + o;
  }
  return v;
}
// slot += (neg ? -w : w) where `cond` holds (one lane per slot).
__device__ __forceinline__ void gput(const DF& w, bool cond, bool neg, double* slot) {
  if (cond) slot_add(slot, neg ? df_neg(w) : w);
}
__device__ __forceinline__ void gput(float w, bool cond, bool neg, double* slot) {
  if (cond) *slot += neg ? -(double)w : (double)w;
}

// ---------------------------------------------------------------------------
// compiled Pauli passes: |psi_j|^2, lambda accumulators
// ---------------------------------------------------------------------------
__device__ __forceinline__ DF pnorm2(const DFC& v) {
  DAcc a = df_prod(v.re, v.re);
  df_mac(a, v.im, v.im);
  return df_norm(a);
}
__device__ __forceinline__ float pnorm2(const float2& v) { return __fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y)); }
template <class A>
__device__ __forceinline__ typename GAcc<A>::V pn2(const typename A::W& w) {
  if constexpr (sizeof(typename GAcc<A>::T) == sizeof(float)) return pnorm2(w);
  else return pnorm2(Dfc<A>::get(w));
}

// lambda_j accumulated per component: double-float for complex128 states,
// float32 for complex64.
template <class A> struct LAcc {
  DAcc re, im;
  __device__ __forceinline__ void init(const typename A::W& w) {
    const DFC v = Dfc<A>::get(w);
    re = DAcc{v.re.h, v.re.l};
    im = DAcc{v.im.h, v.im.l};
  }
  __device__ __forceinline__ void zero() { re = im = DAcc{0.f, 0.f}; }
  // += c * sign * i^PH * w
  template <int PH>
  __device__ __forceinline__ void add(const typename A::W& w, const DF& c, bool neg) {
    const DFC v = Dfc<A>::get(w);
    DF vr = v.re, vi = v.im;
    if (PH & 1) { const DF t = vr; vr = df_neg(vi); vi = t; }
    if (PH & 2) { vr = df_neg(vr); vi = df_neg(vi); }
    if (neg) { vr = df_neg(vr); vi = df_neg(vi); }
    df_mac(re, vr, c);
    df_mac(im, vi, c);
  }
  __device__ __forceinline__ typename A::W out() const;
};
template <> __device__ __forceinline__ DFC LAcc<ArDF>::out() const { return DFC{df_norm(re), df_norm(im)}; }
template <> __device__ __forceinline__ double2 LAcc<ArF64>::out() const {
  return make_double2(df2d(df_norm(re)), df2d(df_norm(im)));
}
template <> struct LAcc<ArF32> {
  float re, im;
  __device__ __forceinline__ void init(const float2& w) { re = w.x; im = w.y; }
  __device__ __forceinline__ void zero() { re = im = 0.f; }
  template <int PH>
  __device__ __forceinline__ void add(const float2& w, float c, bool neg) {
    float vr = w.x, vi = w.y;
    if (PH & 1) { const float t = vr; vr = -vi; vi = t; }
    if (PH & 2) { vr = -vr; vi = -vi; }
    if (neg) { vr = -vr; vi = -vi; }
    re = __fmaf_rn(vr, c, re);
    im = __fmaf_rn(vi, c, im);
  }
  __device__ __forceinline__ float2 out() const { return make_float2(re, im); }
};
// Real coefficient of a Pauli word in the parameter block, per policy.
template <class A> struct PCoef { using T = DF; };
template <> struct PCoef<ArF32> { using T = float; };
// sum of signed coefficients (diagonal words of lambda)
__device__ __forceinline__ void cadd(DAcc& a, const DF& c, bool neg) { df_acc(a, neg ? df_neg(c) : c); }
__device__ __forceinline__ void cadd(float& a, float c, bool neg) { a = neg ? a - c : a + c; }
__device__ __forceinline__ DF cfin(const DAcc& a) { return df_norm(a); }
__device__ __forceinline__ float cfin(float a) { return a; }

// Barrier over a group of warps: named barrier `id` (1..15; 0 is the
// block-wide barrier) for `nthreads` threads, a multiple of 32.
__device__ __forceinline__ void bar_group(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace jit
}  // namespace lqs
