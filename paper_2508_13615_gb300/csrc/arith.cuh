// Arithmetic policies for amplitude updates.
//
//   ArF32 -- complex64 storage, float32 arithmetic.
//   ArF64 -- complex128 storage, native float64 arithmetic.
//   ArDF  -- complex128 storage, double-float arithmetic on the float32 pipes.
//
// Why double-float: GB300's float64 units issue about 2 FMA per clock per SM
// against about 110 float32 FMA, so a native-float64 dense gate on a 30-qubit
// state is bound by float64 throughput at 2-3x the HBM pass time.  Here a
// double x is carried as an unevaluated sum hi + lo of two floats (about 47
// significant bits, Dekker 1971 / Knuth TAOCP 4.2.2 error-free transforms).
// Conversions avoid the float64 pipe: double -> (hi, lo) is pure integer bit
// manipulation, and (hi, lo) -> double is two exact bit-level widenings plus
// one float64 add, which rounds the pair to the nearest double.
//
// Every error-free step uses the explicitly rounded intrinsics (__fadd_rn,
// __fmul_rn, __fmaf_rn) so the compiler cannot contract or reassociate them.
#pragma once
#ifndef __CUDACC_RTC__  // runtime-compiled segment kernels bring their own integer types
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace lqs {

#define LQS_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------------------
// bit-level helpers shared by host and device (host versions allow CPU tests)
// ---------------------------------------------------------------------------
LQS_HD uint32_t f_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u; __builtin_memcpy(&u, &f, 4); return u;
#endif
}
LQS_HD float bits_f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f; __builtin_memcpy(&f, &u, 4); return f;
#endif
}
LQS_HD uint32_t d_hi(double d) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2hiint(d);
#else
  uint64_t u; __builtin_memcpy(&u, &d, 8); return (uint32_t)(u >> 32);
#endif
}
LQS_HD uint32_t d_lo(double d) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2loint(d);
#else
  uint64_t u; __builtin_memcpy(&u, &d, 8); return (uint32_t)u;
#endif
}
LQS_HD double hilo_d(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  uint64_t u = ((uint64_t)hi << 32) | lo; double d; __builtin_memcpy(&d, &u, 8); return d;
#endif
}
LQS_HD float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b; return r;
#endif
}
LQS_HD float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float r = a - b; return r;
#endif
}
LQS_HD float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b; return r;
#endif
}
LQS_HD float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

// Sign flip of a double without the float64 pipe.
LQS_HD double dneg(double d) { return hilo_d(d_hi(d) ^ 0x80000000u, d_lo(d)); }

// ---------------------------------------------------------------------------
// double <-> double-float conversions
// ---------------------------------------------------------------------------
struct DF { float h, l; };

// hi = x truncated to 24 significant bits; lo = the next 23 bits of x rounded
// to nearest, as a float.  Exact decomposition up to 2^-47 |x|.  Magnitudes
// below 2^-102 map to 0 (their float exponent for lo would underflow);
// magnitudes must be below 2^127.
LQS_HD DF d2df(double x) {
  const uint32_t H = d_hi(x), L = d_lo(x);
  const uint32_t s = H & 0x80000000u;
  const uint32_t e11 = (H >> 20) & 0x7FFu;
  // hi: rebias the exponent (1023 -> 127 is -896) and keep 23 mantissa bits.
  const uint32_t Hr = H - (896u << 20);
  const uint32_t hb = (((Hr << 3) | (L >> 29)) & 0x7FFFFFFFu) | s;
  // lo: the low 29 mantissa bits, value rest * 2^(e-52).  Put their top 23
  // bits (rounded) under an implicit one with exponent e-23 and subtract the
  // implicit one exactly: (1 + m/2^23) 2^(e-23) - 2^(e-23) = m 2^(e-46).
  const uint32_t ebs = ((e11 - 919u) << 23) | s;
  const uint32_t m = ((L >> 6) & 0x7FFFFFu) + ((L >> 5) & 1u);  // may carry to 2^23: still exact
  const float lo = fsub(bits_f(ebs + m), bits_f(ebs));
  const bool ok = (e11 - 920u) <= 230u;  // 2^-103 <= |x| < 2^127
  DF r;
  r.h = ok ? bits_f(hb) : 0.0f;
  r.l = ok ? lo : 0.0f;
  return r;
}

// Exact widening of a normal float to double by bit manipulation (zero and
// subnormal floats give a signed zero).
LQS_HD double f2d_bits(float f) {
  const uint32_t b = f_bits(f);
  const uint32_t s = b & 0x80000000u;
  const uint32_t em = b & 0x7FFFFFFFu;
  const bool nz = em >= 0x00800000u;
  const uint32_t H = nz ? (((em >> 3) + (896u << 20)) | s) : s;
  const uint32_t L = nz ? (b << 29) : 0u;
  return hilo_d(H, L);
}

// hi + lo rounded to the nearest double (one float64 add).
LQS_HD double df2d(DF v) { return f2d_bits(v.h) + f2d_bits(v.l); }

// Split a double into a double-float constant: hi = RN(x), lo = RN(x - hi).
// Host-side (coefficients are split once when a gate is prepared).
#ifndef __CUDACC_RTC__
inline DF split_const(double x) {
  DF r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}
#endif

// ---------------------------------------------------------------------------
// double-float arithmetic
// ---------------------------------------------------------------------------

// Accumulator s + e of a sum of products; e collects every rounding error.
struct DAcc { float s, e; };

// a * c exactly split: p = RN(a.h c.h), e = a.h c.h - p + a.h c.l + a.l c.h.
LQS_HD DAcc df_prod(DF a, DF c) {
  const float p = fmul(a.h, c.h);
  float e = ffma(a.h, c.h, -p);
  e = ffma(a.h, c.l, e);
  e = ffma(a.l, c.h, e);
  return DAcc{p, e};
}
// acc += a * c (Knuth's TwoSum on the leading parts).
LQS_HD void df_mac(DAcc& A, DF a, DF c) {
  const DAcc q = df_prod(a, c);
  const float s = fadd(A.s, q.s);
  const float bp = fsub(s, A.s);
  const float err = fadd(fsub(A.s, fsub(s, bp)), fsub(q.s, bp));
  A.s = s;
  A.e = fadd(A.e, fadd(err, q.e));
}
// acc += x (a double-float term).
LQS_HD void df_acc(DAcc& A, DF x) {
  const float s = fadd(A.s, x.h);
  const float bp = fsub(s, A.s);
  const float err = fadd(fsub(A.s, fsub(s, bp)), fsub(x.h, bp));
  A.s = s;
  A.e = fadd(A.e, fadd(err, x.l));
}
// Renormalise to |lo| <= ulp(hi)/2 (Dekker's FastTwoSum).
LQS_HD DF df_norm(DAcc A) {
  const float h = fadd(A.s, A.e);
  const float l = fsub(A.e, fsub(h, A.s));
  return DF{h, l};
}
LQS_HD DF df_neg(DF a) { return DF{-a.h, -a.l}; }
LQS_HD DF df_add(DF a, DF b) { DAcc A{a.h, a.l}; df_acc(A, b); return df_norm(A); }
LQS_HD DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

// ---------------------------------------------------------------------------
// complex types per policy
// ---------------------------------------------------------------------------
struct DFC { DF re, im; };         // working complex (double-float); no alignment, so registers stay free
struct DFK { DF re, im; };         // complex coefficient (double-float)

// 128-bit shared-memory accesses of working amplitudes (the buffers are
// 16-byte aligned per amplitude); other working types use plain accesses.
LQS_HD void st_w(DFC* p, const DFC& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
}
LQS_HD DFC ld_w(const DFC* p) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  return DFC{DF{f.x, f.y}, DF{f.z, f.w}};
}
LQS_HD void st_w(float2* p, const float2& v) { *p = v; }
LQS_HD float2 ld_w(const float2* p) { return *p; }
LQS_HD void st_w(double2* p, const double2& v) { *p = v; }
LQS_HD double2 ld_w(const double2* p) { return *p; }

struct ArF32 {
  using S = float2;  // storage amplitude
  using W = float2;  // working amplitude
  using C = float2;  // complex coefficient
  using R = float;   // real coefficient
  static constexpr int kAmpBytes = 8;
  static LQS_HD C cconst(double re, double im) { return make_float2((float)re, (float)im); }
  static LQS_HD R rconst(double x) { return (float)x; }
  static LQS_HD W load(const S& s) { return s; }
  static LQS_HD S store(W w) { return w; }
  static LQS_HD W zero() { return make_float2(0.f, 0.f); }
  static LQS_HD W cmul(C c, W a) { return make_float2(c.x * a.x - c.y * a.y, c.x * a.y + c.y * a.x); }
  static LQS_HD W cmac2(C c0, W a, C c1, W b) {
    return make_float2(c0.x * a.x - c0.y * a.y + c1.x * b.x - c1.y * b.y,
                       c0.x * a.y + c0.y * a.x + c1.x * b.y + c1.y * b.x);
  }
  static LQS_HD W cmac4(const C* c, const W* a) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      re += c[k].x * a[k].x - c[k].y * a[k].y;
      im += c[k].x * a[k].y + c[k].y * a[k].x;
    }
    return make_float2(re, im);
  }
  static LQS_HD W cmac4_raw(const C* c, const W* a) { return cmac4(c, a); }
  static LQS_HD W rmac2(R c0, W a, R c1, W b) { return make_float2(c0 * a.x + c1 * b.x, c0 * a.y + c1 * b.y); }
  static LQS_HD C kmul(C a, C b) { return cmul(a, b); }
  static LQS_HD C cconst1() { return make_float2(1.f, 0.f); }
  static LQS_HD W neg(W a) { return make_float2(-a.x, -a.y); }
  static LQS_HD W mul_i(W a) { return make_float2(-a.y, a.x); }
  static LQS_HD W add(W a, W b) { return make_float2(a.x + b.x, a.y + b.y); }
  static LQS_HD W sub(W a, W b) { return make_float2(a.x - b.x, a.y - b.y); }
  // raw-storage sign flips / i-multiplies (no arithmetic conversion)
  static LQS_HD S sneg(S a) { return make_float2(-a.x, -a.y); }
  static LQS_HD S smul_i(S a) { return make_float2(-a.y, a.x); }
  // float64 helpers for reductions
  static LQS_HD double re_d(W a) { return (double)a.x; }
  static LQS_HD double im_d(W a) { return (double)a.y; }
};

struct ArF64 {
  using S = double2;
  using W = double2;
  using C = double2;
  using R = double;
  static constexpr int kAmpBytes = 16;
  static LQS_HD C cconst(double re, double im) { return make_double2(re, im); }
  static LQS_HD R rconst(double x) { return x; }
  static LQS_HD W load(const S& s) { return s; }
  static LQS_HD S store(W w) { return w; }
  static LQS_HD W zero() { return make_double2(0.0, 0.0); }
  static LQS_HD W cmul(C c, W a) { return make_double2(c.x * a.x - c.y * a.y, c.x * a.y + c.y * a.x); }
  static LQS_HD W cmac2(C c0, W a, C c1, W b) {
    return make_double2(c0.x * a.x - c0.y * a.y + c1.x * b.x - c1.y * b.y,
                        c0.x * a.y + c0.y * a.x + c1.x * b.y + c1.y * b.x);
  }
  static LQS_HD W cmac4(const C* c, const W* a) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      re += c[k].x * a[k].x - c[k].y * a[k].y;
      im += c[k].x * a[k].y + c[k].y * a[k].x;
    }
    return make_double2(re, im);
  }
  static LQS_HD W cmac4_raw(const C* c, const W* a) { return cmac4(c, a); }
  static LQS_HD W rmac2(R c0, W a, R c1, W b) { return make_double2(c0 * a.x + c1 * b.x, c0 * a.y + c1 * b.y); }
  static LQS_HD C kmul(C a, C b) { return cmul(a, b); }
  static LQS_HD C cconst1() { return make_double2(1.0, 0.0); }
  static LQS_HD W neg(W a) { return make_double2(dneg(a.x), dneg(a.y)); }
  static LQS_HD W mul_i(W a) { return make_double2(dneg(a.y), a.x); }
  static LQS_HD W add(W a, W b) { return make_double2(a.x + b.x, a.y + b.y); }
  static LQS_HD W sub(W a, W b) { return make_double2(a.x - b.x, a.y - b.y); }
  static LQS_HD S sneg(S a) { return make_double2(dneg(a.x), dneg(a.y)); }
  static LQS_HD S smul_i(S a) { return make_double2(dneg(a.y), a.x); }
  static LQS_HD double re_d(W a) { return a.x; }
  static LQS_HD double im_d(W a) { return a.y; }
};

struct ArDF {
  using S = double2;
  using W = DFC;
  using C = DFK;
  using R = DF;
  static constexpr int kAmpBytes = 16;
#ifndef __CUDACC_RTC__  // host-side coefficient preparation
  static inline C cconst(double re, double im) { return DFK{split_const(re), split_const(im)}; }
  static inline R rconst(double x) { return split_const(x); }
#endif
  static LQS_HD W load(const S& s) { return DFC{d2df(s.x), d2df(s.y)}; }
  static LQS_HD S store(W w) { return make_double2(df2d(w.re), df2d(w.im)); }
  static LQS_HD W zero() { return DFC{DF{0.f, 0.f}, DF{0.f, 0.f}}; }
  static LQS_HD W cmul(C c, W a) {
    DAcc re = df_prod(a.re, c.re);
    df_mac(re, df_neg(a.im), c.im);
    DAcc im = df_prod(a.im, c.re);
    df_mac(im, a.re, c.im);
    return DFC{df_norm(re), df_norm(im)};
  }
  static LQS_HD W cmac2(C c0, W a, C c1, W b) {
    DAcc re = df_prod(a.re, c0.re);
    df_mac(re, df_neg(a.im), c0.im);
    df_mac(re, b.re, c1.re);
    df_mac(re, df_neg(b.im), c1.im);
    DAcc im = df_prod(a.im, c0.re);
    df_mac(im, a.re, c0.im);
    df_mac(im, b.im, c1.re);
    df_mac(im, b.re, c1.im);
    return DFC{df_norm(re), df_norm(im)};
  }
  static LQS_HD W cmac4(const C* c, const W* a) {
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
    return DFC{df_norm(re), df_norm(im)};
  }
  // cmac4 without the final renormalisation, for results that go straight
  // to float64 storage (df2d rounds hi + lo however they are split)
  static LQS_HD W cmac4_raw(const C* c, const W* a) {
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
    return DFC{DF{re.s, re.e}, DF{im.s, im.e}};
  }
  static LQS_HD W rmac2(R c0, W a, R c1, W b) {
    DAcc re = df_prod(a.re, c0);
    df_mac(re, b.re, c1);
    DAcc im = df_prod(a.im, c0);
    df_mac(im, b.im, c1);
    return DFC{df_norm(re), df_norm(im)};
  }
  static LQS_HD C kmul(C a, C b) {
    const DFC r = cmul(a, DFC{b.re, b.im});
    return DFK{r.re, r.im};
  }
  static LQS_HD C cconst1() { return DFK{DF{1.f, 0.f}, DF{0.f, 0.f}}; }
  static LQS_HD W neg(W a) { return DFC{df_neg(a.re), df_neg(a.im)}; }
  static LQS_HD W mul_i(W a) { return DFC{df_neg(a.im), a.re}; }
  static LQS_HD W add(W a, W b) { return DFC{df_add(a.re, b.re), df_add(a.im, b.im)}; }
  static LQS_HD W sub(W a, W b) { return DFC{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
  static LQS_HD S sneg(S a) { return make_double2(dneg(a.x), dneg(a.y)); }
  static LQS_HD S smul_i(S a) { return make_double2(dneg(a.y), a.x); }
  static LQS_HD double re_d(W a) { return df2d(a.re); }
  static LQS_HD double im_d(W a) { return df2d(a.im); }
};

}  // namespace lqs
