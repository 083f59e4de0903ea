// Double-float ("df64") arithmetic: a real number is an unevaluated sum h + l
// of two floats with |l| <= ulp(h) / 2, about 48 significant bits.  Used as
// the compute type for complex128 states: the FP64 pipe of a GB300 runs at
// 1/62 of the FP32 rate, so gate and inner-product arithmetic on FP32 pairs
// is several times faster than native FP64 at an error far below the 1e-10
// accuracy target of the complex128 mode.
//
// Algorithms (written from their published statements):
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e == a + b exactly;
//   Fast2Sum (Dekker 1971), valid when |a| >= |b|;
//   TwoProduct with a fused multiply-add: p + e == a * b exactly;
//   double-float add / multiply as in the "sloppy" variants of Hida, Li and
//   Bailey's double-double library (relative error ~2^-47).
// Conversions between IEEE double and df64 split the encoding with integer
// operations (no FP64 instruction on the load side); df64 -> double costs one
// FP64 addition.
//
// The file compiles as CUDA (device and host) and as plain C++ (host only) so
// the conversions and arithmetic are unit-tested on the CPU.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define DF_HD inline
#ifndef __align__
#define __align__(n) alignas(n)
#endif
#endif

namespace sv {

// sv::fma(df, df, df) below must not hide the float / double overloads.
#ifdef __CUDACC__
using ::fma;
#else
using std::fma;
#endif

DF_HD float df_fmaf(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

DF_HD uint64_t df_d2u(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}

DF_HD double df_u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

DF_HD uint32_t df_f2u(float x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}

DF_HD float df_u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

DF_HD float df_u32_to_f(uint32_t r) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(r);
#else
  return (float)r;
#endif
}

DF_HD int df_clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// Exact float -> double by re-encoding the bits (no FP64 instruction),
// subnormal floats included.
DF_HD double df_f2d_exact(float f) {
  const uint32_t u = df_f2u(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t mf = u & 0x7FFFFFu;
  if (e == 0) {
    if (mf == 0) return df_u2d(sign);
    const int p = 31 - df_clz32(mf);  // value = mf * 2^-149, leading bit p
    const uint64_t m = ((uint64_t)mf << (52 - p)) & 0xFFFFFFFFFFFFFull;
    return df_u2d(sign | ((uint64_t)(p - 149 + 1023) << 52) | m);
  }
  const uint64_t m = (uint64_t)mf << 29;
  if (e == 0xFFu) return df_u2d(sign | 0x7FF0000000000000ull | m);
  return df_u2d(sign | ((uint64_t)(e - 127 + 1023) << 52) | m);
}

struct df;
DF_HD df df_make(float h, float l);

struct __align__(8) df {
  float h, l;
  df() = default;
  DF_HD df(float v) : h(v), l(0.f) {}
  DF_HD df(int v) : h((float)v), l(0.f) {}
  DF_HD explicit df(double x);
  DF_HD explicit operator double() const { return df_f2d_exact(h) + df_f2d_exact(l); }
};

DF_HD df df_make(float h, float l) {
  df r;
  r.h = h;
  r.l = l;
  return r;
}

// Knuth TwoSum.
DF_HD df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df_make(s, e);
}

// Dekker Fast2Sum (|a| >= |b|).
DF_HD df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df_make(s, b - (s - a));
}

DF_HD df operator+(df a, df b) {
  const df s = df_two_sum(a.h, b.h);
  return df_fast_two_sum(s.h, s.l + (a.l + b.l));
}

DF_HD df operator-(df a) { return df_make(-a.h, -a.l); }
DF_HD df operator-(df a, df b) { return a + (-b); }

DF_HD df operator*(df a, df b) {
  const float p = a.h * b.h;
  float e = df_fmaf(a.h, b.h, -p);  // TwoProduct error term
  e = df_fmaf(a.h, b.l, df_fmaf(a.l, b.h, e));
  return df_fast_two_sum(p, e);
}

DF_HD df &operator+=(df &a, df b) {
  a = a + b;
  return a;
}

// a * b + c with one renormalisation.
DF_HD df fma(df a, df b, df c) {
  const float p = a.h * b.h;
  float e = df_fmaf(a.h, b.h, -p);
  e = df_fmaf(a.h, b.l, df_fmaf(a.l, b.h, e));
  const df s = df_two_sum(p, c.h);
  return df_fast_two_sum(s.h, s.l + (e + c.l));
}

// IEEE double -> df64: h keeps the top 24 significant bits (exponent rebias
// and a shift of the encoding), l is the remaining 29 bits scaled by
// 2^(E - 52) (down to |x| ~ 2^-100).  Values below 2^-126 flush to zero;
// values beyond the float
// range become +-inf (neither occurs for amplitudes, gate entries or
// coefficients of a normalised state).
DF_HD df::df(double x) {
  const uint64_t b = df_d2u(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;
  if (e == 0 || fe <= 0) {
    h = df_u2f(sign);
    l = 0.f;
    return;
  }
  if (fe >= 255) {
    h = df_u2f(sign | 0x7F800000u);
    l = 0.f;
    return;
  }
  const float hh = df_u2f(sign | ((uint32_t)fe << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
  const uint32_t r = (uint32_t)(b & 0x1FFFFFFFu);
  // r * 2^(E - 52) as (r * 2^-26) * 2^(E - 26): two exact power-of-two scalings,
  // valid for E >= -100 (smaller magnitudes keep only h)
  const int se = fe - 26;  // biased exponent of 2^(E - 26)
  float ll = 0.f;
  if (r != 0 && se >= 1) {
    ll = (df_u32_to_f(r) * df_u2f((uint32_t)(127 - 26) << 23)) * df_u2f((uint32_t)se << 23);
    if (sign) ll = -ll;
  }
  const df n = df_fast_two_sum(hh, ll);
  h = n.h;
  l = n.l;
}

// Lean conversions for single-op streams, where conversion dominates the
// work.  Split: the top 24 significant bits by truncation, the next 29 rounded
// to a float, then one Fast2Sum; magnitudes below 2^-126 become zero and the
// low part is dropped below 2^-74 (never the case that matters for an
// amplitude of a normalised state).  Join: each float re-encoded as a double
// with integer operations (subnormal floats flush to zero), then one FP64
// addition.
DF_HD df df_split_fast(double x) {
  const uint64_t b = df_d2u(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int fe = (int)((b >> 52) & 0x7FF) - 896;  // float biased exponent of x
  const float h = df_u2f(fe > 0 ? (sign | ((uint32_t)fe << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu)) : sign);
  // remainder r * 2^(E - 52): float biased exponent of the scale is fe - 52
  float l = df_u32_to_f((uint32_t)b & 0x1FFFFFFFu) * df_u2f((uint32_t)(fe > 52 ? fe - 52 : 1) << 23);
  l = df_u2f(df_f2u(l) | sign);
  return df_fast_two_sum(h, fe > 52 ? l : 0.f);
}

DF_HD double df_f2d_normal(float f) {
  const uint32_t u = df_f2u(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0) return df_u2d(sign);
  return df_u2d(sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29));
}

DF_HD double df_join_fast(df v) { return df_f2d_normal(v.h) + df_f2d_normal(v.l); }

struct __align__(16) dfc {
  df x, y;  // real, imaginary
};

}  // namespace sv
