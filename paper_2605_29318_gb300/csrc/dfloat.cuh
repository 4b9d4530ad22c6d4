// Double-float arithmetic on the FP32 pipes (internal).
//
// A dfloat is the unevaluated sum h + l of two FP32 numbers; normalised,
// |l| <= ulp(h) / 2, which carries about 48 significant bits at the FP32
// exponent range.  On GB300 an FP64 FMA costs about 64 FP32 ones, while a
// double-float multiply-add below costs 12 FP32 operations, so block products
// that need more than FP32 but much less than FP64's 2^-53 run several times
// faster this way.
//
// Built from the error-free transformations
//   two_sum(a, b)       s + e = a + b exactly, any a, b       (Knuth, TAOCP 4.2.2)
//   fast_two_sum(a, b)  s + e = a + b exactly for |a| >= |b|  (Dekker 1971)
//   two_prod(a, b)      p + e = a * b exactly, by one FMA
// The __fadd_rn / __fmul_rn / __fmaf_rn intrinsics keep the compiler from
// contracting or reordering them.
#pragma once

#include <cuda_runtime.h>

namespace ff {

struct __align__(8) dfloat {
  float h, l;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float a, float b) : h(a), l(b) {}
  __host__ __device__ constexpr explicit dfloat(float a) : h(a), l(0.f) {}
  __host__ __device__ constexpr explicit dfloat(int a) : h((float)a), l(0.f) {}
  __host__ __device__ constexpr explicit dfloat(unsigned a)
      : h((float)a), l((float)((double)a - (double)(float)a)) {}
  // exact split of a double into a rounded head and its remainder
  __host__ __device__ constexpr explicit dfloat(double d)
      : h((float)d), l((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
  __host__ __device__ explicit operator float() const { return h + l; }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// normalised h + l (no magnitude assumption)
__device__ __forceinline__ dfloat df_norm(dfloat x) {
  dfloat r;
  two_sum(x.h, x.l, r.h, r.l);
  return r;
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  dfloat r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  dfloat r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}

// acc += a * b with an accumulator that is left unnormalised: the rounding
// errors of the running sum collect in acc.l (normalise once at the end)
__device__ __forceinline__ void df_mac(dfloat& acc, dfloat a, dfloat b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// acc += a (unnormalised, as df_mac)
__device__ __forceinline__ void df_acc(dfloat& acc, dfloat a) {
  float s, t;
  two_sum(acc.h, a.h, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, a.l));
}

// a / b: the FP32 quotient of the heads, corrected twice from the exact
// remainder a - q b
__device__ __forceinline__ dfloat df_div(dfloat a, dfloat b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const dfloat b1 = df_mul(b, dfloat(q1));
  dfloat r = df_add(a, dfloat(-b1.h, -b1.l));
  const float q2 = __fdiv_rn(r.h, b.h);
  const dfloat b2 = df_mul(b, dfloat(q2));
  r = df_add(r, dfloat(-b2.h, -b2.l));
  const float q3 = __fdiv_rn(r.h, b.h);
  dfloat q;
  fast_two_sum(q1, q2, q.h, q.l);
  return df_add(q, dfloat(q3));
}

// sqrt(a), a >= 0: the FP32 root y of the head, then y + (a - y^2) / (2 y)
__device__ __forceinline__ dfloat df_sqrt(dfloat a) {
  if (!(a.h > 0.f)) return dfloat(0.f, 0.f);
  const float y = __fsqrt_rn(a.h);
  const float p = __fmul_rn(y, y);
  const dfloat e = df_add(a, dfloat(-p, -__fmaf_rn(y, y, -p)));
  dfloat r;
  fast_two_sum(y, __fdiv_rn(e.h, __fmul_rn(2.f, y)), r.h, r.l);
  return r;
}

// exp(x) of a double-float x, |x| < 80.  Cody and Waite's reduction:
// n = nearest integer to x / ln 2, f = x - n ln 2 with ln 2 carried as a
// double-float (|f| <= ln 2 / 2 up to rounding), then the Taylor polynomial of
// e^f to degree 13 by Horner's rule (truncation below (ln2/2)^14 / 14! < 2e-17),
// scaled by 2^n exactly.  About 2^-45 relative: the error of n ln 2 dominates.
__device__ __forceinline__ dfloat df_exp(dfloat x) {
  const float n = rintf(__fmul_rn(x.h, 1.44269504f));
  const dfloat ln2(0.6931471805599453);
  const dfloat nl = df_mul(dfloat(n), ln2);
  const dfloat f = df_add(x, dfloat(-nl.h, -nl.l));
  constexpr double kInvFact[14] = {1.0,
                                   1.0,
                                   1.0 / 2,
                                   1.0 / 6,
                                   1.0 / 24,
                                   1.0 / 120,
                                   1.0 / 720,
                                   1.0 / 5040,
                                   1.0 / 40320,
                                   1.0 / 362880,
                                   1.0 / 3628800,
                                   1.0 / 39916800,
                                   1.0 / 479001600,
                                   1.0 / 6227020800.0};
  dfloat p(kInvFact[13]);
#pragma unroll
  for (int k = 12; k >= 0; --k) p = df_add(df_mul(p, f), dfloat(kInvFact[k]));
  const int e = (int)n;
  return dfloat(ldexpf(p.h, e), ldexpf(p.l, e));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.h, -a.l); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) { return df_div(a, b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = df_add(a, b); }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = df_add(a, -b); }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = df_mul(a, b); }
// comparisons of normalised values: heads first, then tails
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.h == b.h && a.l == b.l; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return !(a == b); }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) {
  return a.h < b.h || (a.h == b.h && a.l < b.l);
}
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }
__device__ __forceinline__ bool operator<=(dfloat a, dfloat b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dfloat a, dfloat b) { return !(a < b); }

// Generic multiply-accumulate and finishing step for the block kernels:
// FMA for float and double, df_mac (unnormalised) for dfloat.
__device__ __forceinline__ void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(dfloat& acc, dfloat a, dfloat b) { df_mac(acc, a, b); }
__device__ __forceinline__ float finish(float a) { return a; }
__device__ __forceinline__ double finish(double a) { return a; }
__device__ __forceinline__ dfloat finish(dfloat a) { return df_norm(a); }

}  // namespace ff

// the math functions the dense Rayleigh-Ritz kernels call, for double-float
// arguments (global overloads beside CUDA's, so unqualified calls resolve)
__device__ __forceinline__ ff::dfloat sqrt(ff::dfloat a) { return ff::df_sqrt(a); }
__device__ __forceinline__ ff::dfloat fabs(ff::dfloat a) { return a.h < 0.f ? -a : a; }
__device__ __forceinline__ ff::dfloat fmax(ff::dfloat a, ff::dfloat b) { return a < b ? b : a; }
__device__ __forceinline__ ff::dfloat fmin(ff::dfloat a, ff::dfloat b) { return b < a ? b : a; }
__device__ __forceinline__ ff::dfloat fma(ff::dfloat a, ff::dfloat b, ff::dfloat c) {
  return ff::df_add(ff::df_mul(a, b), c);
}
__device__ __forceinline__ bool isfinite(ff::dfloat a) { return isfinite(a.h) && isfinite(a.l); }

// shuffles of a dfloat move both halves
__device__ __forceinline__ ff::dfloat __shfl_down_sync(unsigned mask, ff::dfloat v, unsigned d) {
  return ff::dfloat(__shfl_down_sync(mask, v.h, d), __shfl_down_sync(mask, v.l, d));
}
__device__ __forceinline__ ff::dfloat __shfl_sync(unsigned mask, ff::dfloat v, int src) {
  return ff::dfloat(__shfl_sync(mask, v.h, src), __shfl_sync(mask, v.l, src));
}
__device__ __forceinline__ ff::dfloat __shfl_xor_sync(unsigned mask, ff::dfloat v, int lm) {
  return ff::dfloat(__shfl_xor_sync(mask, v.h, lm), __shfl_xor_sync(mask, v.l, lm));
}
