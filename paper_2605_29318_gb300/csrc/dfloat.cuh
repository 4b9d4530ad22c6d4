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
  __host__ __device__ explicit dfloat(float a) : h(a), l(0.f) {}
  __host__ __device__ explicit dfloat(int a) : h((float)a), l(0.f) {}
  __host__ __device__ explicit dfloat(double d) {
    h = (float)d;
    l = (float)(d - (double)h);
  }
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

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.h, -a.l); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = df_add(a, b); }
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.h == b.h && a.l == b.l; }

// Generic multiply-accumulate and finishing step for the block kernels:
// FMA for float and double, df_mac (unnormalised) for dfloat.
__device__ __forceinline__ void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(dfloat& acc, dfloat a, dfloat b) { df_mac(acc, a, b); }
__device__ __forceinline__ float finish(float a) { return a; }
__device__ __forceinline__ double finish(double a) { return a; }
__device__ __forceinline__ dfloat finish(dfloat a) { return df_norm(a); }

}  // namespace ff

// shuffles of a dfloat move both halves
__device__ __forceinline__ ff::dfloat __shfl_down_sync(unsigned mask, ff::dfloat v, unsigned d) {
  return ff::dfloat(__shfl_down_sync(mask, v.h, d), __shfl_down_sync(mask, v.l, d));
}
__device__ __forceinline__ ff::dfloat __shfl_sync(unsigned mask, ff::dfloat v, int src) {
  return ff::dfloat(__shfl_sync(mask, v.h, src), __shfl_sync(mask, v.l, src));
}
