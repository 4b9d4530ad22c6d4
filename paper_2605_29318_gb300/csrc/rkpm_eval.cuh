// Device routines of the corrected RKPM shape functions at one evaluation point
// (internal; shared by the cloud's own shape functions, the two-set
// construction and the skinning weights at query points).  Sec. 3.2,
// Eqs. 7, 9-10; the basis written about the evaluation point (see shape.cu).
#pragma once

#include "dfloat.cuh"
#include "ff_internal.cuh"

namespace ff {
namespace rkpm {

template <class C>
__device__ __forceinline__ void bspline(C q, C& w, C& dwq) {
  if (q <= C(0.5)) {
    w = C(2.0 / 3.0) - C(4) * q * q + C(4) * q * q * q;
    dwq = C(-8) + C(12) * q;
  } else if (q <= C(1)) {
    C t = C(1) - q;
    w = C(4.0 / 3.0) * t * t * t;
    dwq = C(-4) * t * t / q;
  } else {
    w = C(0);
    dwq = C(0);
  }
}

// Raw kernels varphi_k as functors: from the squared distance d2 = |X - p_k|^2
// they give w = varphi_k(X) and gs with grad_X varphi_k = gs (p_k - X).
// BSpline: the cubic B-spline of radius a_k = p.w (the nodal discretisation).
struct BSpline {
  template <class C>
  __device__ __forceinline__ void eval(int, float4 p, C d2, C& w, C& gs) const {
    const C ak = (C)p.w;
    C dwq;
    bspline<C>(sqrt(d2) / ak, w, dwq);
    gs = -dwq / (ak * ak);
  }
};

__device__ __forceinline__ float gauss_exp(float x) { return expf(x); }
__device__ __forceinline__ double gauss_exp(double x) { return exp(x); }
__device__ __forceinline__ dfloat gauss_exp(dfloat x) { return df_exp(x); }

template <class C>
__device__ __forceinline__ C from_f64(double x) { return (C)x; }
template <>
__device__ __forceinline__ dfloat from_f64<dfloat>(double x) { return dfloat(x); }

// Gauss: exp(-|X - p_k|^2 / r_k^2) (Sec. 3.2) with the FP64 radii r_k of the
// two-set construction; grad_X = (2 w / r_k^2)(p_k - X).  In double-float the
// exponential is df_exp (reduction by ln 2 and a Taylor polynomial on the FP32
// pipes).
struct Gauss {
  const double* rad;
  template <class C>
  __device__ __forceinline__ void eval(int k, float4, C d2, C& w, C& gs) const {
    const C rk = from_f64<C>(rad[k]);
    const C rk2 = rk * rk;
    w = gauss_exp(-(d2 / rk2));
    gs = C(2) * w / rk2;
  }
};

template <class C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// symmetric 4x4 packed upper triangle: (0,0)(0,1)(0,2)(0,3)(1,1)(1,2)(1,3)(2,2)(2,3)(3,3)
__device__ __forceinline__ int sidx(int r, int c) {
  if (r > c) { int t = r; r = c; c = t; }
  const int base[4] = {0, 4, 7, 9};
  return base[r] + (c - r);
}

// Cholesky of a 4x4 SPD matrix (packed), returns false if a pivot is not
// positive relative to the trace.  L stored dense row-major lower.
template <class C>
__device__ __forceinline__ bool chol4(const C* m, C* L, C rel_tol) {
  C tr = m[0] + m[4] + m[7] + m[9];
  for (int j = 0; j < 4; ++j) {
    C s = m[sidx(j, j)];
    for (int p = 0; p < j; ++p) s -= L[j * 4 + p] * L[j * 4 + p];
    if (!(s > rel_tol * tr)) return false;
    C d = sqrt(s);
    L[j * 4 + j] = d;
    for (int i = j + 1; i < 4; ++i) {
      C t = m[sidx(i, j)];
      for (int p = 0; p < j; ++p) t -= L[i * 4 + p] * L[j * 4 + p];
      L[i * 4 + j] = t / d;
    }
    for (int i = 0; i < j; ++i) L[i * 4 + j] = C(0);
  }
  return true;
}

template <class C>
__device__ __forceinline__ void chol4_solve(const C* L, const C* b, C* x) {
  C y[4];
  for (int i = 0; i < 4; ++i) {
    C t = b[i];
    for (int p = 0; p < i; ++p) t -= L[i * 4 + p] * y[p];
    y[i] = t / L[i * 4 + i];
  }
  for (int i = 3; i >= 0; --i) {
    C t = y[i];
    for (int p = i + 1; p < 4; ++p) t -= L[p * 4 + i] * x[p];
    x[i] = t / L[i * 4 + i];
  }
}

// Evaluate one row in compute precision C, writing outputs of precision T.
// Returns 0 ok, 1 singular, 2 ill-conditioned (only when check_cond).
template <class C, class T, class Kern = BSpline>
__device__ int shape_row(const float4* __restrict__ pos, long long s, long long e,
                         const int* __restrict__ idx, float4 Xi, T* __restrict__ phi,
                         T* __restrict__ dphi, long long n1, double cond_limit, bool check_cond,
                         const Kern& kern = Kern()) {
  const int lane = threadIdx.x & 31;
  const C xi = (C)Xi.x, yi = (C)Xi.y, zi = (C)Xi.z, si = (C)Xi.w;
  const C isi = C(1) / si;  // the basis scale's reciprocal, once per row
  C m[10], dm[3][10];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    m[q] = C(0);
    dm[0][q] = dm[1][q] = dm[2][q] = C(0);
  }
  // the raw kernel of a lane's first kCache entries is kept for the second
  // pass (the Gaussian's exponential is the costliest step of a pair)
  constexpr int kCache = 4;
  C cw[kCache], cg[kCache];
  int q = 0;
  for (long long t = s + lane; t < e; t += 32, ++q) {
    const int k = idx[t];
    float4 p = pos[k];
    C r0 = (C)p.x - xi, r1 = (C)p.y - yi, r2 = (C)p.z - zi;
    C w, gs;  // grad_X varphi = gs * r
    kern.template eval<C>(k, p, r0 * r0 + r1 * r1 + r2 * r2, w, gs);
#pragma unroll
    for (int u = 0; u < kCache; ++u)
      if (q == u) {
        cw[u] = w;
        cg[u] = gs;
      }
    C P[4] = {C(1), r0 * isi, r1 * isi, r2 * isi};
    C g[3] = {gs * r0, gs * r1, gs * r2};
    int o = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b, ++o) {
        const C pp = P[a] * P[b];
        mac(m[o], w, pp);  // fused (unnormalised in double-float), finished below
        mac(dm[0][o], g[0], pp);
        mac(dm[1][o], g[1], pp);
        mac(dm[2][o], g[2], pp);
      }
  }
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    m[q] = warp_sum(finish(m[q]));
    dm[0][q] = warp_sum(finish(dm[0][q]));
    dm[1][q] = warp_sum(finish(dm[1][q]));
    dm[2][q] = warp_sum(finish(dm[2][q]));
  }
  C L[16];
  if (!chol4<C>(m, L, C(1e-12))) return 1;
  if (check_cond) {
    // 1-norm condition number from the explicit inverse
    C inv_norm = C(0), m_norm = C(0);
    for (int col = 0; col < 4; ++col) {
      C ecol[4] = {C(0), C(0), C(0), C(0)}, x[4];
      ecol[col] = C(1);
      chol4_solve<C>(L, ecol, x);
      C a1 = C(0), a2 = C(0);
      for (int r = 0; r < 4; ++r) {
        a1 += fabs(x[r]);
        a2 += fabs(m[sidx(r, col)]);
      }
      inv_norm = fmax(inv_norm, a1);
      m_norm = fmax(m_norm, a2);
    }
    if ((double)(inv_norm * m_norm) > cond_limit) return 2;
  }
  C Cv[4], dC[3][4];
  {
    C e0[4] = {C(1), C(0), C(0), C(0)};
    chol4_solve<C>(L, e0, Cv);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    C rhs[4];
    for (int r = 0; r < 4; ++r) {
      C t = C(0);
      for (int cc = 0; cc < 4; ++cc) t += dm[d][sidx(r, cc)] * Cv[cc];
      rhs[r] = -t;
    }
    rhs[1 + d] += isi;
    chol4_solve<C>(L, rhs, dC[d]);
  }
  q = 0;
  for (long long t = s + lane; t < e; t += 32, ++q) {
    const int k = idx[t];
    float4 p = pos[k];
    C r0 = (C)p.x - xi, r1 = (C)p.y - yi, r2 = (C)p.z - zi;
    C w, gs;
    if (q < kCache) {
#pragma unroll
      for (int u = 0; u < kCache; ++u)
        if (q == u) {
          w = cw[u];
          gs = cg[u];
        }
    } else {
      kern.template eval<C>(k, p, r0 * r0 + r1 * r1 + r2 * r2, w, gs);
    }
    C P[4] = {C(1), r0 * isi, r1 * isi, r2 * isi};
    C PC = Cv[0];
#pragma unroll
    for (int a = 1; a < 4; ++a) mac(PC, P[a], Cv[a]);
    PC = finish(PC);
    phi[t] = (T)(w * PC);
    C g[3] = {gs * r0, gs * r1, gs * r2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      C PdC = dC[d][0];
#pragma unroll
      for (int a = 1; a < 4; ++a) mac(PdC, P[a], dC[d][a]);
      PdC = finish(PdC);
      dphi[d * n1 + t] = (T)(g[d] * PC + w * PdC);
    }
  }
  return 0;
}

}  // namespace rkpm
}  // namespace ff
