// Block eigensolver for the k lowest pairs of H_w c = lambda M c (Sec. 3.2,
// Eq. 15; Supp. Sec. B "Eigenanalysis" solves the same problem with LOBPCG).
//
// Locally optimal block preconditioned conjugate gradient with an explicit
// M-orthonormal basis [X | W | P]:
//   * the constant mode c0 = 1 / sqrt(1^T M 1) is set analytically (it is an
//     exact null vector of the stored H_w) and deflated from every block;
//   * W = T R, R = H X - M X Theta, with T a Chebyshev polynomial in D^-1 H
//     (D = diag H) approximating H^+ on [beta / ratio, beta] -- FP32 and
//     free of reductions; beta from power iteration capped by Gershgorin;
//   * W is M-projected against X, P and c0 with the blocks M X, M P kept
//     from earlier products, then (H W, M W) comes from one fused pass;
//   * Rayleigh-Ritz on the Gram matrices of the basis (dense.cu) returns the
//     coefficients of the new X and of the new momentum P (already
//     M-orthonormal and M-orthogonal to X), and one block update forms
//     X, P, H X, H P, M X, M P from the old panels;
//   * columns whose relative residual meets tol stop contributing to W.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

#include "linalg.cuh"

namespace ff {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

template <class T>
__global__ void k_random_block(T* X, int ld, long long n, int m, unsigned long long seed,
                               const int* perm) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  long long r = t / m;
  int c = (int)(t % m);
  unsigned long long h = mix64(seed * 0x100000001b3ULL + (unsigned long long)perm[r] * 1024ULL + c);
  double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
  X[r * ld + c] = (T)(2.0 * u - 1.0);
}

template <class T>
__global__ void k_gather_block(const T* __restrict__ X0, long long n, int m,
                               const int* __restrict__ perm, T* __restrict__ X, int ld) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  long long r = t / m;
  int c = (int)(t % m);
  X[r * ld + c] = X0[(long long)c * n + perm[r]];
}

template <class T, class To = T>
__global__ void k_scatter_block(const T* __restrict__ X, int ld, long long n, int m,
                                const int* __restrict__ perm, To* __restrict__ out, long long ldo,
                                int col0) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  long long r = t / m;
  int c = (int)(t % m);
  out[(long long)(c + col0) * ldo + perm[r]] = (To)X[r * ld + c];
}

template <class T>
__global__ void k_fill(T* x, long long n, T v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

template <class T>
__global__ void k_scale(T* x, long long n, const double* s, int mode) {
  // mode 0: x *= 1/sqrt(s[0]);  mode 1: x *= s[0]
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)((double)x[i] * (mode == 0 ? 1.0 / sqrt(s[0]) : s[0]));
}

template <class T>
__global__ void k_d2t(const double* in, T* out, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (T)in[i];
}

// Per-column statistics of the current block, from the recomputed products:
// x.Hx, x.Mx, Hx.Hx, Hx.Mx, Mx.Mx (FP64 accumulation of exact products).
// Partials per row chunk, then a fixed-order reduction (deterministic).
template <class T>
__global__ void k_colstats_partial(const T* __restrict__ X, const T* __restrict__ HX,
                                   const T* __restrict__ MX, int ld, long long n, int m,
                                   long long rows_per_block, double* __restrict__ part) {
  __shared__ double sred[8][5][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * rows_per_block;
  const long long r1 = min(n, r0 + rows_per_block);
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int col = c0 + lane;
    double a[5] = {0, 0, 0, 0, 0};
    if constexpr (std::is_same_v<T, float>) {
      // FP32 blocks: each product exact as a double-float (FMA TwoProduct),
      // summed in double-float -- FP64-grade sums without FP64 arithmetic
      dfloat s5[5] = {dfloat(0), dfloat(0), dfloat(0), dfloat(0), dfloat(0)};
      auto tp = [](float u, float v) {
        const float p = __fmul_rn(u, v);
        return dfloat(p, __fmaf_rn(u, v, -p));
      };
      if (col < m)
        for (long long r = r0 + w; r < r1; r += 8) {
          const float x = X[r * ld + col], h = HX[r * ld + col], mm = MX[r * ld + col];
          df_acc(s5[0], tp(x, h));
          df_acc(s5[1], tp(x, mm));
          df_acc(s5[2], tp(h, h));
          df_acc(s5[3], tp(h, mm));
          df_acc(s5[4], tp(mm, mm));
        }
      for (int q = 0; q < 5; ++q) a[q] = (double)s5[q];
    } else {
      if (col < m)
        for (long long r = r0 + w; r < r1; r += 8) {
          const double x = (double)X[r * ld + col], h = (double)HX[r * ld + col],
                       mm = (double)MX[r * ld + col];
          a[0] += x * h;
          a[1] += x * mm;
          a[2] += h * h;
          a[3] += h * mm;
          a[4] += mm * mm;
        }
    }
    for (int q = 0; q < 5; ++q) sred[w][q][lane] = a[q];
    __syncthreads();
    if (w == 0 && col < m)
      for (int q = 0; q < 5; ++q) {
        double t = 0;
        for (int ww = 0; ww < 8; ++ww) t += sred[ww][q][lane];
        part[((long long)blockIdx.x * 5 + q) * m + col] = t;
      }
    __syncthreads();
  }
}

// The same statistics for double-float blocks with the residual norm taken
// directly: x.Hx and x.Mx in double-float (slots 0, 1), ||Hx - sigma Mx||^2
// with sigma the Ritz values of the last (FP64) Rayleigh-Ritz step (slot 2;
// the residual vector in double-float, its squares summed in FP32 within a
// thread) and ||Mx||^2 (slot 4).  Expanding the norm would need the three sums
// to ~1e-13 relative for a 1e-6 residual, beyond double-float sums over n
// rows; sigma differs from the Rayleigh quotient of the stored block by ~1e-9
// relative, which moves the residual norm by as much.  (FP32 Ritz values are
// far less accurate for the small modes, so FP32 blocks keep the expanded
// form, with exact products and double-float sums.)
template <class T>
__global__ void k_colstats_partial_direct(const T* __restrict__ X, const T* __restrict__ HX,
                                          const T* __restrict__ MX, int ld, long long n, int m,
                                          long long rows_per_block,
                                          const double* __restrict__ sigma,
                                          double* __restrict__ part) {
  __shared__ double sred[8][5][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * rows_per_block;
  const long long r1 = min(n, r0 + rows_per_block);
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int col = c0 + lane;
    T xh(0), xm(0);
    float rr = 0.f, mm2 = 0.f;
    if (col < m) {
      const T ns(-sigma[col]);
      for (long long r = r0 + w; r < r1; r += 8) {
        const T x = X[r * ld + col], h = HX[r * ld + col], mm = MX[r * ld + col];
        df_mac(xh, x, h);
        df_mac(xm, x, mm);
        dfloat res = h;
        df_mac(res, ns, mm);
        const float rf = (float)df_norm(res);
        const float mf = (float)mm;
        rr = fmaf(rf, rf, rr);
        mm2 = fmaf(mf, mf, mm2);
      }
    }
    sred[w][0][lane] = (double)xh;
    sred[w][1][lane] = (double)xm;
    sred[w][2][lane] = rr;
    sred[w][3][lane] = 0.0;
    sred[w][4][lane] = mm2;
    __syncthreads();
    if (w == 0 && col < m)
      for (int q = 0; q < 5; ++q) {
        double t = 0;
        for (int ww = 0; ww < 8; ++ww) t += sred[ww][q][lane];
        part[((long long)blockIdx.x * 5 + q) * m + col] = t;
      }
    __syncthreads();
  }
}

// theta = x.Hx / x.Mx (Rayleigh quotient); ||Hx - theta Mx||^2 expanded in
// FP64, or (direct) the norm summed by the partial kernel.
// One block per column, fixed-order tree reduction over the partials.
__global__ void k_colstats_final(const double* __restrict__ part, int blocks, int m,
                                 double* __restrict__ theta, double* __restrict__ stats,
                                 int direct) {
  __shared__ double sh[5][128];
  const int col = blockIdx.x;
  double a[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < blocks; b += 128)
    for (int q = 0; q < 5; ++q) a[q] += part[((long long)b * 5 + q) * m + col];
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = 64; w; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double th = sh[0][0] / sh[1][0];
    const double r2 =
        direct ? sh[2][0] : fmax(sh[2][0] - 2.0 * th * sh[3][0] + th * th * sh[4][0], 0.0);
    theta[col] = th;
    stats[col] = th;
    stats[m + col] = r2;
    stats[2 * m + col] = sh[4][0];
  }
}

// Chebyshev start: b = active * (HX - MX theta) / diag(H); res = b; d = b / theta_c; x = d.
// The iteration's arrays are n x mc (mc >= m): columns m..mc-1 are zero.
template <class T>
__global__ void k_cheb_init(const T* __restrict__ HX, const T* __restrict__ MX, int ld,
                            const double* __restrict__ theta, const int* __restrict__ active,
                            const float* __restrict__ hdiag, long long n, int m, int mc,
                            float* __restrict__ res, float* __restrict__ d, float* __restrict__ x,
                            float inv_tc, __nv_bfloat16* __restrict__ d16) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * mc) return;
  long long r = t / mc;
  int c = (int)(t % mc);
  float b = 0.f;
  if (c < m && active[c]) {
    if constexpr (std::is_same_v<T, dfloat>) {  // the residual in double-float
      dfloat rr = HX[r * ld + c];
      df_mac(rr, dfloat(-theta[c]), MX[r * ld + c]);
      b = (float)df_norm(rr) / hdiag[r];
    } else if constexpr (std::is_same_v<T, float>) {  // FP32 blocks: in FP32
      b = fmaf(-(float)theta[c], MX[r * ld + c], HX[r * ld + c]) / hdiag[r];
    } else {
      double rr = (double)HX[r * ld + c] - theta[c] * (double)MX[r * ld + c];
      b = (float)(rr / (double)hdiag[r]);
    }
  }
  res[t] = b;
  if (d16) {  // BF16 directions: x starts from the rounded one
    const __nv_bfloat16 q = __float2bfloat16(b * inv_tc);
    d16[t] = q;
    x[t] = __bfloat162float(q);
  } else {
    d[t] = b * inv_tc;
    x[t] = b * inv_tc;
  }
}

// W (n x m of a panel) = x (n x m of a dense array with row stride ldx)
template <class T>
__global__ void k_cast_block(const float* __restrict__ x, int ldx, long long n, int m,
                             T* __restrict__ W, int ld) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  long long r = t / m;
  int c = (int)(t % m);
  W[r * ld + c] = (T)x[r * ldx + c];
}

// Packed Chebyshev start: the same b as k_cheb_init for the columns still
// above tol only, column q of the n x w arrays taken from block column cmap[q]
// (cmap[q] < 0: a padding column, zero).
template <class T>
__global__ void k_cheb_init_packed(const T* __restrict__ HX, const T* __restrict__ MX, int ld,
                                   const double* __restrict__ theta, const int* __restrict__ cmap,
                                   const float* __restrict__ hdiag, long long n, int w,
                                   float* __restrict__ res, float* __restrict__ x, float inv_tc,
                                   __nv_bfloat16* __restrict__ d16) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * w) return;
  long long r = t / w;
  const int c = cmap[(int)(t % w)];
  float b = 0.f;
  if (c >= 0) {
    if constexpr (std::is_same_v<T, dfloat>) {
      dfloat rr = HX[r * ld + c];
      df_mac(rr, dfloat(-theta[c]), MX[r * ld + c]);
      b = (float)df_norm(rr) / hdiag[r];
    } else if constexpr (std::is_same_v<T, float>) {
      b = fmaf(-(float)theta[c], MX[r * ld + c], HX[r * ld + c]) / hdiag[r];
    } else {
      double rr = (double)HX[r * ld + c] - theta[c] * (double)MX[r * ld + c];
      b = (float)(rr / (double)hdiag[r]);
    }
  }
  res[t] = b;
  const __nv_bfloat16 q = __float2bfloat16(b * inv_tc);
  d16[t] = q;
  x[t] = __bfloat162float(q);
}

// W (n x m of a panel) from the packed n x w result: block column c takes
// packed column cinv[c], or zero when it was not preconditioned
template <class T>
__global__ void k_cast_packed(const float* __restrict__ x, int w, const int* __restrict__ cinv,
                              long long n, int m, T* __restrict__ W, int ld) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * m) return;
  long long r = t / m;
  int c = (int)(t % m);
  const int q = cinv[c];
  W[r * ld + c] = q >= 0 ? (T)x[r * w + q] : T(0);
}

// Soft locking of the momentum: the P coefficients (columns nb..2nb-1 of the
// ns x 2nb coefficient matrix YZ) of modes that met tol this iteration are
// zeroed, so their next P column is exactly zero and leaves the basis.  A
// converged mode's momentum is tiny; normalised, it would carry the rounding
// of the products it is formed from into the Gram matrices.
template <class T>
__global__ void k_lock_momentum(T* __restrict__ YZ, int ns, int nb,
                                const int* __restrict__ active) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * nb) return;
  const int r = t / nb, j = t % nb;
  if (!active[j]) YZ[(size_t)r * 2 * nb + nb + j] = T(0);
}

// Soft locking of the basis: the Gram matrices restricted to the kept
// columns (out[i][j] = in[keep[i]][keep[j]], ns x ns -> m x m) ...
__global__ void k_gather_sq(const double* __restrict__ in, int ns, const int* __restrict__ keep,
                            int m, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  const int i = t / m, j = t % m;
  out[t] = in[(size_t)keep[i] * ns + keep[j]];
}

// ... and the Rayleigh-Ritz coefficients (m x q rows) placed back on the full
// basis (ns x q rows; the rows of the columns left out are zeroed first)
template <class T>
__global__ void k_place_rows(const T* __restrict__ in, int m, int q, const int* __restrict__ keep,
                             T* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * q) return;
  const int i = t / q, j = t % q;
  out[(size_t)keep[i] * q + j] = in[t];
}

__global__ void k_round_block(const double* __restrict__ x, float* __restrict__ y, long long m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) y[t] = (float)x[t];
}

__global__ void k_gershgorin(const long long* __restrict__ ptr, const float* __restrict__ hv,
                             const float* __restrict__ hdiag, long long n, unsigned int* out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float g = 0.f;
  if (k < n) {
    float s = 0.f;
    for (long long e = ptr[k]; e < ptr[k + 1]; ++e) s += fabsf(hv[e]);
    g = s / fabsf(hdiag[k]);
  }
  for (int o = 16; o; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(g));
}

}  // namespace

template <class T>
struct Solver {
  ff_ctx* c;
  cudaStream_t st;
  const T* aval;  // interleaved (H, M) of this phase's precision
  long long n;
  int nb, kw, ld;
  int mc;         // columns of the Chebyshev iteration's arrays (nb, or nb
                  // rounded up to 8 for the BF16 / tensor-core steps)
  bool fp64;      // FP64 blocks
  bool rr64;      // FP64 Rayleigh-Ritz
  T *S[2], *HS[2], *MS[2];
  T *c0, *Mc0;
  float *cres, *cd0, *cd1, *cx;
  __nv_bfloat16 *cb0, *cb1;  // BF16 direction vectors of the preconditioner
  double *Ag, *Bg, *G1, *theta_d, *norms_d;
  T *Gt, *YZ;
  int *dropped_d, *active_d;
  double *Ac, *Bc;  // Gram matrices restricted to the kept columns (soft locking)
  T* YZc;           // their Rayleigh-Ritz coefficients
  int* keep_d;      // kept columns
  double* h_pin;  // pinned: theta | ||R||^2 | ||MX||^2 (3 nb)
  int spmm_calls = 0, spmv_calls = 0;

  T* col(T* panel, int c0_) { return panel + c0_; }

  void alloc() {
    ld = ((3 * nb + 3) / 4) * 4;
    for (int b = 0; b < 2; ++b) {
      S[b] = reinterpret_cast<T*>(c->ws[0 + b].ensure(sizeof(T) * n * ld));
      HS[b] = reinterpret_cast<T*>(c->ws[2 + b].ensure(sizeof(T) * n * ld));
      MS[b] = reinterpret_cast<T*>(c->ws[4 + b].ensure(sizeof(T) * n * ld));
    }
    c0 = reinterpret_cast<T*>(c->ws[6].ensure(sizeof(T) * n));
    Mc0 = reinterpret_cast<T*>(c->ws[7].ensure(sizeof(T) * n));
    const int mw = std::max({nb, mc, 4});
    cres = reinterpret_cast<float*>(c->ws[8].ensure(sizeof(float) * n * mw));
    cd0 = reinterpret_cast<float*>(c->ws[9].ensure(sizeof(float) * n * mw));
    cd1 = reinterpret_cast<float*>(c->ws[10].ensure(sizeof(float) * n * mw));
    cb0 = reinterpret_cast<__nv_bfloat16*>(c->ws[24].ensure(sizeof(__nv_bfloat16) * n * mw + 16));
    cb1 = reinterpret_cast<__nv_bfloat16*>(c->ws[25].ensure(sizeof(__nv_bfloat16) * n * mw + 16));
    cx = reinterpret_cast<float*>(c->ws[11].ensure(sizeof(float) * n * mw));
    const int ns = 3 * nb;
    Ag = reinterpret_cast<double*>(c->ws[12].ensure(sizeof(double) * ns * ns));
    Bg = reinterpret_cast<double*>(c->ws[13].ensure(sizeof(double) * ns * ns));
    G1 = reinterpret_cast<double*>(c->ws[14].ensure(sizeof(double) * std::max((2 * nb + 2) * nb, 64)));
    theta_d = reinterpret_cast<double*>(c->ws[15].ensure(sizeof(double) * (nb + 8)));
    norms_d = reinterpret_cast<double*>(c->ws[16].ensure(sizeof(double) * 3 * nb));
    Gt = reinterpret_cast<T*>(c->ws[17].ensure(sizeof(T) * (2 * nb + 2) * nb));
    YZ = reinterpret_cast<T*>(c->ws[18].ensure(sizeof(T) * ns * 2 * nb));
    dropped_d = reinterpret_cast<int*>(c->ws[19].ensure(sizeof(int) * 4));
    // active flags, then the packing maps of the preconditioner: cmap (mc), cinv (nb)
    active_d = reinterpret_cast<int*>(c->ws[20].ensure(sizeof(int) * (2 * nb + mc + 8)));
    h_pin = reinterpret_cast<double*>(c->hflags) + 16;  // pinned scratch after the flags
    Ac = reinterpret_cast<double*>(c->ws[26].ensure(sizeof(double) * 2 * ns * ns));
    Bc = Ac + (size_t)ns * ns;
    unsigned char* yk = reinterpret_cast<unsigned char*>(
        c->ws[27].ensure(sizeof(T) * ns * 2 * nb + sizeof(int) * (ns + 4) + 64));
    YZc = reinterpret_cast<T*>(yk);
    keep_d = reinterpret_cast<int*>(yk + ((sizeof(T) * ns * 2 * nb + 63) / 64) * 64);
  }

  void spmm(const T* X, T* YH, T* YM, int m) {
    spmm_hm_raw<T>(st, c->a_ptr.as<long long>(), c->a_col.as<int>(), aval, n, X, ld, YH, YM, ld,
                   m);
    ++spmm_calls;
  }

  // C(:, cols) += A (p cols) * G  where G = -coeffs (already negated, FP64 p x q)
  void apply_coeffs(const T* A, int lda, int p, const double* Gd, int q, T* C, int ldc) {
    (k_d2t<T><<<(p * q + 255) / 256, 256, 0, st>>>(Gd, Gt, p * q), ::ff::note_launch());
    block_update<T>(st, A, lda, p, Gt, q, C, ldc, n, T(1));
  }

  void deflate(T* X, int m) {
    // X -= c0 (Mc0^T X)
    gram<T>(st, Mc0, 1, 1, X, ld, m, n, G1, -1.0, false, c->scratch[0]);
    apply_coeffs(c0, 1, 1, G1, m, X, ld);
  }
};

// One run of the solver at one precision.  A mixed-precision solve runs an
// FP32 phase (FP32 roundings of H_w and M) that hands its best block to a
// double-float phase.
struct Phase {
  const void* aval = nullptr;      // interleaved (H, M) of the phase's precision
  const float* X0_int = nullptr;   // start block from an earlier phase: internal
                                   // particle order, dense n x nb
  int stall = 50;                  // stop after this many iterations without progress
  double gain = 0.999;             // progress = largest residual below gain x the last mark
  double stall_below = INFINITY;   // iterations only count as stalled below this residual
  int no_best = 40;                // stop after this many iterations without a new
                                   // smallest largest residual, whatever its level
  int best_slot = 22;              // workspace slot that keeps the best block (dense n x nb)
  bool rr_fp32 = false;            // Rayleigh-Ritz in FP32 (else FP64)
  bool update_products = false;    // H X', M X' by the block update instead of a
                                   // fresh block product (a phase that hands over
                                   // well above its rounding floor)
  bool handover_on_breakdown = false;  // a breakdown ends the phase (its best block
                                       // is handed over) instead of a restart
  bool have_best = false;          // out: the best-block slot holds a block
};

// the caller's precision of the modes: FP64 for a double-float phase
template <class T>
using OutOf = std::conditional_t<std::is_same_v<T, dfloat>, double, T>;

template <class T>
ff_status solve(ff_ctx* c, int k, const ff_eig_opts& o, Phase& ph, const T* X0,
                double* eigvals, OutOf<T>* modes, ff_eig_report* rep) {
  using clock = std::chrono::steady_clock;
  const auto t_start = clock::now();
  Solver<T> s;
  s.c = c;
  s.st = c->stream;
  s.aval = static_cast<const T*>(ph.aval);
  s.n = c->n;
  s.fp64 = sizeof(T) == 8;
  s.rr64 = !ph.rr_fp32;
  const bool incl_c0 = !o.exclude_constant;
  s.kw = incl_c0 ? k - 1 : k;
  // block width: the wanted modes plus guard vectors, rounded up to a multiple
  // of four so that every block starts on a 16-byte boundary
  s.nb = (s.kw + std::max(0, o.guard) + 3) / 4 * 4;
  s.nb = std::min<long long>(std::min(s.nb, 340), (s.n - 1) / 3);
  FF_REQUIRE(s.nb >= s.kw && s.nb >= 1, FF_ERR_INVALID_ARG,
             "too few particles for the requested number of modes");
  s.mc = (s.nb + 7) / 8 * 8 <= 256 ? (s.nb + 7) / 8 * 8 : s.nb;
  s.alloc();
  cudaStream_t st = s.st;
  const long long n = s.n;
  const int nb = s.nb, ld = s.ld;
  const int TB = 256;
  auto blocks = [&](long long work) { return (unsigned)((work + TB - 1) / TB); };

  // ---- constant mode: c0 = 1 / sqrt(1^T M 1)
  (k_fill<T><<<blocks(n), TB, 0, st>>>(s.c0, n, T(1)), ::ff::note_launch());
  spmm_hm_raw<T>(st, c->a_ptr.as<long long>(), c->a_col.as<int>(), s.aval, n, s.c0, 1, nullptr,
                 s.Mc0, 1, 1);
  gram<T>(st, s.c0, 1, 1, s.Mc0, 1, 1, n, s.G1, 1.0, false, c->scratch[0]);
  (k_scale<T><<<blocks(n), TB, 0, st>>>(s.c0, n, s.G1, 0), ::ff::note_launch());
  (k_scale<T><<<blocks(n), TB, 0, st>>>(s.Mc0, n, s.G1, 0), ::ff::note_launch());
  FF_LAUNCH_CHECK();

  // ---- Chebyshev interval on D^-1 H
  double beta = 0.0, alpha = 0.0;
  const int deg = std::max(0, o.cheb_degree);
  if (deg > 1) {
    unsigned int* gmax = reinterpret_cast<unsigned int*>(s.dropped_d + 2);
    FF_CUDA(cudaMemsetAsync(gmax, 0, sizeof(unsigned int), st));
    (k_gershgorin<<<blocks(n), TB, 0, st>>>(c->a_ptr.as<long long>(), c->h_f32.as<float>(),
                                           c->hdiag_f32.as<float>(), n, gmax), ::ff::note_launch());
    // power iteration on a 4-column block (reuses the Chebyshev step with res = 0)
    (k_random_block<float><<<blocks(4 * n), TB, 0, st>>>(s.cd0, 4, n, 4, o.seed + 7, c->perm.as<int>()), ::ff::note_launch());
    double est = 0.0;
    float* a = s.cd0;
    float* b = s.cd1;
    for (int it = 0; it < 12; ++it) {
      FF_CUDA(cudaMemsetAsync(s.cres, 0, sizeof(float) * 4 * n, st));
      cheb_step(st, c->a_ptr.as<long long>(), c->a_col.as<int>(), c->h_f32.as<float>(),
                c->hdiag_f32.as<float>(), n, 4, 4, a, b, s.cx, s.cres, 0.f, -1.f, kProfSetup);
      gram<float>(st, a, 4, 4, a, 4, 4, n, s.G1, 1.0, false, c->scratch[0]);
      gram<float>(st, b, 4, 4, b, 4, 4, n, s.G1 + 16, 1.0, false, c->scratch[0]);
      // normalise b (one common factor) and make it the next input
      (k_scale<float><<<blocks(4 * n), TB, 0, st>>>(b, 4 * n, s.G1 + 16, 0), ::ff::note_launch());
      std::swap(a, b);
    }
    double hb[32];
    unsigned int hg = 0;
    FF_CUDA(cudaMemcpyAsync(hb, s.G1, sizeof(hb), cudaMemcpyDeviceToHost, st));
    FF_CUDA(cudaMemcpyAsync(&hg, gmax, sizeof(hg), cudaMemcpyDeviceToHost, st));
    FF_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < 4; ++j) est = std::max(est, std::sqrt(hb[16 + 5 * j] / hb[5 * j]));
    float gf;
    memcpy(&gf, &hg, sizeof(gf));
    beta = std::min(1.2 * est, (double)gf);
    if (!(beta > 0)) beta = gf;
    alpha = beta / std::max(2.0, o.cheb_ratio);
  }

  // ---- starting block
  int warm = 0;
  if (ph.X0_int) {
    (k_cast_block<T><<<blocks(n * nb), TB, 0, st>>>(ph.X0_int, nb, n, nb, s.S[0], ld),
     ::ff::note_launch());
  } else {
    (k_random_block<T><<<blocks(n * nb), TB, 0, st>>>(s.S[0], ld, n, nb, o.seed,
                                                     c->perm.as<int>()), ::ff::note_launch());
    if (X0) {  // the caller's kw + guard columns; any rounding-up columns stay random
      const int mu = std::min(nb, s.kw + std::max(0, o.guard));
      (k_gather_block<T><<<blocks(n * mu), TB, 0, st>>>(X0, n, mu, c->perm.as<int>(), s.S[0], ld),
       ::ff::note_launch());
      warm = 1;
    }
  }
  FF_LAUNCH_CHECK();
  int cur = 0;
  // Rayleigh-Ritz on a block alone (the start block, or the best block after
  // a breakdown): it is the block to orthonormalise.  A warm start is first
  // taken with a loose drop threshold: directions it hardly adds (nearly
  // dependent predicted columns) leave the basis, the block is rotated onto
  // its Ritz vectors (the dropped directions come last, as zero columns) and
  // those columns are refilled from the seeded random generator.
  auto block_rr = [&](bool loose) {
    for (int attempt = 0;; ++attempt) {
      s.deflate(s.S[cur], nb);
      s.spmm(s.S[cur], s.HS[cur], s.MS[cur], nb);
      gram<T>(st, s.S[cur], ld, nb, s.HS[cur], ld, nb, n, s.Ag, 1.0, false, c->scratch[0]);
      gram<T>(st, s.S[cur], ld, nb, s.MS[cur], ld, nb, n, s.Bg, 1.0, false, c->scratch[0]);
      RRDims d0{nb, nb, nb, 0, 0, nb};
      if (loose && attempt == 0) d0.drop = s.fp64 ? 1e-10 : 1e-6;
      rayleigh_ritz<T>(st, s.Ag, s.Bg, d0, s.YZ, s.theta_d, s.dropped_d, c->scratch[1], s.rr64);
      int dropped = 0;
      FF_CUDA(cudaMemcpyAsync(&dropped, s.dropped_d, sizeof(int), cudaMemcpyDeviceToHost, st));
      FF_CUDA(cudaStreamSynchronize(st));
      if (dropped == 0 || attempt == 2) break;
      const int nxt = 1 - cur;
      block_update<T>(st, s.S[cur], ld, nb, s.YZ, nb, s.S[nxt], ld, n, T(0), -1, 0, 2 * nb);
      cur = nxt;
      const int keep = std::max(0, nb - dropped);
      (k_random_block<T><<<blocks(n * (nb - keep)), TB, 0, st>>>(
           s.S[cur] + keep, ld, n, nb - keep, o.seed + 7919ULL * (attempt + 1), c->perm.as<int>()),
       ::ff::note_launch());
      FF_LAUNCH_CHECK();
    }
    const int nxt = 1 - cur;
    block_update<T>(st, s.S[cur], ld, nb, s.YZ, nb, s.S[nxt], ld, n, T(0), -1, 0, 2 * nb);
    s.spmm(s.S[nxt], s.HS[nxt], s.MS[nxt], nb);
    cur = nxt;
  };
  block_rr(warm != 0);

  // ---- iterations
  std::vector<int> active(nb, 1), pack, keep, pact(nb, 1);
  std::vector<double> res(nb, 1.0), theta(nb, 0.0);
  bool has_p = false;
  int it = 0;
  ff_status status = FF_ERR_NOT_CONVERGED;
  const double th_c = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
  // column statistics: chunks of 64 rows (8 per warp), enough blocks in flight
  // to cover the loads' latency
  const long long rpb = std::max<long long>(64, (n + 2047) / 2048);
  const int cs_blocks = (int)((n + rpb - 1) / rpb);
  double* cs_part = reinterpret_cast<double*>(c->scratch[2].ensure(sizeof(double) * cs_blocks * 5 * nb));
  // the block with the smallest largest residual seen, and the progress mark
  T* best = reinterpret_cast<T*>(c->ws[ph.best_slot].ensure(sizeof(T) * n * nb));
  double best_worst = INFINITY, mark = INFINITY, last_worst = INFINITY;
  int mark_it = 0, restarts = 0, best_it = 0;
  std::vector<double> best_res;
  for (;; ++it) {
    // Rayleigh quotients and residual norms of the current X (products recomputed)
    constexpr bool direct = std::is_same_v<T, dfloat>;
    if constexpr (direct)
      (k_colstats_partial_direct<T><<<cs_blocks, 256, 0, st>>>(
           s.S[cur], s.HS[cur], s.MS[cur], ld, n, nb, rpb, s.theta_d, cs_part),
       ::ff::note_launch());
    else
      (k_colstats_partial<T><<<cs_blocks, 256, 0, st>>>(s.S[cur], s.HS[cur], s.MS[cur], ld, n,
                                                       nb, rpb, cs_part),
       ::ff::note_launch());
    (k_colstats_final<<<nb, 128, 0, st>>>(cs_part, cs_blocks, nb, s.theta_d, s.norms_d,
                                          direct ? 1 : 0),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    FF_CUDA(cudaMemcpyAsync(s.h_pin, s.norms_d, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost,
                            st));
    FF_CUDA(cudaStreamSynchronize(st));
    int conv = 0;
    double worst = 0.0;
    bool bad = false;
    for (int j = 0; j < nb; ++j) {
      theta[j] = s.h_pin[j];
      double r = std::sqrt(s.h_pin[nb + j]) / (std::fabs(theta[j]) * std::sqrt(s.h_pin[2 * nb + j]));
      if (!std::isfinite(r)) {
        bad = true;
        r = 1.0;
      }
      res[j] = r;
      active[j] = r > o.tol;
      if (j < s.kw) {
        conv += r <= o.tol;
        worst = std::max(worst, r);
      }
    }
    if (o.verbose)
      fprintf(stderr, "[eigenmodes] it %d  max res %.3e  converged %d/%d\n", it, worst, conv, s.kw);
    last_worst = bad ? INFINITY : worst;
    if (!bad && worst < best_worst) {
      best_worst = worst;
      best_it = it;
      best_res = res;
      FF_CUDA(cudaMemcpy2DAsync(best, sizeof(T) * nb, s.S[cur], sizeof(T) * ld, sizeof(T) * nb, n,
                                cudaMemcpyDeviceToDevice, st));
    }
    if (!bad && (worst < mark * ph.gain || worst >= ph.stall_below)) {
      mark = worst;
      mark_it = it;
    }
    if (bad) {
      status = FF_ERR_NUMERIC;
      break;
    }
    // Breakdown: after the block had come close (best below 0.1) the largest
    // residual is ten times the best seen -- the basis has lost converged
    // directions.  Restart from the best block without momentum (or, in a
    // phase that hands over, end the phase: its best block is handed on).
    if (best_worst < 1e-1 && worst > 10.0 * best_worst && conv < s.kw) {
      if (ph.handover_on_breakdown || restarts >= 3) {
        status = FF_ERR_NOT_CONVERGED;
        break;
      }
      ++restarts;
      FF_CUDA(cudaMemcpy2DAsync(s.S[cur], sizeof(T) * ld, best, sizeof(T) * nb, sizeof(T) * nb, n,
                                cudaMemcpyDeviceToDevice, st));
      block_rr(false);
      has_p = false;
      std::fill(pact.begin(), pact.end(), 1);
      mark = best_worst;
      mark_it = it;
      best_it = it;
      continue;
    }
    if (conv == s.kw) {
      status = FF_OK;
      break;
    }
    if (it >= o.max_iter || (ph.stall > 0 && it - mark_it >= ph.stall) ||
        (ph.no_best > 0 && it - best_it >= ph.no_best)) {
      status = FF_ERR_NOT_CONVERGED;
      break;
    }
    if (o.time_budget_s > 0 &&
        std::chrono::duration<double>(clock::now() - t_start).count() > o.time_budget_s) {
      status = FF_ERR_TIMEOUT;
      break;
    }
    // W = T R  (FP32 Chebyshev polynomial in D^-1 H, or Jacobi when deg <= 1)
    T* W = s.S[cur] + nb;
    // BF16 directions halve the bytes each preconditioner step gathers; their
    // steps take widths in multiples of 8, the padding columns stay zero
    const bool b16 = deg > 1 && s.mc % 8 == 0;
    // packed: only the columns above tol enter the steps, w of them rounded up
    // to 8 (the others are zero either way; on tensor cores W is bit-identical,
    // the CUDA-core step's lane split follows the width, so there W changes at
    // FP32 rounding)
    const bool packed = b16 && o.precond_compact;
    int mc = s.mc;
    if (packed) {
      int nact = 0;
      for (int j = 0; j < nb; ++j) nact += active[j] != 0;
      mc = std::max(8, (nact + 7) / 8 * 8);
      pack.assign(2 * nb + s.mc, -1);
      std::copy(active.begin(), active.end(), pack.begin());
      for (int j = 0, q = 0; j < nb; ++j)
        if (active[j]) {
          pack[nb + q] = j;           // cmap[q] = j
          pack[nb + s.mc + j] = q++;  // cinv[j] = q
        }
      FF_CUDA(cudaMemcpyAsync(s.active_d, pack.data(), sizeof(int) * pack.size(),
                              cudaMemcpyHostToDevice, st));
      (k_cheb_init_packed<T><<<blocks(n * mc), TB, 0, st>>>(
           s.HS[cur], s.MS[cur], ld, s.theta_d, s.active_d + nb, c->hdiag_f32.as<float>(), n, mc,
           s.cres, s.cx, (float)(1.0 / th_c), s.cb0),
       ::ff::note_launch());
    } else {
      FF_CUDA(cudaMemcpyAsync(s.active_d, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                              st));
      (k_cheb_init<T><<<blocks(n * mc), TB, 0, st>>>(s.HS[cur], s.MS[cur], ld, s.theta_d,
                                                    s.active_d, c->hdiag_f32.as<float>(), n, nb,
                                                    mc, s.cres, s.cd0, s.cx,
                                                    deg > 1 ? (float)(1.0 / th_c) : 1.f,
                                                    b16 ? s.cb0 : nullptr), ::ff::note_launch());
    }
    FF_LAUNCH_CHECK();
    if (deg > 1) {
      const double sigma1 = th_c / delta;
      double rho = 1.0 / sigma1;
      float* din = s.cd0;
      float* dout = s.cd1;
      __nv_bfloat16* bin = s.cb0;
      __nv_bfloat16* bout = s.cb1;
      for (int j = 1; j < deg; ++j) {
        const double rn = 1.0 / (2.0 * sigma1 - rho);
        const float c1 = (float)(rn * rho), c2 = (float)(2.0 * rn / delta);
        // the tensor-core step when its tiles exist, else the CUDA-core ones
        const bool tc =
            b16 && o.precond_tc && cheb_step_tc(st, c, mc, bin, bout, s.cx, s.cres, c1, c2);
        if (!tc && b16) {
          cheb_step_b16(st, c->a_ptr.as<long long>(), c->a_col.as<int>(), c->h_f32.as<float>(),
                        c->hdiag_f32.as<float>(), n, mc, bin, bout, s.cx, s.cres, c1, c2);
        } else if (!tc) {
          cheb_step(st, c->a_ptr.as<long long>(), c->a_col.as<int>(), c->h_f32.as<float>(),
                    c->hdiag_f32.as<float>(), n, mc, mc, din, dout, s.cx, s.cres, c1, c2);
        }
        ++s.spmv_calls;
        rho = rn;
        std::swap(din, dout);
        std::swap(bin, bout);
      }
    }
    if (packed)
      (k_cast_packed<T><<<blocks(n * nb), TB, 0, st>>>(s.cx, mc, s.active_d + nb + s.mc, n, nb,
                                                       W, ld), ::ff::note_launch());
    else
      (k_cast_block<T><<<blocks(n * nb), TB, 0, st>>>(s.cx, mc, n, nb, W, ld),
       ::ff::note_launch());
    FF_LAUNCH_CHECK();
    // M-project W against X, P and c0 (with the stored M X, M P, M c0)
    s.deflate(W, nb);
    gram<T>(st, s.MS[cur], ld, nb, W, ld, nb, n, s.G1, -1.0, false, c->scratch[0]);
    s.apply_coeffs(s.S[cur], ld, nb, s.G1, nb, W, ld);
    if (has_p) {
      gram<T>(st, s.MS[cur] + 2 * nb, ld, nb, W, ld, nb, n, s.G1, -1.0, false, c->scratch[0]);
      s.apply_coeffs(s.S[cur] + 2 * nb, ld, nb, s.G1, nb, W, ld);
    }
    s.spmm(W, s.HS[cur] + nb, s.MS[cur] + nb, nb);
    const int ns = has_p ? 3 * nb : 2 * nb;
    gram_rr<T>(st, s.S[cur], s.HS[cur], s.MS[cur], ld, nb, has_p ? 3 : 2, n, s.Ag, s.Bg,
               c->scratch[0]);
    // Soft locking: the Rayleigh-Ritz step keeps X, the W columns of the modes
    // still above tol and the P columns that carry momentum (those of the
    // modes active in the previous iteration); the others are zero and would
    // only be dropped inside it.  Its cost falls from (3 nb)^3 towards
    // (nb + 2 n_active)^3 as the modes converge.
    keep.clear();
    int na = 0;
    for (int j = 0; j < nb; ++j) keep.push_back(j);
    for (int j = 0; j < nb; ++j)
      if (active[j]) {
        keep.push_back(nb + j);
        ++na;
      }
    if (has_p)
      for (int j = 0; j < nb; ++j)
        if (pact[j]) keep.push_back(2 * nb + j);
    const int nsc = (int)keep.size();
    if (nsc < ns && na > 0) {
      FF_CUDA(cudaMemcpyAsync(s.keep_d, keep.data(), sizeof(int) * nsc, cudaMemcpyHostToDevice,
                              st));
      (k_gather_sq<<<blocks((long long)nsc * nsc), TB, 0, st>>>(s.Ag, ns, s.keep_d, nsc, s.Ac),
       ::ff::note_launch());
      (k_gather_sq<<<blocks((long long)nsc * nsc), TB, 0, st>>>(s.Bg, ns, s.keep_d, nsc, s.Bc),
       ::ff::note_launch());
      FF_LAUNCH_CHECK();
      RRDims dc{nsc, nb, nb, 1, nb, na};
      rayleigh_ritz<T>(st, s.Ac, s.Bc, dc, s.YZc, s.theta_d, s.dropped_d, c->scratch[1],
                       s.rr64);
      FF_CUDA(cudaMemsetAsync(s.YZ, 0, sizeof(T) * (size_t)ns * 2 * nb, st));
      (k_place_rows<T><<<blocks((long long)nsc * 2 * nb), TB, 0, st>>>(s.YZc, nsc, 2 * nb,
                                                                      s.keep_d, s.YZ),
       ::ff::note_launch());
      FF_LAUNCH_CHECK();
    } else {
      RRDims dd{ns, nb, nb, 1, nb, nb};
      rayleigh_ritz<T>(st, s.Ag, s.Bg, dd, s.YZ, s.theta_d, s.dropped_d, c->scratch[1], s.rr64);
    }
    pact = active;
    (k_lock_momentum<T><<<blocks((long long)ns * nb), TB, 0, st>>>(s.YZ, ns, nb, s.active_d),
     ::ff::note_launch());
    const int nxt = 1 - cur;
    // X' = S Y, P' = S Z; H P', M P' from the old products; (H X', M X') recomputed
    // from X' itself so that the residual seen by the solver is that of the
    // stored X' (updated products drift from the stored block in FP32) -- or,
    // in a phase that hands over well above that drift, updated as well
    block_update<T>(st, s.S[cur], ld, ns, s.YZ, 2 * nb, s.S[nxt], ld, n, T(0), nb, 2 * nb);
    if (ph.update_products) {
      block_update<T>(st, s.HS[cur], ld, ns, s.YZ, 2 * nb, s.HS[nxt], ld, n, T(0), nb, 2 * nb);
      block_update<T>(st, s.MS[cur], ld, ns, s.YZ, 2 * nb, s.MS[nxt], ld, n, T(0), nb, 2 * nb);
    } else {
      block_update<T>(st, s.HS[cur], ld, ns, s.YZ + nb, nb, s.HS[nxt] + 2 * nb, ld, n, T(0), -1,
                      0, 2 * nb);
      block_update<T>(st, s.MS[cur], ld, ns, s.YZ + nb, nb, s.MS[nxt] + 2 * nb, ld, n, T(0), -1,
                      0, 2 * nb);
      s.spmm(s.S[nxt], s.HS[nxt], s.MS[nxt], nb);
    }
    cur = nxt;
    has_p = true;
  }

  // ---- without convergence, fall back to the best block seen
  ph.have_best = !best_res.empty();
  if (status != FF_OK && !best_res.empty() && !(last_worst <= best_worst)) {
    FF_CUDA(cudaMemcpy2DAsync(s.S[cur], sizeof(T) * ld, best, sizeof(T) * nb, sizeof(T) * nb, n,
                              cudaMemcpyDeviceToDevice, st));
    s.spmm(s.S[cur], s.HS[cur], s.MS[cur], nb);
    res = best_res;
  }

  // ---- eigenvalues as Rayleigh quotients of the final block (FP64-accumulated)
  const int kw = s.kw;
  std::vector<double> hq(2 * (size_t)kw * kw);
  gram<T>(st, s.S[cur], ld, kw, s.HS[cur], ld, kw, n, s.Ag, 1.0, false, c->scratch[0]);
  gram<T>(st, s.S[cur], ld, kw, s.MS[cur], ld, kw, n, s.Bg, 1.0, false, c->scratch[0]);
  FF_CUDA(cudaMemcpyAsync(hq.data(), s.Ag, sizeof(double) * kw * kw, cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaMemcpyAsync(hq.data() + (size_t)kw * kw, s.Bg, sizeof(double) * kw * kw,
                          cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  int out = 0;
  if (incl_c0) eigvals[out++] = 0.0;
  for (int j = 0; j < kw; ++j)
    eigvals[out++] = hq[(size_t)j * kw + j] / hq[(size_t)kw * kw + (size_t)j * kw + j];
  if (modes) {
    int col0 = 0;
    if (incl_c0) {
      (k_scatter_block<T, OutOf<T>><<<blocks(n), TB, 0, st>>>(s.c0, 1, n, 1, c->perm.as<int>(),
                                                               modes, n, 0),
       ::ff::note_launch());
      col0 = 1;
    }
    (k_scatter_block<T, OutOf<T>><<<blocks(n * kw), TB, 0, st>>>(
         s.S[cur], ld, n, kw, c->perm.as<int>(), modes, n, col0),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  FF_CUDA(cudaStreamSynchronize(st));
  if (rep) {
    rep->iterations = it;
    int conv = incl_c0 ? 1 : 0;
    double worst = 0.0;
    for (int j = 0; j < kw; ++j) {
      conv += res[j] <= o.tol;
      worst = std::max(worst, res[j]);
    }
    rep->converged = conv;
    rep->spmm_calls = s.spmm_calls;
    rep->precond_spmv_calls = s.spmv_calls;
    rep->max_residual = worst;
    rep->seconds = std::chrono::duration<double>(clock::now() - t_start).count();
    rep->warm_start_used = warm;
  }
  return status;
}

namespace {
ff_status run_once(ff_ctx* c, int k, const ff_eig_opts& o, const void* X0, double* eigvals,
                   void* modes, ff_eig_report* rep) {
  if (c->prec != FF_PREC_FP64) {
    Phase ph;
    ph.aval = c->a_val.as<float>();
    return solve<float>(c, k, o, ph, static_cast<const float*>(X0), eigvals,
                        static_cast<float*>(modes), rep);
  }
  Phase p64;
  p64.aval = c->a_val.as<double>();
  if (!o.fp32_phase)
    return solve<double>(c, k, o, p64, static_cast<const double*>(X0), eigvals,
                         static_cast<double*>(modes), rep);
  // FP32 phase: to fp32_tol, or until the FP32 residual floor stops it
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  ff_eig_opts o1 = o;
  o1.tol = std::max(o.tol, o.fp32_tol);
  Phase p32;
  p32.aval = c->a_val32.as<float>();
  // hand over once two iterations in a row gain less than 30% (FP32 rounding
  // of H, M and the block sets a floor near 1e-4 on the 50k torus)
  p32.stall = 2;
  p32.gain = 0.7;
  p32.stall_below = 1e-2;
  p32.no_best = 15;
  p32.rr_fp32 = true;
  p32.update_products = true;
  p32.handover_on_breakdown = true;
  p32.best_slot = 21;
  const float* X0f = nullptr;
  if (X0) {  // the caller's FP64 start block, rounded
    const int kw = o.exclude_constant ? k : k - 1;
    const long long m = (long long)c->n * (kw + std::max(0, o.guard));
    float* x = reinterpret_cast<float*>(c->ws[23].ensure(sizeof(float) * m));
    (k_round_block<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(
         static_cast<const double*>(X0), x, m),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    X0f = x;
  }
  std::vector<double> ev1(k);
  ff_eig_report r1{};
  const ff_status s1 = solve<float>(c, k, o1, p32, X0f, ev1.data(), nullptr, &r1);
  // second phase from the FP32 phase's best block
  ff_eig_opts o2 = o;
  o2.max_iter = std::max(0, o.max_iter - r1.iterations);
  if (o.cheb_degree_fp64 > 0) o2.cheb_degree = o.cheb_degree_fp64;
  if (o.time_budget_s > 0) {
    const double used = std::chrono::duration<double>(clock::now() - t0).count();
    o2.time_budget_s = std::max(1e-9, o.time_budget_s - used);
    if (s1 == FF_ERR_TIMEOUT) o2.max_iter = 0;
  }
  // in double-float arithmetic (H, M split into FP32 pairs, ~48-bit significands)
  if (p32.have_best) p64.X0_int = reinterpret_cast<const float*>(c->ws[21].p);
  p64.aval = c->a_valdf.p;
  ff_status s2 = solve<dfloat>(c, k, o2, p64, nullptr, eigvals, static_cast<double*>(modes), rep);
  if (s1 == FF_ERR_TIMEOUT && s2 == FF_ERR_NOT_CONVERGED) s2 = FF_ERR_TIMEOUT;
  if (rep) {
    rep->iterations += r1.iterations;
    rep->fp32_iterations = r1.iterations;
    rep->spmm_calls += r1.spmm_calls;
    rep->precond_spmv_calls += r1.precond_spmv_calls;
    rep->seconds = std::chrono::duration<double>(clock::now() - t0).count();
    rep->warm_start_used = r1.warm_start_used;
  }
  return s2;
}
}  // namespace

// A start block that ends without convergence (not on a timeout) falls back
// to the random start: the solve runs again as a plain call, so the caller's
// block can cost iterations but never the answer.
ff_status run_eigenmodes(ff_ctx* c, int k, const ff_eig_opts& o, const void* X0, double* eigvals,
                         void* modes, ff_eig_report* rep) {
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  ff_eig_report r1{};
  const ff_status s1 = run_once(c, k, o, X0, eigvals, modes, &r1);
  if (!X0 || s1 == FF_OK || s1 == FF_ERR_TIMEOUT) {
    if (rep) *rep = r1;
    return s1;
  }
  ff_eig_opts o2 = o;
  if (o.time_budget_s > 0) {
    const double used = std::chrono::duration<double>(clock::now() - t0).count();
    if (used >= o.time_budget_s) {
      if (rep) *rep = r1;
      return FF_ERR_TIMEOUT;
    }
    o2.time_budget_s = o.time_budget_s - used;
  }
  ff_eig_report r2{};
  const ff_status s2 = run_once(c, k, o2, nullptr, eigvals, modes, &r2);
  if (rep) {
    *rep = r2;
    rep->iterations += r1.iterations;
    rep->fp32_iterations += r1.fp32_iterations;
    rep->spmm_calls += r1.spmm_calls;
    rep->precond_spmv_calls += r1.precond_spmv_calls;
    rep->seconds = std::chrono::duration<double>(clock::now() - t0).count();
    rep->warm_start_used = 2;
  }
  return s2;
}

template <class T>
void spmm_hm(ff_ctx* c, const T* X, int ldx, T* YH, T* YM, int ldy, int m) {
  spmm_hm_raw<T>(c->stream, c->a_ptr.as<long long>(), c->a_col.as<int>(), c->a_val.as<T>(), c->n,
                 X, ldx, YH, YM, ldy, m);
}
template void spmm_hm<float>(ff_ctx*, const float*, int, float*, float*, int, int);
template void spmm_hm<double>(ff_ctx*, const double*, int, double*, double*, int, int);

// caller-order column-major block <-> internal row-major panel (used by ff_apply_operators)
template <class T>
void gather_block(ff_ctx* c, const T* X0, int m, T* X, int ld) {
  (k_gather_block<T><<<(unsigned)((c->n * m + 255) / 256), 256, 0, c->stream>>>(
      X0, c->n, m, c->perm.as<int>(), X, ld), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}
template <class T>
void scatter_block(ff_ctx* c, const T* X, int ld, int m, T* out) {
  (k_scatter_block<T><<<(unsigned)((c->n * m + 255) / 256), 256, 0, c->stream>>>(
      X, ld, c->n, m, c->perm.as<int>(), out, c->n, 0), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}
template void gather_block<float>(ff_ctx*, const float*, int, float*, int);
template void gather_block<double>(ff_ctx*, const double*, int, double*, int);
template void scatter_block<float>(ff_ctx*, const float*, int, int, float*);
template void scatter_block<double>(ff_ctx*, const double*, int, int, double*);

}  // namespace ff
