// Small dense Rayleigh-Ritz step of the block eigensolver (FP64).
//
// The basis S = [X | W | P] (n = nx + nw + np columns) is M-orthonormal except
// for one block O = columns [o0, o0 + no) (the fresh preconditioned residuals W,
// or the whole start block in the first step).  Given the FP64 Gram matrices
// A = S^T H S and B = S^T M S, the nb lowest Ritz pairs of (A, B) -- the trace
// minimisation of Sec. 3.2, Eq. 15 restricted to span S -- are found in four
// launches that hand their results over in a global workspace:
//   k_rr_tridiag  scale the O block by diag(B_OO)^-1/2, Cholesky B_OO = L L^T
//                 with drop (dependent or empty columns leave the basis, as do
//                 columns outside O whose B_ii is not ~1: empty momentum
//                 directions), A <- T^T A T with T = blockdiag(I, L^-T, I), and
//                 Householder tridiagonalisation of A;
//   k_rr_eigvals  the nb smallest eigenvalues of the tridiagonal matrix: an
//                 FP32 multisection on Sturm counts brackets each one, FP64
//                 bisection with a division-free Sturm count refines it;
//   k_rr_invit    their eigenvectors by inverse iteration on the tridiagonal
//                 (LU with partial pivoting), one thread per vector;
//   k_rr_finish   Cholesky QR (twice) of those vectors, the Householder
//                 reflectors applied in reverse, the momentum coefficients Z
//                 (the W and P rows of the Ritz vectors, orthogonalised against
//                 them and orthonormalised -- the next P = S Z is then
//                 M-orthonormal and M-orthogonal to the next X), and the O rows
//                 mapped back through L^-T and the scaling.
// Output YZ = [Y | Z] (n x 2 nb, row-major, context precision) and the Ritz
// values theta (nb).  FP64 throughout: the spectrum of A spans the whole range
// of the basis' Rayleigh quotients and the small eigenvalues need relative
// accuracy.
#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr size_t kMaxDynSmem = 200 * 1024;
constexpr double kDrop = 1e-13;
constexpr double kEps = 1.1e-16;

// global workspace layout (doubles)
struct RRWork {
  double *As, *ref, *L, *dsc, *dg, *e, *e2, *tau, *lam, *V, *Z, *G, *T1, *scr;
  int* keep;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread gets the result
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
  return warp_sum(t);
}

// right-looking Cholesky (lower) of an m x m matrix in place, with drop
__device__ void block_cholesky(double* G, int m, int* keep, double drop_rel) {
  __shared__ int s_keep;
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double piv = G[j * m + j];
      const int k = keep[j] && piv > drop_rel;
      keep[j] = k;
      G[j * m + j] = k ? sqrt(piv) : 1.0;
      s_keep = k;
    }
    __syncthreads();
    const double ljj = G[j * m + j];
    const int kj = s_keep;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) G[i * m + j] = kj ? G[i * m + j] / ljj : 0.0;
    __syncthreads();
    const int r = m - j - 1;
    if (kj)
      for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
        const int i = j + 1 + t / r, l = j + 1 + t % r;
        if (l <= i) G[i * m + l] -= G[i * m + j] * G[l * m + j];
      }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ 1. tridiagonalise
__global__ void __launch_bounds__(kThreads)
    k_rr_tridiag(const double* __restrict__ A, const double* __restrict__ B, int n, int o0, int no,
                 RRWork w, int smem) {
  extern __shared__ double dyn[];
  __shared__ double red[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const size_t nn = (size_t)n * n;
  double* As = smem ? dyn : w.As;
  double* vt = w.T1;            // n
  double* pw = w.T1 + n;        // n
  // scaling: O columns by diag(B)^-1/2; other columns must have B_ii ~ 1
  for (int i = tid; i < n; i += kThreads) {
    const double bii = B[(size_t)i * n + i];
    double s = 1.0;
    int k = 1;
    if (i >= o0 && i < o0 + no) {
      k = bii > 1e-280 && isfinite(bii);
      s = k ? 1.0 / sqrt(bii) : 0.0;
    } else if (!(bii > 0.25 && bii < 4.0)) {
      k = 0;
      s = 0.0;
    }
    w.keep[i] = k;
    w.dsc[i] = s;
  }
  __syncthreads();
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    As[t] = 0.5 * (A[t] + A[(size_t)j * n + i]) * w.dsc[i] * w.dsc[j];
  }
  for (int t = tid; t < no * no; t += kThreads) {
    const int a = t / no, b = t % no, i = o0 + a, j = o0 + b;
    const double v = 0.5 * (B[(size_t)i * n + j] + B[(size_t)j * n + i]) * w.dsc[i] * w.dsc[j];
    w.L[t] = (w.keep[i] && w.keep[j]) ? v : (a == b ? 1.0 : 0.0);
  }
  __syncthreads();
  block_cholesky(w.L, no, w.keep + o0, kDrop);
  // A <- T^T A T: O rows by L^-1, then O columns
  for (int a = 0; a < no; ++a) {
    const int i = o0 + a;
    const double inv = 1.0 / w.L[a * no + a];
    for (int c = tid; c < n; c += kThreads) {
      double acc = As[(size_t)i * n + c];
      for (int b = 0; b < a; ++b) acc -= w.L[a * no + b] * As[(size_t)(o0 + b) * n + c];
      As[(size_t)i * n + c] = acc * inv;
    }
    __syncthreads();
  }
  for (int a = 0; a < no; ++a) {
    const int i = o0 + a;
    const double inv = 1.0 / w.L[a * no + a];
    for (int r = tid; r < n; r += kThreads) {
      double acc = As[(size_t)r * n + i];
      for (int b = 0; b < a; ++b) acc -= w.L[a * no + b] * As[(size_t)r * n + o0 + b];
      As[(size_t)r * n + i] = acc * inv;
    }
    __syncthreads();
  }
  // symmetrise; dropped columns are decoupled with a diagonal just above the
  // spectrum of the kept part (2 ||A_kept||_inf + 1), which keeps them out of
  // the nb lowest without disturbing the scale of the tridiagonal problem
  double rmax = 0.0;
  for (int i = wid; i < n; i += kWarps) {
    if (!w.keep[i]) continue;
    double rs = 0.0;
    for (int j = lane; j < n; j += 32)
      if (w.keep[j]) rs += fabs(As[(size_t)i * n + j]);
    rmax = fmax(rmax, warp_sum(rs));
  }
  {
    __syncthreads();
    if (lane == 0) red[wid] = rmax;
    __syncthreads();
    double t = lane < kWarps ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    rmax = t;
    __syncthreads();
  }
  const double big = 2.0 * rmax + 1.0;
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (!w.keep[i] || !w.keep[j]) As[t] = (i == j) ? big : 0.0;
    else if (i > j) As[t] = 0.5 * (As[t] + As[(size_t)j * n + i]);
  }
  __syncthreads();
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (i < j) As[t] = As[(size_t)j * n + i];
  }
  __syncthreads();
  // Householder: reflector j = [1, v] stored in row j of w.ref (entries j+1..n-1)
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    double part = 0.0;
    for (int i = tid; i < m; i += kThreads) {
      const double x = As[(size_t)(j + 1 + i) * n + j];
      part += x * x;
    }
    const double ss = block_sum(part, red);
    const double x0 = As[(size_t)(j + 1) * n + j];
    const double alpha = sqrt(ss);
    __syncthreads();
    if (!(alpha > 1e-290)) {
      if (tid == 0) {
        w.tau[j] = 0.0;
        w.e[j] = x0;
        w.dg[j] = As[(size_t)j * n + j];
      }
      __syncthreads();
      continue;
    }
    const double beta = x0 >= 0.0 ? -alpha : alpha;
    const double tj = (beta - x0) / beta;
    const double scale = 1.0 / (x0 - beta);
    for (int i = tid; i < m; i += kThreads) {
      const double v = i == 0 ? 1.0 : As[(size_t)(j + 1 + i) * n + j] * scale;
      vt[i] = v;
      w.ref[(size_t)j * n + j + 1 + i] = v;
    }
    if (tid == 0) {
      w.tau[j] = tj;
      w.e[j] = beta;
      w.dg[j] = As[(size_t)j * n + j];
    }
    __syncthreads();
    for (int i = wid; i < m; i += kWarps) {  // p = tau A22 v
      const double* row = As + (size_t)(j + 1 + i) * n + (j + 1);
      double acc = 0.0;
      for (int l = lane; l < m; l += 32) acc += row[l] * vt[l];
      acc = warp_sum(acc);
      if (lane == 0) pw[i] = tj * acc;
    }
    __syncthreads();
    double kp = 0.0;
    for (int i = tid; i < m; i += kThreads) kp += pw[i] * vt[i];
    const double K = 0.5 * tj * block_sum(kp, red);
    __syncthreads();
    for (int i = tid; i < m; i += kThreads) pw[i] -= K * vt[i];
    __syncthreads();
    for (int i = wid; i < m; i += kWarps) {  // A22 -= v w^T + w v^T
      double* row = As + (size_t)(j + 1 + i) * n + (j + 1);
      const double vi = vt[i], wi = pw[i];
      for (int l = lane; l < m; l += 32) row[l] -= vi * pw[l] + wi * vt[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      w.dg[n - 2] = As[(size_t)(n - 2) * n + (n - 2)];
      w.e[n - 2] = As[(size_t)(n - 1) * n + (n - 2)];
      w.tau[n - 2] = 0.0;
    }
    w.dg[n - 1] = As[(size_t)(n - 1) * n + (n - 1)];
    w.e[n - 1] = 0.0;
    w.tau[n - 1] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) w.e2[i] = w.e[i] * w.e[i];
}

// ------------------------------------------------------------------ 2. eigenvalues
__device__ int sturm32(const float* d, const float* e2, int n, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Division-free Sturm count in FP64: sign changes along the leading principal
// minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1), rescaled by
// exact powers of two to stay in range.  A zero minor takes the sign opposite
// to its predecessor.
__device__ int sturm64(const double* d, const double* e2, int n, double x) {
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -1e-300;
  int c = p < 0.0;
  for (int i = 1; i < n; ++i) {
    double q = fma(d[i] - x, p, -e2[i - 1] * pm);
    if (q == 0.0) q = p > 0.0 ? -1e-300 : 1e-300;
    c += (q < 0.0) != (p < 0.0);
    pm = p;
    p = q;
    const double ap = fabs(p);
    if (ap > 0x1p+600 || ap < 0x1p-600) {
      const int ex = ilogb(p);
      p = scalbn(p, -ex);
      pm = scalbn(pm, -ex);
    }
  }
  return c;
}

__global__ void __launch_bounds__(kThreads) k_rr_eigvals(int n, int nb, RRWork w, double* theta) {
  extern __shared__ double dyn[];
  double* dg = dyn;
  double* e2 = dg + n;
  double* bhi = e2 + n;
  double* blo = bhi + nb;
  float* d32 = reinterpret_cast<float*>(blo + nb);
  float* e32 = d32 + n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < n; i += kThreads) {
    dg[i] = w.dg[i];
    e2[i] = w.e2[i];
    d32[i] = (float)w.dg[i];
    e32[i] = (float)w.e2[i];
  }
  __syncthreads();
  double lo = 0.0, hi = 0.0;
  float emax32 = 0.f;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(w.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(w.e[i]) : 0.0);
    const double a = dg[i] - r, b = dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
    emax32 = fmaxf(emax32, e32[i]);
  }
  const double span = fmax(hi - lo, 1e-30);
  lo -= span * 1e-6;
  hi += span * 1e-6;
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const float pivmin32 = fmaxf(1e-37f, 1e-14f * emax32);
  for (int s = wid; s < nb; s += kWarps) {  // FP32 multisection bracket
    float a = (float)lo, b = (float)hi;
    for (int round = 0; round < 30; ++round) {
      const float x = a + (b - a) * (float)(lane + 1) / 33.f;
      const int cnt = sturm32(d32, e32, n, x, pivmin32);
      const unsigned above = __ballot_sync(0xffffffffu, cnt >= s + 1);
      const int first = above ? __ffs(above) - 1 : 32;
      const float na = first == 0 ? a : a + (b - a) * (float)first / 33.f;
      const float nbv = first == 32 ? b : a + (b - a) * (float)(first + 1) / 33.f;
      a = __shfl_sync(0xffffffffu, na, 0);
      b = __shfl_sync(0xffffffffu, nbv, 0);
      if (b - a <= 1e-6f * fmaxf(fabsf(a), fabsf(b))) break;
    }
    if (lane == 0) {
      blo[s] = (double)a;
      bhi[s] = (double)b;
    }
  }
  __syncthreads();
  for (int s = tid; s < nb; s += kThreads) {  // FP64 bisection from the widened bracket
    const double pad = 64.0 * 6e-8 * tnorm;
    double a = fmax(lo, blo[s] - pad), b = fmin(hi, bhi[s] + pad);
    if (!(sturm64(dg, e2, n, a) <= s)) a = lo;
    if (!(sturm64(dg, e2, n, b) >= s + 1)) b = hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (b - a <= 4.0 * kEps * fmax(fabs(a), fabs(b)) || mid <= a || mid >= b) break;
      if (sturm64(dg, e2, n, mid) >= s + 1) b = mid;
      else a = mid;
    }
    w.lam[s] = 0.5 * (a + b);
    theta[s] = 0.5 * (a + b);
  }
}

// ------------------------------------------------------------------ 3. inverse iteration
__global__ void k_rr_invit(int n, int nb, RRWork w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  double lo = 0.0, hi = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(w.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(w.e[i]) : 0.0);
    const double a = w.dg[i] - r, b = w.dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
  }
  const double span = fmax(hi - lo, 1e-30);
  const double tnorm = fmax(fabs(lo - span * 1e-6), fabs(hi + span * 1e-6));
  const double pivmin = fmax(1e-290, kEps * tnorm * 1e-6);
  double* u = w.scr + (size_t)s * 6 * n;  // U diagonal
  double* u1 = u + n;                     // first super-diagonal
  double* u2 = u1 + n;                    // second super-diagonal (pivoting fill)
  double* lm = u2 + n;                    // multipliers
  double* sw = lm + n;                    // row-swap flags
  double* z = sw + n;                     // the vector
  const double lam = w.lam[s];
  // a slightly perturbed shift keeps T - shift I from being exactly singular
  const double shift = lam + kEps * fmax(fabs(lam), span * 1e-3) * 4.0;
  double a_i = w.dg[0] - shift, b_i = n > 1 ? w.e[0] : 0.0, c_i = 0.0;
  for (int i = 0; i < n - 1; ++i) {
    const double sub = w.e[i];
    const double d1 = w.dg[i + 1] - shift;
    const double e1 = i + 2 < n ? w.e[i + 1] : 0.0;
    if (fabs(a_i) >= fabs(sub)) {
      const double pv = fabs(a_i) < pivmin ? (a_i < 0.0 ? -pivmin : pivmin) : a_i;
      const double l = sub / pv;
      u[i] = pv; u1[i] = b_i; u2[i] = c_i; lm[i] = l; sw[i] = 0.0;
      a_i = d1 - l * b_i;
      b_i = e1 - l * c_i;
      c_i = 0.0;
    } else {
      const double l = a_i / sub;
      u[i] = sub; u1[i] = d1; u2[i] = e1; lm[i] = l; sw[i] = 1.0;
      const double na = b_i - l * d1, nc = c_i - l * e1;
      a_i = na;
      b_i = nc;
      c_i = 0.0;
    }
  }
  u[n - 1] = fabs(a_i) < pivmin ? (a_i < 0.0 ? -pivmin : pivmin) : a_i;
  u1[n - 1] = 0.0;
  u2[n - 1] = 0.0;
  unsigned int h = 2166136261u ^ (unsigned)s * 16777619u;  // deterministic start vector
  for (int i = 0; i < n; ++i) {
    h = h * 1664525u + 1013904223u;
    z[i] = 0.5 + (double)((h >> 8) & 0xffff) / 65536.0;
  }
  for (int iter = 0; iter < 3; ++iter) {
    for (int i = 0; i < n - 1; ++i) {
      if (sw[i] != 0.0) {
        const double t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t - lm[i] * z[i];
      } else {
        z[i + 1] -= lm[i] * z[i];
      }
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = z[i];
      if (i + 1 < n) t -= u1[i] * z[i + 1];
      if (i + 2 < n) t -= u2[i] * z[i + 2];
      z[i] = t / u[i];
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm = fmax(nrm, fabs(z[i]));
    const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
    for (int i = 0; i < n; ++i) z[i] *= inv;
  }
  for (int i = 0; i < n; ++i) w.V[(size_t)i * nb + s] = z[i];
}

// ------------------------------------------------------------------ 4. finish
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_rr_finish(int n, int o0, int no, int nx, int nb, int want_p, RRWork w, int smem,
                T* __restrict__ YZ, int* __restrict__ dropped) {
  extern __shared__ double dyn[];
  __shared__ int keep_nb[512];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double* V = smem ? dyn : w.V;                   // n x nb
  double* G = smem ? dyn + (size_t)n * nb : w.G;  // nb x nb
  double* Z = w.Z;
  if (smem)
    for (int t = tid; t < n * nb; t += kThreads) V[t] = w.V[t];
  __syncthreads();
  // Cholesky QR, twice
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = tid; t < nb * nb; t += kThreads) {
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      if (b <= a)
        for (int i = 0; i < n; ++i) acc += V[(size_t)i * nb + a] * V[(size_t)i * nb + b];
      G[t] = acc;
    }
    for (int s = tid; s < nb; s += kThreads) keep_nb[s] = 1;
    __syncthreads();
    block_cholesky(G, nb, keep_nb, 0.0);
    for (int i = tid; i < n; i += kThreads) {
      double* v = V + (size_t)i * nb;
      for (int s = 0; s < nb; ++s) {
        double acc = v[s];
        for (int p = 0; p < s; ++p) acc -= G[s * nb + p] * v[p];
        v[s] = acc / G[s * nb + s];
      }
    }
    __syncthreads();
  }
  // V <- H_0 H_1 ... H_{n-3} V
  for (int j = n - 3; j >= 0; --j) {
    const double tj = w.tau[j];
    if (tj == 0.0) continue;
    const int m = n - j - 1;
    const double* v = w.ref + (size_t)j * n + j + 1;
    for (int s = wid; s < nb; s += kWarps) {
      double acc = 0.0;
      for (int i = lane; i < m; i += 32) acc += v[i] * V[(size_t)(j + 1 + i) * nb + s];
      acc = warp_sum(acc) * tj;
      for (int i = lane; i < m; i += 32) V[(size_t)(j + 1 + i) * nb + s] -= acc * v[i];
    }
    __syncthreads();
  }
  // momentum coefficients (Euclidean in the orthonormal basis)
  if (want_p) {
    for (int t = tid; t < n * nb; t += kThreads) Z[t] = (t / nb) < nx ? 0.0 : V[t];
    __syncthreads();
    for (int t = tid; t < nb * nb; t += kThreads) {  // G = V^T Zp
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += V[(size_t)i * nb + a] * Z[(size_t)i * nb + b];
      G[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < n * nb; t += kThreads) {  // Z = Zp - V G
      const int i = t / nb, b = t % nb;
      double acc = Z[t];
      for (int a = 0; a < nb; ++a) acc -= V[(size_t)i * nb + a] * G[a * nb + b];
      w.T1[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < nb * nb; t += kThreads) {  // G = Z^T Z
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      if (b <= a)
        for (int i = 0; i < n; ++i) acc += w.T1[(size_t)i * nb + a] * w.T1[(size_t)i * nb + b];
      G[t] = acc;
    }
    for (int s = tid; s < nb; s += kThreads) keep_nb[s] = 1;
    __syncthreads();
    double gref = 0.0;
    for (int s = 0; s < nb; ++s) gref = fmax(gref, G[s * nb + s]);
    block_cholesky(G, nb, keep_nb, kDrop * fmax(gref, 1e-300));
    for (int i = tid; i < n; i += kThreads) {  // Z <- Z L^-T, dropped columns zero
      const double* zt = w.T1 + (size_t)i * nb;
      double* zr = Z + (size_t)i * nb;
      for (int s = 0; s < nb; ++s) {
        double acc = zt[s];
        for (int p = 0; p < s; ++p) acc -= G[s * nb + p] * zr[p];
        zr[s] = keep_nb[s] ? acc / G[s * nb + s] : 0.0;
      }
    }
    __syncthreads();
  }
  // O rows back to the original basis: y_O <- D L^-T y_O
  for (int a = no - 1; a >= 0; --a) {
    const int i = o0 + a;
    const double inv = 1.0 / w.L[a * no + a];
    for (int c = tid; c < 2 * nb; c += kThreads) {
      if (c >= nb && !want_p) continue;
      double* M_ = c < nb ? V : Z;
      const int cc = c < nb ? c : c - nb;
      double acc = M_[(size_t)i * nb + cc];
      for (int b = a + 1; b < no; ++b) acc -= w.L[b * no + a] * M_[(size_t)(o0 + b) * nb + cc];
      M_[(size_t)i * nb + cc] = acc * inv;
    }
    __syncthreads();
  }
  for (int t = tid; t < n * nb; t += kThreads) {
    const int i = t / nb, s = t % nb;
    const double d = w.dsc[i];
    YZ[(size_t)i * 2 * nb + s] = (T)(V[t] * d);
    YZ[(size_t)i * 2 * nb + nb + s] = want_p ? (T)(Z[t] * d) : T(0);
  }
  if (tid == 0) {
    int dc = 0;
    for (int a = 0; a < n; ++a) dc += !w.keep[a];
    *dropped = dc;
  }
}

}  // namespace

template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool /*fp64*/, double* /*dbg*/) {
  ProfScope ps(kProfRR);
  FF_REQUIRE(d.ns <= 1024 && d.no <= 1024 && d.nb <= 512 && d.o0 + d.no <= d.ns,
             FF_ERR_INVALID_ARG, "Rayleigh-Ritz basis too large");
  const size_t n = d.ns, nb = d.nb, no = d.no;
  const size_t t1 = std::max(n * nb, 2 * n);
  const size_t total = 2 * n * n + no * no + 5 * n + nb + 2 * n * nb + nb * nb + t1 + 6 * n * nb;
  double* p = reinterpret_cast<double*>(work.ensure(sizeof(double) * total + sizeof(int) * n + 256));
  RRWork w;
  w.As = p; p += n * n;
  w.ref = p; p += n * n;
  w.L = p; p += no * no;
  w.dsc = p; p += n;
  w.dg = p; p += n;
  w.e = p; p += n;
  w.e2 = p; p += n;
  w.tau = p; p += n;
  w.lam = p; p += nb;
  w.V = p; p += n * nb;
  w.Z = p; p += n * nb;
  w.G = p; p += nb * nb;
  w.T1 = p; p += t1;
  w.scr = p; p += 6 * n * nb;
  w.keep = reinterpret_cast<int*>(p);
  static bool attr = false;
  if (!attr) {
    FF_CUDA(cudaFuncSetAttribute(k_rr_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    FF_CUDA(cudaFuncSetAttribute(k_rr_finish<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    FF_CUDA(cudaFuncSetAttribute(k_rr_finish<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    attr = true;
  }
  const size_t tri_bytes = sizeof(double) * n * n;
  const bool tri_smem = tri_bytes <= kMaxDynSmem;
  (k_rr_tridiag<<<1, kThreads, tri_smem ? tri_bytes : 0, st>>>(A, B, d.ns, d.o0, d.no, w,
                                                               tri_smem ? 1 : 0),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const size_t eig_bytes = sizeof(double) * (2 * n + 2 * nb) + sizeof(float) * 2 * n;
  (k_rr_eigvals<<<1, kThreads, eig_bytes, st>>>(d.ns, d.nb, w, theta), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_rr_invit<<<(unsigned)((nb + 31) / 32), 32, 0, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const size_t fin_bytes = sizeof(double) * (n * nb + nb * nb);
  const bool fin_smem = fin_bytes <= kMaxDynSmem;
  (k_rr_finish<T><<<1, kThreads, fin_smem ? fin_bytes : 0, st>>>(
       d.ns, d.o0, d.no, d.nx, d.nb, d.want_p, w, fin_smem ? 1 : 0, YZ, dropped),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template void rayleigh_ritz<float>(cudaStream_t, const double*, const double*, RRDims, float*,
                                   double*, int*, Buf&, bool, double*);
template void rayleigh_ritz<double>(cudaStream_t, const double*, const double*, RRDims, double*,
                                    double*, int*, Buf&, bool, double*);

}  // namespace ff
