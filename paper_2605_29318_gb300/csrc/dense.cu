// Small dense Rayleigh-Ritz step of the block eigensolver, one thread block.
//
// The basis S = [X | W | P] (n = nx + nw + np columns) is M-orthonormal except
// for one block O = columns [o0, o0 + no) (the fresh preconditioned residuals W,
// or the whole start block in the first step).  Given the FP64 Gram matrices
// A = S^T H S and B = S^T M S, the nb lowest Ritz pairs of (A, B) -- the trace
// minimisation of Sec. 3.2, Eq. 15 restricted to span S -- are found by:
//   1. scaling the O block by diag(B_OO)^-1/2 and Cholesky B_OO = L L^T with
//      drop (a column whose pivot falls below the drop tolerance depends on the
//      earlier ones and leaves the basis; exactly-zero columns too);
//   2. A <- T^T A T with T = blockdiag(I, L^-T, I): the basis is orthonormal;
//   3. Householder tridiagonalisation of A (lower part keeps the reflectors);
//   4. the nb smallest eigenvalues of the tridiagonal matrix by multisection
//      on Sturm counts (one warp per eigenvalue, 32 probes per round);
//   5. their eigenvectors by inverse iteration on the tridiagonal (LU with
//      partial pivoting), modified Gram-Schmidt inside clusters of close
//      eigenvalues, then the reflectors applied in reverse;
//   6. momentum coefficients Z: the W and P rows of the Ritz vectors,
//      orthogonalised against the Ritz vectors and orthonormalised (Cholesky of
//      Z^T Z) -- so that the next P = S Z is M-orthonormal and M-orthogonal to
//      the next X without another pass over the panels;
//   7. the O rows mapped back through L^-T and the scaling.
// Output YZ = [Y | Z] (n x 2 nb, row-major, context precision) and the Ritz
// values theta (nb, FP64).  Matrices live in shared memory when they fit.
#include "linalg.cuh"

namespace ff {
namespace {

template <class R>
struct Tol;
template <>
struct Tol<float> {
  static constexpr float drop = 1e-6f, eps = 6e-8f, big = 1e30f, tiny = 1e-35f;
};
template <>
struct Tol<double> {
  static constexpr double drop = 1e-13, eps = 1.1e-16, big = 1e300, tiny = 1e-290;
};

constexpr int kThreads = 1024;
constexpr size_t kMaxDynSmem = 212 * 1024;  // 227 KB per block minus the static part
constexpr int kWarps = kThreads / 32;

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread gets the result
template <class R>
__device__ R block_sum(R v, R* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  R t = lane < kWarps ? red[lane] : R(0);
  t = warp_sum(t);
  return t;
}

// Sturm count: number of eigenvalues of the tridiagonal (d, e) below x
template <class R>
__device__ int sturm(const R* d, const R* e2, int n, R x, R pivmin) {
  int c = 0;
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += q < R(0);
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < R(0);
  }
  return c;
}

template <class R>
struct RRShared {
  R red[kWarps];
  int keep_o[1024];
  double dsc[1024];
};

template <class R, class T>
__global__ void __launch_bounds__(kThreads)
    k_rayleigh_ritz(const double* __restrict__ A, const double* __restrict__ B, int n, int o0,
                    int no, int nx, int nb, int want_p, R* __restrict__ gwork, int smem_mats,
                    T* __restrict__ YZ, double* __restrict__ theta, int* __restrict__ dropped) {
  extern __shared__ unsigned char dyn[];
  __shared__ RRShared<R> sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const size_t nn = (size_t)n * n;
  // matrices: in shared memory when they fit, else in the global workspace
  R* base = smem_mats ? reinterpret_cast<R*>(dyn) : gwork;
  R* As = base;                          // n x n
  R* V = As + nn;                        // n x nb  Ritz vectors
  R* Bs = V + (size_t)n * nb;            // no x no
  R* dg = Bs + (size_t)no * no;          // n  diagonal of T
  R* e = dg + n;                         // n  off-diagonal of T
  R* e2 = e + n;                         // n  squares
  R* tau = e2 + n;                       // n  reflector scales
  R* lam = tau + n;                      // nb eigenvalues
  R* vt = lam + nb;                      // n  current reflector
  R* pw = vt + n;                        // n  p / w
  R* G = pw + n;                         // nb x nb
  // global: momentum coefficients Z (n x nb), then per-vector scratch of the
  // tridiagonal LU (5 n each)
  R* Z = gwork + (smem_mats ? 0 : (nn + (size_t)n * nb + (size_t)no * no + 6 * n + nb +
                                   (size_t)nb * nb));
  R* scr = Z + (size_t)n * nb;

  // ---- 1. load, scale the O block, Cholesky of B_OO
  for (int i = tid; i < n; i += kThreads) {
    double s = 1.0;
    if (i >= o0 && i < o0 + no) {
      const double bii = B[(size_t)i * n + i];
      const int k = bii > 1e-280 && isfinite(bii);
      sh.keep_o[i - o0] = k;
      s = k ? 1.0 / sqrt(bii) : 0.0;
    }
    sh.dsc[i] = s;
  }
  __syncthreads();
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    As[t] = (R)(0.5 * (A[t] + A[(size_t)j * n + i]) * sh.dsc[i] * sh.dsc[j]);
  }
  for (int t = tid; t < no * no; t += kThreads) {
    const int a = t / no, b = t % no;
    const int i = o0 + a, j = o0 + b;
    const double v = 0.5 * (B[(size_t)i * n + j] + B[(size_t)j * n + i]) * sh.dsc[i] * sh.dsc[j];
    Bs[t] = (sh.keep_o[a] && sh.keep_o[b]) ? (R)v : (R)(a == b ? 1 : 0);
  }
  __syncthreads();
  for (int j = 0; j < no; ++j) {
    if (tid == 0) {
      const R piv = Bs[j * no + j];
      const int k = sh.keep_o[j] && piv > Tol<R>::drop;
      sh.keep_o[j] = k;
      Bs[j * no + j] = k ? sqrt(piv) : R(1);
    }
    __syncthreads();
    const R ljj = Bs[j * no + j];
    const int kj = sh.keep_o[j];
    for (int i = j + 1 + tid; i < no; i += kThreads) Bs[i * no + j] = kj ? Bs[i * no + j] / ljj : R(0);
    __syncthreads();
    const int m = no - j - 1;
    if (kj)
      for (int t = tid; t < m * m; t += kThreads) {
        const int i = j + 1 + t / m, l = j + 1 + t % m;
        if (l <= i) Bs[i * no + l] -= Bs[i * no + j] * Bs[l * no + j];
      }
    __syncthreads();
  }
  // ---- 2. A <- T^T A T on the O rows, then the O columns
  for (int a = 0; a < no; ++a) {
    const int i = o0 + a;
    const R inv = R(1) / Bs[a * no + a];
    for (int c = tid; c < n; c += kThreads) {
      R acc = As[(size_t)i * n + c];
      for (int b = 0; b < a; ++b) acc -= Bs[a * no + b] * As[(size_t)(o0 + b) * n + c];
      As[(size_t)i * n + c] = acc * inv;
    }
    __syncthreads();
  }
  for (int a = 0; a < no; ++a) {
    const int i = o0 + a;
    const R inv = R(1) / Bs[a * no + a];
    for (int r = tid; r < n; r += kThreads) {
      R acc = As[(size_t)r * n + i];
      for (int b = 0; b < a; ++b) acc -= Bs[a * no + b] * As[(size_t)r * n + o0 + b];
      As[(size_t)r * n + i] = acc * inv;
    }
    __syncthreads();
  }
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    const bool di = i >= o0 && i < o0 + no && !sh.keep_o[i - o0];
    const bool dj = j >= o0 && j < o0 + no && !sh.keep_o[j - o0];
    if (di || dj) As[t] = (i == j) ? Tol<R>::big : R(0);
    else if (i > j) As[t] = R(0.5) * (As[t] + As[(size_t)j * n + i]);
  }
  __syncthreads();
  for (size_t t = tid; t < nn; t += kThreads) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (i < j) As[t] = As[(size_t)j * n + i];
  }
  __syncthreads();

  // ---- 3. Householder tridiagonalisation (reflector j stored in column j below the diagonal)
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    R part = R(0);
    for (int i = tid; i < m; i += kThreads) {
      const R x = As[(size_t)(j + 1 + i) * n + j];
      part += x * x;
    }
    const R ss = block_sum(part, sh.red);
    const R x0 = As[(size_t)(j + 1) * n + j];
    const R alpha = sqrt(ss);
    __syncthreads();
    if (!(alpha > Tol<R>::tiny)) {
      if (tid == 0) {
        tau[j] = R(0);
        e[j] = x0;
        dg[j] = As[(size_t)j * n + j];
      }
      __syncthreads();
      continue;
    }
    const R beta = x0 >= R(0) ? -alpha : alpha;
    const R tj = (beta - x0) / beta;
    const R scale = R(1) / (x0 - beta);
    for (int i = tid; i < m; i += kThreads) {
      const R v = i == 0 ? R(1) : As[(size_t)(j + 1 + i) * n + j] * scale;
      vt[i] = v;
      As[(size_t)(j + 1 + i) * n + j] = v;
    }
    if (tid == 0) {
      tau[j] = tj;
      e[j] = beta;
      dg[j] = As[(size_t)j * n + j];
    }
    __syncthreads();
    // p = tau A22 v
    for (int i = wid; i < m; i += kWarps) {
      const R* row = As + (size_t)(j + 1 + i) * n + (j + 1);
      R acc = R(0);
      for (int l = lane; l < m; l += 32) acc += row[l] * vt[l];
      acc = warp_sum(acc);
      if (lane == 0) pw[i] = tj * acc;
    }
    __syncthreads();
    R kp = R(0);
    for (int i = tid; i < m; i += kThreads) kp += pw[i] * vt[i];
    const R K = R(0.5) * tj * block_sum(kp, sh.red);
    __syncthreads();
    for (int i = tid; i < m; i += kThreads) pw[i] -= K * vt[i];
    __syncthreads();
    for (int t = tid; t < m * m; t += kThreads) {
      const int i = t / m, l = t % m;
      As[(size_t)(j + 1 + i) * n + (j + 1 + l)] -= vt[i] * pw[l] + pw[i] * vt[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = As[(size_t)(n - 2) * n + (n - 2)];
      e[n - 2] = As[(size_t)(n - 1) * n + (n - 2)];
      tau[n - 2] = R(0);
    }
    dg[n - 1] = As[(size_t)(n - 1) * n + (n - 1)];
    e[n - 1] = R(0);
  }
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) e2[i] = e[i] * e[i];
  __syncthreads();

  // ---- 4. the nb smallest eigenvalues by multisection
  R lo = R(0), hi = R(0), emax = R(0);
  for (int i = 0; i < n; ++i) {
    const R r = (i > 0 ? fabs(e[i - 1]) : R(0)) + (i + 1 < n ? fabs(e[i]) : R(0));
    const R a = dg[i] - r, b = dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
    emax = fmax(emax, e2[i]);
  }
  const R span = fmax(hi - lo, R(1e-30));
  lo -= span * R(1e-6);
  hi += span * R(1e-6);
  const R pivmin = fmax(Tol<R>::tiny, Tol<R>::eps * Tol<R>::eps * emax);
  for (int s = wid; s < nb; s += kWarps) {
    R a = lo, b = hi;
    for (int round = 0; round < 40; ++round) {
      const R x = a + (b - a) * (R)(lane + 1) / R(33);
      const int cnt = sturm(dg, e2, n, x, pivmin);
      const unsigned above = __ballot_sync(0xffffffffu, cnt >= s + 1);
      const int first = above ? __ffs(above) - 1 : 32;
      const R na = first == 0 ? a : a + (b - a) * (R)first / R(33);
      const R nbv = first == 32 ? b : a + (b - a) * (R)(first + 1) / R(33);
      a = __shfl_sync(0xffffffffu, na, 0);
      b = __shfl_sync(0xffffffffu, nbv, 0);
      if (b - a <= R(4) * Tol<R>::eps * fmax(fabs(a), fabs(b)) + pivmin) break;
    }
    if (lane == 0) lam[s] = R(0.5) * (a + b);
  }
  __syncthreads();

  // ---- 5. eigenvectors of the tridiagonal: inverse iteration, one thread per vector
  for (int s = tid; s < nb; s += kThreads) {
    R* u = scr + (size_t)s * 5 * n;   // diag of U
    R* u1 = u + n;                    // first super-diagonal
    R* u2 = u1 + n;                   // second super-diagonal (pivoting fill)
    R* lm = u2 + n;                   // multipliers
    R* z = lm + n;                    // the vector (also written to V)
    // perturb the shift slightly so that T - lambda I is not exactly singular
    const R shift = lam[s] + Tol<R>::eps * fmax(fabs(lam[s]), span * R(1e-3)) * R(4);
    // LU with partial pivoting of the tridiagonal T - shift I (rows i, i+1)
    R a_i = dg[0] - shift, b_i = n > 1 ? e[0] : R(0), c_i = R(0);
    for (int i = 0; i < n - 1; ++i) {
      const R sub = e[i];
      const R d1 = dg[i + 1] - shift;
      const R e1 = i + 2 < n ? e[i + 1] : R(0);
      if (fabs(a_i) >= fabs(sub)) {
        const R piv_ = fabs(a_i) < pivmin ? (a_i < R(0) ? -pivmin : pivmin) : a_i;
        const R l = sub / piv_;
        u[i] = piv_; u1[i] = b_i; u2[i] = c_i; lm[i] = l;
        a_i = d1 - l * b_i;
        b_i = e1 - l * c_i;
        c_i = R(0);
        z[i] = R(0);  // no row swap at step i
      } else {
        const R l = a_i / sub;
        u[i] = sub; u1[i] = d1; u2[i] = e1; lm[i] = l;
        const R na = b_i - l * d1;
        const R nb_ = c_i - l * e1;
        a_i = na;
        b_i = nb_;
        c_i = R(0);
        z[i] = R(1);  // swapped
      }
    }
    u[n - 1] = fabs(a_i) < pivmin ? (a_i < R(0) ? -pivmin : pivmin) : a_i;
    u1[n - 1] = R(0);
    u2[n - 1] = R(0);
    // the row-swap flags go to V's column s until the vector itself is formed
    for (int i = 0; i < n; ++i) V[(size_t)i * nb + s] = z[i];
    // start vector: deterministic pseudo-random
    unsigned int h = 2166136261u ^ (unsigned)s * 16777619u;
    for (int i = 0; i < n; ++i) {
      h = h * 1664525u + 1013904223u;
      z[i] = R(0.5) + (R)((h >> 8) & 0xffff) / R(65536);
    }
    for (int iter = 0; iter < 3; ++iter) {
      // forward: apply the row operations (with the recorded swaps)
      for (int i = 0; i < n - 1; ++i) {
        if (V[(size_t)i * nb + s] != R(0)) {
          const R t = z[i];
          z[i] = z[i + 1];
          z[i + 1] = t - lm[i] * z[i];
        } else {
          z[i + 1] -= lm[i] * z[i];
        }
      }
      // back substitution with U (upper, bandwidth 2)
      R nrm = R(0);
      for (int i = n - 1; i >= 0; --i) {
        R t = z[i];
        if (i + 1 < n) t -= u1[i] * z[i + 1];
        if (i + 2 < n) t -= u2[i] * z[i + 2];
        z[i] = t / u[i];
      }
      for (int i = 0; i < n; ++i) nrm = fmax(nrm, fabs(z[i]));
      const R inv = nrm > R(0) ? R(1) / nrm : R(1);
      for (int i = 0; i < n; ++i) z[i] *= inv;
    }
  }
  __syncthreads();
  for (int t = tid; t < n * nb; t += kThreads) {
    const int i = t / nb, s = t % nb;
    V[t] = scr[(size_t)s * 5 * n + 4 * n + i];
  }
  __syncthreads();
  // orthonormalise the tridiagonal eigenvectors as a block: Cholesky QR, twice
  // (inverse iteration leaves vectors of close eigenvalues slightly
  //  non-orthogonal; two passes of V <- V chol(V^T V)^-T restore it)
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = tid; t < nb * nb; t += kThreads) {
      const int a = t / nb, b = t % nb;
      R acc = R(0);
      if (b <= a)
        for (int i = 0; i < n; ++i) acc += V[(size_t)i * nb + a] * V[(size_t)i * nb + b];
      G[t] = acc;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      if (tid == 0) {
        const R piv = G[j * nb + j];
        G[j * nb + j] = piv > R(0) ? sqrt(piv) : R(1);
      }
      __syncthreads();
      const R ljj = G[j * nb + j];
      for (int i = j + 1 + tid; i < nb; i += kThreads) G[i * nb + j] /= ljj;
      __syncthreads();
      const int m = nb - j - 1;
      for (int t = tid; t < m * m; t += kThreads) {
        const int i = j + 1 + t / m, l = j + 1 + t % m;
        if (l <= i) G[i * nb + l] -= G[i * nb + j] * G[l * nb + j];
      }
      __syncthreads();
    }
    for (int i = tid; i < n; i += kThreads) {
      R* v = V + (size_t)i * nb;
      for (int s = 0; s < nb; ++s) {
        R acc = v[s];
        for (int p = 0; p < s; ++p) acc -= G[s * nb + p] * v[p];
        v[s] = acc / G[s * nb + s];
      }
    }
    __syncthreads();
  }
  // back-transform: V <- H_0 H_1 ... H_{n-3} V
  for (int j = n - 3; j >= 0; --j) {
    const int m = n - j - 1;
    const R tj = tau[j];
    if (tj == R(0)) continue;
    for (int s = wid; s < nb; s += kWarps) {
      R acc = R(0);
      for (int i = lane; i < m; i += 32) acc += As[(size_t)(j + 1 + i) * n + j] * V[(size_t)(j + 1 + i) * nb + s];
      acc = warp_sum(acc) * tj;
      for (int i = lane; i < m; i += 32) V[(size_t)(j + 1 + i) * nb + s] -= acc * As[(size_t)(j + 1 + i) * n + j];
    }
    __syncthreads();
  }
  for (int s = tid; s < nb; s += kThreads) theta[s] = (double)lam[s];

  // ---- 6. momentum coefficients (Euclidean in the orthonormal basis)
  if (want_p) {
    for (int t = tid; t < n * nb; t += kThreads) Z[t] = (t / nb) < nx ? R(0) : V[t];
    __syncthreads();
    for (int t = tid; t < nb * nb; t += kThreads) {   // G = V^T Zp
      const int a = t / nb, b = t % nb;
      R acc = R(0);
      for (int i = 0; i < n; ++i) acc += V[(size_t)i * nb + a] * Z[(size_t)i * nb + b];
      G[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < n * nb; t += kThreads) {   // Z = Zp - V G (written to the o-scratch)
      const int i = t / nb, b = t % nb;
      R acc = Z[t];
      for (int a = 0; a < nb; ++a) acc -= V[(size_t)i * nb + a] * G[a * nb + b];
      scr[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < n * nb; t += kThreads) Z[t] = scr[t];
    __syncthreads();
    for (int t = tid; t < nb * nb; t += kThreads) {   // G = Z^T Z
      const int a = t / nb, b = t % nb;
      R acc = R(0);
      for (int i = 0; i < n; ++i) acc += Z[(size_t)i * nb + a] * Z[(size_t)i * nb + b];
      G[t] = acc;
    }
    __syncthreads();
    // Cholesky with drop, then Z <- Z L^-T (row-wise forward solves)
    for (int j = 0; j < nb; ++j) {
      if (tid == 0) {
        const R piv = G[j * nb + j];
        const R ref = fmax(R(1e-30), G[0]);
        const int k = piv > Tol<R>::drop * ref && piv > R(0);
        sh.keep_o[j] = k;   // keep_o reused: O block is finished
        G[j * nb + j] = k ? sqrt(piv) : R(1);
      }
      __syncthreads();
      const R ljj = G[j * nb + j];
      const int kj = sh.keep_o[j];
      for (int i = j + 1 + tid; i < nb; i += kThreads) G[i * nb + j] = kj ? G[i * nb + j] / ljj : R(0);
      __syncthreads();
      const int m = nb - j - 1;
      if (kj)
        for (int t = tid; t < m * m; t += kThreads) {
          const int i = j + 1 + t / m, l = j + 1 + t % m;
          if (l <= i) G[i * nb + l] -= G[i * nb + j] * G[l * nb + j];
        }
      __syncthreads();
    }
    for (int i = tid; i < n; i += kThreads) {
      R* z = Z + (size_t)i * nb;
      for (int s = 0; s < nb; ++s) {
        R acc = z[s];
        for (int p = 0; p < s; ++p) acc -= G[s * nb + p] * z[p];
        z[s] = sh.keep_o[s] ? acc / G[s * nb + s] : R(0);
      }
    }
    __syncthreads();
  }
  // ---- 7. O rows back to the original basis: y_O <- D L^-T y_O
  // (keep_o was overwritten by the momentum Cholesky; dropped O columns have
  //  zero rows in V and Z because their rows/columns of A were decoupled)
  for (int a = no - 1; a >= 0; --a) {
    const int i = o0 + a;
    const R inv = R(1) / Bs[a * no + a];
    for (int c = tid; c < 2 * nb; c += kThreads) {
      R* M_ = c < nb ? V : Z;
      const int cc = c < nb ? c : c - nb;
      R acc = M_[(size_t)i * nb + cc];
      for (int b = a + 1; b < no; ++b) acc -= Bs[b * no + a] * M_[(size_t)(o0 + b) * nb + cc];
      M_[(size_t)i * nb + cc] = acc * inv;
    }
    __syncthreads();
  }
  for (int t = tid; t < n * nb; t += kThreads) {
    const int i = t / nb, s = t % nb;
    const double d = sh.dsc[i];
    YZ[(size_t)i * 2 * nb + s] = (T)((double)V[t] * d);
    YZ[(size_t)i * 2 * nb + nb + s] = want_p ? (T)((double)Z[t] * d) : T(0);
  }
  if (tid == 0) {
    int dcount = 0;
    for (int a = 0; a < no; ++a) dcount += sh.dsc[o0 + a] == 0.0;
    *dropped = dcount;
  }
}

}  // namespace

template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool /*fp64*/) {
  ProfScope ps(kProfRR);
  FF_REQUIRE(d.ns <= 1024 && d.no <= 1024 && d.o0 + d.no <= d.ns, FF_ERR_INVALID_ARG,
             "Rayleigh-Ritz basis too large");
  // the small dense problem is solved in FP64 in every precision mode: its
  // spectrum spans the whole range of the basis' Rayleigh quotients, and the
  // small eigenvalues need relative accuracy
  using R = double;
  const size_t n = d.ns, nb = d.nb, no = d.no;
  const size_t mats = n * n + n * nb + no * no + 6 * n + nb + nb * nb;
  const size_t glob = n * nb + 5 * n * nb;
  const size_t bytes = sizeof(R) * mats;
  const bool in_smem = bytes <= kMaxDynSmem;
  R* w = reinterpret_cast<R*>(work.ensure(sizeof(R) * (mats + glob + 64)));
  static bool attr = false;
  if (!attr) {
    FF_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz<R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    attr = true;
  }
  (k_rayleigh_ritz<R, T><<<1, kThreads, in_smem ? bytes : 0, st>>>(
      A, B, d.ns, d.o0, d.no, d.nx, d.nb, d.want_p, w, in_smem ? 1 : 0, YZ, theta, dropped), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template void rayleigh_ritz<float>(cudaStream_t, const double*, const double*, RRDims, float*,
                                   double*, int*, Buf&, bool);
template void rayleigh_ritz<double>(cudaStream_t, const double*, const double*, RRDims, double*,
                                    double*, int*, Buf&, bool);

}  // namespace ff
