// Small dense Rayleigh-Ritz step of the block eigensolver, one thread block.
//
// Given the Gram matrices A = S^T H S and B = S^T M S of the basis
// S = [X | W | P] (ns columns), find the nb lowest Ritz pairs of the pencil
// (A, B) (the trace minimisation of Sec. 3.2, Eq. 15, restricted to span S):
//   1. symmetric diagonal scaling D = diag(B)^-1/2; exactly-zero columns dropped
//   2. Cholesky D B D = L L^T; a column whose pivot falls below the drop
//      tolerance is linearly dependent on the earlier ones and is dropped
//   3. C = L^-1 (D A D) L^-T, cyclic Jacobi (round-robin parallel ordering,
//      rotation when |c_pq| > tol sqrt(|c_pp c_qq|)) -> eigenpairs of C
//   4. Y = D L^-T V for the nb smallest eigenvalues (ascending)
//   5. momentum coefficients Z: the W and P rows of Y, made M-orthogonal to
//      the new X = S Y and M-orthonormalised (Cholesky of Z^T B Z), all in the
//      small space, so that P = S Z needs no further pass over the panels.
// Output YZ = [Y | Z] (ns x 2 nb, row-major) and theta (nb) in FP64.
#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kMaxN = 1024;

template <class R>
struct RRTol;
template <>
struct RRTol<float> {
  static constexpr float drop = 1e-6f, jac = 1e-6f, big = 1e30f;
};
template <>
struct RRTol<double> {
  static constexpr double drop = 1e-13, jac = 1e-14, big = 1e300;
};

// in-place right-looking Cholesky of the lower triangle of an n x n matrix;
// dropped columns get a unit pivot and zero sub-column; keep[] updated
template <class R>
__device__ void block_cholesky(R* L, int n, int* keep, R drop_tol) {
  __shared__ int s_keep;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      R piv = L[j * n + j];
      int k = keep[j] && (piv > drop_tol);
      keep[j] = k;
      L[j * n + j] = k ? sqrt(piv) : R(1);
      s_keep = k;
    }
    __syncthreads();
    const R ljj = L[j * n + j];
    const int kj = s_keep;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      L[i * n + j] = kj ? L[i * n + j] / ljj : R(0);
    __syncthreads();
    const int m = n - j - 1;
    if (kj && m > 0) {
      for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int i = j + 1 + t / m, l = j + 1 + t % m;
        if (l <= i) L[i * n + l] -= L[i * n + j] * L[l * n + j];
      }
    }
    __syncthreads();
  }
}

// X (n x m, row-major, leading dim ldx) <- L^-1 X, L lower (n x n)
template <class R>
__device__ void block_forward(const R* L, int n, R* X, int m, int ldx) {
  for (int i = 0; i < n; ++i) {
    const R inv = R(1) / L[i * n + i];
    for (int c = threadIdx.x; c < m; c += blockDim.x) X[i * ldx + c] *= inv;
    __syncthreads();
    const int rows = n - i - 1;
    for (int t = threadIdx.x; t < rows * m; t += blockDim.x) {
      const int r = i + 1 + t / m, c = t % m;
      X[r * ldx + c] -= L[r * n + i] * X[i * ldx + c];
    }
    __syncthreads();
  }
}

// X (n x m) <- L^-T X
template <class R>
__device__ void block_backward_t(const R* L, int n, R* X, int m, int ldx) {
  for (int i = n - 1; i >= 0; --i) {
    const R inv = R(1) / L[i * n + i];
    for (int c = threadIdx.x; c < m; c += blockDim.x) X[i * ldx + c] *= inv;
    __syncthreads();
    for (int t = threadIdx.x; t < i * m; t += blockDim.x) {
      const int r = t / m, c = t % m;
      X[r * ldx + c] -= L[i * n + r] * X[i * ldx + c];
    }
    __syncthreads();
  }
}

// C (n x m) = A (n x k) * B (k x m), all row-major
template <class R>
__device__ void block_gemm(const R* A, int lda, const R* B, int ldb, R* C, int ldc, int n, int k,
                           int m, bool transA = false) {
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    R s = R(0);
    if (!transA)
      for (int p = 0; p < k; ++p) s += A[i * lda + p] * B[p * ldb + j];
    else
      for (int p = 0; p < k; ++p) s += A[p * lda + i] * B[p * ldb + j];
    C[i * ldc + j] = s;
  }
  __syncthreads();
}

template <class R>
__device__ void jacobi(R* Cm, R* V, int n) {
  __shared__ R cs[kMaxN];
  __shared__ R sn[kMaxN];
  __shared__ int pp[kMaxN / 2], qq[kMaxN / 2];
  __shared__ int rot;
  const int m = n + (n & 1);
  const int half = m / 2;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) V[t] = (t / n == t % n) ? R(1) : R(0);
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) rot = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        int p, q;
        if (t == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + t) % (m - 1);
          q = (r - t + (m - 1)) % (m - 1);
        }
        if (p > q) { int x = p; p = q; q = x; }
        R c = R(1), s = R(0);
        if (q < n) {
          const R apq = Cm[p * n + q];
          const R app = Cm[p * n + p], aqq = Cm[q * n + q];
          if (fabs(apq) > RRTol<R>::jac * sqrt(fabs(app * aqq)) && apq != R(0)) {
            const R th = (aqq - app) / (R(2) * apq);
            const R tt = (th >= R(0) ? R(1) : R(-1)) / (fabs(th) + sqrt(th * th + R(1)));
            c = R(1) / sqrt(tt * tt + R(1));
            s = tt * c;
            rot = 1;
          }
        }
        pp[t] = p;
        qq[t] = q;
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      // rows p, q  (C <- J^T C)
      for (int t = threadIdx.x; t < half * n; t += blockDim.x) {
        const int pr = t / n, j = t % n;
        const int p = pp[pr], q = qq[pr];
        if (q >= n || sn[pr] == R(0)) continue;
        const R c = cs[pr], s = sn[pr];
        const R a = Cm[p * n + j], b = Cm[q * n + j];
        Cm[p * n + j] = c * a - s * b;
        Cm[q * n + j] = s * a + c * b;
      }
      __syncthreads();
      // columns p, q (C <- C J) and V <- V J
      for (int t = threadIdx.x; t < half * n; t += blockDim.x) {
        const int pr = t / n, j = t % n;
        const int p = pp[pr], q = qq[pr];
        if (q >= n || sn[pr] == R(0)) continue;
        const R c = cs[pr], s = sn[pr];
        const R a = Cm[j * n + p], b = Cm[j * n + q];
        Cm[j * n + p] = c * a - s * b;
        Cm[j * n + q] = s * a + c * b;
        const R va = V[j * n + p], vb = V[j * n + q];
        V[j * n + p] = c * va - s * vb;
        V[j * n + q] = s * va + c * vb;
      }
      __syncthreads();
    }
    if (rot == 0) break;
    __syncthreads();
  }
}

template <class R, class T>
__global__ void __launch_bounds__(1024)
    k_rayleigh_ritz(const double* __restrict__ A, const double* __restrict__ B, int n, int nx,
                    int nb, int want_p, R* __restrict__ work, T* __restrict__ YZ,
                    double* __restrict__ theta, int* __restrict__ dropped) {
  __shared__ int keep[kMaxN];
  __shared__ double dsc[kMaxN];
  __shared__ R ev[kMaxN];
  __shared__ int order[kMaxN];
  const size_t nn = (size_t)n * n;
  R* Ls = work;           // scaled B -> Cholesky factor
  R* Bo = Ls + nn;        // original B
  R* Cm = Bo + nn;        // projected A
  R* V = Cm + nn;         // eigenvectors / temp
  R* Y = V + nn;          // n x nb
  R* Z = Y + (size_t)n * nb;
  R* T1 = Z + (size_t)n * nb;
  R* G = T1 + (size_t)n * nb;  // nb x nb

  // 1. scaling from diag(B) (in FP64, before any narrowing)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double bii = B[(size_t)i * n + i];
    const int k = bii > 1e-280 && isfinite(bii);
    keep[i] = k;
    dsc[i] = k ? 1.0 / sqrt(bii) : 0.0;
  }
  __syncthreads();
  for (size_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const double b = 0.5 * (B[t] + B[(size_t)j * n + i]);
    const double a = 0.5 * (A[t] + A[(size_t)j * n + i]);
    Bo[t] = (R)b;
    const double s = dsc[i] * dsc[j];
    Ls[t] = (keep[i] && keep[j]) ? (R)(b * s) : (R)(i == j ? 1.0 : 0.0);
    Cm[t] = (keep[i] && keep[j]) ? (R)(a * s) : R(0);
  }
  __syncthreads();
  // 2. Cholesky with drop
  block_cholesky<R>(Ls, n, keep, RRTol<R>::drop);
  // 3. C = L^-1 A L^-1^T
  block_forward<R>(Ls, n, Cm, n, n);
  for (size_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    V[t] = Cm[(size_t)j * n + i];
  }
  __syncthreads();
  block_forward<R>(Ls, n, V, n, n);
  for (size_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    R v = R(0.5) * (V[t] + V[(size_t)j * n + i]);
    if (!keep[i] || !keep[j]) v = (i == j) ? RRTol<R>::big : R(0);
    Cm[t] = v;
  }
  __syncthreads();
  // 4. eigenpairs
  jacobi<R>(Cm, V, n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) ev[i] = Cm[(size_t)i * n + i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = 0;
    const R e = ev[i];
    for (int j = 0; j < n; ++j) r += (ev[j] < e) || (ev[j] == e && j < i);
    order[r] = i;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
    const int i = t / nb, s = t % nb;
    Y[t] = V[(size_t)i * n + order[s]];
  }
  __syncthreads();
  block_backward_t<R>(Ls, n, Y, nb, nb);
  for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
    const int i = t / nb;
    Y[t] = (R)((double)Y[t] * dsc[i]);
  }
  for (int s = threadIdx.x; s < nb; s += blockDim.x) theta[s] = (double)ev[order[s]];
  if (threadIdx.x == 0) {
    int d = 0;
    for (int i = 0; i < n; ++i) d += !keep[i];
    *dropped = d;
  }
  __syncthreads();
  // 5. momentum coefficients
  if (want_p) {
    for (int t = threadIdx.x; t < n * nb; t += blockDim.x) Z[t] = (t / nb) < nx ? R(0) : Y[t];
    __syncthreads();
    block_gemm<R>(Bo, n, Z, nb, T1, nb, n, n, nb);          // T1 = B Zp
    block_gemm<R>(Y, nb, T1, nb, G, nb, nb, n, nb, true);   // G = Y^T B Zp
    for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {  // Z = Zp - Y G
      const int i = t / nb, s = t % nb;
      R acc = Z[t];
      for (int p = 0; p < nb; ++p) acc -= Y[i * nb + p] * G[p * nb + s];
      T1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * nb; t += blockDim.x) Z[t] = T1[t];
    __syncthreads();
    block_gemm<R>(Bo, n, Z, nb, T1, nb, n, n, nb);          // T1 = B Z
    block_gemm<R>(Z, nb, T1, nb, G, nb, nb, n, nb, true);   // G = Z^T B Z
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
      const int i = t / nb, j = t % nb;
      G[t] = R(0.5) * (G[t] + G[j * nb + i]);
    }
    // scale, then Cholesky with drop (keep[] reused for the nb columns)
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const R gii = G[i * nb + i];
      keep[i] = gii > R(0);
      dsc[i] = gii > R(0) ? 1.0 / sqrt((double)gii) : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
      const int i = t / nb, j = t % nb;
      G[t] = (keep[i] && keep[j]) ? (R)((double)G[t] * dsc[i] * dsc[j]) : (R)(i == j ? 1 : 0);
    }
    for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
      const int s = t % nb;
      Z[t] = (R)((double)Z[t] * dsc[s]);
    }
    __syncthreads();
    block_cholesky<R>(G, nb, keep, RRTol<R>::drop);
    // Z <- Z L^-T  : each row z solves L z_new^T = z^T
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      R* z = Z + (size_t)i * nb;
      for (int s = 0; s < nb; ++s) {
        R acc = z[s];
        for (int p = 0; p < s; ++p) acc -= G[s * nb + p] * z[p];
        z[s] = keep[s] ? acc / G[s * nb + s] : R(0);
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * nb; t += blockDim.x) {
    const int i = t / nb, s = t % nb;
    YZ[(size_t)i * 2 * nb + s] = (T)Y[t];
    YZ[(size_t)i * 2 * nb + nb + s] = want_p ? (T)Z[t] : T(0);
  }
}

}  // namespace

template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool fp64) {
  FF_REQUIRE(d.ns <= kMaxN, FF_ERR_INVALID_ARG, "Rayleigh-Ritz basis too large");
  const size_t nn = (size_t)d.ns * d.ns;
  const size_t elems = 4 * nn + 3 * (size_t)d.ns * d.nb + (size_t)d.nb * d.nb + 64;
  if (fp64) {
    double* w = reinterpret_cast<double*>(work.ensure(sizeof(double) * elems));
    k_rayleigh_ritz<double, T><<<1, 1024, 0, st>>>(A, B, d.ns, d.nx, d.nb, d.want_p, w, YZ, theta,
                                                  dropped);
  } else {
    float* w = reinterpret_cast<float*>(work.ensure(sizeof(float) * elems));
    k_rayleigh_ritz<float, T><<<1, 1024, 0, st>>>(A, B, d.ns, d.nx, d.nb, d.want_p, w, YZ, theta,
                                                 dropped);
  }
  FF_LAUNCH_CHECK();
}

template void rayleigh_ritz<float>(cudaStream_t, const double*, const double*, RRDims, float*,
                                   double*, int*, Buf&, bool);
template void rayleigh_ritz<double>(cudaStream_t, const double*, const double*, RRDims, double*,
                                    double*, int*, Buf&, bool);

}  // namespace ff
