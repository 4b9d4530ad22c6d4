// Small dense Rayleigh-Ritz step of the block eigensolver (FP64).
//
// The basis S = [X | W | P] (n = nx + nw + np columns) is M-orthonormal except
// for one block O = columns [o0, o0 + no) (the fresh preconditioned residuals W,
// or the whole start block in the first step).  Given the FP64 Gram matrices
// A = S^T H S and B = S^T M S, the nb lowest Ritz pairs of (A, B) -- the trace
// minimisation of Sec. 3.2, Eq. 15 restricted to span S -- are found by a
// chain of launches that hand their results over in a global workspace.
// GB300 runs FP64 at a small fraction of its FP32 rate on each SM, so every
// stage that can be spread over SMs is:
//   k_rr_tridiag        (one block) scale the O block by diag(B_OO)^-1/2,
//                       Cholesky B_OO = L L^T with drop (dependent or empty
//                       columns leave the basis, as do columns outside O whose
//                       B_ii is not ~1: empty momentum directions),
//                       A <- T^T A T with T = blockdiag(I, L^-T, I); for bases
//                       too large for the cluster it also tridiagonalises;
//   k_rr_house_cluster  Householder tridiagonalisation of A by an 8-block
//                       thread-block cluster, rows spread over the blocks'
//                       shared memory;
//   k_rr_eigvals_mc     the nb smallest eigenvalues of the tridiagonal matrix,
//                       one warp each: FP64 multisection on a division-free
//                       Sturm count;
//   k_rr_invit_sm       their eigenvectors by inverse iteration on the
//                       tridiagonal (LU with partial pivoting), one block each;
//   k_rr_cholqr         Cholesky QR (twice) of those vectors;
//   k_rr_backtransform  the Householder reflectors applied in reverse, one
//                       warp per vector;
//   k_rr_momentum       the momentum coefficients Z (the W and P rows of the
//                       Ritz vectors, orthogonalised against them and
//                       orthonormalised -- the next P = S Z is then
//                       M-orthonormal and M-orthogonal to the next X), and the
//                       O rows mapped back through L^-T and the scaling.
// Output YZ = [Y | Z] (n x 2 nb, row-major, context precision) and the Ritz
// values theta (nb).  FP64 throughout: the spectrum of A spans the whole range
// of the basis' Rayleigh quotients and the small eigenvalues need relative
// accuracy.
#include <cooperative_groups.h>

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
  double *As, *ref, *L, *dsc, *dg, *e, *e2, *tau, *lam, *V, *Z, *G, *T1, *scr, *C, *U;
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
                 RRWork w, int smem, int do_house, double drop) {
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
  // Second projection of the O block against the rest, in coefficient space.
  // The O columns arrive M-projected against the others once, on the
  // N-vectors; once they are mostly made of the other columns (a converging
  // block) that projection leaves a coupling of order eps / |remainder|.  With
  // C = B_{rest,O} (scaled) and T = [I, -C; 0, I], A <- T^T A T and
  // B_OO <- B_OO - C^T C take it out ("twice is enough"); the rest-rest block
  // of B is the identity to rounding.
  const int o1 = o0 + no;
  for (int t = tid; t < n * no; t += kThreads) {
    const int i = t / no, j = o0 + t % no;
    const bool in_o = i >= o0 && i < o1;
    w.C[t] = (!in_o && w.keep[i] && w.keep[j])
                 ? 0.5 * (B[(size_t)i * n + j] + B[(size_t)j * n + i]) * w.dsc[i] * w.dsc[j]
                 : 0.0;
  }
  __syncthreads();
  for (int t = tid; t < n * no; t += kThreads) {  // U = A_{rest,rest} C
    const int i = t / no, a = t % no;
    double acc = 0.0;
    if (i < o0 || i >= o1)
      for (int r = 0; r < n; ++r)
        if (r < o0 || r >= o1) acc += As[(size_t)i * n + r] * w.C[r * no + a];
    w.U[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < no * no; t += kThreads) {
    const int a = t / no, b = t % no, i = o0 + a, j = o0 + b;
    double cc = 0.0, acc = As[(size_t)i * n + j];
    for (int r = 0; r < n; ++r) {
      if (r >= o0 && r < o1) continue;
      const double ca = w.C[r * no + a], cb = w.C[r * no + b];
      cc += ca * cb;
      acc += ca * w.U[r * no + b] - ca * As[(size_t)r * n + j] - As[(size_t)i * n + r] * cb;
    }
    const double v = 0.5 * (B[(size_t)i * n + j] + B[(size_t)j * n + i]) * w.dsc[i] * w.dsc[j] - cc;
    w.L[t] = (w.keep[i] && w.keep[j]) ? v : (a == b ? 1.0 : 0.0);
    As[(size_t)i * n + j] = acc;
  }
  __syncthreads();
  for (int t = tid; t < n * no; t += kThreads) {
    const int i = t / no, j = o0 + t % no;
    if (i >= o0 && i < o1) continue;
    const double v = As[(size_t)i * n + j] - w.U[t];
    As[(size_t)i * n + j] = v;
    As[(size_t)j * n + i] = v;
  }
  __syncthreads();
  block_cholesky(w.L, no, w.keep + o0, drop);
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
  if (!do_house) {  // hand the transformed matrix to the cluster reduction
    if (smem)
      for (size_t t = tid; t < nn; t += kThreads) w.As[t] = As[t];
    return;
  }
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

// ------------------------------------------------------------------ 1b. cluster Householder
// Householder tridiagonalisation of the transformed n x n matrix (w.As) by a
// cluster of kCS thread blocks: row r lives in block r % kCS (distributed
// shared memory), so the O(n^3) FP64 work is spread over kCS SMs.  Per step j
// each block publishes its entries of column j, every block gathers the whole
// column and forms the same reflector; each block computes p = tau A v for its
// rows and publishes them with its share of p^T v; every block gathers p, forms
// w = p - K v and updates its rows.  Two cluster barriers per step; the
// published buffers alternate between steps so no barrier guards their reuse.
constexpr int kCS = 8;
constexpr int kCT = 256;

__device__ double cl_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wdx = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wdx] = v;
  __syncthreads();
  double t = lane < (kCT / 32) ? red[lane] : 0.0;
  return warp_sum(t);
}

__global__ void __cluster_dims__(kCS, 1, 1) __launch_bounds__(kCT)
    k_rr_house_cluster(int n, RRWork w) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int kW = kCT / 32;
  const int rpc = (n + kCS - 1) / kCS;
  extern __shared__ double sm[];
  double* Ar = sm;                      // rpc x n: row rank + kCS * li
  double* vf = Ar + (size_t)rpc * n;    // n: column j, then v
  double* wf = vf + n;                  // n: p, then w
  double* pubc = wf + n;                // 2 x rpc
  double* pubp = pubc + 2 * rpc;        // 2 x rpc
  double* pubs = pubp + 2 * rpc;        // 2
  __shared__ double red[kW];
  for (int t = tid; t < rpc * n; t += kCT) {
    const int li = t / n, c = t % n, r = rank + kCS * li;
    Ar[t] = r < n ? w.As[(size_t)r * n + c] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j + 2 < n; ++j) {
    const int buf = j & 1;
    for (int li = tid; li < rpc; li += kCT) {
      const int r = rank + kCS * li;
      pubc[buf * rpc + li] = (r < n && r >= j + 1) ? Ar[(size_t)li * n + j] : 0.0;
    }
    cl.sync();
    for (int r = j + 1 + tid; r < n; r += kCT) {
      const double* rem = cl.map_shared_rank(pubc + buf * rpc, r % kCS);
      vf[r] = rem[r / kCS];
    }
    __syncthreads();
    double part = 0.0;
    for (int r = j + 1 + tid; r < n; r += kCT) part += vf[r] * vf[r];
    const double ss = cl_block_sum(part, red);
    const double x0 = vf[j + 1];
    const double alpha = sqrt(ss);
    const int own_j = (j % kCS) == rank;
    if (!(alpha > 1e-290)) {
      if (own_j && tid == 0) w.dg[j] = Ar[(size_t)(j / kCS) * n + j];
      if (rank == 0 && tid == 0) {
        w.tau[j] = 0.0;
        w.e[j] = x0;
      }
      __syncthreads();
      continue;
    }
    const double beta = x0 >= 0.0 ? -alpha : alpha;
    const double tj = (beta - x0) / beta;
    const double scale = 1.0 / (x0 - beta);
    __syncthreads();
    for (int r = j + 1 + tid; r < n; r += kCT) {
      const double v = r == j + 1 ? 1.0 : vf[r] * scale;
      vf[r] = v;
      if (rank == 0) w.ref[(size_t)j * n + r] = v;
    }
    if (own_j && tid == 0) w.dg[j] = Ar[(size_t)(j / kCS) * n + j];
    if (rank == 0 && tid == 0) {
      w.tau[j] = tj;
      w.e[j] = beta;
    }
    __syncthreads();
    // p = tau A v for own rows r >= j+1, and this block's share of p^T v
    double kp = 0.0;
    for (int li = wid; li < rpc; li += kW) {
      const int r = rank + kCS * li;
      double acc = 0.0;
      if (r < n && r >= j + 1) {
        const double* row = Ar + (size_t)li * n;
        for (int l = j + 1 + lane; l < n; l += 32) acc += row[l] * vf[l];
      }
      acc = warp_sum(acc) * tj;
      if (lane == 0) {
        pubp[buf * rpc + li] = (r < n && r >= j + 1) ? acc : 0.0;
        if (r < n && r >= j + 1) kp += acc * vf[r];
      }
    }
    const double kpb = cl_block_sum(kp, red);
    if (tid == 0) pubs[buf] = kpb;
    cl.sync();
    double K = 0.0;
    for (int q = 0; q < kCS; ++q) K += cl.map_shared_rank(pubs, q)[buf];
    K *= 0.5 * tj;
    for (int r = j + 1 + tid; r < n; r += kCT) {
      const double* rem = cl.map_shared_rank(pubp + buf * rpc, r % kCS);
      wf[r] = rem[r / kCS] - K * vf[r];
    }
    __syncthreads();
    for (int li = wid; li < rpc; li += kW) {  // A_own -= v w^T + w v^T
      const int r = rank + kCS * li;
      if (r >= n || r < j + 1) continue;
      double* row = Ar + (size_t)li * n;
      const double vr = vf[r], wr = wf[r];
      for (int l = j + 1 + lane; l < n; l += 32) row[l] -= vr * wf[l] + wr * vf[l];
    }
    __syncthreads();
  }
  // the last 2 x 2 block
  if (tid == 0) {
    for (int r = (n >= 2 ? n - 2 : 0); r < n; ++r) {
      if (r % kCS != rank) continue;
      const double* row = Ar + (size_t)(r / kCS) * n;
      w.dg[r] = row[r];
      if (r == n - 1 && n >= 2) w.e[n - 2] = row[n - 2];
    }
    if (rank == 0) {
      if (n >= 2) w.tau[n - 2] = 0.0;
      w.tau[n - 1] = 0.0;
      w.e[n - 1] = 0.0;
    }
  }
  __threadfence();
  cl.sync();
  if (rank == 0)
    for (int i = tid; i < n; i += kCT) w.e2[i] = w.e[i] * w.e[i];
}

// ------------------------------------------------------------------ 2b. eigenvalues, one block each
// FP64 multisection with the division-free Sturm count: one warp per
// eigenvalue, 32 probes per round (a 33-fold shrink of the bracket per round).
__global__ void k_rr_eigvals_mc(int n, int nb, RRWork w, double* theta) {
  const int s = blockIdx.x, lane = threadIdx.x;
  double lo = 0.0, hi = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(w.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(w.e[i]) : 0.0);
    const double a = w.dg[i] - r, b = w.dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
  }
  const double span = fmax(hi - lo, 1e-30);
  double a = lo - span * 1e-6, b = hi + span * 1e-6;
  for (int round = 0; round < 64; ++round) {
    const double x = a + (b - a) * (double)(lane + 1) / 33.0;
    const int cnt = sturm64(w.dg, w.e2, n, x);
    const unsigned above = __ballot_sync(0xffffffffu, cnt >= s + 1);
    const int first = above ? __ffs(above) - 1 : 32;
    const double na = first == 0 ? a : a + (b - a) * (double)first / 33.0;
    const double nbv = first == 32 ? b : a + (b - a) * (double)(first + 1) / 33.0;
    a = __shfl_sync(0xffffffffu, na, 0);
    b = __shfl_sync(0xffffffffu, nbv, 0);
    if (b - a <= 4.0 * kEps * fmax(fabs(a), fabs(b))) break;
  }
  if (lane == 0) {
    w.lam[s] = 0.5 * (a + b);
    theta[s] = 0.5 * (a + b);
  }
}

// ------------------------------------------------------------------ 3b. inverse iteration in shared memory
// kIV threads per block, one vector each, their LU factors in shared memory
// (one thread per block: the pivoting branches of different vectors diverge)
constexpr int kIV = 1;
__global__ void k_rr_invit_sm(int n, int nb, RRWork w) {
  extern __shared__ double sm[];
  const int s = blockIdx.x * kIV + threadIdx.x;
  double* u = sm + (size_t)threadIdx.x * 6 * n;
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
  double* u1 = u + n;
  double* u2 = u1 + n;
  double* lm = u2 + n;
  double* sw = lm + n;
  double* z = sw + n;
  const double lam = w.lam[s];
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
  unsigned int h = 2166136261u ^ (unsigned)s * 16777619u;
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

// ------------------------------------------------------------------ 4a. Cholesky QR (twice) of the tridiagonal eigenvectors
__global__ void __launch_bounds__(kThreads) k_rr_cholqr(int n, int nb, RRWork w) {
  __shared__ int keep_nb[512];
  double* V = w.V;
  double* G = w.G;
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = threadIdx.x; t < nb * nb; t += kThreads) {
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      if (b <= a)
        for (int i = 0; i < n; ++i) acc += V[(size_t)i * nb + a] * V[(size_t)i * nb + b];
      G[t] = acc;
    }
    for (int s2 = threadIdx.x; s2 < nb; s2 += kThreads) keep_nb[s2] = 1;
    __syncthreads();
    block_cholesky(G, nb, keep_nb, 0.0);
    for (int i = threadIdx.x; i < n; i += kThreads) {
      double* v = V + (size_t)i * nb;
      for (int s2 = 0; s2 < nb; ++s2) {
        double acc = v[s2];
        for (int p = 0; p < s2; ++p) acc -= G[s2 * nb + p] * v[p];
        v[s2] = acc / G[s2 * nb + s2];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ 4b. back-transform, one warp per vector
__global__ void k_rr_backtransform(int n, int nb, RRWork w) {
  extern __shared__ double z[];
  const int s = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) z[i] = w.V[(size_t)i * nb + s];
  __syncwarp();
  for (int j = n - 3; j >= 0; --j) {
    const double tj = w.tau[j];
    if (tj == 0.0) continue;
    const double* v = w.ref + (size_t)j * n;
    double acc = 0.0;
    for (int i = j + 1 + lane; i < n; i += 32) acc += v[i] * z[i];
    acc = warp_sum(acc) * tj;
    for (int i = j + 1 + lane; i < n; i += 32) z[i] -= acc * v[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) w.V[(size_t)i * nb + s] = z[i];
}

// ------------------------------------------------------------------ 4c. momentum and mapping back
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_rr_momentum(int n, int o0, int no, int nx, int nb, int want_p, RRWork w,
                  T* __restrict__ YZ, int* __restrict__ dropped) {
  __shared__ int keep_nb[512];
  const int tid = threadIdx.x;
  double* V = w.V;
  double* Z = w.Z;
  double* G = w.G;
  if (want_p) {
    // G = V^T Zp with Zp = V without its X rows, summed over the W and P rows
    // directly: I - V_X^T V_X would cancel catastrophically once the X rows of
    // V are nearly the identity (a converging block)
    for (int t = tid; t < nb * nb; t += kThreads) {
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      for (int i = nx; i < n; ++i) acc += V[(size_t)i * nb + a] * V[(size_t)i * nb + b];
      G[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < n * nb; t += kThreads) {  // Z = Zp - V G
      const int i = t / nb, b = t % nb;
      double acc = i < nx ? 0.0 : V[t];
      for (int a = 0; a < nb; ++a) acc -= V[(size_t)i * nb + a] * G[a * nb + b];
      w.T1[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < nb * nb; t += kThreads) {  // G = Z^T Z (lower)
      const int a = t / nb, b = t % nb;
      double acc = 0.0;
      if (b <= a)
        for (int i = 0; i < n; ++i) acc += w.T1[(size_t)i * nb + a] * w.T1[(size_t)i * nb + b];
      G[t] = acc;
    }
    for (int s2 = tid; s2 < nb; s2 += kThreads) keep_nb[s2] = 1;
    __syncthreads();
    double gref = 0.0;
    for (int s2 = 0; s2 < nb; ++s2) gref = fmax(gref, G[s2 * nb + s2]);
    block_cholesky(G, nb, keep_nb, kDrop * fmax(gref, 1e-300));
    for (int i = tid; i < n; i += kThreads) {  // Z <- Z L^-T, dropped columns zero
      const double* zt = w.T1 + (size_t)i * nb;
      double* zr = Z + (size_t)i * nb;
      for (int s2 = 0; s2 < nb; ++s2) {
        double acc = zt[s2];
        for (int p = 0; p < s2; ++p) acc -= G[s2 * nb + p] * zr[p];
        zr[s2] = keep_nb[s2] ? acc / G[s2 * nb + s2] : 0.0;
      }
    }
    __syncthreads();
  }
  // back to the coefficients of the original basis: y_O <- L^-T y_O, then
  // y_rest <- y_rest - C y_O, then y <- D y
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
  // undo the coefficient-space projection: rest rows -= C y_O
  for (int t = tid; t < n * 2 * nb; t += kThreads) {
    const int i = t / (2 * nb), c = t % (2 * nb);
    if ((i >= o0 && i < o0 + no) || (c >= nb && !want_p)) continue;
    double* M_ = c < nb ? V : Z;
    const int cc = c < nb ? c : c - nb;
    double acc = M_[(size_t)i * nb + cc];
    for (int a = 0; a < no; ++a) acc -= w.C[i * no + a] * M_[(size_t)(o0 + a) * nb + cc];
    M_[(size_t)i * nb + cc] = acc;
  }
  __syncthreads();
  for (int t = tid; t < n * nb; t += kThreads) {
    const int i = t / nb, s2 = t % nb;
    const double d = w.dsc[i];
    YZ[(size_t)i * 2 * nb + s2] = (T)(V[t] * d);
    YZ[(size_t)i * 2 * nb + nb + s2] = want_p ? (T)(Z[t] * d) : T(0);
  }
  if (tid == 0) {
    int dc = 0;
    for (int a = 0; a < n; ++a) dc += !w.keep[a];
    *dropped = dc;
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

}  // namespace

template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool /*fp64*/, double* /*dbg*/) {
  ProfScope ps(kProfRR);
  FF_REQUIRE(d.ns <= 1024 && d.no <= 1024 && d.nb <= 512 && d.o0 + d.no <= d.ns,
             FF_ERR_INVALID_ARG, "Rayleigh-Ritz basis too large");
  const size_t n = d.ns, nb = d.nb, no = d.no;
  const size_t t1 = std::max(n * nb, 2 * n);
  const size_t total =
      2 * n * n + no * no + 5 * n + nb + 2 * n * nb + nb * nb + t1 + 6 * n * nb + 2 * n * no;
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
  w.C = p; p += n * no;
  w.U = p; p += n * no;
  w.keep = reinterpret_cast<int*>(p);
  static bool attr = false;
  if (!attr) {
    FF_CUDA(cudaFuncSetAttribute(k_rr_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    FF_CUDA(cudaFuncSetAttribute(k_rr_house_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    FF_CUDA(cudaFuncSetAttribute(k_rr_invit_sm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem));
    attr = true;
  }
  const size_t tri_bytes = sizeof(double) * n * n;
  const bool tri_smem = tri_bytes <= kMaxDynSmem;
  const size_t rpc = (n + kCS - 1) / kCS;
  const size_t cl_bytes = sizeof(double) * (rpc * n + 2 * n + 4 * rpc + 2);
  const bool use_cluster = cl_bytes <= kMaxDynSmem && n >= 3;
  // transform (one block); Householder by the cluster when its rows fit
  (k_rr_tridiag<<<1, kThreads, tri_smem ? tri_bytes : 0, st>>>(A, B, d.ns, d.o0, d.no, w,
                                                               tri_smem ? 1 : 0,
                                                               use_cluster ? 0 : 1, d.drop),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (use_cluster) {
    (k_rr_house_cluster<<<kCS, kCT, cl_bytes, st>>>(d.ns, w), ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  (k_rr_eigvals_mc<<<(unsigned)nb, 32, 0, st>>>(d.ns, d.nb, w, theta), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const size_t iv_bytes = sizeof(double) * kIV * 6 * n;
  if (iv_bytes <= kMaxDynSmem) {
    (k_rr_invit_sm<<<(unsigned)((nb + kIV - 1) / kIV), kIV, iv_bytes, st>>>(d.ns, d.nb, w),
     ::ff::note_launch());
  } else {
    (k_rr_invit<<<(unsigned)((nb + 31) / 32), 32, 0, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
  (k_rr_cholqr<<<1, kThreads, 0, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_rr_backtransform<<<(unsigned)nb, 32, sizeof(double) * n, st>>>(d.ns, d.nb, w),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_rr_momentum<T><<<1, kThreads, 0, st>>>(d.ns, d.o0, d.no, d.nx, d.nb, d.want_p, w, YZ,
                                            dropped),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template void rayleigh_ritz<float>(cudaStream_t, const double*, const double*, RRDims, float*,
                                   double*, int*, Buf&, bool, double*);
template void rayleigh_ritz<double>(cudaStream_t, const double*, const double*, RRDims, double*,
                                    double*, int*, Buf&, bool, double*);

}  // namespace ff
