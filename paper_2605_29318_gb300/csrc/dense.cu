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
//   k_rr_proj_c, k_rr_proj_v, k_rr_proj_oo
//                       (many blocks) scale the O block by diag(B_OO)^-1/2
//                       (columns outside O whose B_ii is not ~1, empty
//                       momentum directions, leave the basis) and project the
//                       O block against the rest once more in coefficient
//                       space;
//   k_rr_chol, k_rr_ysolve, k_rr_zsolve
//                       Cholesky B_OO = L L^T with drop (dependent or empty
//                       columns leave the basis; one block), then the two
//                       triangular solves of A <- T^T A T with
//                       T = blockdiag(I, L^-T, I) (many blocks);
//   k_rr_tridiag        (one block) the transformed matrix assembled,
//                       symmetrised, dropped columns decoupled; for bases
//                       too large for the cluster it also tridiagonalises;
//   k_rr_house_cluster  Householder tridiagonalisation of A by an 8-block
//                       thread-block cluster, rows spread over the blocks'
//                       shared memory;
//   k_rr_eigvals_mc     the nb smallest eigenvalues of the tridiagonal matrix,
//                       one 4-warp block each: FP32 multisection brackets,
//                       then multisection in the working precision on a
//                       division-free Sturm count;
//   k_rr_invit_sm       their eigenvectors by inverse iteration on the
//                       tridiagonal (LU with partial pivoting), one block each;
//   k_rr_gram_mb, k_rr_cqchol, k_rr_rsolve, k_rr_cholqr
//                       Cholesky QR of those vectors (the Gram and V L^-T
//                       over many blocks, the factor in one; a second pass,
//                       in one block, only when the first finds them far
//                       from orthogonal);
//   k_rr_wy_t, k_rr_backtransform
//                       the Householder reflectors applied in reverse, in
//                       groups of eight in compact WY form;
//   k_rr_gram_mb, k_rr_zp_mb, k_rr_mchol, k_rr_rsolve, k_rr_bsolve
//                       the momentum coefficients Z (the W and P rows of the
//                       Ritz vectors, orthogonalised against them and
//                       orthonormalised -- the next P = S Z is then
//                       M-orthonormal and M-orthogonal to the next X), and the
//                       O rows mapped back through L^-T;
//   k_rr_output         the projection undone and the scaling.
// Output YZ = [Y | Z] (n x 2 nb, row-major, context precision) and the Ritz
// values theta (nb).  Instantiated in FP64 (FP64 blocks), in double-float
// (the double-float phase of the mixed solve) and in FP32 (the FP32 phase):
// the spectrum of A spans the whole range of the basis' Rayleigh quotients and
// the small eigenvalues need relative accuracy, so every phase that must reach
// the FP64 residual bar runs it in FP64 or double-float.
#include <cooperative_groups.h>

#include <cstdlib>
#include <type_traits>

#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr size_t kMaxDynSmem = 220 * 1024;  // opt-in limit less room for static shared memory
// working-precision constants: unit roundoff, smallest magnitude kept apart
// from zero, default Cholesky drop
template <class R>
struct Prec;
template <>
struct Prec<double> {
  static constexpr double eps = 1.1e-16, tiny = 1e-290, drop = 1e-13;
};
template <>
struct Prec<float> {
  static constexpr float eps = 6e-8f, tiny = 1e-30f, drop = 1e-6f;
};
// double-float: ~2^-47 unit roundoff at the FP32 exponent range
template <>
struct Prec<dfloat> {
  static constexpr dfloat eps = dfloat(1.5e-14), tiny = dfloat(1e-30), drop = dfloat(1e-12);
};
__device__ __forceinline__ double scalbn_r(double x, int e) { return scalbn(x, e); }
__device__ __forceinline__ float scalbn_r(float x, int e) { return scalbnf(x, e); }
__device__ __forceinline__ dfloat scalbn_r(dfloat x, int e) {
  return dfloat(scalbnf(x.h, e), scalbnf(x.l, e));
}

// global workspace layout (working precision R)
template <class R>
struct RRWork {
  R *As, *ref, *L, *dsc, *dg, *e, *e2, *tau, *lam, *V, *Z, *G, *T1, *scr, *C, *U;
  int* keep;   // n: basis columns kept
  int* keepz;  // nb: momentum columns kept
  int* flag;   // 1: Cholesky QR's second pass is needed
};

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
  R t = lane < (int)(blockDim.x >> 5) ? red[lane] : R(0.0);
  return warp_sum(t);
}

// Blocked one-block dense factorisation and solves, in panels of kPB columns:
// each panel's few columns are done by short substitutions, and what they
// change in the rest of the matrix is applied as one product in 4 x 4
// register tiles over all threads (4 x 4 for 4-byte types: 16 multiply-adds
// per 8 shared loads; 2 x 4 for 8-byte ones, which would spill), so
// that the serial part is kPB steps long and the bulk runs at full width.
constexpr int kPB = 8;

// Cholesky (lower, row-major m x m) of G in place, with drop: column j is
// kept when keep[j] and its updated pivot g_jj > drop_rel, else it leaves (a
// zero column with l_jj = 1, keep[j] = 0, updating nothing).  L^T is mirrored
// into the upper triangle (g_kj = l_jk for k > j), where the solves below read
// it by rows.  With X (m rows of nx entries, stride ldx) the same elimination
// is applied to X's rows, which leaves L^-1 X in X (a dropped column's row is
// left as it is).  Per panel: the kPB x kPB diagonal block by warp 0, the
// panel's rows below and the panel's rows of X by a thread per row / column
// (substitutions of at most kPB steps), then the trailing lower triangle and
// X's rows below in register tiles; three barriers a panel.
template <class R>
__device__ void block_cholesky(R* G, int m, int* keep, R drop_rel, R* X = nullptr, int ldx = 0,
                               int nx = 0) {
  constexpr int TR = sizeof(R) > 4 ? 2 : 4;  // tile rows: 8-byte types would spill at 4
  const int tid = threadIdx.x, lane = tid & 31;
  for (int j0 = 0; j0 < m; j0 += kPB) {
    const int jb = min(kPB, m - j0);
    R* D = G + (size_t)j0 * m + j0;  // the diagonal block, D[i m + k]
    if (tid < 32) {
      for (int j = 0; j < jb; ++j) {
        const R piv = D[(size_t)j * m + j];
        const int kj = keep[j0 + j] && piv > drop_rel;
        const R l = kj ? sqrt(piv) : R(1.0);
        __syncwarp();
        if (lane > j && lane < jb) {
          const R v = kj ? D[(size_t)lane * m + j] / l : R(0.0);
          D[(size_t)lane * m + j] = v;
          D[(size_t)j * m + lane] = v;
        }
        if (lane == 0) {
          D[(size_t)j * m + j] = l;
          keep[j0 + j] = kj;
        }
        __syncwarp();
        for (int e = lane; e < kPB * kPB; e += 32) {
          const int i = e / kPB, k = e - i * kPB;
          if (k > j && k <= i && i < jb)
            D[(size_t)i * m + k] -= D[(size_t)i * m + j] * D[(size_t)k * m + j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    const int r0 = j0 + jb, nr = m - r0;
    // the panel's rows below: l_ij = (g_ij - sum_{p<j} l_ip l_jp) / l_jj
    for (int i = r0 + tid; i < m; i += blockDim.x) {
      R* gi = G + (size_t)i * m + j0;
      R v[kPB];
#pragma unroll
      for (int j = 0; j < kPB; ++j) {
        if (j < jb) {
          R acc = gi[j];
#pragma unroll
          for (int p = 0; p < j; ++p) acc -= v[p] * D[(size_t)j * m + p];
          v[j] = keep[j0 + j] ? acc / D[(size_t)j * m + j] : R(0.0);
          gi[j] = v[j];
          G[(size_t)(j0 + j) * m + i] = v[j];
        }
      }
    }
    // the panel's rows of X: y_j = (x_j - sum_{p<j} l_jp y_p) / l_jj
    if (X)
      for (int c = tid; c < nx; c += blockDim.x) {
        R v[kPB];
#pragma unroll
        for (int j = 0; j < kPB; ++j) {
          if (j < jb) {
            R acc = X[(size_t)(j0 + j) * ldx + c];
#pragma unroll
            for (int p = 0; p < j; ++p) acc -= D[(size_t)j * m + p] * v[p];
            v[j] = acc / D[(size_t)j * m + j];
            X[(size_t)(j0 + j) * ldx + c] = v[j];
          }
        }
      }
    __syncthreads();
    if (nr > 0) {
      // trailing lower triangle: g_ik -= sum_j l_ij l_kj (k <= i), 4 x 4 tiles
      const int ta = (nr + TR - 1) / TR, tt = (nr + 3) >> 2;
      for (int t = tid; t < ta * tt; t += blockDim.x) {
        const int ia = t / tt, ib = t - ia * tt;
        if (4 * ib > TR * ia + TR - 1) continue;  // above the diagonal
        R acc[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = R(0.0);
        for (int j = 0; j < jb; ++j) {
          R la[TR], lb[4];
          const R* up = G + (size_t)(j0 + j) * m + r0;  // row j of L^T
#pragma unroll
          for (int r = 0; r < TR; ++r) la[r] = TR * ia + r < nr ? up[TR * ia + r] : R(0.0);
#pragma unroll
          for (int c = 0; c < 4; ++c) lb[c] = 4 * ib + c < nr ? up[4 * ib + c] : R(0.0);
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += la[r] * lb[c];
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = TR * ia + r, k = 4 * ib + c;
            if (i < nr && k <= i) G[(size_t)(r0 + i) * m + r0 + k] -= acc[r][c];
          }
      }
      // X's rows below: x_i -= sum_j l_ij y_j, 4 x 4 tiles over (i, c)
      if (X) {
        const int tc = (nx + 3) >> 2;
        for (int t = tid; t < ta * tc; t += blockDim.x) {
          const int ia = t / tc, ib = t - ia * tc;
          R acc[TR][4];
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = R(0.0);
          for (int j = 0; j < jb; ++j) {
            R la[TR], yb[4];
            const R* up = G + (size_t)(j0 + j) * m + r0;
            const R* yj = X + (size_t)(j0 + j) * ldx;
#pragma unroll
            for (int r = 0; r < TR; ++r) la[r] = TR * ia + r < nr ? up[TR * ia + r] : R(0.0);
#pragma unroll
            for (int c = 0; c < 4; ++c) yb[c] = 4 * ib + c < nx ? yj[4 * ib + c] : R(0.0);
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[r][c] += la[r] * yb[c];
          }
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int i = TR * ia + r, cc = 4 * ib + c;
              if (i < nr && cc < nx) X[(size_t)(r0 + i) * ldx + cc] -= acc[r][c];
            }
        }
      }
    }
    __syncthreads();
  }
}

// X <- X L^-T for `rows` rows of X (m entries each, stride ldx): every row is
// a forward substitution along the row.  L is lower (row-major, m x m) with
// L^T mirrored into its upper triangle, as block_cholesky leaves it.  Per
// panel: its columns by a thread per row, then the later columns in 4 x 4
// register tiles (x_k -= sum_j x_j l_kj, l_kj read from the mirror).
template <class R>
__device__ void block_trsm_rt(const R* L, int m, R* X, int ldx, int rows) {
  constexpr int TR = sizeof(R) > 4 ? 2 : 4;
  const int tid = threadIdx.x;
  for (int j0 = 0; j0 < m; j0 += kPB) {
    const int jb = min(kPB, m - j0);
    const R* D = L + (size_t)j0 * m + j0;
    for (int a = tid; a < rows; a += blockDim.x) {
      R* x = X + (size_t)a * ldx + j0;
      R v[kPB];
#pragma unroll
      for (int j = 0; j < kPB; ++j) {
        if (j < jb) {
          R acc = x[j];
#pragma unroll
          for (int p = 0; p < j; ++p) acc -= v[p] * D[(size_t)j * m + p];
          v[j] = acc / D[(size_t)j * m + j];
          x[j] = v[j];
        }
      }
    }
    __syncthreads();
    const int k0 = j0 + jb, nk = m - k0;
    if (nk > 0) {
      const int ta = (rows + TR - 1) / TR, tb = (nk + 3) >> 2;
      for (int t = tid; t < ta * tb; t += blockDim.x) {
        const int ia = t / tb, ib = t - ia * tb;
        R acc[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = R(0.0);
        for (int j = 0; j < jb; ++j) {
          R xa[TR], lb[4];
          const R* up = L + (size_t)(j0 + j) * m + k0;
#pragma unroll
          for (int r = 0; r < TR; ++r)
            xa[r] = TR * ia + r < rows ? X[(size_t)(TR * ia + r) * ldx + j0 + j] : R(0.0);
#pragma unroll
          for (int c = 0; c < 4; ++c) lb[c] = 4 * ib + c < nk ? up[4 * ib + c] : R(0.0);
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += xa[r] * lb[c];
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int a = TR * ia + r, k = 4 * ib + c;
            if (a < rows && k < nk) X[(size_t)a * ldx + k0 + k] -= acc[r][c];
          }
      }
    }
    __syncthreads();
  }
}

// X <- L^-T X for the m rows of X (nc entries each, stride ldx; L lower,
// row-major m x m): a backward substitution down every column.  Per panel,
// from the last: its rows by a thread per column, then the earlier rows in
// 4 x 4 register tiles (x_b -= sum_j l_jb x_j, l_jb read along row j of L).
template <class R>
__device__ void block_trsm_lt(const R* L, int m, R* X, int ldx, int nc) {
  constexpr int TR = sizeof(R) > 4 ? 2 : 4;
  const int tid = threadIdx.x;
  for (int j1 = m; j1 > 0; j1 -= kPB) {
    const int j0 = max(0, j1 - kPB), jb = j1 - j0;
    for (int c = tid; c < nc; c += blockDim.x) {
      R v[kPB];
#pragma unroll
      for (int jj = kPB - 1; jj >= 0; --jj) {
        if (jj < jb) {
          const int j = j0 + jj;
          R acc = X[(size_t)j * ldx + c];
#pragma unroll
          for (int p = jj + 1; p < kPB; ++p)
            if (p < jb) acc -= L[(size_t)(j0 + p) * m + j] * v[p];
          v[jj] = acc / L[(size_t)j * m + j];
          X[(size_t)j * ldx + c] = v[jj];
        }
      }
    }
    __syncthreads();
    if (j0 > 0) {
      const int ta = (j0 + TR - 1) / TR, tb = (nc + 3) >> 2;
      for (int t = tid; t < ta * tb; t += blockDim.x) {
        const int ia = t / tb, ib = t - ia * tb;
        R acc[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = R(0.0);
        for (int j = 0; j < jb; ++j) {
          R la[TR], xb[4];
          const R* lj = L + (size_t)(j0 + j) * m;
          const R* xj = X + (size_t)(j0 + j) * ldx;
#pragma unroll
          for (int r = 0; r < TR; ++r) la[r] = TR * ia + r < j0 ? lj[TR * ia + r] : R(0.0);
#pragma unroll
          for (int c = 0; c < 4; ++c) xb[c] = 4 * ib + c < nc ? xj[4 * ib + c] : R(0.0);
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += la[r] * xb[c];
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int b = TR * ia + r, cc = 4 * ib + c;
            if (b < j0 && cc < nc) X[(size_t)b * ldx + cc] -= acc[r][c];
          }
      }
    }
    __syncthreads();
  }
}

template <class R>
__device__ __forceinline__ R shfl_xor_r(R v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
template <>
__device__ __forceinline__ dfloat shfl_xor_r<dfloat>(dfloat v, int o) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

// The warp sums of 16 values at once by halving exchanges (16 shuffles
// instead of 80): lanes 2q and 2q + 1 end with the sum of v[q].
template <class R>
__device__ __forceinline__ R sum16(R (&v)[16]) {
  const int lane = threadIdx.x & 31;
  R a8[8], a4[4], a2[2];
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    a8[k] = (h4 ? v[k + 8] : v[k]) + shfl_xor_r(h4 ? v[k] : v[k + 8], 16);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    a4[k] = (h3 ? a8[k + 4] : a8[k]) + shfl_xor_r(h3 ? a8[k] : a8[k + 4], 8);
#pragma unroll
  for (int k = 0; k < 2; ++k)
    a2[k] = (h2 ? a4[k + 2] : a4[k]) + shfl_xor_r(h2 ? a4[k] : a4[k + 2], 4);
  R a1 = (h1 ? a2[1] : a2[0]) + shfl_xor_r(h1 ? a2[0] : a2[1], 2);
  return a1 + shfl_xor_r(a1, 1);
}

// C = X^T Y over `rows` rows (X: rows x ma, Y: rows x mb, row-major with row
// strides ldx, ldy), only the entries b <= a when `lower`; C row-major with
// row stride ldc.  Each warp takes 4 x 4 tiles of C in turn, its lanes
// splitting the rows, and reduces the tile with sum16.
template <class R>
__device__ void blk_gram_tn(const R* X, int ldx, const R* Y, int ldy, int rows, int ma, int mb,
                            R* C, int ldc, bool lower) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ta = (ma + 3) >> 2, tb = (mb + 3) >> 2;
  for (int t = wid; t < ta * tb; t += kWarps) {
    const int ia = t / tb, ib = t - ia * tb;
    if (lower && ib > ia) continue;
    R acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = R(0.0);
    for (int i = lane; i < rows; i += 32) {
      R xa[4], yb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        xa[r] = 4 * ia + r < ma ? X[(size_t)i * ldx + 4 * ia + r] : R(0.0);
        yb[r] = 4 * ib + r < mb ? Y[(size_t)i * ldy + 4 * ib + r] : R(0.0);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[4 * r + c] += xa[r] * yb[c];
    }
    const R s = sum16(acc);
    const int q = lane >> 1, a = 4 * ia + (q >> 2), b = 4 * ib + (q & 3);
    if (!(lane & 1) && a < ma && b < mb && (!lower || b <= a)) C[(size_t)a * ldc + b] = s;
  }
}

// ------------------------------------------------------------------ R(0.) coefficient-space projection
// The scaling of basis column i: O columns by B_ii^-1/2 (kept when B_ii is
// positive and finite), the others by 1 (kept when B_ii ~ 1; an empty
// momentum direction leaves the basis).
template <class R>
__device__ __forceinline__ int rr_scale(const double* __restrict__ B, int n, int o0, int no, int i,
                                        R& s) {
  const R bii = (R)B[(size_t)i * n + i];
  int k;
  if (i >= o0 && i < o0 + no) {
    k = bii > Prec<R>::tiny && isfinite(bii);
    s = k ? R(1.0) / sqrt(bii) : R(0.0);
  } else {
    k = bii > R(0.25) && bii < R(4.0);
    s = k ? R(1.0) : R(0.0);
  }
  return k;
}

// Second projection of the O block against the rest, in coefficient space.
// The O columns arrive M-projected against the others once, on the
// N-vectors; once they are mostly made of the other columns (a converging
// block) that projection leaves a coupling of order eps / |remainder|.  With
// the scaled matrices, C = B_{rest,O} and T = [I, -C; 0, I] (C's rows in O
// are zero), T^T A T and T^T B T differ from A and B only in
//   A_{rest,O} <- V = A_{rest,O} - A_{rest,rest} C,
//   A_OO       <- A_OO - C^T V - (C^T A_{rest,O})^T,
//   B_OO       <- B_OO - C^T C,
// and the rest-rest block of B is the identity to rounding ("twice is
// enough").  Three launches spread this over the SMs: the scaling and C, the
// rows of V (a block per kPR rows), the O x O blocks (a block per row).
constexpr int kPR = 8;
constexpr int kPT = 256;

template <class R>
__global__ void __launch_bounds__(kPT)
    k_rr_proj_c(const double* __restrict__ B, int n, int o0, int no, RRWork<R> w) {
  const long long t = (long long)blockIdx.x * kPT + threadIdx.x;
  if (t < n) {
    R s;
    w.keep[t] = rr_scale(B, n, o0, no, (int)t, s);
    w.dsc[t] = s;
    return;
  }
  const long long u = t - n;
  if (u >= (long long)n * no) return;
  const int i = (int)(u / no), b = (int)(u - (long long)i * no), j = o0 + b;
  R c = R(0.0);
  if (!(i >= o0 && i < o0 + no)) {
    R si, sj;
    const int ki = rr_scale(B, n, o0, no, i, si), kj = rr_scale(B, n, o0, no, j, sj);
    if (ki && kj) c = R(0.5) * ((R)B[(size_t)i * n + j] + (R)B[(size_t)j * n + i]) * si * sj;
  }
  w.C[u] = c;
}

// the scaled symmetric A: A_ij d_i d_j and A_ji d_j d_i averaged
template <class R>
__device__ __forceinline__ R rr_asym(const double* __restrict__ A, int n, const R* dsc, int i,
                                     int j) {
  const R di = dsc[i], dj = dsc[j];
  return R(0.5) * ((R)A[(size_t)i * n + j] * di * dj + (R)A[(size_t)j * n + i] * dj * di);
}

template <class R>
__global__ void __launch_bounds__(kPT)
    k_rr_proj_v(const double* __restrict__ A, int n, int o0, int no, RRWork<R> w) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* at = reinterpret_cast<R*>(dyn_raw);  // kPR x n: the block's rows of the scaled A
  const int i0 = blockIdx.x * kPR, o1 = o0 + no;
  for (int t = threadIdx.x; t < kPR * n; t += kPT) {
    const int k = t / kPR, q = t - k * kPR, i = i0 + q;
    at[(size_t)q * n + k] = i < n ? rr_asym(A, n, w.dsc, i, k) : R(0.0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kPR * no; t += kPT) {
    const int q = t / no, b = t - q * no, i = i0 + q;
    if (i >= n || (i >= o0 && i < o1)) continue;
    const R* ar = at + (size_t)q * n;
    const R* cb = w.C + b;
    R s[4] = {R(0.0), R(0.0), R(0.0), R(0.0)};
    for (int seg = 0; seg < 2; ++seg) {
      const int k0 = seg ? o1 : 0, k1 = seg ? n : o0;
      int k = k0;
      for (; k + 4 <= k1; k += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) s[r] += ar[k + r] * cb[(size_t)(k + r) * no];
      }
      for (; k < k1; ++k) s[0] += ar[k] * cb[(size_t)k * no];
    }
    w.U[(size_t)i * no + b] = ar[o0 + b] - ((s[0] + s[1]) + (s[2] + s[3]));
  }
}

template <class R>
__global__ void __launch_bounds__(128)
    k_rr_proj_oo(const double* __restrict__ A, const double* __restrict__ B, int n, int o0, int no,
                 RRWork<R> w) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* ca = reinterpret_cast<R*>(dyn_raw);  // n: column a of C
  R* aa = ca + n;                         // n: column o0 + a of the scaled A
  const int a = blockIdx.x, ia = o0 + a, o1 = o0 + no;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    ca[k] = w.C[(size_t)k * no + a];
    aa[k] = rr_asym(A, n, w.dsc, k, ia);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < no; b += blockDim.x) {
    const int ib = o0 + b;
    R sa[2] = {R(0.0), R(0.0)}, sb[2] = {R(0.0), R(0.0)};
    for (int seg = 0; seg < 2; ++seg) {
      const int k0 = seg ? o1 : 0, k1 = seg ? n : o0;
      for (int k = k0; k < k1; ++k) {
        const R cb = w.C[(size_t)k * no + b];
        sa[k & 1] += ca[k] * w.U[(size_t)k * no + b] + cb * aa[k];
        sb[k & 1] += ca[k] * cb;
      }
    }
    w.G[(size_t)a * no + b] = rr_asym(A, n, w.dsc, ia, ib) - (sa[0] + sa[1]);
    const R bv = R(0.5) * ((R)B[(size_t)ia * n + ib] + (R)B[(size_t)ib * n + ia]) * w.dsc[ia] *
                     w.dsc[ib] -
                 (sb[0] + sb[1]);
    w.L[(size_t)a * no + b] = (w.keep[ia] && w.keep[ib]) ? bv : (a == b ? R(1.0) : R(0.0));
  }
}

// ------------------------------------------------------------------ R(0.5) factor and solves of the transform
// A <- T^T A T with T = blockdiag(I, L^-T, I), L L^T = B_OO - C^T C: with
// Y = L^-1 A_{O,.} (A's O rows after the projection), the rest-O blocks are
// Y's transposes and the O x O block is Y_OO L^-T.  The factor takes one
// block; each column of Y is a forward substitution of its own, and so is
// each row of Y_OO L^-T, so both solves are spread over blocks of kYC
// columns (rows), each with its own copy of L.
constexpr int kYC = 32;

template <class R>
__global__ void __launch_bounds__(kThreads)
    k_rr_chol(int o0, int no, RRWork<R> w, int lsm, R drop) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* Ls = lsm ? reinterpret_cast<R*>(dyn_raw) : w.L;
  __shared__ int keep_o[1024];
  if (lsm)
    for (int t = threadIdx.x; t < no * no; t += kThreads) Ls[t] = w.L[t];
  for (int a = threadIdx.x; a < no; a += kThreads) keep_o[a] = w.keep[o0 + a];
  __syncthreads();
  block_cholesky(Ls, no, keep_o, drop);
  for (int a = threadIdx.x; a < no; a += kThreads) w.keep[o0 + a] = keep_o[a];
  if (lsm)
    for (int t = threadIdx.x; t < no * no; t += kThreads) w.L[t] = Ls[t];
}

// Y (no x n, row-major, in Yg) = L^-1 A_{O,.}: a block per cb columns, each
// column staged as a row of Xt and solved as x L^-T
template <class R>
__global__ void __launch_bounds__(256)
    k_rr_ysolve(int n, int o0, int no, RRWork<R> w, R* __restrict__ Yg, int cb, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* dyn = reinterpret_cast<R*>(dyn_raw);
  const R* L = lsm ? dyn : w.L;
  R* Xt = dyn + (lsm ? (size_t)no * no : 0);
  const int lx = no | 1, c0 = blockIdx.x * cb, nc = min(cb, n - c0);
  if (lsm)
    for (int t = threadIdx.x; t < no * no; t += blockDim.x) dyn[t] = w.L[t];
  for (int t = threadIdx.x; t < nc * no; t += blockDim.x) {
    const int c = t / no, a = t - c * no, col = c0 + c;
    Xt[(size_t)c * lx + a] = (col >= o0 && col < o0 + no) ? w.G[(size_t)a * no + (col - o0)]
                                                          : w.U[(size_t)col * no + a];
  }
  __syncthreads();
  block_trsm_rt(L, no, Xt, lx, nc);
  for (int t = threadIdx.x; t < nc * no; t += blockDim.x) {
    const int a = t / nc, c = t - a * nc;
    Yg[(size_t)a * n + c0 + c] = Xt[(size_t)c * lx + a];
  }
}

// Y_OO <- Y_OO L^-T in place in Yg: a block per cb rows
template <class R>
__global__ void __launch_bounds__(256)
    k_rr_zsolve(int n, int o0, int no, RRWork<R> w, R* __restrict__ Yg, int cb, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* dyn = reinterpret_cast<R*>(dyn_raw);
  const R* L = lsm ? dyn : w.L;
  R* Xs = dyn + (lsm ? (size_t)no * no : 0);
  const int lx = no | 1, a0 = blockIdx.x * cb, nr = min(cb, no - a0);
  if (lsm)
    for (int t = threadIdx.x; t < no * no; t += blockDim.x) dyn[t] = w.L[t];
  for (int t = threadIdx.x; t < nr * no; t += blockDim.x) {
    const int r = t / no, b = t - r * no;
    Xs[(size_t)r * lx + b] = Yg[(size_t)(a0 + r) * n + o0 + b];
  }
  __syncthreads();
  block_trsm_rt(L, no, Xs, lx, nr);
  for (int t = threadIdx.x; t < nr * no; t += blockDim.x) {
    const int r = t / no, b = t - r * no;
    Yg[(size_t)(a0 + r) * n + o0 + b] = Xs[(size_t)r * lx + b];
  }
}

// ------------------------------------------------------------------ R(1.) tridiagonalise
template <class R>
__global__ void __launch_bounds__(kThreads)
    k_rr_tridiag(const double* __restrict__ A, const double* __restrict__ B, int n, int o0, int no,
                 RRWork<R> w, int smem, int do_house, const R* __restrict__ Yg) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* dyn = reinterpret_cast<R*>(dyn_raw);
  __shared__ R red[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // smem = 1: A in shared memory (rows padded to an odd stride, so that a
  // thread per row hits distinct banks)
  const int la = (smem && !do_house) ? (n | 1) : n;
  R* As = smem ? dyn : w.As;
  R* vt = w.T1;            // n (after Yg has been read)
  R* pw = w.T1 + n;        // n
  const int o1 = o0 + no;
  // the scaled matrix (rows by warps, columns by lanes) and its symmetric
  // part; then A's O rows and the rest-O blocks from Y (no x n in Yg, its
  // O x O block already times L^-T), which the solve launches left there
  for (int i = wid; i < n; i += kWarps)
    for (int j = lane; j < n; j += 32)
      As[(size_t)i * la + j] = (R)A[(size_t)i * n + j] * w.dsc[i] * w.dsc[j];
  __syncthreads();
  for (int i = wid; i < n; i += kWarps)
    for (int j = lane; j < i; j += 32) {
      const R v = R(0.5) * (As[(size_t)i * la + j] + As[(size_t)j * la + i]);
      As[(size_t)i * la + j] = v;
      As[(size_t)j * la + i] = v;
    }
  __syncthreads();
  for (int i = wid; i < n; i += kWarps) {
    if (i >= o0 && i < o1) {
      for (int c = lane; c < n; c += 32) As[(size_t)i * la + c] = Yg[(size_t)(i - o0) * n + c];
    } else {
      for (int b = lane; b < no; b += 32) As[(size_t)i * la + o0 + b] = Yg[(size_t)b * n + i];
    }
  }
  __syncthreads();
  // symmetrise; dropped columns are decoupled with a diagonal just above the
  // spectrum of the kept part (2 ||A_kept||_inf + 1), which keeps them out of
  // the nb lowest without disturbing the scale of the tridiagonal problem
  R rmax = R(0.0);
  for (int i = wid; i < n; i += kWarps) {
    if (!w.keep[i]) continue;
    R rs = R(0.0);
    for (int j = lane; j < n; j += 32)
      if (w.keep[j]) rs += fabs(As[(size_t)i * la + j]);
    rmax = fmax(rmax, warp_sum(rs));
  }
  {
    __syncthreads();
    if (lane == 0) red[wid] = rmax;
    __syncthreads();
    R t = lane < kWarps ? red[lane] : R(0.0);
#pragma unroll
    for (int o = 16; o; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    rmax = t;
    __syncthreads();
  }
  const R big = R(2.0) * rmax + R(1.0);
  for (int i = wid; i < n; i += kWarps)
    for (int j = lane; j <= i; j += 32) {
      R v;
      if (!w.keep[i] || !w.keep[j])
        v = (i == j) ? big : R(0.0);
      else
        v = i > j ? R(0.5) * (As[(size_t)i * la + j] + As[(size_t)j * la + i]) : As[(size_t)i * la + j];
      As[(size_t)i * la + j] = v;
    }
  __syncthreads();
  for (int i = wid; i < n; i += kWarps)
    for (int j = lane; j < n; j += 32)
      if (i < j) As[(size_t)i * la + j] = As[(size_t)j * la + i];
  __syncthreads();
  if (!do_house) {  // hand the transformed matrix to the cluster reduction
    if (smem)
      for (int i = wid; i < n; i += kWarps)
        for (int j = lane; j < n; j += 32) w.As[(size_t)i * n + j] = As[(size_t)i * la + j];
    return;
  }
  // Householder: reflector j = [1, v] stored in row j of w.ref (entries j+1..n-1)
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    R part = R(0.0);
    for (int i = tid; i < m; i += kThreads) {
      const R x = As[(size_t)(j + 1 + i) * la + j];
      part += x * x;
    }
    const R ss = block_sum(part, red);
    const R x0 = As[(size_t)(j + 1) * la + j];
    const R alpha = sqrt(ss);
    __syncthreads();
    if (!(alpha > Prec<R>::tiny)) {
      if (tid == 0) {
        w.tau[j] = R(0.0);
        w.e[j] = x0;
        w.dg[j] = As[(size_t)j * la + j];
      }
      __syncthreads();
      continue;
    }
    const R beta = x0 >= R(0.0) ? -alpha : alpha;
    const R tj = (beta - x0) / beta;
    const R scale = R(1.0) / (x0 - beta);
    for (int i = tid; i < m; i += kThreads) {
      const R v = i == 0 ? R(1.0) : As[(size_t)(j + 1 + i) * la + j] * scale;
      vt[i] = v;
      w.ref[(size_t)j * n + j + 1 + i] = v;
    }
    if (tid == 0) {
      w.tau[j] = tj;
      w.e[j] = beta;
      w.dg[j] = As[(size_t)j * la + j];
    }
    __syncthreads();
    for (int i = wid; i < m; i += kWarps) {  // p = tau A22 v
      const R* row = As + (size_t)(j + 1 + i) * n + (j + 1);
      R acc = R(0.0);
      for (int l = lane; l < m; l += 32) acc += row[l] * vt[l];
      acc = warp_sum(acc);
      if (lane == 0) pw[i] = tj * acc;
    }
    __syncthreads();
    R kp = R(0.0);
    for (int i = tid; i < m; i += kThreads) kp += pw[i] * vt[i];
    const R K = R(0.5) * tj * block_sum(kp, red);
    __syncthreads();
    for (int i = tid; i < m; i += kThreads) pw[i] -= K * vt[i];
    __syncthreads();
    for (int i = wid; i < m; i += kWarps) {  // A22 -= v w^T + w v^T
      R* row = As + (size_t)(j + 1 + i) * n + (j + 1);
      const R vi = vt[i], wi = pw[i];
      for (int l = lane; l < m; l += 32) row[l] -= vi * pw[l] + wi * vt[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      w.dg[n - 2] = As[(size_t)(n - 2) * la + (n - 2)];
      w.e[n - 2] = As[(size_t)(n - 1) * la + (n - 2)];
      w.tau[n - 2] = R(0.0);
    }
    w.dg[n - 1] = As[(size_t)(n - 1) * la + (n - 1)];
    w.e[n - 1] = R(0.0);
    w.tau[n - 1] = R(0.0);
  }
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) w.e2[i] = w.e[i] * w.e[i];
}

// ------------------------------------------------------------------ 1b. cluster Householder
// Householder tridiagonalisation of the transformed n x n matrix (w.As) by a
// cluster of CS thread blocks: row r lives in block r % CS (distributed
// shared memory), so the O(n^3) work is spread over CS SMs.  Every block
// holds column j of the current matrix (cf, two buffers); a step
//   1. forms the reflector in every warp (the norm by a warp reduction over
//      the block's copy of column j: the same values everywhere, no barrier;
//      v is formed from column j where it is read);
//   2. computes p = tau A v for the block's rows (a warp per row, four rows
//      at a time) and publishes p, the warps' shares of p^T v and the rows'
//      entries of column j+1 before the update;
//   3. after one cluster barrier, gathers in one round of remote loads (at
//      most one or two per thread) p, the column-j+1 entries and the shares of all
//      blocks into its own shared memory;
//   4. after a block barrier, forms K = tau p^T v / 2, w = p - K v, the
//      updated column j+1 (into the other buffer) and updates its rows
//      (A -= v w^T + w v^T); a block barrier ends the step.
// The published buffers alternate between steps, so no barrier guards their
// reuse.
// The cluster has 16 blocks where the GPU can place such clusters (a
// non-portable size; 8 otherwise) of 512 threads: on n = 216 in FP32 that
// measured 560 us a call against 627 us for 8 blocks of 256 threads.
constexpr int kCT = 512;
constexpr int kCW = kCT / 32;

template <class R, int CS>
__global__ void __launch_bounds__(kCT) k_rr_house_cluster(int n, RRWork<R> w) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rpc = (n + CS - 1) / CS;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* Ar = reinterpret_cast<R*>(sm_raw);  // rpc x n: row rank + CS * li
  R* cf = Ar + (size_t)rpc * n;          // 2 x n: column j (alternating)
  R* wl = cf + 2 * n;                    // n: the gathered p
  R* cn = wl + n;                        // n: the gathered entries of column j+1
  R* kall = cn + n;                      // CS x kCW: the gathered shares of p^T v
  R* pubc = kall + CS * kCW;            // 2 x rpc: own rows' entries of column j+1
  R* pubp = pubc + 2 * rpc;              // 2 x rpc: own rows' p
  R* pubk = pubp + 2 * rpc;              // 2 x kCW: the warps' shares of p^T v
  for (int t = tid; t < rpc * n; t += kCT) {
    const int li = t / n, c = t - li * n, r = rank + CS * li;
    Ar[t] = r < n ? w.As[(size_t)r * n + c] : R(0.0);
  }
  for (int l = tid; l < n; l += kCT) cf[l] = l >= 1 ? w.As[(size_t)l * n] : R(0.0);
  __syncthreads();
  cl.sync();  // every block of the cluster runs before the first remote access
  for (int j = 0; j + 2 < n; ++j) {
    const int buf = j & 1;
    const R* cur = cf + buf * n;
    R* nxt = cf + (buf ^ 1) * n;
    // 1. the reflector, in every warp
    R ss = R(0.0);
    for (int l = j + 1 + lane; l < n; l += 32) ss += cur[l] * cur[l];
    ss = warp_sum(ss);
    const R x0 = cur[j + 1];
    const R alpha = sqrt(ss);
    const bool refl = alpha > Prec<R>::tiny;
    const R beta = x0 >= R(0.0) ? -alpha : alpha;
    const R tj = refl ? (beta - x0) / beta : R(0.0);
    const R scale = refl ? R(1.0) / (x0 - beta) : R(0.0);
    const R v1 = refl ? R(1.0) : R(0.0);  // v_{j+1}
    if (rank == 0 && wid == 0) {
      for (int l = j + 1 + lane; l < n; l += 32)
        w.ref[(size_t)j * n + l] = l == j + 1 ? v1 : cur[l] * scale;
      if (lane == 0) {
        w.tau[j] = tj;
        w.e[j] = refl ? beta : x0;
      }
    }
    if ((j % CS) == rank && wid == (j / CS) % kCW && lane == 0)
      w.dg[j] = Ar[(size_t)(j / CS) * n + j];
    // 2. p = tau A v for own rows r >= j+1, four rows of a warp at a time
    R kp = R(0.0);
    for (int l0 = wid; l0 < rpc; l0 += 4 * kCW) {
      R acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = R(0.0);
        const int li = l0 + q * kCW, r = rank + CS * li;
        if (li < rpc && r < n && r >= j + 1) {
          const R* row = Ar + (size_t)li * n;
          for (int l = j + 1 + lane; l < n; l += 32)
            acc[q] += row[l] * (l == j + 1 ? v1 : cur[l] * scale);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = warp_sum(acc[q]) * tj;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int li = l0 + q * kCW, r = rank + CS * li;
        if (li < rpc && r < n && r >= j + 1) {
          kp += acc[q] * (r == j + 1 ? v1 : cur[r] * scale);
          if (lane == 0) {
            pubp[buf * rpc + li] = acc[q];
            pubc[buf * rpc + li] = Ar[(size_t)li * n + j + 1];
          }
        }
      }
    }
    if (lane == 0) pubk[buf * kCW + wid] = kp;
    cl.sync();
    // 3. one round of remote loads
    for (int l = j + 1 + tid; l < n; l += kCT) {
      const int owner = l % CS, ol = l / CS;
      wl[l] = cl.map_shared_rank(pubp, owner)[buf * rpc + ol];
      cn[l] = cl.map_shared_rank(pubc, owner)[buf * rpc + ol];
    }
    if (tid < CS * kCW) kall[tid] = cl.map_shared_rank(pubk, tid / kCW)[buf * kCW + tid % kCW];
    __syncthreads();
    // 4. K, w, the next column and the update of own rows
    R kq = R(0.0);
    for (int q = lane; q < CS * kCW; q += 32) kq += kall[q];
    const R K = R(0.5) * tj * warp_sum(kq);
    const R wn = wl[j + 1] - K * v1;  // w_{j+1}
    for (int l = j + 2 + tid; l < n; l += kCT) {
      const R vl = cur[l] * scale, wv = wl[l] - K * vl;
      nxt[l] = cn[l] - (vl * wn + wv * v1);
    }
    for (int li = wid; li < rpc; li += kCW) {
      const int r = rank + CS * li;
      if (r >= n || r < j + 1) continue;
      R* row = Ar + (size_t)li * n;
      const R vr = r == j + 1 ? v1 : cur[r] * scale, wr = wl[r] - K * vr;
      for (int l = j + 1 + lane; l < n; l += 32) {
        const R vl = l == j + 1 ? v1 : cur[l] * scale;
        row[l] -= vr * (wl[l] - K * vl) + wr * vl;
      }
    }
    __syncthreads();
  }
  // the last 2 x 2 block
  if (tid == 0) {
    for (int r = (n >= 2 ? n - 2 : 0); r < n; ++r) {
      if (r % CS != rank) continue;
      const R* row = Ar + (size_t)(r / CS) * n;
      w.dg[r] = row[r];
      if (r == n - 1 && n >= 2) w.e[n - 2] = row[n - 2];
    }
    if (rank == 0) {
      if (n >= 2) w.tau[n - 2] = R(0.0);
      w.tau[n - 1] = R(0.0);
      w.e[n - 1] = R(0.0);
    }
  }
  __threadfence();
  cl.sync();  // also: no block leaves while another may still read its buffers
  if (rank == 0)
    for (int i = tid; i < n; i += kCT) w.e2[i] = w.e[i] * w.e[i];
}

// ------------------------------------------------------------------ 2b. eigenvalues, one block each
// FP64 multisection with the division-free Sturm count: one warp per
// eigenvalue, 32 probes per round (a 33-fold shrink of the bracket per round).
// The count is the number of sign changes along the leading principal minors
// p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1), rescaled by exact
// powers of two to stay in range, a zero minor taking the sign opposite to
// its predecessor; the sign and range tests run on the bit patterns (integer
// instructions): per step three floating-point instructions, which matters in
// FP64 on GB300 (64 cycles per FP64 warp instruction).
__device__ __forceinline__ long long bits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ int bits(float v) { return __float_as_int(v); }
template <class R>
__device__ int sturm_bits(const R* d, const R* e2, int n, R x) {
  using I = decltype(bits(R(0)));
  constexpr int kSign = 8 * (int)sizeof(R) - 1;
  constexpr int kMant = sizeof(R) == 8 ? 52 : 23;
  constexpr int kBias = sizeof(R) == 8 ? 1023 : 127;
  constexpr int kMask = sizeof(R) == 8 ? 0x7ff : 0xff;
  constexpr int kSpan = sizeof(R) == 8 ? 600 : 60;
  R pm = R(1.0), p = d[0] - x;
  I bp = bits(p);
  if ((bp << 1) == 0) {
    p = -Prec<R>::tiny;
    bp = bits(p);
  }
  int c = (int)((unsigned long long)(bp >> kSign) & 1ull);
  for (int i = 1; i < n; ++i) {
    R q = fma(d[i] - x, p, -e2[i - 1] * pm);
    I bq = bits(q);
    if ((bq << 1) == 0) {  // a zero minor takes the sign opposite to its predecessor
      q = bp < 0 ? Prec<R>::tiny : -Prec<R>::tiny;
      bq = bits(q);
    }
    c += (int)((unsigned long long)((bq ^ bp) >> kSign) & 1ull);
    pm = p;
    p = q;
    bp = bq;
    const int ex = (int)((bq >> kMant) & kMask) - kBias;
    if (ex > kSpan || ex < -kSpan) {
      p = scalbn_r(p, -ex);
      pm = scalbn_r(pm, -ex);
      bp = bits(p);
    }
  }
  return c;
}

// Double-float: the sign, zero and exponent tests on the (normalised) head.
template <>
__device__ int sturm_bits<dfloat>(const dfloat* d, const dfloat* e2, int n, dfloat x) {
  dfloat pm(1.0f), p = d[0] - x;
  if (p.h == 0.f) p = -Prec<dfloat>::tiny;
  int c = p.h < 0.f;
  for (int i = 1; i < n; ++i) {
    dfloat q = df_add(df_mul(d[i] - x, p), -df_mul(e2[i - 1], pm));
    if (q.h == 0.f) q = p.h < 0.f ? Prec<dfloat>::tiny : -Prec<dfloat>::tiny;
    c += (q.h < 0.f) != (p.h < 0.f);
    pm = p;
    p = q;
    const int ex = ilogbf(p.h);
    if (ex > 60 || ex < -60) {
      p = scalbn_r(p, -ex);
      pm = scalbn_r(pm, -ex);
    }
  }
  return c;
}

// One block of kEW warps per eigenvalue s: multisection with 32 kEW probes a
// round, first on FP32 copies of the tridiagonal (cheap bracketing to FP32
// resolution), then in the working precision from the FP32 bracket widened by
// its error bound and checked by working-precision counts.
constexpr int kEW = 4;
template <class R>
__device__ void multisection(const R* d, const R* e2, int n, int s, R& a, R& b, int max_rounds,
                             R rel, int* sfirst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NP = 32 * kEW;
  for (int round = 0; round < max_rounds; ++round) {
    const R x = a + (b - a) * (R)(threadIdx.x + 1) / (R)(NP + 1);
    const int cnt = sturm_bits<R>(d, e2, n, x);
    const unsigned above = __ballot_sync(0xffffffffu, cnt >= s + 1);
    if (lane == 0) sfirst[wid] = above ? 32 * wid + __ffs(above) - 1 : NP;
    __syncthreads();
    int first = NP;
    for (int q = 0; q < kEW; ++q) first = min(first, sfirst[q]);
    const R na = first == 0 ? a : a + (b - a) * (R)first / (R)(NP + 1);
    const R nbv = first == NP ? b : a + (b - a) * (R)(first + 1) / (R)(NP + 1);
    a = na;
    b = nbv;
    __syncthreads();
    if (b - a <= rel * fmax(fabs(a), fabs(b))) break;
  }
}

template <class R>
__global__ void __launch_bounds__(32 * kEW)
    k_rr_eigvals_mc(int n, int nb, RRWork<R> w, double* theta) {
  extern __shared__ __align__(16) unsigned char ev_raw[];
  R* d = reinterpret_cast<R*>(ev_raw);
  R* e2 = d + n;
  float* d32 = reinterpret_cast<float*>(e2 + n);
  float* e32 = d32 + n;
  __shared__ int sfirst[kEW];
  __shared__ R red[2 * kEW];
  const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  R lo = R(0.0), hi = R(0.0);
  bool any = false;
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = w.dg[i];
    e2[i] = w.e2[i];
    d32[i] = (float)w.dg[i];
    e32[i] = (float)w.e2[i];
    const R r = (i > 0 ? fabs(w.e[i - 1]) : R(0.0)) + (i + 1 < n ? fabs(w.e[i]) : R(0.0));
    const R a = w.dg[i] - r, b = w.dg[i] + r;
    lo = any ? fmin(lo, a) : a;
    hi = any ? fmax(hi, b) : b;
    any = true;
  }
  if (!any) {
    lo = R(1e30);
    hi = R(-1e30);
  }
  for (int o = 16; o; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    red[wid] = lo;
    red[kEW + wid] = hi;
  }
  __syncthreads();
  lo = red[0];
  hi = red[kEW];
  for (int q = 1; q < kEW; ++q) {
    lo = fmin(lo, red[q]);
    hi = fmax(hi, red[kEW + q]);
  }
  const R span = fmax(hi - lo, R(1e-30));
  lo -= span * R(1e-6);
  hi += span * R(1e-6);
  R a = lo, b = hi;
  if (sizeof(R) == 8) {
    // FP32 bracket, then widened by the FP32 count's error bound
    float a32 = (float)lo, b32 = (float)hi;
    multisection<float>(d32, e32, n, s, a32, b32, 16, 4.f * Prec<float>::eps, sfirst);
    const R tnorm = fmax(fabs(lo), fabs(hi));
    const R pad = R(64.0) * R(6e-8) * tnorm;
    a = fmax(lo, (R)a32 - pad);
    b = fmin(hi, (R)b32 + pad);
    // keep the bracket only if working-precision counts confirm it
    if (tid == 0) {
      sfirst[0] = sturm_bits<R>(d, e2, n, a) <= s;
      sfirst[1] = sturm_bits<R>(d, e2, n, b) >= s + 1;
    }
    __syncthreads();
    if (!sfirst[0]) a = lo;
    if (!sfirst[1]) b = hi;
    __syncthreads();
  }
  multisection<R>(d, e2, n, s, a, b, 64, R(4.0) * Prec<R>::eps, sfirst);
  if (tid == 0) {
    w.lam[s] = R(0.5) * (a + b);
    theta[s] = (double)(R(0.5) * (a + b));
  }
}

// ------------------------------------------------------------------ 3b. inverse iteration in shared memory
// kIV threads per block, one vector each, their LU factors in shared memory
// (one thread per block: the pivoting branches of different vectors diverge)
constexpr int kIV = 1;
template <class R>
__global__ void k_rr_invit_sm(int n, int nb, RRWork<R> w) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* sm = reinterpret_cast<R*>(sm_raw);
  const int s = blockIdx.x * kIV + threadIdx.x;
  R* u = sm + (size_t)threadIdx.x * 6 * n;
  if (s >= nb) return;
  R lo = R(0.0), hi = R(0.0);
  for (int i = 0; i < n; ++i) {
    const R r = (i > 0 ? fabs(w.e[i - 1]) : R(0.0)) + (i + 1 < n ? fabs(w.e[i]) : R(0.0));
    const R a = w.dg[i] - r, b = w.dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
  }
  const R span = fmax(hi - lo, R(1e-30));
  const R tnorm = fmax(fabs(lo - span * R(1e-6)), fabs(hi + span * R(1e-6)));
  const R pivmin = fmax(Prec<R>::tiny, Prec<R>::eps * tnorm * R(1e-6));
  R* u1 = u + n;
  R* u2 = u1 + n;
  R* lm = u2 + n;
  R* sw = lm + n;
  R* z = sw + n;
  const R lam = w.lam[s];
  const R shift = lam + Prec<R>::eps * fmax(fabs(lam), span * R(1e-3)) * R(4.0);
  R a_i = w.dg[0] - shift, b_i = n > 1 ? w.e[0] : R(0.0), c_i = R(0.0);
  for (int i = 0; i < n - 1; ++i) {
    const R sub = w.e[i];
    const R d1 = w.dg[i + 1] - shift;
    const R e1 = i + 2 < n ? w.e[i + 1] : R(0.0);
    if (fabs(a_i) >= fabs(sub)) {
      const R pv = fabs(a_i) < pivmin ? (a_i < R(0.0) ? -pivmin : pivmin) : a_i;
      const R l = sub / pv;
      u[i] = pv; u1[i] = b_i; u2[i] = c_i; lm[i] = l; sw[i] = R(0.0);
      a_i = d1 - l * b_i;
      b_i = e1 - l * c_i;
      c_i = R(0.0);
    } else {
      const R l = a_i / sub;
      u[i] = sub; u1[i] = d1; u2[i] = e1; lm[i] = l; sw[i] = R(1.0);
      const R na = b_i - l * d1, nc = c_i - l * e1;
      a_i = na;
      b_i = nc;
      c_i = R(0.0);
    }
  }
  u[n - 1] = fabs(a_i) < pivmin ? (a_i < R(0.0) ? -pivmin : pivmin) : a_i;
  u1[n - 1] = R(0.0);
  u2[n - 1] = R(0.0);
  // the pivots' reciprocals, once: the substitutions below then multiply
  // (independent divisions here instead of one on every step of the chain)
  for (int i = 0; i < n; ++i) u[i] = R(1.0) / u[i];
  unsigned int h = 2166136261u ^ (unsigned)s * 16777619u;
  for (int i = 0; i < n; ++i) {
    h = h * 1664525u + 1013904223u;
    z[i] = R(0.5) + (R)((h >> 8) & 0xffff) / R(65536.0);
  }
  for (int iter = 0; iter < 3; ++iter) {
    for (int i = 0; i < n - 1; ++i) {
      if (sw[i] != R(0.0)) {
        const R t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t - lm[i] * z[i];
      } else {
        z[i + 1] -= lm[i] * z[i];
      }
    }
    for (int i = n - 1; i >= 0; --i) {
      R t = z[i];
      if (i + 1 < n) t -= u1[i] * z[i + 1];
      if (i + 2 < n) t -= u2[i] * z[i + 2];
      z[i] = t * u[i];
    }
    R nrm = R(0.0);
    for (int i = 0; i < n; ++i) nrm = fmax(nrm, fabs(z[i]));
    const R inv = nrm > R(0.0) ? R(1.0) / nrm : R(1.0);
    for (int i = 0; i < n; ++i) z[i] *= inv;
  }
  for (int i = 0; i < n; ++i) w.V[(size_t)i * nb + s] = z[i];
}

// ------------------------------------------------------------------ small dense products over many blocks
// The Gram matrices and the product of the momentum step and the first Gram
// of Cholesky QR, spread over the SMs (on one SM in double-float they cost
// several hundred thousand cycles): G = X_{r0:r1}^T Y_{r0:r1} (lower: only
// the lower triangle) with a warp per 4 x 4 tile of G, lanes over rows; and
// T = Zp - V G (Zp = V with rows below r0 zero) with a thread per 4 entries.
template <class R>
__global__ void __launch_bounds__(256)
    k_rr_gram_mb(const R* __restrict__ X, int ldx, const R* __restrict__ Y, int ldy, int r0,
                 int r1, int ma, int mb, R* __restrict__ G, int ldg, int lower) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int ta = (ma + 3) >> 2, tb = (mb + 3) >> 2;
  if (t >= ta * tb) return;
  const int ia = t / tb, ib = t - ia * tb;
  if (lower && ib > ia) return;
  R acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = R(0.0);
  for (int i = r0 + lane; i < r1; i += 32) {
    R xa[4], yb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      xa[r] = 4 * ia + r < ma ? X[(size_t)i * ldx + 4 * ia + r] : R(0.0);
      yb[r] = 4 * ib + r < mb ? Y[(size_t)i * ldy + 4 * ib + r] : R(0.0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[4 * r + c] += xa[r] * yb[c];
  }
  const R sm = sum16(acc);
  const int q = lane >> 1, a = 4 * ia + (q >> 2), b = 4 * ib + (q & 3);
  if (!(lane & 1) && a < ma && b < mb && (!lower || b <= a)) G[(size_t)a * ldg + b] = sm;
}

template <class R>
__global__ void __launch_bounds__(256)
    k_rr_zp_mb(const R* __restrict__ V, const R* __restrict__ G, int n, int nb, int r0,
               R* __restrict__ T) {
  const int tq = (nb + 3) >> 2;
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  if (t >= (long long)n * tq) return;
  const int i = (int)(t / tq), c0 = 4 * (int)(t - (long long)i * tq);
  const R* vi = V + (size_t)i * nb;
  R acc[4] = {R(0.0), R(0.0), R(0.0), R(0.0)};
  for (int a = 0; a < nb; ++a) {
    const R va = vi[a];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c0 + c < nb) acc[c] += va * G[(size_t)a * nb + c0 + c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (c0 + c < nb) T[(size_t)i * nb + c0 + c] = (i >= r0 ? vi[c0 + c] : R(0.0)) - acc[c];
}

// ------------------------------------------------------------------ 4a. Cholesky QR of the tridiagonal eigenvectors (twice unless once is enough)
// First pass: the Gram V^T V over many blocks (k_rr_gram_mb), its factor in
// one block (k_rr_cqchol, which also decides whether a second pass is
// needed), V <- V L^-T over blocks of rows (k_rr_rsolve); the second pass,
// when needed, in one block (k_rr_cholqr, which returns at once otherwise).
template <class R>
__global__ void __launch_bounds__(kThreads) k_rr_cqchol(int nb, RRWork<R> w, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* G = lsm ? reinterpret_cast<R*>(dyn_raw) : w.G;
  __shared__ int keep_nb[512];
  __shared__ float s_off[kWarps];
  if (lsm)
    for (int t = threadIdx.x; t < nb * nb; t += kThreads) G[t] = w.G[t];
  for (int s2 = threadIdx.x; s2 < nb; s2 += kThreads) keep_nb[s2] = 1;
  __syncthreads();
  // largest off-diagonal of the normalised Gram matrix: at most 1e-3 means
  // (Gershgorin) a condition number below (1 + nb 1e-3) / (1 - nb 1e-3),
  // and one pass leaves the vectors orthonormal to a few units of rounding
  float off = 0.f;
  for (int t = threadIdx.x; t < nb * nb; t += kThreads) {
    const int a = t / nb, b = t - a * nb;
    if (b < a)
      off = fmaxf(off, fabsf((float)G[(size_t)a * nb + b]) /
                           sqrtf((float)G[(size_t)a * nb + a] * (float)G[(size_t)b * nb + b]));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
  if ((threadIdx.x & 31) == 0) s_off[threadIdx.x >> 5] = off;
  __syncthreads();
  off = 0.f;
  for (int q = 0; q < kWarps; ++q) off = fmaxf(off, s_off[q]);
  block_cholesky(G, nb, keep_nb, R(0.0));
  if (threadIdx.x == 0) *w.flag = !(nb * 1e-3f < 0.5f && off <= 1e-3f);
  if (lsm)
    for (int t = threadIdx.x; t < nb * nb; t += kThreads) w.G[t] = G[t];
}
// The second pass.  SM: V (n x nb) and G staged in shared memory (dynamic),
// else worked on in the global workspace
template <class R, bool SM>
__global__ void __launch_bounds__(kThreads) k_rr_cholqr(int n, int nb, RRWork<R> w) {
  if (!*w.flag) return;  // one pass was enough
  __shared__ int keep_nb[512];
  extern __shared__ __align__(16) unsigned char cq_raw[];
  // in shared memory V's rows are padded to an odd stride, so that a thread
  // per row (and the Gram's lanes over rows) hit distinct banks
  const int lv = SM ? (nb | 1) : nb;
  R* V = SM ? reinterpret_cast<R*>(cq_raw) : w.V;
  R* G = SM ? V + (size_t)n * lv : w.G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (SM) {
    for (int i = wid; i < n; i += kWarps)
      for (int c = lane; c < nb; c += 32) V[(size_t)i * lv + c] = w.V[(size_t)i * nb + c];
    __syncthreads();
  }
  blk_gram_tn(V, lv, V, lv, n, nb, nb, G, nb, true);
  for (int s2 = threadIdx.x; s2 < nb; s2 += kThreads) keep_nb[s2] = 1;
  __syncthreads();
  block_cholesky(G, nb, keep_nb, R(0.0));
  block_trsm_rt(G, nb, V, lv, n);  // V <- V L^-T
  if (SM)
    for (int i = wid; i < n; i += kWarps)
      for (int c = lane; c < nb; c += 32) w.V[(size_t)i * nb + c] = V[(size_t)i * lv + c];
}

// ------------------------------------------------------------------ 4b. back-transform, blocked
// The reflectors are applied in groups of kWY in compact WY form: H_j0 ...
// H_{j0+b-1} = I - V T V^T with V the group's vectors (v_j zero above row
// j + 1) and T upper triangular, T_ii = tau_i and T_{0:i,i} = -tau_i
// T_{0:i,0:i} V_{:,0:i}^T v_i.  k_rr_wy_t builds T for every group (a block
// per group: the V^T V products by warps, the recurrence by one thread);
// k_rr_backtransform applies the groups, last first, to kBW vectors per
// block: W = V^T Z, W <- T W, Z -= V W, each a product over the block's
// threads, so a group costs four block barriers instead of kWY dependent
// warp reductions per vector.
constexpr int kWY = 8;
constexpr int kBW = 8;

template <class R>
__global__ void __launch_bounds__(256) k_rr_wy_t(int n, RRWork<R> w, R* __restrict__ T) {
  __shared__ R dd[kWY * kWY];
  const int g = blockIdx.x, j0 = g * kWY, b = min(kWY, n - 2 - j0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = wid; q < kWY * kWY; q += 8) {
    const int k = q / kWY, i = q - k * kWY;
    if (!(k < i && i < b)) continue;
    if (w.tau[j0 + k] == R(0.0) || w.tau[j0 + i] == R(0.0)) {  // H = I: v need not be set
      if (lane == 0) dd[q] = R(0.0);
      continue;
    }
    const R* vk = w.ref + (size_t)(j0 + k) * n;
    const R* vi = w.ref + (size_t)(j0 + i) * n;
    R acc = R(0.0);
    for (int l = j0 + i + 1 + lane; l < n; l += 32) acc += vk[l] * vi[l];
    acc = warp_sum(acc);
    if (lane == 0) dd[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R t[kWY * kWY];
#pragma unroll
    for (int q = 0; q < kWY * kWY; ++q) t[q] = R(0.0);
    for (int i = 0; i < b; ++i) {
      const R ti = w.tau[j0 + i];
      for (int k = 0; k < i; ++k) {
        R s = R(0.0);
        for (int m = k; m < i; ++m) s += t[k * kWY + m] * dd[m * kWY + i];
        t[k * kWY + i] = -ti * s;
      }
      t[i * kWY + i] = ti;
    }
    for (int q = 0; q < kWY * kWY; ++q) T[(size_t)g * kWY * kWY + q] = t[q];
  }
}

template <class R>
__global__ void __launch_bounds__(32 * kBW) k_rr_backtransform(int n, int nb, RRWork<R> w,
                                                               const R* __restrict__ T) {
  extern __shared__ __align__(16) unsigned char z_raw[];
  R* Z = reinterpret_cast<R*>(z_raw);  // n x kBW: the block's vectors, row-major
  R* V = Z + (size_t)n * kBW;          // kWY x n: the group's reflectors
  __shared__ R W[kWY * kBW], W2[kWY * kBW];
  const int tid = threadIdx.x, s0 = blockIdx.x * kBW;
  const int ns = min(kBW, nb - s0);
  for (int t = tid; t < n * kBW; t += blockDim.x) {
    const int i = t / kBW, s = t - i * kBW;
    Z[t] = s < ns ? w.V[(size_t)i * nb + s0 + s] : R(0.0);
  }
  const int ng = n > 2 ? (n - 2 + kWY - 1) / kWY : 0;
  for (int g = ng - 1; g >= 0; --g) {
    const int j0 = g * kWY, b = min(kWY, n - 2 - j0);
    for (int t = tid; t < kWY * n; t += blockDim.x) {
      const int k = t / n, l = t - k * n;
      V[t] = (k < b && l >= j0 + k + 1 && !(w.tau[j0 + k] == R(0.0)))
                 ? w.ref[(size_t)(j0 + k) * n + l]
                 : R(0.0);
    }
    __syncthreads();
    // W = V^T Z: four threads per entry over rows l = p mod 4
    {
      const int o = tid >> 2, p = tid & 3, k = o / kBW, s = o - k * kBW;
      R acc = R(0.0);
      if (k < b)
        for (int l = j0 + k + 1 + p; l < n; l += 4) acc += V[(size_t)k * n + l] * Z[(size_t)l * kBW + s];
      acc += shfl_xor_r(acc, 1);
      acc += shfl_xor_r(acc, 2);
      if (p == 0) W[o] = acc;
    }
    __syncthreads();
    if (tid < kWY * kBW) {  // W <- T W
      const int k = tid / kBW, s = tid - k * kBW;
      const R* tg = T + (size_t)g * kWY * kWY;
      R acc = R(0.0);
      for (int m = k; m < b; ++m) acc += tg[k * kWY + m] * W[m * kBW + s];
      W2[tid] = acc;
    }
    __syncthreads();
    for (int t = tid; t < (n - j0 - 1) * kBW; t += blockDim.x) {  // Z -= V W
      const int l = j0 + 1 + t / kBW, s = t % kBW;
      R acc = R(0.0);
#pragma unroll
      for (int k = 0; k < kWY; ++k) acc += V[(size_t)k * n + l] * W2[k * kBW + s];
      Z[(size_t)l * kBW + s] -= acc;
    }
    __syncthreads();
  }
  for (int t = tid; t < n * kBW; t += blockDim.x) {
    const int i = t / kBW, s = t - i * kBW;
    if (s < ns) w.V[(size_t)i * nb + s0 + s] = Z[t];
  }
}

// ------------------------------------------------------------------ 4c. momentum and mapping back
// The momentum coefficients Z (the W and P rows of the Ritz vectors,
// orthogonalised against them and orthonormalised -- the next P = S Z is
// then M-orthonormal and M-orthogonal to the next X), from the multi-block
// launches' Z = Zp - V G (w.T1) and Z^T Z (w.G): the factor of Z^T Z with
// drop in one block (k_rr_mchol, which also counts the basis columns the
// step dropped), Z <- Z L^-T with dropped columns zero over blocks of rows
// (k_rr_rsolve), and the O rows of V and Z mapped back through the
// transform's factor, y_O <- L^-T y_O, over blocks of columns (k_rr_bsolve);
// then y_rest <- y_rest - C y_O and y <- D y (k_rr_output).
template <class R>
__global__ void __launch_bounds__(kThreads)
    k_rr_mchol(int n, int nb, int want_p, RRWork<R> w, int* __restrict__ dropped, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* G = lsm ? reinterpret_cast<R*>(dyn_raw) : w.G;
  __shared__ int keep_nb[512];
  const int tid = threadIdx.x;
  if (want_p) {
    if (lsm)
      for (int t = tid; t < nb * nb; t += kThreads) G[t] = w.G[t];
    for (int s2 = tid; s2 < nb; s2 += kThreads) keep_nb[s2] = 1;
    __syncthreads();
    R gref = R(0.0);
    for (int s2 = 0; s2 < nb; ++s2) gref = fmax(gref, G[s2 * nb + s2]);
    block_cholesky(G, nb, keep_nb, Prec<R>::drop * fmax(gref, Prec<R>::tiny));
    for (int s2 = tid; s2 < nb; s2 += kThreads) w.keepz[s2] = keep_nb[s2];
    if (lsm)
      for (int t = tid; t < nb * nb; t += kThreads) w.G[t] = G[t];
  }
  if (tid == 0) {
    int dc = 0;
    for (int a = 0; a < n; ++a) dc += !w.keep[a];
    *dropped = dc;
  }
}

// Xout <- Xin L^-T for `rows` rows (m entries each; L as block_cholesky
// leaves it, ld m), entries of columns with mask[c] == 0 set to zero: a
// block per cb rows (Xout may be Xin: a block writes only the rows it read)
template <class R>
__global__ void __launch_bounds__(256)
    k_rr_rsolve(const R* __restrict__ Lg, int m, const R* Xin, int ldin, R* Xout, int ldout,
                int rows, const int* __restrict__ mask, int cb, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* dyn = reinterpret_cast<R*>(dyn_raw);
  const R* L = lsm ? dyn : Lg;
  R* Xs = dyn + (lsm ? (size_t)m * m : 0);
  const int lx = m | 1, r0 = blockIdx.x * cb, nr = min(cb, rows - r0);
  if (lsm)
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) dyn[t] = Lg[t];
  for (int t = threadIdx.x; t < nr * m; t += blockDim.x) {
    const int r = t / m, c = t - r * m;
    Xs[(size_t)r * lx + c] = Xin[(size_t)(r0 + r) * ldin + c];
  }
  __syncthreads();
  block_trsm_rt(L, m, Xs, lx, nr);
  for (int t = threadIdx.x; t < nr * m; t += blockDim.x) {
    const int r = t / m, c = t - r * m;
    Xout[(size_t)(r0 + r) * ldout + c] = (mask && !mask[c]) ? R(0.0) : Xs[(size_t)r * lx + c];
  }
}

// the O rows of V (columns 0..nb-1) and Z (columns nb..ncol-1): y_O <-
// L^-T y_O, a block per cb columns
template <class R>
__global__ void __launch_bounds__(256)
    k_rr_bsolve(const R* __restrict__ Lg, int no, int o0, R* __restrict__ V, R* __restrict__ Z,
                int nb, int ncol, int cb, int lsm) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  R* dyn = reinterpret_cast<R*>(dyn_raw);
  const R* L = lsm ? dyn : Lg;
  R* Xs = dyn + (lsm ? (size_t)no * no : 0);  // no x cb
  const int c0 = blockIdx.x * cb, nc = min(cb, ncol - c0);
  if (lsm)
    for (int t = threadIdx.x; t < no * no; t += blockDim.x) dyn[t] = Lg[t];
  for (int t = threadIdx.x; t < no * nc; t += blockDim.x) {
    const int a = t / nc, c = t - a * nc, col = c0 + c;
    Xs[(size_t)a * cb + c] =
        col < nb ? V[(size_t)(o0 + a) * nb + col] : Z[(size_t)(o0 + a) * nb + col - nb];
  }
  __syncthreads();
  block_trsm_lt(L, no, Xs, cb, nc);
  for (int t = threadIdx.x; t < no * nc; t += blockDim.x) {
    const int a = t / nc, c = t - a * nc, col = c0 + c;
    if (col < nb)
      V[(size_t)(o0 + a) * nb + col] = Xs[(size_t)a * cb + c];
    else
      Z[(size_t)(o0 + a) * nb + col - nb] = Xs[(size_t)a * cb + c];
  }
}

// Output, one block per row i: undo the coefficient-space projection
// (y_i -= sum_a C_ia y_{o0+a} for rows outside O) and scale, for the Ritz
// vectors V and the momentum coefficients Z.
template <class R, class T>
__global__ void k_rr_output(int n, int o0, int no, int nb, int want_p, RRWork<R> w,
                            T* __restrict__ YZ) {
  const int i = blockIdx.x;
  const bool in_o = i >= o0 && i < o0 + no;
  const R d = w.dsc[i];
  for (int c = threadIdx.x; c < 2 * nb; c += blockDim.x) {
    T* out = YZ + (size_t)i * 2 * nb + c;
    if (c >= nb && !want_p) {
      *out = T(0);
      continue;
    }
    const R* M_ = c < nb ? w.V : w.Z;
    const int cc = c < nb ? c : c - nb;
    R acc = M_[(size_t)i * nb + cc];
    if (!in_o)
      for (int a = 0; a < no; ++a) acc -= w.C[i * no + a] * M_[(size_t)(o0 + a) * nb + cc];
    *out = (T)(acc * d);
  }
}

// ------------------------------------------------------------------ R(3.) inverse iteration
template <class R>
__global__ void k_rr_invit(int n, int nb, RRWork<R> w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  R lo = R(0.0), hi = R(0.0);
  for (int i = 0; i < n; ++i) {
    const R r = (i > 0 ? fabs(w.e[i - 1]) : R(0.0)) + (i + 1 < n ? fabs(w.e[i]) : R(0.0));
    const R a = w.dg[i] - r, b = w.dg[i] + r;
    if (i == 0 || a < lo) lo = a;
    if (i == 0 || b > hi) hi = b;
  }
  const R span = fmax(hi - lo, R(1e-30));
  const R tnorm = fmax(fabs(lo - span * R(1e-6)), fabs(hi + span * R(1e-6)));
  const R pivmin = fmax(Prec<R>::tiny, Prec<R>::eps * tnorm * R(1e-6));
  R* u = w.scr + (size_t)s * 6 * n;  // U diagonal
  R* u1 = u + n;                     // first super-diagonal
  R* u2 = u1 + n;                    // second super-diagonal (pivoting fill)
  R* lm = u2 + n;                    // multipliers
  R* sw = lm + n;                    // row-swap flags
  R* z = sw + n;                     // the vector
  const R lam = w.lam[s];
  // a slightly perturbed shift keeps T - shift I from being exactly singular
  const R shift = lam + Prec<R>::eps * fmax(fabs(lam), span * R(1e-3)) * R(4.0);
  R a_i = w.dg[0] - shift, b_i = n > 1 ? w.e[0] : R(0.0), c_i = R(0.0);
  for (int i = 0; i < n - 1; ++i) {
    const R sub = w.e[i];
    const R d1 = w.dg[i + 1] - shift;
    const R e1 = i + 2 < n ? w.e[i + 1] : R(0.0);
    if (fabs(a_i) >= fabs(sub)) {
      const R pv = fabs(a_i) < pivmin ? (a_i < R(0.0) ? -pivmin : pivmin) : a_i;
      const R l = sub / pv;
      u[i] = pv; u1[i] = b_i; u2[i] = c_i; lm[i] = l; sw[i] = R(0.0);
      a_i = d1 - l * b_i;
      b_i = e1 - l * c_i;
      c_i = R(0.0);
    } else {
      const R l = a_i / sub;
      u[i] = sub; u1[i] = d1; u2[i] = e1; lm[i] = l; sw[i] = R(1.0);
      const R na = b_i - l * d1, nc = c_i - l * e1;
      a_i = na;
      b_i = nc;
      c_i = R(0.0);
    }
  }
  u[n - 1] = fabs(a_i) < pivmin ? (a_i < R(0.0) ? -pivmin : pivmin) : a_i;
  u1[n - 1] = R(0.0);
  u2[n - 1] = R(0.0);
  // the pivots' reciprocals, once: the substitutions below then multiply
  // (independent divisions here instead of one on every step of the chain)
  for (int i = 0; i < n; ++i) u[i] = R(1.0) / u[i];
  unsigned int h = 2166136261u ^ (unsigned)s * 16777619u;  // deterministic start vector
  for (int i = 0; i < n; ++i) {
    h = h * 1664525u + 1013904223u;
    z[i] = R(0.5) + (R)((h >> 8) & 0xffff) / R(65536.0);
  }
  for (int iter = 0; iter < 3; ++iter) {
    for (int i = 0; i < n - 1; ++i) {
      if (sw[i] != R(0.0)) {
        const R t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t - lm[i] * z[i];
      } else {
        z[i + 1] -= lm[i] * z[i];
      }
    }
    for (int i = n - 1; i >= 0; --i) {
      R t = z[i];
      if (i + 1 < n) t -= u1[i] * z[i + 1];
      if (i + 2 < n) t -= u2[i] * z[i + 2];
      z[i] = t * u[i];
    }
    R nrm = R(0.0);
    for (int i = 0; i < n; ++i) nrm = fmax(nrm, fabs(z[i]));
    const R inv = nrm > R(0.0) ? R(1.0) / nrm : R(1.0);
    for (int i = 0; i < n; ++i) z[i] *= inv;
  }
  for (int i = 0; i < n; ++i) w.V[(size_t)i * nb + s] = z[i];
}

// the cluster size of the Householder: 16 when the device can place a
// cluster of 16 such blocks (with the largest shared memory a call may ask
// for), else the portable 8; decided once per precision
template <class R>
int house_cluster_size() {
  static const int cs = [] {
    const void* k16 = (const void*)k_rr_house_cluster<R, 16>;
    if (cudaFuncSetAttribute(k16, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
      cudaGetLastError();
      return 8;
    }
    set_max_dyn_smem(k16, (int)kMaxDynSmem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = kMaxDynSmem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_rr_house_cluster<R, 16>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 8;
    }
    return clusters >= 1 ? 16 : 8;
  }();
  return cs;
}

template <class R, int CS>
void launch_house(int n, RRWork<R> w, size_t bytes, cudaStream_t st) {
  set_max_dyn_smem((const void*)k_rr_house_cluster<R, CS>, (int)kMaxDynSmem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  FF_CUDA(cudaLaunchKernelEx(&cfg, k_rr_house_cluster<R, CS>, n, w));
  ::ff::note_launch();
}

// one Rayleigh-Ritz step in working precision R, output in T
template <class R, class T>
void rr_run(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ, double* theta,
            int* dropped, Buf& work) {
  const size_t n = d.ns, nb = d.nb, no = d.no;
  const size_t t1 = std::max(n * nb, 2 * n);
  const size_t total =
      2 * n * n + no * no + 5 * n + nb + 2 * n * nb + nb * nb + t1 + 6 * n * nb + 2 * n * no;
  R* p = reinterpret_cast<R*>(work.ensure(sizeof(R) * total + sizeof(int) * (n + nb + 1) + 256));
  RRWork<R> w;
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
  w.keepz = w.keep + n;
  w.flag = w.keepz + nb;
  for (const void* fn : {(const void*)k_rr_mchol<R>, (const void*)k_rr_rsolve<R>,
                         (const void*)k_rr_cqchol<R>,
                         (const void*)k_rr_bsolve<R>, (const void*)k_rr_tridiag<R>,
                         (const void*)k_rr_invit_sm<R>,
                         (const void*)k_rr_cholqr<R, true>, (const void*)k_rr_backtransform<R>,
                         (const void*)k_rr_proj_v<R>, (const void*)k_rr_chol<R>,
                         (const void*)k_rr_ysolve<R>, (const void*)k_rr_zsolve<R>})
    set_max_dyn_smem(fn, (int)kMaxDynSmem);
  const size_t a_bytes = sizeof(R) * n * (n | 1), l_bytes = sizeof(R) * no * no;
  const int tri_smem = a_bytes <= kMaxDynSmem ? 1 : 0;
  const int ch_lsm = l_bytes <= kMaxDynSmem ? 1 : 0;
  // the solves: L in shared memory when a few staged rows fit beside it
  const size_t lx_bytes = sizeof(R) * (no | 1);
  const int sv_lsm = l_bytes + 8 * lx_bytes <= kMaxDynSmem ? 1 : 0;
  int cb = kYC;
  while (cb > 1 && (sv_lsm ? l_bytes : 0) + cb * lx_bytes > kMaxDynSmem) cb >>= 1;
  const size_t sv_bytes = (sv_lsm ? l_bytes : 0) + cb * lx_bytes;
  R* Yg = w.T1;  // Y = L^-1 A_{O,.}, no x n
  const int cs = house_cluster_size<R>();
  const size_t rpc = (n + cs - 1) / cs;
  const size_t cl_bytes = sizeof(R) * (rpc * n + 4 * n + cs * kCW + 4 * rpc + 2 * kCW);
  const bool use_cluster = cl_bytes <= kMaxDynSmem && n >= 3;
  const R drop = (R)std::max(d.drop, (double)Prec<R>::drop);
  // scaling and projection (many blocks), transform (one block); Householder
  // by the cluster when its rows fit
  (k_rr_proj_c<R><<<(unsigned)((n * no + n + kPT - 1) / kPT), kPT, 0, st>>>(B, d.ns, d.o0, d.no, w),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (no > 0) {
    (k_rr_proj_v<R><<<(unsigned)((n + kPR - 1) / kPR), kPT, sizeof(R) * kPR * n, st>>>(
         A, d.ns, d.o0, d.no, w),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_rr_proj_oo<R><<<(unsigned)no, 128, sizeof(R) * 2 * n, st>>>(A, B, d.ns, d.o0, d.no, w),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  if (no > 0) {
    (k_rr_chol<R><<<1, kThreads, ch_lsm ? l_bytes : 0, st>>>(d.o0, d.no, w, ch_lsm, drop),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_rr_ysolve<R><<<(unsigned)((n + cb - 1) / cb), 256, sv_bytes, st>>>(d.ns, d.o0, d.no, w, Yg,
                                                                         cb, sv_lsm),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_rr_zsolve<R><<<(unsigned)((no + cb - 1) / cb), 256, sv_bytes, st>>>(d.ns, d.o0, d.no, w,
                                                                          Yg, cb, sv_lsm),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  (k_rr_tridiag<R><<<1, kThreads, tri_smem ? a_bytes : 0, st>>>(A, B, d.ns, d.o0, d.no, w,
                                                                tri_smem, use_cluster ? 0 : 1, Yg),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (use_cluster) {
    if (cs == 16)
      launch_house<R, 16>(d.ns, w, cl_bytes, st);
    else
      launch_house<R, 8>(d.ns, w, cl_bytes, st);
  }
  (k_rr_eigvals_mc<R><<<(unsigned)nb, 32 * kEW, (sizeof(R) + sizeof(float)) * 2 * n, st>>>(
       d.ns, d.nb, w, theta),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const size_t iv_bytes = sizeof(R) * kIV * 6 * n;
  if (iv_bytes <= kMaxDynSmem) {
    (k_rr_invit_sm<R><<<(unsigned)((nb + kIV - 1) / kIV), kIV, iv_bytes, st>>>(d.ns, d.nb, w),
     ::ff::note_launch());
  } else {
    (k_rr_invit<R><<<(unsigned)((nb + 31) / 32), 32, 0, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
  // G = X_{r0:r1}^T Y_{r0:r1} over many blocks (a warp per 4 x 4 tile)
  auto gram_mb = [&](const R* X, const R* Y, int r0, int r1, R* G, int lower) {
    const int tiles = (int)(((nb + 3) / 4) * ((nb + 3) / 4));
    (k_rr_gram_mb<R><<<(unsigned)((tiles + 7) / 8), 256, 0, st>>>(X, (int)nb, Y, (int)nb, r0, r1,
                                                                  (int)nb, (int)nb, G, (int)nb,
                                                                  lower),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  };
  // X <- X L^-T (L: m x m as block_cholesky leaves it) over blocks of rows,
  // columns with mask[c] == 0 set to zero
  auto rsolve = [&](const R* Lg, int m, const R* Xin, R* Xout, int rows, const int* mask) {
    const size_t lb = sizeof(R) * m * m, lz = sizeof(R) * (m | 1);
    const int lsm = lb + 8 * lz <= kMaxDynSmem ? 1 : 0;
    int rcb = kYC;
    while (rcb > 1 && (lsm ? lb : 0) + rcb * lz > kMaxDynSmem) rcb >>= 1;
    (k_rr_rsolve<R><<<(unsigned)((rows + rcb - 1) / rcb), 256, (lsm ? lb : 0) + rcb * lz, st>>>(
         Lg, m, Xin, m, Xout, m, rows, mask, rcb, lsm),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  };
  gram_mb(w.V, w.V, 0, (int)n, w.G, 1);  // Cholesky QR's first Gram
  {
    const size_t gq = sizeof(R) * nb * nb;
    const int lsm = gq <= kMaxDynSmem ? 1 : 0;
    (k_rr_cqchol<R><<<1, kThreads, lsm ? gq : 0, st>>>((int)nb, w, lsm), ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  rsolve(w.G, (int)nb, w.V, w.V, (int)n, nullptr);
  const size_t cq_bytes = sizeof(R) * (n * (nb | 1) + nb * nb);
  if (cq_bytes <= kMaxDynSmem)
    (k_rr_cholqr<R, true><<<1, kThreads, cq_bytes, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  else
    (k_rr_cholqr<R, false><<<1, kThreads, 0, st>>>(d.ns, d.nb, w), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const int ngr = n > 2 ? (int)((n - 2 + kWY - 1) / kWY) : 0;
  if (ngr > 0) {
    (k_rr_wy_t<R><<<(unsigned)ngr, 256, 0, st>>>(d.ns, w, w.scr), ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  (k_rr_backtransform<R><<<(unsigned)((nb + kBW - 1) / kBW), 32 * kBW,
                           sizeof(R) * n * (kBW + kWY), st>>>(d.ns, d.nb, w, w.scr),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (d.want_p) {  // the momentum step's Grams and Z = Zp - V G over many blocks
    gram_mb(w.V, w.V, d.nx, (int)n, w.G, 0);
    const long long zt = (long long)n * ((nb + 3) / 4);
    (k_rr_zp_mb<R><<<(unsigned)((zt + 255) / 256), 256, 0, st>>>(w.V, w.G, (int)n, (int)nb, d.nx,
                                                                 w.T1),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    gram_mb(w.T1, w.T1, 0, (int)n, w.G, 1);
  }
  // the momentum factor (one block), Z L^-T (blocks of rows), the O rows
  // mapped back (blocks of columns)
  const size_t g_bytes = sizeof(R) * nb * nb;
  const int mc_lsm = g_bytes <= kMaxDynSmem ? 1 : 0;
  (k_rr_mchol<R><<<1, kThreads, mc_lsm ? g_bytes : 0, st>>>((int)n, (int)nb, d.want_p, w, dropped,
                                                            mc_lsm),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (d.want_p) rsolve(w.G, (int)nb, w.T1, w.Z, (int)n, w.keepz);
  if (no > 0) {
    const int ncol = d.want_p ? 2 * (int)nb : (int)nb;
    const size_t lc = sizeof(R) * no;
    const int bs_lsm = l_bytes + 8 * lc <= kMaxDynSmem ? 1 : 0;
    int bcb = kYC;
    while (bcb > 1 && (bs_lsm ? l_bytes : 0) + bcb * lc > kMaxDynSmem) bcb >>= 1;
    (k_rr_bsolve<R><<<(unsigned)((ncol + bcb - 1) / bcb), 256, (bs_lsm ? l_bytes : 0) + bcb * lc,
                      st>>>(w.L, d.no, d.o0, w.V, w.Z, (int)nb, ncol, bcb, bs_lsm),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  (k_rr_output<R, T><<<(unsigned)n, 128, 0, st>>>(d.ns, d.o0, d.no, d.nb, d.want_p, w, YZ),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

}  // namespace

template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool fp64, double* /*dbg*/) {
  ProfScope ps(kProfRR);
  FF_REQUIRE(d.ns <= 1024 && d.no <= 1024 && d.nb <= 512 && d.o0 + d.no <= d.ns,
             FF_ERR_INVALID_ARG, "Rayleigh-Ritz basis too large");
  if (fp64) {
    // double-float blocks: the dense step in double-float too (GB300's FP64
    // rate holds the FP64 step to a fraction of the FP32 pipes)
    if constexpr (std::is_same_v<T, dfloat>)
      rr_run<dfloat, T>(st, A, B, d, YZ, theta, dropped, work);
    else
      rr_run<double, T>(st, A, B, d, YZ, theta, dropped, work);
  } else {
    rr_run<float, T>(st, A, B, d, YZ, theta, dropped, work);
  }
}

template void rayleigh_ritz<float>(cudaStream_t, const double*, const double*, RRDims, float*,
                                   double*, int*, Buf&, bool, double*);
template void rayleigh_ritz<double>(cudaStream_t, const double*, const double*, RRDims, double*,
                                    double*, int*, Buf&, bool, double*);
template void rayleigh_ritz<dfloat>(cudaStream_t, const double*, const double*, RRDims, dfloat*,
                                    double*, int*, Buf&, bool, double*);

}  // namespace ff
