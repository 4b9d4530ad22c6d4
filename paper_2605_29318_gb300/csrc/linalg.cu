#include <cuda_bf16.h>
// Block kernels of the eigensolver: the fused (H_w, M) block product, the
// Chebyshev preconditioner steps, tall-skinny Gram products and block updates.
// Panels are row-major n x ld (row k of a block of m columns is contiguous), so
// a warp reads one row of a block with unit stride.
#include <type_traits>

#include "linalg.cuh"

namespace ff {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Y_H = H X, Y_M = M X with H in difference form: (H x)_k = sum_l H_kl (x_l - x_k),
// exact because every row of the stored H sums to zero (the diagonal term
// multiplies x_k - x_k = 0).  One warp per row; lanes over block columns.
template <class T>
__global__ void k_spmm_hm(const long long* __restrict__ ptr, const int* __restrict__ col,
                          const T* __restrict__ val, long long n, const T* __restrict__ X, int ldx,
                          T* __restrict__ YH, T* __restrict__ YM, int ldy, int m) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const long long s = ptr[k], e = ptr[k + 1];
    for (int c0 = 0; c0 < m; c0 += 32) {
      const int cc = c0 + lane;
      const bool act = cc < m;
      const T xk = act ? X[k * ldx + cc] : T(0);
      T ah = T(0), am = T(0);
      for (long long e0 = s; e0 < e; e0 += 32) {
        const int cnt = (int)min((long long)32, e - e0);
        int l_l = 0;
        T h_l = T(0), m_l = T(0);
        if (lane < cnt) {
          l_l = col[e0 + lane];
          h_l = val[2 * (e0 + lane)];
          m_l = val[2 * (e0 + lane) + 1];
        }
        for (int j = 0; j < cnt; ++j) {
          const int l = __shfl_sync(kFull, l_l, j);
          const T h = __shfl_sync(kFull, h_l, j);
          const T mm = __shfl_sync(kFull, m_l, j);
          if (act) {
            const T xl = X[(long long)l * ldx + cc];
            ah += h * (xl - xk);
            am += mm * xl;
          }
        }
      }
      if (act) {
        if (YH) YH[k * ldy + cc] = ah;
        if (YM) YM[k * ldy + cc] = am;
      }
    }
  }
}

// One Chebyshev step on D^-1 H (FP32):  res -= D^-1 H d_in;  d_out = c1 d_in + c2 res;
// x += d_out.  (H d)_k in difference form as above.
__global__ void k_cheb_step(const long long* __restrict__ ptr, const int* __restrict__ col,
                            const float* __restrict__ hv, const float* __restrict__ hdiag,
                            long long n, int m, int ld, const float* __restrict__ din,
                            float* __restrict__ dout, float* __restrict__ x,
                            float* __restrict__ res, float c1, float c2) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const long long s = ptr[k], e = ptr[k + 1];
    const float dinv = 1.0f / hdiag[k];
    for (int c0 = 0; c0 < m; c0 += 32) {
      const int cc = c0 + lane;
      const bool act = cc < m;
      const long long o = k * ld + cc;
      const float dk = act ? din[o] : 0.f;
      float acc = 0.f;
      for (long long e0 = s; e0 < e; e0 += 32) {
        const int cnt = (int)min((long long)32, e - e0);
        int l_l = 0;
        float h_l = 0.f;
        if (lane < cnt) {
          l_l = col[e0 + lane];
          h_l = hv[e0 + lane];
        }
        for (int j = 0; j < cnt; ++j) {
          const int l = __shfl_sync(kFull, l_l, j);
          const float h = __shfl_sync(kFull, h_l, j);
          if (act) acc += h * (din[(long long)l * ld + cc] - dk);
        }
      }
      if (act) {
        const float r = res[o] - acc * dinv;
        const float dn = c1 * dk + c2 * r;
        res[o] = r;
        dout[o] = dn;
        x[o] += dn;
      }
    }
  }
}

// Vectorised variants for blocks whose width m is a multiple of the 16-byte
// vector (4 floats / 2 doubles) and at most 32 vectors: a group of G = m / VEC
// lanes reads one neighbour row of the block with 16-byte loads, the warp holds
// P = 32 / G groups that walk different entries of the matrix row, four
// entries per group in flight; the groups' partial sums are combined with
// shuffles at the end of the row.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <class T>
__device__ __forceinline__ void vload(const T* p, T (&v)[Vec16<T>::n]) {
  const typename Vec16<T>::type q = *reinterpret_cast<const typename Vec16<T>::type*>(p);
  if constexpr (Vec16<T>::n == 4) {
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    v[0] = q.x; v[1] = q.y;
  }
}
template <class T>
__device__ __forceinline__ void vstore(T* p, const T (&v)[Vec16<T>::n]) {
  typename Vec16<T>::type q;
  if constexpr (Vec16<T>::n == 4) {
    q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
  } else {
    q.x = v[0]; q.y = v[1];
  }
  *reinterpret_cast<typename Vec16<T>::type*>(p) = q;
}

// GT > 0 fixes the group width G at compile time (the solver's block widths).
template <class T, int GT = 0>
__global__ void k_spmm_hm_vec(const long long* __restrict__ ptr, const int* __restrict__ col,
                              const T* __restrict__ val, long long n, const T* __restrict__ X,
                              int ldx, T* __restrict__ YH, T* __restrict__ YM, int ldy, int m) {
  constexpr int VEC = Vec16<T>::n;
  const int lane = threadIdx.x & 31;
  const int G = GT > 0 ? GT : m / VEC, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * VEC;
  const bool act = g < P;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const long long s = ptr[k], e = ptr[k + 1];
    T xk[VEC], ah[VEC], am[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) ah[u] = am[u] = T(0);
    if (act) vload(X + k * ldx + cv, xk);
    else
#pragma unroll
      for (int u = 0; u < VEC; ++u) xk[u] = T(0);
    // offsets within the row are 32-bit; (H, M) of a nonzero is one 2-vector load
    using T2 = typename std::conditional<std::is_same_v<T, float>, float2, double2>::type;
    const int cnt = (int)(e - s);
    const int* cr = col + s;
    const T2* vr = reinterpret_cast<const T2*>(val) + s;
    int e0 = act ? g : cnt;
    for (; e0 + 3 * P < cnt; e0 += 4 * P) {
      int l[4];
      T h[4], mm[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = e0 + q * P;
        l[q] = __ldg(cr + t);
        const T2 hm = vr[t];
        h[q] = hm.x;
        mm[q] = hm.y;
      }
      T xl[4][VEC];
#pragma unroll
      for (int q = 0; q < 4; ++q) vload(X + (long long)l[q] * ldx + cv, xl[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          ah[u] += h[q] * (xl[q][u] - xk[u]);
          am[u] += mm[q] * xl[q][u];
        }
    }
    for (; e0 < cnt; e0 += P) {
      const int l = __ldg(cr + e0);
      const T2 hm = vr[e0];
      const T h = hm.x, mm = hm.y;
      T xl[VEC];
      vload(X + (long long)l * ldx + cv, xl);
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        ah[u] += h * (xl[u] - xk[u]);
        am[u] += mm * xl[u];
      }
    }
    for (int q = 1; q < P; ++q) {
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const T th = __shfl_down_sync(kFull, ah[u], q * G);
        const T tm = __shfl_down_sync(kFull, am[u], q * G);
        if (g == 0) {
          ah[u] += th;
          am[u] += tm;
        }
      }
    }
    if (g == 0) {
      if (YH) vstore(YH + k * ldy + cv, ah);
      if (YM) vstore(YM + k * ldy + cv, am);
    }
  }
}

__global__ void k_cheb_step_vec(const long long* __restrict__ ptr, const int* __restrict__ col,
                                const float* __restrict__ hv, const float* __restrict__ hdiag,
                                long long n, int m, int ld, const float* __restrict__ din,
                                float* __restrict__ dout, float* __restrict__ x,
                                float* __restrict__ res, float c1, float c2) {
  const int lane = threadIdx.x & 31;
  const int G = m / 4, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * 4;
  const bool act = g < P;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const long long s = ptr[k], e = ptr[k + 1];
    float dk[4] = {0, 0, 0, 0}, acc[4] = {0, 0, 0, 0};
    if (act) vload(din + k * ld + cv, dk);
    long long e0 = act ? s + g : e;
    for (; e0 + 3 * P < e; e0 += 4 * P) {
      int l[4];
      float h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        l[q] = col[e0 + q * P];
        h[q] = hv[e0 + q * P];
      }
      float dl[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) vload(din + (long long)l[q] * ld + cv, dl[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += h[q] * (dl[q][u] - dk[u]);
    }
    for (; e0 < e; e0 += P) {
      const int l = col[e0];
      const float h = hv[e0];
      float dl[4];
      vload(din + (long long)l * ld + cv, dl);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += h * (dl[u] - dk[u]);
    }
    for (int q = 1; q < P; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float t = __shfl_down_sync(kFull, acc[u], q * G);
        if (g == 0) acc[u] += t;
      }
    if (g == 0) {
      const float dinv = 1.0f / hdiag[k];
      const long long o = k * ld + cv;
      float r[4], dn[4], xx[4];
      vload(res + o, r);
      vload(x + o, xx);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        r[u] -= acc[u] * dinv;
        dn[u] = c1 * dk[u] + c2 * r[u];
        xx[u] += dn[u];
      }
      vstore(res + o, r);
      vstore(dout + o, dn);
      vstore(x + o, xx);
    }
  }
}

// Gram partials: P[blk][i][j] = sum_{rows in chunk} A[r][ia + i] * B[r][ib + j]
// (p x q outputs in 32 x 32 tiles; grid.x = row chunks, grid.y = output tiles).
// Accumulates in T inside the chunk, the cross-chunk sum is FP64 (k_gram_reduce).
// Partial tall-skinny products over a chunk of rows: a TW x TW tile of
// A^T B per block (TW = 32, or 40 for the 40-wide blocks of a 40-column
// eigensolver block, so that no lane computes padding -- on GB300 an FP64
// warp instruction costs the same whatever the active lanes).  Thread
// (tx, ty) of TW x 8 owns rows ty + 8u of the tile and column tx.
template <class T, int TW>
__global__ void __launch_bounds__(TW * 8)
    k_gram_partial(const T* __restrict__ A, int lda, int p, const T* __restrict__ B, int ldb,
                   int q, long long n, long long rows_per_chunk, double* __restrict__ part) {
  constexpr int U = TW / 8;
  __shared__ T sa[32][TW + 1];
  __shared__ T sb[32][TW + 1];
  const int tilesq = (q + TW - 1) / TW;
  const int ti = blockIdx.y / tilesq, tj = blockIdx.y % tilesq;
  const int tx = threadIdx.x % TW, ty = threadIdx.x / TW;
  const long long r0 = (long long)blockIdx.x * rows_per_chunk;
  const long long r1 = min(n, r0 + rows_per_chunk);
  T acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = T(0);
  for (long long rb = r0; rb < r1; rb += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const long long r = rb + rr;
      const int ia = ti * TW + tx, ib = tj * TW + tx;
      sa[rr][tx] = (r < r1 && ia < p) ? A[r * lda + ia] : T(0);
      sb[rr][tx] = (r < r1 && ib < q) ? B[r * ldb + ib] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const T bv = sb[rr][tx];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if constexpr (std::is_same_v<T, dfloat>)
          df_mac(acc[u], sa[rr][ty + 8 * u], bv);
        else
          acc[u] += sa[rr][ty + 8 * u] * bv;
      }
    }
    __syncthreads();
  }
  const int jj = tj * TW + tx;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int ii = ti * TW + ty + 8 * u;
    if (ii < p && jj < q) part[((long long)blockIdx.x * p + ii) * q + jj] = (double)acc[u];
  }
}

// Cross-chunk sums of Gram partials: a block of kRedWarps warps per 32
// consecutive entries, warp w summing chunks w, w + kRedWarps, ... and warp 0
// adding the warps' sums in order (a fixed order: results do not depend on
// timing).
constexpr int kRedWarps = 16;
__global__ void __launch_bounds__(32 * kRedWarps)
    k_gram_reduce(const double* __restrict__ part, int chunks, int pq, int q,
                  double* __restrict__ out, int ldo, double alpha, int accumulate) {
  __shared__ double red[kRedWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (t < pq)
#pragma unroll 4
    for (int c = w; c < chunks; c += kRedWarps) s += part[(long long)c * pq + t];
  red[w][lane] = s;
  __syncthreads();
  if (w != 0 || t >= pq) return;
  s = 0.0;
  for (int q2 = 0; q2 < kRedWarps; ++q2) s += red[q2][lane];
  double* o = out + (long long)(t / q) * ldo + t % q;
  *o = accumulate ? *o + alpha * s : alpha * s;
}

// Sums of products for the reductions below: FP64 for FP32 and FP64 blocks,
// double-float for double-float blocks
template <class T>
struct SumOf {
  using type = double;
};
template <>
struct SumOf<dfloat> {
  using type = dfloat;
};
__device__ __forceinline__ void add_prod(double& s, float a, float b) {
  s += (double)a * (double)b;
}
__device__ __forceinline__ void add_prod(double& s, double a, double b) { s += a * b; }
__device__ __forceinline__ void add_prod(dfloat& s, dfloat a, dfloat b) { df_mac(s, a, b); }
__device__ __forceinline__ void add_sum(double& s, double a) { s += a; }
__device__ __forceinline__ void add_sum(dfloat& s, dfloat a) { df_acc(s, a); }

// p == 1: part[chunk][j] = sum over the chunk's rows of a[r] B[r][j]; the 8
// warps of a block take interleaved rows, lanes take columns
template <class T>
__global__ void __launch_bounds__(256)
    k_gram_row(const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb, int q,
               long long n, long long rows_per_chunk, double* __restrict__ part) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * rows_per_chunk;
  const long long r1 = min(n, r0 + rows_per_chunk);
  for (int j0 = 0; j0 < q; j0 += 32) {
    const int j = j0 + lane;
    typename SumOf<T>::type sp(0);
    if (j < q)
      for (long long r = r0 + w; r < r1; r += 8) add_prod(sp, A[r * lda], B[r * ldb + j]);
    red[w][lane] = (double)sp;
    __syncthreads();
    if (w == 0 && j < q) {
      double t = 0.0;
      for (int ww = 0; ww < 8; ++ww) t += red[ww][lane];
      part[(long long)blockIdx.x * q + j] = t;
    }
    __syncthreads();
  }
}

// out[c * ldo + c] = sum_r A[r][c] B[r][c] for the columns c outside [w0, w1)
// (one block per column, FP64 sums)
template <class T>
__global__ void __launch_bounds__(512)
    k_gram_diag(const T* __restrict__ A, const T* __restrict__ B, int ld, long long n, int w0,
                int w1, double* __restrict__ out, int ldo) {
  const int c = (int)blockIdx.x >= w0 ? (int)blockIdx.x + (w1 - w0) : (int)blockIdx.x;
  typename SumOf<T>::type sp(0);
  for (long long r = threadIdx.x; r < n; r += blockDim.x) add_prod(sp, A[r * ld + c], B[r * ld + c]);
  double s = (double)sp;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  __shared__ double red[16];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (threadIdx.x == 0) out[(long long)c * ldo + c] = t;
  }
}

// A: upper block triangle from the lower one; B: W rows from the W columns
__global__ void k_gram_mirror(double* __restrict__ A, double* __restrict__ B, int ns, int nb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * ns) return;
  const int i = t / ns, j = t % ns;
  if (i / nb < j / nb) A[t] = A[(long long)j * ns + i];
  if (i / nb == 1 && j / nb != 1) B[t] = B[(long long)j * ns + i];
}

// C[r][cmap(j)] = beta * C[...] + sum_i A[r][i] * Y[i][j]; cmap sends columns
// j < split to C + j and j >= split to C + off2 + (j - split).
// One warp per row, lanes over 32 columns of the tile; Y tile staged in shared memory.
// C = beta C + A Y over all rows: a group of TW threads per row, thread tx
// owning output column blockIdx.y * TW + tx (TW = 32, or 40 for 40-wide
// outputs so that no lane computes padding); Y's TW columns staged in shared
// memory; columns at or past `split` are written at off2 + (j - split).
template <class T, int TW>
__global__ void k_block_update(const T* __restrict__ A, int lda, int p, const T* __restrict__ Y,
                               int ldy, int q, T* __restrict__ C, int ldc, long long n, T beta,
                               int split, int off2) {
  extern __shared__ unsigned char smraw[];
  T* sy = reinterpret_cast<T*>(smraw);  // p x TW
  const int tx = threadIdx.x % TW, ry = threadIdx.x / TW, rpb = blockDim.x / TW;
  const int j = blockIdx.y * TW + tx;
  for (int t = threadIdx.x; t < p * TW; t += blockDim.x) {
    const int i = t / TW, jj = blockIdx.y * TW + (t % TW);
    sy[t] = jj < q ? Y[(long long)i * ldy + jj] : T(0);
  }
  __syncthreads();
  const int cj = j < split ? j : off2 + (j - split);
  if constexpr (std::is_same_v<T, dfloat>) {
    for (long long r = (long long)blockIdx.x * rpb + ry; r < n; r += (long long)gridDim.x * rpb) {
      const T* a = A + r * lda;
      T acc(0);
#pragma unroll 4
      for (int i = 0; i < p; ++i) df_mac(acc, a[i], sy[i * TW + tx]);
      if (j < q) {
        T* cp = C + r * ldc + cj;
        if (!(beta == T(0))) df_mac(acc, beta, *cp);
        *cp = df_norm(acc);
      }
    }
  } else {
  for (long long r = (long long)blockIdx.x * rpb + ry; r < n; r += (long long)gridDim.x * rpb) {
    const T* a = A + r * lda;
    T acc = T(0);
    int i = 0;
    for (; i + 4 <= p; i += 4) {
      acc += a[i] * sy[i * TW + tx] + a[i + 1] * sy[(i + 1) * TW + tx] +
             a[i + 2] * sy[(i + 2) * TW + tx] + a[i + 3] * sy[(i + 3) * TW + tx];
    }
    for (; i < p; ++i) acc += a[i] * sy[i * TW + tx];
    if (j < q) {
      T* cp = C + r * ldc + cj;
      *cp = beta == T(0) ? acc : beta * *cp + acc;
    }
  }
  }
}

// ------------------------------------------------------------- register-tiled kernels
// A Gram tile: operand panels (first column of the tile in each), destination
// of entry (0, 0) and the valid rows and columns (multiples of 4)
struct GramTile {
  const void* a;
  const void* b;
  double* out;
  int pi, qj;
  int diag_only;
};
constexpr int kMaxGramTiles = 32;
struct GramTiles {
  GramTile t[kMaxGramTiles];
  int count;
};

// Four consecutive values of a row (16-byte aligned): one 16-byte load for
// FP32, two for FP64 and double-float.
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const dfloat* p, dfloat (&v)[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  const float4 b = reinterpret_cast<const float4*>(p)[1];
  v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w); v[2] = dfloat(b.x, b.y);
  v[3] = dfloat(b.z, b.w);
}
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(dfloat* p, const dfloat (&v)[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[2].h, v[2].l, v[3].h, v[3].l);
}

// 16-byte asynchronous copy global -> shared; bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Several Gram tiles in one launch, each with its own operand panels and
// destination: part[chunk][tile][i][j] = sum over the chunk's rows of
// a[r][i] b[r][j] for a TW x TW tile.  The block streams its rows through
// shared memory in 32-row slabs of both panels' TW columns (16-byte
// asynchronous copies, two slabs in flight; rows past the chunk and columns
// past the tile's valid width are zero-filled).  A group of TD x TD threads
// (TD = TW / 4) covers the tile, each thread a 4 x 4 register block; GR
// groups take interleaved rows of a slab and are summed in shared memory at
// the end.  Sums in T within a thread (double-float for double-float panels),
// FP64 from there on.
template <class T, int TW>
__global__ void __launch_bounds__(256)
    k_gram_tiles(GramTiles tiles, int lda, int ldb, long long n, long long rows_per_chunk,
                 double* __restrict__ part) {
  constexpr int TD = TW / 4, TT = TD * TD, GR = 256 / TT, NT = TT * GR;
  constexpr int SL = 32, EPC = 16 / (int)sizeof(T), CPR = TW / EPC;
  constexpr int kSlab = 2 * 2 * SL * TW * (int)sizeof(T);
  constexpr int kRed = (GR - 1) * TT * 16 * 8;
  __shared__ __align__(16) unsigned char sm[kSlab > kRed ? kSlab : kRed];
  T* slab = reinterpret_cast<T*>(sm);  // [buf][panel][row][TW]
  const int tid = threadIdx.x, grp = tid / TT, lt = tid % TT;
  const int ti = lt / TD, tj = lt % TD;
  const GramTile tl = tiles.t[blockIdx.y];
  const T* pa = static_cast<const T*>(tl.a);
  const T* pb = static_cast<const T*>(tl.b);
  const bool live = grp < GR && 4 * ti < tl.pi && 4 * tj < tl.qj;
  const long long r0 = (long long)blockIdx.x * rows_per_chunk;
  const long long r1 = min(n, r0 + rows_per_chunk);
  const int nslab = (int)((r1 - r0 + SL - 1) / SL);
  auto issue = [&](int buf, long long rs) {
    for (int t = tid; t < 2 * SL * CPR; t += NT) {
      const int pan = t / (SL * CPR), w = t % (SL * CPR), rr = w / CPR, cc = (w % CPR) * EPC;
      const long long r = rs + rr;
      const bool ok = r < r1 && cc < (pan == 0 ? tl.pi : tl.qj);
      const T* src = pan == 0 ? pa + (ok ? r * lda + cc : r0 * lda) : pb + (ok ? r * ldb + cc : r0 * ldb);
      cp_async16(slab + ((buf * 2 + pan) * SL + rr) * TW + cc, src, ok ? 16 : 0);
    }
  };
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  if (nslab > 0) issue(0, r0);
  cp_async_commit();
  for (int sl = 0; sl < nslab; ++sl) {
    if (sl + 1 < nslab) issue((sl + 1) & 1, r0 + (long long)(sl + 1) * SL);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    if (live) {
      const T* sa = slab + ((sl & 1) * 2 + 0) * SL * TW + 4 * ti;
      const T* sb = slab + ((sl & 1) * 2 + 1) * SL * TW + 4 * tj;
#pragma unroll 4
      for (int rr = grp; rr < SL; rr += GR) {
        T x[4], y[4];
        load4(sa + rr * TW, x);
        load4(sb + rr * TW, y);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) mac(acc[u][v], x[u], y[v]);
      }
    }
    __syncthreads();
  }
  double* red = reinterpret_cast<double*>(sm);  // [GR - 1][TT][16]
  if (grp > 0 && grp < GR)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) red[((grp - 1) * TT + lt) * 16 + 4 * u + v] = (double)acc[u][v];
  __syncthreads();
  if (grp == 0 && live) {
    double* o = part + ((long long)blockIdx.x * tiles.count + blockIdx.y) * (TW * TW);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double t = (double)acc[u][v];
        for (int g = 1; g < GR; ++g) t += red[((g - 1) * TT + lt) * 16 + 4 * u + v];
        o[(4 * ti + u) * TW + 4 * tj + v] = t;
      }
  }
}

// out = alpha * (sum over chunks) (+ out), per tile entry; tiles marked
// diag_only write their diagonal alone.  Chunks split over the block's warps
// as in k_gram_reduce.
template <int TW>
__global__ void __launch_bounds__(32 * kRedWarps)
    k_gram_tiles_reduce(GramTiles tiles, int chunks, int ldo, double alpha, int accumulate,
                        const double* __restrict__ part) {
  __shared__ double red[kRedWarps][33];
  const int t = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const GramTile tl = tiles.t[t];
  const int i = e / TW, j = e % TW;
  const bool want = e < TW * TW && i < tl.pi && j < tl.qj && !(tl.diag_only && i != j);
  double s = 0.0;
  if (want)
#pragma unroll 4
    for (int c = w; c < chunks; c += kRedWarps)
      s += part[((long long)c * tiles.count + t) * (TW * TW) + e];
  red[w][lane] = s;
  __syncthreads();
  if (w != 0 || !want) return;
  s = 0.0;
  for (int q = 0; q < kRedWarps; ++q) s += red[q][lane];
  double* o = tl.out + (long long)i * ldo + j;
  *o = accumulate ? *o + alpha * s : alpha * s;
}

// C = beta C + A Y for blocks with p, q, lda, ldc, split, off2 multiples of 4:
// each thread computes a 4 x 4 register block (4 consecutive rows, 4
// consecutive output columns) from 16-byte row loads of A and of the Y tile
// staged in shared memory; TD = TW / 4 threads span a TW-column tile and
// RG = 256 / TD row groups share a block.  Columns at or past `split` are
// written at off2 + (j - split).
template <class T, int TW>
__global__ void __launch_bounds__(256)
    k_block_update_rt(const T* __restrict__ A, int lda, int p, const T* __restrict__ Y, int ldy,
                      int q, T* __restrict__ C, int ldc, long long n, T beta, int split,
                      int off2) {
  constexpr int TD = TW / 4, RG = 256 / TD, RR = 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sy = reinterpret_cast<T*>(smraw);  // p x TW
  const int c0 = blockIdx.y * TW;
  for (int t = threadIdx.x; t < p * TW; t += blockDim.x) {
    const int i = t / TW, jj = c0 + (t % TW);
    sy[t] = jj < q ? Y[(long long)i * ldy + jj] : T(0);
  }
  __syncthreads();
  const int tc = threadIdx.x % TD, rg = threadIdx.x / TD;
  const int j0 = c0 + 4 * tc;
  if (rg >= RG || j0 >= q) return;
  const int cj = j0 < split ? j0 : off2 + (j0 - split);
  const T* yb = sy + 4 * tc;
  for (long long rb = ((long long)blockIdx.x * RG + rg) * RR; rb < n;
       rb += (long long)gridDim.x * RG * RR) {
    const T* ar[RR];
#pragma unroll
    for (int rr = 0; rr < RR; ++rr) ar[rr] = A + min(rb + rr, n - 1) * lda;  // tail rows clamped
    T acc[RR][4];
#pragma unroll
    for (int rr = 0; rr < RR; ++rr)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[rr][v] = T(0);
    for (int i = 0; i < p; i += 4) {
      T y[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) load4(yb + (i + kk) * TW, y[kk]);
#pragma unroll
      for (int rr = 0; rr < RR; ++rr) {
        T x[4];
        load4(ar[rr] + i, x);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int v = 0; v < 4; ++v) mac(acc[rr][v], x[kk], y[kk][v]);
      }
    }
#pragma unroll
    for (int rr = 0; rr < RR; ++rr) {
      if (rb + rr >= n) break;
      T* cp = C + (rb + rr) * ldc + cj;
      if (!(beta == T(0))) {
        T old[4];
        load4(cp, old);
#pragma unroll
        for (int v = 0; v < 4; ++v) mac(acc[rr][v], beta, old[v]);
      }
      T o4[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) o4[v] = finish(acc[rr][v]);
      store4(cp, o4);
    }
  }
}

}  // namespace

// FP64 block product (H x, M x) for m % 4 == 0: each lane owns 4 columns (two
// 16-byte loads per gathered row), so a 40-column block keeps 30 of 32 lanes
// busy.  GB300 charges an FP64 warp instruction the same whatever the active
// lanes, so lane use is FP64 throughput; and H x is accumulated as
// sum_l h_kl x_l - (sum_l h_kl) x_k (two FMAs per value and nonzero instead of
// the subtract-and-FMA of the difference form; in FP64 the lost cancellation
// costs ~1e-12 relative).
__global__ void k_spmm_hm_f64x4(const long long* __restrict__ ptr, const int* __restrict__ col,
                                const double* __restrict__ val, long long n,
                                const double* __restrict__ X, int ldx, double* __restrict__ YH,
                                double* __restrict__ YM, int ldy, int m) {
  const int lane = threadIdx.x & 31;
  const int G = m / 4, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * 4;
  const bool act = g < P;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const long long s = ptr[k], e = ptr[k + 1];
    double ah[4] = {0, 0, 0, 0}, am[4] = {0, 0, 0, 0}, hs = 0.0;
    long long e0 = act ? s + g : e;
    for (; e0 + P < e; e0 += 2 * P) {
      const int l0 = col[e0], l1 = col[e0 + P];
      const double2 hm0 = *reinterpret_cast<const double2*>(val + 2 * e0);
      const double2 hm1 = *reinterpret_cast<const double2*>(val + 2 * (e0 + P));
      const double2* p0 = reinterpret_cast<const double2*>(X + (long long)l0 * ldx + cv);
      const double2* p1 = reinterpret_cast<const double2*>(X + (long long)l1 * ldx + cv);
      const double2 a0 = __ldg(p0), b0 = __ldg(p0 + 1), a1 = __ldg(p1), b1 = __ldg(p1 + 1);
      hs += hm0.x + hm1.x;
      ah[0] = fma(hm0.x, a0.x, ah[0]); ah[1] = fma(hm0.x, a0.y, ah[1]);
      ah[2] = fma(hm0.x, b0.x, ah[2]); ah[3] = fma(hm0.x, b0.y, ah[3]);
      am[0] = fma(hm0.y, a0.x, am[0]); am[1] = fma(hm0.y, a0.y, am[1]);
      am[2] = fma(hm0.y, b0.x, am[2]); am[3] = fma(hm0.y, b0.y, am[3]);
      ah[0] = fma(hm1.x, a1.x, ah[0]); ah[1] = fma(hm1.x, a1.y, ah[1]);
      ah[2] = fma(hm1.x, b1.x, ah[2]); ah[3] = fma(hm1.x, b1.y, ah[3]);
      am[0] = fma(hm1.y, a1.x, am[0]); am[1] = fma(hm1.y, a1.y, am[1]);
      am[2] = fma(hm1.y, b1.x, am[2]); am[3] = fma(hm1.y, b1.y, am[3]);
    }
    for (; e0 < e; e0 += P) {
      const int l0 = col[e0];
      const double2 hm0 = *reinterpret_cast<const double2*>(val + 2 * e0);
      const double2* p0 = reinterpret_cast<const double2*>(X + (long long)l0 * ldx + cv);
      const double2 a0 = __ldg(p0), b0 = __ldg(p0 + 1);
      hs += hm0.x;
      ah[0] = fma(hm0.x, a0.x, ah[0]); ah[1] = fma(hm0.x, a0.y, ah[1]);
      ah[2] = fma(hm0.x, b0.x, ah[2]); ah[3] = fma(hm0.x, b0.y, ah[3]);
      am[0] = fma(hm0.y, a0.x, am[0]); am[1] = fma(hm0.y, a0.y, am[1]);
      am[2] = fma(hm0.y, b0.x, am[2]); am[3] = fma(hm0.y, b0.y, am[3]);
    }
    for (int q = 1; q < P; ++q) {  // groups are at most 3 for the 40-column block
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double th = __shfl_down_sync(kFull, ah[u], q * G);
        const double tm = __shfl_down_sync(kFull, am[u], q * G);
        if (g == 0) {
          ah[u] += th;
          am[u] += tm;
        }
      }
      const double ts = __shfl_down_sync(kFull, hs, q * G);
      if (g == 0) hs += ts;
    }
    if (g == 0) {
      const double2* pk = reinterpret_cast<const double2*>(X + k * ldx + cv);
      const double2 xa = pk[0], xb = pk[1];
      if (YH) {
        double2* o = reinterpret_cast<double2*>(YH + k * ldy + cv);
        o[0] = make_double2(fma(-hs, xa.x, ah[0]), fma(-hs, xa.y, ah[1]));
        o[1] = make_double2(fma(-hs, xb.x, ah[2]), fma(-hs, xb.y, ah[3]));
      }
      if (YM) {
        double2* o = reinterpret_cast<double2*>(YM + k * ldy + cv);
        o[0] = make_double2(am[0], am[1]);
        o[1] = make_double2(am[2], am[3]);
      }
    }
  }
}

// Double-float block product (H x, M x) for m % 4 == 0: the values of a
// nonzero are (H.h, H.l, M.h, M.l), one 16-byte load; each lane owns 4
// columns (two 16-byte loads per gathered row); H x accumulated as
// sum_l h_kl x_l - (sum_l h_kl) x_k, as in the FP64 kernel, with unnormalised
// double-float accumulators.
__global__ void __launch_bounds__(256)
    k_spmm_hm_df(const long long* __restrict__ ptr, const int* __restrict__ col,
                 const float4* __restrict__ val, int n, const dfloat* __restrict__ X, int ldx,
                 dfloat* __restrict__ YH, dfloat* __restrict__ YM, int ldy, int m) {
  const int lane = threadIdx.x & 31;
  const int G = m / 4, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * 4;
  const bool act = g < P;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < n; k += warps) {
    const long long s = ptr[k];
    const int cnt = (int)(ptr[k + 1] - s);
    const int* cr = col + s;
    const float4* vr = val + s;
    dfloat ah[4], am[4], hs(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) ah[u] = am[u] = dfloat(0);
    int e = act ? g : cnt;
    for (; e + P < cnt; e += 2 * P) {
      const int l0 = __ldg(cr + e), l1 = __ldg(cr + e + P);
      const float4 v0 = __ldg(vr + e), v1 = __ldg(vr + e + P);
      const float4* p0 = reinterpret_cast<const float4*>(X + (long long)l0 * ldx + cv);
      const float4* p1 = reinterpret_cast<const float4*>(X + (long long)l1 * ldx + cv);
      const float4 a0 = __ldg(p0), b0 = __ldg(p0 + 1), a1 = __ldg(p1), b1 = __ldg(p1 + 1);
      const dfloat x0[4] = {dfloat(a0.x, a0.y), dfloat(a0.z, a0.w), dfloat(b0.x, b0.y),
                            dfloat(b0.z, b0.w)};
      const dfloat x1[4] = {dfloat(a1.x, a1.y), dfloat(a1.z, a1.w), dfloat(b1.x, b1.y),
                            dfloat(b1.z, b1.w)};
      const dfloat h0(v0.x, v0.y), m0(v0.z, v0.w), h1(v1.x, v1.y), m1(v1.z, v1.w);
      df_acc(hs, h0);
      df_acc(hs, h1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        df_mac(ah[u], h0, x0[u]);
        df_mac(am[u], m0, x0[u]);
        df_mac(ah[u], h1, x1[u]);
        df_mac(am[u], m1, x1[u]);
      }
    }
    for (; e < cnt; e += P) {
      const int l0 = __ldg(cr + e);
      const float4 v0 = __ldg(vr + e);
      const float4* p0 = reinterpret_cast<const float4*>(X + (long long)l0 * ldx + cv);
      const float4 a0 = __ldg(p0), b0 = __ldg(p0 + 1);
      const dfloat x0[4] = {dfloat(a0.x, a0.y), dfloat(a0.z, a0.w), dfloat(b0.x, b0.y),
                            dfloat(b0.z, b0.w)};
      const dfloat h0(v0.x, v0.y), m0(v0.z, v0.w);
      df_acc(hs, h0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        df_mac(ah[u], h0, x0[u]);
        df_mac(am[u], m0, x0[u]);
      }
    }
    for (int q = 1; q < P; ++q) {  // groups are at most 3 for the 40-column block
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const dfloat th = __shfl_down_sync(kFull, ah[u], q * G);
        const dfloat tm = __shfl_down_sync(kFull, am[u], q * G);
        if (g == 0) {
          df_acc(ah[u], th);
          df_acc(am[u], tm);
        }
      }
      const dfloat ts = __shfl_down_sync(kFull, hs, q * G);
      if (g == 0) df_acc(hs, ts);
    }
    if (g == 0) {
      const long long o = (long long)k * ldy + cv;
      if (YH) {
        const float4* pk = reinterpret_cast<const float4*>(X + (long long)k * ldx + cv);
        const float4 xa = pk[0], xb = pk[1];
        const dfloat xk[4] = {dfloat(xa.x, xa.y), dfloat(xa.z, xa.w), dfloat(xb.x, xb.y),
                              dfloat(xb.z, xb.w)};
        dfloat r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          df_mac(ah[u], -hs, xk[u]);
          r[u] = df_norm(ah[u]);
        }
        float4* out = reinterpret_cast<float4*>(YH + o);
        out[0] = make_float4(r[0].h, r[0].l, r[1].h, r[1].l);
        out[1] = make_float4(r[2].h, r[2].l, r[3].h, r[3].l);
      }
      if (YM) {
        dfloat r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = df_norm(am[u]);
        float4* out = reinterpret_cast<float4*>(YM + o);
        out[0] = make_float4(r[0].h, r[0].l, r[1].h, r[1].l);
        out[1] = make_float4(r[2].h, r[2].l, r[3].h, r[3].l);
      }
    }
  }
}

// The same product for pencils with few rows and long ones (the two-set
// pencils: ~1,000 rows of a few hundred nonzeros): one warp per row leaves
// most of the GPU idle behind long serial chains, so a block of kSW warps
// shares each row (group q of the block takes nonzeros q, q + Q, ...), the
// warps' partial sums added in shared memory in a fixed order.
constexpr int kSW = 8;
__global__ void __launch_bounds__(32 * kSW)
    k_spmm_hm_df_split(const long long* __restrict__ ptr, const int* __restrict__ col,
                       const float4* __restrict__ val, int n, const dfloat* __restrict__ X,
                       int ldx, dfloat* __restrict__ YH, dfloat* __restrict__ YM, int ldy, int m) {
  __shared__ dfloat part[kSW][32][9];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = m / 4, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * 4;
  const bool act = g < P;
  const int Q = kSW * P;  // groups per row
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const long long s = ptr[k];
    const int cnt = (int)(ptr[k + 1] - s);
    const int* cr = col + s;
    const float4* vr = val + s;
    dfloat ah[4], am[4], hs(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) ah[u] = am[u] = dfloat(0);
    for (int e = act ? wid * P + g : cnt; e < cnt; e += Q) {
      const int l0 = __ldg(cr + e);
      const float4 v0 = __ldg(vr + e);
      const float4* p0 = reinterpret_cast<const float4*>(X + (long long)l0 * ldx + cv);
      const float4 a0 = __ldg(p0), b0 = __ldg(p0 + 1);
      const dfloat x0[4] = {dfloat(a0.x, a0.y), dfloat(a0.z, a0.w), dfloat(b0.x, b0.y),
                            dfloat(b0.z, b0.w)};
      const dfloat h0(v0.x, v0.y), m0(v0.z, v0.w);
      df_acc(hs, h0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        df_mac(ah[u], h0, x0[u]);
        df_mac(am[u], m0, x0[u]);
      }
    }
    for (int q = 1; q < P; ++q) {  // the warp's groups onto group 0
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const dfloat th = __shfl_down_sync(kFull, ah[u], q * G);
        const dfloat tm = __shfl_down_sync(kFull, am[u], q * G);
        if (g == 0) {
          df_acc(ah[u], th);
          df_acc(am[u], tm);
        }
      }
      const dfloat ts = __shfl_down_sync(kFull, hs, q * G);
      if (g == 0) df_acc(hs, ts);
    }
    if (g == 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        part[wid][lane][u] = ah[u];
        part[wid][lane][4 + u] = am[u];
      }
      part[wid][lane][8] = hs;
    }
    __syncthreads();
    if (wid == 0 && g == 0) {
      for (int w = 1; w < kSW; ++w) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          df_acc(ah[u], part[w][lane][u]);
          df_acc(am[u], part[w][lane][4 + u]);
        }
        df_acc(hs, part[w][lane][8]);
      }
      const long long o = (long long)k * ldy + cv;
      if (YH) {
        const float4* pk = reinterpret_cast<const float4*>(X + (long long)k * ldx + cv);
        const float4 xa = pk[0], xb = pk[1];
        const dfloat xk[4] = {dfloat(xa.x, xa.y), dfloat(xa.z, xa.w), dfloat(xb.x, xb.y),
                              dfloat(xb.z, xb.w)};
        dfloat r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          df_mac(ah[u], -hs, xk[u]);
          r[u] = df_norm(ah[u]);
        }
        float4* out = reinterpret_cast<float4*>(YH + o);
        out[0] = make_float4(r[0].h, r[0].l, r[1].h, r[1].l);
        out[1] = make_float4(r[2].h, r[2].l, r[3].h, r[3].l);
      }
      if (YM) {
        dfloat r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = df_norm(am[u]);
        float4* out = reinterpret_cast<float4*>(YM + o);
        out[0] = make_float4(r[0].h, r[0].l, r[1].h, r[1].l);
        out[1] = make_float4(r[2].h, r[2].l, r[3].h, r[3].l);
      }
    }
    __syncthreads();  // part is rewritten for the next row
  }
}

// k_spmm_hm_vec for pencils with few rows and long ones: a block of kSW
// warps per row, the warps' partial sums added in shared memory in a fixed
// order (see k_spmm_hm_df_split)
template <class T>
__global__ void __launch_bounds__(32 * kSW)
    k_spmm_hm_vec_split(const long long* __restrict__ ptr, const int* __restrict__ col,
                        const T* __restrict__ val, long long n, const T* __restrict__ X, int ldx,
                        T* __restrict__ YH, T* __restrict__ YM, int ldy, int m) {
  constexpr int VEC = Vec16<T>::n;
  __shared__ T part[kSW][32][2 * VEC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = m / VEC, P = 32 / G;
  const int g = lane / G, cv = (lane % G) * VEC;
  const bool act = g < P;
  const int Q = kSW * P;
  using T2 = typename std::conditional<std::is_same_v<T, float>, float2, double2>::type;
  for (long long k = blockIdx.x; k < n; k += gridDim.x) {
    const long long s = ptr[k];
    const int cnt = (int)(ptr[k + 1] - s);
    const int* cr = col + s;
    const T2* vr = reinterpret_cast<const T2*>(val) + s;
    T xk[VEC], ah[VEC], am[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) ah[u] = am[u] = T(0);
    if (act) vload(X + k * ldx + cv, xk);
    else
#pragma unroll
      for (int u = 0; u < VEC; ++u) xk[u] = T(0);
    for (int e = act ? wid * P + g : cnt; e < cnt; e += Q) {
      const int l = __ldg(cr + e);
      const T2 hm = vr[e];
      T xl[VEC];
      vload(X + (long long)l * ldx + cv, xl);
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        ah[u] += hm.x * (xl[u] - xk[u]);
        am[u] += hm.y * xl[u];
      }
    }
    for (int q = 1; q < P; ++q) {
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const T th = __shfl_down_sync(kFull, ah[u], q * G);
        const T tm = __shfl_down_sync(kFull, am[u], q * G);
        if (g == 0) {
          ah[u] += th;
          am[u] += tm;
        }
      }
    }
    if (g == 0)
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        part[wid][lane][u] = ah[u];
        part[wid][lane][VEC + u] = am[u];
      }
    __syncthreads();
    if (wid == 0 && g == 0) {
      for (int w = 1; w < kSW; ++w)
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          ah[u] += part[w][lane][u];
          am[u] += part[w][lane][VEC + u];
        }
      if (YH) vstore(YH + k * ldy + cv, ah);
      if (YM) vstore(YM + k * ldy + cv, am);
    }
    __syncthreads();  // part is rewritten for the next row
  }
}

template <class T>
void spmm_hm_raw(cudaStream_t st, const long long* ptr, const int* col, const T* val, long long n,
                 const T* X, int ldx, T* YH, T* YM, int ldy, int m) {
  ProfScope ps(kProfSpmm);
  const int T_ = 256;
  long long blocks = std::min<long long>((n * 32 + T_ - 1) / T_, (long long)sm_count() * 64);
  if constexpr (std::is_same_v<T, dfloat>) {
    const bool df_ok = m % 4 == 0 && m <= 128 && ldx % 2 == 0 && ldy % 2 == 0 &&
                       n * (long long)std::max(ldx, ldy) < (1LL << 31) &&
                       reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                       reinterpret_cast<uintptr_t>(val) % 16 == 0 &&
                       (!YH || reinterpret_cast<uintptr_t>(YH) % 16 == 0) &&
                       (!YM || reinterpret_cast<uintptr_t>(YM) % 16 == 0);
    if (df_ok && n > 0 && n < (long long)sm_count() * 16)  // few rows: a block per row
      (k_spmm_hm_df_split<<<(unsigned)n, 32 * kSW, 0, st>>>(
           ptr, col, reinterpret_cast<const float4*>(val), (int)n, X, ldx, YH, YM, ldy, m),
       ::ff::note_launch());
    else if (df_ok)
      (k_spmm_hm_df<<<(unsigned)blocks, T_, 0, st>>>(ptr, col, reinterpret_cast<const float4*>(val),
                                                     (int)n, X, ldx, YH, YM, ldy, m),
       ::ff::note_launch());
    else
      (k_spmm_hm<T><<<(unsigned)blocks, T_, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM, ldy, m),
       ::ff::note_launch());
    FF_LAUNCH_CHECK();
  } else {
    constexpr int VEC = Vec16<T>::n;
    const bool vec_ok = m % VEC == 0 && m <= 32 * VEC && ldx % VEC == 0 && ldy % VEC == 0 &&
                        reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
                        (!YH || reinterpret_cast<uintptr_t>(YH) % 16 == 0) &&
                        (!YM || reinterpret_cast<uintptr_t>(YM) % 16 == 0);
    if constexpr (std::is_same_v<T, double>) {
      if (vec_ok && m % 4 == 0 && m <= 128 && reinterpret_cast<uintptr_t>(val) % 16 == 0) {
        (k_spmm_hm_f64x4<<<(unsigned)blocks, T_, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM, ldy,
                                                         m),
         ::ff::note_launch());
        FF_LAUNCH_CHECK();
        return;
      }
    }
    if (vec_ok && std::is_same_v<T, float> && n > 0 && n < (long long)sm_count() * 16)
      (k_spmm_hm_vec_split<T><<<(unsigned)n, 32 * kSW, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM,
                                                                 ldy, m),
       ::ff::note_launch());  // few rows: a block per row
    else if (vec_ok && std::is_same_v<T, float> && m == 40)  // the solver's 40-column blocks
      (k_spmm_hm_vec<T, 10><<<(unsigned)blocks, T_, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM,
                                                              ldy, m),
       ::ff::note_launch());
    else if (vec_ok)
      (k_spmm_hm_vec<T><<<(unsigned)blocks, T_, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM, ldy, m),
       ::ff::note_launch());
    else
      (k_spmm_hm<T><<<(unsigned)blocks, T_, 0, st>>>(ptr, col, val, n, X, ldx, YH, YM, ldy, m),
       ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
}

// One warp per row; lanes form groups of G = m / 8 lanes, each lane owning 8
// consecutive columns (one 16-byte load of 8 BF16 values per gathered row);
// the P = 32 / G groups take P nonzeros of the row at a time.  GT > 0 fixes G
// at compile time (the block widths the solver uses), GT = 0 reads it from m.
// Offsets within a row and into the direction block are 32-bit (the host
// checks n * m < 2^31).
__device__ __forceinline__ void bf8_load(const __nv_bfloat16* p, float (&v)[8]) {
  const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
  const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) {  // a BF16 value is the top half of an FP32 one
    v[2 * u] = __uint_as_float(w[u] << 16);
    v[2 * u + 1] = __uint_as_float(w[u] & 0xffff0000u);
  }
}

template <int GT>
__global__ void __launch_bounds__(256)
    k_cheb_step_b16(const long long* __restrict__ ptr, const int* __restrict__ col,
                    const float* __restrict__ hv, const float* __restrict__ hdiag, int n, int m_,
                    const __nv_bfloat16* __restrict__ din, __nv_bfloat16* __restrict__ dout,
                    float* __restrict__ x, float* __restrict__ res, float c1, float c2) {
  const int G = GT > 0 ? GT : m_ / 8;
  const int m = 8 * G, P = 32 / G;
  const int lane = threadIdx.x & 31;
  const int g = lane / G, cv = (lane % G) * 8;
  const bool act = g < P;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  const __nv_bfloat16* dc = din + cv;
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < n; k += warps) {
    const long long s = ptr[k];
    const int cnt = (int)(ptr[k + 1] - s);
    const int* cr = col + s;
    const float* hr = hv + s;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, hs = 0.f;
    int e = act ? g : cnt;
    for (; e + 3 * P < cnt; e += 4 * P) {
      int l[4];
      float h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        l[q] = __ldg(cr + e + q * P);
        h[q] = __ldg(hr + e + q * P);
      }
      float dl[4][8];
#pragma unroll
      for (int q = 0; q < 4; ++q) bf8_load(dc + l[q] * m, dl[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        hs += h[q];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(h[q], dl[q][u], acc[u]);
      }
    }
    for (; e < cnt; e += P) {
      float dl[8];
      const float h = __ldg(hr + e);
      bf8_load(dc + __ldg(cr + e) * m, dl);
      hs += h;
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fmaf(h, dl[u], acc[u]);
    }
#pragma unroll
    for (int off = G; off < 32; off <<= 1) {  // tree over the groups
      const bool in = lane + off < 32;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float t = __shfl_down_sync(kFull, acc[u], off);
        if (in) acc[u] += t;
      }
      const float t = __shfl_down_sync(kFull, hs, off);
      if (in) hs += t;
    }
    if (g == 0) {
      const float dinv = 1.0f / hdiag[k];
      const int o = k * m + cv;
      float dk[8];
      bf8_load(din + o, dk);
      float4* rp = reinterpret_cast<float4*>(res + o);
      float4* xp = reinterpret_cast<float4*>(x + o);
      const float4 r0 = rp[0], r1 = rp[1], x0 = xp[0], x1 = xp[1];
      float r[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      float xx[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      __align__(16) __nv_bfloat16 dn[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        r[u] -= (acc[u] - hs * dk[u]) * dinv;
        const __nv_bfloat16 q = __float2bfloat16(c1 * dk[u] + c2 * r[u]);
        dn[u] = q;
        xx[u] += __bfloat162float(q);
      }
      rp[0] = make_float4(r[0], r[1], r[2], r[3]);
      rp[1] = make_float4(r[4], r[5], r[6], r[7]);
      xp[0] = make_float4(xx[0], xx[1], xx[2], xx[3]);
      xp[1] = make_float4(xx[4], xx[5], xx[6], xx[7]);
      *reinterpret_cast<uint4*>(dout + o) = *reinterpret_cast<const uint4*>(dn);
    }
  }
}

void cheb_step_b16(cudaStream_t st, const long long* ptr, const int* col, const float* hv,
                   const float* hdiag, long long n, int m, const void* din, void* dout, float* x,
                   float* res, float c1, float c2) {
  ProfScope ps(kProfPrecond);
  FF_REQUIRE(m % 8 == 0 && m <= 256 && reinterpret_cast<uintptr_t>(din) % 16 == 0 &&
                 reinterpret_cast<uintptr_t>(dout) % 16 == 0 &&
                 reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                 reinterpret_cast<uintptr_t>(res) % 16 == 0,
             FF_ERR_INVALID_ARG, "BF16 preconditioner step needs m % 8 == 0 and aligned blocks");
  FF_REQUIRE(n * m < (1LL << 31), FF_ERR_INVALID_ARG, "BF16 preconditioner step: n * m >= 2^31");
  const int T_ = 256;
  long long blocks = std::min<long long>((n * 32 + T_ - 1) / T_, (long long)sm_count() * 64);
  const auto* bi = static_cast<const __nv_bfloat16*>(din);
  auto* bo = static_cast<__nv_bfloat16*>(dout);
  const int ni = (int)n;
#define FF_CHEB16(GT)                                                                     \
  (k_cheb_step_b16<GT><<<(unsigned)blocks, T_, 0, st>>>(ptr, col, hv, hdiag, ni, m, bi, bo, x, \
                                                        res, c1, c2),                     \
   ::ff::note_launch())
  switch (m / 8) {
    case 4: FF_CHEB16(4); break;
    case 5: FF_CHEB16(5); break;
    case 6: FF_CHEB16(6); break;
    case 8: FF_CHEB16(8); break;
    default: FF_CHEB16(0); break;
  }
#undef FF_CHEB16
  FF_LAUNCH_CHECK();
}

void cheb_step(cudaStream_t st, const long long* ptr, const int* col, const float* hv,
               const float* hdiag, long long n, int m, int ld, const float* din, float* dout,
               float* x, float* res, float c1, float c2, int prof) {
  ProfScope ps(prof);
  const int T_ = 256;
  long long blocks = std::min<long long>((n * 32 + T_ - 1) / T_, (long long)sm_count() * 64);
  const bool vec_ok = m % 4 == 0 && m <= 128 && ld % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(din) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(dout) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(res) % 16 == 0;
  if (vec_ok)
    (k_cheb_step_vec<<<(unsigned)blocks, T_, 0, st>>>(ptr, col, hv, hdiag, n, m, ld, din, dout, x,
                                                     res, c1, c2), ::ff::note_launch());
  else
    (k_cheb_step<<<(unsigned)blocks, T_, 0, st>>>(ptr, col, hv, hdiag, n, m, ld, din, dout, x, res,
                                                 c1, c2), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

namespace {

bool al16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// append the TW x TW tiles of a (p x q) product A^T B written at out (row
// stride ldo); false when the list would overflow
template <class T>
bool add_tiles(GramTiles& g, int TW, const T* A, int p, const T* B, int q, double* out, int ldo,
               int diag_only = 0) {
  for (int i0 = 0; i0 < p; i0 += TW)
    for (int j0 = 0; j0 < q; j0 += TW) {
      if (diag_only && i0 != j0) continue;
      if (g.count == kMaxGramTiles) return false;
      g.t[g.count++] = GramTile{A + i0, B + j0, out + (long long)i0 * ldo + j0,
                                std::min(TW, p - i0), std::min(TW, q - j0), diag_only};
    }
  return true;
}

template <class T>
void launch_tiles(cudaStream_t st, const GramTiles& g, int TW, int lda, int ldb, long long n,
                  int ldo, double alpha, bool accumulate, Buf& part) {
  // about four blocks per SM in all, at least 64 rows per chunk
  long long chunks = std::max<long long>(1, ((long long)sm_count() * 4) / g.count);
  chunks = std::max<long long>(1, std::min(chunks, (n + 63) / 64));
  const long long rpc = (n + chunks - 1) / chunks;
  chunks = (n + rpc - 1) / rpc;
  double* pp = reinterpret_cast<double*>(part.ensure(sizeof(double) * chunks * g.count * TW * TW));
  dim3 grid((unsigned)chunks, (unsigned)g.count);
  dim3 rgrid((unsigned)((TW * TW + 31) / 32), (unsigned)g.count);
  if (TW == 40) {
    (k_gram_tiles<T, 40><<<grid, 200, 0, st>>>(g, lda, ldb, n, rpc, pp), ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_gram_tiles_reduce<40><<<rgrid, 32 * kRedWarps, 0, st>>>(g, (int)chunks, ldo, alpha,
                                                                accumulate ? 1 : 0, pp),
     ::ff::note_launch());
  } else {
    (k_gram_tiles<T, 32><<<grid, 256, 0, st>>>(g, lda, ldb, n, rpc, pp), ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_gram_tiles_reduce<32><<<rgrid, 32 * kRedWarps, 0, st>>>(g, (int)chunks, ldo, alpha,
                                                                accumulate ? 1 : 0, pp),
     ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
}

}  // namespace

template <class T>
void gram(cudaStream_t st, const T* A, int lda, int p, const T* B, int ldb, int q, long long n,
          double* out, double alpha, bool accumulate, Buf& part, int ldo) {
  if (p <= 0 || q <= 0) return;
  ProfScope ps(kProfGram);
  if (p % 4 == 0 && q % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 && al16(A) && al16(B)) {
    const int TW = p % 40 == 0 && q % 40 == 0 ? 40 : 32;
    GramTiles g;
    g.count = 0;
    if (add_tiles(g, TW, A, p, B, q, out, ldo < 0 ? q : ldo)) {
      launch_tiles<T>(st, g, TW, lda, ldb, n, ldo < 0 ? q : ldo, alpha, accumulate, part);
      return;
    }
  }
  if (p == 1 && q <= 256) {  // a row vector times a block: no tile of padding
    const long long chunks = std::max<long long>(1, std::min<long long>((n + 255) / 256, 608));
    const long long rpc = (n + chunks - 1) / chunks;
    double* pp = reinterpret_cast<double*>(part.ensure(sizeof(double) * chunks * q));
    (k_gram_row<T><<<(unsigned)chunks, 256, 0, st>>>(A, lda, B, ldb, q, n, rpc, pp),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    (k_gram_reduce<<<(q + 31) / 32, 32 * kRedWarps, 0, st>>>(
         pp, (int)chunks, q, q, out, ldo < 0 ? q : ldo, alpha, accumulate ? 1 : 0),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    return;
  }
  const bool w40 = p % 40 == 0 && q % 40 == 0;
  const int TW = w40 ? 40 : 32;
  const int tiles = ((p + TW - 1) / TW) * ((q + TW - 1) / TW);
  long long chunks = std::max<long long>(1, std::min<long long>((n + 511) / 512, 2048 / tiles + 1));
  long long rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + 31) / 32 * 32;
  chunks = std::max<long long>(1, (n + rpc - 1) / rpc);
  double* pp = reinterpret_cast<double*>(part.ensure(sizeof(double) * chunks * p * q));
  dim3 grid((unsigned)chunks, (unsigned)tiles);
  if (w40)
    (k_gram_partial<T, 40><<<grid, 320, 0, st>>>(A, lda, p, B, ldb, q, n, rpc, pp),
     ::ff::note_launch());
  else
    (k_gram_partial<T, 32><<<grid, 256, 0, st>>>(A, lda, p, B, ldb, q, n, rpc, pp),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_gram_reduce<<<(p * q + 31) / 32, 32 * kRedWarps, 0, st>>>(
       pp, (int)chunks, p * q, q, out, ldo < 0 ? q : ldo, alpha, accumulate ? 1 : 0),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

void gram_mirror(cudaStream_t st, double* A, double* B, int ns, int nb) {
  (k_gram_mirror<<<(ns * ns + 255) / 256, 256, 0, st>>>(A, B, ns, nb), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template <class T>
void gram_rr(cudaStream_t st, const T* S, const T* HS, const T* MS, int ld, int nb, int nblk,
             long long n, double* A, double* B, Buf& part) {
  const int ns = nblk * nb;
  // FP32 blocks: split-BF16 x 3 products on the tensor cores when the basis fits
  if constexpr (std::is_same_v<T, float>)
    if (gram_tc_enabled() && gram_rr_tc(st, S, HS, MS, ld, nb, nblk, n, A, B, part)) return;
  if (nb % 4 == 0 && ld % 4 == 0 && al16(S) && al16(HS) && al16(MS)) {
    // all tiles in one launch: the lower block triangle of A, the W columns
    // of B and the diagonals of B's X and P blocks
    const int TW = nb % 40 == 0 ? 40 : 32;
    GramTiles g;
    g.count = 0;
    bool ok = true;
    for (int j = 0; j < nblk && ok; ++j)
      for (int i = j; i < nblk && ok; ++i)
        ok = add_tiles(g, TW, S + i * nb, nb, HS + j * nb, nb, A + (long long)i * nb * ns + j * nb,
                       ns);
    for (int i = 0; i < nblk && ok; ++i)
      ok = add_tiles(g, TW, S + i * nb, nb, MS + nb, nb, B + (long long)i * nb * ns + nb, ns);
    for (int i = 0; i < nblk && ok; ++i)
      if (i != 1)
        ok = add_tiles(g, TW, S + i * nb, nb, MS + i * nb, nb,
                       B + (long long)i * nb * ns + i * nb, ns, 1);
    if (ok) {
      ProfScope ps(kProfGram);
      launch_tiles<T>(st, g, TW, ld, ld, n, ns, 1.0, false, part);
      (k_gram_mirror<<<(ns * ns + 255) / 256, 256, 0, st>>>(A, B, ns, nb), ::ff::note_launch());
      FF_LAUNCH_CHECK();
      return;
    }
  }
  // lower block triangle: A_ij = S_i^T (H S_j) for block i >= j.  The products
  // of the smooth, converging blocks (H X) are the accurate ones; W^T (H X)
  // is taken rather than X^T (H W), whose rounding follows the rough W.
  for (int j = 0; j < nblk; ++j)
    gram<T>(st, S + j * nb, ld, ns - j * nb, HS + j * nb, ld, nb, n,
            A + (long long)j * nb * ns + j * nb, 1.0, false, part, ns);
  gram<T>(st, S, ld, ns, MS + nb, ld, nb, n, B + nb, 1.0, false, part, ns);
  ProfScope ps(kProfGram);
  (k_gram_diag<T><<<(unsigned)(ns - nb), 512, 0, st>>>(S, MS, ld, n, nb, 2 * nb, B, ns),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_gram_mirror<<<(ns * ns + 255) / 256, 256, 0, st>>>(A, B, ns, nb), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template <class T>
void block_update(cudaStream_t st, const T* A, int lda, int p, const T* Y, int q, T* C, int ldc,
                  long long n, T beta, int split, int off2, int ldy) {
  if (q <= 0 || n <= 0) return;
  ProfScope ps(kProfUpdate);
  if (p <= 0) {
    // C = beta * C only; p == 0 never happens in the solver
    return;
  }
  const bool w40 = q % 40 == 0;
  const int TW = w40 ? 40 : 32;
  size_t smem = sizeof(T) * (size_t)p * TW;
  const int sp = split < 0 ? q : split;
  if (p % 4 == 0 && q % 4 == 0 && lda % 4 == 0 && ldc % 4 == 0 && sp % 4 == 0 && off2 % 4 == 0 &&
      al16(A) && al16(C) && smem <= 200 * 1024) {
    if (smem > 48 * 1024)
      set_max_dyn_smem(w40 ? (const void*)k_block_update_rt<T, 40>
                           : (const void*)k_block_update_rt<T, 32>,
                       200 * 1024);
    const int TD = TW / 4, RG = 256 / TD;
    const long long rows_per_block = (long long)RG * 4;
    dim3 grid((unsigned)std::min<long long>((n + rows_per_block - 1) / rows_per_block, (long long)sm_count() * 8),
              (unsigned)((q + TW - 1) / TW));
    if (w40)
      (k_block_update_rt<T, 40><<<grid, TD * RG, smem, st>>>(A, lda, p, Y, ldy < 0 ? q : ldy, q, C,
                                                            ldc, n, beta, sp, off2),
       ::ff::note_launch());
    else
      (k_block_update_rt<T, 32><<<grid, TD * RG, smem, st>>>(A, lda, p, Y, ldy < 0 ? q : ldy, q, C,
                                                            ldc, n, beta, sp, off2),
       ::ff::note_launch());
    FF_LAUNCH_CHECK();
    return;
  }
  const int rpb = 8;  // rows per block (one TW-thread group each)
  if (smem > 48 * 1024)
    set_max_dyn_smem(w40 ? (const void*)k_block_update<T, 40> : (const void*)k_block_update<T, 32>,
                     227 * 1024);
  dim3 grid((unsigned)std::min<long long>((n + rpb - 1) / rpb, (long long)sm_count() * 16),
            (unsigned)((q + TW - 1) / TW));
  if (w40)
    (k_block_update<T, 40><<<grid, 40 * rpb, smem, st>>>(A, lda, p, Y, ldy < 0 ? q : ldy, q, C,
                                                        ldc, n, beta, split < 0 ? q : split, off2),
     ::ff::note_launch());
  else
    (k_block_update<T, 32><<<grid, 32 * rpb, smem, st>>>(A, lda, p, Y, ldy < 0 ? q : ldy, q, C,
                                                        ldc, n, beta, split < 0 ? q : split, off2),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template void spmm_hm_raw<float>(cudaStream_t, const long long*, const int*, const float*,
                                 long long, const float*, int, float*, float*, int, int);
template void spmm_hm_raw<double>(cudaStream_t, const long long*, const int*, const double*,
                                  long long, const double*, int, double*, double*, int, int);
template void gram<float>(cudaStream_t, const float*, int, int, const float*, int, int, long long,
                          double*, double, bool, Buf&, int);
template void gram<double>(cudaStream_t, const double*, int, int, const double*, int, int,
                           long long, double*, double, bool, Buf&, int);
template void gram_rr<float>(cudaStream_t, const float*, const float*, const float*, int, int, int,
                             long long, double*, double*, Buf&);
template void gram_rr<double>(cudaStream_t, const double*, const double*, const double*, int, int,
                              int, long long, double*, double*, Buf&);
template void block_update<float>(cudaStream_t, const float*, int, int, const float*, int, float*,
                                  int, long long, float, int, int, int);
template void block_update<double>(cudaStream_t, const double*, int, int, const double*, int,
                                   double*, int, long long, double, int, int, int);
template void spmm_hm_raw<dfloat>(cudaStream_t, const long long*, const int*, const dfloat*,
                                  long long, const dfloat*, int, dfloat*, dfloat*, int, int);
template void gram<dfloat>(cudaStream_t, const dfloat*, int, int, const dfloat*, int, int,
                           long long, double*, double, bool, Buf&, int);
template void gram_rr<dfloat>(cudaStream_t, const dfloat*, const dfloat*, const dfloat*, int, int,
                              int, long long, double*, double*, Buf&);
template void block_update<dfloat>(cudaStream_t, const dfloat*, int, int, const dfloat*, int,
                                   dfloat*, int, long long, dfloat, int, int, int);

}  // namespace ff
