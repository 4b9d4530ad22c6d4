// The paper's two-set RKPM discretisation (Supp. Sec. B "RKPM construction",
// with the Gaussian kernel of Sec. 3.2).
//
// Quadrature points X_i with volumes v_i (an inside grid of the object, or its
// own points); K kernel centres p_k chosen among them by farthest-point
// sampling; radius r_k = distance from p_k to its second-nearest other centre;
// raw kernel exp(-|X - p_k|^2 / r_k^2), cut at t r_k when t > 0; the corrected
// shape functions of Eqs. 7, 9-10 at the quadrature points.  The result is laid
// out like the nodal discretisation's (rows = quadrature points, columns =
// centres, plus the transposed lists), so the assembly of H_w (Prop. 1) and M
// (Eq. 14) and the eigensolver run unchanged on the K centres.
//
// Every decision taken in floating point is the FP64 one on the FP32-stored
// points, each operation rounded separately:
//   * squared distances ((dx*dx + dy*dy) + dz*dz);
//   * farthest-point sampling from `start`, ties to the lowest index;
//   * r_k = sqrt of the second-smallest squared distance to the other centres;
//   * centre k covers X iff d2 < (t*t) * (r_k*r_k).
// Each is first settled in FP32 with a relative margin of 1e-5 (FP32 and FP64
// squared distances differ by less than 4e-7 relative); only values within
// the margin are evaluated in FP64.  Distances are compared by their FP64 bit
// patterns where they are ordered (non-negative doubles order like integers).
//
// Kernels:
//   k_fps          one 8-block cluster: each block keeps its slice of points
//                  and their running squared distance to the chosen set in
//                  shared memory (global memory when it does not fit); per
//                  chosen centre: update, block arg-max, one cluster barrier,
//                  every block reduces the 8 published candidates itself
//   k_radii        one warp per centre: the two smallest squared distances
//   k_cover_rows   one thread per point: its covering centres, ascending
//   k_cover_cols   one warp per centre: the points it covers, ascending, and
//                  the centre's position in each point's row
//   k_shape_twoset one warp per quadrature point, Eqs. 7, 9-10 with the Gaussian
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "ff_internal.cuh"
#include "rkpm_eval.cuh"

namespace ff {
namespace {

constexpr int kFpsCS = 8;                    // blocks per cluster
constexpr int kFpsT = 1024;                  // threads per block
constexpr int kFpsSmemMax = 200 * 1024;      // dynamic shared memory per block
constexpr int kFpsGridMin = 200000;          // points from which the whole GPU samples
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double d2_f64(float ax, float ay, float az, float bx, float by,
                                         float bz) {
  const double dx = __dsub_rn((double)ax, (double)bx);
  const double dy = __dsub_rn((double)ay, (double)by);
  const double dz = __dsub_rn((double)az, (double)bz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ float d2_f32(float ax, float ay, float az, float bx, float by,
                                        float bz) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// centre (p, l32 = fl32(lim), lim = t^2 r^2 or +inf) covers the point (x, y, z)
__device__ __forceinline__ bool covers2(float x, float y, float z, float4 p, float l32,
                                        double lim) {
  if (l32 >= 1e-30f) {
    const float d32 = d2_f32(x, y, z, p.x, p.y, p.z);
    if (d32 < __fmul_rn(l32, 0.99999f)) return true;
    if (d32 > __fmul_rn(l32, 1.00001f)) return false;
  }
  return d2_f64(x, y, z, p.x, p.y, p.z) < lim;
}

// ------------------------------------------------------------------ validation
__global__ void k_validate_points(const float* __restrict__ X, const float* __restrict__ v,
                                  long long n, int* __restrict__ bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2], vi = v[i];
    const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && fabsf(x) < 1e18f &&
                    fabsf(y) < 1e18f && fabsf(z) < 1e18f && isfinite(vi) && vi > 0.f;
    if (!ok) atomicMin(bad, (int)i);
  }
}

// ------------------------------------------------------------------ farthest-point sampling
struct FpsCand {
  unsigned long long key;  // bit pattern of the squared distance (>= 0)
  int idx;
  float x, y, z;
  int pad;
};

__device__ __forceinline__ void fps_pick(FpsCand& a, unsigned long long key, int idx, float x,
                                         float y, float z) {
  if (key > a.key || (key == a.key && idx < a.idx)) {
    a.key = key;
    a.idx = idx;
    a.x = x;
    a.y = y;
    a.z = z;
  }
}

__device__ __forceinline__ void fps_warp_max(FpsCand& a) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(kFull, a.key, o);
    const int i2 = __shfl_xor_sync(kFull, a.idx, o);
    const float x2 = __shfl_xor_sync(kFull, a.x, o);
    const float y2 = __shfl_xor_sync(kFull, a.y, o);
    const float z2 = __shfl_xor_sync(kFull, a.z, o);
    fps_pick(a, k2, i2, x2, y2, z2);
  }
}

// Block b owns points [b S, min(n, (b + 1) S)).  cur = squared distance to the
// chosen set (FP64), cur32 its FP32 rounding for the filter.  Every block
// computes the same winner from the same 8 candidates, so all leave the loop
// together; the published candidates alternate between two buffers, so the
// one cluster barrier per step also orders their reuse.
__global__ void __cluster_dims__(kFpsCS, 1, 1) __launch_bounds__(kFpsT, 1)
    k_fps(const float* __restrict__ X, int n, int K, int start, int S, int in_smem,
          float* __restrict__ gxyz, double* __restrict__ gcur, float* __restrict__ gcur32,
          long long* __restrict__ chosen, DevFlags* __restrict__ flags) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int p0 = min(rank * S, n);
  const int cnt = min(n - p0, S);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ FpsCand pub[2];
  __shared__ FpsCand red[kFpsT / 32];
  double* cur;
  float *cur32, *xs, *ys, *zs;
  if (in_smem) {
    cur = reinterpret_cast<double*>(sm_raw);
    cur32 = reinterpret_cast<float*>(cur + S);
    xs = cur32 + S;
    ys = xs + S;
    zs = ys + S;
  } else {
    cur = gcur + p0;
    cur32 = gcur32 + p0;
    xs = gxyz + p0;
    ys = gxyz + (size_t)n + p0;
    zs = gxyz + 2 * (size_t)n + p0;
  }
  const float sx = X[3LL * start], sy = X[3LL * start + 1], sz = X[3LL * start + 2];
  for (int p = tid; p < cnt; p += kFpsT) {
    const long long g = (long long)p0 + p;
    const float x = X[3 * g], y = X[3 * g + 1], z = X[3 * g + 2];
    xs[p] = x;
    ys[p] = y;
    zs[p] = z;
    const double d = d2_f64(x, y, z, sx, sy, sz);
    cur[p] = d;
    cur32[p] = (float)d;
  }
  if (rank == 0 && tid == 0) chosen[0] = start;
  __syncthreads();
  float cx = sx, cy = sy, cz = sz;
  for (int j = 1; j < K; ++j) {
    const int buf = j & 1;
    FpsCand best{0ull, INT_MAX, 0.f, 0.f, 0.f, 0};
    for (int p = tid; p < cnt; p += kFpsT) {
      const float x = xs[p], y = ys[p], z = zs[p];
      double c = cur[p];
      if (j > 1) {  // fold in the centre chosen last (the start is in already)
        const float c32 = cur32[p];
        if (c32 < 1e-30f || d2_f32(x, y, z, cx, cy, cz) <= __fmul_rn(c32, 1.00001f)) {
          const double d = d2_f64(x, y, z, cx, cy, cz);
          if (d < c) {
            c = d;
            cur[p] = d;
            cur32[p] = (float)d;
          }
        }
      }
      fps_pick(best, (unsigned long long)__double_as_longlong(c), p0 + p, x, y, z);
    }
    fps_warp_max(best);
    if (lane == 0) red[wid] = best;
    __syncthreads();
    if (wid == 0) {
      FpsCand b = red[lane];
      fps_warp_max(b);
      if (lane == 0) pub[buf] = b;
    }
    cl.sync();
    FpsCand win{0ull, INT_MAX, 0.f, 0.f, 0.f, 0};
#pragma unroll
    for (int q = 0; q < kFpsCS; ++q) {
      const FpsCand r = *cl.map_shared_rank(&pub[buf], q);
      fps_pick(win, r.key, r.idx, r.x, r.y, r.z);
    }
    if (win.key == 0ull || win.idx == INT_MAX) {
      // every remaining point coincides with a chosen centre
      if (rank == 0 && tid == 0 && atomicCAS(&flags->code, 0, (int)FF_ERR_INVALID_ARG) == 0)
        flags->index = j;
      break;
    }
    if (rank == 0 && tid == 0) chosen[j] = win.idx;
    cx = win.x;
    cy = win.y;
    cz = win.z;
  }
  cl.sync();  // no block leaves while another may still read its candidates
}

// The same sampling on the whole GPU: one block per SM in a cooperative
// launch, each holding its slice of the points and their running distances in
// shared memory (global memory when the slice does not fit).  Per centre:
// update, block arg-max, the block's candidate published to global memory
// (two buffers by parity), a grid barrier, and every block reduces all the
// published candidates itself -- the same winner everywhere, so every block
// leaves the loop at the same step.  The barrier is a monotone arrival counter
// in global memory; its wait is bounded (about a second of clock cycles) and
// a block that gives up records FF_ERR_TIMEOUT in the flags and in `abort`, and
// every block leaves the loop at the next barrier it sees it at.
constexpr long long kGridWaitCycles = 2000000000LL;

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* abort,
                                             DevFlags* flags,
                                             long long limit = kGridWaitCycles) {
  __shared__ int s_abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const long long t0 = clock64();
    int ab = 0;
    while (*reinterpret_cast<volatile unsigned*>(bar) < target) {
      if (*reinterpret_cast<volatile int*>(abort)) {
        ab = 1;
        break;
      }
      if (clock64() - t0 > limit) {
        atomicExch(abort, 1);
        if (atomicCAS(&flags->code, 0, (int)FF_ERR_TIMEOUT) == 0) flags->index = -1;
        ab = 1;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_abort = ab || *reinterpret_cast<volatile int*>(abort);
  }
  __syncthreads();
  return s_abort == 0;
}

__global__ void __launch_bounds__(kFpsT, 1)
    k_fps_grid(const float* __restrict__ X, int n, int K, int start, int S, int in_smem,
               float* __restrict__ gxyz, double* __restrict__ gcur, float* __restrict__ gcur32,
               long long* __restrict__ chosen, FpsCand* __restrict__ cand, unsigned* bar,
               int* abort, DevFlags* __restrict__ flags) {
  const int G = gridDim.x, rank = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int p0 = min(rank * S, n);
  const int cnt = min(n - p0, S);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ FpsCand red[kFpsT / 32];
  __shared__ FpsCand s_win;
  double* cur;
  float *cur32, *xs, *ys, *zs;
  if (in_smem) {
    cur = reinterpret_cast<double*>(sm_raw);
    cur32 = reinterpret_cast<float*>(cur + S);
    xs = cur32 + S;
    ys = xs + S;
    zs = ys + S;
  } else {
    cur = gcur + p0;
    cur32 = gcur32 + p0;
    xs = gxyz + p0;
    ys = gxyz + (size_t)n + p0;
    zs = gxyz + 2 * (size_t)n + p0;
  }
  const float sx = X[3LL * start], sy = X[3LL * start + 1], sz = X[3LL * start + 2];
  for (int p = tid; p < cnt; p += kFpsT) {
    const long long g = (long long)p0 + p;
    const float x = X[3 * g], y = X[3 * g + 1], z = X[3 * g + 2];
    xs[p] = x;
    ys[p] = y;
    zs[p] = z;
    const double d = d2_f64(x, y, z, sx, sy, sz);
    cur[p] = d;
    cur32[p] = (float)d;
  }
  if (rank == 0 && tid == 0) chosen[0] = start;
  __syncthreads();
  float cx = sx, cy = sy, cz = sz;
  for (int j = 1; j < K; ++j) {
    FpsCand best{0ull, INT_MAX, 0.f, 0.f, 0.f, 0};
    for (int p = tid; p < cnt; p += kFpsT) {
      const float x = xs[p], y = ys[p], z = zs[p];
      double c = cur[p];
      if (j > 1) {  // fold in the centre chosen last (the start is in already)
        const float c32 = cur32[p];
        if (c32 < 1e-30f || d2_f32(x, y, z, cx, cy, cz) <= __fmul_rn(c32, 1.00001f)) {
          const double d = d2_f64(x, y, z, cx, cy, cz);
          if (d < c) {
            c = d;
            cur[p] = d;
            cur32[p] = (float)d;
          }
        }
      }
      fps_pick(best, (unsigned long long)__double_as_longlong(c), p0 + p, x, y, z);
    }
    fps_warp_max(best);
    if (lane == 0) red[wid] = best;
    __syncthreads();
    if (wid == 0) {
      FpsCand b = red[lane];
      fps_warp_max(b);
      if (lane == 0) cand[(size_t)(j & 1) * G + rank] = b;
    }
    if (!grid_barrier(bar, (unsigned)j * (unsigned)G, abort, flags)) break;
    // every block reduces all the published candidates (L1 bypassed)
    FpsCand w{0ull, INT_MAX, 0.f, 0.f, 0.f, 0};
    const FpsCand* cj = cand + (size_t)(j & 1) * G;
    for (int q = tid; q < G; q += kFpsT) {
      const unsigned long long key = __ldcg(reinterpret_cast<const unsigned long long*>(&cj[q].key));
      const int idx = __ldcg(&cj[q].idx);
      const float x = __ldcg(&cj[q].x), y = __ldcg(&cj[q].y), z = __ldcg(&cj[q].z);
      fps_pick(w, key, idx, x, y, z);
    }
    fps_warp_max(w);
    if (lane == 0) red[wid] = w;
    __syncthreads();
    if (wid == 0) {
      FpsCand b = red[lane];
      fps_warp_max(b);
      if (lane == 0) s_win = b;
    }
    __syncthreads();
    const FpsCand win = s_win;
    if (win.key == 0ull || win.idx == INT_MAX) {
      // every remaining point coincides with a chosen centre
      if (rank == 0 && tid == 0 && atomicCAS(&flags->code, 0, (int)FF_ERR_INVALID_ARG) == 0)
        flags->index = j;
      break;
    }
    if (rank == 0 && tid == 0) chosen[j] = win.idx;
    cx = win.x;
    cy = win.y;
    cz = win.z;
    __syncthreads();  // s_win and red are rewritten in the next step
  }
}

// Self-check of the bounded wait: every block arrives once at a barrier that
// waits for one arrival more than the grid has, so the wait can only end by
// running out (FF_ERR_TIMEOUT in the flags) or through the abort word.
__global__ void k_wait_check(unsigned* bar, int* abort, DevFlags* flags, long long limit) {
  grid_barrier(bar, gridDim.x + 1u, abort, flags, limit);
}

__global__ void k_gather_centres(const float* __restrict__ X, const long long* __restrict__ chosen,
                                 int K, float4* __restrict__ cpos) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const long long i = chosen[k];
  cpos[k] = make_float4(X[3 * i], X[3 * i + 1], X[3 * i + 2], 0.f);
}

// ------------------------------------------------------------------ radii
// r_k = sqrt(second-smallest squared distance to the other centres); lim_k =
// (t*t) * (r_k*r_k) or +inf without a cut.
__global__ void k_radii(const float4* __restrict__ cpos, int K, double tt, double* __restrict__ rad,
                        double* __restrict__ lim, float* __restrict__ lim32,
                        DevFlags* __restrict__ flags) {
  const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (k >= K) return;
  const int lane = threadIdx.x & 31;
  const float4 p = cpos[k];
  double m1 = INFINITY, m2 = INFINITY;
  for (int j = lane; j < K; j += 32) {
    if (j == k) continue;
    const float4 q = cpos[j];
    const double d = d2_f64(q.x, q.y, q.z, p.x, p.y, p.z);
    if (d < m1) {
      m2 = m1;
      m1 = d;
    } else if (d < m2) {
      m2 = d;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double a1 = __shfl_xor_sync(kFull, m1, o);
    const double a2 = __shfl_xor_sync(kFull, m2, o);
    const double lo = fmin(m1, a1);
    const double hi = fmin(fmax(m1, a1), fmin(m2, a2));
    m1 = lo;
    m2 = hi;
  }
  if (lane == 0) {
    const double r = __dsqrt_rn(m2);
    rad[k] = r;
    const double L = tt > 0.0 ? __dmul_rn(tt, __dmul_rn(r, r)) : (double)INFINITY;
    lim[k] = L;
    lim32[k] = (float)L;
    if (!(r > 0.0) || !isfinite(r))
      if (atomicCAS(&flags->code, 0, (int)FF_ERR_INVALID_ARG) == 0) flags->index = k;
  }
}

// ------------------------------------------------------------------ covering lists
// MODE 0: count the centres covering each point; MODE 1: list them, ascending
template <int MODE>
__global__ void __launch_bounds__(256)
    k_cover_rows(const float* __restrict__ Xq, long long nq, const float4* __restrict__ cpos,
                 const float* __restrict__ lim32, const double* __restrict__ lim, int K,
                 int* __restrict__ cnt, const long long* __restrict__ rptr,
                 int* __restrict__ ridx) {
  __shared__ float4 sp[256];
  __shared__ float sl32[256];
  __shared__ double sl[256];
  const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
  const bool live = i < nq;
  float x = 0.f, y = 0.f, z = 0.f;
  long long base = 0, end = 0;
  if (live) {
    x = Xq[3 * i];
    y = Xq[3 * i + 1];
    z = Xq[3 * i + 2];
    if (MODE) {
      base = rptr[i];
      end = rptr[i + 1];
    }
  }
  int c = 0;
  for (int k0 = 0; k0 < K; k0 += 256) {
    __syncthreads();
    if (k0 + (int)threadIdx.x < K) {
      sp[threadIdx.x] = cpos[k0 + threadIdx.x];
      sl32[threadIdx.x] = lim32[k0 + threadIdx.x];
      sl[threadIdx.x] = lim[k0 + threadIdx.x];
    }
    __syncthreads();
    const int kn = min(256, K - k0);
    if (live) {
      for (int q = 0; q < kn; ++q) {
        if (covers2(x, y, z, sp[q], sl32[q], sl[q])) {
          if (MODE && base + c < end) ridx[base + c] = k0 + q;
          ++c;
        }
      }
    }
  }
  if (!MODE && live) cnt[i] = c;
}

// MODE 0: count the points each centre covers; MODE 1: list them (ascending)
// with the position of the centre in each point's (ascending) row
template <int MODE>
__global__ void k_cover_cols(const float* __restrict__ Xq, long long nq,
                             const float4* __restrict__ cpos, const float* __restrict__ lim32,
                             const double* __restrict__ lim, int K, int* __restrict__ cnt,
                             const long long* __restrict__ tptr, int* __restrict__ tidx,
                             long long* __restrict__ tpos, const long long* __restrict__ rptr,
                             const int* __restrict__ ridx, DevFlags* __restrict__ flags) {
  const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (k >= K) return;
  const int lane = threadIdx.x & 31;
  const float4 p = cpos[k];
  const float l32 = lim32[k];
  const double l64 = lim[k];
  const long long base = MODE ? tptr[k] : 0, end = MODE ? tptr[k + 1] : 0;
  long long c = 0;
  for (long long i0 = 0; i0 < nq; i0 += 32) {
    const long long i = i0 + lane;
    bool cov = false;
    if (i < nq) cov = covers2(Xq[3 * i], Xq[3 * i + 1], Xq[3 * i + 2], p, l32, l64);
    const unsigned bal = __ballot_sync(kFull, cov);
    if (MODE && cov) {
      const long long slot = base + c + __popc(bal & ((1u << lane) - 1u));
      if (slot < end) {
        long long lo = rptr[i], hi = rptr[i + 1];
        const long long row_end = hi;
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (ridx[mid] < k)
            lo = mid + 1;
          else
            hi = mid;
        }
        tidx[slot] = (int)i;
        if (lo < row_end && ridx[lo] == k) {
          tpos[slot] = lo;
        } else {  // the two passes disagree: report, keep the position in range
          tpos[slot] = rptr[i];
          if (atomicCAS(&flags->code, 0, (int)FF_ERR_CUDA) == 0) flags->index = k;
        }
      }
    }
    c += __popc(bal);
  }
  if (!MODE && lane == 0) cnt[k] = (int)c;
}

// ------------------------------------------------------------------ shape functions
template <class T>
__global__ void __launch_bounds__(256, 2) k_shape_twoset(const float4* __restrict__ cpos, const double* __restrict__ rad,
                               const float* __restrict__ Xq, float scale,
                               const long long* __restrict__ ptr, const int* __restrict__ idx,
                               long long nq, long long n1, T* __restrict__ phi,
                               T* __restrict__ dphi, double cond_limit,
                               DevFlags* __restrict__ flags) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= nq) return;
  const int lane = threadIdx.x & 31;
  const long long s = ptr[i], e = ptr[i + 1];
  const float4 Xi = make_float4(Xq[3 * i], Xq[3 * i + 1], Xq[3 * i + 2], scale);
  const rkpm::Gauss kern{rad};
  int st = 1;
  if (e > s) {
    if constexpr (sizeof(T) == 4) {
      st = rkpm::shape_row<float, T>(cpos, s, e, idx, Xi, phi, dphi, n1, cond_limit, true, kern);
      if (st != 0) {
        st = rkpm::shape_row<double, T>(cpos, s, e, idx, Xi, phi, dphi, n1, 0.0, false, kern);
        if (lane == 0 && st == 0) atomicAdd(&flags->fallback, 1);
      }
    } else {
      st = rkpm::shape_row<dfloat, T>(cpos, s, e, idx, Xi, phi, dphi, n1, 0.0, false, kern);
    }
  }
  if (st != 0 && lane == 0)
    if (atomicCAS(&flags->code, 0, (int)FF_ERR_SINGULAR_MOMENT) == 0) flags->index = (int)i;
}

__global__ void k_iota(int* __restrict__ a, int* __restrict__ b, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    a[t] = t;
    b[t] = t;
  }
}

__global__ void k_copy_f32(const float* __restrict__ x, float* __restrict__ y, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = x[t];
}

}  // namespace

// Covering lists of arbitrary points (the rows of a shape-function table over
// the two-set centres): count, scan, fill.  Returns the number of pairs.
long long twoset_cover(ff_ctx* c, const float* Q, long long nq, Buf& ptrb, Buf& idxb,
                       Buf& cntb) {
  cudaStream_t st = c->stream;
  const int K = (int)c->n;
  int* cnt = reinterpret_cast<int*>(cntb.ensure(sizeof(int) * (nq + 1)));
  (k_cover_rows<0><<<ceil_div(nq, 256), 256, 0, st>>>(
       Q, nq, c->pos.as<float4>(), c->clim32.as<float>(), c->clim.as<double>(), K, cnt, nullptr,
       nullptr),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  long long* ptr = reinterpret_cast<long long*>(ptrb.ensure(sizeof(long long) * (nq + 1)));
  scan_counts(cnt, ptr, nq, c, c->scratch[3]);
  long long n1 = 0;
  FF_CUDA(cudaMemcpyAsync(&n1, ptr + nq, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  int* idx = reinterpret_cast<int*>(idxb.ensure(sizeof(int) * std::max(n1, 1LL)));
  (k_cover_rows<1><<<ceil_div(nq, 256), 256, 0, st>>>(
       Q, nq, c->pos.as<float4>(), c->clim32.as<float>(), c->clim.as<double>(), K, nullptr, ptr,
       idx),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  return n1;
}

// Gaussian shape functions of the two-set centres at nq points (one warp each);
// outputs of the context precision: in FP64 contexts double-float pairs (for
// the assembly) or FP64 values (fp64_out).  Returns the flags of the pass
// (code FF_ERR_SINGULAR_MOMENT with the point).
DevFlags twoset_shape(ff_ctx* c, const float* Q, long long nq, const long long* ptr,
                      const int* idx, long long n1, void* phi, void* dphi, bool fp64_out) {
  cudaStream_t st = c->stream;
  const int T = 256;
  reset_flags(c);
  ProfScope ps(kProfShape);
  if (c->prec == FF_PREC_FP64 && fp64_out)
    (k_shape_twoset<double><<<ceil_div(nq * 32, T), T, 0, st>>>(
         c->pos.as<float4>(), c->crad.as<double>(), Q, c->qscale, ptr, idx, nq, n1,
         static_cast<double*>(phi), static_cast<double*>(dphi), 1e2, c->flags.as<DevFlags>()),
     ::ff::note_launch());
  else if (!tables_f32(c))
    (k_shape_twoset<dfloat><<<ceil_div(nq * 32, T), T, 0, st>>>(
         c->pos.as<float4>(), c->crad.as<double>(), Q, c->qscale, ptr, idx, nq, n1,
         static_cast<dfloat*>(phi), static_cast<dfloat*>(dphi), 1e2, c->flags.as<DevFlags>()),
     ::ff::note_launch());
  else
    (k_shape_twoset<float><<<ceil_div(nq * 32, T), T, 0, st>>>(
         c->pos.as<float4>(), c->crad.as<double>(), Q, c->qscale, ptr, idx, nq, n1,
         static_cast<float*>(phi), static_cast<float*>(dphi), 1e2, c->flags.as<DevFlags>()),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
  ps.close();
  return read_flags(c);
}

// The transposed covering lists of a two-set cloud: for every centre the
// points it covers (ascending) and its position in each point's row; checked
// against the row lists built before.
void twoset_columns(ff_ctx* c, const float* Xq) {
  cudaStream_t st = c->stream;
  const int T = 256;
  const int K = (int)c->n;
  const long long nq = c->nq, n1 = c->n1;
  const float4* cpos = c->pos.as<float4>();
  const float* lim32 = c->clim32.as<float>();
  const double* lim = c->clim.as<double>();
  int* ccnt = reinterpret_cast<int*>(c->scratch[6].ensure(sizeof(int) * (K + 1)));
  (k_cover_cols<0><<<ceil_div((long long)K * 32, T), T, 0, st>>>(
       Xq, nq, cpos, lim32, lim, K, ccnt, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  long long* tptr = reinterpret_cast<long long*>(c->nbrT_ptr.ensure(sizeof(long long) * (K + 1)));
  scan_counts(ccnt, tptr, K, c, c->scratch[3]);
  long long n1t = 0;
  FF_CUDA(cudaMemcpyAsync(&n1t, tptr + K, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  FF_REQUIRE(n1t == n1, FF_ERR_CUDA, "covering lists disagree between the two passes");
  int* tidx = reinterpret_cast<int*>(c->nbrT_idx.ensure(sizeof(int) * std::max(n1, 1LL)));
  long long* tpos =
      reinterpret_cast<long long*>(c->nbrT_pos.ensure(sizeof(long long) * std::max(n1, 1LL)));
  reset_flags(c);
  (k_cover_cols<1><<<ceil_div((long long)K * 32, T), T, 0, st>>>(
       Xq, nq, cpos, lim32, lim, K, nullptr, tptr, tidx, tpos, c->nbr_ptr.as<long long>(),
       c->nbr_idx.as<int>(), c->flags.as<DevFlags>()),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const DevFlags f = read_flags(c);
  FF_REQUIRE(f.code == 0, FF_ERR_CUDA, "covering lists disagree between the two passes");
  c->has_cols = true;
}

// The grid barrier of the farthest-point sampling with one arrival missing:
// the status the host reads once the bounded wait has run out.
ff_status selftest_device_wait(int device, long long wait_cycles) {
  int coop = 0;
  FF_CUDA(cudaSetDevice(device));
  FF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  FF_REQUIRE(coop, FF_ERR_CUDA, "the device has no cooperative launch");
  unsigned char* mem = nullptr;
  FF_CUDA(cudaMalloc(&mem, 256));
  ff_status out = FF_ERR_CUDA;
  try {
    unsigned* bar = reinterpret_cast<unsigned*>(mem);
    int* abort = reinterpret_cast<int*>(mem + 16);
    DevFlags* flags = reinterpret_cast<DevFlags*>(mem + 64);
    FF_CUDA(cudaMemset(mem, 0, 256));
    long long limit = wait_cycles;
    void* args[] = {&bar, &abort, &flags, &limit};
    FF_CUDA(cudaLaunchCooperativeKernel((const void*)k_wait_check, dim3(sm_count()), dim3(32),
                                        args, 0, nullptr));
    ::ff::note_launch();
    FF_CUDA(cudaDeviceSynchronize());
    DevFlags h{};
    FF_CUDA(cudaMemcpy(&h, flags, sizeof(h), cudaMemcpyDeviceToHost));
    out = h.code == FF_ERR_TIMEOUT ? FF_ERR_TIMEOUT : h.code == 0 ? FF_OK : (ff_status)h.code;
  } catch (...) {
    cudaFree(mem);
    throw;
  }
  cudaFree(mem);
  return out;
}

void build_twoset(ff_ctx* c, const float* Xq, const float* vq, long long nq, int K, double trunc,
                  long long start) {
  cudaStream_t st = c->stream;
  const int T = 256;
  // ---- 1. validation
  int* bad = reinterpret_cast<int*>(c->scratch[0].ensure(64));
  const int imax = INT_MAX;
  FF_CUDA(cudaMemcpyAsync(bad, &imax, sizeof(int), cudaMemcpyHostToDevice, st));
  (k_validate_points<<<(int)std::min<long long>(ceil_div(nq, T), (long long)sm_count() * 8), T, 0, st>>>(Xq, vq, nq,
                                                                                      bad),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  int badi = INT_MAX;
  FF_CUDA(cudaMemcpyAsync(&badi, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  FF_REQUIRE(badi == INT_MAX, FF_ERR_INVALID_ARG,
             "invalid quadrature point " + std::to_string(badi) +
                 ": positions must be finite (|x| < 1e18) and volumes > 0");
  c->n = K;
  c->nq = nq;
  c->twoset = true;
  c->trunc = trunc;

  // ---- 2. farthest-point sampling: on the whole GPU (cooperative launch, one
  // block per SM) when the points are many, else on one thread-block cluster
  const int n = (int)nq;
  long long* chosen = reinterpret_cast<long long*>(c->centre_idx.ensure(sizeof(long long) * K));
  reset_flags(c);
  bool done = false;
  {
    ProfScope ps(kProfFps);
    int coop = 0;
    FF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
    const int G = sm_count();
    if (coop && n >= kFpsGridMin) {
      const int S = (n + G - 1) / G;
      const size_t smem = 24 * (size_t)S;
      const bool in_smem = smem <= (size_t)kFpsSmemMax;
      if (in_smem) set_max_dyn_smem((const void*)k_fps_grid, (int)std::max<size_t>(smem, 16));
      int per_sm = 0;
      FF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fps_grid, kFpsT,
                                                            in_smem ? smem : 0));
      if (per_sm >= 1) {
        float* gxyz = nullptr;
        double* gcur = nullptr;
        float* gcur32 = nullptr;
        if (!in_smem) {
          gxyz = reinterpret_cast<float*>(c->scratch[1].ensure(sizeof(float) * 3 * (size_t)n));
          gcur = reinterpret_cast<double*>(c->scratch[2].ensure(sizeof(double) * (size_t)n));
          gcur32 = reinterpret_cast<float*>(c->scratch[4].ensure(sizeof(float) * (size_t)n));
        }
        // candidates (two buffers of G), then the barrier counter and the abort word
        unsigned char* sync = reinterpret_cast<unsigned char*>(
            c->scratch[7].ensure(2 * sizeof(FpsCand) * G + 64));
        FpsCand* cand = reinterpret_cast<FpsCand*>(sync);
        unsigned* bar = reinterpret_cast<unsigned*>(sync + 2 * sizeof(FpsCand) * G);
        int* abort = reinterpret_cast<int*>(bar + 4);
        FF_CUDA(cudaMemsetAsync(bar, 0, 32, st));
        int nn = n, KK = K, st0 = (int)start, SS = S, ism = in_smem ? 1 : 0;
        DevFlags* fl = c->flags.as<DevFlags>();
        void* args[] = {(void*)&Xq, &nn, &KK, &st0, &SS, &ism, &gxyz, &gcur, &gcur32,
                        &chosen, &cand, &bar, &abort, &fl};
        FF_CUDA(cudaLaunchCooperativeKernel((const void*)k_fps_grid, dim3(G), dim3(kFpsT), args,
                                            in_smem ? smem : 0, st));
        ::ff::note_launch();
        done = true;
      }
    }
    if (!done) {
      const int S = (n + kFpsCS - 1) / kFpsCS;
      const size_t smem = 24 * (size_t)S;
      const bool in_smem = smem <= (size_t)kFpsSmemMax;
      float* gxyz = nullptr;
      double* gcur = nullptr;
      float* gcur32 = nullptr;
      if (in_smem) {
        set_max_dyn_smem((const void*)k_fps, (int)std::max<size_t>(smem, 16));
      } else {
        gxyz = reinterpret_cast<float*>(c->scratch[1].ensure(sizeof(float) * 3 * (size_t)n));
        gcur = reinterpret_cast<double*>(c->scratch[2].ensure(sizeof(double) * (size_t)n));
        gcur32 = reinterpret_cast<float*>(c->scratch[4].ensure(sizeof(float) * (size_t)n));
      }
      (k_fps<<<kFpsCS, kFpsT, in_smem ? smem : 0, st>>>(Xq, n, K, (int)start, S,
                                                        in_smem ? 1 : 0, gxyz, gcur, gcur32,
                                                        chosen, c->flags.as<DevFlags>()),
       ::ff::note_launch());
      FF_LAUNCH_CHECK();
    }
  }
  DevFlags f = read_flags(c);
  FF_REQUIRE(f.code != FF_ERR_TIMEOUT, FF_ERR_TIMEOUT,
             "farthest-point sampling: a grid barrier wait ran out");
  FF_REQUIRE(f.code == 0, FF_ERR_INVALID_ARG,
             "the quadrature points hold fewer than K = " + std::to_string(K) +
                 " distinct positions (farthest-point step " + std::to_string(f.index) + ")");

  // ---- 3. centres and radii
  float4* cpos = reinterpret_cast<float4*>(c->pos.ensure(sizeof(float4) * K));
  (k_gather_centres<<<ceil_div(K, T), T, 0, st>>>(Xq, chosen, K, cpos), ::ff::note_launch());
  double* rad = reinterpret_cast<double*>(c->crad.ensure(sizeof(double) * K));
  double* lim = reinterpret_cast<double*>(c->clim.ensure(sizeof(double) * K));
  float* lim32 = reinterpret_cast<float*>(c->clim32.ensure(sizeof(float) * K));
  reset_flags(c);
  (k_radii<<<ceil_div((long long)K * 32, T), T, 0, st>>>(cpos, K, trunc > 0 ? trunc * trunc : 0.0,
                                                         rad, lim, lim32, c->flags.as<DevFlags>()),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  f = read_flags(c);
  FF_REQUIRE(f.code == 0, FF_ERR_INVALID_ARG,
             "centre " + std::to_string(f.index) + " has a zero radius");
  std::vector<double> hr(K);
  FF_CUDA(cudaMemcpy(hr.data(), rad, sizeof(double) * K, cudaMemcpyDeviceToHost));
  // basis scale of the shape functions (any positive value gives the same
  // functions; the largest radius keeps the moment matrices well scaled)
  c->qscale = (float)*std::max_element(hr.begin(), hr.end());

  // ---- 4. covering lists: rows (point -> centres) and columns (centre -> points)
  ProfScope ps_cover(kProfCover);
  const long long n1 = twoset_cover(c, Xq, nq, c->nbr_ptr, c->nbr_idx, c->scratch[5]);
  c->n1 = n1;
  ps_cover.close();

  // ---- 5. quadrature volumes, identity order of the centres
  float* vol = reinterpret_cast<float*>(c->vol.ensure(sizeof(float) * nq));
  (k_copy_f32<<<ceil_div(nq, T), T, 0, st>>>(vq, vol, nq), ::ff::note_launch());
  float* qpts = reinterpret_cast<float*>(c->qpts.ensure(sizeof(float) * 3 * nq));
  (k_copy_f32<<<ceil_div(3 * nq, T), T, 0, st>>>(Xq, qpts, 3 * nq), ::ff::note_launch());
  // the transposed lists (centre -> the points it covers) serve the row-owner
  // assembly, which runs when K is too large for the dense tiles of the
  // two-set assembly, and the matrix-free operator (built on demand there)
  c->has_cols = false;
  if (!tset_assembly_fits(K)) twoset_columns(c, qpts);
  int* perm = reinterpret_cast<int*>(c->perm.ensure(sizeof(int) * K));
  int* iperm = reinterpret_cast<int*>(c->iperm.ensure(sizeof(int) * K));
  (k_iota<<<ceil_div(K, T), T, 0, st>>>(perm, iperm, K), ::ff::note_launch());
  FF_LAUNCH_CHECK();

  // ---- 6. shape functions at the quadrature points
  const size_t es = tables_f32(c) ? 4 : 8;
  c->phi.ensure(es * std::max(n1, 1LL));
  c->dphi.ensure(3 * es * std::max(n1, 1LL));
  f = twoset_shape(c, Xq, nq, c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), n1, c->phi.p,
                   c->dphi.p, false);
  c->hflags->fallback = f.fallback;
  if (f.code == FF_ERR_SINGULAR_MOMENT)
    throw Error(FF_ERR_SINGULAR_MOMENT,
                "moment matrix of quadrature point " + std::to_string(f.index) +
                    " is singular: fewer than four non-coplanar centres cover it");
}

}  // namespace ff
