// Grid-hash support-neighbour search (nodal RKPM discretisation).
//
// Node k covers the point X iff ||X - p_k||^2 < a_k^2, where the squared
// distance is ((dx*dx + dy*dy) + dz*dz) in FP64 on the FP32-stored inputs with
// no fused multiply-add (Supp. Sec. B "RKPM construction": the kernel support
// decides which nodes enter the moment sum of Sec. 3.2, Eqs. 9-10).  An FP32
// evaluation with a relative margin of 1e-5 settles every pair whose distance
// is not within rounding of the radius; only those are re-tested in FP64, which
// keeps the lists bit-identical to the FP64 rule.
//
// Pipeline (all on the context stream):
//   1. validate inputs, bounding box, largest radius           (1 readback)
//   2. cell keys: 4x4x4-cell bricks in x-y-z order, Morton order inside a
//      brick; counting sort of particles by key, each cell ordered by caller
//      index (deterministic)                          -> perm, pos, vol
//   3. scatter search: every node k scans the cells within ceil(1.001 a_k / h)
//      rings of its own cell, counting the points it covers   -> row counts
//   4. scan, fill (atomic cursor per row), sort each row ascending
//   5. transpose lists (node k -> rows i it covers, with the position of k in row i)
#include "ff_internal.cuh"
#include "grid.cuh"

namespace ff {
namespace {

__device__ __forceinline__ unsigned int f2ord(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// red: [0..2] min xyz (ordered uint), [3..5] max xyz, [6] max a; bad: first invalid index
__global__ void k_validate_bbox(const float* __restrict__ X, const float* __restrict__ v,
                                const float* __restrict__ a, long long n,
                                unsigned int* __restrict__ red, int* __restrict__ bad) {
  unsigned int mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0, 0, 0}, ma = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2], ai = a[i], vi = v[i];
    bool ok = isfinite(x) && isfinite(y) && isfinite(z) && fabsf(x) < 1e18f && fabsf(y) < 1e18f &&
              fabsf(z) < 1e18f && isfinite(ai) && ai > 1e-18f && ai < 1e18f && isfinite(vi) &&
              vi > 0.f;
    if (!ok) {
      atomicMin(bad, (int)i);
      continue;
    }
    float c[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      unsigned int u = f2ord(c[d]);
      mn[d] = min(mn[d], u);
      mx[d] = max(mx[d], u);
    }
    ma = max(ma, f2ord(ai));
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o; o >>= 1) {
      mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  for (int o = 16; o; o >>= 1) ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  if ((threadIdx.x & 31) == 0) {
    for (int d = 0; d < 3; ++d) {
      atomicMin(&red[d], mn[d]);
      atomicMax(&red[3 + d], mx[d]);
    }
    atomicMax(&red[6], ma);
  }
}

__global__ void k_init_red(unsigned int* red, int* bad) {
  for (int d = 0; d < 3; ++d) {
    red[d] = 0xffffffffu;
    red[3 + d] = 0u;
  }
  red[6] = 0u;
  *bad = 0x7fffffff;
}

__global__ void k_decode_red(const unsigned int* red, float* out) {
  for (int d = 0; d < 7; ++d) out[d] = ord2f(red[d]);
}

__global__ void k_keys(const float* __restrict__ X, long long n, GridDev g,
                       int* __restrict__ key, int* __restrict__ cnt) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = cell_coord(X[3 * i], g.o0, g.h, g.d0);
  int cy = cell_coord(X[3 * i + 1], g.o1, g.h, g.d1);
  int cz = cell_coord(X[3 * i + 2], g.o2, g.h, g.d2);
  int k = (int)cell_key(g, cx, cy, cz);
  key[i] = k;
  atomicAdd(&cnt[k], 1);
}

__global__ void k_scatter(const int* __restrict__ key, long long n, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ tmp) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int k = key[i];
  int p = start[k] + atomicAdd(&fill[k], 1);
  tmp[p] = (int)i;
}

// one warp per cell: order the cell's particles by caller index (rank counting)
__global__ void k_order_cells(const int* __restrict__ start, long long ncells,
                              const int* __restrict__ tmp, int* __restrict__ perm) {
  long long cell = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (cell >= ncells) return;
  int s = start[cell], e = start[cell + 1];
  for (int a = s + lane; a < e; a += 32) {
    int va = tmp[a];
    int r = 0;
    for (int b = s; b < e; ++b) r += tmp[b] < va;
    perm[s + r] = va;
  }
}

__global__ void k_gather_particles(const int* __restrict__ perm, long long n,
                                   const float* __restrict__ X, const float* __restrict__ v,
                                   const float* __restrict__ a, float4* __restrict__ pos,
                                   float* __restrict__ vol, int* __restrict__ iperm) {
  long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int i = perm[j];
  pos[j] = make_float4(X[3LL * i], X[3LL * i + 1], X[3LL * i + 2], a[i]);
  vol[j] = v[i];
  iperm[i] = (int)j;
}

// MODE 0: count per row (atomic); MODE 1: fill rows through an atomic cursor
template <int MODE>
__global__ void k_search(const float4* __restrict__ pos, long long n, GridDev g,
                         const int* __restrict__ cstart, int* __restrict__ cnt,
                         const long long* __restrict__ rptr, int* __restrict__ ridx) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float4 p = pos[k];
  int cx = cell_coord(p.x, g.o0, g.h, g.d0);
  int cy = cell_coord(p.y, g.o1, g.h, g.d1);
  int cz = cell_coord(p.z, g.o2, g.h, g.d2);
  int R = (int)ceil(1.001 * (double)p.w / g.h);
  for (int z = max(cz - R, 0); z <= min(cz + R, g.d2 - 1); ++z)
    for (int y = max(cy - R, 0); y <= min(cy + R, g.d1 - 1); ++y)
      for (int x = max(cx - R, 0); x <= min(cx + R, g.d0 - 1); ++x) {
        long long key = cell_key(g, x, y, z);
        int s = cstart[key], e = cstart[key + 1];
        for (int i = s; i < e; ++i) {
          if (covers(pos[i], p)) {
            if (MODE == 0) {
              atomicAdd(&cnt[i], 1);
            } else {
              long long slot = rptr[i] + atomicAdd(&cnt[i], 1);
              ridx[slot] = (int)k;
            }
          }
        }
      }
}

// one warp per row: sort the row ascending in place (rank counting, values unique)
__global__ void k_sort_rows(const long long* __restrict__ ptr, long long n, int* __restrict__ idx,
                            int* __restrict__ tmp) {
  long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  long long s = ptr[row], e = ptr[row + 1];
  for (long long a = s + lane; a < e; a += 32) tmp[a] = idx[a];
  __syncwarp();
  for (long long a = s + lane; a < e; a += 32) {
    int va = tmp[a];
    int r = 0;
    for (long long b = s; b < e; ++b) r += tmp[b] < va;
    idx[s + r] = va;
  }
}

__global__ void k_col_count(const int* __restrict__ idx, long long n1, int* __restrict__ cnt) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n1) atomicAdd(&cnt[idx[e]], 1);
}

__global__ void k_transpose_fill(const long long* __restrict__ ptr, const int* __restrict__ idx,
                                 long long n, const long long* __restrict__ tptr,
                                 int* __restrict__ cur, int* __restrict__ tidx,
                                 long long* __restrict__ tpos) {
  long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  for (long long e = ptr[row] + lane; e < ptr[row + 1]; e += 32) {
    int k = idx[e];
    long long slot = tptr[k] + atomicAdd(&cur[k], 1);
    tidx[slot] = (int)row;
    tpos[slot] = e;
  }
}

// one warp per node: order the transposed list by row index (rows are unique)
__global__ void k_sort_transposed(const long long* __restrict__ tptr, long long n,
                                  int* __restrict__ tidx, long long* __restrict__ tpos,
                                  int* __restrict__ tmpi, long long* __restrict__ tmpp) {
  long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (k >= n) return;
  long long s = tptr[k], e = tptr[k + 1];
  for (long long a = s + lane; a < e; a += 32) {
    tmpi[a] = tidx[a];
    tmpp[a] = tpos[a];
  }
  __syncwarp();
  for (long long a = s + lane; a < e; a += 32) {
    int va = tmpi[a];
    int r = 0;
    for (long long b = s; b < e; ++b) r += tmpi[b] < va;
    tidx[s + r] = va;
    tpos[s + r] = tmpp[a];
  }
}

}  // namespace

void build_neighbours(ff_ctx* c, const float* X, const float* v, const float* a, int64_t n) {
  cudaStream_t st = c->stream;
  const int T = 256;
  // ---- 1. validation, bounding box, largest radius
  Buf& redb = c->scratch[0];
  redb.ensure(64);
  unsigned int* red = redb.as<unsigned int>();
  int* bad = reinterpret_cast<int*>(red + 8);
  float* dec = reinterpret_cast<float*>(red + 9);
  (k_init_red<<<1, 1, 0, st>>>(red, bad), ::ff::note_launch());
  int blocks = (int)std::min<long long>(ceil_div(n, T), (long long)sm_count() * 8);
  (k_validate_bbox<<<blocks, T, 0, st>>>(X, v, a, n, red, bad), ::ff::note_launch());
  (k_decode_red<<<1, 1, 0, st>>>(red, dec), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  struct {
    unsigned int r[9];
    float d[7];
  } h{};
  FF_CUDA(cudaMemcpyAsync(&h, red, sizeof(h), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  int badi = (int)h.r[8];
  FF_REQUIRE(badi == 0x7fffffff, FF_ERR_INVALID_ARG,
             "invalid particle " + std::to_string(badi) +
                 ": positions must be finite, volumes > 0 and support radii > 0");
  double lo[3] = {h.d[0], h.d[1], h.d[2]}, hi[3] = {h.d[3], h.d[4], h.d[5]};
  double amax = h.d[6];
  // cell edge >= 1.001 * largest radius: one ring of cells covers every support;
  // grow it if the box would need more than ~8 cells per particle
  double cell = 1.001 * amax;
  Grid& g = c->grid;
  for (int it = 0; it < 64; ++it) {
    long long tot = 1;
    for (int d = 0; d < 3; ++d) {
      g.dims[d] = (int)std::min<double>(floor((hi[d] - lo[d]) / cell) + 1.0, 1 << 20);
      g.bdims[d] = (g.dims[d] + 3) / 4;
      tot *= g.bdims[d];
    }
    g.ncells = tot * 64;
    if (g.ncells <= std::max<long long>(8 * n, 4096) && g.ncells < (1LL << 30)) break;
    cell *= 1.25;
  }
  for (int d = 0; d < 3; ++d) g.origin[d] = lo[d];
  g.h = cell;
  GridDev gd{g.origin[0], g.origin[1], g.origin[2], g.h, g.dims[0], g.dims[1], g.dims[2],
             g.bdims[0], g.bdims[1], g.bdims[2]};

  // ---- 2. counting sort by cell key
  long long K = g.ncells;
  int* key = reinterpret_cast<int*>(c->scratch[1].ensure(sizeof(int) * n));
  int* cnt = reinterpret_cast<int*>(c->scratch[2].ensure(sizeof(int) * (K + 1)));
  int* cstart = reinterpret_cast<int*>(c->cell_start.ensure(sizeof(int) * (K + 1)));
  FF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (K + 1), st));
  (k_keys<<<ceil_div(n, T), T, 0, st>>>(X, n, gd, key, cnt), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  scan_counts_i32(cnt, cstart, K, c, c->scratch[3]);
  FF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (K + 1), st));
  int* tmp = reinterpret_cast<int*>(c->scratch[4].ensure(sizeof(int) * n));
  (k_scatter<<<ceil_div(n, T), T, 0, st>>>(key, n, cstart, cnt, tmp), ::ff::note_launch());
  int* perm = reinterpret_cast<int*>(c->perm.ensure(sizeof(int) * n));
  (k_order_cells<<<ceil_div(K * 32, T), T, 0, st>>>(cstart, K, tmp, perm), ::ff::note_launch());
  float4* pos = reinterpret_cast<float4*>(c->pos.ensure(sizeof(float4) * n));
  float* vol = reinterpret_cast<float*>(c->vol.ensure(sizeof(float) * n));
  int* iperm = reinterpret_cast<int*>(c->iperm.ensure(sizeof(int) * n));
  (k_gather_particles<<<ceil_div(n, T), T, 0, st>>>(perm, n, X, v, a, pos, vol, iperm), ::ff::note_launch());
  FF_LAUNCH_CHECK();

  // ---- 3-4. scatter search: count, scan, fill, sort rows
  int* rcnt = reinterpret_cast<int*>(c->scratch[5].ensure(sizeof(int) * (n + 1)));
  FF_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int) * (n + 1), st));
  (k_search<0><<<ceil_div(n, 128), 128, 0, st>>>(pos, n, gd, cstart, rcnt, nullptr, nullptr), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  long long* rptr = reinterpret_cast<long long*>(c->nbr_ptr.ensure(sizeof(long long) * (n + 1)));
  scan_counts(rcnt, rptr, n, c, c->scratch[3]);
  long long n1 = 0;
  FF_CUDA(cudaMemcpyAsync(&n1, rptr + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  c->n1 = n1;
  int* ridx = reinterpret_cast<int*>(c->nbr_idx.ensure(sizeof(int) * n1));
  FF_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int) * (n + 1), st));
  (k_search<1><<<ceil_div(n, 128), 128, 0, st>>>(pos, n, gd, cstart, rcnt, rptr, ridx), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  int* rtmp = reinterpret_cast<int*>(c->scratch[6].ensure(sizeof(int) * n1));
  (k_sort_rows<<<ceil_div(n * 32, T), T, 0, st>>>(rptr, n, ridx, rtmp), ::ff::note_launch());
  FF_LAUNCH_CHECK();

  // ---- 5. transpose
  FF_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int) * (n + 1), st));
  (k_col_count<<<ceil_div(n1, T), T, 0, st>>>(ridx, n1, rcnt), ::ff::note_launch());
  long long* tptr = reinterpret_cast<long long*>(c->nbrT_ptr.ensure(sizeof(long long) * (n + 1)));
  scan_counts(rcnt, tptr, n, c, c->scratch[3]);
  FF_CUDA(cudaMemsetAsync(rcnt, 0, sizeof(int) * (n + 1), st));
  int* tidx = reinterpret_cast<int*>(c->nbrT_idx.ensure(sizeof(int) * n1));
  long long* tpos = reinterpret_cast<long long*>(c->nbrT_pos.ensure(sizeof(long long) * n1));
  (k_transpose_fill<<<ceil_div(n * 32, T), T, 0, st>>>(rptr, ridx, n, tptr, rcnt, tidx, tpos), ::ff::note_launch());
  long long* ptmp = reinterpret_cast<long long*>(c->scratch[7].ensure(sizeof(long long) * n1));
  (k_sort_transposed<<<ceil_div(n * 32, T), T, 0, st>>>(tptr, n, tidx, tpos, rtmp, ptmp), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  c->has_cols = true;
}

}  // namespace ff
