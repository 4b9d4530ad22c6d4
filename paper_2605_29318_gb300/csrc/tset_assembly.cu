// Assembly of H_w (Prop. 1) and M (Sec. 3.2, Eq. 14) for the two-set
// discretisation in dense tiles.
//
//   (H_w)_kl = sum_i v_i (lambda_i + 4 mu_i) grad phi_k(X_i) . grad phi_l(X_i)
//   M_kl     = sum_i v_i phi_k(X_i) phi_l(X_i)
//
// With K centres and n quadrature points each covered by c_i centres, the sums
// hold sum_i c_i^2 pair products (6e9 for a million points at ~80 centres
// each): a dense contraction once the points are grouped.  The points are
// grouped by their nearest covering centre (a counting sort over the K
// centres), and cut into tiles of TP consecutive points of that order (TP = 16,
// 24 or 32: smaller tiles let two blocks share an SM).
// A tile's points are close together, so the union U of their covering centres
// is small (~1.5 c_i).  One thread block per tile:
//   1. the union as a bitmap over the centres and its popcount ranks;
//   2. for every pair of 64-column blocks of the union, rows from block
//      A = bj and columns from block B = bi <= bj: the tile's weighted
//      gradients and shape functions of A and the plain ones of B staged
//      densely in shared memory (zeros where a point does not see a centre),
//      then the 64 x 64 block of sum_t (w_t g_A(t)) g_B(t)^T and
//      sum_t (v_t phi_A(t)) phi_B(t)^T in register tiles (4 x 4 per thread,
//      rows 4 tr + r, columns 4 tc + c: one vector read of each of A
//      (broadcast) and B (conflict-free) per point and value).  The last
//      block of the union is usually narrow; it always falls on the row side,
//      where the warps whose rows lie past the union skip the products;
//   3. each non-zero entry of the upper triangle added into dense K x K FP64
//      accumulators (atomic adds).
// The sums inside a tile run in the context's working precision (double-float
// in FP64 contexts, about 2^-47 relative; FP32 otherwise); across tiles they
// are FP64.  The order of the FP64 additions follows the atomics' arrival, so
// the matrices are reproducible to FP64 rounding (not bit for bit).
// A second pass turns the accumulators into the CSR layout of the nodal path
// (ascending columns; an entry is stored where H_w or M is non-zero), with the
// diagonal of H_w set to minus the sum of its row's off-diagonal entries.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "ff_internal.cuh"
#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kTilePtsDefault = 24;  // quadrature points per tile
constexpr int kBlk = 64;       // union columns per register block
constexpr int kThreads = 256;  // 16 x 16 threads, 4 x 4 entries each

// the nearest covering centre of every point (ties: the lower index) and the
// points per centre
__global__ void k_home(const float* __restrict__ Xq, long long nq, const long long* __restrict__ ptr,
                       const int* __restrict__ idx, const float4* __restrict__ cpos,
                       int* __restrict__ home, int* __restrict__ cnt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const float x = Xq[3 * i], y = Xq[3 * i + 1], z = Xq[3 * i + 2];
  float best = INFINITY;
  int h = 0;
  for (long long e = ptr[i]; e < ptr[i + 1]; ++e) {
    const int k = idx[e];
    const float4 p = cpos[k];
    const float dx = x - p.x, dy = y - p.y, dz = z - p.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (d2 < best) {  // ascending k: the first minimum is the lowest index
      best = d2;
      h = k;
    }
  }
  home[i] = h;
  atomicAdd(&cnt[h], 1);
}

__global__ void k_home_scatter(const int* __restrict__ home, long long nq,
                               const long long* __restrict__ start, int* __restrict__ cursor,
                               int* __restrict__ order) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int h = home[i];
  order[start[h] + atomicAdd(&cursor[h], 1)] = (int)i;
}

// rank of centre c in the tile's union (bitmap words and their exclusive
// popcount prefix)
__device__ __forceinline__ int union_rank(const unsigned* bits, const int* wpre, int c) {
  const int w = c >> 5;
  return wpre[w] + __popc(bits[w] & ((1u << (c & 31)) - 1u));
}

// four consecutive values of a staging row (16-byte aligned)
__device__ __forceinline__ void load4(const float* p, float (&x)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  x[0] = q.x;
  x[1] = q.y;
  x[2] = q.z;
  x[3] = q.w;
}
__device__ __forceinline__ void load4(const dfloat* p, dfloat (&x)[4]) {
  const float4 q0 = *reinterpret_cast<const float4*>(p);
  const float4 q1 = *reinterpret_cast<const float4*>(p + 2);
  x[0] = dfloat(q0.x, q0.y);
  x[1] = dfloat(q0.z, q0.w);
  x[2] = dfloat(q1.x, q1.y);
  x[3] = dfloat(q1.z, q1.w);
}

// The tile's points (order[p0 ..]) and the union of their covering centres:
// the bitmap `bits` over the centres, the exclusive popcount prefix of its
// words `wpre` and the union's centres `ucol` in ascending order.  Returns the
// union's size.
template <int TP>
__device__ int tile_union(const int* __restrict__ order, long long nq,
                          const long long* __restrict__ ptr, const int* __restrict__ idx, int nw,
                          int* pts, unsigned* bits, int* wpre, int* ucol, int* s_total, int& np) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long p0 = (long long)blockIdx.x * TP;
  np = (int)min((long long)TP, nq - p0);
  if (tid < TP) pts[tid] = tid < np ? order[p0 + tid] : -1;
  for (int w = tid; w < nw; w += kThreads) bits[w] = 0u;
  __syncthreads();
  for (int j = wid; j < np; j += kThreads / 32) {
    const int i = pts[j];
    for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
      const int c = idx[e];
      atomicOr(&bits[c >> 5], 1u << (c & 31));
    }
  }
  __syncthreads();
  if (wid == 0) {  // exclusive prefix of the words' popcounts
    int run = 0;
    for (int w0 = 0; w0 < nw; w0 += 32) {
      const int w = w0 + lane;
      const int v = w < nw ? __popc(bits[w]) : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (w < nw) wpre[w] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      wpre[nw] = run;
      *s_total = run;
    }
  }
  __syncthreads();
  for (int w = tid; w < nw; w += kThreads) {
    unsigned b = bits[w];
    int r = wpre[w];
    while (b) {
      const int q = __ffs(b) - 1;
      ucol[r++] = (w << 5) + q;
      b &= b - 1u;
    }
  }
  __syncthreads();
  return *s_total;
}

// The upper triangle of one 64 x 64 block's non-zero entries into the dense
// FP64 accumulators.
template <class T>
__device__ __forceinline__ void add_block(const T (&h)[4][4], const T (&m)[4][4], bool live,
                                          int a0, int b0, int tr, int tc, int U, const int* ucol,
                                          int K, double* __restrict__ Hd,
                                          double* __restrict__ Md) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int ur = a0 + 4 * tr + r, uc = b0 + 4 * tc + c;
      if (!live || ur >= U || uc >= U || ur < uc) continue;
      const double hv = (double)finish(h[r][c]), mv = (double)finish(m[r][c]);
      if (hv == 0.0 && mv == 0.0) continue;
      const long long at = (long long)ucol[uc] * K + ucol[ur];  // upper triangle
      atomicAdd(&Hd[at], hv);
      atomicAdd(&Md[at], mv);
    }
}

// Every pair of 64-column blocks of the union, each staged on its own: the
// weighted values of block A = bj and the plain ones of block B = bi <= bj in
// sA[4][TP][kBlk] and sB[4][TP][kBlk] (zeros where a point does not see a
// centre), then the block's products and its entries.
template <class T, int TP>
__device__ void tile_pairs(const int* pts, int np, int U, const unsigned* bits, const int* wpre,
                           const int* ucol, const long long* __restrict__ ptr,
                           const int* __restrict__ idx, const T* __restrict__ phi,
                           const T* __restrict__ dphi, long long n1, const T* __restrict__ wh,
                           const float* __restrict__ vol, int K, double* __restrict__ Hd,
                           double* __restrict__ Md, T* sA, T* sB) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tr = tid >> 4, tc = tid & 15;
  const int nblk = (U + kBlk - 1) / kBlk;
  constexpr int kPlane = TP * kBlk;  // one value plane of a staging array
  for (int bi = 0; bi < nblk; ++bi)
    for (int bj = bi; bj < nblk; ++bj) {
      const int a0 = bj * kBlk, b0 = bi * kBlk;  // rows: block bj, columns: block bi
      const bool live = 4 * tr < U - a0;         // the thread has a row in the union
      for (int q = tid; q < 4 * kPlane; q += kThreads) {
        sA[q] = T(0);
        sB[q] = T(0);
      }
      __syncthreads();
      for (int j = wid; j < np; j += kThreads / 32) {
        const int i = pts[j];
        const T w = wh[i];
        const T v = T(vol[i]);
        for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
          const int r = union_rank(bits, wpre, idx[e]);
          const bool inA = r >= a0 && r < a0 + kBlk, inB = r >= b0 && r < b0 + kBlk;
          if (!inA && !inB) continue;
          const T g0 = dphi[e], g1 = dphi[n1 + e], g2 = dphi[2 * n1 + e], f = phi[e];
          if (inA) {
            const int o = j * kBlk + (r - a0);
            sA[o] = w * g0;
            sA[kPlane + o] = w * g1;
            sA[2 * kPlane + o] = w * g2;
            sA[3 * kPlane + o] = v * f;
          }
          if (inB) {
            const int o = j * kBlk + (r - b0);
            sB[o] = g0;
            sB[kPlane + o] = g1;
            sB[2 * kPlane + o] = g2;
            sB[3 * kPlane + o] = f;
          }
        }
      }
      __syncthreads();
      T h[4][4], m[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          h[r][c] = T(0);
          m[r][c] = T(0);
        }
      for (int j = 0; j < (live ? np : 0); ++j) {
#pragma unroll
        for (int val = 0; val < 4; ++val) {
          T a[4], b[4];
          load4(sA + val * kPlane + j * kBlk + 4 * tr, a);
          load4(sB + val * kPlane + j * kBlk + 4 * tc, b);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              if (val < 3)
                mac(h[r][c], a[r], b[c]);
              else
                mac(m[r][c], a[r], b[c]);
            }
        }
      }
      add_block(h, m, live, a0, b0, tr, tc, U, ucol, K, Hd, Md);
      __syncthreads();  // the staging arrays are refilled next
    }
}

// One block per tile.  Shared memory (dynamic): bitmap (nw words), word
// prefix (nw + 1), union columns (K), then the staging arrays
// sA[4][TP][kBlk] and sB[4][TP][kBlk] of T.
template <class T, int TP>
__global__ void __launch_bounds__(kThreads, TP == 32 ? 1 : 2)
    k_tset_tiles(const int* __restrict__ order, long long nq, const long long* __restrict__ ptr,
                 const int* __restrict__ idx, const T* __restrict__ phi,
                 const T* __restrict__ dphi, long long n1, const T* __restrict__ wh,
                 const float* __restrict__ vol, int K, double* __restrict__ Hd,
                 double* __restrict__ Md) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nw = (K + 31) >> 5;
  unsigned* bits = reinterpret_cast<unsigned*>(sm_raw);
  int* wpre = reinterpret_cast<int*>(bits + nw);
  int* ucol = wpre + nw + 1;
  size_t off = (size_t)(2 * nw + 1 + K) * 4;
  off = (off + 15) & ~size_t(15);
  T* sA = reinterpret_cast<T*>(sm_raw + off);
  T* sB = sA + 4 * TP * kBlk;
  __shared__ int pts[TP];
  __shared__ int s_total;
  int np = 0;
  const int U = tile_union<TP>(order, nq, ptr, idx, nw, pts, bits, wpre, ucol, &s_total, np);
  tile_pairs<T, TP>(pts, np, U, bits, wpre, ucol, ptr, idx, phi, dphi, n1, wh, vol, K, Hd, Md, sA,
                    sB);
}

// FP32 sums: the tile's plain values over the whole union staged once,
// G[4][TP][Up] (Up = the union rounded up to 64, at most kStageCols), with
// the points' weights beside them; every pair of 64-column blocks then reads
// the same read-only staging (the weight applied to the row block's values
// as they are read, the same rounding as a weighted copy), so the pairs need
// no barrier between them.  A tile whose union exceeds kStageCols takes the
// per-pair staging.
constexpr int kStageCols = 256;
template <int TP>
__global__ void __launch_bounds__(kThreads, TP == 16 ? 3 : 2)
    k_tset_tiles_once(const int* __restrict__ order, long long nq,
                      const long long* __restrict__ ptr, const int* __restrict__ idx,
                      const float* __restrict__ phi, const float* __restrict__ dphi, long long n1,
                      const float* __restrict__ wh, const float* __restrict__ vol, int K,
                      double* __restrict__ Hd, double* __restrict__ Md) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nw = (K + 31) >> 5;
  unsigned* bits = reinterpret_cast<unsigned*>(sm_raw);
  int* wpre = reinterpret_cast<int*>(bits + nw);
  int* ucol = wpre + nw + 1;
  size_t off = (size_t)(2 * nw + 1 + K) * 4;
  off = (off + 15) & ~size_t(15);
  float* G = reinterpret_cast<float*>(sm_raw + off);
  __shared__ int pts[TP];
  __shared__ int s_total;
  __shared__ float wj[TP], vj[TP];
  int np = 0;
  const int U = tile_union<TP>(order, nq, ptr, idx, nw, pts, bits, wpre, ucol, &s_total, np);
  if (U > kStageCols) {
    tile_pairs<float, TP>(pts, np, U, bits, wpre, ucol, ptr, idx, phi, dphi, n1, wh, vol, K, Hd,
                          Md, G, G + 4 * TP * kBlk);
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nblk = (U + kBlk - 1) / kBlk;
  const int Up = nblk * kBlk;
  const int plane = TP * Up;
  for (int q = tid; q < 4 * plane; q += kThreads) G[q] = 0.f;
  __syncthreads();
  for (int j = wid; j < np; j += kThreads / 32) {
    const int i = pts[j];
    if (lane == 0) {
      wj[j] = wh[i];
      vj[j] = vol[i];
    }
    for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
      const int o = j * Up + union_rank(bits, wpre, idx[e]);
      G[o] = dphi[e];
      G[plane + o] = dphi[n1 + e];
      G[2 * plane + o] = dphi[2 * n1 + e];
      G[3 * plane + o] = phi[e];
    }
  }
  __syncthreads();
  const int tr = tid >> 4, tc = tid & 15;
  for (int bi = 0; bi < nblk; ++bi)
    for (int bj = bi; bj < nblk; ++bj) {
      const int a0 = bj * kBlk, b0 = bi * kBlk;
      const bool live = 4 * tr < U - a0;
      float h[4][4], m[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          h[r][c] = 0.f;
          m[r][c] = 0.f;
        }
      for (int j = 0; j < (live ? np : 0); ++j) {
        const float wt = wj[j], vt = vj[j];
#pragma unroll
        for (int val = 0; val < 4; ++val) {
          float a[4], b[4];
          load4(G + val * plane + j * Up + a0 + 4 * tr, a);
          load4(G + val * plane + j * Up + b0 + 4 * tc, b);
          const float s = val < 3 ? wt : vt;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float ar = s * a[r];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              if (val < 3)
                h[r][c] = fmaf(ar, b[c], h[r][c]);
              else
                m[r][c] = fmaf(ar, b[c], m[r][c]);
            }
          }
        }
      }
      add_block(h, m, live, a0, b0, tr, tc, U, ucol, K, Hd, Md);
    }
}

__device__ __forceinline__ bool stored(const double* Hd, const double* Md, long long at) {
  return Hd[at] != 0.0 || Md[at] != 0.0;
}

// row k of the symmetric matrices from the upper-triangle accumulators
__device__ __forceinline__ long long at_sym(int k, int l, int K) {
  return k <= l ? (long long)k * K + l : (long long)l * K + k;
}

// entries per row (the diagonal always)
__global__ void k_dense_count(const double* __restrict__ Hd, const double* __restrict__ Md, int K,
                              int* __restrict__ cnt) {
  const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (k >= K) return;
  const int lane = threadIdx.x & 31;
  int c = 0;
  for (int l = lane; l < K; l += 32) c += (l == k) || stored(Hd, Md, at_sym(k, l, K));
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) cnt[k] = c;
}

// CSR rows with ascending columns; diagonal of H_w = -(sum of the row's
// off-diagonal entries), summed in a fixed order
template <class TO>
__global__ void k_dense_fill(const double* __restrict__ Hd, const double* __restrict__ Md, int K,
                             const long long* __restrict__ aptr, int* __restrict__ acol,
                             TO* __restrict__ aval, float* __restrict__ hf32,
                             float* __restrict__ hdiag) {
  const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (k >= K) return;
  const int lane = threadIdx.x & 31;
  double off = 0.0;
  for (int l = lane; l < K; l += 32)
    if (l != k) off += (double)(TO)Hd[at_sym(k, l, K)];
#pragma unroll
  for (int o = 16; o; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
  long long pos = aptr[k];
  for (int l0 = 0; l0 < K; l0 += 32) {
    const int l = l0 + lane;
    const bool has = l < K && (l == k || stored(Hd, Md, at_sym(k, l, K)));
    const unsigned bal = __ballot_sync(0xffffffffu, has);
    if (has) {
      const long long e = pos + __popc(bal & ((1u << lane) - 1u));
      const long long at = at_sym(k, l, K);
      const TO hv = l == k ? (TO)(-off) : (TO)Hd[at];
      acol[e] = l;
      aval[2 * e] = hv;
      aval[2 * e + 1] = (TO)Md[at];
      hf32[e] = (float)hv;
      if (l == k) hdiag[k] = (float)hv;
    }
    pos += __popc(bal);
  }
}

template <class T>
size_t tile_smem(int K, int tp) {
  const int nw = (K + 31) >> 5;
  size_t off = (size_t)(2 * nw + 1 + K) * 4;
  off = (off + 15) & ~size_t(15);
  // FP32: the whole-union staging (which also holds the per-pair arrays)
  const size_t stage = std::is_same_v<T, float> ? 4 * (size_t)tp * kStageCols
                                                : 2 * 4 * (size_t)tp * kBlk;
  return off + stage * sizeof(T);
}

// points per tile: FF_TSET_TILE = 16, 24 or 32 (for measurements), else the default
int tile_points() {
  static const int tp = [] {
    const char* e = std::getenv("FF_TSET_TILE");
    const int v = e ? std::atoi(e) : 0;
    return (v == 16 || v == 24 || v == 32) ? v : kTilePtsDefault;
  }();
  return tp;
}

template <class T, int TP>
void launch_tiles(ff_ctx* c, const int* order, int K, double* Hd, double* Md) {
  const long long nq = c->nq;
  const size_t smem = tile_smem<T>(K, TP);
  const unsigned tiles = (unsigned)((nq + TP - 1) / TP);
  if constexpr (std::is_same_v<T, float>) {
    set_max_dyn_smem((const void*)k_tset_tiles_once<TP>, (int)smem);
    (k_tset_tiles_once<TP><<<tiles, kThreads, smem, c->stream>>>(
         order, nq, c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->phi.as<float>(),
         c->dphi.as<float>(), c->n1, c->wh.as<float>(), c->vol.as<float>(), K, Hd, Md),
     ::ff::note_launch());
  } else {
    set_max_dyn_smem((const void*)k_tset_tiles<T, TP>, (int)smem);
    (k_tset_tiles<T, TP><<<tiles, kThreads, smem, c->stream>>>(
         order, nq, c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->phi.as<T>(),
         c->dphi.as<T>(), c->n1, c->wh.as<T>(), c->vol.as<float>(), K, Hd, Md),
     ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
}

template <class T>
void launch_tiles(ff_ctx* c, const int* order, int K, double* Hd, double* Md) {
  switch (tile_points()) {
    case 16: launch_tiles<T, 16>(c, order, K, Hd, Md); break;
    case 32: launch_tiles<T, 32>(c, order, K, Hd, Md); break;
    default: launch_tiles<T, 24>(c, order, K, Hd, Md); break;
  }
}

}  // namespace

bool tset_assembly_fits(long long K) { return K >= 1 && K <= kTsetMaxCentres; }

// H_w and M of a two-set cloud (c->wh holds the material weights).  Leaves
// a_ptr, a_col, a_val, h_f32, hdiag_f32 and c->n2 as the row-owner assembly does.
void tset_assemble(ff_ctx* c) {
  cudaStream_t st = c->stream;
  const long long nq = c->nq, n1 = c->n1;
  const int K = (int)c->n;
  const bool f64 = c->prec == FF_PREC_FP64;
  const bool tdf = !tables_f32(c);  // double-float tables and tile sums
  const int TB = 256;
  // ---- grouping by the nearest covering centre
  int* home = reinterpret_cast<int*>(c->scratch[5].ensure(sizeof(int) * (nq + 1)));
  int* order = reinterpret_cast<int*>(c->scratch[6].ensure(sizeof(int) * (nq + 1)));
  int* cnt = reinterpret_cast<int*>(c->scratch[7].ensure(sizeof(int) * 2 * (K + 1)));
  int* cursor = cnt + (K + 1);
  long long* start = reinterpret_cast<long long*>(c->scratch[4].ensure(sizeof(long long) * (K + 1)));
  FF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (K + 1), st));
  {
    ProfScope ps(kProfPattern);
    (k_home<<<ceil_div(nq, TB), TB, 0, st>>>(c->qpts.as<float>(), nq, c->nbr_ptr.as<long long>(),
                                             c->nbr_idx.as<int>(), c->pos.as<float4>(), home, cnt),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    scan_counts(cnt, start, K, c, c->scratch[3]);
    (k_home_scatter<<<ceil_div(nq, TB), TB, 0, st>>>(home, nq, start, cursor, order),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  // ---- dense accumulators
  const size_t kk = (size_t)K * K;
  double* Hd = reinterpret_cast<double*>(c->scratch[2].ensure(2 * sizeof(double) * kk));
  double* Md = Hd + kk;
  FF_CUDA(cudaMemsetAsync(Hd, 0, 2 * sizeof(double) * kk, st));
  {
    ProfScope ps(kProfAsmValues);
    if (tdf)
      launch_tiles<dfloat>(c, order, K, Hd, Md);
    else
      launch_tiles<float>(c, order, K, Hd, Md);
  }
  // ---- CSR
  int* rc = reinterpret_cast<int*>(c->scratch[5].ensure(sizeof(int) * (nq + 1)));
  (k_dense_count<<<ceil_div((long long)K * 32, TB), TB, 0, st>>>(Hd, Md, K, rc),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  long long* aptr = reinterpret_cast<long long*>(c->a_ptr.ensure(sizeof(long long) * (K + 1)));
  scan_counts(rc, aptr, K, c, c->scratch[3]);
  long long n2 = 0;
  FF_CUDA(cudaMemcpyAsync(&n2, aptr + K, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  c->n2 = n2;
  const size_t tb = f64 ? 8 : 4;
  c->a_col.ensure(sizeof(int) * n2);
  c->a_val.ensure(2 * tb * n2);
  c->h_f32.ensure(sizeof(float) * n2);
  c->hdiag_f32.ensure(sizeof(float) * K);
  if (f64)
    (k_dense_fill<double><<<ceil_div((long long)K * 32, TB), TB, 0, st>>>(
         Hd, Md, K, aptr, c->a_col.as<int>(), c->a_val.as<double>(), c->h_f32.as<float>(),
         c->hdiag_f32.as<float>()),
     ::ff::note_launch());
  else
    (k_dense_fill<float><<<ceil_div((long long)K * 32, TB), TB, 0, st>>>(
         Hd, Md, K, aptr, c->a_col.as<int>(), c->a_val.as<float>(), c->h_f32.as<float>(),
         c->hdiag_f32.as<float>()),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

}  // namespace ff
