// Skinning weight fields and linear blend skinning at query points.
//
// The reduced-order basis of the paper is the set of weight fields
// W^j(X) = sum_k phi_k(X) c_k^j (Sec. 3.2): the corrected RKPM shape functions
// of the built cloud (the same kernel, supports and linear basis as the
// cloud's own shape functions, Eqs. 6-11) evaluated at X, times the nodal
// values c (the eigenmodes).  The deformation is linear blend skinning,
// Eq. 1: x = X + sum_j W^j(X) Z_j [X; 1] with Z_j in R^{3x4}.
//
// Pipeline: a gather search (each query point scans the 27 cells around its
// cell -- the cell edge is at least the largest support, so those hold every
// node that covers it; points outside the box are clamped to the boundary
// cells, which still hold every node within one support of them), the moment
// solve and shape functions per query point (one warp each; double-float in
// FP64 contexts, FP32 with the FP64 redo of ill-conditioned points in FP32
// ones), and the weights as one warp per point over the modes.  Clouds of the
// two-set discretisation take its own covering test over the K centres and
// its Gaussian shape functions (twoset.cu).
#include "grid.cuh"
#include "rkpm_eval.cuh"

namespace ff {
namespace {

using rkpm::shape_row;

// MODE 0: count the nodes covering each query point; MODE 1: list them (in
// cell order, then node order inside a cell: deterministic)
template <int MODE>
__global__ void k_query_search(const float* __restrict__ Q, long long nq,
                               const float4* __restrict__ pos, GridDev g,
                               const int* __restrict__ cstart, int* __restrict__ cnt,
                               const long long* __restrict__ qptr, int* __restrict__ qidx) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float4 X = make_float4(Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], 0.f);
  const int cx = cell_coord(X.x, g.o0, g.h, g.d0);
  const int cy = cell_coord(X.y, g.o1, g.h, g.d1);
  const int cz = cell_coord(X.z, g.o2, g.h, g.d2);
  int c = 0;
  const long long base = MODE ? qptr[q] : 0;
  for (int z = max(cz - 1, 0); z <= min(cz + 1, g.d2 - 1); ++z)
    for (int y = max(cy - 1, 0); y <= min(cy + 1, g.d1 - 1); ++y)
      for (int x = max(cx - 1, 0); x <= min(cx + 1, g.d0 - 1); ++x) {
        const long long key = cell_key(g, x, y, z);
        for (int i = cstart[key]; i < cstart[key + 1]; ++i)
          if (covers(X, pos[i])) {
            if (MODE) qidx[base + c] = i;
            ++c;
          }
      }
  if (!MODE) cnt[q] = c;
}

// shape functions of query point q (one warp): FP64 contexts in double-float
// with FP64 output, FP32 contexts in FP32 with the FP64 redo when the moment
// matrix is ill-conditioned.  scale normalises the linear basis (any positive
// value gives the same functions; the support size keeps M well scaled).
template <class T>
__global__ void k_query_shape(const float4* __restrict__ pos, const float* __restrict__ Q,
                              const long long* __restrict__ qptr, const int* __restrict__ qidx,
                              long long nq, long long nq1, float scale, T* __restrict__ phi,
                              T* __restrict__ dphi, double cond_limit,
                              DevFlags* __restrict__ flags) {
  const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= nq) return;
  const int lane = threadIdx.x & 31;
  const long long s = qptr[q], e = qptr[q + 1];
  const float4 Xq = make_float4(Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], scale);
  int st = 1;
  if (e > s) {
    if constexpr (sizeof(T) == 4) {
      st = shape_row<float, T>(pos, s, e, qidx, Xq, phi, dphi, nq1, cond_limit, true);
      if (st != 0) st = shape_row<double, T>(pos, s, e, qidx, Xq, phi, dphi, nq1, 0.0, false);
    } else {
      st = shape_row<dfloat, T>(pos, s, e, qidx, Xq, phi, dphi, nq1, 0.0, false);
    }
  }
  if (st != 0 && lane == 0)
    if (atomicCAS(&flags->code, 0, (int)FF_ERR_SINGULAR_MOMENT) == 0) flags->index = (int)q;
}

// W[q][j] = sum over the nodes k covering q of phi_k(X_q) C[j][perm k]
// (C column-major n x m in the caller's order); one warp per point, lanes
// over the modes
template <class T>
__global__ void k_query_weights(const long long* __restrict__ qptr, const int* __restrict__ qidx,
                                const T* __restrict__ phi, long long nq,
                                const int* __restrict__ perm, const T* __restrict__ C,
                                long long n, int m, T* __restrict__ W) {
  const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= nq) return;
  const int lane = threadIdx.x & 31;
  const long long s = qptr[q], e = qptr[q + 1];
  for (int j = lane; j < m; j += 32) {
    T acc = T(0);
    for (long long t = s; t < e; ++t) acc += phi[t] * C[(long long)j * n + perm[qidx[t]]];
    W[q * m + j] = acc;
  }
}

// x_q = X_q + sum_j W[q][j] Z_j [X_q; 1]  (Z row-major m x 3 x 4)
template <class T>
__global__ void k_lbs(const float* __restrict__ Q, long long nq, const T* __restrict__ W, int m,
                      const T* __restrict__ Z, T* __restrict__ x) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const T X0 = (T)Q[3 * q], X1 = (T)Q[3 * q + 1], X2 = (T)Q[3 * q + 2];
  T o0 = X0, o1 = X1, o2 = X2;
  for (int j = 0; j < m; ++j) {
    const T w = W[q * m + j];
    const T* z = Z + 12LL * j;
    o0 += w * (z[0] * X0 + z[1] * X1 + z[2] * X2 + z[3]);
    o1 += w * (z[4] * X0 + z[5] * X1 + z[6] * X2 + z[7]);
    o2 += w * (z[8] * X0 + z[9] * X1 + z[10] * X2 + z[11]);
  }
  x[3 * q] = o0;
  x[3 * q + 1] = o1;
  x[3 * q + 2] = o2;
}

template <class T>
void weights_t(ff_ctx* c, const float* Q, long long nq, const T* C, int m, T* W) {
  cudaStream_t st = c->stream;
  const int TB = 256;
  if (c->twoset) {
    const long long nq1 = twoset_cover(c, Q, nq, c->sk_ptr, c->sk_idx, c->sk_cnt);
    const long long* qptr = c->sk_ptr.as<long long>();
    const int* qidx = c->sk_idx.as<int>();
    T* phi = reinterpret_cast<T*>(c->sk_phi.ensure(sizeof(T) * 4 * std::max(nq1, 1LL)));
    const DevFlags f = twoset_shape(c, Q, nq, qptr, qidx, nq1, phi, phi + nq1, true);
    if (f.code == FF_ERR_SINGULAR_MOMENT)
      throw Error(FF_ERR_SINGULAR_MOMENT,
                  "query point " + std::to_string(f.index) +
                      " is covered by fewer than four non-coplanar centres");
    (k_query_weights<T><<<ceil_div(nq * 32, TB), TB, 0, st>>>(qptr, qidx, phi, nq,
                                                              c->perm.as<int>(), C, c->n, m, W),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    FF_CUDA(cudaStreamSynchronize(st));
    return;
  }
  const Grid& g = c->grid;
  const GridDev gd{g.origin[0], g.origin[1], g.origin[2], g.h, g.dims[0], g.dims[1], g.dims[2],
                   g.bdims[0], g.bdims[1], g.bdims[2]};
  int* cnt = reinterpret_cast<int*>(c->sk_cnt.ensure(sizeof(int) * (nq + 1)));
  long long* qptr = reinterpret_cast<long long*>(c->sk_ptr.ensure(sizeof(long long) * (nq + 1)));
  (k_query_search<0><<<ceil_div(nq, TB), TB, 0, st>>>(Q, nq, c->pos.as<float4>(), gd,
                                                      c->cell_start.as<int>(), cnt, nullptr,
                                                      nullptr),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  scan_counts(cnt, qptr, nq, c, c->scratch[3]);
  long long nq1 = 0;
  FF_CUDA(cudaMemcpyAsync(&nq1, qptr + nq, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  int* qidx = reinterpret_cast<int*>(c->sk_idx.ensure(sizeof(int) * std::max(nq1, 1LL)));
  (k_query_search<1><<<ceil_div(nq, TB), TB, 0, st>>>(Q, nq, c->pos.as<float4>(), gd,
                                                      c->cell_start.as<int>(), nullptr, qptr,
                                                      qidx),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  T* phi = reinterpret_cast<T*>(c->sk_phi.ensure(sizeof(T) * 4 * std::max(nq1, 1LL)));
  T* dphi = phi + nq1;
  reset_flags(c);
  (k_query_shape<T><<<ceil_div(nq * 32, TB), TB, 0, st>>>(
       c->pos.as<float4>(), Q, qptr, qidx, nq, nq1, (float)(g.h / 1.001), phi, dphi, 1e2,
       c->flags.as<DevFlags>()),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const DevFlags f = read_flags(c);
  if (f.code == FF_ERR_SINGULAR_MOMENT)
    throw Error(FF_ERR_SINGULAR_MOMENT,
                "query point " + std::to_string(f.index) +
                    " is covered by fewer than four non-coplanar nodes");
  (k_query_weights<T><<<ceil_div(nq * 32, TB), TB, 0, st>>>(qptr, qidx, phi, nq,
                                                            c->perm.as<int>(), C, c->n, m, W),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  FF_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

void skinning_weights(ff_ctx* c, const float* Q, long long nq, const void* C, int m, void* W) {
  if (nq == 0) return;
  if (c->prec == FF_PREC_FP64)
    weights_t<double>(c, Q, nq, static_cast<const double*>(C), m, static_cast<double*>(W));
  else
    weights_t<float>(c, Q, nq, static_cast<const float*>(C), m, static_cast<float*>(W));
}

void lbs_deform(ff_ctx* c, const float* Q, long long nq, const void* W, int m, const void* Z,
                void* x) {
  if (nq == 0) return;
  const int TB = 256;
  if (c->prec == FF_PREC_FP64)
    (k_lbs<double><<<ceil_div(nq, TB), TB, 0, c->stream>>>(Q, nq, static_cast<const double*>(W),
                                                           m, static_cast<const double*>(Z),
                                                           static_cast<double*>(x)),
     ::ff::note_launch());
  else
    (k_lbs<float><<<ceil_div(nq, TB), TB, 0, c->stream>>>(Q, nq, static_cast<const float*>(W), m,
                                                          static_cast<const float*>(Z),
                                                          static_cast<float*>(x)),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
  FF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace ff
