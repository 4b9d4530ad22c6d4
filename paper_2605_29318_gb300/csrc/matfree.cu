// Matrix-free application of H_w and M (Prop. 1 and Eq. 14 without
// assembling either matrix).
//
// Prop. 1 writes H_w as a sum over the quadrature points of rank-3 terms:
//   H_w X = sum_s G_s^T D G_s X,   M X = Phi^T V Phi X,
// with (G_s)_ik = d_s phi_k(X_i), Phi_ik = phi_k(X_i), D = diag(v_i (lambda_i +
// 4 mu_i)) and V = diag(v_i).  Two passes over the shape-function tables:
//   k_mf_gather   one warp per quadrature point i: Y_i = [G_0 X, G_1 X, G_2 X,
//                 Phi X]_i (4 m values, lanes over the columns), scaled by the
//                 point's weights;
//   k_mf_scatter  one warp per node k, over the points that node covers (the
//                 transposed lists, ascending): (H X)_k = sum_i sum_s
//                 d_s phi_k(X_i) Y_i,s and (M X)_k = sum_i phi_k(X_i) Y_i,3 --
//                 fixed order, no atomics.
// It reads the tables (n1 pairs x 4 values) twice and the block once per pair,
// where an assembled product reads n2 matrix entries: the smaller of the two
// wherever n2 / n1 is large.  The sums are FP64 in FP64 contexts (the tables'
// double-float pairs rounded to FP64) and FP32 otherwise.
#include <type_traits>

#include "dfloat.cuh"
#include "ff_internal.cuh"

namespace ff {

template <class T>
void gather_block(ff_ctx* c, const T* X0, int m, T* X, int ld);
template <class T>
void scatter_block(ff_ctx* c, const T* X, int ld, int m, T* out);

namespace {

template <class S>
__device__ __forceinline__ double as_f64(S x) {
  return (double)x;
}

// C: compute type (double or float); S: stored table / weight type
template <class C, class S>
__global__ void k_mf_gather(const long long* __restrict__ ptr, const int* __restrict__ idx,
                            const S* __restrict__ phi, const S* __restrict__ dphi, long long n1,
                            const S* __restrict__ wh, const float* __restrict__ vol, long long nq,
                            const C* __restrict__ X, int m, C* __restrict__ Y) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= nq) return;
  const int lane = threadIdx.x & 31;
  const C w = (C)as_f64(wh[i]), v = (C)vol[i];
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int col = c0 + lane;
    C a0 = C(0), a1 = C(0), a2 = C(0), a3 = C(0);
    if (col < m)
      for (long long e = ptr[i]; e < ptr[i + 1]; ++e) {
        const C x = X[(long long)idx[e] * m + col];
        a0 += (C)as_f64(dphi[e]) * x;
        a1 += (C)as_f64(dphi[n1 + e]) * x;
        a2 += (C)as_f64(dphi[2 * n1 + e]) * x;
        a3 += (C)as_f64(phi[e]) * x;
      }
    if (col < m) {
      C* y = Y + i * 4LL * m;
      y[col] = w * a0;
      y[m + col] = w * a1;
      y[2 * m + col] = w * a2;
      y[3 * m + col] = v * a3;
    }
  }
}

template <class C, class S>
__global__ void k_mf_scatter(const long long* __restrict__ tptr, const int* __restrict__ tidx,
                             const long long* __restrict__ tpos, const S* __restrict__ phi,
                             const S* __restrict__ dphi, long long n1, long long n,
                             const C* __restrict__ Y, int m, C* __restrict__ YH,
                             C* __restrict__ YM) {
  const long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= n) return;
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int col = c0 + lane;
    C h = C(0), mm = C(0);
    if (col < m)
      for (long long a = tptr[k]; a < tptr[k + 1]; ++a) {
        const long long e = tpos[a];
        const C* y = Y + (long long)tidx[a] * 4 * m;
        h += (C)as_f64(dphi[e]) * y[col] + (C)as_f64(dphi[n1 + e]) * y[m + col] +
             (C)as_f64(dphi[2 * n1 + e]) * y[2 * m + col];
        mm += (C)as_f64(phi[e]) * y[3 * m + col];
      }
    if (col < m) {
      YH[k * m + col] = h;
      YM[k * m + col] = mm;
    }
  }
}

template <class C, class S>
void run(ff_ctx* c, const C* Xp, int m, C* YHp, C* YMp, const S* wh) {
  cudaStream_t st = c->stream;
  const long long n = c->n, nq = c->nq, n1 = c->n1;
  const int T = 256;
  C* Y = reinterpret_cast<C*>(c->scratch[1].ensure(sizeof(C) * 4 * (size_t)nq * m));
  (k_mf_gather<C, S><<<ceil_div(nq * 32, T), T, 0, st>>>(
       c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->phi.as<S>(), c->dphi.as<S>(), n1, wh,
       c->vol.as<float>(), nq, Xp, m, Y),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_mf_scatter<C, S><<<ceil_div(n * 32, T), T, 0, st>>>(
       c->nbrT_ptr.as<long long>(), c->nbrT_idx.as<int>(), c->nbrT_pos.as<long long>(),
       c->phi.as<S>(), c->dphi.as<S>(), n1, n, Y, m, YHp, YMp),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

}  // namespace

void apply_matfree(ff_ctx* c, const float* E, const float* nu, double E0, double nu0,
                   const void* X, int m, void* YH, void* YM) {
  if (!c->has_cols) twoset_columns(c, c->qpts.as<float>());
  const long long n = c->n, nq = c->nq;
  const bool f64 = c->prec == FF_PREC_FP64;
  void* wh = c->scratch[0].ensure((tables_f32(c) ? 4 : 8) * (size_t)nq + 64);
  material_weights(c, E, nu, E0, nu0, wh);
  auto go = [&](auto tag) {
    using C = decltype(tag);
    C* in = reinterpret_cast<C*>(c->scratch[4].ensure(sizeof(C) * n * m));
    C* oh = reinterpret_cast<C*>(c->scratch[6].ensure(sizeof(C) * n * m));
    C* om = reinterpret_cast<C*>(c->scratch[7].ensure(sizeof(C) * n * m));
    gather_block<C>(c, static_cast<const C*>(X), m, in, m);
    if constexpr (std::is_same_v<C, double>) {
      if (tables_f32(c))
        run<double, float>(c, in, m, oh, om, static_cast<const float*>(wh));
      else
        run<double, dfloat>(c, in, m, oh, om, static_cast<const dfloat*>(wh));
    } else
      run<float, float>(c, in, m, oh, om, static_cast<const float*>(wh));
    if (YH) scatter_block<C>(c, oh, m, m, static_cast<C*>(YH));
    if (YM) scatter_block<C>(c, om, m, m, static_cast<C*>(YM));
    FF_CUDA(cudaStreamSynchronize(c->stream));
  };
  if (f64)
    go(double{});
  else
    go(float{});
}

}  // namespace ff
