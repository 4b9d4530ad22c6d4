// Corrected RKPM shape functions and gradients, one warp per evaluation point.
//
// Sec. 3.2, Eqs. 7, 9-10: phi_k(X) = varphi_k(X) P(p_k)^T C(X), M(X) C(X) = P(X),
// M(X) = sum_k varphi_k(X) P(p_k) P(p_k)^T with the linear basis.  The basis is
// written about the evaluation point, P_o(p) = [1, (p - X_i)/a_i] (an invertible
// affine change of [1, x, y, z], so phi is unchanged and M is well scaled).  The
// gradient follows from differentiating M C = P_o:
//   d_s C = M^{-1} (e_{1+s}/a_i - (d_s M) C),
//   d_s phi_k = d_s varphi_k P_k^T C + varphi_k P_k^T d_s C.
// Raw kernel: cubic B-spline w(q), q = |X - p_k| / a_k, grad = (w'(q)/q)(X - p_k)/a_k^2.
//
// Lanes stride over the row's neighbours and accumulate the 10 distinct entries
// of M and the 30 of d M; a butterfly reduction gives every lane the sums; every
// lane then solves the 4x4 system (Cholesky) and writes phi / grad phi for its
// own neighbours.  In FP32 mode a row whose moment matrix has a 1-norm condition
// number above `cond_fp64` is recomputed entirely in FP64.  FP64 mode computes
// and stores double-float pairs (FP32 head and tail, ~2^-47 relative).
#include "dfloat.cuh"
#include "ff_internal.cuh"
#include "rkpm_eval.cuh"

namespace ff {
namespace {

using rkpm::shape_row;

template <class T>
__global__ void k_shape(const float4* __restrict__ pos, const long long* __restrict__ ptr,
                        const int* __restrict__ idx, long long n, long long n1,
                        T* __restrict__ phi, T* __restrict__ dphi, double cond_limit,
                        DevFlags* __restrict__ flags) {
  long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const int lane = threadIdx.x & 31;
  long long s = ptr[i], e = ptr[i + 1];
  float4 Xi = pos[i];
  int st;
  if (sizeof(T) == 4) {
    st = shape_row<float, T>(pos, s, e, idx, Xi, phi, dphi, n1, cond_limit, true);
    if (st != 0) {
      st = shape_row<double, T>(pos, s, e, idx, Xi, phi, dphi, n1, 0.0, false);
      if (lane == 0 && st == 0) atomicAdd(&flags->fallback, 1);
    }
  } else {
    // FP64 outputs computed in double-float (~2^-47 relative; GB300's FP64
    // rate made this kernel FP64-bound)
    st = shape_row<dfloat, T>(pos, s, e, idx, Xi, phi, dphi, n1, 0.0, false);
  }
  if (st == 1 && lane == 0) {
    if (atomicCAS(&flags->code, 0, (int)FF_ERR_SINGULAR_MOMENT) == 0) flags->index = (int)i;
  }
}

}  // namespace

void build_shape(ff_ctx* c) {
  const long long n = c->n, n1 = c->n1;
  const int T = 256;
  reset_flags(c);
  size_t es = c->prec == FF_PREC_FP64 ? 8 : 4;
  c->phi.ensure(es * n1);
  c->dphi.ensure(3 * es * n1);
  const double cond_limit = 1e2;
  ProfScope ps(kProfShape);
  if (c->prec == FF_PREC_FP64) {  // stored as double-float pairs for the assembly
    (k_shape<dfloat><<<ceil_div(n * 32, T), T, 0, c->stream>>>(
        c->pos.as<float4>(), c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), n, n1,
        c->phi.as<dfloat>(), c->dphi.as<dfloat>(), cond_limit, c->flags.as<DevFlags>()), ::ff::note_launch());
  } else {
    (k_shape<float><<<ceil_div(n * 32, T), T, 0, c->stream>>>(
        c->pos.as<float4>(), c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), n, n1,
        c->phi.as<float>(), c->dphi.as<float>(), cond_limit, c->flags.as<DevFlags>()), ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
  ps.close();
  DevFlags f = read_flags(c);
  c->hflags->fallback = f.fallback;
  if (f.code == FF_ERR_SINGULAR_MOMENT) {
    int orig = -1;
    FF_CUDA(cudaMemcpy(&orig, c->perm.as<int>() + f.index, sizeof(int), cudaMemcpyDeviceToHost));
    throw Error(FF_ERR_SINGULAR_MOMENT,
                "moment matrix of particle " + std::to_string(orig) +
                    " is singular: fewer than four non-coplanar nodes cover it");
  }
}

}  // namespace ff
