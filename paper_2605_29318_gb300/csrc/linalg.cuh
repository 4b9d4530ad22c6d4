// Block linear-algebra launchers used by the eigensolver (internal).
#pragma once

#include "dfloat.cuh"
#include "ff_internal.cuh"

namespace ff {

template <class T>
void spmm_hm_raw(cudaStream_t st, const long long* ptr, const int* col, const T* val, long long n,
                 const T* X, int ldx, T* YH, T* YM, int ldy, int m);

void cheb_step(cudaStream_t st, const long long* ptr, const int* col, const float* hv,
               const float* hdiag, long long n, int m, int ld, const float* din, float* dout,
               float* x, float* res, float c1, float c2, int prof = kProfPrecond);

// The same step with the direction vectors d stored in BF16 (m % 8 == 0):
// each gathered row is half the bytes; the residual and the accumulated x stay
// FP32, and x accumulates the rounded directions that H is applied to.
void cheb_step_b16(cudaStream_t st, const long long* ptr, const int* col, const float* hv,
                   const float* hdiag, long long n, int m, const void* din, void* dout, float* x,
                   float* res, float c1, float c2);

// Tensor-core form of the BF16 step (chebtc.cu): cheb_tc_build lays out the
// block-dense tiles after assembly (false: spans too wide, the CUDA-core step
// stays in use); cheb_step_tc runs one step (false: not built or m outside
// 8..120 in steps of 8 -- nothing launched).
bool cheb_tc_build(ff_ctx* c);
bool cheb_step_tc(cudaStream_t st, const ff_ctx* c, int m, const void* din, void* dout, float* x,
                  float* res, float c1, float c2);

// out (p x q, row-major with leading dimension ldo (default q), FP64)
// (+)= alpha * A^T B over n rows
template <class T>
void gram(cudaStream_t st, const T* A, int lda, int p, const T* B, int ldb, int q, long long n,
          double* out, double alpha, bool accumulate, Buf& part, int ldo = -1);

// Gram matrices of the Rayleigh-Ritz step on the basis S = [X | W | P] (nblk
// blocks of nb columns, ns = nblk * nb): A = S^T H S (the block lower triangle,
// mirrored) and of B = S^T M S the W columns and rows and the diagonal -- the
// only entries the Rayleigh-Ritz step reads, since X and P are M-orthonormal
// and M-orthogonal to each other by construction
template <class T>
void gram_rr(cudaStream_t st, const T* S, const T* HS, const T* MS, int ld, int nb, int nblk,
             long long n, double* A, double* B, Buf& part);

// the same Gram matrices for FP32 blocks on the tensor cores (gram_tc.cu):
// split-BF16 x 3 tcgen05 products with FP32 accumulation in TMEM, FP64 sums
// across row ranges; false (nothing launched) when ns > 256 or n < 2048
bool gram_rr_tc(cudaStream_t st, const float* S, const float* HS, const float* MS, int ld, int nb,
                int nblk, long long n, double* A, double* B, Buf& part);
// whether gram_rr takes the tensor-core path for FP32 blocks (default on;
// the environment variable FF_GRAM_TC=0 turns it off for comparisons)
bool gram_tc_enabled();
// A: upper block triangle from the lower one; B: the W rows from the W columns
void gram_mirror(cudaStream_t st, double* A, double* B, int ns, int nb);

// C (n x q, with the column split described in linalg.cu) = beta C + A Y, Y p x q row-major
// with leading dimension ldy (default q)
template <class T>
void block_update(cudaStream_t st, const T* A, int lda, int p, const T* Y, int q, T* C, int ldc,
                  long long n, T beta, int split = -1, int off2 = 0, int ldy = -1);

// small dense Rayleigh-Ritz (dense.cu)
struct RRDims {
  int ns;      // basis columns used (nx + nw + np)
  int nx;      // columns of X at the front
  int nb;      // Ritz vectors kept
  int want_p;  // 1: also build the P coefficients Z
  int o0, no;  // the block that is not yet M-orthonormal: columns [o0, o0 + no)
  double drop = 1e-13;  // O columns whose M-orthogonal remainder has squared
                        // relative norm below this leave the basis
};
template <class T>
void rayleigh_ritz(cudaStream_t st, const double* A, const double* B, RRDims d, T* YZ,
                   double* theta, int* dropped, Buf& work, bool fp64, double* dbg = nullptr);

}  // namespace ff
