// Learned warm start: particle features, the point network (forward, loss,
// backward, Adam) and the start block handed to the eigensolver.
//
// The paper starts LOBPCG from a random block (Supp. Sec. B); this layer
// predicts a start block for the same eigenproblem (Sec. 3.2, Eq. 15).  The
// features, network, loss and optimiser are the ones declared in freeform.h.
//
// GB300 mapping: every layer is one tiled GEMM (64 x 64 tiles, BF16 or FP32
// operands staged in shared memory as FP32, FP32 accumulation) whose epilogue
// fuses bias, ReLU, the backward ReLU mask, BF16 rounding of the stored
// activation and, for the second layer, the max-pool over particles (an
// atomicMax on a packed (value, ~row) key, so h2 is never stored).  Weight
// gradients are split-K GEMMs over the particles with FP32 atomics.  The loss
// needs three small Gram matrices of the output block; they are accumulated
// in FP64 per entry, and the 32 x 32 algebra runs in one block in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "linalg.cuh"

struct ff_net {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  long long t = 0;             // Adam steps taken
  ff::Buf master, m1, m2;      // FP32 parameters and Adam moments
  ff::Buf w16;                 // BF16 copy used by the kernels
  ff::Buf grad;                // FP32 gradient
  long long cap = 0;           // particles the activation buffers hold
  ff::Buf f16, h1, h3, h4, y;  // activations (BF16 except y)
  ff::Buf dy, dh4, dh3, dh1;   // FP32 gradients of the activations
  ff::Buf pool, g, arg, c3, dg;
  ff::Buf lsum, small;         // loss Grams (FP64) and the 32 x 32 results
  double* h_small = nullptr;   // pinned
};

namespace ff {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kF = FF_WS_FEATURES, kO = FF_WS_OUTPUTS;
constexpr int kH1 = 128, kH2 = 256, kH3 = 256, kH4 = 128, kZ = kH1 + kH2;
constexpr long long oW1 = 0, oB1 = oW1 + kH1 * kF, oW2 = oB1 + kH1, oB2 = oW2 + kH2 * kH1,
                    oW3 = oB2 + kH2, oB3 = oW3 + kH3 * kZ, oW4 = oB3 + kH3,
                    oB4 = oW4 + kH4 * kH3, oW5 = oB4 + kH4, oB5 = oW5 + kO * kH4,
                    kP = oB5 + kO;
static_assert(kP == 170784, "parameter count");
constexpr int kMaxModes = 32;
constexpr int kLossEntries = kO * kO + kO * kMaxModes + kMaxModes * kMaxModes;

// ------------------------------------------------------------------ GEMM
// C[m][n] = epilogue(sum_k A(m, k) B(k, n)), A(m, k) = A[m * sam + k * sak],
// B(k, n) = B[k * sbk + n * sbn]; operands BF16 or FP32.
struct Gemm {
  int M = 0, N = 0, K = 0;
  const void* A = nullptr;
  int a16 = 0;
  long long sam = 0, sak = 0;
  const void* B = nullptr;
  int b16 = 0;
  long long sbk = 0, sbn = 0;
  const float* bias = nullptr;   // + bias[n]
  const float* bias2 = nullptr;  // + bias2[n]
  int relu = 0;
  const bf16* mask = nullptr;    // zero where mask[m * ldmask + n] <= 0
  long long ldmask = 0;
  void* C = nullptr;
  int c16 = 0;
  long long ldc = 0;
  int atomic = 0;                      // C += (FP32, split-K)
  unsigned long long* pool = nullptr;  // max-pool over m instead of a store
  int kchunk = 0;
};

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ float ldv(const void* p, int b16, long long off) {
  return b16 ? __bfloat162float(static_cast<const bf16*>(p)[off])
             : static_cast<const float*>(p)[off];
}

__global__ void __launch_bounds__(256) k_gemm(Gemm g) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int kb = blockIdx.z * g.kchunk;
  const int ke = min(g.K, kb + g.kchunk);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const bool a_kfast = g.sak == 1;
  const bool b_nfast = g.sbn == 1;
  for (int k0 = kb; k0 < ke; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      const int mm = a_kfast ? e / TK : e % TM;
      const int kk = a_kfast ? e % TK : e / TM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < ke) ? ldv(g.A, g.a16, (long long)m * g.sam + (long long)k * g.sak)
                                       : 0.f;
    }
    for (int e = tid; e < TN * TK; e += 256) {
      const int nn = b_nfast ? e % TN : e / TK;
      const int kk = b_nfast ? e / TN : e % TK;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < ke) ? ldv(g.B, g.b16, (long long)k * g.sbk + (long long)n * g.sbn)
                                       : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      if (g.bias) v += g.bias[n];
      if (g.bias2) v += g.bias2[n];
      if (g.relu) v = v > 0.f ? v : 0.f;
      if (g.mask && !(__bfloat162float(g.mask[(long long)m * g.ldmask + n]) > 0.f)) v = 0.f;
      const long long o = (long long)m * g.ldc + n;
      if (g.pool) {  // v >= 0 here: its bits order like the value; ties -> lowest row
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(v) << 32) | (0xffffffffu - (unsigned)m);
        atomicMax(&g.pool[n], key);
      } else if (g.atomic) {
        atomicAdd(static_cast<float*>(g.C) + o, v);
      } else if (g.c16) {
        static_cast<bf16*>(g.C)[o] = __float2bfloat16(v);
      } else {
        static_cast<float*>(g.C)[o] = v;
      }
    }
  }
}

void gemm(cudaStream_t st, Gemm g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return;
  const int tiles = ceil_div(g.M, TM) * ceil_div(g.N, TN);
  if (g.kchunk <= 0) {
    if (g.atomic) {  // split the reduction so that ~2 blocks run per SM
      const int splits = std::max(1, std::min(ceil_div(304, tiles), ceil_div(g.K, 256)));
      g.kchunk = ceil_div(ceil_div(g.K, splits), TK) * TK;
    } else {
      g.kchunk = ceil_div(g.K, TK) * TK;
    }
  }
  dim3 grid(ceil_div(g.N, TN), ceil_div(g.M, TM), ceil_div(g.K, g.kchunk));
  (k_gemm<<<grid, 256, 0, st>>>(g), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ elementwise
__global__ void k_f2bf(const float* __restrict__ x, bf16* __restrict__ y, long long m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) y[t] = __float2bfloat16(x[t]);
}

// column sums of a row-major n x w FP32 matrix (w <= 256), added into out
__global__ void k_colsum(const float* __restrict__ X, long long n, int w, float* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= w) return;
  const long long r0 = (long long)blockIdx.x * 256;
  const long long r1 = r0 + 256 < n ? r0 + 256 : n;
  float s = 0.f;
  for (long long r = r0; r < r1; ++r) s += X[r * w + c];
  atomicAdd(out + c, s);
}

__global__ void k_pool_finish(const unsigned long long* __restrict__ pool, float* __restrict__ g,
                              int* __restrict__ arg) {
  const int c = threadIdx.x;
  if (c >= kH2) return;
  const unsigned long long key = pool[c];
  g[c] = __uint_as_float((unsigned)(key >> 32));
  arg[c] = (int)(0xffffffffu - (unsigned)(key & 0xffffffffu));
}

// c3 = W3[:, 128:] g + b3 (one warp per output)
__global__ void k_global_term(const bf16* __restrict__ w, const float* __restrict__ g,
                              const float* __restrict__ b3, float* __restrict__ c3) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= kH3) return;
  float s = 0.f;
  for (int c = lane; c < kH2; c += 32)
    s = fmaf(__bfloat162float(w[oW3 + (long long)j * kZ + kH1 + c]), g[c], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) c3[j] = s + b3[j];
}

// ------------------------------------------------------------------ loss
// Unnormalised sums: G0 = sum v y y^T (32 x 32), Z = sum v y c^T (32 x m),
// K = sum v c c^T (m x m) and sum v, accumulated per entry in FP64.
__global__ void __launch_bounds__(256)
    k_loss_gram(const float* __restrict__ Y, const float* __restrict__ C, const float* __restrict__ vol,
                long long n, int m, double* __restrict__ out) {
  __shared__ double ys[32][kO + 1];
  __shared__ double cs[32][kMaxModes + 1];
  __shared__ double vs[32];
  const int tid = threadIdx.x;
  const int E = kO * kO + kO * m + m * m;
  double acc[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) acc[r] = 0.0;
  double vsum = 0.0;
  for (long long p0 = (long long)blockIdx.x * 32; p0 < n; p0 += (long long)gridDim.x * 32) {
    for (int e = tid; e < 32 * kO; e += 256) {
      const int pl = e / kO, j = e % kO;
      const long long p = p0 + pl;
      ys[pl][j] = p < n ? (double)Y[p * kO + j] : 0.0;
    }
    for (int e = tid; e < 32 * m; e += 256) {
      const int j = e / 32, pl = e % 32;
      const long long p = p0 + pl;
      cs[pl][j] = p < n ? (double)C[(long long)j * n + p] : 0.0;
    }
    if (tid < 32) vs[tid] = p0 + tid < n ? (double)vol[p0 + tid] : 0.0;
    __syncthreads();
    if (tid == 0)
      for (int pl = 0; pl < 32; ++pl) vsum += vs[pl];
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      const int e = tid + 256 * r;
      if (e >= E) break;
      int xa, zb;
      if (e < kO * kO) {
        xa = e / kO;
        zb = e % kO;
        double s = acc[r];
        for (int pl = 0; pl < 32; ++pl) s = fma(vs[pl] * ys[pl][xa], ys[pl][zb], s);
        acc[r] = s;
      } else if (e < kO * kO + kO * m) {
        const int q = e - kO * kO;
        xa = q / m; zb = q % m;
        double s = acc[r];
        for (int pl = 0; pl < 32; ++pl) s = fma(vs[pl] * ys[pl][xa], cs[pl][zb], s);
        acc[r] = s;
      } else {
        const int q = e - kO * kO - kO * m;
        xa = q / m; zb = q % m;
        double s = acc[r];
        for (int pl = 0; pl < 32; ++pl) s = fma(vs[pl] * cs[pl][xa], cs[pl][zb], s);
        acc[r] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    const int e = tid + 256 * r;
    if (e < E) atomicAdd(out + e, acc[r]);
  }
  if (tid == 0) atomicAdd(out + kLossEntries, vsum);
}

// in-place inverse of an SPD q x q matrix held in shared memory (Gauss-Jordan
// without pivoting; aug is q x 2q scratch, fac q scratch)
__device__ void spd_inverse(double* A, int q, double* aug, double* fac) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < q * 2 * q; t += nt) {
    const int i = t / (2 * q), j = t % (2 * q);
    aug[t] = j < q ? A[i * q + j] : (j - q == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int p = 0; p < q; ++p) {
    const double piv = aug[p * 2 * q + p];
    __syncthreads();
    for (int j = tid; j < 2 * q; j += nt) aug[p * 2 * q + j] /= piv;
    for (int i = tid; i < q; i += nt) fac[i] = aug[i * 2 * q + p];
    __syncthreads();
    for (int t = tid; t < q * 2 * q; t += nt) {
      const int i = t / (2 * q), j = t % (2 * q);
      if (i != p) aug[t] -= fac[i] * aug[p * 2 * q + j];
    }
    __syncthreads();
  }
  for (int t = tid; t < q * q; t += nt) A[t] = aug[(t / q) * 2 * q + q + t % q];
  __syncthreads();
}

// 32 x 32 algebra of the loss: P1 = K^-1 Z^T G^-1, P2' = G^-1 Z P1 + e q I,
// L = 1 - trace(P1 Z) / m, coef = -2 / (m sum v)
__global__ void __launch_bounds__(1024)
    k_loss_small(const double* __restrict__ sums, int m, float* __restrict__ P1o,
                 float* __restrict__ P2o, double* __restrict__ scal) {
  __shared__ double G[kO * kO], Kq[kMaxModes * kMaxModes], Z[kO * kMaxModes];
  __shared__ double aug[kO * 2 * kO];
  __shared__ double fac[kO], red[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double V = sums[kLossEntries];
  for (int t = tid; t < kO * kO; t += nt) G[t] = sums[t] / V;
  for (int t = tid; t < kO * m; t += nt) Z[t] = sums[kO * kO + t] / V;
  for (int t = tid; t < m * m; t += nt) Kq[t] = sums[kO * kO + kO * m + t] / V;
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < kO; ++i) tr += G[i * kO + i];
    red[0] = 1e-6 * tr / kO;
  }
  __syncthreads();
  if (tid < kO) G[tid * kO + tid] += red[0];
  __syncthreads();
  spd_inverse(G, kO, aug, fac);
  spd_inverse(Kq, m, aug, fac);
  double* P1 = aug;                // m x 32
  double* GZ = aug + kMaxModes * kO;  // 32 x m
  for (int t = tid; t < kO * m; t += nt) {  // GZ = G^-1 Z
    const int i = t / m, j = t % m;
    double s = 0.0;
    for (int l = 0; l < kO; ++l) s += G[i * kO + l] * Z[l * m + j];
    GZ[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < m * kO; t += nt) {  // P1 = K^-1 (G^-1 Z)^T
    const int a = t / kO, j = t % kO;
    double s = 0.0;
    for (int b = 0; b < m; ++b) s += Kq[a * m + b] * GZ[j * m + b];
    P1[t] = s;
  }
  __syncthreads();
  double* P2 = G;                  // G^-1 is no longer needed
  for (int t = tid; t < kO * kO; t += nt) {  // P2 = (G^-1 Z) P1
    const int i = t / kO, j = t % kO;
    double s = 0.0;
    for (int a = 0; a < m; ++a) s += GZ[i * m + a] * P1[a * kO + j];
    P2[t] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double tz = 0.0, q = 0.0;
    for (int a = 0; a < m; ++a)
      for (int j = 0; j < kO; ++j) {
        tz += P1[a * kO + j] * Z[j * m + a];
        q += P1[a * kO + j] * GZ[j * m + a];
      }
    red[1] = q;
    scal[0] = 1.0 - tz / m;
    scal[1] = -2.0 / (m * V);
  }
  __syncthreads();
  const double eq = 1e-6 / kO * red[1];
  for (int t = tid; t < m * kO; t += nt) P1o[t] = (float)P1[t];
  for (int t = tid; t < kO * kO; t += nt)
    P2o[t] = (float)(P2[t] + ((t / kO) == (t % kO) ? eq : 0.0));
}

// dy[p][j] = coef v_p (sum_a C[a][p] P1[a][j] - sum_b y[p][b] P2'[b][j])
__global__ void k_loss_dy(const float* __restrict__ Y, const float* __restrict__ C,
                          const float* __restrict__ vol, long long n, int m,
                          const float* __restrict__ P1g, const float* __restrict__ P2g,
                          const double* __restrict__ scal, float* __restrict__ dy) {
  __shared__ float P1[kMaxModes * kO], P2[kO * kO];
  for (int t = threadIdx.x; t < m * kO; t += blockDim.x) P1[t] = P1g[t];
  for (int t = threadIdx.x; t < kO * kO; t += blockDim.x) P2[t] = P2g[t];
  __syncthreads();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float acc[kO];
#pragma unroll
  for (int j = 0; j < kO; ++j) acc[j] = 0.f;
  for (int a = 0; a < m; ++a) {
    const float c = C[(long long)a * n + p];
#pragma unroll
    for (int j = 0; j < kO; ++j) acc[j] = fmaf(c, P1[a * kO + j], acc[j]);
  }
  for (int b = 0; b < kO; ++b) {
    const float yb = Y[p * kO + b];
#pragma unroll
    for (int j = 0; j < kO; ++j) acc[j] = fmaf(-yb, P2[b * kO + j], acc[j]);
  }
  const float s = (float)scal[1] * vol[p];
#pragma unroll
  for (int j = 0; j < kO; ++j) dy[p * kO + j] = s * acc[j];
}

// ------------------------------------------------------------------ backward pieces
// dW3[:, 128:] = s3 g^T with s3 = db3 (column sums of dh3)
__global__ void k_outer_w3(const float* __restrict__ s3, const float* __restrict__ g,
                           float* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kH3 * kH2) return;
  const int j = t / kH2, c = t % kH2;
  grad[oW3 + (long long)j * kZ + kH1 + c] += s3[j] * g[c];
}

// dg = W3[:, 128:]^T s3
__global__ void k_dg(const bf16* __restrict__ w, const float* __restrict__ s3, float* __restrict__ dg) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kH2) return;
  float s = 0.f;
  for (int j = 0; j < kH3; ++j) s = fmaf(__bfloat162float(w[oW3 + (long long)j * kZ + kH1 + c]), s3[j], s);
  dg[c] = s;
}

// max-pool backward: channel c's gradient goes to its maximiser (if active)
__global__ void k_pool_backward(const float* __restrict__ g, const int* __restrict__ arg,
                                const float* __restrict__ dg, const bf16* __restrict__ h1,
                                const bf16* __restrict__ w, float* __restrict__ grad,
                                float* __restrict__ dh1) {
  const int c = blockIdx.x, i = threadIdx.x;
  if (!(g[c] > 0.f)) return;
  const long long p = arg[c];
  const float d = dg[c];
  if (i < kH1) {
    grad[oW2 + (long long)c * kH1 + i] += d * __bfloat162float(h1[p * kH1 + i]);
    atomicAdd(dh1 + p * kH1 + i, d * __bfloat162float(w[oW2 + (long long)c * kH1 + i]));
  }
  if (i == 0) grad[oB2 + c] += d;
}

__global__ void k_relu_mask(float* __restrict__ d, const bf16* __restrict__ h, long long m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m && !(__bfloat162float(h[t]) > 0.f)) d[t] = 0.f;
}

// Adam (Kingma & Ba, Algorithm 1), then the BF16 copy
__global__ void k_adam(float* __restrict__ th, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ gr, bf16* __restrict__ w, long long P, float lr,
                       float c1, float c2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const float gi = gr[t];
  const float a = 0.9f * m1[t] + 0.1f * gi;
  const float b = 0.999f * m2[t] + 0.001f * gi * gi;
  m1[t] = a;
  m2[t] = b;
  const float mh = a / c1, vh = b / c2;
  const float v = th[t] - lr * mh / (sqrtf(vh) + 1e-8f);
  th[t] = v;
  w[t] = __float2bfloat16(v);
}

__device__ __forceinline__ unsigned long long splitmix(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// He-normal weights (Box-Muller on counter-based uniforms), zero biases
__global__ void k_init(float* __restrict__ th, bf16* __restrict__ w, unsigned long long seed) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kP) return;
  const long long offs[5] = {oW1, oW2, oW3, oW4, oW5};
  const long long bofs[5] = {oB1, oB2, oB3, oB4, oB5};
  const int fan[5] = {kF, kH1, kZ, kH3, kH4};
  float v = 0.f;
  for (int l = 0; l < 5; ++l)
    if (t >= offs[l] && t < bofs[l]) {
      const unsigned long long r = splitmix(seed * 0x100000001b3ULL + (unsigned long long)t);
      const double u1 = ((r >> 11) + 1.0) * 0x1.0p-53, u2 = ((splitmix(r) >> 11) + 0.5) * 0x1.0p-53;
      v = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2) * sqrt(2.0 / fan[l]));
    }
  th[t] = v;
  w[t] = __float2bfloat16(v);
}

// ------------------------------------------------------------------ features
// global sums in FP64: [0] sum v, [1..3] sum v X, [4] sum |N|, [5..10] sum v d d^T,
// [11..13] third moments along the axes
__global__ void k_feat_moments(const float4* __restrict__ pos, const float* __restrict__ vol,
                               const long long* __restrict__ nptr, long long n, int pass,
                               const double* __restrict__ frame, double* __restrict__ sums) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const float4 p = pos[r];
    const double v = vol[r];
    if (pass == 0) {
      acc[0] += v;
      acc[1] += v * p.x;
      acc[2] += v * p.y;
      acc[3] += v * p.z;
      acc[4] += (double)(nptr[r + 1] - nptr[r]);
    } else {
      const double d0 = p.x - frame[0], d1 = p.y - frame[1], d2 = p.z - frame[2];
      if (pass == 1) {
        acc[0] += v * d0 * d0;
        acc[1] += v * d0 * d1;
        acc[2] += v * d0 * d2;
        acc[3] += v * d1 * d1;
        acc[4] += v * d1 * d2;
        acc[5] += v * d2 * d2;
      } else {
        for (int j = 0; j < 3; ++j) {
          const double u = d0 * frame[3 + j] + d1 * frame[6 + j] + d2 * frame[9 + j];
          acc[j] += v * u * u * u;
        }
      }
    }
  }
  const int base = pass == 0 ? 0 : pass == 1 ? 5 : 11;
  const int cnt = pass == 0 ? 5 : pass == 1 ? 6 : 3;
  for (int j = 0; j < cnt; ++j) {
    double s = acc[j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sums + base + j, s);
  }
}

// frame layout: [0..2] mu, [3..11] R row-major (column j = axis j), [12..14]
// principal variances (descending), [15] s, [16] mean count, [17] mean volume
__global__ void k_feat_frame(double* __restrict__ sums, double* __restrict__ frame, long long n,
                             int stage) {
  if (threadIdx.x != 0) return;
  if (stage == 0) {
    const double V = sums[0];
    frame[0] = sums[1] / V;
    frame[1] = sums[2] / V;
    frame[2] = sums[3] / V;
    frame[16] = sums[4] / (double)n;
    frame[17] = V / (double)n;
    return;
  }
  if (stage == 1) {  // cyclic Jacobi on the 3 x 3 covariance (Golub & Van Loan, Sec. 8.5)
    const double V = sums[0];
    double A[3][3] = {{sums[5] / V, sums[6] / V, sums[7] / V},
                      {sums[6] / V, sums[8] / V, sums[9] / V},
                      {sums[7] / V, sums[9] / V, sums[10] / V}};
    double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 50; ++sweep) {
      const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
      const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
      if (!(off > 1e-36 * dia)) break;
      for (int p = 0; p < 2; ++p)
        for (int q = p + 1; q < 3; ++q) {
          if (A[p][q] == 0.0) continue;
          const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
          const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
          for (int k = 0; k < 3; ++k) {  // A <- A J
            const double akp = A[k][p], akq = A[k][q];
            A[k][p] = c * akp - s * akq;
            A[k][q] = s * akp + c * akq;
          }
          for (int k = 0; k < 3; ++k) {  // A <- J^T A
            const double apk = A[p][k], aqk = A[q][k];
            A[p][k] = c * apk - s * aqk;
            A[q][k] = s * apk + c * aqk;
          }
          for (int k = 0; k < 3; ++k) {  // Q <- Q J
            const double qkp = Q[k][p], qkq = Q[k][q];
            Q[k][p] = c * qkp - s * qkq;
            Q[k][q] = s * qkp + c * qkq;
          }
        }
    }
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (A[ord[j]][ord[j]] > A[ord[i]][ord[i]]) {
          const int t = ord[i];
          ord[i] = ord[j];
          ord[j] = t;
        }
    for (int j = 0; j < 3; ++j) {
      frame[12 + j] = A[ord[j]][ord[j]];
      for (int k = 0; k < 3; ++k) frame[3 + 3 * k + j] = Q[k][ord[j]];
    }
    frame[15] = sqrt(frame[12] + frame[13] + frame[14]);
    return;
  }
  for (int j = 0; j < 3; ++j)  // stage 2: signs from the third moments
    if (sums[11 + j] < 0.0)
      for (int k = 0; k < 3; ++k) frame[3 + 3 * k + j] = -frame[3 + 3 * k + j];
}

__global__ void k_features(const float4* __restrict__ pos, const float* __restrict__ vol,
                           const long long* __restrict__ nptr, const int* __restrict__ nidx,
                           const int* __restrict__ perm, long long n,
                           const double* __restrict__ frame, float* __restrict__ feat) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float R[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) R[t] = (float)frame[3 + t];
  const float4 p = pos[r];
  float sx = 0.f, sy = 0.f, sz = 0.f, sxx = 0.f, sxy = 0.f, sxz = 0.f, syy = 0.f, syz = 0.f, szz = 0.f;
  const long long e0 = nptr[r], e1 = nptr[r + 1];
  for (long long e = e0; e < e1; ++e) {
    const float4 q = pos[nidx[e]];
    const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    sx += dx; sy += dy; sz += dz;
    sxx += dx * dx; sxy += dx * dy; sxz += dx * dz;
    syy += dy * dy; syz += dy * dz; szz += dz * dz;
  }
  const float inv = 1.f / (float)(e1 - e0);
  const float mx = sx * inv, my = sy * inv, mz = sz * inv;
  const float cxx = sxx * inv - mx * mx, cxy = sxy * inv - mx * my, cxz = sxz * inv - mx * mz;
  const float cyy = syy * inv - my * my, cyz = syz * inv - my * mz, czz = szz * inv - mz * mz;
  const double s = frame[15];
  const double ox = p.x - frame[0], oy = p.y - frame[1], oz = p.z - frame[2];
  float* f = feat + (long long)perm[r] * kF;
  const float ia = 1.f / p.w;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float r0 = R[j], r1 = R[3 + j], r2 = R[6 + j];
    f[j] = (float)((ox * frame[3 + j] + oy * frame[6 + j] + oz * frame[9 + j]) / s);
    f[3 + j] = (mx * r0 + my * r1 + mz * r2) * ia;
    const float q = r0 * (cxx * r0 + cxy * r1 + cxz * r2) + r1 * (cxy * r0 + cyy * r1 + cyz * r2) +
                    r2 * (cxz * r0 + cyz * r1 + czz * r2);
    f[6 + j] = q * ia * ia;
  }
  f[9] = (float)((double)(e1 - e0) / frame[16]);
  f[10] = (float)(p.w / s);
  f[11] = (float)(vol[r] / frame[17]);
  f[12] = (float)sqrt(frame[13] / frame[12]);
  f[13] = (float)sqrt(frame[14] / frame[12]);
  f[14] = (float)(log((double)n) / 16.0);
  f[15] = 1.f;
}

// column-major caller-order start block: network columns, then seeded guard columns
template <class T>
__global__ void k_pack_start(const float* __restrict__ y, long long n, int cols, int ncols_net,
                             unsigned long long seed, T* __restrict__ X0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * cols) return;
  const int j = (int)(t / n);
  const long long i = t % n;
  float v;
  if (j < ncols_net) {
    v = y[i * kO + j];
  } else {
    const unsigned long long r = splitmix(seed ^ ((unsigned long long)j << 40) ^ (unsigned long long)i);
    v = (float)((double)(r >> 11) * 0x1.0p-53 * 2.0 - 1.0);
  }
  X0[t] = (T)v;
}

// ------------------------------------------------------------------ host side
unsigned blocks(long long work, int tb = 256) { return (unsigned)((work + tb - 1) / tb); }

void net_reserve(ff_net* w, long long n) {
  if (n <= w->cap) return;
  w->f16.ensure(sizeof(bf16) * n * kF);
  w->h1.ensure(sizeof(bf16) * n * kH1);
  w->h3.ensure(sizeof(bf16) * n * kH3);
  w->h4.ensure(sizeof(bf16) * n * kH4);
  w->y.ensure(sizeof(float) * n * kO);
  w->dy.ensure(sizeof(float) * n * kO);
  w->dh4.ensure(sizeof(float) * n * kH4);
  w->dh3.ensure(sizeof(float) * n * kH3);
  w->dh1.ensure(sizeof(float) * n * kH1);
  w->cap = n;
}

// forward on stream st; the output block lands in w->y (n x 32, FP32)
void net_forward(ff_net* w, cudaStream_t st, const float* feat, long long n) {
  net_reserve(w, n);
  const bf16* W = w->w16.as<bf16>();
  const float* th = w->master.as<float>();
  bf16* f16 = w->f16.as<bf16>();
  (k_f2bf<<<blocks(n * kF), 256, 0, st>>>(feat, f16, n * kF), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  Gemm g;
  // h1 = relu(f W1^T + b1)
  g = Gemm{};
  g.M = (int)n; g.N = kH1; g.K = kF;
  g.A = f16; g.a16 = 1; g.sam = kF; g.sak = 1;
  g.B = W + oW1; g.b16 = 1; g.sbk = 1; g.sbn = kF;
  g.bias = th + oB1; g.relu = 1;
  g.C = w->h1.p; g.c16 = 1; g.ldc = kH1;
  gemm(st, g);
  // g = max_p relu(h1 W2^T + b2)
  FF_CUDA(cudaMemsetAsync(w->pool.p, 0, sizeof(unsigned long long) * kH2, st));
  g = Gemm{};
  g.M = (int)n; g.N = kH2; g.K = kH1;
  g.A = w->h1.p; g.a16 = 1; g.sam = kH1; g.sak = 1;
  g.B = W + oW2; g.b16 = 1; g.sbk = 1; g.sbn = kH1;
  g.bias = th + oB2; g.relu = 1;
  g.pool = w->pool.as<unsigned long long>();
  gemm(st, g);
  (k_pool_finish<<<1, kH2, 0, st>>>(w->pool.as<unsigned long long>(), w->g.as<float>(),
                                     w->arg.as<int>()), ::ff::note_launch());
  (k_global_term<<<kH3 / 8, 256, 0, st>>>(W, w->g.as<float>(), th + oB3, w->c3.as<float>()),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  // h3 = relu(h1 W3[:, :128]^T + (W3[:, 128:] g + b3))
  g = Gemm{};
  g.M = (int)n; g.N = kH3; g.K = kH1;
  g.A = w->h1.p; g.a16 = 1; g.sam = kH1; g.sak = 1;
  g.B = W + oW3; g.b16 = 1; g.sbk = 1; g.sbn = kZ;
  g.bias = w->c3.as<float>(); g.relu = 1;
  g.C = w->h3.p; g.c16 = 1; g.ldc = kH3;
  gemm(st, g);
  // h4 = relu(h3 W4^T + b4)
  g = Gemm{};
  g.M = (int)n; g.N = kH4; g.K = kH3;
  g.A = w->h3.p; g.a16 = 1; g.sam = kH3; g.sak = 1;
  g.B = W + oW4; g.b16 = 1; g.sbk = 1; g.sbn = kH3;
  g.bias = th + oB4; g.relu = 1;
  g.C = w->h4.p; g.c16 = 1; g.ldc = kH4;
  gemm(st, g);
  // y = h4 W5^T + b5
  g = Gemm{};
  g.M = (int)n; g.N = kO; g.K = kH4;
  g.A = w->h4.p; g.a16 = 1; g.sam = kH4; g.sak = 1;
  g.B = W + oW5; g.b16 = 1; g.sbk = 1; g.sbn = kH4;
  g.bias = th + oB5;
  g.C = w->y.p; g.ldc = kO;
  gemm(st, g);
}

// loss and dL/dy (into w->dy); the loss lands in w->h_small[0] after a sync
void net_loss(ff_net* w, cudaStream_t st, const float* vol, long long n, const float* C, int m) {
  double* sums = w->lsum.as<double>();
  FF_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (kLossEntries + 1), st));
  const unsigned gb = (unsigned)std::min<long long>(ceil_div(n, 32), 2LL * sm_count());
  (k_loss_gram<<<gb, 256, 0, st>>>(w->y.as<float>(), C, vol, n, m, sums), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  float* P1 = w->small.as<float>();
  float* P2 = P1 + kMaxModes * kO;
  double* scal = reinterpret_cast<double*>(P2 + kO * kO);
  (k_loss_small<<<1, 1024, 0, st>>>(sums, m, P1, P2, scal), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_loss_dy<<<blocks(n, 128), 128, 0, st>>>(w->y.as<float>(), C, vol, n, m, P1, P2, scal,
                                              w->dy.as<float>()), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  FF_CUDA(cudaMemcpyAsync(w->h_small, scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
}

// gradient of the loss through the network into w->grad (zeroed here)
void net_backward(ff_net* w, cudaStream_t st, long long n) {
  const bf16* W = w->w16.as<bf16>();
  float* gr = w->grad.as<float>();
  FF_CUDA(cudaMemsetAsync(gr, 0, sizeof(float) * kP, st));
  const unsigned cb = (unsigned)ceil_div(n, 256);
  Gemm g;
  // layer 5
  g = Gemm{};
  g.M = kO; g.N = kH4; g.K = (int)n;
  g.A = w->dy.p; g.sam = 1; g.sak = kO;
  g.B = w->h4.p; g.b16 = 1; g.sbk = kH4; g.sbn = 1;
  g.C = gr + oW5; g.ldc = kH4; g.atomic = 1;
  gemm(st, g);
  (k_colsum<<<cb, 256, 0, st>>>(w->dy.as<float>(), n, kO, gr + oB5), ::ff::note_launch());
  g = Gemm{};
  g.M = (int)n; g.N = kH4; g.K = kO;
  g.A = w->dy.p; g.sam = kO; g.sak = 1;
  g.B = W + oW5; g.b16 = 1; g.sbk = kH4; g.sbn = 1;
  g.mask = w->h4.as<bf16>(); g.ldmask = kH4;
  g.C = w->dh4.p; g.ldc = kH4;
  gemm(st, g);
  // layer 4
  g = Gemm{};
  g.M = kH4; g.N = kH3; g.K = (int)n;
  g.A = w->dh4.p; g.sam = 1; g.sak = kH4;
  g.B = w->h3.p; g.b16 = 1; g.sbk = kH3; g.sbn = 1;
  g.C = gr + oW4; g.ldc = kH3; g.atomic = 1;
  gemm(st, g);
  (k_colsum<<<cb, 256, 0, st>>>(w->dh4.as<float>(), n, kH4, gr + oB4), ::ff::note_launch());
  g = Gemm{};
  g.M = (int)n; g.N = kH3; g.K = kH4;
  g.A = w->dh4.p; g.sam = kH4; g.sak = 1;
  g.B = W + oW4; g.b16 = 1; g.sbk = kH3; g.sbn = 1;
  g.mask = w->h3.as<bf16>(); g.ldmask = kH3;
  g.C = w->dh3.p; g.ldc = kH3;
  gemm(st, g);
  // layer 3: per-particle half, then the global half through g
  g = Gemm{};
  g.M = kH3; g.N = kH1; g.K = (int)n;
  g.A = w->dh3.p; g.sam = 1; g.sak = kH3;
  g.B = w->h1.p; g.b16 = 1; g.sbk = kH1; g.sbn = 1;
  g.C = gr + oW3; g.ldc = kZ; g.atomic = 1;
  gemm(st, g);
  (k_colsum<<<cb, 256, 0, st>>>(w->dh3.as<float>(), n, kH3, gr + oB3), ::ff::note_launch());
  (k_outer_w3<<<blocks(kH3 * kH2), 256, 0, st>>>(gr + oB3, w->g.as<float>(), gr),
   ::ff::note_launch());
  (k_dg<<<1, kH2, 0, st>>>(W, gr + oB3, w->dg.as<float>()), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  g = Gemm{};
  g.M = (int)n; g.N = kH1; g.K = kH3;
  g.A = w->dh3.p; g.sam = kH3; g.sak = 1;
  g.B = W + oW3; g.b16 = 1; g.sbk = kZ; g.sbn = 1;
  g.C = w->dh1.p; g.ldc = kH1;
  gemm(st, g);
  // layer 2 through the max pool, then the ReLU of h1
  (k_pool_backward<<<kH2, kH1, 0, st>>>(w->g.as<float>(), w->arg.as<int>(), w->dg.as<float>(),
                                         w->h1.as<bf16>(), W, gr, w->dh1.as<float>()),
   ::ff::note_launch());
  (k_relu_mask<<<blocks(n * kH1), 256, 0, st>>>(w->dh1.as<float>(), w->h1.as<bf16>(), n * kH1),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  // layer 1
  g = Gemm{};
  g.M = kH1; g.N = kF; g.K = (int)n;
  g.A = w->dh1.p; g.sam = 1; g.sak = kH1;
  g.B = w->f16.p; g.b16 = 1; g.sbk = kF; g.sbn = 1;
  g.C = gr + oW1; g.ldc = kF; g.atomic = 1;
  gemm(st, g);
  (k_colsum<<<cb, 256, 0, st>>>(w->dh1.as<float>(), n, kH1, gr + oB1), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

template <class F>
ff_status net_guarded(ff_net* w, F&& f) {
  if (!w) return FF_ERR_INVALID_ARG;
  w->err.clear();
  try {
    FF_CUDA(cudaSetDevice(w->device));
    f();
    return FF_OK;
  } catch (const ff::Error& e) {
    w->err = e.what();
    (void)cudaGetLastError();
    return e.code;
  } catch (const std::exception& e) {
    w->err = e.what();
    return FF_ERR_CUDA;
  }
}

void check_cloud(const float* feat, const float* vol, long long n, const float* modes, int m) {
  FF_REQUIRE(feat && vol && modes && n >= 1, FF_ERR_INVALID_ARG, "null input or n < 1");
  FF_REQUIRE(m >= 1 && m <= kMaxModes && m < n, FF_ERR_INVALID_ARG, "m must be in [1, 32] and < n");
  FF_REQUIRE(n < (1LL << 31), FF_ERR_INVALID_ARG, "n too large");
}

}  // namespace

void warmstart_features(ff_ctx* c, float* feat);

// warm-start block for the eigensolver
void warmstart_block(ff_ctx* c, ff_net* w, int k, const ff_eig_opts& o, void* X0) {
  cudaStream_t st = c->stream;
  const long long n = c->n;
  float* feat = reinterpret_cast<float*>(c->scratch[4].ensure(sizeof(float) * n * kF));
  warmstart_features(c, feat);
  net_forward(w, st, feat, n);
  const int kw = o.exclude_constant ? k : k - 1;
  const int cols = kw + std::max(0, o.guard);
  const int net_cols = std::min(cols, kO);
  if (c->prec == FF_PREC_FP64)
    (k_pack_start<double><<<blocks(n * cols), 256, 0, st>>>(w->y.as<float>(), n, cols, net_cols,
                                                            o.seed + 0x5bd1e995ULL,
                                                            static_cast<double*>(X0)),
     ::ff::note_launch());
  else
    (k_pack_start<float><<<blocks(n * cols), 256, 0, st>>>(w->y.as<float>(), n, cols, net_cols,
                                                           o.seed + 0x5bd1e995ULL,
                                                           static_cast<float*>(X0)),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

void warmstart_features(ff_ctx* c, float* feat) {
  cudaStream_t st = c->stream;
  const long long n = c->n;
  double* sums = reinterpret_cast<double*>(c->scratch[5].ensure(sizeof(double) * 40));
  double* frame = sums + 16;
  FF_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 40, st));
  const unsigned gb = (unsigned)std::min<long long>(ceil_div(n, 256), 4LL * sm_count());
  const float4* pos = c->pos.as<float4>();
  const float* vol = c->vol.as<float>();
  const long long* nptr = c->nbr_ptr.as<long long>();
  (k_feat_moments<<<gb, 256, 0, st>>>(pos, vol, nptr, n, 0, frame, sums), ::ff::note_launch());
  (k_feat_frame<<<1, 32, 0, st>>>(sums, frame, n, 0), ::ff::note_launch());
  (k_feat_moments<<<gb, 256, 0, st>>>(pos, vol, nptr, n, 1, frame, sums), ::ff::note_launch());
  (k_feat_frame<<<1, 32, 0, st>>>(sums, frame, n, 1), ::ff::note_launch());
  (k_feat_moments<<<gb, 256, 0, st>>>(pos, vol, nptr, n, 2, frame, sums), ::ff::note_launch());
  (k_feat_frame<<<1, 32, 0, st>>>(sums, frame, n, 2), ::ff::note_launch());
  (k_features<<<blocks(n), 256, 0, st>>>(pos, vol, nptr, c->nbr_idx.as<int>(), c->perm.as<int>(),
                                          n, frame, feat), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

}  // namespace ff

// ------------------------------------------------------------------ C ABI
extern "C" {

int64_t ff_net_num_params(void) { return ff::kP; }

ff_status ff_net_create(ff_net** out, int device, void* cuda_stream) {
  if (!out) return FF_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    (void)cudaGetLastError();
    return FF_ERR_INVALID_ARG;
  }
  ff_net* w = new ff_net();
  w->device = device;
  w->stream = static_cast<cudaStream_t>(cuda_stream);
  const ff_status s = ff::net_guarded(w, [&] {
    using namespace ff;
    w->master.ensure(sizeof(float) * kP);
    w->m1.ensure(sizeof(float) * kP);
    w->m2.ensure(sizeof(float) * kP);
    w->grad.ensure(sizeof(float) * kP);
    w->w16.ensure(sizeof(bf16) * kP);
    w->pool.ensure(sizeof(unsigned long long) * kH2);
    w->g.ensure(sizeof(float) * kH2);
    w->arg.ensure(sizeof(int) * kH2);
    w->c3.ensure(sizeof(float) * kH3);
    w->dg.ensure(sizeof(float) * kH2);
    w->lsum.ensure(sizeof(double) * (kLossEntries + 1));
    w->small.ensure(sizeof(float) * (kMaxModes * kO + kO * kO) + sizeof(double) * 4);
    FF_CUDA(cudaMallocHost(&w->h_small, sizeof(double) * 4));
    FF_CUDA(cudaMemsetAsync(w->master.p, 0, sizeof(float) * kP, w->stream));
    FF_CUDA(cudaMemsetAsync(w->m1.p, 0, sizeof(float) * kP, w->stream));
    FF_CUDA(cudaMemsetAsync(w->m2.p, 0, sizeof(float) * kP, w->stream));
    FF_CUDA(cudaMemsetAsync(w->w16.p, 0, sizeof(bf16) * kP, w->stream));
    FF_CUDA(cudaStreamSynchronize(w->stream));
  });
  if (s != FF_OK) {
    ff_net_destroy(w);
    return s;
  }
  *out = w;
  return FF_OK;
}

void ff_net_destroy(ff_net* w) {
  if (!w) return;
  cudaSetDevice(w->device);
  if (w->h_small) cudaFreeHost(w->h_small);
  delete w;
}

const char* ff_net_last_error(const ff_net* w) { return w ? w->err.c_str() : "null network"; }

ff_status ff_net_init(ff_net* w, uint64_t seed) {
  return ff::net_guarded(w, [&] {
    using namespace ff;
    (k_init<<<blocks(kP), 256, 0, w->stream>>>(w->master.as<float>(), w->w16.as<bf16>(), seed),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    FF_CUDA(cudaMemsetAsync(w->m1.p, 0, sizeof(float) * kP, w->stream));
    FF_CUDA(cudaMemsetAsync(w->m2.p, 0, sizeof(float) * kP, w->stream));
    w->t = 0;
    FF_CUDA(cudaStreamSynchronize(w->stream));
  });
}

ff_status ff_net_set_params(ff_net* w, const float* params, int64_t count) {
  return ff::net_guarded(w, [&] {
    using namespace ff;
    FF_REQUIRE(params && count == kP, FF_ERR_INVALID_ARG, "params must hold ff_net_num_params() floats");
    FF_CUDA(cudaMemcpyAsync(w->master.p, params, sizeof(float) * kP, cudaMemcpyHostToDevice, w->stream));
    (k_f2bf<<<blocks(kP), 256, 0, w->stream>>>(w->master.as<float>(), w->w16.as<bf16>(), kP),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    FF_CUDA(cudaMemsetAsync(w->m1.p, 0, sizeof(float) * kP, w->stream));
    FF_CUDA(cudaMemsetAsync(w->m2.p, 0, sizeof(float) * kP, w->stream));
    w->t = 0;
    FF_CUDA(cudaStreamSynchronize(w->stream));
  });
}

ff_status ff_net_get_params(ff_net* w, float* params, int64_t count) {
  return ff::net_guarded(w, [&] {
    FF_REQUIRE(params && count == ff::kP, FF_ERR_INVALID_ARG, "params must hold ff_net_num_params() floats");
    FF_CUDA(cudaMemcpyAsync(params, w->master.p, sizeof(float) * ff::kP, cudaMemcpyDeviceToHost, w->stream));
    FF_CUDA(cudaStreamSynchronize(w->stream));
  });
}

ff_status ff_net_forward(ff_net* w, const float* feat, int64_t n, float* out) {
  return ff::net_guarded(w, [&] {
    FF_REQUIRE(feat && out && n >= 1 && n < (1LL << 31), FF_ERR_INVALID_ARG, "bad arguments");
    ff::net_forward(w, w->stream, feat, n);
    FF_CUDA(cudaMemcpyAsync(out, w->y.p, sizeof(float) * n * ff::kO, cudaMemcpyDeviceToDevice, w->stream));
    FF_CUDA(cudaStreamSynchronize(w->stream));
  });
}

ff_status ff_net_loss_grad(ff_net* w, const float* feat, const float* vol, int64_t n,
                           const float* modes, int m, double* loss, float* grad) {
  return ff::net_guarded(w, [&] {
    ff::check_cloud(feat, vol, n, modes, m);
    ff::net_forward(w, w->stream, feat, n);
    ff::net_loss(w, w->stream, vol, n, modes, m);
    ff::net_backward(w, w->stream, n);
    if (grad)
      FF_CUDA(cudaMemcpyAsync(grad, w->grad.p, sizeof(float) * ff::kP, cudaMemcpyDeviceToHost, w->stream));
    FF_CUDA(cudaStreamSynchronize(w->stream));
    if (loss) *loss = w->h_small[0];
  });
}

ff_status ff_net_train_step(ff_net* w, const float* feat, const float* vol, int64_t n,
                            const float* modes, int m, float lr, double* loss) {
  return ff::net_guarded(w, [&] {
    using namespace ff;
    check_cloud(feat, vol, n, modes, m);
    FF_REQUIRE(lr > 0.f && std::isfinite(lr), FF_ERR_INVALID_ARG, "lr must be > 0");
    net_forward(w, w->stream, feat, n);
    net_loss(w, w->stream, vol, n, modes, m);
    net_backward(w, w->stream, n);
    w->t += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)w->t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)w->t));
    (k_adam<<<blocks(kP), 256, 0, w->stream>>>(w->master.as<float>(), w->m1.as<float>(),
                                                 w->m2.as<float>(), w->grad.as<float>(),
                                                 w->w16.as<bf16>(), kP, lr, c1, c2),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    FF_CUDA(cudaStreamSynchronize(w->stream));
    if (loss) *loss = w->h_small[0];
  });
}

}  // extern "C"
