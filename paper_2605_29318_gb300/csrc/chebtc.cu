// Tensor-core step of the Chebyshev preconditioner (internal).
//
// The preconditioner applies H (FP32 values) to 40-column blocks of BF16
// direction vectors several hundred times per solve; on CUDA cores that step
// is bound by instruction issue (a gathered row and a multiply-add per nonzero
// and column).  Rows in the internal (cell) order are spatially local, so 16
// consecutive rows share most of their columns: per block of 16 rows the H
// entries are laid out as a dense 16 x K BF16 tile over the sorted union of the
// block's columns (K rounded up to 16; on the 50k torus K averages ~450 and
// ~35% of the tile is nonzero), stored in the A-fragment order of
// mma.m16n8k16 so that a k-step is one 16-byte load per lane.  A step gathers the 16 union rows of the
// direction block into shared memory once (16-byte asynchronous copies),
// forms the B fragments with ldmatrix.trans and accumulates in FP32.
//
// The tile entries are the BF16 roundings of H's values; the row sums hs used
// by the step's difference form (H d)_k = sum_l h_kl d_l - (sum_l h_kl) d_k are
// sums of the same rounded values, so the rounded operator still maps the
// constant vector to zero.  The preconditioner is a polynomial in the rounded
// matrix, which is symmetric like H.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kTcRows = 16;            // rows per block (the M of the MMA)
constexpr int kTcMaxWords = 8192;      // bitmap words: column spans up to 262144
constexpr unsigned kFullMask = 0xffffffffu;

// column span of each block and the number of k-steps its union needs
__global__ void __launch_bounds__(256)
    k_tc_count(const long long* __restrict__ ptr, const int* __restrict__ col, int n,
               int* __restrict__ nks, int* __restrict__ lo_out, int* __restrict__ words_out) {
  extern __shared__ unsigned bm[];
  __shared__ int s_min, s_max, s_cnt;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int k0 = b * kTcRows, k1 = min(n, k0 + kTcRows);
  const long long e0 = ptr[k0], e1 = ptr[k1];
  if (tid == 0) {
    s_min = 0x7fffffff;
    s_max = -1;
    s_cnt = 0;
  }
  __syncthreads();
  int mn = 0x7fffffff, mx = -1;
  for (long long e = e0 + tid; e < e1; e += blockDim.x) {
    const int c = col[e];
    mn = min(mn, c);
    mx = max(mx, c);
  }
  atomicMin(&s_min, mn);
  atomicMax(&s_max, mx);
  __syncthreads();
  const int lo = s_min;
  const int words = s_max >= lo ? (s_max - lo) / 32 + 1 : 0;
  if (words > kTcMaxWords) {
    if (tid == 0) nks[b] = -1;
    return;
  }
  for (int wd = tid; wd < words; wd += blockDim.x) bm[wd] = 0u;
  __syncthreads();
  for (long long e = e0 + tid; e < e1; e += blockDim.x) {
    const int off = col[e] - lo;
    atomicOr(&bm[off >> 5], 1u << (off & 31));
  }
  __syncthreads();
  int cnt = 0;
  for (int wd = tid; wd < words; wd += blockDim.x) cnt += __popc(bm[wd]);
  atomicAdd(&s_cnt, cnt);
  __syncthreads();
  if (tid == 0) {
    nks[b] = (s_cnt + 15) / 16;
    lo_out[b] = lo;
    words_out[b] = words;
  }
}

// union columns, tile entries (fragment order) and rounded row sums
__global__ void __launch_bounds__(256)
    k_tc_fill(const long long* __restrict__ ptr, const int* __restrict__ col,
              const float* __restrict__ hv, int n, const int* __restrict__ kofs,
              const int* __restrict__ lo_in, const int* __restrict__ words_in,
              int* __restrict__ ucol, unsigned short* __restrict__ tile, float* __restrict__ hs) {
  extern __shared__ unsigned smw[];
  __shared__ int wsum[8];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k0 = b * kTcRows, k1 = min(n, k0 + kTcRows);
  const long long e0 = ptr[k0], e1 = ptr[k1];
  const int lo = lo_in[b], words = words_in[b];
  const long long s0 = kofs[b];
  const int ns = kofs[b + 1] - kofs[b];
  unsigned* bm = smw;          // words
  unsigned* pre = smw + words; // words: union entries before each word
  for (int wd = tid; wd < words; wd += blockDim.x) bm[wd] = 0u;
  // this block's tile region to zero (16-byte units: 32 per k-step)
  uint4* t4 = reinterpret_cast<uint4*>(tile) + s0 * 32;
  for (int q = tid; q < ns * 32; q += blockDim.x) t4[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (long long e = e0 + tid; e < e1; e += blockDim.x) {
    const int off = col[e] - lo;
    atomicOr(&bm[off >> 5], 1u << (off & 31));
  }
  __syncthreads();
  // exclusive scan of the popcounts: each thread a contiguous run of words
  const int per = (words + blockDim.x - 1) / blockDim.x;
  const int w0 = min(words, tid * per), w1 = min(words, w0 + per);
  int run = 0;
  for (int wd = w0; wd < w1; ++wd) run += __popc(bm[wd]);
  int incl = run;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  int base = 0;
  for (int q = 0; q < wid; ++q) base += wsum[q];
  int acc = base + incl - run;
  for (int wd = w0; wd < w1; ++wd) {
    pre[wd] = acc;
    acc += __popc(bm[wd]);
  }
  int total = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) total += wsum[q];
  __syncthreads();
  // union columns in ascending order; padding repeats the first column
  int* uc = ucol + s0 * 16;
  for (int wd = tid; wd < words; wd += blockDim.x) {
    unsigned bits = bm[wd];
    int r = pre[wd];
    while (bits) {
      const int j = __ffs(bits) - 1;
      uc[r++] = lo + 32 * wd + j;
      bits &= bits - 1;
    }
  }
  for (int r = total + tid; r < ns * 16; r += blockDim.x) uc[r] = lo;
  // entries: warp wid takes rows wid and wid + 8 of the block
  for (int rr = wid; rr < kTcRows; rr += 8) {
    const int k = k0 + rr;
    if (k >= n) break;
    float sum = 0.f;
    for (long long e = ptr[k] + lane; e < ptr[k + 1]; e += 32) {
      const int off = col[e] - lo;
      const int rank = pre[off >> 5] + __popc(bm[off >> 5] & ((1u << (off & 31)) - 1u));
      const int s = rank >> 4, kk = rank & 15;
      const int fl = (rr & 7) * 4 + ((kk & 7) >> 1);  // fragment lane
      const int reg = (rr >> 3) + 2 * (kk >> 3);      // a0..a3
      const __nv_bfloat16 q = __float2bfloat16(hv[e]);
      tile[((s0 + s) * 32 + fl) * 8 + reg * 2 + (kk & 1)] = __bfloat16_as_ushort(q);
      sum += __bfloat162float(q);
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(kFullMask, sum, o);
    if (lane == 0) hs[k] = sum;
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint4& a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// One block of WB warps per 16-row block; warp w takes the block's k-steps
// w, w + WB, ...: three staging buffers per warp keep the union rows of two
// later steps in flight while a step is multiplied (their union columns and
// A fragments loaded earlier still).  The warps' partial 16 x m products are
// summed through the same shared memory and each warp finishes a share of the
// column tiles: res -= D^-1 (H d), d' = c1 d + c2 res (BF16), x += d'.
// WB = 4 where the row blocks fill the GPU; WB = 16 where they are few (a
// K x K pencil of a two-set cloud: 63 row blocks for K = 1,000), so that each
// warp's chain of k-steps is four times shorter.
template <int WB>
constexpr size_t tc_step_smem(int NT) {
  return std::max<size_t>((size_t)WB * 3 * kTcRows * 8 * NT * 2, (size_t)WB * 32 * 4 * NT * 4);
}

template <int NT, int WB>
__global__ void __launch_bounds__(32 * WB)
    k_cheb_step_tc(const int* __restrict__ kofs, const int* __restrict__ ucol,
                   const uint4* __restrict__ tile, const float* __restrict__ hs,
                   const float* __restrict__ hdiag, int n, const __nv_bfloat16* __restrict__ din,
                   __nv_bfloat16* __restrict__ dout, float* __restrict__ x,
                   float* __restrict__ res, float c1, float c2) {
  constexpr int kWB = WB;
  constexpr int m = 8 * NT, PIECES = kTcRows * NT, ITERS = (PIECES + 31) / 32, NB = 3;
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(smem) + w * NB * kTcRows * m;
  const int s0 = kofs[b], ns = kofs[b + 1] - s0;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  auto ucol_of = [&](int s) {
    return (s < ns && lane < 16) ? __ldg(ucol + (long long)(s0 + s) * 16 + lane) : 0;
  };
  auto tile_of = [&](int s, const uint4& dflt) {
    return s < ns ? __ldg(tile + (long long)(s0 + s) * 32 + lane) : dflt;
  };
  auto stage_step = [&](int buf, int u) {  // u: lane r < 16 holds the step's union column r
    __nv_bfloat16* dst = stage + buf * kTcRows * m;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
      const int p = it * 32 + lane;
      const int rr = min(p / NT, kTcRows - 1), pc = p % NT;
      const int row = __shfl_sync(kFullMask, u, rr);
      if (p < PIECES) cp_async16(dst + rr * m + pc * 8, din + (long long)row * m + pc * 8);
    }
  };
  // Registers rotate without moves (a move would wait for its load): A[p]
  // holds the fragments of the step multiplied in phase p, U[p] the union
  // columns of the step staged in phase p; each is reloaded right after use
  // for the step three phases on.
  int s = w;
  if (s < ns) stage_step(0, ucol_of(s));
  cp_commit();
  if (s + kWB < ns) stage_step(1, ucol_of(s + kWB));
  cp_commit();
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  uint4 A[3] = {tile_of(s, zero4), tile_of(s + kWB, zero4), tile_of(s + 2 * kWB, zero4)};
  int U[3] = {ucol_of(s + 2 * kWB), ucol_of(s + 3 * kWB), ucol_of(s + 4 * kWB)};
  auto phase = [&](const int p) {
    if (s + 2 * kWB < ns) stage_step((p + 2) % 3, U[p]);
    cp_commit();
    U[p] = ucol_of(s + 5 * kWB);
    cp_wait2();
    __syncwarp();
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(stage + p * kTcRows * m);
    const int mat = lane >> 3, krow = (mat & 1) * 8 + (lane & 7);
#pragma unroll
    for (int j = 0; j + 1 < NT; j += 2) {
      unsigned r0, r1, r2, r3;
      const unsigned addr = sbase + (unsigned)(krow * m * 2 + (j + (mat >> 1)) * 16);
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                   : "r"(addr));
      mma_bf16(acc[j], A[p], r0, r1);
      mma_bf16(acc[j + 1], A[p], r2, r3);
    }
    if (NT & 1) {
      constexpr int j = NT - 1;
      unsigned r0, r1;
      const unsigned addr =
          sbase + (unsigned)(((lane >> 3) & 1) * 8 * m * 2 + (lane & 7) * m * 2 + j * 16);
      asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                   : "=r"(r0), "=r"(r1)
                   : "r"(addr));
      mma_bf16(acc[j], A[p], r0, r1);
    }
    __syncwarp();
    A[p] = tile_of(s + 3 * kWB, zero4);
    s += kWB;
  };
  while (s < ns) {
    phase(0);
    if (s >= ns) break;
    phase(1);
    if (s >= ns) break;
    phase(2);
  }
  cp_wait0();
  __syncthreads();  // every warp is done with its staging buffers
  float* red = reinterpret_cast<float*>(smem);  // [kWB][32][4 NT]
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[(w * 32 + lane) * 4 * NT + 4 * j + q] = acc[j][q];
  __syncthreads();
  // warp w finishes the column tiles j = w, w + kWB, ...
  const int g = lane >> 2, t = lane & 3;
  for (int j = w; j < NT; j += kWB) {
    float c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float t = 0.f;
      for (int v = 0; v < kWB; ++v) t += red[(v * 32 + lane) * 4 * NT + 4 * j + q];
      c[q] = t;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = b * kTcRows + g + 8 * h;
      if (k >= n) continue;
      const float dinv = 1.0f / hdiag[k], hsk = hs[k];
      const long long o = (long long)k * m + 8 * j + 2 * t;
      const __nv_bfloat162 dk2 = *reinterpret_cast<const __nv_bfloat162*>(din + o);
      const float2 dk = __bfloat1622float2(dk2);
      float2 r = *reinterpret_cast<const float2*>(res + o);
      float2 xx = *reinterpret_cast<const float2*>(x + o);
      r.x -= (c[2 * h] - hsk * dk.x) * dinv;
      r.y -= (c[2 * h + 1] - hsk * dk.y) * dinv;
      const __nv_bfloat16 q0 = __float2bfloat16(c1 * dk.x + c2 * r.x);
      const __nv_bfloat16 q1 = __float2bfloat16(c1 * dk.y + c2 * r.y);
      xx.x += __bfloat162float(q0);
      xx.y += __bfloat162float(q1);
      *reinterpret_cast<float2*>(res + o) = r;
      *reinterpret_cast<float2*>(x + o) = xx;
      __nv_bfloat162 qq;
      qq.x = q0;
      qq.y = q1;
      *reinterpret_cast<__nv_bfloat162*>(dout + o) = qq;
    }
  }
}

}  // namespace

bool cheb_tc_build(ff_ctx* c) {
  cudaStream_t st = c->stream;
  c->tc_ksteps = 0;
  const long long n = c->n;
  if (n <= 0 || n >= (1LL << 30)) return false;
  const int nblk = (int)((n + kTcRows - 1) / kTcRows);
  int* nks = reinterpret_cast<int*>(c->scratch[4].ensure(sizeof(int) * 3 * (size_t)nblk));
  int* lo = nks + nblk;
  int* words = lo + nblk;
  set_max_dyn_smem((const void*)k_tc_count, (int)(sizeof(unsigned) * kTcMaxWords));
  set_max_dyn_smem((const void*)k_tc_fill, (int)(2 * sizeof(unsigned) * kTcMaxWords));
  (k_tc_count<<<nblk, 256, sizeof(unsigned) * kTcMaxWords, st>>>(
       c->a_ptr.as<long long>(), c->a_col.as<int>(), (int)n, nks, lo, words),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  std::vector<int> h(nblk);
  FF_CUDA(cudaMemcpyAsync(h.data(), nks, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  std::vector<int> ofs(nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) {
    if (h[b] < 0) return false;  // a block's columns span too far: CUDA-core step
    ofs[b + 1] = ofs[b] + h[b];
    if (ofs[b + 1] >= (1 << 26)) return false;
  }
  const long long S = ofs[nblk];
  int* kofs = reinterpret_cast<int*>(c->tc_kofs.ensure(sizeof(int) * (nblk + 1)));
  FF_CUDA(cudaMemcpyAsync(kofs, ofs.data(), sizeof(int) * (nblk + 1), cudaMemcpyHostToDevice, st));
  int* uc = reinterpret_cast<int*>(c->tc_ucol.ensure(sizeof(int) * 16 * (size_t)std::max(S, 1LL)));
  auto* tl = reinterpret_cast<unsigned short*>(c->tc_tile.ensure(512 * (size_t)std::max(S, 1LL)));
  float* hs = reinterpret_cast<float*>(c->tc_hs.ensure(sizeof(float) * n));
  (k_tc_fill<<<nblk, 256, 2 * sizeof(unsigned) * kTcMaxWords, st>>>(
       c->a_ptr.as<long long>(), c->a_col.as<int>(), c->h_f32.as<float>(), (int)n, kofs, lo,
       words, uc, tl, hs),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  FF_CUDA(cudaStreamSynchronize(st));
  c->tc_ksteps = S;
  return true;
}

bool cheb_step_tc(cudaStream_t st, const ff_ctx* c, int m, const void* din, void* dout, float* x,
                  float* res, float c1, float c2) {
  // widths 8..120 in steps of 8 (the staging buffers stay in static shared memory)
  if (c->tc_ksteps <= 0 || m % 8 != 0 || m < 8 || m > 120 || c->n * m >= (1LL << 31)) return false;
  ProfScope ps(kProfPrecond);
  const int nblk = (int)((c->n + kTcRows - 1) / kTcRows);
  const auto* bi = static_cast<const __nv_bfloat16*>(din);
  auto* bo = static_cast<__nv_bfloat16*>(dout);
  const bool few = nblk < 2 * sm_count();
  auto go = [&](auto nt) {
    constexpr int NT = decltype(nt)::value;
    if (few) {
      const size_t sm = tc_step_smem<16>(NT);
      set_max_dyn_smem((const void*)k_cheb_step_tc<NT, 16>, (int)sm);
      (k_cheb_step_tc<NT, 16><<<nblk, 32 * 16, sm, st>>>(
           c->tc_kofs.as<int>(), c->tc_ucol.as<int>(),
           reinterpret_cast<const uint4*>(c->tc_tile.p), c->tc_hs.as<float>(),
           c->hdiag_f32.as<float>(), (int)c->n, bi, bo, x, res, c1, c2),
       ::ff::note_launch());
    } else {
      const size_t sm = tc_step_smem<4>(NT);
      set_max_dyn_smem((const void*)k_cheb_step_tc<NT, 4>, (int)sm);
      (k_cheb_step_tc<NT, 4><<<nblk, 32 * 4, sm, st>>>(
           c->tc_kofs.as<int>(), c->tc_ucol.as<int>(),
           reinterpret_cast<const uint4*>(c->tc_tile.p), c->tc_hs.as<float>(),
           c->hdiag_f32.as<float>(), (int)c->n, bi, bo, x, res, c1, c2),
       ::ff::note_launch());
    }
  };
#define FF_TC(NT) go(std::integral_constant<int, NT>{})
  switch (m / 8) {
    case 1: FF_TC(1); break;
    case 2: FF_TC(2); break;
    case 3: FF_TC(3); break;
    case 4: FF_TC(4); break;
    case 5: FF_TC(5); break;
    case 6: FF_TC(6); break;
    case 7: FF_TC(7); break;
    case 8: FF_TC(8); break;
    case 9: FF_TC(9); break;
    case 10: FF_TC(10); break;
    case 11: FF_TC(11); break;
    case 12: FF_TC(12); break;
    case 13: FF_TC(13); break;
    case 14: FF_TC(14); break;
    default: FF_TC(15); break;
  }
#undef FF_TC
  FF_LAUNCH_CHECK();
  return true;
}

}  // namespace ff
