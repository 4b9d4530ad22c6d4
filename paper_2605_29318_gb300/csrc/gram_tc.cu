// Gram products of the Rayleigh-Ritz step on the 5th-generation tensor cores
// (tcgen05), for FP32 blocks: CA = S^T (H S) and CB = S^T (M S) over n rows,
// the basis S = [X | W | P] of ns <= 256 columns.
//
// Split BF16 x 3: every FP32 value a = a_hi + a_lo with a_hi = bf16(a),
// a_lo = bf16(a - a_hi); a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped
// a_lo b_lo is below 2^-16 of the product), three BF16 MMAs accumulating in
// FP32.  One CTA (4 warps) per 128-row tile of the output (basis columns
// m0..m0+127) and per range of rows of S:
//   * rows in chunks of 32.  The 32 rows of S, H S and M S of a chunk are
//     contiguous in global memory (row-major panels): one thread copies them
//     into shared memory with three cp.async.bulk copies (the bulk-copy engine,
//     completion counted in bytes on an mbarrier), two chunks ahead of the
//     tensor cores;
//   * every thread then reads 8 consecutive rows of one column from the FP32
//     copy, splits them and stores the 8 hi and 8 lo values as one 16-byte
//     K-major core-matrix row each (K-major, no swizzle: core matrices of
//     8 rows x 16 bytes, 128 bytes apart along K, 256 bytes apart along M / N),
//     double-buffered;
//   * one thread issues per 16-row slice three tcgen05.mma (M = 128, N = ns
//     rounded up to 16, K = 16) for CA and three for CB, accumulating in TMEM
//     (CA in columns 0..255, CB in 256..511 of a 512-column allocation), and
//     commits them to the stage's mbarrier, which frees the stage for the
//     chunk after next;
//   * the epilogue reads the accumulators back with tcgen05.ld (warp w owns
//     TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, i.e. output rows, and every
//     fourth 16-column group from 16 (w / 4) on) into an FP32 partial per
//     CTA; a second kernel sums the partials of all CTAs in a fixed order in
//     FP64 and writes the entries the Rayleigh-Ritz step reads.  16 warps
//     share the conversion of the chunks (4 per scheduler).
// Waits on the mbarriers are bounded; a wait that runs out (a fault of the
// hardware, not of the data) poisons the partial with NaN, which the solver
// reports as a non-finite residual.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kGT = 512;        // threads: 16 warps, four per set of 32 TMEM lanes
constexpr int kKC = 32;         // rows per chunk (two K = 16 slices)
constexpr int kMT = 128;        // output rows per tile (the M of the MMA)
constexpr long long kSpin = 1LL << 26;

__device__ __forceinline__ unsigned su32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long sdesc(unsigned addr) {
  // start address, leading (K) byte offset 128, stride (M/N) byte offset 256,
  // descriptor version 1 (tcgen05), no swizzle
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(256 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(unsigned d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mbar)
               : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false if it ran out
__device__ __forceinline__ bool wait_parity(unsigned mbar, unsigned parity) {
  for (long long spin = 0; spin < kSpin; ++spin) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of element (row r of the operand, k) in a K-major chunk of R rows
__device__ __forceinline__ int kmaj(int r, int k, int R) {
  return (k >> 4) * (R * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16;
}

// split 8 FP32 values into hi / lo BF16 and store each as one 16-byte row
__device__ __forceinline__ void split_store(const float (&v)[8], unsigned char* hi,
                                            unsigned char* lo) {
  unsigned h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat16 h0 = __float2bfloat16(v[2 * q]), h1 = __float2bfloat16(v[2 * q + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16(v[2 * q] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16(v[2 * q + 1] - __bfloat162float(h1));
    h[q] = (unsigned)__bfloat16_as_ushort(h0) | ((unsigned)__bfloat16_as_ushort(h1) << 16);
    l[q] = (unsigned)__bfloat16_as_ushort(l0) | ((unsigned)__bfloat16_as_ushort(l1) << 16);
  }
  *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Shared memory: two BF16 operand stages (A hi, A lo: 128 x 32 each; H S hi /
// lo and M S hi / lo: npad x 32 each), then two FP32 stages holding the
// chunk's 32 rows of S, H S and M S as they lie in global memory (ld floats
// per row).
__host__ __device__ constexpr int stage_bytes(int npad) { return 2 * kMT * kKC * 2 + 4 * npad * kKC * 2; }
__host__ __device__ constexpr int fstage_bytes(int ld) { return 3 * kKC * ld * 4; }

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__global__ void __launch_bounds__(kGT, 1)
    k_gram_tc(const float* __restrict__ S, const float* __restrict__ HS,
              const float* __restrict__ MS, int ld, int ns, int npad, long long n,
              long long rows_per_cta, float* __restrict__ part) {
  extern __shared__ __align__(1024) unsigned char sm[];
  // mbarriers: 0, 1 the BF16 stages (MMAs done), 2 all MMAs done, 3, 4 the
  // FP32 stages (bulk copies landed)
  __shared__ __align__(8) unsigned long long mbar[5];
  __shared__ unsigned s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, g = blockIdx.y, G = gridDim.y;
  const int m0 = mt * kMT;
  const long long r0 = (long long)g * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  const int nchunk = (int)((max(r1 - r0, 0LL) + kKC - 1) / kKC);
  const int SB = stage_bytes(npad), FB = fstage_bytes(ld);
  unsigned char* fst = sm + 2 * SB;  // the two FP32 stages
  if (tid == 0) {
    for (int q = 0; q < 5; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[q])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        su32(&s_tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tbase = s_tmem;
  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(npad >> 3) << 17) |
                         ((unsigned)(kMT >> 4) << 24);
  // chunk q's rows into FP32 stage q & 1 (one thread; rows past r1 are not
  // copied and read as zero below)
  auto fetch = [&](int q) {
    const long long rc = r0 + (long long)q * kKC;
    const int rows = (int)min((long long)kKC, r1 - rc);
    const unsigned bytes = (unsigned)rows * (unsigned)ld * 4u;
    const unsigned mb = su32(&mbar[3 + (q & 1)]);
    const unsigned dst = su32(fst + (q & 1) * FB);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(3u * bytes)
                 : "memory");
    bulk_g2s(dst, S + rc * ld, bytes, mb);
    bulk_g2s(dst + kKC * ld * 4, HS + rc * ld, bytes, mb);
    bulk_g2s(dst + 2 * kKC * ld * 4, MS + rc * ld, bytes, mb);
  };
  if (tid == 0) {
    if (nchunk > 0) fetch(0);
    if (nchunk > 1) fetch(1);
  }
  bool ok = true;
  for (int q = 0; q < nchunk; ++q) {
    const int s = q & 1;
    unsigned char* st = sm + s * SB;
    const float* fs = reinterpret_cast<const float*>(fst + s * FB);
    const int rows = (int)min((long long)kKC, r1 - (r0 + (long long)q * kKC));
    ok = ok && wait_parity(su32(&mbar[3 + s]), (unsigned)((q / 2) & 1));  // rows landed
    if (q >= 2) ok = ok && wait_parity(su32(&mbar[s]), (unsigned)((q / 2 - 1) & 1));  // MMAs done
    // A = S^T: rows m0..m0+127 of the tile (basis columns), 4 groups of 8 rows
    for (int it = tid; it < kMT * 4; it += kGT) {
      const int col = it % kMT, rg = it / kMT;
      const int c = m0 + col;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = rg * 8 + i;
        v[i] = (c < ns && r < rows) ? fs[r * ld + c] : 0.f;
      }
      const int o = kmaj(col, rg * 8, kMT);
      split_store(v, st + o, st + kMT * kKC * 2 + o);
    }
    // B = H S and M S: npad columns
    unsigned char* bh = st + 2 * kMT * kKC * 2;
    const int bsz = npad * kKC * 2;
    const float* fh = fs + kKC * ld;
    const float* fm = fs + 2 * kKC * ld;
    for (int it = tid; it < npad * 4; it += kGT) {
      const int c = it % npad, rg = it / npad;
      float vh[8], vm[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = rg * 8 + i;
        const bool in = c < ns && r < rows;
        vh[i] = in ? fh[r * ld + c] : 0.f;
        vm[i] = in ? fm[r * ld + c] : 0.f;
      }
      const int o = kmaj(c, rg * 8, npad);
      split_store(vh, bh + o, bh + bsz + o);
      split_store(vm, bh + 2 * bsz + o, bh + 3 * bsz + o);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();  // the BF16 stage is written; the FP32 stage is free again
    if (tid == 0) {
      if (q + 2 < nchunk) fetch(q + 2);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a_hi = su32(st), a_lo = a_hi + kMT * kKC * 2;
      const unsigned h_hi = su32(bh), h_lo = h_hi + bsz, m_hi = h_lo + bsz, m_lo = m_hi + bsz;
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks) {
        const unsigned ao = ks * kMT * 32, bo = ks * npad * 32;
        const unsigned acc0 = (q > 0 || ks > 0) ? 1u : 0u;
        mma_bf16(tbase, sdesc(a_hi + ao), sdesc(h_hi + bo), idesc, acc0);
        mma_bf16(tbase, sdesc(a_hi + ao), sdesc(h_lo + bo), idesc, 1u);
        mma_bf16(tbase, sdesc(a_lo + ao), sdesc(h_hi + bo), idesc, 1u);
        mma_bf16(tbase + 256, sdesc(a_hi + ao), sdesc(m_hi + bo), idesc, acc0);
        mma_bf16(tbase + 256, sdesc(a_hi + ao), sdesc(m_lo + bo), idesc, 1u);
        mma_bf16(tbase + 256, sdesc(a_lo + ao), sdesc(m_hi + bo), idesc, 1u);
      }
      commit(su32(&mbar[s]));
    }
  }
  // all MMAs done (the last commit covers every earlier one of this thread)
  if (tid == 0 && nchunk > 0) commit(su32(&mbar[2]));
  if (nchunk > 0) ok = ok && wait_parity(su32(&mbar[2]), 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: row m0 + 32 (warp % 4) + lane of CA and CB into this CTA's partial
  const int lw = warp & 3;
  const int row = 32 * lw + lane;
  float* pa = part + ((long long)(mt * G + g) * 2) * kMT * npad;
  float* pb = pa + (long long)kMT * npad;
  for (int c0 = 16 * (warp >> 2); c0 < npad; c0 += 64) {
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      unsigned r[16];
      const unsigned addr = tbase + ((unsigned)(32 * lw) << 16) + (unsigned)(which * 256 + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float* out = (which ? pb : pa) + (long long)row * npad + c0;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        out[j] = nchunk == 0 ? 0.f : ok ? __uint_as_float(r[j]) : __int_as_float(0x7fc00000);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

// Sum of the partials (fixed order, FP64) and the entries the Rayleigh-Ritz
// step reads: A on and below the block diagonal, B in the W columns and on the
// diagonal (k_gram_mirror completes both).  A block of 32 x 8 threads per 32
// consecutive entries of one row: thread (x, y) sums the partials y, y + 8, ...
// of entry x, and the eight sums are added in order.
__global__ void __launch_bounds__(256)
    k_gram_tc_reduce(const float* __restrict__ part, int ns, int npad, int nb, int G,
                     double* __restrict__ A, double* __restrict__ B) {
  __shared__ double sa[8][33], sb[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = blockIdx.y, j = blockIdx.x * 32 + tx;
  const int mt = i / kMT, row = i % kMT;
  double a = 0.0, b = 0.0;
  if (j < ns)
    for (int g = ty; g < G; g += 8) {
      const float* p = part + ((long long)(mt * G + g) * 2) * kMT * npad + (long long)row * npad + j;
      a += (double)p[0];
      b += (double)p[(long long)kMT * npad];
    }
  sa[ty][tx] = a;
  sb[ty][tx] = b;
  __syncthreads();
  if (ty == 0 && j < ns) {
    double ta = 0.0, tb = 0.0;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      ta += sa[y][tx];
      tb += sb[y][tx];
    }
    const long long t = (long long)i * ns + j;
    if (i / nb >= j / nb) A[t] = ta;
    if (j / nb == 1 || i == j) B[t] = tb;
  }
}

}  // namespace

bool gram_tc_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("FF_GRAM_TC");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool gram_rr_tc(cudaStream_t st, const float* S, const float* HS, const float* MS, int ld, int nb,
                int nblk, long long n, double* A, double* B, Buf& part) {
  const int ns = nblk * nb;
  // the basis within one M tile and its rows (ld floats) bulk-copyable:
  // 16-byte aligned panels and rows, both stages within shared memory
  if (ns > kMT || ns < 1 || n < 2048 || ld < ns || ld % 4 != 0 || n >= (1LL << 31) / ld)
    return false;
  if ((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(HS) |
       reinterpret_cast<uintptr_t>(MS)) % 16 != 0)
    return false;
  const int npad = (ns + 15) / 16 * 16;
  const int mtiles = (ns + kMT - 1) / kMT;
  const int G = (int)std::max<long long>(
      1, std::min<long long>((n + 255) / 256, std::max(1, sm_count() / mtiles)));
  const long long rpc = ((n + G - 1) / G + kKC - 1) / kKC * kKC;
  const int smem = 2 * stage_bytes(npad) + 2 * fstage_bytes(ld);
  if (smem > 220 * 1024) return false;
  float* p = reinterpret_cast<float*>(part.ensure(sizeof(float) * 2 * (size_t)mtiles * G * kMT * npad));
  set_max_dyn_smem((const void*)k_gram_tc, smem);
  ProfScope ps(kProfGram);
  (k_gram_tc<<<dim3(mtiles, G), kGT, smem, st>>>(S, HS, MS, ld, ns, npad, n, rpc, p),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_gram_tc_reduce<<<dim3((ns + 31) / 32, ns), 256, 0, st>>>(p, ns, npad, nb, G, A, B),
   ::ff::note_launch());
  FF_LAUNCH_CHECK();
  gram_mirror(st, A, B, ns, nb);
  return true;
}

}  // namespace ff
