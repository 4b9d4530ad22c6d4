// Scans, device-flag helpers, launch counting and the event profiler.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "ff_internal.cuh"

namespace ff {

// The limit only grows: contexts driven from several host threads may launch
// the same kernel with different sizes, and a larger limit never affects a
// smaller launch (the attribute is an upper bound, not an allocation).
void set_max_dyn_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  FF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  int& cur = limit[std::make_pair(fn, dev)];
  if (bytes <= cur) return;
  FF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
}

// Streaming multiprocessors of the current device (queried once per device).
int sm_count() {
  static std::mutex mu;
  static std::map<int, int> count;
  int dev = 0;
  FF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  int& n = count[dev];
  if (n == 0) {
    FF_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    if (n <= 0) n = 1;
  }
  return n;
}

thread_local ff_ctx* g_ctx = nullptr;

namespace {
std::atomic<long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int cls_) : cls(cls_) {
  ff_ctx* c = g_ctx;
  if (!c || !c->prof.on || !((c->prof.mask >> cls_) & 1u)) return;
  Profiler& p = c->prof;
  const size_t need = 2 * (size_t)(p.used[cls] + 1);
  while (p.ev[cls].size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    p.ev[cls].push_back(e);
  }
  cudaEvent_t start = p.ev[cls][2 * p.used[cls]];
  stop = p.ev[cls][2 * p.used[cls] + 1];
  p.used[cls]++;
  cudaEventRecord(start, c->stream);
}

void ProfScope::close() {
  if (stop && g_ctx) cudaEventRecord(stop, g_ctx->stream);
  stop = nullptr;
}

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class TI, class TO>
__global__ void k_scan_tile(const TI* __restrict__ in, TO* __restrict__ out,
                            TO* __restrict__ tile_sums, long long n) {
  __shared__ TO warp_tot[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO run = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    long long i = base + j;
    TO x = i < n ? (TO)in[i] : (TO)0;
    v[j] = run;
    run += x;
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TO incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    TO y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    TO t = lane < kScanThreads / 32 ? warp_tot[lane] : (TO)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  TO off = (incl - run) + (warp > 0 ? warp_tot[warp - 1] : (TO)0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    long long i = base + j;
    if (i < n) out[i] = v[j] + off;
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = off + run;
}

template <class TO>
__global__ void k_add_tile_offsets(TO* __restrict__ out, const TO* __restrict__ offs, long long n) {
  long long i = (long long)blockIdx.x * kScanTile + threadIdx.x;
  TO o = offs[blockIdx.x];
  for (int j = 0; j < kScanItems; ++j, i += kScanThreads)
    if (i < n) out[i] += o;
}

template <class TO>
__global__ void k_set_last(TO* out, long long n, const TO* v) { out[n] = *v; }

template <class TI, class TO>
void scan_impl(const TI* in, TO* out, long long n, ff_ctx* c, Buf& tmp, size_t tmp_off) {
  // out must hold n + 1 entries; out[n] = total
  long long tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) {
    FF_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), c->stream));
    return;
  }
  size_t need = tmp_off + sizeof(TO) * (size_t)(2 * tiles + 2);
  // tmp is sized by the caller for the recursion depth (see scan_counts)
  FF_REQUIRE(need <= tmp.bytes, FF_ERR_CUDA, "scan workspace too small");
  TO* sums = reinterpret_cast<TO*>(reinterpret_cast<char*>(tmp.p) + tmp_off);
  TO* sums_scan = sums + tiles;
  (k_scan_tile<TI, TO><<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, out, sums, n), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (tiles == 1) {
    (k_set_last<TO><<<1, 1, 0, c->stream>>>(out, n, sums), ::ff::note_launch());
    FF_LAUNCH_CHECK();
    return;
  }
  scan_impl<TO, TO>(sums, sums_scan, tiles, c, tmp, tmp_off + sizeof(TO) * (size_t)(2 * tiles + 2));
  (k_add_tile_offsets<TO><<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(out, sums_scan, n), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  (k_set_last<TO><<<1, 1, 0, c->stream>>>(out, n, sums_scan + tiles), ::ff::note_launch());
  FF_LAUNCH_CHECK();
}

size_t scan_tmp_bytes(long long n, size_t elem) {
  size_t total = 0;
  while (true) {
    long long tiles = (n + kScanTile - 1) / kScanTile;
    total += elem * (size_t)(2 * tiles + 2);
    if (tiles <= 1) break;
    n = tiles;
  }
  return total + 256;
}
}  // namespace

void scan_counts(const int* in, long long* out, long long n, ff_ctx* c, Buf& tmp) {
  tmp.ensure(scan_tmp_bytes(n, sizeof(long long)));
  scan_impl<int, long long>(in, out, n, c, tmp, 0);
}

void scan_counts_i32(const int* in, int* out, long long n, ff_ctx* c, Buf& tmp) {
  tmp.ensure(scan_tmp_bytes(n, sizeof(int)));
  scan_impl<int, int>(in, out, n, c, tmp, 0);
}

void reset_flags(ff_ctx* c) {
  c->flags.ensure(sizeof(DevFlags));
  FF_CUDA(cudaMemsetAsync(c->flags.p, 0, sizeof(DevFlags), c->stream));
}

DevFlags read_flags(ff_ctx* c) {
  FF_CUDA(cudaMemcpyAsync(c->hflags, c->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost,
                          c->stream));
  FF_CUDA(cudaStreamSynchronize(c->stream));
  return *c->hflags;
}

}  // namespace ff
