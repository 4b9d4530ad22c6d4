// Many objects in one call (eigenmodes_batched): a pool of host threads, each
// with its own context on its own non-blocking stream, takes the objects
// largest first from a shared counter and runs the single-object calls on
// them.  One object's solve is a chain of small latency-bound launches with a
// host read-back per iteration, so a single object leaves most SMs idle;
// several objects in flight on separate streams fill them.  Each item runs the
// same kernels as alone, so its results do not depend on the batch.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "ff_internal.cuh"

extern "C" {

ff_status eigenmodes_batched(int device, int precision, ff_batch_item* items, int count,
                             const ff_eig_opts* opts, int workers) {
  if (count < 0 || (count > 0 && !items)) return FF_ERR_INVALID_ARG;
  if (precision != FF_PREC_FP32 && precision != FF_PREC_FP64) return FF_ERR_INVALID_ARG;
  if (workers < 0 || workers > 256) return FF_ERR_INVALID_ARG;
  if (count == 0) return FF_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    items[i].status = FF_ERR_CUDA;
    std::strncpy(items[i].error, "not run: no worker could create a context",
                 sizeof(items[i].error) - 1);
    items[i].error[sizeof(items[i].error) - 1] = '\0';
  }
  // largest objects first (longest-processing-time order); ties by index
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return items[a].n > items[b].n; });
  const int nw = std::min(count, workers > 0 ? workers : 8);
  std::atomic<int> next{0};
  auto work = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    ff_ctx* c = nullptr;
    if (ff_create(&c, device, st, precision) != FF_OK) {
      cudaStreamDestroy(st);
      return;
    }
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= count) break;
      ff_batch_item& it = items[order[q]];
      ff_status s = rkpm_build(c, it.particles, it.volumes, it.support, it.n);
      if (s == FF_OK) s = assemble_hessian(c, it.E, it.nu, it.E0, it.nu0);
      if (s == FF_OK) s = eigenmodes(c, it.k, opts, nullptr, it.eigvals, it.modes, it.report);
      it.status = s;
      const char* msg = s == FF_OK ? "" : ff_last_error(c);
      std::strncpy(it.error, msg, sizeof(it.error) - 1);
      it.error[sizeof(it.error) - 1] = '\0';
    }
    ff_destroy(c);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  pool.reserve(nw);
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (items[i].status != FF_OK) return items[i].status;
  return FF_OK;
}

}  // extern "C"
