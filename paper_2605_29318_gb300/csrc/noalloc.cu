// Allocation-free variant of ff_apply_operators.
//
// ff_apply_operators stages the caller's block in three device panels that the
// context allocates on demand (cudaMalloc).  Some callers cannot allocate at
// that point: real-time loops that forbid driver allocations (a cudaMalloc can
// synchronise the device and take milliseconds), processes whose device memory
// is fully reserved by another allocator (a caching allocator or a memory pool
// that owns the rest of the GPU), and hosts that hand a plug-in a fixed memory
// budget.  This entry point uses a fixed scratch array that lives in the
// library's own device image instead: a file-scope __device__ array of
// kStaticScratchBytes, which every GPU that loads the library holds until the
// process exits.
//
// Host code must not use the array's name as a device address (on the host it
// names a stand-in object); the device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, and cached; the first call
// on a device does this set-up.  Every call shares the one array and leaves
// its contents behind; nothing in it needs to start at zero (each call
// overwrites every byte it reads).  Calls that overlap on the GPU -- on two
// streams, or from two threads -- race on the array and must be serialised by
// the caller.  Like the library's other calls, it synchronises the context's
// stream before it returns.
#include <mutex>

#include "linalg.cuh"

namespace ff {
template <class T>
void gather_block(ff_ctx* c, const T* X0, int m, T* X, int ld);
template <class T>
void scatter_block(ff_ctx* c, const T* X, int ld, int m, T* out);
}  // namespace ff

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// device address of the static scratch on `device` (which must be current)
void* static_scratch(int device) {
  FF_REQUIRE(device >= 0 && device < kMaxDevices, FF_ERR_INVALID_ARG, "device index too large");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      throw ff::Error(FF_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                       cudaGetErrorString(e));
    }
    g_scratch_addr[device] = p;
  }
  return g_scratch_addr[device];
}

}  // namespace

extern "C" ff_status ff_apply_operators_noalloc(ff_ctx* c, const void* X, int m, void* YH,
                                                void* YM) {
  if (!c) return FF_ERR_INVALID_ARG;
  c->err.clear();
  // the profiler attributes the block products to this context, as in
  // ff_apply_operators
  ff::g_ctx = c;
  struct Reset {
    ~Reset() { ff::g_ctx = nullptr; }
  } reset;
  try {
    FF_CUDA(cudaSetDevice(c->device));
    FF_REQUIRE(c->stage >= 2, FF_ERR_STATE, "matrices not assembled");
    FF_REQUIRE(X && m >= 1 && m <= 512, FF_ERR_INVALID_ARG, "bad block");
    const size_t esz = c->prec == FF_PREC_FP64 ? 8 : 4;
    const size_t panel = ((size_t)c->n * m * esz + 255) / 256 * 256;
    if (3 * panel > kStaticScratchBytes)
      throw ff::Error(FF_ERR_INVALID_ARG,
                      "block too large for the static scratch: n * m * " + std::to_string(esz) +
                          " bytes * 3 panels must fit in " +
                          std::to_string(kStaticScratchBytes) + " bytes");
    unsigned char* base = static_cast<unsigned char*>(static_scratch(c->device));
    auto run = [&](auto tag) {
      using T = decltype(tag);
      T* in = reinterpret_cast<T*>(base);
      T* oh = reinterpret_cast<T*>(base + panel);
      T* om = reinterpret_cast<T*>(base + 2 * panel);
      ff::gather_block<T>(c, static_cast<const T*>(X), m, in, m);
      ff::spmm_hm<T>(c, in, m, oh, om, m, m);
      if (YH) ff::scatter_block<T>(c, oh, m, m, static_cast<T*>(YH));
      if (YM) ff::scatter_block<T>(c, om, m, m, static_cast<T*>(YM));
      FF_CUDA(cudaStreamSynchronize(c->stream));
    };
    if (c->prec == FF_PREC_FP64)
      run(double{});
    else
      run(float{});
    return FF_OK;
  } catch (const ff::Error& e) {
    c->err = e.what();
    (void)cudaGetLastError();
    return e.code;
  } catch (const std::exception& e) {
    c->err = e.what();
    return FF_ERR_CUDA;
  }
}
