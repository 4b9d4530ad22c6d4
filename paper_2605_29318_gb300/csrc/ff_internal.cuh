// Internal declarations of the freeform-gb300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/freeform.h"

namespace ff {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
  ff_status code;
  Error(ff_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define FF_CUDA(x)                                                                     \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      throw ::ff::Error(e_ == cudaErrorMemoryAllocation ? FF_ERR_OOM : FF_ERR_CUDA,    \
                        std::string(#x) + ": " + cudaGetErrorString(e_));              \
    }                                                                                  \
  } while (0)

#define FF_LAUNCH_CHECK() FF_CUDA(cudaGetLastError())

#define FF_REQUIRE(cond, code, msg)            \
  do {                                         \
    if (!(cond)) throw ::ff::Error(code, msg); \
  } while (0)

// ---------------------------------------------------------------- device buffer
// Owning device allocation (cudaMalloc); grows on demand, never shrinks.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void* ensure(size_t b) {
    if (b == 0) b = 16;
    if (b > bytes) {
      release();
      cudaError_t e = cudaMalloc(&p, b);
      if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw Error(FF_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed");
      }
      bytes = b;
    }
    return p;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Device-side error word written by kernels (never a trap).
struct DevFlags {
  int code;          // ff_status of the first error a kernel hit (0 = none)
  int index;         // particle (internal order) or row that raised it
  int fallback;      // number of moment solves redone in FP64
  int max_row;       // largest count seen by a pass that reports one
  double red[8];     // small reductions returned to the host
};

// Per-class CUDA-event timing of the library's launches (off by default).
enum ProfClass {
  kProfPrecond = 0,  // Chebyshev preconditioner steps (H-only block products)
  kProfSpmm,         // fused (H, M) block products
  kProfGram,         // tall-skinny Gram products
  kProfRR,           // small dense Rayleigh-Ritz
  kProfUpdate,       // block updates
  kProfBuild,        // rkpm_build (whole stage)
  kProfAssemble,     // assemble_hessian (whole stage)
  kProfSetup,        // eigensolver set-up (power iteration)
  kProfFps,          // farthest-point sampling of the two-set centres
  kProfCover,        // covering lists of the two-set construction
  kProfShape,        // shape-function kernels (moment solves)
  kProfPattern,      // assembly: the sparsity pattern of H_w and M
  kProfAsmValues,    // assembly: the values of H_w and M
  kProfN
};

struct Profiler {
  bool on = false;
  unsigned mask = ~0u;  // classes recorded while on (bit 1 << class)
  std::vector<cudaEvent_t> ev[kProfN];  // start/stop pairs
  int used[kProfN] = {};
};

// count of kernel launches issued by the library (process-wide)
void note_launch();
long long launch_count();

// Uniform grid used by the neighbour search.
struct Grid {
  double origin[3];
  double h;          // cell edge
  int dims[3];       // cells per axis
  int bdims[3];      // 4x4x4-cell bricks per axis
  long long ncells;  // bdims product * 64 (key space)
};

}  // namespace ff

// ---------------------------------------------------------------- context
struct ff_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int prec = FF_PREC_FP32;
  std::string err;
  int stage = 0;  // 0 empty, 1 built, 2 assembled
  int64_t n = 0, n1 = 0, n2 = 0;  // unknowns (nodes or centres), shape pairs, matrix entries
  // quadrature points (rows of the shape-function lists): n for the nodal
  // discretisation, the given points for the two-set one
  int64_t nq = 0;
  bool twoset = false;  // two-set discretisation: farthest-point centres, Gaussian kernel
  double trunc = 0.0;   // its cut radius in units of r_k (0: untruncated)
  float qscale = 1.f;   // its basis scale
  // FP64 contexts: FP32 shape functions and tile sums for two-set clouds
  // (ff_set_build_precision), the matrices still stored in FP64
  bool build32 = false;
  bool t32 = false;  // the built cloud's tables are FP32 (set at each build)

  ff::Grid grid{};
  // particles in internal (cell) order
  // (two-set: the centres in their farthest-point order, pos.w = 0; the radii
  // are kept in FP64 in crad)
  ff::Buf perm;      // int[n]   internal -> caller index
  ff::Buf iperm;     // int[n]   caller -> internal index
  ff::Buf pos;       // float4[n] (x, y, z, a)
  ff::Buf vol;       // float[nq] quadrature volumes
  ff::Buf cell_start;// int[ncells + 1]
  // two-set centres
  ff::Buf centre_idx;// int64[K]  quadrature point chosen as centre k
  ff::Buf crad;      // double[K] r_k
  ff::Buf clim;      // double[K] t^2 r_k^2 (+inf untruncated)
  ff::Buf clim32;    // float[K]  its FP32 rounding (filter)
  ff::Buf qpts;      // float[3 nq] the quadrature points (x, y, z), caller order
  bool has_cols = false;  // the transposed lists nbrT_* are built
  // neighbours (internal order)
  ff::Buf nbr_ptr;   // int64[nq+1]
  ff::Buf nbr_idx;   // int[n1]
  ff::Buf nbrT_ptr;  // int64[n+1]  node k -> rows i it covers
  ff::Buf nbrT_idx;  // int[n1]     row i
  ff::Buf nbrT_pos;  // int64[n1]   position of k inside row i
  // shape functions (context precision), aligned with nbr_idx
  ff::Buf phi;       // T[n1]
  ff::Buf dphi;      // T[3 * n1]
  // matrices (internal order), CSR with the diagonal stored
  ff::Buf a_ptr;     // int64[n+1]
  ff::Buf a_col;     // int[n2]
  ff::Buf a_val;     // T2[n2] interleaved (H, M)
  ff::Buf a_val32;   // float2[n2] (H, M) rounded from a_val (FP64 contexts)
  ff::Buf a_valdf;   // float4[n2] (H.h, H.l, M.h, M.l) double-float split of a_val
                     // (FP64 contexts)
  ff::Buf h_f32;     // float[n2] H values for the preconditioner
  // the same H in 16-row blocks, each a dense BF16 tile over the union of its
  // rows' columns in mma.m16n8k16 A-fragment order (tensor-core
  // preconditioner step); tc_ksteps = 0 when not built
  ff::Buf tc_kofs;   // int[nblk + 1] first k-step (16 union columns) of each block
  ff::Buf tc_ucol;   // int[16 * ksteps] union columns
  ff::Buf tc_tile;   // uint4[32 * ksteps] A fragments
  ff::Buf tc_hs;     // float[n] row sums of the rounded entries
  long long tc_ksteps = 0;
  ff::Buf hdiag_f32; // float[n] diag(H)
  // skinning weights at query points (scratch of the last call)
  ff::Buf sk_cnt;    // int[nq + 1]
  ff::Buf sk_ptr;    // int64[nq + 1]
  ff::Buf sk_idx;    // int[nq1]  covering nodes (internal order)
  ff::Buf sk_phi;    // T[4 * nq1] shape functions and gradients
  ff::Buf wh;        // T[nq] v_i (lambda_i + 4 mu_i)
  // device flags
  ff::Buf flags;     // DevFlags
  ff::DevFlags* hflags = nullptr;  // pinned mirror
  // generic scratch
  ff::Buf scratch[8];
  // device copies of host inputs and outputs of the host-buffer calls
  ff::Buf host_in[5];
  ff::Buf host_out;
  // eigen-solver workspace
  ff::Buf ws[28];
  ff::Profiler prof;
};

namespace ff {

// context of the C-ABI call running on this thread (profiling hooks)
extern thread_local ff_ctx* g_ctx;

// records a start/stop event pair around a scope when profiling is on
struct ProfScope {
  int cls;
  cudaEvent_t stop = nullptr;
  explicit ProfScope(int cls_);
  ~ProfScope() { close(); }
  void close();  // record the stop event now (once)
};

// ---------------------------------------------------------------- helpers
inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// whether the shape-function tables (and the material weights and tile sums
// of the assembly) are FP32: FP32 contexts, and two-set clouds of FP64
// contexts built with FP32 build precision; else double-float pairs
inline bool tables_f32(const ff_ctx* c) { return c->t32; }

// raise a kernel's dynamic shared-memory limit on the current device (only
// ever raised, per kernel and device; thread-safe; the attribute belongs to
// the device's context)
void set_max_dyn_smem(const void* fn, int bytes);

// number of streaming multiprocessors of the current device (cached per device)
int sm_count();

void reset_flags(ff_ctx* c);
DevFlags read_flags(ff_ctx* c);

// exclusive scan of int counts -> int64 offsets (out has n+1 entries)
void scan_counts(const int* in, long long* out, long long n, ff_ctx* c, Buf& tmp);
// exclusive scan of int -> int (out has n+1 entries)
void scan_counts_i32(const int* in, int* out, long long n, ff_ctx* c, Buf& tmp);

// stages
void build_neighbours(ff_ctx* c, const float* X, const float* v, const float* a, int64_t n);
void build_shape(ff_ctx* c);
void build_matrices(ff_ctx* c, const float* E, const float* nu, double E0, double nu0);
// v_i (lambda_i + 4 mu_i) per quadrature point (context precision) into wh
void material_weights(ff_ctx* c, const float* E, const float* nu, double E0, double nu0,
                      void* wh);
// the grid barrier's bounded wait run out on purpose (one arrival missing)
ff_status selftest_device_wait(int device, long long wait_cycles);
// the transposed lists of a two-set cloud (built on demand)
void twoset_columns(ff_ctx* c, const float* Xq);
// H_w X and M X from the shape-function tables (matfree.cu)
void apply_matfree(ff_ctx* c, const float* E, const float* nu, double E0, double nu0,
                   const void* X, int m, void* YH, void* YM);

// the two-set discretisation (twoset.cu): centres, radii, covering lists and
// shape functions at the quadrature points
void build_twoset(ff_ctx* c, const float* Xq, const float* vq, long long nq, int K, double trunc,
                  long long start);
// dense-tile assembly of a two-set cloud's H_w and M (tset_assembly.cu), for
// K up to kTsetMaxCentres centres
constexpr long long kTsetMaxCentres = 4096;
bool tset_assembly_fits(long long K);
void tset_assemble(ff_ctx* c);
// covering lists of arbitrary points over the centres (returns the pair count)
// and the Gaussian shape functions there (returns the pass's flags)
long long twoset_cover(ff_ctx* c, const float* Q, long long nq, Buf& ptrb, Buf& idxb, Buf& cntb);
DevFlags twoset_shape(ff_ctx* c, const float* Q, long long nq, const long long* ptr,
                      const int* idx, long long n1, void* phi, void* dphi, bool fp64_out);

// skinning weight fields and linear blend skinning at query points (skinning.cu)
void skinning_weights(ff_ctx* c, const float* Q, long long nq, const void* C, int m, void* W);
void lbs_deform(ff_ctx* c, const float* Q, long long nq, const void* W, int m, const void* Z,
                void* x);

// operator application on internal-order row-major panels
template <class T>
void spmm_hm(ff_ctx* c, const T* X, int ldx, T* YH, T* YM, int ldy, int m);

// eigen solver
ff_status run_eigenmodes(ff_ctx* c, int k, const ff_eig_opts& o, const void* X0,
                         double* eigvals, void* modes, ff_eig_report* rep);

}  // namespace ff
