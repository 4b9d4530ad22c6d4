// C ABI of the library: argument checks, error model and inspection exports.
#include <algorithm>
#include <numeric>

#include "linalg.cuh"

namespace ff {
void warmstart_features(ff_ctx* c, float* feat);
void warmstart_block(ff_ctx* c, ff_net* w, int k, const ff_eig_opts& o, void* X0);
template <class T>
void gather_block(ff_ctx* c, const T* X0, int m, T* X, int ld);
template <class T>
void scatter_block(ff_ctx* c, const T* X, int ld, int m, T* out);
}  // namespace ff

namespace {

template <class F>
ff_status guarded(ff_ctx* c, F&& f) {
  if (!c) return FF_ERR_INVALID_ARG;
  c->err.clear();
  ff::g_ctx = c;
  struct Reset {
    ~Reset() { ff::g_ctx = nullptr; }
  } reset;
  try {
    FF_CUDA(cudaSetDevice(c->device));
    f();
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

}  // namespace

namespace {
template <class T>
std::vector<double> to_host_f64(const ff::Buf& b, size_t count) {
  std::vector<T> tmp(count);
  if (count) FF_CUDA(cudaMemcpy(tmp.data(), b.p, sizeof(T) * count, cudaMemcpyDeviceToHost));
  return std::vector<double>(tmp.begin(), tmp.end());
}
// double-float pairs (head, tail) to FP64: head + tail
std::vector<double> to_host_df(const ff::Buf& b, size_t count) {
  std::vector<float> tmp(2 * count);
  if (count) FF_CUDA(cudaMemcpy(tmp.data(), b.p, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost));
  std::vector<double> out(count);
  for (size_t i = 0; i < count; ++i) out[i] = (double)tmp[2 * i] + (double)tmp[2 * i + 1];
  return out;
}
template <class T>
std::vector<T> to_host(const ff::Buf& b, size_t count) {
  std::vector<T> tmp(count);
  if (count) FF_CUDA(cudaMemcpy(tmp.data(), b.p, sizeof(T) * count, cudaMemcpyDeviceToHost));
  return tmp;
}

// internal-order CSR (+ aligned values) -> caller-order CSR with ascending columns
void remap_csr(const std::vector<int>& perm, const std::vector<int>& iperm,
               const std::vector<long long>& p, const std::vector<int>& idx,
               std::vector<const std::vector<double>*> vals, int64_t* optr, int32_t* oidx,
               std::vector<double*> ovals, const std::vector<size_t>& strides_in,
               const std::vector<size_t>& strides_out, const std::vector<int>& reps) {
  const long long n = (long long)perm.size();
  long long off = 0;
  std::vector<std::pair<int, long long>> row;
  for (long long i = 0; i < n; ++i) {
    const long long j = iperm[i];
    optr[i] = off;
    row.clear();
    for (long long e = p[j]; e < p[j + 1]; ++e) row.emplace_back(perm[idx[e]], e);
    std::sort(row.begin(), row.end());
    for (size_t t = 0; t < row.size(); ++t) {
      oidx[off + t] = row[t].first;
      for (size_t v = 0; v < vals.size(); ++v) {
        if (!ovals[v]) continue;
        for (int r = 0; r < reps[v]; ++r)
          ovals[v][r * strides_out[v] + off + t] = (*vals[v])[r * strides_in[v] + row[t].second];
      }
    }
    off += (long long)row.size();
  }
  optr[n] = off;
}
}  // namespace

extern "C" {

const char* ff_version(void) { return "freeform-gb300 0.1"; }

ff_status ff_create(ff_ctx** out, int device, void* cuda_stream, int precision) {
  if (!out) return FF_ERR_INVALID_ARG;
  *out = nullptr;
  if (precision != FF_PREC_FP32 && precision != FF_PREC_FP64) return FF_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  ff_ctx* c = new ff_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->prec = precision;
  ff_status s = guarded(c, [&] {
    c->flags.ensure(sizeof(ff::DevFlags));
    void* h = nullptr;
    FF_CUDA(cudaMallocHost(&h, 64 * 1024));
    c->hflags = static_cast<ff::DevFlags*>(h);
  });
  if (s != FF_OK) {
    delete c;
    return s;
  }
  *out = c;
  return FF_OK;
}

void ff_destroy(ff_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& v : c->prof.ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  if (c->hflags) cudaFreeHost(c->hflags);
  delete c;
}

const char* ff_last_error(const ff_ctx* c) { return c ? c->err.c_str() : "null context"; }

ff_status rkpm_build(ff_ctx* c, const float* particles, const float* volumes, const float* support,
                     int64_t n) {
  return guarded(c, [&] {
    FF_REQUIRE(particles && volumes && support, FF_ERR_INVALID_ARG, "NULL input pointer");
    FF_REQUIRE(n >= 1 && n <= 0x7fffffffLL, FF_ERR_INVALID_ARG, "n out of range");
    c->stage = 0;
    c->n = n;
    c->nq = n;
    c->twoset = false;
    c->t32 = c->prec != FF_PREC_FP64;
    c->n1 = c->n2 = 0;
    ff::ProfScope ps(ff::kProfBuild);
    ff::build_neighbours(c, particles, volumes, support, n);
    ff::build_shape(c);
    c->stage = 1;
  });
}

ff_status rkpm_build_twoset(ff_ctx* c, const float* points, const float* volumes, int64_t n,
                            int32_t K, double trunc, int64_t start) {
  return guarded(c, [&] {
    FF_REQUIRE(points && volumes, FF_ERR_INVALID_ARG, "NULL input pointer");
    FF_REQUIRE(n >= 4 && n <= 0x7fffffffLL, FF_ERR_INVALID_ARG, "n out of range");
    FF_REQUIRE(K >= 4 && (int64_t)K <= n, FF_ERR_INVALID_ARG, "K must lie in 4..n");
    FF_REQUIRE(std::isfinite(trunc) && trunc >= 0.0, FF_ERR_INVALID_ARG,
               "trunc must be finite and >= 0 (0: untruncated)");
    FF_REQUIRE(start >= 0 && start < n, FF_ERR_INVALID_ARG, "start out of range");
    c->stage = 0;
    c->n1 = c->n2 = 0;
    c->t32 = c->prec != FF_PREC_FP64 || c->build32;
    ff::ProfScope ps(ff::kProfBuild);
    ff::build_twoset(c, points, volumes, n, K, trunc, start);
    c->stage = 1;
  });
}

ff_status assemble_hessian(ff_ctx* c, const float* E, const float* nu, double E0, double nu0) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "assemble_hessian before rkpm_build");
    if (!E) FF_REQUIRE(E0 > 0 && std::isfinite(E0), FF_ERR_INVALID_ARG, "E0 must be > 0");
    if (!nu) FF_REQUIRE(nu0 >= 0 && nu0 < 0.5, FF_ERR_INVALID_ARG, "nu0 must be in [0, 0.5)");
    c->stage = 1;
    ff::ProfScope ps(ff::kProfAssemble);
    ff::build_matrices(c, E, nu, E0, nu0);
    c->stage = 2;
  });
}

void ff_eig_opts_default(ff_eig_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->max_iter = 500;
  o->guard = 8;
  o->cheb_degree = 16;
  o->cheb_ratio = 300.0;
  o->seed = 0;
  o->time_budget_s = 0.0;
  o->exclude_constant = 0;
  o->verbose = 0;
  o->fp32_phase = 1;
  o->fp32_tol = 1e-4;
  o->cheb_degree_fp64 = 48;
  o->precond_tc = 1;
  o->precond_compact = 0;
}

ff_status eigenmodes(ff_ctx* c, int k, const ff_eig_opts* opts, const void* X0, double* eigvals,
                     void* modes, ff_eig_report* rep) {
  ff_status result = FF_OK;
  ff_status s = guarded(c, [&] {
    FF_REQUIRE(c->stage >= 2, FF_ERR_STATE, "eigenmodes before assemble_hessian");
    FF_REQUIRE(eigvals, FF_ERR_INVALID_ARG, "eigvals must not be NULL");
    FF_REQUIRE(k >= 1 && k <= 256 && k <= c->n - 1, FF_ERR_INVALID_ARG, "k out of range");
    ff_eig_opts o;
    ff_eig_opts_default(&o);
    if (opts) o = *opts;
    FF_REQUIRE(o.tol > 0 && o.max_iter >= 0 && o.guard >= 0 && o.fp32_tol > 0 &&
                   o.cheb_degree_fp64 >= 0, FF_ERR_INVALID_ARG,
               "bad options");
    if (rep) *rep = ff_eig_report{};
    result = ff::run_eigenmodes(c, k, o, X0, eigvals, modes, rep);
    if (result == FF_ERR_NOT_CONVERGED) c->err = "max_iter reached or residual stalled before tol";
    if (result == FF_ERR_TIMEOUT) c->err = "time budget exhausted";
    if (result == FF_ERR_NUMERIC) c->err = "non-finite residual";
  });
  return s != FF_OK ? s : result;
}

ff_status ff_set_build_precision(ff_ctx* c, int precision) {
  return guarded(c, [&] {
    FF_REQUIRE(precision == FF_PREC_FP32 || precision == FF_PREC_FP64, FF_ERR_INVALID_ARG,
               "build precision must be FF_PREC_FP32 or FF_PREC_FP64");
    FF_REQUIRE(c->prec == FF_PREC_FP64 || precision == FF_PREC_FP32, FF_ERR_INVALID_ARG,
               "an FP32 context builds in FP32");
    c->build32 = precision == FF_PREC_FP32;
  });
}

ff_status ff_profile_enable(ff_ctx* c, int on) {
  return ff_profile_classes(c, on ? ~0u : 0u);
}

ff_status ff_profile_classes(ff_ctx* c, uint32_t mask) {
  return guarded(c, [&] {
    FF_CUDA(cudaStreamSynchronize(c->stream));
    c->prof.on = mask != 0;
    c->prof.mask = mask;
    for (int k = 0; k < ff::kProfN; ++k) c->prof.used[k] = 0;
  });
}

}  // extern "C"

namespace {
// device copy of a host array on the context stream (nullptr stays nullptr)
template <class T>
const T* stage_in(ff_ctx* c, int slot, const T* h, long long count) {
  if (!h) return nullptr;
  T* d = reinterpret_cast<T*>(c->host_in[slot].ensure(sizeof(T) * std::max(count, 1LL)));
  FF_CUDA(cudaMemcpyAsync(d, h, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
  return d;
}

// the eigenmodes step of the host-buffer calls: modes to a device buffer of
// the context, then copied to the caller's host array
ff_status host_eigenmodes(ff_ctx* c, int k, const ff_eig_opts* opts, double* eigvals, void* modes,
                          ff_eig_report* rep) {
  const size_t esz = c->prec == FF_PREC_FP64 ? 8 : 4;
  size_t bytes = 0;
  void* dmodes = nullptr;
  ff_status s = guarded(c, [&] {
    FF_REQUIRE(k >= 1 && k <= 256 && k <= c->n - 1, FF_ERR_INVALID_ARG, "k out of range");
    bytes = esz * (size_t)c->n * k;
    if (modes) dmodes = c->host_out.ensure(bytes);
  });
  if (s != FF_OK) return s;
  const ff_status r = eigenmodes(c, k, opts, nullptr, eigvals, dmodes, rep);
  if (r != FF_OK && r != FF_ERR_NOT_CONVERGED && r != FF_ERR_TIMEOUT && r != FF_ERR_NUMERIC)
    return r;
  if (modes) {
    s = guarded(c, [&] {
      FF_CUDA(cudaMemcpyAsync(modes, dmodes, bytes, cudaMemcpyDeviceToHost, c->stream));
      FF_CUDA(cudaStreamSynchronize(c->stream));
    });
    if (s != FF_OK) return s;
  }
  return r;
}
}  // namespace

extern "C" {

ff_status ff_subspace_host(ff_ctx* c, const float* particles, const float* volumes,
                           const float* support, const float* E, const float* nu, int64_t n,
                           double E0, double nu0, int k, const ff_eig_opts* opts,
                           double* eigvals, void* modes, ff_eig_report* rep) {
  const float *dX = nullptr, *dv = nullptr, *da = nullptr, *dE = nullptr, *dnu = nullptr;
  ff_status s = guarded(c, [&] {
    FF_REQUIRE(particles && volumes && support, FF_ERR_INVALID_ARG, "NULL input pointer");
    FF_REQUIRE(n >= 1 && n <= 0x7fffffffLL, FF_ERR_INVALID_ARG, "n out of range");
    dX = stage_in(c, 0, particles, 3 * n);
    dv = stage_in(c, 1, volumes, n);
    da = stage_in(c, 2, support, n);
    dE = stage_in(c, 3, E, n);
    dnu = stage_in(c, 4, nu, n);
  });
  if (s != FF_OK) return s;
  if ((s = rkpm_build(c, dX, dv, da, n)) != FF_OK) return s;
  if ((s = assemble_hessian(c, dE, dnu, E0, nu0)) != FF_OK) return s;
  return host_eigenmodes(c, k, opts, eigvals, modes, rep);
}

ff_status ff_subspace_twoset_host(ff_ctx* c, const float* points, const float* volumes,
                                  const float* E, const float* nu, int64_t n, int32_t K,
                                  double trunc, int64_t start, double E0, double nu0, int k,
                                  const ff_eig_opts* opts, double* eigvals, void* modes,
                                  ff_eig_report* rep) {
  const float *dX = nullptr, *dv = nullptr, *dE = nullptr, *dnu = nullptr;
  ff_status s = guarded(c, [&] {
    FF_REQUIRE(points && volumes, FF_ERR_INVALID_ARG, "NULL input pointer");
    FF_REQUIRE(n >= 4 && n <= 0x7fffffffLL, FF_ERR_INVALID_ARG, "n out of range");
    dX = stage_in(c, 0, points, 3 * n);
    dv = stage_in(c, 1, volumes, n);
    dE = stage_in(c, 3, E, n);
    dnu = stage_in(c, 4, nu, n);
  });
  if (s != FF_OK) return s;
  if ((s = rkpm_build_twoset(c, dX, dv, n, K, trunc, start)) != FF_OK) return s;
  if ((s = assemble_hessian(c, dE, dnu, E0, nu0)) != FF_OK) return s;
  return host_eigenmodes(c, k, opts, eigvals, modes, rep);
}

ff_status ff_profile_read(ff_ctx* c, int cls, int64_t* launches, double* total_ms) {
  return guarded(c, [&] {
    FF_REQUIRE(cls >= 0 && cls < ff::kProfN, FF_ERR_INVALID_ARG, "unknown profile class");
    FF_CUDA(cudaStreamSynchronize(c->stream));
    double ms = 0.0;
    for (int i = 0; i < c->prof.used[cls]; ++i) {
      float t = 0.f;
      FF_CUDA(cudaEventElapsedTime(&t, c->prof.ev[cls][2 * i], c->prof.ev[cls][2 * i + 1]));
      ms += t;
    }
    if (launches) *launches = c->prof.used[cls];
    if (total_ms) *total_ms = ms;
  });
}

int64_t ff_launch_count(void) { return ff::launch_count(); }

ff_status ff_selftest_device_wait(int device, int64_t wait_cycles) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    (void)cudaGetLastError();
    return FF_ERR_CUDA;
  }
  if (wait_cycles < 1000000 || wait_cycles > 4000000000LL) return FF_ERR_INVALID_ARG;
  try {
    return ff::selftest_device_wait(device, wait_cycles);
  } catch (const ff::Error& e) {
    (void)cudaGetLastError();
    return e.code;
  } catch (...) {
    return FF_ERR_CUDA;
  }
}

ff_status ff_get_sizes(const ff_ctx* c, int64_t* n, int64_t* n1, int64_t* n2) {
  if (!c) return FF_ERR_INVALID_ARG;
  if (n) *n = c->stage >= 1 ? c->n : 0;
  if (n1) *n1 = c->stage >= 1 ? c->n1 : 0;
  if (n2) *n2 = c->stage >= 2 ? c->n2 : 0;
  return FF_OK;
}

ff_status ff_get_twoset(const ff_ctx* cc, int64_t* n_points, int32_t* K, int64_t* centres,
                        double* radii) {
  ff_ctx* c = const_cast<ff_ctx*>(cc);
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1 && c->twoset, FF_ERR_STATE, "no two-set cloud built");
    if (n_points) *n_points = c->nq;
    if (K) *K = (int32_t)c->n;
    FF_CUDA(cudaStreamSynchronize(c->stream));
    if (centres)
      FF_CUDA(cudaMemcpy(centres, c->centre_idx.p, sizeof(int64_t) * c->n,
                         cudaMemcpyDeviceToHost));
    if (radii) FF_CUDA(cudaMemcpy(radii, c->crad.p, sizeof(double) * c->n, cudaMemcpyDeviceToHost));
  });
}

ff_status ff_skinning_weights(ff_ctx* c, const float* Q, int64_t nq, const void* C, int m,
                              void* W) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "no cloud built");
    FF_REQUIRE(nq >= 0 && nq < (1LL << 26) && m >= 1 && m <= 4096, FF_ERR_INVALID_ARG,
               "bad sizes");
    FF_REQUIRE(nq == 0 || (Q && C && W), FF_ERR_INVALID_ARG, "NULL array");
    ff::skinning_weights(c, Q, nq, C, m, W);
  });
}

ff_status ff_lbs_deform(ff_ctx* c, const float* Q, int64_t nq, const void* W, int m,
                        const void* Z, void* x) {
  return guarded(c, [&] {
    FF_REQUIRE(nq >= 0 && nq < (1LL << 26) && m >= 1 && m <= 4096, FF_ERR_INVALID_ARG,
               "bad sizes");
    FF_REQUIRE(nq == 0 || (Q && W && Z && x), FF_ERR_INVALID_ARG, "NULL array");
    ff::lbs_deform(c, Q, nq, W, m, Z, x);
  });
}

ff_status ff_get_precond_layout(const ff_ctx* c, int64_t* row_blocks, int64_t* ksteps) {
  if (!c) return FF_ERR_INVALID_ARG;
  const bool built = c->stage >= 2 && c->tc_ksteps > 0;
  if (row_blocks) *row_blocks = built ? (c->n + 15) / 16 : 0;
  if (ksteps) *ksteps = built ? c->tc_ksteps : 0;
  return FF_OK;
}


ff_status ff_export_rkpm(const ff_ctx* cc, int64_t* ptr, int32_t* idx, double* phi, double* dphi) {
  ff_ctx* c = const_cast<ff_ctx*>(cc);
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "no cloud built");
    FF_REQUIRE(ptr && idx, FF_ERR_INVALID_ARG, "NULL output");
    FF_CUDA(cudaStreamSynchronize(c->stream));
    const size_t n = c->n, n1 = c->n1, nq = c->nq;
    auto p = to_host<long long>(c->nbr_ptr, nq + 1);
    auto ix = to_host<int>(c->nbr_idx, n1);
    std::vector<double> ph, dph;
    if (!ff::tables_f32(c)) {
      ph = to_host_df(c->phi, n1);
      dph = to_host_df(c->dphi, 3 * n1);
    } else {
      ph = to_host_f64<float>(c->phi, n1);
      dph = to_host_f64<float>(c->dphi, 3 * n1);
    }
    if (c->twoset) {  // rows and centres are already in the caller's order
      std::copy(p.begin(), p.end(), ptr);
      std::copy(ix.begin(), ix.end(), idx);
      if (phi) std::copy(ph.begin(), ph.end(), phi);
      if (dphi) std::copy(dph.begin(), dph.end(), dphi);
      return;
    }
    auto perm = to_host<int>(c->perm, n);
    auto iperm = to_host<int>(c->iperm, n);
    remap_csr(perm, iperm, p, ix, {&ph, &dph}, ptr, idx, {phi, dphi}, {n1, n1}, {n1, n1}, {1, 3});
  });
}

ff_status ff_export_row_ptr(const ff_ctx* cc, int64_t* ptr) {
  ff_ctx* c = const_cast<ff_ctx*>(cc);
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "no cloud built");
    FF_REQUIRE(ptr, FF_ERR_INVALID_ARG, "NULL output");
    FF_CUDA(cudaStreamSynchronize(c->stream));
    const size_t nq = c->nq;
    auto p = to_host<long long>(c->nbr_ptr, nq + 1);
    if (c->twoset) {
      std::copy(p.begin(), p.end(), ptr);
      return;
    }
    auto perm = to_host<int>(c->perm, nq);  // internal -> caller
    std::vector<long long> cnt(nq);
    for (size_t j = 0; j < nq; ++j) cnt[perm[j]] = p[j + 1] - p[j];
    ptr[0] = 0;
    for (size_t i = 0; i < nq; ++i) ptr[i + 1] = ptr[i] + cnt[i];
  });
}

ff_status ff_export_matrices(const ff_ctx* cc, int64_t* row_ptr, int32_t* col, double* H,
                             double* M) {
  ff_ctx* c = const_cast<ff_ctx*>(cc);
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 2, FF_ERR_STATE, "matrices not assembled");
    FF_REQUIRE(row_ptr && col, FF_ERR_INVALID_ARG, "NULL output");
    FF_CUDA(cudaStreamSynchronize(c->stream));
    const size_t n = c->n, n2 = c->n2;
    auto perm = to_host<int>(c->perm, n);
    auto iperm = to_host<int>(c->iperm, n);
    auto p = to_host<long long>(c->a_ptr, n + 1);
    auto ix = to_host<int>(c->a_col, n2);
    std::vector<double> v = c->prec == FF_PREC_FP64 ? to_host<double>(c->a_val, 2 * n2)
                                                    : to_host_f64<float>(c->a_val, 2 * n2);
    std::vector<double> hv(n2), mv(n2);
    for (size_t e = 0; e < n2; ++e) {
      hv[e] = v[2 * e];
      mv[e] = v[2 * e + 1];
    }
    remap_csr(perm, iperm, p, ix, {&hv, &mv}, row_ptr, col, {H, M}, {0, 0}, {0, 0}, {1, 1});
  });
}

ff_status ff_apply_operators(ff_ctx* c, const void* X, int m, void* YH, void* YM) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 2, FF_ERR_STATE, "matrices not assembled");
    FF_REQUIRE(X && m >= 1 && m <= 512, FF_ERR_INVALID_ARG, "bad block");
    const long long n = c->n;
    auto run = [&](auto tag) {
      using T = decltype(tag);
      T* in = reinterpret_cast<T*>(c->scratch[4].ensure(sizeof(T) * n * m));
      T* oh = reinterpret_cast<T*>(c->scratch[6].ensure(sizeof(T) * n * m));
      T* om = reinterpret_cast<T*>(c->scratch[7].ensure(sizeof(T) * n * m));
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
  });
}

ff_status ff_apply_operators_matfree(ff_ctx* c, const float* E, const float* nu, double E0,
                                     double nu0, const void* X, int m, void* YH, void* YM) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "no cloud built");
    FF_REQUIRE(X && m >= 1 && m <= 512, FF_ERR_INVALID_ARG, "bad block");
    if (!E) FF_REQUIRE(E0 > 0 && std::isfinite(E0), FF_ERR_INVALID_ARG, "E0 must be > 0");
    if (!nu) FF_REQUIRE(nu0 >= 0 && nu0 < 0.5, FF_ERR_INVALID_ARG, "nu0 must be in [0, 0.5)");
    ff::apply_matfree(c, E, nu, E0, nu0, X, m, YH, YM);
  });
}

ff_status ff_warmstart_features(ff_ctx* c, float* feat) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "features before rkpm_build");
    FF_REQUIRE(!c->twoset, FF_ERR_STATE, "the warm start takes a nodal cloud (rkpm_build)");
    FF_REQUIRE(feat, FF_ERR_INVALID_ARG, "feat must not be NULL");
    ff::warmstart_features(c, feat);
    FF_CUDA(cudaStreamSynchronize(c->stream));
  });
}

ff_status ff_warmstart_block(ff_ctx* c, ff_net* net, int k, const ff_eig_opts* opts, void* X0) {
  return guarded(c, [&] {
    FF_REQUIRE(c->stage >= 1, FF_ERR_STATE, "warm start before rkpm_build");
    FF_REQUIRE(!c->twoset, FF_ERR_STATE, "the warm start takes a nodal cloud (rkpm_build)");
    FF_REQUIRE(net && X0, FF_ERR_INVALID_ARG, "net and X0 must not be NULL");
    FF_REQUIRE(k >= 1 && k <= 256 && k <= c->n - 1, FF_ERR_INVALID_ARG, "k out of range");
    ff_eig_opts o;
    ff_eig_opts_default(&o);
    if (opts) o = *opts;
    FF_REQUIRE(o.guard >= 0, FF_ERR_INVALID_ARG, "bad options");
    ff::warmstart_block(c, net, k, o, X0);
    FF_CUDA(cudaStreamSynchronize(c->stream));
  });
}

}  // extern "C"
