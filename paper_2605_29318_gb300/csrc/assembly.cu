// Assembly of the weight-space Hessian H_w (Prop. 1) and the RKPM mass matrix
// (Sec. 3.2, Eq. 14) in CSR, one warp per matrix row.
//
//   (H_w)_kl = sum_i v_i (lambda_i + 4 mu_i) grad phi_k(X_i) . grad phi_l(X_i)
//   M_kl     = sum_i v_i phi_k(X_i) phi_l(X_i)
// over the quadrature points X_i covered by both nodes k and l.
//
// Row-owner gather: the warp of row k walks the points i that node k covers
// (transposed neighbour lists, ascending i), and for each i its lanes add the
// contribution of every node l of row i into a shared-memory accumulator slot.
// Within one i the lanes touch distinct slots and the walk over i is
// sequential, so every entry is summed in a fixed order (deterministic, no
// atomics).  Column slots come from a shared-memory hash set of the row's
// 2-hop pattern; pass 1 counts the unique columns, pass 2 sorts them and
// accumulates the values.  The diagonal of H_w is replaced by minus the sum of
// the off-diagonal entries of its row, which makes H_w 1 = 0 exact in storage
// (the constant mode of Supp. Sec. B is an exact null vector).
#include <type_traits>

#include "ff_internal.cuh"
#include "linalg.cuh"

namespace ff {
namespace {

constexpr int kEmpty = -1;

__device__ __forceinline__ unsigned int hash32(unsigned int x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// insert key into a warp-private table; returns the slot (or -1 when full)
__device__ __forceinline__ int hset_insert(int* tab, int tsize, int key, bool& fresh) {
  unsigned int h = hash32((unsigned int)key) & (tsize - 1);
  for (int probe = 0; probe < tsize; ++probe) {
    int prev = atomicCAS(&tab[h], kEmpty, key);
    if (prev == kEmpty) {
      fresh = true;
      return (int)h;
    }
    if (prev == key) {
      fresh = false;
      return (int)h;
    }
    h = (h + 1) & (tsize - 1);
  }
  fresh = false;
  return -1;
}

__device__ __forceinline__ int hset_find(const int* tab, int tsize, int key) {
  unsigned int h = hash32((unsigned int)key) & (tsize - 1);
  for (int probe = 0; probe < tsize; ++probe) {
    int v = tab[h];
    if (v == key) return (int)h;
    if (v == kEmpty) return -1;
    h = (h + 1) & (tsize - 1);
  }
  return -1;
}

template <class T>
__global__ void k_material(const int* __restrict__ perm, long long n, const float* __restrict__ vol,
                           const float* __restrict__ E, const float* __restrict__ nu, double E0,
                           double nu0, T* __restrict__ wh, DevFlags* flags) {
  long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int i = perm ? perm[j] : (int)j;  // caller index of quadrature point j
  double e = E ? (double)E[i] : E0;
  double p = nu ? (double)nu[i] : nu0;
  if (!(e > 0.0) || !(p >= 0.0) || !(p < 0.5) || !isfinite(e)) {
    if (atomicCAS(&flags->code, 0, (int)FF_ERR_INVALID_ARG) == 0) flags->index = i;
    return;
  }
  double lam = e * p / ((1.0 + p) * (1.0 - 2.0 * p));
  double mu = e / (2.0 * (1.0 + p));
  wh[j] = (T)((double)vol[j] * (lam + 4.0 * mu));
}

// pass 1: unique 2-hop columns per row
__global__ void k_pattern_count(const long long* __restrict__ ptr, const int* __restrict__ idx,
                                const long long* __restrict__ tptr, const int* __restrict__ tidx,
                                long long n, int tsize, int* __restrict__ cnt,
                                DevFlags* __restrict__ flags) {
  extern __shared__ int sm_tab[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* tab = sm_tab + wib * tsize;
  const long long rows_per_grid = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long k = (long long)blockIdx.x * (blockDim.x >> 5) + wib; k < n; k += rows_per_grid) {
    for (int q = lane; q < tsize; q += 32) tab[q] = kEmpty;
    __syncwarp();
    int fresh_cnt = 0;
    bool overflow = false;
    for (long long a = tptr[k]; a < tptr[k + 1]; ++a) {
      int i = tidx[a];
      for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
        bool fresh;
        int slot = hset_insert(tab, tsize, idx[e], fresh);
        if (slot < 0) overflow = true;
        fresh_cnt += fresh;
      }
    }
    fresh_cnt = __reduce_add_sync(0xffffffffu, fresh_cnt);
    overflow = __any_sync(0xffffffffu, overflow);
    if (lane == 0) {
      cnt[k] = fresh_cnt;
      atomicMax(&flags->max_row, fresh_cnt);
      if (overflow || 2 * fresh_cnt > tsize) {
        if (atomicCAS(&flags->code, 0, (int)FF_ERR_INVALID_ARG) == 0) flags->index = (int)k;
      }
    }
    __syncwarp();
  }
}

// pass 2: sorted columns and values
// T: shape functions, material weights and sums (double-float for FP64
// contexts); TO: the stored matrix values
template <class T, class TO = T>
__global__ void k_assemble(const long long* __restrict__ ptr, const int* __restrict__ idx,
                           const long long* __restrict__ tptr, const int* __restrict__ tidx,
                           const long long* __restrict__ tpos, const T* __restrict__ phi,
                           const T* __restrict__ dphi, long long n1, const float* __restrict__ vol,
                           const T* __restrict__ wh, long long n, int tsize, int maxrow,
                           const long long* __restrict__ aptr, int* __restrict__ acol,
                           TO* __restrict__ aval, float* __restrict__ hf32,
                           float* __restrict__ hdiag) {
  extern __shared__ unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  // per-warp layout: tab[tsize], rnk[tsize], keys[maxrow], skeys[maxrow] (int),
  // then vh[maxrow], vm[maxrow] (T)
  size_t per_warp = (size_t)tsize * 8 + (size_t)maxrow * 8;
  per_warp = (per_warp + 15) & ~size_t(15);
  size_t per_warp_T = per_warp + (size_t)maxrow * 2 * sizeof(T);
  per_warp_T = (per_warp_T + 15) & ~size_t(15);
  unsigned char* base = sm_raw + per_warp_T * wib;
  int* tab = reinterpret_cast<int*>(base);
  int* rnk = tab + tsize;
  int* keys = rnk + tsize;
  int* skeys = keys + maxrow;
  T* vh = reinterpret_cast<T*>(base + per_warp);
  T* vm = vh + maxrow;
  const long long rows_per_grid = (long long)gridDim.x * wpb;
  for (long long k = (long long)blockIdx.x * wpb + wib; k < n; k += rows_per_grid) {
    for (int q = lane; q < tsize; q += 32) tab[q] = kEmpty;
    __syncwarp();
    for (long long a = tptr[k]; a < tptr[k + 1]; ++a) {
      int i = tidx[a];
      for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
        bool fresh;
        hset_insert(tab, tsize, idx[e], fresh);
      }
    }
    __syncwarp();
    // compact the keys
    int m = 0;
    for (int q0 = 0; q0 < tsize; q0 += 32) {
      int v = tab[q0 + lane];
      bool has = v != kEmpty;
      unsigned int bal = __ballot_sync(0xffffffffu, has);
      if (has) keys[m + __popc(bal & ((1u << lane) - 1))] = v;
      m += __popc(bal);
    }
    __syncwarp();
    // rank of every key (columns ascending), recorded at its hash slot
    for (int q = lane; q < m; q += 32) {
      int v = keys[q];
      int r = 0;
      for (int b = 0; b < m; ++b) r += keys[b] < v;
      rnk[hset_find(tab, tsize, v)] = r;
      vh[q] = T(0);
      vm[q] = T(0);
    }
    __syncwarp();
    // accumulate over the points i covered by node k, ascending i
    for (long long a = tptr[k]; a < tptr[k + 1]; ++a) {
      int i = tidx[a];
      long long eik = tpos[a];
      T fk = phi[eik];
      T gk0 = dphi[eik], gk1 = dphi[n1 + eik], gk2 = dphi[2 * n1 + eik];
      T wi = wh[i], vi = (T)vol[i];
      T cH0 = wi * gk0, cH1 = wi * gk1, cH2 = wi * gk2, cM = vi * fk;
      for (long long e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
        int r = rnk[hset_find(tab, tsize, idx[e])];
        if constexpr (std::is_same_v<T, dfloat>) {  // unnormalised sums, normalised below
          df_mac(vh[r], cH0, dphi[e]);
          df_mac(vh[r], cH1, dphi[n1 + e]);
          df_mac(vh[r], cH2, dphi[2 * n1 + e]);
          df_mac(vm[r], cM, phi[e]);
        } else {
          vh[r] += cH0 * dphi[e] + cH1 * dphi[n1 + e] + cH2 * dphi[2 * n1 + e];
          vm[r] += cM * phi[e];
        }
      }
      __syncwarp();
    }
    // keys in rank (ascending column) order; vh / vm are already indexed by rank
    for (int q = lane; q < m; q += 32) {
      int v = keys[q];
      skeys[rnk[hset_find(tab, tsize, v)]] = v;
    }
    __syncwarp();
    T off = T(0);
    for (int r = lane; r < m; r += 32)
      if (skeys[r] != (int)k) off += finish(vh[r]);
#pragma unroll
    for (int o = 16; o; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    const long long row0 = aptr[k];
    for (int r = lane; r < m; r += 32) {
      int col = skeys[r];
      const TO h = (col == (int)k) ? (TO)(-off) : (TO)finish(vh[r]);
      acol[row0 + r] = col;
      aval[2 * (row0 + r)] = h;
      aval[2 * (row0 + r) + 1] = (TO)finish(vm[r]);
      hf32[row0 + r] = (float)h;
    }
    if (lane == 0) hdiag[k] = (float)(TO)(-off);
    __syncwarp();
  }
}

size_t assemble_smem_per_warp(int tsize, int maxrow, size_t tbytes) {
  size_t per_warp = (size_t)tsize * 8 + (size_t)maxrow * 8;
  per_warp = (per_warp + 15) & ~size_t(15);
  size_t t = per_warp + (size_t)maxrow * 2 * tbytes;
  return (t + 15) & ~size_t(15);
}

__global__ void k_round_f32(const double* __restrict__ x, float* __restrict__ y, long long m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) y[t] = (float)x[t];
}

// x = h + l with h = fl32(x), l = fl32(x - h): the double-float split
__global__ void k_split_df(const double* __restrict__ x, float2* __restrict__ y, long long m) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) {
    const float h = (float)x[t];
    y[t] = make_float2(h, (float)(x[t] - (double)h));
  }
}

}  // namespace

void finish_matrices(ff_ctx* c);

// v_i (lambda_i + 4 mu_i) per quadrature point into wh (double-float pairs in
// FP64 contexts, FP32 otherwise); throws FF_ERR_INVALID_ARG on a bad material
void material_weights(ff_ctx* c, const float* E, const float* nu, double E0, double nu0,
                      void* wh) {
  cudaStream_t st = c->stream;
  const long long nq = c->nq;
  const int T = 256;
  const int* qperm = c->twoset ? nullptr : c->perm.as<int>();
  reset_flags(c);
  if (!tables_f32(c))
    (k_material<dfloat><<<ceil_div(nq, T), T, 0, st>>>(qperm, nq, c->vol.as<float>(), E, nu, E0,
                                                     nu0, static_cast<dfloat*>(wh),
                                                     c->flags.as<DevFlags>()),
     ::ff::note_launch());
  else
    (k_material<float><<<ceil_div(nq, T), T, 0, st>>>(qperm, nq, c->vol.as<float>(), E, nu, E0,
                                                    nu0, static_cast<float*>(wh),
                                                    c->flags.as<DevFlags>()),
     ::ff::note_launch());
  FF_LAUNCH_CHECK();
  const DevFlags f = read_flags(c);
  if (f.code == FF_ERR_INVALID_ARG)
    throw Error(FF_ERR_INVALID_ARG, "invalid material (need E > 0, 0 <= nu < 0.5) at point " +
                                        std::to_string(f.index));
}

void build_matrices(ff_ctx* c, const float* E, const float* nu, double E0, double nu0) {
  cudaStream_t st = c->stream;
  const long long n = c->n, n1 = c->n1, nq = c->nq;
  const int T = 256;
  const bool f64 = c->prec == FF_PREC_FP64;
  const bool tdf = !tables_f32(c);  // double-float tables, weights and sums
  const size_t tb = f64 ? 8 : 4;
  reset_flags(c);
  DevFlags f{};
  // material weights per quadrature point (the nodal points are in cell
  // order, the two-set quadrature points in the caller's)
  c->wh.ensure((tdf ? 8 : 4) * nq);
  const int* qperm = c->twoset ? nullptr : c->perm.as<int>();
  if (tdf)  // FP64 contexts: material weights in double-float, like the shape functions
    (k_material<dfloat><<<ceil_div(nq, T), T, 0, st>>>(qperm, nq, c->vol.as<float>(), E, nu, E0,
                                                     nu0, c->wh.as<dfloat>(),
                                                     c->flags.as<DevFlags>()), ::ff::note_launch());
  else
    (k_material<float><<<ceil_div(nq, T), T, 0, st>>>(qperm, nq, c->vol.as<float>(), E, nu, E0,
                                                    nu0, c->wh.as<float>(),
                                                    c->flags.as<DevFlags>()), ::ff::note_launch());
  FF_LAUNCH_CHECK();
  if (c->twoset && tset_assembly_fits(n)) {
    // two-set clouds: dense tiles of points grouped by their nearest centre
    f = read_flags(c);
    if (f.code == FF_ERR_INVALID_ARG)
      throw Error(FF_ERR_INVALID_ARG, "invalid material (need E > 0, 0 <= nu < 0.5) at point " +
                                          std::to_string(f.index));
    tset_assemble(c);
    finish_matrices(c);
    return;
  }
  // pass 1: unique columns per row, in a table of 2048 slots per warp (4 warps
  // per block); clouds of uneven density (wide supports reaching into dense
  // regions) retry with 16384 slots per warp (2 warps per block)
  int* cnt = reinterpret_cast<int*>(c->scratch[5].ensure(sizeof(int) * (n + 1)));
  int tsize1 = 2048;
  ProfScope ps_pattern(kProfPattern);
  for (int attempt = 0; attempt < 2; ++attempt) {
    tsize1 = attempt == 0 ? 2048 : 16384;
    const int wpb1 = attempt == 0 ? 4 : 2;
    const size_t smem1 = sizeof(int) * tsize1 * wpb1;
    if (smem1 > 48 * 1024) set_max_dyn_smem((const void*)k_pattern_count, (int)smem1);
    if (attempt > 0) reset_flags(c);
    int grid1 = (int)std::min<long long>(ceil_div(n, wpb1), (long long)sm_count() * 16);
    (k_pattern_count<<<grid1, 32 * wpb1, smem1, st>>>(
        c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->nbrT_ptr.as<long long>(),
        c->nbrT_idx.as<int>(), n, tsize1, cnt, c->flags.as<DevFlags>()), ::ff::note_launch());
    FF_LAUNCH_CHECK();
    f = read_flags(c);
    const bool overflow =
        f.code == FF_ERR_INVALID_ARG && f.max_row > 0 && f.max_row * 2 > tsize1;
    if (!overflow) break;
  }
  ps_pattern.close();
  if (f.code == FF_ERR_INVALID_ARG) {
    throw Error(FF_ERR_INVALID_ARG,
                f.max_row > 0 && f.max_row * 2 > tsize1
                    ? "a Hessian row has more than " + std::to_string(tsize1 / 2) +
                          " distinct columns (support too large)"
                    : "invalid material (need E > 0, 0 <= nu < 0.5) at point " +
                          std::to_string(f.index));
  }
  const int maxrow = std::max(f.max_row, 1);
  long long* aptr = reinterpret_cast<long long*>(c->a_ptr.ensure(sizeof(long long) * (n + 1)));
  scan_counts(cnt, aptr, n, c, c->scratch[3]);
  long long n2 = 0;
  FF_CUDA(cudaMemcpyAsync(&n2, aptr + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FF_CUDA(cudaStreamSynchronize(st));
  c->n2 = n2;
  c->a_col.ensure(sizeof(int) * n2);
  c->a_val.ensure(2 * tb * n2);
  c->h_f32.ensure(sizeof(float) * n2);
  c->hdiag_f32.ensure(sizeof(float) * n);
  int tsize2 = 64;
  while (tsize2 < 2 * maxrow) tsize2 <<= 1;
  size_t pw = assemble_smem_per_warp(tsize2, maxrow, tdf ? 8 : 4);
  int wpb2 = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / pw));
  size_t smem = pw * wpb2;
  int grid2 = (int)std::min<long long>(ceil_div(n, wpb2), (long long)sm_count() * 32);
  ProfScope ps_values(kProfAsmValues);
  if (f64 && !tdf) {  // FP32 tables and sums, FP64 storage
    set_max_dyn_smem((const void*)k_assemble<float, double>,
                     (int)std::max<size_t>(smem, 48 * 1024));
    (k_assemble<float, double><<<grid2, 32 * wpb2, smem, st>>>(
        c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->nbrT_ptr.as<long long>(),
        c->nbrT_idx.as<int>(), c->nbrT_pos.as<long long>(), c->phi.as<float>(),
        c->dphi.as<float>(), n1, c->vol.as<float>(), c->wh.as<float>(), n, tsize2, maxrow, aptr,
        c->a_col.as<int>(), c->a_val.as<double>(), c->h_f32.as<float>(), c->hdiag_f32.as<float>()), ::ff::note_launch());
  } else if (f64) {
    set_max_dyn_smem((const void*)k_assemble<dfloat, double>,
                     (int)std::max<size_t>(smem, 48 * 1024));
    (k_assemble<dfloat, double><<<grid2, 32 * wpb2, smem, st>>>(
        c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->nbrT_ptr.as<long long>(),
        c->nbrT_idx.as<int>(), c->nbrT_pos.as<long long>(), c->phi.as<dfloat>(),
        c->dphi.as<dfloat>(), n1, c->vol.as<float>(), c->wh.as<dfloat>(), n, tsize2, maxrow, aptr,
        c->a_col.as<int>(), c->a_val.as<double>(), c->h_f32.as<float>(), c->hdiag_f32.as<float>()), ::ff::note_launch());
  } else {
    set_max_dyn_smem((const void*)k_assemble<float>, (int)std::max<size_t>(smem, 48 * 1024));
    (k_assemble<float><<<grid2, 32 * wpb2, smem, st>>>(
        c->nbr_ptr.as<long long>(), c->nbr_idx.as<int>(), c->nbrT_ptr.as<long long>(),
        c->nbrT_idx.as<int>(), c->nbrT_pos.as<long long>(), c->phi.as<float>(),
        c->dphi.as<float>(), n1, c->vol.as<float>(), c->wh.as<float>(), n, tsize2, maxrow, aptr,
        c->a_col.as<int>(), c->a_val.as<float>(), c->h_f32.as<float>(), c->hdiag_f32.as<float>()), ::ff::note_launch());
  }
  FF_LAUNCH_CHECK();
  ps_values.close();
  finish_matrices(c);
}

// the copies of (H, M) the eigensolver reads besides the stored values, and
// the preconditioner's tensor-core tiles
void finish_matrices(ff_ctx* c) {
  cudaStream_t st = c->stream;
  const long long n2 = c->n2;
  const bool f64 = c->prec == FF_PREC_FP64;
  if (f64) {  // FP32 rounding of (H, M) for the FP32 phase of the eigensolver
    float* v32 = reinterpret_cast<float*>(c->a_val32.ensure(2 * sizeof(float) * n2));
    const long long m = 2 * n2;
    (k_round_f32<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c->a_val.as<double>(), v32, m),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
    // and the double-float split for its second phase
    float2* vdf = reinterpret_cast<float2*>(c->a_valdf.ensure(2 * sizeof(float2) * n2));
    (k_split_df<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c->a_val.as<double>(), vdf, m),
     ::ff::note_launch());
    FF_LAUNCH_CHECK();
  }
  cheb_tc_build(c);
  FF_CUDA(cudaStreamSynchronize(st));
}

}  // namespace ff
