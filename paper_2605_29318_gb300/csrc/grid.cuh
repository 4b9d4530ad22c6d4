// Uniform grid of the neighbour search and the coverage predicate (internal;
// shared by the neighbour search of the cloud and of query points).
#pragma once

#include "ff_internal.cuh"

namespace ff {

struct GridDev {
  double o0, o1, o2, h;
  int d0, d1, d2, b0, b1, b2;
};

__device__ __forceinline__ int cell_coord(float x, double o, double h, int dim) {
  int c = (int)floor(((double)x - o) / h);
  return min(max(c, 0), dim - 1);
}

__device__ __forceinline__ unsigned int spread3(unsigned int v) {  // 2 bits -> positions 0, 3
  return (v & 1u) | ((v & 2u) << 2);
}

__device__ __forceinline__ long long cell_key(const GridDev& g, int cx, int cy, int cz) {
  long long brick = ((long long)(cz >> 2) * g.b1 + (cy >> 2)) * g.b0 + (cx >> 2);
  unsigned int m = spread3(cx & 3) | (spread3(cy & 3) << 1) | (spread3(cz & 3) << 2);
  return brick * 64 + m;
}

// the coverage predicate: FP32 with a margin, FP64 (no FMA) inside the margin
__device__ __forceinline__ bool covers(float4 X, float4 p) {
  float dx = __fsub_rn(X.x, p.x), dy = __fsub_rn(X.y, p.y), dz = __fsub_rn(X.z, p.z);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  float a2 = __fmul_rn(p.w, p.w);
  if (d2 < a2 * 0.99999f) return true;
  if (d2 > a2 * 1.00001f) return false;
  double ex = __dsub_rn((double)X.x, (double)p.x);
  double ey = __dsub_rn((double)X.y, (double)p.y);
  double ez = __dsub_rn((double)X.z, (double)p.z);
  double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return e2 < __dmul_rn((double)p.w, (double)p.w);
}


}  // namespace ff
