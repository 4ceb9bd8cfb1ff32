// Plane staging for z-marching tile kernels: cp.async 16-byte copies of a
// (rows x kW) window of one x-y plane into shared memory, with zero fill on
// Dirichlet ghost rows / planes and wrap on periodic axes.
#pragma once

#include "internal.h"

namespace vsv {
namespace tile {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

constexpr int kTX = 128;              // tile width (x)
constexpr int kTY = 16;               // tile height (y)
constexpr int kHX = 4;                // halo columns (one 16-byte vector)
constexpr int kW = kTX + 2 * kHX;     // staged row length (floats)
constexpr int kNV = kW / 4;           // 16-byte vectors per staged row
constexpr int kThreads = 256;         // 32 (x groups of 4) x 8 (rows)

struct Geom {
  int nx, ny, nz;
  int per_y, per_z;
  int ntx, nty;          // tiles along x, y
  int zchunk;
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Per-thread staging descriptors: shared offset, global row offset within a
// plane (j * nx + x) and whether the row exists (else zero fill).
template <int NS>
struct StageDesc {
  int soff[NS];
  int goff[NS];
  bool ok[NS];
  bool used[NS];
  __device__ __forceinline__ void init(const Geom& G, int x0, int y0, int hr, int rows) {
    for (int s = 0; s < NS; ++s) {
      const int t = threadIdx.x + kThreads * s;
      used[s] = t < rows * kNV;
      const int r = t / kNV, v = t - r * kNV;
      int j = y0 - hr + r;
      bool okr = true;
      if (G.per_y) j = wrapi(j, G.ny);
      else if (j < 0 || j >= G.ny) okr = false;
      const int x = wrapi(x0 - kHX + 4 * v, G.nx);
      soff[s] = r * kW + 4 * v;
      goff[s] = okr ? j * G.nx + x : 0;
      ok[s] = okr;
    }
  }
  __device__ __forceinline__ void stage(float* slot, const float* __restrict__ src, const Geom& G,
                                        int plane, bool zero) const {
    bool pvalid = !zero;
    int k = plane;
    if (G.per_z) k = wrapi(k, G.nz);
    else if (k < 0 || k >= G.nz) pvalid = false;
    const float* base = src + (pvalid ? (long long)k * G.ny * G.nx : 0LL);
    for (int s = 0; s < NS; ++s)
      if (used[s]) cp_async16(slot + soff[s], base + goff[s], pvalid && ok[s]);
  }
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Can the tiled kernels handle this level?  (All three axes active, x
// periodic, tile-aligned extents.)
inline bool level_ok(const Level& L) {
  return L.act[0] && L.act[1] && L.act[2] && L.per[0] && L.n[0] % kTX == 0 &&
         L.n[1] % kTY == 0 && L.n[2] >= 2;
}

inline Geom geom(const Level& L, int zchunk) {
  Geom G;
  G.nx = L.n[0]; G.ny = L.n[1]; G.nz = L.n[2];
  G.per_y = L.per[1]; G.per_z = L.per[2];
  G.ntx = L.n[0] / kTX; G.nty = L.n[1] / kTY;
  G.zchunk = zchunk > 0 ? (zchunk < L.n[2] ? zchunk : L.n[2]) : L.n[2];
  return G;
}

}  // namespace tile
}  // namespace vsv
