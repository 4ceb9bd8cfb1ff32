// Plane staging for z-marching tile kernels: cp.async 16-byte copies of a
// (rows x kW) window of one x-y plane into shared memory, with zero fill on
// Dirichlet ghost rows / planes and wrap on periodic axes; and, for the fused
// sweep, a split layout (tile body, then its halo groups) whose body a TMA
// tensor-map box fills, with mbarrier helpers whose waits are bounded.
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
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::); }

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
// i mod n in [0, n) for any i (a tile may span several periods of a short axis)
__device__ __forceinline__ int modi(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// Per-thread staging descriptors for the (up to three) 16-byte vectors a
// thread copies per plane: shared offset (-1: unused), global row offset
// within a plane (j * nx + x), and whether the row exists (else zero fill).
// Plain scalar members, so the descriptors stay in registers.
struct StageVec {
  int soff, goff;
  bool ok;
  __device__ __forceinline__ void init(const Geom& G, int t, int x0, int y0, int hr, int rows) {
    const int r = t / kNV, v = t - r * kNV;
    int j = y0 - hr + r;
    ok = true;
    if (G.per_y) j = modi(j, G.ny);
    else if (j < 0 || j >= G.ny) ok = false;
    const int x = modi(x0 - kHX + 4 * v, G.nx);   // nx is a multiple of 4
    soff = t < rows * kNV ? r * kW + 4 * v : -1;
    goff = ok ? j * G.nx + x : 0;
  }
  __device__ __forceinline__ void issue(float* slot, const float* base, bool pvalid) const {
    if (soff >= 0) cp_async16(slot + soff, base + goff, pvalid && ok);
  }
};

template <int NS>
struct StageDesc {
  static_assert(NS >= 1 && NS <= 3, "at most three vectors per thread and plane");
  StageVec v0, v1, v2;
  __device__ __forceinline__ void init(const Geom& G, int x0, int y0, int hr, int rows) {
    v0.init(G, threadIdx.x, x0, y0, hr, rows);
    v1.init(G, threadIdx.x + kThreads, x0, y0, hr, NS > 1 ? rows : 0);
    v2.init(G, threadIdx.x + 2 * kThreads, x0, y0, hr, NS > 2 ? rows : 0);
  }
  __device__ __forceinline__ void stage(float* slot, const float* __restrict__ src, const Geom& G,
                                        int plane, bool zero) const {
    bool pvalid = !zero;
    int k = plane;
    if (G.per_z) k = wrapi(k, G.nz);
    else if (k < 0 || k >= G.nz) pvalid = false;
    const float* base = src + (pvalid ? (long long)k * G.ny * G.nx : 0LL);
    v0.issue(slot, base, pvalid);
    if (NS > 1) v1.issue(slot, base, pvalid);
    if (NS > 2) v2.issue(slot, base, pvalid);
  }
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// ---------------------------------------------------------------- tensor-map staging
// On tile-aligned levels the tile's own columns of a staged plane come as one
// box of a tensor map, loaded by the tensor memory accelerator (TMA) into a
// ring slot; a shared-memory mbarrier counts the arrival of each step's
// bytes.  Waits on it are bounded (kCopyLimitNs by default), after which a
// status bit (kCopyTimeout) is set and the kernel returns.
constexpr unsigned long long kCopyLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// makes the initialised barriers visible to the copy engine
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// orders this thread's earlier shared-memory accesses before later copies
// of the tensor memory accelerator into the same memory
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of `bar`, at most limit_ns; on timeout sets
// kCopyTimeout in *status.  Every thread of the CTA calls it; the CTA-wide
// vote makes the outcome the same for all of them (false: leave the kernel).
__device__ __forceinline__ bool mbar_wait_cta(unsigned long long* bar, unsigned parity,
                                              int* status, unsigned long long limit_ns) {
  int late = 0;
  if (!mbar_test(bar, parity)) {
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
      if (global_ns() - t0 > limit_ns) {
        late = 1;
        break;
      }
    }
  }
  if (__syncthreads_or(late)) {
    if (late && status) atomicOr(status, kCopyTimeout);
    return false;
  }
  return true;
}

// Waits at most limit_ns for phase `parity` of `bar` (one thread, on the
// way out after a timeout: the CTA's shared memory stays allocated until
// copies still in flight have landed or the bound has passed).
__device__ __forceinline__ void mbar_drain(unsigned long long* bar, unsigned parity,
                                           unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity) && global_ns() - t0 < limit_ns) {
  }
}

// One box of a 3-D tensor map (x, y, z element coordinates of its first
// element; parts outside the tensor read as zero) into shared memory at
// `dst` (128-byte aligned), counted on `bar` in bytes.  `map` is the
// generic address of a tensor map in kernel parameter space.
__device__ __forceinline__ void tma_load_3d(float* dst, const void* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- split layout
// A staged plane in the split layout: `rows` body rows of kTX floats (the
// tile's own columns x0 .. x0 + kTX - 1: one tensor-map box), then `rows`
// halo rows of kHP floats, the 16-byte groups left (x0 - 4 .. x0 - 1) and
// right (x0 + kTX .. x0 + kTX + 3) of the tile, wrapped around periodic x.
constexpr int kHP = 2 * kHX;
__device__ __forceinline__ float* halo_row(float* slot, int rows, int r) {
  return slot + rows * kTX + r * kHP;
}
__device__ __forceinline__ const float* halo_row(const float* slot, int rows, int r) {
  return slot + rows * kTX + r * kHP;
}

// cp.async staging of one 16-byte vector of a split-layout plane: vector v of
// staged row r (t = r * kNV + v; v = 0 the left halo group, 1 .. kTX / 4 the
// body, kNV - 1 the right halo group).  halo_only: only the two halo vectors
// of each row (t = 2 r + side), the body coming as a tensor-map box.
struct SplitVec {
  int soff, goff;
  bool ok;
  __device__ __forceinline__ void init(const Geom& G, int t, int x0, int y0, int hr, int rows,
                                       bool halo_only) {
    int r, v;
    if (halo_only) {
      r = t >> 1;
      v = (t & 1) ? kNV - 1 : 0;
    } else {
      r = t / kNV;
      v = t - r * kNV;
    }
    int j = y0 - hr + r;
    ok = true;
    if (G.per_y) j = modi(j, G.ny);
    else if (j < 0 || j >= G.ny) ok = false;
    const int x = modi(x0 - kHX + 4 * v, G.nx);   // nx is a multiple of 4
    const bool mine = t >= 0 && r < rows;
    if (!mine) soff = -1;
    else if (v == 0) soff = rows * kTX + r * kHP;
    else if (v == kNV - 1) soff = rows * kTX + r * kHP + kHX;
    else soff = r * kTX + 4 * (v - 1);
    goff = ok ? j * G.nx + x : 0;
  }
  __device__ __forceinline__ void issue(float* slot, const float* base, bool pvalid) const {
    if (soff >= 0) cp_async16(slot + soff, base + goff, pvalid && ok);
  }
};

template <int NS>
struct SplitDesc {
  static_assert(NS >= 1 && NS <= 3, "at most three vectors per thread and plane");
  SplitVec v0, v1, v2;
  // whole planes: vectors tid, tid + kThreads, tid + 2 kThreads
  __device__ __forceinline__ void init(const Geom& G, int x0, int y0, int hr, int rows) {
    const int t = (int)threadIdx.x;
    v0.init(G, t, x0, y0, hr, rows, false);
    v1.init(G, NS > 1 ? t + kThreads : -1, x0, y0, hr, rows, false);
    v2.init(G, NS > 2 ? t + 2 * kThreads : -1, x0, y0, hr, rows, false);
  }
  // halo vectors only: this thread's is t (-1: none)
  __device__ __forceinline__ void init_halo(const Geom& G, int t, int x0, int y0, int hr, int rows) {
    v0.init(G, t < 2 * rows ? t : -1, x0, y0, hr, rows, true);
    v1.soff = -1;
    v2.soff = -1;
  }
  __device__ __forceinline__ void stage(float* slot, const float* __restrict__ src, const Geom& G,
                                        int plane) const {
    bool pvalid = true;
    int k = plane;
    if (G.per_z) k = wrapi(k, G.nz);
    else if (k < 0 || k >= G.nz) pvalid = false;
    const float* base = src + (pvalid ? (long long)k * G.ny * G.nx : 0LL);
    v0.issue(slot, base, pvalid);
    if (NS > 1) v1.issue(slot, base, pvalid);
    if (NS > 2) v2.issue(slot, base, pvalid);
  }
};

// Can the tiled kernels handle this level?  (All three axes active, x
// periodic, tile-aligned extents.)
inline bool level_ok(const Level& L) {
  return L.act[0] && L.act[1] && L.act[2] && L.per[0] && L.n[0] % kTX == 0 &&
         L.n[1] % kTY == 0 && L.n[2] >= 2;
}

// Ragged tiling (partial tiles at the x and y edges): every axis active, x
// periodic with an extent that is a multiple of one 16-byte vector, and at
// least two cells along y and z so that a cell meets at most one wall per
// axis.
inline bool ragged_ok(const Level& L) {
  return L.act[0] && L.act[1] && L.act[2] && L.per[0] && L.n[0] % 4 == 0 && L.n[1] >= 2 &&
         L.n[2] >= 2;
}

// Fraction of a level's tiles that holds cells (1 for tile-aligned levels).
inline double tile_fill(const Level& L) {
  const int tx = (L.n[0] + kTX - 1) / kTX, ty = (L.n[1] + kTY - 1) / kTY;
  return (double)L.n[0] * L.n[1] / ((double)tx * kTX * ty * kTY);
}

// z-chunk length for a tiled z-marching kernel on level L: the grid is
// (tiles x chunks x ncomp) CTAs, `slots` of which are resident at a time, and
// a chunk costs its planes plus about `halo` extra planes of pipeline fill.
// Picks the chunk that minimises waves x (chunk + halo), chunks of at least
// `min_chunk` planes unless the whole extent is shorter.
inline int pick_zchunk(const Level& L, int ncomp, int slots, int halo, int min_chunk = 8) {
  const int nz = L.n[2];
  const long long tiles =
      (long long)((L.n[0] + kTX - 1) / kTX) * ((L.n[1] + kTY - 1) / kTY) * ncomp;
  if (slots < 1) slots = 1;
  double best = 0.0;
  int best_chunk = nz;
  for (int nzc = 1; nzc <= nz; ++nzc) {
    const int chunk = (nz + nzc - 1) / nzc;
    if (chunk < min_chunk && nzc > 1) break;
    const long long blocks = tiles * ((nz + chunk - 1) / chunk);
    const long long waves = (blocks + slots - 1) / slots;
    const double eff = (double)(tiles * nz) / ((double)waves * slots * (chunk + halo));
    if (eff > best * (1.0 + 1e-9)) {
      best = eff;
      best_chunk = chunk;
    }
  }
  return best_chunk;
}

inline Geom geom(const Level& L, int zchunk) {
  Geom G;
  G.nx = L.n[0]; G.ny = L.n[1]; G.nz = L.n[2];
  G.per_y = L.per[1]; G.per_z = L.per[2];
  G.ntx = (L.n[0] + kTX - 1) / kTX; G.nty = (L.n[1] + kTY - 1) / kTY;
  G.zchunk = zchunk > 0 ? (zchunk < L.n[2] ? zchunk : L.n[2]) : L.n[2];
  return G;
}

}  // namespace tile
}  // namespace vsv
