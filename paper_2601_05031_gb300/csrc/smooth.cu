// Fused red-black Gauss-Seidel sweep: one full sweep (red then black) of the
// 7-point Poisson operator in a single pass over memory.
//
// A CTA owns a TX x TY tile of the (x, y) plane and marches along z.  At
// step p it updates the red cells of plane p (reading the old black values of
// planes p-1, p, p+1) and then the black cells of plane p-1 (reading the new
// red values of planes p-2, p-1, p), and stores the finished plane p-1.  The
// sweep reads x from A and writes it to B (ping-pong), so no CTA ever reads a
// value another CTA writes: red cells are recomputed on a one-cell halo ring
// around the tile from A (which needs a two-cell halo of A).  The result is
// bit-identical to the in-place red-then-black sweep.
//
// Planes are staged in shared memory by cp.async (16-byte vectors, zero fill
// for Dirichlet ghost rows/planes, wrap on periodic axes): a ring of five
// x-planes and three rhs planes, two planes of loads in flight.
#include "internal.h"

namespace vsv {

namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

constexpr int kTX = 128;   // tile width (x), multiple of 4
constexpr int kTY = 16;    // tile height (y)
constexpr int kH = 2;      // halo rows of x
constexpr int kHX = 4;     // halo columns (one 16-byte vector)
constexpr int kW = kTX + 2 * kHX;     // staged row length
constexpr int kRA = kTY + 2 * kH;     // staged x rows
constexpr int kRB = kTY + 2 * (kH - 1);  // staged rhs rows
constexpr int kNA = 5;     // x-plane ring slots
constexpr int kNB = 3;     // rhs-plane ring slots
constexpr int kThreads = 256;

struct FusedGeom {
  int nx, ny, nz;
  int per_y, per_z;
  int ntx, nty;          // tiles along x, y
  int zchunk;
  float alpha;           // Dirichlet closure of this level (0 on the finest)
  float h2;
  float beta;            // b = beta * B + S
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// stage one plane of `src` (rows y0-hr .. y0-hr+rows-1, columns x0-kHX ..)
__device__ __forceinline__ void stage_plane(float* dst, const float* __restrict__ src,
                                            const FusedGeom& G, int x0, int y0, int hr, int rows,
                                            int plane) {
  bool pvalid = true;
  int k = plane;
  if (G.per_z) k = wrapi(k, G.nz);
  else if (k < 0 || k >= G.nz) pvalid = false;
  const int nv = kW / 4;
  const int total = rows * nv;
  for (int t = threadIdx.x; t < total; t += kThreads) {
    const int r = t / nv, v = t - r * nv;
    int j = y0 - hr + r;
    bool valid = pvalid;
    if (G.per_y) j = wrapi(j, G.ny);
    else if (j < 0 || j >= G.ny) valid = false;
    const int x = wrapi(x0 - kHX + 4 * v, G.nx);
    const float* g = valid ? src + ((long long)k * G.ny + j) * G.nx + x : src;
    cp_async16(dst + r * kW + 4 * v, g, valid);
  }
}

}  // namespace

// One full red-black sweep A -> B for one component per blockIdx.z.
// Grid: x = ntx * nty tiles, y = z chunks, z = components.
__global__ void __launch_bounds__(kThreads, 2)
k_rbgs_fused(FusedGeom G, Comp3<float> A, Comp3<float> B, Rhs3<float> R) {
  extern __shared__ float4 smem_f4[];
  float* sA = reinterpret_cast<float*>(smem_f4);
  float* sB = sA + kNA * kRA * kW;
  const int comp = blockIdx.z;
  const float* __restrict__ a = A.p[comp];
  float* __restrict__ out = B.p[comp];
  const float* __restrict__ bsrc = R.B[comp];
  const float* __restrict__ S = R.S[comp];
  const int tx = blockIdx.x % G.ntx, ty = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = ty * kTY;
  const int zb = blockIdx.y * G.zchunk;
  const int ze = min(zb + G.zchunk, G.nz);
  const float beta = G.beta, h2 = G.h2;

  auto slotA = [&](int plane) { return sA + (((plane % kNA) + kNA) % kNA) * (kRA * kW); };
  auto slotB = [&](int plane) { return sB + (((plane % kNB) + kNB) % kNB) * (kRB * kW); };
  auto plane_is_ghost = [&](int p) { return !G.per_z && (p < 0 || p >= G.nz); };

  // Step p needs x planes p-2 .. p+1 and rhs planes p-1, p; it issues the
  // loads of step p+1 (x plane p+2, rhs plane p+1) before waiting for its own.
  // Prologue: what step zb-1 needs.
  stage_plane(slotA(zb - 2), a, G, x0, y0, kH, kRA, zb - 2);
  stage_plane(slotA(zb - 1), a, G, x0, y0, kH, kRA, zb - 1);
  stage_plane(slotA(zb), a, G, x0, y0, kH, kRA, zb);
  stage_plane(slotB(zb - 1), bsrc, G, x0, y0, kH - 1, kRB, zb - 1);
  cp_async_commit();

  for (int p = zb - 1; p <= ze; ++p) {
    if (p + 1 <= ze) {
      stage_plane(slotA(p + 2), a, G, x0, y0, kH, kRA, p + 2);
      stage_plane(slotB(p + 1), bsrc, G, x0, y0, kH - 1, kRB, p + 1);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    // ---- red cells of plane p on the tile plus a one-cell ring
    if (!plane_is_ghost(p)) {
      float* cA = slotA(p);
      const float* mA = slotA(p - 1);
      const float* pA = slotA(p + 1);
      const float* cB = slotB(p);
      const int ncol = (kTX + 2) / 2;
      const int items = (kRA - 2) * ncol;
      for (int t = threadIdx.x; t < items; t += kThreads) {
        const int rr = t / ncol, m = t - rr * ncol;
        const int r = rr + 1;
        const int j = y0 - kH + r;
        if (!G.per_y && (j < 0 || j >= G.ny)) continue;
        const int cf = kHX - 1 + ((x0 - 1 + j + p) & 1);
        const int c = cf + 2 * m;
        const int idx = r * kW + c;
        const float s = cA[idx - 1] + cA[idx + 1] + cA[idx - kW] + cA[idx + kW] + mA[idx] + pA[idx];
        int nwall = 0;
        if (!G.per_y) nwall += (j == 0) + (j == G.ny - 1);
        if (!G.per_z) nwall += (p == 0) + (p == G.nz - 1);
        const int jj = G.per_y ? wrapi(j, G.ny) : j;
        const int kk = G.per_z ? wrapi(p, G.nz) : p;
        float b = beta * cB[(r - 1) * kW + c];
        if (S) b += S[jj + (long long)kk * G.ny];
        cA[idx] = (s - b * h2) / (6.f + G.alpha * (float)nwall);
      }
    }
    __syncthreads();
    // ---- black cells of plane p-1 on the tile, then store the plane
    const int q = p - 1;
    if (q >= zb && q < ze) {
      float* cA = slotA(q);
      const float* mA = slotA(q - 1);
      const float* pA = slotA(q + 1);
      const float* cB = slotB(q);
      const int ncol = kTX / 2;
      const int items = kTY * ncol;
      for (int t = threadIdx.x; t < items; t += kThreads) {
        const int rr = t / ncol, m = t - rr * ncol;
        const int r = rr + kH;
        const int j = y0 + rr;
        const int cf = kHX + ((x0 + j + q + 1) & 1);
        const int c = cf + 2 * m;
        const int idx = r * kW + c;
        const float s = cA[idx - 1] + cA[idx + 1] + cA[idx - kW] + cA[idx + kW] + mA[idx] + pA[idx];
        int nwall = 0;
        if (!G.per_y) nwall += (j == 0) + (j == G.ny - 1);
        if (!G.per_z) nwall += (q == 0) + (q == G.nz - 1);
        float b = beta * cB[(r - 1) * kW + c];
        if (S) b += S[j + (long long)q * G.ny];
        cA[idx] = (s - b * h2) / (6.f + G.alpha * (float)nwall);
      }
      __syncthreads();
      const int nv = kTX / 4;
      for (int t = threadIdx.x; t < kTY * nv; t += kThreads) {
        const int rr = t / nv, v = t - rr * nv;
        const float4 val = *reinterpret_cast<const float4*>(cA + (rr + kH) * kW + kHX + 4 * v);
        *reinterpret_cast<float4*>(out + ((long long)q * G.ny + y0 + rr) * G.nx + x0 + 4 * v) = val;
      }
    }
    __syncthreads();
  }
  cp_async_wait0();
}

// Can the fused sweep handle this level?  (All three axes active, x
// periodic, tile-aligned extents.)
bool fused_sweep_ok(const Level& L) {
  return L.act[0] && L.act[1] && L.act[2] && L.per[0] && L.n[0] % kTX == 0 &&
         L.n[1] % kTY == 0 && L.n[2] >= 2;
}

size_t fused_sweep_smem() { return (size_t)(kNA * kRA + kNB * kRB) * kW * sizeof(float); }

// One fused full sweep A -> B on `ncomp` components.
void launch_rbgs_fused(Ctx& cx, const Level& L, Comp3<float> A, Comp3<float> B, Rhs3<float> R,
                       int ncomp, int zchunk, int kclass) {
  static bool attr_set = false;
  const size_t smem = fused_sweep_smem();
  if (!attr_set) {
    cudaFuncSetAttribute(k_rbgs_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  FusedGeom G;
  G.nx = L.n[0]; G.ny = L.n[1]; G.nz = L.n[2];
  G.per_y = L.per[1]; G.per_z = L.per[2];
  G.ntx = L.n[0] / kTX; G.nty = L.n[1] / kTY;
  G.zchunk = zchunk > 0 ? std::min(zchunk, L.n[2]) : L.n[2];
  G.alpha = L.alphaf;
  G.h2 = (float)(1.0 / L.inv_h2);
  G.beta = R.beta;
  const int nzc = (L.n[2] + G.zchunk - 1) / G.zchunk;
  dim3 grid(G.ntx * G.nty, nzc, ncomp);
  cx.before(kclass);
  k_rbgs_fused<<<grid, kThreads, smem, cx.stream>>>(G, A, B, R);
  cx.after(kclass);
}

}  // namespace vsv
