// Fused red-black Gauss-Seidel sweep: one full sweep (red then black) of the
// 7-point Poisson operator in a single pass over memory.
//
// A CTA owns a 128 x 16 tile of the (x, y) plane and marches along z.  At
// step p it updates the red cells of plane p (reading the old black values of
// planes p-1, p, p+1), then the black cells of plane p-1 (reading the new red
// values of planes p-2, p-1, p), and stores the finished plane p-1.  The sweep
// reads x from A and writes B (ping-pong), so no CTA reads a value another CTA
// writes: red cells are recomputed on a one-cell ring around the tile from A
// (two-cell halo of A).  Same arithmetic, same summation order as the
// per-colour kernel, hence bit-identical results.
//
// Work mapping: thread (gx, ty) of 32 x 8 owns the float4 column groups at
// x = x0 + 4 gx, rows ty and ty + 8.  It keeps its groups of planes p-2 .. p+1
// in registers (z-neighbours never touch shared memory); x / y neighbours come
// from the staged plane in shared memory by 128-bit loads.  Warps 0 and 7
// also do the red cells of the halo rows, 36 threads the two halo columns.
// Planes are staged by cp.async (16-byte vectors, zero fill on Dirichlet
// ghosts, wrap on periodic axes; two planes in flight) into a ring of five
// x-planes and three rhs planes.
#include "tile.cuh"

namespace vsv {

using namespace tile;

namespace {

constexpr int kH = 2;                    // halo rows of x
constexpr int kRA = kTY + 2 * kH;        // staged x rows
constexpr int kRB = kTY + 2 * (kH - 1);  // staged rhs rows
constexpr int kNA = 5;                   // x-plane ring slots
constexpr int kNB = 3;                   // rhs-plane ring slots
constexpr int kStageA = (kRA * kNV + kThreads - 1) / kThreads;   // vectors per thread
constexpr int kStageB = (kRB * kNV + kThreads - 1) / kThreads;

struct FusedGeom : Geom {
  float rc[7];           // 1 / (6 + alpha * nwall), as in Level::rcf
  float h2;
  float beta;            // b = beta * B + S
};

// Red (or black) update of one float4 group: the two cells at offsets par and
// par + 2, given own V (centre row), U / D (rows above / below), M / P
// (planes below / above), the scalar neighbours Lx / Rx and the rhs group
// Bv.  Returns V with those two components replaced.  Summation order x-, x+,
// y-, y+, z-, z+ as in the per-colour kernel.
__device__ __forceinline__ float4 rb_group(float4 V, float4 U, float4 D, float4 M, float4 P, float Lx,
                                           float Rx, float4 Bv, int par, float beta, float S,
                                           float h2, float rc) {
  if (par == 0) {
    const float b0 = beta * Bv.x + S, b2 = beta * Bv.z + S;
    const float s0 = Lx + V.y + U.x + D.x + M.x + P.x;
    const float s2 = V.y + V.w + U.z + D.z + M.z + P.z;
    V.x = (s0 - b0 * h2) * rc;
    V.z = (s2 - b2 * h2) * rc;
  } else {
    const float b1 = beta * Bv.y + S, b3 = beta * Bv.w + S;
    const float s1 = V.x + V.z + U.y + D.y + M.y + P.y;
    const float s3 = V.z + Rx + U.w + D.w + M.w + P.w;
    V.y = (s1 - b1 * h2) * rc;
    V.w = (s3 - b3 * h2) * rc;
  }
  return V;
}

}  // namespace

// One full red-black sweep A -> B for one component per blockIdx.z.
// Grid: x = ntx * nty tiles, y = z chunks, z = components.  ZERO_IN: A is
// taken as zero (first sweep of a correction from e = 0; A is not read).
template <bool ZERO_IN, bool HAS_S>
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
  const int tx = blockIdx.x % G.ntx, tyb = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = tyb * kTY;
  const int zb = blockIdx.y * G.zchunk;
  const int ze = min(zb + G.zchunk, G.nz);
  const float beta = G.beta, h2 = G.h2;
  const int tid = threadIdx.x, gx = tid & 31, ty = tid >> 5;
  const int q = gx + 1;                    // own float4 group (staged columns 4q .. 4q+3)

  auto slotA = [&](int plane) { return sA + (((plane % kNA) + kNA) % kNA) * (kRA * kW); };
  auto slotB = [&](int plane) { return sB + (((plane % kNB) + kNB) % kNB) * (kRB * kW); };
  auto ghost_plane = [&](int p) { return !G.per_z && (p < 0 || p >= G.nz); };
  auto zwall = [&](int p) { return G.per_z ? 0 : (p == 0) + (p == G.nz - 1); };
  auto srow = [&](int j, int p) -> float {
    if (!HAS_S) return 0.f;
    const int kk = G.per_z ? wrapi(p, G.nz) : p;
    return S[(G.per_y ? wrapi(j, G.ny) : j) + (long long)kk * G.ny];
  };

  StageDesc<kStageA> da;
  StageDesc<kStageB> db;
  da.init(G, x0, y0, kH, kRA);
  db.init(G, x0, y0, kH - 1, kRB);

  // own rows
  int rown[2], jown[2], ywall[2];
  for (int h = 0; h < 2; ++h) {
    rown[h] = ty + 8 * h + kH;
    jown[h] = y0 + ty + 8 * h;
    ywall[h] = G.per_y ? 0 : (jown[h] == 0) + (jown[h] == G.ny - 1);
  }

  // prologue: x planes zb-2 .. zb and rhs plane zb-1
  da.stage(slotA(zb - 2), a, G, zb - 2, ZERO_IN);
  da.stage(slotA(zb - 1), a, G, zb - 1, ZERO_IN);
  da.stage(slotA(zb), a, G, zb, ZERO_IN);
  db.stage(slotB(zb - 1), bsrc, G, zb - 1, false);
  cp_async_commit();
  cp_async_wait0();
  __syncthreads();
  // register pipeline: MM = plane p-2, M = p-1, V = p, P = p+1 (own groups);
  // rotated at the top of every step
  float4 MM[2], M[2], V[2], P[2];
  for (int h = 0; h < 2; ++h) {
    V[h] = lds4(slotA(zb - 2) + rown[h] * kW + 4 * q);
    P[h] = lds4(slotA(zb - 1) + rown[h] * kW + 4 * q);
    M[h] = V[h];
    MM[h] = V[h];
  }

  for (int p = zb - 1; p <= ze; ++p) {
    if (p + 1 <= ze) {
      da.stage(slotA(p + 2), a, G, p + 2, ZERO_IN);
      db.stage(slotB(p + 1), bsrc, G, p + 1, false);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    float* cA = slotA(p);
    const float* cB = slotB(p);
    for (int h = 0; h < 2; ++h) {
      MM[h] = M[h];
      M[h] = V[h];
      V[h] = P[h];
      P[h] = lds4(slotA(p + 1) + rown[h] * kW + 4 * q);
    }
    // ---- red cells of plane p: own groups, halo rows, halo columns
    if (!ghost_plane(p)) {
      const int zw = zwall(p);
      for (int h = 0; h < 2; ++h) {
        const int r = rown[h], j = jown[h];
        const float* row = cA + r * kW;
        const float4 U = lds4(row - kW + 4 * q), D = lds4(row + kW + 4 * q);
        const float Lx = row[4 * q - 1], Rx = row[4 * q + 4];
        const float4 Bv = lds4(cB + (r - 1) * kW + 4 * q);
        const int par = (j + p) & 1;
        V[h] = rb_group(V[h], U, D, M[h], P[h], Lx, Rx, Bv, par, beta, srow(j, p), h2,
                        G.rc[ywall[h] + zw]);
        float* dst = cA + r * kW + 4 * q;
        if (par == 0) { dst[0] = V[h].x; dst[2] = V[h].z; }
        else { dst[1] = V[h].y; dst[3] = V[h].w; }
      }
      if (ty == 0 || ty == 7) {   // halo rows y0 - 1 and y0 + kTY
        const int r = (ty == 0) ? 1 : kRA - 2;
        const int j = y0 - kH + r;
        if (G.per_y || (j >= 0 && j < G.ny)) {
          const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
          const float* row = cA + r * kW;
          const float4 Vh = lds4(row + 4 * q), U = lds4(row - kW + 4 * q), D = lds4(row + kW + 4 * q);
          const float4 Mh = lds4(slotA(p - 1) + r * kW + 4 * q);
          const float4 Ph = lds4(slotA(p + 1) + r * kW + 4 * q);
          const float Lx = row[4 * q - 1], Rx = row[4 * q + 4];
          const float4 Bv = lds4(cB + (r - 1) * kW + 4 * q);
          const int par = (j + p) & 1;
          const float4 Vn = rb_group(Vh, U, D, Mh, Ph, Lx, Rx, Bv, par, beta, srow(j, p), h2,
                                     G.rc[jw + zw]);
          float* dst = cA + r * kW + 4 * q;
          if (par == 0) { dst[0] = Vn.x; dst[2] = Vn.z; }
          else { dst[1] = Vn.y; dst[3] = Vn.w; }
        }
      }
      if (tid >= 32 && tid < 32 + 2 * (kRA - 2)) {   // halo columns x0 - 1 and x0 + kTX
        const int idx = tid - 32;
        const int r = 1 + (idx >> 1);
        const int c = (idx & 1) ? kHX + kTX : kHX - 1;
        const int j = y0 - kH + r;
        const int x = x0 - kHX + c;
        if ((G.per_y || (j >= 0 && j < G.ny)) && (((x + j + p) & 1) == 0)) {
          const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
          const int id = r * kW + c;
          const float s = cA[id - 1] + cA[id + 1] + cA[id - kW] + cA[id + kW] + slotA(p - 1)[id] +
                          slotA(p + 1)[id];
          const float bb = beta * cB[(r - 1) * kW + c] + srow(j, p);
          cA[id] = (s - bb * h2) * G.rc[jw + zw];
        }
      }
    }
    __syncthreads();
    // ---- black cells of plane p-1 on the tile, stored straight from registers
    const int qp = p - 1;
    if (qp >= zb && qp < ze) {
      const int zw = zwall(qp);
      const float* cAq = slotA(qp);
      const float* cBq = slotB(qp);
      for (int h = 0; h < 2; ++h) {
        const int r = rown[h], j = jown[h];
        const float* row = cAq + r * kW;
        const float4 U = lds4(row - kW + 4 * q), D = lds4(row + kW + 4 * q);
        const float Lx = row[4 * q - 1], Rx = row[4 * q + 4];
        const float4 Bv = lds4(cBq + (r - 1) * kW + 4 * q);
        const int par = (j + qp + 1) & 1;
        M[h] = rb_group(M[h], U, D, MM[h], V[h], Lx, Rx, Bv, par, beta, srow(j, qp), h2,
                        G.rc[ywall[h] + zw]);
        *reinterpret_cast<float4*>(out + ((long long)qp * G.ny + j) * G.nx + x0 + 4 * gx) = M[h];
      }
    }
    __syncthreads();
  }
  cp_async_wait0();
}

// Can the fused sweep handle this level?  (All three axes active, x
// periodic, tile-aligned extents.)
bool fused_sweep_ok(const Level& L) { return level_ok(L); }

size_t fused_sweep_smem() { return (size_t)(kNA * kRA + kNB * kRB) * kW * sizeof(float); }

template <bool Z, bool HS>
static void launch_variant(dim3 grid, size_t smem, cudaStream_t s, const FusedGeom& G,
                           Comp3<float> A, Comp3<float> B, Rhs3<float> R) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_rbgs_fused<Z, HS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  k_rbgs_fused<Z, HS><<<grid, kThreads, smem, s>>>(G, A, B, R);
}

// One fused full sweep A -> B on `ncomp` components (zero_in: A taken as 0).
void launch_rbgs_fused(Ctx& cx, const Level& L, Comp3<float> A, Comp3<float> B, Rhs3<float> R,
                       int ncomp, int zchunk, int kclass, bool zero_in) {
  const size_t smem = fused_sweep_smem();
  FusedGeom G;
  G.nx = L.n[0]; G.ny = L.n[1]; G.nz = L.n[2];
  G.per_y = L.per[1]; G.per_z = L.per[2];
  G.ntx = L.n[0] / kTX; G.nty = L.n[1] / kTY;
  G.zchunk = zchunk > 0 ? std::min(zchunk, L.n[2]) : L.n[2];
  for (int q = 0; q < 7; ++q) G.rc[q] = L.rcf[q];
  G.h2 = (float)(1.0 / L.inv_h2);
  G.beta = R.beta;
  const int nzc = (L.n[2] + G.zchunk - 1) / G.zchunk;
  dim3 grid(G.ntx * G.nty, nzc, ncomp);
  const bool hs = R.S[0] != nullptr;
  cx.before(kclass);
  if (zero_in) {
    if (hs) launch_variant<true, true>(grid, smem, cx.stream, G, A, B, R);
    else launch_variant<true, false>(grid, smem, cx.stream, G, A, B, R);
  } else {
    if (hs) launch_variant<false, true>(grid, smem, cx.stream, G, A, B, R);
    else launch_variant<false, false>(grid, smem, cx.stream, G, A, B, R);
  }
  cx.after(kclass);
}

}  // namespace vsv
