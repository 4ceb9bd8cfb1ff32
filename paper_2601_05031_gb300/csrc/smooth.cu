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
// also do the red cells of the halo rows, warp 1 those of the two halo
// columns beside the owned rows (the ring's corners are never read: the
// black cells next to them are not updated).
//
// Staging (two steps of copies in flight, a ring of six x planes and five
// rhs planes in shared memory, split layout of tile.cuh: body rows of the
// tile's 128 columns, then the 4-column halo groups left and right of it):
// on tile-aligned levels without periodic y the body of a plane is one box
// of a TMA tensor map (zeros beyond a y or z wall come from the box's
// out-of-bounds fill), the halo groups -- wrapped around periodic x, which a
// box cannot do -- are 16-byte cp.async copies; elsewhere every 16-byte
// vector is a cp.async copy with zero fill on Dirichlet ghosts.
#include <cuda.h>   // CUtensorMap and the encoder's types; the driver is reached at run time

#include <algorithm>
#include <cstring>

#include "tile.cuh"

namespace vsv {

using namespace tile;

namespace {

constexpr int kH = 2;                    // halo rows of x
constexpr int kRA = kTY + 2 * kH;        // staged x rows
constexpr int kRB = kTY + 2 * (kH - 1);  // staged rhs rows
constexpr int kNA = 6;                   // x-plane ring slots
constexpr int kNB = 5;                   // rhs-plane ring slots
// slot sizes (floats): body and halo rows, rounded up to 128 bytes so that
// every slot can take a box
constexpr int kSlotA = (kRA * (kTX + kHP) + 31) / 32 * 32;
constexpr int kSlotB = (kRB * (kTX + kHP) + 31) / 32 * 32;
constexpr int kStageA = (kRA * kNV + kThreads - 1) / kThreads;   // vectors per thread
constexpr int kStageB = (kRB * kNV + kThreads - 1) / kThreads;
constexpr int kIssueTid = 160;           // issues the boxes (warp 5: no halo duties)
constexpr int kHaloTid = 128;            // first of the 2 kRA + 2 kRB halo-copy threads
constexpr unsigned kBoxA = kRA * kTX * 4, kBoxB = kRB * kTX * 4;   // bytes per box
static_assert(kHaloTid + 2 * (kRA + kRB) <= kThreads, "halo copies need a thread each");

struct FusedGeom : Geom {
  // omega / (6 + alpha * nwall) for nwall = 0, 1, 2: the relaxation weight
  // times Level::rcf, rounded as relax() expects
  float rc0, rc1, rc2;
  float h2;
  float beta;            // b = beta * B + S
  float c1;              // 1 - omega
  int* status;           // device flag word (kCopyTimeout)
  unsigned long long limit_ns;   // bound of each wait for staged planes
  // > 0 only in the check of that bound: every copy group expects this
  // many bytes and no box is loaded, so each wait runs out
  unsigned probe_tx;
};

// tensor maps of the three components' x (boxes of kRA rows) and rhs (kRB
// rows); unused by the cp.async variant
struct FusedMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

// nwall is at most 2 on a tile-aligned level (ny >= 16 and nz >= 2 keep the
// two walls of an axis apart, and x is periodic).
__device__ __forceinline__ float rc_of(const FusedGeom& G, int nwall) {
  return nwall == 0 ? G.rc0 : (nwall == 1 ? G.rc1 : G.rc2);
}

// Red (or black) update of one float4 group: the two cells at offsets par and
// par + 2, given own V (centre row), U / D (rows above / below), M / P
// (planes below / above), the scalar neighbours Lx / Rx and the rhs group
// Bv.  Returns V with those two components replaced (relaxed by omega from
// their old values).  Neighbours summed as ((x- + x+) + (y- + y+)) +
// (z- + z+), as in the per-colour kernel.
__device__ __forceinline__ float4 rb_group(float4 V, float4 U, float4 D, float4 M, float4 P, float Lx,
                                           float Rx, float4 Bv, int par, float beta, float S,
                                           float h2, float wrc, float c1) {
  if (par == 0) {
    const float b0 = beta * Bv.x + S, b2 = beta * Bv.z + S;
    const float s0 = ((Lx + V.y) + (U.x + D.x)) + (M.x + P.x);
    const float s2 = ((V.y + V.w) + (U.z + D.z)) + (M.z + P.z);
    V.x = relax(V.x, nb_term(s0, b0, h2), wrc, c1);
    V.z = relax(V.z, nb_term(s2, b2, h2), wrc, c1);
  } else {
    const float b1 = beta * Bv.y + S, b3 = beta * Bv.w + S;
    const float s1 = ((V.x + V.z) + (U.y + D.y)) + (M.y + P.y);
    const float s3 = ((V.z + Rx) + (U.w + D.w)) + (M.w + P.w);
    V.y = relax(V.y, nb_term(s1, b1, h2), wrc, c1);
    V.w = relax(V.w, nb_term(s3, b3, h2), wrc, c1);
  }
  return V;
}

__device__ __forceinline__ float* ring(float* base, int plane, int slots, int slot_elems) {
  return base + ((unsigned)(plane + slots) % (unsigned)slots) * slot_elems;   // plane >= -slots
}

}  // namespace

// One full red-black sweep A -> B for one component per blockIdx.z.
// Grid: x = ntx * nty tiles, y = z chunks, z = components.  ZERO_IN: A is
// taken as zero (first sweep of a correction from e = 0; A is not read).
// UPD: the swept values are not stored to B but added to the double-word
// iterate, (XH, XL) <- (XH, XL) + e, with the arithmetic of k_update_dw (the
// last sweep of a correction's V-cycle; e itself is not needed afterwards).
// RAGGED: partial edge tiles, every staged vector a cp.async copy; else a
// tile-aligned level without periodic y whose plane bodies are boxes of the
// tensor maps M.
//
// Pipeline: step p updates the red cells of plane p and the black cells of
// plane p - 2.  The two phases are independent (the black cells need the red
// values of planes p - 3 .. p - 1, finished in earlier steps), so their
// loads and arithmetic overlap.  At step p the CTA waits for the copies of
// step p - 2 (x plane p + 1, rhs plane p), passes the one barrier of the
// step and then issues the copies of x plane p + 3 and rhs plane p + 2, so
// two steps of copies are in flight.  Within a step the red phase writes only
// red cells of slot p and reads black cells of slots p - 1 .. p + 1, and the
// black phase reads slot p - 2 plus registers; issuing after the barrier
// keeps the copies out of the slots of plane p - 3, which the black phase of
// step p - 1 read (six x and five rhs slots).  The boxes of step group s
// (the planes step zb - 1 + s needs) are counted on mbarrier s & 1.
template <bool ZERO_IN, bool HAS_S, bool UPD, bool RAGGED>
__global__ void __launch_bounds__(kThreads, 2)
k_rbgs_fused(FusedGeom G, Comp3<float> A, Comp3<float> B, Rhs3<float> R, Comp3<float> XH,
             Comp3<float> XL, const __grid_constant__ FusedMaps M) {
  pdl_begin();
  constexpr bool TMA = !RAGGED;
  extern __shared__ float4 smem_f4[];
  // boxes land on 128-byte boundaries: align the rings' base (by pointer
  // arithmetic on the shared array, so that accesses stay shared-space ones)
  float* sA = reinterpret_cast<float*>(smem_f4) + (((128u - (smem_u32(smem_f4) & 127u)) & 127u) >> 2);
  float* sB = sA + kNA * kSlotA;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sB + kNB * kSlotB);
  const int comp = blockIdx.z;
  const float* __restrict__ a = A.at(comp);
  float* __restrict__ out = B.at(comp);
  float* __restrict__ uh = XH.at(comp);
  float* __restrict__ ul = XL.at(comp);
  const float* __restrict__ bsrc = R.b_at(comp);
  const float* __restrict__ S = R.s_at(comp);
  const int tx = blockIdx.x % G.ntx, tyb = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = tyb * kTY;
  const int zb = blockIdx.y * G.zchunk;
  const int ze = min(zb + G.zchunk, G.nz);
  const int sLast = ze - zb + 1;             // last copy group
  const float beta = G.beta, h2 = G.h2, c1 = G.c1;
  const int tid = threadIdx.x, gx = tid & 31, ty = tid >> 5;

  auto slotA = [&](int plane) { return ring(sA, plane, kNA, kSlotA); };
  auto slotB = [&](int plane) { return ring(sB, plane, kNB, kSlotB); };
  // halo row r of an x or rhs slot: [0, kHX) left of the tile, [kHX, kHP) right
  auto hA = [&](auto* slot, int r) { return halo_row(slot, kRA, r); };
  auto hB = [&](auto* slot, int r) { return halo_row(slot, kRB, r); };
  auto ghost_plane = [&](int p) { return !G.per_z && (p < 0 || p >= G.nz); };
  auto zwall = [&](int p) { return G.per_z ? 0 : (p == 0) + (p == G.nz - 1); };
  auto srow = [&](int j, int p) -> float {
    if (!HAS_S) return 0.f;
    const int kk = G.per_z ? wrapi(p, G.nz) : p;
    return S[(G.per_y ? (RAGGED ? modi(j, G.ny) : wrapi(j, G.ny)) : j) + (long long)kk * G.ny];
  };

  // cp.async vectors of this thread: whole planes (RAGGED) or one halo group
  // of an x or rhs row (threads kHaloTid ..)
  SplitDesc<kStageA> da;
  SplitDesc<kStageB> db;
  if constexpr (RAGGED) {
    da.init(G, x0, y0, kH, kRA);
    db.init(G, x0, y0, kH - 1, kRB);
  } else {
    da.init_halo(G, tid - kHaloTid, x0, y0, kH, kRA);
    db.init_halo(G, tid - kHaloTid - 2 * kRA, x0, y0, kH - 1, kRB);
  }
  auto stage_x = [&](float* slot, int plane) {
    if constexpr (!ZERO_IN) da.stage(slot, a, G, plane);
  };
  auto stage_b = [&](float* slot, int plane) { db.stage(slot, bsrc, G, plane); };
  // boxes (one thread; planes beyond a z wall lie outside the tensor and
  // read as zero): arm the group's barrier with its bytes -- false in the
  // check of the wait bound, which loads no box -- then load
  auto arm = [&](unsigned long long* bar, unsigned bytes) {
    mbar_arrive_expect_tx(bar, G.probe_tx ? G.probe_tx : bytes);
    return G.probe_tx == 0u;
  };
  auto box_x = [&](float* slot, int plane, unsigned long long* bar) {
    tma_load_3d(slot, &M.a[comp], x0, y0 - kH, G.per_z ? wrapi(plane, G.nz) : plane, bar);
  };
  auto box_b = [&](float* slot, int plane, unsigned long long* bar) {
    tma_load_3d(slot, &M.b[comp], x0, y0 - (kH - 1), G.per_z ? wrapi(plane, G.nz) : plane, bar);
  };
  // after a wait that ran out: boxes of groups grp and grp + 1 may still be
  // in flight into this CTA's shared memory, and this thread's cp.async copies
  auto bail = [&](int grp) {
    cp_async_wait0();
    if (tid == 0)
      for (int g = grp; g <= grp + 1 && g <= sLast; ++g)
        mbar_drain(&bars[g & 1], (g >> 1) & 1, G.limit_ns);
  };

  // own rows (2 ty and 2 ty + 1: each is the other's y neighbour, straight
  // from registers) and their 1 / diagonal for z-interior (0) and z-wall (1)
  // planes
  int rown[2], jown[2];
  float rco[2][2];
  // RAGGED (partial edge tiles): a row past a wall stays the staged zero
  // ghost (not updated); a row or column past the extent of a periodic axis
  // holds a wrapped copy whose updates repeat its owner's (same inputs, same
  // arithmetic), so only the stores to memory are masked
  bool upd_row[2], st_row[2];
  const bool xok = !RAGGED || x0 + 4 * gx < G.nx;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    rown[h] = 2 * ty + h + kH;
    jown[h] = y0 + 2 * ty + h;
    upd_row[h] = !RAGGED || G.per_y || jown[h] < G.ny;
    st_row[h] = !RAGGED || (jown[h] < G.ny && xok);
    const int yw = G.per_y ? 0 : (jown[h] == 0) + (jown[h] == G.ny - 1);
    rco[h][0] = rc_of(G, yw);
    rco[h][1] = rc_of(G, yw + 1);
  }

  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_mbar_init();
    }
  }
  // ZERO_IN: x is not staged at all.  The ring is zeroed once; afterwards
  // only red positions of in-range cells are ever written (the ring length 6
  // is even, so a slot position keeps its colour), and within a plane no red
  // value is read before that plane's red phase writes it.  So every value a
  // sweep from zero reads -- black cells, wall rows, halo values -- is the
  // zero that staging would have copied.  Planes beyond a z wall are taken
  // as zero in registers (their slots hold an earlier plane's red values).
  if constexpr (ZERO_IN) {
    float4* a4 = reinterpret_cast<float4*>(sA);
    for (int t = tid; t < kNA * kSlotA / 4; t += kThreads) a4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if constexpr (TMA) __syncthreads();   // initialised barriers before the first box
  // prologue: group 0 = x planes zb-2 .. zb, rhs plane zb-1 (step zb-1);
  // group 1 = x plane zb+1, rhs plane zb (step zb)
  if constexpr (TMA) {
    if (tid == kIssueTid && arm(&bars[0], (ZERO_IN ? 0u : 3u * kBoxA) + kBoxB)) {
      if constexpr (!ZERO_IN)
        for (int i = -2; i <= 0; ++i) box_x(slotA(zb + i), zb + i, &bars[0]);
      box_b(slotB(zb - 1), zb - 1, &bars[0]);
    }
  }
  for (int i = -2; i <= 0; ++i) stage_x(slotA(zb + i), zb + i);
  stage_b(slotB(zb - 1), zb - 1);
  cp_async_commit();
  if constexpr (TMA) {
    if (tid == kIssueTid && arm(&bars[1], (ZERO_IN ? 0u : kBoxA) + kBoxB)) {
      if constexpr (!ZERO_IN) box_x(slotA(zb + 1), zb + 1, &bars[1]);
      box_b(slotB(zb), zb, &bars[1]);
    }
  }
  stage_x(slotA(zb + 1), zb + 1);
  stage_b(slotB(zb), zb);
  cp_async_commit();
  cp_async_wait1();
  if constexpr (TMA) {
    if (!mbar_wait_cta(&bars[0], 0u, G.status, G.limit_ns)) {
      bail(0);
      return;
    }
  } else {
    __syncthreads();
  }
  // register pipeline: MMM = plane p-3, MM = p-2, M = p-1, V = p, P = p+1
  // (own groups); rotated at the top of every step
  float4 MMM[2], MM[2], M_[2], V[2], P[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    V[h] = lds4(slotA(zb - 2) + rown[h] * kTX + 4 * gx);
    P[h] = lds4(slotA(zb - 1) + rown[h] * kTX + 4 * gx);
    M_[h] = V[h];
    MM[h] = V[h];
    MMM[h] = V[h];
  }
  // ring slots (offsets into the rings, in floats) of x planes p - 2 .. p + 3
  // and rhs planes p - 2 .. p + 2 at the top of step p, rotated at its end
  // (no divisions in the loop)
  auto offA = [&](int plane) { return (int)(slotA(plane) - sA); };
  auto offB = [&](int plane) { return (int)(slotB(plane) - sB); };
  int oa0 = offA(zb - 3), oa1 = offA(zb - 2), oa2 = offA(zb - 1), oa3 = offA(zb), oa4 = offA(zb + 1),
      oa5 = offA(zb + 2);
  int ob0 = offB(zb - 3), ob1 = offB(zb - 2), ob2 = offB(zb - 1), ob3 = offB(zb), ob4 = offB(zb + 1);

  for (int p = zb - 1; p <= ze + 1; ++p) {
    float* const xa0 = sA + oa0;
    float* const xa1 = sA + oa1;
    float* const xa2 = sA + oa2;
    float* const xa3 = sA + oa3;
    float* const xa5 = sA + oa5;
    const float* const rb0 = sB + ob0;
    const float* const rb2 = sB + ob2;
    float* const rb4 = sB + ob4;
    const int qp = p - 2;
    const bool black = qp >= zb && qp < ze;
    // UPD: the iterate of plane p - 2, loaded ahead of the barrier so that
    // its latency overlaps the wait
    float4 XHp[2], XLp[2];
    if constexpr (UPD) {
      if (black) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!st_row[h]) continue;
          const long long gi = ((long long)qp * G.ny + jown[h]) * G.nx + x0 + 4 * gx;
          XHp[h] = *reinterpret_cast<const float4*>(uh + gi);
          XLp[h] = *reinterpret_cast<const float4*>(ul + gi);
        }
      }
    }
    // the copies of step p - 2 (x plane p + 1, rhs plane p) have landed;
    // after the barrier no warp is in step p - 1 any more, so the slots of
    // planes p - 3 (x) and p - 3 (rhs), last read by the black phase of step
    // p - 1, are free for the copies this step issues
    cp_async_wait1();
    if constexpr (TMA) {
      // this thread's earlier shared-memory writes (red values) are ordered
      // before the boxes loaded after the barrier
      fence_proxy_async();
      const int grp = p - zb + 1;
      if (grp <= sLast) {
        if (!mbar_wait_cta(&bars[grp & 1], (unsigned)(grp >> 1) & 1u, G.status, G.limit_ns)) {
          bail(grp);
          return;
        }
      } else {
        __syncthreads();
      }
    } else {
      __syncthreads();
    }
    if (p + 2 <= ze) {
      if constexpr (TMA) {
        unsigned long long* bar = &bars[(p - zb + 3) & 1];
        if (tid == kIssueTid && arm(bar, (ZERO_IN ? 0u : kBoxA) + kBoxB)) {
          if constexpr (!ZERO_IN) box_x(xa5, p + 3, bar);
          box_b(rb4, p + 2, bar);
        }
      }
      stage_x(xa5, p + 3);
      stage_b(rb4, p + 2);
    }
    cp_async_commit();
    float* cA = xa2;
    const float* cB = rb2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      MMM[h] = MM[h];
      MM[h] = M_[h];
      M_[h] = V[h];
      V[h] = P[h];
      // ZERO_IN: the black values of plane p + 1 are zero and its red ones
      // are written by the red phase of the next step before any read
      P[h] = (ZERO_IN || p > ze) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                 : lds4(xa3 + rown[h] * kTX + 4 * gx);
    }
    // the black phase's operands from shared memory: the y neighbours of
    // the two rows, their rhs groups and, at the tile edges, the x halo
    float4 U0, D1, Bq0, Bq1;
    float Le[2], Re[2];
    auto black_load = [&]() {
      if (black) {
        const float* cAq = xa0;
        const float* cBq = rb0;
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          // lanes 0 and 31 need x0 - 1 and x0 + kTX: one load for both
          const float e = hA(cAq, rown[h])[gx == 31 ? kHX : kHX - 1];
          Le[h] = gx == 0 ? e : 0.f;
          Re[h] = gx == 31 ? e : 0.f;
        }
        U0 = lds4(cAq + (rown[0] - 1) * kTX + 4 * gx);
        D1 = lds4(cAq + (rown[1] + 1) * kTX + 4 * gx);
        Bq0 = lds4(cBq + (rown[0] - 1) * kTX + 4 * gx);
        Bq1 = lds4(cBq + (rown[1] - 1) * kTX + 4 * gx);
      }
    };
    auto black_phase = [&]() {
      // ---- black cells of plane p-2 on the tile, stored straight from
      // registers.  They need the red values of planes p-3 .. p-1, all final,
      // so this phase does not depend on the red phase of the same step.
      if (black) {
        const int zw = zwall(qp);
        const int par = (jown[0] + qp + 1) & 1;     // black offset of row 2ty
        float Lq[2], Rq[2];
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          Lq[h] = __shfl_up_sync(0xffffffffu, MM[h].w, 1);
          Rq[h] = __shfl_down_sync(0xffffffffu, MM[h].x, 1);
          if (gx == 0) Lq[h] = Le[h];
          if (gx == 31) Rq[h] = Re[h];
        }
        const float4 M0 = MM[0];
        if (upd_row[0])
          MM[0] = rb_group(MM[0], U0, MM[1], MMM[0], M_[0], Lq[0], Rq[0], Bq0, par, beta,
                           srow(jown[0], qp), h2, zw ? rco[0][1] : rco[0][0], c1);
        if (upd_row[1])
          MM[1] = rb_group(MM[1], M0, D1, MMM[1], M_[1], Lq[1], Rq[1], Bq1, 1 - par, beta,
                           srow(jown[1], qp), h2, zw ? rco[1][1] : rco[1][0], c1);
      }
    };
    auto black_store = [&]() {
      if (black) {
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!st_row[h]) continue;
          const long long gi = ((long long)qp * G.ny + jown[h]) * G.nx + x0 + 4 * gx;
          if constexpr (UPD) {
            const FF v0 = ff_add_f(FF{XHp[h].x, XLp[h].x}, MM[h].x);
            const FF v1 = ff_add_f(FF{XHp[h].y, XLp[h].y}, MM[h].y);
            const FF v2 = ff_add_f(FF{XHp[h].z, XLp[h].z}, MM[h].z);
            const FF v3 = ff_add_f(FF{XHp[h].w, XLp[h].w}, MM[h].w);
            *reinterpret_cast<float4*>(uh + gi) = make_float4(v0.hi, v1.hi, v2.hi, v3.hi);
            *reinterpret_cast<float4*>(ul + gi) = make_float4(v0.lo, v1.lo, v2.lo, v3.lo);
          } else {
            *reinterpret_cast<float4*>(out + gi) = MM[h];
          }
        }
      }
    };
    // the red phase's shared-memory operands for the own groups (same
    // roles as the black phase's)
    const bool red = p <= ze && !ghost_plane(p);
    float4 U0r, D1r, B0r, B1r;
    float Ler[2], Rer[2];
    auto red_load = [&]() {
      if (red) {
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float e = hA(cA, rown[h])[gx == 31 ? kHX : kHX - 1];
          Ler[h] = gx == 0 ? e : 0.f;
          Rer[h] = gx == 31 ? e : 0.f;
        }
        U0r = lds4(cA + (rown[0] - 1) * kTX + 4 * gx);
        D1r = lds4(cA + (rown[1] + 1) * kTX + 4 * gx);
        B0r = lds4(cB + (rown[0] - 1) * kTX + 4 * gx);
        B1r = lds4(cB + (rown[1] - 1) * kTX + 4 * gx);
      }
    };
    // ZERO_IN: every neighbour of a red cell is black and still zero, so the
    // red update is the scaled rhs alone: (0 - b h^2) rc, the value the
    // general form gives with a zero neighbour sum
    auto red_phase_zero = [&]() {
      if (!red) return;
      const int zw = zwall(p);
      const int par = (jown[0] + p) & 1;          // red offset of row 2ty
  #pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!upd_row[h]) continue;
        const float4 Bv = h == 0 ? B0r : B1r;
        const float sr = srow(jown[h], p), rc = zw ? rco[h][1] : rco[h][0];
        float* dst = cA + rown[h] * kTX + 4 * gx;
        if ((h == 0 ? par : 1 - par) == 0) {
          V[h].x = relax(0.f, nb_term(0.f, beta * Bv.x + sr, h2), rc, c1);
          V[h].z = relax(0.f, nb_term(0.f, beta * Bv.z + sr, h2), rc, c1);
          dst[0] = V[h].x; dst[2] = V[h].z;
        } else {
          V[h].y = relax(0.f, nb_term(0.f, beta * Bv.y + sr, h2), rc, c1);
          V[h].w = relax(0.f, nb_term(0.f, beta * Bv.w + sr, h2), rc, c1);
          dst[1] = V[h].y; dst[3] = V[h].w;
        }
      }
      if (ty == 0 || ty == 7) {   // halo rows y0 - 1 and y0 + kTY
        const int r = (ty == 0) ? 1 : kRA - 2;
        const int j = y0 - kH + r;
        if (G.per_y || (j >= 0 && j < G.ny)) {
          const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
          const float4 Bv = lds4(cB + (r - 1) * kTX + 4 * gx);
          const float sr = srow(j, p), rc = rc_of(G, jw + zw);
          float* dst = cA + r * kTX + 4 * gx;
          if (((j + p) & 1) == 0) {
            dst[0] = relax(0.f, nb_term(0.f, beta * Bv.x + sr, h2), rc, c1);
            dst[2] = relax(0.f, nb_term(0.f, beta * Bv.z + sr, h2), rc, c1);
          } else {
            dst[1] = relax(0.f, nb_term(0.f, beta * Bv.y + sr, h2), rc, c1);
            dst[3] = relax(0.f, nb_term(0.f, beta * Bv.w + sr, h2), rc, c1);
          }
        }
      }
      if ((tid >> 5) == 1) {   // halo columns x0 - 1 and x0 + kTX beside the own rows
        const int idx = tid - 32;
        const int r = kH + (idx >> 1);
        const int side = idx & 1;                     // 0: x0 - 1, 1: x0 + kTX
        const int hc = side ? kHX : kHX - 1;          // its place in the halo row
        const int j = y0 - kH + r;
        const int x = side ? x0 + kTX : x0 - 1;
        if ((G.per_y || (j >= 0 && j < G.ny)) && (((x + j + p) & 1) == 0)) {
          const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
          const float bb = beta * hB(cB, r - 1)[hc] + srow(j, p);
          hA(cA, r)[hc] = relax(0.f, nb_term(0.f, bb, h2), rc_of(G, jw + zw), c1);
        }
      }
    };
    auto red_phase = [&]() {
      // ---- red cells of plane p: own groups, halo rows, halo columns
      if constexpr (ZERO_IN) {
        red_phase_zero();
        return;
      }
      if (red) {
        const int zw = zwall(p);
        // rows 2ty and 2ty+1 have opposite parity; each row's red cells need the
        // other row's black values (registers) and one more row from shared
        // memory; the x neighbours come from the adjacent lanes' registers
        // (black values, which this phase does not change) and, at the tile
        // edges, from the staged halo columns
        const int par = (jown[0] + p) & 1;          // red offset of row 2ty
        float Lx[2], Rx[2];
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          Lx[h] = __shfl_up_sync(0xffffffffu, V[h].w, 1);
          Rx[h] = __shfl_down_sync(0xffffffffu, V[h].x, 1);
          if (gx == 0) Lx[h] = Ler[h];
          if (gx == 31) Rx[h] = Rer[h];
        }
        const float4 U0 = U0r, D1 = D1r, B0 = B0r, B1 = B1r;
        const float4 V0 = V[0];
        if (upd_row[0])
          V[0] = rb_group(V[0], U0, V[1], M_[0], P[0], Lx[0], Rx[0], B0, par, beta,
                          srow(jown[0], p), h2, zw ? rco[0][1] : rco[0][0], c1);
        if (upd_row[1])
          V[1] = rb_group(V[1], V0, D1, M_[1], P[1], Lx[1], Rx[1], B1, 1 - par, beta,
                          srow(jown[1], p), h2, zw ? rco[1][1] : rco[1][0], c1);
        {
          float* dst = cA + rown[0] * kTX + 4 * gx;
          if (upd_row[0]) {
            if (par == 0) { dst[0] = V[0].x; dst[2] = V[0].z; }
            else { dst[1] = V[0].y; dst[3] = V[0].w; }
          }
          dst += kTX;
          if (upd_row[1]) {
            if (par == 0) { dst[1] = V[1].y; dst[3] = V[1].w; }
            else { dst[0] = V[1].x; dst[2] = V[1].z; }
          }
        }
        if (ty == 0 || ty == 7) {   // halo rows y0 - 1 and y0 + kTY
          const int r = (ty == 0) ? 1 : kRA - 2;
          const int j = y0 - kH + r;
          if (G.per_y || (j >= 0 && j < G.ny)) {
            const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
            const float* row = cA + r * kTX;
            const float4 Vh = lds4(row + 4 * gx), U = lds4(row - kTX + 4 * gx),
                         D = lds4(row + kTX + 4 * gx);
            const float4 Mh = lds4(xa1 + r * kTX + 4 * gx);
            const float4 Ph = lds4(xa3 + r * kTX + 4 * gx);
            const float Lx = gx == 0 ? hA(cA, r)[kHX - 1] : row[4 * gx - 1];
            const float Rx = gx == 31 ? hA(cA, r)[kHX] : row[4 * gx + 4];
            const float4 Bv = lds4(cB + (r - 1) * kTX + 4 * gx);
            const int par = (j + p) & 1;
            const float4 Vn = rb_group(Vh, U, D, Mh, Ph, Lx, Rx, Bv, par, beta, srow(j, p), h2,
                                       rc_of(G, jw + zw), c1);
            float* dst = cA + r * kTX + 4 * gx;
            if (par == 0) { dst[0] = Vn.x; dst[2] = Vn.z; }
            else { dst[1] = Vn.y; dst[3] = Vn.w; }
          }
        }
        if ((tid >> 5) == 1) {   // halo columns x0 - 1 and x0 + kTX beside the own rows
          const int idx = tid - 32;
          const int r = kH + (idx >> 1);
          const int side = idx & 1;                     // 0: x0 - 1, 1: x0 + kTX
          const int hc = side ? kHX : kHX - 1;          // its place in the halo row
          const int j = y0 - kH + r;
          const int x = side ? x0 + kTX : x0 - 1;
          if ((G.per_y || (j >= 0 && j < G.ny)) && (((x + j + p) & 1) == 0)) {
            const int jw = G.per_y ? 0 : (j == 0) + (j == G.ny - 1);
            float* hr = hA(cA, r);
            // x - 1 and x + 1: the halo group's inner neighbour and the tile's
            // edge column
            const float xm = side ? cA[r * kTX + kTX - 1] : hr[kHX - 2];
            const float xp = side ? hr[kHX + 1] : cA[r * kTX];
            const float s = ((xm + xp) + (hA(cA, r - 1)[hc] + hA(cA, r + 1)[hc])) +
                            (hA(xa1, r)[hc] + hA(xa3, r)[hc]);
            const float bb = beta * hB(cB, r - 1)[hc] + srow(j, p);
            hr[hc] = relax(hr[hc], nb_term(s, bb, h2), rc_of(G, jw + zw), c1);
          }
        }
      }
    };
    // The plain sweep runs the black phase first: it writes only global
    // memory, so the compiler may start the red phase's shared-memory loads
    // early (measured 292.5 -> 282.1 us per finest-level launch).  The
    // zero-input and update variants were slower that way (234.9 -> 243.2
    // and 419.7 -> 446.4 us) and keep the red phase first.  The zero-input
    // variant loads both phases' shared-memory operands ahead of the red
    // phase, whose stores the compiler cannot tell apart from the black
    // phase's loads (234.4 -> 218.2 us); in the plain sweep the same
    // hoisting raises the registers to 128 and costs 5 %.  The black cells
    // go to memory at the end of the step, after the red phase's loads
    // (plain sweep 261.5 -> 256.9 us).
    if constexpr (!ZERO_IN && !UPD) {
      black_load();
      black_phase();
      red_load();
      red_phase();
      black_store();
    } else if constexpr (ZERO_IN) {
      black_load();
      red_load();
      red_phase();
      black_phase();
      black_store();
    } else {
      red_load();
      red_phase();
      black_load();
      black_phase();
      black_store();
    }
    {
      const int t = oa0;
      oa0 = oa1; oa1 = oa2; oa2 = oa3; oa3 = oa4; oa4 = oa5; oa5 = t;
      const int u = ob0;
      ob0 = ob1; ob1 = ob2; ob2 = ob3; ob3 = ob4; ob4 = u;
    }
  }
  cp_async_wait0();
}

// Can the fused sweep handle this level?  Tile-aligned levels always; other
// levels with ragged edge tiles when at least a quarter of the tiles' cells
// exist (below that the idle lanes cost more than the second per-colour
// launch saves) and the level has at least 2^17 cells (on smaller levels
// the few CTAs' z-march takes longer than two per-colour launches: measured
// 16.8 us against 2 x 5.9 us at 64 x 32 x 32; with four-plane chunks 11.0 us,
// yet the graph-replayed step was slower with it, 1,795 against 1,801
// Mcell-steps/s).
bool fused_sweep_ok(const Level& L, bool ragged) {
  if (level_ok(L)) return true;
  return ragged && ragged_ok(L) && tile_fill(L) >= 0.25 && L.cells() >= (1 << 17);
}

// the two rings, two mbarriers and the slack that aligns the rings to 128 bytes
size_t fused_sweep_smem() {
  return (size_t)(kNA * kSlotA + kNB * kSlotB) * sizeof(float) + 2 * sizeof(unsigned long long) +
         128;
}

namespace {

static_assert(sizeof(CUtensorMap) == sizeof(TensorMapEntry::map), "opaque tensor map size");

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null if unavailable
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of the FP32 field `ptr` of level L (x fastest, then y, then z)
// with boxes of kTX x rows x 1, zero fill outside; encoded once per context
// (the grid's fields never move).  False if it cannot be encoded.
bool field_map(Ctx& cx, const float* ptr, const Level& L, int rows, CUtensorMap* out) {
  for (const TensorMapEntry& e : cx.tmaps)
    if (e.ptr == ptr && e.rows == rows && e.n[0] == L.n[0] && e.n[1] == L.n[1] && e.n[2] == L.n[2]) {
      std::memcpy(out, e.map, sizeof(CUtensorMap));
      return true;
    }
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || !ptr || (reinterpret_cast<uintptr_t>(ptr) & 15)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)L.n[0], (cuuint64_t)L.n[1], (cuuint64_t)L.n[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)L.n[0] * 4, (cuuint64_t)L.n[0] * L.n[1] * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kTX, (cuuint32_t)rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  TensorMapEntry e{};
  e.ptr = ptr;
  e.n[0] = L.n[0]; e.n[1] = L.n[1]; e.n[2] = L.n[2];
  e.rows = rows;
  CUtensorMap m;
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(ptr), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  std::memcpy(e.map, &m, sizeof(CUtensorMap));
  if (cx.tmaps.size() >= 512) cx.tmaps.clear();   // bounded (a handful of fields per level)
  cx.tmaps.push_back(e);
  *out = m;
  return true;
}

// tensor maps for a launch of the TMA variant (x unless zero_in, rhs)
bool fused_maps(Ctx& cx, const Level& L, Comp3<float> A, Rhs3<float> R, int ncomp, bool zero_in,
                FusedMaps* M) {
  for (int c = 0; c < ncomp; ++c) {
    if (!zero_in && !field_map(cx, A.at(c), L, kRA, &M->a[c])) return false;
    if (!field_map(cx, R.b_at(c), L, kRB, &M->b[c])) return false;
  }
  return true;
}

template <bool Z, bool HS, bool U, bool RG>
void launch_variant(dim3 grid, size_t smem, const Ctx& cx, const FusedGeom& G, Comp3<float> A,
                    Comp3<float> B, Rhs3<float> R, Comp3<float> XH, Comp3<float> XL,
                    const FusedMaps& M) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_rbgs_fused<Z, HS, U, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_rbgs_fused<Z, HS, U, RG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         100);
    attr_set = true;
  }
  launch_k(cx, k_rbgs_fused<Z, HS, U, RG>, grid, kThreads, smem, G, A, B, R, XH, XL, M);
}

template <bool RG>
void launch_pick(dim3 grid, size_t smem, const Ctx& cx, const FusedGeom& G, Comp3<float> A,
                 Comp3<float> B, Rhs3<float> R, Comp3<float> XH, Comp3<float> XL,
                 const FusedMaps& M, bool upd, bool zero_in, bool hs) {
  if (upd) {
    if (hs) launch_variant<false, true, true, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
    else launch_variant<false, false, true, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
  } else if (zero_in) {
    if (hs) launch_variant<true, true, false, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
    else launch_variant<true, false, false, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
  } else {
    if (hs) launch_variant<false, true, false, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
    else launch_variant<false, false, false, RG>(grid, smem, cx, G, A, B, R, XH, XL, M);
  }
}

FusedGeom fused_geom(Ctx& cx, const Level& L, Rhs3<float> R, int ncomp, int zchunk, float omega) {
  FusedGeom G;
  G.nx = L.n[0]; G.ny = L.n[1]; G.nz = L.n[2];
  G.per_y = L.per[1]; G.per_z = L.per[2];
  G.ntx = (L.n[0] + kTX - 1) / kTX; G.nty = (L.n[1] + kTY - 1) / kTY;
  // a step costs about three planes of pipeline fill; chunks down to four
  // planes let the small levels spread over more SMs
  if (zchunk <= 0) zchunk = pick_zchunk(L, std::max(ncomp, cx.chunk_comps), 2 * cx.sms, 3, 4);
  G.zchunk = std::min(zchunk, L.n[2]);
  // omega rc and 1 - omega rounded in FP32 as relax() and wscale() form them
  G.rc0 = omega * L.rcf[0];
  G.rc1 = omega * L.rcf[1];
  G.rc2 = omega * L.rcf[2];
  G.c1 = 1.f - omega;
  G.h2 = (float)(1.0 / L.inv_h2);
  G.beta = R.beta;
  G.status = cx.status;
  G.limit_ns = kCopyLimitNs;
  G.probe_tx = 0u;
  return G;
}

}  // namespace

// One fused full sweep A -> B on `ncomp` components (zero_in: A taken as 0;
// zchunk <= 0: chosen for whole waves of two CTAs per SM).  With upd_hi /
// upd_lo given (and zero_in false) the result is added to that double-word
// iterate instead of being stored to B.  Tile-aligned levels without
// periodic y stage by TMA boxes, the others by cp.async.
void launch_rbgs_fused(Ctx& cx, const Level& L, Comp3<float> A, Comp3<float> B, Rhs3<float> R,
                       int ncomp, int zchunk, int kclass, bool zero_in, const Comp3<float>* upd_hi,
                       const Comp3<float>* upd_lo, float omega) {
  const size_t smem = fused_sweep_smem();
  const FusedGeom G = fused_geom(cx, L, R, ncomp, zchunk, omega);
  const int nzc = (L.n[2] + G.zchunk - 1) / G.zchunk;
  dim3 grid(G.ntx * G.nty, nzc, ncomp);
  const bool hs = R.S[0] != nullptr;
  const bool upd = upd_hi && upd_lo && !zero_in;
  const Comp3<float> XH = upd ? *upd_hi : Comp3<float>{{nullptr, nullptr, nullptr}};
  const Comp3<float> XL = upd ? *upd_lo : Comp3<float>{{nullptr, nullptr, nullptr}};
  FusedMaps M;
  std::memset(&M, 0, sizeof M);
  const bool tma = level_ok(L) && !L.per[1] && fused_maps(cx, L, A, R, ncomp, zero_in, &M);
  // algorithmic bytes per cell: rhs and result (+ x unless zero_in, + the
  // iterate's two words read and written when updating)
  const double bpc = zero_in ? 8.0 : (upd ? 24.0 : 12.0);
  cx.before(kclass);
  if (tma) launch_pick<false>(grid, smem, cx, G, A, B, R, XH, XL, M, upd, zero_in, hs);
  else launch_pick<true>(grid, smem, cx, G, A, B, R, XH, XL, M, upd, zero_in, hs);
  cx.after(kclass, bpc * (double)L.cells() * ncomp);
}

// The bound of the fused sweep's waits for its staged planes: one sweep from
// zero of component 0 of R into B on the tile-aligned level L (without
// periodic y), every copy group armed with probe_tx bytes (> 0) and no box
// loaded, so that every wait gives up after limit_ns and sets kCopyTimeout
// in the flag word.  Returns false (nothing launched) unless L is such a
// level.
bool launch_copy_wait_probe(Ctx& cx, const Level& L, Comp3<float> B, Rhs3<float> R,
                            unsigned probe_tx, unsigned long long limit_ns) {
  if (!level_ok(L) || L.per[1] || probe_tx == 0u) return false;
  FusedGeom G = fused_geom(cx, L, R, 1, 0, 1.f);
  G.limit_ns = limit_ns;
  G.probe_tx = probe_tx;
  const int nzc = (L.n[2] + G.zchunk - 1) / G.zchunk;
  dim3 grid(G.ntx * G.nty, nzc, 1);
  const Comp3<float> none{{nullptr, nullptr, nullptr}};
  FusedMaps M;
  std::memset(&M, 0, sizeof M);
  launch_pick<false>(grid, fused_sweep_smem(), cx, G, none, B, R, none, none, M, false, true,
                     R.S[0] != nullptr);
  return cudaPeekAtLastError() == cudaSuccess;
}

}  // namespace vsv
