// Tiled grid transfers of the multigrid V-cycle (FP32 storage) for
// tile-aligned levels coarsened by two on every axis: the residual
// restriction r_c = R (b - L e) and the prolongation e += P e_c.  Both march
// along z over a 128 x 16 fine tile (64 x 8 coarse), so every fine value is
// read from memory once; they do the same arithmetic, in the same order, as
// k_restrict_block / k_prolong_block (mg.cu), hence the same bits.
#include "tile.cuh"

namespace vsv {

using namespace tile;

namespace {

// ---------------------------------------------------------------- restriction
constexpr int kRR = kTY + 2;   // staged fine rows (one halo row each side)
constexpr int kRS = 5;         // ring slots
constexpr int kRStage = (kRR * kNV + kThreads - 1) / kThreads;

struct RGeom : Geom {
  float ih2, alpha, beta, sh2;
  int cnx, cny;   // coarse extents (x, y)
};

__device__ __forceinline__ float c4(const float4& v, int o) {
  return o == 0 ? v.x : (o == 1 ? v.y : (o == 2 ? v.z : v.w));
}

}  // namespace

// Thread (gx, ty) owns fine columns x0 + 4 gx .. + 3 of rows 2 ty, 2 ty + 1,
// i.e. coarse cells (I0 + 2 gx, I0 + 2 gx + 1) of coarse row J0 + ty, and
// accumulates their children plane by plane (planes 2K then 2K + 1, rows
// 2J then 2J + 1, x 2I then 2I + 1: the order of k_restrict_block).  Fine
// neighbours in x / y come from the staged plane, z neighbours from the
// thread's registers.  Copies run two steps ahead; five ring slots make one
// barrier per step enough (as in the tiled defect kernel).
// RAGGED: partial edge tiles; threads whose fine cells lie past the extent
// read no rhs and store nothing (their staged neighbours are wrapped copies
// or zero ghosts, never used for an owned cell's result).
template <bool HAS_S, bool RAGGED>
__global__ void __launch_bounds__(kThreads, 3)
k_restrict_tiled(RGeom G, Comp3<float> X, Rhs3<float> R, Comp3<float> RC) {
  pdl_begin();
  extern __shared__ float4 smem_r4[];
  float* sX = reinterpret_cast<float*>(smem_r4);
  const int comp = blockIdx.z;
  const float* __restrict__ x = X.at(comp);
  const float* __restrict__ bsrc = R.b_at(comp);
  const float* __restrict__ S = R.s_at(comp);
  float* __restrict__ rc = RC.at(comp);
  const int tx = blockIdx.x % G.ntx, tyb = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = tyb * kTY;
  const int zb = blockIdx.y * G.zchunk;            // zchunk is even
  const int ze = min(zb + G.zchunk, G.nz);
  const int tid = threadIdx.x, gx = tid & 31, ty = tid >> 5;
  const int q = gx + 1;
  auto slot = [&](int plane) {
    return sX + ((unsigned)(plane + kRS) % (unsigned)kRS) * (kRR * kW);   // plane >= -1
  };
  StageDesc<kRStage> ds;
  ds.init(G, x0, y0, 1, kRR);
  int rown[2], jown[2], yw[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    jown[h] = y0 + 2 * ty + h;
    rown[h] = 2 * ty + h + 1;
    yw[h] = G.per_y ? 0 : (jown[h] == 0) + (jown[h] == G.ny - 1);
  }
  // both fine rows of a thread lie inside or outside together (ny is even)
  const bool act = !RAGGED || (jown[0] < G.ny && x0 + 4 * gx < G.nx);
  for (int pl = zb - 1; pl <= zb + 1; ++pl) ds.stage(slot(pl), x, G, pl, false);
  cp_async_commit();
  if (zb + 2 <= ze) ds.stage(slot(zb + 2), x, G, zb + 2, false);
  cp_async_commit();
  // rhs of plane zb
  float4 Bn[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
  if (act) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      Bn[h] = *reinterpret_cast<const float4*>(bsrc + ((long long)zb * G.ny + jown[h]) * G.nx + x0 +
                                               4 * gx);
  }
  cp_async_wait1();
  __syncthreads();
  float4 Mz[2], Vz[2], Pz[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    Vz[h] = lds4(slot(zb - 1) + rown[h] * kW + 4 * q);
    Pz[h] = lds4(slot(zb) + rown[h] * kW + 4 * q);
  }
  float acc0 = 0.f, acc1 = 0.f;
  for (int p = zb; p < ze; ++p) {
    if (p + 3 <= ze) ds.stage(slot(p + 3), x, G, p + 3, false);
    cp_async_commit();
    float4 Bc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Bc[h] = Bn[h];
      if (p + 1 < ze && act)
        Bn[h] = *reinterpret_cast<const float4*>(bsrc + ((long long)(p + 1) * G.ny + jown[h]) * G.nx +
                                                 x0 + 4 * gx);
    }
    cp_async_wait2();
    __syncthreads();
    const float* cX = slot(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Mz[h] = Vz[h];
      Vz[h] = Pz[h];
      Pz[h] = lds4(slot(p + 1) + rown[h] * kW + 4 * q);
    }
    const int zw = G.per_z ? 0 : (p == 0) + (p == G.nz - 1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float* row = cX + rown[h] * kW;
      const float4 U = lds4(row - kW + 4 * q), D = lds4(row + kW + 4 * q);
      const float Lx = row[4 * q - 1], Rx = row[4 * q + 4];
      const float s_ = (HAS_S && act) ? S[jown[h] + (long long)p * G.ny] : 0.f;
      const int nwall = yw[h] + zw;
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float xm = o == 0 ? Lx : c4(Vz[h], o - 1);
        const float xp = o == 3 ? Rx : c4(Vz[h], o + 1);
        const float s = ((xm + xp) + (c4(U, o) + c4(D, o))) + (c4(Mz[h], o) + c4(Pz[h], o));
        const float b = G.beta * c4(Bc[h], o) + s_;
        const float r = b - (s - (6.f + G.alpha * (float)nwall + G.sh2) * c4(Vz[h], o)) * G.ih2;
        if (o < 2) acc0 += r; else acc1 += r;
      }
    }
    if ((p & 1) && act) {   // plane pair complete: store the two coarse cells
      const int K = p >> 1, J = (y0 >> 1) + ty, I = (x0 >> 1) + 2 * gx;
      *reinterpret_cast<float2*>(rc + ((long long)K * G.cny + J) * G.cnx + I) =
          make_float2(acc0 * 0.125f, acc1 * 0.125f);
      acc0 = 0.f;
      acc1 = 0.f;
    }
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------- prolongation
namespace {
constexpr int kPRows = kTY / 2 + 2;      // staged coarse rows (J0 - 1 .. J0 + 8)
constexpr int kPW = kTX / 2 + 2 * kHX;   // staged coarse row length (I0 - 4 .. I0 + 67)
constexpr int kPNV = kPW / 4;            // 16-byte vectors per staged coarse row
constexpr int kPS = 6;                   // coarse-plane ring slots
static_assert(kPRows * kPNV <= kThreads, "one staging vector per thread");

struct PGeom {
  int nx, ny, nz;                  // fine extents
  int cnx, cny, cnz;               // coarse extents
  int per_y, per_z;                // coarse (= fine) periodicity of y, z
  int ntx, nty, zchunk;            // fine tiles and z chunk (even)
  float malpha;                    // -alpha of the coarse level
};
}  // namespace

// Thread (gx, ty) owns fine columns x0 + 4 gx .. + 3 of rows 2 ty, 2 ty + 1:
// coarse cells I0 + 2 gx, I0 + 2 gx + 1 of coarse row J = J0 + ty, whose x
// neighbours are I0 + 2 gx - 1 and I0 + 2 gx + 2 (x is periodic).  Coarse
// planes are staged (rows J0 - 1 .. J0 + 8) two steps ahead into a six-slot
// ring; a step handles the fine planes 2K and 2K + 1 of coarse plane K, whose
// fine values are read and written straight from registers.
// RAGGED: partial edge tiles (coarse x extent a multiple of 4); threads whose
// fine cells lie past the extent read and write nothing.
template <bool RAGGED>
__global__ void __launch_bounds__(kThreads, 3)
k_prolong_tiled(PGeom G, Comp3<float> X, Comp3<float> E) {
  pdl_begin();
  __shared__ __align__(16) float sE[kPS * kPRows * kPW];
  const int comp = blockIdx.z;
  float* __restrict__ x = X.at(comp);
  const float* __restrict__ e = E.at(comp);
  const int tx = blockIdx.x % G.ntx, tyb = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = tyb * kTY;
  const int I0 = x0 >> 1, J0 = y0 >> 1;
  const int Kb = (blockIdx.y * G.zchunk) >> 1;
  const int Ke = min(blockIdx.y * G.zchunk + G.zchunk, G.nz) >> 1;
  const int tid = threadIdx.x, gx = tid & 31, ty = tid >> 5;
  auto slot = [&](int K) { return sE + ((unsigned)(K + kPS) % (unsigned)kPS) * (kPRows * kPW); };
  // staging descriptor: one 16-byte vector per thread (tid < kPRows * kPNV)
  const bool st_used = tid < kPRows * kPNV;
  const int st_r = tid / kPNV, st_v = tid - st_r * kPNV;
  int st_j = J0 - 1 + st_r;
  bool st_ok = st_used;
  if (G.per_y) st_j = RAGGED ? modi(st_j, G.cny) : wrapi(st_j, G.cny);
  else if (st_j < 0 || st_j >= G.cny) st_ok = false;
  const int st_i = RAGGED ? modi(I0 - kHX + 4 * st_v, G.cnx) : wrapi(I0 - kHX + 4 * st_v, G.cnx);
  const bool act = !RAGGED || (y0 + 2 * ty < G.ny && x0 + 4 * gx < G.nx);
  const int st_goff = st_ok ? st_j * G.cnx + st_i : 0;
  const int st_soff = st_r * kPW + 4 * st_v;
  auto stage = [&](int K) {
    if (!st_used) return;
    bool ok = st_ok;
    int k = K;
    if (G.per_z) k = wrapi(k, G.cnz);
    else if (k < 0 || k >= G.cnz) ok = false;
    const float* src = e + (ok ? (long long)k * G.cny * G.cnx + st_goff : 0LL);
    cp_async16(slot(K) + st_soff, src, ok);
  };
  // y neighbours of coarse row J0 + ty: the row above (b = 0) and below (b = 1)
  const int J = J0 + ty;
  int rowN[2];
  float fyN[2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int jn = J + (b ? 1 : -1);
    const bool in = G.per_y || (jn >= 0 && jn < G.cny);
    rowN[b] = in ? ty + 1 + (b ? 1 : -1) : ty + 1;   // staged row index
    fyN[b] = in ? 1.f : G.malpha;
  }
  const int colC0 = kHX + 2 * gx;   // staged column of coarse I0 + 2 gx

  stage(Kb - 1);   // group 0: planes Kb-1 .. Kb+1 (step Kb); group 1: plane Kb+2
  stage(Kb);
  stage(Kb + 1);
  cp_async_commit();
  if (Kb + 2 <= Ke) stage(Kb + 2);
  cp_async_commit();
  for (int K = Kb; K < Ke; ++K) {
    if (K + 3 <= Ke) stage(K + 3);   // plane K + 3 is needed by step K + 2
    cp_async_commit();
    // fine values of planes 2K, 2K+1, rows 2ty, 2ty+1
    float4 F[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        F[c][b] = act ? *reinterpret_cast<const float4*>(
                            x + ((long long)(2 * K + c) * G.ny + y0 + 2 * ty + b) * G.nx + x0 + 4 * gx)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    cp_async_wait2();
    __syncthreads();
    // coarse planes: centre K and the neighbour below (c = 0) / above (c = 1)
    const float* pC = slot(K);
    const float* pN[2];
    float fzN[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int kn = K + (c ? 1 : -1);
      const bool in = G.per_z || (kn >= 0 && kn < G.cnz);
      pN[c] = in ? slot(kn) : pC;
      fzN[c] = in ? 1.f : G.malpha;
    }
    // the four coarse x values (I-1, I, I+1, I+2 with I = I0 + 2 gx) of a staged row
    auto row4 = [&](const float* pl, int r, float v[4]) {
      const float* rp = pl + r * kPW + colC0;
      v[0] = rp[-1];
      const float2 m = *reinterpret_cast<const float2*>(rp);
      v[1] = m.x;
      v[2] = m.y;
      v[3] = rp[2];
    };
    float cc[4];
    row4(pC, ty + 1, cc);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float zc[4];
      row4(pN[c], ty + 1, zc);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float yc[4], zy[4];
        row4(pC, rowN[b], yc);
        row4(pN[c], rowN[b], zy);
        // boundary factors: n = (fz * fy) * e (x is periodic, its factor 1),
        // the same values prolong_children forms
        const float fy = fyN[b], fz = fzN[c], fzy = fz * fy;
        float out[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int ic = 1 + (o >> 1);                // own coarse x in the 4-vector
          const int in = (o & 1) ? ic + 1 : ic - 1;   // its x neighbour on this child's side
          out[o] = prolong_value<float>(cc[ic], cc[in], fy * yc[ic], fy * yc[in], fz * zc[ic],
                                        fz * zc[in], fzy * zy[ic], fzy * zy[in]);
        }
        float4 v = F[c][b];
        v.x += out[0];
        v.y += out[1];
        v.z += out[2];
        v.w += out[3];
        if (act)
          *reinterpret_cast<float4*>(x + ((long long)(2 * K + c) * G.ny + y0 + 2 * ty + b) * G.nx +
                                   x0 + 4 * gx) = v;
      }
    }
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------- launchers
// ragged: also levels with partial edge tiles (fine x extent a multiple of 8,
// so that coarse rows stage as whole 16-byte vectors), under the size and
// fill thresholds of the fused sweep
bool tiled_transfer_ok(const Level& F, const Level& C, bool ragged) {
  for (int a = 0; a < 3; ++a)
    if (F.n[a] != 2 * C.n[a]) return false;
  if (level_ok(F)) return true;
  return ragged && ragged_ok(F) && F.n[0] % 8 == 0 && tile_fill(F) >= 0.25 &&
         F.cells() >= (1 << 17);
}

static int even_chunk(const Level& F, int ncomp, int sms, int halo) {
  int chunk = pick_zchunk(F, ncomp, 3 * sms, halo);
  chunk += chunk & 1;
  return std::min(chunk, F.n[2]);
}

bool launch_restrict_tiled(Ctx& cx, const Level& F, const Level& C, Comp3<float> X,
                           Rhs3<float> R, Comp3<float> RC, int ncomp) {
  if (!tiled_transfer_ok(F, C, cx.ragged)) return false;
  const bool rg = !level_ok(F);
  RGeom G;
  static_cast<Geom&>(G) = geom(F, even_chunk(F, std::max(ncomp, cx.chunk_comps), cx.sms, 2));
  G.ih2 = F.inv_h2f;
  G.alpha = F.alphaf;
  G.sh2 = F.sh2f;
  G.beta = R.beta;
  G.cnx = C.n[0];
  G.cny = C.n[1];
  const size_t smem = (size_t)kRS * kRR * kW * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_restrict_tiled<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_restrict_tiled<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_restrict_tiled<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_restrict_tiled<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  dim3 grid(G.ntx * G.nty, (F.n[2] + G.zchunk - 1) / G.zchunk, ncomp);
  cx.before(VSV_KCLASS_RESTRICT);
  if (R.S[0]) {
    if (rg) launch_k(cx, k_restrict_tiled<true, true>, grid, kThreads, smem, G, X, R, RC);
    else launch_k(cx, k_restrict_tiled<true, false>, grid, kThreads, smem, G, X, R, RC);
  } else {
    if (rg) launch_k(cx, k_restrict_tiled<false, true>, grid, kThreads, smem, G, X, R, RC);
    else launch_k(cx, k_restrict_tiled<false, false>, grid, kThreads, smem, G, X, R, RC);
  }
  cx.after(VSV_KCLASS_RESTRICT, 8.5 * (double)F.cells() * ncomp);   // e, b read; r_c written
  return true;
}

bool launch_prolong_tiled(Ctx& cx, const Level& F, const Level& C, Comp3<float> X, Comp3<float> E,
                          int ncomp) {
  if (!tiled_transfer_ok(F, C, cx.ragged)) return false;
  const bool rg = !level_ok(F);
  PGeom G;
  G.nx = F.n[0]; G.ny = F.n[1]; G.nz = F.n[2];
  G.cnx = C.n[0]; G.cny = C.n[1]; G.cnz = C.n[2];
  G.per_y = C.per[1]; G.per_z = C.per[2];
  G.ntx = (F.n[0] + kTX - 1) / kTX; G.nty = (F.n[1] + kTY - 1) / kTY;
  G.zchunk = even_chunk(F, std::max(ncomp, cx.chunk_comps), cx.sms, 2);
  G.malpha = -C.alphaf;
  dim3 grid(G.ntx * G.nty, (F.n[2] + G.zchunk - 1) / G.zchunk, ncomp);
  cx.before(VSV_KCLASS_PROLONG);
  if (rg) launch_k(cx, k_prolong_tiled<true>, grid, kThreads, 0, G, X, E);
  else launch_k(cx, k_prolong_tiled<false>, grid, kThreads, 0, G, X, E);
  cx.after(VSV_KCLASS_PROLONG, 8.5 * (double)F.cells() * ncomp);   // e read and written, e_c read
  return true;
}

}  // namespace vsv
