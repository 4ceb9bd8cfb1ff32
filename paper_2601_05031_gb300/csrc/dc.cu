// Outer defect correction of the mixed path with a double-word iterate.
//
// The iterate x = x_hi + x_lo (two FP32 words, about 44 significant bits) is
// refined by   r = b - L_h x  (the hi words of the stencil by error-free
// cascaded summation, the cancelling rhs and stencil terms by error-free
// sums, only O(u)-small terms added in FP32: the error is a rounding of r
// plus O(u^2) of the terms),   L_h e = r  (one FP32 multigrid V-cycle from
// e = 0),   x <- x + e (double-word addition).  The defect sees x to
// FP64-class accuracy, so the refinement converges to the discrete solution
// below FP32 rounding and the relative residual is a meaningful stopping test.
#include <algorithm>

#include "tile.cuh"

namespace vsv {

namespace {

__device__ __forceinline__ int wrapd(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Neighbour fetch on the fine level with zero data on Dirichlet ghosts.
struct NbFetch {
  const float* __restrict__ a;
  int nx, ny, nz, per[3], act[3];
  __device__ __forceinline__ float get(int i, int j, int k) const {
    if (i < 0 || i >= nx) { if (!per[0]) return 0.f; i = wrapd(i, nx); }
    if (j < 0 || j >= ny) { if (!per[1]) return 0.f; j = wrapd(j, ny); }
    if (k < 0 || k >= nz) { if (!per[2]) return 0.f; k = wrapd(k, nz); }
    return a[lin(i, j, k, nx, ny)];
  }
};

// r = (b1 + b2 + s) - (p + rest) where b1 + b2 is the rhs pair, s the row
// source, p the leading word of L x and rest its O(u) remainder.  b1 (+ s)
// and p cancel almost completely near convergence, so they go through
// error-free TwoSums; b2, rest and the TwoSum errors are O(u) of the terms
// and are added in FP32 (their rounding is O(u^2) of the terms).
__device__ __forceinline__ float defect_combine(float b1, float b2, bool has_b2, float s,
                                                bool has_s, float p, float rest) {
  float h = b1, lo = 0.f;
  if (has_s) two_sum(b1, s, h, lo);
  float d, e;
  two_sum(h, -p, d, e);
  lo = has_s ? __fadd_rn(lo, e) : e;
  if (has_b2) lo = __fadd_rn(lo, b2);
  lo = __fsub_rn(lo, rest);
  return __fadd_rn(d, lo);
}

}  // namespace

// r = beta (B_hi + B_lo) + S(y, z) - L_h (x_hi + x_lo) to a rounding of r plus
// O(u^2) of the terms; optional FP64 partial sums of ||r||^2 and ||b||^2 per
// block.
__global__ void k_defect_dw(Level L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                            Comp3<float> BL, Comp3<float> OUT, double* partials, float ih_hi,
                            float ih_lo) {
  pdl_begin();
  const int comp = blockIdx.y;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  NbFetch H{XH.at(comp), nx, ny, nz, {L.per[0], L.per[1], L.per[2]}, {L.act[0], L.act[1], L.act[2]}};
  NbFetch Lo{XL.at(comp), nx, ny, nz, {L.per[0], L.per[1], L.per[2]}, {L.act[0], L.act[1], L.act[2]}};
  const float* __restrict__ bh = R.b_at(comp);
  const float* __restrict__ bl = BL.at(comp);
  const float* __restrict__ S = R.s_at(comp);
  float* __restrict__ out = OUT.at(comp);
  const float beta = R.beta;
  // diagonal 2 d + s h^2 as a pair (alpha = 0 on the finest level)
  const float dch = L.cdh[0], dcl = L.cdl[0];
  double rr = 0.0, bb = 0.0;
  for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    const float s = S ? S[j + (long long)k * ny] : 0.f;
    float r2 = 0.f, b2 = 0.f;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long t = lin(i, j, k, nx, ny);
      // hi words: cascade from the first active direction's x- neighbour
      // on, in the order x-, x+, y-, y+, z-, z+; lo words: the per-axis
      // pair sums added in axis order
      CascadeSum lh(0.f);
      float llo = 0.f;
      bool first = true;
      for (int a = 0; a < 3; ++a) {
        if (!L.act[a]) continue;
        const int di = a == 0, dj = a == 1, dk = a == 2;
        const float hm = H.get(i - di, j - dj, k - dk), hp = H.get(i + di, j + dj, k + dk);
        const float pl = __fadd_rn(Lo.get(i - di, j - dj, k - dk), Lo.get(i + di, j + dj, k + dk));
        if (first) { lh = CascadeSum(hm); llo = pl; first = false; }
        else { lh.add(hm); llo = __fadd_rn(llo, pl); }
        lh.add(hp);
      }
      lh.add_scaled(-dch, H.a[t]);
      if (dcl != 0.f) lh.add(-dcl * H.a[t]);   // adding -0 would change nothing
      llo = __fmaf_rn(-dch, Lo.a[t], llo);
      // L x = (lh.hi + lh.lo + llo) * inv_h2, leading product split exactly
      const float p = __fmul_rn(ih_hi, lh.hi);
      const float pe = __fmaf_rn(ih_hi, lh.hi, -p);
      const float rest = __fmaf_rn(ih_hi, __fadd_rn(lh.lo, llo), __fmaf_rn(ih_lo, lh.hi, pe));
      const float b1 = beta * bh[t];
      const float rv = defect_combine(b1, bl ? beta * bl[t] : 0.f, bl != nullptr, s, S != nullptr,
                                      p, rest);
      out[t] = rv;
      if (partials) {
        const float bv = b1 + (bl ? beta * bl[t] : 0.f) + s;
        r2 = __fmaf_rn(rv, rv, r2);
        b2 = __fmaf_rn(bv, bv, b2);
      }
    }
    rr += (double)r2;
    bb += (double)b2;
  }
  if (partials) {
    rr = block_sum(rr);
    bb = block_sum(bb);
    if (threadIdx.x == 0) {
      double* o = partials + ((long long)comp * gridDim.x + blockIdx.x) * 2;
      o[0] = rr;
      o[1] = bb;
    }
  }
}

// (x_hi, x_lo) <- (x_hi, x_lo) + e
__global__ void k_update_dw(Comp3<float> XH, Comp3<float> XL, Comp3<float> E, long long n) {
  pdl_begin();
  const int comp = blockIdx.y;
  float* __restrict__ xh = XH.at(comp);
  float* __restrict__ xl = XL.at(comp);
  const float* __restrict__ e = E.at(comp);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const FF v = ff_add_f(FF{xh[t], xl[t]}, e[t]);
    xh[t] = v.hi;
    xl[t] = v.lo;
  }
}

// First guess from the history, written into the oldest buffer C (A = x^n,
// B = x^{n-1}, C = x^{n-2}): A plus the extrapolation increment
// d = 0 (order 0), A - B (order 1: 2A - B) or 2A - 3B + C (order 2:
// 3A - 3B + C).  Only A must be exact (its two words); d is formed in FP32
// from the high words, so its rounding, of order u |x|, is an error of the
// first guess, which the cycles of the solve contract like any other.  The
// low words of B and C are not read.
__global__ void k_extrapolate_rot_dw(Comp3<float> AH, Comp3<float> AL, Comp3<float> BH,
                                     Comp3<float> CH, Comp3<float> CL, long long n, int order) {
  pdl_begin();
  const int comp = blockIdx.y;
  const float* __restrict__ ah = AH.at(comp);
  const float* __restrict__ al = AL.at(comp);
  const float* __restrict__ bh = BH.at(comp);
  float* __restrict__ ch = CH.at(comp);
  float* __restrict__ cl = CL.at(comp);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const FF a{ah[t], al[t]};
    FF v = a;
    if (order == 1) {
      v = ff_add_f(a, a.hi - bh[t]);
    } else if (order == 2) {
      v = ff_add_f(a, __fmaf_rn(2.f, a.hi, __fmaf_rn(-3.f, bh[t], ch[t])));
    }
    ch[t] = v.hi;
    cl[t] = v.lo;
  }
}

// (YH, YL) += a (XH, XL) in double-word arithmetic, a given in FP64 and
// split into an FP32 pair (the inertial right-hand side f - s omega'^n).
__global__ void k_axpy_dw(Comp3<float> YH, Comp3<float> YL, Comp3<float> XH, Comp3<float> XL,
                          float a_hi, float a_lo, long long n) {
  pdl_begin();
  const int comp = blockIdx.y;
  float* __restrict__ yh = YH.at(comp);
  float* __restrict__ yl = YL.at(comp);
  const float* __restrict__ xh = XH.at(comp);
  const float* __restrict__ xl = XL.at(comp);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const FF v = ff_add(FF{yh[t], yl[t]}, ff_mul(FF{xh[t], xl[t]}, FF{a_hi, a_lo}));
    yh[t] = v.hi;
    yl[t] = v.lo;
  }
}

void launch_defect_dw(Ctx& cx, const Level& L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                      Comp3<float> BL, Comp3<float> OUT, int ncomp, double* partials, int nblocks) {
  const float ih_hi = (float)L.inv_h2, ih_lo = (float)(L.inv_h2 - (double)ih_hi);
  dim3 grid(nblocks, ncomp);
  cx.before(VSV_KCLASS_RESTRICT);
  launch_k(cx, k_defect_dw, grid, kBlock, 0, L, XH, XL, R, BL, OUT, partials, ih_hi, ih_lo);
  cx.after(VSV_KCLASS_RESTRICT, (BL.p[0] ? 20.0 : 16.0) * (double)L.cells() * ncomp);
}

// ---------------------------------------------------------------- tiled defect
// The same defect as k_defect_dw (same summation order, hence the same
// bits) on a 128 x 16 tile marching along z: x_hi and x_lo planes staged in
// shared memory (one-cell halo), each thread's own float4 groups of the
// planes below and above held in registers, rhs read straight from memory.
// At step p the CTA issues the copies of plane p + 3 and waits for those of
// plane p + 1 (two steps of copies in flight); five ring slots keep the copies
// clear of the planes p - 1 and p that a warp still in step p - 1 may read,
// so one barrier per step suffices.
namespace {
constexpr int kDS = 5;   // ring slots
// ROWS rows per thread: a tile of 8 ROWS rows, 8 ROWS + 2 staged with the halo
template <int ROWS>
struct DefShape {
  static constexpr int kRows = 8 * ROWS;
  static constexpr int kDR = kRows + 2;
  static constexpr int kStage = (kDR * tile::kNV + tile::kThreads - 1) / tile::kThreads;
  static constexpr size_t kSmem = (size_t)2 * kDS * kDR * tile::kW * sizeof(float);
};

struct DefGeom : tile::Geom {
  float ih_hi, ih_lo, beta;
  float dch, dcl;   // diagonal 6 + s h^2 as a pair (alpha = 0 on the finest level)
};

__device__ __forceinline__ float comp4(const float4& v, int o) {
  return o == 0 ? v.x : (o == 1 ? v.y : (o == 2 ? v.z : v.w));
}

// b - L x at one cell, the same arithmetic as k_defect_dw with every axis
// active: hi neighbours by cascaded summation in the order x-, x+, y-, y+,
// z-, z+, then -6 x_c; lo parts as per-axis pair sums in FP32.
__device__ __forceinline__ float defect_cell(float xmh, float xph, float ymh, float yph, float zmh,
                                             float zph, float ch, float xml, float xpl, float yml,
                                             float ypl, float zml, float zpl, float cl, float b1,
                                             float b2, bool has_b2, float s, bool has_s,
                                             float ih_hi, float ih_lo, float dch, float dcl) {
  CascadeSum lh(xmh);
  lh.add(xph);
  lh.add(ymh); lh.add(yph);
  lh.add(zmh); lh.add(zph);
  float llo = __fadd_rn(__fadd_rn(__fadd_rn(xml, xpl), __fadd_rn(yml, ypl)), __fadd_rn(zml, zpl));
  lh.add_scaled(-dch, ch);
  if (dcl != 0.f) lh.add(-dcl * ch);   // adding -0 would change nothing
  llo = __fmaf_rn(-dch, cl, llo);
  const float p = __fmul_rn(ih_hi, lh.hi);
  const float pe = __fmaf_rn(ih_hi, lh.hi, -p);
  const float rest = __fmaf_rn(ih_hi, __fadd_rn(lh.lo, llo), __fmaf_rn(ih_lo, lh.hi, pe));
  return defect_combine(b1, b2, has_b2, s, has_s, p, rest);
}
}  // namespace

// RAGGED: partial edge tiles; cells past the extent (wrapped copies or zero
// ghost rows in the staged planes) are skipped.  NORMS: FP64 partial sums of
// ||r||^2 and ||b||^2 per block (the fixed-cycle solves go without).
template <int ROWS, bool RAGGED, bool NORMS>
__global__ void __launch_bounds__(tile::kThreads, ROWS == 1 ? 3 : 2)
k_defect_tiled(DefGeom G, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R, Comp3<float> BL,
               Comp3<float> OUT, double* partials) {
  pdl_begin();
  using namespace tile;
  constexpr int kDR = DefShape<ROWS>::kDR, kRows = DefShape<ROWS>::kRows;
  constexpr int kDStage = DefShape<ROWS>::kStage;
  extern __shared__ float4 smem_d4[];
  float* sH = reinterpret_cast<float*>(smem_d4);
  float* sL = sH + kDS * kDR * kW;
  const int comp = blockIdx.z;
  const float* __restrict__ xh = XH.at(comp);
  const float* __restrict__ xl = XL.at(comp);
  const float* __restrict__ bh = R.b_at(comp);
  const float* __restrict__ bl = BL.at(comp);
  const float* __restrict__ S = R.s_at(comp);
  float* __restrict__ out = OUT.at(comp);
  const int tx = blockIdx.x % G.ntx, tyb = blockIdx.x / G.ntx;
  const int x0 = tx * kTX, y0 = tyb * kRows;
  const int zb = blockIdx.y * G.zchunk;
  const int ze = min(zb + G.zchunk, G.nz);
  const int tid = threadIdx.x, gx = tid & 31, ty = tid >> 5;
  const int q = gx + 1;
  const float beta = G.beta;
  auto slot = [&](float* base, int plane) {
    return base + ((unsigned)(plane + kDS) % (unsigned)kDS) * (kDR * kW);   // plane >= -1
  };
  StageDesc<kDStage> ds;
  ds.init(G, x0, y0, 1, kDR);
  int rown[ROWS], jown[ROWS];
#pragma unroll
  for (int h = 0; h < ROWS; ++h) {
    rown[h] = ty + 8 * h + 1;
    jown[h] = y0 + ty + 8 * h;
  }
  // group 0: planes zb-1 .. zb+1 (step zb); group 1: plane zb+2 (step zb+1)
  for (int pl = zb - 1; pl <= zb + 1; ++pl) {
    ds.stage(slot(sH, pl), xh, G, pl, false);
    ds.stage(slot(sL, pl), xl, G, pl, false);
  }
  cp_async_commit();
  if (zb + 2 <= ze) {
    ds.stage(slot(sH, zb + 2), xh, G, zb + 2, false);
    ds.stage(slot(sL, zb + 2), xl, G, zb + 2, false);
  }
  cp_async_commit();
  cp_async_wait1();
  __syncthreads();
  float4 Mh[ROWS], Ml[ROWS], Vh[ROWS], Vl[ROWS], Ph[ROWS], Pl[ROWS];
#pragma unroll
  for (int h = 0; h < ROWS; ++h) {
    Vh[h] = lds4(slot(sH, zb - 1) + rown[h] * kW + 4 * q);
    Vl[h] = lds4(slot(sL, zb - 1) + rown[h] * kW + 4 * q);
    Ph[h] = lds4(slot(sH, zb) + rown[h] * kW + 4 * q);
    Pl[h] = lds4(slot(sL, zb) + rown[h] * kW + 4 * q);
  }
  double rr = 0.0, bb = 0.0;
  // global offsets of the thread's groups in plane zb, advanced by a plane
  // per step, and the ring slot of plane p, advanced with p
  const long long plane_n = (long long)G.ny * G.nx;
  long long gown[ROWS];
#pragma unroll
  for (int h = 0; h < ROWS; ++h) gown[h] = ((long long)zb * G.ny + jown[h]) * G.nx + x0 + 4 * gx;
  for (int p = zb, is = zb % kDS; p < ze;
       ++p, is = (is == kDS - 1) ? 0 : is + 1) {
    auto sl = [&](float* base, int k) {   // slot of plane p + k, 0 <= k < kDS
      const int t = is + k;
      return base + (t >= kDS ? t - kDS : t) * (kDR * kW);
    };
    // the step's rhs words and row source, loaded ahead of the barrier so
    // that their latency overlaps the wait for the staged planes
    float4 B1s[ROWS], B2s[ROWS];
    float Ss[ROWS];
#pragma unroll
    for (int h = 0; h < ROWS; ++h) {
      const int j = jown[h];
      const bool ok = !RAGGED || (j < G.ny && x0 + 4 * gx < G.nx);
      const long long gi = gown[h] + (long long)(p - zb) * plane_n;
      B1s[h] = ok ? *reinterpret_cast<const float4*>(bh + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
      B2s[h] = ok && bl ? *reinterpret_cast<const float4*>(bl + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
      Ss[h] = ok && S ? S[j + (long long)p * G.ny] : 0.f;
    }
    if (p + 3 <= ze) {   // plane p+3 is needed by step p+2
      ds.stage(sl(sH, 3), xh, G, p + 3, false);
      ds.stage(sl(sL, 3), xl, G, p + 3, false);
    }
    cp_async_commit();
    cp_async_wait2();
    __syncthreads();
    const float* cH = sl(sH, 0);
    const float* cL = sl(sL, 0);
#pragma unroll
    for (int h = 0; h < ROWS; ++h) {
      Mh[h] = Vh[h]; Ml[h] = Vl[h];
      Vh[h] = Ph[h]; Vl[h] = Pl[h];
      Ph[h] = lds4(sl(sH, 1) + rown[h] * kW + 4 * q);
      Pl[h] = lds4(sl(sL, 1) + rown[h] * kW + 4 * q);
    }
    float r2 = 0.f, b2 = 0.f;
#pragma unroll
    for (int h = 0; h < ROWS; ++h) {
      const int r = rown[h], j = jown[h];
      if (RAGGED && (j >= G.ny || x0 + 4 * gx >= G.nx)) continue;
      const float* rowH = cH + r * kW;
      const float* rowL = cL + r * kW;
      const float4 Uh = lds4(rowH - kW + 4 * q), Dh = lds4(rowH + kW + 4 * q);
      const float4 Ul = lds4(rowL - kW + 4 * q), Dl = lds4(rowL + kW + 4 * q);
      const float Lh = rowH[4 * q - 1], Rh = rowH[4 * q + 4];
      const float Ll = rowL[4 * q - 1], Rl = rowL[4 * q + 4];
      const long long gi = gown[h] + (long long)(p - zb) * plane_n;
      const float4 B1 = B1s[h], B2 = B2s[h];
      const float s = Ss[h];
      float res[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float xmh = o == 0 ? Lh : comp4(Vh[h], o - 1), xph = o == 3 ? Rh : comp4(Vh[h], o + 1);
        const float xml = o == 0 ? Ll : comp4(Vl[h], o - 1), xpl = o == 3 ? Rl : comp4(Vl[h], o + 1);
        const float b1v = beta * comp4(B1, o), b2v = beta * comp4(B2, o);
        res[o] = defect_cell(xmh, xph, comp4(Uh, o), comp4(Dh, o), comp4(Mh[h], o), comp4(Ph[h], o),
                             comp4(Vh[h], o), xml, xpl, comp4(Ul, o), comp4(Dl, o), comp4(Ml[h], o),
                             comp4(Pl[h], o), comp4(Vl[h], o), b1v, b2v, bl != nullptr, s,
                             S != nullptr, G.ih_hi, G.ih_lo, G.dch, G.dcl);
        if (NORMS) {
          const float bv = b1v + (bl ? b2v : 0.f) + s;
          r2 = __fmaf_rn(res[o], res[o], r2);
          b2 = __fmaf_rn(bv, bv, b2);
        }
      }
      *reinterpret_cast<float4*>(out + gi) = make_float4(res[0], res[1], res[2], res[3]);
    }
    if (NORMS) {
      rr += (double)r2;
      bb += (double)b2;
    }
  }
  cp_async_wait0();
  if (NORMS) {
    rr = block_sum(rr);
    bb = block_sum(bb);
    if (threadIdx.x == 0) {
      const long long nb = (long long)gridDim.x * gridDim.y;
      double* o = partials + ((long long)comp * nb + blockIdx.x + (long long)gridDim.x * blockIdx.y) * 2;
      o[0] = rr;
      o[1] = bb;
    }
  }
}

// launches the tiled defect when the level allows it; returns the number of
// partial-sum blocks per component (0 if it did not launch)
int launch_defect_tiled(Ctx& cx, const Level& L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                        Comp3<float> BL, Comp3<float> OUT, int ncomp, double* partials, int max_blocks,
                        bool ragged) {
  const bool aligned = tile::level_ok(L);
  if (!aligned && !(ragged && tile::ragged_ok(L) && tile::tile_fill(L) >= 0.25 &&
                    L.cells() >= (1 << 17)))
    return 0;
  // one row per thread: 8-row tiles, three CTAs per SM (four, at 64
  // registers, spill and run slower)
  constexpr int ROWS = 1;
  using Sh = DefShape<ROWS>;
  const int ntx = (L.n[0] + tile::kTX - 1) / tile::kTX, nty = (L.n[1] + Sh::kRows - 1) / Sh::kRows;
  const int tiles = ntx * nty;
  int chunk = tile::pick_zchunk(L, std::max(ncomp, cx.chunk_comps), 3 * cx.sms, 2);
  chunk = std::max(chunk, 1);
  // pick_zchunk counts 128 x 16 tiles; there are twice as many 8-row tiles
  chunk = std::min(L.n[2], 2 * chunk);
  while (tiles * ((L.n[2] + chunk - 1) / chunk) * ncomp > max_blocks && chunk < L.n[2]) ++chunk;
  const int nz = (L.n[2] + chunk - 1) / chunk;
  if (tiles * nz * ncomp > max_blocks) return 0;
  DefGeom G;
  static_cast<tile::Geom&>(G) = tile::geom(L, chunk);
  G.nty = nty;
  G.ih_hi = (float)L.inv_h2;
  G.ih_lo = (float)(L.inv_h2 - (double)G.ih_hi);
  G.beta = R.beta;
  G.dch = L.cdh[0];
  G.dcl = L.cdl[0];
  static bool attr = false;
  if (!attr) {
    auto set = [](auto kern) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::kSmem);
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    };
    set(k_defect_tiled<ROWS, false, false>);
    set(k_defect_tiled<ROWS, true, false>);
    set(k_defect_tiled<ROWS, false, true>);
    set(k_defect_tiled<ROWS, true, true>);
    attr = true;
  }
  dim3 grid(tiles, nz, ncomp);
  auto kern = aligned ? (partials ? k_defect_tiled<ROWS, false, true> : k_defect_tiled<ROWS, false, false>)
                      : (partials ? k_defect_tiled<ROWS, true, true> : k_defect_tiled<ROWS, true, false>);
  cx.before(VSV_KCLASS_RESTRICT);
  launch_k(cx, kern, grid, tile::kThreads, Sh::kSmem, G, XH, XL, R, BL, OUT, partials);
  // x_hi, x_lo, b_hi (, b_lo) read, r written
  cx.after(VSV_KCLASS_RESTRICT, (BL.p[0] ? 20.0 : 16.0) * (double)L.cells() * ncomp);
  return tiles * nz;
}

void launch_update_dw(Ctx& cx, Comp3<float> XH, Comp3<float> XL, Comp3<float> E, long long n,
                      int ncomp) {
  const long long b = std::min<long long>((n + kBlock - 1) / kBlock, 8LL * cx.sms);
  dim3 grid((unsigned)b, ncomp);
  cx.before(VSV_KCLASS_PROLONG);
  launch_k(cx, k_update_dw, grid, kBlock, 0, XH, XL, E, n);
  cx.after(VSV_KCLASS_PROLONG, 20.0 * (double)n * ncomp);   // x_hi, x_lo, e read; x_hi, x_lo written
}

void launch_extrapolate_rot_dw(Ctx& cx, Comp3<float> AH, Comp3<float> AL, Comp3<float> BH,
                               Comp3<float> BL, Comp3<float> CH, Comp3<float> CL, long long n,
                               int ncomp, int order) {
  const long long b = std::min<long long>((n + kBlock - 1) / kBlock, 8LL * cx.sms);
  dim3 grid((unsigned)b, ncomp);
  cx.before(-1);
  launch_k(cx, k_extrapolate_rot_dw, grid, kBlock, 0, AH, AL, BH, CH, CL, n, order);
  // read: A's two words and the high words of B (order >= 1) and C (order
  // 2); written: the guess's two words
  cx.after(-1, (16.0 + 4.0 * (double)order) * (double)n * ncomp);
}

void launch_axpy_dw(Ctx& cx, Comp3<float> YH, Comp3<float> YL, Comp3<float> XH, Comp3<float> XL,
                    double a, long long n, int ncomp) {
  const long long b = std::min<long long>((n + kBlock - 1) / kBlock, 8LL * cx.sms);
  dim3 grid((unsigned)b, ncomp);
  const float a_hi = (float)a, a_lo = (float)(a - (double)a_hi);
  cx.before(-1);
  launch_k(cx, k_axpy_dw, grid, kBlock, 0, YH, YL, XH, XL, a_hi, a_lo, n);
  cx.after(-1, 24.0 * (double)n * ncomp);   // y, x read, y written (two words each)
}

}  // namespace vsv
