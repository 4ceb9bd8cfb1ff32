// Outer defect correction of the mixed path with a double-word iterate.
//
// The iterate x = x_hi + x_lo (two FP32 words, about 44 significant bits) is
// refined by   r = b - L_h x  (exact: cascaded summation of every FP32 term,
// one final rounding),   L_h e = r  (one FP32 multigrid V-cycle from e = 0),
// x <- x + e (double-word addition).  The defect sees x to FP64-class
// accuracy, so the refinement converges to the discrete solution below FP32
// rounding and the relative residual is a meaningful stopping test.
#include <algorithm>

#include "internal.h"

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

}  // namespace

// r = beta (B_hi + B_lo) + S(y, z) - L_h (x_hi + x_lo), exactly up to the final
// rounding; optional FP64 partial sums of ||r||^2 and ||b||^2 per block.
__global__ void k_defect_dw(Level L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                            Comp3<float> BL, Comp3<float> OUT, double* partials, float ih_hi,
                            float ih_lo) {
  const int comp = blockIdx.y;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  NbFetch H{XH.p[comp], nx, ny, nz, {L.per[0], L.per[1], L.per[2]}, {L.act[0], L.act[1], L.act[2]}};
  NbFetch Lo{XL.p[comp], nx, ny, nz, {L.per[0], L.per[1], L.per[2]}, {L.act[0], L.act[1], L.act[2]}};
  const float* __restrict__ bh = R.B[comp];
  const float* __restrict__ bl = BL.p[comp];
  const float* __restrict__ S = R.S[comp];
  float* __restrict__ out = OUT.p[comp];
  const float beta = R.beta;
  const float dcoef = (float)(2 * (L.act[0] + L.act[1] + L.act[2]));
  double rr = 0.0, bb = 0.0;
  for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
    const int j = row % ny, k = row / ny;
    const float s = S ? S[j + (long long)k * ny] : 0.f;
    float r2 = 0.f, b2 = 0.f;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long t = lin(i, j, k, nx, ny);
      CascadeSum lh(0.f);
      float llo = 0.f;
      if (L.act[0]) {
        lh.add(H.get(i - 1, j, k)); lh.add(H.get(i + 1, j, k));
        llo += Lo.get(i - 1, j, k) + Lo.get(i + 1, j, k);
      }
      if (L.act[1]) {
        lh.add(H.get(i, j - 1, k)); lh.add(H.get(i, j + 1, k));
        llo += Lo.get(i, j - 1, k) + Lo.get(i, j + 1, k);
      }
      if (L.act[2]) {
        lh.add(H.get(i, j, k - 1)); lh.add(H.get(i, j, k + 1));
        llo += Lo.get(i, j, k - 1) + Lo.get(i, j, k + 1);
      }
      lh.add_scaled(-dcoef, H.a[t]);
      llo = __fmaf_rn(-dcoef, Lo.a[t], llo);
      // L x = (lh.hi + lh.lo + llo) * inv_h2, leading product split exactly
      const float p = __fmul_rn(ih_hi, lh.hi);
      const float pe = __fmaf_rn(ih_hi, lh.hi, -p);
      const float rest = __fmaf_rn(ih_hi, __fadd_rn(lh.lo, llo), __fmaf_rn(ih_lo, lh.hi, pe));
      const float b1 = beta * bh[t];
      CascadeSum r(b1);
      if (bl) r.add(beta * bl[t]);
      r.add(s);
      r.add(-p);
      r.add(-rest);
      const float rv = r.value();
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
  const int comp = blockIdx.y;
  float* __restrict__ xh = XH.p[comp];
  float* __restrict__ xl = XL.p[comp];
  const float* __restrict__ e = E.p[comp];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const FF v = ff_add_f(FF{xh[t], xl[t]}, e[t]);
    xh[t] = v.hi;
    xl[t] = v.lo;
  }
}

// x <- 2 x - xp and xp <- old x in double-word arithmetic (extrapolate = 1);
// xp <- x only (extrapolate = 0).
__global__ void k_extrapolate_dw(Comp3<float> XH, Comp3<float> XL, Comp3<float> PH, Comp3<float> PL,
                                 long long n, int extrapolate) {
  const int comp = blockIdx.y;
  float* __restrict__ xh = XH.p[comp];
  float* __restrict__ xl = XL.p[comp];
  float* __restrict__ ph = PH.p[comp];
  float* __restrict__ pl = PL.p[comp];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const FF x{xh[t], xl[t]};
    if (extrapolate) {
      const FF v = ff_add(FF{2.f * x.hi, 2.f * x.lo}, ff_neg(FF{ph[t], pl[t]}));
      xh[t] = v.hi;
      xl[t] = v.lo;
    }
    ph[t] = x.hi;
    pl[t] = x.lo;
  }
}

void launch_defect_dw(Ctx& cx, const Level& L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                      Comp3<float> BL, Comp3<float> OUT, int ncomp, double* partials, int nblocks) {
  const float ih_hi = (float)L.inv_h2, ih_lo = (float)(L.inv_h2 - (double)ih_hi);
  dim3 grid(nblocks, ncomp);
  cx.before(VSV_KCLASS_RESTRICT);
  k_defect_dw<<<grid, kBlock, 0, cx.stream>>>(L, XH, XL, R, BL, OUT, partials, ih_hi, ih_lo);
  cx.after(VSV_KCLASS_RESTRICT);
}

void launch_update_dw(Ctx& cx, Comp3<float> XH, Comp3<float> XL, Comp3<float> E, long long n,
                      int ncomp) {
  const long long b = std::min<long long>((n + kBlock - 1) / kBlock, 8 * 152);
  dim3 grid((unsigned)b, ncomp);
  cx.before(VSV_KCLASS_PROLONG);
  k_update_dw<<<grid, kBlock, 0, cx.stream>>>(XH, XL, E, n);
  cx.after(VSV_KCLASS_PROLONG);
}

void launch_extrapolate_dw(Ctx& cx, Comp3<float> XH, Comp3<float> XL, Comp3<float> PH,
                           Comp3<float> PL, long long n, int ncomp, int extrapolate) {
  const long long b = std::min<long long>((n + kBlock - 1) / kBlock, 8 * 152);
  dim3 grid((unsigned)b, ncomp);
  cx.before(-1);
  k_extrapolate_dw<<<grid, kBlock, 0, cx.stream>>>(XH, XL, PH, PL, n, extrapolate);
  cx.after(-1);
}

}  // namespace vsv
