// Poisson kernels: red-black Gauss-Seidel / SOR sweeps, exact-defect
// residual with restriction, trilinear prolongation, coarsest-level solve and
// residual norms.  Main-text eqs. gen1 and gen3 are Poisson problems per
// Cartesian component; the paper solves them "using an iterative method"
// (numerical-implementation section) -- this file is that method on the GPU:
// cell-centred multigrid V-cycles (or red-black SOR), templated on the
// storage type (float for the mixed path, double for the FP64 path).
#include <algorithm>

#include "internal.h"

namespace vsv {

// Visit the neighbour values of cell (i,j,k) on level L in the order x-, x+,
// y-, y+, z-, z+, skipping Dirichlet ghosts, which are counted in nwall
// instead (their value is -alpha * x_c, zero on the fine level).
template <class T, class F>
__device__ __forceinline__ void for_nb(const T* __restrict__ x, const Level& L, int i, int j, int k,
                                       long long c, int& nwall, F&& f) {
  nwall = 0;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const long long sy = nx, sz = (long long)nx * ny;
  if (L.act[0]) {
    if (i > 0) f(x[c - 1]); else if (L.per[0]) f(x[c + nx - 1]); else ++nwall;
    if (i < nx - 1) f(x[c + 1]); else if (L.per[0]) f(x[c - (nx - 1)]); else ++nwall;
  }
  if (L.act[1]) {
    if (j > 0) f(x[c - sy]); else if (L.per[1]) f(x[c + (ny - 1) * sy]); else ++nwall;
    if (j < ny - 1) f(x[c + sy]); else if (L.per[1]) f(x[c - (ny - 1) * sy]); else ++nwall;
  }
  if (L.act[2]) {
    if (k > 0) f(x[c - sz]); else if (L.per[2]) f(x[c + (nz - 1) * sz]); else ++nwall;
    if (k < nz - 1) f(x[c + sz]); else if (L.per[2]) f(x[c - (nz - 1) * sz]); else ++nwall;
  }
}

// Sum of the neighbour values as ((x- + x+) + (y- + y+)) + (z- + z+), a
// Dirichlet ghost or an inactive axis contributing zero.  Every sweep,
// residual and transfer kernel sums in this order, so they agree bit for bit.
template <class T>
__device__ __forceinline__ T sum_nb(const T* __restrict__ x, const Level& L, int i, int j, int k,
                                    long long c, int& nwall) {
  nwall = 0;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const long long sy = nx, sz = (long long)nx * ny;
  T a = 0, b = 0, s[3];
  if (L.act[0]) {
    if (i > 0) a = x[c - 1]; else if (L.per[0]) a = x[c + nx - 1]; else ++nwall;
    if (i < nx - 1) b = x[c + 1]; else if (L.per[0]) b = x[c - (nx - 1)]; else ++nwall;
  }
  s[0] = a + b;
  a = 0; b = 0;
  if (L.act[1]) {
    if (j > 0) a = x[c - sy]; else if (L.per[1]) a = x[c + (ny - 1) * sy]; else ++nwall;
    if (j < ny - 1) b = x[c + sy]; else if (L.per[1]) b = x[c - (ny - 1) * sy]; else ++nwall;
  }
  s[1] = a + b;
  a = 0; b = 0;
  if (L.act[2]) {
    if (k > 0) a = x[c - sz]; else if (L.per[2]) a = x[c + (nz - 1) * sz]; else ++nwall;
    if (k < nz - 1) b = x[c + sz]; else if (L.per[2]) b = x[c - (nz - 1) * sz]; else ++nwall;
  }
  s[2] = a + b;
  return (s[0] + s[1]) + s[2];
}

template <class T>
__device__ __forceinline__ T rhs_at(const Rhs3<T>& R, int comp, long long c, int j, int k, int ny) {
  T b = R.beta * R.b_at(comp)[c];
  if (R.s_at(comp)) b += R.s_at(comp)[j + (long long)k * ny];
  return b;
}

__device__ __forceinline__ int n_active(const Level& L) { return L.act[0] + L.act[1] + L.act[2]; }

// ---------------------------------------------------------------- residual value
// r = b - L_h x at one cell, plain arithmetic in T.
template <class T>
__device__ __forceinline__ T resid_plain(const T* __restrict__ x, const Level& L, int i, int j, int k,
                                         long long c, T b) {
  int nwall;
  const T s = sum_nb(x, L, i, j, k, c, nwall);
  T coef = (T)(2 * n_active(L)) + lv_alpha<T>(L) * (T)nwall + lv_sh2<T>(L);
  return b - (s - coef * x[c]) * lv_ih2<T>(L);
}

// Exact defect in FP32 storage: every term of b - (sum_nb - coef x_c)/h^2 is
// accumulated by cascaded summation, so the result equals the real-number
// defect up to one final rounding (the diagonal coefficient enters as an
// FP32 pair; it is the integer 2 d on the fine level of a Poisson problem).
__device__ __forceinline__ float resid_exact(const float* __restrict__ x, const Level& L, int i,
                                             int j, int k, long long c, float b, float ih_hi,
                                             float ih_lo) {
  int nwall;
  CascadeSum t(0.f);
  for_nb(x, L, i, j, k, c, nwall, [&](float v) { t.add(v); });
  t.add_scaled(-L.cdh[nwall], x[c]);
  if (L.cdl[nwall] != 0.f) t.add(-L.cdl[nwall] * x[c]);   // adding -0 would change nothing
  if (ih_hi == 1.f && ih_lo == 0.f) {
    CascadeSum r(b);
    r.add(-t.hi);
    r.add(-t.lo);
    return r.value();
  }
  // (ih_hi + ih_lo) * (t.hi + t.lo) with the leading product split exactly
  float p = __fmul_rn(ih_hi, t.hi);
  float pe = __fmaf_rn(ih_hi, t.hi, -p);
  float rest = __fmaf_rn(ih_hi, t.lo, __fmaf_rn(ih_lo, t.hi, pe));
  CascadeSum r(b);
  r.add(-p);
  r.add(-rest);
  return r.value();
}

template <class T, bool EXACT>
__device__ __forceinline__ T resid_at(const T* __restrict__ x, const Level& L, int i, int j, int k,
                                      long long c, T b, float ih_hi, float ih_lo) {
  if constexpr (EXACT) {
    return resid_exact(x, L, i, j, k, c, b, ih_hi, ih_lo);
  } else {
    return resid_plain(x, L, i, j, k, c, b);
  }
}

// ---------------------------------------------------------------- sweeps
// One colour of a red-black Gauss-Seidel sweep (omega = 1) or SOR sweep
// (the red-black SOR solver, or over-relaxed multigrid smoothing),
// colour = (i + j + k) & 1, in place.  Thread t handles the t-th cell of the
// colour in its x row.
template <class T>
__global__ void k_rb_sweep(Level L, Comp3<T> X, Rhs3<T> R, int color, T omega, T h2) {
  pdl_begin();
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  int i2, j, k, comp;
  if (!cell3((nx + 1) >> 1, ny, nz, i2, j, k, comp)) return;
  T* __restrict__ x = X.at(comp);
  const int i = 2 * i2 + ((j + k + color) & 1);
  if (i >= nx) return;
  const long long c = lin(i, j, k, nx, ny);
  int nwall;
  const T s = sum_nb(x, L, i, j, k, c, nwall);
  const T b = rhs_at(R, comp, c, j, k, ny);
  x[c] = relax(x[c], nb_term(s, b, h2), wscale(omega, lv_rc<T>(L, nwall)), (T)1 - omega);
}

// Residual of the fine (or any) level, restricted to the next coarser level
// by averaging the children of each coarse cell.
template <class T, bool EXACT>
__global__ void k_resid_restrict(Level F, Level C, Comp3<T> X, Rhs3<T> R, Comp3<T> RC, float ih_hi,
                                 float ih_lo) {
  pdl_begin();
  int I, J, K, comp;
  if (!cell3(C.n[0], C.n[1], C.n[2], I, J, K, comp)) return;
  const T* __restrict__ x = X.at(comp);
  const long long t = lin(I, J, K, C.n[0], C.n[1]);
  const int fx = F.n[0] / C.n[0], fy = F.n[1] / C.n[1], fz = F.n[2] / C.n[2];
  T acc = 0;
  for (int dk = 0; dk < fz; ++dk)
    for (int dj = 0; dj < fy; ++dj)
      for (int di = 0; di < fx; ++di) {
        const int i = I * fx + di, j = J * fy + dj, k = K * fz + dk;
        const long long c = lin(i, j, k, F.n[0], F.n[1]);
        const T b = rhs_at(R, comp, c, j, k, F.n[1]);
        acc += resid_at<T, EXACT>(x, F, i, j, k, c, b, ih_hi, ih_lo);
      }
  RC.at(comp)[t] = acc / (T)(fx * fy * fz);
}

// One axis of the cell-centred linear interpolation: the two coarse indices
// and weights for fine index i (child of I = i / f).
template <class T>
struct Interp1 {
  int idx[2];
  T w[2];
};

template <class T>
__device__ __forceinline__ Interp1<T> interp_axis(int i, int f, int nC, int per, T alpha) {
  Interp1<T> r;
  if (f == 1) {
    r.idx[0] = r.idx[1] = i;
    r.w[0] = (T)1;
    r.w[1] = (T)0;
    return r;
  }
  const int I = i >> 1;
  const int off = (i & 1) ? 1 : -1;
  int I2 = I + off;
  r.idx[0] = I;
  r.w[0] = (T)0.75;
  if (I2 < 0 || I2 >= nC) {
    if (per) {
      I2 = (I2 + nC) % nC;
      r.idx[1] = I2;
      r.w[1] = (T)0.25;
    } else {  // ghost = -alpha * e(I)
      r.idx[1] = I;
      r.w[1] = (T)(-0.25) * alpha;
    }
  } else {
    r.idx[1] = I2;
    r.w[1] = (T)0.25;
  }
  return r;
}

// x_fine += P e_coarse (trilinear, cell centred).
template <class T>
__global__ void k_prolong_add(Level F, Level C, Comp3<T> X, Comp3<T> E) {
  pdl_begin();
  int i, j, k, comp;
  if (!cell3(F.n[0], F.n[1], F.n[2], i, j, k, comp)) return;
  const long long t = lin(i, j, k, F.n[0], F.n[1]);
  const T al = lv_alpha<T>(C);
  const Interp1<T> ax = interp_axis<T>(i, F.n[0] / C.n[0], C.n[0], C.per[0], al);
  const Interp1<T> ay = interp_axis<T>(j, F.n[1] / C.n[1], C.n[1], C.per[1], al);
  const Interp1<T> az = interp_axis<T>(k, F.n[2] / C.n[2], C.n[2], C.per[2], al);
  const T* __restrict__ e = E.at(comp);
  T acc = 0;
  for (int c2 = 0; c2 < 2; ++c2)
    for (int b2 = 0; b2 < 2; ++b2)
      for (int a2 = 0; a2 < 2; ++a2) {
        const T w = ax.w[a2] * ay.w[b2] * az.w[c2];
        if (w != (T)0) acc += w * e[lin(ax.idx[a2], ay.idx[b2], az.idx[c2], C.n[0], C.n[1])];
      }
  X.at(comp)[t] += acc;
}

template <class T>
__global__ void k_zero(Comp3<T> X, long long n) {
  pdl_begin();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) X.at(blockIdx.y)[t] = (T)0;
}

// First guess of a solve from the history, written into the oldest buffer
// C: order 0: A; 1: 2A - B; 2: 3(A - B) + C (A = x^n, B = x^{n-1}, C =
// x^{n-2}; extrapolation in time of order 0, 1, 2).
template <class T>
__global__ void k_extrapolate_rot(Comp3<T> A, Comp3<T> B, Comp3<T> C, long long n, int order) {
  pdl_begin();
  const int comp = blockIdx.y;
  const T* __restrict__ a = A.at(comp);
  const T* __restrict__ b = B.at(comp);
  T* __restrict__ c = C.at(comp);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const T x = a[t];
    if (order == 0) c[t] = x;
    else if (order == 1) c[t] = (T)2 * x - b[t];
    else c[t] = (T)3 * (x - b[t]) + c[t];
  }
}

// y += a x (the inertial right-hand side f - s omega'^n, FP64 path).
template <class T>
__global__ void k_axpy(Comp3<T> Y, Comp3<T> X, T a, long long n) {
  pdl_begin();
  const int comp = blockIdx.y;
  T* __restrict__ y = Y.at(comp);
  const T* __restrict__ x = X.at(comp);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}

// Coarsest level: e = 0, then `sweeps` red-black Gauss-Seidel sweeps in
// shared memory by one block per component.
template <class T>
__global__ void k_coarse_solve(Level L, Comp3<T> E, Comp3<T> RR, int sweeps, T h2) {
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  T* e = reinterpret_cast<T*>(smem_raw);
  const int comp = blockIdx.y;
  const long long n = L.cells();
  const T* __restrict__ r = RR.at(comp);
  T* rs = e + n;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    e[t] = 0;
    rs[t] = r[t];
  }
  __syncthreads();
  const int nx = L.n[0], ny = L.n[1], nxh = (nx + 1) >> 1;
  const int nh = nxh * ny * L.n[2];   // cells of one colour, rounded up per row
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (int t2 = threadIdx.x; t2 < nh; t2 += blockDim.x) {
        const int i2 = t2 % nxh, q = t2 / nxh;
        const int j = q % ny, k = q / ny;
        const int i = 2 * i2 + ((j + k + color) & 1);
        if (i >= nx) continue;
        const int t = (k * ny + j) * nx + i;
        int nwall;
        const T sum = sum_nb(e, L, i, j, k, t, nwall);
        e[t] = relax(e[t], nb_term(sum, rs[t], h2), lv_rc<T>(L, nwall), (T)0);
      }
      __syncthreads();
    }
  for (long long t = threadIdx.x; t < n; t += blockDim.x) E.at(comp)[t] = e[t];
}

// Per-block partial sums of ||b - L x||^2 and ||b||^2 (FP64 accumulation).
template <class T, bool EXACT>
__global__ void k_resid_norm(Level L, Comp3<T> X, Rhs3<T> R, double* partials, float ih_hi,
                             float ih_lo) {
  pdl_begin();
  const int comp = blockIdx.y;
  const T* __restrict__ x = X.at(comp);
  const int rows = L.n[1] * L.n[2];
  double rr = 0.0, bb = 0.0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % L.n[1], k = row / L.n[1];
    T r2 = 0, b2 = 0;   // per-row partial in T, then FP64 across rows
    for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
      const long long t = lin(i, j, k, L.n[0], L.n[1]);
      const T b = rhs_at(R, comp, t, j, k, L.n[1]);
      const T r = resid_at<T, EXACT>(x, L, i, j, k, t, b, ih_hi, ih_lo);
      r2 += r * r;
      b2 += b * b;
    }
    rr += (double)r2;
    bb += (double)b2;
  }
  rr = block_sum(rr);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    double* out = partials + ((long long)comp * gridDim.x + blockIdx.x) * 2;
    out[0] = rr;
    out[1] = bb;
  }
}

// Sum the partials of k_resid_norm in a fixed order (one block per comp).
__global__ void k_norm_finalize(const double* partials, int nblocks, Scalars* S) {
  pdl_begin();
  const int comp = blockIdx.x;
  double rr = 0.0, bb = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    rr += partials[((long long)comp * nblocks + b) * 2];
    bb += partials[((long long)comp * nblocks + b) * 2 + 1];
  }
  rr = block_sum(rr);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    S->rnorm2[comp] = rr;
    S->bnorm2[comp] = bb;
  }
}

// ---------------------------------------------------------------- blocked transfers
// Both kernels below take one coarse cell per thread and handle its 2x2x2
// fine children together; they require every axis to be coarsened by two
// (the coarse-level index I owns fine cells 2I and 2I+1 on every axis).

// Index of an outer neighbour (one cell beyond a 2-cell block) along one
// axis: wrapped on a periodic axis, -1 for a Dirichlet ghost.
__device__ __forceinline__ int outer_idx(int i, int n, int per) {
  if (i < 0) return per ? i + n : -1;
  if (i >= n) return per ? i - n : -1;
  return i;
}

template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <class T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
  const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(p);
  a = v.x;
  b = v.y;
}

// Residual of the 8 children, averaged onto the coarse cell (plain
// arithmetic, neighbours summed pairwise as in sum_nb).  The
// children of coarse x index I are fine 2I, 2I+1 (an aligned pair).
template <class T>
__global__ void k_restrict_block(Level F, Level C, Comp3<T> X, Rhs3<T> R, Comp3<T> RC) {
  pdl_begin();
  int I, J, K, comp;
  if (!cell3(C.n[0], C.n[1], C.n[2], I, J, K, comp)) return;
  const T* __restrict__ x = X.at(comp);
  const int nx = F.n[0], ny = F.n[1], nz = F.n[2];
  const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
  const int xm = outer_idx(i0 - 1, nx, F.per[0]), xp = outer_idx(i0 + 2, nx, F.per[0]);
  const int ym = outer_idx(j0 - 1, ny, F.per[1]), yp = outer_idx(j0 + 2, ny, F.per[1]);
  const int zm = outer_idx(k0 - 1, nz, F.per[2]), zp = outer_idx(k0 + 2, nz, F.per[2]);
  auto row = [&](int j, int k) { return x + ((long long)k * ny + j) * nx; };
  T c[2][2][2], fxm[2][2], fxp[2][2], fym[2][2], fyp[2][2], fzm[2][2], fzp[2][2], b[2][2][2];
#pragma unroll
  for (int kz = 0; kz < 2; ++kz)
#pragma unroll
    for (int jy = 0; jy < 2; ++jy) {
      const T* r = row(j0 + jy, k0 + kz);
      ld2(r + i0, c[kz][jy][0], c[kz][jy][1]);
      fxm[kz][jy] = xm >= 0 ? r[xm] : (T)0;
      fxp[kz][jy] = xp >= 0 ? r[xp] : (T)0;
      const long long t = ((long long)(k0 + kz) * ny + j0 + jy) * nx + i0;
      ld2(R.b_at(comp) + t, b[kz][jy][0], b[kz][jy][1]);
      const T s = R.s_at(comp) ? R.s_at(comp)[j0 + jy + (long long)(k0 + kz) * ny] : (T)0;
      b[kz][jy][0] = R.beta * b[kz][jy][0] + s;
      b[kz][jy][1] = R.beta * b[kz][jy][1] + s;
    }
#pragma unroll
  for (int kz = 0; kz < 2; ++kz) {
    if (ym >= 0) ld2(row(ym, k0 + kz) + i0, fym[kz][0], fym[kz][1]); else fym[kz][0] = fym[kz][1] = (T)0;
    if (yp >= 0) ld2(row(yp, k0 + kz) + i0, fyp[kz][0], fyp[kz][1]); else fyp[kz][0] = fyp[kz][1] = (T)0;
  }
#pragma unroll
  for (int jy = 0; jy < 2; ++jy) {
    if (zm >= 0) ld2(row(j0 + jy, zm) + i0, fzm[jy][0], fzm[jy][1]); else fzm[jy][0] = fzm[jy][1] = (T)0;
    if (zp >= 0) ld2(row(j0 + jy, zp) + i0, fzp[jy][0], fzp[jy][1]); else fzp[jy][0] = fzp[jy][1] = (T)0;
  }
  const T ih2 = lv_ih2<T>(F), al = lv_alpha<T>(F), sh = lv_sh2<T>(F);
  T acc = 0;
#pragma unroll
  for (int kz = 0; kz < 2; ++kz)
#pragma unroll
    for (int jy = 0; jy < 2; ++jy)
#pragma unroll
      for (int ix = 0; ix < 2; ++ix) {
        const T v_xm = ix == 0 ? fxm[kz][jy] : c[kz][jy][0];
        const T v_xp = ix == 1 ? fxp[kz][jy] : c[kz][jy][1];
        const T v_ym = jy == 0 ? fym[kz][ix] : c[kz][0][ix];
        const T v_yp = jy == 1 ? fyp[kz][ix] : c[kz][1][ix];
        const T v_zm = kz == 0 ? fzm[jy][ix] : c[0][jy][ix];
        const T v_zp = kz == 1 ? fzp[jy][ix] : c[1][jy][ix];
        const int nwall = (ix == 0 && xm < 0) + (ix == 1 && xp < 0) + (jy == 0 && ym < 0) +
                          (jy == 1 && yp < 0) + (kz == 0 && zm < 0) + (kz == 1 && zp < 0);
        const T s = ((v_xm + v_xp) + (v_ym + v_yp)) + (v_zm + v_zp);
        acc += b[kz][jy][ix] - (s - ((T)6 + al * (T)nwall + sh) * c[kz][jy][ix]) * ih2;
      }
  RC.at(comp)[lin(I, J, K, C.n[0], C.n[1])] = acc * (T)0.125;
}

// Increments P e for the 8 children of coarse cell (I,J,K): weights 3/4 and
// 1/4 per axis; the coarse neighbours come from the coarse level's boundary
// rule: periodic wrap, or -alpha * (adjacent cell) per out-of-range axis (the
// linear extrapolation through zero at the wall).  v[c][b][a] is the child
// (2K+c, 2J+b, 2I+a).
template <class T>
__device__ __forceinline__ void prolong_children(const Level& C, const T* __restrict__ e, int I,
                                                 int J, int K, T v[2][2][2]) {
  const int cx_ = C.n[0], cy = C.n[1], cz = C.n[2];
  const T ma = -lv_alpha<T>(C);
  int ix[3], iy[3], iz[3];
  T fx[3], fy[3], fz[3];
  ix[1] = I; iy[1] = J; iz[1] = K;
  fx[1] = fy[1] = fz[1] = (T)1;
#pragma unroll
  for (int s = 0; s < 3; s += 2) {
    const int d = s - 1;
    int t = outer_idx(I + d, cx_, C.per[0]);
    ix[s] = t >= 0 ? t : I; fx[s] = t >= 0 ? (T)1 : ma;
    t = outer_idx(J + d, cy, C.per[1]);
    iy[s] = t >= 0 ? t : J; fy[s] = t >= 0 ? (T)1 : ma;
    t = outer_idx(K + d, cz, C.per[2]);
    iz[s] = t >= 0 ? t : K; fz[s] = t >= 0 ? (T)1 : ma;
  }
  T n[3][3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T* r = e + ((long long)iz[c] * cy + iy[b]) * cx_;
      const T f = fz[c] * fy[b];
#pragma unroll
      for (int a = 0; a < 3; ++a) n[c][b][a] = f * fx[a] * r[ix[a]];
    }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int ax = 2 * a, by = 2 * b, cz2 = 2 * c;
        v[c][b][a] = prolong_value<T>(n[1][1][1], n[1][1][ax], n[1][by][1], n[1][by][ax],
                                      n[cz2][1][1], n[cz2][1][ax], n[cz2][by][1], n[cz2][by][ax]);
      }
}

// x_fine += P e for the 8 children of one coarse cell per thread.
template <class T>
__global__ void k_prolong_block(Level F, Level C, Comp3<T> X, Comp3<T> E) {
  pdl_begin();
  int I, J, K, comp;
  if (!cell3(C.n[0], C.n[1], C.n[2], I, J, K, comp)) return;
  T v[2][2][2];
  prolong_children<T>(C, E.at(comp), I, J, K, v);
  T* __restrict__ x = X.at(comp);
  const int nx = F.n[0], ny = F.n[1];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      T* p = x + ((long long)(2 * K + c) * ny + 2 * J + b) * nx + 2 * I;
      typename Vec2<T>::type cur = *reinterpret_cast<typename Vec2<T>::type*>(p);
      cur.x += v[c][b][0];
      cur.y += v[c][b][1];
      *reinterpret_cast<typename Vec2<T>::type*>(p) = cur;
    }
}

__host__ __device__ bool blocked_transfer_ok(const Level& F, const Level& C) {
  for (int a = 0; a < 3; ++a)
    if (F.n[a] != 2 * C.n[a]) return false;
  return true;
}

// ---------------------------------------------------------------- coarse V-cycle in one CTA
// The levels from `first` down to the coarsest are small enough to live in
// shared memory; one CTA per component runs the whole lower part of the
// V-cycle there (same operations as the level-by-level kernels: red-black
// sweeps, residual restricted by averaging, trilinear prolongation), which
// replaces dozens of latency-bound launches per V-cycle by one.

// q = a / d, with rem = a - q d (0 <= a, 0 < d): a shift and a mask where d
// is a power of two (every level of a power-of-two grid), else a division.
__device__ __forceinline__ int cv_divmod(int a, int d, int& rem) {
  if ((d & (d - 1)) == 0) {
    rem = a & (d - 1);
    return a >> (__ffs(d) - 1);
  }
  const int q = a / d;
  rem = a - q * d;
  return q;
}

// The thread's cells of one colour are visited with the index (i2, j, k)
// advanced by the block size incrementally (adds and carries instead of two
// integer divisions per cell).  The neighbour sum, the wall count and the
// update are those of sum_nb and the per-colour sweep (same operands, same
// order of the additions), with 32-bit offsets into shared memory, and with
// the level's geometry and the weights omega rc (one per count of wall
// neighbours, in shared memory) formed once per call instead of per cell.
template <class T>
__device__ void cv_sweep(const Level& L, T* e, const T* r, int sweeps, T h2, T omega) {
  __shared__ T wtab[8];
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2], nxh = (nx + 1) >> 1;
  const int sz = nx * ny;
  const int nh = nxh * ny * nz;   // cells of one colour, rounded up per row
  const bool ax = L.act[0], ay = L.act[1], az = L.act[2];
  const bool px = L.per[0], py = L.per[1], pz = L.per[2];
  const T c1 = (T)1 - omega;
  const int B = blockDim.x;
  int Bi, Bj, i20, j0;
  const int Bk = cv_divmod(cv_divmod(B, nxh, Bi), ny, Bj);
  const int k0 = cv_divmod(cv_divmod((int)threadIdx.x, nxh, i20), ny, j0);
  if (threadIdx.x < 7) wtab[threadIdx.x] = wscale(omega, lv_rc<T>(L, (int)threadIdx.x));
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      int i2 = i20, j = j0, k = k0;
      for (int t2 = threadIdx.x; t2 < nh; t2 += B) {
        if (t2 != threadIdx.x) {
          i2 += Bi;
          int cj = Bj;
          if (i2 >= nxh) { i2 -= nxh; ++cj; }
          j += cj;
          int ck = Bk;
          while (j >= ny) { j -= ny; ++ck; }
          k += ck;
        }
        const int i = 2 * i2 + ((j + k + color) & 1);
        if (i >= nx) continue;
        const int t = (k * ny + j) * nx + i;
        int nwall = 0;
        T a = 0, b = 0;
        if (ax) {
          if (i > 0) a = e[t - 1]; else if (px) a = e[t + nx - 1]; else ++nwall;
          if (i < nx - 1) b = e[t + 1]; else if (px) b = e[t - (nx - 1)]; else ++nwall;
        }
        const T s0 = a + b;
        a = 0; b = 0;
        if (ay) {
          if (j > 0) a = e[t - nx]; else if (py) a = e[t + (ny - 1) * nx]; else ++nwall;
          if (j < ny - 1) b = e[t + nx]; else if (py) b = e[t - (ny - 1) * nx]; else ++nwall;
        }
        const T s1 = a + b;
        a = 0; b = 0;
        if (az) {
          if (k > 0) a = e[t - sz]; else if (pz) a = e[t + (nz - 1) * sz]; else ++nwall;
          if (k < nz - 1) b = e[t + sz]; else if (pz) b = e[t - (nz - 1) * sz]; else ++nwall;
        }
        const T s2 = a + b;
        e[t] = relax(e[t], nb_term((s0 + s1) + s2, r[t], h2), wtab[nwall], c1);
      }
      __syncthreads();
    }
}

template <class T>
__device__ void cv_restrict(const Level& F, const Level& C, const T* e, const T* r, T* rc) {
  const int nc = (int)C.cells();
  const int fx = F.n[0] / C.n[0], fy = F.n[1] / C.n[1], fz = F.n[2] / C.n[2];
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    int I, J;
    const int K = cv_divmod(cv_divmod(t, C.n[0], I), C.n[1], J);
    T acc = 0;
    for (int dk = 0; dk < fz; ++dk)
      for (int dj = 0; dj < fy; ++dj)
        for (int di = 0; di < fx; ++di) {
          const int i = I * fx + di, j = J * fy + dj, k = K * fz + dk;
          const int c = (k * F.n[1] + j) * F.n[0] + i;
          acc += resid_plain(e, F, i, j, k, c, r[c]);
        }
    rc[t] = acc / (T)(fx * fy * fz);
  }
  __syncthreads();
}

template <class T>
__device__ void cv_prolong(const Level& F, const Level& C, T* e, const T* ec) {
  if (blocked_transfer_ok(F, C)) {   // as k_prolong_block
    const int nc = (int)C.cells();
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      int I, J;
      const int K = cv_divmod(cv_divmod(t, C.n[0], I), C.n[1], J);
      T v[2][2][2];
      prolong_children<T>(C, ec, I, J, K, v);
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            e[((2 * K + c) * F.n[1] + 2 * J + b) * F.n[0] + 2 * I + a] += v[c][b][a];
    }
    __syncthreads();
    return;
  }
  const int nf = (int)F.cells();   // as k_prolong_add
  const T al = lv_alpha<T>(C);
  for (int t = threadIdx.x; t < nf; t += blockDim.x) {
    const int i = t % F.n[0], q = t / F.n[0];
    const int j = q % F.n[1], k = q / F.n[1];
    const Interp1<T> ax = interp_axis<T>(i, F.n[0] / C.n[0], C.n[0], C.per[0], al);
    const Interp1<T> ay = interp_axis<T>(j, F.n[1] / C.n[1], C.n[1], C.per[1], al);
    const Interp1<T> az = interp_axis<T>(k, F.n[2] / C.n[2], C.n[2], C.per[2], al);
    T acc = 0;
    for (int c2 = 0; c2 < 2; ++c2)
      for (int b2 = 0; b2 < 2; ++b2)
        for (int a2 = 0; a2 < 2; ++a2) {
          const T w = ax.w[a2] * ay.w[b2] * az.w[c2];
          if (w != (T)0) acc += w * ec[(az.idx[c2] * C.n[1] + ay.idx[b2]) * C.n[0] + ax.idx[a2]];
        }
    e[t] += acc;
  }
  __syncthreads();
}

// The lower V-cycle of one component in one CTA: rhs rr (level CC.first,
// global memory) -> correction e_out, every level in shared memory `base`.
template <class T>
__device__ void coarse_vcycle_cta(const CoarseCycle& CC, const T* __restrict__ rr,
                                  T* __restrict__ e_out, T* base) {
  const int f = CC.first, l_last = CC.last;
  // (e, r) of level l in shared memory; CC is a grid-constant parameter, so
  // its tables are read in place at run-time indices (no local copies)
  auto e = [&](int l) { return base + CC.off[l]; };
  auto r = [&](int l) { return base + CC.off[l] + CC.lv[l].cells(); };
  const int n0 = (int)CC.lv[f].cells();
  for (int t = threadIdx.x; t < n0; t += blockDim.x) {
    r(f)[t] = rr[t];
    e(f)[t] = (T)0;
  }
  __syncthreads();
  for (int l = f; l < l_last; ++l) {
    cv_sweep<T>(CC.lv[l], e(l), r(l), CC.nu1, (T)CC.h2[l], (T)CC.omega);
    cv_restrict<T>(CC.lv[l], CC.lv[l + 1], e(l), r(l), r(l + 1));
    const int nc = (int)CC.lv[l + 1].cells();
    T* ec = e(l + 1);
    for (int t = threadIdx.x; t < nc; t += blockDim.x) ec[t] = (T)0;
    __syncthreads();
  }
  cv_sweep<T>(CC.lv[l_last], e(l_last), r(l_last), CC.coarse_sweeps, (T)CC.h2[l_last], (T)1);
  for (int l = l_last - 1; l >= f; --l) {
    cv_prolong<T>(CC.lv[l], CC.lv[l + 1], e(l), e(l + 1));
    cv_sweep<T>(CC.lv[l], e(l), r(l), CC.nu2, (T)CC.h2[l], (T)CC.omega);
  }
  const T* e0 = e(f);
  for (int t = threadIdx.x; t < n0; t += blockDim.x) e_out[t] = e0[t];
}

template <class T>
__global__ void __launch_bounds__(1024)
k_coarse_vcycle(const __grid_constant__ CoarseCycle CC, Comp3<T> E, Comp3<T> RR) {
  pdl_begin();
  extern __shared__ unsigned char smem_cv[];
  const int comp = blockIdx.x;
  coarse_vcycle_cta<T>(CC, RR.at(comp), E.at(comp), reinterpret_cast<T*>(smem_cv));
}

template <class T>
bool launch_coarse_vcycle(Ctx& cx, const CoarseCycle& CC, Comp3<T> E, Comp3<T> R, int ncomp) {
  const size_t smem = (size_t)CC.total * sizeof(T);
  if (smem > kCoarseCycleSmem) return false;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_coarse_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return false;
  cx.before(VSV_KCLASS_SMOOTH);
  launch_k(cx, k_coarse_vcycle<T>, ncomp, 1024, smem, CC, E, R);
  // r of the first level read, e written; the rest stays in shared memory
  cx.after(VSV_KCLASS_SMOOTH, 2.0 * (double)sizeof(T) * (double)CC.lv[CC.first].cells() * ncomp);
  return true;
}

// ---------------------------------------------------------------- persistent lower V-cycle
// The levels below the finest fit in L2 and are bound by launch and
// barrier latency when run level by level (dozens of launches of a few to
// tens of microseconds each per V-cycle).  One cooperative launch runs them
// instead: every CTA of the grid (all co-resident) sweeps, restricts and
// prolongs levels first .. cc-1 with grid-stride loops, separated by grid
// barriers, and the levels cc .. last run as the one-CTA coarse cycle above
// (CTAs 0 .. ncomp-1, one component each) while the others wait.  Every
// operation is the per-colour reference kernels' arithmetic (sum_nb, relax,
// resid_plain, prolong_children / interp_axis), so the result is bit for
// bit that of the level-by-level V-cycle.

// Cells (a, j, k, comp) of a [ncomp][nz][ny][na] index space visited by a
// grid-stride loop: the flat index advances by the total thread count with
// carries instead of divisions.
struct StrideWalk {
  int a, j, k, c;
  int sa, sj, sk, sc;
  int na, ny, nz;
  __device__ __forceinline__ void init(long long t0, long long stride, int na_, int ny_, int nz_) {
    na = na_; ny = ny_; nz = nz_;
    long long q = t0;
    a = (int)(q % na); q /= na; j = (int)(q % ny); q /= ny; k = (int)(q % nz); c = (int)(q / nz);
    q = stride;
    sa = (int)(q % na); q /= na; sj = (int)(q % ny); q /= ny; sk = (int)(q % nz);
    sc = (int)(q / nz);
  }
  __device__ __forceinline__ void next() {
    a += sa;
    int cj = sj;
    if (a >= na) { a -= na; ++cj; }
    j += cj;
    int ck = sk;
    if (j >= ny) { j -= ny; ++ck; }
    k += ck;
    int cc = sc;
    if (k >= nz) { k -= nz; ++cc; }
    c += cc;
  }
};

// Bounded grid barrier (see GridBarrier).  Arrivals count up monotonically
// from zero (the host zeroes the counter before each launch), so barrier n
// waits until n * (gridDim.x + extra) arrivals.  Returns false when the
// wait ran out (bit kSyncTimeout of *status set, by this CTA or another);
// the caller then leaves the kernel.
__device__ __forceinline__ bool grid_sync(const GridBarrier& B, unsigned& epoch) {
  __shared__ int ok_s;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();                                    // publish this CTA's writes
    atomicAdd(B.count, 1u);
    const unsigned target = epoch * (gridDim.x + B.extra);
    const volatile unsigned* vc = B.count;
    const volatile int* vs = B.status;
    const unsigned long long t0 = global_ns();
    while (*vc < target) {
      if (*vs & kSyncTimeout) { ok = 0; break; }
      if (global_ns() - t0 > B.limit_ns) {
        atomicOr(B.status, kSyncTimeout);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();                                    // see the other CTAs' writes
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Number of Dirichlet ghosts among the 7-point neighbours of (i, j, k).
__device__ __forceinline__ int wall_count(const Level& L, int i, int j, int k) {
  int n = 0;
  if (L.act[0] && !L.per[0]) n += (i == 0) + (i == L.n[0] - 1);
  if (L.act[1] && !L.per[1]) n += (j == 0) + (j == L.n[1] - 1);
  if (L.act[2] && !L.per[2]) n += (k == 0) + (k == L.n[2] - 1);
  return n;
}

// One colour of a red-black sweep of level l, every component.  first:
// e is not yet initialised (a correction from zero): the red cells take
// their value from the rhs alone and the black cells are set to zero, as
// zeroing e and sweeping its red cells does.
template <class T>
__device__ void lc_sweep(const LowerCycle<T>& P, int l, int color, bool first, T omega) {
  const Level& L = P.lv[l];
  const int nx = L.n[0], nxh = (nx + 1) >> 1;
  const T h2 = (T)P.h2[l];
  StrideWalk w;
  w.init((long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, nxh,
         L.n[1], L.n[2]);
  for (; w.c < P.ncomp; w.next()) {
    T* __restrict__ x = P.e[l][w.c];
    const T* __restrict__ b = P.r[l][w.c];
    const int red = 2 * w.a + ((w.j + w.k + color) & 1);
    const long long row = lin(0, w.j, w.k, nx, L.n[1]);
    if (first) {
      // color is 0 here: the pair (2a, 2a + 1) holds one red and one black cell
      const int blk = red ^ 1;
      if (red < nx) {
        const long long c = row + red;
        x[c] = relax((T)0, nb_term((T)0, b[c], h2),
                     wscale(omega, lv_rc<T>(L, wall_count(L, red, w.j, w.k))), (T)1 - omega);
      }
      if (blk < nx) x[row + blk] = (T)0;
      continue;
    }
    if (red >= nx) continue;
    const long long c = row + red;
    int nwall;
    const T sn = sum_nb(x, L, red, w.j, w.k, c, nwall);
    x[c] = relax(x[c], nb_term(sn, b[c], h2), wscale(omega, lv_rc<T>(L, nwall)), (T)1 - omega);
  }
}

// Residual of level l restricted to level l + 1 (as k_resid_restrict).
template <class T>
__device__ void lc_restrict(const LowerCycle<T>& P, int l) {
  const Level& F = P.lv[l];
  const Level& C = P.lv[l + 1];
  const int fx = F.n[0] / C.n[0], fy = F.n[1] / C.n[1], fz = F.n[2] / C.n[2];
  StrideWalk w;
  w.init((long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
         C.n[0], C.n[1], C.n[2]);
  for (; w.c < P.ncomp; w.next()) {
    const T* __restrict__ x = P.e[l][w.c];
    const T* __restrict__ b = P.r[l][w.c];
    T acc = 0;
    for (int dk = 0; dk < fz; ++dk)
      for (int dj = 0; dj < fy; ++dj)
        for (int di = 0; di < fx; ++di) {
          const int i = w.a * fx + di, j = w.j * fy + dj, k = w.k * fz + dk;
          const long long c = lin(i, j, k, F.n[0], F.n[1]);
          acc += resid_plain(x, F, i, j, k, c, b[c]);
        }
    P.r[l + 1][w.c][lin(w.a, w.j, w.k, C.n[0], C.n[1])] = acc / (T)(fx * fy * fz);
  }
}

// e(l) += P e(l + 1) (as k_prolong_block, or k_prolong_add where an axis
// is not coarsened).
template <class T>
__device__ void lc_prolong(const LowerCycle<T>& P, int l) {
  const Level& F = P.lv[l];
  const Level& C = P.lv[l + 1];
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  StrideWalk w;
  if (blocked_transfer_ok(F, C)) {
    w.init(t0, stride, C.n[0], C.n[1], C.n[2]);
    for (; w.c < P.ncomp; w.next()) {
      T v[2][2][2];
      prolong_children<T>(C, P.e[l + 1][w.c], w.a, w.j, w.k, v);
      T* __restrict__ x = P.e[l][w.c];
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b) {
          T* p = x + ((long long)(2 * w.k + c) * F.n[1] + 2 * w.j + b) * F.n[0] + 2 * w.a;
          p[0] += v[c][b][0];
          p[1] += v[c][b][1];
        }
    }
    return;
  }
  const T al = lv_alpha<T>(C);
  w.init(t0, stride, F.n[0], F.n[1], F.n[2]);
  for (; w.c < P.ncomp; w.next()) {
    const Interp1<T> ax = interp_axis<T>(w.a, F.n[0] / C.n[0], C.n[0], C.per[0], al);
    const Interp1<T> ay = interp_axis<T>(w.j, F.n[1] / C.n[1], C.n[1], C.per[1], al);
    const Interp1<T> az = interp_axis<T>(w.k, F.n[2] / C.n[2], C.n[2], C.per[2], al);
    const T* __restrict__ ec = P.e[l + 1][w.c];
    T acc = 0;
    for (int c2 = 0; c2 < 2; ++c2)
      for (int b2 = 0; b2 < 2; ++b2)
        for (int a2 = 0; a2 < 2; ++a2) {
          const T wt = ax.w[a2] * ay.w[b2] * az.w[c2];
          if (wt != (T)0) acc += wt * ec[lin(ax.idx[a2], ay.idx[b2], az.idx[c2], C.n[0], C.n[1])];
        }
    P.e[l][w.c][lin(w.a, w.j, w.k, F.n[0], F.n[1])] += acc;
  }
}

// e(l) = 0 (a correction from zero that takes no pre-smoothing sweep).
template <class T>
__device__ void lc_zero(const LowerCycle<T>& P, int l) {
  const Level& L = P.lv[l];
  StrideWalk w;
  w.init((long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
         L.n[0], L.n[1], L.n[2]);
  for (; w.c < P.ncomp; w.next()) P.e[l][w.c][lin(w.a, w.j, w.k, L.n[0], L.n[1])] = (T)0;
}

template <class T>
__global__ void __launch_bounds__(1024)
k_lower_vcycle(const __grid_constant__ LowerCycle<T> P) {
  extern __shared__ unsigned char smem_lc[];
  unsigned epoch = 0;
  const T om = (T)P.omega;
  auto sweeps = [&](int l, int nu, bool from_zero) -> bool {
    if (nu == 0 && from_zero) {
      lc_zero<T>(P, l);
      return grid_sync(P.bar, epoch);
    }
    for (int s = 0; s < nu; ++s)
      for (int color = 0; color < 2; ++color) {
        lc_sweep<T>(P, l, color, from_zero && s == 0 && color == 0, om);
        if (!grid_sync(P.bar, epoch)) return false;
      }
    return true;
  };
  const int lw = P.cc;   // first level of the one-CTA part (last + 1: none)
  for (int l = P.first; l < lw; ++l) {
    if (l == P.last) {   // coarsest level solved grid-wide: plain Gauss-Seidel from zero
      for (int s = 0; s < P.coarse_sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
          lc_sweep<T>(P, l, color, s == 0 && color == 0, (T)1);
          if (!grid_sync(P.bar, epoch)) return;
        }
      break;
    }
    if (!sweeps(l, P.nu1, true)) return;
    lc_restrict<T>(P, l);
    if (!grid_sync(P.bar, epoch)) return;
  }
  if (lw <= P.last) {
    if (blockIdx.x < (unsigned)P.ncomp)
      coarse_vcycle_cta<T>(P.cc_plan, P.r[lw][blockIdx.x], P.e[lw][blockIdx.x],
                           reinterpret_cast<T*>(smem_lc));
    if (!grid_sync(P.bar, epoch)) return;
  }
  for (int l = min(lw, P.last) - 1; l >= P.first; --l) {
    lc_prolong<T>(P, l);
    if (!grid_sync(P.bar, epoch)) return;
    if (!sweeps(l, P.nu2, false)) return;
  }
}

// The barrier alone, for tests of its bound: `rounds` barriers of a grid
// that expects `extra` arrivals more per barrier than it has CTAs (extra > 0
// means the wait can only end by running out).
__global__ void k_barrier_probe(GridBarrier B, int rounds) {
  unsigned epoch = 0;
  for (int r = 0; r < rounds; ++r)
    if (!grid_sync(B, epoch)) return;
}

template <class T>
int lower_cycle_blocks(int sms, size_t smem) {
  int per_sm = 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_lower_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lower_vcycle<T>, 1024, smem) !=
      cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <class T>
bool launch_lower_vcycle(Ctx& cx, const LowerCycle<T>& P) {
  const size_t smem = P.cc <= P.last ? (size_t)P.cc_plan.total * sizeof(T) : 0;
  if (smem > kCoarseCycleSmem) return false;
  const int nb = lower_cycle_blocks<T>(cx.sms, smem);
  if (nb < P.ncomp || nb < 1) return false;
  if (cudaMemsetAsync(P.bar.count, 0, sizeof(unsigned), cx.stream) != cudaSuccess) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nb);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = cx.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs co-resident, or no launch
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cx.before(VSV_KCLASS_SMOOTH);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_lower_vcycle<T>, P);
  // r of the first level read, e written; the lower levels stay in L2
  cx.after(VSV_KCLASS_SMOOTH, 2.0 * (double)sizeof(T) * (double)P.lv[P.first].cells() * P.ncomp);
  return e == cudaSuccess;
}

int barrier_probe_max_blocks(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, 128, 0) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

bool launch_barrier_probe(cudaStream_t s, GridBarrier B, int blocks, int rounds) {
  if (cudaMemsetAsync(B.count, 0, sizeof(unsigned), s) != cudaSuccess) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_probe, B, rounds) == cudaSuccess;
}

// ---------------------------------------------------------------- launchers
static inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <class T>
void launch_rb_sweep(Ctx& cx, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, int color,
                     double omega, double h2, int kclass) {
  const dim3 grid = grid3((L.n[0] + 1) / 2, L.n[1], L.n[2], ncomp);
  cx.before(kclass);
  launch_k(cx, k_rb_sweep<T>, grid, block3(), 0, L, X, R, color, (T)omega, (T)h2);
  // one colour: the other colour's values and this colour's rhs read, this colour written
  // (and read, for SOR): 1.5 words per cell
  cx.after(kclass, (omega == 1.0 ? 1.5 : 2.0) * (double)sizeof(T) * (double)L.cells() * ncomp);
}

template <class T>
void launch_resid_restrict(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Rhs3<T> R,
                           Comp3<T> RC, int ncomp, bool exact) {
  const dim3 grid = grid3(C.n[0], C.n[1], C.n[2], ncomp);
  if constexpr (std::is_same<T, float>::value) {
    if (!exact && cx.tiled && launch_restrict_tiled(cx, F, C, X, R, RC, ncomp)) return;
  }
  if (!exact && blocked_transfer_ok(F, C)) {
    cx.before(VSV_KCLASS_RESTRICT);
    launch_k(cx, k_restrict_block<T>, grid, block3(), 0, F, C, X, R, RC);
    cx.after(VSV_KCLASS_RESTRICT, 2.125 * (double)sizeof(T) * (double)F.cells() * ncomp);
    return;
  }
  cx.before(VSV_KCLASS_RESTRICT);
  float ih_hi = (float)F.inv_h2, ih_lo = (float)(F.inv_h2 - (double)ih_hi);
  if constexpr (std::is_same<T, float>::value) {
    if (exact)
      launch_k(cx, k_resid_restrict<float, true>, grid, block3(), 0, F, C, X, R, RC, ih_hi, ih_lo);
    else
      launch_k(cx, k_resid_restrict<float, false>, grid, block3(), 0, F, C, X, R, RC, ih_hi, ih_lo);
  } else {
    launch_k(cx, k_resid_restrict<T, false>, grid, block3(), 0, F, C, X, R, RC, ih_hi, ih_lo);
  }
  cx.after(VSV_KCLASS_RESTRICT, (2.0 * (double)F.cells() + (double)C.cells()) * (double)sizeof(T) * ncomp);
}

template <class T>
void launch_prolong_add(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Comp3<T> E, int ncomp) {
  if constexpr (std::is_same<T, float>::value) {
    if (cx.tiled && launch_prolong_tiled(cx, F, C, X, E, ncomp)) return;
  }
  if (blocked_transfer_ok(F, C)) {
    cx.before(VSV_KCLASS_PROLONG);
    launch_k(cx, k_prolong_block<T>, grid3(C.n[0], C.n[1], C.n[2], ncomp), block3(), 0, F, C, X, E);
    cx.after(VSV_KCLASS_PROLONG, 2.125 * (double)sizeof(T) * (double)F.cells() * ncomp);
    return;
  }
  const dim3 grid = grid3(F.n[0], F.n[1], F.n[2], ncomp);
  cx.before(VSV_KCLASS_PROLONG);
  launch_k(cx, k_prolong_add<T>, grid, block3(), 0, F, C, X, E);
  cx.after(VSV_KCLASS_PROLONG, (2.0 * (double)F.cells() + (double)C.cells()) * (double)sizeof(T) * ncomp);
}

template <class T>
void launch_zero(Ctx& cx, Comp3<T> X, long long n, int ncomp) {
  dim3 grid(blocks_for(n), ncomp);
  cx.before(-1);
  launch_k(cx, k_zero<T>, grid, kBlock, 0, X, n);
  cx.after(-1, (double)sizeof(T) * (double)n * ncomp);
}

template <class T>
void launch_extrapolate_rot(Ctx& cx, Comp3<T> A, Comp3<T> B, Comp3<T> C, long long n, int ncomp,
                            int order) {
  const long long b = std::min<long long>(blocks_for(n), 4LL * cx.sms);
  dim3 grid((unsigned)b, ncomp);
  cx.before(-1);
  launch_k(cx, k_extrapolate_rot<T>, grid, kBlock, 0, A, B, C, n, order);
  // the history words read (A; A, B; A, B, C), the guess written
  cx.after(-1, (double)(order + 2) * (double)sizeof(T) * (double)n * ncomp);
}

template <class T>
void launch_axpy(Ctx& cx, Comp3<T> Y, Comp3<T> X, double a, long long n, int ncomp) {
  const long long b = std::min<long long>(blocks_for(n), 4LL * cx.sms);
  dim3 grid((unsigned)b, ncomp);
  cx.before(-1);
  launch_k(cx, k_axpy<T>, grid, kBlock, 0, Y, X, (T)a, n);
  cx.after(-1, 3.0 * (double)sizeof(T) * (double)n * ncomp);
}

template <class T>
bool launch_coarse_solve(Ctx& cx, const Level& L, Comp3<T> E, Comp3<T> R, int ncomp, int sweeps,
                         double h2) {
  const long long n = L.cells();
  const size_t smem = (size_t)n * 2 * sizeof(T);
  if (smem > 96 * 1024) return false;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_coarse_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(1, ncomp);
  cx.before(VSV_KCLASS_SMOOTH);
  launch_k(cx, k_coarse_solve<T>, grid, 512, smem, L, E, R, sweeps, (T)h2);
  cx.after(VSV_KCLASS_SMOOTH, 2.0 * (double)sizeof(T) * (double)n * ncomp);
  return true;
}

template <class T>
void launch_resid_norm(Ctx& cx, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, bool exact,
                       double* partials, int nblocks, Scalars* S) {
  dim3 grid(nblocks, ncomp);
  float ih_hi = (float)L.inv_h2, ih_lo = (float)(L.inv_h2 - (double)ih_hi);
  cx.before(-1);
  if constexpr (std::is_same<T, float>::value) {
    if (exact)
      launch_k(cx, k_resid_norm<float, true>, grid, kBlock, 0, L, X, R, partials, ih_hi, ih_lo);
    else
      launch_k(cx, k_resid_norm<float, false>, grid, kBlock, 0, L, X, R, partials, ih_hi, ih_lo);
  } else {
    launch_k(cx, k_resid_norm<T, false>, grid, kBlock, 0, L, X, R, partials, ih_hi, ih_lo);
  }
  cx.after(-1);
  cx.before(-1);
  launch_k(cx, k_norm_finalize, ncomp, kBlock, 0, partials, nblocks, S);
  cx.after(-1);
}

void launch_norm_finalize(Ctx& cx, const double* partials, int nblocks, int ncomp, Scalars* S) {
  cx.before(-1);
  launch_k(cx, k_norm_finalize, ncomp, kBlock, 0, partials, nblocks, S);
  cx.after(-1);
}

#define VSV_INST(T)                                                                                \
  template void launch_rb_sweep<T>(Ctx&, const Level&, Comp3<T>, Rhs3<T>, int, int, double, double, \
                                   int);                                                           \
  template void launch_resid_restrict<T>(Ctx&, const Level&, const Level&, Comp3<T>, Rhs3<T>,      \
                                         Comp3<T>, int, bool);                                     \
  template void launch_prolong_add<T>(Ctx&, const Level&, const Level&, Comp3<T>, Comp3<T>, int);  \
  template void launch_zero<T>(Ctx&, Comp3<T>, long long, int);                                    \
  template void launch_axpy<T>(Ctx&, Comp3<T>, Comp3<T>, double, long long, int);                  \
  template void launch_extrapolate_rot<T>(Ctx&, Comp3<T>, Comp3<T>, Comp3<T>, long long, int, int); \
  template bool launch_coarse_vcycle<T>(Ctx&, const CoarseCycle&, Comp3<T>, Comp3<T>, int);        \
  template bool launch_lower_vcycle<T>(Ctx&, const LowerCycle<T>&);                                \
  template bool launch_coarse_solve<T>(Ctx&, const Level&, Comp3<T>, Comp3<T>, int, int, double);  \
  template void launch_resid_norm<T>(Ctx&, const Level&, Comp3<T>, Rhs3<T>, int, bool, double*,    \
                                     int, Scalars*);
VSV_INST(float)
VSV_INST(double)
#undef VSV_INST

}  // namespace vsv
