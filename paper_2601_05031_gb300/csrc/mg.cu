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

// Neighbour values of cell (i,j,k) on level L; Dirichlet ghosts are not
// returned but counted in nwall (their value is -alpha * x_c, zero on the
// fine level).  Returns the number of values written to v.
template <class T>
__device__ __forceinline__ int gather_nb(const T* __restrict__ x, const Level& L, int i, int j,
                                         int k, long long c, T* v, int& nwall) {
  int m = 0;
  nwall = 0;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const long long sy = nx, sz = (long long)nx * ny;
  if (L.act[0]) {
    if (i > 0) v[m++] = x[c - 1]; else if (L.per[0]) v[m++] = x[c + nx - 1]; else ++nwall;
    if (i < nx - 1) v[m++] = x[c + 1]; else if (L.per[0]) v[m++] = x[c - (nx - 1)]; else ++nwall;
  }
  if (L.act[1]) {
    if (j > 0) v[m++] = x[c - sy]; else if (L.per[1]) v[m++] = x[c + (ny - 1) * sy]; else ++nwall;
    if (j < ny - 1) v[m++] = x[c + sy]; else if (L.per[1]) v[m++] = x[c - (ny - 1) * sy]; else ++nwall;
  }
  if (L.act[2]) {
    if (k > 0) v[m++] = x[c - sz]; else if (L.per[2]) v[m++] = x[c + (nz - 1) * sz]; else ++nwall;
    if (k < nz - 1) v[m++] = x[c + sz]; else if (L.per[2]) v[m++] = x[c - (nz - 1) * sz]; else ++nwall;
  }
  return m;
}

template <class T>
__device__ __forceinline__ T rhs_at(const Rhs3<T>& R, int comp, long long c, int j, int k, int ny) {
  T b = R.beta * R.B[comp][c];
  if (R.S[comp]) b += R.S[comp][j + (long long)k * ny];
  return b;
}

__device__ __forceinline__ int n_active(const Level& L) { return L.act[0] + L.act[1] + L.act[2]; }

// ---------------------------------------------------------------- residual value
// r = b - L_h x at one cell, plain arithmetic in T.
template <class T>
__device__ __forceinline__ T resid_plain(const T* __restrict__ x, const Level& L, int i, int j, int k,
                                         long long c, T b) {
  T v[6];
  int nwall;
  int m = gather_nb(x, L, i, j, k, c, v, nwall);
  T s = 0;
  for (int q = 0; q < m; ++q) s += v[q];
  T coef = (T)(2 * n_active(L)) + lv_alpha<T>(L) * (T)nwall;
  return b - (s - coef * x[c]) * lv_ih2<T>(L);
}

// Exact defect in FP32 storage: every term of b - (sum_nb - coef x_c)/h^2 is
// accumulated by cascaded summation, so the result equals the real-number
// defect up to one final rounding (coef is an integer on the fine level).
__device__ __forceinline__ float resid_exact(const float* __restrict__ x, const Level& L, int i,
                                             int j, int k, long long c, float b, float ih_hi,
                                             float ih_lo) {
  float v[6];
  int nwall;
  int m = gather_nb(x, L, i, j, k, c, v, nwall);
  const float coef = (float)(2 * n_active(L)) + L.alphaf * (float)nwall;
  CascadeSum t(0.f);
  for (int q = 0; q < m; ++q) t.add(v[q]);
  t.add_scaled(-coef, x[c]);
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
// One colour of a red-black Gauss-Seidel sweep (omega = 1) or SOR sweep,
// colour = (i + j + k) & 1, in place.  Thread t handles the t-th cell of the
// colour in its x row.
template <class T>
__global__ void k_rb_sweep(Level L, Comp3<T> X, Rhs3<T> R, int color, T omega, T h2) {
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  int i2, j, k, comp;
  if (!cell3((nx + 1) >> 1, ny, nz, i2, j, k, comp)) return;
  T* __restrict__ x = X.p[comp];
  const int i = 2 * i2 + ((j + k + color) & 1);
  if (i >= nx) return;
  const long long c = lin(i, j, k, nx, ny);
  T v[6];
  int nwall;
  const int m = gather_nb(x, L, i, j, k, c, v, nwall);
  T s = 0;
  for (int q = 0; q < m; ++q) s += v[q];
  const T b = rhs_at(R, comp, c, j, k, ny);
  const T gs = (s - b * h2) * lv_rc<T>(L, nwall);
  x[c] = (omega == (T)1) ? gs : x[c] + omega * (gs - x[c]);
}

// Residual of the fine (or any) level, restricted to the next coarser level
// by averaging the children of each coarse cell.
template <class T, bool EXACT>
__global__ void k_resid_restrict(Level F, Level C, Comp3<T> X, Rhs3<T> R, Comp3<T> RC, float ih_hi,
                                 float ih_lo) {
  int I, J, K, comp;
  if (!cell3(C.n[0], C.n[1], C.n[2], I, J, K, comp)) return;
  const T* __restrict__ x = X.p[comp];
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
  RC.p[comp][t] = acc / (T)(fx * fy * fz);
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
  int i, j, k, comp;
  if (!cell3(F.n[0], F.n[1], F.n[2], i, j, k, comp)) return;
  const long long t = lin(i, j, k, F.n[0], F.n[1]);
  const T al = lv_alpha<T>(C);
  const Interp1<T> ax = interp_axis<T>(i, F.n[0] / C.n[0], C.n[0], C.per[0], al);
  const Interp1<T> ay = interp_axis<T>(j, F.n[1] / C.n[1], C.n[1], C.per[1], al);
  const Interp1<T> az = interp_axis<T>(k, F.n[2] / C.n[2], C.n[2], C.per[2], al);
  const T* __restrict__ e = E.p[comp];
  T acc = 0;
  for (int c2 = 0; c2 < 2; ++c2)
    for (int b2 = 0; b2 < 2; ++b2)
      for (int a2 = 0; a2 < 2; ++a2) {
        const T w = ax.w[a2] * ay.w[b2] * az.w[c2];
        if (w != (T)0) acc += w * e[lin(ax.idx[a2], ay.idx[b2], az.idx[c2], C.n[0], C.n[1])];
      }
  X.p[comp][t] += acc;
}

template <class T>
__global__ void k_zero(Comp3<T> X, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) X.p[blockIdx.y][t] = (T)0;
}

// Linear extrapolation in time of the initial guess: x <- 2 x - xp and
// xp <- x (old); with extrapolate = 0 only xp <- x.
template <class T>
__global__ void k_extrapolate(Comp3<T> X, Comp3<T> XP, long long n, int extrapolate) {
  const int comp = blockIdx.y;
  T* __restrict__ x = X.p[comp];
  T* __restrict__ xp = XP.p[comp];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const T a = x[t];
    if (extrapolate) x[t] = (T)2 * a - xp[t];
    xp[t] = a;
  }
}

// Coarsest level: e = 0, then `sweeps` red-black Gauss-Seidel sweeps in
// shared memory by one block per component.
template <class T>
__global__ void k_coarse_solve(Level L, Comp3<T> E, Comp3<T> RR, int sweeps, T h2) {
  extern __shared__ unsigned char smem_raw[];
  T* e = reinterpret_cast<T*>(smem_raw);
  const int comp = blockIdx.y;
  const long long n = L.cells();
  const T* __restrict__ r = RR.p[comp];
  T* rs = e + n;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    e[t] = 0;
    rs[t] = r[t];
  }
  __syncthreads();
  const int nx = L.n[0], ny = L.n[1];
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = (int)(t % nx);
        const long long q = t / nx;
        const int j = (int)(q % ny), k = (int)(q / ny);
        if (((i + j + k) & 1) != color) continue;
        T v[6];
        int nwall;
        const int m = gather_nb(e, L, i, j, k, t, v, nwall);
        T sum = 0;
        for (int q2 = 0; q2 < m; ++q2) sum += v[q2];
        e[t] = (sum - rs[t] * h2) * lv_rc<T>(L, nwall);
      }
      __syncthreads();
    }
  for (long long t = threadIdx.x; t < n; t += blockDim.x) E.p[comp][t] = e[t];
}

// Per-block partial sums of ||b - L x||^2 and ||b||^2 (FP64 accumulation).
template <class T, bool EXACT>
__global__ void k_resid_norm(Level L, Comp3<T> X, Rhs3<T> R, double* partials, float ih_hi,
                             float ih_lo) {
  const int comp = blockIdx.y;
  const T* __restrict__ x = X.p[comp];
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

// ---------------------------------------------------------------- launchers
static inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <class T>
void launch_rb_sweep(Ctx& cx, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, int color,
                     double omega, double h2, int kclass) {
  const dim3 grid = grid3((L.n[0] + 1) / 2, L.n[1], L.n[2], ncomp);
  cx.before(kclass);
  k_rb_sweep<T><<<grid, block3(), 0, cx.stream>>>(L, X, R, color, (T)omega, (T)h2);
  cx.after(kclass);
}

template <class T>
void launch_resid_restrict(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Rhs3<T> R,
                           Comp3<T> RC, int ncomp, bool exact) {
  const dim3 grid = grid3(C.n[0], C.n[1], C.n[2], ncomp);
  cx.before(VSV_KCLASS_RESTRICT);
  float ih_hi = (float)F.inv_h2, ih_lo = (float)(F.inv_h2 - (double)ih_hi);
  if constexpr (std::is_same<T, float>::value) {
    if (exact)
      k_resid_restrict<float, true><<<grid, block3(), 0, cx.stream>>>(F, C, X, R, RC, ih_hi, ih_lo);
    else
      k_resid_restrict<float, false><<<grid, block3(), 0, cx.stream>>>(F, C, X, R, RC, ih_hi, ih_lo);
  } else {
    k_resid_restrict<T, false><<<grid, block3(), 0, cx.stream>>>(F, C, X, R, RC, ih_hi, ih_lo);
  }
  cx.after(VSV_KCLASS_RESTRICT);
}

template <class T>
void launch_prolong_add(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Comp3<T> E, int ncomp) {
  const dim3 grid = grid3(F.n[0], F.n[1], F.n[2], ncomp);
  cx.before(VSV_KCLASS_PROLONG);
  k_prolong_add<T><<<grid, block3(), 0, cx.stream>>>(F, C, X, E);
  cx.after(VSV_KCLASS_PROLONG);
}

template <class T>
void launch_zero(Ctx& cx, Comp3<T> X, long long n, int ncomp) {
  dim3 grid(blocks_for(n), ncomp);
  cx.before(-1);
  k_zero<T><<<grid, kBlock, 0, cx.stream>>>(X, n);
  cx.after(-1);
}

template <class T>
void launch_extrapolate(Ctx& cx, Comp3<T> X, Comp3<T> XP, long long n, int ncomp, int extrapolate) {
  const long long b = std::min<long long>(blocks_for(n), 4 * 152);
  dim3 grid((unsigned)b, ncomp);
  cx.before(-1);
  k_extrapolate<T><<<grid, kBlock, 0, cx.stream>>>(X, XP, n, extrapolate);
  cx.after(-1);
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
  k_coarse_solve<T><<<grid, 512, smem, cx.stream>>>(L, E, R, sweeps, (T)h2);
  cx.after(VSV_KCLASS_SMOOTH);
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
      k_resid_norm<float, true><<<grid, kBlock, 0, cx.stream>>>(L, X, R, partials, ih_hi, ih_lo);
    else
      k_resid_norm<float, false><<<grid, kBlock, 0, cx.stream>>>(L, X, R, partials, ih_hi, ih_lo);
  } else {
    k_resid_norm<T, false><<<grid, kBlock, 0, cx.stream>>>(L, X, R, partials, ih_hi, ih_lo);
  }
  cx.after(-1);
  cx.before(-1);
  k_norm_finalize<<<ncomp, kBlock, 0, cx.stream>>>(partials, nblocks, S);
  cx.after(-1);
}

void launch_norm_finalize(Ctx& cx, const double* partials, int nblocks, int ncomp, Scalars* S) {
  cx.before(-1);
  k_norm_finalize<<<ncomp, kBlock, 0, cx.stream>>>(partials, nblocks, S);
  cx.after(-1);
}

#define VSV_INST(T)                                                                                \
  template void launch_rb_sweep<T>(Ctx&, const Level&, Comp3<T>, Rhs3<T>, int, int, double, double, \
                                   int);                                                           \
  template void launch_resid_restrict<T>(Ctx&, const Level&, const Level&, Comp3<T>, Rhs3<T>,      \
                                         Comp3<T>, int, bool);                                     \
  template void launch_prolong_add<T>(Ctx&, const Level&, const Level&, Comp3<T>, Comp3<T>, int);  \
  template void launch_zero<T>(Ctx&, Comp3<T>, long long, int);                                    \
  template void launch_extrapolate<T>(Ctx&, Comp3<T>, Comp3<T>, long long, int, int);              \
  template bool launch_coarse_solve<T>(Ctx&, const Level&, Comp3<T>, Comp3<T>, int, int, double);  \
  template void launch_resid_norm<T>(Ctx&, const Level&, Comp3<T>, Rhs3<T>, int, bool, double*,    \
                                     int, Scalars*);
VSV_INST(float)
VSV_INST(double)
#undef VSV_INST

}  // namespace vsv
