// Shared device/host definitions of the vorticity--stream-vector library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace vsv {

constexpr int kMaxLevels = 16;
constexpr int kBlock = 256;

// One grid level of a Poisson problem (the fine grid is level 0).
// Dirichlet walls sit on the ghost nodes of the fine grid; on a coarse level
// l the wall lies between the ghost and the first cell, and the ghost value
// is the linear extrapolation through zero at the wall:
//   ghost = -alpha_l * (adjacent cell),  alpha_l = (2^l - 1) / (2^l + 1).
// A level may carry a diagonal shift: the operator is L_h - s (the
// backward-Euler vorticity step of the inertial variant), which adds
// sh2 = s h_l^2 to the diagonal coefficient 2 d + alpha * nwall.
struct Level {
  int n[3];          // nx, ny, nz
  int per[3];        // 1 = periodic axis
  int act[3];        // 0 for a periodic axis of extent 1 (no coupling)
  double alpha;      // Dirichlet closure coefficient (0 on the fine level)
  double inv_h2;     // 1 / h_l^2
  float alphaf;      // the same in FP32 (FP32 kernels never touch FP64 units)
  float inv_h2f;
  double sh2;        // s h_l^2 (0: plain Poisson)
  float sh2f;
  // 1 / (2 d + alpha * nwall + sh2) for nwall = 0..6 wall neighbours: the
  // smoothers multiply by these instead of dividing (same table in every
  // sweep kernel)
  float rcf[7];
  double rcd[7];
  // the diagonal coefficient 2 d + alpha * nwall + sh2 as an FP32 pair
  // (hi + lo) for the exact defect
  float cdh[7], cdl[7];
  __host__ __device__ long long cells() const { return (long long)n[0] * n[1] * n[2]; }
};

template <class T> __host__ __device__ inline T lv_rc(const Level& L, int nwall);
template <> __host__ __device__ inline float lv_rc<float>(const Level& L, int nwall) { return L.rcf[nwall]; }
template <> __host__ __device__ inline double lv_rc<double>(const Level& L, int nwall) { return L.rcd[nwall]; }

template <class T> __host__ __device__ inline T lv_alpha(const Level& L);
template <> __host__ __device__ inline float lv_alpha<float>(const Level& L) { return L.alphaf; }
template <> __host__ __device__ inline double lv_alpha<double>(const Level& L) { return L.alpha; }
template <class T> __host__ __device__ inline T lv_sh2(const Level& L);
template <> __host__ __device__ inline float lv_sh2<float>(const Level& L) { return L.sh2f; }
template <> __host__ __device__ inline double lv_sh2<double>(const Level& L) { return L.sh2; }
template <class T> __host__ __device__ inline T lv_ih2(const Level& L);
template <> __host__ __device__ inline float lv_ih2<float>(const Level& L) { return L.inv_h2f; }
template <> __host__ __device__ inline double lv_ih2<double>(const Level& L) { return L.inv_h2; }

// Up to three components processed by one launch (gridDim.y = component).
template <class T>
struct Comp3 {
  T* p[3];
  // p[c] without a runtime index into the array (a kernel parameter indexed
  // at run time is copied to local memory first)
  __host__ __device__ __forceinline__ T* at(int c) const {
    return c == 0 ? p[0] : (c == 1 ? p[1] : p[2]);
  }
};

// Prolongation increment of one fine cell (cell-centred trilinear, weights
// 3/4 and 1/4 per axis).  The arguments are the (x-centre, x-neighbour) pairs
// of coarse values, already multiplied by their boundary factors, for the
// (centre plane, centre row), (centre plane, neighbour row), (neighbour
// plane, centre row) and (neighbour plane, neighbour row).  Every
// prolongation kernel calls this, so they agree bit for bit.
template <class T>
__device__ __forceinline__ T prolong_value(T aC, T aX, T bC, T bX, T cC, T cX, T dC, T dX) {
  const T w1 = (T)0.75, w2 = (T)0.25;
  T acc = 0;
  acc += w1 * w1 * (w1 * aC + w2 * aX);
  acc += w1 * w2 * (w1 * bC + w2 * bX);
  acc += w2 * w1 * (w1 * cC + w2 * cX);
  acc += w2 * w2 * (w1 * dC + w2 * dX);
  return acc;
}

// Weighted red-black update of one cell (red-black SOR smoothing; an
// over-relaxed smoother contracts a multigrid V-cycle faster):
// x <- x + omega (gs - x) with the Gauss-Seidel value gs = t rc, where
// t = (neighbour sum) - b h^2 and rc = 1 / diagonal, evaluated as
// t (omega rc) + (1 - omega) x in one fused multiply-add.  Every sweep
// kernel forms t with nb_term and updates through relax, with the same
// rounded constants wrc = omega rc and c1 = 1 - omega, so the fused and
// per-colour sweeps agree bit for bit; omega = 1 (c1 = 0, wrc = rc) gives
// the Gauss-Seidel value t rc itself.
template <class T>
__device__ __forceinline__ T nb_term(T s, T b, T h2) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(-b, h2, s);
  else return __fma_rn(-b, h2, s);
}
template <class T>
__device__ __forceinline__ T relax(T x, T t, T wrc, T c1) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(t, wrc, __fmul_rn(c1, x));
  else return __fma_rn(t, wrc, __dmul_rn(c1, x));
}
template <class T>
__device__ __forceinline__ T wscale(T omega, T rc) {
  if constexpr (sizeof(T) == 4) return __fmul_rn(omega, rc);
  else return __dmul_rn(omega, rc);
}

// The GPU's global timer in nanoseconds (bounds of every wait on other
// threads, CTAs or copies).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// First statement of every kernel that launch_k() launches.  Under
// programmatic stream serialisation a kernel can be scheduled while the
// kernel before it in the stream is still running: griddepcontrol.wait
// blocks until every prerequisite grid has completed and its memory
// operations are visible (it returns at once for a plain launch), so nothing
// before it may touch global memory.  launch_dependents then lets the next
// kernel of the stream be scheduled once every CTA of this one has got here;
// its CTAs take SM slots that this kernel's last wave leaves free and wait
// in the same way.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Right-hand side b = beta * B[c] + S[j + k * ny] (S may be null).
template <class T>
struct Rhs3 {
  const T* B[3];
  const T* S[3];
  T beta;
  __host__ __device__ __forceinline__ const T* b_at(int c) const {
    return c == 0 ? B[0] : (c == 1 ? B[1] : B[2]);
  }
  __host__ __device__ __forceinline__ const T* s_at(int c) const {
    return c == 0 ? S[0] : (c == 1 ? S[1] : S[2]);
  }
};

// Device scalars written by reductions and read by later kernels.
struct Scalars {
  double V, A, V0, A0;
  double lambda_v, gamma_a;
  double k_vol, k_area, eps;   // copies of the penalty parameters
  double h3;
  double rnorm2[3], bnorm2[3];
  float lambda_vf, gamma_af;   // FP32 copies read by the FP32 kernels
  int nonfinite;
  int pad;
};

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline long long lin(int i, int j, int k, int nx, int ny) {
  return ((long long)k * ny + j) * nx + i;
}

// Cell-parallel launches use a 3-D grid: x threads along a row, y blocks
// over rows, z blocks over (plane, component) -- no per-cell division.
constexpr int kBX = 64, kBY = 4;
inline dim3 grid3(int nx, int ny, int nz, int ncomp) {
  return dim3((unsigned)((nx + kBX - 1) / kBX), (unsigned)((ny + kBY - 1) / kBY),
              (unsigned)(nz * ncomp));
}
inline dim3 block3() { return dim3(kBX, kBY, 1); }
__device__ __forceinline__ bool cell3(int nx, int ny, int nz, int& i, int& j, int& k, int& comp) {
  i = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  comp = (int)(blockIdx.z / (unsigned)nz);
  k = (int)blockIdx.z - comp * nz;
  return i < nx && j < ny;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-word ("float-float") value hi + lo with |lo| <= ulp(hi) / 2, built
// from the error-free transforms TwoSum (Knuth), Fast2Sum (Dekker) and
// TwoProd by FMA; the sloppy add / multiply of Joldes, Muller and Popescu
// (2017) give a relative error of a few 2^-44.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_from(float a) { return FF{a, 0.f}; }
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  return fast_two_sum(s, __fadd_rn(e, a.lo));
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float ff_round(FF a) { return __fadd_rn(a.hi, a.lo); }

// Cascaded (compensated) summation accumulator, Ogita-Rump-Oishi "Sum2":
// the running sum is kept as hi + lo with every rounding error of hi
// collected in lo.
struct CascadeSum {
  float hi, lo;
  __device__ __forceinline__ CascadeSum(float a) : hi(a), lo(0.f) {}
  __device__ __forceinline__ void add(float t) {
    float s, e;
    two_sum(hi, t, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  // exact product of a float by a small integer constant (error term by FMA)
  __device__ __forceinline__ void add_scaled(float c, float x) {
    float p = __fmul_rn(c, x);
    float pe = __fmaf_rn(c, x, -p);
    add(p);
    lo = __fadd_rn(lo, pe);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

}  // namespace vsv
