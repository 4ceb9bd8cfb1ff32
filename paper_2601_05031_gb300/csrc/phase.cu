// Phase-field kernels: explicit phi update (eq. gen2), chemical potentials
// (eq. 31 Cahn-Hilliard; eq. 30 / SM eq. 35 Helfrich), vorticity source
// (eq. gen1), volume / area reductions (SM eqs. 32, 37-38), velocity
// v = curl psi (eq. vecpot), the observables of the in-plane-shear and
// results sections, and the FP64 base-flow tables of the channel flows
// (boundary-conditions section).
//
// Fields are [nz][ny][nx] without halos.  Scalars (phi, mu, g) use the
// face mirror at walls and wrap on periodic axes; the flow perturbation
// psi' = psi - psi0 is zero on the wall nodes.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace vsv {

__device__ __forceinline__ int mirror_idx(int j, int n) {
  return j < 0 ? -1 - j : (j >= n ? 2 * n - 1 - j : j);
}
__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <class T>
struct ScalarView {  // periodic x, mirror y, mirror / periodic z
  const T* __restrict__ a;
  int nx, ny, nz, zper;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    i = wrap_idx(i, nx);
    j = mirror_idx(j, ny);
    k = zper ? wrap_idx(k, nz) : mirror_idx(k, nz);
    return a[lin(i, j, k, nx, ny)];
  }
};

template <class T>
struct PertView {  // periodic x, zero on the wall nodes
  const T* __restrict__ a;
  int nx, ny, nz, zper;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    i = wrap_idx(i, nx);
    if (zper) k = wrap_idx(k, nz);
    if (j < 0 || j >= ny || k < 0 || k >= nz) return (T)0;
    return a[lin(i, j, k, nx, ny)];
  }
};

template <class T, class V>
__device__ __forceinline__ T lap7(const V& f, int i, int j, int k, T ih2) {
  return (f(i + 1, j, k) + f(i - 1, j, k) + f(i, j + 1, k) + f(i, j - 1, k) + f(i, j, k + 1) +
          f(i, j, k - 1) - (T)6 * f(i, j, k)) * ih2;
}

__device__ __forceinline__ void cell_of(long long t, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(t % nx);
  const long long q = t / nx;
  j = (int)(q % ny);
  k = (int)(q / ny);
}

template <class T> __device__ __forceinline__ T sc_lambda(const Scalars* S);
template <> __device__ __forceinline__ float sc_lambda<float>(const Scalars* S) { return S->lambda_vf; }
template <> __device__ __forceinline__ double sc_lambda<double>(const Scalars* S) { return S->lambda_v; }
template <class T> __device__ __forceinline__ T sc_gamma(const Scalars* S);
template <> __device__ __forceinline__ float sc_gamma<float>(const Scalars* S) { return S->gamma_af; }
template <> __device__ __forceinline__ double sc_gamma<double>(const Scalars* S) { return S->gamma_a; }

static inline unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// ---------------------------------------------------------------- phi update (eq. gen2)
// phi^{n+1} = phi^n + dt [ M (lap mu + lambda_V) - v . grad phi ],
// v = v0(y, z) + curl psi' (central differences).
template <class T>
__global__ void k_phi_update(PhaseParams P, const T* __restrict__ phi, const T* __restrict__ mu,
                             Comp3<T> psi, Comp3<T> v0, Scalars* S, T dt, T* __restrict__ out) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const T ih2 = (T)P.inv_h2, hih = (T)(0.5 * P.inv_h);
  ScalarView<T> M{mu, P.nx, P.ny, P.nz, P.zper};
  ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
  PertView<T> X{psi.p[0], P.nx, P.ny, P.nz, P.zper};
  PertView<T> Y{psi.p[1], P.nx, P.ny, P.nz, P.zper};
  PertView<T> Z{psi.p[2], P.nx, P.ny, P.nz, P.zper};
  const T lmu = lap7<T>(M, i, j, k, ih2);
  const T gx = (F(i + 1, j, k) - F(i - 1, j, k)) * hih;
  const T gy = (F(i, j + 1, k) - F(i, j - 1, k)) * hih;
  const T gz = (F(i, j, k + 1) - F(i, j, k - 1)) * hih;
  const long long jk = j + (long long)k * P.ny;
  const T vx = v0.p[0][jk] + ((Z(i, j + 1, k) - Z(i, j - 1, k)) - (Y(i, j, k + 1) - Y(i, j, k - 1))) * hih;
  const T vy = v0.p[1][jk] + ((X(i, j, k + 1) - X(i, j, k - 1)) - (Z(i + 1, j, k) - Z(i - 1, j, k))) * hih;
  const T vz = v0.p[2][jk] + ((Y(i + 1, j, k) - Y(i - 1, j, k)) - (X(i, j + 1, k) - X(i, j - 1, k))) * hih;
  const T rate = (T)P.mobility * (lmu + sc_lambda<T>(S)) - (vx * gx + vy * gy + vz * gz);
  const T v = phi[t] + dt * rate;
  out[t] = v;
  if (!isfinite(v)) atomicOr(&S->nonfinite, 1);
}

// ---------------------------------------------------------------- reductions (SM eqs. 32, 37)
// Per-block partial sums of sum(phi) and of the area density
// 3/(2 sqrt2) [eps/2 |grad phi|^2 + (phi^2 - 1)^2 / (4 eps)].
template <class T>
__global__ void k_reduce_va(PhaseParams P, const T* __restrict__ phi, const T* __restrict__ phi_lo,
                            double* partials) {
  ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
  const T hih = (T)(0.5 * P.inv_h);
  const T c_a = (T)(3.0 / (2.0 * 1.4142135623730951));
  const T he = (T)(0.5 * P.eps), q = (T)(0.25 / P.eps);
  double sphi = 0.0, sarea = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    // The penalty multipliers use the small differences V - V0 and A - A0,
    // so both sums are formed in double-word arithmetic from phi = hi + lo.
    ScalarView<float> FL{phi_lo, P.nx, P.ny, P.nz, P.zper};
    CascadeSum cp(0.f), ca(0.f);
    // density c_A (eps/2 |grad phi|^2 + (phi^2 - 1)^2 / (4 eps)) from the
    // raw central differences, the constant factors folded into two pairs
    const FF agf{P.ag_hi, P.ag_lo}, awf{P.aw_hi, P.aw_lo};
    for (int row = blockIdx.x; row < P.ny * P.nz; row += gridDim.x) {
     const int j = row % P.ny, k = row / P.ny;
     for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
      const long long t = lin(i, j, k, P.nx, P.ny);
      const FF f{phi[t], phi_lo[t]};
      auto diff = [&](int i1, int j1, int k1, int i0, int j0, int k0) {
        const FF a{F(i1, j1, k1), FL(i1, j1, k1)}, b{F(i0, j0, k0), FL(i0, j0, k0)};
        return ff_add(a, ff_neg(b));
      };
      const FF gx = diff(i + 1, j, k, i - 1, j, k);
      const FF gy = diff(i, j + 1, k, i, j - 1, k);
      const FF gz = diff(i, j, k + 1, i, j, k - 1);
      const FF g2 = ff_add(ff_add(ff_mul(gx, gx), ff_mul(gy, gy)), ff_mul(gz, gz));
      const FF w = ff_add_f(ff_mul(f, f), -1.f);
      const FF dens = ff_add(ff_mul(g2, agf), ff_mul(ff_mul(w, w), awf));
      cp.add(f.hi);
      cp.add(f.lo);
      ca.add(dens.hi);
      ca.add(dens.lo);
     }
    }
    sphi = (double)cp.hi + (double)cp.lo;
    sarea = (double)ca.hi + (double)ca.lo;
  } else {
    for (int row = blockIdx.x; row < P.ny * P.nz; row += gridDim.x) {
     const int j = row % P.ny, k = row / P.ny;
     for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
      const long long t = lin(i, j, k, P.nx, P.ny);
      const double f = phi[t];
      const double gx = (F(i + 1, j, k) - F(i - 1, j, k)) * hih;
      const double gy = (F(i, j + 1, k) - F(i, j - 1, k)) * hih;
      const double gz = (F(i, j, k + 1) - F(i, j, k - 1)) * hih;
      const double w = f * f - 1.0;
      sphi += f;
      sarea += c_a * (he * (gx * gx + gy * gy + gz * gz) + w * w * q);
     }
    }
  }
  sphi = block_sum(sphi);
  sarea = block_sum(sarea);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sphi;
    partials[2 * blockIdx.x + 1] = sarea;
  }
}

// Fixed-order total of the partials; sets V, A and the multipliers
// lambda_V = K_V (V - V0), gamma_A = K_A (A - A0) 3 eps / (2 sqrt 2).
__global__ void k_va_finalize(const double* partials, int nblocks, long long ncells, Scalars* S,
                              int init) {
  pdl_begin();
  double sp = 0.0, sa = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    sp += partials[2 * b];
    sa += partials[2 * b + 1];
  }
  sp = block_sum(sp);
  sa = block_sum(sa);
  if (threadIdx.x == 0) {
    const double V = 0.5 * S->h3 * ((double)ncells - sp);
    const double A = S->h3 * sa;
    S->V = V;
    S->A = A;
    if (init) {
      S->V0 = V;
      S->A0 = A;
    }
    S->lambda_v = S->k_vol * (V - S->V0);
    S->gamma_a = S->k_area * (A - S->A0) * 3.0 * S->eps / (2.0 * 1.4142135623730951);
    S->lambda_vf = (float)S->lambda_v;
    S->gamma_af = (float)S->gamma_a;
  }
}

// ---------------------------------------------------------------- chemical potential
// Helfrich: g = phi^3 - phi - eps^2 lap phi.
template <class T>
__global__ void k_helfrich_g(PhaseParams P, const T* __restrict__ phi, T* __restrict__ g) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
  const T f = phi[t];
  g[t] = f * f * f - f - (T)(P.eps * P.eps) * lap7<T>(F, i, j, k, (T)P.inv_h2);
}

// CH (fe_kind 0): mu = phi^3 - phi - sigma lap phi.
// Helfrich: mu = cf2 [(3 phi^2 - 1) g - eps^2 lap g] - gamma_A lap phi
//           (+ beta_t g with a membrane tension).
template <class T>
__global__ void k_mu(PhaseParams P, const T* __restrict__ phi, const T* __restrict__ g,
                     const Scalars* S, T* __restrict__ mu) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const T ih2 = (T)P.inv_h2;
  ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
  const T f = phi[t];
  const T lphi = lap7<T>(F, i, j, k, ih2);
  if (P.fe_kind == VSV_CAHN_HILLIARD) {
    mu[t] = f * f * f - f - (T)P.sigma * lphi;
  } else {
    ScalarView<T> G{g, P.nx, P.ny, P.nz, P.zper};
    const T lg = lap7<T>(G, i, j, k, ih2);
    T m = (T)P.cf2 * (((T)3 * f * f - (T)1) * g[t] - (T)(P.eps * P.eps) * lg) -
          sc_gamma<T>(S) * lphi;
    if (P.beta_t != 0.0) m += (T)P.beta_t * g[t];
    mu[t] = m;
  }
}

// ---------------------------------------------------------------- vorticity source (eq. gen1)
// f = grad phi x grad mu / eta - s_omega(y, z)   (rhs of lap omega' = f - s_omega)
template <class T>
__global__ void k_source(PhaseParams P, const T* __restrict__ phi, const T* __restrict__ mu,
                         Comp3<T> s_omega, Comp3<T> f) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const T hih = (T)(0.5 * P.inv_h), ie = (T)P.inv_eta;
  ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
  ScalarView<T> M{mu, P.nx, P.ny, P.nz, P.zper};
  const T ax = (F(i + 1, j, k) - F(i - 1, j, k)) * hih;
  const T ay = (F(i, j + 1, k) - F(i, j - 1, k)) * hih;
  const T az = (F(i, j, k + 1) - F(i, j, k - 1)) * hih;
  const T bx = (M(i + 1, j, k) - M(i - 1, j, k)) * hih;
  const T by = (M(i, j + 1, k) - M(i, j - 1, k)) * hih;
  const T bz = (M(i, j, k + 1) - M(i, j, k - 1)) * hih;
  const long long jk = j + (long long)k * P.ny;
  f.p[0][t] = (ay * bz - az * by) * ie - s_omega.p[0][jk];
  f.p[1][t] = (az * bx - ax * bz) * ie - s_omega.p[1][jk];
  f.p[2][t] = (ax * by - ay * bx) * ie - s_omega.p[2][jk];
}

// ---------------------------------------------------------------- velocity (eq. vecpot)
// psi_lo (low words of a double-word psi', mixed path) may be null; the
// difference of the double-word values is formed exactly before rounding.
template <class T>
__global__ void k_velocity(PhaseParams P, Comp3<T> psi, Comp3<T> psi_lo, Comp3<T> v0, Comp3<T> v) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const T hih = (T)(0.5 * P.inv_h);
  PertView<T> X{psi.p[0], P.nx, P.ny, P.nz, P.zper};
  PertView<T> Y{psi.p[1], P.nx, P.ny, P.nz, P.zper};
  PertView<T> Z{psi.p[2], P.nx, P.ny, P.nz, P.zper};
  const long long jk = j + (long long)k * P.ny;
  if (psi_lo.p[0]) {
    PertView<T> XL{psi_lo.p[0], P.nx, P.ny, P.nz, P.zper};
    PertView<T> YL{psi_lo.p[1], P.nx, P.ny, P.nz, P.zper};
    PertView<T> ZL{psi_lo.p[2], P.nx, P.ny, P.nz, P.zper};
    // d(a)/dx with a = hi + lo: (a+ - a-) = (hi+ - hi-) + (lo+ - lo-)
    auto d = [&](const PertView<T>& H, const PertView<T>& L, int i1, int j1, int k1, int i0, int j0,
                 int k0) {
      return ((H(i1, j1, k1) - H(i0, j0, k0)) + (L(i1, j1, k1) - L(i0, j0, k0))) * hih;
    };
    v.p[0][t] = v0.p[0][jk] + (d(Z, ZL, i, j + 1, k, i, j - 1, k) - d(Y, YL, i, j, k + 1, i, j, k - 1));
    v.p[1][t] = v0.p[1][jk] + (d(X, XL, i, j, k + 1, i, j, k - 1) - d(Z, ZL, i + 1, j, k, i - 1, j, k));
    v.p[2][t] = v0.p[2][jk] + (d(Y, YL, i + 1, j, k, i - 1, j, k) - d(X, XL, i, j + 1, k, i, j - 1, k));
    return;
  }
  v.p[0][t] = v0.p[0][jk] + ((Z(i, j + 1, k) - Z(i, j - 1, k)) - (Y(i, j, k + 1) - Y(i, j, k - 1))) * hih;
  v.p[1][t] = v0.p[1][jk] + ((X(i, j, k + 1) - X(i, j, k - 1)) - (Z(i + 1, j, k) - Z(i - 1, j, k))) * hih;
  v.p[2][t] = v0.p[2][jk] + ((Y(i + 1, j, k) - Y(i - 1, j, k)) - (X(i, j + 1, k) - X(i, j - 1, k))) * hih;
}

// Velocity of the mixed path as a double word (hi + lo) for the observables
// and FP64 exports: v = v0 + curl psi' formed in FP64 from the double-word
// stream vector and the FP64 base-flow table, then split into its rounded
// FP32 value and the FP32 rounding of the remainder (about 48 significant
// bits).  Not on the time-stepping path.
__global__ void k_velocity_dw(PhaseParams P, Comp3<float> psi, Comp3<float> psi_lo,
                              Comp3<const double> v0d, Comp3<float> v, Comp3<float> v_lo) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const double hih = 0.5 * P.inv_h;
  PertView<float> X{psi.p[0], P.nx, P.ny, P.nz, P.zper};
  PertView<float> Y{psi.p[1], P.nx, P.ny, P.nz, P.zper};
  PertView<float> Z{psi.p[2], P.nx, P.ny, P.nz, P.zper};
  PertView<float> XL{psi_lo.p[0], P.nx, P.ny, P.nz, P.zper};
  PertView<float> YL{psi_lo.p[1], P.nx, P.ny, P.nz, P.zper};
  PertView<float> ZL{psi_lo.p[2], P.nx, P.ny, P.nz, P.zper};
  auto d = [&](const PertView<float>& H, const PertView<float>& L, int i1, int j1, int k1, int i0,
               int j0, int k0) {
    return (((double)H(i1, j1, k1) + (double)L(i1, j1, k1)) -
            ((double)H(i0, j0, k0) + (double)L(i0, j0, k0))) * hih;
  };
  const long long jk = j + (long long)k * P.ny;
  double w[3];
  w[0] = v0d.p[0][jk] + (d(Z, ZL, i, j + 1, k, i, j - 1, k) - d(Y, YL, i, j, k + 1, i, j, k - 1));
  w[1] = v0d.p[1][jk] + (d(X, XL, i, j, k + 1, i, j, k - 1) - d(Z, ZL, i + 1, j, k, i - 1, j, k));
  w[2] = v0d.p[2][jk] + (d(Y, YL, i + 1, j, k, i - 1, j, k) - d(X, XL, i, j + 1, k, i, j - 1, k));
  for (int c = 0; c < 3; ++c) {
    const float hi = __double2float_rn(w[c]);
    v.at(c)[t] = hi;
    v_lo.at(c)[t] = __double2float_rn(w[c] - (double)hi);
  }
}

// ---------------------------------------------------------------- observables
// Velocity (materialised; lo: the low words of a double-word velocity, or
// null) with the no-slip wall velocity on the wall nodes.
template <class T>
struct VelView {
  const T* __restrict__ a;
  const T* __restrict__ lo;
  int nx, ny, nz, zper, comp;
  const PhaseParams* P;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    i = wrap_idx(i, nx);
    if (zper) k = wrap_idx(k, nz);
    if (j < 0) return P->vwall[0][comp];
    if (j >= ny) return P->vwall[1][comp];
    if (k < 0) return P->vwall[2][comp];
    if (k >= nz) return P->vwall[3][comp];
    const long long t = lin(i, j, k, nx, ny);
    return lo ? (double)a[t] + (double)lo[t] : (double)a[t];
  }
};

// A double-word perturbation field (hi + lo; lo may be null) read in FP64,
// zero on the wall nodes.
template <class T>
struct PertView2 {
  PertView<T> hi, lo;
  bool has_lo;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    return has_lo ? (double)hi(i, j, k) + (double)lo(i, j, k) : (double)hi(i, j, k);
  }
};

// Base-flow velocity table (x-invariant) with the same wall values.
struct V0View {
  const double* a;
  int ny, nz, zper, comp;
  const PhaseParams* P;
  __device__ __forceinline__ double operator()(int j, int k) const {
    if (zper) k = wrap_idx(k, nz);
    if (j < 0) return P->vwall[0][comp];
    if (j >= ny) return P->vwall[1][comp];
    if (k < 0) return P->vwall[2][comp];
    if (k >= nz) return P->vwall[3][comp];
    return a[j + (long long)k * ny];
  }
};

// q: 0 dissipation integrand, 1 body-free dissipation integrand, 2 |omega'|^2,
// 3 |psi'|^2, 4 w = (1-phi)/2, 5..7 w x, w y, w z, 8 energy density,
// 9 max |div v|, 10 max |div psi|, 11 max sigma_t, 12 (Helfrich with a
// membrane tension) the face-difference area density over c_A / eps.
// vel_lo, om_lo, ps_lo: low words of double-word velocity, omega' and psi'
// (mixed path), or null pointers.
template <class T>
__global__ void k_diag(PhaseParams P, const T* __restrict__ phi, const T* __restrict__ phi_lo,
                       const T* __restrict__ g, const T* __restrict__ g_lo, Comp3<T> vel,
                       Comp3<T> vel_lo, Comp3<T> omega, Comp3<T> om_lo, Comp3<T> psi,
                       Comp3<T> ps_lo, Comp3<const double> psi0r, Comp3<const double> v0d,
                       T* sigma_t, double* partials) {
  double q[kDiagQ];
  for (int a = 0; a < kDiagQ; ++a) q[a] = 0.0;
  const double hih = 0.5 * P.inv_h, eta = 1.0 / P.inv_eta, h = P.h;
  const int ny2 = P.ny + 2;
  for (int row = blockIdx.x; row < P.ny * P.nz; row += gridDim.x) {
   const int j = row % P.ny, k = row / P.ny;
   for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
    const long long t = lin(i, j, k, P.nx, P.ny);
    double G[3][3], G0[3][3];
    for (int c = 0; c < 3; ++c) {
      VelView<T> V{vel.p[c], vel_lo.p[c], P.nx, P.ny, P.nz, P.zper, c, &P};
      G[c][0] = (V(i + 1, j, k) - V(i - 1, j, k)) * hih;
      G[c][1] = (V(i, j + 1, k) - V(i, j - 1, k)) * hih;
      G[c][2] = (V(i, j, k + 1) - V(i, j, k - 1)) * hih;
      V0View W{v0d.p[c], P.ny, P.nz, P.zper, c, &P};
      G0[c][0] = 0.0;
      G0[c][1] = (W(j + 1, k) - W(j - 1, k)) * hih;
      G0[c][2] = (W(j, k + 1) - W(j, k - 1)) * hih;
    }
    double d = 0.0, d0 = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double e = G[a][b] + G[b][a], e0 = G0[a][b] + G0[b][a];
        d += e * e;
        d0 += e0 * e0;
      }
    q[0] += d;
    q[1] += d0;
    double o2 = 0.0, p2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double o = (double)omega.p[c][t] + (om_lo.p[c] ? (double)om_lo.p[c][t] : 0.0);
      const double p = (double)psi.p[c][t] + (ps_lo.p[c] ? (double)ps_lo.p[c][t] : 0.0);
      o2 += o * o;
      p2 += p * p;
    }
    q[2] += o2;
    q[3] += p2;
    const double f = (double)phi[t] + (phi_lo ? (double)phi_lo[t] : 0.0);
    const double w = 0.5 * (1.0 - f);
    q[4] += w;
    q[5] += w * (i + 0.5) * h;
    q[6] += w * (j + 1.0) * h;
    q[7] += w * (P.zper ? (k + 0.5) : (k + 1.0)) * h;
    if (P.fe_kind == VSV_HELFRICH) {
      const double gg = (double)g[t] + (g_lo ? (double)g_lo[t] : 0.0);
      q[8] += gg * gg;
      if (P.beta_t != 0.0) {   // membrane tension: the face-difference area density
        ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
        ScalarView<T> FL{phi_lo ? phi_lo : phi, P.nx, P.ny, P.nz, P.zper};
        auto val = [&](int ii, int jj, int kk) {
          return (double)F(ii, jj, kk) + (phi_lo ? (double)FL(ii, jj, kk) : 0.0);
        };
        const double dx = (val(i + 1, j, k) - f) * P.inv_h;
        double faces = dx * dx;
        if (j + 1 < P.ny) {
          const double dy = (val(i, j + 1, k) - f) * P.inv_h;
          faces += dy * dy;
        }
        if (P.zper || k + 1 < P.nz) {
          const double dz = (val(i, j, k + 1) - f) * P.inv_h;
          faces += dz * dz;
        }
        q[12] += 0.25 * (f * f - 1.0) * (f * f - 1.0) + 0.5 * P.eps * P.eps * faces;
      }
    } else {
      ScalarView<T> F{phi, P.nx, P.ny, P.nz, P.zper};
      double e = 0.25 * (f * f - 1.0) * (f * f - 1.0);
      const double dx = ((double)F(i + 1, j, k) - f) * P.inv_h;
      double faces = dx * dx;
      if (j + 1 < P.ny) {
        const double dy = ((double)F(i, j + 1, k) - f) * P.inv_h;
        faces += dy * dy;
      }
      if (P.zper || k + 1 < P.nz) {
        const double dz = ((double)F(i, j, k + 1) - f) * P.inv_h;
        faces += dz * dz;
      }
      q[8] += e + 0.5 * P.sigma * faces;
    }
    q[9] = fmax(q[9], fabs(G[0][0] + G[1][1] + G[2][2]));
    // div psi with psi = psi0(y, z) + psi'; psi0 ring table holds the wall data
    const bool pl = ps_lo.p[0] != nullptr;
    PertView2<T> PX{{psi.p[0], P.nx, P.ny, P.nz, P.zper}, {pl ? ps_lo.p[0] : psi.p[0], P.nx, P.ny, P.nz, P.zper}, pl};
    PertView2<T> PY{{psi.p[1], P.nx, P.ny, P.nz, P.zper}, {pl ? ps_lo.p[1] : psi.p[1], P.nx, P.ny, P.nz, P.zper}, pl};
    PertView2<T> PZ{{psi.p[2], P.nx, P.ny, P.nz, P.zper}, {pl ? ps_lo.p[2] : psi.p[2], P.nx, P.ny, P.nz, P.zper}, pl};
    auto r0 = [&](int c, int jj, int kk) -> double {
      if (P.zper) kk = wrap_idx(kk, P.nz);
      return psi0r.p[c][(jj + 1) + (long long)(kk + 1) * ny2];
    };
    const double dpx = (PX(i + 1, j, k) - PX(i - 1, j, k)) * hih;
    const double dpy = (PY(i, j + 1, k) - PY(i, j - 1, k) + r0(1, j + 1, k) -
                        r0(1, j - 1, k)) * hih;
    const double dpz = (PZ(i, j, k + 1) - PZ(i, j, k - 1) + r0(2, j, k + 1) -
                        r0(2, j, k - 1)) * hih;
    q[10] = fmax(q[10], fabs(dpx + dpy + dpz));
    const double sxy = eta * (G[0][1] + G[1][0]);
    const double syz = eta * (G[1][2] + G[2][1]);
    const double sxz = eta * (G[0][2] + G[2][0]);
    const double st = sqrt(sxy * sxy + syz * syz + sxz * sxz);
    q[11] = fmax(q[11], st);
    if (sigma_t) sigma_t[t] = (T)st;
   }
  }
  for (int a = 0; a < 9; ++a) {
    const double s = block_sum(q[a]);
    if (threadIdx.x == 0) partials[(long long)blockIdx.x * kDiagQ + a] = s;
  }
  for (int a = 9; a < 12; ++a) {
    const double s = block_max(q[a]);
    if (threadIdx.x == 0) partials[(long long)blockIdx.x * kDiagQ + a] = s;
  }
  {
    const double s = block_sum(q[12]);
    if (threadIdx.x == 0) partials[(long long)blockIdx.x * kDiagQ + 12] = s;
  }
}

__global__ void k_diag_finalize(const double* partials, int nblocks, double* out) {
  for (int a = 0; a < 13; ++a) {   // 0..8 and 12 are sums, 9..11 maxima
    const bool sum = a < 9 || a == 12;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double v = partials[(long long)b * kDiagQ + a];
      s = sum ? s + v : fmax(s, v);
    }
    s = sum ? block_sum(s) : block_max(s);
    if (threadIdx.x == 0) out[a] = s;
  }
}

// <sigma_xy>(y): one block per y row, fixed-order sum over x and z.
template <class T>
__global__ void k_stress_profile(PhaseParams P, Comp3<T> vel, Comp3<T> vel_lo, double* out) {
  const int j = blockIdx.x;
  const double hih = 0.5 * P.inv_h, eta = 1.0 / P.inv_eta;
  VelView<T> VX{vel.p[0], vel_lo.p[0], P.nx, P.ny, P.nz, P.zper, 0, &P};
  VelView<T> VY{vel.p[1], vel_lo.p[1], P.nx, P.ny, P.nz, P.zper, 1, &P};
  double s = 0.0;
  const long long m = (long long)P.nx * P.nz;
  for (long long t = threadIdx.x; t < m; t += blockDim.x) {
    const int i = (int)(t % P.nx), k = (int)(t / P.nx);
    const double dvx_dy = (VX(i, j + 1, k) - VX(i, j - 1, k)) * hih;
    const double dvy_dx = (VY(i + 1, j, k) - VY(i - 1, j, k)) * hih;
    s += eta * (dvx_dy + dvy_dx);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s / (double)m;
}

// ---------------------------------------------------------------- small utilities
template <class Tin, class Tout>
__global__ void k_convert(const Tin* __restrict__ in, Tout* __restrict__ out, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (Tout)in[t];
}

// out = pert + table(y, z); ring = 1: table in ring layout ((ny+2) x (nz+2)).
template <class T>
__global__ void k_full_field(PhaseParams P, const T* __restrict__ pert, const T* __restrict__ lo,
                             const double* __restrict__ tab, int ring, T* __restrict__ out) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const double b = ring ? tab[(j + 1) + (long long)(k + 1) * (P.ny + 2)] : tab[j + (long long)k * P.ny];
  out[t] = (T)((double)pert[t] + (lo ? (double)lo[t] : 0.0) + b);
}

// Full field in FP64 from a double-word perturbation: out = hi + lo + table.
__global__ void k_full_field_dw(PhaseParams P, const float* __restrict__ hi, const float* __restrict__ lo,
                                const double* __restrict__ tab, int ring, double* __restrict__ out) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const double b = tab ? (ring ? tab[(j + 1) + (long long)(k + 1) * (P.ny + 2)] : tab[j + (long long)k * P.ny]) : 0.0;
  out[t] = (double)hi[t] + (double)lo[t] + b;
}

void launch_full_field_dw(Ctx& cx, const PhaseParams& P, const float* hi, const float* lo,
                          const double* tab, int ring, double* out) {
  cx.before(-1);
  k_full_field_dw<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, hi, lo, tab, ring, out);
  cx.after(-1);
}

template <class T>
__global__ void k_scale_copy(const T* __restrict__ in, T* __restrict__ out, long long n, T a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = a * in[t];
}

// ---------------------------------------------------------------- time-dependent walls
// One thread: the device time of the wall data, advanced by one step (or
// set), so that a captured graph of steps carries the time with it.
__global__ void k_wall_time(double* t_dev, double dt, int set_time, double t_set) {
  *t_dev = set_time ? t_set : *t_dev + dt;
}

__device__ __forceinline__ double wall_speed(const WallTables& W, int w, double t) {
  return W.s0[w] + W.ramp[w] * t + W.amp[w] * sin(2.0 * 3.14159265358979323846 * W.freq[w] * t +
                                                  W.phase[w]);
}

// Current tables = s_0(t) B_0 + s_1(t) B_1, every table and component in
// one grid-stride loop over a flat index.
template <class T>
__global__ void k_wall_tables(const __grid_constant__ WallTables W) {
  const double t = *W.t_dev;
  const double a = wall_speed(W, 0, t), b = wall_speed(W, 1, t);
  const long long nr = W.n_ring, nt = W.n_tab;
  const long long total = 3 * (2 * nr + 3 * nt);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int c = (int)(r / (2 * nr + 3 * nt));
    r -= c * (2 * nr + 3 * nt);
    if (r < nr) {
      W.om[c][r] = a * W.bom[0][c][r] + b * W.bom[1][c][r];
    } else if ((r -= nr) < nr) {
      W.ps[c][r] = a * W.bps[0][c][r] + b * W.bps[1][c][r];
    } else if ((r -= nr) < nt) {
      const double v = a * W.bv0[0][c][r] + b * W.bv0[1][c][r];
      W.v0[c][r] = v;
      ((T*)W.v0t[c])[r] = (T)v;
    } else if ((r -= nt) < nt) {
      const double v = a * W.bsom[0][c][r] + b * W.bsom[1][c][r];
      W.som[c][r] = v;
      ((T*)W.somt[c])[r] = (T)v;
    } else {
      r -= nt;
      const double v = a * W.bsps[0][c][r] + b * W.bsps[1][c][r];
      W.sps[c][r] = v;
      ((T*)W.spsnt[c])[r] = (T)(-v);
    }
  }
}

template <class T>
void launch_wall_tables(Ctx& cx, const WallTables& W, double dt, bool set_time, double t_set) {
  cx.before(-1);
  k_wall_time<<<1, 1, 0, cx.stream>>>(W.t_dev, dt, set_time ? 1 : 0, t_set);
  cx.after(-1);
  const long long total = 3LL * (2LL * W.n_ring + 3LL * W.n_tab);
  const unsigned blocks = (unsigned)std::min<long long>((total + kBlock - 1) / kBlock, 4LL * cx.sms);
  cx.before(-1);
  k_wall_tables<T><<<blocks, kBlock, 0, cx.stream>>>(W);
  cx.after(-1, 8.0 * (double)total * 3.0);
}
template void launch_wall_tables<float>(Ctx&, const WallTables&, double, bool, double);
template void launch_wall_tables<double>(Ctx&, const WallTables&, double, bool, double);

// ---------------------------------------------------------------- base-flow tables (FP64)
// Ring layout: entry (j, k), j in [-1, ny], k in [-1, nz], at (j+1) + (k+1)(ny+2).
__device__ __forceinline__ long long ring_at(int j, int k, int ny) {
  return (j + 1) + (long long)(k + 1) * (ny + 2);
}

// Duct wall data from u0 and chi (interior layout j + k ny): normal
// derivative on a wall node by (4 f_1 - f_2) / (2h) (f = 0 on the wall),
// tangential derivatives zero.
__global__ void k_duct_ring(int ny, int nz, double h, const double* u0, const double* chi,
                            double* omy, double* omz, double* psy, double* psz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double ih = 1.0 / (2.0 * h);
  if (t < nz) {  // y walls at row k = t
    const int k = t;
    const double* u = u0 + (long long)k * ny;
    const double* c = chi + (long long)k * ny;
    const double du_lo = (4.0 * u[0] - u[1]) * ih, du_hi = -(4.0 * u[ny - 1] - u[ny - 2]) * ih;
    const double dc_lo = (4.0 * c[0] - c[1]) * ih, dc_hi = -(4.0 * c[ny - 1] - c[ny - 2]) * ih;
    omz[ring_at(-1, k, ny)] = -du_lo;
    omz[ring_at(ny, k, ny)] = -du_hi;
    psz[ring_at(-1, k, ny)] = dc_lo;
    psz[ring_at(ny, k, ny)] = dc_hi;
    omy[ring_at(-1, k, ny)] = 0.0;
    omy[ring_at(ny, k, ny)] = 0.0;
    psy[ring_at(-1, k, ny)] = 0.0;
    psy[ring_at(ny, k, ny)] = 0.0;
  }
  if (t < ny) {  // z walls at column j = t
    const int j = t;
    const double el = (4.0 * u0[j] - u0[j + ny]) * ih;
    const double eh = -(4.0 * u0[j + (long long)(nz - 1) * ny] - u0[j + (long long)(nz - 2) * ny]) * ih;
    const double cl = (4.0 * chi[j] - chi[j + ny]) * ih;
    const double ch = -(4.0 * chi[j + (long long)(nz - 1) * ny] - chi[j + (long long)(nz - 2) * ny]) * ih;
    omy[ring_at(j, -1, ny)] = el;
    omy[ring_at(j, nz, ny)] = eh;
    psy[ring_at(j, -1, ny)] = -cl;
    psy[ring_at(j, nz, ny)] = -ch;
    omz[ring_at(j, -1, ny)] = 0.0;
    omz[ring_at(j, nz, ny)] = 0.0;
    psz[ring_at(j, -1, ny)] = 0.0;
    psz[ring_at(j, nz, ny)] = 0.0;
  }
}

// out = scale * in - (wall-node contribution of `ring` to the 2-D
// Laplacian), both walls in y and z (the duct section).
__global__ void k_ring_rhs(int ny, int nz, double h, const double* ring, double scale,
                           const double* in, double* out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ny * nz) return;
  const int j = (int)(t % ny), k = (int)(t / ny);
  double b = 0.0;
  if (j == 0) b += ring[ring_at(-1, k, ny)];
  if (j == ny - 1) b += ring[ring_at(ny, k, ny)];
  if (k == 0) b += ring[ring_at(j, -1, ny)];
  if (k == nz - 1) b += ring[ring_at(j, nz, ny)];
  out[t] = (in ? scale * in[t] : 0.0) - b / (h * h);
}

__global__ void k_ring_fill(int ny, int nz, const double* interior, double* ring) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ny * nz) return;
  const int j = (int)(t % ny), k = (int)(t / ny);
  ring[ring_at(j, k, ny)] = interior[t];
}

// v0 = curl psi0 (x-invariant), s_omega = lap omega0, s_psi = lap psi0 + omega0,
// all on the interior (y, z) cells from ring tables.
__global__ void k_base_derived(int ny, int nz, int zper, double h, Comp3<const double> om,
                               Comp3<const double> ps, Comp3<double> v0, Comp3<double> som,
                               Comp3<double> sps) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ny * nz) return;
  const int j = (int)(t % ny), k = (int)(t / ny);
  auto at = [&](const double* r, int jj, int kk) -> double {
    if (zper) kk = wrap_idx(kk, nz);
    return r[ring_at(jj, kk, ny)];
  };
  const double hih = 0.5 / h, ih2 = 1.0 / (h * h);
  const double* px = ps.p[0];
  const double* py = ps.p[1];
  const double* pz = ps.p[2];
  v0.p[0][t] = ((at(pz, j + 1, k) - at(pz, j - 1, k)) - (at(py, j, k + 1) - at(py, j, k - 1))) * hih;
  v0.p[1][t] = (at(px, j, k + 1) - at(px, j, k - 1)) * hih;
  v0.p[2][t] = -(at(px, j + 1, k) - at(px, j - 1, k)) * hih;
  for (int c = 0; c < 3; ++c) {
    const double* o = om.p[c];
    const double* p = ps.p[c];
    const double lo = (at(o, j + 1, k) + at(o, j - 1, k) + at(o, j, k + 1) + at(o, j, k - 1) -
                       4.0 * at(o, j, k)) * ih2;
    const double lp = (at(p, j + 1, k) + at(p, j - 1, k) + at(p, j, k + 1) + at(p, j, k - 1) -
                       4.0 * at(p, j, k)) * ih2;
    som.p[c][t] = lo;
    sps.p[c][t] = lp + at(o, j, k);
  }
}

__global__ void k_max_abs(const double* x, long long n, double* out) {
  double m = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) m = fmax(m, fabs(x[t]));
  m = block_max(m);
  if (threadIdx.x == 0) *out = m;
}

__global__ void k_fill(double* x, long long n, double v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = v;
}

// ---------------------------------------------------------------- mixed path: double-word phi
// Unscaled 7-point Laplacian sum (x+ + x- + y+ + y- + z+ + z- - 6 c) of a
// double-word field: the hi parts are summed by cascaded summation
// (error-free up to the final rounding), the lo parts in FP32 (their own
// rounding is below 2^-48 of the field).  Callers apply 1/h^2 together with
// their own coefficient, as one double-word product.
template <class V>
__device__ __forceinline__ FF lap7_ff(const V& H, const V& L, int i, int j, int k) {
  CascadeSum s(H(i + 1, j, k));
  s.add(H(i - 1, j, k));
  s.add(H(i, j + 1, k));
  s.add(H(i, j - 1, k));
  s.add(H(i, j, k + 1));
  s.add(H(i, j, k - 1));
  s.add_scaled(-6.f, H(i, j, k));
  const float lsum = L(i + 1, j, k) + L(i - 1, j, k) + L(i, j + 1, k) + L(i, j - 1, k) +
                     L(i, j, k + 1) + L(i, j, k - 1) - 6.f * L(i, j, k);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, lsum));
}

// phi^{n+1} = phi^n + dt * rate with phi^n = hi + lo; the rate itself is an
// O(1e-4) increment and is formed in FP32 as in the FP64 path.
__global__ void k_phi_update_ff(PhaseParams P, const float* __restrict__ phi,
                                const float* __restrict__ phi_lo, const float* __restrict__ mu,
                                Comp3<float> psi, Comp3<float> v0, Scalars* S, float dt,
                                float* __restrict__ out, float* __restrict__ out_lo) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  const float ih2 = (float)P.inv_h2, hih = (float)(0.5 * P.inv_h);
  ScalarView<float> M{mu, P.nx, P.ny, P.nz, P.zper};
  ScalarView<float> F{phi, P.nx, P.ny, P.nz, P.zper};
  PertView<float> X{psi.p[0], P.nx, P.ny, P.nz, P.zper};
  PertView<float> Y{psi.p[1], P.nx, P.ny, P.nz, P.zper};
  PertView<float> Z{psi.p[2], P.nx, P.ny, P.nz, P.zper};
  const float lmu = lap7<float>(M, i, j, k, ih2);
  const float gx = (F(i + 1, j, k) - F(i - 1, j, k)) * hih;
  const float gy = (F(i, j + 1, k) - F(i, j - 1, k)) * hih;
  const float gz = (F(i, j, k + 1) - F(i, j, k - 1)) * hih;
  const long long jk = j + (long long)k * P.ny;
  const float vx = v0.p[0][jk] + ((Z(i, j + 1, k) - Z(i, j - 1, k)) - (Y(i, j, k + 1) - Y(i, j, k - 1))) * hih;
  const float vy = v0.p[1][jk] + ((X(i, j, k + 1) - X(i, j, k - 1)) - (Z(i + 1, j, k) - Z(i - 1, j, k))) * hih;
  const float vz = v0.p[2][jk] + ((Y(i + 1, j, k) - Y(i - 1, j, k)) - (X(i, j + 1, k) - X(i, j - 1, k))) * hih;
  const float rate = (float)P.mobility * (lmu + S->lambda_vf) - (vx * gx + vy * gy + vz * gz);
  const FF v = ff_add_f(FF{phi[t], phi_lo[t]}, dt * rate);
  out[t] = v.hi;
  out_lo[t] = v.lo;
  if (!isfinite(v.hi)) atomicOr(&S->nonfinite, 1);
}

// g = phi^3 - phi - eps^2 lap phi in double-word arithmetic.
__global__ void k_helfrich_g_ff(PhaseParams P, const float* __restrict__ phi,
                                const float* __restrict__ phi_lo, float* __restrict__ g,
                                float* __restrict__ g_lo) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  ScalarView<float> H{phi, P.nx, P.ny, P.nz, P.zper};
  ScalarView<float> L{phi_lo, P.nx, P.ny, P.nz, P.zper};
  const FF f{phi[t], phi_lo[t]};
  const FF lphi = lap7_ff(H, L, i, j, k);
  const FF cubic = ff_mul(f, ff_add_f(ff_mul(f, f), -1.f));
  const FF r = ff_add(cubic, ff_neg(ff_mul(lphi, FF{P.e2ih_hi, P.e2ih_lo})));
  g[t] = r.hi;
  g_lo[t] = r.lo;
}

// CH:       mu = phi^3 - phi - sigma lap phi
// Helfrich: mu = cf2 [(3 phi^2 - 1) g - eps^2 lap g] - gamma_A lap phi (+ beta_t g)
__global__ void k_mu_ff(PhaseParams P, const float* __restrict__ phi, const float* __restrict__ phi_lo,
                        const float* __restrict__ g, const float* __restrict__ g_lo,
                        const Scalars* S, float* __restrict__ mu, float* __restrict__ mu_lo) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  ScalarView<float> H{phi, P.nx, P.ny, P.nz, P.zper};
  ScalarView<float> L{phi_lo, P.nx, P.ny, P.nz, P.zper};
  const FF f{phi[t], phi_lo[t]};
  const FF lphi = lap7_ff(H, L, i, j, k);
  if (P.fe_kind == VSV_CAHN_HILLIARD) {
    const FF cubic = ff_mul(f, ff_add_f(ff_mul(f, f), -1.f));
    const FF m = ff_add(cubic, ff_neg(ff_mul(lphi, FF{P.sgih_hi, P.sgih_lo})));
    mu[t] = m.hi;
    mu_lo[t] = m.lo;
    return;
  }
  ScalarView<float> GH{g, P.nx, P.ny, P.nz, P.zper};
  ScalarView<float> GL{g_lo, P.nx, P.ny, P.nz, P.zper};
  const FF gg{g[t], g_lo[t]};
  const FF lg = lap7_ff(GH, GL, i, j, k);
  const FF w = ff_add_f(ff_mul_f(ff_mul(f, f), 3.f), -1.f);
  const FF inner = ff_add(ff_mul(w, gg), ff_neg(ff_mul(lg, FF{P.e2ih_hi, P.e2ih_lo})));
  const FF gih = ff_mul_f(FF{P.ih2_hi, P.ih2_lo}, S->gamma_af);   // gamma_A / h^2
  FF m = ff_add(ff_mul(inner, FF{P.cf2_hi, P.cf2_lo}), ff_neg(ff_mul(lphi, gih)));
  if (P.bt_hi != 0.f) m = ff_add(m, ff_mul(gg, FF{P.bt_hi, P.bt_lo}));
  mu[t] = m.hi;
  mu_lo[t] = m.lo;
}

__global__ void k_split_ff(const double* __restrict__ in, float* __restrict__ hi,
                           float* __restrict__ lo, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double d = in[t];
  const float h = (float)d;
  hi[t] = h;
  lo[t] = (float)(d - (double)h);
}

__global__ void k_merge_ff(const float* __restrict__ hi, const float* __restrict__ lo,
                           double* __restrict__ out, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (double)hi[t] + (double)lo[t];
}

// The same splits and merges four elements per thread with 16-byte accesses
// (every array 16-byte aligned), grid-strided; the last n % 4 elements are
// done one per thread.  Used for device buffers and for mapped host memory,
// where fewer, wider requests cross the host link.
__global__ void k_split_ff_v4(const double* __restrict__ in, float* __restrict__ hi,
                              float* __restrict__ lo, long long n) {
  const long long n4 = n >> 2, stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double2* in2 = reinterpret_cast<const double2*>(in);
  for (long long t = t0; t < n4; t += stride) {
    const double2 a = in2[2 * t], b = in2[2 * t + 1];
    const float4 h = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    const float4 l = make_float4((float)(a.x - (double)h.x), (float)(a.y - (double)h.y),
                                 (float)(b.x - (double)h.z), (float)(b.y - (double)h.w));
    reinterpret_cast<float4*>(hi)[t] = h;
    reinterpret_cast<float4*>(lo)[t] = l;
  }
  const long long r = 4 * n4 + t0;
  if (r < n) {
    const double d = in[r];
    const float h = (float)d;
    hi[r] = h;
    lo[r] = (float)(d - (double)h);
  }
}

__global__ void k_merge_ff_v4(const float* __restrict__ hi, const float* __restrict__ lo,
                              double* __restrict__ out, long long n) {
  const long long n4 = n >> 2, stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double2* out2 = reinterpret_cast<double2*>(out);
  for (long long t = t0; t < n4; t += stride) {
    const float4 h = reinterpret_cast<const float4*>(hi)[t];
    const float4 l = reinterpret_cast<const float4*>(lo)[t];
    out2[2 * t] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    out2[2 * t + 1] = make_double2((double)h.z + (double)l.z, (double)h.w + (double)l.w);
  }
  const long long r = 4 * n4 + t0;
  if (r < n) out[r] = (double)hi[r] + (double)lo[r];
}

// ---------------------------------------------------------------- 4-cell kernels
// The same double-word kernels with one thread per 4 consecutive x cells
// (nx a multiple of 4): the own cells and the y / z neighbours are 16-byte
// loads, the x neighbours two scalars, and the boundary index arithmetic is
// done once per row instead of once per access.  Per-cell arithmetic is that
// of the 1-cell kernels above, term for term.
namespace {

// A field around the 4 cells (i0 .. i0+3, j, k): own values c, the rows
// above / below (ym, yp), the planes below / above (zm, zp) and the x
// neighbours xl (i0 - 1) and xr (i0 + 4).
struct St4 {
  float4 c, ym, yp, zm, zp;
  float xl, xr;
};

__device__ __forceinline__ float e4(const float4& v, int o) {
  return o == 0 ? v.x : (o == 1 ? v.y : (o == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 ld4g(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Row offsets of the 4-cell group's neighbourhood, with the boundary rule of
// scalars (mirror at walls) or of the flow perturbation (zero beyond walls,
// flagged by a negative offset); x wraps in both.
struct Geo4 {
  long long rc, rym, ryp, rzm, rzp;   // row offsets (plane * ny + row) * nx
  int il, ir;                          // x indices of the two x neighbours
  int i0;
};

__device__ __forceinline__ Geo4 geo4(const PhaseParams& P, int i0, int j, int k, bool pert) {
  Geo4 G;
  const long long nx = P.nx, ny = P.ny;
  auto row = [&](int jj, int kk) { return ((long long)kk * ny + jj) * nx; };
  G.i0 = i0;
  G.il = i0 == 0 ? P.nx - 1 : i0 - 1;
  G.ir = i0 + 4 == P.nx ? 0 : i0 + 4;
  G.rc = row(j, k);
  if (pert) {
    G.rym = j > 0 ? row(j - 1, k) : -1;
    G.ryp = j < P.ny - 1 ? row(j + 1, k) : -1;
    const int km = P.zper ? wrap_idx(k - 1, P.nz) : k - 1;
    const int kp = P.zper ? wrap_idx(k + 1, P.nz) : k + 1;
    G.rzm = km >= 0 ? row(j, km) : -1;
    G.rzp = kp < P.nz ? row(j, kp) : -1;
  } else {
    G.rym = row(mirror_idx(j - 1, P.ny), k);
    G.ryp = row(mirror_idx(j + 1, P.ny), k);
    G.rzm = row(j, P.zper ? wrap_idx(k - 1, P.nz) : mirror_idx(k - 1, P.nz));
    G.rzp = row(j, P.zper ? wrap_idx(k + 1, P.nz) : mirror_idx(k + 1, P.nz));
  }
  return G;
}

__device__ __forceinline__ St4 load4(const float* __restrict__ a, const Geo4& G) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  St4 S;
  S.c = ld4g(a + G.rc + G.i0);
  S.ym = G.rym >= 0 ? ld4g(a + G.rym + G.i0) : z;
  S.yp = G.ryp >= 0 ? ld4g(a + G.ryp + G.i0) : z;
  S.zm = G.rzm >= 0 ? ld4g(a + G.rzm + G.i0) : z;
  S.zp = G.rzp >= 0 ? ld4g(a + G.rzp + G.i0) : z;
  S.xl = a[G.rc + G.il];
  S.xr = a[G.rc + G.ir];
  return S;
}

// neighbours of cell o of the group
__device__ __forceinline__ float xp4(const St4& S, int o) { return o == 3 ? S.xr : e4(S.c, o + 1); }
__device__ __forceinline__ float xm4(const St4& S, int o) { return o == 0 ? S.xl : e4(S.c, o - 1); }

// lap7_ff on cell o (same order of operations)
// lap7_ff on cell o of a 4-cell group: the unscaled sum, same order
__device__ __forceinline__ FF lap7_ff4(const St4& H, const St4& L, int o) {
  CascadeSum s(xp4(H, o));
  s.add(xm4(H, o));
  s.add(e4(H.yp, o));
  s.add(e4(H.ym, o));
  s.add(e4(H.zp, o));
  s.add(e4(H.zm, o));
  s.add_scaled(-6.f, e4(H.c, o));
  const float lsum = xp4(L, o) + xm4(L, o) + e4(L.yp, o) + e4(L.ym, o) + e4(L.zp, o) +
                     e4(L.zm, o) - 6.f * e4(L.c, o);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, lsum));
}

// lap7 in plain FP32 on cell o (same order as lap7)
__device__ __forceinline__ float lap7_4(const St4& M, int o, float ih2) {
  return (xp4(M, o) + xm4(M, o) + e4(M.yp, o) + e4(M.ym, o) + e4(M.zp, o) + e4(M.zm, o) -
          6.f * e4(M.c, o)) * ih2;
}

__device__ __forceinline__ bool cell4(const PhaseParams& P, int& i0, int& j, int& k) {
  i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  j = blockIdx.y * blockDim.y + threadIdx.y;
  k = blockIdx.z;
  return i0 < P.nx && j < P.ny;
}

}  // namespace

__global__ void __launch_bounds__(256, 3) k_phi_update_ff4(PhaseParams P, const float* __restrict__ phi,
                                 const float* __restrict__ phi_lo, const float* __restrict__ mu,
                                 Comp3<float> psi, Comp3<float> v0, Scalars* S, float dt,
                                 float* __restrict__ out, float* __restrict__ out_lo) {
  pdl_begin();
  int i0, j, k;
  if (!cell4(P, i0, j, k)) return;
  const float ih2 = (float)P.inv_h2, hih = (float)(0.5 * P.inv_h);
  const Geo4 Gs = geo4(P, i0, j, k, false), Gp = geo4(P, i0, j, k, true);
  const St4 M = load4(mu, Gs), F = load4(phi, Gs);
  const St4 X = load4(psi.p[0], Gp), Y = load4(psi.p[1], Gp), Z = load4(psi.p[2], Gp);
  const long long jk = j + (long long)k * P.ny;
  const float v0x = v0.p[0][jk], v0y = v0.p[1][jk], v0z = v0.p[2][jk];
  const float lam = S->lambda_vf, mob = (float)P.mobility;
  const float4 fh = ld4g(phi + Gs.rc + i0), fl = ld4g(phi_lo + Gs.rc + i0);
  float oh[4], ol[4];
  bool finite = true;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float lmu = lap7_4(M, o, ih2);
    const float gx = (xp4(F, o) - xm4(F, o)) * hih;
    const float gy = (e4(F.yp, o) - e4(F.ym, o)) * hih;
    const float gz = (e4(F.zp, o) - e4(F.zm, o)) * hih;
    const float vx = v0x + ((e4(Z.yp, o) - e4(Z.ym, o)) - (e4(Y.zp, o) - e4(Y.zm, o))) * hih;
    const float vy = v0y + ((e4(X.zp, o) - e4(X.zm, o)) - (xp4(Z, o) - xm4(Z, o))) * hih;
    const float vz = v0z + ((xp4(Y, o) - xm4(Y, o)) - (e4(X.yp, o) - e4(X.ym, o))) * hih;
    const float rate = mob * (lmu + lam) - (vx * gx + vy * gy + vz * gz);
    const FF v = ff_add_f(FF{e4(fh, o), e4(fl, o)}, dt * rate);
    oh[o] = v.hi;
    ol[o] = v.lo;
    finite = finite && isfinite(v.hi);
  }
  *reinterpret_cast<float4*>(out + Gs.rc + i0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
  *reinterpret_cast<float4*>(out_lo + Gs.rc + i0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
  if (!finite) atomicOr(&S->nonfinite, 1);
}

__global__ void __launch_bounds__(256) k_helfrich_g_ff4(PhaseParams P, const float* __restrict__ phi,
                                 const float* __restrict__ phi_lo, float* __restrict__ g,
                                 float* __restrict__ g_lo) {
  pdl_begin();
  int i0, j, k;
  if (!cell4(P, i0, j, k)) return;
  const Geo4 G = geo4(P, i0, j, k, false);
  const St4 H = load4(phi, G), L = load4(phi_lo, G);
  float oh[4], ol[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const FF f{e4(H.c, o), e4(L.c, o)};
    const FF lphi = lap7_ff4(H, L, o);
    const FF cubic = ff_mul(f, ff_add_f(ff_mul(f, f), -1.f));
    const FF r = ff_add(cubic, ff_neg(ff_mul(lphi, FF{P.e2ih_hi, P.e2ih_lo})));
    oh[o] = r.hi;
    ol[o] = r.lo;
  }
  *reinterpret_cast<float4*>(g + G.rc + i0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
  *reinterpret_cast<float4*>(g_lo + G.rc + i0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
}

__global__ void __launch_bounds__(256) k_mu_ff4(PhaseParams P, const float* __restrict__ phi,
                                                const float* __restrict__ phi_lo,
                                                const float* __restrict__ g,
                                                const float* __restrict__ g_lo, const Scalars* S,
                                                float* __restrict__ mu, float* __restrict__ mu_lo) {
  pdl_begin();
  int i0, j, k;
  if (!cell4(P, i0, j, k)) return;
  const Geo4 G = geo4(P, i0, j, k, false);
  const St4 H = load4(phi, G), L = load4(phi_lo, G);
  float oh[4], ol[4];
  if (P.fe_kind == VSV_CAHN_HILLIARD) {
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const FF f{e4(H.c, o), e4(L.c, o)};
      const FF lphi = lap7_ff4(H, L, o);
      const FF cubic = ff_mul(f, ff_add_f(ff_mul(f, f), -1.f));
      const FF mm = ff_add(cubic, ff_neg(ff_mul(lphi, FF{P.sgih_hi, P.sgih_lo})));
      oh[o] = mm.hi;
      ol[o] = mm.lo;
    }
  } else {
    const St4 GH = load4(g, G), GL = load4(g_lo, G);
    const FF gih = ff_mul_f(FF{P.ih2_hi, P.ih2_lo}, S->gamma_af);   // gamma_A / h^2
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const FF f{e4(H.c, o), e4(L.c, o)};
      const FF lphi = lap7_ff4(H, L, o);
      const FF gg{e4(GH.c, o), e4(GL.c, o)};
      const FF lg = lap7_ff4(GH, GL, o);
      const FF w = ff_add_f(ff_mul_f(ff_mul(f, f), 3.f), -1.f);
      const FF inner = ff_add(ff_mul(w, gg), ff_neg(ff_mul(lg, FF{P.e2ih_hi, P.e2ih_lo})));
      FF mm = ff_add(ff_mul(inner, FF{P.cf2_hi, P.cf2_lo}), ff_neg(ff_mul(lphi, gih)));
      if (P.bt_hi != 0.f) mm = ff_add(mm, ff_mul(gg, FF{P.bt_hi, P.bt_lo}));
      oh[o] = mm.hi;
      ol[o] = mm.lo;
    }
  }
  *reinterpret_cast<float4*>(mu + G.rc + i0) = make_float4(oh[0], oh[1], oh[2], oh[3]);
  *reinterpret_cast<float4*>(mu_lo + G.rc + i0) = make_float4(ol[0], ol[1], ol[2], ol[3]);
}

__global__ void __launch_bounds__(256) k_source_ff4(PhaseParams P, const float* __restrict__ phi,
                                                    const float* __restrict__ phi_lo,
                                                    const float* __restrict__ mu,
                                                    const float* __restrict__ mu_lo,
                                                    Comp3<float> s_omega, Comp3<float> f,
                                                    Comp3<float> f_lo) {
  pdl_begin();
  int i0, j, k;
  if (!cell4(P, i0, j, k)) return;
  const Geo4 G = geo4(P, i0, j, k, false);
  const St4 FH = load4(phi, G), FL = load4(phi_lo, G), MH = load4(mu, G), ML = load4(mu_lo, G);
  // raw central differences; (1/2h)^2 / eta is applied once to each
  // component of the cross product
  const FF ie{P.src_hi, P.src_lo};
  const long long jk = j + (long long)k * P.ny;
  const float s0 = s_omega.p[0][jk], s1 = s_omega.p[1][jk], s2 = s_omega.p[2][jk];
  auto dd = [&](float ah, float al, float bh, float bl) {
    return ff_add(FF{ah, al}, ff_neg(FF{bh, bl}));
  };
  float o0h[4], o0l[4], o1h[4], o1l[4], o2h[4], o2l[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const FF ax = dd(xp4(FH, o), xp4(FL, o), xm4(FH, o), xm4(FL, o));
    const FF ay = dd(e4(FH.yp, o), e4(FL.yp, o), e4(FH.ym, o), e4(FL.ym, o));
    const FF az = dd(e4(FH.zp, o), e4(FL.zp, o), e4(FH.zm, o), e4(FL.zm, o));
    const FF bx = dd(xp4(MH, o), xp4(ML, o), xm4(MH, o), xm4(ML, o));
    const FF by = dd(e4(MH.yp, o), e4(ML.yp, o), e4(MH.ym, o), e4(ML.ym, o));
    const FF bz = dd(e4(MH.zp, o), e4(ML.zp, o), e4(MH.zm, o), e4(ML.zm, o));
    const FF c0 = ff_add_f(ff_mul(ff_add(ff_mul(ay, bz), ff_neg(ff_mul(az, by))), ie), -s0);
    const FF c1 = ff_add_f(ff_mul(ff_add(ff_mul(az, bx), ff_neg(ff_mul(ax, bz))), ie), -s1);
    const FF c2 = ff_add_f(ff_mul(ff_add(ff_mul(ax, by), ff_neg(ff_mul(ay, bx))), ie), -s2);
    o0h[o] = c0.hi; o0l[o] = c0.lo;
    o1h[o] = c1.hi; o1l[o] = c1.lo;
    o2h[o] = c2.hi; o2l[o] = c2.lo;
  }
  const long long t = G.rc + i0;
  *reinterpret_cast<float4*>(f.p[0] + t) = make_float4(o0h[0], o0h[1], o0h[2], o0h[3]);
  *reinterpret_cast<float4*>(f_lo.p[0] + t) = make_float4(o0l[0], o0l[1], o0l[2], o0l[3]);
  *reinterpret_cast<float4*>(f.p[1] + t) = make_float4(o1h[0], o1h[1], o1h[2], o1h[3]);
  *reinterpret_cast<float4*>(f_lo.p[1] + t) = make_float4(o1l[0], o1l[1], o1l[2], o1l[3]);
  *reinterpret_cast<float4*>(f.p[2] + t) = make_float4(o2h[0], o2h[1], o2h[2], o2h[3]);
  *reinterpret_cast<float4*>(f_lo.p[2] + t) = make_float4(o2l[0], o2l[1], o2l[2], o2l[3]);
}

// Partial sums of sum(phi) and of the area density over 4-cell groups; one
// (phi, area) pair per block, as k_reduce_va.  Each warp takes whole x rows
// (row index and plane from one 32-bit division per row), its lanes the
// rows' 4-cell groups.  WITH_G: the Helfrich g of the same cells is formed
// from the same staged stencil and stored as k_helfrich_g_ff4 stores it
// (same operations, same values), saving that kernel's pass over phi.
template <bool WITH_G>
__global__ void __launch_bounds__(256) k_reduce_va_ff4(PhaseParams P, const float* __restrict__ phi,
                                                       const float* __restrict__ phi_lo,
                                                       double* partials, float* __restrict__ g,
                                                       float* __restrict__ g_lo) {
  pdl_begin();
  const int ng = P.nx >> 2;
  const int rows = P.ny * P.nz;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const FF agf{P.ag_hi, P.ag_lo}, awf{P.aw_hi, P.aw_lo};
  CascadeSum cp(0.f), ca(0.f);
  for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += gridDim.x * wpb)
  for (int gi = lane; gi < ng; gi += 32) {
    const int k = row / P.ny, j = row - k * P.ny;
    const Geo4 G = geo4(P, 4 * gi, j, k, false);
    const St4 H = load4(phi, G), L = load4(phi_lo, G);
    float oh[4], ol[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const FF f{e4(H.c, o), e4(L.c, o)};
      auto diff = [&](float ah, float al, float bh, float bl) {
        return ff_add(FF{ah, al}, ff_neg(FF{bh, bl}));
      };
      const FF gx = diff(xp4(H, o), xp4(L, o), xm4(H, o), xm4(L, o));
      const FF gy = diff(e4(H.yp, o), e4(L.yp, o), e4(H.ym, o), e4(L.ym, o));
      const FF gz = diff(e4(H.zp, o), e4(L.zp, o), e4(H.zm, o), e4(L.zm, o));
      const FF g2 = ff_add(ff_add(ff_mul(gx, gx), ff_mul(gy, gy)), ff_mul(gz, gz));
      const FF w = ff_add_f(ff_mul(f, f), -1.f);
      const FF dens = ff_add(ff_mul(g2, agf), ff_mul(ff_mul(w, w), awf));
      cp.add(f.hi);
      cp.add(f.lo);
      ca.add(dens.hi);
      ca.add(dens.lo);
      if constexpr (WITH_G) {
        // g = phi (phi^2 - 1) - eps^2 lap phi, as k_helfrich_g_ff4 (w is its
        // phi^2 - 1)
        const FF r = ff_add(ff_mul(f, w),
                            ff_neg(ff_mul(lap7_ff4(H, L, o), FF{P.e2ih_hi, P.e2ih_lo})));
        oh[o] = r.hi;
        ol[o] = r.lo;
      }
    }
    if constexpr (WITH_G) {
      *reinterpret_cast<float4*>(g + G.rc + 4 * gi) = make_float4(oh[0], oh[1], oh[2], oh[3]);
      *reinterpret_cast<float4*>(g_lo + G.rc + 4 * gi) = make_float4(ol[0], ol[1], ol[2], ol[3]);
    }
  }
  double sphi = (double)cp.hi + (double)cp.lo;
  double sarea = (double)ca.hi + (double)ca.lo;
  sphi = block_sum(sphi);
  sarea = block_sum(sarea);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sphi;
    partials[2 * blockIdx.x + 1] = sarea;
  }
}

static bool use4(const PhaseParams& P) { return P.nx % 4 == 0 && P.nx >= 8; }
static dim3 grid4(const PhaseParams& P) {
  return dim3((unsigned)((P.nx / 4 + 31) / 32), (unsigned)((P.ny + 7) / 8), (unsigned)P.nz);
}

void launch_phi_update_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo,
                          const float* mu, Comp3<float> psi, Comp3<float> v0, const Scalars* S,
                          float dt, float* out, float* out_lo) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_PHASE);
  if (use4(P))
    launch_k(cx, k_phi_update_ff4, grid4(P), dim3(32, 8), 0, P, phi, phi_lo, mu, psi, v0,
             const_cast<Scalars*>(S), dt, out, out_lo);
  else
    k_phi_update_ff<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(
        P, phi, phi_lo, mu, psi, v0, const_cast<Scalars*>(S), dt, out, out_lo);
  // phi (two words), mu, psi' (3) read; phi (two words) written
  cx.after(VSV_KCLASS_PHASE, 32.0 * (double)n);
}

void launch_mu_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo, float* g,
                  float* g_lo, float* mu, float* mu_lo, const Scalars* S, bool g_ready) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  if (P.fe_kind == VSV_HELFRICH && !g_ready) {
    cx.before(VSV_KCLASS_PHASE);
    if (use4(P))
      launch_k(cx, k_helfrich_g_ff4, grid4(P), dim3(32, 8), 0, P, phi, phi_lo, g, g_lo);
    else
      k_helfrich_g_ff<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, phi_lo, g, g_lo);
    cx.after(VSV_KCLASS_PHASE, 16.0 * (double)n);   // phi read, g written (two words each)
  }
  cx.before(VSV_KCLASS_PHASE);
  if (use4(P))
    launch_k(cx, k_mu_ff4, grid4(P), dim3(32, 8), 0, P, phi, phi_lo, g, g_lo, S, mu, mu_lo);
  else
    k_mu_ff<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, phi_lo, g, g_lo, S, mu,
                                                                       mu_lo);
  // phi (and g for Helfrich) read, mu written, two words each
  cx.after(VSV_KCLASS_PHASE, (P.fe_kind == VSV_HELFRICH ? 24.0 : 16.0) * (double)n);
}

// f = grad phi x grad mu / eta - s_omega in double-word arithmetic from
// phi = hi + lo and mu = hi + lo; written as hi + lo.  The stream vector
// psi' = L^{-2}(-f) is dominated by the small low-wavenumber content of this
// dipole-like source, so FP32 rounding of f would be amplified ~10^3 in psi'.
__global__ void k_source_ff(PhaseParams P, const float* __restrict__ phi, const float* __restrict__ phi_lo,
                            const float* __restrict__ mu, const float* __restrict__ mu_lo,
                            Comp3<float> s_omega, Comp3<float> f, Comp3<float> f_lo) {
  int i, j, k, comp_;
  if (!cell3(P.nx, P.ny, P.nz, i, j, k, comp_)) return;
  const long long t = lin(i, j, k, P.nx, P.ny);
  ScalarView<float> FH{phi, P.nx, P.ny, P.nz, P.zper}, FL{phi_lo, P.nx, P.ny, P.nz, P.zper};
  ScalarView<float> MH{mu, P.nx, P.ny, P.nz, P.zper}, ML{mu_lo, P.nx, P.ny, P.nz, P.zper};
  // raw central differences; (1/2h)^2 / eta is applied once to each
  // component of the cross product
  auto dd = [&](const ScalarView<float>& H, const ScalarView<float>& L, int i1, int j1, int k1, int i0,
                int j0, int k0) {
    const FF a{H(i1, j1, k1), L(i1, j1, k1)}, b{H(i0, j0, k0), L(i0, j0, k0)};
    return ff_add(a, ff_neg(b));
  };
  const FF ax = dd(FH, FL, i + 1, j, k, i - 1, j, k), ay = dd(FH, FL, i, j + 1, k, i, j - 1, k),
           az = dd(FH, FL, i, j, k + 1, i, j, k - 1);
  const FF bx = dd(MH, ML, i + 1, j, k, i - 1, j, k), by = dd(MH, ML, i, j + 1, k, i, j - 1, k),
           bz = dd(MH, ML, i, j, k + 1, i, j, k - 1);
  const FF ie{P.src_hi, P.src_lo};
  const long long jk = j + (long long)k * P.ny;
  const FF c0 = ff_add_f(ff_mul(ff_add(ff_mul(ay, bz), ff_neg(ff_mul(az, by))), ie), -s_omega.p[0][jk]);
  const FF c1 = ff_add_f(ff_mul(ff_add(ff_mul(az, bx), ff_neg(ff_mul(ax, bz))), ie), -s_omega.p[1][jk]);
  const FF c2 = ff_add_f(ff_mul(ff_add(ff_mul(ax, by), ff_neg(ff_mul(ay, bx))), ie), -s_omega.p[2][jk]);
  f.p[0][t] = c0.hi; f_lo.p[0][t] = c0.lo;
  f.p[1][t] = c1.hi; f_lo.p[1][t] = c1.lo;
  f.p[2][t] = c2.hi; f_lo.p[2][t] = c2.lo;
}

void launch_source_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo,
                      const float* mu, const float* mu_lo, Comp3<float> s_omega, Comp3<float> f,
                      Comp3<float> f_lo) {
  cx.before(VSV_KCLASS_PHASE);
  if (use4(P))
    launch_k(cx, k_source_ff4, grid4(P), dim3(32, 8), 0, P, phi, phi_lo, mu, mu_lo, s_omega, f, f_lo);
  else
    k_source_ff<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, phi_lo, mu, mu_lo,
                                                                         s_omega, f, f_lo);
  // phi, mu read, f (3) written, two words each
  cx.after(VSV_KCLASS_PHASE, 40.0 * (double)((long long)P.nx * P.ny * P.nz));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }
static unsigned v4_blocks(const Ctx& cx, long long n) {
  const long long want = (n / 4 + kBlock - 1) / kBlock;
  return (unsigned)std::max<long long>(1, std::min<long long>(want, 16LL * cx.sms));
}

void launch_split_ff(Ctx& cx, const double* in, float* hi, float* lo, long long n) {
  cx.before(-1);
  if (aligned16(in) && aligned16(hi) && aligned16(lo))
    k_split_ff_v4<<<v4_blocks(cx, n), kBlock, 0, cx.stream>>>(in, hi, lo, n);
  else
    k_split_ff<<<nblk(n), kBlock, 0, cx.stream>>>(in, hi, lo, n);
  cx.after(-1);
}

void launch_merge_ff(Ctx& cx, const float* hi, const float* lo, double* out, long long n) {
  cx.before(-1);
  if (aligned16(out) && aligned16(hi) && aligned16(lo))
    k_merge_ff_v4<<<v4_blocks(cx, n), kBlock, 0, cx.stream>>>(hi, lo, out, n);
  else
    k_merge_ff<<<nblk(n), kBlock, 0, cx.stream>>>(hi, lo, out, n);
  cx.after(-1);
}

// ---------------------------------------------------------------- launchers
template <class T>
void launch_phi_update(Ctx& cx, const PhaseParams& P, const T* phi, const T* mu, Comp3<T> psi,
                       Comp3<T> v0, const Scalars* S, T dt, T* out) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_PHASE);
  k_phi_update<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, mu, psi, v0, const_cast<Scalars*>(S),
                                                     dt, out);
  cx.after(VSV_KCLASS_PHASE, 6.0 * sizeof(T) * (double)n);   // phi, mu, psi' (3) read, phi written
}

template <class T>
bool launch_reduce_va(Ctx& cx, const PhaseParams& P, const T* phi, const T* phi_lo,
                      double* partials, int nblocks, Scalars* S, int init, float* g, float* g_lo) {
  bool with_g = false;
  cx.before(VSV_KCLASS_PHASE);
  if constexpr (std::is_same<T, float>::value) {
    if (use4(P)) {
      with_g = g && g_lo;
      if (with_g)
        launch_k(cx, k_reduce_va_ff4<true>, nblocks, kBlock, 0, P, phi, phi_lo, partials, g, g_lo);
      else
        launch_k(cx, k_reduce_va_ff4<false>, nblocks, kBlock, 0, P, phi, phi_lo, partials,
                 (float*)nullptr, (float*)nullptr);
    } else {
      k_reduce_va<T><<<nblocks, kBlock, 0, cx.stream>>>(P, phi, phi_lo, partials);
    }
  } else {
    k_reduce_va<T><<<nblocks, kBlock, 0, cx.stream>>>(P, phi, phi_lo, partials);
  }
  // phi read (two FP32 words, or one FP64); g written (two words)
  cx.after(VSV_KCLASS_PHASE, (with_g ? 16.0 : 8.0) * (double)((long long)P.nx * P.ny * P.nz));
  cx.before(-1);
  launch_k(cx, k_va_finalize, 1, kBlock, 0, partials, nblocks, (long long)P.nx * P.ny * P.nz, S,
           init);
  cx.after(-1);
  return with_g;
}

template <class T>
void launch_mu(Ctx& cx, const PhaseParams& P, const T* phi, T* g, T* mu, const Scalars* S) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  if (P.fe_kind == VSV_HELFRICH) {
    cx.before(VSV_KCLASS_PHASE);
    k_helfrich_g<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, g);
    cx.after(VSV_KCLASS_PHASE, 2.0 * sizeof(T) * (double)n);
  }
  cx.before(VSV_KCLASS_PHASE);
  k_mu<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, g, S, mu);
  cx.after(VSV_KCLASS_PHASE, (P.fe_kind == VSV_HELFRICH ? 3.0 : 2.0) * sizeof(T) * (double)n);
}

template <class T>
void launch_source(Ctx& cx, const PhaseParams& P, const T* phi, const T* mu, Comp3<T> s_omega,
                   Comp3<T> f) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_PHASE);
  k_source<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, phi, mu, s_omega, f);
  cx.after(VSV_KCLASS_PHASE, 5.0 * sizeof(T) * (double)n);   // phi, mu read, f (3) written
}

template <class T>
void launch_velocity(Ctx& cx, const PhaseParams& P, Comp3<T> psi, Comp3<T> psi_lo, Comp3<T> v0,
                     Comp3<T> v) {
  cx.before(-1);
  k_velocity<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, psi, psi_lo, v0, v);
  cx.after(-1);
}

void launch_velocity_dw(Ctx& cx, const PhaseParams& P, Comp3<float> psi, Comp3<float> psi_lo,
                        Comp3<const double> v0d, Comp3<float> v, Comp3<float> v_lo) {
  cx.before(-1);
  k_velocity_dw<<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, psi, psi_lo, v0d, v,
                                                                        v_lo);
  cx.after(-1);
}

template <class T>
void launch_diag(Ctx& cx, const PhaseParams& P, const T* phi, const T* phi_lo, const T* g,
                 const T* g_lo, Comp3<T> vel, Comp3<T> vel_lo, Comp3<T> omega, Comp3<T> om_lo,
                 Comp3<T> psi, Comp3<T> ps_lo, Comp3<const double> psi0_ring,
                 Comp3<const double> v0d, T* sigma_t, double* partials, int nblocks, double* out) {
  cx.before(-1);
  k_diag<T><<<nblocks, kBlock, 0, cx.stream>>>(P, phi, phi_lo, g, g_lo, vel, vel_lo, omega, om_lo,
                                               psi, ps_lo, psi0_ring, v0d, sigma_t, partials);
  cx.after(-1);
  cx.before(-1);
  k_diag_finalize<<<1, kBlock, 0, cx.stream>>>(partials, nblocks, out);
  cx.after(-1);
}

template <class T>
void launch_stress_profile(Ctx& cx, const PhaseParams& P, Comp3<T> vel, Comp3<T> vel_lo,
                           double* out) {
  cx.before(-1);
  k_stress_profile<T><<<P.ny, kBlock, 0, cx.stream>>>(P, vel, vel_lo, out);
  cx.after(-1);
}

template <class Tin, class Tout>
void launch_convert(Ctx& cx, const Tin* in, Tout* out, long long n) {
  cx.before(-1);
  k_convert<Tin, Tout><<<nblk(n), kBlock, 0, cx.stream>>>(in, out, n);
  cx.after(-1);
}

template <class T>
void launch_full_field(Ctx& cx, const PhaseParams& P, const T* pert, const T* lo, const double* tab,
                       int ring, T* out) {
  cx.before(-1);
  k_full_field<T><<<grid3(P.nx, P.ny, P.nz, 1), block3(), 0, cx.stream>>>(P, pert, lo, tab, ring, out);
  cx.after(-1);
}

template <class T>
void launch_scale_copy(Ctx& cx, const T* in, T* out, long long n, double a) {
  cx.before(-1);
  k_scale_copy<T><<<nblk(n), kBlock, 0, cx.stream>>>(in, out, n, (T)a);
  cx.after(-1);
}

void launch_duct_ring(Ctx& cx, int ny, int nz, double h, const double* u0, const double* chi,
                      double* omy, double* omz, double* psy, double* psz) {
  const int m = ny > nz ? ny : nz;
  cx.before(-1);
  k_duct_ring<<<nblk(m), kBlock, 0, cx.stream>>>(ny, nz, h, u0, chi, omy, omz, psy, psz);
  cx.after(-1);
}

void launch_ring_boundary_rhs(Ctx& cx, int ny, int nz, double h, const double* ring, double scale,
                              const double* in, double* out) {
  cx.before(-1);
  k_ring_rhs<<<nblk((long long)ny * nz), kBlock, 0, cx.stream>>>(ny, nz, h, ring, scale, in, out);
  cx.after(-1);
}

void launch_ring_fill_interior(Ctx& cx, int ny, int nz, const double* interior, double* ring) {
  cx.before(-1);
  k_ring_fill<<<nblk((long long)ny * nz), kBlock, 0, cx.stream>>>(ny, nz, interior, ring);
  cx.after(-1);
}

void launch_base_derived(Ctx& cx, int ny, int nz, int zper, double h, const double* om[3],
                         const double* ps[3], double* v0[3], double* s_om[3], double* s_ps[3]) {
  Comp3<const double> O{{om[0], om[1], om[2]}}, Pp{{ps[0], ps[1], ps[2]}};
  Comp3<double> V{{v0[0], v0[1], v0[2]}}, SO{{s_om[0], s_om[1], s_om[2]}},
      SP{{s_ps[0], s_ps[1], s_ps[2]}};
  cx.before(-1);
  k_base_derived<<<nblk((long long)ny * nz), kBlock, 0, cx.stream>>>(ny, nz, zper, h, O, Pp, V, SO, SP);
  cx.after(-1);
}

double device_max_abs(Ctx& cx, const double* x, long long n, double* scratch) {
  cx.before(-1);
  k_max_abs<<<1, 1024, 0, cx.stream>>>(x, n, scratch);
  cx.after(-1);
  double h = 0.0;
  cudaMemcpyAsync(&h, scratch, sizeof(double), cudaMemcpyDeviceToHost, cx.stream);
  cudaStreamSynchronize(cx.stream);
  return h;
}

void launch_fill(Ctx& cx, double* x, long long n, double v) {
  cx.before(-1);
  k_fill<<<nblk(n), kBlock, 0, cx.stream>>>(x, n, v);
  cx.after(-1);
}

#define VSV_INST(T)                                                                               \
  template void launch_phi_update<T>(Ctx&, const PhaseParams&, const T*, const T*, Comp3<T>,      \
                                     Comp3<T>, const Scalars*, T, T*);                            \
  template bool launch_reduce_va<T>(Ctx&, const PhaseParams&, const T*, const T*, double*, int,   \
                                    Scalars*, int, float*, float*);                               \
  template void launch_mu<T>(Ctx&, const PhaseParams&, const T*, T*, T*, const Scalars*);         \
  template void launch_source<T>(Ctx&, const PhaseParams&, const T*, const T*, Comp3<T>,          \
                                 Comp3<T>);                                                       \
  template void launch_velocity<T>(Ctx&, const PhaseParams&, Comp3<T>, Comp3<T>, Comp3<T>,       \
                                   Comp3<T>);                                                     \
  template void launch_diag<T>(Ctx&, const PhaseParams&, const T*, const T*, const T*, const T*,  \
                               Comp3<T>, Comp3<T>, Comp3<T>, Comp3<T>, Comp3<T>, Comp3<T>,        \
                               Comp3<const double>, Comp3<const double>, T*, double*, int,        \
                               double*);                                                          \
  template void launch_stress_profile<T>(Ctx&, const PhaseParams&, Comp3<T>, Comp3<T>, double*);  \
  template void launch_full_field<T>(Ctx&, const PhaseParams&, const T*, const T*, const double*,  \
                                     int, T*);                                                    \
  template void launch_scale_copy<T>(Ctx&, const T*, T*, long long, double);
VSV_INST(float)
VSV_INST(double)
#undef VSV_INST
template void launch_convert<float, double>(Ctx&, const float*, double*, long long);
template void launch_convert<double, float>(Ctx&, const double*, float*, long long);
template void launch_convert<float, float>(Ctx&, const float*, float*, long long);
template void launch_convert<double, double>(Ctx&, const double*, double*, long long);

}  // namespace vsv
