// Discrete adjoint of the time step (FP64 kernels).
//
// Reverse mode of the step of main-text eqs. gen2, gen1, gen3 as the forward
// kernels compute it: phi^{n+1} = phi^n + dt [M (L_m mu^n + lambda^n) -
// v^n . D_m phi^n], gamma^{n+1} from A[phi^{n+1}], mu^{n+1} (eq. 31 or eq. 30 /
// SM eq. 35, plus sigma A_f for a membrane tension), f = D_m phi x D_m mu /
// eta, L omega' = f - s_omega, L psi' = -omega' - s_psi, v = v0 + curl psi'.
// The transposes used (with respect to the plain sum over cells):
//   L_m, L      symmetric (the adjoint Poisson problems are the same problems);
//   D_m^T w   = -D_odd w: the central difference of w with odd ghosts at a
//               mirror face (ghost -1 <- -w_0), wrapped on periodic axes;
//   curl^T    = curl with zero ghosts on the walls;
//   d mu/d phi  symmetric: cf2 [6 phi g + G G] + beta G - gamma L_m (Helfrich,
//               G = (3 phi^2 - 1) - eps^2 L_m), (3 phi^2 - 1) - sigma L_m (CH).
// One thread per cell (x fastest, coalesced); neighbour values through small
// views that apply the closure of each field.  Reductions are per-block
// partial sums totalled in fixed order by one block, so every gradient is
// bitwise reproducible.
#include "internal.h"

namespace vsv {

namespace {

constexpr int kAB = 256;   // threads per block of the adjoint kernels
constexpr double kCA = 1.0606601717798212;   // 3 / (2 sqrt 2)

__device__ __forceinline__ int wrapi_(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// index map of the scalar closure along a mirrored axis; flips `sgn` when the
// index was reflected (odd extension)
__device__ __forceinline__ int mirror_(int j, int n, double& sgn) {
  if (j < 0) { sgn = -sgn; return -1 - j; }
  if (j >= n) { sgn = -sgn; return 2 * n - 1 - j; }
  return j;
}

struct Dims {
  int nx, ny, nz, zper;
  __device__ __forceinline__ long long at(int i, int j, int k) const {
    return ((long long)k * ny + j) * nx + i;
  }
};

// even (mirror) extension of a scalar field: phi, mu, g and their adjoints
struct Even {
  const double* __restrict__ a;
  Dims d;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    double s = 1.0;
    i = wrapi_(i, d.nx);
    j = mirror_(j, d.ny, s);
    k = d.zper ? wrapi_(k, d.nz) : mirror_(k, d.nz, s);
    return a[d.at(i, j, k)];
  }
};

// odd extension (the transpose of the mirror central difference)
struct Odd {
  const double* __restrict__ a;
  Dims d;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    double s = 1.0;
    i = wrapi_(i, d.nx);
    j = mirror_(j, d.ny, s);
    k = d.zper ? wrapi_(k, d.nz) : mirror_(k, d.nz, s);
    return s * a[d.at(i, j, k)];
  }
};

// zero on the wall nodes (flow perturbations and their adjoints)
struct Zero {
  const double* __restrict__ a;
  Dims d;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    i = wrapi_(i, d.nx);
    if (d.zper) k = wrapi_(k, d.nz);
    if (j < 0 || j >= d.ny || k < 0 || k >= d.nz) return 0.0;
    return a[d.at(i, j, k)];
  }
};

template <class V>
__device__ __forceinline__ double lap_(const V& f, int i, int j, int k, double ih2) {
  return (f(i + 1, j, k) + f(i - 1, j, k) + f(i, j + 1, k) + f(i, j - 1, k) + f(i, j, k + 1) +
          f(i, j, k - 1) - 6.0 * f(i, j, k)) * ih2;
}

// central difference along axis a (0 x, 1 y, 2 z)
template <class V>
__device__ __forceinline__ double d_(const V& f, int a, int i, int j, int k, double hih) {
  if (a == 0) return (f(i + 1, j, k) - f(i - 1, j, k)) * hih;
  if (a == 1) return (f(i, j + 1, k) - f(i, j - 1, k)) * hih;
  return (f(i, j, k + 1) - f(i, j, k - 1)) * hih;
}

__device__ __forceinline__ bool cell_(const Dims& d, long long& t, int& i, int& j, int& k) {
  t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)d.nx * d.ny * d.nz;
  if (t >= n) return false;
  i = (int)(t % d.nx);
  const long long q = t / d.nx;
  j = (int)(q % d.ny);
  k = (int)(q / d.ny);
  return true;
}

// sum of v over the block (blockDim.x == kAB); every thread gets the total
__device__ __forceinline__ double bsum_(double v) { return block_sum(v); }

}  // namespace

namespace {

__device__ __forceinline__ Dims dims_(const AdjParams& P) { return Dims{P.nx, P.ny, P.nz, P.zper}; }

// abar = (D_m mu x fbar) / eta, bbar = (fbar x D_m phi) / eta: the adjoint of
// the source f = D_m phi x D_m mu / eta for the adjoint fbar of f.
__global__ void __launch_bounds__(kAB) k_adj_source(AdjParams P, const double* __restrict__ phi,
                                                   const double* __restrict__ mu, Comp3<const double> fb,
                                                   Comp3<double> ab, Comp3<double> bb) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  if (!cell_(d, t, i, j, k)) return;
  Even F{phi, d}, M{mu, d};
  const double a0 = d_(F, 0, i, j, k, P.hih), a1 = d_(F, 1, i, j, k, P.hih), a2 = d_(F, 2, i, j, k, P.hih);
  const double b0 = d_(M, 0, i, j, k, P.hih), b1 = d_(M, 1, i, j, k, P.hih), b2 = d_(M, 2, i, j, k, P.hih);
  const double f0 = fb.p[0][t], f1 = fb.p[1][t], f2 = fb.p[2][t];
  const double ie = P.inv_eta;
  ab.p[0][t] = (b1 * f2 - b2 * f1) * ie;
  ab.p[1][t] = (b2 * f0 - b0 * f2) * ie;
  ab.p[2][t] = (b0 * f1 - b1 * f0) * ie;
  bb.p[0][t] = (f1 * a2 - f2 * a1) * ie;
  bb.p[1][t] = (f2 * a0 - f0 * a2) * ie;
  bb.p[2][t] = (f0 * a1 - f1 * a0) * ie;
}

// outA += D_m^T A = -sum_a D_odd,a A_a (and the same for B when given)
__global__ void __launch_bounds__(kAB) k_adj_divt(AdjParams P, Comp3<const double> A, double* __restrict__ outA,
                                                 Comp3<const double> B, double* __restrict__ outB) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  if (!cell_(d, t, i, j, k)) return;
  {
    Odd X{A.p[0], d}, Y{A.p[1], d}, Z{A.p[2], d};
    outA[t] -= d_(X, 0, i, j, k, P.hih) + d_(Y, 1, i, j, k, P.hih) + d_(Z, 2, i, j, k, P.hih);
  }
  if (outB) {
    Odd X{B.p[0], d}, Y{B.p[1], d}, Z{B.p[2], d};
    outB[t] -= d_(X, 0, i, j, k, P.hih) + d_(Y, 1, i, j, k, P.hih) + d_(Z, 2, i, j, k, P.hih);
  }
}

// Helfrich: g = phi^3 - phi - eps^2 L_m phi and w = G mubar =
// (3 phi^2 - 1) mubar - eps^2 L_m mubar
__global__ void __launch_bounds__(kAB) k_adj_g(AdjParams P, const double* __restrict__ phi,
                                              const double* __restrict__ mub, double* __restrict__ g,
                                              double* __restrict__ w) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  if (!cell_(d, t, i, j, k)) return;
  Even F{phi, d}, U{mub, d};
  const double f = phi[t];
  g[t] = f * f * f - f - P.e2 * lap_(F, i, j, k, P.ih2);
  w[t] = (3.0 * f * f - 1.0) * mub[t] - P.e2 * lap_(U, i, j, k, P.ih2);
}

// phib += (d mu / d phi)^T mubar; per-block partial sums of
// <d mu / d kappa, mubar>, <d mu / d sigma, mubar>, <d mu / d gamma, mubar>
__global__ void __launch_bounds__(kAB) k_adj_mu(AdjParams P, const double* __restrict__ phi,
                                               const double* __restrict__ mub, const double* __restrict__ g,
                                               const double* __restrict__ w, const double* gamma,
                                               double* __restrict__ phib, double* __restrict__ partials) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  double pk = 0.0, ps = 0.0, pg = 0.0;
  if (cell_(d, t, i, j, k)) {
    Even F{phi, d}, U{mub, d};
    const double f = phi[t], u = mub[t];
    const double lphi = lap_(F, i, j, k, P.ih2);
    const double lu = lap_(U, i, j, k, P.ih2);
    if (P.fe_kind == VSV_CAHN_HILLIARD) {
      phib[t] += (3.0 * f * f - 1.0) * u - P.sigma * lu;
      ps = -lphi * u;
    } else {
      Even G{g, d}, W{w, d};
      const double gg = g[t], ww = w[t];
      const double gam = gamma ? *gamma : 0.0;
      const double q = 3.0 * f * f - 1.0;
      phib[t] += P.cf2 * (6.0 * f * gg * u + q * ww - P.e2 * lap_(W, i, j, k, P.ih2)) + P.beta * ww -
                 gam * lu;
      pk = P.cf2_per_kappa * (q * gg - P.e2 * lap_(G, i, j, k, P.ih2)) * u;
      ps = kCA / P.eps * gg * u;
      pg = -lphi * u;
    }
  }
  pk = bsum_(pk);
  ps = bsum_(ps);
  pg = bsum_(pg);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = pk;
    partials[3 * blockIdx.x + 1] = ps;
    partials[3 * blockIdx.x + 2] = pg;
  }
}

// Fixed-order totals of k_adj_mu: kappabar, sigmabar accumulate; with the
// area penalty gamma = K_A c_g (A - A0) passes gammabar on as the
// coefficient c = gammabar K_A c_g of dA/dphi and as -c to A0bar.
__global__ void k_adj_mu_finalize(AdjParams P, const double* partials, int nblocks, double* acc,
                                  int area) {
  double sk = 0.0, ss = 0.0, sg = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    sk += partials[3 * b];
    ss += partials[3 * b + 1];
    sg += partials[3 * b + 2];
  }
  sk = block_sum(sk);
  ss = block_sum(ss);
  sg = block_sum(sg);
  if (threadIdx.x == 0) {
    acc[kAccKappa] += sk;
    acc[kAccSigma] += ss;
    acc[kAccGamma] = sg;
    const double c = area ? sg * P.k_area * 3.0 * P.eps / (2.0 * 1.4142135623730951) : 0.0;
    acc[kAccAreaCoef] = c;
    acc[kAccA0] -= c;
  }
}

// phib += coef * dA/dphi + add_scale * add, dA/dphi = h^3 c_A [eps D_m^T
// D_m phi + (phi^2 - 1) phi / eps] (central-difference area of SM eq. 32)
__global__ void __launch_bounds__(kAB) k_adj_area(AdjParams P, const double* __restrict__ phi,
                                                 const double* coef, const double* add,
                                                 double add_scale, double* __restrict__ phib) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  if (!cell_(d, t, i, j, k)) return;
  const double c = coef ? *coef : 0.0;
  const double a = add ? add_scale * *add : 0.0;
  if (c == 0.0) {
    phib[t] += a;
    return;
  }
  Even F{phi, d};
  // q_a = D_a phi at the neighbour m along axis a, odd extension past a mirror face
  auto q = [&](int ax, int ii, int jj, int kk) {
    double s = 1.0;
    ii = wrapi_(ii, d.nx);
    jj = mirror_(jj, d.ny, s);
    kk = d.zper ? wrapi_(kk, d.nz) : mirror_(kk, d.nz, s);
    return s * d_(F, ax, ii, jj, kk, P.hih);
  };
  const double dtd = -((q(0, i + 1, j, k) - q(0, i - 1, j, k)) + (q(1, i, j + 1, k) - q(1, i, j - 1, k)) +
                       (q(2, i, j, k + 1) - q(2, i, j, k - 1))) * P.hih;
  const double f = phi[t];
  phib[t] += c * P.h3 * kCA * (P.eps * dtd + (f * f - 1.0) * f / P.eps) + a;
}

// Reverse of the phi update, first half: s_a = v_a phibar, vbar_a = -dt
// phibar D_a phi^n, mubar^n = dt M L_m phibar, and partial sums of phibar;
// v = v0(y, z) + curl psi'^n.
__global__ void __launch_bounds__(kAB) k_adj_update1(AdjParams P, const double* __restrict__ phib,
                                                    const double* __restrict__ phi, Comp3<const double> psi,
                                                    Comp3<const double> v0, double dt, Comp3<double> s,
                                                    Comp3<double> vb, double* __restrict__ mub,
                                                    double* __restrict__ partials) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  double part = 0.0;
  if (cell_(d, t, i, j, k)) {
    Even F{phi, d}, U{phib, d};
    Zero X{psi.p[0], d}, Y{psi.p[1], d}, Z{psi.p[2], d};
    const long long jk = j + (long long)k * d.ny;
    const double vx = v0.p[0][jk] + (d_(Z, 1, i, j, k, P.hih) - d_(Y, 2, i, j, k, P.hih));
    const double vy = v0.p[1][jk] + (d_(X, 2, i, j, k, P.hih) - d_(Z, 0, i, j, k, P.hih));
    const double vz = v0.p[2][jk] + (d_(Y, 0, i, j, k, P.hih) - d_(X, 1, i, j, k, P.hih));
    const double u = phib[t];
    s.p[0][t] = vx * u;
    s.p[1][t] = vy * u;
    s.p[2][t] = vz * u;
    vb.p[0][t] = -dt * u * d_(F, 0, i, j, k, P.hih);
    vb.p[1][t] = -dt * u * d_(F, 1, i, j, k, P.hih);
    vb.p[2][t] = -dt * u * d_(F, 2, i, j, k, P.hih);
    mub[t] = dt * P.mobility * lap_(U, i, j, k, P.ih2);
    part = u;
  }
  part = bsum_(part);
  if (threadIdx.x == 0) partials[blockIdx.x] = part;
}

// lambdabar = dt M sum phibar; V0bar -= K_V lambdabar; the constant added to
// phibar^n is K_V lambdabar dV/dphi = -K_V lambdabar h^3 / 2
__global__ void k_adj_lambda_finalize(AdjParams P, const double* partials, int nblocks, double dt,
                                      double* acc) {
  double sp = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) sp += partials[b];
  sp = block_sum(sp);
  if (threadIdx.x == 0) {
    const double lam = dt * P.mobility * sp;
    acc[kAccLambda] = lam;
    acc[kAccV0] -= lam * P.k_vol;
    acc[kAccPhiAdd] = -0.5 * P.h3 * lam * P.k_vol;
  }
}

// Second half: phibar^n = phibar - dt D_m^T s + const (in place: a thread
// reads phibar only at its own cell), psibar'^n = curl vbar (zero ghosts).
__global__ void __launch_bounds__(kAB) k_adj_update2(AdjParams P, double* __restrict__ phib,
                                                    Comp3<const double> s, Comp3<const double> vb,
                                                    double dt, const double* acc, Comp3<double> psib) {
  const Dims d = dims_(P);
  long long t;
  int i, j, k;
  if (!cell_(d, t, i, j, k)) return;
  Odd SX{s.p[0], d}, SY{s.p[1], d}, SZ{s.p[2], d};
  const double dts = d_(SX, 0, i, j, k, P.hih) + d_(SY, 1, i, j, k, P.hih) + d_(SZ, 2, i, j, k, P.hih);
  phib[t] = phib[t] + dt * dts + acc[kAccPhiAdd];
  Zero X{vb.p[0], d}, Y{vb.p[1], d}, Z{vb.p[2], d};
  psib.p[0][t] = d_(Z, 1, i, j, k, P.hih) - d_(Y, 2, i, j, k, P.hih);
  psib.p[1][t] = d_(X, 2, i, j, k, P.hih) - d_(Z, 0, i, j, k, P.hih);
  psib.p[2][t] = d_(Y, 0, i, j, k, P.hih) - d_(X, 1, i, j, k, P.hih);
}

// x = a * y (n doubles): the terminal adjoint and copies with scale
__global__ void k_adj_scale(const double* __restrict__ y, double* __restrict__ x, long long n, double a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = a * y[t];
}

// z = a x + b y (n doubles); z may alias x or y
__global__ void k_adj_axpby(double* z, const double* x, const double* y, long long n, double a,
                            double b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) z[t] = a * x[t] + b * y[t];
}

unsigned nb_(long long n) { return (unsigned)((n + kAB - 1) / kAB); }

}  // namespace

int adj_blocks(long long ncells) { return (int)nb_(ncells); }

void launch_adj_source(Ctx& cx, const AdjParams& P, const double* phi, const double* mu,
                       Comp3<const double> fb, Comp3<double> ab, Comp3<double> bb) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_source<<<nb_(n), kAB, 0, cx.stream>>>(P, phi, mu, fb, ab, bb);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * 11 * (double)n);   // phi, mu, fbar(3) read; abar, bbar written
}

void launch_adj_divt(Ctx& cx, const AdjParams& P, Comp3<const double> A, double* outA,
                     Comp3<const double> B, double* outB) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_divt<<<nb_(n), kAB, 0, cx.stream>>>(P, A, outA, B, outB);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * (outB ? 10 : 5) * (double)n);
}

void launch_adj_mu(Ctx& cx, const AdjParams& P, const double* phi, const double* mub,
                   const double* gamma, double* g, double* w, double* phib, double* partials,
                   double* acc, bool area) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const unsigned nb = nb_(n);
  if (P.fe_kind == VSV_HELFRICH) {
    cx.before(VSV_KCLASS_ADJOINT);
    k_adj_g<<<nb, kAB, 0, cx.stream>>>(P, phi, mub, g, w);
    cx.after(VSV_KCLASS_ADJOINT, 8.0 * 4 * (double)n);
  }
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_mu<<<nb, kAB, 0, cx.stream>>>(P, phi, mub, g, w, gamma, phib, partials);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * (P.fe_kind == VSV_HELFRICH ? 6 : 4) * (double)n);
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_mu_finalize<<<1, kAB, 0, cx.stream>>>(P, partials, (int)nb, acc,
                                              area && P.fe_kind == VSV_HELFRICH && P.k_area != 0.0);
  cx.after(VSV_KCLASS_ADJOINT);
}

void launch_adj_area(Ctx& cx, const AdjParams& P, const double* phi, const double* coef,
                     const double* add, double add_scale, double* phib) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_area<<<nb_(n), kAB, 0, cx.stream>>>(P, phi, coef, add, add_scale, phib);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * 3 * (double)n);
}

void launch_adj_update(Ctx& cx, const AdjParams& P, double* phib, const double* phi,
                       Comp3<const double> psi, Comp3<const double> v0, double dt, Comp3<double> s,
                       Comp3<double> vb, double* mub, Comp3<double> psib, double* partials,
                       double* acc) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const unsigned nb = nb_(n);
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_update1<<<nb, kAB, 0, cx.stream>>>(P, phib, phi, psi, v0, dt, s, vb, mub, partials);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * 12 * (double)n);   // phib, phi, psi'(3) read; s, vb (6), mub written
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_lambda_finalize<<<1, kAB, 0, cx.stream>>>(P, partials, (int)nb, dt, acc);
  cx.after(VSV_KCLASS_ADJOINT);
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_update2<<<nb, kAB, 0, cx.stream>>>(P, phib, Comp3<const double>{{s.p[0], s.p[1], s.p[2]}},
                                           Comp3<const double>{{vb.p[0], vb.p[1], vb.p[2]}}, dt, acc,
                                           psib);
  cx.after(VSV_KCLASS_ADJOINT, 8.0 * 11 * (double)n);   // phib, s, vb read; phib, psib written
}

void launch_adj_axpby(Ctx& cx, double* z, double a, const double* x, double b, const double* y,
                      long long n) {
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_axpby<<<nb_(n), kAB, 0, cx.stream>>>(z, x, y, n, a, b);
  cx.after(VSV_KCLASS_ADJOINT, 24.0 * (double)n);
}

void launch_adj_scale(Ctx& cx, const double* y, double* x, long long n, double a) {
  cx.before(VSV_KCLASS_ADJOINT);
  k_adj_scale<<<nb_(n), kAB, 0, cx.stream>>>(y, x, n, a);
  cx.after(VSV_KCLASS_ADJOINT, 16.0 * (double)n);
}

}  // namespace vsv
