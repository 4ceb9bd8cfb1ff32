// Host-side internals shared by the kernel files and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/vsv.h"
#include "common.cuh"

namespace vsv {

// An encoded TMA tensor map (the driver's opaque 128-byte object) of one
// FP32 field of extent n[0] x n[1] x n[2] with boxes of kTX x rows x 1.
struct TensorMapEntry {
  const void* ptr;
  int n[3];
  int rows;
  alignas(64) unsigned char map[128];
};

// Launch context: the caller's stream, a launch counter and optional CUDA
// event brackets around every launch of one kernel class.
struct Ctx {
  cudaStream_t stream = nullptr;
  int sms = 148;                 // multiprocessors of the grid's device (set at create)
  int tiled = 1;                 // use the tiled transfer kernels (solver variants 0 and 2)
  int ragged = 1;                // also with partial edge tiles (solver variant 0)
  int* status = nullptr;         // device flag word (bounded waits report timeouts here)
  // > 0: the z-marching kernels pick their z-chunks as for this many
  // components (one-component launches of the component streams, which run
  // side by side, keep the chunks of the three-component launch)
  int chunk_comps = 0;
  // launch the kernels that begin with pdl_begin() with programmatic stream
  // serialisation (solver launch_overlap); never while events bracket a
  // kernel class, so that those brackets time one kernel alone
  int overlap = 1;
  std::vector<TensorMapEntry> tmaps;   // tensor maps encoded so far (fields do not move)
  long long launches = 0;
  int prof_class = -1;
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  int ev_used = 0;               // pairs recorded since enable
  long long prof_launches = 0;
  double prof_bytes = 0.0;
  double bytes_total = 0.0;      // algorithmic bytes of every tallied launch so far
  int pending = 0;

  bool match(int kclass) const {
    if (prof_class < 0 || kclass < 0) return false;
    if (prof_class == kclass) return true;
    return prof_class == VSV_KCLASS_SMOOTH && kclass == VSV_KCLASS_SMOOTH_FINE;
  }
  void before(int kclass) {
    ++launches;
    pending = 0;
    if (match(kclass) && 2 * ev_used + 1 < (int)ev.size()) {
      cudaEventRecord(ev[2 * ev_used], stream);
      pending = 1;
    }
  }
  // bytes: the launch's algorithmic memory traffic (0 where not tallied)
  void after(int kclass, double bytes = 0.0) {
    bytes_total += bytes;
    if (pending) {
      cudaEventRecord(ev[2 * ev_used + 1], stream);
      ++ev_used;
      ++prof_launches;
      prof_bytes += bytes;
      pending = 0;
    }
  }
};

// Launch of kernel `kern` on cx.stream (grid, block, dynamic shared memory,
// arguments as for <<< >>>).  With cx.overlap the launch carries programmatic
// stream serialisation: the kernel may be scheduled while the previous kernel
// of the stream finishes and waits for it in pdl_begin(), which must be its
// first statement.  Errors are left for cudaGetLastError, as with <<< >>>.
template <class... P, class... A>
void launch_k(const Ctx& cx, void (*kern)(P...), dim3 grid, dim3 block, size_t smem, A&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = cx.stream;
  cfg.attrs = at;
  cfg.numAttrs = (cx.overlap && cx.prof_class < 0) ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// FP64 block reduction (all threads get the block total); blockDim.x must be a
// multiple of 32 and at most 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_buf[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_buf[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? red_buf[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  if (threadIdx.x == 0) red_buf[0] = t;
  __syncthreads();
  const double r = red_buf[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double redm_buf[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) redm_buf[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? redm_buf[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  __syncthreads();
  if (threadIdx.x == 0) redm_buf[0] = t;
  __syncthreads();
  const double r = redm_buf[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- Poisson launchers (mg.cu)
template <class T>
void launch_rb_sweep(Ctx& cx, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, int color,
                     double omega, double h2, int kclass);
template <class T>
void launch_resid_restrict(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Rhs3<T> R,
                           Comp3<T> RC, int ncomp, bool exact);
template <class T>
void launch_prolong_add(Ctx& cx, const Level& F, const Level& C, Comp3<T> X, Comp3<T> E, int ncomp);
template <class T>
void launch_zero(Ctx& cx, Comp3<T> X, long long n, int ncomp);
// Y += a X
template <class T>
void launch_axpy(Ctx& cx, Comp3<T> Y, Comp3<T> X, double a, long long n, int ncomp);
// first guess of order 0..2 from (A, B, C) = (x^n, x^{n-1}, x^{n-2}), written into C
template <class T>
void launch_extrapolate_rot(Ctx& cx, Comp3<T> A, Comp3<T> B, Comp3<T> C, long long n, int ncomp,
                            int order);
template <class T>
bool launch_coarse_solve(Ctx& cx, const Level& L, Comp3<T> E, Comp3<T> R, int ncomp, int sweeps,
                         double h2);
template <class T>
void launch_resid_norm(Ctx& cx, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, bool exact,
                       double* partials, int nblocks, Scalars* S);

// Lower part of a V-cycle (levels first .. last) run by one CTA per component
// in shared memory: E (level first) <- approximate solution of L e = R.
struct CoarseCycle {
  Level lv[kMaxLevels];
  int first, last;
  int nu1, nu2, coarse_sweeps;
  double omega;                // relaxation weight of the nu1 / nu2 sweeps (coarsest: 1)
  double h2[kMaxLevels];       // 1 / inv_h2 of each level (rounded to T in the kernel)
  long long off[kMaxLevels];   // element offset of level l's (e, r) pair
  long long total;             // elements of shared memory
};
constexpr size_t kCoarseCycleSmem = 200 * 1024;
template <class T>
bool launch_coarse_vcycle(Ctx& cx, const CoarseCycle& CC, Comp3<T> E, Comp3<T> R, int ncomp);

// Bounded grid-wide barrier of a cooperative launch.  count: arrival
// counter in device memory, zeroed before each launch; status: device flag
// word, bit kSyncTimeout set when a CTA's wait exceeded limit_ns
// nanoseconds (the global timer); extra: arrivals expected beyond the
// grid's CTAs per barrier (0; a test sets it to make the wait run out).
constexpr int kSyncTimeout = 2;
// bit of the same word set when a wait of the fused sweep for its staged
// planes (bulk copies) exceeded one second
constexpr int kCopyTimeout = 4;
constexpr unsigned long long kSyncLimitNs = 1000000000ull;   // 1 s
struct GridBarrier {
  unsigned* count;
  int* status;
  unsigned long long limit_ns;
  unsigned extra;
};

// The levels first .. last of a V-cycle in one cooperative launch (mg.cu):
// levels first .. cc-1 grid-wide, levels cc .. last (cc <= last) as the
// one-CTA coarse cycle cc_plan.  e[first] <- correction for rhs r[first].
template <class T>
struct LowerCycle {
  Level lv[kMaxLevels];
  double h2[kMaxLevels];
  T* e[kMaxLevels][3];
  T* r[kMaxLevels][3];
  int first, cc, last;
  int ncomp, nu1, nu2, coarse_sweeps;
  double omega;
  CoarseCycle cc_plan;
  GridBarrier bar;
};
template <class T>
bool launch_lower_vcycle(Ctx& cx, const LowerCycle<T>& P);
// `rounds` bounded barriers of `blocks` co-resident CTAs (tests of the bound)
bool launch_barrier_probe(cudaStream_t s, GridBarrier B, int blocks, int rounds);
int barrier_probe_max_blocks(int sms);

// outer defect correction with double-word iterates (dc.cu)
void launch_defect_dw(Ctx& cx, const Level& L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                      Comp3<float> BL, Comp3<float> OUT, int ncomp, double* partials, int nblocks);
void launch_update_dw(Ctx& cx, Comp3<float> XH, Comp3<float> XL, Comp3<float> E, long long n,
                      int ncomp);
// ragged: also levels that are not tile multiples (partial edge tiles)
int launch_defect_tiled(Ctx& cx, const Level& L, Comp3<float> XH, Comp3<float> XL, Rhs3<float> R,
                        Comp3<float> BL, Comp3<float> OUT, int ncomp, double* partials,
                        int max_blocks, bool ragged);
// first guess of order 0..2 from (A, B, C) = (x^n, x^{n-1}, x^{n-2}), written into C
void launch_extrapolate_rot_dw(Ctx& cx, Comp3<float> AH, Comp3<float> AL, Comp3<float> BH,
                               Comp3<float> BL, Comp3<float> CH, Comp3<float> CL, long long n,
                               int ncomp, int order);
void launch_norm_finalize(Ctx& cx, const double* partials, int nblocks, int ncomp, Scalars* S);
// (YH, YL) += a (XH, XL), double-word
void launch_axpy_dw(Ctx& cx, Comp3<float> YH, Comp3<float> YL, Comp3<float> XH, Comp3<float> XL,
                    double a, long long n, int ncomp);

// tiled restriction / prolongation for tile-aligned levels halved on every
// axis (transfer.cu); false: not applicable, nothing launched
bool launch_restrict_tiled(Ctx& cx, const Level& F, const Level& C, Comp3<float> X,
                           Rhs3<float> R, Comp3<float> RC, int ncomp);
bool launch_prolong_tiled(Ctx& cx, const Level& F, const Level& C, Comp3<float> X, Comp3<float> E,
                          int ncomp);

// fused single-pass red-black sweep (smooth.cu)
// ragged: also levels whose extents are not multiples of the tile (partial
// edge tiles), where enough of the tiles' cells exist
bool fused_sweep_ok(const Level& L, bool ragged);
// omega: relaxation weight of the sweep (1: Gauss-Seidel)
void launch_rbgs_fused(Ctx& cx, const Level& L, Comp3<float> A, Comp3<float> B, Rhs3<float> R,
                       int ncomp, int zchunk, int kclass, bool zero_in,
                       const Comp3<float>* upd_hi = nullptr, const Comp3<float>* upd_lo = nullptr,
                       float omega = 1.f);
// Check of the bound of the fused sweep's waits for staged planes (no copy
// issued; every wait gives up after limit_ns): false unless L is tile-aligned.
bool launch_copy_wait_probe(Ctx& cx, const Level& L, Comp3<float> B, Rhs3<float> R,
                            unsigned probe_tx, unsigned long long limit_ns);

// ---------------------------------------------------------------- phase-field (phase.cu)
struct PhaseParams {
  int nx, ny, nz, zper;
  double h, inv_h, inv_h2;
  int fe_kind;
  double sigma, eps, cf2;       // cf2 = prefactor of the Helfrich mu
  double beta_t;                // Helfrich with tension sigma: mu += beta_t g, beta_t = sigma c_A / eps
  double mobility, inv_eta;
  // the same coefficients as double-word FP32 pairs (hi, lo) for the mixed path
  float ih2_hi, ih2_lo, cf2_hi, cf2_lo;
  float e2ih_hi, e2ih_lo, sgih_hi, sgih_lo;   // eps^2 / h^2 and sigma / h^2
  float src_hi, src_lo;   // (1 / 2h)^2 / eta: scale of the raw-difference cross product
  float ag_hi, ag_lo, aw_hi, aw_lo;   // area density: c_A eps/2 (1/2h)^2 and c_A / (4 eps)
  float bt_hi, bt_lo;                                              // beta_t
  // wall velocity on the wall nodes: [0] y = 0 wall, [1] y = H, [2] z = 0, [3] z = H
  double vwall[4][3];
};

template <class T>
void launch_phi_update(Ctx& cx, const PhaseParams& P, const T* phi, const T* mu, Comp3<T> psi,
                       Comp3<T> v0, const Scalars* S, T dt, T* phi_out);
// V, A (and the multipliers) of phi into S.  On the mixed path with g and
// g_lo given and x extents in 4-cell groups, the same pass also stores the
// Helfrich g of phi there; returns whether it did.
template <class T>
bool launch_reduce_va(Ctx& cx, const PhaseParams& P, const T* phi, const T* phi_lo,
                      double* partials, int nblocks, Scalars* S, int init, float* g = nullptr,
                      float* g_lo = nullptr);
// Mixed path: phi carried as FP32 pairs (hi, lo); mu and g computed with
// double-word FP32 arithmetic, mu rounded to FP32.
void launch_phi_update_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo,
                          const float* mu, Comp3<float> psi, Comp3<float> v0, const Scalars* S,
                          float dt, float* out, float* out_lo);
// g_ready: the Helfrich g of phi is already in g, g_lo (launch_reduce_va)
void launch_mu_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo, float* g,
                  float* g_lo, float* mu, float* mu_lo, const Scalars* S, bool g_ready = false);
void launch_source_ff(Ctx& cx, const PhaseParams& P, const float* phi, const float* phi_lo,
                      const float* mu, const float* mu_lo, Comp3<float> s_omega, Comp3<float> f,
                      Comp3<float> f_lo);
void launch_split_ff(Ctx& cx, const double* in, float* hi, float* lo, long long n);
void launch_merge_ff(Ctx& cx, const float* hi, const float* lo, double* out, long long n);
template <class T>
void launch_mu(Ctx& cx, const PhaseParams& P, const T* phi, T* g, T* mu, const Scalars* S);
template <class T>
void launch_source(Ctx& cx, const PhaseParams& P, const T* phi, const T* mu, Comp3<T> s_omega,
                   Comp3<T> f);
template <class T>
void launch_velocity(Ctx& cx, const PhaseParams& P, Comp3<T> psi, Comp3<T> psi_lo, Comp3<T> v0,
                     Comp3<T> v);
// Diagnostic partial sums; out has kDiagQ doubles per block.
constexpr int kDiagQ = 16;
// vel_lo, om_lo, ps_lo: low words of the double-word velocity, omega' and
// psi' of the mixed path (null pointers on the FP64 path)
template <class T>
void launch_diag(Ctx& cx, const PhaseParams& P, const T* phi, const T* phi_lo, const T* g,
                 const T* g_lo, Comp3<T> vel, Comp3<T> vel_lo, Comp3<T> omega, Comp3<T> om_lo,
                 Comp3<T> psi, Comp3<T> ps_lo, Comp3<const double> psi0_ring,
                 Comp3<const double> v0d, T* sigma_t, double* partials, int nblocks, double* out);
template <class T>
void launch_stress_profile(Ctx& cx, const PhaseParams& P, Comp3<T> vel, Comp3<T> vel_lo,
                           double* out);
// Mixed path: v = v0 + curl psi' in FP64 from the double-word psi' and the
// FP64 base-flow table, stored as a double word (v, v_lo).
void launch_velocity_dw(Ctx& cx, const PhaseParams& P, Comp3<float> psi, Comp3<float> psi_lo,
                        Comp3<const double> v0d, Comp3<float> v, Comp3<float> v_lo);
template <class Tin, class Tout>
void launch_convert(Ctx& cx, const Tin* in, Tout* out, long long n);
template <class T>
void launch_full_field(Ctx& cx, const PhaseParams& P, const T* pert, const T* lo,
                       const double* table2d, int ring, T* out);
void launch_full_field_dw(Ctx& cx, const PhaseParams& P, const float* hi, const float* lo,
                          const double* tab, int ring, double* out);
template <class T>
void launch_scale_copy(Ctx& cx, const T* in, T* out, long long n, double a);

// base-flow helpers (FP64 2-D tables; phase.cu)
void launch_duct_ring(Ctx& cx, int ny, int nz, double h, const double* u0, const double* chi,
                      double* om_ring_y, double* om_ring_z, double* ps_ring_y, double* ps_ring_z);
void launch_ring_boundary_rhs(Ctx& cx, int ny, int nz, double h, const double* ring, double scale_in,
                              const double* in, double* out);
void launch_ring_fill_interior(Ctx& cx, int ny, int nz, const double* interior, double* ring);
// Time-dependent walls: the current base-flow tables as the combination
// s_0(t) B_0 + s_1(t) B_1 of the unit-speed tables B_w at the device time
// *t_dev (advanced by dt, or set to t_set when set_time), with the typed
// copies the kernels read (T: v0t, s_om_t, and s_ps_neg_t = -s_ps).
struct WallTables {
  int n_ring, n_tab;                       // (ny+2)(nz+2), ny nz
  const double* bom[2][3]; const double* bps[2][3];
  const double* bv0[2][3]; const double* bsom[2][3]; const double* bsps[2][3];
  double* om[3]; double* ps[3]; double* v0[3]; double* som[3]; double* sps[3];
  void* v0t[3]; void* somt[3]; void* spsnt[3];
  double s0[2], ramp[2], amp[2], freq[2], phase[2];
  double* t_dev;
};
template <class T>
void launch_wall_tables(Ctx& cx, const WallTables& W, double dt, bool set_time, double t_set);

void launch_base_derived(Ctx& cx, int ny, int nz, int zper, double h, const double* om_ring[3],
                         const double* ps_ring[3], double* v0[3], double* s_om[3], double* s_ps[3]);
double device_max_abs(Ctx& cx, const double* x, long long n, double* scratch);
void launch_fill(Ctx& cx, double* x, long long n, double v);

// ---------------------------------------------------------------- discrete adjoint (adjoint.cu)
// Coefficients of the adjoint kernels (FP64 throughout).
struct AdjParams {
  int nx, ny, nz, zper;
  double h, hih, ih2, h3;            // h, 1 / (2h), 1 / h^2, h^3
  int fe_kind;
  double sigma, eps, e2;             // e2 = eps^2
  double cf2, cf2_per_kappa;         // prefactor of the bending mu, and per unit kappa
  double beta;                       // Helfrich tension coefficient sigma c_A / eps
  double inv_eta, mobility, k_vol, k_area;
};
// slots of the device accumulator array (doubles)
constexpr int kAccKappa = 0;     // dJ / dkappa
constexpr int kAccSigma = 1;     // dJ / dsigma
constexpr int kAccV0 = 2;        // adjoint of the constant V0
constexpr int kAccA0 = 3;        // adjoint of the constant A0
constexpr int kAccAreaCoef = 4;  // gammabar K_A c_g of the current step
constexpr int kAccPhiAdd = 5;    // constant added to phibar by the volume penalty
constexpr int kAccGamma = 6;     // gammabar of the current step
constexpr int kAccLambda = 7;    // lambdabar of the current step
constexpr int kAccCount = 8;
int adj_blocks(long long ncells);   // partial-sum blocks of one reduction (3 doubles each)
void launch_adj_source(Ctx& cx, const AdjParams& P, const double* phi, const double* mu,
                       Comp3<const double> fb, Comp3<double> ab, Comp3<double> bb);
void launch_adj_divt(Ctx& cx, const AdjParams& P, Comp3<const double> A, double* outA,
                     Comp3<const double> B, double* outB);
void launch_adj_mu(Ctx& cx, const AdjParams& P, const double* phi, const double* mub,
                   const double* gamma, double* g, double* w, double* phib, double* partials,
                   double* acc, bool area);
// phib += (*coef) dA/dphi + add_scale (*add); null pointers read as 0
void launch_adj_area(Ctx& cx, const AdjParams& P, const double* phi, const double* coef,
                     const double* add, double add_scale, double* phib);
void launch_adj_update(Ctx& cx, const AdjParams& P, double* phib, const double* phi,
                       Comp3<const double> psi, Comp3<const double> v0, double dt, Comp3<double> s,
                       Comp3<double> vb, double* mub, Comp3<double> psib, double* partials,
                       double* acc);
void launch_adj_scale(Ctx& cx, const double* y, double* x, long long n, double a);
// z = a x + b y (n doubles)
void launch_adj_axpby(Ctx& cx, double* z, double a, const double* x, double b, const double* y,
                      long long n);

}  // namespace vsv
