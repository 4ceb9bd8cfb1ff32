// C ABI of the vorticity--stream-vector library (declared in include/vsv.h):
// workspace layout, multigrid / SOR drivers, base-flow set-up and the time
// step of main-text eqs. gen2, gen1, gen3 in the segregated order of the
// numerical-implementation section.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace vsv;

struct vsv_grid {
  Ctx cx;
  int nx = 0, ny = 0, nz = 0;
  double h = 1.0;
  int prec = VSV_MIXED;
  size_t tsize = 4;
  long long N = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;

  vsv_flow_params flow{};
  vsv_fe_params fe{};
  vsv_solver_params sol{};
  bool flow_set = false, phi_set = false, phase_stale = false;

  void* phi[2] = {nullptr, nullptr};
  float* phi_lo[2] = {nullptr, nullptr};   // mixed path: low words of phi
  int cur = 0;
  void* mu = nullptr;
  void* g = nullptr;
  float* g_lo = nullptr;
  float* mu_lo = nullptr;    // mixed path: low words of mu and of the source f
  float* f_lo[3] = {};
  void* f[3] = {};
  void* om[3] = {};
  void* ps[3] = {};
  // the two previous steps' solutions (initial-guess extrapolation); the
  // three buffers of a field rotate instead of being copied
  void* om_prev[3] = {};
  void* ps_prev[3] = {};
  void* om_prev2[3] = {};
  void* ps_prev2[3] = {};
  int hist = 0;              // how many of those previous solutions are valid (0..2)
  // mixed path: low words of the double-word iterates, the FP32 correction e
  // and defect r of the outer defect correction
  float* om_lo[3] = {};
  float* ps_lo[3] = {};
  float* om_prev_lo[3] = {};
  float* ps_prev_lo[3] = {};
  float* om_prev2_lo[3] = {};
  float* ps_prev2_lo[3] = {};
  float* e0[3] = {};
  float* r0[3] = {};
  void* stage_a = nullptr;   // N * 8 bytes
  void* stage_b = nullptr;   // N * 8 bytes
  // mixed path: staging of the asynchronous FP64 phi transfers (N * 8 bytes
  // each), used by nothing else, the copy streams that move them and the
  // events that order them against the grid's stream
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  cudaStream_t io_in = nullptr, io_out = nullptr;
  cudaEvent_t in_ready = nullptr, in_free = nullptr, out_ready = nullptr, out_free = nullptr;
  void* mg_e[kMaxLevels][3] = {};
  void* mg_r[kMaxLevels][3] = {};
  void* mg_t[kMaxLevels][3] = {};  // ping-pong partner of the fused sweep (mixed path)
  long long mg_cap[kMaxLevels] = {};
  int mg_nlev_cap = 0;

  double* om_ring[3] = {};   // (ny+2)(nz+2) FP64, ring + interior body-free values
  double* ps_ring[3] = {};
  double* v0d[3] = {};       // ny nz FP64
  double* s_om_d[3] = {};
  double* s_ps_d[3] = {};
  void* v0t[3] = {};         // typed copies (T)
  void* s_om_t[3] = {};
  void* s_ps_neg_t[3] = {};
  // time-dependent walls: the base-flow tables of unit wall speeds (basis 0:
  // the y = 0 wall or the Poiseuille speed, basis 1: the y = H wall), of
  // which the current tables are the combination at the device time t_dev
  double* wb_om[2][3] = {};
  double* wb_ps[2][3] = {};
  double* wb_v0[2][3] = {};
  double* wb_som[2][3] = {};
  double* wb_sps[2][3] = {};
  double* t_dev = nullptr;
  bool motion_on = false;
  vsv_wall_motion motion{};
  double* su0 = nullptr;     // 2-D set-up scratch (ny nz each)
  double* schi = nullptr;
  double* sx = nullptr;
  double* sb = nullptr;

  double* partials = nullptr;
  int red_blocks = 0;
  Scalars* S = nullptr;
  double* dout = nullptr;     // kDiagQ doubles
  double* profile = nullptr;  // ny doubles
  double* scratch1 = nullptr;

  std::vector<Level> flow_levels;
  // inertial variant: the hierarchy of L_h - s, s = rho / (eta dt), for the
  // vorticity solves, rebuilt when dt changes
  std::vector<Level> omega_levels;
  double omega_dt = 0.0;
  int* flag_host = nullptr;        // pinned copy of the device non-finite flag
  int* flag_dev = nullptr;         // its device address (mapped)
  // component-parallel flow solves: the first component of the
  // per-component scratch the current solve uses, the two extra streams the
  // components 1 and 2 run on, and the events that fork and join them
  int c0 = 0;
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[2] = {nullptr, nullptr};
  // the step's first guesses, extrapolated on component stream 0 while the
  // grid's stream runs the phase kernels: done (this step) and their event
  bool guesses_done = false;
  cudaEvent_t ext_ev = nullptr;
  unsigned* bar_count = nullptr;   // arrival counter of the persistent V-cycle's grid barriers
  cudaEvent_t flag_event = nullptr;
  bool flag_pending = false;
  int last_cycles[2] = {0, 0};
  double last_relres[2] = {-1.0, -1.0};
  double time = 0.0;
  long long steps = 0;
  std::string err;
};

namespace {

const size_t kAlign = 256;

// Default relaxation weight of the multigrid smoothing sweeps.  Red-black
// SOR smoothing near 1.25-1.3 contracts a V(2,2)-cycle of this cell-centred
// hierarchy (7-point operator, averaging restriction, trilinear
// prolongation, linear wall closure on coarse levels) by about 0.03 per
// cycle asymptotically, against about 0.1 for plain Gauss-Seidel
// smoothing, at no extra memory traffic in the fused sweep; two or three
// cycles from an extrapolated first guess came out most accurate at 1.3.
const double kDefaultMgWeight = 1.3;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Upper bound of the multigrid hierarchy: halve every axis longer than one
// cell while all of them are even (any boundary choice coarsens no further).
int plan_levels(int nx, int ny, int nz, long long* cells) {
  int n[3] = {nx, ny, nz};
  int L = 0;
  cells[L++] = (long long)nx * ny * nz;
  while (L < kMaxLevels) {
    bool ok = true, any = false;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1) {
        any = true;
        if (n[a] % 2) ok = false;
      }
    if (!ok || !any) break;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1) n[a] /= 2;
    cells[L++] = (long long)n[0] * n[1] * n[2];
  }
  return L;
}

int reduction_blocks(long long N) {
  long long b = (N + kBlock - 1) / kBlock;
  return (int)std::max(1LL, std::min(b, 1216LL));
}

// Carve the workspace (g == nullptr: only measure).
size_t carve(int nx, int ny, int nz, int prec, vsv_grid* g, char* base) {
  const size_t ts = (prec == VSV_FP64) ? 8 : 4;
  const long long N = (long long)nx * ny * nz;
  const long long N2 = (long long)ny * nz;
  const long long R2 = (long long)(ny + 2) * (nz + 2);
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = base ? (void*)(base + off) : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  auto tf = [&](long long n) { return take((size_t)n * ts); };
  auto df = [&](long long n) { return (double*)take((size_t)n * 8); };
  void* p;
  p = tf(N); if (g) g->phi[0] = p;
  p = tf(N); if (g) g->phi[1] = p;
  p = tf(N); if (g) g->mu = p;
  p = tf(N); if (g) g->g = p;
  if (prec == VSV_MIXED) {
    p = take((size_t)N * 4); if (g) g->phi_lo[0] = (float*)p;
    p = take((size_t)N * 4); if (g) g->phi_lo[1] = (float*)p;
    p = take((size_t)N * 4); if (g) g->g_lo = (float*)p;
    p = take((size_t)N * 4); if (g) g->mu_lo = (float*)p;
    for (int c = 0; c < 3; ++c) {
      p = take((size_t)N * 4); if (g) g->f_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->om_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->ps_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->om_prev_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->ps_prev_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->om_prev2_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->ps_prev2_lo[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->e0[c] = (float*)p;
      p = take((size_t)N * 4); if (g) g->r0[c] = (float*)p;
    }
  }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->f[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->om[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->ps[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->om_prev[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->ps_prev[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->om_prev2[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N); if (g) g->ps_prev2[c] = p; }
  p = take((size_t)N * 8); if (g) g->stage_a = p;
  p = take((size_t)N * 8); if (g) g->stage_b = p;
  if (prec == VSV_MIXED) {
    p = take((size_t)N * 8); if (g) g->stage_in = p;
    p = take((size_t)N * 8); if (g) g->stage_out = p;
  }
  long long cells[kMaxLevels];
  const int nl = plan_levels(nx, ny, nz, cells);
  if (g) g->mg_nlev_cap = nl;
  for (int l = 1; l < nl; ++l) {
    for (int c = 0; c < 3; ++c) { p = tf(cells[l]); if (g) g->mg_e[l][c] = p; }
    for (int c = 0; c < 3; ++c) { p = tf(cells[l]); if (g) g->mg_r[l][c] = p; }
    if (g) g->mg_cap[l] = cells[l];
  }
  if (prec == VSV_MIXED)
    for (int l = 0; l < nl; ++l)
      for (int c = 0; c < 3; ++c) { p = tf(cells[l]); if (g) g->mg_t[l][c] = p; }
  for (int c = 0; c < 3; ++c) { double* d = df(R2); if (g) g->om_ring[c] = d; }
  for (int c = 0; c < 3; ++c) { double* d = df(R2); if (g) g->ps_ring[c] = d; }
  for (int c = 0; c < 3; ++c) { double* d = df(N2); if (g) g->v0d[c] = d; }
  for (int c = 0; c < 3; ++c) { double* d = df(N2); if (g) g->s_om_d[c] = d; }
  for (int c = 0; c < 3; ++c) { double* d = df(N2); if (g) g->s_ps_d[c] = d; }
  for (int c = 0; c < 3; ++c) { p = tf(N2); if (g) g->v0t[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N2); if (g) g->s_om_t[c] = p; }
  for (int c = 0; c < 3; ++c) { p = tf(N2); if (g) g->s_ps_neg_t[c] = p; }
  double* d;
  d = df(N2); if (g) g->su0 = d;
  d = df(N2); if (g) g->schi = d;
  d = df(N2); if (g) g->sx = d;
  d = df(N2); if (g) g->sb = d;
  const int rb = reduction_blocks(N);
  d = df((long long)rb * 32); if (g) { g->partials = d; g->red_blocks = rb; }
  p = take(sizeof(Scalars)); if (g) g->S = (Scalars*)p;
  d = df(kDiagQ); if (g) g->dout = d;
  d = df(ny); if (g) g->profile = d;
  d = df(8); if (g) g->scratch1 = d;
  p = take(sizeof(unsigned)); if (g) g->bar_count = (unsigned*)p;
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 3; ++c) {
      d = df(R2); if (g) g->wb_om[b][c] = d;
      d = df(R2); if (g) g->wb_ps[b][c] = d;
      d = df(N2); if (g) g->wb_v0[b][c] = d;
      d = df(N2); if (g) g->wb_som[b][c] = d;
      d = df(N2); if (g) g->wb_sps[b][c] = d;
    }
  d = df(1); if (g) g->t_dev = d;
  return off;
}

bool valid_shape(int nx, int ny, int nz) {
  return nx >= 1 && ny >= 2 && nz >= 1 && (long long)nx * ny * nz <= (1LL << 33);
}

vsv_status fail(vsv_grid* g, vsv_status s, const char* fmt, const char* detail = "") {
  if (g) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail);
    g->err = buf;
  }
  return s;
}

// Status of the device flag word: bit 1 non-finite phi, bit kSyncTimeout a
// grid barrier of the persistent V-cycle whose wait ran out, bit
// kCopyTimeout a fused sweep whose staged planes did not arrive in time
// (the sweep's result is then unusable; the flag stays set).
vsv_status flag_status(vsv_grid* g, int flag) {
  if (flag & 1) return fail(g, VSV_ENONFINITE, "non-finite phi%s");
  if (flag & kSyncTimeout)
    return fail(g, VSV_ECUDA, "a grid barrier of the persistent multigrid launch ran out of time%s");
  if (flag & kCopyTimeout)
    return fail(g, VSV_ECUDA, "a wait of the fused sweep for its staged planes ran out of time%s");
  return VSV_OK;
}

// The step's status word into the handle's page-locked, mapped host word.
// A kernel writes it rather than a copy, so it does not queue behind large
// transfers on the copy engines (an asynchronous export of phi, say).
__global__ void k_flag_out(const int* __restrict__ flag, int* host_flag) {
  *reinterpret_cast<volatile int*>(host_flag) = *flag;
  __threadfence_system();
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(g, VSV_ECUDA, #call ": %s", cudaGetErrorString(e_)); \
  } while (0)

#define CKL()                                                                          \
  do {                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess) return fail(g, VSV_ECUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
  } while (0)

bool z_periodic(const vsv_grid* g) {
  return g->flow.kind == VSV_COUETTE || g->flow.kind == VSV_POISEUILLE_PLANAR;
}

// Multigrid levels for per-axis periodic flags: all active axes are halved
// together while every active extent is even (periodic extents must stay
// even); coarse wall closure alpha_l = (2^l - 1) / (2^l + 1).
void set_reciprocals(Level& L) {
  const int d2 = 2 * (L.act[0] + L.act[1] + L.act[2]);
  for (int q = 0; q < 7; ++q) {
    const double cd = (double)d2 + L.alpha * q + L.sh2;
    const float cf = (float)d2 + L.alphaf * (float)q + L.sh2f;
    L.rcd[q] = cd > 0 ? 1.0 / cd : 0.0;
    L.rcf[q] = cf > 0 ? 1.0f / cf : 0.0f;
    L.cdh[q] = (float)cd;
    L.cdl[q] = (float)(cd - (double)L.cdh[q]);
  }
}

// shift: s of the operator L_h - s (0 for the Poisson problems)
std::vector<Level> build_levels(int nx, int ny, int nz, double h, const int per[3], int max_levels,
                                int cap_levels, double shift = 0.0) {
  std::vector<Level> lv;
  Level L{};
  L.n[0] = nx; L.n[1] = ny; L.n[2] = nz;
  for (int a = 0; a < 3; ++a) {
    L.per[a] = per[a];
    L.act[a] = !(per[a] && L.n[a] == 1);
  }
  L.alpha = 0.0;
  L.inv_h2 = 1.0 / (h * h);
  L.alphaf = 0.f;
  L.inv_h2f = (float)L.inv_h2;
  L.sh2 = shift * h * h;
  L.sh2f = (float)L.sh2;
  set_reciprocals(L);
  lv.push_back(L);
  const int maxl = std::min(std::max(max_levels, 1), cap_levels);
  while ((int)lv.size() < maxl) {
    const Level& P = lv.back();
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      if (!P.act[a]) continue;
      if (P.n[a] < 2 || P.n[a] % 2) ok = false;
      else if (P.per[a] && (P.n[a] / 2) % 2) ok = false;
    }
    bool any = false;
    for (int a = 0; a < 3; ++a) any |= (P.act[a] && P.n[a] > 1);
    if (!ok || !any) break;
    Level C = P;
    for (int a = 0; a < 3; ++a)
      if (P.act[a] && P.n[a] > 1) C.n[a] = P.n[a] / 2;
    const int l = (int)lv.size();
    const double p2 = std::ldexp(1.0, l);
    C.alpha = (p2 - 1.0) / (p2 + 1.0);
    C.inv_h2 = 1.0 / (h * h * p2 * p2);
    C.alphaf = (float)C.alpha;
    C.inv_h2f = (float)C.inv_h2;
    C.sh2 = shift * h * h * p2 * p2;
    C.sh2f = (float)C.sh2;
    set_reciprocals(C);
    lv.push_back(C);
  }
  return lv;
}

double sor_weight(const Level& L) {
  double lam = 0.0;
  int d = 0;
  for (int a = 0; a < 3; ++a) {
    if (!L.act[a]) continue;
    ++d;
    if (!L.per[a]) lam += 2.0 - 2.0 * std::cos(M_PI / (L.n[a] + 1.0));
  }
  if (d == 0) return 1.0;
  const double rho = 1.0 - lam / (2.0 * d);
  return 2.0 / (1.0 + std::sqrt(std::max(0.0, 1.0 - rho * rho)));
}

Comp3<const double> ring3(double* const p[3]) { return Comp3<const double>{{p[0], p[1], p[2]}}; }

template <class T>
Comp3<T> comp3(void* a, void* b, void* c) {
  return Comp3<T>{{(T*)a, (T*)b, (T*)c}};
}

// The velocity v = v0 + curl psi' for the observables and the field
// exports, written over the source buffer f (scratch between steps): FP64
// values on the FP64 path, double words (f, f_lo) formed in FP64 on the
// mixed path.  *VL gets the low words (null pointers on the FP64 path).
template <class T>
void output_velocity(vsv_grid* g, const PhaseParams& P, Comp3<T>* V, Comp3<T>* VL) {
  *V = comp3<T>(g->f[0], g->f[1], g->f[2]);
  if constexpr (std::is_same<T, float>::value) {
    *VL = comp3<float>(g->f_lo[0], g->f_lo[1], g->f_lo[2]);
    launch_velocity_dw(g->cx, P, comp3<float>(g->ps[0], g->ps[1], g->ps[2]),
                       comp3<float>(g->ps_lo[0], g->ps_lo[1], g->ps_lo[2]), ring3(g->v0d), *V,
                       *VL);
  } else {
    *VL = Comp3<T>{{nullptr, nullptr, nullptr}};
    launch_velocity<T>(g->cx, P, comp3<T>(g->ps[0], g->ps[1], g->ps[2]),
                       Comp3<T>{{nullptr, nullptr, nullptr}},
                       comp3<T>(g->v0t[0], g->v0t[1], g->v0t[2]), *V);
  }
}

// Low words of omega' and psi' (mixed path) for the observables.
template <class T>
Comp3<T> om_low(vsv_grid* g) {
  if constexpr (std::is_same<T, float>::value) return comp3<float>(g->om_lo[0], g->om_lo[1], g->om_lo[2]);
  else return Comp3<T>{{nullptr, nullptr, nullptr}};
}
template <class T>
Comp3<T> ps_low(vsv_grid* g) {
  if constexpr (std::is_same<T, float>::value) return comp3<float>(g->ps_lo[0], g->ps_lo[1], g->ps_lo[2]);
  else return Comp3<T>{{nullptr, nullptr, nullptr}};
}

// ---------------------------------------------------------------- solvers
// Components c0, c0 + 1, ... of a per-component buffer array (a solve of
// fewer than three components from component c0 uses the leading ones).
template <class T, class P>
Comp3<T> cview(P* const a[3], int c0) {
  return Comp3<T>{{(T*)a[c0], c0 + 1 < 3 ? (T*)a[c0 + 1] : nullptr,
                   c0 + 2 < 3 ? (T*)a[c0 + 2] : nullptr}};
}

// Relaxation weight of the multigrid smoothing sweeps (all levels but the
// coarsest, which is solved by plain Gauss-Seidel sweeps): omega_mg, with 0
// meaning 1.
double mg_weight(const vsv_grid* g) { return g->sol.omega_mg > 0.0 ? g->sol.omega_mg : 1.0; }

// nu red-black sweeps on level l: the fused single-pass kernel (ping-pong
// with the level's scratch) where it applies, else the per-colour kernels.
// x_zero: X is known to be zero (a correction from e = 0): the first fused
// sweep then does not read it, and the per-colour path zeroes it first.
// uh / ul (FP32 storage only): a double-word iterate to which the result is
// to be added; returns true if the last fused sweep did that (X then does not
// hold the result), false if the caller still has to.
template <class T>
bool smooth(vsv_grid* g, const Level& L, int l, Comp3<T> X, Rhs3<T> R, int ncomp, int nu,
            bool x_zero, const Comp3<float>* uh = nullptr, const Comp3<float>* ul = nullptr) {
  const double h2 = 1.0 / L.inv_h2;
  const int kc = (l == 0) ? VSV_KCLASS_SMOOTH_FINE : VSV_KCLASS_SMOOTH;
  const double w = mg_weight(g);
  if constexpr (std::is_same<T, float>::value) {
    if (g->sol.variant != 1 && fused_sweep_ok(L, g->sol.variant == 0) && g->mg_t[l][0] && nu >= 2) {
      Comp3<float> Tt = cview<float>(g->mg_t[l], g->c0);
      const int zchunk = 0;   // chosen by the launcher
      const bool fuse_upd = uh && ul && nu % 2 == 0;
      bool z = x_zero;
      for (int s = 0; s + 1 < nu; s += 2) {
        const bool last = s + 2 == nu;
        launch_rbgs_fused(g->cx, L, X, Tt, R, ncomp, zchunk, kc, z, nullptr, nullptr, (float)w);
        launch_rbgs_fused(g->cx, L, Tt, X, R, ncomp, zchunk, kc, false,
                          fuse_upd && last ? uh : nullptr, fuse_upd && last ? ul : nullptr,
                          (float)w);
        z = false;
      }
      if (nu % 2) {
        launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 0, w, h2, kc);
        launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 1, w, h2, kc);
      }
      return fuse_upd;
    }
  }
  if (x_zero) launch_zero<T>(g->cx, X, L.cells(), ncomp);
  for (int s = 0; s < nu; ++s) {
    launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 0, w, h2, kc);
    launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 1, w, h2, kc);
  }
  return false;
}

// Red-black sweeps on the coarsest level: the solver's coarse_sweeps, but no
// more than twice the level's longest extent (at least 4).  Gauss-Seidel on
// a level of a few cells converges in a few sweeps; on the 2 x 1 x 1 level
// of a 512 x 256 x 256 grid 4 sweeps give the same velocity as 24.
int coarsest_sweeps(const Level& L, int cap) {
  const int m = std::max(L.n[0], std::max(L.n[1], L.n[2]));
  return std::min(cap, std::max(4, 2 * m));
}

// Levels m .. last of hierarchy lv as a one-CTA coarse cycle plan (shared
// memory offsets of every level's (e, r) pair); false if they do not fit.
bool coarse_plan(const vsv_grid* g, const std::vector<Level>& lv, int m, CoarseCycle* CC,
                 size_t elem) {
  *CC = CoarseCycle{};
  CC->first = m;
  CC->last = (int)lv.size() - 1;
  CC->nu1 = g->sol.nu1;
  CC->nu2 = g->sol.nu2;
  CC->omega = mg_weight(g);
  CC->coarse_sweeps = coarsest_sweeps(lv.back(), g->sol.coarse_sweeps);
  long long off = 0;
  for (int q = m; q <= CC->last; ++q) {
    CC->lv[q] = lv[q];
    CC->h2[q] = 1.0 / lv[q].inv_h2;
    CC->off[q] = off;
    off += 2 * lv[q].cells();
  }
  CC->total = off;
  return (size_t)off * elem <= kCoarseCycleSmem;
}

// Should the levels from l down run as one cooperative launch?  Only when
// the solver asks for it (lower_cycle = 1) and where the levels do not all
// fit the one-CTA coarse cycle (which is then the cheaper single launch).
// It is not the default: measured on GB300 it is slower than the
// level-by-level kernels at every size tried (512 x 256 x 256: 16.7 ms per
// step from the 4.2 M-cell level, 15.0 from the 0.5 M-cell level, against
// 14.7 level by level; 256 x 128 x 128: 3.06 against 2.75 ms), because
// per-colour grid-wide sweeps move twice the bytes of the fused sweep and
// its grid barriers (about 1.45 us each) do not beat the launches they
// replace.
bool lower_cycle_wanted(const vsv_grid* g, const std::vector<Level>& lv, int l) {
  if (g->sol.lower_cycle != 1 || l + 1 >= (int)lv.size()) return false;
  CoarseCycle CC;
  return !coarse_plan(g, lv, l, &CC, g->prec == VSV_FP64 ? 8 : 4);
}

template <class T>
bool run_lower_cycle(vsv_grid* g, const std::vector<Level>& lv, int l, Comp3<T> E, Comp3<T> R,
                     int ncomp) {
  LowerCycle<T> P{};
  P.first = l;
  P.last = (int)lv.size() - 1;
  P.ncomp = ncomp;
  P.nu1 = g->sol.nu1;
  P.nu2 = g->sol.nu2;
  P.coarse_sweeps = coarsest_sweeps(lv.back(), g->sol.coarse_sweeps);
  P.omega = mg_weight(g);
  for (int q = l; q <= P.last; ++q) {
    P.lv[q] = lv[q];
    P.h2[q] = 1.0 / lv[q].inv_h2;
    for (int c = 0; c < 3; ++c) {
      P.e[q][c] = q == l ? E.p[c] : (T*)g->mg_e[q][c];
      P.r[q][c] = q == l ? R.p[c] : (T*)g->mg_r[q][c];
    }
  }
  // the one-CTA part: the first level below l from which the rest fits
  P.cc = P.last + 1;
  for (int m = l + 1; m <= P.last; ++m)
    if (coarse_plan(g, lv, m, &P.cc_plan, sizeof(T))) {
      P.cc = m;
      break;
    }
  P.bar = GridBarrier{g->bar_count, &g->S->nonfinite, kSyncLimitNs, 0u};
  return launch_lower_vcycle<T>(g->cx, P);
}

// One V-cycle from level l for L x = R.  uh / ul as in smooth(): returns
// true if the correction was added to that iterate by the last sweep.
template <class T>
bool vcycle(vsv_grid* g, const std::vector<Level>& lv, int l, Comp3<T> X, Rhs3<T> R, int ncomp,
            bool exact_fine = true, bool x_zero = false, const Comp3<float>* uh = nullptr,
            const Comp3<float>* ul = nullptr) {
  const Level& L = lv[l];
  const double h2 = 1.0 / L.inv_h2;
  const bool last = (l + 1 == (int)lv.size());
  const int kc = (l == 0) ? VSV_KCLASS_SMOOTH_FINE : VSV_KCLASS_SMOOTH;
  if (last) {
    if (l > 0) {
      Comp3<T> E = X;
      Comp3<T> RR{{(T*)R.B[0], (T*)R.B[1], (T*)R.B[2]}};
      if (launch_coarse_solve<T>(g->cx, L, E, RR, ncomp, coarsest_sweeps(L, g->sol.coarse_sweeps),
                                 h2))
        return false;
      launch_zero<T>(g->cx, E, L.cells(), ncomp);
    } else if (x_zero) {
      launch_zero<T>(g->cx, X, L.cells(), ncomp);
    }
    const int cs = coarsest_sweeps(L, g->sol.coarse_sweeps);
    for (int s = 0; s < cs; ++s) {
      launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 0, 1.0, h2, kc);
      launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 1, 1.0, h2, kc);
    }
    return false;
  }
  if (l > 0 && x_zero && g->sol.variant == 0 && R.beta == (T)1 && !R.S[0] && !R.S[1] && !R.S[2] &&
      lower_cycle_wanted(g, lv, l)) {
    // the levels from l down in one cooperative launch
    Comp3<T> RR{{(T*)R.B[0], (T*)R.B[1], (T*)R.B[2]}};
    if (run_lower_cycle<T>(g, lv, l, X, RR, ncomp)) return false;
  }
  if (l > 0 && x_zero && g->sol.variant != 1 && R.beta == (T)1 && !R.S[0] && !R.S[1] && !R.S[2]) {
    // the remaining levels fit in one CTA's shared memory: one launch
    CoarseCycle CC;
    coarse_plan(g, lv, l, &CC, sizeof(T));
    Comp3<T> RR{{(T*)R.B[0], (T*)R.B[1], (T*)R.B[2]}};
    if (launch_coarse_vcycle<T>(g->cx, CC, X, RR, ncomp)) return false;
  }
  smooth<T>(g, L, l, X, R, ncomp, g->sol.nu1, x_zero);
  const Level& C = lv[l + 1];
  Comp3<T> EC = cview<T>(g->mg_e[l + 1], g->c0);
  Comp3<T> RC = cview<T>(g->mg_r[l + 1], g->c0);
  const bool exact = std::is_same<T, float>::value && l == 0 && exact_fine;
  launch_resid_restrict<T>(g->cx, L, C, X, R, RC, ncomp, exact);
  Rhs3<T> RCr{{RC.p[0], RC.p[1], RC.p[2]}, {nullptr, nullptr, nullptr}, (T)1};
  vcycle<T>(g, lv, l + 1, EC, RCr, ncomp, exact_fine, true);
  launch_prolong_add<T>(g->cx, L, C, X, EC, ncomp);
  return smooth<T>(g, L, l, X, R, ncomp, g->sol.nu2, false, uh, ul);
}

// relres = max over components of ||b - L x|| / ||b|| (||b|| = 0 -> ||r||).
template <class T>
vsv_status residual(vsv_grid* g, const Level& L, Comp3<T> X, Rhs3<T> R, int ncomp, double* relres) {
  launch_resid_norm<T>(g->cx, L, X, R, ncomp, std::is_same<T, float>::value, g->partials,
                       g->red_blocks, g->S);
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, g->S, sizeof(Scalars), cudaMemcpyDeviceToHost, g->cx.stream));
  CK(cudaStreamSynchronize(g->cx.stream));
  double m = 0.0;
  for (int c = 0; c < ncomp; ++c) {
    const double rn = std::sqrt(hs.rnorm2[c]), bn = std::sqrt(hs.bnorm2[c]);
    m = std::max(m, bn > 0 ? rn / bn : rn);
  }
  *relres = m;
  return VSV_OK;
}

// Solve L x = b (per component) on hierarchy lv.  fixed > 0: exactly that many
// cycles (SOR: sweeps), no synchronisation; else to tol within max_cycles.
template <class T>
vsv_status solve(vsv_grid* g, const std::vector<Level>& lv, Comp3<T> X, Rhs3<T> R, int ncomp,
                 int kind, int fixed, double tol, int max_cycles, int check_every, int* cycles_out,
                 double* relres_out) {
  const Level& L = lv[0];
  double w = g->sol.omega_sor > 0 ? g->sol.omega_sor : sor_weight(L);
  const double h2 = 1.0 / L.inv_h2;
  auto one = [&]() {
    if (kind == VSV_SOLVER_SOR) {
      launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 0, w, h2, VSV_KCLASS_SMOOTH_FINE);
      launch_rb_sweep<T>(g->cx, L, X, R, ncomp, 1, w, h2, VSV_KCLASS_SMOOTH_FINE);
    } else {
      vcycle<T>(g, lv, 0, X, R, ncomp);
    }
  };
  if (fixed > 0) {
    for (int c = 0; c < fixed; ++c) one();
    CKL();
    if (cycles_out) *cycles_out = fixed;
    if (relres_out) *relres_out = -1.0;
    return VSV_OK;
  }
  const int every = std::max(1, check_every);
  double rr = 0.0;
  vsv_status st = residual<T>(g, L, X, R, ncomp, &rr);
  if (st != VSV_OK) return st;
  int c = 0;
  double prev = rr;
  int stall = 0;
  bool floor_reached = false;
  while (rr > tol && c < max_cycles) {
    const int todo = std::min(every, max_cycles - c);
    for (int q = 0; q < todo; ++q) one();
    c += todo;
    CKL();
    st = residual<T>(g, L, X, R, ncomp, &rr);
    if (st != VSV_OK) return st;
    if (!(rr < 0.9 * prev)) {
      if (++stall >= 3) {
        // No further decrease: the iterate sits at the rounding floor of its
        // storage.  In FP32 storage that floor is u ||L|| ||x|| / ||b||
        // (often 1e-6 .. 1e-4 for smooth solutions) while the error of x
        // itself is O(u): accepted as converged for the mixed precision.
        floor_reached = std::is_same<T, float>::value && rr < 1e-3;
        break;
      }
    } else {
      stall = 0;
    }
    prev = std::min(prev, rr);
  }
  if (cycles_out) *cycles_out = c;
  if (relres_out) *relres_out = rr;
  if (!std::isfinite(rr)) return fail(g, VSV_ENONFINITE, "non-finite residual%s");
  if (rr > tol && !floor_reached) return fail(g, VSV_ENOCONV, "Poisson solve stopped above tolerance%s");
  return VSV_OK;
}

// Mixed-path solve of L x = b with the double-word iterate x = (XH, XL) by
// outer defect correction: r = b - L x exactly, one FP32 V-cycle for L e = r
// from e = 0, x += e.  fixed > 0: exactly that many corrections without
// synchronisation; else correct until ||r|| <= tol ||b|| or max_cycles.
vsv_status solve_dc(vsv_grid* g, const std::vector<Level>& lv, Comp3<float> XH, Comp3<float> XL,
                    Rhs3<float> R, Comp3<float> BL, int ncomp, int fixed, double tol,
                    int max_cycles, int check_every, int* cycles_out, double* relres_out) {
  const Level& L = lv[0];
  Comp3<float> E = cview<float>(g->e0, g->c0);
  Comp3<float> RR = cview<float>(g->r0, g->c0);
  Rhs3<float> RE{{RR.p[0], RR.p[1], RR.p[2]}, {nullptr, nullptr, nullptr}, 1.f};
  auto correct = [&]() {
    if (!vcycle<float>(g, lv, 0, E, RE, ncomp, false, true, &XH, &XL))
      launch_update_dw(g->cx, XH, XL, E, L.cells(), ncomp);
  };
  // defect r = b - L x (tiled kernel where the level allows it); returns the
  // number of partial-sum blocks per component written when `norms`
  auto defect = [&](bool norms) -> int {
    double* part = norms ? g->partials : nullptr;
    if (g->sol.variant != 1) {
      const int nb = launch_defect_tiled(g->cx, L, XH, XL, R, BL, RR, ncomp, part,
                                         g->red_blocks * 32 / (2 * ncomp), g->sol.variant == 0);
      if (nb > 0) return nb;
    }
    launch_defect_dw(g->cx, L, XH, XL, R, BL, RR, ncomp, part, g->red_blocks);
    return g->red_blocks;
  };
  if (fixed > 0) {
    for (int c = 0; c < fixed; ++c) {
      defect(false);
      correct();
    }
    CKL();
    if (cycles_out) *cycles_out = fixed;
    if (relres_out) *relres_out = -1.0;
    return VSV_OK;
  }
  const int every = std::max(1, check_every);
  int c = 0;
  double rr = INFINITY;
  while (true) {
    const bool check = (c % every == 0) || c >= max_cycles;
    const int nb = defect(check);
    if (check) {
      launch_norm_finalize(g->cx, g->partials, nb, ncomp, g->S);
      Scalars hs;
      CK(cudaMemcpyAsync(&hs, g->S, sizeof(Scalars), cudaMemcpyDeviceToHost, g->cx.stream));
      CK(cudaStreamSynchronize(g->cx.stream));
      rr = 0.0;
      for (int q = 0; q < ncomp; ++q) {
        const double rn = std::sqrt(hs.rnorm2[q]), bn = std::sqrt(hs.bnorm2[q]);
        rr = std::max(rr, bn > 0 ? rn / bn : rn);
      }
      if (rr <= tol || c >= max_cycles) break;
    }
    correct();
    ++c;
  }
  CKL();
  if (cycles_out) *cycles_out = c;
  if (relres_out) *relres_out = rr;
  if (!std::isfinite(rr)) return fail(g, VSV_ENONFINITE, "non-finite residual%s");
  if (rr > tol) return fail(g, VSV_ENOCONV, "Poisson solve stopped above tolerance%s");
  return VSV_OK;
}

// ---------------------------------------------------------------- phase-field helpers
// Speed of wall w (0: y = 0 wall or Poiseuille speed, 1: y = H wall) at time t.
double wall_speed(const vsv_grid* g, int w, double t) {
  const double s0 = g->flow.kind == VSV_COUETTE ? (w == 0 ? g->flow.v_lo : g->flow.v_hi)
                                                : (w == 0 ? g->flow.u_max : 0.0);
  if (!g->motion_on) return s0;
  const vsv_wall_motion& m = g->motion;
  return s0 + m.ramp[w] * t + m.amplitude[w] * std::sin(2.0 * M_PI * m.frequency[w] * t + m.phase[w]);
}

WallTables wall_tables(const vsv_grid* g) {
  WallTables W{};
  W.n_ring = (g->ny + 2) * (g->nz + 2);
  W.n_tab = g->ny * g->nz;
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 3; ++c) {
      W.bom[b][c] = g->wb_om[b][c];
      W.bps[b][c] = g->wb_ps[b][c];
      W.bv0[b][c] = g->wb_v0[b][c];
      W.bsom[b][c] = g->wb_som[b][c];
      W.bsps[b][c] = g->wb_sps[b][c];
    }
  for (int c = 0; c < 3; ++c) {
    W.om[c] = g->om_ring[c];
    W.ps[c] = g->ps_ring[c];
    W.v0[c] = g->v0d[c];
    W.som[c] = g->s_om_d[c];
    W.sps[c] = g->s_ps_d[c];
    W.v0t[c] = g->v0t[c];
    W.somt[c] = g->s_om_t[c];
    W.spsnt[c] = g->s_ps_neg_t[c];
  }
  const bool cou = g->flow.kind == VSV_COUETTE;
  W.s0[0] = cou ? g->flow.v_lo : g->flow.u_max;
  W.s0[1] = cou ? g->flow.v_hi : 0.0;
  for (int w = 0; w < 2; ++w) {
    W.ramp[w] = g->motion.ramp[w];
    W.amp[w] = g->motion.amplitude[w];
    W.freq[w] = g->motion.frequency[w];
    W.phase[w] = g->motion.phase[w];
  }
  W.t_dev = g->t_dev;
  return W;
}

PhaseParams phase_params(const vsv_grid* g) {
  PhaseParams P{};
  P.nx = g->nx; P.ny = g->ny; P.nz = g->nz;
  P.zper = z_periodic(g);
  P.h = g->h; P.inv_h = 1.0 / g->h; P.inv_h2 = 1.0 / (g->h * g->h);
  P.fe_kind = g->fe.kind;
  P.sigma = g->fe.sigma;
  P.eps = g->fe.eps;
  const double cf = 3.0 * std::sqrt(2.0) * g->fe.kappa / (8.0 * std::pow(g->fe.eps, 3));
  P.cf2 = g->fe.mu_prefactor_half ? cf : 2.0 * cf;
  // membrane tension: sigma times the face-difference area functional adds
  // (c_A / eps) sigma g to the Helfrich mu, c_A = 3 / (2 sqrt 2)
  P.beta_t = g->fe.kind == VSV_HELFRICH ? g->fe.sigma * 3.0 / (2.0 * std::sqrt(2.0) * g->fe.eps) : 0.0;
  P.mobility = g->fe.mobility;
  P.inv_eta = 1.0 / g->flow.eta;
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  split(P.inv_h2, P.ih2_hi, P.ih2_lo);
  split(g->fe.eps * g->fe.eps * P.inv_h2, P.e2ih_hi, P.e2ih_lo);
  split(P.cf2, P.cf2_hi, P.cf2_lo);
  split(g->fe.sigma * P.inv_h2, P.sgih_hi, P.sgih_lo);
  split(0.25 * P.inv_h2 / g->flow.eta, P.src_hi, P.src_lo);
  split(3.0 / (2.0 * std::sqrt(2.0)) * 0.5 * g->fe.eps * 0.25 * P.inv_h2, P.ag_hi, P.ag_lo);
  split(3.0 / (2.0 * std::sqrt(2.0)) * 0.25 / g->fe.eps, P.aw_hi, P.aw_lo);
  split(P.beta_t, P.bt_hi, P.bt_lo);
  std::memset(P.vwall, 0, sizeof P.vwall);
  if (g->flow.kind == VSV_COUETTE) {   // the walls of the current time
    P.vwall[0][0] = wall_speed(g, 0, g->time);
    P.vwall[1][0] = wall_speed(g, 1, g->time);
  }
  return P;
}

void upload_scalar_params(vsv_grid* g) {
  // k_vol, k_area, eps, h3 live in the device scalars (read by the finalizer)
  struct { double k_vol, k_area, eps, h3; } v{g->fe.k_vol, g->fe.k_area, g->fe.eps,
                                                g->h * g->h * g->h};
  cudaMemcpyAsync(&g->S->k_vol, &v, sizeof v, cudaMemcpyHostToDevice, g->cx.stream);
  cudaStreamSynchronize(g->cx.stream);
}

template <class T>
Rhs3<T> rhs_omega(vsv_grid* g) {
  return Rhs3<T>{{(T*)g->f[0], (T*)g->f[1], (T*)g->f[2]}, {nullptr, nullptr, nullptr}, (T)1};
}
template <class T>
Rhs3<T> rhs_psi(vsv_grid* g) {
  return Rhs3<T>{{(T*)g->om[0], (T*)g->om[1], (T*)g->om[2]},
                 {(T*)g->s_ps_neg_t[0], (T*)g->s_ps_neg_t[1], (T*)g->s_ps_neg_t[2]}, (T)-1};
}

// First guess of a solve from the field's history: x^n (order 0), 2 x^n -
// x^{n-1} (order 1) or 3 x^n - 3 x^{n-1} + x^{n-2} (order 2), limited by how
// many previous solutions exist.  The guess is written into the oldest
// buffer, and the three buffers rotate: (x, x_prev, x_prev2) <- (guess, x^n,
// x^{n-1}), so no field is copied.
template <class T>
void guess_from_history(vsv_grid* g, void* x[3], void* xp[3], void* xpp[3], float* xl[3],
                        float* xpl[3], float* xppl[3], int order, int c0 = 0, int ncomp = 3) {
  const bool mixed = std::is_same<T, float>::value && g->prec == VSV_MIXED;
  if (mixed)
    launch_extrapolate_rot_dw(g->cx, cview<float>(x, c0), cview<float>(xl, c0), cview<float>(xp, c0),
                              cview<float>(xpl, c0), cview<float>(xpp, c0), cview<float>(xppl, c0),
                              g->N, ncomp, order);
  else
    launch_extrapolate_rot<T>(g->cx, cview<T>(x, c0), cview<T>(xp, c0), cview<T>(xpp, c0), g->N,
                              ncomp, order);
  for (int c = c0; c < c0 + ncomp; ++c) {
    void* t = xpp[c];
    xpp[c] = xp[c];
    xp[c] = x[c];
    x[c] = t;
    if (mixed) {
      float* tl = xppl[c];
      xppl[c] = xpl[c];
      xpl[c] = xl[c];
      xl[c] = tl;
    }
  }
}

// Whether a step's mixed fixed-cycle solves run on the component streams:
// fixed cycles (no norms across components), component streams wanted (2:
// grids of at least 2^24 cells; on smaller ones the tripled launch count
// costs more than the overlap gains: a batch of 64 grids of 0.5 M cells on
// average ran at 859 instead of 1,456 Mcell-steps/s on streams, 1,284
// instead of 1,359 through the graph), no single-launch lower cycle (its
// barrier counter is shared), and no kernel class being timed by events
// (they assume one launch at a time).
bool solves_branched(const vsv_grid* g) {
  const vsv_solver_params& s = g->sol;
  const int fixed_psi = s.fixed_cycles_psi > 0 ? s.fixed_cycles_psi : s.fixed_cycles;
  const bool streams = s.component_streams == 1 || (s.component_streams == 2 && g->N >= (1LL << 24));
  return g->prec == VSV_MIXED && s.fixed_cycles > 0 && fixed_psi > 0 && streams &&
         s.lower_cycle == 0 && g->cx.prof_class < 0;
}

// The fixed-cycle mixed solves with the three components on three streams:
// component c's vorticity solve, then its stream-vector solve (whose rhs is
// -omega'_c - s_psi,c alone), forked from the grid's stream after the source
// and joined back before the step goes on.  Every kernel sees the component
// it would see in the three-component launches, with the same arithmetic,
// so the results are bit-identical; what changes is that one component's
// latency-bound lower levels overlap the other components' bandwidth-bound
// finest-level kernels.
vsv_status flow_solves_branched(vsv_grid* g, int fixed, int fixed_psi, int order, bool guessed) {
  const vsv_solver_params& s = g->sol;
  const cudaStream_t main = g->cx.stream;
  // on every way out (errors included) the grid's stream waits for both
  // component streams again, so nothing later overlaps their work
  struct Restore {
    vsv_grid* g;
    cudaStream_t main;
    bool forked = false;
    ~Restore() {
      g->cx.stream = main;
      g->c0 = 0;
      g->cx.chunk_comps = 0;
      if (forked)
        for (int i = 0; i < 2; ++i)
          if (cudaEventRecord(g->join_ev[i], g->aux[i]) == cudaSuccess)
            cudaStreamWaitEvent(main, g->join_ev[i], 0);
    }
  } restore{g, main};
  g->cx.chunk_comps = 3;
  CK(cudaEventRecord(g->fork_ev, main));
  for (int i = 0; i < 2; ++i) CK(cudaStreamWaitEvent(g->aux[i], g->fork_ev, 0));
  restore.forked = true;
  const std::vector<Level>& lvo =
      (g->flow.rho > 0.0 && !g->omega_levels.empty()) ? g->omega_levels : g->flow_levels;
  for (int c = 0; c < 3; ++c) {
    g->cx.stream = c == 0 ? main : g->aux[c - 1];
    g->c0 = c;
    if (guessed) CK(cudaStreamWaitEvent(g->cx.stream, g->ext_ev, 0));
    else
      guess_from_history<float>(g, g->om, g->om_prev, g->om_prev2, g->om_lo, g->om_prev_lo,
                                g->om_prev2_lo, order, c, 1);
    const Rhs3<float> RO{{(const float*)g->f[c], nullptr, nullptr}, {nullptr, nullptr, nullptr}, 1.f};
    vsv_status st = solve_dc(g, lvo, cview<float>(g->om, c), cview<float>(g->om_lo, c), RO,
                             cview<float>(g->f_lo, c), 1, fixed, s.tol, s.max_cycles,
                             s.check_every, &g->last_cycles[0], &g->last_relres[0]);
    if (st != VSV_OK) return st;
    if (!guessed)
      guess_from_history<float>(g, g->ps, g->ps_prev, g->ps_prev2, g->ps_lo, g->ps_prev_lo,
                                g->ps_prev2_lo, order, c, 1);
    const Rhs3<float> RP{{(const float*)g->om[c], nullptr, nullptr},
                         {(const float*)g->s_ps_neg_t[c], nullptr, nullptr}, -1.f};
    st = solve_dc(g, g->flow_levels, cview<float>(g->ps, c), cview<float>(g->ps_lo, c), RP,
                  cview<float>(g->om_lo, c), 1, fixed_psi, s.tol, s.max_cycles, s.check_every,
                  &g->last_cycles[1], &g->last_relres[1]);
    if (st != VSV_OK) return st;
  }
  return VSV_OK;   // joined by the guard
}

vsv_status flow_solves_mixed(vsv_grid* g, bool initial) {
  const vsv_solver_params& s = g->sol;
  const int fixed = initial ? 0 : s.fixed_cycles;
  const int fixed_psi = (initial || !s.fixed_cycles) ? fixed
                        : (s.fixed_cycles_psi > 0 ? s.fixed_cycles_psi : s.fixed_cycles);
  const int order = std::min(s.extrapolate, g->hist);
  // the first guesses were already extrapolated early in the step
  const bool guessed = !initial && g->guesses_done;
  g->guesses_done = false;
  if (!initial && solves_branched(g)) {
    const vsv_status st = flow_solves_branched(g, fixed, fixed_psi, order, guessed);
    g->hist = std::min(g->hist + 1, 2);
    return st;
  }
  if (guessed) CK(cudaStreamWaitEvent(g->cx.stream, g->ext_ev, 0));
  if (!initial && !guessed)
    guess_from_history<float>(g, g->om, g->om_prev, g->om_prev2, g->om_lo, g->om_prev_lo,
                              g->om_prev2_lo, order);
  Comp3<float> OH = comp3<float>(g->om[0], g->om[1], g->om[2]);
  Comp3<float> OL = comp3<float>(g->om_lo[0], g->om_lo[1], g->om_lo[2]);
  Comp3<float> FL = comp3<float>(g->f_lo[0], g->f_lo[1], g->f_lo[2]);
  const std::vector<Level>& lvo =
      (!initial && g->flow.rho > 0.0 && !g->omega_levels.empty()) ? g->omega_levels : g->flow_levels;
  vsv_status st = solve_dc(g, lvo, OH, OL, rhs_omega<float>(g), FL, 3, fixed, s.tol,
                           s.max_cycles, s.check_every, &g->last_cycles[0], &g->last_relres[0]);
  if (st != VSV_OK) return st;
  if (!initial && !guessed)
    guess_from_history<float>(g, g->ps, g->ps_prev, g->ps_prev2, g->ps_lo, g->ps_prev_lo,
                              g->ps_prev2_lo, order);
  Comp3<float> PH = comp3<float>(g->ps[0], g->ps[1], g->ps[2]);
  Comp3<float> PL = comp3<float>(g->ps_lo[0], g->ps_lo[1], g->ps_lo[2]);
  // rhs of the stream-vector problem: -(omega'_hi + omega'_lo) - s_psi
  st = solve_dc(g, g->flow_levels, PH, PL, rhs_psi<float>(g), OL, 3, fixed_psi, s.tol, s.max_cycles,
                s.check_every, &g->last_cycles[1], &g->last_relres[1]);
  g->hist = initial ? 0 : std::min(g->hist + 1, 2);
  return st;
}

template <class T>
vsv_status flow_solves(vsv_grid* g, bool initial) {
  if constexpr (std::is_same<T, float>::value) return flow_solves_mixed(g, initial);
  const vsv_solver_params& s = g->sol;
  const int fixed = initial ? 0 : s.fixed_cycles;
  const int fixed_psi = (initial || !s.fixed_cycles) ? fixed
                        : (s.fixed_cycles_psi > 0 ? s.fixed_cycles_psi : s.fixed_cycles);
  const int order = std::min(s.extrapolate, g->hist);
  if (!initial)
    guess_from_history<T>(g, g->om, g->om_prev, g->om_prev2, nullptr, nullptr, nullptr, order);
  Comp3<T> O = comp3<T>(g->om[0], g->om[1], g->om[2]);
  const std::vector<Level>& lvo =
      (!initial && g->flow.rho > 0.0 && !g->omega_levels.empty()) ? g->omega_levels : g->flow_levels;
  vsv_status st = solve<T>(g, lvo, O, rhs_omega<T>(g), 3, s.kind, fixed, s.tol,
                           s.max_cycles, s.check_every, &g->last_cycles[0], &g->last_relres[0]);
  if (st != VSV_OK) return st;
  if (!initial)
    guess_from_history<T>(g, g->ps, g->ps_prev, g->ps_prev2, nullptr, nullptr, nullptr, order);
  Comp3<T> Pp = comp3<T>(g->ps[0], g->ps[1], g->ps[2]);
  st = solve<T>(g, g->flow_levels, Pp, rhs_psi<T>(g), 3, s.kind, fixed_psi, s.tol, s.max_cycles,
                s.check_every, &g->last_cycles[1], &g->last_relres[1]);
  g->hist = initial ? 0 : std::min(g->hist + 1, 2);
  return st;
}

// mu (and V, A, multipliers) of the current phi; init fixes V0, A0.
template <class T>
void refresh_phase(vsv_grid* g, int init) {
  PhaseParams P = phase_params(g);
  T* phi = (T*)g->phi[g->cur];
  if constexpr (std::is_same<T, float>::value) {
    const float* lo = g->phi_lo[g->cur];
    // Helfrich: g from the reduction's pass over phi (variant 1: the
    // separate kernel, same values)
    const bool fuse_g = P.fe_kind == VSV_HELFRICH && g->sol.variant != 1;
    const bool g_ready =
        launch_reduce_va<float>(g->cx, P, phi, lo, g->partials, g->red_blocks, g->S, init,
                                fuse_g ? (float*)g->g : nullptr, fuse_g ? g->g_lo : nullptr);
    launch_mu_ff(g->cx, P, phi, lo, (float*)g->g, g->g_lo, (float*)g->mu, g->mu_lo, g->S, g_ready);
  } else {
    launch_reduce_va<T>(g->cx, P, phi, nullptr, g->partials, g->red_blocks, g->S, init);
    launch_mu<T>(g->cx, P, phi, (T*)g->g, (T*)g->mu, g->S);
  }
}

// f = grad phi x grad mu / eta - s_omega of the current phi and mu
template <class T>
void launch_flow_source(vsv_grid* g, const PhaseParams& P) {
  Comp3<T> SO = comp3<T>(g->s_om_t[0], g->s_om_t[1], g->s_om_t[2]);
  Comp3<T> F = comp3<T>(g->f[0], g->f[1], g->f[2]);
  const T* phi = (const T*)g->phi[g->cur];
  if constexpr (std::is_same<T, float>::value)
    launch_source_ff(g->cx, P, phi, g->phi_lo[g->cur], (const float*)g->mu, g->mu_lo, SO, F,
                     comp3<float>(g->f_lo[0], g->f_lo[1], g->f_lo[2]));
  else
    launch_source<T>(g->cx, P, phi, (const T*)g->mu, SO, F);
}

template <class T>
vsv_status step_impl(vsv_grid* g, double dt) {
  PhaseParams P = phase_params(g);
  g->guesses_done = false;
  if (g->phase_stale) {
    refresh_phase<T>(g, 0);
    g->phase_stale = false;
  }
  T* phi = (T*)g->phi[g->cur];
  T* phin = (T*)g->phi[1 - g->cur];
  Comp3<T> Pp = comp3<T>(g->ps[0], g->ps[1], g->ps[2]);
  Comp3<T> V0 = comp3<T>(g->v0t[0], g->v0t[1], g->v0t[2]);
  // With the component streams (and no inertia, whose right-hand side reads
  // omega'^n), the first guesses of the step's solves depend on the history
  // alone: component stream 0 extrapolates them (bandwidth-bound) while the
  // grid's stream runs the phi update and the phase kernels (ALU-bound).  The
  // fork is recorded before the phi update, which reads psi'^n (the newest
  // history word, never overwritten by a guess).
  const bool early = std::is_same<T, float>::value && solves_branched(g) && g->flow.rho == 0.0;
  if (early) CK(cudaEventRecord(g->fork_ev, g->cx.stream));
  // 1-3: explicit phi update with v^n = v0 + curl psi'^n and lambda_V^n
  if constexpr (std::is_same<T, float>::value)
    launch_phi_update_ff(g->cx, P, phi, g->phi_lo[g->cur], (const float*)g->mu, Pp, V0, g->S,
                         (float)dt, phin, g->phi_lo[1 - g->cur]);
  else
    launch_phi_update<T>(g->cx, P, phi, (const T*)g->mu, Pp, V0, g->S, (T)dt, phin);
  if (early) {
    const cudaStream_t main = g->cx.stream;
    const int order = std::min(g->sol.extrapolate, g->hist);
    CK(cudaStreamWaitEvent(g->aux[0], g->fork_ev, 0));
    g->cx.stream = g->aux[0];
    guess_from_history<T>(g, g->om, g->om_prev, g->om_prev2, g->om_lo, g->om_prev_lo,
                          g->om_prev2_lo, order);
    guess_from_history<T>(g, g->ps, g->ps_prev, g->ps_prev2, g->ps_lo, g->ps_prev_lo,
                          g->ps_prev2_lo, order);
    g->cx.stream = main;
    CK(cudaEventRecord(g->ext_ev, g->aux[0]));
    g->guesses_done = true;
  }
  g->cur = 1 - g->cur;
  // moving walls: the base-flow tables of t^{n+1} for the solves
  if (g->motion_on) launch_wall_tables<T>(g->cx, wall_tables(g), dt, false, 0.0);
  // 4-5: V, A of phi^{n+1}, gamma_A, then mu^{n+1}
  refresh_phase<T>(g, 0);
  // 6: source f = grad phi x grad mu / eta - s_omega
  launch_flow_source<T>(g, P);
  // inertial variant (SM eq. 36), backward Euler: (L_h - s) omega'^{n+1} =
  // f - s_omega - s omega'^n, s = rho / (eta dt); omega' still holds omega'^n
  if (g->flow.rho > 0.0) {
    const double s = g->flow.rho / (g->flow.eta * dt);
    if (g->omega_dt != dt || g->omega_levels.empty()) {
      const int per[3] = {1, 0, z_periodic(g) ? 1 : 0};
      g->omega_levels = build_levels(g->nx, g->ny, g->nz, g->h, per, g->sol.max_levels,
                                     g->mg_nlev_cap, s);
      g->omega_dt = dt;
    }
    Comp3<T> F = comp3<T>(g->f[0], g->f[1], g->f[2]);
    Comp3<T> O = comp3<T>(g->om[0], g->om[1], g->om[2]);
    if constexpr (std::is_same<T, float>::value)
      launch_axpy_dw(g->cx, F, comp3<float>(g->f_lo[0], g->f_lo[1], g->f_lo[2]), O,
                     comp3<float>(g->om_lo[0], g->om_lo[1], g->om_lo[2]), -s, g->N, 3);
    else
      launch_axpy<T>(g->cx, F, O, -s, g->N, 3);
  }
  CKL();
  // 7-8: vorticity then stream-vector Poisson solves
  vsv_status st = flow_solves<T>(g, false);
  g->time += dt;
  g->steps += 1;
  return st;
}

template <class T>
vsv_status set_phi_impl(vsv_grid* g) {
  refresh_phase<T>(g, 1);
  PhaseParams P = phase_params(g);
  launch_flow_source<T>(g, P);
  launch_zero<T>(g->cx, comp3<T>(g->om[0], g->om[1], g->om[2]), g->N, 3);
  launch_zero<T>(g->cx, comp3<T>(g->ps[0], g->ps[1], g->ps[2]), g->N, 3);
  if constexpr (std::is_same<T, float>::value) {
    launch_zero<float>(g->cx, comp3<float>(g->om_lo[0], g->om_lo[1], g->om_lo[2]), g->N, 3);
    launch_zero<float>(g->cx, comp3<float>(g->ps_lo[0], g->ps_lo[1], g->ps_lo[2]), g->N, 3);
  }
  CKL();
  g->phase_stale = false;
  return flow_solves<T>(g, true);
}

// ---------------------------------------------------------------- data movement
// Copy `n` elements of dtype `dt` from user memory into a T buffer `dst`.
template <class T>
vsv_status import_field(vsv_grid* g, const void* src, int dt, int on_device, T* dst, long long n) {
  const size_t in_sz = (dt == VSV_DTYPE_F64) ? 8 : 4;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (in_sz == sizeof(T)) {
    CK(cudaMemcpyAsync(dst, src, n * in_sz, kind, g->cx.stream));
  } else {
    CK(cudaMemcpyAsync(g->stage_b, src, n * in_sz, kind, g->cx.stream));
    if (dt == VSV_DTYPE_F64) launch_convert<double, T>(g->cx, (const double*)g->stage_b, dst, n);
    else launch_convert<float, T>(g->cx, (const float*)g->stage_b, dst, n);
    CKL();
  }
  if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
  return VSV_OK;
}

template <class T>
vsv_status export_field(vsv_grid* g, const T* src, int dt, int on_device, void* dst, long long n) {
  const size_t out_sz = (dt == VSV_DTYPE_F64) ? 8 : 4;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (out_sz == sizeof(T)) {
    CK(cudaMemcpyAsync(dst, src, n * out_sz, kind, g->cx.stream));
  } else {
    if (dt == VSV_DTYPE_F64) launch_convert<T, double>(g->cx, src, (double*)g->stage_b, n);
    else launch_convert<T, float>(g->cx, src, (float*)g->stage_b, n);
    CKL();
    CK(cudaMemcpyAsync(dst, g->stage_b, n * out_sz, kind, g->cx.stream));
  }
  if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
  return VSV_OK;
}

// Device address of host memory that the GPU may access in place: page-
// locked memory mapped into the device's address space (cudaHostAlloc,
// cudaMallocHost, or cudaHostRegister'ed memory under unified addressing),
// as the runtime reports it.  nullptr for anything else (pageable memory,
// unknown pointers): that goes through a copy.  A kernel then moves the data
// across the host link itself, fused with the split or merge of the words,
// instead of a copy into a staging buffer followed by a kernel.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// FP64 host or device words split into the hi + lo pair (hi, lo): in place
// from mapped host memory, else through the staging buffer.
vsv_status split_in(vsv_grid* g, const void* src, int on_device, float* hi, float* lo) {
  const void* m = on_device ? src : mapped_host(src);
  if (m) {
    launch_split_ff(g->cx, (const double*)m, hi, lo, g->N);
  } else {
    CK(cudaMemcpyAsync(g->stage_b, src, g->N * 8, cudaMemcpyHostToDevice, g->cx.stream));
    launch_split_ff(g->cx, (const double*)g->stage_b, hi, lo, g->N);
  }
  return VSV_OK;
}

// phi in: FP64 input splits into hi + lo words on the mixed path.
template <class T>
vsv_status import_phi(vsv_grid* g, const void* src, int dt, int on_device) {
  T* hi = (T*)g->phi[g->cur];
  if constexpr (std::is_same<T, float>::value) {
    float* lo = g->phi_lo[g->cur];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (dt == VSV_DTYPE_F64 && on_device == VSV_HOST_ASYNC) {
      // the copy engine fills the import stage on its own stream once the
      // previous split has read it; the split waits for the copy; the call
      // returns at once
      CK(cudaStreamWaitEvent(g->io_in, g->in_free, 0));
      CK(cudaMemcpyAsync(g->stage_in, src, g->N * 8, cudaMemcpyHostToDevice, g->io_in));
      CK(cudaEventRecord(g->in_ready, g->io_in));
      CK(cudaStreamWaitEvent(g->cx.stream, g->in_ready, 0));
      launch_split_ff(g->cx, (const double*)g->stage_in, hi, lo, g->N);
      CKL();
      CK(cudaEventRecord(g->in_free, g->cx.stream));
      return VSV_OK;
    }
    if (dt == VSV_DTYPE_F64) {
      const vsv_status st = split_in(g, src, on_device, hi, lo);
      if (st != VSV_OK) return st;
    } else {
      CK(cudaMemcpyAsync(hi, src, g->N * 4, kind, g->cx.stream));
      CK(cudaMemsetAsync(lo, 0, g->N * 4, g->cx.stream));
    }
    CKL();
    if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
    return VSV_OK;
  } else {
    return import_field<T>(g, src, dt, on_device, hi, g->N);
  }
}

template <class T>
vsv_status export_phi(vsv_grid* g, int dt, int on_device, void* dst) {
  if constexpr (std::is_same<T, float>::value) {
    if (dt == VSV_DTYPE_F64) {
      // merged in place into device memory; host memory (mapped or not) gets
      // the merged words from the staging buffer by the copy engine, which
      // crosses the host link about twice as fast as a kernel writing mapped
      // memory (193 against 81 GB/s measured on GB300 at 268 MB)
      if (on_device == VSV_HOST_ASYNC) {
        // merged into the export stage once its previous copy has left, then
        // copied out on the export stream while the grid's stream goes on
        CK(cudaStreamWaitEvent(g->cx.stream, g->out_free, 0));
        launch_merge_ff(g->cx, (const float*)g->phi[g->cur], g->phi_lo[g->cur],
                        (double*)g->stage_out, g->N);
        CKL();
        CK(cudaEventRecord(g->out_ready, g->cx.stream));
        CK(cudaStreamWaitEvent(g->io_out, g->out_ready, 0));
        CK(cudaMemcpyAsync(dst, g->stage_out, g->N * 8, cudaMemcpyDeviceToHost, g->io_out));
        CK(cudaEventRecord(g->out_free, g->io_out));
        return VSV_OK;
      }
      if (on_device) {
        launch_merge_ff(g->cx, (const float*)g->phi[g->cur], g->phi_lo[g->cur], (double*)dst, g->N);
        CKL();
      } else {
        launch_merge_ff(g->cx, (const float*)g->phi[g->cur], g->phi_lo[g->cur], (double*)g->stage_a,
                        g->N);
        CKL();
        CK(cudaMemcpyAsync(dst, g->stage_a, g->N * 8, cudaMemcpyDeviceToHost, g->cx.stream));
      }
      if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
      return VSV_OK;
    }
  }
  return export_field<T>(g, (const T*)g->phi[g->cur], dt, on_device, dst, g->N);
}

template <class T>
vsv_status get_field_impl(vsv_grid* g, int field, void* dst, int dt, int on_device) {
  PhaseParams P = phase_params(g);
  if (g->phase_stale && (field == VSV_FIELD_MU || field == VSV_FIELD_STRESS_T)) {
    refresh_phase<T>(g, 0);
    g->phase_stale = false;
  }
  const T* src = nullptr;
  T* tmp = (T*)g->stage_a;
  const bool mixed = std::is_same<T, float>::value;
  const cudaMemcpyKind dkind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // double-word perturbation (mixed path) exported in FP64: hi + lo (+ base)
  auto export_dw = [&](const float* hi, const float* lo, const double* tab) -> vsv_status {
    launch_full_field_dw(g->cx, P, hi, lo, tab, 1, (double*)g->stage_a);
    CKL();
    CK(cudaMemcpyAsync(dst, g->stage_a, g->N * 8, dkind, g->cx.stream));
    if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
    return VSV_OK;
  };
  if (field == VSV_FIELD_PHI) return export_phi<T>(g, dt, on_device, dst);
  else if (field == VSV_FIELD_MU) {
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)g->mu, g->mu_lo, nullptr);
    src = (const T*)g->mu;
  }
  else if (field >= VSV_FIELD_OMEGA_X && field <= VSV_FIELD_OMEGA_Z) {
    const int c = field - VSV_FIELD_OMEGA_X;
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)g->om[c], g->om_lo[c], g->om_ring[c]);
    launch_full_field<T>(g->cx, P, (const T*)g->om[c], (const T*)g->om_lo[c], g->om_ring[c], 1, tmp);
    src = tmp;
  } else if (field >= VSV_FIELD_PSI_X && field <= VSV_FIELD_PSI_Z) {
    const int c = field - VSV_FIELD_PSI_X;
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)g->ps[c], g->ps_lo[c], g->ps_ring[c]);
    launch_full_field<T>(g->cx, P, (const T*)g->ps[c], (const T*)g->ps_lo[c], g->ps_ring[c], 1, tmp);
    src = tmp;
  } else if (field >= VSV_FIELD_VEL_X && field <= VSV_FIELD_VEL_Z) {
    Comp3<T> V, VL;
    output_velocity<T>(g, P, &V, &VL);
    const int c = field - VSV_FIELD_VEL_X;
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)V.p[c], (const float*)VL.p[c], nullptr);
    src = V.p[c];
  } else if (field == VSV_FIELD_STRESS_T) {
    Comp3<T> V, VL;
    output_velocity<T>(g, P, &V, &VL);
    launch_diag<T>(g->cx, P, (const T*)g->phi[g->cur], (const T*)g->phi_lo[g->cur],
                   (const T*)g->g, (const T*)g->g_lo, V, VL,
                   comp3<T>(g->om[0], g->om[1], g->om[2]), om_low<T>(g),
                   comp3<T>(g->ps[0], g->ps[1], g->ps[2]), ps_low<T>(g),
                   ring3(g->ps_ring), ring3(g->v0d), tmp, g->partials, g->red_blocks, g->dout);
    src = tmp;
  } else if (field >= VSV_FIELD_OMEGA_PERT_X && field <= VSV_FIELD_OMEGA_PERT_Z) {
    const int c = field - VSV_FIELD_OMEGA_PERT_X;
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)g->om[c], g->om_lo[c], nullptr);
    src = (const T*)g->om[c];
  } else if (field >= VSV_FIELD_PSI_PERT_X && field <= VSV_FIELD_PSI_PERT_Z) {
    const int c = field - VSV_FIELD_PSI_PERT_X;
    if (mixed && dt == VSV_DTYPE_F64) return export_dw((const float*)g->ps[c], g->ps_lo[c], nullptr);
    src = (const T*)g->ps[c];
  } else {
    return fail(g, VSV_EINVAL, "unknown field%s");
  }
  CKL();
  return export_field<T>(g, src, dt, on_device, dst, g->N);
}

// ---------------------------------------------------------------- base flow
vsv_status upload_d(vsv_grid* g, double* dst, const std::vector<double>& v) {
  CK(cudaMemcpyAsync(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice, g->cx.stream));
  CK(cudaStreamSynchronize(g->cx.stream));
  return VSV_OK;
}

// 2-D (y, z) FP64 solve of lap x = b, zero data on the wall nodes (duct).
vsv_status solve2d(vsv_grid* g, double* x, const double* b, double tol) {
  const int per[3] = {1, 0, 0};
  std::vector<Level> lv = build_levels(1, g->ny, g->nz, g->h, per, 1, 1);
  Comp3<double> X{{x, nullptr, nullptr}};
  Rhs3<double> R{{b, nullptr, nullptr}, {nullptr, nullptr, nullptr}, 1.0};
  launch_fill(g->cx, x, (long long)g->ny * g->nz, 0.0);
  int cyc = 0;
  double rr = 0.0;
  vsv_status st = solve<double>(g, lv, X, R, 1, VSV_SOLVER_SOR, 0, tol, 200000, 50, &cyc, &rr);
  if (st == VSV_ENOCONV && rr < 1e-11) st = VSV_OK;   // rounding floor of the 2-D solve
  return st;
}

template <class T>
void typed_tables(vsv_grid* g) {
  const long long n2 = (long long)g->ny * g->nz;
  for (int c = 0; c < 3; ++c) {
    launch_convert<double, T>(g->cx, g->v0d[c], (T*)g->v0t[c], n2);
    launch_convert<double, T>(g->cx, g->s_om_d[c], (T*)g->s_om_t[c], n2);
    launch_scale_copy<double>(g->cx, g->s_ps_d[c], g->sx, n2, -1.0);
    launch_convert<double, T>(g->cx, g->sx, (T*)g->s_ps_neg_t[c], n2);
  }
}

vsv_status build_base_flow(vsv_grid* g) {
  const int ny = g->ny, nz = g->nz;
  const long long R2 = (long long)(ny + 2) * (nz + 2), n2 = (long long)ny * nz;
  const double h = g->h;
  for (int c = 0; c < 3; ++c) {
    launch_fill(g->cx, g->om_ring[c], R2, 0.0);
    launch_fill(g->cx, g->ps_ring[c], R2, 0.0);
  }
  const double H = (ny + 1) * h;
  auto ridx = [&](int j, int k) { return (size_t)((j + 1) + (long long)(k + 1) * (ny + 2)); };
  if (g->flow.kind == VSV_COUETTE || g->flow.kind == VSV_POISEUILLE_PLANAR) {
    // closed forms on every node (y = (j + 1) h), x- and z-invariant
    std::vector<double> om(R2, 0.0), ps(R2, 0.0);
    for (int k = -1; k <= nz; ++k)
      for (int j = -1; j <= ny; ++j) {
        const double y = (j + 1) * h;
        double o, p;
        if (g->flow.kind == VSV_COUETTE) {
          const double vl = g->flow.v_lo, vh = g->flow.v_hi;
          p = vl * y + (vh - vl) * y * y / (2.0 * H);
          o = -(vh - vl) / H;
        } else {
          const double U = g->flow.u_max;
          p = 4.0 * U * (H * y * y / 2.0 - y * y * y / 3.0) / (H * H);
          o = -4.0 * U * (H - 2.0 * y) / (H * H);
        }
        om[ridx(j, k)] = o;
        ps[ridx(j, k)] = p;
      }
    vsv_status st = upload_d(g, g->om_ring[2], om);
    if (st != VSV_OK) return st;
    st = upload_d(g, g->ps_ring[2], ps);
    if (st != VSV_OK) return st;
  } else if (g->flow.kind == VSV_POISEUILLE_DUCT) {
    if (ny < 2 || nz < 2) return fail(g, VSV_EINVAL, "duct needs ny, nz >= 2%s");
    // u0: lap u0 = -1, scaled to max U; chi: lap chi = u0 (zero wall data)
    launch_fill(g->cx, g->sb, n2, -1.0);
    vsv_status st = solve2d(g, g->su0, g->sb, 1e-13);
    if (st != VSV_OK) return st;
    const double mx = device_max_abs(g->cx, g->su0, n2, g->scratch1);
    launch_scale_copy<double>(g->cx, g->su0, g->su0, n2, g->flow.u_max / mx);
    st = solve2d(g, g->schi, g->su0, 1e-13);
    if (st != VSV_OK) return st;
    launch_duct_ring(g->cx, ny, nz, h, g->su0, g->schi, g->om_ring[1], g->om_ring[2], g->ps_ring[1],
                     g->ps_ring[2]);
    // body-free interior: lap omega0 = 0, lap psi0 = -omega0 with the ring
    // data (u0 and chi are no longer needed: their buffers hold omega0_y, _z)
    double* om_int[3] = {nullptr, g->su0, g->schi};
    for (int c = 1; c < 3; ++c) {
      launch_ring_boundary_rhs(g->cx, ny, nz, h, g->om_ring[c], 0.0, nullptr, g->sb);
      st = solve2d(g, g->sx, g->sb, 1e-12);
      if (st != VSV_OK) return st;
      launch_ring_fill_interior(g->cx, ny, nz, g->sx, g->om_ring[c]);
      launch_scale_copy<double>(g->cx, g->sx, om_int[c], n2, 1.0);
    }
    for (int c = 1; c < 3; ++c) {
      launch_ring_boundary_rhs(g->cx, ny, nz, h, g->ps_ring[c], -1.0, om_int[c], g->sb);
      st = solve2d(g, g->sx, g->sb, 1e-12);
      if (st != VSV_OK) return st;
      launch_ring_fill_interior(g->cx, ny, nz, g->sx, g->ps_ring[c]);
    }
  } else if (g->flow.kind != VSV_QUIESCENT) {
    return fail(g, VSV_EINVAL, "unknown flow kind%s");
  }
  const double* om[3] = {g->om_ring[0], g->om_ring[1], g->om_ring[2]};
  const double* ps[3] = {g->ps_ring[0], g->ps_ring[1], g->ps_ring[2]};
  launch_base_derived(g->cx, ny, nz, z_periodic(g), h, om, ps, g->v0d, g->s_om_d, g->s_ps_d);
  if (g->prec == VSV_FP64) typed_tables<double>(g);
  else typed_tables<float>(g);
  CKL();
  CK(cudaStreamSynchronize(g->cx.stream));
  return VSV_OK;
}

// Programmatic dependent launches for this grid (solver launch_overlap; 2:
// on grids of at least 2^24 cells).  Small grids usually run many at a time
// on their own streams, where the CTAs that wait for their predecessor hold
// SM slots the other streams' kernels would use: measured slower there.
bool overlap_on(const vsv_grid* g) {
  return g->sol.launch_overlap == 1 || (g->sol.launch_overlap == 2 && g->N >= (1LL << 24));
}

void default_solver(vsv_solver_params* s, int prec) {
  s->kind = VSV_SOLVER_MG;
  s->tol = prec == VSV_FP64 ? 1e-12 : 1e-10;
  s->max_cycles = 200;
  s->fixed_cycles = 0;
  s->check_every = 1;
  s->nu1 = 2;
  s->nu2 = 2;
  s->max_levels = kMaxLevels;
  s->coarse_sweeps = 24;
  s->omega_sor = 0.0;
  s->variant = 0;
  s->extrapolate = 1;
  s->fixed_cycles_psi = 0;
  s->omega_mg = kDefaultMgWeight;
  s->lower_cycle = 0;
  s->component_streams = 2;
  s->launch_overlap = 2;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

const char* vsv_version(void) { return "vsv-gb300 0.1 (sm_103a)"; }

size_t vsv_workspace_bytes(int nx, int ny, int nz, int precision) {
  if (!valid_shape(nx, ny, nz) || (precision != VSV_FP64 && precision != VSV_MIXED)) return 0;
  return carve(nx, ny, nz, precision, nullptr, nullptr);
}

vsv_status vsv_create(vsv_grid** out, int nx, int ny, int nz, double h, int precision,
                      void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (!out) return VSV_EINVAL;
  *out = nullptr;
  if (!valid_shape(nx, ny, nz) || !(h > 0) || (precision != VSV_FP64 && precision != VSV_MIXED))
    return VSV_EINVAL;
  if ((nx > 1 && nx % 2) || !workspace || ((uintptr_t)workspace % kAlign)) return VSV_EINVAL;
  const size_t need = carve(nx, ny, nz, precision, nullptr, nullptr);
  if (ws_bytes < need) return VSV_ENOMEM;
  vsv_grid* g = new vsv_grid();
  g->nx = nx; g->ny = ny; g->nz = nz; g->h = h;
  g->prec = precision;
  g->tsize = precision == VSV_FP64 ? 8 : 4;
  g->N = (long long)nx * ny * nz;
  g->ws = (char*)workspace;
  g->ws_bytes = ws_bytes;
  g->cx.stream = (cudaStream_t)cuda_stream;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      g->cx.sms = sms;
  }
  carve(nx, ny, nz, precision, g, g->ws);
  g->cx.status = &g->S->nonfinite;
  g->flow = vsv_flow_params{VSV_QUIESCENT, 0.0, 0.0, 0.0, 1.0, 0.0};
  g->fe = vsv_fe_params{VSV_CAHN_HILLIARD, 1.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0};
  default_solver(&g->sol, precision);
  g->cx.overlap = overlap_on(g);
  if (cudaMemsetAsync(g->S, 0, sizeof(Scalars), g->cx.stream) != cudaSuccess) {
    delete g;
    return VSV_ECUDA;
  }
  // the handle's page-locked word for vsv_step's deferred status, and the
  // event that marks its arrival (created here: stepping allocates nothing)
  bool ok = cudaMallocHost((void**)&g->flag_host, sizeof(int)) == cudaSuccess &&
            cudaHostGetDevicePointer((void**)&g->flag_dev, g->flag_host, 0) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->flag_event, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->ext_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaStreamCreateWithFlags(&g->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->join_ev[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&g->io_in, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&g->io_out, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t* e : {&g->in_ready, &g->in_free, &g->out_ready, &g->out_free})
    ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    vsv_destroy(g);
    return VSV_ECUDA;
  }
  *g->flag_host = 0;
  upload_scalar_params(g);
  *out = g;
  return VSV_OK;
}

vsv_status vsv_destroy(vsv_grid* g) {
  if (!g) return VSV_OK;
  for (auto e : g->cx.ev) cudaEventDestroy(e);
  if (g->flag_event) {
    cudaEventSynchronize(g->flag_event);
    cudaEventDestroy(g->flag_event);
  }
  if (g->flag_host) cudaFreeHost(g->flag_host);
  for (int i = 0; i < 2; ++i) {
    if (g->aux[i]) {
      cudaStreamSynchronize(g->aux[i]);
      cudaStreamDestroy(g->aux[i]);
    }
    if (g->join_ev[i]) cudaEventDestroy(g->join_ev[i]);
  }
  if (g->fork_ev) cudaEventDestroy(g->fork_ev);
  if (g->ext_ev) cudaEventDestroy(g->ext_ev);
  for (cudaStream_t st : {g->io_in, g->io_out})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t e : {g->in_ready, g->in_free, g->out_ready, g->out_free})
    if (e) cudaEventDestroy(e);
  delete g;
  return VSV_OK;
}

vsv_status vsv_default_solver(vsv_solver_params* out, int precision) {
  if (!out) return VSV_EINVAL;
  default_solver(out, precision);
  return VSV_OK;
}

vsv_status vsv_set_flow(vsv_grid* g, const vsv_flow_params* fp) {
  if (!g || !fp) return VSV_EINVAL;
  if (fp->kind < 0 || fp->kind > VSV_QUIESCENT || !(fp->eta > 0) || !(fp->rho >= 0) ||
      !std::isfinite(fp->rho))
    return fail(g, VSV_EINVAL, "invalid flow parameters%s");
  const bool zper = fp->kind == VSV_COUETTE || fp->kind == VSV_POISEUILLE_PLANAR;
  if (zper && g->nz > 1 && g->nz % 2) return fail(g, VSV_EINVAL, "periodic z needs even nz%s");
  g->flow = *fp;
  g->motion_on = false;
  const int per[3] = {1, 0, zper ? 1 : 0};
  g->flow_levels = build_levels(g->nx, g->ny, g->nz, g->h, per, g->sol.max_levels, g->mg_nlev_cap);
  g->omega_levels.clear();
  vsv_status st = build_base_flow(g);
  if (st != VSV_OK) return st;
  g->flow_set = true;
  g->phi_set = false;
  return VSV_OK;
}

vsv_status vsv_set_free_energy(vsv_grid* g, const vsv_fe_params* fe) {
  if (!g || !fe) return VSV_EINVAL;
  if ((fe->kind != VSV_CAHN_HILLIARD && fe->kind != VSV_HELFRICH) || !(fe->eps > 0) ||
      fe->mobility < 0 || fe->k_vol < 0 || fe->k_area < 0)
    return fail(g, VSV_EINVAL, "invalid free-energy parameters%s");
  g->fe = *fe;
  upload_scalar_params(g);
  if (g->phi_set) g->phase_stale = true;
  return VSV_OK;
}

vsv_status vsv_set_wall_motion(vsv_grid* g, const vsv_wall_motion* m) {
  if (!g) return VSV_EINVAL;
  if (!g->flow_set) return fail(g, VSV_ESTATE, "vsv_set_flow must precede vsv_set_wall_motion%s");
  bool any = false;
  if (m) {
    for (int w = 0; w < 2; ++w) {
      const double v[4] = {m->ramp[w], m->amplitude[w], m->frequency[w], m->phase[w]};
      for (double x : v) {
        if (!std::isfinite(x)) return fail(g, VSV_EINVAL, "non-finite wall motion%s");
        any = any || x != 0.0;
      }
    }
    const bool w1 = m->ramp[1] != 0.0 || m->amplitude[1] != 0.0;
    if (any && g->flow.kind == VSV_QUIESCENT)
      return fail(g, VSV_EINVAL, "a quiescent flow has no moving walls%s");
    if (w1 && g->flow.kind != VSV_COUETTE)
      return fail(g, VSV_EINVAL, "wall 1 moves in Couette flow only%s");
    if (any && g->flow.rho > 0.0)
      return fail(g, VSV_EINVAL, "moving walls are provided for the non-inertial flow only%s");
  }
  if (!any) {   // steady walls: the tables of vsv_set_flow, exactly
    const bool was = g->motion_on;
    g->motion_on = false;
    g->motion = vsv_wall_motion{};
    return was ? build_base_flow(g) : VSV_OK;
  }
  // tables of unit wall speeds (the base flow is linear in them)
  const vsv_flow_params keep = g->flow;
  const long long R2 = (long long)(g->ny + 2) * (g->nz + 2), n2 = (long long)g->ny * g->nz;
  vsv_status st = VSV_OK;
  for (int w = 0; w < 2 && st == VSV_OK; ++w) {
    if (keep.kind != VSV_COUETTE && w == 1) {
      for (int c = 0; c < 3; ++c) {
        launch_fill(g->cx, g->wb_om[1][c], R2, 0.0);
        launch_fill(g->cx, g->wb_ps[1][c], R2, 0.0);
        launch_fill(g->cx, g->wb_v0[1][c], n2, 0.0);
        launch_fill(g->cx, g->wb_som[1][c], n2, 0.0);
        launch_fill(g->cx, g->wb_sps[1][c], n2, 0.0);
      }
      break;
    }
    g->flow = keep;
    if (keep.kind == VSV_COUETTE) {
      g->flow.v_lo = w == 0 ? 1.0 : 0.0;
      g->flow.v_hi = w == 1 ? 1.0 : 0.0;
    } else {
      g->flow.u_max = 1.0;
    }
    g->motion_on = false;
    st = build_base_flow(g);
    for (int c = 0; c < 3 && st == VSV_OK; ++c) {
      const cudaStream_t s = g->cx.stream;
      if (cudaMemcpyAsync(g->wb_om[w][c], g->om_ring[c], R2 * 8, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(g->wb_ps[w][c], g->ps_ring[c], R2 * 8, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(g->wb_v0[w][c], g->v0d[c], n2 * 8, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(g->wb_som[w][c], g->s_om_d[c], n2 * 8, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(g->wb_sps[w][c], g->s_ps_d[c], n2 * 8, cudaMemcpyDeviceToDevice, s))
        st = fail(g, VSV_ECUDA, "copy of the wall-speed tables failed%s");
    }
  }
  g->flow = keep;
  if (st != VSV_OK) {
    build_base_flow(g);
    return st;
  }
  g->motion = *m;
  g->motion_on = true;
  if (g->prec == VSV_FP64) launch_wall_tables<double>(g->cx, wall_tables(g), 0.0, true, g->time);
  else launch_wall_tables<float>(g->cx, wall_tables(g), 0.0, true, g->time);
  CKL();
  if (g->phi_set) g->phase_stale = true;
  return VSV_OK;
}

vsv_status vsv_set_solver(vsv_grid* g, const vsv_solver_params* sp) {
  if (!g || !sp) return VSV_EINVAL;
  if (sp->kind != VSV_SOLVER_MG && sp->kind != VSV_SOLVER_SOR) return fail(g, VSV_EINVAL, "bad solver kind%s");
  if (sp->kind == VSV_SOLVER_SOR && g->prec != VSV_FP64)
    return fail(g, VSV_EINVAL, "SOR is provided for the FP64 precision only%s");
  if (sp->nu1 < 0 || sp->nu2 < 0 || sp->nu1 + sp->nu2 < 1 || sp->coarse_sweeps < 1 ||
      sp->max_cycles < 1 || sp->fixed_cycles < 0 || sp->fixed_cycles_psi < 0 || sp->max_levels < 1 || !(sp->tol >= 0) ||
      sp->variant < 0 || sp->variant > 2 || sp->extrapolate < 0 || sp->extrapolate > 2 ||
      !(sp->omega_mg >= 0.0 && sp->omega_mg < 2.0) || sp->lower_cycle < 0 ||
      sp->lower_cycle > 1 || sp->component_streams < 0 || sp->component_streams > 2 ||
      sp->launch_overlap < 0 || sp->launch_overlap > 2)
    return fail(g, VSV_EINVAL, "invalid solver parameters%s");
  g->sol = *sp;
  g->cx.tiled = sp->variant != 1;
  g->cx.ragged = sp->variant == 0;
  g->cx.overlap = overlap_on(g);
  if (g->flow_set) {
    const int per[3] = {1, 0, z_periodic(g) ? 1 : 0};
    g->flow_levels = build_levels(g->nx, g->ny, g->nz, g->h, per, g->sol.max_levels, g->mg_nlev_cap);
    g->omega_levels.clear();   // rebuilt with the new depth at the next step
  }
  return VSV_OK;
}

// on_device as the transfer calls take it: VSV_HOST_ASYNC is honoured for
// FP64 phi on the mixed path; anywhere else it means synchronous host memory.
static int transfer_kind(const vsv_grid* g, int field, int dtype, int on_device) {
  if (on_device != VSV_HOST_ASYNC) return on_device;
  return (field == VSV_FIELD_PHI && dtype == VSV_DTYPE_F64 && g->prec == VSV_MIXED) ? VSV_HOST_ASYNC
                                                                                    : 0;
}

vsv_status vsv_set_phi(vsv_grid* g, const void* phi, int dtype, int on_device) {
  if (!g || !phi || (dtype != VSV_DTYPE_F32 && dtype != VSV_DTYPE_F64) || on_device < 0 ||
      on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  if (on_device == VSV_HOST_ASYNC) on_device = 0;   // the initial solves synchronise anyway
  if (!g->flow_set) return fail(g, VSV_ESTATE, "vsv_set_flow must precede vsv_set_phi%s");
  g->err.clear();
  vsv_status st;
  if (g->motion_on) {   // the walls of t = 0 for the initial solves
    if (g->prec == VSV_FP64) launch_wall_tables<double>(g->cx, wall_tables(g), 0.0, true, 0.0);
    else launch_wall_tables<float>(g->cx, wall_tables(g), 0.0, true, 0.0);
    CKL();
  }
  if (g->prec == VSV_FP64) {
    st = import_phi<double>(g, phi, dtype, on_device);
    if (st == VSV_OK) st = set_phi_impl<double>(g);
  } else {
    st = import_phi<float>(g, phi, dtype, on_device);
    if (st == VSV_OK) st = set_phi_impl<float>(g);
  }
  g->time = 0.0;
  g->steps = 0;
  if (st == VSV_OK || st == VSV_ENOCONV) g->phi_set = true;
  return st;
}

vsv_status vsv_stability_limit(const vsv_grid* g, double* dt_max) {
  if (!g || !dt_max) return VSV_EINVAL;
  const double h2 = g->h * g->h;
  int d = 1 + (g->ny > 1) + (g->nz > 1);
  if (g->nx > 1) d = 3;
  const double lam = 4.0 * d / h2;   // largest eigenvalue of -lap
  const double M = g->fe.mobility;
  double lim = INFINITY;
  if (M > 0) {
    if (g->fe.kind == VSV_CAHN_HILLIARD) {
      lim = 2.0 / (M * lam * (2.0 + g->fe.sigma * lam));
    } else {
      const double e2 = g->fe.eps * g->fe.eps;
      const double cf = 3.0 * std::sqrt(2.0) * g->fe.kappa / (8.0 * std::pow(g->fe.eps, 3));
      const double c2 = g->fe.mu_prefactor_half ? cf : 2.0 * cf;
      const double t = 2.0 + e2 * lam;
      const double beta = g->fe.sigma * 3.0 / (2.0 * std::sqrt(2.0) * g->fe.eps);
      lim = 2.0 / (M * lam * t * (c2 * t + std::max(beta, 0.0)));
    }
    if (g->fe.k_vol > 0) {
      const double v = 4.0 / (M * g->fe.k_vol * (double)g->N * g->h * h2);
      lim = std::min(lim, v);
    }
  }
  *dt_max = lim;
  return VSV_OK;
}

vsv_status vsv_step(vsv_grid* g, int nsteps, double dt) {
  if (!g || nsteps < 0 || !(dt > 0)) return VSV_EINVAL;
  if (!g->phi_set) return fail(g, VSV_ESTATE, "vsv_set_phi must precede vsv_step%s");
  double lim;
  vsv_stability_limit(g, &lim);
  if (dt > lim) {
    char buf[128];
    snprintf(buf, sizeof buf, " (dt %.3g > limit %.3g)", dt, lim);
    return fail(g, VSV_EUNSTABLE, "time step above the explicit stability bound%s", buf);
  }
  // flag of an earlier call, read without waiting if its copy has landed
  if (g->flag_pending && cudaEventQuery(g->flag_event) == cudaSuccess) {
    g->flag_pending = false;
    if (*g->flag_host) return flag_status(g, *g->flag_host);
  }
  for (int s = 0; s < nsteps; ++s) {
    vsv_status st = g->prec == VSV_FP64 ? step_impl<double>(g, dt) : step_impl<float>(g, dt);
    if (st != VSV_OK) return st;
  }
  CKL();
  // (not counted in the grid's launches, like the copy it replaces: a
  // captured batch of the same steps reads the word its own way)
  k_flag_out<<<1, 1, 0, g->cx.stream>>>(&g->S->nonfinite, g->flag_dev);
  CKL();
  CK(cudaEventRecord(g->flag_event, g->cx.stream));
  g->flag_pending = true;
  return VSV_OK;
}

// ---------------------------------------------------------------- batches
}  // extern "C"

struct vsv_batch {
  std::vector<vsv_grid*> grids;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  double dt = 0.0;
  std::vector<long long> launches_per_replay;
  std::vector<double> bytes_per_replay;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
};

namespace {

constexpr int kReplaySteps = 6;   // phi ping-pong (2) x history rotation (3)

// the host-side state a step advances
struct GridHostState {
  int cur, hist;
  void *om[3], *ps[3], *om_prev[3], *ps_prev[3], *om_prev2[3], *ps_prev2[3];
  float *om_lo[3], *ps_lo[3], *om_prev_lo[3], *ps_prev_lo[3], *om_prev2_lo[3], *ps_prev2_lo[3];
  double time;
  long long steps, launches;
  double bytes;
};

GridHostState save_host(const vsv_grid* g) {
  GridHostState s;
  s.cur = g->cur;
  s.hist = g->hist;
  for (int c = 0; c < 3; ++c) {
    s.om[c] = g->om[c]; s.ps[c] = g->ps[c];
    s.om_prev[c] = g->om_prev[c]; s.ps_prev[c] = g->ps_prev[c];
    s.om_prev2[c] = g->om_prev2[c]; s.ps_prev2[c] = g->ps_prev2[c];
    s.om_lo[c] = g->om_lo[c]; s.ps_lo[c] = g->ps_lo[c];
    s.om_prev_lo[c] = g->om_prev_lo[c]; s.ps_prev_lo[c] = g->ps_prev_lo[c];
    s.om_prev2_lo[c] = g->om_prev2_lo[c]; s.ps_prev2_lo[c] = g->ps_prev2_lo[c];
  }
  s.time = g->time;
  s.steps = g->steps;
  s.launches = g->cx.launches;
  s.bytes = g->cx.bytes_total;
  return s;
}

bool same_layout(const GridHostState& a, const GridHostState& b) {
  if (a.cur != b.cur || a.hist != b.hist) return false;
  for (int c = 0; c < 3; ++c)
    if (a.om[c] != b.om[c] || a.ps[c] != b.ps[c] || a.om_prev[c] != b.om_prev[c] ||
        a.ps_prev[c] != b.ps_prev[c] || a.om_prev2[c] != b.om_prev2[c] ||
        a.ps_prev2[c] != b.ps_prev2[c] || a.om_lo[c] != b.om_lo[c] || a.ps_lo[c] != b.ps_lo[c] ||
        a.om_prev_lo[c] != b.om_prev_lo[c] || a.ps_prev_lo[c] != b.ps_prev_lo[c] ||
        a.om_prev2_lo[c] != b.om_prev2_lo[c] || a.ps_prev2_lo[c] != b.ps_prev2_lo[c])
      return false;
  return true;
}

// A grid can be captured once its history and phase fields no longer
// change the work a step enqueues.
bool steady(const vsv_grid* g) { return g->hist == 2 && !g->phase_stale; }

vsv_status step_one(vsv_grid* g, double dt) {
  return g->prec == VSV_FP64 ? step_impl<double>(g, dt) : step_impl<float>(g, dt);
}

}  // namespace

extern "C" {

vsv_status vsv_batch_create(vsv_batch** out, vsv_grid* const* grids, int n, void* cuda_stream) {
  if (!out || !grids || n < 1) return VSV_EINVAL;
  *out = nullptr;
  // graphs cannot be captured on the legacy default stream
  if (cuda_stream == nullptr || (cudaStream_t)cuda_stream == cudaStreamLegacy) return VSV_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!grids[i]) return VSV_EINVAL;
    for (int j = 0; j < i; ++j)
      if (grids[j] == grids[i]) return VSV_EINVAL;
  }
  vsv_batch* b = new vsv_batch();
  b->grids.assign(grids, grids + n);
  b->stream = (cudaStream_t)cuda_stream;
  b->join.resize(n, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i)
    ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    vsv_batch_destroy(b);
    return VSV_ECUDA;
  }
  *out = b;
  return VSV_OK;
}

vsv_status vsv_batch_destroy(vsv_batch* b) {
  if (!b) return VSV_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  delete b;
  return VSV_OK;
}

vsv_status vsv_batch_step(vsv_batch* b, int nsteps, double dt) {
  if (!b || nsteps < 0 || !(dt > 0)) return VSV_EINVAL;
  const int n = (int)b->grids.size();
  for (vsv_grid* g : b->grids) {
    if (!g->phi_set) return fail(g, VSV_ESTATE, "vsv_set_phi must precede vsv_batch_step%s");
    if (g->sol.fixed_cycles <= 0)
      return fail(g, VSV_EINVAL, "batched steps need fixed_cycles > 0%s");
    if (g->cx.prof_class >= 0) return fail(g, VSV_ESTATE, "profiling is on for a batched grid%s");
    double lim;
    vsv_stability_limit(g, &lim);
    if (dt > lim) return fail(g, VSV_EUNSTABLE, "time step above the explicit stability bound%s");
  }
  int done = 0;
  // plain steps until every grid is steady
  while (done < nsteps) {
    bool all = true;
    for (vsv_grid* g : b->grids) all = all && steady(g);
    if (all) break;
    for (vsv_grid* g : b->grids) {
      const vsv_status st = step_one(g, dt);
      if (st != VSV_OK) return st;
    }
    ++done;
  }
  if (nsteps - done >= kReplaySteps && (!b->exec || b->dt != dt)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    std::vector<GridHostState> saved;
    for (vsv_grid* g : b->grids) saved.push_back(save_host(g));
    cudaGraph_t graph = nullptr;
    vsv_grid* g0 = b->grids[0];
    const cudaError_t eb = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (eb != cudaSuccess) {
      cudaGetLastError();
      return fail(g0, VSV_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(eb));
    }
    vsv_status st = VSV_OK;
    cudaEventRecord(b->fork, b->stream);
    for (vsv_grid* g : b->grids) cudaStreamWaitEvent(g->cx.stream, b->fork, 0);
    for (int k = 0; k < kReplaySteps && st == VSV_OK; ++k)
      for (vsv_grid* g : b->grids) {
        st = step_one(g, dt);
        if (st != VSV_OK) break;
      }
    for (int i = 0; i < n; ++i) {
      cudaEventRecord(b->join[i], b->grids[i]->cx.stream);
      cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
    b->launches_per_replay.assign(n, 0);
    b->bytes_per_replay.assign(n, 0.0);
    bool layout_ok = true;
    for (int i = 0; i < n; ++i) {
      vsv_grid* g = b->grids[i];
      const GridHostState after = save_host(g);
      layout_ok = layout_ok && same_layout(after, saved[i]);
      b->launches_per_replay[i] = after.launches - saved[i].launches;
      b->bytes_per_replay[i] = after.bytes - saved[i].bytes;
      g->time = saved[i].time;   // the captured steps have not run yet
      g->steps = saved[i].steps;
      g->cx.launches = saved[i].launches;
      g->cx.bytes_total = saved[i].bytes;
    }
    if (st != VSV_OK || ec != cudaSuccess || !layout_ok) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != VSV_OK ? st : fail(g0, VSV_ECUDA, "capture of the batched steps failed%s");
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      b->exec = nullptr;
      return fail(g0, VSV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
    b->dt = dt;
  }
  if (nsteps - done >= kReplaySteps && b->exec) {
    // work queued on the grids' streams first, then the replays, then the grids wait
    for (int i = 0; i < n; ++i) {
      cudaEventRecord(b->join[i], b->grids[i]->cx.stream);
      cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    while (nsteps - done >= kReplaySteps) {
      const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
      if (e != cudaSuccess)
        return fail(b->grids[0], VSV_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
      for (int i = 0; i < n; ++i) {
        vsv_grid* g = b->grids[i];
        g->time += kReplaySteps * dt;
        g->steps += kReplaySteps;
        g->cx.launches += b->launches_per_replay[i];
        g->cx.bytes_total += b->bytes_per_replay[i];
      }
      done += kReplaySteps;
    }
    cudaEventRecord(b->fork, b->stream);
    for (vsv_grid* g : b->grids) cudaStreamWaitEvent(g->cx.stream, b->fork, 0);
  }
  for (; done < nsteps; ++done)
    for (vsv_grid* g : b->grids) {
      const vsv_status st = step_one(g, dt);
      if (st != VSV_OK) return st;
    }
  return VSV_OK;
}

vsv_status vsv_solve_poisson(vsv_grid* g, const void* rhs, void* x, int dtype, int on_device,
                             const vsv_bc* bc, double tol, int max_cycles, int* cycles_out,
                             double* relres_out) {
  if (!g || !rhs || !x || !bc || max_cycles < 1 || (dtype != VSV_DTYPE_F32 && dtype != VSV_DTYPE_F64) ||
      on_device < 0 || on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  if (on_device == VSV_HOST_ASYNC) on_device = 0;
  const int per[3] = {bc->periodic[0] ? 1 : 0, bc->periodic[1] ? 1 : 0, bc->periodic[2] ? 1 : 0};
  const int n[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a)
    if (per[a] && n[a] > 1 && n[a] % 2) return fail(g, VSV_EINVAL, "periodic axes need even extent%s");
  if (!(bc->shift >= 0) || !std::isfinite(bc->shift))
    return fail(g, VSV_EINVAL, "shift must be finite and >= 0%s");
  if (per[0] && per[1] && per[2] && bc->shift == 0.0)
    return fail(g, VSV_EINVAL, "all-periodic problem is singular%s");
  g->err.clear();
  std::vector<Level> lv = build_levels(g->nx, g->ny, g->nz, g->h, per, g->sol.max_levels,
                                       g->mg_nlev_cap, bc->shift);
  vsv_status st;
  g->phi_set = false;
  auto run = [&](auto tag) -> vsv_status {
    using T = decltype(tag);
    T* b = (T*)g->f[0];
    T* xx = (T*)g->f[1];
    vsv_status s = import_field<T>(g, rhs, dtype, on_device, b, g->N);
    if (s != VSV_OK) return s;
    s = import_field<T>(g, x, dtype, on_device, xx, g->N);
    if (s != VSV_OK) return s;
    Comp3<T> X{{xx, nullptr, nullptr}};
    Rhs3<T> R{{b, nullptr, nullptr}, {nullptr, nullptr, nullptr}, (T)1};
    vsv_status s2 = solve<T>(g, lv, X, R, 1, g->sol.kind, 0, tol, max_cycles, g->sol.check_every,
                             cycles_out, relres_out);
    s = export_field<T>(g, xx, dtype, on_device, x, g->N);
    if (s != VSV_OK) return s;
    return s2;
  };
  // mixed path: double-word rhs and iterate, outer defect correction
  auto run_mixed = [&]() -> vsv_status {
    if (g->sol.kind != VSV_SOLVER_MG) return fail(g, VSV_EINVAL, "mixed precision solves use MG%s");
    float* bh = (float*)g->f[0];
    float* bl = (float*)g->stage_a;           // first N floats of the FP64 stage
    float* xh = (float*)g->f[1];
    float* xl = (float*)g->f[2];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    auto split_in = [&](const void* src, float* hi, float* lo) -> vsv_status {
      if (dtype == VSV_DTYPE_F64) {
        CK(cudaMemcpyAsync(g->stage_b, src, g->N * 8, kind, g->cx.stream));
        launch_split_ff(g->cx, (const double*)g->stage_b, hi, lo, g->N);
      } else {
        CK(cudaMemcpyAsync(hi, src, g->N * 4, kind, g->cx.stream));
        CK(cudaMemsetAsync(lo, 0, g->N * 4, g->cx.stream));
      }
      CK(cudaStreamSynchronize(g->cx.stream));
      return VSV_OK;
    };
    vsv_status s = split_in(rhs, bh, bl);
    if (s != VSV_OK) return s;
    s = split_in(x, xh, xl);
    if (s != VSV_OK) return s;
    Comp3<float> XH{{xh, nullptr, nullptr}}, XL{{xl, nullptr, nullptr}}, BL{{bl, nullptr, nullptr}};
    Rhs3<float> R{{bh, nullptr, nullptr}, {nullptr, nullptr, nullptr}, 1.f};
    vsv_status s2 = solve_dc(g, lv, XH, XL, R, BL, 1, 0, tol, max_cycles, g->sol.check_every,
                             cycles_out, relres_out);
    const cudaMemcpyKind okind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dtype == VSV_DTYPE_F64) {
      launch_merge_ff(g->cx, xh, xl, (double*)g->stage_b, g->N);
      CK(cudaMemcpyAsync(x, g->stage_b, g->N * 8, okind, g->cx.stream));
    } else {
      CK(cudaMemcpyAsync(x, xh, g->N * 4, okind, g->cx.stream));
    }
    CK(cudaStreamSynchronize(g->cx.stream));
    return s2;
  };
  if (g->prec == VSV_FP64) st = run(double{});
  else st = run_mixed();
  return st;
}

vsv_status vsv_get_field(vsv_grid* g, int field, void* dst, int dtype, int on_device) {
  if (!g || !dst || field < 0 || field >= VSV_FIELD_COUNT ||
      (dtype != VSV_DTYPE_F32 && dtype != VSV_DTYPE_F64) || on_device < 0 ||
      on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  on_device = transfer_kind(g, field, dtype, on_device);
  if (!g->phi_set) return fail(g, VSV_ESTATE, "no state: call vsv_set_phi first%s");
  return g->prec == VSV_FP64 ? get_field_impl<double>(g, field, dst, dtype, on_device)
                             : get_field_impl<float>(g, field, dst, dtype, on_device);
}

vsv_status vsv_set_field(vsv_grid* g, int field, const void* src, int dtype, int on_device) {
  if (!g || !src || (dtype != VSV_DTYPE_F32 && dtype != VSV_DTYPE_F64) || on_device < 0 ||
      on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  on_device = transfer_kind(g, field, dtype, on_device);
  if (!g->phi_set) return fail(g, VSV_ESTATE, "no state: call vsv_set_phi first%s");
  void* dst = nullptr;
  if (field == VSV_FIELD_PHI) {
    vsv_status st = g->prec == VSV_FP64 ? import_phi<double>(g, src, dtype, on_device)
                                        : import_phi<float>(g, src, dtype, on_device);
    if (st == VSV_OK) g->phase_stale = true;
    return st;
  } else if (field >= VSV_FIELD_OMEGA_PERT_X && field <= VSV_FIELD_OMEGA_PERT_Z)
    dst = g->om[field - VSV_FIELD_OMEGA_PERT_X];
  else if (field >= VSV_FIELD_PSI_PERT_X && field <= VSV_FIELD_PSI_PERT_Z)
    dst = g->ps[field - VSV_FIELD_PSI_PERT_X];
  else
    return fail(g, VSV_EINVAL, "field cannot be set%s");
  vsv_status st;
  if (g->prec == VSV_FP64) {
    st = import_field<double>(g, src, dtype, on_device, (double*)dst, g->N);
  } else {
    float* lo = (field <= VSV_FIELD_OMEGA_PERT_Z) ? g->om_lo[field - VSV_FIELD_OMEGA_PERT_X]
                                                   : g->ps_lo[field - VSV_FIELD_PSI_PERT_X];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (dtype == VSV_DTYPE_F64) {
      const vsv_status sst = split_in(g, src, on_device, (float*)dst, lo);
      if (sst != VSV_OK) return sst;
    } else {
      CK(cudaMemcpyAsync(dst, src, g->N * 4, kind, g->cx.stream));
      CK(cudaMemsetAsync(lo, 0, g->N * 4, g->cx.stream));
    }
    CKL();
    if (!on_device) CK(cudaStreamSynchronize(g->cx.stream));
    st = VSV_OK;
  }
  if (st == VSV_OK && field == VSV_FIELD_PHI) g->phase_stale = true;
  if (st == VSV_OK && field != VSV_FIELD_PHI) g->hist = 0;
  return st;
}

vsv_status vsv_get_diagnostics(vsv_grid* g, vsv_diag* out) {
  if (!g || !out) return VSV_EINVAL;
  if (!g->phi_set) return fail(g, VSV_ESTATE, "no state: call vsv_set_phi first%s");
  PhaseParams P = phase_params(g);
  auto run = [&](auto tag) {
    using T = decltype(tag);
    if (g->phase_stale) {
      refresh_phase<T>(g, 0);
      g->phase_stale = false;
    }
    Comp3<T> V, VL;
    output_velocity<T>(g, P, &V, &VL);
    launch_diag<T>(g->cx, P, (const T*)g->phi[g->cur], (const T*)g->phi_lo[g->cur],
                   (const T*)g->g, (const T*)g->g_lo, V, VL,
                   comp3<T>(g->om[0], g->om[1], g->om[2]), om_low<T>(g),
                   comp3<T>(g->ps[0], g->ps[1], g->ps[2]), ps_low<T>(g),
                   ring3(g->ps_ring), ring3(g->v0d), (T*)nullptr, g->partials, g->red_blocks,
                   g->dout);
  };
  if (g->prec == VSV_FP64) run(double{});
  else run(float{});
  CKL();
  double q[kDiagQ];
  Scalars hs;
  CK(cudaMemcpyAsync(q, g->dout, sizeof q, cudaMemcpyDeviceToHost, g->cx.stream));
  CK(cudaMemcpyAsync(&hs, g->S, sizeof hs, cudaMemcpyDeviceToHost, g->cx.stream));
  CK(cudaStreamSynchronize(g->cx.stream));
  const double h3 = g->h * g->h * g->h, eta = g->flow.eta;
  std::memset(out, 0, sizeof *out);
  out->time = g->time;
  out->steps = g->steps;
  out->volume = hs.V;
  out->area = hs.A;
  out->volume0 = hs.V0;
  out->area0 = hs.A0;
  out->reduced_volume = hs.A > 0 ? hs.V / (4.0 / 3.0 * M_PI * std::pow(hs.A / (4.0 * M_PI), 1.5)) : 0.0;
  if (g->fe.kind == VSV_HELFRICH) {
    const double cf = 3.0 * std::sqrt(2.0) * g->fe.kappa / (8.0 * std::pow(g->fe.eps, 3));
    out->energy = cf * h3 * q[8];
    // membrane tension sigma times the face-difference area, (c_A / eps) h^3 q12
    if (g->fe.sigma != 0.0)
      out->energy += g->fe.sigma * 3.0 / (2.0 * std::sqrt(2.0) * g->fe.eps) * h3 * q[12];
  } else {
    out->energy = h3 * q[8];
  }
  out->lambda_v = hs.lambda_v;
  out->gamma_a = hs.gamma_a;
  for (int a = 0; a < 3; ++a) out->com[a] = q[4] > 0 ? q[5 + a] / q[4] : 0.0;
  out->dissipation = 0.5 * eta * h3 * q[0];
  out->dissipation0 = 0.5 * eta * h3 * q[1];
  out->resistance_rel = out->dissipation0 > 0 ? (out->dissipation - out->dissipation0) / out->dissipation0 : 0.0;
  out->omega_dev2 = h3 * q[2];
  out->psi_dev2 = h3 * q[3];
  out->max_div_v = q[9];
  out->max_div_psi = q[10];
  out->max_sigma_t = q[11];
  out->last_cycles_omega = g->last_cycles[0];
  out->last_cycles_psi = g->last_cycles[1];
  out->last_relres_omega = g->last_relres[0];
  out->last_relres_psi = g->last_relres[1];
  out->nonfinite = hs.nonfinite;
  return VSV_OK;
}

vsv_status vsv_get_stress_profile(vsv_grid* g, double* out) {
  if (!g || !out) return VSV_EINVAL;
  if (!g->phi_set) return fail(g, VSV_ESTATE, "no state: call vsv_set_phi first%s");
  PhaseParams P = phase_params(g);
  auto run = [&](auto tag) {
    using T = decltype(tag);
    Comp3<T> V, VL;
    output_velocity<T>(g, P, &V, &VL);
    launch_stress_profile<T>(g->cx, P, V, VL, g->profile);
  };
  if (g->prec == VSV_FP64) run(double{});
  else run(float{});
  CKL();
  CK(cudaMemcpyAsync(out, g->profile, g->ny * sizeof(double), cudaMemcpyDeviceToHost, g->cx.stream));
  CK(cudaStreamSynchronize(g->cx.stream));
  return VSV_OK;
}

struct StateHeader {
  char magic[8];
  int nx, ny, nz, prec;
  double V0, A0, time;
  long long steps;
  int hist, pad;
};

// Device buffers of the state blob, in blob order: phi, omega'(3), psi'(3),
// the two previous steps' omega'(3) and psi'(3); on the mixed path then the
// low words of phi and of those eighteen double-word fields.
std::vector<std::pair<void*, size_t>> state_fields(const vsv_grid* g) {
  std::vector<std::pair<void*, size_t>> v;
  const size_t fb = (size_t)g->N * g->tsize, lb = (size_t)g->N * 4;
  v.push_back({g->phi[g->cur], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->om[c], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->ps[c], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->om_prev[c], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->ps_prev[c], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->om_prev2[c], fb});
  for (int c = 0; c < 3; ++c) v.push_back({g->ps_prev2[c], fb});
  if (g->prec == VSV_MIXED) {
    v.push_back({g->phi_lo[g->cur], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->om_lo[c], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->ps_lo[c], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->om_prev_lo[c], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->ps_prev_lo[c], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->om_prev2_lo[c], lb});
    for (int c = 0; c < 3; ++c) v.push_back({g->ps_prev2_lo[c], lb});
  }
  return v;
}

size_t vsv_state_bytes(const vsv_grid* g) {
  if (!g) return 0;
  size_t s = sizeof(StateHeader);
  for (auto& f : state_fields(g)) s += f.second;
  return s;
}

vsv_status vsv_get_state(vsv_grid* g, void* dst, size_t bytes) {
  if (!g || !dst || bytes < vsv_state_bytes(g)) return VSV_EINVAL;
  if (!g->phi_set) return fail(g, VSV_ESTATE, "no state: call vsv_set_phi first%s");
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, g->S, sizeof hs, cudaMemcpyDeviceToHost, g->cx.stream));
  char* p = (char*)dst;
  size_t off = sizeof(StateHeader);
  for (auto& f : state_fields(g)) {
    CK(cudaMemcpyAsync(p + off, f.first, f.second, cudaMemcpyDeviceToHost, g->cx.stream));
    off += f.second;
  }
  CK(cudaStreamSynchronize(g->cx.stream));
  StateHeader hd{};
  std::memcpy(hd.magic, "VSVSTAT", 8);
  hd.nx = g->nx; hd.ny = g->ny; hd.nz = g->nz; hd.prec = g->prec;
  hd.V0 = hs.V0; hd.A0 = hs.A0; hd.time = g->time; hd.steps = g->steps;
  hd.hist = g->hist;
  std::memcpy(p, &hd, sizeof hd);
  return VSV_OK;
}

vsv_status vsv_set_state(vsv_grid* g, const void* src, size_t bytes) {
  if (!g || !src || bytes < vsv_state_bytes(g)) return VSV_EINVAL;
  if (!g->flow_set) return fail(g, VSV_ESTATE, "vsv_set_flow must precede vsv_set_state%s");
  StateHeader hd;
  std::memcpy(&hd, src, sizeof hd);
  if (std::memcmp(hd.magic, "VSVSTAT", 8) || hd.nx != g->nx || hd.ny != g->ny || hd.nz != g->nz ||
      hd.prec != g->prec)
    return fail(g, VSV_EINVAL, "state blob does not match this grid%s");
  const char* p = (const char*)src;
  size_t off = sizeof(StateHeader);
  for (auto& f : state_fields(g)) {
    CK(cudaMemcpyAsync(f.first, p + off, f.second, cudaMemcpyHostToDevice, g->cx.stream));
    off += f.second;
  }
  double v[2] = {hd.V0, hd.A0};
  CK(cudaMemcpyAsync(&g->S->V0, v, sizeof v, cudaMemcpyHostToDevice, g->cx.stream));
  CK(cudaStreamSynchronize(g->cx.stream));
  g->time = hd.time;
  g->steps = hd.steps;
  g->phi_set = true;
  g->phase_stale = true;
  g->hist = (hd.hist >= 0 && hd.hist <= 2) ? hd.hist : 0;
  if (g->motion_on) {   // the walls of the restored time
    if (g->prec == VSV_FP64) launch_wall_tables<double>(g->cx, wall_tables(g), 0.0, true, g->time);
    else launch_wall_tables<float>(g->cx, wall_tables(g), 0.0, true, g->time);
    CKL();
  }
  return VSV_OK;
}

vsv_status vsv_check(vsv_grid* g) {
  if (!g) return VSV_EINVAL;
  CK(cudaStreamSynchronize(g->cx.stream));
  if (g->io_in) CK(cudaStreamSynchronize(g->io_in));
  if (g->io_out) CK(cudaStreamSynchronize(g->io_out));
  CKL();
  int flag = 0;
  CK(cudaMemcpy(&flag, &g->S->nonfinite, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return flag_status(g, flag);
  return VSV_OK;
}

vsv_status vsv_barrier_check(vsv_grid* g, int blocks, int rounds, int extra_arrivals,
                             double limit_ms) {
  if (!g || blocks < 1 || rounds < 1 || extra_arrivals < 0 || !(limit_ms > 0) || limit_ms > 1e4)
    return VSV_EINVAL;
  if (blocks > barrier_probe_max_blocks(g->cx.sms))
    return fail(g, VSV_EINVAL, "more CTAs than can be co-resident%s");
  const GridBarrier B{g->bar_count, &g->S->nonfinite,
                      (unsigned long long)(limit_ms * 1e6), (unsigned)extra_arrivals};
  if (!launch_barrier_probe(g->cx.stream, B, blocks, rounds))
    return fail(g, VSV_ECUDA, "barrier check launch failed%s");
  CK(cudaStreamSynchronize(g->cx.stream));
  int flag = 0;
  CK(cudaMemcpy(&flag, &g->S->nonfinite, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag & kSyncTimeout) {
    const int cleared = flag & ~kSyncTimeout;
    CK(cudaMemcpy(&g->S->nonfinite, &cleared, sizeof(int), cudaMemcpyHostToDevice));
    return flag_status(g, kSyncTimeout);
  }
  return VSV_OK;
}

vsv_status vsv_copy_wait_check(vsv_grid* g, int probe_bytes, double limit_ms) {
  if (!g || probe_bytes < 16 || probe_bytes > (1 << 19) || probe_bytes % 16 || !(limit_ms > 0) ||
      limit_ms > 1e4)
    return VSV_EINVAL;
  if (g->prec != VSV_MIXED || !g->mg_t[0][0] || !g->r0[0])
    return fail(g, VSV_EINVAL, "the fused sweep runs on mixed-precision grids only%s");
  const int per[3] = {1, 0, 1};
  const std::vector<Level> lv = build_levels(g->nx, g->ny, g->nz, g->h, per, 1, 1);
  const Comp3<float> B{{(float*)g->mg_t[0][0], nullptr, nullptr}};
  const Rhs3<float> R{{(const float*)g->r0[0], nullptr, nullptr}, {nullptr, nullptr, nullptr}, 1.f};
  if (!launch_copy_wait_probe(g->cx, lv[0], B, R, (unsigned)probe_bytes,
                              (unsigned long long)(limit_ms * 1e6)))
    return fail(g, VSV_EINVAL, "copy wait check: the grid is not tile-aligned or the launch failed%s");
  CK(cudaStreamSynchronize(g->cx.stream));
  int flag = 0;
  CK(cudaMemcpy(&flag, &g->S->nonfinite, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag & kCopyTimeout) {
    const int cleared = flag & ~kCopyTimeout;
    CK(cudaMemcpy(&g->S->nonfinite, &cleared, sizeof(int), cudaMemcpyHostToDevice));
    return flag_status(g, kCopyTimeout);
  }
  return VSV_OK;
}

const char* vsv_last_error(const vsv_grid* g) { return g ? g->err.c_str() : "null handle"; }

int64_t vsv_kernel_launches(const vsv_grid* g) { return g ? g->cx.launches : 0; }

double vsv_kernel_bytes(const vsv_grid* g) { return g ? g->cx.bytes_total : 0.0; }

vsv_status vsv_profile_enable(vsv_grid* g, int kclass, int enable) {
  if (!g || kclass < 0 || kclass >= VSV_KCLASS_COUNT) return VSV_EINVAL;
  if (g->cx.ev.empty()) {
    g->cx.ev.resize(2 * 8192);
    for (auto& e : g->cx.ev) CK(cudaEventCreate(&e));
  }
  g->cx.prof_class = enable ? kclass : -1;
  g->cx.ev_used = 0;
  g->cx.prof_launches = 0;
  g->cx.prof_bytes = 0.0;
  return VSV_OK;
}

vsv_status vsv_profile_read(vsv_grid* g, int kclass, double* total_ms, int64_t* launches,
                            double* alg_bytes) {
  if (!g || !total_ms || !launches) return VSV_EINVAL;
  if (g->cx.prof_class != kclass) return fail(g, VSV_ESTATE, "profiling not enabled for this class%s");
  CK(cudaStreamSynchronize(g->cx.stream));
  double t = 0.0;
  for (int i = 0; i < g->cx.ev_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, g->cx.ev[2 * i], g->cx.ev[2 * i + 1]));
    t += ms;
  }
  *total_ms = t;
  *launches = g->cx.prof_launches;
  if (alg_bytes) *alg_bytes = g->cx.prof_bytes;
  return VSV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- adjoint tape
// Reverse mode over a recorded trajectory with checkpointing: the forward
// pass keeps the full state (the state blob's fields, on the device) every
// `every` steps and at the last step; the backward pass walks the segments
// from the last to the first, re-runs each segment from its checkpoint while
// recording phi, mu, psi' (FP64) and gamma_A of every step, then reverses its
// steps with the adjoint kernels.  Memory: checkpoints of the state plus one
// segment of (every + 1) x 5 fields, instead of the whole trajectory.
struct vsv_tape {
  vsv_grid* g = nullptr;
  int every = 20;
  double tol = 1e-11;
  int fixed = 0;                       // > 0: cycles per adjoint solve, no host synchronisation
  int nsteps = 0;
  double dt = 0.0;
  bool recorded = false;
  size_t ck_bytes = 0;                 // bytes of one checkpoint
  std::vector<char*> ck;               // device checkpoints ...
  std::vector<int> ck_step;            // ... of the states at these steps
  std::vector<StateHeader> ck_hdr;     // their host-side counters
  double* rec = nullptr;               // (every + 1) x 5 N doubles: phi, mu, psi'(3)
  double* gam = nullptr;               // (every + 1) gamma_A (device)
  double* buf = nullptr;               // adjoint fields, FP64
  float* fbuf = nullptr;               // mixed path: double-word solve iterates and rhs
  double* acc = nullptr;               // kAccCount accumulators
  double* partials = nullptr;          // 3 per reduction block
  size_t dev_bytes = 0;
  // caller-owned device memory (vsv_tape_create_in): every buffer and the
  // checkpoint slots are carved from it; nothing is allocated or freed
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int max_ck = 0;                      // checkpoint slots in ws
  char* ck_pool = nullptr;             // the first of them
  long long adj_cycles = 0;            // cycles of the adjoint solves, last backward pass
  long long recomputed = 0;            // steps re-run by the last backward pass
  // views into buf / fbuf
  double *phib, *mub, *psib[3], *ab[3], *bb[3], *fb[3], *x1[3], *gsc, *wsc;
  double *omc[3], *omt[3];   // inertial variant: the carried vorticity adjoint, a temporary
  float *x1h[3], *x1l[3], *fbh[3], *fbl[3], *bh[3], *bl[3];
};

namespace {

AdjParams adj_params(const vsv_grid* g) {
  AdjParams P{};
  P.nx = g->nx; P.ny = g->ny; P.nz = g->nz;
  P.zper = z_periodic(g) ? 1 : 0;
  P.h = g->h; P.hih = 0.5 / g->h; P.ih2 = 1.0 / (g->h * g->h); P.h3 = g->h * g->h * g->h;
  P.fe_kind = g->fe.kind;
  P.sigma = g->fe.sigma;
  P.eps = g->fe.eps;
  P.e2 = g->fe.eps * g->fe.eps;
  const double cf1 = 3.0 * std::sqrt(2.0) / (8.0 * std::pow(g->fe.eps, 3));   // C_F per unit kappa
  P.cf2_per_kappa = g->fe.mu_prefactor_half ? cf1 : 2.0 * cf1;
  P.cf2 = P.cf2_per_kappa * g->fe.kappa;
  P.beta = g->fe.kind == VSV_HELFRICH ? g->fe.sigma * 3.0 / (2.0 * std::sqrt(2.0) * g->fe.eps) : 0.0;
  P.inv_eta = 1.0 / g->flow.eta;
  P.mobility = g->fe.mobility;
  P.k_vol = g->fe.k_vol;
  P.k_area = g->fe.k_area;
  return P;
}

template <class T>
Comp3<const T> cc3(T* const a[3]) { return Comp3<const T>{{a[0], a[1], a[2]}}; }
template <class T>
Comp3<T> mc3(T* const a[3]) { return Comp3<T>{{a[0], a[1], a[2]}}; }

void tape_free_ckpts(vsv_tape* t) {
  if (!t->ws)
    for (char* p : t->ck) cudaFree(p);
  t->ck.clear();
  t->ck_step.clear();
  t->ck_hdr.clear();
}

// Bytes of one checkpoint: the state fields plus V0 and A0.
size_t tape_ck_bytes(const vsv_grid* g) {
  size_t b = 2 * sizeof(double);
  for (auto& f : state_fields(g)) b += f.second;
  return b;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes of a tape's buffers (without checkpoints), each rounded up
// to 256 bytes as the caller-owned layout carves them.
size_t tape_buffer_bytes(const vsv_grid* g, int every) {
  const size_t N = (size_t)g->N;
  size_t b = round256((size_t)(every + 1) * 5 * N * 8) + round256((size_t)(every + 1) * 8) +
             round256(25 * N * 8) + round256(kAccCount * 8) + round256((size_t)3 * adj_blocks(g->N) * 8);
  if (g->prec == VSV_MIXED) b += round256(18 * N * 4);
  return b;
}

// checkpoints a forward pass of nsteps records: step 0 and every segment end
int tape_ck_count(int nsteps, int every) { return 1 + (nsteps + every - 1) / every; }

vsv_status tape_alloc(vsv_tape* t) {
  vsv_grid* g = t->g;
  const long long N = g->N;
  size_t carved = 0;
  auto dmalloc = [&](void** p, size_t b) -> vsv_status {
    if (t->ws) {
      *p = t->ws + carved;
      carved += round256(b);
      return VSV_OK;
    }
    CK(cudaMalloc(p, b));
    t->dev_bytes += b;
    return VSV_OK;
  };
  vsv_status st;
  if ((st = dmalloc((void**)&t->rec, (size_t)(t->every + 1) * 5 * N * 8)) != VSV_OK) return st;
  if ((st = dmalloc((void**)&t->gam, (size_t)(t->every + 1) * 8)) != VSV_OK) return st;
  if ((st = dmalloc((void**)&t->buf, (size_t)25 * N * 8)) != VSV_OK) return st;
  if ((st = dmalloc((void**)&t->acc, kAccCount * 8)) != VSV_OK) return st;
  if ((st = dmalloc((void**)&t->partials, (size_t)3 * adj_blocks(N) * 8)) != VSV_OK) return st;
  double* p = t->buf;
  auto take = [&]() { double* q = p; p += N; return q; };
  t->phib = take();
  t->mub = take();
  for (int c = 0; c < 3; ++c) t->psib[c] = take();
  for (int c = 0; c < 3; ++c) t->ab[c] = take();
  for (int c = 0; c < 3; ++c) t->bb[c] = take();
  for (int c = 0; c < 3; ++c) t->fb[c] = take();
  for (int c = 0; c < 3; ++c) t->x1[c] = take();
  t->gsc = take();
  t->wsc = take();
  for (int c = 0; c < 3; ++c) t->omc[c] = take();
  for (int c = 0; c < 3; ++c) t->omt[c] = take();
  if (g->prec == VSV_MIXED) {
    if ((st = dmalloc((void**)&t->fbuf, (size_t)18 * N * 4)) != VSV_OK) return st;
    float* f = t->fbuf;
    auto takef = [&]() { float* q = f; f += N; return q; };
    for (int c = 0; c < 3; ++c) t->x1h[c] = takef();
    for (int c = 0; c < 3; ++c) t->x1l[c] = takef();
    for (int c = 0; c < 3; ++c) t->fbh[c] = takef();
    for (int c = 0; c < 3; ++c) t->fbl[c] = takef();
    for (int c = 0; c < 3; ++c) t->bh[c] = takef();
    for (int c = 0; c < 3; ++c) t->bl[c] = takef();
  }
  if (t->ws) t->ck_pool = t->ws + carved;   // checkpoint slots follow the buffers
  return VSV_OK;
}

// state -> checkpoint slot (device to device, asynchronous)
vsv_status tape_save(vsv_tape* t, int step) {
  vsv_grid* g = t->g;
  char* dst = nullptr;
  if (t->ws) {
    if ((int)t->ck.size() >= t->max_ck) return fail(g, VSV_ENOMEM, "tape checkpoint slots exhausted%s");
    dst = t->ck_pool + t->ck.size() * round256(t->ck_bytes);
  } else {
    CK(cudaMalloc((void**)&dst, t->ck_bytes));
  }
  // a failed copy frees a new slot before returning (not yet on the tape)
  auto copy = [&](void* to, const void* from, size_t n) -> cudaError_t {
    const cudaError_t e = cudaMemcpyAsync(to, from, n, cudaMemcpyDeviceToDevice, g->cx.stream);
    if (e != cudaSuccess && !t->ws) cudaFree(dst);
    return e;
  };
  size_t off = 0;
  for (auto& f : state_fields(g)) {
    CK(copy(dst + off, f.first, f.second));
    off += f.second;
  }
  CK(copy(dst + off, &g->S->V0, 2 * sizeof(double)));   // V0, A0 (adjacent in Scalars)
  if (!t->ws) t->dev_bytes += t->ck_bytes;
  StateHeader hd{};
  hd.time = g->time;
  hd.steps = g->steps;
  hd.hist = g->hist;
  t->ck.push_back(dst);
  t->ck_step.push_back(step);
  t->ck_hdr.push_back(hd);
  return VSV_OK;
}

vsv_status tape_restore(vsv_tape* t, int i) {
  vsv_grid* g = t->g;
  const char* src = t->ck[i];
  size_t off = 0;
  for (auto& f : state_fields(g)) {
    CK(cudaMemcpyAsync(f.first, src + off, f.second, cudaMemcpyDeviceToDevice, g->cx.stream));
    off += f.second;
  }
  CK(cudaMemcpyAsync(&g->S->V0, src + off, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                     g->cx.stream));
  g->time = t->ck_hdr[i].time;
  g->steps = t->ck_hdr[i].steps;
  g->hist = t->ck_hdr[i].hist;
  g->phi_set = true;
  g->phase_stale = true;
  return VSV_OK;
}

double* rec_field(vsv_tape* t, int slot, int q) { return t->rec + ((size_t)slot * 5 + q) * t->g->N; }

// phi, mu, psi' (FP64) and gamma_A of the grid's current state into a slot
vsv_status tape_record(vsv_tape* t, int slot) {
  vsv_grid* g = t->g;
  const int fields[5] = {VSV_FIELD_PHI, VSV_FIELD_MU, VSV_FIELD_PSI_PERT_X, VSV_FIELD_PSI_PERT_Y,
                         VSV_FIELD_PSI_PERT_Z};
  for (int q = 0; q < 5; ++q) {
    vsv_status st = g->prec == VSV_FP64
                        ? get_field_impl<double>(g, fields[q], rec_field(t, slot, q), VSV_DTYPE_F64, 1)
                        : get_field_impl<float>(g, fields[q], rec_field(t, slot, q), VSV_DTYPE_F64, 1);
    if (st != VSV_OK) return st;
  }
  // mu's export refreshed the phase of a restored state: gamma_A is current
  CK(cudaMemcpyAsync(t->gam + slot, &g->S->gamma_a, sizeof(double), cudaMemcpyDeviceToDevice,
                     g->cx.stream));
  return VSV_OK;
}

// fbar = L^-1 (-L^-1 psibar) per component: the adjoint of the vorticity and
// stream-vector solves (L symmetric, zero wall data), warm-started from the
// previous reverse step's solutions.  Inertial variant (rho > 0): the
// vorticity of a step came from (L - s) omega = f - s omega_prev, so
// fbar = (L - s)^-1 (omc - L^-1 psibar) with omc the vorticity adjoint
// carried from the later step, and the carry becomes omc = -s fbar;
// `shifted` false (the initial state, whose vorticity is the Stokes one)
// solves with L and leaves the carry alone.
vsv_status tape_solves_inertial(vsv_tape* t, bool shifted);
vsv_status tape_solves(vsv_tape* t, bool shifted) {
  vsv_grid* g = t->g;
  if (g->flow.rho > 0.0) return tape_solves_inertial(t, shifted);
  const int every = std::max(1, g->sol.check_every);
  int c1 = 0, c2 = 0;
  double r1 = 0.0, r2 = 0.0;
  vsv_status st;
  if (g->prec == VSV_FP64) {
    Rhs3<double> R1{{t->psib[0], t->psib[1], t->psib[2]}, {nullptr, nullptr, nullptr}, 1.0};
    st = solve<double>(g, g->flow_levels, mc3(t->x1), R1, 3, VSV_SOLVER_MG, t->fixed, t->tol, 400, every,
                       &c1, &r1);
    if (st != VSV_OK) return st;
    Rhs3<double> R2{{t->x1[0], t->x1[1], t->x1[2]}, {nullptr, nullptr, nullptr}, -1.0};
    st = solve<double>(g, g->flow_levels, mc3(t->fb), R2, 3, VSV_SOLVER_MG, t->fixed, t->tol, 400, every,
                       &c2, &r2);
    if (st != VSV_OK) return st;
  } else {
    for (int c = 0; c < 3; ++c) launch_split_ff(g->cx, t->psib[c], t->bh[c], t->bl[c], g->N);
    Rhs3<float> R1{{t->bh[0], t->bh[1], t->bh[2]}, {nullptr, nullptr, nullptr}, 1.f};
    st = solve_dc(g, g->flow_levels, mc3(t->x1h), mc3(t->x1l), R1, mc3(t->bl), 3, t->fixed, t->tol, 400,
                  every, &c1, &r1);
    if (st != VSV_OK) return st;
    Rhs3<float> R2{{t->x1h[0], t->x1h[1], t->x1h[2]}, {nullptr, nullptr, nullptr}, -1.f};
    st = solve_dc(g, g->flow_levels, mc3(t->fbh), mc3(t->fbl), R2, mc3(t->x1l), 3, t->fixed, t->tol, 400,
                  every, &c2, &r2);
    if (st != VSV_OK) return st;
    for (int c = 0; c < 3; ++c) launch_merge_ff(g->cx, t->fbh[c], t->fbl[c], t->fb[c], g->N);
  }
  t->adj_cycles += c1 + c2;
  return VSV_OK;
}

vsv_status tape_solves_inertial(vsv_tape* t, bool shifted) {
  vsv_grid* g = t->g;
  const long long N = g->N;
  const int every = std::max(1, g->sol.check_every);
  const double s = g->flow.rho / (g->flow.eta * t->dt);
  if (shifted && g->omega_levels.empty())
    return fail(g, VSV_ESTATE, "no shifted hierarchy for the inertial adjoint%s");
  const std::vector<Level>& lv2 = shifted ? g->omega_levels : g->flow_levels;
  int c1 = 0, c2 = 0;
  double r1 = 0.0, r2 = 0.0;
  vsv_status st;
  if (g->prec == VSV_FP64) {
    Rhs3<double> R1{{t->psib[0], t->psib[1], t->psib[2]}, {nullptr, nullptr, nullptr}, 1.0};
    st = solve<double>(g, g->flow_levels, mc3(t->x1), R1, 3, VSV_SOLVER_MG, t->fixed, t->tol, 400,
                       every, &c1, &r1);
    if (st != VSV_OK) return st;
    for (int c = 0; c < 3; ++c) launch_adj_axpby(g->cx, t->omt[c], 1.0, t->omc[c], -1.0, t->x1[c], N);
    Rhs3<double> R2{{t->omt[0], t->omt[1], t->omt[2]}, {nullptr, nullptr, nullptr}, 1.0};
    st = solve<double>(g, lv2, mc3(t->fb), R2, 3, VSV_SOLVER_MG, t->fixed, t->tol, 400, every, &c2,
                       &r2);
    if (st != VSV_OK) return st;
  } else {
    for (int c = 0; c < 3; ++c) launch_split_ff(g->cx, t->psib[c], t->bh[c], t->bl[c], N);
    Rhs3<float> R1{{t->bh[0], t->bh[1], t->bh[2]}, {nullptr, nullptr, nullptr}, 1.f};
    st = solve_dc(g, g->flow_levels, mc3(t->x1h), mc3(t->x1l), R1, mc3(t->bl), 3, t->fixed, t->tol,
                  400, every, &c1, &r1);
    if (st != VSV_OK) return st;
    for (int c = 0; c < 3; ++c) {
      launch_merge_ff(g->cx, t->x1h[c], t->x1l[c], t->omt[c], N);
      launch_adj_axpby(g->cx, t->omt[c], 1.0, t->omc[c], -1.0, t->omt[c], N);
      launch_split_ff(g->cx, t->omt[c], t->bh[c], t->bl[c], N);
    }
    Rhs3<float> R2{{t->bh[0], t->bh[1], t->bh[2]}, {nullptr, nullptr, nullptr}, 1.f};
    st = solve_dc(g, lv2, mc3(t->fbh), mc3(t->fbl), R2, mc3(t->bl), 3, t->fixed, t->tol, 400, every,
                  &c2, &r2);
    if (st != VSV_OK) return st;
    for (int c = 0; c < 3; ++c) launch_merge_ff(g->cx, t->fbh[c], t->fbl[c], t->fb[c], N);
  }
  if (shifted)
    for (int c = 0; c < 3; ++c) launch_adj_scale(g->cx, t->fb[c], t->omc[c], N, -s);
  CKL();
  t->adj_cycles += c1 + c2;
  return VSV_OK;
}

// adjoint of the flow solve and of mu at a recorded state (slot s); with
// `step` the area penalty of gamma_A = K_A c_g (A - A0) too
vsv_status tape_state_adjoint(vsv_tape* t, const AdjParams& P, int s, bool step) {
  vsv_grid* g = t->g;
  vsv_status st = tape_solves(t, step);
  if (st != VSV_OK) return st;
  const double* phi = rec_field(t, s, 0);
  const double* mu = rec_field(t, s, 1);
  launch_adj_source(g->cx, P, phi, mu, cc3(t->fb), mc3(t->ab), mc3(t->bb));
  launch_adj_divt(g->cx, P, cc3(t->ab), t->phib, cc3(t->bb), t->mub);
  launch_adj_mu(g->cx, P, phi, t->mub, step ? t->gam + s : nullptr, t->gsc, t->wsc, t->phib,
                t->partials, t->acc, step);
  if (step && P.fe_kind == VSV_HELFRICH && P.k_area != 0.0)
    launch_adj_area(g->cx, P, phi, t->acc + kAccAreaCoef, nullptr, 0.0, t->phib);
  CKL();
  return VSV_OK;
}

}  // namespace

extern "C" {

vsv_status vsv_tape_create(vsv_tape** out, vsv_grid* g, int every, double tol) {
  if (!out || !g || every < 1 || !(tol >= 0) || !std::isfinite(tol)) return VSV_EINVAL;
  *out = nullptr;
  vsv_tape* t = new vsv_tape();
  t->g = g;
  t->every = every;
  t->tol = tol > 0 ? tol : 1e-11;
  vsv_status st = tape_alloc(t);
  if (st != VSV_OK) {
    vsv_tape_destroy(t);
    return st;
  }
  *out = t;
  return VSV_OK;
}

vsv_status vsv_tape_workspace_bytes(const vsv_grid* g, int every, int max_steps, size_t* bytes) {
  if (!g || !bytes || every < 1 || max_steps < 1) return VSV_EINVAL;
  *bytes = tape_buffer_bytes(g, every) +
           (size_t)tape_ck_count(max_steps, every) * round256(tape_ck_bytes(g));
  return VSV_OK;
}

vsv_status vsv_tape_create_in(vsv_tape** out, vsv_grid* g, int every, int max_steps, double tol,
                              void* workspace, size_t workspace_bytes) {
  if (!out) return VSV_EINVAL;
  *out = nullptr;
  if (!g || every < 1 || max_steps < 1 || !(tol >= 0) || !std::isfinite(tol) || !workspace ||
      ((uintptr_t)workspace & 255))
    return VSV_EINVAL;
  size_t need = 0;
  vsv_tape_workspace_bytes(g, every, max_steps, &need);
  if (workspace_bytes < need) return VSV_ENOMEM;
  cudaPointerAttributes pa{};
  int dev = -1;
  if (cudaPointerGetAttributes(&pa, workspace) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
      cudaGetDevice(&dev) != cudaSuccess || pa.device != dev) {
    cudaGetLastError();
    return VSV_EINVAL;
  }
  vsv_tape* t = new vsv_tape();
  t->g = g;
  t->every = every;
  t->tol = tol > 0 ? tol : 1e-11;
  t->ws = (char*)workspace;
  t->ws_bytes = workspace_bytes;
  t->max_ck = tape_ck_count(max_steps, every);
  t->ck_bytes = tape_ck_bytes(g);
  t->dev_bytes = need;
  vsv_status st = tape_alloc(t);
  if (st != VSV_OK) {
    vsv_tape_destroy(t);
    return st;
  }
  *out = t;
  return VSV_OK;
}

vsv_status vsv_tape_destroy(vsv_tape* t) {
  if (!t) return VSV_OK;
  if (t->g) cudaStreamSynchronize(t->g->cx.stream);
  tape_free_ckpts(t);
  if (!t->ws) {
    cudaFree(t->rec);
    cudaFree(t->gam);
    cudaFree(t->buf);
    cudaFree(t->fbuf);
    cudaFree(t->acc);
    cudaFree(t->partials);
  }
  delete t;
  return VSV_OK;
}

size_t vsv_tape_bytes(const vsv_tape* t) { return t ? t->dev_bytes : 0; }

vsv_status vsv_tape_set_cycles(vsv_tape* t, int fixed_cycles) {
  if (!t || fixed_cycles < 0) return VSV_EINVAL;
  t->fixed = fixed_cycles;
  return VSV_OK;
}

vsv_status vsv_tape_info(const vsv_tape* t, int64_t* adjoint_cycles, int64_t* recomputed_steps,
                         int* checkpoints) {
  if (!t) return VSV_EINVAL;
  if (adjoint_cycles) *adjoint_cycles = t->adj_cycles;
  if (recomputed_steps) *recomputed_steps = t->recomputed;
  if (checkpoints) *checkpoints = (int)t->ck.size();
  return VSV_OK;
}

}  // extern "C"

extern "C" {

vsv_status vsv_tape_forward(vsv_tape* t, const void* phi0, int dtype, int on_device, int nsteps,
                            double dt) {
  if (!t || !phi0 || nsteps < 1 || !(dt > 0) || on_device < 0 || on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  if (on_device == VSV_HOST_ASYNC) on_device = 0;
  vsv_grid* g = t->g;
  if (!g->flow_set) return fail(g, VSV_ESTATE, "vsv_set_flow must precede vsv_tape_forward%s");
  if (g->motion_on)
    return fail(g, VSV_EINVAL, "the adjoint tape needs steady walls (vsv_set_wall_motion)%s");
  if (t->ws && tape_ck_count(nsteps, t->every) > t->max_ck)
    return fail(g, VSV_ENOMEM, "more steps than the tape's workspace was sized for%s");
  CK(cudaStreamSynchronize(g->cx.stream));
  tape_free_ckpts(t);
  if (!t->ws)
    t->dev_bytes = (size_t)(t->every + 1) * 5 * g->N * 8 + (size_t)(t->every + 1) * 8 +
                   (size_t)25 * g->N * 8 + kAccCount * 8 + (size_t)3 * adj_blocks(g->N) * 8 +
                   (g->prec == VSV_MIXED ? (size_t)18 * g->N * 4 : 0);
  t->recorded = false;
  t->ck_bytes = tape_ck_bytes(g);
  vsv_status st = vsv_set_phi(g, phi0, dtype, on_device);
  if (st != VSV_OK) return st;
  if ((st = tape_save(t, 0)) != VSV_OK) return st;
  int done = 0;
  while (done < nsteps) {
    const int k = std::min(t->every, nsteps - done);
    if ((st = vsv_step(g, k, dt)) != VSV_OK) return st;
    done += k;
    if ((st = tape_save(t, done)) != VSV_OK) return st;
  }
  if ((st = vsv_check(g)) != VSV_OK) return st;
  t->nsteps = nsteps;
  t->dt = dt;
  t->recorded = true;
  return VSV_OK;
}

vsv_status vsv_tape_backward(vsv_tape* t, const double* phibar_final, double* phibar0,
                             int on_device, double* param_bar) {
  if (!t || !phibar_final || !phibar0 || on_device < 0 || on_device > VSV_HOST_ASYNC)
    return VSV_EINVAL;
  if (on_device == VSV_HOST_ASYNC) on_device = 0;
  vsv_grid* g = t->g;
  if (!t->recorded) return fail(g, VSV_ESTATE, "vsv_tape_forward must precede vsv_tape_backward%s");
  const long long N = g->N;
  const AdjParams P = adj_params(g);
  cudaStream_t s = g->cx.stream;
  t->adj_cycles = 0;
  t->recomputed = 0;
  // terminal adjoint: phibar^N given, mubar^N = psibar'^N = 0; zero warm starts
  CK(cudaMemcpyAsync(t->phib, phibar_final, N * 8,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(t->mub, 0, N * 8, s));
  for (int c = 0; c < 3; ++c) {
    CK(cudaMemsetAsync(t->omc[c], 0, N * 8, s));
    CK(cudaMemsetAsync(t->psib[c], 0, N * 8, s));
    CK(cudaMemsetAsync(t->fb[c], 0, N * 8, s));
    CK(cudaMemsetAsync(t->x1[c], 0, N * 8, s));
  }
  if (t->fbuf) CK(cudaMemsetAsync(t->fbuf, 0, (size_t)18 * N * 4, s));
  CK(cudaMemsetAsync(t->acc, 0, kAccCount * 8, s));
  Comp3<const double> V0{{g->v0d[0], g->v0d[1], g->v0d[2]}};
  vsv_status st;
  const int nck = (int)t->ck.size();
  for (int seg = nck - 2; seg >= 0; --seg) {
    const int a = t->ck_step[seg], b = t->ck_step[seg + 1];
    // re-run the segment from its checkpoint, recording every state
    if ((st = tape_restore(t, seg)) != VSV_OK) return st;
    if ((st = tape_record(t, 0)) != VSV_OK) return st;
    for (int n = a; n < b; ++n) {
      st = g->prec == VSV_FP64 ? step_impl<double>(g, t->dt) : step_impl<float>(g, t->dt);
      if (st != VSV_OK) return st;
      if ((st = tape_record(t, n + 1 - a)) != VSV_OK) return st;
      ++t->recomputed;
    }
    // reverse its steps: state n + 1 (flow solve, mu, gamma_A), then the update n -> n + 1
    for (int n = b - 1; n >= a; --n) {
      if ((st = tape_state_adjoint(t, P, n + 1 - a, true)) != VSV_OK) return st;
      launch_adj_update(g->cx, P, t->phib, rec_field(t, n - a, 0),
                        Comp3<const double>{{rec_field(t, n - a, 2), rec_field(t, n - a, 3),
                                             rec_field(t, n - a, 4)}},
                        V0, t->dt, mc3(t->ab), mc3(t->bb), t->mub, mc3(t->psib), t->partials, t->acc);
      CKL();
    }
  }
  // the initial state: mu^0 and psi^0 of phi^0 (gamma^0 = 0 identically),
  // then V0 = V[phi^0] and A0 = A[phi^0]
  if ((st = tape_state_adjoint(t, P, 0, false)) != VSV_OK) return st;
  launch_adj_area(g->cx, P, rec_field(t, 0, 0), P.fe_kind == VSV_HELFRICH ? t->acc + kAccA0 : nullptr,
                  t->acc + kAccV0, -0.5 * P.h3, t->phib);
  CKL();
  CK(cudaMemcpyAsync(phibar0, t->phib, N * 8,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  double hacc[kAccCount];
  CK(cudaMemcpyAsync(hacc, t->acc, sizeof hacc, cudaMemcpyDeviceToHost, s));
  // leave the grid at the end of the trajectory
  if ((st = tape_restore(t, nck - 1)) != VSV_OK) return st;
  CK(cudaStreamSynchronize(s));
  if (param_bar) {
    param_bar[0] = hacc[kAccKappa];
    param_bar[1] = hacc[kAccSigma];
  }
  return VSV_OK;
}

}  // extern "C"
