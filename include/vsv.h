/*
 * vsv.h -- C ABI of the GB300 vorticity--stream-vector phase-field library.
 *
 * The library advances the system of Gallen et al. ("Deformable bodies in a
 * 3-dimensional viscous flow: vorticity-stream vector formulation"),
 * main-text eqs. gen2, gen1, gen3 (= supplementary eq. 29):
 *
 *     d(phi)/dt  = M (lap mu + lambda_V) - (curl psi) . grad phi
 *     lap omega  = (1/eta) grad phi x grad mu
 *     lap psi    = -omega,          v = curl psi   (eq. vecpot)
 *
 * on a uniform cubic grid (numerical-implementation section), forward Euler
 * for phi and the segregated order "advance phi, solve omega, solve psi"
 * within one step.  Every step runs as CUDA kernels on one GPU, enqueued on
 * the caller's stream; there is no CPU fallback.
 *
 * Grid and layout.  nx x ny x nz cells of spacing h; x is the periodic flow
 * axis (boundary-conditions section: periodic in the flow direction), y is
 * always walled, z is walled (duct, quiescent) or periodic (Couette, planar
 * Poiseuille).  Every field crossing this ABI is a dense C-ordered array
 * [nz][ny][nx] (x fastest) without halos.  Flow walls sit on the ghost
 * nodes j = -1 and j = n, where omega and psi take the body-free flow's
 * values (boundary-conditions section); phi and mu have no-flux (mirror)
 * walls.
 *
 * Precision.  VSV_FP64 stores and computes everything in FP64.  VSV_MIXED
 * stores fields in FP32 and smooths in FP32; the defect b - L x driving each
 * multigrid correction is evaluated exactly (error-free FP32 transforms,
 * i.e. at least FP64 accuracy) before rounding, and all volume / area /
 * norm / stress reductions accumulate in FP64.
 *
 * Ownership.  The caller owns the device workspace, the stream and every
 * input / output buffer; the library owns only the opaque host handle.  The
 * workspace must stay valid until vsv_destroy.  A handle is not thread-safe;
 * calls on one handle must be serialised by the caller.
 *
 * Errors.  Every function returns a vsv_status (0 = success); none aborts or
 * exits.  After a failure vsv_last_error() describes it.  Kernel launches are
 * asynchronous: faults inside kernels surface at the next synchronising call
 * (vsv_check, vsv_get_field to host, vsv_get_diagnostics).
 */
#ifndef VSV_H
#define VSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vsv_grid vsv_grid;

typedef enum {
  VSV_OK = 0,
  VSV_EINVAL = -1,       /* bad argument or shape; nothing was launched        */
  VSV_ENOMEM = -2,       /* workspace smaller than vsv_workspace_bytes()       */
  VSV_ECUDA = -3,        /* a CUDA runtime call failed (message has the name)  */
  VSV_ENOCONV = -4,      /* Poisson solve hit max_cycles above tol; fields valid */
  VSV_ENONFINITE = -5,   /* a NaN / Inf appeared in phi (device flag)          */
  VSV_EUNSTABLE = -6,    /* dt above the explicit stability bound              */
  VSV_ESTATE = -7        /* call out of order (e.g. step before set_phi)       */
} vsv_status;

typedef enum { VSV_FP64 = 0, VSV_MIXED = 1 } vsv_precision;

/* Body-free flows supplying the wall data (boundary-conditions section). */
typedef enum {
  VSV_POISEUILLE_DUCT = 0,   /* walls in y and z, pressure-driven along x     */
  VSV_POISEUILLE_PLANAR = 1, /* walls in y, z periodic                        */
  VSV_COUETTE = 2,           /* walls in y moving along x, z periodic         */
  VSV_QUIESCENT = 3          /* walls in y and z at rest                      */
} vsv_flow_kind;

/* Free energies: Cahn-Hilliard (eq. 31) or phase-field Helfrich (eq. 30). */
typedef enum { VSV_CAHN_HILLIARD = 0, VSV_HELFRICH = 1 } vsv_fe_kind;

typedef enum { VSV_SOLVER_MG = 0, VSV_SOLVER_SOR = 1 } vsv_solver_kind;
typedef enum { VSV_DTYPE_F32 = 0, VSV_DTYPE_F64 = 1 } vsv_dtype;

/* Memory kind of the on_device argument of the transfer calls: 0 host
 * memory (synchronous: the call returns when the data has moved), 1 device
 * memory, VSV_HOST_ASYNC page-locked host memory moved asynchronously (FP64
 * phi on the mixed path: vsv_set_field and vsv_get_field enqueue the copy on
 * a copy stream of the grid's and return at once; the host buffer must stay
 * unchanged after a set, and holds the data after a get, only once vsv_check
 * has returned; for every other field, dtype or precision it acts as 0). */
#define VSV_HOST_ASYNC 2

typedef enum {
  VSV_FIELD_PHI = 0,
  VSV_FIELD_MU = 1,
  VSV_FIELD_OMEGA_X = 2, VSV_FIELD_OMEGA_Y = 3, VSV_FIELD_OMEGA_Z = 4,   /* full omega */
  VSV_FIELD_PSI_X = 5, VSV_FIELD_PSI_Y = 6, VSV_FIELD_PSI_Z = 7,         /* full psi   */
  VSV_FIELD_VEL_X = 8, VSV_FIELD_VEL_Y = 9, VSV_FIELD_VEL_Z = 10,        /* v = curl psi */
  VSV_FIELD_STRESS_T = 11,          /* sigma_t of the in-plane-shear section        */
  VSV_FIELD_OMEGA_PERT_X = 12, VSV_FIELD_OMEGA_PERT_Y = 13, VSV_FIELD_OMEGA_PERT_Z = 14,
  VSV_FIELD_PSI_PERT_X = 15, VSV_FIELD_PSI_PERT_Y = 16, VSV_FIELD_PSI_PERT_Z = 17,
  VSV_FIELD_COUNT = 18
} vsv_field;

/* Body-free flow.  u_max: Poiseuille maximum speed over the cells;
 * v_lo / v_hi: Couette wall speeds (along x) at the y = 0 and y = H walls;
 * eta: dynamic viscosity (eq. gen1).
 * rho: fluid density.  0 (the paper's results) gives the non-inertial
 * vorticity equation gen1.  rho > 0 selects the inertial variant of SM
 * eq. 36, (rho / eta) d omega / dt - lap omega = -(1/eta) grad phi x grad mu,
 * advanced by one backward-Euler step per time step:
 * (lap - s) omega^{n+1} = f - s omega^n with s = rho / (eta dt), solved by the
 * same multigrid with the shifted operator.  vsv_set_phi still starts from
 * the non-inertial vorticity of phi^0.  rho < 0 or non-finite: VSV_EINVAL. */
typedef struct {
  int kind;
  double u_max;
  double v_lo;
  double v_hi;
  double eta;
  double rho;
} vsv_flow_params;

/* Time-dependent walls (supplementary material, the time-dependency
 * paragraph after eq. 36: a flow that speeds up, slows down or oscillates
 * changes only the boundary conditions).  Wall w's speed at time t becomes
 *   s_w(t) = s_w + ramp[w] t + amplitude[w] sin(2 pi frequency[w] t + phase[w])
 * where s_w is the steady speed of vsv_set_flow: w = 0 is the Couette wall at
 * y = 0 (v_lo) or the Poiseuille speed u_max, w = 1 the Couette wall at
 * y = H (v_hi; must be all zero for Poiseuille).  t is the simulation time
 * (0 at vsv_set_phi; restored by vsv_set_state). */
typedef struct {
  double ramp[2];
  double amplitude[2];
  double frequency[2];
  double phase[2];
} vsv_wall_motion;

/* Free energy.  sigma: CH gradient coefficient, or for the Helfrich kind the
 * membrane tension, which adds sigma A_f[phi] to the energy (A_f: the area
 * functional of SM eq. 32 with the gradient summed over cell faces) and
 * (3 / (2 sqrt2 eps)) sigma g to mu; kappa, eps: Helfrich bending
 * modulus and interface width (also the width in the area functional, SM
 * eq. 32); mobility M; k_area, k_vol: penalty stiffnesses of the area and
 * volume multipliers (gamma_A = k_area (A - A0) 3 eps / (2 sqrt 2),
 * lambda_V = k_vol (V - V0)); mu_prefactor_half selects the SM eq. 35
 * prefactor 3 sqrt2 kappa / (8 eps^3) instead of the exact derivative of
 * eq. 30 (twice that). */
typedef struct {
  int kind;
  double sigma;
  double kappa;
  double eps;
  double mobility;
  double k_area;
  double k_vol;
  int mu_prefactor_half;
} vsv_fe_params;

/* Poisson solver (the paper says only "an iterative method").
 * kind: MG (cell-centred V-cycles, red-black Gauss-Seidel smoothing) or SOR
 *   (red-black, FP64 only).
 * fixed_cycles > 0: every solve inside vsv_step runs exactly that many
 *   V-cycles (SOR: sweeps) with no host synchronisation; 0: iterate until
 *   ||b - L x||_2 <= tol ||b||_2 or max_cycles, checking every check_every.
 * nu1 / nu2: pre / post smoothing sweeps; max_levels: multigrid depth cap;
 * coarse_sweeps: red-black sweeps on the coarsest level (capped at twice
 *   that level's longest extent, and at least 4); omega_sor <= 0
 * picks the optimal SOR weight for the grid.  variant 0 uses the fastest
 * kernels available for each level (fused single-pass red-black sweeps,
 * tiled transfers and defects where the tile shape allows, the lower levels
 * of a V-cycle in one launch), with partial edge tiles on levels whose
 * extents are not multiples of the 128 x 16 tile; 1 forces the reference
 * per-level, per-colour kernels (same arithmetic, bit-identical results; for
 * cross-checks); 2 is 0 without partial tiles (fast kernels on tile-aligned
 * levels only, per-colour kernels elsewhere; also bit-identical).
 * extrapolate: order of the first guess of each solve of a time step, from
 * the previous solutions: 0 starts from x^n; 1 from 2 x^n - x^{n-1} (linear
 * extrapolation in time, initial error O(dt^2) instead of O(dt)); 2 from
 * 3 x^n - 3 x^{n-1} + x^{n-2} (quadratic, O(dt^3)).  The order drops to what
 * the history allows for the first steps after vsv_set_phi, vsv_set_field
 * of omega' / psi', or vsv_set_state of a blob without history.  It changes
 * the iterate, not the converged answer.  Values outside 0..2: VSV_EINVAL. */
typedef struct {
  int kind;
  double tol;
  int max_cycles;
  int fixed_cycles;
  int check_every;
  int nu1;
  int nu2;
  int max_levels;
  int coarse_sweeps;
  double omega_sor;
  int variant;
  int extrapolate;
  int fixed_cycles_psi;   /* > 0: fixed cycle count of the stream-vector solves
                             (fixed_cycles then applies to the vorticity
                             solves only); 0: same as fixed_cycles */
  double omega_mg;        /* relaxation weight of the multigrid smoothing
                             sweeps, red-black SOR (every level but the
                             coarsest, which keeps Gauss-Seidel): x <- x +
                             omega_mg (x_GS - x).  0 or 1: Gauss-Seidel.
                             Default 1.3, where a V(2,2)-cycle contracts
                             the error about 3x more than with 1.  It
                             changes the iterate, not the converged answer.
                             Outside [0, 2): VSV_EINVAL. */
  int lower_cycle;        /* the levels below the finest of a V-cycle (variant
                             0 only): 0 (default) level by level; 1 in one
                             cooperative launch (grid-wide red-black sweeps
                             and transfers separated by bounded grid
                             barriers, then the one-CTA coarse cycle) where
                             those levels do not fit one CTA's shared memory.
                             Bit-identical results either way; on GB300 the
                             single launch measured slower at every size
                             tried.  Outside 0..1: VSV_EINVAL. */
  int component_streams;  /* 1: fixed-cycle mixed-precision steps run each
                             component's vorticity and stream-vector solves
                             on a stream of its own (two created with the
                             grid, forked from and joined back to the grid's
                             stream within the step, also inside captured
                             graphs), so that one component's latency-bound
                             coarse levels overlap the others' finest-level
                             kernels; bit-identical results.  0: the
                             components together on the grid's stream.  2
                             (default): 1 on grids of at least 2^24 cells,
                             else 0 (on small grids the tripled launch count
                             costs more than the overlap gains).  Off while
                             a kernel class is being profiled or with
                             lower_cycle = 1.  Outside 0..2: VSV_EINVAL. */
  int launch_overlap;     /* 1: the step's solver and phase-field kernels
                             are launched with programmatic stream
                             serialisation, so that each is scheduled onto
                             the SMs while the kernel before it in its
                             stream drains and starts work the moment that
                             kernel has completed (it waits for it before
                             its first memory access); 0: plain launches.
                             2 (default): 1 on grids of at least 2^24
                             cells, else 0 (small grids usually run many
                             side by side, where the waiting kernels hold
                             SM slots that the other grids' kernels would
                             use).  Bit-identical results.  Plain launches
                             while a kernel class is being profiled.
                             Outside 0..2: VSV_EINVAL. */
} vsv_solver_params;

/* Per-axis boundary of a standalone Poisson problem: periodic (1) or zero
 * Dirichlet data on the ghost nodes -1 and n (0).  Order x, y, z.
 * shift >= 0: solve the shifted problem (L_h - shift) x = rhs instead (the
 * operator of one backward-Euler step of the inertial vorticity equation,
 * SM eq. 36); 0 for the Poisson problem. */
typedef struct {
  int periodic[3];
  double shift;
} vsv_bc;

/* Observables (in-plane-shear section, results section, SM eq. 40). */
typedef struct {
  double time;
  int64_t steps;
  double volume;          /* V = h^3/2 sum (1 - phi)                          */
  double area;            /* A of SM eq. 32                                   */
  double volume0, area0;  /* reference values fixed by vsv_set_phi             */
  double reduced_volume;  /* SM eq. 40                                        */
  double energy;          /* Helfrich C_F h^3 sum g^2, or CH energy            */
  double lambda_v, gamma_a;
  double com[3];          /* centre of the body, weights (1 - phi)/2          */
  double dissipation;     /* (eta/2) int sum_ij (d_j v_i + d_i v_j)^2           */
  double dissipation0;    /* same for the body-free flow                        */
  double resistance_rel;  /* (D - D0) / D0                                      */
  double omega_dev2;      /* int |omega - omega0|^2                             */
  double psi_dev2;        /* int |psi - psi0|^2                                 */
  double max_div_v, max_div_psi, max_sigma_t;
  int last_cycles_omega, last_cycles_psi;   /* of the last step's solves        */
  double last_relres_omega, last_relres_psi;/* -1 when not measured             */
  int nonfinite;
} vsv_diag;

/* Library version string. */
const char* vsv_version(void);

/* Bytes of device workspace a grid needs (all fields, the multigrid
 * hierarchy, base-flow tables, reduction scratch).  0 for invalid shapes. */
size_t vsv_workspace_bytes(int nx, int ny, int nz, int precision);

/* Create a grid over caller-owned device memory `workspace` (>= 256-byte
 * aligned, ws_bytes >= vsv_workspace_bytes) and caller stream `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  Periodic axes must have
 * even extent or extent 1.  Defaults: quiescent flow, eta = 1, CH with
 * sigma = eps = M = 1, default solver for the precision.  The handle holds
 * all the library's own memory: host state, one page-locked 4-byte word
 * into which vsv_step copies its deferred status, and CUDA events; no call
 * on the grid allocates device memory (the tape's convenience constructor
 * vsv_tape_create aside). */
vsv_status vsv_create(vsv_grid** out, int nx, int ny, int nz, double h, int precision,
                      void* workspace, size_t ws_bytes, void* cuda_stream);

/* Free the host handle with its page-locked word and events (the
 * workspace stays the caller's).  NULL is a no-op. */
vsv_status vsv_destroy(vsv_grid* g);

/* Choose the body-free flow (builds the wall data and base-flow tables on
 * the device; a duct runs 2-D FP64 Poisson solves).  Must precede set_phi. */
vsv_status vsv_set_flow(vsv_grid* g, const vsv_flow_params* fp);
vsv_status vsv_set_free_energy(vsv_grid* g, const vsv_fe_params* fe);

/* Make the walls of the flow time-dependent (vsv_wall_motion; NULL or all
 * zero: steady walls again).  A step n -> n+1 advects phi with the flow of
 * time t^n and solves for omega, psi with the wall data of t^{n+1}; the
 * base-flow tables are recombined on the device every step from tables of
 * unit wall speeds, so CUDA graphs of steps (vsv_batch_step) replay it too.
 * Exports and observables see the walls of the current time.  Must follow
 * vsv_set_flow (which resets the walls to steady); takes effect at the
 * current time.  VSV_EINVAL: non-finite entries, motion of a quiescent flow
 * or of wall 1 of a Poiseuille flow, or an inertial flow (rho > 0);
 * VSV_ESTATE before vsv_set_flow.  The adjoint tape refuses a grid with
 * moving walls (VSV_EINVAL from vsv_tape_forward). */
vsv_status vsv_set_wall_motion(vsv_grid* g, const vsv_wall_motion* m);
vsv_status vsv_set_solver(vsv_grid* g, const vsv_solver_params* sp);
vsv_status vsv_default_solver(vsv_solver_params* out, int precision);

/* Load phi^0 (dtype VSV_DTYPE_*, host or device pointer), then compute mu,
 * V0 = V[phi^0], A0 = A[phi^0] and solve omega, psi for phi^0 (zero initial
 * guess, iterating to tol).  Returns VSV_ENOCONV if a solve stalls. */
vsv_status vsv_set_phi(vsv_grid* g, const void* phi, int dtype, int on_device);

/* Advance nsteps steps of size dt (step order in the file comment).
 * Asynchronous when the solver uses fixed_cycles; returns VSV_EUNSTABLE if
 * dt exceeds vsv_stability_limit, VSV_ENONFINITE if the previous step set
 * the non-finite flag. */
vsv_status vsv_step(vsv_grid* g, int nsteps, double dt);

/* Largest dt the explicit update tolerates (linear analysis about phi = +-1:
 * Model-B diffusion of the chosen mu, and the volume penalty). */
vsv_status vsv_stability_limit(const vsv_grid* g, double* dt_max);

/* Standalone Poisson solve L_h x = rhs (or (L_h - bc->shift) x = rhs) on
 * this grid's shape with boundary `bc`, spacing h, using the grid's solver
 * and precision.  All-periodic boundaries need shift > 0 (else VSV_EINVAL,
 * as for a negative or non-finite shift).  rhs and x are
 * [nz][ny][nx] arrays of dtype on host or device; x holds the initial guess
 * on entry.  Uses the grid's scratch (it clobbers the grid's flow
 * perturbation of component z; call vsv_set_phi again afterwards to resume
 * time stepping).  cycles_out / relres_out may be NULL. */
vsv_status vsv_solve_poisson(vsv_grid* g, const void* rhs, void* x, int dtype, int on_device,
                             const vsv_bc* bc, double tol, int max_cycles, int* cycles_out,
                             double* relres_out);

/* Copy a field out (full omega / psi include the base flow).  Synchronous
 * for host destinations (on_device 0).  On the mixed path an FP64 phi is
 * merged from its two words into a device staging buffer and crosses to
 * host memory by the copy engine (faster over the host link than a kernel
 * writing mapped memory); with on_device = VSV_HOST_ASYNC that copy runs on
 * the grid's export stream and the call returns at once (valid after
 * vsv_check).  The bits are the same either way; dst needs no alignment. */
vsv_status vsv_get_field(vsv_grid* g, int field, void* dst, int dtype, int on_device);

/* Replace phi (mu, V, A are recomputed before the next step; V0, A0 and the
 * flow are kept) or a perturbation component OMEGA_PERT_* / PSI_PERT_*.  On
 * the mixed path FP64 input in page-locked, mapped host memory is read in
 * place by the kernel that splits it into the two words; other host memory
 * is copied through a staging buffer first.  With on_device =
 * VSV_HOST_ASYNC (FP64 phi, mixed path) the copy engine fills a staging
 * buffer on the grid's import stream, overlapping the grid's earlier work,
 * the split waits for it, and the call returns at once (src must stay
 * unchanged until vsv_check). */
vsv_status vsv_set_field(vsv_grid* g, int field, const void* src, int dtype, int on_device);

/* Observables of the current state; synchronises. */
vsv_status vsv_get_diagnostics(vsv_grid* g, vsv_diag* out);

/* <sigma_xy> averaged over x and z, one value per y row (ny doubles, host). */
vsv_status vsv_get_stress_profile(vsv_grid* g, double* out);

/* Checkpoint / resume: a flat host blob of the state (phi, omega', psi', the
 * previous step's omega' and psi', V0, A0, time, step count); resuming from
 * it continues bit-identically. */
size_t vsv_state_bytes(const vsv_grid* g);
vsv_status vsv_get_state(vsv_grid* g, void* dst, size_t bytes);
vsv_status vsv_set_state(vsv_grid* g, const void* src, size_t bytes);

/* Volume and area of a phase field without any device allocation.  The
 * paper has no counterpart: this is an interface for callers that may not
 * allocate device memory -- a plugin whose host application owns every
 * device allocation, or a latency-critical loop that cannot afford the
 * device-wide synchronisation a cudaMalloc / cudaFree may cause.
 * It computes the two numbers vsv_get_diagnostics reports as volume and
 * area: V = h^3/2 sum (1 - phi), and A = h^3 sum of the area density
 * 3/(2 sqrt2) [eps/2 |grad phi|^2 + (phi^2 - 1)^2 / (4 eps)] with central
 * differences (periodic x, mirror y, mirror or periodic z), with its
 * scratch in a fixed 1 MiB file-scope device array of per-row partial sums.
 *   phi: device pointer to an FP64 [nz][ny][nx] field (read only).
 *   out: device pointer to two doubles, written V then A.
 *   cuda_stream: cudaStream_t to run on (NULL = legacy default stream); the
 *   call is asynchronous on it.
 * phi and out must be device (or managed) memory of the current device, and
 * the stream a stream of that device; otherwise VSV_EINVAL and nothing is
 * launched.  An error already pending from earlier work on this thread
 * (cudaPeekAtLastError) makes the call return VSV_ECUDA without launching
 * and without clearing it.
 * Limit: ny * nz <= 65536 (y, z) rows; larger shapes return VSV_EINVAL and
 * launch nothing.  The first call on a device looks up the array's device
 * address while that device is current; make that first call before any
 * stream capture.  All calls in the process share the array, which keeps
 * the last call's partial sums; two calls whose kernels overlap on the GPU
 * race on it.  Never calls cudaMalloc or cudaFree. */
vsv_status vsv_volume_area_static(const double* phi, int nx, int ny, int nz, double h, double eps,
                                  int z_periodic, double* out, void* cuda_stream);

/* Synchronise the stream and report deferred kernel errors / flags: a
 * non-finite phi (VSV_ENONFINITE), a grid barrier of the single-launch lower
 * V-cycle whose wait ran out, or a fused smoothing sweep whose staged planes
 * did not arrive in time (VSV_ECUDA; every such wait gives up after about a
 * second, so no launch can hang; the flag stays set). */
vsv_status vsv_check(vsv_grid* g);

/* Check of the bounded grid barrier that the single-launch lower V-cycle
 * uses (the paper has no counterpart; this serves tests).  Runs `rounds`
 * barriers of a cooperative launch of `blocks` CTAs on the grid's stream,
 * each barrier expecting `extra_arrivals` more CTAs than the launch has:
 * with 0 every barrier completes; with more, arrivals that never come, so
 * every wait runs out after limit_ms milliseconds and the kernel returns.
 * Synchronises.  Returns VSV_OK when all barriers completed, VSV_ECUDA (the
 * timeout message) when a wait ran out, VSV_EINVAL for bad arguments
 * (blocks < 1 or more than can be co-resident, rounds < 1, limit_ms <= 0
 * or above 10000).  It uses the grid's barrier counter and a flag bit it
 * clears again before returning; it touches no field. */
vsv_status vsv_barrier_check(vsv_grid* g, int blocks, int rounds, int extra_arrivals,
                             double limit_ms);

/* Check of the bounded waits of the fused smoothing sweep for its staged
 * planes (the paper has no counterpart; this serves tests).  On tile-aligned
 * mixed-precision grids (nx a multiple of 128, ny of 16) the sweep stages
 * rows of x and of the right-hand side by bulk copies whose arrival a
 * shared-memory barrier counts in bytes.  This runs one such sweep on the
 * grid's finest-level scratch buffers with every copy group expecting
 * probe_bytes bytes (a multiple of 16, 16 .. 524288) that no copy delivers:
 * every wait runs out after limit_ms milliseconds, the kernel sets a flag bit
 * and returns.  Synchronises.  Returns VSV_ECUDA (the timeout message) when
 * the waits ran out, as they must; VSV_EINVAL for bad arguments or a grid
 * the sweep does not serve.  It clears the flag bit again before returning;
 * the scratch buffers' contents are not defined afterwards (every solve
 * rewrites them), no field is touched. */
vsv_status vsv_copy_wait_check(vsv_grid* g, int probe_bytes, double limit_ms);

/* Message of the last failure on this handle ("" if none); the pointer stays
 * valid until the next call on the handle. */
const char* vsv_last_error(const vsv_grid* g);

/* Kernel accounting.  vsv_kernel_launches: kernels this handle has launched.
 * Profiling brackets every launch of one kernel class with CUDA events on the
 * grid's stream; vsv_profile_read synchronises and returns the summed device
 * time and launch count since the last vsv_profile_enable, and (alg_bytes not
 * NULL) the summed algorithmic memory traffic of those launches: the bytes
 * each kernel must read and write at least (fused sweep: 12 per cell and
 * component, 8 when the input is known to be zero, 24 when it also updates
 * the double-word iterate; tiled defect 16 or 20, tiled restriction and
 * prolongation 8.5 per fine cell).  Launches of kernels without a tally add
 * 0.  Fails with VSV_ESTATE if that class is not being profiled. */
typedef enum {
  VSV_KCLASS_SMOOTH = 0,        /* red-black Gauss-Seidel sweeps, all levels   */
  VSV_KCLASS_SMOOTH_FINE = 1,   /* red-black sweeps on the finest level only   */
  VSV_KCLASS_RESTRICT = 2,      /* exact residual + restriction                */
  VSV_KCLASS_PROLONG = 3,       /* prolongation + correction                   */
  VSV_KCLASS_PHASE = 4,         /* phi update, mu, source, reductions          */
  VSV_KCLASS_ADJOINT = 5,       /* stencil kernels of the discrete adjoint     */
  VSV_KCLASS_COUNT = 6
} vsv_kernel_class;
int64_t vsv_kernel_launches(const vsv_grid* g);
/* Algorithmic memory traffic, in bytes, of all kernels this handle has
 * launched that carry a tally (every kernel of vsv_step and of the solves):
 * for each launch, the bytes it must read and write at least (each input
 * word read once, each output word written once; the per-kernel counts are
 * listed with vsv_profile_read).  A host-side counter; no synchronisation.
 * Divided by a measured time it gives the achieved HBM bandwidth of a step
 * in the algorithmic sense.  0 for a NULL handle. */
double vsv_kernel_bytes(const vsv_grid* g);
vsv_status vsv_profile_enable(vsv_grid* g, int kernel_class, int enable);
vsv_status vsv_profile_read(vsv_grid* g, int kernel_class, double* total_ms, int64_t* launches,
                            double* alg_bytes);

/* Batched stepping of independent grids.  The paper simulates one body at a
 * time and has no counterpart; this serves many small problems at once (a
 * parameter sweep), where launch latency, not bandwidth, bounds a step.
 *
 * vsv_batch_create groups n existing grids (each with its own workspace and
 * stream, vsv_set_phi done, solver in fixed_cycles mode) under a master
 * stream `cuda_stream`, which must be a created stream (graphs cannot be
 * captured on the legacy default stream).  The batch does not own the
 * grids: destroy it before them.  VSV_EINVAL on n < 1, NULL or repeated
 * grids, or a NULL / legacy master stream.
 *
 * vsv_batch_step advances every grid by nsteps steps of dt.  Each grid first
 * takes plain steps, on its own stream, until its solution history is full
 * and its phase fields are current.  Then one CUDA graph is captured with
 * six steps of every grid, each grid on its own branch so that small grids
 * run concurrently, and replayed; six steps bring the phi double buffer and
 * the three-buffer solution histories back to the captured layout.  Steps
 * left over run plainly.  The graph is captured again when dt changes.
 * Results are bit-identical to vsv_step on each grid.  Every grid must
 * satisfy its stability bound (else VSV_EUNSTABLE), must use fixed_cycles
 * > 0 (else VSV_EINVAL), and must not be profiling (else VSV_ESTATE).
 * Work already queued on a grid's stream completes first, and later work on
 * it waits for the batch.  Non-finite flags are not read per step: call
 * vsv_check on a grid for them.
 *
 * vsv_batch_destroy frees the graph and the events (NULL is a no-op). */
typedef struct vsv_batch vsv_batch;
vsv_status vsv_batch_create(vsv_batch** out, vsv_grid* const* grids, int n, void* cuda_stream);
vsv_status vsv_batch_step(vsv_batch* b, int nsteps, double dt);
vsv_status vsv_batch_destroy(vsv_batch* b);

/* Discrete adjoint with checkpointing.  Differentiates the map
 * (phi^0, kappa, sigma) -> phi^N of vsv_set_phi followed by N steps of
 * vsv_step (eqs. gen2, gen1, gen3 in the segregated order of the
 * numerical-implementation section), as the kernels compute it: reverse mode
 * of the discrete step, with the transposes of its central-difference and
 * mirror stencils and adjoint Poisson problems that are the same problems as
 * the forward ones (the 7-point operator with zero wall data is symmetric).
 * Adjoint fields are FP64; the adjoint solves use the grid's precision
 * (FP64 multigrid, or FP32 V-cycles with double-word defect correction) to
 * the relative residual `tol`.  With the inertial variant (rho > 0) the
 * adjoint of the vorticity is carried from step to step through the same
 * shifted operator L - s as the backward-Euler step.  The area and volume
 * constants A0 = A[phi^0], V0 = V[phi^0] depend on phi^0 and are
 * differentiated.
 *
 * vsv_tape_create_in binds a tape to grid g (which must outlive it): every
 * >= 1 steps between checkpoints, forward passes of up to max_steps >= 1
 * steps, tol > 0 (0 selects 1e-11).  All its device memory -- one segment's
 * record ((every + 1) x 5 FP64 fields), the adjoint fields and the
 * checkpoint slots -- is carved from `workspace`: caller-owned device memory
 * on the current device, 256-byte aligned, of workspace_bytes >=
 * vsv_tape_workspace_bytes(g, every, max_steps) bytes, which the caller
 * keeps until vsv_tape_destroy.  The tape allocates and frees no device
 * memory.  VSV_EINVAL on bad arguments (including a host or misaligned
 * workspace), VSV_ENOMEM when workspace_bytes is too small.
 * vsv_tape_workspace_bytes: that size (buffers plus 1 + ceil(max_steps /
 * every) checkpoints of the grid's state); VSV_EINVAL on bad arguments.
 *
 * vsv_tape_create: the same, with the tape allocating its device memory
 * itself (cudaMalloc; checkpoints as they are saved) and freeing it in
 * vsv_tape_destroy; no step limit.  VSV_EINVAL on bad arguments,
 * VSV_ECUDA when memory runs out.
 *
 * vsv_tape_forward runs vsv_set_phi(phi0, dtype, on_device) and nsteps steps
 * of dt, saving the full state on the device at step 0, every `every` steps
 * and at step nsteps.  The grid's flow, free energy and solver settings
 * must stay unchanged until the matching backward pass.  VSV_EINVAL for
 * bad arguments, VSV_ENOMEM (nothing run) when nsteps exceeds the max_steps
 * of a tape over caller-owned memory; errors of vsv_set_phi / vsv_step pass
 * through.
 *
 * vsv_tape_backward takes phibar_final = dJ/dphi^N (N cells, FP64, device
 * memory when on_device, else host) and writes phibar0 = dJ/dphi^0 (same
 * memory kind) and, when param_bar is not NULL, param_bar[0] = dJ/dkappa and
 * param_bar[1] = dJ/dsigma (host).  It re-runs each segment from its
 * checkpoint and leaves the grid at the state of step nsteps.  It returns
 * when the results are written.  VSV_ESTATE without a forward pass.
 *
 * vsv_tape_set_cycles: fixed_cycles > 0 runs every adjoint solve for exactly
 * that many cycles (V-cycles, or defect corrections on the mixed path) from
 * the previous reverse step's solution, with no host synchronisation; 0
 * (the default) solves to `tol`.  VSV_EINVAL for a NULL tape or a negative
 * count.
 * vsv_tape_destroy frees the tape (and, for vsv_tape_create, its device
 * memory; NULL is a no-op).
 * vsv_tape_bytes: device bytes the tape uses (checkpoints included; the
 * workspace size it needs for vsv_tape_create_in).
 * vsv_tape_info: adjoint solve cycles and re-run steps of the last backward
 * pass, checkpoints held. */
typedef struct vsv_tape vsv_tape;
vsv_status vsv_tape_workspace_bytes(const vsv_grid* g, int every, int max_steps, size_t* bytes);
vsv_status vsv_tape_create_in(vsv_tape** out, vsv_grid* g, int every, int max_steps, double tol,
                              void* workspace, size_t workspace_bytes);
vsv_status vsv_tape_create(vsv_tape** out, vsv_grid* g, int every, double tol);
vsv_status vsv_tape_destroy(vsv_tape* t);
vsv_status vsv_tape_forward(vsv_tape* t, const void* phi0, int dtype, int on_device, int nsteps,
                            double dt);
vsv_status vsv_tape_backward(vsv_tape* t, const double* phibar_final, double* phibar0,
                             int on_device, double* param_bar);
vsv_status vsv_tape_set_cycles(vsv_tape* t, int fixed_cycles);
size_t vsv_tape_bytes(const vsv_tape* t);
vsv_status vsv_tape_info(const vsv_tape* t, int64_t* adjoint_cycles, int64_t* recomputed_steps,
                         int* checkpoints);

#ifdef __cplusplus
}
#endif
#endif /* VSV_H */
