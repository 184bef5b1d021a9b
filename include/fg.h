/*
 * fg.h -- C ABI of the GB300 FFT chemo-mechanical fracture solver.
 *
 * The library advances the three coupled fields of the paper "An FFT based
 * chemo-mechanical framework with fracture" (arXiv 2411.16583): the deformation
 * gradient F, the ion concentration c and the phase field d, on a periodic
 * nx x ny x nz voxel grid (Sec. 3.1, Eq. Fsplit).  Each time step is the paper's
 * global staggered scheme (Alg. 4): one backward-Euler Newton-CG solve of the Fick
 * problem (Alg. 3), then mechanical Newton-CG (Alg. 1) and phase-field PCG (Alg. 2)
 * repeated until the equilibrium residual (Eq. mechresiduum) is below tolerance.
 * Every Krylov iteration applies a matrix-free Fourier operator (Eqs. mechanicalsolve,
 * PFFA, PFFprecond, ChemresidualFourier_A) built from the library's own CUDA FFT.
 *
 * Conventions
 *   - Voxel arrays are x-fastest: index (z * ny + y) * nx + x.  A tensor field is
 *     9 such arrays back to back, component (i, j) at offset (3 i + j) * V.
 *   - nz = 1 is plane strain.  nx must be even; nx, ny, nz must be among the
 *     transform lengths the library was built for (fg_supported_size).
 *   - Host arrays passed to fg_setup are copied; the caller keeps ownership.
 *   - Device pointers passed to fg_apply / fg_get_field(on_device=1) belong to the
 *     caller and must hold the stated number of elements.
 *   - All GPU work is enqueued on opts.cuda_stream (NULL: the legacy default stream);
 *     calls return after that work has completed unless stated otherwise.
 *   - Functions return FG_OK (0) or a negative FG_ERR_* code, and never throw;
 *     fg_last_error() gives the calling thread's last message.
 *   - With the environment variable FG_VERBOSE set, the mechanical Newton solver
 *     prints one line per iteration (residual, CG iterations, damping, shifts) to
 *     stderr; nothing else reads the environment.
 */
#ifndef FG_H
#define FG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FG_OK 0
#define FG_ERR_INVALID (-1) /* bad argument, size or unsupported option */
#define FG_ERR_OOM (-2)     /* device allocation failed */
#define FG_ERR_CUDA (-3)    /* a CUDA call failed */
#define FG_ERR_NOCONV (-4)  /* a Newton, Krylov or staggered loop hit its cap */
#define FG_ERR_DOMAIN (-5)  /* c left (0, 1) or det F / J_c <= 0 */
#define FG_ERR_NUMERIC (-6) /* NaN or Inf met, or a Krylov operator was not positive */

#define FG_SVK 0       /* Saint-Venant-Kirchhoff (Eqs. Ee, psie0) */
#define FG_NEOHOOKE 1  /* compressible Neo-Hookean */

#define FG_FP64 0      /* every operator and solve in FP64 */
#define FG_MIXED 1     /* FP32 Krylov operators, FP64 residuals and updates */

/* operators of fg_apply */
#define FG_OP_MECH 0     /* y = F^-1[G : F[K : x]]          (9 comps, Eq. mechanicalsolve) */
#define FG_OP_PFF 1      /* y = A(x) of Eq. PFFA            (1 comp) */
#define FG_OP_PFF_PREC 2 /* y = P(x) of Eq. PFFprecond      (1 comp) */
#define FG_OP_CHEM 3     /* y = x c(1-c) + dt L x, the Newton operator of Eq. Chemderfc
                            in the variable x = dc / (c (1-c))   (1 comp) */
#define FG_OP_GRES 4     /* y = F^-1[G : F[x]], FP64 only   (9 comps, Eq. mechresiduum) */

/* fields of fg_get_field / fg_set_field */
#define FG_FIELD_C 0  /* concentration, V doubles */
#define FG_FIELD_F 1  /* deformation gradient, 9 V doubles */
#define FG_FIELD_D 2  /* phase field, V doubles */
#define FG_FIELD_H 3  /* history H, V doubles */
#define FG_FIELD_P 4  /* first Piola stress of the current (F, c, d), 9 V doubles (get) */

typedef struct {
  int nx, ny, nz;        /* voxels per axis */
  double hx, hy, hz;     /* voxel size per axis (m) */
} fg_grid;

typedef struct {
  int law;           /* FG_NEOHOOKE or FG_SVK; all phases of a context use one law */
  double E, nu;      /* Young's modulus (Pa), Poisson ratio */
  double Omega;      /* swelling: J_c = 1 + Omega (c - c0) (Eq. Fc) */
  double c0;         /* stress-free concentration */
  double D;          /* diffusivity (m^2/s) (Eq. mobility) */
  double sigma_max;  /* damage threshold stress (Pa) (Eq. SigDrivingForce) */
} fg_phase;

typedef struct {
  int precision;      /* FG_FP64 or FG_MIXED */
  double gc, lc;      /* fracture toughness (J/m^2), length scale (m) (Eq. PFF) */
  double RT;          /* gas constant x temperature (J/mol) */
  double cmax;        /* molar density scaling mu_e (mol/m^3) */
  double tol_newton;  /* mechanical Newton tolerance on err_res */
  double tol_cg;      /* relative Krylov tolerance (FP64 mode; mixed mode: floor) */
  double tol_chem;    /* ||dc|| / ||c_t|| (Eq. Chemerror) */
  double tol_chem_cg; /* relative Krylov tolerance of the chemistry solve */
  double tol_pff_cg;  /* relative tolerance of the phase-field solve */
  double tol_stag;    /* staggered loop: err_res threshold */
  double cg_forcing;  /* mixed mode: relative tolerance of each FP32 inner solve */
  int max_newton, max_cg, max_chem_newton, max_stag;
  void* cuda_stream;  /* cudaStream_t, NULL for the legacy default stream */
  double l2_fraction; /* share of L2 one chunk of kx planes of the spectrum may take
                         between the Y and Z passes (0 or >= 1: no chunking) */
  int cg_indefinite;  /* a CG direction p of negative curvature <p, A p> < 0 in the
                         mechanical Newton system A dF = -G P:
                         2 = shift (default): solve again with A + sigma I,
                             sigma = 2 (sigma + |<p, (A + sigma) p>| / |p|^2), that
                             quotient at least 1e-6 of <b, A b> / |b|^2, until no such
                             direction is met; sigma shrinks 4-fold per Newton iteration
                             (Levenberg-Marquardt-type Newton),
                         1 = take it (the Galerkin iterate exists while <p, A p> != 0),
                         0 = stop there and keep the iterate (truncated CG).
                         <p, A p> = 0 or a non-finite value always stops a solve */
  int chem_full_jacobian; /* 0 (default): the chemistry Newton of Alg. 3 with the Jacobian
                         of the ideal part mu_c' only; 1: also the elastic part
                         d(mu_e/RT)/dc (same root; converges where mu_e reaches several RT,
                         e.g. Omega = 1.3 with E = 15 GPa).  FG_ERR_NUMERIC where the full
                         dmu~/dc <= 0 */
  int l2_prefetch;    /* 1: the X passes hand the real-space rows each block reads to the
                         bulk-copy unit as L2 prefetches (cp.async.bulk.prefetch.L2) before
                         they start; 0 (default): plain loads.  fg_autotune overrides it with
                         the faster choice */
  int residual_ff;    /* mixed mode only: 1 (default): the residual transforms that stay in
                         FP64 storage (the equilibrium residual G*P of Eq. mechresiduum and its
                         norm, the FP64 projection of each Newton correction, and the Fick
                         residual of Eq. Chemresidualfc) run their FFTs in float-float
                         arithmetic (pairs of FP32, about 48 significant bits, error-free
                         TwoSum/TwoProduct) on the FP32 pipes; 0: in FP64 arithmetic.  The
                         fields, updates, norms and sums stay FP64 either way */
  int z_columns;      /* kx-ky columns per block of the FP32 projection pass where the
                         transform length along z is a square (64, 256): 0 (default) the
                         built-in tile, 1 or 4; fg_autotune overrides it */
  int cluster_pass;   /* 1 (default): where ny = nz is 128 or 256, the FP32 operators run
                         their y transform, frequency-space operator and inverse y transform
                         (the mechanical projection; the chemistry's gradient and divergence)
                         as one pass whose kx planes stay in the distributed shared memory of
                         16-CTA thread-block clusters (if the device can keep such a cluster
                         resident); fg_autotune keeps each only where it is faster.  0: the
                         three separate passes */
} fg_opts;

typedef struct {
  int newton_chem, newton_mech, cg_chem, cg_mech, cg_pff, stag;
  int inner_refine;   /* FP64 residual refinements of mixed-mode phase-field solves */
  int cg_truncated;   /* Krylov solves stopped early: mechanical CG at non-positive
                         curvature, or an FP32 inner solve of the mixed mode at max_cg */
  int newton_damped;  /* halvings of mechanical Newton corrections */
  int cg_negcurv;     /* CG directions of negative curvature taken (cg_indefinite 1) */
  int newton_shifted; /* mechanical Newton systems solved again with a larger shift */
  int newton_minres;  /* mechanical solves that fell back to FP64 MINRES after a CG
                         correction failed to lower the FP64 residual (a MINRES solve at
                         max_cg keeps its iterate; the Newton loop's test decides) */
  int cg_graph_replays; /* 16-iteration chunks of the mechanical CG replayed from captured
                         CUDA graphs (contexts on a stream other than the legacy default
                         stream, profiling off, no shift) */
  double err_mech;    /* final err_res */
  double err_chem;    /* final ||dc|| / ||c_t|| */
  double mass;        /* sum of c after the step */
  double mass_err;    /* sum c - (sum c_t + dt sum cdot_B), relative to sum c */
  int status;         /* FG_OK or the error code of the step */
} fg_stats;

typedef struct fg_ctx fg_ctx;

/* Default options: FP64, gc = 1, lc = 2e-7, RT = 8.314462618 * 298.15, cmax = 3e4,
 * tolerances 1e-9 (Newton, chem, staggered) and 1e-10 (Krylov), cg_forcing 1e-5,
 * caps 30 / 5000 / 50 / 50, no L2 chunking, cg_indefinite 2. */
void fg_default_opts(fg_opts* o);

/* 1 when the transform length n is compiled in, else 0.  The library is built with
 * 1, 8, 12, 16, 24, 32, 48, 64, 80, 96, 100, 128, 256 and 512 (own Stockham FFT with
 * radices 2, 4, 8, 16, 3 and 5; nx must be even). */
int fg_supported_size(int n);

/*
 * Creates a solver context (Sec. 3.1 problem statement; Alg. 4 initial state).
 *   grid, phases[nphases]   geometry and per-phase constants; every phase uses one law
 *   phase_id[V]             phase of each voxel (< nphases); the paper's compliant
 *                           buffer material around the particle is one of the phases
 *   cdot_B[V]               influx volume source (1/s), nonzero only in the band of
 *                           width dL inside the particle surface (Eqs. neumann1-2)
 *   c_init[V]               initial concentration, or NULL for phases[id].c0
 *   log_E[V], log_D[V]      optional per-voxel log-scale of E and D (NULL: none)
 *   log_gc[V]               optional per-voxel log-scale of the toughness, g_c(x) =
 *                           opts.gc exp(log_gc) (NULL: uniform).  It scales the history
 *                           H = max(H_t, g_c(x)/(2 l_c) D_f), and the phase-field equation
 *                           g_c(x) (d/l_c - l_c lap d) = 2 (1 - d) H is solved divided by
 *                           g_c(x)/g_c, i.e. Eq. PFFA with H replaced by H g_c/g_c(x)
 *   log_smax[V]             optional per-voxel log-scale of the strength, sigma_max(x) =
 *                           phases[id].sigma_max exp(log_smax) in the driving force of
 *                           Eq. SigDrivingForce (Sec. 5.1 draws it per voxel from the
 *                           law of Eq. Gumbell; NULL: the phase value).  It is a fixed
 *                           input: fg_adjoint returns no gradient with respect to it
 * Initial state F = I, d = 0, H = 0 (Alg. 4).  Allocates all device memory.
 * Errors: FG_ERR_INVALID (sizes, ids, law), FG_ERR_OOM, FG_ERR_CUDA.
 */
int fg_setup(fg_ctx** out, const fg_grid* grid, const fg_phase* phases, int nphases,
             const uint8_t* phase_id, const double* cdot_B, const double* c_init,
             const double* log_E, const double* log_D, const double* log_gc,
             const double* log_smax, const fg_opts* opts);

/*
 * One time step of Alg. 4 from the stored state (F_t, c_t, d_t, H_t) to t + dt with the
 * macroscopic deformation gradient Fbar[9] (row-major) at t + dt.  On success the new
 * state is stored.  On FG_ERR_NOCONV / FG_ERR_DOMAIN / FG_ERR_NUMERIC the stored state
 * is left at the start of the step.  st may be NULL.
 */
int fg_step(fg_ctx* ctx, double dt, const double Fbar[9], fg_stats* st);

/*
 * Residuals of the stored state: err_mech = ||G*P(F)|| / ||G*P(Fbar)|| (Eq. mechresiduum,
 * with the fallbacks ||P(Fbar)|| then 1 when the comparison stress has no incompatible
 * part), err_chem = ||f(c)|| / ||c_t|| of Eq. Chemresidualfc for the last step's data
 * (0 before the first step), mass_sum = sum of c.  Any output pointer may be NULL.
 */
int fg_residual(fg_ctx* ctx, double* err_mech, double* err_chem, double* mass_sum);

/*
 * One operator application y = op(x) at the stored state, for tests and benchmarks.
 *   op         FG_OP_*;  prec: 0 = FP64 (x, y double), 1 = FP32 (x, y float), 2 = FG_OP_GRES
 *              with float-float transforms (x, y double; mixed context with residual_ff)
 *   x, y       device pointers, 9 V (MECH, GRES) or V (others) elements
 *   dt         time step of FG_OP_CHEM (ignored otherwise)
 *   dot        if not NULL receives <x, y> accumulated in FP64
 * MECH uses the tangent at the stored (F, c, d); CHEM uses c_t = c, d_t = d, F_t = F;
 * PFF and PFF_PREC use the stored H.  Enqueued on the context stream; returns when done.
 */
int fg_apply(fg_ctx* ctx, int op, int prec, const void* x, void* y, double dt, double* dot);

/* Copies a field out (host or device destination, see FG_FIELD_*). */
int fg_get_field(fg_ctx* ctx, int field, void* dst, int on_device);

/* Overwrites a stored field (C, F, D or H) from host or device memory, for tests and
 * restarts.  The step's t-state is the stored state.  Refused (FG_ERR_INVALID) while the
 * tape holds recorded steps (fg_tape_begin), whose trajectory fg_adjoint recomputes. */
int fg_set_field(fg_ctx* ctx, int field, const void* src, int on_device);

/* Runs n applications of op back to back on the stream between two CUDA events and
 * reports the mean time per application in ms (no synchronisation inside); prec as in
 * fg_apply. */
int fg_time_apply(fg_ctx* ctx, int op, int prec, int n, double* ms_per_apply);

/* Mechanical equilibrium alone (Alg. 1) at the stored c and d: the stored F is shifted by
 * Fbar - (previous Fbar) and brought to err_res <= tol_newton in place. */
int fg_solve_mech(fg_ctx* ctx, const double Fbar[9], fg_stats* st);

/*
 * Hand-written adjoint of that equilibrium at the stored (converged) F, c, d.  For a loss
 * L(F) with dL/dF = W (9 V doubles, host or device), solves the transposed tangent system
 * G K G lambda = G W with the same fused mechanical CG (the tangent is self-adjoint) and
 * writes the gradient of L with respect to the per-voxel log stiffness,
 * grad_logE[v] = -lambda(v) : P(v) (V doubles, host or device).  iters (may be NULL)
 * receives the adjoint CG iterations.
 */
int fg_adjoint_mech(fg_ctx* ctx, const double* W, double* grad_logE, int* iters);

/* Autotuner: times the run-time selectable schedule of the mechanical operator on this
 * context's grid (how many kx planes the Y-Z-Y passes take per L2-sized chunk, L2 prefetch
 * of the X passes on or off, and a one-component-per-block or nine-component X-inv CG
 * update) and keeps the fastest.  ms_per_iteration (may be NULL) receives the best
 * operator time.  Allocates two temporary 9 V vectors.
 * In a mixed context it also times the FP32 projection pass with 1 and 4 kx-ky columns
 * per block against its default tile, and the clustered Y-Z-Y pass (cluster_pass) against
 * the best separate passes.
 * fg_autotune_report returns the choices in force, choice[5] = {kx planes per chunk of
 * the Krylov precision, X-inv update one component per block (1) or nine (0), L2 prefetch
 * (1) or not (0), columns per block of the FP32 projection pass (0: default), clustered
 * Y-Z-Y passes: bit 0 the projection chain, bit 1 the chemistry's chains}, and
 * (xinv_ms, may be NULL) the autotuner's X-inv update times [prefetch off, nine; off, one;
 * on, nine; on, one] in ms (zeros before fg_autotune). */
int fg_autotune(fg_ctx* ctx, double* ms_per_iteration);
int fg_autotune_report(fg_ctx* ctx, int choice[5], double xinv_ms[4]);

/* Launch-site profiling.  While a site is enabled, every launch at that site is
 * bracketed by two CUDA events on the context stream (at most 32768 launches are recorded
 * after each enable).  Sites: 0-4 the five passes of the mechanical operator (X-fwd with
 * the tangent, Y-fwd, Z with the projection, Y-inv, X-inv with the dot product), 5 the
 * Krylov update of the mechanical CG (unfused path).  fg_profile_read synchronises the stream and returns
 * the number of recorded launches, their summed device time and (volumes, may be NULL)
 * the number of full grid volumes they covered (the Y and Z passes run on chunks of kx
 * planes, each a fraction of the volume); launches shorter than a
 * fifth of the median (kernels that returned at once because their Krylov loop had
 * already converged) are left out of both. */
int fg_profile(fg_ctx* ctx, int site, int enable);
int fg_profile_read(fg_ctx* ctx, int site, int* launches, double* total_ms, double* volumes);

/*
 * Batches of independent RVEs (many particles of uneven grid sizes).  fg_batch_setup
 * gives every member context its own non-blocking CUDA stream (restored by
 * fg_batch_destroy; members must outlive the batch and not be stepped on their own
 * meanwhile).  fg_batch_step advances every member by one time step of Alg. 4 with the
 * same dt and Fbar; a pool of host threads drives the members concurrently, so their
 * kernels overlap on the GPU.  st (may be NULL) receives n fg_stats.  Returns FG_OK or
 * the first member's error (every member is attempted; a failed member keeps its state).
 */
typedef struct fg_batch fg_batch;
int fg_batch_setup(fg_batch** out, int n, fg_ctx* const* members);
int fg_batch_step(fg_batch* batch, double dt, const double Fbar[9], fg_stats* st);
void fg_batch_destroy(fg_batch* batch);

/*
 * Grouped operator application over a batch (the mechanical operator G*(K:x) of Eq.
 * mechanicalsolve, as fg_apply with FG_OP_MECH).  Members whose grids are equal form a group
 * (run with the schedule the autotuner chose for the group's first member); each FFT pass
 * of a group runs as ONE kernel launch over all its members, block m P + b of the launch
 * running block b of member m, with the members' pass arguments read from a device table
 * (a device-side work list).  The groups run concurrently, each on a stream of its own.  x[i], y[i]: member i's
 * 9 x V input and output (device pointers, precision prec: 0 = FP64, 1 = FP32; host
 * pointers in the emulation build), owned by the caller.  Builds each member's tangent
 * state from its F first (as fg_apply does).  Runs on a stream of the batch and returns
 * after the applications completed; the members' streams are synchronised first.  Errors:
 * FG_ERR_INVALID (op other than FG_OP_MECH, bad precision, a null vector, members on
 * different devices), FG_ERR_CUDA.
 *
 * fg_batch_time_apply times napply applications of every member's operator (zero inputs in
 * buffers of its own) four ways and writes milliseconds per batch application to ms:
 * ms[0] the grouped launches captured once as a CUDA graph and replayed, ms[1] the grouped
 * launches issued one by one, ms[2] every member's own launches member after member on one
 * stream, ms[3] every member's own launches on its own stream, all members at once.
 * info (may be NULL): [0] groups, [1] launches per grouped application, [2] launches per
 * application of all members one by one.  GPU build only (FG_ERR_INVALID in the emulation).
 */
int fg_batch_apply(fg_batch* batch, int op, int prec, const void* const* x, void* const* y);
int fg_batch_time_apply(fg_batch* batch, int prec, int napply, double ms[4], int info[3]);

/*
 * Mixed macroscopic control (the paper's Sec. 3 allows prescribing macroscopic stress
 * components instead of F-bar components).  Bit 3 i + j of mask marks component (i, j) as
 * stress-controlled: the mean first Piola stress P-bar_ij is prescribed (Pbar[9],
 * row-major) and the mean F-bar_ij becomes an unknown.  The projection keeps those
 * components of the zero-frequency mode (the orthogonal projection onto compatible
 * zero-mean fields plus uniform fields on the mask, so the Newton operator stays
 * symmetric), and the residual is G P - M P-bar.  In fg_step, the Fbar argument's
 * controlled components are only the starting guess; after a step the stored F-bar holds
 * their solved mean.  mask = 0 restores full strain control.  fg_adjoint differentiates
 * steps under a mask as well; the mask cannot change while the tape holds recorded steps.
 * Errors: FG_ERR_INVALID (mask outside 0..511, Pbar NULL with a mask, steps recorded on
 * the tape).
 */
int fg_set_stress_control(fg_ctx* ctx, int mask, const double Pbar[9]);

/*
 * Discrete adjoint of recorded time steps (a hand-written reverse of Alg. 4; the paper's
 * forward equations Eqs. Chemresidualfc, mechanicalsolve, Hist, SigDrivingForce, PFFA
 * differentiated at each converged step).
 *
 * fg_tape_begin starts recording at the stored state: every later successful fg_step is
 * recorded (dt, Fbar), and the state before every ckpt_every-th recorded step is kept as a
 * checkpoint (12 V doubles of device memory each).  A new call drops the old tape.
 *
 * fg_adjoint runs the recorded steps backwards.  Each segment between checkpoints is
 * recomputed forward from its checkpoint (ckpt_every + 1 states of 12 V doubles held at a
 * time), then every step is reversed: the (F, H, d) block by transposed block Gauss-Seidel
 * sweeps accelerated by GMRES on the phase-field multiplier (mechanical CG on G K G,
 * phase-field PCG; the couplings are dP/dd and dpsi/dF on the active branch of
 * H = max(H_t, psi)), then the chemistry by its exact Jacobian transpose
 * I + dt dmu~/dc L, solved as a symmetric system by CG.  All adjoint solves run in FP64
 * at the options' tolerances (tol_cg, tol_pff_cg, tol_chem_cg; GMRES to tol_stag within
 * max_stag), and an iteration cap is an error in both precision modes.
 *   loss        FG_LOSS_CRACK_ENERGY: Gamma_E = sum g_c(x) (d^2/(2 l_c) + l_c/2 |grad_f d|^2)
 *               h^3 of the final phase field (Eq. crack); the seeds are ignored.
 *               FG_LOSS_SEEDS: L with dL/dc, dL/dF, dL/dd of the final state given in
 *               seed_c (V), seed_F (9 V, component (i, j) at (3 i + j) V), seed_d (V),
 *               host or device arrays, NULL meaning zero.
 *   loss_value  (may be NULL) Gamma_E, or 0 for FG_LOSS_SEEDS
 *   grad_*      (host or device, V doubles each, may be NULL) dL/dlog E, dL/dlog g_c,
 *               dL/dlog D per voxel (log g_c as in fg_setup's log_gc)
 * On return the stored state is the one at the call and the tape is kept.  Errors:
 * FG_ERR_INVALID (no recorded step, bad loss), FG_ERR_NOCONV (an adjoint solve hit its
 * cap), FG_ERR_NUMERIC (dmu~/dc <= 0 somewhere: the chemistry Jacobian is not positive),
 * FG_ERR_DOMAIN, FG_ERR_OOM, FG_ERR_CUDA.
 */
#define FG_LOSS_CRACK_ENERGY 0
#define FG_LOSS_SEEDS 1

typedef struct {
  int steps;       /* steps reversed */
  int recomputed;  /* forward steps recomputed from checkpoints */
  int sweeps;      /* transposed Gauss-Seidel sweeps (one mechanical + one phase-field solve) */
  int gmres;       /* GMRES iterations on the phase-field multiplier */
  int cg_mech, cg_pff, cg_chem;  /* Krylov iterations of the adjoint solves */
} fg_adjoint_stats;

int fg_tape_begin(fg_ctx* ctx, int ckpt_every);
int fg_adjoint(fg_ctx* ctx, int loss, const double* seed_c, const double* seed_F,
               const double* seed_d, double* loss_value, double* grad_logE, double* grad_loggc,
               double* grad_logD, fg_adjoint_stats* st);

/*
 * Displacement at the voxel corners, for losses on displacements (e.g. a mismatch with
 * measured displacements) in the adjoint.  From the split F = Fbar + grad u~ of Eq. Fsplit:
 *   u = (Fbar - I) x + u~,  x_j = i_j h_j the position of corner i (the lower corner of
 *   voxel i), u~ periodic with zero mean and its rotated-scheme gradient (Sec. 3.2) equal
 *   to F - mean(F) in least squares: exactly, for a compatible F, up to the scheme's null
 *   modes (several axes at their Nyquist frequency), which carry no strain.
 *   F[9 V], Fbar[9]  deformation gradient (component (i, j) at (3 i + j) V) and its mean,
 *                    row-major; both NULL: the context's current state
 *   u[3 V]           output, component i at i V
 * fg_displacement_adjoint applies the transpose of F -> u~: g[9 V] = (du~/dF)^T r for
 * r[3 V].  With r = dL/du of a loss L on the displacement, g is dL/dF at fixed Fbar, the
 * seed_F of fg_adjoint with FG_LOSS_SEEDS.
 * Pointers may be host or device memory (on_device is informational); the work runs in
 * FP64 in either precision mode.  Errors: FG_ERR_INVALID (null argument, or only one of F
 * and Fbar given), FG_ERR_OOM, FG_ERR_CUDA.
 */
int fg_displacement(fg_ctx* ctx, const double* F, const double* Fbar, double* u, int on_device);
int fg_displacement_adjoint(fg_ctx* ctx, const double* r, double* g, int on_device);

/*
 * Restart files: fg_save writes the evolving state of the context (c, F, d, H, the
 * t-state of the last step, Fbar, the previous Fbar, the last dt, and the mixed-control
 * mask and prescribed Pbar of fg_set_stress_control) to a binary file; fg_load reads one
 * into a context set up with the same grid, law and materials (the file holds no
 * material data), which then steps as the saved one would.  Doubles in the machine's byte
 * order.  fg_load is refused while the tape holds recorded steps.  Errors: FG_ERR_INVALID
 * (file cannot be opened, written or read, is not a state file, its grid or law differs,
 * or the tape holds steps), FG_ERR_CUDA.
 */
int fg_save(fg_ctx* ctx, const char* path);
int fg_load(fg_ctx* ctx, const char* path);

/* Releases the context, its tape and its device memory.  NULL is ignored. */
void fg_destroy(fg_ctx* ctx);

/*
 * fg_mech_apply_noalloc -- the FP32 mechanical operator application of fg_apply
 * (FG_OP_MECH, prec 1) of a context under full strain control (the projection G, no
 * stress-control mask), for callers that cannot allocate GPU memory.  The paper has no
 * counterpart: this is a deployment variant.  It suits code that may only hand over
 * pointers, e.g. a plug-in running inside a host framework that owns all device memory
 * through its own pool, or a service whose device-memory budget is fixed after start-up,
 * where a library that calls cudaMalloc would break the pool or the budget.
 *
 * Inputs are the caller's device arrays: F (9 V doubles, component (i, j) at
 * (3 i + j) V), c, d and the per-voxel Lame constants lam, mu, swelling Omega and
 * stress-free c0 (V doubles each); x (9 V floats) in, y (9 V floats) out, y = G : F^-1[
 * F[K(F, c, d) : x]].  dot (host, may be NULL) receives <x, y>.  Work is enqueued on
 * `stream` (cudaStream_t, NULL: legacy default) and the call returns when it is done.
 *
 * All scratch (spectra, packed tangent, tables, partial sums: about 32 MB) is one
 * static device array that every GPU loading the library holds until the process exits.
 * Limits: nx even, every edge <= 64 (so V <= 262,144) and a compiled transform length;
 * larger grids return FG_ERR_INVALID without touching the GPU.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current.  Every call copies its inputs from host memory and waits for its work.  Every
 * call reuses the same array and leaves the last call's contents in it; calls that overlap on
 * the GPU (other streams, other host threads) race on it.  No cudaMalloc, cudaFree or
 * other allocating routine is called.  Errors: FG_ERR_INVALID, FG_ERR_DOMAIN
 * (det F <= 0 or J_c <= 0), FG_ERR_CUDA; message in fg_last_error().
 */
int fg_mech_apply_noalloc(int nx, int ny, int nz, double hx, double hy, double hz,
                          const double* F, const double* c, const double* d,
                          const double* lam, const double* mu, const double* Omega,
                          const double* c0, const float* x, float* y, double* dot,
                          void* stream);

/* Number of CUDA kernels the library has launched since it was loaded (all contexts). */
long long fg_kernel_launches(void);

/* Message of the calling thread's last failing call ("" if none). */
const char* fg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FG_H */
