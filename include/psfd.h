/*
 * psfd.h -- C ABI of the B300 Lippmann-Schwinger PSFD solver for EUV mask scattering.
 *
 * The library solves the scattering of plane waves by an absorber layer on top of a
 * planar multilayer stack, following arXiv 2606.25541 (Lee, Gillijns, Kim):
 *   - Sec. 2, Eqs. (1)-(3): the stack is removed from the computational domain and
 *     acts through its reflection operator R (background-field decomposition);
 *   - Sec. 3, Eq. (9): R acts per transverse Fourier mode through the stack's
 *     reflection matrix T_R, obtained by the transfer-matrix / generalized reflection
 *     coefficient recursion;
 *   - Sec. 3, Eqs. (11)-(18): the remaining free-space problem is solved in
 *     Lippmann-Schwinger form x - G*(V x) = b with V = k0^2 (eps - eps_bg), the
 *     convolution done by FFTs with a windowed dyadic Green's function.
 * For periodic clips the Green's function is taken exactly per transverse Bloch mode
 * and windowed in z only (|z| < L = nf*dz/2), and R is folded into the operator:
 *   A u = u - (I + R) G*(V u),   b = E_inc + R[E_inc],
 * u being the total field on the absorber planes.
 *
 * Conventions: lengths in nm; time dependence exp(-i w t); complex numbers are stored
 * as interleaved (re, im) pairs of double (or float where stated); field vectors are
 * laid out [rhs][component 3][plane nslab][y ny][x nx] with x fastest; absorber plane
 * p (0-based) sits at height (p + 1/2) dz above the stack interface z_top.
 *
 * Ownership: the context owns every device buffer it allocates in psfd_create and
 * frees them in psfd_destroy. Input arrays are read during the call only. Output
 * arrays are provided by the caller. A context is bound to one CUDA stream and is not
 * thread safe; calls on one context must not overlap.
 *
 * Errors: every function returns PSFD_OK (0) or a negative PSFD_E_* code; the
 * context keeps a human-readable description, see psfd_last_error().
 */
#ifndef PSFD_H
#define PSFD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSFD_OK 0
#define PSFD_E_ARG (-1)           /* invalid argument (null pointer, bad size, unsupported length) */
#define PSFD_E_NOMEM (-2)         /* device allocation failed */
#define PSFD_E_BUDGET (-3)        /* request exceeds the context's HBM budget */
#define PSFD_E_CUDA (-4)          /* a CUDA runtime call failed */
#define PSFD_E_NOT_CONVERGED (-5) /* iteration cap reached before the tolerance */
#define PSFD_E_BREAKDOWN (-6)     /* Krylov breakdown (zero or non-finite scalar) */
#define PSFD_E_ANOMALY (-7)       /* a diffraction order grazes the interface (beta ~ 0) */
#define PSFD_E_TIMEOUT (-8)       /* a bounded device wait gave up */
#define PSFD_E_STATE (-9)         /* call out of order (e.g. solve before set_illumination) */

#define PSFD_FP64 0         /* every step in complex FP64 */
#define PSFD_FP32_REFINED 1 /* complex FP32 Krylov inside FP64 defect correction */
#define PSFD_FP64_DF 2      /* psfd_apply only: FP64 data, z pass in double-float (see below) */

#define PSFD_HOST 0   /* pointer argument is host memory */
#define PSFD_DEVICE 1 /* pointer argument is device memory of the context's GPU */

typedef struct psfd_ctx psfd_ctx;

/* Discretisation of one mask clip (Sec. 3, Eq. (4): Fourier basis on a uniform grid). */
typedef struct {
  int nx, ny;        /* transverse grid; x and y are periodic with pitch nx*dx, ny*dy */
  int nslab;         /* absorber planes (the support of V) */
  int nf;            /* z FFT length, nf >= 2*nslab + 2 and psfd_supported_length(nf) */
  double dx, dy, dz; /* grid spacing, nm */
  double wavelength; /* vacuum wavelength, nm */
  double eps_bg;     /* real permittivity of the background medium (1 = vacuum) */
} psfd_grid;

/* Options of psfd_solve. Zero-initialised fields take the defaults in brackets. */
typedef struct {
  double tol;       /* target relative residual ||b - A x|| / ||b|| in FP64 [1e-10] */
  int max_iter;     /* Krylov iteration cap per solve or per refinement sweep [500] */
  int max_outer;    /* refinement sweep cap for PSFD_FP32_REFINED [12] */
  double inner_tol; /* tightest relative tolerance of an FP32 inner solve [1e-4]: a sweep
                       starting from FP64 residual rho (relative) is solved to
                       min(1/2, max(inner_tol, tol / (4 rho))), i.e. only as far as the
                       target still needs */
  int check_every;  /* iterations between host reads of the device convergence flags [4] */
  int krylov;       /* PSFD_BICGSTAB [default] or PSFD_GMRES */
  int restart;      /* GMRES basis size per sweep [PSFD_KRYLOV_MAX] (<= PSFD_KRYLOV_MAX) */
  int reserved[2];
} psfd_solve_opts;

/* Krylov methods. GMRES(m) (classical Gram-Schmidt, Givens rotations) needs fewer operator
 * applications; BiCGStab needs no growing basis, and on B300 its two cheap vector passes
 * per iteration make it the faster of the two at the bench sizes. */
#define PSFD_BICGSTAB 0
#define PSFD_GMRES 1
#define PSFD_KRYLOV_MAX 24 /* Krylov vectors a context reserves per illumination */

typedef struct {
  int iterations;   /* Krylov iterations (operator applications / 2), max over RHS */
  int outer;        /* refinement sweeps performed */
  double relres;    /* true FP64 relative residual after the solve, max over RHS */
  double seconds;   /* wall time of psfd_solve */
  int status;       /* PSFD_OK or the first failure */
  int reserved[3];
} psfd_report;

/* Text of a status code (static storage). */
const char* psfd_strerror(int status);

/* Description of the last failure on this context ("" if none). */
const char* psfd_last_error(const psfd_ctx* ctx);

/* 1 if n is an FFT length the kernels are built for, else 0: 4, 8, 16, 32, 64, 96, 128, 160,
 * 192, 256, 320, 384, 512, 640, 768, 1024. */
int psfd_supported_length(int n);

/* Device bytes psfd_create would allocate for this grid, precision and RHS capacity. The
 * Krylov pool is sized for BiCGStab (7 vectors per illumination); the first PSFD_GMRES solve
 * on a context grows it to restart + 3 vectors (and fails with PSFD_E_BUDGET or
 * PSFD_E_NOMEM if that does not fit). */
int psfd_workspace_bytes(const psfd_grid* grid, int precision, int max_rhs, size_t* bytes);

/* Create a solver context on the current CUDA device.
 *   grid       discretisation; validated (supported lengths, nf >= 2*nslab+2)
 *   precision  PSFD_FP64 or PSFD_FP32_REFINED
 *   max_rhs    capacity in illuminations solved together
 *   hbm_budget bytes the context may allocate (0 = no limit); PSFD_E_BUDGET if exceeded
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 * On success *out receives the context. */
int psfd_create(psfd_ctx** out, const psfd_grid* grid, int precision, int max_rhs,
                size_t hbm_budget, void* stream);

/* Free every resource of the context (NULL is accepted). */
int psfd_destroy(psfd_ctx* ctx);

/* Rebind the context to another stream. */
int psfd_set_stream(psfd_ctx* ctx, void* stream);

/* Green's function of the operator. PSFD_GREEN_PERIODIC (default): the clip is periodic in x
 * and y (diffraction orders), the kernel is exact per transverse mode and windowed in z only.
 * PSFD_GREEN_SPHERICAL: an isolated clip (Sec. 3, Eqs. (13)-(17)): the dyadic Green's function
 * truncated to |r| < R, F[G_R](k) = A(|k|) I + B(|k|) khat khat^T, evaluated at
 * k = (q_x, q_y, kz_l), with no stack reflection (free space around the clip). The caller pads
 * the clip transversally in the grid (eps = eps_bg in the border) so that every period exceeds
 * the scatterer's extent plus R, and R exceeds the scatterer's diameter; z is padded
 * internally to nf, which must satisfy nf dz >= nslab dz + R. Unknowns remain Bloch envelopes
 * (the field times exp(-i q_inc . r)), the right-hand side the incident envelope.
 * Must precede psfd_set_illumination (it discards the current illuminations). The kernel is
 * tabulated per illumination: (nf/2 + 1) nx ny entries of 32 B (FP64) + 16 B (FP32) per
 * illumination slot, allocated here under the context's budget. The diffraction-order calls
 * keep their periodic meaning and are not defined for this kind.
 * Errors: PSFD_E_ARG (unknown kind, R <= 0, R above a transverse period, nf too short),
 * PSFD_E_BUDGET / PSFD_E_NOMEM. */
#define PSFD_GREEN_PERIODIC 0
#define PSFD_GREEN_SPHERICAL 1
int psfd_set_green(psfd_ctx* ctx, int kind, double R);

/* CUDA graphs for the Krylov loop (on by default; no counterpart in the paper, which states
 * no execution model). Each engine tick runs check_every Krylov iterations of the active
 * illuminations; that launch sequence depends only on the batch width, the method and the
 * options, so it is captured once per configuration (on a private stream of the context)
 * and replayed as one graph launch on the context's stream. Results are bitwise the same
 * either way. enable = 0 waits for the context's stream and frees the captured graphs.
 * Profiling (psfd_profile_enable) bypasses the graphs. */
int psfd_set_graphs(psfd_ctx* ctx, int enable);

/* Device-side sweep loop (on by default; needs graphs on; no counterpart in the paper). While
 * every busy illumination of the context is inside a Krylov sweep, the ticks of that sweep
 * run inside one graph launch: a conditional WHILE node repeats the tick's graph, and a
 * one-block kernel at the end of each tick records every slot's Krylov estimate and clears
 * the condition once no slot is active (or after max_iter / check_every + 1 ticks, after
 * which any slot still active goes on in ordinary ticks). The host then waits once per sweep
 * instead of once per tick. Slots whose sweep ends early wait for the others before their
 * FP64 residual. Results, iteration counts and the residual history are bitwise those of the
 * host-driven ticks. Contexts of the serving loop keep host-driven ticks, so that requests
 * are admitted between ticks. */
int psfd_set_device_loop(psfd_ctx* ctx, int enable);

/* Autotuner (no counterpart in the paper). Tile shapes of the operator's passes that leave
 * every element's arithmetic and every reduction order unchanged are chosen at run time:
 *   zx  x-modes per CTA of the z pass (K2), 1-16; the lane-group z transforms (nf = 64,
 *       128, 256, and 160 in FP32) take 4, 8 or 16;
 *   rb  rows per CTA of the forward row pass on planes too large for one CTA;
 *   cx  columns per CTA of the column passes on such planes;
 *   pf  on planes split into two half-plane CTAs (FP32 128 x 128): each CTA of the inverse pass
 *       (and of the forward pass with the plain input stage) asks the bulk-copy unit to
 *       prefetch into L2 the planes of the CTA pf launches later (0: none).
 * psfd_autotune times the candidate shapes on the context's own grid, illuminations and
 * buffers (CUDA events around 3 applications each, one tunable at a time, each from the best
 * shape so far) in the precision of the context's Krylov loop (FP32 for PSFD_FP32_REFINED,
 * FP64 for PSFD_FP64), and stores the fastest in a process-wide table keyed by (precision,
 * nx, ny, nslab, nf) that every context of that grid then uses. A grid already in the table
 * is not timed again unless force != 0. Results are bitwise the same for every shape. The
 * call synchronises the context's stream, overwrites two of its Krylov scratch vectors (not
 * the solution), drops its captured graphs, and needs set_potential and set_illumination
 * first (PSFD_E_STATE). Contexts that captured graphs before keep the old shapes in them.
 * report (may be NULL): the built-in and the tuned time of one application in ms (0 when the
 * table already held the grid), the chosen shapes (0 = built-in) and the shapes timed.
 * psfd_tune_set stores given shapes for a grid and precision (0 = built-in; PSFD_E_ARG for a
 * shape the kernels cannot take); psfd_tune_reset empties the table. */
typedef struct {
  double default_ms, tuned_ms;
  int zx, rb, cx;
  int candidates;
  int pf;
} psfd_tune_report;
int psfd_autotune(psfd_ctx* ctx, int force, psfd_tune_report* report);
int psfd_tune_set(const psfd_grid* grid, int precision, int zx, int rb, int cx, int pf);
int psfd_tune_reset(void);

/* Arithmetic of the FP64 residual r = b - A x that certifies a PSFD_FP32_REFINED solve
 * (no counterpart in the paper; the defect correction is not one of its steps).
 *   PSFD_RESID_FP64    every step in FP64;
 *   PSFD_RESID_DFLOAT  (default) in double-float (a pair of FP32 numbers, about 48
 *                      significant bits, ~1e-14 normwise): the z pass's transforms and dyadic
 *                      products on nf = 64 or 128 with the periodic kernel, and the y
 *                      transforms of planes too large for one CTA (ny = 128 or 256, nx a
 *                      multiple of 8); FP64 elsewhere. B300 runs FP32 about sixty times
 *                      faster than FP64, and the refinement needs the residual only to well
 *                      below its tolerance.
 * Vectors, the x passes, the Green's scalars and the reflection stay FP64 either way.
 * Contexts of precision PSFD_FP64 ignore the setting. Errors: PSFD_E_ARG (unknown kind). */
#define PSFD_RESID_FP64 0
#define PSFD_RESID_DFLOAT 1
int psfd_set_residual_arith(psfd_ctx* ctx, int kind);

/* Planar stack below z_top (Sec. 2, Fig. 1): n_layers layers listed top to bottom with
 * complex refractive index n_complex[2*j], n_complex[2*j+1] and thickness thickness_nm[j],
 * on a substrate of index n_sub[0] + i n_sub[1]. eps = n^2. n_layers may be 0. */
int psfd_set_stack(psfd_ctx* ctx, int n_layers, const double* n_complex,
                   const double* thickness_nm, const double* n_sub);

/* Absorber permittivity eps on the nslab x ny x nx cells, complex interleaved, laid out
 * [plane][y][x] (where = PSFD_HOST or PSFD_DEVICE). V = k0^2 (eps - eps_bg) is formed on
 * the device in FP64 and FP32 (Sec. 2, Eq. (1)). */
int psfd_set_potential(psfd_ctx* ctx, const double* eps_complex, int where);

/* Plane-wave illuminations (host arrays of length n_rhs <= max_rhs): polar angle theta
 * and azimuth phi in degrees (k_inc = k_bg (sin t cos f, sin t sin f, -cos t)) and
 * polarisation pol (0 = s, i.e. E along z x q; 1 = p). Builds, on the device and in FP64,
 * the per-mode stack reflection r_s, r_p by the Parratt recursion and the right-hand side
 * b = E_inc + R[E_inc]. Returns PSFD_E_ANOMALY if some order has |beta| < 1e-9 k0. */
int psfd_set_illumination(psfd_ctx* ctx, int n_rhs, const double* theta_deg,
                          const double* phi_deg, const int* pol);

/* Solve A u = b for every illumination (Krylov: BiCGStab; PSFD_FP32_REFINED runs it in
 * complex FP32 inside FP64 defect correction r = b - A u, u += A^-1 r). opts may be NULL.
 * The Krylov loop stays on the device; the host reads the convergence flags once per sweep
 * (psfd_set_device_loop), or every check_every iterations with the loop off. report may be
 * NULL. Returns PSFD_E_NOT_CONVERGED if some
 * right-hand side missed the tolerance (the solution is still stored). */
int psfd_solve(psfd_ctx* ctx, const psfd_solve_opts* opts, psfd_report* report);

/* psfd_solve on n distinct contexts at once (no counterpart in the paper: a way to run a
 * batch of illuminations split over several contexts, e.g. the two halves of a set of
 * angles). Each context is solved by its own host thread on its own stream, so the
 * contexts' kernels run side by side: the z pass, bound by instruction issue, overlaps the
 * latency-bound plane passes of the other context. Each context's results are bitwise those
 * of psfd_solve on it alone (the arithmetic of a context does not depend on the others).
 *   ctxs     host array of n context pointers, all distinct and non-null; contexts sharing
 *            one stream are correct but run one after the other
 *   opts     as for psfd_solve, applied to every context (may be NULL)
 *   reports  host array of n reports, or NULL
 * Returns PSFD_OK, PSFD_E_ARG (null, n < 1 or a repeated context), or the first non-OK status
 * of the contexts in order (every context is solved either way). Per-pass profiling
 * (psfd_profile_enable) records launches of one context at a time: leave it off here. */
int psfd_solve_group(psfd_ctx* const* ctxs, int n, const psfd_solve_opts* opts, psfd_report* reports);

/* The paper's outer fixed-point iteration (Sec. 3, Eqs. (8)-(9)) in place of the folded
 * operator: outer step k solves the free-space problem u_k - G*(V u_k) = b_k with
 * b_k = E_inc + R[E_inc + E_mask^(k-1)], E_mask^(0) = 0, so R is rebuilt from the mask
 * field of the previous step. Each step runs the same engine as psfd_solve (the same
 * Krylov method, precision and opts) with R left out of the operator, warm-started from the
 * previous step and solved to step_tol ||b_k|| (0 = tol / 10). Between steps the folded
 * FP64 residual ||b - A u_k|| / ||b|| (b = E_inc + R[E_inc]) is formed: it is the change of
 * the reflected field over the step plus the step's own residual, and an illumination stops
 * once it is <= opts->tol; at the fixed point u solves A u = b, so solution, orders and
 * residual mean what they mean after psfd_solve. max_steps <= 0 means 50. report->outer is
 * the number of outer steps, report->iterations the Krylov iterations over all of them,
 * report->relres the folded residual. The residual history records kind 2 = the folded
 * residual after each outer step (kinds 0 and 1 refer to the step's own system).
 * Memory: one more FP64 vector per illumination slot, allocated on the first call under
 * the context's budget (PSFD_E_BUDGET / PSFD_E_NOMEM otherwise).
 * Errors: PSFD_E_STATE before potential/illumination, PSFD_E_ARG (step_tol outside [0, 1)),
 * PSFD_E_NOT_CONVERGED if an illumination is still above tol after max_steps (or one of its
 * steps missed step_tol), PSFD_E_BREAKDOWN on a non-finite residual. */
int psfd_solve_fixed_point(psfd_ctx* ctx, const psfd_solve_opts* opts, int max_steps, double step_tol,
                           psfd_report* report);

/* Number of propagating reflected orders (|q_mn| < k_bg) of illumination rhs. */
int psfd_num_orders(psfd_ctx* ctx, int rhs, int* n_orders);

/* Reflected diffraction orders of illumination rhs after psfd_solve (Sec. 2, Eq. (3);
 * Sec. 3, Eq. (9)): for each propagating order (m, n), written to host arrays of
 * capacity `capacity` orders,
 *   mn[2k], mn[2k+1]  signed order indices,
 *   amp[6k..6k+5]     complex field vector A_mn (x, y, z) referenced at z_top,
 *   sp[4k..4k+3]      complex s and p amplitudes (bilinear projections on s, p+),
 *   eff[k]            diffraction efficiency |A|^2 Re(beta_mn) / beta_00.
 * Any of amp, sp, eff may be NULL. *n_orders receives the count. */
int psfd_diffraction_orders(psfd_ctx* ctx, int rhs, int capacity, int* n_orders, int* mn,
                            double* amp, double* sp, double* eff);

/* One operator application out = A u for right-hand sides rhs0 .. rhs0+n_rhs-1 with the
 * current potential and illumination tables (the Krylov hot path, Eq. (18) with Eq. (9)).
 * precision selects complex FP64 (double pairs) or complex FP32 (float pairs) data;
 * PSFD_FP64_DF applies the operator as a refined solve's residual does under
 * PSFD_RESID_DFLOAT (FP64 data, the z pass in double-float where supported).
 * u and out are device arrays [n_rhs][3][nslab][ny][nx]; they must not alias. */
int psfd_apply(psfd_ctx* ctx, int precision, int rhs0, int n_rhs, const void* u, void* out);

/* Copy the FP64 solution u (or the right-hand side b) of illumination rhs,
 * [3][nslab][ny][nx] complex double, to dst (where = PSFD_HOST or PSFD_DEVICE). */
int psfd_get_solution(psfd_ctx* ctx, int rhs, double* dst, int where);
int psfd_get_rhs(psfd_ctx* ctx, int rhs, double* dst, int where);

/* Warm start: the next psfd_solve starts illumination rhs from x ([3][nslab][ny][nx] complex
 * double, host or device as `where` says) instead of zero -- a solution from a nearby
 * problem, or this problem's own solution at a looser tolerance, so that a solve can be
 * continued to a tighter one. The solve first forms the FP64 residual b - A x; when that is
 * already below tol it takes no Krylov iteration. Call after psfd_set_illumination (which
 * discards guesses); x is copied before the call returns. Errors: PSFD_E_ARG (rhs out of
 * range, null x, bad where). */
int psfd_set_initial_guess(psfd_ctx* ctx, int rhs, const double* x, int where);

/* Convergence curve of illumination rhs in the latest solve (the residual-vs-iteration record
 * the paper plots, Sec. 4): entry k is (iteration[k] Krylov iterations so far, kind[k],
 * relres[k]); kind 1 = the FP64 relative residual ||b - A x|| / ||b|| (the start of the solve
 * and the end of every sweep), kind 0 = the Krylov estimate after a batch of check_every
 * iterations (BiCGStab only: its recursive residual times the sweep's starting residual),
 * kind 2 = the folded FP64 residual after an outer step of psfd_solve_fixed_point.
 * Copies min(capacity, *n) entries; *n = the number recorded (at most 100000). */
int psfd_residual_history(psfd_ctx* ctx, int rhs, int capacity, int* n, int* iteration, int* kind, double* relres);

/* Per-mode tables of illumination rhs, each [ny][nx] complex double on the host:
 * beta (z wavenumber, Im >= 0) and the stack reflection coefficients r_s, r_p. */
int psfd_get_mode_tables(psfd_ctx* ctx, int rhs, double* beta, double* r_s, double* r_p);

/* ---------------------------------------------------------------------------------
 * Serving loop: continuous batching of mask-clip solves (any number of clips, each with
 * its own grid, stack, permittivity and 1..n illuminations).
 *
 * Requests are copied on submit and queued. Each psfd_server_progress call admits queued
 * requests, in arrival order, into a context of the same grid (a "bucket" with
 * slots_per_context illumination slots and as many potential slots) as soon as slots are
 * free -- also while other requests of the bucket are mid-solve -- creating a bucket when
 * its device footprint fits the HBM budget (idle buckets are released to make room).
 * Buckets advance independently: each has its own streams, and progress enqueues the next
 * step of the solve engine for every bucket whose previous step has finished (the FP32 /
 * FP64 Krylov iterations, FP64 residuals and orders of all its admitted illuminations share
 * launches), completes the steps that have finished and retires requests whose
 * illuminations are all done; it never waits for a bucket's running step (it polls for at
 * most 2 ms when nothing can move). The bucket holding the oldest running request runs on
 * the highest-priority stream, the next oldest on the next level, so the device serves
 * requests in arrival order and younger ones fill idle SMs. A request's orders do not
 * depend on which other requests shared its bucket. Single threaded: the caller drives
 * progress. */
typedef struct psfd_server psfd_server;

typedef struct {
  psfd_grid grid;          /* discretisation (as for psfd_create) */
  int n_layers;            /* stack, as for psfd_set_stack */
  const double* n_complex;
  const double* thickness_nm;
  const double* n_sub;
  const double* eps;       /* host, complex double [nslab][ny][nx] permittivity */
  int n_rhs;               /* illuminations, as for psfd_set_illumination */
  const double* theta_deg;
  const double* phi_deg;
  const int* pol;
} psfd_request;

/* precision: PSFD_FP64 or PSFD_FP32_REFINED; hbm_budget: bytes of all buckets (0 = no
 * limit); opts: solve options for every request (NULL = defaults). */
int psfd_server_create(psfd_server** out, int precision, size_t hbm_budget, int slots_per_context,
                       const psfd_solve_opts* opts);
int psfd_server_destroy(psfd_server* s);
/* Queue a request (inputs copied); *ticket identifies it. */
int psfd_server_submit(psfd_server* s, const psfd_request* req, long long* ticket);
/* Complete finished engine steps, admit, enqueue the next step of idle buckets, retire;
 * *n_pending = queued + running. */
int psfd_server_progress(psfd_server* s, int* n_pending);
/* Fused rounds (no counterpart in the paper; off by default). With ticks_per_round > 0 every
 * bucket runs on one stream of the server and progress() works in rounds: when the previous
 * round has finished, every bucket completes, queued requests are admitted, each bucket's
 * phase work (norms, FP64 residuals, sweep starts, orders) is enqueued, and then ONE graph
 * launch advances every bucket that is inside a Krylov sweep -- clips of different grids side
 * by side -- through up to ticks_per_round ticks of check_every iterations each (one
 * conditional WHILE node per bucket, see psfd_set_device_loop). The graph is captured once per
 * set of buckets and batch widths and replayed. A request's results are bitwise the same as
 * with independent buckets. Admission happens between rounds. 0 returns to independent
 * buckets on priority streams. Call between progress() calls with no round in flight
 * (PSFD_E_STATE otherwise). */
int psfd_server_set_rounds(psfd_server* s, int ticks_per_round);
/* Requests in flight at once over all buckets (no counterpart in the paper). n > 0: a
 * queued request is admitted only while fewer than n requests are running, still in arrival
 * order; the running ones share the device (the oldest on the highest stream priority).
 * Sharing shortens the waits of short requests but stretches the long ones that set the
 * tail latency; a small n keeps most of the overlap and the tail close to one request at a
 * time. 0 (default): every request that fits is admitted. Takes effect at the next
 * admission. Errors: PSFD_E_ARG (null server or n < 0). */
int psfd_server_set_max_running(psfd_server* s, int n);
/* *state: 0 queued, 1 running, 2 done; *status: PSFD_OK or the request's failure. */
int psfd_server_status(psfd_server* s, long long ticket, int* state, int* status);
/* Orders of illumination rhs of a finished request (layout as psfd_diffraction_orders). */
int psfd_server_orders(psfd_server* s, long long ticket, int rhs, int capacity, int* n_orders, int* mn,
                       double* amp, double* sp, double* eff);
/* Forget a finished request, or cancel a queued one; PSFD_E_STATE for a running request
 * (it keeps its slots until it finishes). A request whose bucket alone exceeds the HBM
 * budget finishes at admission with status PSFD_E_BUDGET; one whose bucket cannot be
 * allocated while no other request runs finishes with PSFD_E_NOMEM (with requests running,
 * it waits for their memory). */
int psfd_server_release(psfd_server* s, long long ticket);
/* Device bytes held by the buckets and their number. */
int psfd_server_memory(psfd_server* s, size_t* used, int* n_contexts);

/* Number of CUDA kernels the library has launched since it was loaded (all contexts). */
int psfd_launch_count(unsigned long long* count);

/* Per-pass timing for measurement: psfd_profile_enable(1) clears earlier records and
 * brackets each operator pass (K1, K2, K3 in FP32 and FP64) and each BiCGStab vector
 * update with CUDA events on the stream it runs on; psfd_profile_enable(0) stops.
 * psfd_profile_get folds the finished records (synchronising on their events) into
 * per-class totals: class name (static storage), launches, summed event time in ms,
 * and the algorithmic bytes and flops of those launches (every vector read or written
 * once; 5 N log2 N flops per complex FFT of length N). cls in [0, psfd_profile_classes()). */
int psfd_profile_enable(int on);
int psfd_profile_classes(void);
int psfd_profile_get(int cls, const char** name, unsigned long long* launches, double* ms, double* bytes,
                     double* flops);

/* ---------------------------------------------------------------------------------
 * Allocation-free operator application. The paper has no counterpart: this is a
 * deployment variant of psfd_apply for callers that cannot call cudaMalloc -- systems
 * whose device memory is fixed at start-up (real-time or certified deployments that
 * forbid allocation after initialisation) and hosts whose own allocator owns the
 * device, where an outside cudaMalloc/cudaFree would break its accounting or
 * synchronise the device. Such callers cannot use psfd_create, which allocates.
 *
 * out = A u for one illumination, with the same FP32 kernels as psfd_apply(...,
 * PSFD_FP32_REFINED, ...), computed without any context:
 *   grid                   discretisation (same rules as psfd_create)
 *   n_layers, n_complex, thickness_nm, n_sub   stack, as in psfd_set_stack (<= 256 layers)
 *   theta_deg, phi_deg     illumination (polarisation does not enter A)
 *   eps                    device, complex double [nslab][ny][nx] permittivity
 *   u, out                 device, complex float [3][nslab][ny][nx]; must not alias
 *   stream                 cudaStream_t (NULL = legacy default stream)
 * It allocates nothing (no cudaMalloc, cudaFree or allocating library call): every
 * intermediate lives in one static device array of PSFD_STATIC_SCRATCH_BYTES that the
 * library holds on every GPU it is loaded on until the process exits. A grid needs
 * about nx*ny*(152 + 32*nslab) + 16 KiB of it (128 x 128 x 60: 34.0 MB); larger grids
 * are rejected with PSFD_E_BUDGET before any device work. The first call on each
 * device does a one-time set-up: it looks the array's device address up
 * (cudaGetSymbolAddress) with that device current, so make the first call on a device
 * before any stream capture begins. All calls share the array and it keeps the previous
 * call's contents: calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller. The stack arrays are read before return. A stack
 * with at most 8 distinct media, 16 distinct interfaces and 8 distinct (medium,
 * thickness) layers -- the Ru / Mo/Si stacks -- is passed to the kernels by value; any
 * other stack is copied into the array and the call then synchronises the stream once.
 * Returns PSFD_OK, PSFD_E_ARG, PSFD_E_BUDGET, PSFD_E_ANOMALY or PSFD_E_CUDA. */
#define PSFD_STATIC_SCRATCH_BYTES (48u * 1024u * 1024u)
int psfd_apply_fp32_static(const psfd_grid* grid, int n_layers, const double* n_complex,
                           const double* thickness_nm, const double* n_sub, double theta_deg,
                           double phi_deg, const void* eps, const void* u, void* out, void* stream);

/* ---------------------------------------------------------------------------------
 * The conventional differential PSFD operator (Sec. 3, Eqs. (4)-(7)), the formulation the
 * paper measures its Lippmann-Schwinger form against:
 *   out = curl curl E - k0^2 eps E
 * on Bloch envelopes of a periodic clip whose z column (free space, PML at both ends) holds
 * the absorber. Derivatives are spectral (Eq. (6)): along x and y exact per transverse mode
 * (d/dx -> i q_x, q = q_inc + 2 pi m / P), along z by an FFT over the column divided by the
 * stretch s(z) = 1 + i sigma(z) (Eq. (7)). The paper gives no PML profile; this one is
 * sigma(z) = sigma_max (depth / L)^3 over n_pml planes at each end, sigma_max =
 * -4 ln(1e-8) / (2 kb L), L = n_pml dz, plane k at z = (k + 1/2) dz. Complex FP64 throughout.
 *   n                 transverse points, nx = ny = n in {8, 16, 32, 64}; dx = dy
 *   nz                planes of the column in {32, 64, 128}; 0 <= 2 n_pml < nz
 *   wavelength, eps_bg, theta_deg, phi_deg   as in psfd_grid / psfd_set_illumination
 *   eps               device, complex double [nz][n][n]
 *   E, out            device, complex double [3][nz][n][n]; must not alias
 *   work              device, complex double [3][nz][n][n], caller-owned scratch
 *   stream            cudaStream_t (NULL = legacy default stream)
 * Three launches (FFT_xy; per-mode curls with the z derivatives; inverse FFT_xy with the
 * k0^2 eps term), no allocation, no synchronisation. Returns PSFD_OK, PSFD_E_ARG
 * (unsupported size, null pointer, non-positive spacing) or PSFD_E_CUDA. */
int psfd_apply_differential(int n, int nz, int n_pml, double dx, double dz, double wavelength, double eps_bg,
                            double theta_deg, double phi_deg, const double* eps, const double* E, double* out,
                            double* work, void* stream);

/* GMRES(restart) solve of the differential system A x = b of psfd_apply_differential (the
 * paper's comparator, Sec. 3, Eqs. (4)-(7); its preconditioner table), FP64, on the device:
 *   precond 0  none;
 *   precond 1  the spectral damping D(k) = min(1, kb^2 / |k|^2) on the column's 3-D Fourier
 *              grid (k = (q_x, q_y, k_z), q = q_inc + 2 pi m / P), applied on the left: the
 *              system M A x = M b is solved and its residual is what rtol bounds.
 * Arnoldi with classical Gram-Schmidt and one reorthogonalisation pass (on the device),
 * Givens rotations and the triangular solve on the host (one host wait per iteration); the
 * residual M (b - A x) is recomputed at every restart. Arguments as psfd_apply_differential,
 * and:
 *   b, x          device, complex double [3][nz][n][n]; x is overwritten (start: 0)
 *   work          device scratch of psfd_solve_differential_work(...) complex doubles
 *   restart       basis size per cycle (1 .. 512); max_matvecs bounds the operator applications
 *                 of the Arnoldi steps (the restart residuals are not counted)
 *   matvecs, relres (may be NULL) applications taken, final relative residual
 * Returns PSFD_OK, PSFD_E_NOT_CONVERGED (x holds the last iterate), PSFD_E_ARG or PSFD_E_CUDA. */
int psfd_solve_differential(int n, int nz, int n_pml, double dx, double dz, double wavelength, double eps_bg,
                            double theta_deg, double phi_deg, int precond, const double* eps, const double* b,
                            double* x, double* work, int restart, int max_matvecs, double rtol, int* matvecs,
                            double* relres, void* stream);
/* Complex doubles of work psfd_solve_differential needs: (restart + 4) fields plus the partial sums. */
size_t psfd_solve_differential_work(int n, int nz, int restart);

/* Measurement of the z pass's forward transform (K2 at nf = 128) on two kinds of units, for
 * deciding whether the tensor cores pay (no counterpart in the paper):
 *   method 0  CUDA cores: the register four-step transform of K2 (16 x 8 points, FP32);
 *   method 1  tensor cores: the transform as dense real DFT products, Re/Im of 128 columns as
 *             the 256 columns of B, the cos and -sin matrices as A (128 bins x 64 planes),
 *             every operand split into BF16 hi + lo and three products (hi hi, hi lo, lo hi)
 *             accumulated in FP32 (tcgen05.mma kind::f16 from shared memory into tensor
 *             memory; accuracy about 1e-5 normwise against 1e-7 for method 0).
 *   in   device, complex float [nsets][nslab][ny][nx]: plane p sits at z index p + 1 of a
 *        column of 128 (zero elsewhere); 1 <= nslab <= 63
 *   out  device, complex float [nsets][128][ny][nx]: the unnormalised DFT along z
 * nx must be a multiple of 128 (method 1) or 32 (method 0). Runs on `stream` without
 * synchronising; the first call on a device builds its tables (and synchronises).
 * psfd_zdft_status returns the device's error flag of method 1: 0, or 1 / 2 when a bounded
 * wait for the table copy / the products gave up (the output is then not written).
 * Returns PSFD_OK, PSFD_E_ARG, PSFD_E_NOMEM or PSFD_E_CUDA. */
int psfd_zdft_measure(int method, int nx, int ny, int nsets, int nslab, const void* in, void* out, void* stream);
int psfd_zdft_status(int* flag);

/* Test hook for the device FFT: `count` contiguous transforms of length n, in place, on
 * device data (complex double if fp64 else complex float). inverse = 1 applies the
 * unnormalised inverse. Runs on the legacy default stream and synchronises. */
int psfd_test_fft(int n, int count, int inverse, int fp64, void* data);

#ifdef __cplusplus
}
#endif
#endif /* PSFD_H */
