/*
 * fvns.h -- C ABI of the GB300 (sm_103a) library for the linear-stability
 * method of A. Yu. Gelfgat, "Linear instability of the lid-driven flow in a
 * cubic cavity" (arXiv 1704.08521).
 *
 * Problem (Section 2, Eqs. 1-4): incompressible flow in the unit cube,
 * no-slip walls, the lid z = 1 moving with (u, v) = (cos alpha, sin alpha),
 * Reynolds number Re.  Discretisation (Section 3): second-order staggered
 * finite volumes on a stretched nx x ny x nz grid.
 *
 * ---------------------------------------------------------------- layout --
 * Every array argument is a DEVICE pointer to float64 data owned by the
 * caller (the library never frees it) unless a comment says "host".
 *   cell field  : nz*ny*nx values, C order [k][j][i], i (x) fastest.
 *   velocity    : 3 cell-sized blocks [u | v | w] (n_vel = 3*nz*ny*nx).
 *                 u[k][j][i] is the x-velocity on the face x_i, the low face
 *                 of cell i; u[k][j][0] is the wall x = 0.  Likewise
 *                 v[k][0][i] and w[0][j][i] are walls.  Wall entries are
 *                 ignored on input and written as 0 on output.  The high
 *                 walls (x = 1, y = 1, z = 1) are not stored.
 * The lid velocity of Eq. 4 is never stored: it enters through the stencils.
 *
 * ---------------------------------------------------------------- errors --
 * Every call returns fv_status; on failure fv_last_error() gives a message
 * (thread-local).  Invalid arguments give FV_EINVAL and launch nothing.
 * Iteration caps give FV_ENOCONV with the stats filled in.  No call traps,
 * asserts or exits.
 *
 * ---------------------------------------------------------------- streams --
 * All work is queued on the stream given to fv_grid_create.  Calls that
 * return host scalars (stats, eigenvalues) synchronise that stream.
 */
#ifndef FVNS_H
#define FVNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FV_OK = 0,
  FV_EINVAL = 1,   /* bad size, null pointer, bad option */
  FV_ENOMEM = 2,   /* device allocation failed */
  FV_ECUDA = 3,    /* a CUDA call failed (message in fv_last_error) */
  FV_ENOCONV = 4,  /* an iteration cap was reached */
  FV_ENAN = 5,     /* a NaN/Inf appeared in a norm */
  FV_ETIMEOUT = 6  /* a bounded device-side wait gave up (the tensor-core
                      pressure transforms of FV_MIXED / FV_FF); the grid's
                      sticky timeout word is cleared once reported */
} fv_status;

/* Grid stretching.  Section 3, Eq. 5: x -> x - 0.0975 sin(2 pi x) applied to
 * the uniform points i/N (FV_MAP_SINE0975); FV_MAP_COSINE is
 * x_i = (1 - cos(pi i / N)) / 2; FV_MAP_UNIFORM is x_i = i / N. */
typedef enum { FV_MAP_SINE0975 = 0, FV_MAP_COSINE = 1, FV_MAP_UNIFORM = 2 } fv_map;

/* Arithmetic of the stencil and pressure-correction sweeps.
 * FV_FP64 : everything in float64 (on GB300 the FP64 pipes run at ~1/70 of
 *           the FP32 rate: this is the plain reference form).
 * FV_MIXED: J.v and the tensor-product pressure-correction solve in float32;
 *           the defect-correction state (velocity, pressure) and its
 *           divergence in float-float (hi + lo float pairs, ~48 bits).
 * FV_FF   : as FV_MIXED, but J.v also in float-float: results agree with
 *           FV_FP64 to ~1e-12 relative, on the FP32 pipes (for eigenvalues
 *           to 1e-7 and below).  Graph path only for simple_krylov_solve. */
typedef enum { FV_FP64 = 0, FV_MIXED = 1, FV_FF = 2 } fv_prec;

typedef struct fv_grid fv_grid; /* opaque: metrics, solver tables, workspace */

typedef struct {
  int nx, ny, nz;
  int64_t n_cell; /* nx*ny*nz           */
  int64_t n_vel;  /* 3*n_cell            */
  int64_t n_unknown_vel; /* (nx-1)ny nz + nx(ny-1)nz + nx ny(nz-1) */
  int64_t workspace_bytes; /* device memory the grid holds */
} fv_grid_info;

/* Options of one Krylov-vector evaluation (Section 3, the algorithm after
 * Eq. 10).  Zero-initialised fields take the defaults in brackets. */
typedef struct {
  double eps;     /* stop when ||phi_k||_inf <= eps * ||phi_1||_inf  [1e-8] */
  int max_pass;   /* cap on SIMPLE passes                            [200] */
  int prec;       /* fv_prec                                 [FV_FP64 = 0] */
  double omega;   /* under-relaxation of each correction, (0, 1]     [1.0] */
  double sigma;   /* >0: return P(L_U v + sigma v) - sigma v, the shifted
                     operator used inside GMRES and Arnoldi; 0: the plain
                     Krylov vector P L_U v of Eqs. 8-9                 [0] */
  int async;      /* FV_MIXED only: 1 = do not synchronise; the call then
                     returns FV_OK once queued and stats are not filled
                     (a non-converged loop is not reported)              [0] */
  int pressure;   /* solver of each pass's pressure correction: 0 the
                     tensor-product factorisation, 1 the multigrid solve of
                     fv_pressure_solve_mg (FV_FP64 only)                  [0] */
  double pressure_rtol; /* multigrid: relative residual of each pass's
                     solve; the later passes correct the rest          [1e-3] */
} fv_simple_opts;

typedef struct {
  int passes;          /* SIMPLE passes done                                */
  double phi_first;    /* ||phi_1||_inf                                     */
  double phi_last;     /* ||phi_last||_inf                                  */
  double div_max;      /* max |D v_out| after the last pass                 */
} fv_simple_stats;

typedef struct {
  double tol;        /* ||F||_inf target                              [1e-10] */
  int max_newton;    /* Newton iteration cap                             [30] */
  int gmres_m;       /* GMRES restart length (Section 3: 100)           [100] */
  int gmres_max_it;  /* GMRES iteration cap per Newton step           [20000] */
  double gmres_rtol; /* relative GMRES tolerance per Newton step       [1e-8] */
  int prec;          /* fv_prec of the Krylov vectors           [FV_FP64 = 0] */
  double sigma;      /* shift of the gradient complement                 [10] */
  double simple_eps; /* SIMPLE tolerance inside GMRES                  [1e-10] */
  int linear;        /* fv_linear: solver of each Newton correction
                        [FV_LIN_GMRES_BICGSTAB = 0] */
  double gmres_sat;  /* a GMRES(m) restart cycle whose residual W-norm ends
                        above gmres_sat x its start counts as saturated [0.5] */
  int precond;       /* 0: the paper's unpreconditioned Krylov vectors; 1: a
                        Stokes-type right preconditioner M^-1 = P (s - Lap/Re)^-1
                        (vector Laplacian of the momentum equations, s =
                        precond_sigma, then the projection onto divergence-free
                        fields) with flexible GMRES(m) and, after its
                        saturation (linear = FV_LIN_GMRES_BICGSTAB), the
                        right-preconditioned BiCGstab(2).  Same corrections;
                        far fewer operator products on strongly stretched
                        grids                                              [0] */
  double precond_sigma; /* s >= 0 of the preconditioner                    [0] */
  int forcing;       /* 0: every correction to gmres_rtol; 1: Eisenstat-Walker
                        forcing terms eta_k = 0.9 (||F_k|| / ||F_k-1||)^2 in
                        [gmres_rtol, 0.1] (loose early, tight near the root) [0] */
  int gmres_aug;     /* precond = 1: the last gmres_aug (<= 4) steps of each
                        flexible GMRES cycle take the corrections of the
                        previous cycles as their directions (the LGMRES
                        augmentation of Baker, Jessup & Manteuffel 2005,
                        against the stagnation of restarted GMRES)        [0] */
  double tau;        /* >= 0: each correction solves (A - tau I) du = F
                        instead of A du = F (a shifted, pseudo-transient
                        Newton step: same steady state; error modes of
                        eigenvalue lambda contract by tau / |lambda - tau|
                        per step; moves the weakly damped oscillatory
                        modes near the imaginary axis away from it, where
                        restarted Krylov solvers stagnate)                [0] */
} fv_newton_opts;

/* Section 3: the Newton corrections are computed by restarted GMRES or by
 * BiCGstab(2) (Sleijpen & Fokkema 1993); when GMRES(100) saturates, its last
 * approximation is the initial guess of BiCGstab(2). */
typedef enum {
  FV_LIN_GMRES_BICGSTAB = 0,  /* GMRES(m) cycles until saturated, then BiCGstab(2) */
  FV_LIN_GMRES = 1,           /* GMRES(m) only                                     */
  FV_LIN_BICGSTAB = 2         /* BiCGstab(2) only, from a zero correction           */
} fv_linear;

typedef struct {
  int iterations;          /* Newton steps taken                        */
  int gmres_total;         /* GMRES iterations summed over all steps    */
  double res_hist[64];     /* ||F||_inf before each step (first 64)     */
  double res_final;
  int bicgstab_total;      /* BiCGstab(2) operator applications, summed */
  double lin_hist[64];     /* per Newton step: the linear solver's final residual
                              W-norm over ||F_m||_W (GMRES: its last restart's
                              estimate; BiCGstab(2): its smallest recursive one) */
} fv_newton_stats;

typedef struct {
  double tol;        /* Ritz residual <= tol * max(|theta|, eps^(2/3))  [1e-10] */
  int max_restarts;  /* implicit-restart cap                           [5000] */
  int prec;          /* fv_prec of the Krylov vectors           [FV_FP64 = 0] */
  double sigma;      /* shift of the gradient complement (must exceed minus
                        the real part of every wanted eigenvalue)        [10] */
  double simple_eps; /* SIMPLE tolerance per Krylov vector             [1e-10] */
} fv_arnoldi_opts;

typedef struct {
  int restarts;
  int matvecs;
  double ritz_resid[64]; /* estimated residual of each returned pair */
} fv_arnoldi_stats;

/* Section 2-3: allocate a grid of nx x ny x nz finite volumes (each >= 4,
 * <= 1024, n_vel < 2^31) with map fv_map, lid angle alpha (radians; 0 = lid
 * parallel to the x sidewall, pi/4 = parallel to the diagonal plane) and
 * Reynolds number re > 0.  `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream).  Builds the metrics and the tensor-product eigenbases
 * of the pressure-correction operator and allocates all workspace, so later
 * calls never allocate.  *out receives the handle. */
fv_status fv_grid_create(int nx, int ny, int nz, int map, double alpha, double re,
                         void* cuda_stream, fv_grid** out);
/* Change the grid's Reynolds number (re > 0).  A change synchronises the
 * grid's stream and drops the captured evaluation graphs, which are captured
 * again by the next FV_MIXED / FV_FF evaluation (outside any stream capture). */
fv_status fv_grid_set_re(fv_grid* g, double re);
fv_status fv_grid_set_stream(fv_grid* g, void* cuda_stream);
fv_status fv_grid_get_info(const fv_grid* g, fv_grid_info* info /* host */);
void fv_grid_destroy(fv_grid* g);
const char* fv_last_error(void);

/* Eqs. 1-4 discretised: steady residual of (U, P).
 * F_mom[n_vel] = (1/Re) Lap U - div(U (x) U) - grad P at the velocity faces
 * (lid velocity of Eq. 4 in the wall stencils), F_div[n_cell] = D U. */
fv_status ns_residual(const fv_grid* g, const double* U, const double* P,
                      double* F_mom, double* F_div);

/* Eq. 6 / Eq. 10: Jv[n_vel] = (1/Re) Lap v - div(U (x) v) - div(v (x) U),
 * the linearised momentum operator about U with homogeneous wall values
 * (the momentum predictor w of Eq. 10).  prec selects float64 or float32
 * arithmetic (inputs and output stay float64). */
fv_status ns_jacvec(const fv_grid* g, const double* U, const double* v, double* Jv, int prec);

/* Register U[n_vel] as the grid's base flow (Eq. 6: the steady state the
 * operator is linearised about).  Krylov methods apply the operator about
 * one U thousands of times; the float32 rounding and float-float split of U
 * that the FV_MIXED and FV_FF stencils read are made here once instead of in
 * every evaluation.  Afterwards simple_krylov_solve accepts U = NULL and then
 * uses these copies (and, for FV_FP64, this array, which the caller keeps
 * alive and unchanged while it is used that way).  Register again after
 * changing U.  newton_steady and arnoldi_leading register their U
 * themselves (this replaces any earlier registration). */
fv_status fv_grid_set_base(fv_grid* g, const double* U);

/* Section 3, Eqs. 8-10 and the SIMPLE-like algorithm: from v_in compute
 * w = L_U v_in (Eq. 10), then repeat { solve D G phi = D v (Neumann);
 * v -= omega G phi; p += omega phi } until the stop test of opts.  Returns
 * the divergence-free v_out[n_vel] and p_out[n_cell] (zero mean; may be
 * NULL).  v_in and v_out may not alias.  stats may be NULL.
 * FV_MIXED runs the whole evaluation as one CUDA graph launch whose pass
 * loop is decided on the device; the graph is captured on the first such
 * call for a grid (make that call outside any stream capture).  U = NULL:
 * the base flow registered by fv_grid_set_base. */
fv_status simple_krylov_solve(const fv_grid* g, const double* U, const double* v_in,
                              double* v_out, double* p_out,
                              const fv_simple_opts* opts, fv_simple_stats* stats);

/* Section 3, Newton steps 1-4 at the grid's current Re: U[n_vel] (in: guess,
 * e.g. all zeros = rest; out: steady state) and P[n_cell] (out).  Each
 * correction solves P L_U u = P F_mom (in the shifted form A_sigma) by the
 * opts.linear solver -- restarted GMRES(m), BiCGstab(2), or GMRES(m) until
 * it saturates followed by BiCGstab(2) -- whose operator applications come
 * from simple_krylov_solve.  gmres_max_it caps the operator applications of
 * both solvers per correction.  Returns FV_ENOCONV if ||F||_inf >= tol after
 * max_newton steps. */
fv_status newton_steady(fv_grid* g, double* U, double* P,
                        const fv_newton_opts* opts, fv_newton_stats* stats);

/* Section 3, Eq. 7: the nev (<= 64) eigenvalues of largest real part of the
 * linearised operator about the steady U, by implicitly restarted Arnoldi
 * (Krylov dimension m, nev + 2 <= m <= 128) in regular mode.  The Arnoldi
 * steps of a cycle build the FP64 Hessenberg matrix in device memory with no
 * host round trip; the small dense restart work (Ritz values by Francis
 * QR, exact shifts) takes one copy of it per cycle.  v0[n_vel] is
 * the start vector (device; e.g. a seeded Gaussian; it is projected first).
 * lam_re/lam_im (host, nev each) receive the eigenvalues sorted by
 * descending real part, conjugate pairs adjacent (positive imaginary part
 * first).  evec (device, optional, 2*n_vel: real then imaginary part)
 * receives the leading eigenvector, unit W-norm, phase such that its
 * largest-modulus entry is real positive. */
fv_status arnoldi_leading(const fv_grid* g, const double* U, const double* v0,
                          int m, int nev, double* lam_re, double* lam_im, double* evec,
                          const fv_arnoldi_opts* opts, fv_arnoldi_stats* stats);

/* Options / statistics of the critical-Re search. */
typedef struct {
  double rtol;        /* stop when |Re_{k+1} - Re_k| <= rtol Re_{k+1}       [1e-8] */
  int max_iter;       /* secant steps after the two starting points          [30] */
  int m, nev;         /* Arnoldi Krylov dimension / eigenvalues          [30, 4] */
  int prec;           /* fv_prec of the Krylov vectors              [FV_FP64 = 0] */
  double newton_tol;  /* ||F||_inf of each steady state                  [1e-10] */
  double arnoldi_tol; /* Ritz tolerance                                  [1e-10] */
  int precond;        /* fv_newton_opts.precond of the steady states          [0] */
  double precond_sigma; /* fv_newton_opts.precond_sigma                       [0] */
  int forcing;        /* fv_newton_opts.forcing                                [0] */
  int max_restarts;   /* fv_arnoldi_opts.max_restarts (0: its default)         [0] */
  double tau;         /* fv_newton_opts.tau                                    [0] */
  int max_newton;     /* fv_newton_opts.max_newton (0: its default)            [0] */
} fv_critical_opts;

typedef struct {
  int evaluations;        /* sigma(Re) evaluations (Newton + Arnoldi)    */
  double re_hist[64];     /* Re of each evaluation                       */
  double sigma_hist[64];  /* real part of the leading eigenvalue         */
  double omega_hist[64];  /* |imaginary part| of the leading eigenvalue  */
} fv_critical_stats;

/* Section 3: the critical Reynolds number, where the real part of the
 * leading eigenvalue Lambda (largest real part) crosses zero, and the
 * critical circular frequency omega_cr ~ |Im Lambda|.  Secant iteration on
 * sigma(Re) = Re(Lambda(Re)) from re0 and re1 (the paper does not say how it
 * brackets Re_cr).  Each evaluation sets the grid's Re, runs newton_steady
 * warm-started from U, P (in: a steady state near re0; out: the steady
 * state at Re_cr) and arnoldi_leading from v0.  re_cr / omega_cr: host. */
fv_status fv_critical_re(fv_grid* g, double* U, double* P, const double* v0, double re0, double re1,
                         const fv_critical_opts* opts, double* re_cr, double* omega_cr,
                         fv_critical_stats* stats);

/* ------------------------------------------------------------ batching --
 * Several instances (grids of uneven sizes, Reynolds numbers and lid
 * angles, e.g. the bracketing points of a critical-Re search) advance one
 * mixed-precision Krylov-vector evaluation each in ONE CUDA graph launch:
 * the momentum predictors of all instances in one persistent work-queue
 * kernel, then the SIMPLE loops as concurrent graph branches, each with a
 * device-side WHILE node.  The batch borrows the grids (their workspace;
 * an instance's Re is read when fv_batch_krylov is called, so fv_grid_set_re
 * between calls takes effect).  The graph is captured on the first
 * fv_batch_krylov call (outside any stream capture). */
typedef struct fv_batch fv_batch;
fv_status fv_batch_create(int n /* 1..32 */, fv_grid* const* grids /* host array */,
                          void* cuda_stream, fv_batch** out);
void fv_batch_destroy(fv_batch* b);
/* out[i] = P (L_{U[i]} x[i] + sigma x[i]) - sigma x[i] for every instance
 * (host arrays of device pointers; Eqs. 8-10 with the stop test of
 * simple_krylov_solve, tolerance eps).  passes (host, n, optional): SIMPLE
 * passes per instance; when given, the call synchronises and reports
 * FV_ENOCONV / FV_ENAN of any instance. */
fv_status fv_batch_krylov(fv_batch* b, const double* const* U, const double* const* x,
                          double* const* out, double eps, double sigma, int* passes);
/* Time the batched momentum kernel with 1, 2, 4, 8 z-planes per work item
 * (ms: host, 4 entries, optional) and keep the fastest (returned in *best). */
fv_status fv_batch_autotune(fv_batch* b, int* best, double* ms);
/* Set the z-planes per work item explicitly (e.g. from a cached tuning). */
fv_status fv_batch_set_tile(fv_batch* b, int planes);

/* Section 3 step 1, right-hand side: r[n_cell] = D v, the finite-volume
 * divergence of v[n_vel] (outflux of each cell over its volume; the wall
 * faces carry zero normal velocity).  float64, device. */
fv_status ns_divergence(const fv_grid* g, const double* v, double* r);

/* ------------------------------------------------------- learned guess --
 * Optional first pass of the SIMPLE-like loop of Section 3 from a learned
 * guess of the pressure correction.  The paper has no counterpart: the
 * paper's loop starts every evaluation from phi = 0 and an exact solve.
 * A 3-D convolutional U-Net (4 levels of 16/32/48/64 channels, two 3x3x3
 * convolutions + ReLU per level, 2x2x2 mean pooling, nearest upsampling
 * with skip concatenation, a 1x1x1 output layer; BF16 weights and
 * activations, float32 accumulation on the tensor cores) maps the
 * right-hand side in index units, q = r (dx_i dy_j dz_k)^(2/3) with
 * r = D w, scaled by 1/S (S = rms of q), and the metric channels
 * log(n_x dx_i), log(n_y dy_j), log(n_z dz_k) to phi / S.  Grid
 * dimensions: multiples of 8 in [8, 1024].  The network owns its parameters (float32 + BF16 mirror, Adam
 * moments) and an activation workspace that grows to the largest grid it
 * has seen.  Parameter layout (float32): for each of the 14 convolutions,
 * in order encoder 0a, 0b, 1a, 1b, 2a, 2b, bottom a, b, decoder 2a, 2b, 1a,
 * 1b, 0a, 0b, the weights W[27][cout][cin] (tap 9(dz+1)+3(dy+1)+(dx+1))
 * then the bias[cout]; last the 16 output weights and the output bias.
 * Channels (cin -> cout): 16->16, 16->16, 16->32, 32->32, 32->48, 48->48,
 * 48->64, 64->64, 112->48, 48->48, 80->32, 32->32, 48->16, 16->16; decoder
 * inputs are [upsampled coarser output, skip of the same level].  The
 * network input has 16 channels: the 4 above, then 12 zeros. */
typedef struct fv_unet fv_unet;
/* He-normal weights from seed, zero biases; work on cuda_stream. */
fv_status fv_unet_create(uint64_t seed, void* cuda_stream, fv_unet** out);
void fv_unet_destroy(fv_unet* u);
int fv_unet_param_count(const fv_unet* u);
fv_status fv_unet_set_stream(fv_unet* u, void* cuda_stream);
/* Copy all parameters in (device, float32, param_count); resets Adam. */
fv_status fv_unet_set_params(fv_unet* u, const float* params);
/* Copy parameters and/or the gradients of the last backward pass out
 * (device, float32, param_count; either may be NULL). */
fv_status fv_unet_get_params(const fv_unet* u, float* params, float* grads);
/* Raw forward pass: in[4][n_cell] (device float32 input planes, cells x
 * fastest), out[n_cell] (device float32). */
fv_status fv_unet_forward(fv_unet* u, int nx, int ny, int nz, const float* in, float* out);
/* Gradients of the mean-free square loss L = mean((e - mean e)^2),
 * e = out - target (target: device float32, n_cell), with respect to every
 * parameter, for the last forward pass.  *loss (host, optional) = L; the
 * call then synchronises the network's stream. */
fv_status fv_unet_backward(fv_unet* u, const float* target, double* loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradients. */
fv_status fv_unet_adam(fv_unet* u, float lr);
/* phi[n_cell] (device float64) = the network's guess for the Poisson
 * right-hand side r[n_cell] (device float64) on grid g (g's stream). */
fv_status fv_unet_guess(fv_unet* u, const fv_grid* g, const double* r, double* phi);
/* One training step on the pair (r, phi) of grid g: normalise, forward,
 * backward, Adam; *loss (host, optional) = the loss before the step. */
fv_status fv_unet_train_step(fv_unet* u, const fv_grid* g, const double* r, const double* phi,
                             float lr, double* loss);
/* simple_krylov_solve (prec FV_MIXED or FV_FF, host-driven loop) whose
 * first pass takes phi from the network instead of the exact solve; the
 * following passes are the exact tensor-product solves of the paper's loop.
 * The stop test keeps the tolerance of the plain loop: corrections are
 * compared with the pressure after the first exact pass (guess + its
 * correction), the plain loop's first correction.  stats->passes counts
 * the guess pass; a net whose guess does not converge under the same test
 * returns FV_ENOCONV like the plain loop. */
fv_status simple_krylov_solve_guess(const fv_grid* g, fv_unet* u, const double* U,
                                    const double* v_in, double* v_out, double* p_out,
                                    const fv_simple_opts* opts, fv_simple_stats* stats);

/* Section 4, Eqs. 11-17: the divergence-free projection of the velocity
 * v[n_vel] (float64, device) onto a set of coordinate planes and its vector
 * potential.  plane 0: the (x, z) planes -> v_1 = (u_1, 0, w_1) and
 * Psi^(y); 1: the (y, z) planes -> v_2 = (0, v_2, w_2) and Psi^(x); 2: the
 * (x, y) planes -> v_3 = (u_3, v_3, 0) and Psi^(z).  vp[n_vel] (device)
 * receives the projection: the two in-plane components of v minus the
 * gradient of phi, (L_a + L_c) phi = (in-plane divergence of v) solved
 * exactly in every plane (Neumann walls), so that the in-plane divergence
 * (Eqs. 12-14) vanishes to round-off; the normal component is zero.
 * psi (device, optional) receives the potential on the corners of the
 * planes' cells: a [k][j][i] array with n + 1 entries along the two in-plane
 * axes and n along the normal one (e.g. (nz+1) x ny x (nx+1) for plane 0),
 * zero on the walls, with v_1 = rot(0, Psi, 0), v_2 = rot(Psi, 0, 0),
 * v_3 = rot(0, 0, Psi).  Wall entries of v are ignored.  v and vp may not
 * alias.  float64 throughout. */
fv_status fv_plane_projection(const fv_grid* g, const double* v, int plane, double* vp,
                              double* psi);

/* W-weighted inner product <a, b> = sum over velocity faces of the momentum
 * control-volume size times a b (wall faces excluded).  Result to host. */
fv_status fv_dot_w(const fv_grid* g, const double* a, const double* b, double* out /* host */);

/* Section 3 step 1 alone: phi[n_cell] = zero-mean solution of D G phi = r
 * (Neumann) by the tensor-product factorisation; prec as above. */
fv_status fv_pressure_solve(const fv_grid* g, const double* r, double* phi, int prec);

/* Section 3 step 1 by multigrid: phi[n_cell] (device, float64) = the
 * solution of D G phi = r[n_cell] (device, float64) with Neumann walls, of
 * zero volume-weighted mean -- the same phi as fv_pressure_solve.  Conjugate
 * gradients in float64 on the symmetric form -V D G phi = -V r (r first made
 * compatible with the null space: r - sum(V r)/sum(V)), preconditioned by
 * one float32 V-cycle per iteration: full coarsening while an axis has more
 * than 4 cells, alternating-direction zebra line Gauss-Seidel smoothing (one
 * tridiagonal solve per grid line), linear interpolation between coarse
 * centres and its transpose, rediscretised coarse operators, an exact
 * separable solve on the coarsest grid.  guess (device, optional, may equal
 * phi) is the initial phi, zero if NULL.  Stops at ||b - A phi||_2 <=
 * rtol ||b||_2; FV_ENOCONV (stats filled) after max_iter iterations.  The
 * hierarchy and its workspace (~6 float32 and 5 float64 cell arrays) are
 * built on the first call and kept with the grid.  Runs on the grid's
 * stream; returns after the last convergence check (the final mean removal
 * is queued). */
typedef struct {
  double rtol;     /* relative residual target                        [1e-10] */
  int max_iter;    /* conjugate-gradient iteration cap                  [100] */
  int nu;          /* smoothing sweeps (each x, y, z) before and after  [1]   */
  double omega;    /* relaxation factor of the line sweeps              [1.0] */
} fv_mg_opts;

typedef struct {
  int iterations;  /* conjugate-gradient iterations (one V-cycle each)         */
  int levels;      /* grids of the hierarchy, the finest included              */
  double rel_res;  /* ||b - A phi||_2 / ||b||_2 at the end                     */
} fv_mg_stats;

fv_status fv_pressure_solve_mg(fv_grid* g, const double* r, double* phi, const double* guess,
                               const fv_mg_opts* opts, fv_mg_stats* stats);

/* Allocation-free variant of fv_pressure_solve (prec = FV_MIXED) for callers
 * that cannot allocate device memory -- code running inside a memory pool it
 * does not own and may not grow, or embedded users with no access to an
 * allocator.  The paper has no counterpart: this is a property of the
 * library, not of the method.  It needs no grid handle: nx, ny, nz (each in
 * [4, 128], nx*ny*nz <= 1048576) and map describe the grid; r[n_cell]
 * (device, float64) is the right-hand side, phi[n_cell] (device, float64)
 * receives the zero-mean solution of D G phi = r, work is queued on
 * cuda_stream.  The call makes no cudaMalloc, cudaFree or other allocating
 * call: all scratch (eigenbases and two float32 transform buffers, ~8.4 MB)
 * lives in one fixed device array inside the library, which every GPU that
 * uses it holds until the process exits.  The library's device code is
 * loaded lazily, so the FIRST call on each device (with that device
 * current) loads it, reserves the array and looks up its device address:
 * make that first call before entering any region where the driver may not
 * reserve memory; later calls reserve nothing.  The host-side tables of
 * each (dimension, map) are computed on first use and kept.  Sizes beyond
 * the limits give FV_EINVAL.  Calls share the array: calls that overlap on
 * the GPU race on it. */
fv_status fv_pressure_solve_noalloc(int nx, int ny, int nz, int map, const double* r,
                                    double* phi, void* cuda_stream);

/* ------------------------------------------------------- instrumentation --
 * Kernel classes timed by the optional per-grid profiler (CUDA events
 * recorded on the grid's stream around every launch of that class). */
typedef enum {
  FV_K_MOMENTUM = 0,   /* J.v / residual stencil                       */
  FV_K_DIVERGENCE = 1, /* D v                                           */
  FV_K_CORRECT = 2,    /* SIMPLE correction + divergence pass           */
  FV_K_TPF_X = 3,      /* pressure solve: x-axis transforms             */
  FV_K_TPF_YZ = 4,     /* pressure solve: y- and z-axis transforms      */
  FV_K_DOTS = 5,       /* weighted inner products                       */
  FV_K_VECTOR = 6,     /* other vector kernels (updates, scaling, ...)  */
  FV_K_TPF_XINV = 7,   /* pressure solve: inverse x-y transforms        */
  FV_K_MG_SMOOTH = 8,  /* multigrid: line Gauss-Seidel smoothing sweeps */
  FV_K_MG_OTHER = 9,   /* multigrid: transfers, coarse solve, CG steps  */
  FV_NKIND = 10
} fv_kernel_kind;

/* Start (on != 0) or stop recording; starting clears earlier records. */
fv_status fv_profile_enable(fv_grid* g, int on);
/* Synchronise the grid's stream and report, per fv_kernel_kind, the summed
 * device time in ms and the number of launches since fv_profile_enable. */
fv_status fv_profile_read(fv_grid* g, double* ms /* host, FV_NKIND */,
                          int64_t* launches /* host, FV_NKIND */);
/* Total number of launches (kernel launches and graph launches) this
 * library has issued in the process. */
int64_t fv_launch_count(void);
/* Error-path testing without a device fault: set the grid's sticky device
 * timeout word exactly as a tensor-core pressure transform does when one of
 * its bounded mbarrier waits gives up, so that the next FV_MIXED / FV_FF
 * evaluation (or Krylov cycle) on the grid reports FV_ETIMEOUT.  Only
 * status == FV_ETIMEOUT is accepted (else FV_EINVAL).  Queued on the grid's
 * stream. */
fv_status fv_debug_inject_status(fv_grid* g, int status);
/* Time `reps` back-to-back launches of one FV_MIXED kernel class
 * (FV_K_MOMENTUM, FV_K_DIVERGENCE, FV_K_CORRECT, FV_K_TPF_X = one forward
 * x-y slab transform, FV_K_TPF_XINV = one inverse x-y slab transform,
 * FV_K_TPF_YZ = one z-axis transform) on the grid's workspace with CUDA events on its
 * stream; *ms_per_launch (host) receives the mean device time.  Needs one
 * earlier FV_MIXED simple_krylov_solve on the grid. */
fv_status fv_bench_kernel(fv_grid* g, int kind, int reps, double* ms_per_launch);

#ifdef __cplusplus
}
#endif

#endif /* FVNS_H */
