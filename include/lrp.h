/*
 * lrp.h — C ABI of the GB300 low-rank posterior-covariance library.
 *
 * The library computes, on one GPU, the hot path of the low-rank posterior
 * covariance method for a linear Bayesian inverse problem whose parameter is
 * the initial condition u of a parabolic PDE (Benner, Qiu, Stoll,
 * "Low-rank computation of posterior covariance matrices in Bayesian inverse
 * problems", Sec. 6 Eq. (pde)):
 *
 *   y_t - div(kappa grad y) = 0 (or the convection-diffusion equation
 *   y_t - nu Laplace y + w . grad y = 0 of Sec. 6.2, upwind) on the unit
 *   square/cube, y = 0 on the boundary, y(0) = u; finite differences with
 *   n interior nodes per axis
 *   (h = 1/(n+1)), implicit Euler with tau = T/nt:
 *   (I + tau L) y_n = y_{n-1}  (block row of Sec. 6.1 Eq. (st_pde), M = I).
 *   Data: point sensors read the bilinear/trilinear interpolant of y at the
 *   observed steps obs_every, 2*obs_every, ..., nt (Sec. 6 Eq. (obj),
 *   Eq. (dis_obj)). Gamma_noise = sigma^2 I.
 *   Prior: Gamma_prior = R^-2, R = I + alpha L0 (L0 the constant-coefficient
 *   Laplacian), so Gamma_prior^{1/2} = R^{-1}; or Gamma_prior = gamma I
 *   (R^{-1} = sqrt(gamma) I, prior_kind LRP_PRIOR_IDENTITY).
 *   F = parameter-to-observable map; H_mis = F^T F / sigma^2;
 *   Htilde = R^{-1} H_mis R^{-1}  (Sec. 2 Eq. (prior_pre), Sec. 6.1 Eq. (misfit)).
 *
 * Conventions (all entry points):
 *  - Grid vectors have nx = n^dim entries, node (i0,i1,i2) at flat index
 *    i0 + n*i1 + n*n*i2 (first coordinate fastest).
 *  - Blocks of vectors are column-major: column j of a block X with leading
 *    dimension ldx starts at X + j*ldx.
 *  - Observation vectors (one per column) have n_data = n_obs * n_steps
 *    entries, step-major: (k-th observed step, sensor s) at k*n_obs + s.
 *  - Array arguments may be host or device pointers; the library detects
 *    which with cudaPointerGetAttributes and stages host arrays through the
 *    device. The caller owns every array it passes. Device arrays must be
 *    on the problem's device; device memory of another GPU is rejected with
 *    LRP_EINVAL (managed memory is accepted).
 *  - All work is ordered on the problem's CUDA stream; every call returns
 *    after that work has completed (synchronous).
 *  - Errors: a call returns a status; on error the outputs are undefined and
 *    lrp_last_error() describes the failure. A solve that misses its
 *    tolerance within its iteration cap still fills its outputs and stats
 *    and returns LRP_ENOCONV.
 *  - Handles are not thread-safe: one host thread per handle at a time.
 */
#ifndef LRP_H
#define LRP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRP_OK = 0,
  LRP_EINVAL = 1,     /* invalid argument */
  LRP_ENOMEM = 2,     /* device or host allocation failed */
  LRP_ENOCONV = 3,    /* a solve or the eigensolver missed its tolerance */
  LRP_ENONFINITE = 4, /* NaN or Inf in an input */
  LRP_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  LRP_EBUDGET = 6,    /* request exceeds the configured memory budget */
  LRP_ECUDA = 7       /* CUDA runtime error */
} lrp_status;

/* precision of the inner (PCG / multigrid) arithmetic */
enum {
  LRP_FP64 = 0,  /* everything in FP64 */
  LRP_MIXED = 1  /* FP32 multigrid-PCG corrections inside FP64 iterative refinement */
};

/* PDE operator (lrp_problem_desc.pde) */
enum { LRP_PDE_HEAT = 0, LRP_PDE_CONVDIFF = 1 };

/* prior covariance (lrp_problem_desc.prior_kind) */
enum {
  LRP_PRIOR_LAPLACE = 0,  /* Gamma_prior = (I + alpha L0)^-2, Gamma_prior^{1/2} = (I + alpha L0)^-1 */
  LRP_PRIOR_IDENTITY = 1  /* Gamma_prior = gamma I, Gamma_prior^{1/2} = sqrt(gamma) I */
};

/* flags of lrp_hessian_apply */
enum {
  LRP_PRIOR_PRECOND = 0,      /* default: Y = Htilde X */
  LRP_MISFIT_ONLY = 1u << 0,  /* Y = H_mis X (no prior factors) */
  LRP_KEEP_TRAJ_FACTORS = 1u << 1, /* also compress the forward trajectory of
                                      each column to low-rank-in-time factors
                                      Y ~ W V^T (Sec. 3); ranks in the stats */
  LRP_LOWRANK_SOURCE = 1u << 2,    /* the product of Sec. 4 Algorithm 1 "up to the
                                      truncation tolerance": the state trajectory
                                      and the adjoint trajectory are kept as
                                      W V^T truncated to time_trunc_tol (rank cap
                                      time_rank_max), the adjoint's data are the
                                      observations of the truncated state and the
                                      result is the truncated adjoint's first
                                      step (then the prior factor). No longer
                                      exactly symmetric: the operator of
                                      lrp_arnoldi. Ranks and truncation errors of
                                      both trajectories in the stats. Not with
                                      LRP_KEEP_TRAJ_FACTORS. */
  LRP_ALS_SOLVES = 1u << 3         /* the forward and the adjoint space-time systems
                                      (Sec. 6.1, Eq. (st_pde)) are solved by the
                                      alternating low-rank solver of lrp_als_solve
                                      (rank als_rank, als_sweeps sweeps from the
                                      first als_rank unit time vectors) instead of
                                      time stepping: the state Y ~ W_Y V_Y^T, the
                                      adjoint's source B^T B W_Y V_Y^T / sigma^2 at
                                      the observed steps, the result the adjoint
                                      solution's first step (then the prior
                                      factor). Equals Htilde X up to the solver's
                                      residual. Stats: time_rank_max / adj_rank_max
                                      = the rank, time_trunc_err / adj_trunc_err =
                                      the largest final relative residual of the
                                      forward / adjoint solves, n_solves = the
                                      preconditioner's spatial solves per column.
                                      Not with LRP_KEEP_TRAJ_FACTORS or
                                      LRP_LOWRANK_SOURCE; also a flag of lrp_arnoldi. */
};

typedef struct lrp_problem lrp_problem;     /* opaque, library-owned */
typedef struct lrp_posterior lrp_posterior; /* opaque, library-owned, device-resident factors */

typedef struct {
  int dim;                  /* 2 or 3 */
  int n;                    /* interior nodes per axis; n = 2^L - 1, 3 <= n <= 511 */
  int nt;                   /* time steps */
  double T;                 /* final time */
  const double* kappa_faces;/* host; NULL -> kappa = 1. Else the face values of kappa:
                               faces normal to axis 0, then axis 1 (then 2); along
                               their own axis a face index runs 0..n (face i lies
                               between nodes i-1 and i), along the other axes 0..n-1;
                               first coordinate fastest within each block. */
  double prior_alpha;       /* R = I + alpha*L0 */
  int n_obs;                /* number of sensors (>= 1) */
  const double* obs_xyz;    /* host, n_obs*dim sensor coordinates in (0,1)^dim, point-major */
  int obs_every;            /* observed steps obs_every, 2*obs_every, ..., <= nt */
  double sigma;             /* noise standard deviation */
  int precision;            /* LRP_FP64 or LRP_MIXED */
  double time_trunc_tol;    /* relative Frobenius tolerance of the time factors (<= 0 -> 1e-8) */
  int time_rank_max;        /* rank cap of the time factors (e.g. 40) */
  int time_chunk;           /* steps buffered between recompressions (0 -> 16, at most 64) */
  double solve_rtol;        /* relative residual per spatial solve (0 -> 1e-13 FP64, 1e-10 mixed) */
  int pcg_maxit;            /* PCG iteration cap per solve (0 -> 200) */
  /* tuning (0 -> autotuned or default) */
  int team_ctas;            /* CTAs per thread-block cluster working on one column group */
  int team_cols;            /* columns per cluster: 1, 2, 4, 8 or 16 */
  int mg_nu;                /* Jacobi sweeps before and after the coarse correction (finest level) */
  double inner_rtol;        /* LRP_MIXED: FP32 inner relative tolerance (0 -> 1e-4) */
  int coarse_items;         /* multigrid levels with at most this many points x columns are
                               solved by every CTA of a team in shared memory (0 -> 1024) */
  int kernel_variant;       /* 0 auto; 1 the generic sweep kernel; 2 the band kernel (2D, kappa = 1,
                               LRP_MIXED, team_cols 1: each CTA keeps its band of rows of the finest
                               grid in shared memory, every coarse level in every CTA); 3 the band
                               kernel with the first coarse level split across the cluster like the
                               finest one (each CTA owning >= 2 of its rows); LRP_EINVAL if the
                               requested variant does not apply. Auto takes 3, else 2, else 1. */
  int mg_nu_coarse;         /* Jacobi sweeps before and after on the coarser levels of the band
                               kernel (0 -> mg_nu) */
  int prior_kind;           /* LRP_PRIOR_LAPLACE: Gamma_prior = (I + prior_alpha L0)^-2 (the default);
                               LRP_PRIOR_IDENTITY: Gamma_prior = prior_gamma I (the paper's
                               experiments, Sec. 6.1: Gamma_prior = 10 I) */
  double prior_gamma;       /* LRP_PRIOR_IDENTITY: the prior variance (> 0) */
  int pde;                  /* LRP_PDE_HEAT (L = -div(kappa grad)) or LRP_PDE_CONVDIFF (L = -conv_nu
                               Laplace + wind . grad with first-order upwind differences: the
                               convection-diffusion operator of Sec. 6.2; not symmetric, so every
                               implicit-Euler step is solved by Jacobi-preconditioned BiCGStab and
                               the adjoint sweep solves with (I + tau L)^T; LRP_FP64 only, kappa NULL) */
  double conv_nu;           /* LRP_PDE_CONVDIFF: diffusivity nu (>= 0) */
  double wind[3];           /* LRP_PDE_CONVDIFF: constant wind vector w (dim entries used) */
  int mg_levels;            /* multigrid levels of the time-step operator I + tau L: 0 = down to one
                               node; 3..L cuts the hierarchy there, and the coarsest kept level is
                               smoothed by 2 mg_nu_coarse damped Jacobi sweeps (a fixed symmetric
                               polynomial, so PCG stays valid) instead of solved exactly. On the
                               coarse levels of a time step the operator is close to the identity
                               (c/h^2 small), so the deep levels cost latency and add little. The
                               prior operator always keeps the whole hierarchy. 0 -> autotuned or 0 */
  int als_rank;             /* LRP_ALS_SOLVES: rank of the alternating solves (0 -> 16; capped at
                               min(64, nt, nx)) */
  int als_sweeps;           /* LRP_ALS_SOLVES: sweeps per solve (0 -> 3) */
  double als_tol;           /* LRP_ALS_SOLVES: stop a solve once its relative residual is <= als_tol
                               (0 -> always als_sweeps sweeps) */
  double als_prec_rtol;     /* alternating solves (lrp_als_solve, LRP_ALS_SOLVES): > 0 -> the spatial
                               solves that apply the space step's preconditioner run to this relative
                               residual (never below solve_rtol); 0 -> als_prec_its iterations each */
  int als_prec_its;         /* alternating solves: multigrid-preconditioned CG iterations per
                               preconditioner solve, from zero (LRP_MIXED: one FP32 inner solve and one
                               FP64 residual update), when als_prec_rtol is 0 (0 -> 2) */
  int mg_bf16;              /* LRP_MIXED: 1 -> the multigrid smoother iterates and coarse right-hand sides
                               of the levels held in global memory are stored in BF16 (rounded to
                               nearest even; the arithmetic stays FP32, the PCG vectors FP32, the
                               refinement FP64). Runs the generic sweep kernel (the 2D band kernel keeps
                               its vectors in shared memory in FP32 and has no BF16 form). The V-cycle
                               is then not exactly the same operator in every application; the FP64
                               refinement keeps the result at the solve tolerance, and a solve that
                               does not converge returns LRP_ENOCONV. 0 -> FP32 storage */
} lrp_problem_desc;

typedef struct {
  int n_solves;             /* spatial solves performed (per column) */
  int pcg_iters_max;        /* largest PCG iteration count of any solve */
  double pcg_iters_mean;    /* mean PCG iterations per solve */
  int refine_max;           /* LRP_MIXED: largest number of refinement sweeps of any solve */
  double max_rel_residual;  /* largest final relative residual of any solve */
  int time_rank_max;        /* largest time rank of the kept trajectory factors (0 if not kept) */
  double time_trunc_err;    /* largest certified relative truncation error bound of the factors */
  double ms;                /* wall time of the call */
  int adj_rank_max;         /* LRP_LOWRANK_SOURCE: largest time rank of the adjoint trajectory factors */
  double adj_trunc_err;     /* LRP_LOWRANK_SOURCE: their largest certified relative truncation error */
} lrp_apply_stats;

typedef struct {
  int n_iter;               /* Lanczos block steps */
  int n_matvec;             /* Htilde applications to single vectors */
  int k_converged;          /* Ritz pairs meeting the residual test */
  double max_ritz_resid;    /* max over the returned pairs of ||Htilde v - theta v|| / theta_1 */
  double ms;                /* wall time */
  double ms_apply;          /* of which Hessian applications */
} lrp_lanczos_stats;

/* query kinds */
enum { LRP_Q_MEAN = 1, LRP_Q_VARIANCE = 2, LRP_Q_SAMPLES = 4 };

typedef struct {
  unsigned kind;            /* mask of LRP_Q_* */
  const double* y_obs;      /* n_data observations (host or device); needed for MEAN and SAMPLES */
  double sigma;             /* noise level of this request; 0 -> the problem's sigma */
  int n_points;             /* VARIANCE: number of query nodes */
  const int* points;        /* VARIANCE: flat node indices (host or device) */
  int n_samples;            /* SAMPLES: number of samples */
  const double* xi;         /* SAMPLES: nx*n_samples standard normals, column-major (host or device) */
} lrp_query;

typedef struct {
  double* mean;             /* nx (host or device), written for MEAN and SAMPLES requests if non-NULL */
  double* variance;         /* n_points (host or device) */
  double* samples;          /* nx*n_samples column-major (host or device) */
  double ms;                /* wall time */
} lrp_query_result;

/* ---------------------------------------------------------------------------
 * Problem setup (Sec. 6: grid, operators, sensors, prior).
 * Builds the multigrid hierarchy of I + tau*L and I + alpha*L0, the sensor
 * interpolation lists and their transpose, and uploads them. cuda_stream: a
 * cudaStream_t (NULL = the default stream); the current device at this call
 * becomes the problem's device. On success *out owns all device memory of
 * the problem until lrp_problem_destroy.
 * Errors: LRP_EINVAL (bad sizes: n not 2^L-1, dim not 2/3, nt < 1, sensor
 * outside (0,1)^dim, ...), LRP_ENONFINITE, LRP_ENOMEM, LRP_ECUDA. */
lrp_status lrp_setup_problem(const lrp_problem_desc* desc, void* cuda_stream, lrp_problem** out);
void lrp_problem_destroy(lrp_problem* p);

/* Basic sizes of a problem: nx, n_obs, number of observed steps, n_data. */
lrp_status lrp_problem_sizes(const lrp_problem* p, int* nx, int* n_obs, int* n_steps, int* n_data);

/* ---------------------------------------------------------------------------
 * Y = Htilde X (Sec. 2 Eq. (prior_pre); Sec. 6.1 Eq. (misfit)) for nvec
 * columns: prior half-apply, forward implicit-Euler sweep with the fused
 * observation and 1/sigma^2 weighting, adjoint sweep with the fused
 * B^T source, prior half-apply. With LRP_MISFIT_ONLY: Y = H_mis X.
 * X: nx x nvec (ldx >= nx), Y: nx x nvec (ldy >= nx); X and Y may not overlap.
 * st may be NULL. */
lrp_status lrp_hessian_apply(lrp_problem* p, int nvec, const double* X, int ldx,
                             double* Y, int ldy, unsigned flags, lrp_apply_stats* st);

/* Allocation-free variant of lrp_hessian_apply (the paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory while they run, e.g. a process whose device memory is reserved up
 * front by another allocator, or a loop where a cudaMalloc would synchronise
 * the device). Computes Y = Htilde X exactly as lrp_hessian_apply does, but
 * the solver workspace is a fixed 64 MiB array in device memory that the
 * library holds on every GPU that loads it until the process exits; the call
 * makes no cudaMalloc or cudaFree. X and Y must be device arrays (host arrays
 * are rejected: staging them would allocate). A call whose workspace would
 * exceed 64 MiB (it grows with nvec, the grid and the number of observations)
 * returns LRP_EINVAL with the required size in lrp_last_error(); split the
 * columns into smaller calls. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the one
 * array, so calls that overlap on the GPU (different threads or streams,
 * any problems) race: serialise them. The array keeps the previous call's
 * contents; nothing in the computation reads it before writing it. */
lrp_status lrp_hessian_apply_noalloc(lrp_problem* p, int nvec, const double* X, int ldx,
                                     double* Y, int ldy, lrp_apply_stats* st);

/* Autotuner for blocks of nvec columns. Stage 1 times, for each cluster size
 * (1..8, 12, 16 CTAs), CTA size (256 or 512 threads) and columns per cluster
 * (1, 2), with or without running in several waves for clusters of 8 or
 * more, the prior solve and the first `steps` forward implicit-Euler steps
 * (0 -> 16); stage 2 varies the smoothing sweeps (finest and coarse levels,
 * 1 or 2 each) and (LRP_MIXED) the inner
 * tolerance on the two best shapes; stage 3 times one whole Hessian apply for
 * the five best; stage 4 times the stage-1 screen for one column at larger
 * cluster sizes (team_ctas_narrow of lrp_tuning). The winner stays in the
 * problem handle for later calls.
 * All candidates iterate to the same tolerances. *best_ms (may be NULL)
 * receives the winner's Hessian-apply time. Allocates two nx x nvec blocks
 * for the duration of the call. No counterpart in the paper. */
lrp_status lrp_autotune(lrp_problem* p, int nvec, int steps, double* best_ms);

/* D = F U (no noise weighting): forward sweep and observation.
 * U: nx x nvec, D: n_data x nvec. */
lrp_status lrp_forward_observe(lrp_problem* p, int nvec, const double* U, int ldu,
                               double* D, int ldd, lrp_apply_stats* st);

/* U = F^T D: adjoint sweep (backward recursion with the B^T source).
 * D: n_data x nvec, U: nx x nvec. */
lrp_status lrp_adjoint(lrp_problem* p, int nvec, const double* D, int ldd,
                       double* U, int ldu, lrp_apply_stats* st);

/* Y = Gamma_prior^{1/2} X = (I + alpha L0)^{-1} X. */
lrp_status lrp_prior_half(lrp_problem* p, int nvec, const double* X, int ldx,
                          double* Y, int ldy, lrp_apply_stats* st);

/* Forward trajectory of each column of U in low-rank-in-time form (Sec. 3):
 * Y = [y_1 .. y_nt] ~ W V^T with W: nx x r and V: nt x r (column j's factors
 * at W + j*nx*rmax and V + j*nt*rmax, column-major, ld nx and nt).
 * ranks[j] receives r for column j (<= time_rank_max). W, V must hold
 * nvec*nx*time_rank_max and nvec*nt*time_rank_max doubles. */
lrp_status lrp_trajectory_factors(lrp_problem* p, int nvec, const double* U, int ldu,
                                  double* W, double* V, int* ranks, lrp_apply_stats* st);

/* ---------------------------------------------------------------------------
 * Low-rank posterior (Sec. 4 Algorithm 1, as block Lanczos with full
 * reorthogonalisation on the symmetric Htilde; Sec. 2 SMW form).
 * Computes the k leading eigenpairs of Htilde with blocks of `block`
 * columns (1..64) until every returned Ritz pair has
 * ||Htilde v - theta v|| <= eig_tol * theta_1 (eig_tol 0 -> 1e-6), or the
 * Krylov space reaches max_basis columns (0 -> min(nx, 4k+2*block)).
 * eig_threshold > 0 keeps only eigenvalues >= eig_threshold (the paper's
 * threshold epsilon, Sec. 6.1) among the k, and the iteration stops as soon
 * as every Ritz value above the threshold meets the residual test and some
 * Ritz value lies below it (k is then a cap). start: optional nx x block start block
 * (host or device), NULL -> a fixed pseudo-random block.
 * The posterior keeps V_k, G = R^{-1} V_k and lambda on the device.
 * Returns LRP_ENOCONV (with a usable posterior) if the basis cap is hit or a
 * solve of a Hessian apply missed its tolerance within pcg_maxit. */
lrp_status lrp_lowrank_posterior(lrp_problem* p, int k, int block, double eig_tol,
                                 double eig_threshold, int max_basis, const double* start,
                                 lrp_posterior** out, lrp_lanczos_stats* st);
void lrp_posterior_destroy(lrp_posterior* post);

/* Batched low-rank posterior (no counterpart in the paper: the batching
 * form). Runs the block Lanczos of lrp_lowrank_posterior (eig_threshold 0,
 * default basis cap, pseudo-random start) on `count` independent problems of
 * any sizes at once: every block step of every problem not yet converged is
 * enqueued on a stream of that problem's own (created for the call; the
 * problem's stream is drained first and restored at the end) and, with
 * use_graph, the whole step is captured into one CUDA graph and launched
 * once (otherwise launched directly); problems drop out as they converge.
 * The problems must be distinct and on one device. outs[i] and stats[i]
 * (stats may be NULL) as in
 * lrp_lowrank_posterior; *bst (may be NULL) gets totals. Each result equals
 * that of lrp_lowrank_posterior on the same problem (same kernels in the
 * same order on its stream). max_steps > 0 stops after that many block
 * steps (a bounded sample: the posteriors then hold the current Ritz pairs).
 * Returns LRP_ENOCONV if any problem stopped before converging (its
 * posterior is still usable). */
typedef struct {
  int steps;             /* block steps (graph launches with use_graph) */
  long long graph_nodes; /* nodes of all step graphs together */
  long long n_matvec;    /* Htilde applications over all problems */
  double ms_steps;       /* wall time of the steps */
  double ms;             /* wall time of the call */
} lrp_batch_stats;
lrp_status lrp_batch_lowrank_posterior(lrp_problem* const* probs, int count, int k, int block, double eig_tol,
                                       int use_graph, int max_steps, lrp_posterior** outs,
                                       lrp_lanczos_stats* stats, lrp_batch_stats* bst);

/* ---------------------------------------------------------------------------
 * Arnoldi process of Sec. 4 Algorithm 1, as printed: single vectors; step j
 * applies the operator to v_j, orthogonalises the result against v_1 .. v_j
 * one at a time (modified Gram-Schmidt; the coefficients are column j of the
 * Hessenberg matrix H), H_{j+1,j} = its norm, v_{j+1} = it / H_{j+1,j}.
 * The operator is Htilde (flags 0), H_mis (LRP_MISFIT_ONLY) or the truncated
 * product of Algorithm 1 (LRP_LOWRANK_SOURCE, see lrp_hessian_apply), which
 * is not exactly symmetric: hence Arnoldi rather than Lanczos (Sec. 4).
 * Ritz values: the eigenvalues of the leading m x m block of H
 * (lrp_hessenberg_eig), possibly complex. Ritz vectors of the real ones by
 * back substitution on the Schur factor; residual estimate
 * |H_{m+1,m}| |e_m^T y| (||y|| = 1).
 * Stops after max_steps steps, on an invariant subspace, or once the wanted
 * Ritz values all have residual estimates <= eig_tol |theta_1| (eig_tol 0 ->
 * 1e-6): with eig_threshold > 0 (the threshold epsilon of Sec. 6.1) the
 * wanted ones are those with real part >= eig_threshold, and some Ritz value
 * must lie below it; otherwise the k leading ones. A complex Ritz value
 * among the wanted ones keeps the run going. The test runs after every step
 * up to 32 steps, then every floor(m/16)-th step; with a threshold, not
 * before step 8.
 * Outputs (each may be NULL; host or device):
 *   theta_re, theta_im [max_steps]: the m Ritz values of the last H_m by
 *     decreasing real part;
 *   H [(max_steps+1) x max_steps], column-major, ld max_steps+1 (zero beyond
 *     column m);
 *   ranks_y, ranks_q [max_steps] (host): with LRP_LOWRANK_SOURCE, the time
 *     ranks of the state and adjoint trajectory factors at each step
 *     (0 otherwise);
 *   out: a posterior from the wanted real Ritz pairs with theta > 0, the
 *     Ritz vectors orthonormalised (block CGS2) in order of decreasing theta
 *     (not with LRP_MISFIT_ONLY).
 * start: nx vector (host or device) or NULL (a fixed pseudo-random vector).
 * Returns LRP_ENOCONV (outputs written) if max_steps is reached first or a
 * solve missed its tolerance; LRP_EINVAL for max_steps outside
 * 1..min(nx, 2048), k < 1 without a threshold, or LRP_KEEP_TRAJ_FACTORS. */
typedef struct {
  int n_steps;           /* Arnoldi steps m (Hessian applications) */
  int k_converged;       /* wanted real Ritz values that met the test (0 if it failed) */
  int n_complex;         /* Ritz values of H_m with nonzero imaginary part */
  double max_imag;       /* largest |Im theta| / |theta_1| */
  double hess_asym;      /* ||H_m - H_m^T||_F / ||H_m||_F */
  double max_ritz_resid; /* largest residual estimate of the wanted pairs / |theta_1| */
  int time_rank_max;     /* LRP_LOWRANK_SOURCE: largest state-trajectory rank over the steps */
  int adj_rank_max;      /* LRP_LOWRANK_SOURCE: largest adjoint-trajectory rank over the steps */
  double ms;             /* wall time of the call */
  double ms_apply;       /* wall time of the operator applications */
} lrp_arnoldi_stats;
lrp_status lrp_arnoldi(lrp_problem* p, int max_steps, int k, double eig_tol, double eig_threshold,
                       unsigned flags, const double* start, double* theta_re, double* theta_im,
                       double* H, int* ranks_y, int* ranks_q, lrp_posterior** out,
                       lrp_arnoldi_stats* st);

/* ---------------------------------------------------------------------------
 * A space-time parameter (Sec. 4: a distributed source u(x, t) as the
 * uncertain quantity, the case the low-rank Krylov vectors are made for):
 * y_t + L y = u, y(0) = 0, implicit Euler (I + tau L) y_n = y_{n-1} + tau u_n;
 * U = [u_1 .. u_nt] (nx x nt). Observations, noise and the spatial prior as
 * for the initial condition; Gamma_prior = I_nt (x) Gamma_x. Then
 * F^T d = tau [q_1 .. q_nt] (the adjoint recursion's whole trajectory) and
 * Htilde U = Gamma_x^{1/2} F^T F Gamma_x^{1/2} U / sigma^2.
 * Low-rank vectors U = W V^T (W: nx x r, V: nt x r, column-major).
 *
 * lrp_st_hessian_apply: Htilde (W V^T) as factors: the prior factor on the r
 * columns of W, one forward sweep with the factored source added before each
 * step's solve and the fused observation, the adjoint sweep storing its
 * trajectory, the streaming truncation of that trajectory (time_trunc_tol,
 * time_rank_max, time_chunk), the prior factor on its space factor. Wout
 * (nx x time_rank_max, ld nx) and Vout (nt x time_rank_max, ld nt) receive
 * the *r_out result columns; host or device arrays. Stats: adj_rank_max and
 * adj_trunc_err describe the truncation. */
lrp_status lrp_st_hessian_apply(lrp_problem* p, int r, const double* W, int ldw, const double* V, int ldv,
                                double* Wout, double* Vout, int* r_out, lrp_apply_stats* st);

/* Algorithm 1 on low-rank space-time vectors (Sec. 4, Eq. (lanczos1)-
 * (lanczos2)): w = Htilde v_j (lrp_st_hessian_apply); for i = 1..j:
 * h_ij = <w, v_i> (trace of the factor products), w <- round(w - h_ij v_i)
 * (factors concatenated, then rounded: thin QR of both factors, SVD of the
 * small core, smallest rank whose discarded Frobenius tail is at most
 * time_trunc_tol ||w||_F, capped at time_rank_max); h_{j+1,j} = ||w||_F,
 * v_{j+1} = w / h_{j+1,j}. Ritz values, the stopping rule, theta_re/theta_im
 * and H as in lrp_arnoldi. Start: r0 factor columns W0 (nx x r0), V0
 * (nt x r0) (host or device; rounded and normalised), or r0 = 0 for a fixed
 * pseudo-random rank-1 start. ranks [max_steps] (host, may be NULL): the rank
 * of v_{j+1}. Stats: time_rank_max = the largest rank of a Krylov vector,
 * adj_rank_max = the largest rank of a product Htilde v_j. Needs
 * time_rank_max <= 56; LRP_EINVAL otherwise. */
lrp_status lrp_st_arnoldi(lrp_problem* p, int max_steps, int k, double eig_tol, double eig_threshold, int r0,
                          const double* W0, const double* V0, double* theta_re, double* theta_im, double* H,
                          int* ranks, lrp_arnoldi_stats* st);

/* ---------------------------------------------------------------------------
 * Alternating low-rank solver of the space-time system (Sec. 6.1: the
 * all-at-once system Eq. (st_pde), solved in low-rank form by alternating
 * Galerkin projections, Eq. (amen_1) and Eq. (amen_2), the first by a Krylov
 * method with the preconditioner of Eq. (pre_1)). With A = I + tau L the
 * problem's time-step operator, the forward system (transpose = 0) is
 *   A y_n = y_{n-1} + f_n, n = 1..nt, y_0 = 0, i.e. A Y - Y S^T = F,
 * and the adjoint system (transpose = 1) is
 *   A^T q_n = q_{n+1} + f_n, n = nt..1, q_{nt+1} = 0,
 * with Y = [y_1 .. y_nt] (nx x nt) and the source F = Wf Vf^T given as
 * factors Wf (nx x rf, ld ldwf), Vf (nt x rf, ld ldvf; row n-1 = step n).
 * An initial condition u is the source u e_1^T (rf = 1, Vf = e_1).
 * The solution is returned as Y ~ W V^T, W: nx x r (ld ldw), V: nt x r
 * (ld ldv, orthonormal columns, row n-1 = step n). One sweep is
 *  - the space step: V fixed, the Galerkin projection onto span(V) in time,
 *    A W - W T = F V with T = V^T S^T V (T[i, j] = sum_n V[n-1, i] V[n, j];
 *    the adjoint uses the same with time reversed), an nx r system solved by
 *    flexible GMRES to a relative residual of max(10 solve_rtol, 1e-12),
 *    right-preconditioned by blockdiag(A - T_jj I), each block applied by
 *    als_prec_its (0 -> 2) multigrid-preconditioned CG iterations from zero
 *    (the problem's solver and precision), or a solve to als_prec_rtol if
 *    that is > 0 (the GMRES is flexible: the preconditioner may change from
 *    one iteration to the next);
 *  - the time step: W orthonormalised to Q, the Galerkin projection onto
 *    span(Q) in space, Q^T A Q z_n - z_{n-1} = Q^T f_n (r x r, direct),
 *    then V = the orthonormalised Z and W = Q R_Z^T.
 * V0 (nt x r, ld ldv0): the start (orthonormalised first). The rank is fixed
 * (AMEn's residual-based enrichment is not done); basis directions that
 * become numerically dependent are dropped (zero columns). Runs `sweeps`
 * sweeps, or stops after the first whose relative residual
 * ||A Y - Y S^T - F||_F / ||F||_F (A^T Q - Q S - F for the adjoint) is
 * <= tol (tol > 0). res (host, may be NULL): that residual after each sweep
 * (0 past the last one taken). All arrays host or device.
 * Errors: LRP_EINVAL for r outside 1..min(64, nt, nx), rf outside 0..64,
 * sweeps < 1, short leading dimensions; LRP_ENOCONV (outputs written) if a
 * GMRES space step or a spatial solve missed its tolerance. */
typedef struct {
  int sweeps;           /* sweeps taken */
  int gmres_iters;      /* GMRES iterations over all space steps */
  int gmres_iters_max;  /* largest count of one space step */
  int precond_solves;   /* spatial solves of the preconditioner, per column */
  double residual;      /* relative residual after the last sweep */
  double ms;            /* wall time */
  double ms_space;      /* of which space steps */
  double ms_time;       /* of which time steps and residuals */
} lrp_als_stats;
lrp_status lrp_als_solve(lrp_problem* p, int transpose, int rf, const double* Wf, int ldwf, const double* Vf,
                         int ldvf, int r, const double* V0, int ldv0, int sweeps, double tol, double* W, int ldw,
                         double* V, int ldv, double* res, lrp_als_stats* st);

/* Eigenvalues of a real upper Hessenberg matrix by the Francis double-shift
 * QR iteration (the eigensolver of lrp_arnoldi; Golub & Van Loan Sec. 7.5),
 * on the current device, synchronously. H: m x m column-major (ld ldh >= m),
 * host or device; entries below the first subdiagonal are ignored.
 * wr, wi (host, m): the eigenvalues in the order of the diagonal of the real
 * Schur form (a complex pair adjacent, positive imaginary part first).
 * T, Z (each may be NULL; host or device, m x m, ld m): the quasi-upper-
 * triangular Schur factor and the orthogonal Schur vectors, H = Z T Z^T.
 * LRP_ENOCONV if the iteration used 30 m double-shift steps without
 * finishing (outputs as far as reached); LRP_EINVAL for m outside 1..4096. */
lrp_status lrp_hessenberg_eig(int m, const double* H, int ldh, double* wr, double* wi,
                              double* T, double* Z);

/* Copies the r <= k eigenvalues (decreasing) and optionally the eigenvectors
 * (nx x r column-major, ld ldv) out of a posterior. *r receives the count. */
lrp_status lrp_posterior_eigs(const lrp_posterior* post, int* r, double* lambda,
                              double* V, int ldv);

/* Posterior queries (Sec. 2: posterior mean = MAP point, pointwise variance
 * diag(Gamma_post), samples u_mean + R^{-1}(I + V Lambda V^T)^{-1/2} xi),
 * with the eigenvalues rescaled to the request's sigma
 * (lambda(sigma) = lambda(sigma0) sigma0^2 / sigma^2). If a solve of the
 * query misses its tolerance within pcg_maxit, the outputs are still written
 * and the call returns LRP_ENOCONV. */
lrp_status lrp_posterior_query(lrp_posterior* post, const lrp_query* q, lrp_query_result* r);

/* Checkpoint: write / read the posterior factors and a hash of the problem.
 * Save writes `path`.tmp and renames it to `path` when complete (a failed
 * save leaves no partial file). Load rejects (LRP_EINVAL) a file of another
 * problem, a header whose rank exceeds nx and a truncated file. */
lrp_status lrp_posterior_save(const lrp_posterior* post, const char* path);
lrp_status lrp_posterior_load(lrp_problem* p, const char* path, lrp_posterior** out);

/* Message of the last error on this host thread (never NULL). */
const char* lrp_last_error(void);

/* Library version string. */
const char* lrp_version(void);

/* Sweep-kernel ledger. mode 1: reset and start recording, for every launch
 * of a sweep kernel on this problem, its CUDA-event duration and its
 * algorithmic bytes (passes over the fine-level vectors implied by the
 * solver's iteration counts); mode 0: reset and stop; mode -1: read only.
 * kernel selects what is returned: 0 all sweep launches, 1 the generic team
 * kernel, 2 the 2D band kernel. The accumulated values before the reset are
 * returned in *ms, *launches and *algo_bytes (each may be NULL). kernel 3
 * (generic) and 4 (band) select the launches that run a whole Hessian apply
 * (prior solve, forward sweep, adjoint sweep, prior solve), e.g. the block
 * applies of the Lanczos iteration. */
lrp_status lrp_sweep_profile(lrp_problem* p, int mode, int kernel, double* ms, unsigned long long* launches,
                             double* algo_bytes);

/* Current launch/multigrid settings of a problem (set by lrp_setup_problem's
 * descriptor or chosen by lrp_autotune) and what the last sweep launch used:
 * last_kernel 1 = generic team kernel, 2 = 2D band kernel, 0 = none yet;
 * last_team_ctas = the cluster size it ran with (the requested size is
 * halved until every team is resident). No counterpart in the paper. */
typedef struct lrp_tuning {
  int team_ctas, team_cols, mg_nu, mg_nu_coarse;
  double inner_rtol;
  int last_kernel, last_team_ctas;
  int threads;  /* threads per CTA */
  int waves;    /* 1: clusters of the requested size even if they run in several waves */
  int team_ctas_narrow; /* cluster size for launches with few columns, used when all of their
                           clusters fit on the GPU at once at that size; 0 = team_ctas */
  int mg_levels;        /* time-step operator's multigrid levels (0 = all; see lrp_problem_desc) */
} lrp_tuning;
lrp_status lrp_problem_tuning(const lrp_problem* p, lrp_tuning* out);
/* Sets a problem's launch shape and multigrid settings from t (team_ctas,
 * team_cols, mg_nu, mg_nu_coarse, inner_rtol, threads 256 or 512, waves,
 * team_ctas_narrow 0..16, mg_levels 0 or 3..levels; the
 * last_* fields are ignored), e.g. to reuse one autotuned setting for
 * problems of the same size. LRP_EINVAL on values out of range. */
lrp_status lrp_set_tuning(lrp_problem* p, const lrp_tuning* t);

/* ---------------------------------------------------------------------------
 * Posterior-query server (no counterpart in the paper; it serves the
 * low-rank posterior of Sec. 2 to a stream of requests).
 *
 * A model is a problem with its rank-k factors, computed by
 * lrp_lowrank_posterior when the model is added (or read from a checkpoint).
 * Requests (lrp_query: mean, pointwise variance, samples; each with its own
 * data and noise level, the stored eigenvalues being rescaled by
 * sigma0^2/sigma^2) are queued by lrp_server_submit and served by `slots`
 * worker threads, each with its own CUDA stream: a free worker takes the
 * model of the oldest pending request and serves up to max_batch of its
 * pending requests in one batch (one adjoint sweep and one prior sweep over
 * all the batch's columns). Requests arriving while batches run join the
 * next batch a worker forms, and batches overlap on the device.
 * Memory: factors, per-worker problem handles and batch scratch are counted
 * against hbm_budget; a model whose factors are not on the device is admitted
 * by evicting least recently used idle models (factors kept in pinned host
 * memory); a request whose model cannot fit even alone fails with
 * LRP_EBUDGET. A result does not depend on the batch it was served in beyond
 * the solver tolerance. The device current at lrp_server_create is used.
 * Thread safety: submit, wait and info may be called from any threads. */
typedef struct lrp_server lrp_server;

typedef struct {
  size_t hbm_budget;  /* device bytes the server may hold; 0 -> 16 GiB */
  int slots;          /* worker threads / streams (batches in flight); 0 -> 4, <= 64 */
  int max_batch;      /* requests per batch; 0 -> 16, <= 256 */
  int max_samples;    /* largest n_samples of a request; 0 -> 8, <= 64 */
  int max_points;     /* largest n_points of a request; 0 -> 1024 */
  int autotune;       /* 1: run lrp_autotune for max_batch columns on every model as it is added */
} lrp_server_config;

typedef struct {
  double t_submit_ms;  /* milliseconds since lrp_server_create */
  double t_start_ms;   /* its batch was formed */
  double t_done_ms;    /* its results were on the host */
  int batch;           /* requests in that batch */
  int slot;            /* worker that served it */
  int admitted;        /* 1 if the model's factors were brought onto the device for this batch */
} lrp_request_stats;

typedef struct {
  size_t device_bytes;  /* accounted device bytes held now */
  int models, resident;
  long long admissions, evictions, batches, served, pending;
} lrp_server_stats;

lrp_status lrp_server_create(const lrp_server_config* cfg, lrp_server** out);
/* Adds a model: sets the problem up from d, computes its rank-k factors
 * (block, eig_tol as in lrp_lowrank_posterior) or, if factors_path names an
 * existing checkpoint of the same problem, reads them (a non-NULL path that
 * does not exist yet receives the computed factors). *model receives its id. */
lrp_status lrp_server_add_model(lrp_server* s, const lrp_problem_desc* d, int k, int block, double eig_tol,
                                const char* factors_path, int* model, lrp_lanczos_stats* st);
/* Queues a request (its inputs are copied; q's arrays may be reused at once). */
lrp_status lrp_server_submit(lrp_server* s, int model, const lrp_query* q, unsigned long long* ticket);
/* Waits for a request (timeout_s <= 0: no limit; LRP_ETIMEOUT otherwise),
 * copies its results into r's HOST buffers (each may be NULL) and releases
 * the ticket. Returns the request's own status; LRP_ENOCONV means a solve of
 * the batch the request was served in missed its tolerance within pcg_maxit
 * (every request of that batch gets it), and the results are still copied. */
lrp_status lrp_server_wait(lrp_server* s, unsigned long long ticket, double timeout_s, lrp_query_result* r,
                           lrp_request_stats* st);
lrp_status lrp_server_info(lrp_server* s, lrp_server_stats* out);
/* Finishes the queued requests, stops the workers, frees everything. */
void lrp_server_destroy(lrp_server* s);

/* Diagnostics: number of CUDA kernels this library has launched in this
 * process so far (all problems, all threads). */
unsigned long long lrp_kernel_launches(void);

/* Peak rates of the current device measured with the library's own kernels
 * (no counterpart in the paper; the denominators of the roofline figures of
 * kernels not bound by HBM bandwidth): shared-memory bandwidth over all SMs
 * (16-byte loads and stores, conflict-free), FP64 and FP32 FMA throughput
 * (8 independent chains per thread). Each is the best of three timed
 * launches; the call takes well under a second. */
typedef struct {
  double smem_gbs;         /* shared-memory bytes loaded + stored per second / 1e9 */
  double fp64_fma_tflops;  /* 2 x FP64 FMAs per second / 1e12 */
  double fp32_fma_tflops;  /* 2 x FP32 FMAs per second / 1e12 */
  int sm_count;
  double clock_mhz;        /* the device's nominal SM clock */
} lrp_device_peaks;
lrp_status lrp_measure_device_peaks(lrp_device_peaks* out);

/* Test hook (failure injection on the host, no counterpart in the paper):
 * after `after` further successful device allocations by this library, the
 * next one fails as if the device were out of memory (once, in any thread);
 * after < 0 disarms it. The call that meets the failure returns LRP_ENOMEM
 * and releases what it had allocated. */
void lrp_debug_fail_alloc(long long after);

#ifdef __cplusplus
}
#endif
#endif /* LRP_H */
