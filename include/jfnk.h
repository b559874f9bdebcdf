/*
 * jfnk.h -- C ABI of libjfnk.so: a GB300 (sm_103a) implementation of the
 * Jacobian-free Newton-Krylov method with a Jacobian-free geometric multigrid
 * preconditioner of Kothari, Kopanicakova & Krause, "A Multigrid
 * Preconditioner for Jacobian-free Newton-Krylov Methods" (arXiv:2103.13890).
 *
 * The problem statement (Sec. 1): find x with F(x) = 0, using only the
 * actions F(x) and J(x)v ~ (F(x + eps v) - F(x)) / eps, preconditioned by the
 * V-cycle MG(x, F(x), b, l) of Algorithm 1.
 *
 * Conventions shared by every entry point
 *   - Vectors are FULL node grids of a uniform structured grid on the unit
 *     square / cube with n elements per direction: (n+1)^2 or (n+1)^3 values,
 *     x fastest, then y, then z, densely packed.  Boundary entries hold the
 *     Dirichlet data for an iterate and are zero for residuals, corrections and
 *     Krylov vectors (results always have zero boundary entries).
 *   - Every vector pointer is a DEVICE pointer owned by the caller.  The
 *     library never allocates device memory: its scratch lives in a workspace
 *     the caller allocates (jfnk_workspace_size / jfnk_set_workspace).
 *   - Calls are asynchronous on the given CUDA stream (may be 0), except
 *     jfnk_solve, jfnk_solve_batched and jfnk_adjoint_solve, which synchronise
 *     the stream to test convergence on the host.
 *   - Calls on one problem must not run concurrently (they share its
 *     workspace).  Distinct problems are independent.
 *   - Errors are returned as jfnk_status, never thrown; jfnk_last_error()
 *     gives a message for the calling thread.  A CUDA error is reported as
 *     JFNK_ERR_CUDA.  The library never traps on the device.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JFNK_OK = 0,
    JFNK_ERR_INVALID_ARG = 1,   /* bad sizes, kinds, levels, null pointers */
    JFNK_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    JFNK_ERR_NONFINITE = 3,     /* NaN/Inf in a norm, eps or Hessenberg entry */
    JFNK_ERR_NOT_CONVERGED = 4, /* Newton iteration limit reached */
    JFNK_ERR_BREAKDOWN = 5,     /* Krylov breakdown with a nonzero residual */
    JFNK_ERR_LINESEARCH = 6,    /* backtracking found no sufficient decrease */
    JFNK_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
    JFNK_ERR_NOT_IMPLEMENTED = 8,
    JFNK_ERR_WORKSPACE = 9      /* workspace missing or too small */
} jfnk_status;

typedef enum { JFNK_F32 = 0, JFNK_F64 = 1 } jfnk_dtype;

/* Problems (Sec. 3, and nonlinear diffusion), Q1 elements, 2^d Gauss points:
 *  JFNK_BRATU2D  F_i = int grad u.grad phi_i - lambda exp(u) phi_i   (Sec. 3, Bratu)
 *  JFNK_ND3D     F_i = int (1+u^2) grad u.grad phi_i - int f phi_i, f manufactured
 *                from u* = sin(pi x) sin(pi y) sin(pi z)
 *  JFNK_NDK3D    F_i = sum_e kappa_e int_e (1+u^2) grad u.grad phi_i - int phi_i
 *  JFNK_MINSURF2D F_i = int grad u.grad phi_i / sqrt(1 + |grad u|^2)  (Sec. 3, minimal
 *                surface; its Dirichlet data x(1-x) / 0 are the boundary entries of u)
 *  JFNK_BEAM3D   Neo-Hookean beam (Sec. 3, hyperelasticity): F_a = int P(F) grad phi_a,
 *                P = mu F + (lam ln J - mu) F^-T, E = 10, nu = 0.3, on (0,10)x(0,1)^2 with
 *                10 n_elem x n_elem x n_elem cube elements; vectors hold 3 displacement
 *                components per node (component fastest: shape (n+1, n+1, 10n+1, 3));
 *                Dirichlet data (u = 0 at x = 0, the end rotation at x = 10) are the
 *                entries of u on those faces; the other faces are free (their nodes are
 *                unknowns).  n_elem / 2^(levels-1) >= 1. */
typedef enum { JFNK_BRATU2D = 0, JFNK_ND3D = 1, JFNK_NDK3D = 2, JFNK_MINSURF2D = 3, JFNK_BEAM3D = 4 } jfnk_kind;

/* Finite-difference step (Sec. 1):
 *  JFNK_EPS_PAPER  eps = (1/(n ||v||_2)) sum_i sqrt(eps_p)(1+|x_i|), eps_p = 2^-52,
 *                  n = interior unknowns
 *  JFNK_EPS_FP32   eps = sqrt(2^-23)(1 + ||x||_2) / ||v||_2  (single-precision PC) */
typedef enum { JFNK_EPS_PAPER = 0, JFNK_EPS_FP32 = 1 } jfnk_eps_mode;

typedef struct jfnk_problem jfnk_problem; /* opaque */

typedef struct {
    int kind;            /* jfnk_kind */
    int n_elem;          /* elements per direction on the finest level; n_elem / 2^(levels-1) >= 2 */
    int levels;          /* multigrid levels L+1 >= 1 (Sec. 2: l = 0 coarsest .. L finest) */
    double lambda;       /* Bratu parameter (Sec. 3 uses 5) */
    const double* load;  /* ND3D: optional device FP64 finest-level load vector int f phi_i;
                            NULL = the library computes the manufactured load itself */
    const double* kappa; /* NDK3D: device FP64 per-element coefficient, n_elem^3 values, x fastest;
                            copied into the workspace by jfnk_set_workspace */
} jfnk_problem_desc;

typedef struct {
    int nu_pre, nu_post;     /* V(nu1, nu2) (Alg. 1): smoothing applications per side */
    int cheb_degree;         /* degree k of each Chebyshev application (k FD actions) */
    double cheb_lo, cheb_hi; /* interval [lo, hi] * lambda_l (Sec. 2: 0.06, 1.2) */
    int power_iters;         /* power-method iterations (Sec. 2: at most 30) */
    double power_tol;        /* > 0: also stop when |dlambda| < tol * lambda (Sec. 2: 1e-2) */
    int restart;             /* FGMRES restart length m (<= 64) */
    int max_linear;          /* FGMRES iterations per Newton step */
    double rtol_newton;      /* stop when ||F|| <= rtol ||F_0|| */
    double atol_newton;      /* > 0: also stop when ||F|| < atol (Sec. 3: 1e-6) */
    int eta_mode;            /* 0: eta = min(eta_max, ||F||/||F_0||); 1: min(eta_max, ||F||) (Sec. 3) */
    double eta_max;          /* 0.5 (Sec. 3) */
    double coarse_tol;       /* coarse GMRES stop (Sec. 3: 1e-12) */
    int coarse_tol_mode;     /* 0: relative to ||r_0||, 1: absolute */
    int coarse_maxit;        /* 0: number of coarse unknowns (Sec. 3) */
    int pc_dtype;            /* jfnk_dtype of the preconditioner (smoother, transfers, coarse solve) */
    int eps_mode_pc;         /* jfnk_eps_mode used inside the preconditioner */
    int max_newton;
    int line_search;         /* 1: cubic backtracking (Sec. 3), 0: full steps */
    int ls_max;              /* backtracking steps */
    uint64_t seed;           /* power-method start vector (SplitMix64 stream) */
    int use_graph;           /* 1: capture the V-cycle once in a CUDA graph and replay it */
    /* The paper's own solver variant (Sec. 2 "The coarse level solver", Alg. 1, Sec. 3) */
    int outer;               /* JFNK_OUTER_FGMRES (default) or JFNK_OUTER_CG (Sec. 3) */
    int coarse_method;       /* JFNK_COARSE_GMRES or JFNK_COARSE_CGQN: CG preconditioned by L-BFGS,
                                stopped on negative curvature, re-run with the spectral shift (Alg. 1) */
    int lbfgs_pairs;         /* secant pairs kept for the L-BFGS preconditioner (Sec. 3: 20; <= 32) */
    double shift_gamma;      /* gamma of the shift update lambda_c+ = gamma min(lambda_c, lambda_c+) (Sec. 3: 5) */
} jfnk_options;

typedef enum { JFNK_OUTER_FGMRES = 0, JFNK_OUTER_CG = 1 } jfnk_outer;
typedef enum { JFNK_COARSE_GMRES = 0, JFNK_COARSE_CGQN = 1 } jfnk_coarse_method;

#define JFNK_MAX_LEVELS 16
#define JFNK_MAX_HIST 64

typedef struct {
    int newton_its;
    int linear_its;
    int status;                          /* jfnk_status of the solve */
    int converged;
    double res_hist[JFNK_MAX_HIST];      /* ||F_k||_2 */
    double alpha_hist[JFNK_MAX_HIST];    /* line-search steps */
    int lin_hist[JFNK_MAX_HIST];         /* FGMRES iterations per Newton step */
    double ge;                           /* GE = sum_l 2^(-d(L-l)) GE_l (Sec. 3) */
    long long nF[JFNK_MAX_LEVELS];       /* residual evaluations per level (FD actions included) */
    double lambda_max[JFNK_MAX_LEVELS];  /* last power-method estimates */
    double setup_ms, solve_ms;
    int coarse_shifts;                   /* shifted coarse CG calls (Alg. 1 while-loop) */
    int coarse_negcurv;                  /* coarse CG calls ended by negative curvature */
    int outer_negcurv;                   /* outer CG solves ended by negative curvature */
    long long nJv[JFNK_MAX_LEVELS];      /* FD Jacobian actions per level (part of nF; the
                                            coarse Krylov iterations count on level 0) */
    int ls_hist[JFNK_MAX_HIST];          /* residual evaluations of the line search per Newton
                                            step; when none gives a sufficient decrease the
                                            step is not taken (alpha_hist 0, u and ||F||
                                            unchanged) and the solve returns JFNK_ERR_LINESEARCH */
} jfnk_stats;

/* Defaults of the 2D Bratu workload: V(3,3), degree 3, [0.1, 1.1] lambda_max,
 * 10 power iterations, FGMRES(30), rtol 1e-10, FP64 preconditioner. */
void jfnk_default_options(jfnk_options* opts);

/* The paper's own settings (Sec. 2, Sec. 3 "Setup"): outer CG preconditioned by
 * one V(5,5) cycle (read as one degree-5 Chebyshev application per side),
 * interval [0.06, 1.2] lambda_l, power method to 30 iterations or a relative
 * change below 1e-2, coarse CG with 20 L-BFGS secant pairs and the spectral
 * shift gamma = 5, eta = min(0.5, ||F||), stop at ||F|| < 1e-6, FP64.
 * The paper has no counterpart of use_graph (left at 1). */
void jfnk_paper_options(jfnk_options* opts);

/* Create / destroy a problem description on the current CUDA device.
 * Allocates only host memory.  INVALID_ARG on bad kind/sizes/levels.
 * The 3D kernel choice per level is read from the environment here; it
 * changes speed only (results differ at rounding level):
 *   JFNK_EP3D_MAX_N_F64 / _F32  levels with n <= this run the element-parallel
 *                               kernels (defaults 2^20 / 64)
 *   JFNK_V2_THREADS_F64 / _F32  CTA-size cap of the halo-free kernel (default
 *                               1024; < 0: that kernel is not used)
 *   JFNK_V3_F32                 FP32 halo-free levels: 0 one element a thread,
 *                               1 / 2 two elements a thread with one / two CTAs
 *                               per SM, 3 (default) two, CTAs chosen per mode
 *   JFNK_ZM3D_MIN_N_F64 / _F32  element-parallel levels with n >= this (> 0)
 *                               march element columns along z (default 0: no)
 *   JFNK_EP3D_CLUSTER_MIN_N / _MAX_N  FP32 element-parallel levels with n in
 *                               this range (at most 32) run in one thread-block
 *                               cluster (defaults 16 / 16; _MAX_N 0: never) */
jfnk_status jfnk_problem_create(const jfnk_problem_desc* desc, jfnk_problem** out);
jfnk_status jfnk_problem_destroy(jfnk_problem* p);

/* Bytes of device workspace needed by every call on this problem with these
 * options (opts may be NULL for residual / jvp only). */
jfnk_status jfnk_workspace_size(const jfnk_problem* p, const jfnk_options* opts, size_t* bytes);

/* Attach caller-owned device workspace (>= jfnk_workspace_size bytes, 256-byte
 * aligned).  Zero-fills it, copies kappa (and computes the manufactured load
 * when desc.load is NULL) on `stream`.  The workspace must stay allocated while
 * the problem is used. */
jfnk_status jfnk_set_workspace(jfnk_problem* p, const jfnk_options* opts, void* dev_ptr, size_t bytes, void* stream);

/* F(u) on level `level` (0 coarsest .. levels-1 finest), dtype of u and F.
 * Finest level: F = A(u) - load.  Coarse levels rediscretise the operator A only
 * (the constant load cancels in every FD action).  Sec. 1 / Sec. 3. */
jfnk_status jfnk_residual(jfnk_problem* p, int level, int dtype, const void* u, void* F, void* stream);

/* Jv = (F(u + eps v) - F(u)) / eps  (Sec. 1), with F(u) given as Fu (as returned
 * by jfnk_residual on the same level).  eps > 0 is used as given; eps <= 0
 * selects eps_mode (jfnk_eps_mode).  Boundary entries of v are ignored. */
jfnk_status jfnk_jvp(jfnk_problem* p, int level, int dtype, const void* u, const void* Fu,
                     const void* v, void* Jv, double eps, int eps_mode, void* stream);

/* Per-Newton-step set-up of the hierarchy at the finest iterate u (FP64):
 * x_(l-1) = P x_l (Sec. 2, projection 2^-d I^T), F(x_l) on every level, and the
 * power-method estimate lambda_l on every smoothed level (Sec. 2).  `newton_step`
 * 0 starts the power method from the seeded random vector, later steps from the
 * previous eigenvector. */
jfnk_status jfnk_mg_setup(jfnk_problem* p, const jfnk_options* opts, const double* u,
                          int newton_step, void* stream);

/* s = MG(x_L, F(x_L), b, L): one V(nu1,nu2)-cycle of Algorithm 1 on the finest
 * level, FP64 in and out (converted to/from opts->pc_dtype internally).
 * Requires jfnk_mg_setup. */
jfnk_status jfnk_mg_vcycle(jfnk_problem* p, const jfnk_options* opts, const double* b, double* s, void* stream);

/* Inexact JFNK solve (Sec. 1, Sec. 3): Newton with MG-preconditioned FGMRES(m)
 * (opts->outer = JFNK_OUTER_FGMRES) or CG (JFNK_OUTER_CG, the paper's choice;
 * negative curvature p.Jp <= 0 ends it with the current iterate, or the first
 * search direction at the first iteration) and backtracking; u_inout (FP64) is
 * the initial guess with its Dirichlet data on the boundary and receives the
 * solution.  stats may be NULL. */
jfnk_status jfnk_solve(jfnk_problem* p, const jfnk_options* opts, double* u_inout, jfnk_stats* stats, void* stream);

/* Batched solve (FGMRES outer and GMRES coarse solves only; NOT_IMPLEMENTED
 * otherwise) of `count` independent 2D Bratu problems of uneven sizes and
 * parameters (e.g. 129^2 / 257^2 / 513^2 nodes, different lambda) whose
 * hierarchies end at the same coarse grid.  Each problem keeps its own
 * workspace (laid out for opts); u_inout[i] is instance i's iterate.  The
 * instances advance in lock step (Newton, FGMRES(m), line search per
 * instance), and every device operation is one launch over all instances it
 * applies to -- each level operation of the V-cycle of Algorithm 1 over the
 * instances that have that level, the coarse GMRES with one CTA per instance
 * -- replayed from a CUDA graph when opts->use_graph is set.  Per instance the
 * method and its arithmetic are those of jfnk_solve.  stats (nullable) is an
 * array of count entries.  Synchronises the stream. */
jfnk_status jfnk_solve_batched(jfnk_problem* const* problems, int count, const jfnk_options* opts,
                               double* const* u_inout, jfnk_stats* stats, void* stream);

/* ---- building blocks of Algorithm 1, exposed one by one ---------------- */

typedef enum {
    JFNK_RESTRICT = 0,    /* out(level-1) = R in(level) = I^T in  (Sec. 2; coarse boundary 0) */
    JFNK_PROLONG_ADD = 1, /* out(level) += I in(level-1)          (Sec. 2; coarse boundary taken as 0) */
    JFNK_PROJECT = 2      /* out(level-1) = P in(level) = 2^-d I^T in on interior nodes, injection
                             of the Dirichlet data on the boundary (Sec. 2) */
} jfnk_transfer_op;

/* Transfer between `level` (fine) and `level-1` (coarse), vectors of dtype. */
jfnk_status jfnk_transfer(jfnk_problem* p, int op, int level, int dtype, const void* in, void* out, void* stream);

/* nu Chebyshev smoothing applications of degree opts->cheb_degree for
 * J(x_l) s = b on [cheb_lo, cheb_hi] * lambda_l (Sec. 2, "Smoothers"), in
 * place on s.  Vectors in opts->pc_dtype; s_is_zero = 1 skips the first
 * residual evaluation.  Requires jfnk_mg_setup. */
jfnk_status jfnk_smooth(jfnk_problem* p, const jfnk_options* opts, int level, const void* b, void* s, int nu,
                        int s_is_zero, void* stream);

/* Coarse solve of Algorithm 1 on level 0 (Sec. 2, "The coarse level solver"),
 * in one CTA: GMRES (opts->coarse_method = JFNK_COARSE_GMRES) or the paper's
 * CG preconditioned by L-BFGS with the spectral shift (JFNK_COARSE_CGQN): the
 * first call after jfnk_mg_setup(newton_step = 0) collects the secant pairs and
 * keeps opts->lbfgs_pairs of them (uniform sampling) for every later call; a
 * CG run that meets negative curvature is repeated on A - lambda_c+ I with
 * lambda_c+ = shift_gamma min(lambda_c, lambda_c+) (at most 30 times).  The
 * adjoint solve always uses GMRES.  Vectors in opts->pc_dtype.  Requires
 * jfnk_mg_setup. */
jfnk_status jfnk_coarse_solve(jfnk_problem* p, const jfnk_options* opts, const void* b, void* s, void* stream);

/* Host copies of the level scalars set by jfnk_mg_setup: lambda_l (power
 * method), sum|x_i| and ||x||_2 over interior nodes.  Synchronises `stream`. */
jfnk_status jfnk_level_info(jfnk_problem* p, int level, double* lambda_max, double* xstat_l1, double* xstat_l2,
                            void* stream);

/* Copy a level vector set by jfnk_mg_setup into out (opts->pc_dtype):
 * which = 0: x_l, 1: A(x_l), 2: the power-method vector -- the output J v/||v||
 * of the last power iteration, whose direction is the eigenvector estimate and
 * whose norm is lambda_l (the adjoint solve keeps it normalised). */
jfnk_status jfnk_level_vector(jfnk_problem* p, int level, int which, void* out, void* stream);

/* ---- adjoint: vector-Jacobian products and the adjoint solve --------------
 * For the 3D diffusion problems F_i = sum_e kappa_e int_e (1+u^2) grad u.grad phi_i - b_i
 * (kappa = 1 for ND3D) the transposed Jacobian acts as
 *   (J^T w)_j = sum_e kappa_e int_e (1+u^2) grad w.grad phi_j + 2u (grad u.grad w) phi_j
 * and (dF/dkappa_e)^T w = int_e (1+u^2) grad u.grad w (boundary entries of w ignored).
 * The paper has no adjoint; these follow from differentiating its F. */

/* JTw = J(u)^T w on a level (dtype vectors, full node grids); dFdkappa_w
 * (nullable, NDK3D only, n_l^3 per-element values) = (dF/dkappa)^T w. */
jfnk_status jfnk_vjp(jfnk_problem* p, int level, int dtype, const void* u, const void* w, void* JTw,
                     void* dFdkappa_w, void* stream);

/* Replace the coefficient field of an NDK3D problem (device FP64, n_elem^3,
 * copied) and rebuild the coarse-level coefficients (arithmetic means). */
jfnk_status jfnk_set_kappa(jfnk_problem* p, const double* kappa, void* stream);

/* Adjoint solve at a solution u (FP64): J(u)^T lambda = g by FGMRES(m) with
 * the V-cycle of Algorithm 1 run on J^T (Chebyshev smoothing, restriction,
 * coarse GMRES with the exact vector-Jacobian product; preconditioner in
 * opts->pc_dtype), to ||g - J^T lambda|| <= rtol ||g||.  g's boundary entries
 * are ignored.  If grad_kappa is given (NDK3D): grad_kappa = -(dF/dkappa)^T lambda,
 * the gradient of L(u(kappa)) with dL/du = g (implicit-function theorem).
 * Synchronises the stream; stats (nullable) gets iteration counts and GE. */
jfnk_status jfnk_adjoint_solve(jfnk_problem* p, const jfnk_options* opts, const double* u, const double* g,
                               double* lambda, double* grad_kappa, double rtol, jfnk_stats* stats, void* stream);

/* ---- workspace-free FD Jacobian action ------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc (code that runs where device allocation is forbidden
 * or would stall, or whose device memory is fully reserved by another
 * allocator) and therefore cannot provide the workspace jfnk_jvp needs.
 *
 * Computes the same Jv = (F(u + eps v) - F(u)) / eps as jfnk_jvp on the finest
 * level of a one-level problem described inline: kind, n_elem, lambda (Bratu),
 * kappa (NDK3D, per element, in dtype) and load (ND3D, nullable, in dtype: the
 * load vector included in Fu; NDK3D always includes its unit load).  eps > 0 is
 * used as given, eps <= 0 selects eps_mode.
 *
 * It allocates nothing: its scratch (reduction partials for up to 2048 CTAs,
 * completion counters, the FD step; about 16 KB) is a file-scope __device__
 * array that every GPU which loads libjfnk.so holds until the process exits.
 * Sizes: 2 <= n_elem <= JFNK_NOALLOC_MAX_N3D (3D) or JFNK_NOALLOC_MAX_N2D (2D);
 * larger grids return JFNK_ERR_INVALID_ARG.  Every call looks up the scratch's
 * device address on the current device (cudaGetSymbolAddress); the first lookup
 * on a device may load the library's device code there, so make the first call
 * on each device before any stream capture.  Every call clears the completion counters it needs
 * on `stream` and otherwise reuses the previous call's scratch contents, so calls
 * that overlap on the GPU (other streams, other threads) race on the scratch:
 * serialise them. */
#define JFNK_NOALLOC_MAX_N3D 512
#define JFNK_NOALLOC_MAX_N2D 16384
jfnk_status jfnk_jvp_noalloc(int kind, int n_elem, double lambda, const void* kappa, const void* load, int dtype,
                             const void* u, const void* Fu, const void* v, void* Jv, double eps, int eps_mode,
                             void* stream);

/* Limits of the single-CTA coarse solver and of FGMRES. */
#define JFNK_COARSE_MAX_NODES 1024
#define JFNK_COARSE_MAX_IT 1024
#define JFNK_MAX_RESTART 64

/* Message for the last error on the calling thread. */
const char* jfnk_last_error(void);

/* Measured arithmetic peaks of the current GPU (the paper has no counterpart;
 * these are the denominators of the element kernels' ALU rooflines): FMA
 * operations per second of independent FMA chains on every SM, FP64, FP32, and
 * FP32 in the packed fma.rn.f32x2 form (two FMAs per instruction).  Any output
 * pointer may be NULL to skip that measurement.  Host pointers; launches a few
 * 5-20 ms kernels on `stream` and synchronises it.  Allocates nothing. */
jfnk_status jfnk_measure_peaks(double* fp64_fma_per_s, double* fp32_fma_per_s, double* fp32x2_fma_per_s,
                               void* stream);

/* Bounds record of a bounds-checked build (compiled with -DJFNK_DEBUG_BOUNDS;
 * the paper has no counterpart).  Such a build checks the computed indices of
 * the element kernels, transfers and reductions before each access; an index
 * out of range is clamped into range (no fault, no trap) and the source line
 * of the first one is recorded in device memory.  *enabled = 1 in such a build,
 * 0 otherwise; *line = the first recorded line (0: none; the file is in
 * jfnk_last_error()); reset = 1 clears the record.  Host pointers; reads device
 * memory synchronously. */
jfnk_status jfnk_debug_bounds(int* enabled, unsigned int* line, int reset);

/* Number of kernels this library launched on the calling thread since the last
 * reset (returns the count; reset = 1 then clears it).  A replayed V-cycle
 * graph adds the number of kernels it contains. */
long long jfnk_kernel_launches(int reset);

/* Event timing of the element-residual kernels, per kernel class (problem,
 * precision, fused epilogue, grid size): on = 1 starts a fresh record, 0 stops.
 * Events are recorded on the launching stream around each launch. */
void jfnk_profile_enable(int on);
/* Synchronises the device and fills up to max_classes entries: class names
 * (name_len bytes each), launch counts, summed durations in ms and elements per
 * launch.  Returns the number of classes recorded. */
int jfnk_profile_read(int max_classes, char* names, int name_len, long long* launches, double* total_ms,
                      double* work_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* JFNK_H */
