/*
 * lbfmm: GB300-native fast integral-equation solver for the Laplace-Beltrami
 * Dirichlet problem on the unit sphere with M islands
 * (Kropinski & Nigam, "Fast integral equation methods for the Laplace-Beltrami
 * equation on the sphere").
 *
 * The method (Sec. 3-5): project the island curves stereographically to the
 * plane, discretise the double-layer second-kind equation with the trapezoidal
 * rule (Nystrom), border it with one point source per island (Eq. u_multi,
 * sum_ak, constraints), and solve the bordered system (Eq. matrix_eqns) with
 * GMRES preconditioned by the block matrix [[I, E], [F, D]] (Eq.
 * matrix_eqns_c), computing each matvec with a 2D fast multipole method.
 *
 * Conventions
 *   - Every call returns an int status: 0 = LBF_OK, > 0 = soft (the result is
 *     usable), < 0 = hard error (outputs undefined).  No exception or exit
 *     crosses this interface.
 *   - Array arguments are DEVICE pointers unless marked "host"; the caller owns
 *     them.  Arrays are contiguous, double precision, row-major.
 *   - Calls are asynchronous on the given stream unless marked "synchronous".
 *     Device-side errors (a node at the projection pole, ...) are recorded in a
 *     status word that lbf_sync_status() returns.
 *   - Node ordering: nodes are grouped by island through the CSR array
 *     island_ptr[M+1] (host, int64): island k owns nodes
 *     island_ptr[k] .. island_ptr[k+1]-1, equispaced in the curve parameter
 *     alpha in [0, 2 pi) (h_k = 2 pi / N_k, Sec. 5), curve oriented
 *     counter-clockwise about the island seen from outside the sphere.  Island 0
 *     plays the role of C_1 (the curve that encircles the north pole, Sec. 3)
 *     and is exempt from the density constraint (Eq. disc_constr).
 *   - Unknown vector of the bordered system: [sigma (N); a (M)] (Eq. matrix_eqns),
 *     right-hand side [2 g; 0] (the paper's doubled scaling, Eq. disc_sphere).
 */
#ifndef LBFMM_H
#define LBFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lbf_stream_t; /* a cudaStream_t; NULL = legacy default stream */
typedef struct lbf_plan lbf_plan;

/* status codes */
#define LBF_OK 0
#define LBF_NOCONV 1        /* GMRES hit maxit before tol; outputs are the last iterate */
#define LBF_EINVAL (-1)     /* bad argument (null pointer, size, option out of range) */
#define LBF_EPOLE (-2)      /* a node lies at the projection pole: 1 - x3 < 1e-12 */
#define LBF_EDEPTH (-3)     /* reserved: the tree needs more than max_depth levels */
#define LBF_EWORKSPACE (-4) /* workspace too small; see lbf_plan_create */
#define LBF_ECUDA (-5)      /* a CUDA runtime call failed */
#define LBF_ETIMEOUT (-6)   /* a bounded device wait gave up */
#define LBF_ENOTBUILT (-7)  /* the plan was created without the parts this call needs */
#define LBF_ESINGULAR (-8)  /* the Schur complement S = D - F E of the border is singular */

/* matvec choice */
#define LBF_MATVEC_FMM 0
#define LBF_MATVEC_DIRECT 1

/* operators for lbf_apply */
#define LBF_OP_FULL 0           /* bordered matrix A = [[I+K, E],[F, D]], in/out N+M */
#define LBF_OP_K_ONLY 1         /* density block (I + K) sigma, in/out N   */
#define LBF_OP_PRECONDITIONED 2 /* P^-1 A with P = [[I, E],[F, D]], in/out N+M */

/* Solver and FMM options.  Defaults (lbf_default_options) follow Sec. 6:
 * GMRES restart 50; tolerance 1e-12 (the paper uses 1e-11); FMM accurate to
 * about 1e-12 relative. */
typedef struct lbf_options {
    double tol;           /* GMRES stop: ||P^-1 (b - A x)|| <= tol ||P^-1 b|| */
    int restart;          /* GMRES restart length m (1..200) */
    int maxit;            /* maximum GMRES iterations in total */
    int p;                /* FMM expansion order: terms 0..p (4..63) */
    int leaf_size;        /* a quadtree box is split while it holds more nodes (1..1024) */
    int max_depth;        /* quadtree depth limit D (1..30) */
    int matvec;           /* LBF_MATVEC_FMM or LBF_MATVEC_DIRECT */
    int border;           /* 1: build E, F, D and the Schur complement (needed by
                             LBF_OP_FULL, LBF_OP_PRECONDITIONED, gmres and a-terms
                             of evaluate); 0: density block only */
    int64_t box_capacity; /* quadtree boxes reserved in the workspace; 0 = estimate */
    int precision;        /* LBF_PRECISION_FP64 or LBF_PRECISION_FP32_REFINE */
    int p32;              /* expansion order of the FP32 FMM (4..31) */
    double inner_tol;     /* FP32_REFINE: relative tolerance of each inner solve
                             (default 3e-4) */
    int max_refine;       /* FP32_REFINE: maximum refinement steps */
    int graphs;           /* GMRES steps replayed from a CUDA graph captured once per plan
                             (stream must not be the legacy default stream): 1 on, 0 off,
                             -1 automatic (on for N <= 262144, where launches dominate);
                             per-kernel tracing skips graph-replayed kernels */
    int fmm64;            /* arithmetic of the accurate (double) FMM operator: 0 double,
                             1 double-float (pairs of floats, ~48-bit significands; this
                             GPU issues float 64 times faster than double) */
    int schur;            /* how the preconditioner applies S^-1 (S = D - F E, Sec. 5, Eq.
                             matrix_eqns_c): LBF_SCHUR_AUTO, LBF_SCHUR_GJ or LBF_SCHUR_LU */
    int p2p_warps;        /* near-field tile: warps (leaves) per block of the leaf pass,
                             1..8 (0: 4) */
    int precond;          /* 1: GMRES on P^-1 A (Eq. matrix_eqns_c); 0: on A itself, the
                             unpreconditioned comparison of Sec. 6, Example 1 (the stopping
                             test is then on ||[2g; 0] - A x||) */
} lbf_options;

/* schur: LBF_SCHUR_GJ forms S^-1 by Gauss-Jordan elimination in double (2 M^3 flops on
 * the double pipe; S^-1 to about cond(S) 2^-52) and applies it as a matrix-vector
 * product; LBF_SCHUR_LU factors S = P^T L U in double-float arithmetic on the float pipes
 * (M^3 / 3 multiply-adds; about cond(S) 2^-46) and applies S^-1 by two triangular solves.
 * Either is a preconditioner: the GMRES solution meets tol whichever is used.
 * LBF_SCHUR_AUTO takes GJ for M <= 1024 and LU above. */
#define LBF_SCHUR_AUTO 0
#define LBF_SCHUR_GJ 1
#define LBF_SCHUR_LU 2

/* precision of gmres_solve:
 *   FP64:        every operator application in double;
 *   FP32_REFINE: iterative refinement (GMRES-IR): the FP64 residual
 *                r = P^-1 ([2g; 0] - A x) is formed with the double FMM, the
 *                correction solves P^-1 A d = r with GMRES whose operator runs
 *                the FMM in float (expansions, translations and near field;
 *                node offsets, self terms, the sphere correction, the border
 *                blocks, the rows of each island's mean density -- added
 *                exactly from the discrete Gauss identity -- and the Hessenberg
 *                matrix and Givens rotations stay in double; the Krylov basis
 *                of these inner solves is stored in float, its dot products
 *                summed in double), and x += d until ||r|| <= tol ||P^-1 [2g; 0]||. */
#define LBF_PRECISION_FP64 0
#define LBF_PRECISION_FP32_REFINE 1
/* lbf_apply: OR this into op to run the FMM part in float (plans built with
 * LBF_PRECISION_FP32_REFINE) */
#define LBF_OP_FP32 16
/* lbf_apply: OR this into op to apply the transposed operator instead (the
 * adjoint system): K_ONLY -> (I + 2K)^T, FULL -> A^T, PRECONDITIONED -> P^-T A^T */
#define LBF_OP_TRANSPOSE 32

int lbf_default_options(lbf_options *opt /* host */);

/* Human-readable name of a status code (static string). */
const char *lbf_status_string(int status);

/* Bytes of device workspace a plan over these islands needs (synchronous, host
 * only).  The quadtree part is an estimate from N and leaf_size unless
 * opt->box_capacity is set; lbf_plan_create reports the exact need if the
 * estimate was short. */
int lbf_workspace_size(int M, const int64_t *island_ptr /* host, M+1 */, const lbf_options *opt,
                       size_t *bytes /* host out */);

/* Build a plan: project the nodes to the plane (Sec. 3), precompute the
 * trapezoidal weights w_j = h xi'_j, the self terms and the rank-one sphere
 * correction (Sec. 5, Eq. disc_sphere with Eq. cont_kern), build the Morton
 * quadtree and its interaction lists, and (opt->border) build the lists of the
 * multiplier potential E y (evaluated on the quadtree, E is never formed) and
 * invert the Schur complement S = D - F E (Sec. 5, Eq. matrix_eqns_c).
 *
 *   x, dx, d2x : N x 3 nodes on the unit sphere and their first and second
 *                derivatives with respect to alpha (device)
 *   centres    : M x 3 points c_k inside island k carrying the multiplier
 *                sources A_k G(x, c_k) (Eq. u_multi) (device)
 *   pole_rotation : host 3x3 row-major rotation applied to every point before
 *                projection, or NULL for none (Sec. 3 "without loss of generality")
 *   workspace, bytes : device memory owned by the caller, >= lbf_workspace_size;
 *                it must stay allocated and untouched until lbf_plan_destroy.
 *   box_capacity_needed : host out (nullable): on LBF_EWORKSPACE, the
 *                box_capacity to retry with (then query lbf_workspace_size again).
 * Synchronous: returns after the plan is built.  The library allocates a few KB
 * of pinned host memory here and no device memory anywhere. */
int lbf_plan_create(lbf_plan **plan, int M, const int64_t *island_ptr, const double *x,
                    const double *dx, const double *d2x, const double *centres,
                    const double *pole_rotation, const lbf_options *opt, void *workspace,
                    size_t bytes, int64_t *box_capacity_needed, lbf_stream_t stream);

/* The same plan from nodes given in the stereographic plane (Sec. 3), for
 * callers whose variables are the planar node positions (derivatives with
 * respect to xi_j, with xi'_j and xi''_j held fixed, use this form):
 *   xi, dxi, d2xi : N x 2 (re, im) planar nodes and their first and second
 *                   derivatives with respect to alpha (device)
 *   centres       : M x 3 multiplier sites on the unit sphere (device)
 * No pole rotation (the plane is the caller's); everything else as
 * lbf_plan_create. */
int lbf_plan_create_planar(lbf_plan **plan, int M, const int64_t *island_ptr, const double *xi,
                           const double *dxi, const double *d2xi, const double *centres,
                           const lbf_options *opt, void *workspace, size_t bytes,
                           int64_t *box_capacity_needed, lbf_stream_t stream);

int lbf_plan_destroy(lbf_plan *plan);

/* Plan facts (host out, all nullable): total nodes, islands, quadtree boxes,
 * leaves, deepest level, expansion order. */
int lbf_plan_info(const lbf_plan *plan, int64_t *N, int *M, int64_t *nbox, int64_t *nleaf,
                  int *depth, int *p);

/* Projected geometry in the caller's node order (all nullable, device out):
 *   xi     : N x 2, the stereographic image (x1 + i x2)/(1 - x3) (Sec. 3)
 *   normal : N x 2, unit normal into the island in the plane, -i xi'/|xi'|
 *   weight : N x 2, complex trapezoidal weight h_k xi'_j
 *   arc_weight : N, h_k |xi'_j| */
int lbf_geometry_out(const lbf_plan *plan, double *xi, double *normal, double *weight,
                     double *arc_weight, lbf_stream_t stream);

/* out = op(in) for one of LBF_OP_* (device in/out, caller's node order).
 * LBF_OP_K_ONLY needs N entries in and out; the others N + M. */
int lbf_apply(lbf_plan *plan, int op, const double *in, double *out, lbf_stream_t stream);

/* Solve [[I+K, E],[F, D]] [sigma; a] = [2 g; 0] with restarted GMRES on the
 * left-preconditioned system (Eq. matrix_eqns_c; opt.precond = 0: on the system itself).  g: N boundary values
 * (device); sigma (N), a (M): device out; x0: initial guess [sigma; a] (N+M,
 * device, nullable = zero).  iters, rel_res: host out (nullable): iterations
 * done and the final preconditioned relative residual.  Synchronous.
 * Returns LBF_NOCONV (> 0) when maxit is reached before tol. */
int lbf_gmres_solve(lbf_plan *plan, const double *g, double *sigma, double *a, const double *x0,
                    int *iters, double *rel_res, lbf_stream_t stream);

/* Several right-hand sides of one geometry (the system of Sec. 5, Eq. matrix_eqns, with
 * the options of lbf_gmres_solve), solved together: their GMRES iterations advance in
 * lockstep, groups of up to 16, and every launch of an Arnoldi step, restart or
 * operator application covers the whole group (one CUDA block row per right-hand side,
 * each gated by its own GMRES state), the step replayed from one CUDA graph per group
 * when graphs are on; with FP32_REFINE every refinement round forms the FP64 residuals
 * of the open right-hand sides together and runs their float inner solves in lockstep.
 * Each right-hand side runs the kernels and fixed-order reductions of lbf_gmres_solve on
 * its own buffers, except the near field of the native-double FMM operator (fmm64 = 0),
 * which one pass forms for the whole group, a pair's geometry once for all densities (a
 * different rounding: results agree with separate solves to the solver's tolerance).
 * With direct sums, the double-float operator, or the float one alone, sigma, a, iters
 * and rel_res equal those of nrhs separate lbf_gmres_solve calls bit for bit.  A
 * right-hand side that converges stops while the others go on.  Plans whose S^-1 is
 * applied by LU factors (LBF_SCHUR_LU, or M > 1024 with LBF_SCHUR_AUTO) solve the
 * right-hand sides one after another with lbf_gmres_solve (workspace 0).
 *   g: device, nrhs x N, caller order (right-hand side r at g + r N)
 *   sigma: device out, nrhs x N; a: device out, nrhs x M (nullable)
 *   iters, rel_res: host out, nrhs each (nullable)
 *   work, bytes: device memory, 256-byte aligned, of at least lbf_gmres_workspace_many
 *   bytes (the buffers of each right-hand side of a group: charges, expansions,
 *   Krylov basis; the caller owns it and may reuse it after the call)
 * Synchronous.  LBF_EWORKSPACE when work is short, LBF_NOCONV (soft) when some
 * right-hand side reached maxit. */
int lbf_gmres_workspace_many(const lbf_plan *plan, int nrhs, size_t *bytes /* host out */);
int lbf_gmres_solve_many(lbf_plan *plan, int nrhs, const double *g, double *sigma, double *a,
                         int *iters, double *rel_res, void *work, size_t bytes,
                         lbf_stream_t stream);

/* The adjoint system (Sec. 5, the bordered Eq. matrix_eqns transposed): solve
 * A^T lam = r by GMRES on P^-T A^T (left preconditioning with P^T, the same
 * tolerance, restart, precision and refinement options as lbf_gmres_solve).
 *   r, lam : N + M device vectors in caller order (node part, then one entry per
 *            constraint row, the last one the row of Eq. sum_ak); x0 nullable.
 * Synchronous; LBF_NOCONV (soft) when maxit is reached. */
int lbf_gmres_solve_transpose(lbf_plan *plan, const double *r, double *lam, const double *x0,
                              int *iters, double *rel_res, lbf_stream_t stream);

/* Transposed evaluation (adjoint of lbf_evaluate, Eq. u_multi): for u = C [sigma; a]
 * at the targets, [sbar; abar] = C^T ubar, i.e.
 *   sbar_j = sum_t ubar_t ( (1/2pi) Im(w_j / (xi_j - xi_t)) + beta_j ),
 *   abar_m = sum_t ubar_t G(t, c_m).
 *   targets : T x 3 on the unit sphere; ubar : T; sbar : N; abar : M (nullable);
 *   device, caller order.  Asynchronous; needs the border.  LBF_EWORKSPACE when
 *   the plan's basis region (restart + 1 vectors) holds fewer than 4 N doubles. */
int lbf_evaluate_transpose(lbf_plan *plan, int64_t T, const double *targets, const double *ubar,
                           double *sbar, double *abar, lbf_stream_t stream);

/* Gradient of a target functional L(u) with respect to the planar node positions
 * (d/dRe xi_j, d/dIm xi_j; xi'_j and xi''_j held fixed, so the weights and the
 * diagonal-limit terms are constant):
 *   dL/dxi_j = d/dxi_j (ubar^T C z) - lam^T (dA/dxi_j) z,   A^T lam = C^T ubar,
 * for the solution z = [sigma; a] of lbf_gmres_solve, ubar = dL/du at the targets
 * and lam from lbf_gmres_solve_transpose (r = C^T ubar from lbf_evaluate_transpose).
 * (dL/dg comes from lbf_gradient_data.)  sigma (N), a (M), lam (N + M), ubar (T),
 * targets (T x 3), grad (N x 2 out): device, caller order.  Asynchronous, FP64;
 * LBF_EWORKSPACE when the basis region holds fewer than 12 N doubles. */
int lbf_gradient_nodes(lbf_plan *plan, const double *sigma, const double *a, const double *lam,
                       int64_t T, const double *targets, const double *ubar, double *grad,
                       lbf_stream_t stream);

/* Gradient of a target functional with respect to the Dirichlet data g: the data
 * enter the bordered system (Eq. matrix_eqns) only through its right-hand side
 * [2 g; 0] (the doubled scaling of Eq. disc_sphere), so dL/dg_j = 2 lam_j with lam
 * the adjoint solution of lbf_gmres_solve_transpose (A^T lam = C^T ubar).
 *   lam : N + M (device, caller order; only the first N entries are read)
 *   grad_g : N (device out, caller order).  Asynchronous. */
int lbf_gradient_data(lbf_plan *plan, const double *lam, double *grad_g, lbf_stream_t stream);

/* Batched solves of independent geometries: many instances of the bordered system
 * of Sec. 5, each with nrhs right-hand sides (the paper solves one instance at a
 * time; this is an interface of the library).  nworkers host threads, each with its
 * own CUDA stream, take the items largest first (nodes x right-hand sides); per
 * item: a plan (lbf_plan_create, no pole rotation); the right-hand sides solved with
 * opt by lbf_gmres_solve_many when the item's workspace has room for it after the
 * plan's (lbf_batch_workspace_size), else by lbf_gmres_solve one after another; when
 * T > 0 and u != NULL, lbf_evaluate at the targets; then the plan is destroyed.  Synchronous.  Returns LBF_EINVAL for a bad
 * item, LBF_ECUDA if a worker could not start; each item's own outcome is in its
 * status (LBF_EWORKSPACE with box_capacity_needed set when its workspace was short). */
typedef struct lbf_batch_item {
    /* in */
    int M;                                  /* islands */
    const int64_t *island_ptr;              /* host, M + 1 */
    const double *x, *dx, *d2x, *centres;   /* device, as lbf_plan_create */
    void *workspace;                        /* device, >= lbf_workspace_size(M, island_ptr, opt);
                                               lbf_batch_workspace_size(..., nrhs) bytes for the
                                               right-hand sides in lockstep */
    size_t bytes;
    int nrhs;                               /* right-hand sides */
    const double *g;                        /* device, nrhs x N: right-hand side r at g + r N */
    double *sigma, *a;                      /* device out, nrhs x N and nrhs x M (a nullable) */
    int64_t T;                              /* targets (0: no evaluation) */
    const double *targets;                  /* device, T x 3 */
    double *u;                              /* device out, nrhs x T (nullable) */
    int64_t box_capacity;                   /* this item's opt->box_capacity (0: estimate) */
    /* out (host) */
    int status, iters;                      /* worst status; GMRES iterations over the rhs */
    int64_t fp64_applies, fp32_applies;     /* operator applications over the rhs */
    double max_rel_res;                     /* largest final relative residual */
    int64_t box_capacity_needed;            /* see lbf_plan_create */
} lbf_batch_item;
int lbf_batch_run(int nitems, lbf_batch_item *items, const lbf_options *opt, int nworkers);
/* Workspace of one batch item whose right-hand sides are solved in lockstep
 * (lbf_gmres_solve_many) by lbf_batch_run: the plan's bytes (lbf_workspace_size),
 * rounded up to 256, then lbf_gmres_workspace_many's for nrhs right-hand sides (none
 * where those are solved one after another).  An item whose workspace holds less
 * solves its right-hand sides one after another.  Host call, no GPU work. */
int lbf_batch_workspace_size(int M, const int64_t *island_ptr, const lbf_options *opt, int nrhs,
                             size_t *bytes /* host out */);

/* Autotuner of the FMM's free parameters for one geometry (the paper fixes neither
 * the expansion order nor the leaf size; Sec. 6 gives only the FMM tolerance):
 * timed trials of the density operator (I + 2K) sigma on a seeded density, against a
 * reference at order 44.  For each leaf size in {32, 48, 64} the order p rises from 16
 * until the relative l2 error is at most target / 4; the fastest such (p, leaf) is
 * kept, then the near-field tile (p2p_warps 2, 4, 8).  A trial's time is its accurate
 * application's, plus, when base asks for FP32_REFINE, 10 times its float application's
 * (about the float applications per FP64 residual of a refinement solve).  Trial plans
 * are built without the border, one at a time, in the caller's workspace.
 *   geometry and pole_rotation: as lbf_plan_create (device arrays; rotation host/NULL)
 *   base: options to start from (precision, fmm64, ...: kept in *best)
 *   target: the largest acceptable rel-l2 error of the operator
 *   workspace, bytes: device memory; with workspace = NULL only *bytes_needed is set
 *   best: host out, base with p, leaf_size and p2p_warps chosen
 *   table, table_len: host out (nullable), every trial as JSON text
 * Synchronous.  LBF_NOCONV (soft) when no trial met the target (best = base). */
int lbf_autotune(int M, const int64_t *island_ptr, const double *x, const double *dx,
                 const double *d2x, const double *centres, const double *pole_rotation,
                 const lbf_options *base, double target, void *workspace, size_t bytes,
                 size_t *bytes_needed, lbf_options *best, char *table, size_t table_len,
                 lbf_stream_t stream);

/* Work of the plan's last lbf_gmres_solve (host out): stats[0] Arnoldi steps,
 * [1] FP64 operator applications, [2] FP32 operator applications,
 * [3] refinement steps (0 for LBF_PRECISION_FP64). */
int lbf_solve_stats(const lbf_plan *plan, int64_t stats[4]);

/* u at T points t (T x 3 on the sphere, off the curves, device) from the
 * representation formula (Eq. u_multi): the double layer of sigma plus
 * sum_m a_m G(t, c_m).  a may be NULL (no multiplier sources). */
int lbf_evaluate(lbf_plan *plan, const double *sigma, const double *a, int64_t T,
                 const double *targets, double *u, lbf_stream_t stream);

/* out_q = sum_s gamma_s G(t_q, p_s), G the generalized fundamental solution
 * (Sec. 1.1, Eq. greens_func): Dirichlet data of point sources or vortices
 * (Sec. 6, Example 2).  t: T x 3, p: S x 3, gamma: S, out: T (device). */
int lbf_green_sum(int64_t T, const double *t, int64_t S, const double *p, const double *gamma,
                  double *out, lbf_stream_t stream);

/* out_q = (1/2) sum_s Re 1 / (xi(t_q) - xi(p_s)), xi the stereographic image (Sec. 3):
 * the exact solution of Sec. 6, Examples 1 and 3 (Eq. exact_bcs), harmonic in the plane
 * away from the xi(p_s) and hence Laplace-Beltrami harmonic on the sphere.  A source at the
 * north pole (xi = infinity) adds nothing.  t: T x 3, p: S x 3, out: T (device), in the
 * frame whose north pole is the projection pole. */
int lbf_dipole_sum(int64_t T, const double *t, int64_t S, const double *p, double *out,
                   lbf_stream_t stream);

/* Point vortices in the ocean (Sec. 6, Example 2): the stream function
 * psi = psi* + sum_s gamma_s G(., v_s) with psi = 0 on every curve, where the regular
 * part psi* solves the Dirichlet problem with data -sum_s gamma_s G(x, v_s) on the curves
 * (composed in the library: that data from the plan's nodes, lbf_gmres_solve, then
 * lbf_evaluate plus the vortices' own term at the targets).
 *   vortices : S x 3 points on the sphere in the ocean (device, caller's frame)
 *   gamma    : S strengths (device)
 *   targets  : T x 3 off-curve points (device, caller's frame); u: T (device out)
 *   sigma, a : N and M (device out): the density and multipliers of psi*; sigma also
 *              holds the data while the solve reads it
 *   iters, rel_res : host out (nullable), as lbf_gmres_solve.
 * Synchronous (the solve is); LBF_NOCONV (soft) when GMRES reached maxit. */
int lbf_point_vortices(lbf_plan *plan, int64_t S, const double *vortices, const double *gamma,
                       int64_t T, const double *targets, double *u, double *sigma, double *a,
                       int *iters, double *rel_res, lbf_stream_t stream);

/* The quadtree of a plan (Sec. 6, Example 3), for inspection and tests
 * (device out, synchronous, all nullable):
 *   perm  : N entries, perm[i] = caller index of the i-th node in Morton order
 *   boxes : nbox x 8 int32 rows {level, ix, iy, parent, first_child, nchild,
 *           begin, end}; boxes are numbered level by level, in Morton order
 *           within a level; [begin, end) indexes the Morton-ordered nodes.
 * The integer specification of keys and splitting is given in lbf_tree.cu. */
int lbf_tree_export(const lbf_plan *plan, int32_t *perm, int32_t *boxes, lbf_stream_t stream);

/* One interaction list of the adaptive FMM in CSR form over boxes
 * (kind 0..3 = U, V, W, X; device out, synchronous).  ptr: nbox + 1 entries;
 * idx: *len entries (pass idx = NULL to query *len, host out). */
int lbf_list_export(const lbf_plan *plan, int kind, int32_t *ptr, int32_t *idx, int64_t *len,
                    lbf_stream_t stream);

/* Work counts of a plan's FMM (host out, synchronous), for algorithmic-FLOP
 * accounting: counts[0] N, [1] near-field pairs (P2P, self excluded),
 * [2] M2M shifts, [3] M2L translations (V lists), [4] L2L shifts,
 * [5] (target node, W box) pairs, [6] (source node, X box) pairs, [7] leaves. */
int lbf_plan_counts(const lbf_plan *plan, int64_t counts[8], lbf_stream_t stream);

/* Work counts of the multiplier potential E y (Sec. 4.1, Eq. u_multi; the FMM
 * evaluation of E a suggested in Sec. 5), host out, synchronous:
 * counts[0] (box, centre) P2L pairs, [1] (node, centre) pairs summed directly
 * (adjacent leaves), [2] centres summed directly at every node (outside the
 * tree's square), [3] sum over nodes of the local expansions evaluated by the
 * float operator (tree levels >= 2 on the path from the node's leaf to the
 * root), [4] terms of its double local expansions, [5] terms of its float
 * local expansions.  LBF_ENOTBUILT without the border. */
int lbf_border_counts(const lbf_plan *plan, int64_t counts[6], lbf_stream_t stream);

/* Tracing: while enabled, every launch of the kernels below is bracketed by a
 * pair of CUDA events recorded on the stream it is launched on.  Host calls;
 * lbf_profile_read synchronizes on the recorded events and returns, per kernel,
 * the launches and their summed device time. */
#define LBF_KERNEL_UP 0     /* upward pass: P2M + M2M, one launch */
#define LBF_KERNEL_DOWN 1   /* downward pass: L2L + M2L + P2L, one launch per level */
                            /* (the float pass: M2L + P2L, one launch, no L2L) */
#define LBF_KERNEL_LEAF 2   /* L2P + M2P + P2P + combine */
#define LBF_KERNEL_DIRECT 3
#define LBF_KERNEL_ARNOLDI 4
#define LBF_KERNEL_ESUM 5   /* multiplier potential E y: P2L, L2L and L2P + direct centres
                               (float: the evaluation at the nodes only) */
#define LBF_KERNEL_UP32 6   /* the three FMM passes of the float operator */
#define LBF_KERNEL_DOWN32 7
#define LBF_KERNEL_LEAF32 8
#define LBF_KERNEL_ESUM32 9 /* the multiplier potential of the float operator */
/* stages of lbf_plan_create (every launch of the stage between one event pair) */
#define LBF_STAGE_GEOMETRY 10 /* projection, quadtree, interaction lists, gather */
#define LBF_STAGE_BORDER 11   /* multiplier-potential lists and the Schur complement */
#define LBF_STAGE_INVERSE 12  /* Gauss-Jordan inverse of the Schur complement */
/* the double-float LU of the Schur complement (schur = LBF_SCHUR_LU) */
#define LBF_KERNEL_LU_PANEL 13  /* panel elimination with the pivot search (per panel) */
#define LBF_KERNEL_LU_UPDATE 14 /* interchanges, U12 = L11^-1 A12, diagonal-block inverses */
#define LBF_KERNEL_LU_GEMM 15   /* trailing update A22 -= L21 U12 */
#define LBF_KERNEL_LU_SOLVE 16  /* the two triangular solves of each S^-1 application */
#define LBF_KERNEL_COUNT 17
int lbf_profile_enable(int on);
int lbf_profile_reset(void);
int lbf_profile_read(int kernel, int64_t *launches /* host out */, double *total_ms /* host out */);

/* lbf_evaluate_noalloc: the same off-curve evaluation as lbf_evaluate, for
 * callers that cannot allocate device memory at all -- no plan, no workspace,
 * no allocator call.  (The paper has no counterpart: this is an interface
 * convenience of this library.)  Useful where no allocator is reachable or
 * allowed: a loop running on a fixed memory budget set at start-up, a
 * foreign-language binding without access to the framework's allocator, a
 * plugin that must not grow its host library's pool.
 *   xi, weight : N x 2 projected nodes and complex weights h xi', as returned by
 *                lbf_geometry_out (any node order, the same for sigma)
 *   sigma      : N densities; a (M), centres (M x 3): multiplier sources in the
 *                same rotated frame as xi (M = 0: none); targets: T x 3, same frame
 *   u          : T outputs.  All arrays are device memory owned by the caller.
 * Its scratch (q = sigma w and the reduction partials, about 4 MB) is one
 * static device array, so N is limited to LBF_NOALLOC_MAX_NODES: larger N
 * returns LBF_EINVAL without touching the device.  Every call shares that
 * array: calls that overlap on the GPU race, so serialise them.  The first call
 * on a device looks up the array's address with that device current; make it
 * before any stream capture.  Asynchronous on the stream. */
#define LBF_NOALLOC_MAX_NODES 262144
int lbf_evaluate_noalloc(int64_t N, const double *xi, const double *weight, const double *sigma,
                         int M, const double *a, const double *centres, int64_t T,
                         const double *targets, double *u, lbf_stream_t stream);

/* The double reciprocals of the operator's sums, exposed for tests against IEEE
 * division.  Every near-field pair of Sec. 5's discretised double layer needs
 * 1/|xi_j - xi_i|^2; the library refines a single-precision seed x with e = 1 - a x:
 *   variant 0: the general form, seeded by the float reciprocal of (float)a, two
 *              Newton-Raphson steps x <- x + x e; outside [1e-30, 1e30] it falls back
 *              to the division operator;
 *   variant 1: the near-field and far-field form, for a in [2^-126, 2^126] only: the
 *              seed is built from a's bits by integer operations (no conversion
 *              instruction on the double pipe), then one third-order step
 *              x <- x + x (e + e^2).
 * a, out: n doubles (device).  Asynchronous. */
int lbf_selftest_rcp(int variant, int64_t n, const double *a, double *out, lbf_stream_t stream);

/* Failure injection, for tests of the bounded device waits (every wait polls a bounded
 * number of times, then records LBF_ETIMEOUT in the plan's status word and lets its
 * kernel finish, so the context stays usable):
 *   LBF_INJECT_CHAIN (plan given): the plan's waits give up after `polls` polls, and the
 *     next accurate operator application's one-launch L2L chain (the downward pass)
 *     skips the boxes of levels 0-2 in its second phase, so the parent waits of their
 *     children run out; lbf_sync_status then returns LBF_ETIMEOUT;
 *   LBF_INJECT_BARRIER (plan NULL): the next lbf_plan_create on this thread gives its
 *     waits `polls` polls and starts the grid barrier of the Schur complement's inverse
 *     (or factorisation) already past its count, so it never opens; that creation
 *     returns LBF_ETIMEOUT.
 * Synchronous.  lbf_debug_clear resets a plan's status word and poll limit. */
#define LBF_INJECT_CHAIN 1
#define LBF_INJECT_BARRIER 2
int lbf_debug_inject(lbf_plan *plan, int what, unsigned polls, lbf_stream_t stream);
int lbf_debug_clear(lbf_plan *plan, lbf_stream_t stream);

/* Wait for the stream and return the first device-side error recorded by
 * this plan's kernels (LBF_OK if none).  Synchronous. */
int lbf_sync_status(lbf_plan *plan, lbf_stream_t stream);

/* Number of kernels this library has launched in this process (a kernel
 * replayed inside a CUDA graph counts once per replay). */
int64_t lbf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LBFMM_H */
