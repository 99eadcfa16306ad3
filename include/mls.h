/*
 * mls.h -- C ABI of the GB300 (sm_103a) multilevel elastodynamics timestep
 * library: the per-Newton-iteration linear solve of arXiv 2508.13386,
 * "Sparse, Geometry- and Material-Aware Bases for Multilevel Elastodynamic
 * Simulation", and the Newton loop around it.
 *
 * What one timestep computes (Sec. 3.1, Eq. IP with implicit Euler):
 *   x^{t+1} = argmin_x E(x),
 *   E(x) = 1/2 sum_{v free} m_v |x_v - x_tilde_v|^2
 *          + h^2 ( sum_e vol_e psi(F_e(x)) + kappa sum_v b(n . x_v - o) ),
 *   x_tilde = x^t + h v^t + h^2 g,      v^{t+1} = (x^{t+1} - x^t) / h,
 * with the non-inverting Neo-Hookean psi of Sec. 4 (psi = mu/2 (tr F^T F - 3)
 * - mu ln J + lam/2 ln^2 J), the point-plane IPC log barrier
 * b(d) = -(d - dhat)^2 ln(d / dhat) on (0, dhat), lumped masses, and
 * Dirichlet vertices held at x^t.  Each Newton iteration solves H d = -g
 * (Eq. 5) with H the element-wise PSD-projected Hessian, by conjugate
 * gradient preconditioned either with 3x3 block Jacobi or with the two-level
 * cycle built from the paper's sparse LBS basis (Eq. LBS, Sec. 3.5): smoothing
 * by block Jacobi plus the Galerkin coarse correction U (U^T H U)^{-1} U^T
 * (Alg. 2 / Sec. 3.7.1, here with the coarse operator formed explicitly and
 * factored by dense Cholesky).  A filtered backtracking line search (Sec. 3.9)
 * follows: the point-plane CCD bound, J > 0 on every tet, Armijo on E.
 *
 * Conventions for every entry point:
 *  - Units are SI; positions, velocities and energies are float64.
 *  - Arrays are C-contiguous.  "[n][3]" means n rows of (x, y, z).
 *  - Pointers documented as DEVICE must be device memory of the current
 *    CUDA device (for example torch.Tensor.data_ptr() of a CUDA tensor); those
 *    documented as HOST are ordinary host memory.  The caller owns every
 *    pointer it passes; uploads copy into library-owned device buffers, and
 *    the library keeps no caller pointer after a call returns.
 *  - Every call runs on the context's stream (mls_options.stream, 0 = the
 *    legacy default stream) and returns only after its work on that stream
 *    has completed, so results are ready when the call returns.
 *  - Errors are returned as a negative mls_status with a message available
 *    from mls_last_error(); no call aborts, traps or throws across the ABI.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef MLS_H_
#define MLS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mls_status {
  MLS_OK = 0,
  MLS_EINVAL = -1,      /* bad argument, size or call order */
  MLS_ENOMEM = -2,      /* device or host allocation failed */
  MLS_ECUDA = -3,       /* a CUDA runtime call failed */
  MLS_ENOTCONV = -4,    /* Newton or PCG hit its iteration cap */
  MLS_ELINESEARCH = -5, /* no acceptable step after the halving cap */
  MLS_ECHOL = -6,       /* coarse operator not positive definite */
  MLS_ENONFINITE = -7,  /* NaN or Inf in an input or an iterate */
  MLS_ETIMEOUT = -8,    /* a bounded device-side wait gave up */
  MLS_EINVERTED = -9    /* an input state has a tet with J <= 0 or a vertex on/below the plane */
} mls_status;

/* Arithmetic of the linear solve.  Gradients, energies, norms, dot products,
 * the line search and the coarse Cholesky factorisation are float64 in every
 * mode. */
enum {
  MLS_FP64 = 0,        /* element Hessians, H, PCG vectors: float64 */
  MLS_MIXED_FP32 = 1,  /* element Hessians, H, PCG vectors, smoothing and
                          basis projection: float32 with float32 accumulation */
  MLS_MIXED_BF16 = 2   /* as MIXED_FP32, but H's values stored as bfloat16 */
};

enum {
  MLS_PRECOND_BLOCK_JACOBI = 0, /* 3x3 block-diagonal inverse */
  MLS_PRECOND_TWO_LEVEL = 1     /* block-Jacobi smoothing + Galerkin coarse correction */
};

enum {
  MLS_CYCLE_ADDITIVE = 0,       /* z = omega D^-1 r + U A_c^-1 U^T r */
  MLS_CYCLE_MULTIPLICATIVE = 1  /* smooth, coarse-correct the residual, smooth (symmetric) */
};

typedef struct mls_options {
  int precision;       /* MLS_FP64 | MLS_MIXED_FP32 | MLS_MIXED_BF16 */
  int preconditioner;  /* MLS_PRECOND_BLOCK_JACOBI | MLS_PRECOND_TWO_LEVEL */
  int cycle;           /* MLS_CYCLE_* (two-level only) */
  double omega;        /* block-Jacobi damping in the two-level cycle; 0 chooses it at
                          every coarse build: 0.9 x 2 / lambda, lambda the largest
                          Ritz value of 20 Lanczos steps on D^-1 H (D the 3x3 block
                          diagonal of H).  The symmetric cycle is positive
                          definite only while omega lambda_max(D^-1 H) < 2; a PCG
                          breakdown with the automatic choice retries the solve
                          with omega x 0.8 (up to three times).  Not for batches. */
  double newton_tol;   /* stop when |d|_inf <= newton_tol * max(|x - x^t|_inf, h^2 |g|) */
  double pcg_rtol;     /* PCG stops at |r|_2 <= eta |b|_2, eta = min(pcg_rtol, forcing term) */
  int max_newton;      /* Newton iteration cap per timestep */
  int max_pcg;         /* PCG iteration cap per Newton iteration */
  int coarse_refresh;  /* 0: rebuild U^T H U and its factor every Newton iteration;
                          k > 0: at the first iteration of a step and then every k */
  int coarse_lag_steps; /* 0 (default): a step's first Newton iteration always
                          rebuilds the coarse operator; s > 0: it keeps a factor
                          built at most s steps earlier (a lagged preconditioner:
                          PCG still solves the current Newton system; ignored
                          with direction 1).  If that first solve takes more
                          than 1.5 x + 8 the PCG iterations of the first
                          solve of the first step after the last build, the
                          factor is rebuilt at the next Newton iteration. */
  int pcg_check_every; /* PCG iterations launched between host convergence checks
                          (separate-kernel mode) */
  int persistent;      /* 1: run the PCG iterations in one cooperative persistent
                          kernel per solve; 0 (default): one launch per phase */
  int persist_blocks_per_sm; /* resident blocks per SM of the persistent kernel
                          (0: the library's choice; capped by occupancy) */
  int direction;       /* 0 (default): each Newton direction solves H d = -g by PCG
                          to the forcing tolerance, and Newton stops on the step
                          test newton_tol.  1: the paper's inexact direction
                          (Alg. 1, Alg. 2; two-level preconditioner required):
                          d_s = U (U^T H U)^{-1} U^T (-g) from the factored
                          Galerkin operator, plus refine_iters block-Jacobi CG
                          iterations on H d_f = -g - H d_s from d_f = 0;
                          Newton stops after the update when the mean vertex
                          speed of the subspace step, sum_v |d_s,v|_2 /
                          (h n_vertices), is below paper_tol (m/s, Sec. 3.9).
                          2: as 1, with the subspace direction of Alg. 2 as
                          printed: the affine level (one handle at the centre
                          of mass, phi = 1; left out when the mesh has
                          Dirichlet vertices) solved on its 12 x 12 operator,
                          then PCG on (U^T H U) q = U^T (-g - H d_a) with 12 x 12
                          block-Jacobi preconditioning and the matrix-free
                          product U^T (H (U q)), to relative residual sub_rtol;
                          no coarse factorisation */
  int refine_iters;    /* directions 1, 2: fixed full-space CG iterations (20-40) */
  double paper_tol;    /* directions 1, 2: subspace-decrement tolerance (1e-3) */
  void* stream;        /* cudaStream_t the context runs on (0 = legacy default) */
  double sub_rtol;     /* direction 2: relative residual of the subspace PCG (1e-4,
                          Sec. 3.7.1) */
  int hessian_lag;     /* directions 1, 2: 1 = the refinement CG solves with H_lag
                          (Sec. 3.7.2): the element Hessians saved at the last
                          refresh, with the mass, contact and friction blocks
                          of the current iterate.  H_lag is refreshed at the
                          first Newton iteration of a step and whenever the
                          mean of the last three line-search step sizes falls
                          below 0.5, at most once every five iterations.
                          0 (default): the refinement uses the fresh H */
} mls_options;

typedef struct mls_stats {
  int newton_iters;        /* Newton iterations taken */
  int pcg_iters;           /* PCG iterations summed over the Newton iterations */
  int line_search_trials;  /* energy evaluations in the line search */
  int coarse_builds;       /* Galerkin builds + factorisations */
  double step_rel;         /* final |d|_inf / max(|x - x^t|_inf, h^2 |g|); with the
                              paper's direction, sum_v |d_s,v|_2 / (h n_vertices) */
  double grad_norm;        /* |g|_2 at the last evaluated iterate */
  double energy;           /* E at the returned iterate */
  int64_t kernel_launches; /* CUDA kernels this call launched */
  int warm_start_used;     /* 1 if the step started from the network's prediction */
  int coarse_shifts;       /* coarse factorisations retried with a diagonal shift:
                              a non-positive pivot in U^T H U is retried on
                              U^T H U + sigma diag(U^T H U), sigma = 1e-7, 1e-5,
                              1e-3, 1e-1 (the operator only preconditions, so the
                              converged direction does not change) */
  int coarse_fallbacks;    /* Newton iterations preconditioned by block Jacobi
                              because U^T H U stayed indefinite after the shift
                              retries (the next iteration builds it again) */
  int subspace_iters;      /* direction 2: subspace PCG iterations summed over the
                              Newton iterations (the affine level counts one per
                              Newton iteration) */
  int hessian_refreshes;   /* hessian_lag: refreshes of H_lag in the step */
  int contact_pairs;       /* mesh-mesh pairs within dhat at the last assembly (mls_set_bodies) */
} mls_stats;

typedef struct mls_ctx mls_ctx;

/* Fill *opt with defaults: FP64, block Jacobi, newton_tol 1e-10, pcg_rtol
 * 1e-4 (the paper's subspace PCG tolerance, Sec. 3.7.1), 50 Newton and 20000
 * PCG iterations, additive cycle, omega 1, coarse_refresh 0, check every 16,
 * one launch per PCG phase, default stream.  Returns MLS_EINVAL if opt is NULL. */
mls_status mls_default_options(mls_options* opt);

/* Create a context on the current CUDA device.  opt may be NULL (defaults).
 * *out receives the context; free it with mls_destroy. */
mls_status mls_create(mls_ctx** out, const mls_options* opt);

/* Free a context and all its device memory.  NULL is a no-op. */
mls_status mls_destroy(mls_ctx* ctx);

/* Message for the last failed call on ctx ("" if none).  Owned by ctx. */
const char* mls_last_error(const mls_ctx* ctx);

/* Change options after creation (same meaning as in mls_create). */
mls_status mls_set_options(mls_ctx* ctx, const mls_options* opt);

/* The block-Jacobi damping the two-level cycle applies now (*omega, HOST):
 * opt.omega, or with opt.omega = 0 the choice made at the last coarse
 * build, whose estimate of lambda_max(D^-1 H) goes to *lambda_max (HOST,
 * nullable; 0 before any automatic choice). */
mls_status mls_smoother_omega(mls_ctx* ctx, double* omega, double* lambda_max);

/* Largest eigenvalue of the symmetric tridiagonal matrix with diagonal
 * d[0..k-1] and off-diagonal e[0..k-2] (HOST arrays), by bisection on the
 * Sturm count; the result bounds it from above to rounding.  NaN for k < 1
 * or null arrays.  Used by the automatic damping; exported for testing. */
double mls_tridiag_max_eig(const double* d, const double* e, int k);

/* Upload the tet mesh and its materials (Sec. 3.1 discretisation; Sec. 4
 * material model).  All HOST pointers:
 *   rest_xyz  [n_verts][3]  rest positions X
 *   tets      [n_tets][4]   vertex indices, each tet positively oriented at rest
 *   youngs, poisson, density   [n_tets]  E (Pa), nu, rho (kg/m^3)
 *   dirichlet [n_verts]     1 = vertex held at its current position, 0 = free;
 *                           NULL = none
 * Builds rest shapes, lumped masses and the BSR sparsity of H.  Replaces a
 * previous mesh and drops an uploaded basis.  MLS_EINVAL for n_verts < 1,
 * n_tets < 1, an index out of range, a non-positive rest volume, E <= 0,
 * nu outside (-1, 0.5) or rho <= 0. */
mls_status mls_upload_mesh(mls_ctx* ctx, int32_t n_verts, const double* rest_xyz,
                           int32_t n_tets, const int32_t* tets, const double* youngs,
                           const double* poisson, const double* density,
                           const uint8_t* dirichlet);

/* Upload a sparse LBS basis (Eq. LBS): handle origins and, per vertex, the
 * handles whose weight phi_j(v) is nonzero (Sec. 3.5), as HOST arrays:
 *   origins [n_handles][3]    handle origins o_j
 *   vrow    [n_verts + 1]     CSR row pointer over vertices
 *   handle  [vrow[n]]         handle index of each entry, 0 <= j < n_handles
 *   phi     [vrow[n]]         weight phi_j(v)
 * Column 12 j + 4 c + l of U at row 3 v + c is phi_j(v) a_l with
 * a = [1, X_v - o_j].  Needed by MLS_PRECOND_TWO_LEVEL.  MLS_EINVAL for
 * sizes or indices out of range or a call before mls_upload_mesh. */
mls_status mls_upload_basis(mls_ctx* ctx, int32_t n_handles, const double* origins,
                            const int32_t* vrow, const int32_t* handle, const double* phi);

/* Cubature of the elastic term in the coarse operator (Sec. 3.8): scale
 * [n_tets] HOST, per element the factor w_e / vol_e of a cubature with
 * weights w_e (0 off the cubature; see paper_2508_13386_gb300/cubature.py for
 * the modal moment fitting of Alg. 3).  From the next coarse build on,
 * U^T H U is built from H_cub = M + h^2 (sum_e scale_e H_e + barrier), the
 * mass and barrier terms whole; the fine H and every other use of H are
 * unchanged.  NULL removes the cubature.  MLS_EINVAL for a negative or
 * non-finite factor or a call before mls_upload_mesh. */
mls_status mls_upload_cubature(mls_ctx* ctx, const double* scale);

/* External loads (HOST arrays of 3): gravity g (m/s^2); when contact != 0 the
 * ground plane {x : n . x = o} with unit normal plane_n, barrier distance
 * dhat > 0 and stiffness kappa > 0.  Defaults: g = (0, 0, -9.81), no contact. */
mls_status mls_set_forces(mls_ctx* ctx, const double* gravity, int contact,
                          const double* plane_n, double plane_o, double dhat, double kappa);

/* Lagged point-plane friction, the term D of Eq. IP (Sec. 3.1, which takes
 * IPC's mollified friction potential without writing it out).  For each
 * vertex v, with distance d_v^t = n . x_v^t - o to the plane of
 * mls_set_forces and h the timestep:
 *   lam_v = -kappa b'(d_v^t)                   normal force, lagged at x^t
 *   u_v   = (I - n n^T)(x_v - x_v^t),  y = |u_v|   tangential slip
 *   D     = sum_v mu lam_v f0(y),  f0' = f1 = 2y/eps - y^2/eps^2 (y < eps), 1 (y >= eps),
 *           f0(0) = eps / 3,  eps = eps_v h,
 * added to E with the same h^2 (BDF2: (4/9) h^2) factor as the elastic energy;
 * its gradient, its (PSD) diagonal Hessian blocks and its energy enter the
 * assembly and the line search.  mu = 0 turns it off (the default).
 * With bodies set (mls_set_bodies) the same mu and eps_v also give the
 * friction between them, the ground form with the plane replaced by each
 * pair's closest points: every point-triangle and edge-edge pair of
 * different bodies within dhat at x^t keeps, for the step, the weights w of
 * its closest-point difference (sum_j w_j x_j, the weights summing to zero),
 * the unit normal n along it and lam = -kappa b'(d); its slip is
 *   u = (I - n n^T) sum_j w_j (x_j - x_j^t)
 * and it adds mu lam f0(|u|), with PSD 12 x 12 Hessian w w^T (x) mu lam K,
 * K = (f1/y)(I - n n^T) + (f1' - f1/y) u^ u^T.
 * MLS_EINVAL for mu < 0, eps_v <= 0 with mu > 0, or mu > 0 with neither the
 * contact plane nor bodies (call mls_set_forces with contact, or
 * mls_set_bodies, first; turning either off later suspends its term). */
mls_status mls_set_friction(mls_ctx* ctx, double mu, double eps_v);

/* Mesh-mesh contact (Eq. IP term B, Sec. 3.1, which takes IPC's barrier on
 * surface primitives without writing it out; the CCD filter of Sec. 3.9).
 * body [n_verts] HOST labels each vertex with its body (>= 0).  The surface
 * is the set of faces that belong to one tet only, their edges and their
 * vertices.  Every point-triangle pair (surface vertex, face) and edge-edge
 * pair of different bodies at distance d < dhat adds
 *     kappa b(d),  b(d) = -(d - dhat)^2 ln(d / dhat),
 * to E with the same h^2 factor as the elastic energy; d is the distance of
 * the closest points of the closed primitives.  The Hessian of each pair is
 * projected to the positive semi-definite cone (12 x 12 per pair).  The line
 * search's first step is also bounded by conservative advancement, which
 * keeps every pair of different bodies at >= 0.1 of its distance, and the
 * start iterate is x^t + a (x_tilde - x^t) with a that bound.
 * Blocks of H between vertices of different bodies go to spare slots of the
 * surface-vertex rows: spare slots per row (0 = 32).  Call after
 * mls_upload_mesh and before mls_upload_basis / mls_upload_cubature; it
 * rebuilds H's sparsity.  body = NULL turns mesh-mesh contact off.  With
 * mls_set_friction mu > 0 the pairs also carry friction (see there).
 * MLS_EINVAL for a negative label, dhat <= 0 or kappa <= 0, spare < 0, no
 * mesh, or an uploaded basis or cubature.  A timestep fails with MLS_ENOMEM
 * when a vertex touches more vertices of other bodies than its spare slots
 * hold. */
mls_status mls_set_bodies(mls_ctx* ctx, const int32_t* body, double dhat, double kappa, int32_t spare);

/* One implicit-Euler timestep.  DEVICE pointers:
 *   x [n][3] positions x^t, v [n][3] velocities v^t (read only),
 *   dx_out [n][3] receives x^{t+1} - x^t.
 * stats_out (HOST, may be NULL) receives iteration counts.  The start iterate
 * is x_tilde with Dirichlet vertices at x^t, or x^t when x_tilde is
 * infeasible.  MLS_EINVERTED if x^t itself is infeasible, MLS_ENOTCONV if the
 * Newton cap is hit (dx_out then holds the last iterate's displacement). */
mls_status mls_newton_step(mls_ctx* ctx, const double* x, const double* v, double dt,
                           double* dx_out, mls_stats* stats_out);

/* Same as mls_newton_step with HOST x, v and dx_out: copies x and v to the
 * device and dx back inside the call. */
mls_status mls_newton_step_host(mls_ctx* ctx, const double* x, const double* v, double dt,
                                double* dx_out, mls_stats* stats_out);

/* One BDF2 timestep (Sec. 3.1, Eq. IP with alpha = 4/9).  DEVICE pointers:
 *   x, v [n][3]            x^t and v^t,
 *   x_prev, v_prev [n][3]  x^{t-1} and v^{t-1} (read only),
 *   dx_out [n][3]          receives x^{t+1} - x^t.
 * The predictor is x_tilde = (4 x^t - x^{t-1}) / 3 + (2 dt / 9)(4 v^t - v^{t-1})
 * + (4/9) dt^2 g, and E = 1/2 |x - x_tilde|_M^2 + (4/9) dt^2 (Psi + B + D):
 * the implicit-Euler potential of the step 2 dt / 3, so the Newton loop,
 * its options, line search and stopping test (scaled by dt) are those of
 * mls_newton_step.  The caller forms v^{t+1} = (3 x^{t+1} - 4 x^t + x^{t-1}) / (2 dt).
 * Statuses as mls_newton_step. */
mls_status mls_newton_step_bdf2(mls_ctx* ctx, const double* x, const double* v, const double* x_prev,
                                const double* v_prev, double dt, double* dx_out, mls_stats* stats_out);

/* ---- Stage entry points: one step of the path on the context's state ----
 * These run single rows of the hot path so each can be checked on its own.
 * All array arguments are DEVICE pointers unless stated otherwise. */

/* Per-tet element evaluation (Sec. 4 Neo-Hookean, element-wise PSD
 * projection of dP/dF): for positions x [n][3] write, per tet e,
 *   energy [t]        vol_e psi(F_e)   (+inf where J <= 0)   (nullable)
 *   grad   [t][12]    d(vol psi)/dx_e, element DOF 3 a + c   (nullable)
 *   hess   [t][12][12] vol B^T [dP/dF]_+ B in the context's precision,
 *                      widened to float64                      (nullable) */
mls_status mls_eval_elements(mls_ctx* ctx, const double* x, double* energy, double* grad,
                             double* hess);

/* Assemble the gradient g [n][3] (float64, written to grad_out, nullable) and
 * the projected Hessian H (kept in the context) at x for the timestep whose
 * predictor uses x_t and v_t (all [n][3]) and step dt. */
mls_status mls_assemble(mls_ctx* ctx, const double* x, const double* x_t, const double* v_t,
                        double dt, double* grad_out);

/* Copy the assembled H out as HOST block-CSR: row_ptr [n+1], col [nnzb],
 * val [nnzb][3][3] (float64).  *nnzb receives the block count; pass NULL
 * arrays to query it first. */
mls_status mls_get_hessian(mls_ctx* ctx, int32_t* row_ptr, int32_t* col, double* val,
                           int64_t* nnzb);

/* y = H x with the assembled H in its storage precision (float64 in and out). */
mls_status mls_spmv(mls_ctx* ctx, const double* x, double* y);

/* z = M^{-1} r with the current preconditioner (float64 in and out). */
mls_status mls_precond_apply(mls_ctx* ctx, const double* r, double* z);

/* Solve H d = b by PCG from d = 0 to |r| <= rtol |b|: b, d [n][3] float64;
 * *iters and *rel_res (HOST, nullable) receive the iteration count and final
 * |r|/|b| of the recursively updated residual. */
mls_status mls_pcg_solve(mls_ctx* ctx, const double* b, double* d, double rtol, int max_iter,
                         int* iters, double* rel_res);

/* w = U q (prolongation, Eq. LBS): q [m][12] -> w [n][3]. */
mls_status mls_prolong(mls_ctx* ctx, const double* q, double* w);

/* z = U^T r (restriction): r [n][3] -> z [m][12]. */
mls_status mls_restrict(mls_ctx* ctx, const double* r, double* z);

/* Build the Galerkin operator A_c = U^T H U from the assembled H (summed in
 * float64 from H's stored values in every precision) and factor it (dense
 * Cholesky, float64).  A non-positive pivot retries the factorisation of
 * A_c + sigma diag(A_c) for sigma = 1e-7, 1e-5, 1e-3, 1e-1; MLS_ECHOL if the
 * last retry fails too.  mls_get_coarse returns the unshifted A_c. */
mls_status mls_build_coarse(mls_ctx* ctx);

/* Copy A_c (HOST, [12m][12m] float64, before factorisation) out. */
mls_status mls_get_coarse(mls_ctx* ctx, double* A);

/* Copy the Cholesky factor of the last coarse build out (stage entry point,
 * for testing the factorisation): L (HOST, [12m][12m] float64, row-major)
 * receives the lower triangle of L with L L^T = A_c (1 + sigma diag, see
 * mls_coarse_shift); the strict upper triangle is set to zero.
 * MLS_EINVAL without a factored coarse operator. */
mls_status mls_get_coarse_factor(mls_ctx* ctx, double* L);

/* *sigma (HOST) = the relative diagonal shift of the current coarse factor:
 * 0 when U^T H U factored as built, else the sigma of the retry that
 * succeeded (see mls_build_coarse).  MLS_EINVAL for a null argument. */
mls_status mls_coarse_shift(mls_ctx* ctx, double* sigma);

/* Energy E(x + alpha d) for the current timestep (after mls_assemble) and
 * whether the point is feasible (every J > 0 and every vertex above the
 * plane).  x, d DEVICE [n][3]; *E and *feasible HOST. */
mls_status mls_energy(mls_ctx* ctx, const double* x, const double* d, double alpha, double* E,
                      int* feasible);

/* Point-plane CCD step bound min(1, 0.9 min_v dist_v / (-n . d_v)) over
 * vertices approaching the plane; 1 without contact.  *alpha HOST. */
mls_status mls_ccd_bound(mls_ctx* ctx, const double* x, const double* d, double* alpha);

/* ---- Kernel timing (tracing) ---------------------------------------------
 * Opt-in CUDA-event timing of the library's kernel classes, recorded on the
 * context's stream around each launch of the enabled classes, for measuring
 * kernel durations inside a running timestep.  Events cost about a
 * microsecond per launch, so enable only the classes being measured. */
enum {
  MLS_PROF_ELEMENTS = 0,  /* per-tet energy/gradient/Hessian */
  MLS_PROF_ASSEMBLE = 1,  /* gradient gather + H assembly */
  MLS_PROF_SPMV = 2,      /* the PCG product kernel (H z, direction update, p.q) */
  MLS_PROF_PCG_UPDATE = 3,/* PCG vector update + block-Jacobi + dots */
  MLS_PROF_PRECOND = 4,   /* two-level preconditioner kernels */
  MLS_PROF_GALERKIN = 5,  /* U^T H U */
  MLS_PROF_CHOLESKY = 6,  /* coarse factorisation and inverse */
  MLS_PROF_LINESEARCH = 7,/* energy / CCD / norm reductions */
  MLS_PROF_PCG_FUSED = 8, /* the persistent PCG kernel (one launch per solve) */
  MLS_PROF_COUNT = 9
};

/* Enable timing for the classes whose bits are set in mask (bit k = class k;
 * 0 disables) and reset the accumulated totals. */
mls_status mls_profile_enable(mls_ctx* ctx, uint32_t mask);

/* Read accumulated totals: ms[MLS_PROF_COUNT] milliseconds and
 * launches[MLS_PROF_COUNT] launch counts (HOST arrays, either nullable). */
mls_status mls_profile_read(mls_ctx* ctx, double* ms, int64_t* launches);

/* Mesh-mesh contact pairs (stage entry point, for testing): the broad and
 * narrow phase over x [n][3] (DEVICE) with d = NULL (pairs of different
 * bodies at distance < dhat), or over the segment x -> x + d (d DEVICE
 * [n][3]: every pair whose boxes, grown by dhat, meet on the segment, the
 * candidates of the CCD filter and the line search).  Writes up to cap
 * pairs each as HOST int32 [cap][4]: point-triangle (v, a, b, c) and
 * edge-edge (p0, p1, q0, q1) vertex indices; *npt and *nee receive the full
 * counts.  MLS_EINVAL without mls_set_bodies. */
mls_status mls_contact_pairs(mls_ctx* ctx, const double* x, const double* d, int64_t cap, int32_t* pt, int64_t* npt,
                             int32_t* ee, int64_t* nee);

/* Distance derivatives of n primitive pairs (for testing; no context).
 * DEVICE arrays: kind [n] (0 point-triangle with X = (p, a, b, c), 1
 * edge-edge with X = (p0, p1, q0, q1)), X [n][4][3]; outputs dist [n],
 * grad [n][12] and hess_d [n][12][12] of the distance over the 12 stacked
 * coordinates (the formula of the closest feature: plane, line or point),
 * and hess_b [n][12][12] = kappa (b''(d) grad grad^T + b'(d) hess_d)
 * projected to the positive semi-definite cone.  Runs on the legacy
 * default stream and waits.  MLS_EINVAL for n < 0, null arrays, dhat <= 0 or
 * kappa <= 0; MLS_ECUDA on a launch error. */
mls_status mls_contact_pair_derivatives(const int32_t* kind, const double* X, int32_t n, double kappa, double dhat,
                                        double* dist, double* grad, double* hess_d, double* hess_b);

/* ---- Dense bf16 product on the tensor cores ------------------------------
 * Not in the paper: the matrix product under the learned warm start's
 * network (and exported so that it can be tested on its own).
 *   C[M x N] = A[M x K] B[N x K]^T
 * with A [M][lda] and B [N][ldb] bfloat16 row-major DEVICE arrays (K
 * contiguous; lda, ldb >= K and multiples of 8; 16-byte aligned) and C
 * float32 [M][ldc] (DEVICE, ldc >= N).  Products of bf16 values are exact
 * and sums accumulate in float32 (tcgen05 with a tensor-memory accumulator,
 * operands staged by TMA).  Waits for completion on stream (cudaStream_t,
 * NULL = legacy default).  MLS_EINVAL for bad sizes, pitches or alignment;
 * MLS_ETIMEOUT if a bounded device wait gave up (the result is then
 * undefined).  Calls from several host threads are serialised. */
mls_status mls_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B, int32_t ldb,
                         float* C, int32_t ldc, void* stream);

/* ---- Learned warm start: MLP trained and run by the library's kernels ----
 * Not in the paper (an extension): a 3-layer MLP, h1 = relu(x W1^T + b1),
 * h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3, maps coarse-state features to
 * the coarse increment of a timestep.  Products run on tensor cores with
 * BF16 weights and operands and FP32 accumulation; parameters are kept as
 * FP32 master copies updated by Adam (beta1 0.9, beta2 0.999, eps 1e-8) on
 * the loss 1/(2B) sum_b |y_b - t_b|^2.  Parameter layout (one flat FP32
 * array): W1 [h][in], b1 [h], W2 [h][h], b2 [h], W3 [out][h], b3 [out]. */
typedef struct mls_mlp mls_mlp;

/* Create a network with the given widths, batches of up to max_batch rows,
 * initial parameters init_params (HOST, flat layout above), kernels queued
 * on stream (cudaStream_t, NULL = legacy default). */
mls_status mls_mlp_create(mls_mlp** out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                          int32_t max_batch, const float* init_params, void* stream);
/* Free the network's device buffers; NULL is accepted. */
mls_status mls_mlp_destroy(mls_mlp* mlp);
/* Number of parameters (length of the flat array). */
int64_t mls_mlp_param_count(const mls_mlp* mlp);
/* Y [batch][out] = net(X [batch][in]); DEVICE float32 arrays; any batch size. */
mls_status mls_mlp_forward(mls_mlp* mlp, const float* X, int32_t batch, float* Y);
/* Loss gradient for one batch (batch <= max_batch) into grad_out (DEVICE,
 * flat layout, nullable); *loss_out (HOST, nullable) receives the loss. */
mls_status mls_mlp_gradients(mls_mlp* mlp, const float* X, const float* T, int32_t batch,
                             float* grad_out, double* loss_out);
/* One Adam update with the given gradient (DEVICE, flat layout). */
mls_status mls_mlp_adam_step(mls_mlp* mlp, const float* grad, float lr);
/* Train on minibatches: rows order[0..batch), order[batch..2 batch), ... of
 * X [n_samples][in] with targets T [n_samples][out] (DEVICE), order a DEVICE
 * int32 array of n_order sample indices (a shuffled epoch, drawn by the
 * caller); one Adam step per full minibatch.  *loss_out (HOST, nullable):
 * mean minibatch loss. */
mls_status mls_mlp_train(mls_mlp* mlp, const float* X, const float* T, int32_t n_samples,
                         const int32_t* order, int32_t n_order, int32_t batch, float lr,
                         double* loss_out);
/* Copy the FP32 master parameters to HOST. */
mls_status mls_mlp_get_params(mls_mlp* mlp, float* host_params);
/* Standardise inputs and targets inside the network: inputs enter as
 * (x - mean_in) / std_in, training targets as (t - mean_out) / std_out, and
 * mls_mlp_forward returns y std_out + mean_out.  DEVICE float arrays (copied);
 * non-positive standard deviations are treated as 1.  All NULL: no
 * standardisation. */
mls_status mls_mlp_set_normalization(mls_mlp* mlp, const float* mean_in, const float* std_in,
                                     const float* mean_out, const float* std_out);
/* Column means and standard deviations (population) of DEVICE X [n][d]
 * into DEVICE mean [d], sd [d]. */
mls_status mls_mlp_column_stats(const float* X, int32_t n, int32_t d, float* mean, float* sd,
                                void* stream);

/* ---- Warm start from the coarse state ------------------------------------
 * Coarse coordinates q(x) = (U^T M U)^{-1} U^T M (x - X) of the uploaded SMS
 * basis.  While enabled, every mls_newton_step records q(x^t) in a history and
 * forms the features f = [q^t, q^{t-1}, q(X + h^2 g)] (the coarse coordinates of
 * the last two steps and of the gravity displacement);
 * when recording it also computes, after the step, the target
 * dq = (U^T H U)^{-1} U^T H (x^{t+1} - x_tilde) (the Galerkin coarse
 * projection of the step, H and its coarse factor taken at the first Newton
 * iterate; requires coarse_refresh >= the Newton count).  With a network
 * attached (3r inputs, r outputs, r = 12 handles) the step starts from
 * x_tilde + U dq_hat, dq_hat = net(f), when that point is feasible and has
 * lower energy than x_tilde; otherwise from x_tilde.  With bodies set
 * (mls_set_bodies) the candidate must also be reachable from x^t on a
 * straight path the CCD filter does not cut, and it is compared with the
 * start the step would otherwise take (x_tilde cut by the same filter).
 * The converged step does not depend on the start.  Not in the paper. */
/* enable: 0 off, 1 history/features (and prediction when a network is
 * attached), 2 as 1 plus recording targets (two-level preconditioner only).
 * The first enable factors U^T M U (float64 Cholesky). */
mls_status mls_warm_start_enable(mls_ctx* ctx, int enable);
/* Forget the history (start of a new trajectory). */
mls_status mls_warm_start_reset(mls_ctx* ctx);
/* Attach a trained network (not owned; NULL detaches). */
mls_status mls_warm_start_attach(mls_ctx* ctx, mls_mlp* mlp);
/* Copy the last step's features (DEVICE float [3r]) and target (DEVICE float [r]). */
mls_status mls_warm_start_sample(mls_ctx* ctx, float* features, float* target);
/* q(x) for DEVICE x [n][3] into DEVICE q [m][12] (float64). */
mls_status mls_coarse_project(mls_ctx* ctx, const double* x, double* q);

/* ---- Batched timestep of many independent meshes -----------------------
 * Advances B independent meshes by one implicit-Euler step each (the
 * timestep of mls_newton_step: projected Newton on the incremental potential,
 * Eq. 5, with the filtered line search of Sec. 3.9), solving every Newton
 * system with block-Jacobi PCG.  Each mesh keeps its own Newton and PCG
 * scalars, tolerances and stopping decisions; a finished mesh idles while the
 * others continue.  One timestep is one CUDA graph launch: the Newton, PCG
 * and line-search loops are WHILE conditional nodes whose conditions are set
 * on the device from the per-mesh states.  The first step times candidate
 * launch shapes of the PCG kernels on the assembled system and keeps the
 * fastest (mls_batch_retune forgets the choice).
 *
 * Options as for mls_create.  preconditioner: block Jacobi, or two-level
 * with per-mesh bases (mls_batch_upload_basis; the symmetric multiplicative
 * cycle with damping omega, coarse operators U_m^T H U_m built and factored
 * once per step at the start iterate, in float64, one block per mesh).
 * cycle, coarse_refresh and the persistent settings are ignored.  Forces (gravity, ground plane, barrier) are shared by
 * all meshes.  The batch owns a context and an internal stream, ordered after
 * opt->stream on every step.  Not in the paper. */
typedef struct mls_batch mls_batch;

typedef struct mls_batch_mesh_stats {
  int32_t status;             /* MLS_OK, MLS_ENOTCONV, MLS_ELINESEARCH, MLS_ENONFINITE, MLS_EINVERTED,
                                 MLS_ECHOL (a coarse block not positive definite after
                                 the diagonal-shift retries of mls_build_coarse) */
  int32_t newton_iters;
  int32_t pcg_iters;          /* summed over the mesh's Newton iterations */
  int32_t line_search_trials;
  double step_rel;            /* last |d|_inf / max(|x - x^t|_inf, h^2 |g|) */
  double grad_norm;           /* |g|_2 at the last Newton iteration */
  double energy;              /* E at the returned state */
} mls_batch_mesh_stats;

typedef struct mls_batch_info {
  int64_t kernel_launches;    /* kernels run by the step (graph nodes executed + 2) */
  int32_t graph_launches;     /* graph launches of the step (1) */
  int32_t newton_rounds;      /* Newton loop bodies run (max Newton count over meshes) */
  int32_t pcg_rounds;         /* PCG loop bodies run (2 iterations each) */
  int32_t line_search_rounds; /* line-search loop bodies run */
  int32_t spmv_lanes;         /* tuned lanes per row of the product (4 or 8) */
  int32_t row_threads;        /* tuned threads per block of the row kernels */
  int32_t rows_per_thread;    /* tuned rows per thread of the row kernels */
  double tune_ms;             /* time spent timing candidates (first step) */
} mls_batch_info;

/* Create an empty batch with options opt (HOST; NULL = mls_default_options)
 * on opt->stream.  MLS_EINVAL for invalid options, MLS_ENOMEM / MLS_ECUDA when
 * the context or the internal stream cannot be made. */
mls_status mls_batch_create(mls_batch** out, const mls_options* opt);
/* Free the batch, its context, graph and device buffers; NULL is accepted. */
mls_status mls_batch_destroy(mls_batch* b);
/* The message of the batch's last failing call (owned by the batch, valid
 * until its next call); "" when there is none. */
const char* mls_batch_last_error(const mls_batch* b);
/* B meshes concatenated: mesh m owns vertices [vert_offsets[m],
 * vert_offsets[m+1]) and tets [tet_offsets[m], tet_offsets[m+1]); tets hold
 * GLOBAL vertex indices of the concatenation, each tet within its own mesh.
 * rest_xyz [V][3], tets [T][4], youngs/poisson/density [T], dirichlet [V]
 * (nullable), all HOST arrays, copied.  MLS_EINVAL for an empty mesh, a tet
 * crossing meshes, or anything mls_upload_mesh rejects. */
mls_status mls_batch_upload(mls_batch* b, int32_t n_meshes, const int32_t* vert_offsets,
                            const int32_t* tet_offsets, const double* rest_xyz, const int32_t* tets,
                            const double* youngs, const double* poisson, const double* density,
                            const uint8_t* dirichlet);
/* Per-mesh SMS bases (Sec. 3.5-3.6) for two-level preconditioning: mesh m
 * owns handles [handle_offsets[m], handle_offsets[m+1]) (1 to 128 per mesh);
 * origins [n_handles][3]; vrow [V+1], handle [nnz] (global handle ids, each
 * vertex's handles within its own mesh), phi [nnz] in the batch's vertex
 * numbering; HOST arrays, copied.  MLS_EINVAL on any violation. */
mls_status mls_batch_upload_basis(mls_batch* b, int32_t n_handles, const int32_t* handle_offsets,
                                  const double* origins, const int32_t* vrow, const int32_t* handle,
                                  const double* phi);
/* Loads shared by every mesh: the arguments and errors of mls_set_forces
 * (Eq. IP: gravity in the predictor, the point-plane barrier B).  The next
 * step rebuilds its graph. */
mls_status mls_batch_set_forces(mls_batch* b, const double* gravity, int contact, const double* plane_n,
                                double plane_o, double dhat, double kappa);
/* Lagged point-plane friction for every mesh of the batch: the term and the
 * arguments of mls_set_friction (Eq. IP, term D), with the mollifier width
 * eps_v dt of each step's dt.  Call after mls_batch_set_forces with contact;
 * the next step rebuilds its graph.  MLS_EINVAL as mls_set_friction. */
mls_status mls_batch_set_friction(mls_batch* b, double mu, double eps_v);
/* Forget the tuned launch shape: the next step times the candidates again
 * and rebuilds its graph. */
mls_status mls_batch_retune(mls_batch* b);
/* One timestep of every mesh from DEVICE x, v [V][3] (float64, concatenated)
 * into DEVICE dx [V][3].  stats (HOST [B], nullable) receives per-mesh
 * results, info (HOST, nullable) the launch counts.  Returns MLS_OK when every
 * mesh succeeded, else the status of the first failing mesh (dx is written
 * for all meshes; a mesh with MLS_ENOTCONV returns its last iterate). */
mls_status mls_batch_step(mls_batch* b, const double* x, const double* v, double dt, double* dx_out,
                          mls_batch_mesh_stats* stats, mls_batch_info* info);
/* One BDF2 timestep of every mesh (Sec. 3.1, Eq. IP with alpha = 4/9), as
 * mls_newton_step_bdf2 for each mesh: DEVICE x, v [V][3] (x^t, v^t) and
 * x_prev, v_prev [V][3] (x^{t-1}, v^{t-1}), concatenated like x.  The first
 * call allocates two history buffers of [V][3] float64 (kept until the
 * next mls_batch_upload or mls_batch_destroy).  Switching between this and
 * mls_batch_step rebuilds the step graph.  Statuses as mls_batch_step, and
 * MLS_ENOMEM when the history buffers cannot be allocated. */
mls_status mls_batch_step_bdf2(mls_batch* b, const double* x, const double* v, const double* x_prev,
                               const double* v_prev, double dt, double* dx_out, mls_batch_mesh_stats* stats,
                               mls_batch_info* info);

/* ---- Self-test of the bounded device wait -------------------------------
 * The persistent PCG kernel separates its phases with a grid barrier whose
 * wait is bounded: a block that polls more than a limit flags an error and
 * the kernel returns (the solve reports MLS_ETIMEOUT) instead of hanging.
 * This entry point exercises that path on its own: `blocks` co-resident
 * blocks of 256 threads each arrive once at a barrier expecting `expected`
 * arrivals, polling at most spin_limit times.  With expected <= blocks the
 * barrier releases (MLS_OK, *gave_up = 0); with expected > blocks every
 * block gives up (MLS_ETIMEOUT, *gave_up = blocks).  Allocates 128 bytes of
 * device memory for the call; waits on `stream` (a cudaStream_t, NULL =
 * legacy default).  MLS_EINVAL for non-positive arguments; MLS_ECUDA when
 * the blocks cannot all be resident.  Not in the paper. */
mls_status mls_selftest_barrier(int32_t blocks, int32_t expected, int32_t spin_limit, int32_t* gave_up,
                                void* stream);

/* ---- Allocation-free elastic energy ------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they run (a fixed memory budget, a
 * host framework that owns all device allocations, or code where an
 * allocation's implicit synchronisation is not allowed).  It needs no
 * context and calls no allocator: its reduction scratch is a file-scope
 * device array (about 48 KB per device that uses it, held until the library
 * is unloaded).
 *
 * Computes, with DEVICE pointers,
 *   *energy_out  = sum_e vol_e psi(F_e(x))  (the Neo-Hookean energy of
 *                  mls_eval_elements, summed in block order; rest shapes are
 *                  formed from rest_xyz on the fly)
 *   *invalid_out = number of tets skipped because an index lies outside
 *                  [0, n_verts), the rest volume is <= 0 or J <= 0
 * from rest_xyz [n_verts][3], x [n_verts][3], tets [n_tets][4] (int32),
 * mu, lam [n_tets] (Lame parameters).  Work is queued on stream (a
 * cudaStream_t, NULL = legacy default) and the call returns without waiting;
 * results are valid once the stream reaches that point.
 * Limits: n_tets <= MLS_NOALLOC_MAX_TETS, else MLS_EINVAL.  All calls share
 * the scratch: calls whose kernels can overlap on the GPU (other streams or
 * host threads on the same device) race and must be serialised.  The first
 * call on each device looks up the scratch address with that device current;
 * make it before any stream capture.  That address belongs to the device's
 * primary context and stays cached for the life of the process: after
 * cudaDeviceReset on a device, do not call this entry point on it again. */
#define MLS_NOALLOC_MAX_TETS (4096 * 256)
mls_status mls_elastic_energy_noalloc(int32_t n_verts, int32_t n_tets, const double* rest_xyz,
                                      const int32_t* tets, const double* mu, const double* lam,
                                      const double* x, double* energy_out, int32_t* invalid_out,
                                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MLS_H_ */
