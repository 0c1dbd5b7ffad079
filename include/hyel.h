/*
 * hyel.h -- C ABI of libhyel: one Newton step of the VMS / generalized-alpha
 * hyper-elastodynamics scheme on P1 tetrahedra, with the nested block
 * preconditioned FGMRES solve, on one NVIDIA GB300 (sm_103a).
 *
 * Method: J. Liu, A. L. Marsden, "A robust and efficient iterative method for
 * hyper-elastodynamics with nested block preconditioning" (arXiv:1809.06350).
 * Section, equation, algorithm and appendix references below are to that
 * paper; equations are named by their LaTeX labels.
 *
 * Conventions (every entry point):
 *   - The context's device is made current for the call and the caller's
 *     current device is restored before it returns.
 *   - Returns int: HYEL_OK (0) or a negative HYEL_E* code. After a non-zero
 *     return, hyel_last_error(ctx) holds a one-line message.
 *   - The caller owns every pointer it passes. Host arrays are copied before
 *     the call returns. Device arrays are borrowed for the duration of the call
 *     and must be valid on the context's device.
 *   - All device work is ordered on the CUDA stream given to hyel_create (or
 *     hyel_set_stream). A call synchronizes that stream only when it returns
 *     host-visible results (norms, statistics, convergence decisions).
 *   - The context allocates and owns its internal device workspace (mesh,
 *     matrix, Krylov bases); it never allocates outputs for the caller.
 *   - Vectors of the reduced linear system are ordered x = [x_v ; x_p]:
 *     x_v[3a+i] (node a, component i) then x_p[a]; length 4N.
 *   - Nodal vectors: u, v, udot, vdot are [N][3] interleaved; p, pdot are [N].
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef HYEL_H
#define HYEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HYEL_OK           0
#define HYEL_EINVAL      -1  /* invalid argument (null pointer, bad size, bad enum) */
#define HYEL_ECUDA       -2  /* a CUDA runtime call failed */
#define HYEL_ENOMEM      -3  /* device allocation failed */
#define HYEL_ENOCONV     -4  /* a solver level or Newton hit its iteration cap */
#define HYEL_EBREAKDOWN  -5  /* GMRES breakdown without convergence */
#define HYEL_ENAN        -6  /* NaN or Inf met in a norm */
#define HYEL_EINVERTED   -7  /* an element has J <= 0 (or V <= 0 at upload) */
#define HYEL_ESINGULAR   -8  /* a 3x3 diagonal block of A is singular */
#define HYEL_ESTATE      -9  /* call out of order (e.g. solve before assemble) */

typedef struct hyel_ctx hyel_ctx;

/* ---------------------------------------------------------------- inputs */

/* Volumetric model (§2, §5): Gibbs energy of the compressible neo-Hookean
 * model of §5.1 (rho(p) = rho0 (p + sqrt(p^2+kappa^2))/kappa,
 * beta(p) = 1/sqrt(p^2+kappa^2)), or the fully incompressible G_vol = p/rho0
 * of §5.2 (rho = rho0, beta = 0). */
enum { HYEL_VOL_GIBBS = 0, HYEL_VOL_INCOMPRESSIBLE = 1 };

/* Material (§2 constitutive relations, §5.1 and §5.2 energies).
 * Isochoric energy per unit reference volume:
 *   mu/2 (tr C~ - 3) + sum_{i=1..n_fibres} k1/(2 k2) (exp(k2 E_i^2) - 1),
 *   E_i = H_i : C~ - 1,  H_i = kd I + (1 - 3 kd) a_i (x) a_i.
 * tau_M = c_m h^e / (c rho0), h^e the longest reference edge of the element,
 * c = sqrt((kappa + 4 mu/3)/rho0) (Gibbs) or sqrt(mu/rho0) (incompressible)
 * evaluated with the element's mu, kappa (§3.1).
 * Per-element host arrays (length E) override the global values when given. */
typedef struct {
    int32_t vol_model;          /* HYEL_VOL_* */
    int32_t n_fibres;           /* 0 (neo-Hookean) or 2 (HGO) */
    double  rho0;               /* reference density */
    double  mu, kappa;          /* shear and bulk moduli (kappa unused if incompressible) */
    double  k1, k2, kd;         /* fibre stiffness, exponent, dispersion */
    double  c_m;                /* stabilization constant (paper: 1e-3) */
    double  body[3];            /* body force per unit mass b */
    const double *mu_e;         /* host [E] or NULL */
    const double *kappa_e;      /* host [E] or NULL */
    const double *k1_e;         /* host [E] or NULL */
    const double *k2_e;         /* host [E] or NULL */
    const double *fibre_a1;     /* host [E][3], required when n_fibres == 2 */
    const double *fibre_a2;     /* host [E][3], required when n_fibres == 2 */
} hyel_material;

/* Boundary data (eq. strong_form_dirichlet_u).
 * Dirichlet: u_i = g = value * s(t), v_i = dg/dt on the listed (node, comp),
 * s(t) = min(t / t_ramp, 1). Neumann: a dead nominal traction
 * H = p_max * s(t) * traction_dir on the listed reference triangles; it enters
 * R_m as -int N_A H_i dGamma_X (Appendix A), i.e. a third of each triangle's
 * reference area to each vertex. */
typedef struct {
    int64_t        n_dirichlet;
    const int32_t *dir_node;      /* host [n_dirichlet] */
    const int32_t *dir_comp;      /* host [n_dirichlet], 0..2 */
    const double  *dir_value;     /* host [n_dirichlet] or NULL (all zero) */
    int64_t        n_traction_tris;
    const int32_t *traction_tris; /* host [n_traction_tris][3] */
    double         traction_dir[3];
    double         p_max;
    double         t_ramp;        /* > 0 */
} hyel_bc;

/* Device state arrays (caller-owned). For hyel_assemble they hold stage
 * values: u, p, v at t_{n+alpha_f} and udot, pdot, vdot at t_{n+alpha_m}.
 * For hyel_newton_step they hold y_n and ydot_n on entry and y_{n+1},
 * ydot_{n+1} on return. Lengths: u, v, udot, vdot [3N]; p, pdot [N]. */
typedef struct {
    double *u, *p, *v;
    double *udot, *pdot, *vdot;
} hyel_state;

/* Time stepping and Newton control (§3.2, §3.3).
 * alpha_m = (3 - rho_inf)/(2 (1 + rho_inf)), alpha_f = gamma = 1/(1 + rho_inf).
 * Newton stops when ||R||/||R_(0)|| <= tol_r or ||R|| <= tol_a, ||R_(0)|| being
 * the residual norm at the predictor. rhs_literal = 0 uses the exact
 * right-hand side of eq. NR_smaller_eqn_1 (with the K_{.,udot} R_k terms);
 * 1 uses -[R_m ; R_p] as printed in step 5 of the multi-corrector stage. */
typedef struct {
    double  rho_inf;
    double  dt;
    double  t_n;
    double  tol_r, tol_a;
    int32_t l_max;
    int32_t rhs_literal;
} hyel_time_params;

/* Precision of the preconditioner levels (intermediate and inner solvers,
 * their SpMVs and Gram-Schmidt). The outer FGMRES, its Gram-Schmidt and
 * Givens, the residual assembly and the Newton update are always FP64.
 * HYEL_PREC_BF16S: as HYEL_PREC_FP32, except that the A-SpMVs of the A-solves
 * read each scaled 3x3 block of A as nine BF16 values times one FP32 scale
 * (s = max |entry|, stored entries = bf16_rn(float(a) / s)), accumulating in
 * FP32. B, C, D, the block-Jacobi inverses and diag(S^) stay FP32. */
enum { HYEL_PREC_FP64 = 0, HYEL_PREC_FP32 = 1, HYEL_PREC_BF16S = 2 };

/* One Krylov level: stop when ||r|| <= max(rtol ||b||, atol) or after maxit
 * iterations; restart every `restart` iterations. Zero initial guess. */
typedef struct {
    double  rtol, atol;
    int32_t maxit, restart;
} hyel_krylov_level;

/* Nested solver (§4.4): outer FGMRES on the scaled system with the SCR
 * preconditioner of Algorithm 1 (or the block variant block_precond selects);
 * `a` controls the two intermediate A-solves (eq. seg_sol_int_disp,
 * seg_sol_disp), `s` the Schur solve (eq. seg_sol_pres), right-preconditioned
 * as s_precond selects (point-Jacobi on diag(S^), S^ = D - C diag(A)^-1 B, by
 * default), and `inner` the A-solve inside the matrix-free S product
 * (Algorithm 2, eq. S_inner_A_eqn). A-solves are right-preconditioned as
 * a_precond selects (the inverses of the 3x3 node-diagonal blocks of A by
 * default).
 * graph = 1 (default): the whole nested solve is one CUDA graph whose Krylov
 * loops are device-driven `while` conditional nodes (no host round trip until
 * the solve ends); the graph is built once per context and parameter set.
 * graph = 0: the host drives the kernel-per-step loops, reading the level
 * state after every iteration. Both run the same kernels and give the same
 * iterates. With block-Jacobi A-solves (the default), each intermediate
 * A-solve is one cooperative launch of a persistent GMRES kernel on A M^-1 (M
 * the 3x3 block diagonal of A), and each S-solve, its inner A-solves
 * included, is one cooperative launch too, in both modes. check_every (>= 1)
 * is validated and otherwise unused. */
/* Preconditioner of the A-solves (intermediate and inner):
 * HYEL_APREC_BJACOBI: 3x3 block-Jacobi, folded into the operator (A M^-1) of a
 *   persistent GMRES kernel (the default);
 * HYEL_APREC_AMG: one V-cycle of smoothed-aggregation multigrid (the
 *   stand-in for the paper's algebraic multigrid, §4.4) as the right
 *   preconditioner of an FGMRES A-level: the coarse space holds the rigid-body
 *   modes of every aggregate (two 3x3 block-nodes each: translation and
 *   rotation), the prolongator is smoothed once by damped block-Jacobi,
 *   Galerkin levels, a degree-3 Chebyshev smoother, a dense inverse on the
 *   coarsest level (at most 96 block-nodes); the cycle runs in FP32 for FP64
 *   and FP32 levels alike (the level's own products keep its precision).
 *   The hierarchy's pattern is built once per mesh (on the host), its
 *   operators once per assembly (after the scaling, on the GPU);
 *   hyel_amg_info reports its levels;
 * HYEL_APREC_CHEB: the polynomial p(M^-1 A) M^-1 of degree a_cheb_degree
 *   (1..16), M the 3x3 block diagonal of A: that many steps of the Chebyshev
 *   iteration for A z = v from z = 0 on [lmin, lmax] from Ritz values of
 *   M^-1 A (12 Arnoldi steps in the M-inner product, FP32; lmax = 1.05
 *   theta_max, lmin = theta_min / 2 clamped to [lmax / 1000, lmax / 1.5]),
 *   rebuilt after every scaling of a new assembly. The polynomial reads A in
 *   FP32 with FP32 directions; the A-solves (GMRES on A p(M^-1 A) M^-1, one
 *   persistent launch each, the inner ones inside the S-solve) multiply by A
 *   in the level's precision (FP32 for HYEL_PREC_BF16S: no BF16 copy). For
 *   stiffness-dominated A, where block-Jacobi alone needs long GMRES cycles. */
enum { HYEL_APREC_BJACOBI = 0, HYEL_APREC_AMG = 1, HYEL_APREC_CHEB = 2 };
/* Preconditioner of the S-solve (§4.2):
 * HYEL_SPREC_JACOBI: diag(S^)^-1, S^ = D - C diag(A)^-1 B (the default);
 * HYEL_SPREC_CHEB: the polynomial p(diag(S^)^-1 S^) diag(S^)^-1 of degree
 *   s_cheb_degree (1..16) given by that many steps of the Chebyshev iteration
 *   for S^ z = v from z = 0 on an interval [lmin, lmax], with the explicit
 *   sparse S^ (distance-2 node pattern, see hyel_schur_hat_setup). lmax and an
 *   estimate of lmin come from Ritz values (hyel_schur_hat_setup);
 *   s_cheb_ratio = 0 uses that lmin (clamped to [lmax / 1000, lmax / 1.5]),
 *   s_cheb_ratio > 1 fixes lmin = lmax / s_cheb_ratio. Rebuilt after every
 *   scaling of a new assembly. A fixed linear operator, applied inside the
 *   persistent S-solve (one grid barrier per degree), which keeps P^-1 v_j
 *   for every Krylov vector (flexible form: x = Z y at the end of a cycle);
 *   the paper's own choice is algebraic multigrid built from S^ (§5). Not
 *   with a_precond = HYEL_APREC_AMG. */
enum { HYEL_SPREC_JACOBI = 0, HYEL_SPREC_CHEB = 1 };
/* The block preconditioner of the outer FGMRES (§4.2–4.4; the factorization
 * of eq. a_ldu_block_factorization):
 * HYEL_BLOCK_LDU: Algorithm 1 (P_SCR, the default): A xhat = r_v,
 *   S x_p = r_p - C xhat (the S-solve), A x_v = r_v - B x_p;
 * HYEL_BLOCK_DU: the upper triangular part [[A, B], [O, S]]: S x_p = r_p,
 *   A x_v = r_v - B x_p;
 * HYEL_BLOCK_D: the block diagonal [[A, O], [O, S]]: A x_v = r_v, S x_p = r_p;
 * HYEL_BLOCK_SIMPLE: H1 = H2 = diag(A)^-1, the paper's comparison baseline:
 *   A xhat = r_v, S^ x_p = r_p - C xhat with the explicit S^ (GMRES on S^ with
 *   the s-level controls, preconditioned by s_precond, one persistent launch;
 *   FP64 S^ values in FP64 levels, FP32 in mixed ones), x_v = xhat -
 *   diag(A)^-1 B x_p.
 * A-solves use the a-level controls, S-solves (matrix-free S, inner A-solves)
 * the s- and inner-level controls. */
enum { HYEL_BLOCK_LDU = 0, HYEL_BLOCK_DU = 1, HYEL_BLOCK_D = 2, HYEL_BLOCK_SIMPLE = 3 };
/* The inner A-solve of Algorithm 2 (the matrix-free S product):
 * HYEL_INNER_GMRES: GMRES on A M^-1 with the inner-level controls (default);
 * HYEL_INNER_CG_SYM: preconditioned CG on the symmetrized A_sym = (A + A^T)/2
 *   with the 3x3 block-Jacobi preconditioner of A_sym (the paper's conclusion:
 *   symmetrize the inner system and use CG), in the single-reduction form of
 *   Chronopoulos and Gear, stopping at ||r|| <= max(rtol ||b||, atol) with the
 *   inner-level controls (restart unused). The S product then applies
 *   S_sym = D - C A_sym^-1 B, an approximation of S that the outer FGMRES
 *   corrects. Needs a_precond = HYEL_APREC_BJACOBI. */
enum { HYEL_INNER_GMRES = 0, HYEL_INNER_CG_SYM = 1 };

typedef struct {
    hyel_krylov_level outer, a, s, inner;
    int32_t precision;      /* HYEL_PREC_* */
    int32_t check_every;
    int32_t graph;
    int32_t a_precond;      /* HYEL_APREC_* */
    int32_t s_precond;      /* HYEL_SPREC_* */
    int32_t s_cheb_degree;  /* HYEL_SPREC_CHEB: polynomial degree, 1..16 */
    double  s_cheb_ratio;   /* HYEL_SPREC_CHEB: 0 (estimated lmin) or lmax / lmin > 1 */
    int32_t block_precond;  /* HYEL_BLOCK_* */
    int32_t inner_solver;   /* HYEL_INNER_* */
    int32_t a_cheb_degree;  /* HYEL_APREC_CHEB: polynomial degree, 1..16 */
    int32_t reserved_;      /* must be 0 */
} hyel_solver_params;

typedef struct {
    int32_t status;         /* HYEL_OK or the failing code */
    int32_t outer_its;      /* FGMRES iterations */
    int64_t a_its, s_its, inner_its;       /* total iterations per level */
    int32_t a_solves, s_solves, inner_solves;
    double  rel_residual;   /* true ||r - A x|| / ||r|| of the scaled system */
    double  ms_setup, ms_solve;
} hyel_solve_stats;

typedef struct {
    int32_t status;
    int32_t iterations;     /* Newton corrections taken */
    int32_t converged;
    int32_t pad_;
    double  res_norm0, res_norm;
    int64_t outer_its, a_its, s_its, inner_its;
    double  ms_assemble, ms_solve, ms_total;
} hyel_newton_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`; all work goes to `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream). */
int hyel_create(hyel_ctx **out, int device, void *cuda_stream);
int hyel_destroy(hyel_ctx *ctx);
int hyel_set_stream(hyel_ctx *ctx, void *cuda_stream);
/* Message of the last failure on this context ("" if none). NULL ctx gives the
 * message of the last failed hyel_create on this thread. */
const char *hyel_last_error(const hyel_ctx *ctx);

/* ---------------------------------------------------------------- mesh */

/* Upload a P1 tetrahedral mesh (§3.1). X: host [n_nodes][3] reference
 * coordinates; tets: host [n_tets][4] node indices. Tetrahedra with negative
 * signed volume are reoriented; a zero-volume tetrahedron is HYEL_EINVERTED.
 * Builds the node-adjacency block pattern (SELL-32: rows in slices of 32), the
 * element-to-block-slot gather lists and the per-element reference geometry
 * (shape-function gradients, volume, tau_M). Replaces any previous mesh. */
int hyel_mesh_upload(hyel_ctx *ctx, int64_t n_nodes, const double *X,
                     int64_t n_tets, const int32_t *tets,
                     const hyel_bc *bc, const hyel_material *mat);

/* info[0] = N, [1] = E, [2] = nnzb (node-pair blocks), [3] = padded block
 * slots (multiple of 32), [4] = device bytes held by the context. */
int hyel_mesh_info(hyel_ctx *ctx, int64_t *info, int n);

/* ---------------------------------------------------------------- assembly */

/* What hyel_assemble computes: HYEL_RES the residual (the element pass that
 * Newton's stopping test needs, §3.3 step 2), HYEL_TAN the consistent tangent
 * (§3.3 step 4) with the residual and the right-hand side that come with it. */
#define HYEL_RES 1u
#define HYEL_TAN 2u

/* Assemble at a stage state (Appendix A; §3.3 steps 2 and 4): residuals R_m,
 * R_p (with traction at t_n + alpha_f dt) and, with HYEL_TAN in flags, the
 * consistent tangent blocks
 * A = K_{m,vdot} + (a_f g dt/a_m) K_{m,udot}, B = K_{m,pdot},
 * C = K_{p,vdot} + (a_f g dt/a_m) K_{p,udot}, D = K_{p,pdot}
 * (eq. def_matrix_A, def_matrix_D), stored internally with Dirichlet rows and
 * columns of constrained velocity components replaced by identity.
 *   flags    HYEL_RES (residual only: the stored blocks are left as they
 *            were), HYEL_TAN or HYEL_RES | HYEL_TAN (residual and tangent);
 *            anything else is HYEL_EINVAL.
 *   res_out  device [4N] or NULL: [R_m ; R_p], zero on Dirichlet components.
 *   rhs_out  device [4N] or NULL: right-hand side of eq. NR_smaller_eqn_1
 *            (or the literal step-5 form), zero on Dirichlet components;
 *            needs HYEL_TAN (HYEL_EINVAL otherwise).
 *   norms_out host [4] or NULL: ||R||, ||R_k||, ||R_p||, ||R_m|| over free
 *            components, R_k = udot_{n+am} - v_{n+af}. (Synchronizes.)
 * Returns HYEL_EINVERTED if some element has J <= 0 (then outputs are void). */
int hyel_assemble(hyel_ctx *ctx, const hyel_time_params *tp, const hyel_state *stage, unsigned flags,
                  double *res_out, double *rhs_out, double *norms_out);

/* Copy the assembled (unscaled) blocks to host arrays in block-CSR order:
 * row_ptr [N+1], col [nnzb] (ascending within a row), A [nnzb][3][3]
 * (row-major), B [nnzb][3], C [nnzb][3], D [nnzb]. Any pointer may be NULL. */
int hyel_matrix_download(hyel_ctx *ctx, int32_t *row_ptr, int32_t *col,
                         double *A, double *B, double *C, double *D);

/* ---------------------------------------------------------------- operators */

enum { HYEL_OP_FULL = 0, HYEL_OP_A = 1, HYEL_OP_B = 2, HYEL_OP_C = 3, HYEL_OP_D = 4, HYEL_OP_AM = 5,
       HYEL_OP_SHAT = 6 };
enum { HYEL_MAT_ASSEMBLED = 0, HYEL_MAT_SCALED64 = 1, HYEL_MAT_SCALED32 = 2, HYEL_MAT_TRANSPOSED = 3,
       HYEL_MAT_SCALED_BF16S = 4 };

/* y = op(M) x on device vectors. FULL: [4N] -> [4N]; A: [3N] -> [3N];
 * B: [N] -> [3N]; C: [3N] -> [N]; D: [N] -> [N]. x, y are double for the
 * FP64 matrices and float for HYEL_MAT_SCALED32. Scaled matrices exist after
 * hyel_solve_setup (or a solve) on the current assembly.
 * HYEL_MAT_TRANSPOSED (FULL only): y = [[A^T, C^T], [B^T, D^T]] x, the
 * transpose of the assembled operator, built on first use after each
 * assembly (the block pattern is symmetric; block (i, c) of the transpose is
 * taken from block (c, i)).
 * HYEL_MAT_SCALED_BF16S (A and AM only, float x and y): the BF16-with-block-
 * scale copies described at HYEL_PREC_BF16S.
 * AM ([3N] -> [3N], scaled matrices only): y = A M^-1 x with M the 3x3 block
 * diagonal of the scaled A, i.e. A right-preconditioned by block-Jacobi; the
 * A-solves iterate on this operator (stored block by block as A_(r,c) M_c^-1).
 * SHAT ([N] -> [N], HYEL_MAT_SCALED64 or HYEL_MAT_SCALED32): y = S^ x with
 * the explicit S^ of hyel_schur_hat_setup (HYEL_ESTATE before it).
 * x and y must be distinct, non-overlapping ranges (HYEL_EINVAL otherwise):
 * each row reads entries of x that other rows' threads are writing into y. */
int hyel_spmv(hyel_ctx *ctx, int op, int matrix, const void *x, void *y);

/* Prepare the scaled system for the current assembly (§4.1): W_ii =
 * |A_ii|^-1/2 (1 if |A_ii| < 1e-15), scaled FP64 and FP32 blocks, the
 * BF16-with-block-scale copy of the scaled A, 3x3
 * block-Jacobi inverses of A and diag(S^). w_out: device [4N] or NULL. */
int hyel_solve_setup(hyel_ctx *ctx, double *w_out);

/* Explicit S^ = D - C diag(A)^-1 B of the scaled system (§4.2, the matrix
 * the paper builds the S-solve's preconditioner from), diag(A) the scalar
 * diagonal of the scaled A. Runs hyel_solve_setup if needed, then (unless
 * current for this assembly) sums S^ on the GPU on the distance-2 node
 * pattern (row i couples i with every node two block-graph steps away; the
 * pattern and the per-contribution entry positions are built on the host on
 * first use for the mesh) in FP32 from the FP32 scaled blocks (an FP64 copy is
 * summed from the FP64 blocks on the first FP64 use), and estimates the spectrum of
 * diag(S^)^-1 S^: 12 Arnoldi steps (two classical Gram-Schmidt passes each)
 * on |M|^-1/2 S^ |M|^-1/2, M = diag(S^), from x0_i = 2 u_i - 1 (u_i the top 53
 * bits of output i of SplitMix64 seeded with 0, over 2^53); the eigenvalues
 * theta of the symmetric part of the 12 x 12 Hessenberg matrix give
 * lmin = theta_min / 2 and lmax = 1.05 theta_max (in FP32, sums across
 * blocks in FP64). Synchronizes.
 *   bounds_out host [2] or NULL: lmin, lmax.
 *   info       host [n_info] or NULL: [0] nonzeros of S^, [1] padded slots,
 *              [2] summed contributions, [3] longest row.
 * HYEL_EINVAL if a row is longer than 800 entries; HYEL_ENAN if the Arnoldi
 * run meets NaN/Inf or no positive Ritz value. */
int hyel_schur_hat_setup(hyel_ctx *ctx, double *bounds_out, int64_t *info, int n_info);

/* y = p(diag(S^)^-1 S^) diag(S^)^-1 x: `degree` steps of the Chebyshev
 * iteration for S^ y = x from y = 0 on the interval HYEL_SPREC_CHEB uses
 * (ratio = 0: the estimated one; ratio > 1: [lmax / ratio, lmax]), FP64
 * vectors. matrix: HYEL_MAT_SCALED64 (FP64 values of S^) or HYEL_MAT_SCALED32
 * (FP32 values, as inside the S-solve, where the polynomial reads S^ in FP32
 * at every precision). x, y: device [N] double, distinct, non-overlapping.
 * HYEL_ESTATE before hyel_schur_hat_setup on the current assembly; HYEL_EINVAL
 * for overlapping x and y, another matrix, degree outside 1..16 or another
 * ratio. Synchronizes. */
int hyel_schur_hat_cheb(hyel_ctx *ctx, int matrix, int32_t degree, double ratio, const double *x, double *y);

/* y = S x for the scaled system (Algorithm 2: D x - C A^-1 (B x)), the inner
 * A-solve controlled by params->inner, params->inner_solver (A_sym with CG)
 * and params->precision. x, y: device [N] double, distinct, non-overlapping
 * ranges (HYEL_EINVAL otherwise). */
int hyel_schur_apply(hyel_ctx *ctx, const hyel_solver_params *params,
                     const double *x, double *y, hyel_solve_stats *stats);

/* The HYEL_APREC_CHEB interval of M^-1 A for the current scaled system (runs
 * hyel_solve_setup if needed; built unless current). bounds_out: host [2]
 * (lmin, lmax) or NULL. Synchronizes. */
int hyel_a_cheb_setup(hyel_ctx *ctx, double *bounds_out);

/* y = p(M^-1 A) M^-1 x, the HYEL_APREC_CHEB polynomial of the given degree
 * (1..16) on the interval of hyel_a_cheb_setup, as inside the A-solves: FP32
 * A values and directions, FP64 residual and result. x, y: device [3N]
 * double, distinct, non-overlapping (HYEL_EINVAL otherwise). HYEL_ESTATE before
 * hyel_a_cheb_setup on the current assembly. Synchronizes. */
int hyel_a_cheb_apply(hyel_ctx *ctx, int32_t degree, const double *x, double *y);

/* The multigrid hierarchy of HYEL_APREC_AMG, the stand-in for the paper's
 * algebraic multigrid of §4.4 and §5 (built by the first solve that
 * selects it on the current mesh): info[0] = number of levels L (0 before
 * that solve), then per level l = 0..L-1 info[1 + 2l] = block-nodes (3
 * unknowns each; level 0 is the mesh's nodes) and info[2 + 2l] = stored 3x3
 * blocks. Writes at most n entries of the host array info; HYEL_EINVAL if
 * info is NULL or n < 1. */
int hyel_amg_info(hyel_ctx *ctx, int64_t *info, int n);

/* z = P^-1 r once, P the block preconditioner of params->block_precond on the
 * scaled system (§4.2–4.4), its sub-solves controlled by params (precision,
 * levels, A- and S-preconditioners) exactly as inside hyel_solve_nested.
 * r, z: device [4N] double ([v ; p] ordering), distinct, non-overlapping
 * (HYEL_EINVAL otherwise). stats: host or NULL (a, s and inner counts). Synchronizes. */
int hyel_block_precond_apply(hyel_ctx *ctx, const hyel_solver_params *params,
                             const double *r, double *z, hyel_solve_stats *stats);

/* ---------------------------------------------------------------- solve */

/* Solve A x = rhs for the last assembled matrix (§4): symmetric diagonal
 * scaling, FGMRES with the nested SCR preconditioner (or the block variant
 * params->block_precond selects), unscaling.
 * rhs, x: device [4N] double. stats: host or NULL. Returns HYEL_ENOCONV if the
 * outer solver reached its iteration cap (x then holds the last iterate). */
int hyel_solve_nested(hyel_ctx *ctx, const hyel_solver_params *params,
                      const double *rhs, double *x, hyel_solve_stats *stats);

/* One generalized-alpha time step (§3.3): predictor, then up to l_max Newton
 * corrections, each assembling, solving with hyel_solve_nested and updating
 * by eq. NR_smaller_eqn_2 and step 7. state: y_n, ydot_n in, y_{n+1},
 * ydot_{n+1} out (overwritten only on return). With Chebyshev preconditioners
 * the intervals estimated at the first correction are kept at the later ones
 * of the same step (S^ and A themselves are rebuilt every time). */
int hyel_newton_step(hyel_ctx *ctx, const hyel_time_params *tp,
                     const hyel_solver_params *sp, hyel_state *state,
                     hyel_newton_stats *stats);

/* ---------------------------------------------------------------- adjoint */

/* Replace the moduli of the uploaded mesh (mu, kappa, k1, k2; global or per
 * element) and recompute tau_M; geometry, models, rho0, c_m, body force and
 * fibre directions are kept. Invalidates the current assembly. */
int hyel_update_material(hyel_ctx *ctx, const hyel_material *mat);

/* Solve A^T x = rhs for the last assembled matrix: the nested solver of
 * hyel_solve_nested applied to the transposed blocks [[A^T, C^T], [B^T, D^T]]
 * (same scaling W; S^T = D^T - B^T A^-T C^T applied matrix-free). rhs, x:
 * device [4N], ordered [x_v ; x_p] as in hyel_solve_nested. */
int hyel_solve_nested_transpose(hyel_ctx *ctx, const hyel_solver_params *params,
                                const double *rhs, double *x, hyel_solve_stats *stats);

/* grad[e][k] -= sum over element e of lambda . dF_e/dtheta_k for the element
 * parameters theta = (mu, kappa, k1, k2), F = [R_k bar ; R_p ; R_m] the residual
 * of Appendix A at the stage state (R_k bar does not depend on theta).
 * lambda: device [7N] ordered [lam_k 3N | lam_p N | lam_m 3N] (Dirichlet
 * components are ignored); grad: device [E][4], accumulated. Synchronizes. */
int hyel_param_sensitivity(hyel_ctx *ctx, const hyel_state *stage, const double *lambda, double *grad);

/* One reverse step of the discrete adjoint of the generalized-alpha Newton
 * step (§3.2, §3.3) for an objective of the final state. state_n holds y_n,
 * ydot_n and state_np1 the converged y_{n+1}, ydot_{n+1} (device, read only).
 * ybar, ydotbar: device [7N] ([u|p|v] and [udot|pdot|vdot]), dJ/dy_{n+1} and
 * dJ/dydot_{n+1} on entry, dJ/dy_n and dJ/dydot_n on return. grad: device
 * [E][4] or NULL, accumulates dJ/dtheta. lambda_out: device [7N] or NULL, the
 * step's adjoint [lam_k | lam_p | lam_m]. The transposed linear system is
 * solved with `sp` (stats: that solve). Dirichlet constraints must be
 * homogeneous; their components carry zero adjoint. Leaves the context
 * without a valid assembly. */
int hyel_adjoint_step(hyel_ctx *ctx, const hyel_time_params *tp, const hyel_solver_params *sp,
                      const hyel_state *state_n, const hyel_state *state_np1, double *ybar,
                      double *ydotbar, double *grad, double *lambda_out, hyel_solve_stats *stats);

/* ---------------------------------------------------------------- profiling */

/* Kernel classes timed with CUDA events on the context's stream when enabled
 * (launches made while a solve runs as a CUDA graph are not timed).
 * HYEL_K_GMRES_A is the persistent A-solve kernel (one launch per
 * intermediate A-solve), HYEL_K_GMRES_S the persistent S-solve kernel (one
 * launch per S-solve, its inner A-solves included); their algorithmic bytes
 * are counted on the device per iteration (the operator's values and indices
 * plus the passes over the Krylov vectors) and added when the solve returns.
 * HYEL_K_SCHUR_HAT times the numeric S^ and its Ritz interval together.
 * HYEL_K_ASSEMBLE is the element pass with the tangent (Appendix A residual
 * and blocks), HYEL_K_ASSEMBLE_CORR the same pass that also forms the
 * K_{.,udot} R_k right-hand-side terms (the first correction of a step), and
 * HYEL_K_ASSEMBLE_RES the residual-only element pass (Newton's stopping
 * test). */
enum { HYEL_K_SPMV_A64 = 0, HYEL_K_SPMV_A32 = 1, HYEL_K_SPMV_FULL64 = 2,
       HYEL_K_ASSEMBLE = 3, HYEL_K_GATHER = 4, HYEL_K_SPMV_A16 = 5, HYEL_K_GMRES_A = 6,
       HYEL_K_GMRES_S = 7, HYEL_K_SCHUR_HAT = 8, HYEL_K_ASSEMBLE_RES = 9, HYEL_K_ASSEMBLE_CORR = 10,
       HYEL_K_NCLASSES = 11 };

/* enable != 0 starts event timing of the kernel classes (and clears the
 * totals); 0 stops it. */
int hyel_profile(hyel_ctx *ctx, int enable);
/* Totals since the last enable: ms[k], launches[k], algorithmic bytes[k] for
 * k < HYEL_K_NCLASSES (arrays of HYEL_K_NCLASSES, any may be NULL).
 * Synchronizes. */
int hyel_profile_read(hyel_ctx *ctx, double *ms, int64_t *launches, double *bytes);

/* ---------------------------------------------------------------- failure detection */

/* The persistent solver kernels (one cooperative launch per A-, S- or
 * S^-solve and per Ritz-interval estimate) synchronize their blocks with grid
 * barriers. Every wait at such a barrier is bounded: a block that waits
 * longer than the limit sets an abort word, every block leaves at its next
 * barrier, and the entry point returns HYEL_ECUDA with the context still
 * usable (no device fault, no lost context). The paper has no counterpart
 * (its solvers run on CPUs); the limit guards against a stalled or
 * pre-empted block turning into a hang of the whole device.
 * seconds: the limit, 1e-6 .. 60 (default 1). Takes effect at the next launch
 * (also in CUDA graphs already built: the limit is read from device memory
 * when a launch starts). Synchronizes. */
int hyel_set_wait_limit(hyel_ctx *ctx, double seconds);

/* Host-made fault injection for tests of the failure path above:
 * HYEL_FAULT_BARRIER_SKIP makes block 0 of the next persistent launch leave
 * one grid barrier without arriving, so the other blocks' waits run into the
 * limit and the call reports HYEL_ECUDA; one launch takes it, later ones run
 * normally. HYEL_FAULT_NONE withdraws a pending injection. Nothing here
 * faults the device or waits without a bound. Synchronizes. */
enum { HYEL_FAULT_NONE = 0, HYEL_FAULT_BARRIER_SKIP = 1 };
int hyel_inject_fault(hyel_ctx *ctx, int kind);

/* A measurement aid (the paper has no counterpart): one launch of a
 * compute-only kernel of independent FP64 FMA chains (no memory traffic in
 * its loop), 8 blocks of 256 threads per SM, each thread 8 chains of `iters`
 * FMAs (1 <= iters <= 2^24; HYEL_EINVAL otherwise). The caller times the
 * launch on the context's stream; *flops_out (host, or NULL) receives the
 * launch's FP64 flop count (2 per FMA), so that flops / time is the device's
 * FP64 FMA rate, the peak of the FP64-bound element kernel. sink: device [1]
 * double, never written in practice (it keeps the chains alive). Stream-
 * ordered, no synchronization. */
int hyel_fp64_fma_probe(hyel_ctx *ctx, int64_t iters, double *sink, double *flops_out);

/* A measurement aid (the paper has no counterpart): one launch that reads
 * `bytes` of the device buffer `buf` once with 16-byte loads (8 blocks of 256
 * threads per SM, grid-stride), the plain streaming read of that size. Timed
 * by the caller like the SpMVs, it gives the read rate a kernel reading that
 * many bytes once can reach, launch ramp and tail included. bytes: a positive
 * multiple of 16; buf: 16-byte aligned (HYEL_EINVAL otherwise). sink: device
 * [1] double, never written in practice. Stream-ordered. */
int hyel_stream_read_probe(hyel_ctx *ctx, const void *buf, int64_t bytes, double *sink);

/* Number of kernel launches this library has issued in the process so far
 * (all contexts). count: host. */
int hyel_launch_count(int64_t *count);

/* ---------------------------------------------------------------- no-allocation variant */

/* Residual norms of the coupled operator without any device allocation:
 * out[0] = ||b - M x||_2, out[1] = ||b||_2 with M = [[A, B], [C, D]] the
 * assembled (HYEL_MAT_ASSEMBLED) or scaled (HYEL_MAT_SCALED64, after
 * hyel_solve_setup) matrix. x, b: device [4N] double; out: device [2] double.
 * Stream-ordered, no synchronization.
 *
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory where they need a residual check (frameworks whose pool
 * allocator owns all device memory and forbids cudaMalloc beside it, callers
 * whose device-memory budget is spent, latency-critical loops where an
 * allocation costs more than the check). Its reduction scratch is a fixed
 * 128 KB file-scope device array, held by every GPU that loads the library
 * until the process exits; it calls no cudaMalloc, cudaFree or allocating
 * routine. Limit: N <= 1,048,576 nodes (HYEL_EINVAL beyond; HYEL_ESTATE with
 * no mesh). The first call on a device looks up the array's device address
 * and caches it for the process; make that first call before any stream
 * capture, and do not call again after a cudaDeviceReset of that device (the
 * cached address is then stale). All calls share the one array: calls whose
 * kernels overlap on the GPU (different streams or contexts at the same time)
 * race and give wrong results; serialize them. */
int hyel_residual_norm_static(hyel_ctx *ctx, int matrix, const double *x, const double *b, double *out);

#ifdef __cplusplus
}
#endif
#endif /* HYEL_H */
