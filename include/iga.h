/*
 * iga.h -- C ABI of the GB300 isogeometric Bratu library (libiga.so).
 *
 * The library assembles, on one GPU, the residual vector and Jacobian matrix of
 * the Galerkin weak form of the Bratu problem
 *      -div(kappa grad u) - lambda exp(u) = 0,  u = g on the boundary,
 * on a tensor-product NURBS space, and drives a Newton-Krylov solve.  It follows
 * the PetIGA paper (Dalcin, Collier, Vignal, Cortes, Calo):
 *   - B-spline bases (Sec. 2.1, Eqs. 1-3), tensor products (Sec. 2.2, Eq. 5),
 *     NURBS bases and derivatives (Sec. 2.3, Eqs. 6-7, drational);
 *   - the CSR adjacency pattern from BasisStencil (Sec. 2.5, Algorithm 2);
 *   - element-by-element Gauss-Legendre assembly (Sec. 2.7, Algorithm 3);
 *   - the geometry map, its inverse and spatial gradients (Appendix A);
 *   - the Bratu residual and Jacobian (Sec. 3.1, Eqs. residual and jacobian),
 *     with kappa = 1 unless a log-kappa field is given (an extension);
 *   - the problem set-up calls of Sec. 3.2 (IGASetDim/SetDof/SetFromOptions/
 *     SetUp, IGASetBoundaryValue, IGASetFormFunction/Jacobian, SNESSolve).
 *
 * Conventions shared by every call:
 *   - Natural ordering (Sec. 2.2): the control variable of tensor index
 *     (i0, i1, i2) is A = i0 + n0*(i1 + n1*i2); rows and columns of the Jacobian
 *     use the same numbering.
 *   - Every compute call is asynchronous on the CUDA stream given to iga_create
 *     (NULL = the legacy default stream) unless stated otherwise.  Pointers
 *     documented as "device" must be device (or managed) memory of the current
 *     device; the library never frees caller memory.
 *   - No call throws; each returns an iga_status.  IGA_EINVAL means the
 *     arguments were rejected before any work was queued; nothing was written.
 *     iga_last_error() gives a one-line reason.
 *   - Results are deterministic: the kernels use no floating-point atomics and
 *     every sum is taken in a fixed order, so two calls with the same input give
 *     bit-identical output.
 */
#ifndef IGA_H
#define IGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iga_s *iga_t;

typedef enum {
  IGA_OK = 0,
  IGA_EINVAL = 1,    /* invalid argument or unsupported discretisation */
  IGA_ENOMEM = 2,    /* device allocation failed */
  IGA_ECUDA = 3,     /* a CUDA runtime call failed */
  IGA_ENOCONV = 4,   /* Newton did not reach the tolerance within its cap */
  IGA_EDIVERGED = 5, /* line search failed or the residual grew without bound */
  IGA_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  IGA_ENAN = 7       /* a NaN or Inf appeared in the input or in the iterates */
} iga_status;

typedef enum {
  IGA_FP64 = 0,     /* FP64 element arithmetic, FP64 values (double *) */
  IGA_JAC_TF32 = 1, /* element contraction with TF32 operands, FP32 accumulate; float * values */
  IGA_JAC_BF16 = 2, /* element contraction with BF16 operands, FP32 accumulate; float * values */
  IGA_JAC_FP32 = 3, /* global sum factorisation in FP32 on the CUDA cores; float * values */
  IGA_JAC_FD = 5,   /* local numerical differentiation, Sec. 2.8 Eq. (fdjac): forward differences
                       of the quadrature-point integrand in each element value, step
                       sqrt(eps) sqrt(1 + ||U_e||_2); FP64 (double *) values; 3D p <= 3, 2D p <= 4 */
  IGA_JAC_NONE = 4  /* Newton only: matrix-free Newton-Krylov, no assembled Jacobian; the Krylov
                       solver applies J(U) exactly on the fly (sum-factorised element passes,
                       iga_apply_jacobian_mf) with Jacobi preconditioning from
                       iga_form_jacobian_diagonal (the -snes_mf run of Sec. 2.8, with exact
                       products instead of finite differences) */
} iga_precision;

/* Discretisation (the IGASetDim / IGASetFromOptions data of Sec. 3.2).
 *  dim            2 or 3 (Sec. 3.2 IGASetDim); one scalar field (IGASetDof = 1).
 *  degree[d]      polynomial degree p, 1..4, equal in every direction.
 *  nel[d]         elements per direction (used when knots[d] == NULL).
 *  continuity[d]  inter-element continuity k, 0..p-1; -1 means p-1 (the default
 *                 space of Sec. 3.2 is C^{p-1}).  Used when knots[d] == NULL.
 *  knots[d]       explicit open knot vector of nknots[d] entries (host memory),
 *                 non-decreasing, p+1 repeated end knots; NULL: uniform on [0,1].
 *  quad[d]        Gauss-Legendre points per direction; 0 means p+1 (the rule of
 *                 Sec. 5 and App. C); only p+1 is supported.
 *  ctrl           host array N*dim of physical control points (natural order,
 *                 coordinates contiguous), or NULL for the identity map x = xi.
 *  weights        host array N of rational weights, or NULL for all ones.
 *  periodic[d]    0: not periodic.  k+1 (1..p): direction d is periodic with C^k
 *                 continuity across the boundary (Sec. 2.4): its open knot vector
 *                 (explicit or uniform) is unclamped by Eqs. (unclamp-left) and
 *                 (unclamp-right), the k+1 redundant functions are eliminated and
 *                 every function index wraps as mod(i, n-k) (Eq. map-wrap), so the
 *                 direction has n-k functions; needs n-k >= k+1.  N, ctrl, weights
 *                 and log-kappa count the wrapped functions only.  A periodic axis
 *                 takes no Dirichlet value; the pattern stays Algorithm 2's with
 *                 wrapped columns, ascending in each row.  Periodic handles assemble
 *                 the FP64 and FP32 Jacobians (IGA_FP64, IGA_JAC_FP32) and solve with
 *                 them; the element-matrix, matrix-free and no-allocation entry
 *                 points return IGA_EINVAL. */
typedef struct {
  int dim;
  int degree[3];
  int nel[3];
  int continuity[3];
  const double *knots[3];
  int nknots[3];
  int quad[3];
  const double *ctrl;
  const double *weights;
  int periodic[3];
} iga_desc;

/* Problem parameters: lambda of Eq. (strong), and an optional host array of N
 * log-kappa coefficients (kappa = exp(sum logkappa_A N_A); NULL: kappa = 1). */
typedef struct {
  double lambda;
  const double *log_kappa;
} iga_bratu;

/* Create a discretisation (IGACreate + IGASetUp of Sec. 3.2): validates the
 * description, builds knot vectors, Gauss rules and 1D basis tables, the CSR
 * pattern (Algorithm 2), and the per-quadrature-point geometry factors on the
 * device.  `stream` is a cudaStream_t (NULL: default stream); all library-owned
 * device memory is allocated here with cudaMalloc and freed by iga_destroy.
 * Synchronises the stream before returning.  On failure *out is NULL.
 * IGA_EINVAL also for more than 2^28 control variables (int32 column and
 * thread indices). */
iga_status iga_create(const iga_desc *desc, const iga_bratu *bratu, void *stream, iga_t *out);

/* IGASetBoundaryValue(iga, axis, side, 0, value) of Sec. 3.2: Dirichlet value on
 * the face `side` (0 = left, 1 = right) of parametric direction `axis`.  Rows of
 * boundary control variables become F_A = U_A - value and identity rows of the
 * Jacobian, with the column zeroed in the other rows (symmetric form).  When
 * faces meet, the face set later in the order (axis 0 side 0, axis 0 side 1,
 * axis 1 side 0, ...) gives the value.  A periodic axis has no faces: IGA_EINVAL. */
iga_status iga_set_boundary_value(iga_t iga, int axis, int side, double value);

/* Failure detection of the tensor-core Jacobian (a library facility; the paper has no
 * counterpart).  Every wait of its pipeline on a shared-memory barrier is bounded: after
 * `seconds` (default 2; accepted range (0, 60]) the kernel stops issuing copies and
 * tensor-core operations, waits at most 2 s more for those it has issued, frees its
 * tensor memory and returns, and the call (iga_form_jacobian, iga_solve_newton) reports
 * IGA_ETIMEOUT.  The handle stays usable; the next call runs normally. */
iga_status iga_set_wait_limit(iga_t iga, double seconds);

/* Test hook of that path: the next BF16/TF32 element-GEMM Jacobian on this handle waits
 * once, before issuing any work, on a barrier phase that nothing completes, so the wait
 * gives up after the limit and the call returns IGA_ETIMEOUT.  Later calls are unaffected.
 * Faults nothing: the give-up is the bounded wait's normal exit. */
iga_status iga_inject_stall(iga_t iga);

/* Form of the GMRES orthogonalisation (a library facility): fused = 1 (default) runs each
 * Arnoldi step's Gram-Schmidt passes, norm and Givens step as one cooperative launch when
 * the row partition fits the GPU's resident blocks (up to about 2.5M unknowns), else as
 * separate pass kernels; fused = 0 always takes the separate kernels (the same arithmetic
 * up to the norm's summation order).  Other values: IGA_EINVAL. */
iga_status iga_set_gmres_fused(iga_t iga, int fused);

/* Plan of the sum-factorised stiffness (a library facility): general = 0 (default) lets
 * create-time classification pick the diagonal-S plan where every off-diagonal S_ab of the
 * geometry cache is below 5e-13 of the diagonal (an orthogonal parametrisation such as the
 * annulus: those terms are zero in exact arithmetic); general = 1 always contracts every
 * term.  Other values: IGA_EINVAL. */
iga_status iga_set_jacobian_plan(iga_t iga, int general);

/* Change lambda after creation (used by the batched and learned-start drivers). */
iga_status iga_set_lambda(iga_t iga, double lambda);

/* Sizes and the device CSR pattern (library-owned, valid until iga_destroy):
 * rowptr int64[n+1], colidx int32[nnz], columns ascending within each row,
 * every BasisStencil entry present (explicit zeros included). */
iga_status iga_get_pattern(iga_t iga, int64_t *n, int64_t *nnz, const int64_t **rowptr,
                           const int32_t **colidx);

/* Residual F(U) of Eq. (residual), Algorithm 3, FP64.  U and F: device double[n],
 * caller-owned, must not overlap.  Dirichlet rows as set by iga_set_boundary_value. */
iga_status iga_form_residual(iga_t iga, const double *U, double *F);

/* Residual F(U) exactly as iga_form_residual, for callers that cannot allocate
 * device memory at call time (an allocator they do not own holds the device, a
 * real-time loop cannot take an allocation's latency or failure): this call
 * allocates nothing.  The paper has no counterpart; it is a library-level
 * variant.  Its element-vector scratch is a fixed array of
 * IGA_NOALLOC_MAX_ELEMENT_VALUES doubles (16 MiB) in the library's device memory.
 *  - iga_create (non-periodic handles) looks the array's address up on the current
 *    device; this loads the library code that holds the array and reserves its
 *    16 MiB on that device, which keeps it until the process exits.  Should that
 *    look-up fail at creation, the first call repeats it and may then be the one
 *    that reserves the array: make that call before any stream capture.
 *  - The current device must be the one that was current at iga_create
 *    (IGA_EINVAL otherwise).
 *  - Problems with elements x (p+1)^dim above the array's size are rejected with
 *    IGA_EINVAL (nothing is written); iga_form_residual has no such limit.
 *  - All calls share the array: calls that overlap on the GPU race.  Nothing in
 *    it needs to start at zero (every entry read was written by the same call).
 * U and F: device double[n], caller-owned, distinct; stream-ordered like the other
 * calls; the kernels are those of iga_form_residual, so the results are
 * bit-identical to it. */
#define IGA_NOALLOC_MAX_ELEMENT_VALUES 2097152u
iga_status iga_form_residual_noalloc(iga_t iga, const double *U, double *F);

/* Jacobian J(U) of Eq. (jacobian) into CSR values on the library's pattern.
 * vals: device memory, caller-owned, nnz entries of double (IGA_FP64, IGA_JAC_FD) or
 * float (IGA_JAC_TF32, IGA_JAC_BF16, IGA_JAC_FP32).  IGA_JAC_NONE is not a format:
 * IGA_EINVAL.  IGA_JAC_TF32 / IGA_JAC_BF16 synchronise the stream at the end to read the
 * tensor-core pipeline's give-up flag: IGA_ETIMEOUT (the values are then invalid) when
 * a bounded wait gave up (see iga_set_wait_limit). */
iga_status iga_form_jacobian(iga_t iga, const double *U, void *vals, iga_precision prec);

/* y = J x for CSR values on the library's pattern (the operator product of the
 * Krylov solvers of Sec. 5; PETSc's MatMult).  vals as written by
 * iga_form_jacobian: double for IGA_FP64, float for the other precisions (their
 * values are widened; x, y and the sums are FP64).  x and y: device double[n],
 * caller-owned, distinct.  Columns are not read: they follow from the stencil
 * structure of the pattern.  Stream-ordered, deterministic. */
iga_status iga_apply_jacobian(iga_t iga, const void *vals, iga_precision prec, const double *x, double *y);

/* y = J(U) x without assembling J: the linearisation of Eq. (residual) at U applied
 * to x by the same sum-factorised element passes as the residual (columns of
 * Dirichlet variables zero, identity Dirichlet rows), gathered per row in a fixed
 * order.  Equal to iga_form_jacobian(U) followed by iga_apply_jacobian up to
 * rounding.  U, x, y: device double[n], caller-owned, x != y.  Stream-ordered. */
iga_status iga_apply_jacobian_mf(iga_t iga, const double *U, const double *x, double *y);

/* d = diag(J(U)) (1 on Dirichlet rows) without assembling J: per element and local
 * function, the quadratic form of Eq. (jacobian) over the Gauss points, gathered
 * per row.  d: device double[n], caller-owned.  Stream-ordered. */
iga_status iga_form_jacobian_diagonal(iga_t iga, const double *U, double *d);

/* Newton-Krylov options (SNESSolve of Sec. 3.2; -snes_atol, -ksp_* analogues). */
typedef struct {
  double atol;         /* stop when ||F||_2 <= atol (default 1e-10) */
  int max_newton;      /* Newton iteration cap (default 50) */
  int gmres_restart;   /* GMRES(m) restart length (default 60) */
  int max_krylov;      /* Krylov iteration cap per Newton step (default 4000) */
  double krylov_rtol;  /* forcing term cap; the solve uses min(krylov_rtol, ||F_k||) (default 1e-2) */
  iga_precision jac;   /* Jacobian precision used to steer Newton (default IGA_FP64);
                          IGA_JAC_NONE: matrix-free (no assembled Jacobian) */
  int reuse_stiffness; /* 1: assemble the U-independent part K of J once per solve and add
                          the reaction term each step (default 1); every residual of the solve
                          (FP64 with every Jacobian type, except matrix-free, local ND and periodic
                          solves) is then the FP64 product K U plus the reaction term (equal to
                          Eq. (residual) up to rounding); 0: full assembly each step */
  int ksp;             /* Krylov method: IGA_KSP_GMRES (default) or IGA_KSP_CG (Jacobi-
                          preconditioned conjugate gradients, the -ksp_type cg run of App. B;
                          valid because the Jacobian with symmetric Dirichlet rows is symmetric) */
  int gmres_cgs_refine; /* second classical Gram-Schmidt pass of each GMRES (Arnoldi) step:
                          IGA_CGS_REFINE_NEVER (default: one pass, the default refinement type
                          of PETSc's GMRES, the solver behind the paper's SNESSolve),
                          IGA_CGS_REFINE_ALWAYS (classical Gram-Schmidt twice) or
                          IGA_CGS_REFINE_IFNEEDED (a second pass only when the first removes
                          at least half of ||w||^2, i.e. ||w - V h|| <= ||w|| / sqrt(2)); other
                          values: IGA_EINVAL.  Where the orthogonalisation runs as separate
                          pass kernels (iga_set_gmres_fused) IFNEEDED refines always. */
} iga_newton_opts;
#define IGA_KSP_GMRES 0
#define IGA_KSP_CG 1
#define IGA_CGS_REFINE_NEVER 0
#define IGA_CGS_REFINE_IFNEEDED 1
#define IGA_CGS_REFINE_ALWAYS 2

typedef struct {
  int newton_its;         /* Newton steps taken */
  int krylov_its;         /* total Krylov iterations */
  double fnorm0, fnorm;   /* ||F(U_0)||_2 and ||F(U_final)||_2 */
  double fnorm_hist[64];  /* ||F||_2 after each step (index 0 = initial) */
  iga_status status;      /* IGA_OK when ||F|| <= atol */
} iga_newton_report;

/* Fill opts with the defaults above. */
void iga_newton_defaults(iga_newton_opts *opts);

/* Solve F(U) = 0 by Newton with GMRES(m) + Jacobi (right preconditioning) on
 * the device, starting from U (device double[n], in/out).  Each step solves
 * J(U_k) dU = -F(U_k) to the forcing tolerance and backtracks (halving, at most
 * 10 times) until ||F|| decreases.  Synchronises the stream; fills *report
 * (may be NULL).  Returns report->status. */
iga_status iga_solve_newton(iga_t iga, double *U, const iga_newton_opts *opts,
                            iga_newton_report *report);

/* Same as iga_solve_newton with U in HOST memory: copies U to the device, solves,
 * copies the solution back. */
iga_status iga_solve_newton_host(iga_t iga, double *U_host, const iga_newton_opts *opts,
                                 iga_newton_report *report);

/* ---- Time-dependent problems: generalized-alpha (Sec. 4.2, Eq. ga) ----
 * The transient Bratu problem u_t - div(kappa grad u) - lambda e^u = 0 in the
 * semi-discrete form of Sec. 4.2: with U-dot the rates of the control variables,
 *   R_A(U-dot, U) = (N_A, u-dot^h) + [Eq. (residual)]_A   (rows without Dirichlet data),
 *   R_A = U_A - g_A                                        (Dirichlet rows; no U-dot),
 * u-dot^h = sum_B U-dot_B N_B, integrated by the same Gauss rule as Eq. (residual). */

/* R(V, U) with V = U-dot.  V, U, F: device double[n], caller-owned; F distinct from V
 * and U.  Stream-ordered, deterministic. */
iga_status iga_form_residual_ts(iga_t iga, const double *V, const double *U, double *F);

/* dR/dU + shift dR/dU-dot at U (the shifted Jacobian of an implicit time step): the
 * Jacobian of Eq. (jacobian) plus shift times the mass matrix (N_A, N_B), with the
 * Dirichlet fix of iga_form_jacobian.  vals: caller-owned device memory, nnz doubles
 * (IGA_FP64) or floats (IGA_JAC_FP32); other precisions: IGA_EINVAL. */
iga_status iga_form_jacobian_ts(iga_t iga, double shift, const double *U, void *vals, iga_precision prec);

typedef struct {
  double dt;       /* time step t_{n+1} - t_n, > 0 */
  double rho_inf;  /* spectral radius at dt -> infinity, in [0, 1]; 1 = implicit midpoint rule */
} iga_ts_opts;

/* One generalized-alpha step (Sec. 4.2, Eq. ga) with
 *   alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = 1 / (1 + rho_inf),
 *   gamma = 1/2 + alpha_m - alpha_f.
 * In: U = U_n, V = U-dot_n (device double[n], caller-owned, distinct; U_n should meet
 * the Dirichlet data and V_n be zero there).  Newton-Krylov (opts as for
 * iga_solve_newton; jac IGA_FP64, IGA_JAC_FP32 or IGA_JAC_NONE, others IGA_EINVAL) solves
 * R(U-dot_{n+alpha_m}, U_{n+alpha_f}) = 0 for W = U_{n+alpha_f} starting from W = U_n;
 * its Jacobian is the shifted one with shift alpha_m / (alpha_f gamma dt).  Out, when the
 * report's status is IGA_OK: U = U_{n+1}, V = U-dot_{n+1}; otherwise U and V keep
 * U_n and U-dot_n.  The U-independent stiffness is assembled on the first step and
 * kept by the later ones.  Synchronises the stream; returns report->status. */
iga_status iga_ts_alpha_step(iga_t iga, const iga_ts_opts *ts, double *U, double *V, const iga_newton_opts *opts,
                             iga_newton_report *report);

/* ---- Batched solves: many independent 2D problems in one persistent launch ----
 * Each instance i is a 2D Bratu problem described by descs[i] (dim 2, identity
 * map: ctrl = weights = NULL, equal degree 1..3 and equal knot vectors in both
 * directions; knots or nel/continuity as for iga_create) and params[i] (lambda,
 * optional host log-kappa of the instance's N_i control variables), with
 * homogeneous Dirichlet values on all four sides.  Instances with identical
 * descriptions share their tables and CSR pattern.  The paper solves one problem
 * per SNESSolve; the batch is this library's extension for many small problems.
 * iga_batch_create allocates every device buffer (cudaMalloc) and the work
 * arenas; its stream argument is unused (the batch runs on an internal stream). */
typedef struct iga_batch_s *iga_batch_t;
typedef struct {
  int solved;       /* instances that reached ||F|| <= atol */
  int *newton_its;  /* host arrays of length count, or NULL */
  int *krylov_its;
  double *fnorm;
  int *status;      /* iga_status per instance */
  double *solve_us; /* device time of each instance's solve in microseconds (%globaltimer
                       from the first to the last step of the CTA that solved it), or NULL */
} iga_batch_report;
iga_status iga_batch_create(int count, const iga_desc *descs, const iga_bratu *params, void *stream,
                            iga_batch_t *out);
/* offsets[count+1]: instance i owns U[offsets[i] .. offsets[i+1]) of the
 * concatenated solution array (natural order within an instance). */
iga_status iga_batch_offsets(iga_batch_t batch, int64_t *offsets);
/* Launch shape of the persistent kernel: CTAs per SM and threads per CTA (256 or 512;
 * ctas_per_sm * threads_per_cta <= 2048).  Default 1 x 512.  IGA_EINVAL otherwise.
 * The autotuner in paper_1305_4452_gb300/autotune.py chooses it. */
iga_status iga_batch_set_launch(iga_batch_t batch, int ctas_per_sm, int threads_per_cta);
/* Work-unit and tile shapes of the persistent kernel.
 * dot_chunks: each of the j+1 Gram-Schmidt dot products of an orthogonalisation pass is
 *   split into dot_chunks row ranges, one warp per (dot, range), their sums added in
 *   range order (0: as many ranges as keep every warp busy, at most 16).  Default 1 (one
 *   warp per dot).  Results depend on it only through the order of additions.
 * jac_lines: element tile of the Jacobian's first sum-factorisation stage (Eq. jacobian,
 *   axis 0): Gauss lines whose Q00 and kappa values are staged in shared memory at once,
 *   each pair-table value then serving that many lines (1, 2, 4 or 8; fewer when the
 *   lines of a large instance do not fit).  Default 4.  The Jacobian does not depend on
 *   it (same terms, same order).
 * Out-of-range values return IGA_EINVAL and change nothing.  The autotuner in
 * paper_1305_4452_gb300/autotune.py chooses both with the launch shape. */
iga_status iga_batch_set_tiles(iga_batch_t batch, int dot_chunks, int jac_lines);
/* Solve every instance from the initial values in U (device, concatenated,
 * in/out) with Newton + GMRES(m, at most 64) + Jacobi (Jacobi CG with
 * opts->ksp = IGA_KSP_CG), FP64 residual and norms, FP32 sum-factorised Jacobian.  One graph launch (captured on the first call
 * and replayed): argument copy, work-counter reset, the persistent kernel (each
 * CTA takes the next instance, largest first, until none is left) and the
 * report copy.  Synchronises the device.  Returns IGA_OK when every instance
 * converged, IGA_ENOCONV otherwise (see report->status). */
iga_status iga_batch_solve(iga_batch_t batch, double *U, const iga_newton_opts *opts, iga_batch_report *report);
void iga_batch_destroy(iga_batch_t batch);
const char *iga_batch_last_error(iga_batch_t batch);

/* ---- Learned initial guess: a convolutional neural operator (not in the paper) ----
 * An L-layer network of 3x3 convolutions (dilation dilations[l], zero padding) on
 * an height x width grid, in_channels inputs per grid point, `hidden` channels
 * between layers, SiLU activations and one linear output channel multiplied by a
 * mask.  Forward and input-gradient convolutions run as implicit GEMMs on the
 * tcgen05 tensor cores, weight gradients as im2col + mma.sync GEMMs, all BF16 x
 * BF16 -> FP32; master weights, gradients, Adam moments and the loss are FP32.
 * Parameters: a flat FP32 vector, per layer W[cout][3][3][cin] then b[cout].
 * Inputs are NHWC FP32 device arrays; batch size <= max_batch.  Shapes:
 * in_channels 1..16, hidden 16, 32 or 64, 2..16 layers, max_batch*height*width
 * <= 2^28; anything else is IGA_EINVAL before any device work.  iga_nn_create
 * allocates all device memory; weights are He-uniform from `seed`.
 * iga_nn_forward and iga_nn_loss_grad synchronise the stream; IGA_ETIMEOUT if a
 * tensor-core pipeline wait gave up (the call's outputs are then invalid). */
typedef struct iga_nn_s *iga_nn_t;
iga_status iga_nn_create(int height, int width, int in_channels, int hidden, int layers, const int *dilations,
                         int max_batch, uint64_t seed, void *stream, iga_nn_t *out);
iga_status iga_nn_num_params(iga_nn_t nn, int64_t *count);
iga_status iga_nn_get_params(iga_nn_t nn, float *host);        /* host float[count] */
iga_status iga_nn_set_params(iga_nn_t nn, const float *host);  /* also resets Adam */
/* y[B][H][W] = mask * net(x); x: device float[B][H][W][in_channels]; mask: device float[H][W] or NULL */
iga_status iga_nn_forward(iga_nn_t nn, const float *x, int B, const float *mask, float *y);
/* forward + backward of the masked mean-squared error against tgt[B][H][W]; *loss
 * (host) gets the loss; grads_out (device float[count]) gets the gradient if non-NULL */
iga_status iga_nn_loss_grad(iga_nn_t nn, const float *x, const float *tgt, const float *mask, int B, float *loss,
                            float *grads_out);
/* Loss = [sum mask (y-t)^2 + beta * sum over grid edges ((y-t)_i - (y-t)_j)^2] / sum mask:
 * beta >= 0 weights a discrete H1 seminorm of the error (default 0).  The Newton
 * residual of a guess is dominated by its oscillatory error, which this term targets. */
iga_status iga_nn_set_h1_weight(iga_nn_t nn, float beta);
/* one Adam update with the gradient of the last iga_nn_loss_grad */
iga_status iga_nn_adam_step(iga_nn_t nn, float lr, float beta1, float beta2, float eps);
void iga_nn_destroy(iga_nn_t nn);
const char *iga_nn_last_error(iga_nn_t nn);

/* Per-kernel-class launch counts and device times (the tracing facility; the
 * paper's -snes_monitor / -log_view analogue).  Classes, in order:
 *   0 geometry factors, 1 residual element kernel, 2 residual gather, 3 Q00 /
 *   u at Gauss points, 4 Jacobian stage 1, 5 Jacobian stage 2, 6 Jacobian final
 *   stage, 7 SpMV, 8 Gram-Schmidt multi-dot/update, 9 GMRES scalar kernels,
 *   10 vector kernels, 11 stiffness + reaction combine, 12 CSR pattern,
 *   13 tensor-core element matrices, 14 element-matrix gather, 15 the stiffness
 *   product K U of the split residual (class 7 is then the Krylov products alone).
 * iga_profile_enable(iga, mask): classes whose bit is set get a CUDA event pair
 * recorded around each launch on the library's stream (mask 0: timing off;
 * launches are always counted).  iga_profile_read synchronises the stream,
 * returns the totals since the last read (ms[c], timed[c] = timed launches,
 * launches[c] = all launches) and resets them. */
#define IGA_NCLASS 16
typedef struct {
  double ms[16];
  long long timed[16];
  long long launches[16];
} iga_profile;
iga_status iga_profile_enable(iga_t iga, unsigned mask);
iga_status iga_profile_read(iga_t iga, iga_profile *out);

/* ---- Roofline denominators (measurement; the paper has no counterpart) ----
 * Peak rates of the current device, measured by micro-benchmarks on `stream`
 * (a cudaStream_t, NULL: default stream):
 *   fp64_tflops  FP64 fused multiply-adds (CUDA cores, DFMA), flops = 2 per FMA;
 *   fp32_tflops  FP32 fused multiply-adds (FFMA);
 *   copy_gbs     device-to-device copy of a 512 MiB buffer, read + write bytes;
 *   sms          streaming multiprocessors of the device.
 * Each figure is the best of several launches timed with CUDA events (about 0.2 s
 * in all).  Allocates (and frees) 1 GiB of scratch; synchronises the stream.
 * IGA_ENOMEM or IGA_ECUDA on failure (*out unchanged). */
typedef struct {
  double fp64_tflops;
  double fp32_tflops;
  double copy_gbs;
  int sms;
} iga_peaks;
iga_status iga_measure_peaks(void *stream, iga_peaks *out);

/* y[i] = e^x[i], i < n, with the FP64 exponential that the residual, Q00 and reaction
 * kernels evaluate at the Gauss points (the Bratu term lambda e^u of Eq. residual and
 * Eq. jacobian): the table-driven method of Tang (ACM TOMS 1989), about one unit in the
 * last place.  x and y are device arrays of n doubles (caller-owned; they may be the same
 * array); stream-ordered on `stream`, no synchronisation.  n = 0 does nothing;
 * n < 0 or a NULL array with n > 0 returns IGA_EINVAL. */
iga_status iga_exp_eval(void *stream, const double *x, double *y, int64_t n);

/* Release every library-owned device buffer.  NULL is accepted. */
void iga_destroy(iga_t iga);

/* One-line description of the last error on this handle (or of the last failed
 * iga_create when iga == NULL).  Never NULL. */
const char *iga_last_error(iga_t iga);

#ifdef __cplusplus
}
#endif
#endif /* IGA_H */
