/*
 * bm.h - C ABI of the GB300 direct-indirect Burton-Miller solver for 2-D Helmholtz
 * transmission problems (Matsumoto & Matsushima, "Efficient LU factorization exploiting
 * direct-indirect Burton-Miller equation for Helmholtz transmission problems").
 *
 * The library assembles the Nystrom discretisation of either boundary integral system,
 * factors it and solves it on one GPU (sm_103a):
 *
 *  - the 3N x 3N direct-indirect ("mixed") system of Eq. dis_mixedBM (section 4), stored as
 *    its four dense blocks M13, M23, M31, M32 of Theorem thm:LU (section 4.1) - the two
 *    identity and three zero blocks are never materialised;
 *  - the 2N x 2N ordinary Burton-Miller system of Eq. dis_BM (section 4), the comparison.
 *
 * Factorisation of the mixed system follows Theorem thm:LU: U33 = -M31 M13 - M32 M23, then a
 * dense complex LU with partial pivoting of U33.  Solves with arbitrary 3N right-hand sides
 * follow Corollary lem:for_ssm_RHS.
 *
 * Conventions shared by every entry point:
 *  - Complex numbers are bm_c64 (interleaved re, im; FP64).  Right-hand sides and solutions
 *    are column-major with leading dimension >= the system size (3N mixed, 2N ordinary).
 *    Mixed unknowns are ordered (u, q, phi), ordinary ones (u, q).
 *  - Pointers flagged "on_device" are device pointers on the handle's device (for example
 *    torch data_ptr()); otherwise they are host pointers and the call copies through them.
 *  - The handle owns every device buffer it allocates (blocks, factors, pivots, workspace);
 *    the caller owns B, X, angles and outputs.  All work is enqueued on the handle's stream
 *    and calls return after the stream has finished the work they enqueued.
 *  - A handle is not thread-safe: use one handle per host thread.
 *  - Every function returns BM_OK (0) or an error code; bm_strerror names it and
 *    bm_last_error returns a message with the details of the most recent failure.
 */
#ifndef BM_H
#define BM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BM_OK = 0,
    BM_EINVAL = 1,      /* invalid argument (size, pointer, leading dimension, enum value) */
    BM_ENOMEM = 2,      /* request exceeds the handle's HBM budget, or a device allocation failed */
    BM_ESINGULAR = 3,   /* exactly zero pivot; *info holds the 1-based column (LAPACK style) */
    BM_ENOTCONV = 4,    /* iterative refinement did not reach refine_tol within refine_maxit */
    BM_ENONFINITE = 5,  /* NaN or Inf in an input (right-hand side, wavenumber, curve data) */
    BM_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    BM_ESTATE = 7,      /* call order violated (solve before factor, factor before assemble) */
    BM_ECUDA = 8        /* a CUDA runtime call failed; bm_last_error has its message */
} bm_status;

typedef enum { BM_MIXED = 0, BM_ORDINARY = 1 } bm_formulation;

/* Arithmetic of the factorisation.
 *  BM_FP64          : FP64 throughout (assembly, Schur GEMM, LU, solve).
 *  BM_CF32_TF32_IR  : FP64 assembly; Schur GEMM and LU trailing updates in complex TF32 on the
 *                     tensor cores (FP32 accumulation), panels and triangular solves in FP32;
 *                     FP64 residuals and iterative refinement to refine_tol (backward error).
 *  BM_CF32_3XTF32_IR: as above with each tensor-core product split hi/lo (3 TF32 products,
 *                     about FP32 accuracy), which needs fewer refinement steps. */
typedef enum { BM_FP64 = 0, BM_CF32_TF32_IR = 1, BM_CF32_3XTF32_IR = 2 } bm_precision;

typedef struct { double re, im; } bm_c64;

/* Curves, parametrised counter-clockwise over t in [0, 2 pi) (the normal nu = (y', -x')/|x'|
 * then points into the exterior domain, section 2.1):
 *  BM_CURVE_CIRCLE : p = {R, cx, cy, -}      x = (cx + R cos t, cy + R sin t)
 *  BM_CURVE_ELLIPSE: p = {a, b, -, -}        x = (a cos t, b sin t)
 *  BM_CURVE_STAR   : p = {r0, amp, lobes, -} x = (r0 + amp cos(lobes t)) (cos t, sin t)
 *  BM_CURVE_KITE   : p = {c, b, -, -}        x = (cos t + c cos 2t - c, b sin t)
 *  BM_CURVE_USER   : user = host array of 6N doubles, node-major
 *                    {x, y, x', y', x'', y''} at t_j = 2 pi j / N. */
typedef enum {
    BM_CURVE_CIRCLE = 0, BM_CURVE_ELLIPSE = 1, BM_CURVE_STAR = 2, BM_CURVE_KITE = 3, BM_CURVE_USER = 4
} bm_curve_kind;

typedef struct {
    int kind;
    double p[4];
    const double* user;
} bm_curve;

/* Options; pass NULL for the defaults.
 *  eps0          : exterior material constant (default 1).
 *  eps1, eps_set : interior material constant; if eps_set == 0 it is eps0 (k_in/k_out)^2,
 *                  from k_i = omega sqrt(eps_i) (section 2.1) with omega = k_out / sqrt(eps0).
 *  beta, beta_set: Burton-Miller constant (needs Im beta != 0, section 3.1); default i / k_out.
 *  prec          : bm_precision (default BM_FP64).
 *  refine_tol    : backward-error target of refinement (default 1e-9).
 *  refine_maxit  : refinement iteration cap (default 30).
 *  nb            : outer LU block size, a multiple of 32 in [32, 256] (0 = library default).
 *  refine_residual: how refinement forms r = b - A x (bm_refine_residual):
 *     BM_RESID_TC_UPDATE (0, default): the first residual from exact integer products on the
 *        tensor cores - A (once, after assembly) and x split into seven base-128 digits per row /
 *        column scale, digit pairs multiplied in bf16 with exact FP32 sums over chunks of 256 and
 *        double-float sums across chunks (FP64-level accuracy, ~1e-15 of |A||x|); later ones
 *        updated as r -= A d with the product in FP32 (d, the last correction, is small by then,
 *        so the update error stays far below refine_tol);
 *     BM_RESID_FP64_UPDATE (1): the first residual in FP64, later ones updated as above;
 *     BM_RESID_FP64_ALL (2): every residual in FP64;
 *     BM_RESID_DF_UPDATE (3): the first residual in double-float arithmetic on the FP32 cores (each
 *        FP64 operand split into two FP32 parts, exact products, compensated sums: ~1e-12 of
 *        |A||x|), later ones updated as in mode 0;
 *     BM_RESID_TC_ALL (4): every residual from exact tensor-core digit products as in mode 0, with
 *        nine digits per operand (~2^-64 of the row and column scales).
 *  The updated residuals of modes 0, 1 and 3 carry the FP32 product error of each update, so the
 *  backward error they track is reliable down to about 1e-12; refine_tol below 1e-12 needs
 *  BM_RESID_FP64_ALL or BM_RESID_TC_ALL (bm_assemble returns BM_EINVAL otherwise).
 * zeta_p: quadrature.  0 (default) is the one-point zeta-corrected rule of section 4.  1..20 adds
 *  the high-order zeta corrections of section 5.3 ("order 31" is zeta_p = 14): weights derived
 *  from the Euler-Maclaurin expansion of the punctured trapezoid sum (zeta'(-2k) for the log
 *  parts of S, D, D*, N; the two-term expansion of N's x^-2 part with a central second-derivative
 *  stencil) on the 2 zeta_p + 1 (log parts) and 2 zeta_p + 3 (N) nodes around each diagonal, for
 *  an O(h^(2 zeta_p + 3)) rule.  Needs N >= 2 zeta_p + 3, and |arg k| <= 60 degrees for both
 *  wavenumbers unless |k| (zeta_p + 1) h max|x'| < 2.9 (BM_EINVAL otherwise).
 * Launch and diagnostic settings (0 selects the default for each; none changes a result beyond
 * rounding order, except test_wait_timeout):
 *  eager             : 1 launches every kernel of bm_factor and of the refinement corrections directly
 *                      instead of replaying the CUDA graphs captured on first use (for profilers that
 *                      cannot replay graph-captured cluster launches).
 *  panel_cluster_max : cap on the CTAs of one LU panel cluster, 1 .. 16 (0: as many as the device
 *                      co-schedules).  Fewer CTAs put more rows on each thread.
 *  panel_kernel      : 0 runs FP32 panels on the lane-per-column kernel wherever it fits; 1 keeps them
 *                      on the register-row kernel (the kernel the FP64 path always uses).
 *  test_wait_timeout : test hook for the device-wait error path.  1 makes every tensor-core product
 *                      wait on a barrier that nothing completes; the wait gives up after about 1 ms,
 *                      the product skips its output and bm_factor returns BM_ETIMEOUT (the FP64
 *                      precision, which has no tensor-core product, is unaffected).  2 makes one wait
 *                      of the FP32 triangular solve wait on a flag that nothing sets; it gives up
 *                      after about 1 s, the rest of that solve stops waiting, and bm_solve returns
 *                      BM_ETIMEOUT.  Nothing is left running on the device, and the handle stays
 *                      usable after a new bm_assemble.  Other values: BM_EINVAL. */
typedef struct {
    double eps0;
    bm_c64 eps1;
    bm_c64 beta;
    int eps_set;
    int beta_set;
    int prec;
    double refine_tol;
    int refine_maxit;
    int nb;
    int refine_residual;
    int zeta_p;
    int eager;
    int panel_cluster_max;
    int panel_kernel;
    int test_wait_timeout;
} bm_opts;

typedef enum {
    BM_RESID_TC_UPDATE = 0, BM_RESID_FP64_UPDATE = 1, BM_RESID_FP64_ALL = 2, BM_RESID_DF_UPDATE = 3,
    BM_RESID_TC_ALL = 4
} bm_refine_residual;

/* Per-solve report.  Times are device times (CUDA events) of the solve's phases. */
typedef struct {
    int iterations;          /* refinement corrections applied (0 for BM_FP64) */
    double backward_error;   /* max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf),
                                A the FP64 assembled system; computed on the device in FP64 */
    double t_solve_ms;       /* whole bm_solve device time, including refinement */
    double t_residual_ms;    /* part of it spent in FP64 residuals */
} bm_solve_info;

typedef struct bm_ctx bm_ctx;

/* Create a handle on CUDA device `device`.  cuda_stream (a cudaStream_t, may be NULL) is the
 * stream all work is enqueued on; NULL makes the handle create and own a non-blocking stream.
 * hbm_budget_bytes bounds the device memory the handle may hold (0 = 90 % of free memory at
 * creation).  The Hankel Taylor table (about 3 MB, see bm_hankel_taylor_table) is built on the
 * host on first use and uploaded once per device and CUDA context by the first bm_create there;
 * every handle on the device shares that copy, which is not counted against any handle's budget
 * and lives as long as the context. */
bm_status bm_create(bm_ctx** out, int device, void* cuda_stream, size_t hbm_budget_bytes);

/* Assemble the Nystrom system (section 4, Eq. dis_mixedBM or Eq. dis_BM) for N nodes on the
 * curve, exterior/interior wavenumbers k_out = k0, k_in = k1 (complex; the principal branch is
 * used, Re k > 0 required).  Kernels of section 2.2 off the diagonal; the one-point
 * zeta-corrected diagonal of section 4 on it (opts->zeta_p > 0: plus the high-order corrections
 * on the band around it, see bm_opts).  The right-hand side of a plane wave is made by
 * bm_rhs_plane_wave.  Replaces any previous system and factorisation of the handle.
 * Errors: BM_EINVAL (N < 8, N > 65536, bad kind/params, Re k <= 0, |arg k| > 60 degrees),
 * BM_ENONFINITE, BM_ENOMEM (admission: the bytes the system and its factorisation need
 * exceed the budget; nothing is allocated then). */
bm_status bm_assemble(bm_ctx* ctx, const bm_curve* curve, int N, bm_c64 k_out, bm_c64 k_in,
                      bm_formulation formulation, const bm_opts* opts);

/* Factor the assembled system.  Mixed: U33 = -M31 M13 - M32 M23 (Theorem thm:LU), then
 * P U33 = L U with partial pivoting (pivot = first index of max |Re|+|Im|).  Ordinary: P A = L U
 * of the 2N matrix.  The assembled FP64 operator is kept for residuals.
 * *info (may be NULL) is 0, or the 1-based column of the first exactly zero pivot, in which
 * case BM_ESINGULAR is returned and bm_solve refuses to run.  Errors: BM_ESTATE. */
bm_status bm_factor(bm_ctx* ctx, int* info);

/* Right-hand sides of plane waves exp(i k0 (cos a, sin a).x) for nrhs incidence angles
 * (host array, radians): b3 = -u_in - beta du_in/dnu placed as (0, 0, b3) for the mixed
 * system (Theorem thm:LU) or (b3, 0) for the ordinary one (Eq. dis_BM).  B has ldb >= the
 * system size. */
bm_status bm_rhs_plane_wave(bm_ctx* ctx, const double* angles, int nrhs, bm_c64* B, int ldb,
                            int on_device);

/* Solve A X = B for nrhs right-hand sides (any 3N or 2N data; Corollary lem:for_ssm_RHS for
 * the mixed system).  FP64: one factored solve.  CF32 precisions: x0 from the FP32 factors,
 * then x += A^{-1}_{fp32} (b - A x) with the residual in FP64 until the backward error (as in
 * bm_solve_info) is <= refine_tol; BM_ENOTCONV if refine_maxit corrections do not get there
 * (X then holds the last iterate).  X may not alias B.  info may be NULL.
 * Errors: BM_ESTATE (not factored or singular), BM_EINVAL, BM_ENONFINITE (B not finite). */
bm_status bm_solve(bm_ctx* ctx, int nrhs, const bm_c64* B, int ldb, bm_c64* X, int ldx,
                   int on_device, bm_solve_info* info);

/* Solve the mixed system for the block-diagonal right-hand side diag(B1, B2, B3) of Corollary
 * lem:block_LU (§4.1, toward the leaf level of a fast direct solver): B1, B2, B3 are N x c1,
 * N x c2, N x c3 (ld >= N; a block with c = 0 may be NULL), X is 3N x (c1 + c2 + c3) (ldx >= 3N):
 *   X = [ B1 - M13 Z31   -M13 Z32        -M13 Z33 ]    Z31 = -U33^{-1} M31 B1
 *       [ -M23 Z31       B2 - M23 Z32    -M23 Z33 ]    Z32 = -U33^{-1} M32 B2
 *       [ Z31            Z32             Z33      ]    Z33 =  U33^{-1} B3,  U33 = -M31 M13 - M32 M23,
 * which is the Corollary lem:for_ssm_RHS solve of the block-diagonal columns: it runs as bm_solve
 * on them (same precision and refinement; info as bm_solve's).  B and X on the host or (on_device)
 * the device.  The device form stages the 3N x (c1 + c2 + c3) right-hand side in a buffer charged
 * to the HBM budget.  Errors: BM_ESTATE (not factored, or the ordinary formulation), BM_EINVAL,
 * BM_ENOMEM, and those of bm_solve. */
bm_status bm_solve_block(bm_ctx* ctx, int c1, const bm_c64* B1, int ld1, int c2, const bm_c64* B2, int ld2, int c3,
                         const bm_c64* B3, int ld3, bm_c64* X, int ldx, int on_device, bm_solve_info* info);

/* Diagnostic (host only, no GPU needed): the weights of the high-order zeta corrections for
 * zeta_p = p (1..20), as bm_assemble uses them.  tau[0..p]: tau[0] = sigma_0 = -2 sum tau_m (the
 * diagonal's log weight beyond ln(h/2pi)), tau[m] the log-part weight at offset +-m; c2[0..p+1]:
 * the central second-derivative stencil applied to N's x^-2 part.  Errors: BM_EINVAL. */
bm_status bm_zeta_weights(int p, double* tau, double* c2);

/* Far-field pattern of solutions X (nrhs columns, as returned by bm_solve) at M observation
 * angles: u_inf(xhat) = e^{i pi/4}/sqrt(8 pi k0) sum_j w_j [-i k0 (xhat.nu_j) u_j - eps0 q_j]
 * exp(-i k0 xhat.x_j), from the exterior Green representation of the total field
 * (section 3.1), normalised so that u_sc ~ e^{i k0 r} r^{-1/2} u_inf.  Uinf is M x nrhs,
 * column-major, ldu >= M.  angles is a host array.  Errors: BM_EINVAL, BM_ESTATE, BM_ENONFINITE (an
 * angle is not finite), BM_ENOMEM, BM_ECUDA. */
bm_status bm_far_field(bm_ctx* ctx, const bm_c64* X, int ldx, int nrhs, const double* angles,
                       int M, bm_c64* Uinf, int ldu, int on_device);

/* The far field of bm_far_field (same kernel, same result) for callers that must not allocate
 * device memory while they run; the paper has no counterpart, it is a library service.
 * bm_far_field allocates and frees a small device buffer for the angles on each call, charged to
 * the handle's HBM budget: once resident systems have used the budget up it fails with BM_ENOMEM,
 * and each allocation may have to grow the device's memory pool, which a caller holding a
 * fixed device-memory footprint (a serving loop sized to the GPU) cannot allow.  This call copies the
 * angles into a fixed device array of BM_FAR_FIELD_STATIC_MAX_ANGLES doubles (64 KB) built into
 * the library, and allocates nothing.
 *  X    : device array, nsys x nrhs column-major solutions (ldx >= nsys), as from bm_solve.
 *  Uinf : device array, M x nrhs column-major output (ldu >= M), fully overwritten.
 *  angles: host array of M observation angles (radians), 1 <= M <= BM_FAR_FIELD_STATIC_MAX_ANGLES.
 * Nothing in the fixed array needs to start at zero: each call writes the M angles it reads.
 * The first call on a device looks up the array's device address once for that device (and again
 * after the device's context has been replaced, e.g. by cudaDeviceReset); make it before any
 * stream capture starts on the device.  The array is shared by all handles and threads
 * on a device: calls that overlap in time race on it.  The call waits for the handle's stream
 * before it returns, so calls made one after another are safe.
 * Errors: BM_EINVAL (M above the limit - bm_last_error says so -, bad sizes or pointers),
 * BM_ENONFINITE (an angle is not finite), BM_ESTATE (nothing assembled), BM_ECUDA. */
#define BM_FAR_FIELD_STATIC_MAX_ANGLES 8192
bm_status bm_far_field_static(bm_ctx* ctx, const bm_c64* X, int ldx, int nrhs, const double* angles,
                              int M, bm_c64* Uinf, int ldu);

/* ---- Contour eigenvalue solver (section 5.3, sec:ssm) ----
 * The paper finds the complex omega at which the discretised system is singular with the
 * Sakurai-Sugiura projection method, solving the system at the quadrature points of a closed
 * contour for random right-hand sides (which Corollary lem:for_ssm_RHS serves for the mixed
 * system); it cites the method without its steps.  bm_ssm takes the block Hankel variant:
 *   points   z_p = center + radius zeta_p, zeta_p = exp(i 2 pi (p + 1/2) / npoints), p < npoints,
 *            in the k_out = omega plane (eps0 = 1), with k_in = k_ratio z_p (eps1 = k_ratio^2 fixed;
 *            beta = i / k_out unless opts fix it);
 *   moments  mu_k = sum_p w_p zeta_p^k V^H T(z_p)^{-1} V, w_p = radius zeta_p / npoints, k < 2M
 *            (L x L each; V holds L probe columns of the system's size);
 *   Hankel   H = [mu_{i+j}], Hs = [mu_{i+j+1}] (LM x LM block Hankel matrices);
 *   rank     H = W1 S W2^H, r = #{s_i > rank_tol s_1};
 *   pencil   the eigenvalues zeta of W1_r^H Hs W2_r S_r^{-1} give omega = center + radius zeta.
 * The contour points run in batches of up to `batch` points (one handle each) and each phase covers
 * a whole batch: one launch assembles every point's system (grid.z = point); for the CF32 precisions
 * one launch forms every point's Schur complement on the tensor cores (a tensor map set per point);
 * the points' LU factorisations replay their captured graphs on the points' streams at once, with the
 * panel cluster size picked on the first batch by timing each candidate (the autotuner); `workers`
 * host threads run the refined solves (bm_solve, precision opts->prec); one launch projects every
 * point's solutions.  The moments, Hankel matrices and the small pencil are formed on the device,
 * the small SVD and eigenvalue problem (size L M at most 256) use cuSOLVER. */
typedef struct {
    bm_c64 center;    /* contour centre in the k_out plane */
    double radius;    /* circle radius, > 0 */
    int npoints;      /* trapezoid points, 4 .. 4096 */
    int nmoments;     /* M, 1 .. 16 */
    bm_c64 k_ratio;   /* k_in = k_ratio * k_out on the contour */
    double rank_tol;  /* relative singular-value cut; 0 selects 1e-8 */
    int workers;      /* host threads running the points' refined solves, 1 .. 64; 0 selects 16 */
    int batch;        /* contour points per batched launch, 1 .. 64; 0 selects min(npoints, 32) */
    int panel_cluster;/* LU panel cluster size, 1 .. 16; 0 lets the autotuner pick it on the first batch */
} bm_ssm_opts;

typedef struct {
    int rank;            /* r */
    int n_inside;        /* eigenvalues inside the contour (|zeta| < 1), listed first in omega */
    int max_iterations;  /* most refinement iterations over the contour points (CF32 precisions) */
    double max_backward_error;  /* largest backward error of the contour solves */
    double t_total_ms;   /* wall time of the call */
    double t_points_ms;  /* wall time of the contour points (assemble + factor + solve + projection) */
    double t_assemble_ms, t_factor_ms, t_solve_ms;  /* wall time of each phase, summed over batches */
    int batch;           /* points per batched launch */
    int panel_cluster;   /* LU panel cluster size used */
    double tune_ms[3];   /* autotuner: factor-phase wall time of the first batch with clusters of 16, 8, 4
                            CTAs (0 when not tuned) */
} bm_ssm_info;

/* Eigenvalues of the discretised system `form` (curve, N as in bm_assemble) inside a circle.
 *  V      : host array, nsys x L column-major (ldv >= nsys; nsys = 3N mixed, 2N ordinary), the
 *           probe right-hand sides (also used as the left projection), 1 <= L, L * M <= 256.
 *  omega  : output, the r eigenvalues (cap >= L * M): those inside the contour first, each group
 *           ordered by real part.  sigma: output, the L * M singular values of H (may be NULL).
 * Errors: BM_EINVAL (arguments), BM_ESINGULAR (a contour point hits an exactly singular system),
 * BM_ENOTCONV (refinement), BM_ENOMEM, BM_ECUDA; bm_last_error names the point. */
bm_status bm_ssm(int device, const bm_curve* curve, int N, bm_formulation form, const bm_opts* opts,
                 const bm_ssm_opts* ssm, const bm_c64* V, int ldv, int L, bm_c64* omega, int cap,
                 double* sigma, bm_ssm_info* info);

/* bm_ssm keeps the handles and device buffers of its last batch of contour points (and the panel
 * cluster size its autotuner picked) for the next call with the same device, N, formulation,
 * options, batch size and L: repeated contour solves then reuse them instead of allocating again.
 * bm_ssm_release frees what is kept for `device` (every device when device < 0). */
bm_status bm_ssm_release(int device);

/* ---- Serving: continuous batching of independent solves ----
 * A library service around the solver (the paper has no counterpart; its solves arrive as a
 * stream, for instance the contour points of section 5.3).  A server owns `slots` worker handles,
 * each with its own stream and host thread.  Requests (any curve, N, wavenumbers, formulation and
 * nrhs) queue in arrival order; the head of the queue is admitted as soon as a slot is free and
 * its device bytes fit what the HBM budget leaves beside the requests in flight, so requests that
 * arrive while others run join them and their work overlaps on the device.  A worker assembles,
 * factors (the factors stay on the device for the solve) and solves its request, then releases the
 * request's device memory before taking the next one.  Every kernel is deterministic and each
 * request has its own buffers, so a result is the same whether it ran alone or in the mix. */
typedef struct bm_server bm_server;

typedef struct {
    int slots;                /* requests on the device at once, 1 .. 32 */
    size_t hbm_budget_bytes;  /* admission budget over the requests in flight (0: 80 % of free memory) */
    bm_opts opts;             /* options of every request (precision, refinement, block size) */
} bm_server_opts;

typedef struct {
    bm_curve curve;
    int N;
    bm_c64 k_out, k_in;
    int formulation;          /* bm_formulation */
    int nrhs;
    const bm_c64* B;          /* host, nsys x nrhs (ldb >= nsys) */
    int ldb;
    bm_c64* X;                /* host output, nsys x nrhs (ldx >= nsys) */
    int ldx;
} bm_request;                 /* B, X (and a user curve) must stay valid until bm_server_wait returns */

typedef struct {
    int status;               /* bm_status of the request */
    int slot;                 /* worker that ran it */
    int iterations;           /* refinement corrections */
    double backward_error;
    double t_queue_ms;        /* submit -> admitted */
    double t_service_ms;      /* admitted -> done */
    size_t bytes;             /* device bytes admitted for it */
} bm_result;

typedef struct {
    unsigned long long submitted, completed;
    size_t max_in_flight_bytes;  /* high-water mark of admitted bytes (never above the budget) */
    int max_in_flight;           /* high-water mark of requests on the device at once */
    size_t budget_bytes;
} bm_server_stats;

bm_status bm_server_create(bm_server** out, int device, const bm_server_opts* opts);
/* Queue a request; returns at once with its ticket.  BM_ENOMEM if it alone exceeds the budget,
 * BM_EINVAL for bad sizes or pointers. */
bm_status bm_server_submit(bm_server* s, const bm_request* req, unsigned long long* ticket);
/* Wait for a request and collect its result (each ticket once: a call for a ticket that is already
 * collected, or that another thread collects while this one waits, returns BM_EINVAL). */
bm_status bm_server_wait(bm_server* s, unsigned long long ticket, bm_result* res);
bm_status bm_server_stats_get(bm_server* s, bm_server_stats* st);
/* Finish every queued request, stop the workers, release the handles. */
bm_status bm_server_destroy(bm_server* s);

/* Copy one assembled FP64 block to dst (column-major, ldd >= rows).
 * Mixed: which = 0..3 selects M13, M23, M31, M32 (N x N).
 * Ordinary: which = 0 selects the whole 2N x 2N matrix. */
bm_status bm_copy_block(bm_ctx* ctx, int which, bm_c64* dst, int ldd, int on_device);

/* Evaluate the device special functions H0^(1)(z), H1^(1)(z) used by assembly at n points
 * (section 2.2 kernels; principal branch, Re z > 0).  All arrays are device arrays when
 * on_device, else host arrays. */
bm_status bm_hankel01(bm_ctx* ctx, const bm_c64* z, int n, bm_c64* h0, bm_c64* h1, int on_device);

/* Run the device's integer FP64 -> FP32 rounding (used where the operator's magnitudes are formed
 * in FP32, e.g. its row norms) on n host values x: rn[i] = x[i] rounded to the nearest FP32, ties to
 * even, formed from the bit pattern by integer operations.  This call exposes it so it can be
 * compared with the IEEE conversion.  Both arrays are host arrays. */
bm_status bm_f32_convert(bm_ctx* ctx, const double* x, int n, float* rn);

/* Host copy of the anchor table the device Taylor zone of bm_hankel01 expands about:
 * H0^(1)(z0), H1^(1)(z0) at z0 = re0 + ix*step + i (im0 + iy*step), stored as
 * out[4*(iy*nx + ix) + {0,1,2,3}] = {Re H0, Im H0, Re H1, Im H1}; anchors outside the annulus
 * 2.5 <= |z0| <= 21 are zero.  Built once per process on the host (no GPU needed); out may be
 * NULL to query the sizes, else it must hold cap_anchors >= nx*ny anchors. */
bm_status bm_hankel_anchor_table(double* out, int cap_anchors, int* nx, int* ny, double* re0, double* im0,
                                 double* step);

/* Host copy of the Taylor coefficients the device Taylor zone of bm_hankel01 evaluates: for every
 * anchor of bm_hankel_anchor_table (same nx, ny, re0, im0, step), H0^(1)(z0 + d) = sum_k a_k d^k
 * (a_0 = H0(z0), a_1 = -H1(z0), the rest from Bessel's equation; H1 = -dH0/dz), k = 0 .. nterms-1,
 * stored as out[2*(nterms*(iy*nx + ix) + k) + {0,1}] = {Re a_k, Im a_k}.  The device holds a_0 .. a_8
 * in FP64 and the rest in FP32; they are returned as the device holds them, widened to double.
 * Zero outside the annulus 2.5 <= |z0| <= 21.  Built once per process on the host (no GPU
 * needed); out may be NULL to query nterms, else it must hold cap_anchors >= nx*ny anchors. */
bm_status bm_hankel_taylor_table(double* out, int cap_anchors, int* nterms);

/* Timing probe: enqueue `reps` launches of one hot kernel on the handle's stream and return
 * without synchronising, so a caller can bracket them with its own events on that stream.
 *  which = BM_PROBE_SCHUR   : the Schur-complement product U33 = -[M31 M32][M13; M23] of
 *                             Theorem thm:LU (mixed system; tensor cores for the CF32 precisions,
 *                             FP64 CUDA cores for BM_FP64).  It overwrites U33, so the handle
 *                             returns to the assembled-but-not-factored state.
 *  which = BM_PROBE_RESIDUAL: the first refinement residual r = b - A x of the last bm_solve (same
 *                             nrhs), in the arithmetic the handle uses for it (FP64 or double-float).
 * Errors: BM_ESTATE (nothing assembled / solved yet), BM_EINVAL. */
enum { BM_PROBE_SCHUR = 0, BM_PROBE_RESIDUAL = 1 };
bm_status bm_enqueue_probe(bm_ctx* ctx, int which, int reps);

/* Per-kernel device times of one factorisation and solve (a diagnostic; the paper has no
 * counterpart).  Runs bm_factor, then bm_solve(nrhs, B, ldb, X, ldx, on_device), with every kernel
 * launched directly (no graph replay) and each launch bracketed by two events on the handle's
 * stream, and reports the launches grouped by kernel name: count and summed device time.  The
 * factors and X are those of a normal call; the times add up to the serial device time of the two
 * calls (kernels that a normal call overlaps are timed one after another here).
 *  out: cap entries (may be NULL to query the count); *count receives the number of groups.
 * Errors: those of bm_factor and bm_solve. */
typedef struct {
    char name[64];
    int launches;
    double ms;
} bm_kernel_time;
bm_status bm_profile(bm_ctx* ctx, int nrhs, const bm_c64* B, int ldb, bm_c64* X, int ldx, int on_device,
                     bm_kernel_time* out, int cap, int* count);

/* Number of CUDA kernels this handle has launched so far (kernel nodes of every replayed CUDA
 * graph plus kernels launched outside graphs). */
bm_status bm_kernel_launches(bm_ctx* ctx, unsigned long long* count);

/* Device bytes the handle currently holds, and its budget. */
bm_status bm_memory(bm_ctx* ctx, size_t* held_bytes, size_t* budget_bytes);

/* Release every device buffer and the handle (the stream too, if the handle created it). */
bm_status bm_destroy(bm_ctx* ctx);

const char* bm_strerror(bm_status s);

/* Details of the most recent failure on this host thread (empty string if none). */
const char* bm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BM_H */
