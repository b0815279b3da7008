/*
 * wcs.h -- C ABI of the GB300 Woodbury-circulant direct solver for the
 * preconditioned TE combined-field integral equation on a convex 2D PEC
 * contour (Consoli et al., "On the Fast Direct Solution of a Preconditioned
 * Electromagnetic Integral Equation", arXiv 2203.13283).
 *
 * Conventions for every call:
 *  - Complex numbers are interleaved (re, im) doubles (FP64).
 *  - Blocks of right-hand sides / solutions are column-major N x B with a
 *    leading dimension ld >= N (column c starts at element c * ld).
 *  - "_dev" pointers are device pointers on the context's device; "_host"
 *    pointers are host memory.  The caller owns every pointer it passes; the
 *    library keeps no caller pointer after the call returns.  All device work
 *    is ordered on the stream given to wcs_create; calls return after their
 *    work is enqueued unless stated otherwise (calls that return host data,
 *    and the setup calls, synchronise the stream).
 *  - Every call returns a wcs_status; on failure wcs_last_error() describes
 *    it (thread-local).  No exception crosses the ABI.
 *  - Setup must proceed contour -> wcs_mesh -> wcs_assemble -> wcs_skeleton
 *    -> wcs_factor -> solves; a call made before its prerequisites returns
 *    WCS_ERR_STATE.  Setting a new contour or mesh invalidates later stages.
 */
#ifndef WCS_H
#define WCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wcs_ctx wcs_ctx;

typedef enum wcs_status {
  WCS_OK = 0,
  WCS_ERR_ARG = 1,          /* invalid argument (null pointer, size, ld) */
  WCS_ERR_NOT_CONVEX = 2,   /* contour has negative curvature somewhere */
  WCS_ERR_CUDA = 3,         /* CUDA runtime error */
  WCS_ERR_OOM = 4,          /* device allocation failed */
  WCS_ERR_SINGULAR = 5,     /* capacitance matrix numerically singular */
  WCS_ERR_RANK_CAP = 6,     /* skeleton reached max_rank before the tolerance */
  WCS_ERR_NOT_CONVERGED = 7,/* iterative refinement did not reach its tolerance */
  WCS_ERR_TIMEOUT = 8,      /* reserved: a bounded device wait gave up */
  WCS_ERR_STATE = 9,        /* call made out of order */
  WCS_ERR_UNSUPPORTED = 10  /* option combination not built */
} wcs_status;

typedef enum wcs_precision {
  WCS_PREC_FP64 = 0,        /* every stage in complex FP64 */
  WCS_PREC_MIXED = 1        /* operator products on the tensor cores (split-bf16, FP32
                               accumulation; exact fixed-point products for the residual
                               with exact_residual), element-pair integrals in FP64 except
                               far pairs beyond zfast (FP32); FP64 circulant eigenvalues,
                               capacitance matrix and refinement vectors */
} wcs_precision;

/* Tunables.  Obtain defaults with wcs_default_options, then override. */
typedef struct wcs_options {
  int precision;      /* wcs_precision */
  int q_far;          /* Gauss points per element for element pairs farther than near_band
                         (default 0 = automatic: 6 in the FP64 form, 4 in the mixed form) */
  int q_near;         /* Gauss points per element for near and singular pairs (default 0 =
                         automatic: 12 in the FP64 form, 8 in the mixed form, where entries
                         need ~1e-9; max 16) */
  int near_band;      /* periodic element distance treated as near (default 4) */
  int block;          /* randomized sampling block width (default 32, max 64) */
  int max_refine;     /* maximum iterative-refinement steps per solve (default 12) */
  double refine_tol;  /* target relative residual ||b - C x|| / ||b|| per column (default 1e-12) */
  int rhs_chunk;      /* right-hand sides processed per pass (default 256) */
  int mixed_planes;   /* mixed form: bf16 planes per operator entry (default 3, max 3) */
  int rhs_planes;     /* mixed form: bf16 planes per staged vector entry (= mixed_planes) */
  double zfast;       /* mixed form: far pairs with k R >= zfast + 2 k h are integrated in FP32
                         around float-float element-centre phases (9 is the smallest safe value),
                         nearer ones in FP64; 0: every pair in FP64.  Default -1 = automatic:
                         1000 in the mixed form.  Measured at N = 32768 (superellipse, k = 3642)
                         against the FP64 form, for incidence grazing the flat faces: 9.8e-7 with
                         zfast = 9, 7.8e-7 with 500, 6.1e-7 with 1000 (assembly 1.7 s), 3.8e-7
                         with 2000 (2.3 s), 2.4e-7 with 0.  The FP32 part loses accuracy where the two terms of the
                         Maue form of N cancel (pairs on one flat face), and there its roundings
                         repeat along each diagonal of the operator. */
  int sample_planes;  /* mixed form: bf16 planes of each operand in the skeleton's sampling
                         products (default 0 = 2; 1 = one product per pass, ~4e-3 relative) */
  int exact_residual; /* mixed form: 1 = evaluate the refinement residual b - C x exactly (fixed-
                         point slices of the operator planes and of x, integer products on the
                         tensor cores, float-float and FP64 sums; see wcs_gemm_exact), so
                         refinement reaches refine_tol down to ~1e-11 against the stored operator;
                         costs 6 bf16 slices of each operator (96 N^2 bytes in all, built at the
                         first such solve).  Adjoint solves keep the drained residual.  0
                         (default): residuals in split-bf16 with FP32 accumulation, which floor
                         near 2e-7. */
} wcs_options;

typedef struct wcs_info {
  int64_t N;          /* unknowns = elements */
  double L;           /* perimeter of gamma (= perimeter of gamma_c) */
  double h;           /* element length L / N */
  double a;           /* radius of gamma_c, L / (2 pi); also the curvature average of k~ */
  double k;           /* wavenumber */
  double kt_re, kt_im;/* k~ = k + 0.4 i k^{1/3} a^{-2/3} (Sec. III) */
  int rank;           /* skeleton rank (after wcs_skeleton), else -1 */
  double norm_cc;     /* ||C_c||_2 = max |mu_C| (after wcs_assemble) */
  double min_curvature; /* minimum curvature found by the convexity check */
  double zfast;       /* far-pair FP32 threshold in effect (mixed form; 0 in the FP64 form) */
  double capacitance_residual; /* ||I - K K^-1||_F / sqrt(rank) of the last wcs_factor, measured
                         with exact products when K^-1 came from the tensor-core iteration
                         (mixed form, rank >= 256); -1 when not measured */
} wcs_info;

/* Entries of wcs_solve_info::history. */
#define WCS_HISTORY 32

typedef struct wcs_solve_info {
  int refine_steps;   /* iterative-refinement steps taken (max over chunks) */
  double rel_residual;/* max over columns of ||b - C x|| / ||b|| at exit */
  int history_len;    /* entries of history[] that describe steps taken (<= WCS_HISTORY) */
  double history[WCS_HISTORY]; /* history[i]: max over columns of the relative residual
                         after i refinement steps (i = 0: the Woodbury solve of Eq. 9 alone).
                         A chunk that stopped earlier contributes its final residual.  In the
                         mixed form a step's entry is the residual carried by the updates
                         R <- R - C dx unless it was recomputed at that step. */
} wcs_solve_info;

/* Operators selectable by wcs_apply / wcs_circulant_eigs. */
typedef enum wcs_op {
  WCS_OP_C = 0,       /* C of Eq. (6) on gamma */
  WCS_OP_CH = 1,      /* C^H */
  WCS_OP_CC = 2,      /* C_c: C on the equivalent circle (circulant) */
  WCS_OP_CCH = 3,     /* C_c^H */
  WCS_OP_CC_INV = 4,  /* C_c^{-1} */
  WCS_OP_S = 5,       /* S^k~ Galerkin matrix on gamma */
  WCS_OP_D = 6,       /* D^k */
  WCS_OP_DT = 7,      /* D^k~ */
  WCS_OP_N = 8,       /* N^k */
  WCS_OP_G = 9,       /* Gram matrix of the hats */
  WCS_OP_SKEL = 10,   /* U V^T, the skeleton of C - C_c (Eq. 7) */
  WCS_OP_GINV = 11,   /* G^-1 (cyclic tridiagonal solve) */
  WCS_OP_CCH_INV = 12 /* C_c^{-H} */
} wcs_op;

/* Library version string. */
const char* wcs_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* wcs_last_error(void);

/* Fill *opt with the defaults documented in wcs_options. */
int wcs_default_options(wcs_options* opt);

/* Create a solver context on the current CUDA device.  stream: a cudaStream_t
 * (NULL = legacy default stream) on which all device work is ordered.  opt may
 * be NULL for defaults. */
int wcs_create(wcs_ctx** out, const wcs_options* opt, void* stream);

/* Free every device buffer of ctx and the context itself (NULL is a no-op). */
int wcs_destroy(wcs_ctx* ctx);

/* --- contour gamma (Sec. II: a convex 2D contour), as r(theta) = rho(theta) (cos, sin) --- */
/* Circle of radius a. */
int wcs_contour_circle(wcs_ctx* ctx, double a);
/* Ellipse x^2/ax^2 + y^2/ay^2 = 1. */
int wcs_contour_ellipse(wcs_ctx* ctx, double ax, double ay);
/* Superellipse |x/ax|^p + |y/ay|^p = 1 with p >= 2. */
int wcs_contour_superellipse(wcs_ctx* ctx, double ax, double ay, double p);
/* rho(theta) = sum_{m<count} cos_c[m] cos(m theta) + sin_c[m] sin(m theta); host arrays,
 * count <= 64.  The unit circle is count = 1, cos_c[0] = 1. */
int wcs_contour_fourier(wcs_ctx* ctx, int count, const double* cos_c, const double* sin_c);

/* Mesh gamma uniformly in arc length with N piecewise-linear elements (Sec. V),
 * node 0 at polar angle 0, and fix the wavenumbers: k > 0 as given, k <= 0 means
 * 10 elements per wavelength (k = 2 pi (N/10) / L).  k~ follows Sec. III with
 * a = L / (2 pi).  Builds the same mesh on the equivalent circle gamma_c.
 * Rejects non-convex contours (WCS_ERR_NOT_CONVEX) and k h > 2.5. */
int wcs_mesh(wcs_ctx* ctx, int64_t N, double k);

/* Geometry and wavenumbers of the current mesh. */
int wcs_query(const wcs_ctx* ctx, wcs_info* info);

/* Positions, outward normals and curvature at arc lengths s_host[0..count):
 * out_host receives 5 * count doubles (x, y, nx, ny, kappa blocks). */
int wcs_geometry_sample(wcs_ctx* ctx, int64_t count, const double* s_host, double* out_host);

/* Assemble the Galerkin matrices S^k~, D^k, D^k~, N^k of Eq. (4)/(5) on gamma
 * (device-resident: dense complex FP64 in the FP64 form; in the mixed form
 * split-bf16 planes of each operator and of its transpose, from entries
 * integrated in FP64, or for far pairs in FP32 when zfast > 0) and the
 * circulant eigenvalues of the same operators on gamma_c (always FP64), from
 * which mu_C of C_c (Eq. 6 on the circle) follows. */
int wcs_assemble(wcs_ctx* ctx);

/* Entries of (S~, D, D~, N) at (rows_host[t], cols_host[t]), computed point-wise
 * with the same quadrature as wcs_assemble: out_host gets 4 * count complex
 * values (operator-major).  Needs wcs_mesh only. */
int wcs_operator_entries(wcs_ctx* ctx, int64_t count, const int64_t* rows_host,
                         const int64_t* cols_host, double* out_host);

/* mu_X(m), m = 0..N-1, of the circle operator X in {WCS_OP_G, S, D, DT, N, CC}:
 * eigenvalue for the eigenvector exp(2 pi i m j / N).  out_dev: N complex. */
int wcs_circulant_eigs(wcs_ctx* ctx, int op, double* out_dev);

/* Y = op X for B columns (X, Y device, column-major, may not alias).
 * The circulant operators (CC, CCH, CC_INV, CCH_INV) are applied by FFT with
 * the FP64 eigenvalues mu_C.  In the mixed form, for power-of-two N in
 * [1024, 65536], the transform itself runs in FP32 (relative error ~1e-6:
 * these applies serve the Woodbury approximate inverse of Eq. 9 and the
 * sampling of C - C_c, both corrected by refinement); otherwise in FP64. */
int wcs_apply(wcs_ctx* ctx, int op, int64_t B, const double* X_dev, int64_t ldx, double* Y_dev,
              int64_t ldy);

/* Skeleton C - C_c = U V^T (Eq. 7) by an adaptive blocked randomized range
 * finder on the matrix-free operator C - C_c: Gaussian test blocks (Philox,
 * seed), projected samples, stopping when every new projected sample has norm
 * below tol * ||C_c||_2 / (10 sqrt(2/pi)), so ||C - C_c - U V^T|| <= tol ||C_c||
 * with high probability.  U is orthonormal; V^T = U^H (C - C_c).  max_rank <= 0
 * means N.  *rank_out receives the rank.  Returns WCS_ERR_RANK_CAP (with the
 * skeleton kept) when max_rank is reached first. */
int wcs_skeleton(wcs_ctx* ctx, double tol, int max_rank, uint64_t seed, int* rank_out);

/* Factor C = C_c (I + C_c^{-1} U V^T) (Eq. 8): W = C_c^{-1} U by FFT, the
 * capacitance matrix K = I + V^T W and its inverse, for the Woodbury identity
 * of Eq. (9).  K^-1: FP64 Gauss-Jordan in the FP64 form and for rank < 256;
 * in the mixed form otherwise a Newton-Schulz iteration on the tensor cores,
 * closed by one step with the drained three-plane product and then by steps
 * with exact fixed-point products until ||I - K K^-1||_F / sqrt(rank),
 * measured with an exact product after each, is below 1e-10 (at most three;
 * ~3e-11 at rank 4096; reported in wcs_info.capacitance_residual).  Returns
 * WCS_ERR_SINGULAR when K is singular, the iteration does not converge, or
 * the closing steps leave that residual at 1e-6 or above. */
int wcs_factor(wcs_ctx* ctx);

/* Checkpoint of a factored context.  The paper defines no file format; this
 * stores what the solve of Eq. (9) needs beyond the operators: the single
 * skeleton U V^T of Eq. (7) (U = Q and V_w = conj(V), N x rank each) and
 * W~ = C_c^-1 U (I + V^T C_c^-1 U)^-1 and the capacitance inverse
 * (I + V^T C_c^-1 U)^-1 (rank x rank, for wcs_solve_adjoint), plus the
 * contour, N, k and the options, in a host file at `path` (complex FP64,
 * about 48 N rank bytes).  wcs_save writes format version 3, which ends with
 * a 64-bit FNV-1a checksum of the whole file; wcs_load checks the file's
 * length and checksum before any device work, so a truncated or corrupted
 * file is rejected with the context left as it was.  Files of versions 1
 * and 2 (no checksum) still load; version-1 contexts solve forward only.
 * The operators are not stored.  wcs_load re-runs the mesh and the assembly,
 * which are deterministic, on a context created with the same precision and
 * quadrature options (else WCS_ERR_ARG), then restores the factors; the
 * context is then in the factored state.  Both synchronise the context
 * stream.  Errors: WCS_ERR_STATE (save before wcs_factor), WCS_ERR_ARG
 * (null arguments, unreadable/truncated/corrupted/foreign file, option
 * mismatch), or the status of the mesh/assembly step. */
int wcs_save(wcs_ctx* ctx, const char* path);
int wcs_load(wcs_ctx* ctx, const char* path);

/* x = C^-1 b through Eq. (9) only (no refinement), B columns, device pointers. */
int wcs_woodbury_apply(wcs_ctx* ctx, int64_t B, const double* b_dev, int64_t ldb, double* x_dev,
                       int64_t ldx);

/* Solve Eq. (5) for B plane waves with propagation angles angles_host[0..B)
 * (radians, d = (cos, sin), phase reference at the origin): project
 * e/eta and h (Eq. 4), form the preconditioned right-hand side of Eq. (5),
 * apply Eq. (9), then refine x <- x + C^-1 (b - C x) until refine_tol.
 * j_dev receives the hat coefficients of the current (N x B, ldj). */
int wcs_solve_planewaves(wcs_ctx* ctx, int64_t B, const double* angles_host, double* j_dev,
                         int64_t ldj, wcs_solve_info* info);

/* Same as wcs_solve_planewaves with the solution returned in host memory
 * (j_host, N x B, ldj); includes the device-to-host copy; synchronises. */
int wcs_solve_planewaves_host(wcs_ctx* ctx, int64_t B, const double* angles_host, double* j_host,
                              int64_t ldj, wcs_solve_info* info);

/* Solve Eq. (5) for user Galerkin data e/eta and h (device, N x B, ld). */
int wcs_solve_rhs(wcs_ctx* ctx, int64_t B, const double* e_dev, const double* h_dev, int64_t ld,
                  double* j_dev, int64_t ldj, wcs_solve_info* info);

/* Shape perturbation of the current contour (any family): adds
 * sum_{m<M} alpha[m] cos(m theta) + sum_{m=1..M} beta[m-1] sin(m theta) to its
 * radial function rho(theta) (Sec. II: gamma star-shaped and convex; a
 * non-convex result fails in wcs_mesh with WCS_ERR_NOT_CONVEX).  Replaces an
 * earlier perturbation; M = 0 removes it.  Host arrays of M doubles each,
 * 0 <= M <= 32.  Like the contour setters it discards the mesh and
 * everything built on it.  Errors: WCS_ERR_STATE (no contour yet),
 * WCS_ERR_ARG. */
int wcs_contour_perturb(wcs_ctx* ctx, int M, const double* alpha, const double* beta);

/* Gradient of the far-field objective J = sum_b sum_o |F(phi_o; angle_b)|^2
 * (B plane-wave incidences, nphi observation angles; F as in wcs_farfield)
 * with respect to the 2M shape parameters of wcs_contour_perturb, at the
 * context's current contour: grad[m] = dJ/d alpha_m (m < M), grad[M+m-1] =
 * dJ/d beta_m (m = 1..M).  N and k stay fixed; the mesh, k~ (Sec. III) and
 * everything else follow the contour.  Adjoint route: one forward solve
 * (Eq. 5 through Eq. 9), one adjoint solve lam = C^-H E^H F, then
 * dJ/dp = 2 Re sum_b [F_b^H dE j_b + lam_b^H dR_b] with R = b - C j written
 * through the four operators (Eq. 5, 6).  The derivatives of S~, D, D~, N
 * enter as bilinear forms evaluated for all parameters in one pass over the
 * far element pairs (analytic derivatives of the Hankel kernels with respect
 * to the points, normals and k~, contracted with the motion of the
 * arc-length mesh); the near band (log-singular rules), the mesh motion, the
 * right-hand sides and the far-field map are central differences with step
 * delta (delta <= 0 means 1e-6), all O(N) per parameter.  angles_host (B),
 * phi_host (nphi) and the outputs J_host (1) and grad_host (2M) are host
 * memory.  Needs a factored context; device scratch 4 N^2 complex FP64 plus
 * a few N x B blocks.  Synchronises the stream.  Errors: WCS_ERR_STATE,
 * WCS_ERR_ARG, WCS_ERR_NOT_CONVEX (a perturbed contour), WCS_ERR_NOT_CONVERGED
 * (a solve missed refine_tol; outputs still written). */
int wcs_shape_gradient(wcs_ctx* ctx, int64_t B, const double* angles_host, int nphi, const double* phi_host,
                       int M, double delta, double* J_host, double* grad_host);

/* wcs_shape_gradient for the parameters i0 <= i < i1 only (0 <= i0 <= i1 <=
 * 2M, same numbering): grad_host[i - i0] = dJ/dp_i.  J_host is always
 * written.  The parameters are independent, so ranks of a multi-GPU job can
 * each take a contiguous range and gather the pieces.  Same errors as
 * wcs_shape_gradient; grad_host may be null when i0 == i1. */
int wcs_shape_gradient_range(wcs_ctx* ctx, int64_t B, const double* angles_host, int nphi,
                             const double* phi_host, int M, double delta, int i0, int i1, double* J_host,
                             double* grad_host);

/* Shape derivatives of one Galerkin operator as bilinear forms:
 * out[2 (i - i0) + {0, 1}] = (re, im) of sum_b u_b^H (dX / dp_i) v_b for the
 * shape parameters i0 <= i < i1 of wcs_contour_perturb (numbering as in
 * wcs_shape_gradient), X = op (0 S~, 1 D, 2 D~, 3 N; Sec. II Eq. 4 and the
 * S~ of Eq. 5).  The derivative moves the arc-length mesh with the contour
 * at fixed N and k (k~ follows a = L / 2 pi).  Far pairs: one pass of the
 * analytic derivative kernel; near band: central differences (step delta,
 * <= 0 means 1e-6).  u_dev, v_dev: complex FP64 device blocks N x B
 * (column-major, ld >= N).  Needs wcs_assemble.  Device scratch 4 N^2
 * complex FP64; synchronises.  The terms of wcs_shape_gradient's adjoint
 * formula, offered separately for checks and for other objectives. */
int wcs_shape_operator_forms(wcs_ctx* ctx, int op, int64_t B, const double* u_dev, const double* v_dev, int64_t ld,
                             int M, double delta, int i0, int i1, double* out_host);

/* Solve C x = b for B general right-hand sides b of Eq. (5)'s preconditioned
 * system (device, complex FP64, column-major N x B, ldb, ldx >= N): Eq. (9)
 * then refinement x <- x + C~^-1 (b - C x) with the exact product C, to
 * refine_tol.  wcs_solve_rhs is the same solve with b formed from e/eta and
 * h.  x must not alias b.  Errors: WCS_ERR_STATE (before wcs_factor),
 * WCS_ERR_ARG (null pointer with B > 0, ld < N), WCS_ERR_NOT_CONVERGED (x
 * still written). */
int wcs_solve(wcs_ctx* ctx, int64_t B, const double* b_dev, int64_t ldb, double* x_dev, int64_t ldx,
              wcs_solve_info* info);

/* Adjoint solve C^H x = b (Eq. 5's operator C conjugate-transposed), B
 * columns of complex FP64, device, column-major N x B (ldb, ldx >= N).  The
 * approximate inverse is the adjoint of Eq. (9): with C~ = C_c + U V^T,
 * C~^-H b = y - C_c^-H V_w K^-H (U^H y), y = C_c^-H b, K = I + V^T C_c^-1 U;
 * C_c^-H is Eq. (8) with conjugated eigenvalues.  Refinement uses C^H, so the
 * result meets refine_tol against the exact adjoint.  Needs the capacitance
 * inverse that wcs_factor forms and wcs_save stores (a context restored
 * from a version-1 file has none: WCS_ERR_STATE until wcs_factor runs
 * again).  x must not alias b.  Errors:
 * WCS_ERR_STATE, WCS_ERR_ARG (null pointer with B > 0, ld < N),
 * WCS_ERR_NOT_CONVERGED (x still written). */
int wcs_solve_adjoint(wcs_ctx* ctx, int64_t B, const double* b_dev, int64_t ldb, double* x_dev,
                      int64_t ldx, wcs_solve_info* info);

/* Plane-wave Galerkin projections e/eta and h of Eq. (4) (device, N x B, ld). */
int wcs_planewave_rhs(wcs_ctx* ctx, int64_t B, const double* angles_host, double* e_dev,
                      double* h_dev, int64_t ld);

/* Far field F(phi_o) for B currents (device j, N x B, ldj) at nphi observation
 * angles: H^s ~ F e^{i k rho} / sqrt(rho).  F_dev: nphi x B, column-major, ldf. */
int wcs_farfield(wcs_ctx* ctx, int64_t B, const double* j_dev, int64_t ldj, int nphi,
                 const double* phi_host, double* F_dev, int64_t ldf);

/* Real contraction on the tensor cores (tcgen05, sm_103a) with split-bf16
 * operands: D (M x Nc) = A (M x K) * B (Nc x K)^T, all FP64 row-major device
 * arrays (lda, ldb >= K, ldd >= Nc).  Each operand is rounded to `planes`
 * bf16 terms (1: bf16, 2: ~16 bits, 3: ~24 bits) and every product of
 * combined order < planes is accumulated in FP32 in tensor memory.  This is
 * the contraction behind the mixed-precision operator products of Eq. (5)-(7).
 * When the output tiles cannot fill the GPU (few rows and columns, long K)
 * and accurate == 0, K is split over the grid and the FP32 partials are summed
 * in FP64 in a fixed order; the split depends on the shape alone, so results
 * are reproducible.  Allocates its own staging buffers; ordered on `stream`;
 * synchronises.  Returns WCS_ERR_TIMEOUT if a bounded device wait expired. */
int wcs_gemm_split_bf16(int64_t M, int64_t Nc, int64_t K, const double* A_dev, int64_t lda,
                        const double* B_dev, int64_t ldb, int planes, double* D_dev, int64_t ldd,
                        void* stream);

/* wcs_gemm_split_bf16 with a choice of accumulation.  The accumulator of the
 * MMA truncates, so its error grows with the number of K = 16 steps it spans.
 * accurate = 1 drains the tensor-memory accumulator into FP32 register sums
 * after every step (~1e-7 relative with 3 planes); accurate = n > 1 drains
 * every n steps (n = 64: ~1e-5 at close to the speed of accurate = 0).
 * accurate = 4 drains once per shared-memory stage of K = 64 and issues the
 * stage's products smallest first across its four steps, which keeps the
 * error of accurate = 1 at ~80% of its time (the solver's refinement
 * residual uses it).  planes must be 2 or 3 when accurate != 0. */
int wcs_gemm_split_bf16_ex(int64_t M, int64_t Nc, int64_t K, const double* A_dev, int64_t lda,
                           const double* B_dev, int64_t ldb, int planes, int accurate, double* D_dev,
                           int64_t ldd, void* stream);

/* The contraction of wcs_gemm_split_bf16 without any device allocation.  The
 * paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc (a real-time loop running on a frozen memory pool, a plug-in
 * whose host application owns all device memory, code between two
 * synchronisation points that must not allocate).  Same arguments and result
 * as wcs_gemm_split_bf16; the staging planes, the split-K partials and the
 * error flag live in one file-scope device array of 32 MiB that every GPU
 * loading the library holds until the process exits.  Sizes whose
 * (M + Nc) * ceil64(K) * planes * 2 bytes plus split-K partials exceed that
 * limit are rejected with WCS_ERR_ARG.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the array: calls whose GPU
 * work overlaps (other streams, other host threads) race on it.  Each call
 * clears the parts that must start at zero.  Synchronises `stream`. */
int wcs_gemm_split_bf16_noalloc(int64_t M, int64_t Nc, int64_t K, const double* A_dev, int64_t lda,
                                const double* B_dev, int64_t ldb, int planes, double* D_dev,
                                int64_t ldd, void* stream);

/* Exact real contraction D (M x Nc) = A (M x K) * B (Nc x K)^T on the tensor
 * cores, all FP64 row-major device arrays (lda, ldb >= K, ldd >= Nc).  The
 * operator products of the refinement residual (Eq. 5 with C of Eq. 6) in
 * the mixed form's exact_residual mode use the same method: each row is cut
 * into chunks of 1024 K values, each chunk scaled by a power of two so its
 * entries lie in (-1, 1) and written as six 7-bit fixed-point slices (bf16
 * integers); the 21 slice pairs of combined order < 6 are multiplied with
 * one split of K per chunk, where the FP32 accumulation of integer products
 * below 2^24 is exact, and the scaled partials are summed in float-float and
 * FP64.  Error of D_ij <= 2^-40 sum_k (cmax_A |B_jk| + |A_ik| cmax_B +
 * cmax_A cmax_B), cmax the largest magnitude in the value's chunk of 1024;
 * for data of similar size within each chunk that is ~2^-40 (|A| |B|^T),
 * independent of K.  Values must lie within 2^-100 .. 2^100.  Allocates
 * about 12 (M + Nc) K + 4 (K / 1024) M Nc bytes; ordered on `stream`;
 * synchronises.  Errors: WCS_ERR_ARG, WCS_ERR_OOM, WCS_ERR_CUDA,
 * WCS_ERR_TIMEOUT (a bounded device wait expired). */
int wcs_gemm_exact(int64_t M, int64_t Nc, int64_t K, const double* A_dev, int64_t lda, const double* B_dev,
                   int64_t ldb, double* D_dev, int64_t ldd, void* stream);

/* Per-contour outcome of wcs_batch_solve_fourier. */
typedef struct wcs_batch_stats {
  int status;         /* wcs_status of the contour's setup and solve (WCS_ERR_NOT_CONVERGED: solved,
                         refine_tol missed) */
  int rank;           /* skeleton rank */
  int refine_steps;   /* iterative-refinement steps of its solve */
  double rel_residual;/* max over its columns of ||b - C x|| / ||b|| */
  double setup_s;     /* wall-clock seconds of mesh, assembly, skeleton and factor */
  double solve_s;     /* wall-clock seconds of the plane-wave solve, including the copy to the host */
  int worker;         /* host worker (stream) that took it */
} wcs_batch_stats;

/* Batched form: `count` contours solved for the same B plane waves (Sec. V:
 * any number of right-hand sides per contour; here also many contours).
 * Contour c has radial function rho(theta) = sum_{m<nf} cos_c[c nf + m]
 * cos(m theta) + sin_c[c nf + m] sin(m theta) (sin_c may be NULL), N[c]
 * elements and wavenumber k[c] (<= 0: 10 elements per wavelength), with the
 * options `opt` (NULL: defaults).  Each contour is meshed, assembled,
 * skeletonised at tolerance tol with rank cap N[c] / rank_div (rank_div <= 0:
 * no cap; WCS_ERR_RANK_CAP is accepted), factored and solved; its current
 * (N[c] x B complex FP64, column-major, ld N[c]) is written to host memory at
 * j_host + 2 B sum_{c' < c} N[c'] doubles.  `workers` (1..8) host threads
 * each drive one context on its own stream and take contours from a queue
 * ordered by decreasing N, so the GPU overlaps one contour's setup with
 * another's solve and device memory holds at most `workers` contours.  stats
 * (optional, count entries) receives each contour's outcome.  Returns the
 * first hard error (after finishing the other contours), else
 * WCS_ERR_NOT_CONVERGED if a contour missed refine_tol, else WCS_OK.
 * Errors before any work: WCS_ERR_ARG. */
int wcs_batch_solve_fourier(const wcs_options* opt, int count, int nf, const double* cos_c, const double* sin_c,
                            const int64_t* N, const double* k, int64_t B, const double* angles_host, double tol,
                            int rank_div, uint64_t seed, int workers, double* j_host, wcs_batch_stats* stats);

/* Number of CUDA kernel launches the library has issued in this process. */
uint64_t wcs_launch_count(void);

/* Per-kernel timing with CUDA events recorded on the context stream around
 * each instrumented launch (enable != 0 turns it on; off by default). */
int wcs_profile(wcs_ctx* ctx, int enable);

/* Sum the recorded launches by category (synchronises): out_host gets 16 x 4
 * doubles {launches, total ms, algorithmic work, bytes} for the categories, in
 * order: tensor-core contraction (work = useful real flops 2 M Nc K of the
 * complex product), assembly (work = far point pairs), FFT circulant applies
 * (bytes), FP64 GEMM, skeleton, factor, solve, drained tensor-core
 * contraction, skeleton sampling, projection, orthonormalisation, V_w,
 * capacitance inverse, exact contraction (work = useful flops, as the first),
 * FP32 far-pair assembly kernel (work = far point pairs of its tiles; the
 * assembly category then counts the FP64 kernel over the other tiles),
 * periodically drained tensor-core contraction (work as the first; the
 * drained category then counts the three-plane product drained once per
 * K = 64 stage only).
 * reset != 0 clears the records. */
int wcs_profile_read(wcs_ctx* ctx, int reset, double* out_host);

/* Measured issue rate of the FMA pipe (precision 64: FP64, 32: FP32) on the
 * current device, in flops per second (an FMA counts as 2): a dependency-free
 * stream of `iters` rounds of 8 independent FMA chains per thread over a grid
 * of 8 CTAs of 256 threads per SM, timed with CUDA events on `stream`.  The
 * paper has no counterpart: this gives the roofline denominator of the
 * point-pair integration kernels (Eq. 4), which run on these pipes.
 * Allocates a small output buffer; synchronises the stream. */
int wcs_fma_rate(int precision, int iters, void* stream, double* flops_per_s);

/* Host-only: product-integration weights of the near-field rule with q points
 * (3 * q * q doubles: coincident, next-neighbour, previous-neighbour pairs). */
int wcs_quadrature_tables(int q, double* out_host);

#ifdef __cplusplus
}
#endif

#endif /* WCS_H */
