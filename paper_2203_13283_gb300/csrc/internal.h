// Internal interfaces between the translation units of the solver library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace wcs {

// A one-time set-up step per CUDA device.  Kernel attributes (the opt-in to
// more than 48 KB of dynamic shared memory) and __constant__ tables belong to
// a device, so a process that uses several devices repeats the step on each.
// need() is true until done() has been called with that device current;
// device indices >= 64 are not remembered (the step then runs every time).
struct DeviceOnce {
  bool flag[64] = {};
  static int device() {
    int d = -1;
    return (cudaGetDevice(&d) == cudaSuccess) ? d : -1;
  }
  bool need() const {
    const int d = device();
    return d < 0 || d >= 64 || !flag[d];
  }
  void done() {
    const int d = device();
    if (d >= 0 && d < 64) flag[d] = true;
  }
};

// ---------------------------------------------------------------- geometry
enum ContourFamily { FAM_CIRCLE = 0, FAM_ELLIPSE = 1, FAM_SUPERELLIPSE = 2, FAM_FOURIER = 3 };
constexpr int kMaxFourier = 64;
constexpr int kMaxPerturb = 33;

struct Contour {
  int family;
  double a;             // circle radius
  double ax, ay, p;     // ellipse / superellipse
  int nf;               // Fourier: number of coefficients (m = 0..nf-1)
  double fc[kMaxFourier], fs[kMaxFourier];
  // shape perturbation added to rho of any family:
  // sum_{m < np} pc[m] cos(m theta) + ps[m] sin(m theta)   (ps[0] = 0)
  int np;
  double pc[kMaxPerturb], ps[kMaxPerturb];
};

// Structure-of-arrays point table: positions, unit outward normals, curvature.
struct Points {
  double *x = nullptr, *y = nullptr, *nx = nullptr, *ny = nullptr, *kappa = nullptr;
  int64_t n = 0;
};

// Arc-length tables of a contour: panel cumulative lengths in theta.
struct ArcTable {
  double* cum = nullptr;  // P + 1 entries, cum[P] = L
  int P = 0;
  double L = 0.0;
};

int arc_table_build(const Contour& c, ArcTable& t, cudaStream_t s);
// Points at arc lengths s_j = (e + xi[g]) * h for e < N, g < nq (index e*nq + g).
int points_build(const Contour& c, const ArcTable& t, int64_t N, double h, const double* xi_dev,
                 int nq, Points& out, cudaStream_t s);
// Minimum curvature over a dense sample of the contour (convexity check).
int min_curvature(const Contour& c, const ArcTable& t, int64_t samples, double* kmin, cudaStream_t s);

// ---------------------------------------------------------------- quadrature
struct QuadTables {
  int q_far = 6, q_near = 12, near_band = 4;
  double xf[16], wf[16];         // far rule on [0,1]
  double xn[16], wn[16];         // near rule on [0,1]
  // product-integration weights for log d on the near grid (q_near^2 each):
  // 0: self (d = |xi - eta|), 1: f = e + 1 (d = 1 - xi + eta), 2: f = e - 1 (d = xi + 1 - eta)
  std::vector<double> wlog[3];
};
void gauss_legendre01(int n, double* x, double* w);
void build_quad_tables(QuadTables& q);

// ---------------------------------------------------------------- assembly
// FP32 constants of the far-pair path, formed once on the host
struct FastConsts {
  float kf = 0.f, beta = 0.f;      // k, Im k~
  float ck[2] = {0.f, 0.f};        // sqrt(2 / (pi k~))
  float ik[2] = {0.f, 0.f};        // i / k~
  float kt4[2] = {0.f, 0.f};       // i k~ / 4
  float ampk = 0.f;                // sqrt(2 / (pi k))
  float kk2h2 = 0.f, h2 = 0.f;     // k^2 h^2, h^2
  float beta_lo = 0.f;             // Im k~ - beta (float-float tail)
  float zfast2 = 0.f;              // zfast^2 (pair test k^2 |c_e - c_f|^2 >= zfast^2)
  float k_hi = 0.f, k_lo = 0.f;    // k as a float-float pair
  float twopi[3] = {0.f, 0.f, 0.f};   // 2 pi = twopi[0] + twopi[1] + twopi[2]
};

struct AsmArgs {
  int64_t N;
  double h, k;
  zd kt;
  int kt_pair = 0;                 // 1: both wavenumbers from one real evaluation (k~ = k (1 + i t))
  int rot_ok = 0;                  // 1: far element pairs may share a reference phase (k h <= 1.2, t <= 0.019)
  KtPair ktp;
  int q_far, q_near, near_band;
  Points far, near;                // point tables (far: q_far per element, near: q_near)
  const double* wlog;              // 3 * q_near^2 product weights (device)
  zd *S, *D, *Dt, *Nk;             // outputs
  int64_t ld;                      // row-major leading dimension
  // mixed-precision form: far pairs with k R >= zfast are integrated in FP32
  // around the FP64 element-centre distance; output written as split-bf16
  // planes [op][layout][plane] (layout 0: X, layout 1: X^T; each row-major
  // complex as real N x 2N, leading dimension ldp).
  int mixed = 0;
  int planes = 0;
  uint16_t* P[4][2][3];
  int64_t ldp = 0;
  const double *cx = nullptr, *cy = nullptr;     // element centres (xi = 1/2)
  const float *ox = nullptr, *oy = nullptr;      // far points minus their element centre
  const float *nxf = nullptr, *nyf = nullptr;    // far-point normals (FP32)
  const float *nxl = nullptr, *nyl = nullptr;    // their float-float tails
  const float *oxl = nullptr, *oyl = nullptr;    // float-float tails of the offsets
  // FP64 factors of the FP32 far-pair path, applied once per stored entry (a
  // constant rounded to FP32 would bias every far entry of an operator alike)
  zd fS, fD, fDt, fN;              // S~, D, D~, N (see pair_fast_f)
  double kk2h2 = 0.0;              // k^2 h^2 of the Maue form
  const float4* cff = nullptr;                   // element centres as float-float (x hi, x lo, y hi, y lo)
  double zfast = 1e300;
  FastConsts fk;
  const uint8_t* tile_flags = nullptr;           // mixed tile kernel: only flagged tiles
};
// Fill kp.asym for kp.t and the term-count thresholds kp.xth for relative
// tolerance tol (host).
void fill_asymptotic(KtPair& kp, double tol);
int assemble_dense(const AsmArgs& a, cudaStream_t s);
// Mixed form: the same operators written as split-bf16 planes (see AsmArgs):
// the FP32 far-pair kernel over the tiles it can take, then the FP64 kernel
// over the rest.  mid (optional, two events) is recorded between the two;
// fp64_tiles and tiles (optional) receive the tile counts.
int assemble_planes(const AsmArgs& a, cudaStream_t s, cudaEvent_t* mid = nullptr, int64_t* fp64_tiles = nullptr,
                    int64_t* tiles = nullptr);
// FP32 offset tables of the far points relative to element centres.
int far_offsets(const Points& far, const double* cx, const double* cy, int64_t N, int q, float* ox,
                float* oy, float* nxf, float* nyf, float* nxl, float* nyl, float* oxl, float* oyl, float4* cff,
                cudaStream_t s);
// First row of the four circulant operators on the circle (row 0, N entries each).
int assemble_circle_row(const AsmArgs& a, cudaStream_t s);
// Sampled entries (row, col) of the four operators, computed point-wise.
int assemble_entries(const AsmArgs& a, int64_t count, const int64_t* rows, const int64_t* cols,
                     zd* out4, cudaStream_t s);

// Shape derivative of bilinear forms (the gradient of Sec. II-V with respect
// to the contour).  W[X] (row-major N x N, X = S~, D, D~, N) are node-pair
// coefficients; the forms are T = sum_X sum_ij W[X]_ij X_ij.
struct ShapeArgs {
  AsmArgs A;                       // base geometry, rules and wavenumbers (far tables used)
  const zd* W[4] = {nullptr, nullptr, nullptr, nullptr};
  double* Gr = nullptr;            // per far point: dT/dr (complex x, complex y) as 4 doubles
  double* Gn = nullptr;            // per far point: dT/dn (4 doubles)
  double* scal = nullptr;          // dT/dk~ (2 doubles), sum of the h^2-scaled far terms (2 doubles)
};
// Far element pairs (periodic distance > near_band), one pass for every
// parameter: accumulates Gr, Gn (zeroed by the caller) and scal.
int shape_far_forms(const ShapeArgs& a, cudaStream_t s);
// sum over near element pairs (distance <= near_band) of sum_X sum_ab
// W[X](e + a, f + b) X_ef,ab with the pair integrals of A's geometry;
// part holds per-block partial sums (2 doubles each), *nparts set.
int shape_near_forms(const AsmArgs& A, const zd* const* W, double* part, int* nparts, cudaStream_t s);

// ---------------------------------------------------------------- FFT
struct FFTPlan {
  int64_t n = 0;
  bool pow2 = true;
  int64_t m = 0;                   // Bluestein length (power of two >= 2n-1)
  zd* twiddle = nullptr;           // device twiddles for the power-of-two length
  zd* chirp = nullptr;             // Bluestein chirp (n)
  zd* chirp_hat = nullptr;         // FFT of the Bluestein filter (m)
  zd* work = nullptr;              // Bluestein work (m * batch_cap)
  int64_t work_cols = 0;
};
// FP32 circulant applies of the mixed form (circ32.cu): y = F^-1 diag(s) F x
// with s = mu, conj(mu), 1/mu, 1/conj(mu) (mode 0..3) for power-of-two
// 1024 <= n <= 65536; x, y FP64 columns (y may alias x).
struct Circ32 {
  int64_t n = 0;
  int n1 = 0, n2 = 0;
  float2* scale = nullptr;   // 4 x n, permuted to the middle pass's register layout, times 1/n
  int64_t scale_n = 0;
  float2* work = nullptr;    // FP32 scratch columns
  int64_t work_elems = 0;
  bool ready = false;
};
bool circ32_supported(int64_t n);
int circ32_prepare(Circ32& p, const zd* mu, int64_t n, cudaStream_t s);
int circ32_apply(Circ32& p, const zd* x, int64_t ldx, zd* y, int64_t ldy, int64_t cols, int mode, cudaStream_t s);
void circ32_release(Circ32& p);
int fft_plan_create(FFTPlan& p, int64_t n, cudaStream_t s);
void fft_plan_destroy(FFTPlan& p);
// In-place batched transform of `cols` columns of length n (column-major, ld).
// sign = -1: forward (e^{-2 pi i jk/n}); +1: inverse without 1/n scaling.
int fft_columns(FFTPlan& p, zd* x, int64_t ld, int64_t cols, int sign, cudaStream_t s);
// x[:, c] <- x[:, c] * mu (mu length n), or / mu when divide, conj(mu) when conj_mu.
int scale_columns(zd* x, int64_t n, int64_t ld, int64_t cols, const zd* mu, bool divide,
                  bool conj_mu, double extra, cudaStream_t s);

// ---------------------------------------------------------------- dense linear algebra (FP64)
// General strided complex matrix view: element (i, j) at p[i * rs + j * cs], optionally conjugated.
struct ZView {
  const zd* p;
  int64_t rs, cs;
  bool conj;
};
// C (m x n, column-major ldc) = alpha * A (m x k) * B (k x n) + beta * C.
int zgemm(int64_t m, int64_t n, int64_t k, zd alpha, ZView A, ZView B, zd beta, zd* C, int64_t ldc,
          cudaStream_t s);
// Y = G^{-1} X for the cyclic Gram matrix of hats (h/6 [1 4 1]), column-major; may alias.
// work: caller-owned device scratch of n * cols complex values.
int gram_inverse(const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t n, int64_t cols, double h,
                 zd* work, cudaStream_t s);
// Y = alpha * G X + beta * Y (cyclic tridiagonal), column-major.
int gram_apply(const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t n, int64_t cols, double h,
               double alpha, double beta, cudaStream_t s);
// Column 2-norms of an m x n column-major block into out (device, n doubles).
int column_norms(const zd* X, int64_t ld, int64_t m, int64_t n, double* out, cudaStream_t s);
// out[c] = sum_i conj(X[i, c]) Y[i, c] for the n columns of m x n blocks (device, n complex).
int column_dotc(const zd* X, int64_t ldx, const zd* Y, int64_t ldy, int64_t m, int64_t n, zd* out,
                cudaStream_t s);
// Complex Gaussian samples (unit variance per complex entry), Philox-4x32 counter based.
int gaussian_fill(zd* X, int64_t ld, int64_t m, int64_t n, uint64_t seed, uint64_t offset,
                  cudaStream_t s);
// Y(:, c) = a X(:, c) + b Y(:, c)
int axpby(int64_t m, int64_t n, zd a, const zd* X, int64_t ldx, zd b, zd* Y, int64_t ldy,
          cudaStream_t s);
// G (b x b, column-major) = X^H X for X m x b (b <= 64); work holds
// ceil(m/256) * b * b partial sums.
int gram_matrix(const zd* X, int64_t ld, int64_t m, int b, zd* G, zd* work, cudaStream_t s);
// Pivoted Cholesky of a Hermitian b x b Gram (device, column-major ld = b): returns
// numerical rank r (pivots >= tol^2 * max) and writes R (upper, r x b in permuted order)
// and the pivot permutation.  Runs in one thread block.
int pivoted_cholesky(zd* Gm, int b, double rel_tol, int* perm, int* rank_dev, cudaStream_t s);
// Y(:, 0:r) = X(:, perm[0:r]) R[0:r, 0:r]^{-1} (b <= 64; work: r x r scratch for
// R^{-1}; Y must not alias X)
int trsm_right_upper(const zd* X, int64_t ldx, int64_t m, const zd* R, int b, const int* perm,
                     const int* rank_dev, int rank_host, zd* Y, int64_t ldy, zd* work, cudaStream_t s);
// LU with partial pivoting of an n x n column-major matrix (in place) and explicit inverse.
int lu_inverse(zd* A, int64_t n, zd* Ainv, int* piv, int* info_dev, double* minpiv_dev,
               cudaStream_t s);

// ---------------------------------------------------------------- right-hand sides / far field
// split_phase: FP64 phase at one point per hat and FP32 offsets (~1e-7; mixed form)
int planewave_rhs(const Points& near, const double* wn, const double* xn, int q, int64_t N,
                  double h, double k, const double* angles, int B, zd* e, zd* hv, int64_t ld,
                  cudaStream_t s, bool split_phase = false);
int farfield_matrix(const Points& near, const double* wn, const double* xn, int q, int64_t N,
                    double h, double k, const double* phi, int nphi, zd* E, int64_t lde,
                    cudaStream_t s);

}  // namespace wcs
