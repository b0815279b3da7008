// C ABI and host orchestration of the Woodbury-circulant solver.
//
// Sec. III, Eq. (5)/(6): C = (G/2 + D~) G^{-1} (G/2 - D) + S~ G^{-1} N is
// never formed; it is applied matrix-free from the four assembled operators.
// Sec. V: C_c (the same operator on the circle of equal perimeter) is
// circulant; its eigenvalues mu_C come from the FFT of the first rows of the
// circle operators.  Eq. (7): C - C_c = U V^T by randomized range finding;
// Eq. (8)/(9): Woodbury with the capacitance K = I + V^T C_c^{-1} U.
#include <algorithm>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wcs.h"
#include "internal.h"
#include "gemm_tc.h"
#include "exact.h"

namespace wcs {
std::atomic<unsigned long long> g_launches{0};
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
}  // namespace wcs

using namespace wcs;

enum Stage { ST_NEW = 0, ST_CONTOUR = 1, ST_MESH = 2, ST_ASSEMBLED = 3, ST_SKELETON = 4, ST_FACTORED = 5 };

// Owned device buffer: grows on demand (contents not kept), freed by release()
// or when it goes out of scope; not copyable.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int ensure(size_t b) {
    if (b <= bytes) return 0;
    cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (cudaMalloc(&p, b) != cudaSuccess) { set_error("out of device memory"); return WCS_ERR_OOM; }
    bytes = b;
    return 0;
  }
  void release() { cudaFree(p); p = nullptr; bytes = 0; }
  zd* z() { return (zd*)p; }
  double* d() { return (double*)p; }
};

struct wcs_ctx {
  wcs_options opt;
  cudaStream_t s = nullptr;
  int stage = ST_NEW;
  Contour contour{}, circle{};
  ArcTable arc{}, arc_c{};
  int64_t N = 0, ld = 0;
  double L = 0, h = 0, a = 0, k = 0, kmin = 0;
  zd kt = mkz(0.0);
  QuadTables quad;
  DevBuf xf, xn, wn, wlog;                // device rule nodes / weights
  DevBuf pts_far, pts_near, pts_far_c, pts_near_c;
  Points far, near, far_c, near_c;
  DevBuf ops;                             // S, D, Dt, N (row-major, ld)
  zd *S = nullptr, *D = nullptr, *Dt = nullptr, *Nk = nullptr;
  DevBuf mu;                              // 6 x N: G, S, D, Dt, N, C
  double norm_cc = 0;
  FFTPlan fft{};
  bool fft_ready = false;
  Circ32 circ{};                          // mixed form: FP32 circulant applies (built from mu_C on first use)
  double kinv_res = -1.0;                 // ||I - K K^-1||_F / sqrt(r) of the last factor (-1: not measured)
  int rank = -1;
  DevBuf U, Vw, Wt;                       // N x rank each
  DevBuf w1, w2, w3, w4, w5;              // N x chunk scratch
  DevBuf small;                           // small scratch
  DevBuf gwork;                           // work of the Gram inverse (N x cols)
  // mixed-precision form
  bool mixed = false;
  int planes = 2, rhs_planes = 2;
  int64_t ldp = 0;                        // plane leading dimension (bf16 elements)
  DevBuf opplanes;                        // [op][layout][plane] N x ldp bf16
  DevBuf centres, offs;                   // element centres (FP64), far offsets (FP32)
  DevBuf stage0, stage1, stage2;          // staged right-hand blocks (bf16 planes)
  int64_t stage_cols = 0;
  DevBuf tcerr;
  DevBuf gW;                 // split-K workspace of the small contractions (FP32)
  DevBuf qh, qt;             // skeleton basis as resident bf16 planes: rows conj(q_i); rows of Q
  DevBuf gA, gB;                          // staging for general complex tensor products
  DevBuf sol_e, sol_h, sol_b, sol_ang, sol_j;   // solve blocks (grow-only, kept across calls)
  DevBuf Kinv;                            // r x r capacitance inverse (adjoint solves)
  DevBuf Wa;                              // N x r: C_c^-H V_w, formed at the first adjoint solve
  // exact residuals (mixed form, exact_residual = 1): fixed-point slices of
  // the four operators (layout 0), built at the first solve that needs them
  DevBuf exops, exrhs, exws;
  ExactOperand exA[4];
  bool exact_ready = false;
  // optional per-kernel timing: CUDA events on the context stream
  bool profile = false;
  struct Rec { int cat; cudaEvent_t a, b; double flops, bytes; };
  std::vector<Rec> recs;
};

enum StatCat { CAT_GEMM_TC = 0, CAT_ASSEMBLY = 1, CAT_FFT = 2, CAT_ZGEMM = 3, CAT_SKELETON = 4,
               CAT_FACTOR = 5, CAT_SOLVE = 6, CAT_GEMM_ACC = 7, CAT_SAMPLE = 8, CAT_PROJECT = 9,
               CAT_ORTH = 10, CAT_VW = 11, CAT_INVERSE = 12, CAT_GEMM_EXACT = 13, CAT_ASSEMBLY_FAST = 14,
               CAT_GEMM_PER = 15, CAT_COUNT = 16 };

struct ProfScope {
  wcs_ctx* c;
  int cat;
  double flops, bytes;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(wcs_ctx* c_, int cat_, double f, double by) : c(c_), cat(cat_), flops(f), bytes(by) {
    if (!c->profile) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->s);
  }
  ~ProfScope() {
    if (!c->profile) return;
    cudaEventRecord(b, c->s);
    c->recs.push_back({cat, a, b, flops, bytes});
  }
};

static uint16_t* plane_ptr(wcs_ctx* c, int op, int layout, int plane) {
  const int64_t per = c->N * c->ldp;
  return (uint16_t*)c->opplanes.p + (((int64_t)op * 2 + layout) * c->planes + plane) * per;
}

static zd* mu_ptr(wcs_ctx* c, int which) { return c->mu.z() + (int64_t)which * c->N; }
enum { MU_G = 0, MU_S = 1, MU_D = 2, MU_DT = 3, MU_N = 4, MU_C = 5 };

// ----------------------------------------------------------------------------- helpers
static ZView op_view(const zd* A, int64_t ld, bool adjoint) {
  if (!adjoint) return ZView{A, ld, 1, false};
  return ZView{A, 1, ld, true};
}
static ZView blk(const zd* X, int64_t ld) { return ZView{X, 1, ld, false}; }
static ZView blkH(const zd* X, int64_t ld) { return ZView{X, ld, 1, true}; }

#define TRY(x)              \
  do {                      \
    int _r = (x);           \
    if (_r) return _r;      \
  } while (0)

// Y = G^{-1} X (cyclic Gram matrix) with the context's own work buffer.
static int ginv(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols) {
  if (cols <= 0) return 0;
  TRY(c->gwork.ensure(sizeof(zd) * c->N * cols));
  return gram_inverse(X, ldx, Y, ldy, c->N, cols, c->h, c->gwork.z(), c->s);
}

static int ensure_work(wcs_ctx* c, int64_t cols) {
  size_t b = sizeof(zd) * c->N * std::max<int64_t>(cols, 1);
  TRY(c->w1.ensure(b));
  TRY(c->w2.ensure(b));
  TRY(c->w3.ensure(b));
  TRY(c->w4.ensure(b));
  TRY(c->w5.ensure(b));
  return 0;
}

// the device flag of the bounded waits in the tensor-core kernels: zeroed when allocated
static int ensure_tcerr(wcs_ctx* c) {
  if (c->tcerr.p) return 0;
  TRY(c->tcerr.ensure(sizeof(int)));
  cudaMemsetAsync(c->tcerr.p, 0, sizeof(int), c->s);
  return 0;
}

static int ensure_stage(wcs_ctx* c, int64_t cols) {
  if (cols <= c->stage_cols) return 0;
  const size_t b = sizeof(uint16_t) * (size_t)(2 * cols) * c->ldp * c->rhs_planes;
  TRY(c->stage0.ensure(b));
  TRY(c->stage1.ensure(b));
  TRY(c->stage2.ensure(b));
  TRY(ensure_tcerr(c));
  c->stage_cols = cols;
  return 0;
}

static int stage(wcs_ctx* c, DevBuf& buf, const zd* X, int64_t ldx, int64_t cols, int conj) {
  uint16_t* P[3];
  const int64_t per = 2 * c->stage_cols * c->ldp;
  for (int p = 0; p < 3; ++p) P[p] = (uint16_t*)buf.p + p * per;
  return stage_rhs(X, c->N, cols, ldx, conj, c->rhs_planes, P, c->ldp, c->s);
}

// Y = alpha * op(X) + beta * Y on the tensor cores, op one of the assembled
// operators (0 S~, 1 D, 2 D~, 3 N), X already staged in `buf`.  adjoint uses
// the transposed planes: A^H x = conj(A^T conj(x)) (buf staged with conj).
static bool debug_finite();
static int check_tc(wcs_ctx* c);

// Precision of a tensor-core operator product (mixed form):
//   PREC_FAST      two leading planes, one accumulator over all of K (~1e-4 at
//                  K ~ 1e5): Woodbury products, the range finder's projections
//   PREC_ACCURATE  all stored planes, accumulator drained every ACC_DRAIN
//                  K = 16 steps (~1e-7): refinement residual
//   PREC_PERIODIC  two leading planes, accumulator drained every 64 steps
//                  (~1e-5): residual updates R <- R - C dx, whose error scales
//                  with |dx|; the skeleton's samples and V_w (the wide-tile
//                  kernel is also the faster one at these widths)
//   PREC_FAST1     leading plane only, one product (~4e-3): optional skeleton
//                  sampling (sample_planes = 1)
//   PREC_EXACT     fixed-point slices of operator and vector, integer
//                  products, FP64 sums (exact.cu): residuals of refinement
//                  below the accurate floor (forward products only)
enum { PREC_FAST = 0, PREC_ACCURATE = 1, PREC_PERIODIC = 2, PREC_FAST1 = 3, PREC_EXACT = 4 };

// K = 16 steps per drain of the accurate product: one shared-memory stage
// (K = 64), whose products the kernel issues smallest first across the four
// steps.  Measured at N = 32768 (K = 65536, 1024 plane waves) against a solve
// with exact residuals: drain 1 took 45.1 ms per product and left 3.0e-7
// (max over 64 columns), drain 4 issued step by step 36.7 ms and 3.5e-7; the
// error floor is set by the three-plane split, not by the drain.
constexpr int ACC_DRAIN = 4;

// Algorithmic HBM bytes of one contraction: every plane of A and B read once,
// the complex FP64 output written (and read when beta != 0).
static double tc_bytes(const TcArgs& t, int pa, int pb) {
  const double out = 16.0 * t.M * (t.Nc / 2) * ((t.beta.x != 0.0 || t.beta.y != 0.0) ? 2.0 : 1.0);
  return 2.0 * ((double)pa * t.M * t.K + (double)pb * t.Nc * t.K) + out;
}

static int tc_apply(wcs_ctx* c, int op, bool adjoint, DevBuf& buf, int64_t cols, zd alpha, zd beta, zd* Y,
                    int64_t ldy, int mode = PREC_FAST) {
  const bool accurate = (mode == PREC_ACCURATE);
  const int P = accurate ? std::min(c->planes, c->rhs_planes)
                         : (mode == PREC_FAST1 ? 1 : std::min(2, std::min(c->planes, c->rhs_planes)));
  TcOperand A, B;
  A.planes = P;
  A.ld = c->ldp;
  for (int p = 0; p < P; ++p) A.plane[p] = plane_ptr(c, op, adjoint ? 1 : 0, p);
  B.planes = P;
  B.ld = c->ldp;
  const int64_t per = 2 * c->stage_cols * c->ldp;
  for (int p = 0; p < P; ++p) B.plane[p] = (uint16_t*)buf.p + p * per;
  TcArgs t;
  t.M = (int)c->N;
  t.Nc = (int)(2 * cols);
  t.K = (int)(2 * c->N);
  tc_products(P, t);
  t.epi = EPI_CPLX_F64;
  t.conj_out = adjoint ? 1 : 0;
  t.out = Y;
  t.ldo = ldy;
  t.alpha = alpha;
  t.beta = beta;
  t.err = (int*)c->tcerr.p;
  t.drain = (mode == PREC_PERIODIC) ? 64 : (accurate ? ACC_DRAIN : 1);
  const bool drained = (mode == PREC_ACCURATE || mode == PREC_PERIODIC);
  ProfScope ps(c, mode == PREC_PERIODIC ? CAT_GEMM_PER : (drained ? CAT_GEMM_ACC : CAT_GEMM_TC),
               2.0 * t.M * (double)t.Nc * t.K,
               tc_bytes(t, P, P));
  TRY(drained ? gemm_tc_accurate(A, B, t, c->s) : gemm_tc(A, B, t, c->s));
  if (debug_finite()) {
    int r = check_tc(c);
    if (r) fprintf(stderr, "[wcs debug] operator product op=%d adj=%d mode=%d M=%d Nc=%d K=%d: %s\n", op,
                   (int)adjoint, mode, t.M, t.Nc, t.K, g_err.c_str());
    return r;
  }
  return 0;
}

static int check_tc(wcs_ctx* c) {
  int e = 0;
  // the flag exists once a tensor-core product has run on this context
  if (c->tcerr.p) {
    const cudaError_t m = cudaMemcpyAsync(&e, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (m != cudaSuccess) { set_error(std::string("device: ") + cudaGetErrorString(m)); return WCS_ERR_CUDA; }
  }
  cudaError_t r = cudaStreamSynchronize(c->s);
  if (r != cudaSuccess) { set_error(std::string("device: ") + cudaGetErrorString(r)); return WCS_ERR_CUDA; }
  if (e) { set_error("tensor-core contraction: a bounded wait expired"); return WCS_ERR_TIMEOUT; }
  return 0;
}

// C (m x n, column-major ldc) = alpha * A (m x k view) * X (k x n, column-major) + beta * C.
// Mixed form: on the tensor cores through staged split-bf16 planes; FP64 form: zgemm.
static int cgemm(wcs_ctx* c, int64_t m, int64_t n, int64_t k, zd alpha, ZView A, const zd* X, int64_t ldx,
                 zd beta, zd* C, int64_t ldc, bool accurate = false) {
  if (m <= 0 || n <= 0) return 0;
  if (!c->mixed || k < 64) return zgemm(m, n, k, alpha, A, blk(X, ldx), beta, C, ldc, c->s);
  // fast: two planes, one accumulator; accurate: three planes, the drained
  // accumulation of the refinement residual
  const int P = accurate ? 3 : 2;
  const int64_t ldk = ((2 * k + 63) / 64) * 64;
  // grow the staging buffers geometrically: the skeleton calls this with a
  // basis that widens block by block
  const size_t needA = sizeof(uint16_t) * (size_t)m * ldk * P, needB = sizeof(uint16_t) * (size_t)(2 * n) * ldk * P;
  if (needA > c->gA.bytes) TRY(c->gA.ensure(std::max(needA, c->gA.bytes + c->gA.bytes / 2)));
  if (needB > c->gB.bytes) TRY(c->gB.ensure(std::max(needB, c->gB.bytes + c->gB.bytes / 2)));
  TRY(ensure_tcerr(c));
  uint16_t *pa[3], *pb[3];
  for (int p = 0; p < 3; ++p) {
    pa[p] = (uint16_t*)c->gA.p + (int64_t)p * m * ldk;
    pb[p] = (uint16_t*)c->gB.p + (int64_t)p * 2 * n * ldk;
  }
  if (ldk != 2 * k) {   // zero the padding of the K dimension
    cudaMemsetAsync(c->gA.p, 0, sizeof(uint16_t) * (size_t)m * ldk * P, c->s);
    cudaMemsetAsync(c->gB.p, 0, sizeof(uint16_t) * (size_t)(2 * n) * ldk * P, c->s);
  }
  TRY(stage_view(A.p, m, k, A.rs, A.cs, A.conj ? 1 : 0, P, pa, ldk, c->s));
  TRY(stage_rhs(X, k, n, ldx, 0, P, pb, ldk, c->s));
  TcOperand oa, ob;
  oa.planes = ob.planes = P;
  oa.ld = ob.ld = ldk;
  for (int p = 0; p < P; ++p) { oa.plane[p] = pa[p]; ob.plane[p] = pb[p]; }
  TcArgs t;
  t.M = (int)m; t.Nc = (int)(2 * n); t.K = (int)(2 * k);
  tc_products(P, t);
  t.epi = EPI_CPLX_F64;
  t.out = C; t.ldo = ldc; t.alpha = alpha; t.beta = beta;
  t.err = (int*)c->tcerr.p;
  TRY(c->gW.ensure((size_t)32 << 20));
  t.ws = (float*)c->gW.p;
  t.ws_elems = (int64_t)(c->gW.bytes / sizeof(float));
  ProfScope ps(c, accurate ? CAT_GEMM_ACC : CAT_GEMM_TC, 2.0 * t.M * (double)t.Nc * t.K, tc_bytes(t, P, P));
  if (accurate) {
    t.drain = ACC_DRAIN;
    TRY(gemm_tc_accurate(oa, ob, t, c->s));
  } else {
    TRY(gemm_tc(oa, ob, t, c->s));
  }
  return 0;
}

// cgemm with A already held as two split-bf16 planes (row-major real M x 2K,
// leading dimension lda); A_view is the same matrix for the FP64 fallback.
static int cgemm_planes(wcs_ctx* c, int64_t m, int64_t n, int64_t k, zd alpha, const uint16_t* A0,
                        const uint16_t* A1, int64_t lda, ZView A_view, const zd* X, int64_t ldx, zd beta, zd* C,
                        int64_t ldc) {
  if (m <= 0 || n <= 0) return 0;
  if (!c->mixed || k < 64) return cgemm(c, m, n, k, alpha, A_view, X, ldx, beta, C, ldc);
  const int P = 2;
  const int64_t ldk = ((2 * k + 63) / 64) * 64;
  const size_t needB = sizeof(uint16_t) * (size_t)(2 * n) * ldk * P;
  if (needB > c->gB.bytes) TRY(c->gB.ensure(std::max(needB, c->gB.bytes + c->gB.bytes / 2)));
  TRY(ensure_tcerr(c));
  uint16_t* pb[3];
  for (int p = 0; p < 3; ++p) pb[p] = (uint16_t*)c->gB.p + (int64_t)p * 2 * n * ldk;
  TRY(stage_rhs(X, k, n, ldx, 0, P, pb, ldk, c->s));
  TcOperand oa, ob;
  oa.planes = ob.planes = P;
  oa.ld = lda;
  ob.ld = ldk;
  oa.plane[0] = A0; oa.plane[1] = A1;
  ob.plane[0] = pb[0]; ob.plane[1] = pb[1];
  TcArgs t;
  t.M = (int)m; t.Nc = (int)(2 * n); t.K = (int)(2 * k);
  tc_products(P, t);
  t.epi = EPI_CPLX_F64;
  t.out = C; t.ldo = ldc; t.alpha = alpha; t.beta = beta;
  t.err = (int*)c->tcerr.p;
  TRY(c->gW.ensure((size_t)32 << 20));
  t.ws = (float*)c->gW.p;
  t.ws_elems = (int64_t)(c->gW.bytes / sizeof(float));
  ProfScope ps(c, CAT_GEMM_TC, 2.0 * t.M * (double)t.Nc * t.K, tc_bytes(t, P, P));
  TRY(gemm_tc(oa, ob, t, c->s));
  return 0;
}

// The operators' exact slices (from their layout-0 split-bf16 planes), once per assembly.
static int ensure_exact_ops(wcs_ctx* c) {
  if (c->exact_ready) return 0;
  int64_t ld = 0, nch = 0;
  size_t sb = 0, eb = 0;
  exact_operand_alloc_bytes(c->N, 2 * c->N, &ld, &nch, &sb, &eb);
  const size_t per_op = ((EX_SLICES * sb + eb + 255) / 256) * 256;   // keeps every slice 256-byte aligned
  TRY(c->exops.ensure(4 * per_op));
  char* base = (char*)c->exops.p;
  for (int op = 0; op < 4; ++op) {
    ExactOperand& o = c->exA[op];
    o.ld = ld;
    o.nchunks = nch;
    for (int q = 0; q < EX_SLICES; ++q) o.slice[q] = (uint16_t*)(base + op * per_op + q * sb);
    o.expo = (int16_t*)(base + op * per_op + EX_SLICES * sb);
    const uint16_t* P[3] = {plane_ptr(c, op, 0, 0), c->planes > 1 ? plane_ptr(c, op, 0, 1) : nullptr,
                            c->planes > 2 ? plane_ptr(c, op, 0, 2) : nullptr};
    TRY(exact_slice_planes(P, c->planes, c->N, 2 * c->N, c->ldp, o, c->s));
  }
  c->exact_ready = true;
  return 0;
}

// Y = alpha * op X + beta * Y, exactly up to FP64 sums (op 0 S~, 1 D, 2 D~, 3 N).
static int ex_apply(wcs_ctx* c, int op, const zd* X, int64_t ldx, int64_t cols, zd alpha, zd beta, zd* Y,
                    int64_t ldy) {
  if (cols <= 0) return 0;
  TRY(ensure_exact_ops(c));
  TRY(ensure_tcerr(c));
  const int64_t N = c->N, G = 256;   // right-hand sides per pass: bounds the split-K workspace
  int64_t ld = 0, nch = 0;
  size_t sb = 0, eb = 0;
  exact_operand_alloc_bytes(2 * G, 2 * N, &ld, &nch, &sb, &eb);
  const size_t sbr = ((sb + 255) / 256) * 256;
  TRY(c->exrhs.ensure(EX_SLICES * sbr + sizeof(int16_t) * (size_t)G * nch + 256));
  const int64_t ws_elems = nch * 2 * G * N;
  TRY(c->exws.ensure(sizeof(float) * (size_t)ws_elems));
  ExactOperand B;
  B.ld = ld;
  B.nchunks = nch;
  for (int q = 0; q < EX_SLICES; ++q) B.slice[q] = (uint16_t*)((char*)c->exrhs.p + q * sbr);
  B.expo = (int16_t*)((char*)c->exrhs.p + EX_SLICES * sbr);
  ProfScope ps(c, CAT_GEMM_EXACT, 2.0 * N * (2.0 * cols) * (2.0 * N), 0.0);
  for (int64_t c0 = 0; c0 < cols; c0 += G) {
    const int64_t cc = std::min(G, cols - c0);
    TRY(exact_slice_rhs(X + c0 * ldx, N, cc, ldx, 0, B, c->s));
    TRY(exact_product(c->exA[op], (int)N, B, (int)cc, (int)(2 * N), alpha, beta, 0, Y + c0 * ldy, ldy,
                      (float*)c->exws.p, ws_elems, (int*)c->tcerr.p, c->s));
  }
  return 0;
}

// C X (forward) with exact operator products; FP64 Gram algebra between them.
static int apply_C_exact(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols) {
  const int64_t N = c->N;
  zd* T1 = c->w1.z();
  zd* T2 = c->w2.z();
  const zd one = mkz(1.0), zero = mkz(0.0), mone = mkz(-1.0);
  TRY(ex_apply(c, 1, X, ldx, cols, mone, zero, T1, N));    // -D X
  TRY(ex_apply(c, 3, X, ldx, cols, one, zero, T2, N));     // N X
  TRY(gram_apply(X, ldx, T1, N, N, cols, c->h, 0.5, 1.0, c->s));
  TRY(ginv(c, T1, N, T1, N, cols));
  TRY(ginv(c, T2, N, T2, N, cols));
  TRY(ex_apply(c, 2, T1, N, cols, one, zero, Y, ldy));     // D~ T1
  TRY(ex_apply(c, 0, T2, N, cols, one, one, Y, ldy));      // + S~ T2
  TRY(gram_apply(T1, N, Y, ldy, N, cols, c->h, 0.5, 1.0, c->s));
  return 0;
}

static int apply_C_mixed(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols, bool adj,
                         int acc) {
  if (acc == PREC_EXACT && !adj) return apply_C_exact(c, X, ldx, Y, ldy, cols);
  if (acc == PREC_EXACT) acc = PREC_ACCURATE;   // adjoint products: the drained split-bf16 product
  const int64_t N = c->N;
  zd* T1 = c->w1.z();
  zd* T2 = c->w2.z();
  const zd one = mkz(1.0), zero = mkz(0.0), mone = mkz(-1.0);
  TRY(ensure_stage(c, cols));
  const int cj = adj ? 1 : 0;
  TRY(stage(c, c->stage0, X, ldx, cols, cj));
  if (!adj) {
    TRY(tc_apply(c, 1, false, c->stage0, cols, mone, zero, T1, N, acc));   // -D X
    TRY(tc_apply(c, 3, false, c->stage0, cols, one, zero, T2, N, acc));    // N X
  } else {
    TRY(tc_apply(c, 2, true, c->stage0, cols, one, zero, T1, N, acc));     // D~^H X
    TRY(tc_apply(c, 0, true, c->stage0, cols, one, zero, T2, N, acc));     // S~^H X
  }
  TRY(gram_apply(X, ldx, T1, N, N, cols, c->h, 0.5, 1.0, c->s));
  TRY(ginv(c, T1, N, T1, N, cols));
  TRY(ginv(c, T2, N, T2, N, cols));
  TRY(stage(c, c->stage1, T1, N, cols, cj));
  TRY(stage(c, c->stage2, T2, N, cols, cj));
  if (!adj) {
    TRY(tc_apply(c, 2, false, c->stage1, cols, one, zero, Y, ldy, acc));   // D~ T1
    TRY(tc_apply(c, 0, false, c->stage2, cols, one, one, Y, ldy, acc));    // + S~ T2
  } else {
    TRY(tc_apply(c, 1, true, c->stage1, cols, mone, zero, Y, ldy, acc));   // -D^H T1
    TRY(tc_apply(c, 3, true, c->stage2, cols, one, one, Y, ldy, acc));     // + N^H T2
  }
  TRY(gram_apply(T1, N, Y, ldy, N, cols, c->h, 0.5, 1.0, c->s));
  return 0;
}

// Y = C X (adjoint: C^H X); uses w1, w2 as temporaries.  Y must not alias X.
static int apply_C(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols, bool adj,
                   int mode = PREC_FAST) {
  if (c->mixed) return apply_C_mixed(c, X, ldx, Y, ldy, cols, adj, mode);
  const int64_t N = c->N;
  zd* T1 = c->w1.z();
  zd* T2 = c->w2.z();
  const zd one = mkz(1.0), zero = mkz(0.0), mone = mkz(-1.0);
  if (!adj) {
    // T1 = (G/2 - D) X, T2 = N X
    TRY(zgemm(N, cols, N, mone, op_view(c->D, c->ld, false), blk(X, ldx), zero, T1, N, c->s));
    TRY(gram_apply(X, ldx, T1, N, N, cols, c->h, 0.5, 1.0, c->s));
    TRY(zgemm(N, cols, N, one, op_view(c->Nk, c->ld, false), blk(X, ldx), zero, T2, N, c->s));
    TRY(ginv(c, T1, N, T1, N, cols));
    TRY(ginv(c, T2, N, T2, N, cols));
    // Y = (G/2 + D~) T1 + S~ T2
    TRY(zgemm(N, cols, N, one, op_view(c->Dt, c->ld, false), blk(T1, N), zero, Y, ldy, c->s));
    TRY(zgemm(N, cols, N, one, op_view(c->S, c->ld, false), blk(T2, N), one, Y, ldy, c->s));
    TRY(gram_apply(T1, N, Y, ldy, N, cols, c->h, 0.5, 1.0, c->s));
  } else {
    // C^H = (G/2 - D)^H G^{-1} (G/2 + D~)^H + N^H G^{-1} S~^H   (G real symmetric)
    TRY(zgemm(N, cols, N, one, op_view(c->Dt, c->ld, true), blk(X, ldx), zero, T1, N, c->s));
    TRY(gram_apply(X, ldx, T1, N, N, cols, c->h, 0.5, 1.0, c->s));
    TRY(zgemm(N, cols, N, one, op_view(c->S, c->ld, true), blk(X, ldx), zero, T2, N, c->s));
    TRY(ginv(c, T1, N, T1, N, cols));
    TRY(ginv(c, T2, N, T2, N, cols));
    TRY(zgemm(N, cols, N, mone, op_view(c->D, c->ld, true), blk(T1, N), zero, Y, ldy, c->s));
    TRY(zgemm(N, cols, N, one, op_view(c->Nk, c->ld, true), blk(T2, N), one, Y, ldy, c->s));
    TRY(gram_apply(T1, N, Y, ldy, N, cols, c->h, 0.5, 1.0, c->s));
  }
  return 0;
}

// Y = C_c X, C_c^H X or C_c^{-1} X by FFT (mode 0, 1, 2).  Y may alias X.
static int apply_Cc(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols, int mode) {
  const int64_t N = c->N;
  if (c->mixed && circ32_supported(N)) {
    // mixed form: the three-pass FP32 transform (x and y read and written
    // once in FP64, one FP32 scratch round trip in between)
    if (!c->circ.ready) TRY(circ32_prepare(c->circ, mu_ptr(c, MU_C), N, c->s));
    ProfScope ps(c, CAT_FFT, 0.0, 64.0 * (double)N * cols);
    return circ32_apply(c->circ, X, ldx, Y, ldy, cols, mode, c->s);
  }
  if (X != Y) {
    cudaError_t e = cudaMemcpy2DAsync(Y, sizeof(zd) * ldy, X, sizeof(zd) * ldx, sizeof(zd) * N, cols,
                                      cudaMemcpyDeviceToDevice, c->s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  }
  ProfScope ps(c, CAT_FFT, 0.0, 4.0 * 16.0 * (double)N * cols);
  TRY(fft_columns(c->fft, Y, ldy, cols, -1, c->s));
  // mode 0: C_c, 1: C_c^H, 2: C_c^-1, 3: C_c^-H (eigenvalues mu_C, conj(mu_C))
  TRY(scale_columns(Y, N, ldy, cols, mu_ptr(c, MU_C), mode == 2 || mode == 3, mode == 1 || mode == 3,
                    1.0 / (double)N, c->s));
  TRY(fft_columns(c->fft, Y, ldy, cols, +1, c->s));
  return 0;
}

// Y = (C - C_c) X or its adjoint; uses w1, w2, w3.
static int apply_remainder(wcs_ctx* c, const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t cols,
                           bool adj, int mode = PREC_FAST) {
  TRY(apply_C(c, X, ldx, Y, ldy, cols, adj, mode));
  zd* T3 = c->w3.z();
  TRY(apply_Cc(c, X, ldx, T3, c->N, cols, adj ? 1 : 0));
  TRY(axpby(c->N, cols, mkz(-1.0), T3, c->N, mkz(1.0), Y, ldy, c->s));
  return 0;
}

// X = C^{-1} B through Eq. (9); uses w3 for Y = C_c^{-1} B and small for Z.
static int woodbury(wcs_ctx* c, const zd* B, int64_t ldb, zd* X, int64_t ldx, int64_t cols) {
  const int64_t N = c->N;
  TRY(apply_Cc(c, B, ldb, X, ldx, cols, 2));
  if (c->rank <= 0) return 0;
  const int64_t r = c->rank;
  TRY(c->small.ensure(sizeof(zd) * r * cols));
  zd* Z = c->small.z();
  // Z = V^T Y = Vw^H Y ; X = Y - Wt Z
  TRY(cgemm(c, r, cols, N, mkz(1.0), blkH(c->Vw.z(), N), X, ldx, mkz(0.0), Z, r));
  TRY(cgemm(c, N, cols, r, mkz(-1.0), blk(c->Wt.z(), N), Z, r, mkz(1.0), X, ldx));
  return 0;
}

// X = C^{-H} B through the adjoint of Eq. (9).  With C~ = C_c + Q V_w^H:
//   C~^-H B = Y - (C_c^-H V_w) K^-H (Q^H Y),  Y = C_c^-H B,  K = I + V_w^H C_c^-1 Q,
// the capacitance matrix of the forward solve.  C_c^-H V_w is formed once.
static int woodbury_adj(wcs_ctx* c, const zd* B, int64_t ldb, zd* X, int64_t ldx, int64_t cols) {
  const int64_t N = c->N;
  TRY(apply_Cc(c, B, ldb, X, ldx, cols, 3));
  if (c->rank <= 0) return 0;
  const int64_t r = c->rank;
  if (!c->Kinv.p) { set_error("adjoint solve: capacitance inverse missing (factor again)"); return WCS_ERR_STATE; }
  if (!c->Wa.p) {
    TRY(c->Wa.ensure(sizeof(zd) * N * r));
    TRY(apply_Cc(c, c->Vw.z(), N, c->Wa.z(), N, r, 3));
  }
  TRY(c->small.ensure(sizeof(zd) * 2 * r * cols));
  zd* T = c->small.z();
  zd* Z = T + r * cols;
  TRY(cgemm(c, r, cols, N, mkz(1.0), blkH(c->U.z(), N), X, ldx, mkz(0.0), T, r));    // Q^H Y
  TRY(cgemm(c, r, cols, r, mkz(1.0), blkH(c->Kinv.z(), r), T, r, mkz(0.0), Z, r));   // K^-H (Q^H Y)
  TRY(cgemm(c, N, cols, r, mkz(-1.0), blk(c->Wa.z(), N), Z, r, mkz(1.0), X, ldx));   // Y - C_c^-H V_w Z
  return 0;
}

// WCS_DEBUG_FINITE=1: check device buffers for non-finite values after each
// stage of the skeleton (diagnostic; synchronises)
static bool debug_finite() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("WCS_DEBUG_FINITE"); v = (e && e[0] == '1') ? 1 : 0; }
  return v == 1;
}
static int dbg_check(wcs_ctx* c, const zd* p, int64_t rows, int64_t cols, int64_t ld, const char* what) {
  if (!debug_finite() || rows <= 0 || cols <= 0) return 0;
  std::vector<zd> h(rows);
  for (int64_t j = 0; j < cols; ++j) {
    cudaMemcpyAsync(h.data(), p + j * ld, sizeof(zd) * rows, cudaMemcpyDeviceToHost, c->s);
    cudaStreamSynchronize(c->s);
    for (int64_t i = 0; i < rows; ++i)
      if (!std::isfinite(h[i].x) || !std::isfinite(h[i].y) || std::fabs(h[i].x) > 1e30 || std::fabs(h[i].y) > 1e30) {
        fprintf(stderr, "[wcs debug] non-finite or huge after %s at (%lld, %lld): %g %g\n", what, (long long)i,
                (long long)j, h[i].x, h[i].y);
        set_error(std::string("debug: non-finite after ") + what);
        return WCS_ERR_CUDA;
      }
  }
  return 0;
}

static int sync(wcs_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) { set_error(std::string("device: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  return 0;
}

// ----------------------------------------------------------------------------- kernels local to this file
__global__ void k_mu_finish(zd* mu, int64_t N, double h) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  double s, co;
  sincospi(2.0 * (double)m / (double)N, &s, &co);
  const zd G = mkz(h * (2.0 + co) / 3.0);
  mu[m] = G;
  const zd S = mu[N + m], D = mu[2 * N + m], Dt = mu[3 * N + m], Nk = mu[4 * N + m];
  const zd half = 0.5 * G;
  mu[5 * N + m] = zdiv((half + Dt) * (half - D) + S * Nk, G);
}

__global__ void k_absmax(const zd* x, int64_t n, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, zabs(x[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// X0 = K^H / (||K||_1 ||K||_inf): column/row absolute sums
// column sums: one block per column (contiguous); row sums: one thread per row
// (consecutive threads read consecutive rows of a column)
__global__ void k_col_abs_sums(const zd* K, int64_t r, double* colsum) {
  __shared__ double red[256];
  const int64_t i = blockIdx.x;
  double cs = 0.0;
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) cs += zabs(K[i * r + j]);
  red[threadIdx.x] = cs;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) colsum[i] = red[0];
}

__global__ void k_row_abs_sums(const zd* K, int64_t r, double* rowsum) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  double rs = 0.0;
  for (int64_t j = 0; j < r; ++j) rs += zabs(K[j * r + i]);
  rowsum[i] = rs;
}

__global__ void k_scaled_adjoint(const zd* K, int64_t r, const double* colsum, const double* rowsum, zd* X) {
  __shared__ double n1, ninf;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int64_t i = 0; i < r; ++i) { a = fmax(a, colsum[i]); b = fmax(b, rowsum[i]); }
    n1 = a;
    ninf = b;
  }
  __syncthreads();
  const double sc = 1.0 / (n1 * ninf);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % r, j = t / r;   // X(i, j) = conj(K(j, i)) * sc
    X[j * r + i] = sc * conj(K[i * r + j]);
  }
}

// T = 2I - T (in place)
__global__ void k_two_minus(zd* T, int64_t r) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= r * r) return;
  const int64_t i = t % r, j = t / r;
  zd v = -T[t];
  if (i == j) v.x += 2.0;
  T[t] = v;
}

// At = A^T for an r x r complex column-major A (At row-major A)
__global__ void k_transpose_z(const zd* __restrict__ A, int64_t r, zd* __restrict__ At) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= r * r) return;
  const int64_t i = t / r, j = t % r;   // At row i, column j (coalesced writes)
  At[t] = A[i + j * r];
}

// ||I - T||_F^2 partial sums (one block)
// ||T - I||_F in two deterministic stages: per-block partial sums, then one block
constexpr int EYE_BLOCKS = 304;
__global__ void k_eye_partial(const zd* T, int64_t r, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % r, j = t / r;
    zd v = T[t];
    if (i == j) v.x -= 1.0;
    s += abs2(v);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_eye_finish(const double* part, int n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

__global__ void k_add_identity(zd* K, int64_t r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) K[i * r + i] += mkz(1.0);
}

// per-column squared norms of an N x cols block
__global__ void k_colnorm2(const zd* X, int64_t ld, int64_t m, double* out) {
  __shared__ double red[256];
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += abs2(X[c * ld + i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// ----------------------------------------------------------------------------- C ABI
extern "C" {

const char* wcs_version(void) { return "wcs-gb300 0.1 (sm_103a, FP64 path)"; }

const char* wcs_last_error(void) { return g_err.c_str(); }

int wcs_default_options(wcs_options* o) {
  if (!o) { set_error("null options"); return WCS_ERR_ARG; }
  std::memset(o, 0, sizeof(*o));
  o->precision = WCS_PREC_FP64;
  o->q_far = 0;   // automatic: 6 (FP64 form) or 4 (mixed form)
  o->q_near = 0;   // automatic: 12 (FP64 form) or 8 (mixed form)
  o->near_band = 4;
  o->block = 32;
  o->max_refine = 12;
  o->refine_tol = 1e-12;
  o->rhs_chunk = 256;
  o->mixed_planes = 3;
  o->rhs_planes = 3;
  o->zfast = -1.0;  // automatic: 1000 in the mixed form (FP32 far pairs beyond k R = 1000), unused in FP64
  return WCS_OK;
}

int wcs_create(wcs_ctx** out, const wcs_options* opt, void* stream) {
  if (!out) { set_error("null output pointer"); return WCS_ERR_ARG; }
  wcs_options o;
  if (opt) o = *opt; else wcs_default_options(&o);
  if (o.precision != WCS_PREC_FP64 && o.precision != WCS_PREC_MIXED) { set_error("unknown precision mode"); return WCS_ERR_ARG; }
  if (o.precision == WCS_PREC_MIXED && (o.mixed_planes < 1 || o.mixed_planes > 3 || o.rhs_planes != o.mixed_planes)) {
    set_error("mixed form: 1 <= mixed_planes <= 3 and rhs_planes == mixed_planes");
    return WCS_ERR_ARG;
  }
  if (o.q_far == 0) o.q_far = (o.precision == WCS_PREC_MIXED) ? 4 : 6;
  if (o.q_near == 0) o.q_near = (o.precision == WCS_PREC_MIXED) ? 8 : 12;
  if (o.sample_planes == 0) o.sample_planes = 2;
  // FP32 far pairs beyond k R = 1000: at N = 32768 (k = 3642, superellipse)
  // this keeps the error against the FP64 form at 6.1e-7 for grazing
  // incidence (2000: 3.8e-7; all far pairs in FP32: 9.8e-7) with 1.7 s of
  // assembly (2000: 2.3 s); smaller problems have few pairs that far and stay
  // mostly in FP64
  if (o.zfast < 0.0) o.zfast = (o.precision == WCS_PREC_MIXED) ? 1000.0 : 0.0;
  if (o.sample_planes < 1 || o.sample_planes > 2) { set_error("sample_planes must be 1 or 2"); return WCS_ERR_ARG; }
  if (o.exact_residual != 0 && o.exact_residual != 1) { set_error("exact_residual must be 0 or 1"); return WCS_ERR_ARG; }
  if (o.q_far < 2 || o.q_far > 16 || o.q_near < 4 || o.q_near > 16 || o.near_band < 1 ||
      o.block < 1 || o.block > 64 || o.rhs_chunk < 1 || o.max_refine < 0) {
    set_error("option out of range");
    return WCS_ERR_ARG;
  }
  wcs_ctx* c = new wcs_ctx();
  c->opt = o;
  c->s = (cudaStream_t)stream;
  c->mixed = (o.precision == WCS_PREC_MIXED);
  c->planes = o.mixed_planes;
  c->rhs_planes = o.rhs_planes;
  c->quad.q_far = o.q_far;
  c->quad.q_near = o.q_near;
  c->quad.near_band = o.near_band;
  build_quad_tables(c->quad);
  *out = c;
  return WCS_OK;
}

static void free_mesh(wcs_ctx* c) {
  cudaFree(c->arc.cum); c->arc.cum = nullptr;
  cudaFree(c->arc_c.cum); c->arc_c.cum = nullptr;
  c->pts_far.release(); c->pts_near.release(); c->pts_far_c.release(); c->pts_near_c.release();
  c->ops.release(); c->mu.release();
  c->opplanes.release(); c->centres.release(); c->offs.release();
  c->stage0.release(); c->stage1.release(); c->stage2.release(); c->stage_cols = 0;
  c->gA.release(); c->gB.release(); c->gW.release(); c->qh.release(); c->qt.release();
  c->U.release(); c->Vw.release(); c->Wt.release(); c->Kinv.release(); c->Wa.release();
  c->sol_e.release(); c->sol_h.release(); c->sol_b.release(); c->sol_ang.release(); c->sol_j.release();
  c->exops.release(); c->exrhs.release(); c->exws.release(); c->exact_ready = false;
  if (c->fft_ready) { fft_plan_destroy(c->fft); c->fft_ready = false; }
  circ32_release(c->circ);
  c->kinv_res = -1.0;
  c->rank = -1;
}

int wcs_destroy(wcs_ctx* c) {
  if (!c) return WCS_OK;
  free_mesh(c);
  c->xf.release(); c->xn.release(); c->wn.release(); c->wlog.release();
  c->w1.release(); c->w2.release(); c->w3.release(); c->w4.release(); c->w5.release();
  c->small.release(); c->tcerr.release(); c->gwork.release();
  delete c;
  return WCS_OK;
}

static int set_contour(wcs_ctx* c, const Contour& k) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  free_mesh(c);
  c->contour = k;
  c->stage = ST_CONTOUR;
  return WCS_OK;
}

int wcs_contour_circle(wcs_ctx* c, double a) {
  if (!(a > 0)) { set_error("radius must be positive"); return WCS_ERR_ARG; }
  Contour k{};
  k.family = FAM_CIRCLE;
  k.a = a;
  return set_contour(c, k);
}

int wcs_contour_ellipse(wcs_ctx* c, double ax, double ay) {
  if (!(ax > 0 && ay > 0)) { set_error("semi-axes must be positive"); return WCS_ERR_ARG; }
  Contour k{};
  k.family = FAM_ELLIPSE;
  k.ax = ax;
  k.ay = ay;
  return set_contour(c, k);
}

int wcs_contour_superellipse(wcs_ctx* c, double ax, double ay, double p) {
  if (!(ax > 0 && ay > 0 && p >= 2.0)) { set_error("superellipse needs ax, ay > 0 and p >= 2"); return WCS_ERR_ARG; }
  Contour k{};
  k.family = FAM_SUPERELLIPSE;
  k.ax = ax;
  k.ay = ay;
  k.p = p;
  return set_contour(c, k);
}

int wcs_contour_fourier(wcs_ctx* c, int count, const double* cc, const double* ss) {
  if (count < 1 || count > kMaxFourier || !cc) { set_error("fourier: 1 <= count <= 64 and cos_c required"); return WCS_ERR_ARG; }
  if (!(cc[0] > 0)) { set_error("fourier: mean radius must be positive"); return WCS_ERR_ARG; }
  Contour k{};
  k.family = FAM_FOURIER;
  k.nf = count;
  for (int m = 0; m < count; ++m) { k.fc[m] = cc[m]; k.fs[m] = ss ? ss[m] : 0.0; }
  return set_contour(c, k);
}

int wcs_contour_perturb(wcs_ctx* c, int M, const double* alpha, const double* beta) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_CONTOUR) { set_error("set a contour first"); return WCS_ERR_STATE; }
  if (M < 0 || M > kMaxPerturb - 1 || (M > 0 && (!alpha || !beta))) {
    set_error("perturbation: 0 <= M <= 32 and alpha, beta required");
    return WCS_ERR_ARG;
  }
  Contour k = c->contour;
  k.np = M > 0 ? M + 1 : 0;
  for (int m = 0; m < kMaxPerturb; ++m) { k.pc[m] = 0.0; k.ps[m] = 0.0; }
  for (int m = 0; m < M; ++m) { k.pc[m] = alpha[m]; k.ps[m + 1] = beta[m]; }
  return set_contour(c, k);
}

static int build_points(wcs_ctx* c, const Contour& k, const ArcTable& t, DevBuf& buf, Points& P,
                        const double* xi_dev, int q, bool with_kappa) {
  const int64_t n = c->N * q;
  TRY(buf.ensure(sizeof(double) * n * 5));
  double* b = buf.d();
  P.x = b; P.y = b + n; P.nx = b + 2 * n; P.ny = b + 3 * n; P.kappa = with_kappa ? b + 4 * n : nullptr;
  P.n = n;
  return points_build(k, t, c->N, c->h, xi_dev, q, P, c->s);
}

int wcs_mesh(wcs_ctx* c, int64_t N, double k) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_CONTOUR) { set_error("set a contour first"); return WCS_ERR_STATE; }
  if (N < 12 || N > (int64_t)1 << 22) { set_error("N must be in [12, 4194304]"); return WCS_ERR_ARG; }
  free_mesh(c);
  c->stage = ST_CONTOUR;
  TRY(arc_table_build(c->contour, c->arc, c->s));
  c->L = c->arc.L;
  c->N = N;
  c->ld = (N + 7) & ~(int64_t)7;
  c->h = c->L / (double)N;
  c->a = c->L / (2.0 * WCS_PI);
  c->k = (k > 0) ? k : 2.0 * WCS_PI * ((double)N / 10.0) / c->L;
  if (c->k * c->h > 2.5) { set_error("k h > 2.5: mesh too coarse for the wavenumber"); return WCS_ERR_ARG; }
  c->kt = mkz(c->k, 0.4 * cbrt(c->k) * pow(c->a, -2.0 / 3.0));
  TRY(min_curvature(c->contour, c->arc, std::max<int64_t>(16 * N, 65536), &c->kmin, c->s));
  if (c->kmin < -1e-9) { set_error("contour is not convex (negative curvature)"); return WCS_ERR_NOT_CONVEX; }
  // equivalent circle
  c->circle = Contour{};
  c->circle.family = FAM_CIRCLE;
  c->circle.a = c->a;
  TRY(arc_table_build(c->circle, c->arc_c, c->s));
  // rules on device
  const int qf = c->opt.q_far, qn = c->opt.q_near;
  TRY(c->xf.ensure(sizeof(double) * 16));
  TRY(c->xn.ensure(sizeof(double) * 16));
  TRY(c->wn.ensure(sizeof(double) * 16));
  TRY(c->wlog.ensure(sizeof(double) * 3 * qn * qn));
  cudaMemcpyAsync(c->xf.p, c->quad.xf, sizeof(double) * qf, cudaMemcpyHostToDevice, c->s);
  cudaMemcpyAsync(c->xn.p, c->quad.xn, sizeof(double) * qn, cudaMemcpyHostToDevice, c->s);
  cudaMemcpyAsync(c->wn.p, c->quad.wn, sizeof(double) * qn, cudaMemcpyHostToDevice, c->s);
  for (int t = 0; t < 3; ++t)
    cudaMemcpyAsync(c->wlog.d() + t * qn * qn, c->quad.wlog[t].data(), sizeof(double) * qn * qn,
                    cudaMemcpyHostToDevice, c->s);
  TRY(build_points(c, c->contour, c->arc, c->pts_far, c->far, c->xf.d(), qf, false));
  TRY(build_points(c, c->contour, c->arc, c->pts_near, c->near, c->xn.d(), qn, true));
  TRY(build_points(c, c->circle, c->arc_c, c->pts_far_c, c->far_c, c->xf.d(), qf, false));
  TRY(build_points(c, c->circle, c->arc_c, c->pts_near_c, c->near_c, c->xn.d(), qn, true));
  TRY(fft_plan_create(c->fft, N, c->s));
  c->fft_ready = true;
  TRY(sync(c));
  c->stage = ST_MESH;
  return WCS_OK;
}

int wcs_query(const wcs_ctx* c, wcs_info* info) {
  if (!c || !info) { set_error("null argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("no mesh yet"); return WCS_ERR_STATE; }
  info->N = c->N; info->L = c->L; info->h = c->h; info->a = c->a; info->k = c->k;
  info->kt_re = c->kt.x; info->kt_im = c->kt.y;
  info->rank = c->stage >= ST_SKELETON ? c->rank : -1;
  info->norm_cc = c->stage >= ST_ASSEMBLED ? c->norm_cc : 0.0;
  info->min_curvature = c->kmin;
  info->zfast = c->mixed ? c->opt.zfast : 0.0;
  info->capacitance_residual = c->kinv_res;
  return WCS_OK;
}

static AsmArgs asm_args(wcs_ctx* c, bool circle) {
  AsmArgs A{};
  A.N = c->N; A.h = c->h; A.k = c->k; A.kt = c->kt;
  A.q_far = c->opt.q_far; A.q_near = c->opt.q_near; A.near_band = c->opt.near_band;
  A.far = circle ? c->far_c : c->far;
  A.near = circle ? c->near_c : c->near;
  A.wlog = c->wlog.d();
  A.ld = c->ld;
  // k~ = k (1 + i t): both Hankel evaluations of a point pair from one real one
  const double t = c->kt.y / c->k;
  if (c->kt.x == c->k && t >= 0.0 && t <= 0.1) {
    const std::complex<double> z(1.0, t);
    const std::complex<double> c1 = 1.0 / z, c2 = 1.0 / std::sqrt(z);
    A.kt_pair = 1;
    A.ktp.t = t;
    A.ktp.c1 = mkz(c1.real(), c1.imag());
    A.ktp.c2 = mkz(c2.real(), c2.imag());
    // the mixed form stores entries to 24 bits: its expansion stops at 1e-13;
    // the FP64 form and the circle rows (the eigenvalues) keep 1e-16
    fill_asymptotic(A.ktp, (c->mixed && !circle) ? 1e-13 : 1e-16);
    // the reference-phase route of the far pairs needs |k R - x0| <= 1.05
    // (points within 0.45 h of their element's reference point) and
    // |(k R - x0) t| <= 0.02 (see hankel01_asymptotic_rot)
    A.rot_ok = (c->k * c->h <= 1.2 && t <= 0.019) ? 1 : 0;
  }
  return A;
}

// FP32 constants of the mixed form's far-pair path (after A.zfast is set)
static void set_fast_consts(AsmArgs& A) {
  const std::complex<double> kt(A.kt.x, A.kt.y);
  const std::complex<double> ck = std::sqrt((2.0 / WCS_PI) / kt), ik = std::complex<double>(0.0, 1.0) / kt;
  const std::complex<double> kt4 = std::complex<double>(0.0, 0.25) * kt;
  FastConsts& F = A.fk;
  F.kf = (float)A.k;
  F.beta = (float)A.kt.y;
  F.beta_lo = (float)(A.kt.y - (double)F.beta);
  F.ck[0] = (float)ck.real(); F.ck[1] = (float)ck.imag();
  F.ik[0] = (float)ik.real(); F.ik[1] = (float)ik.imag();
  F.kt4[0] = (float)kt4.real(); F.kt4[1] = (float)kt4.imag();
  F.ampk = (float)std::sqrt(2.0 / (WCS_PI * A.k));
  F.kk2h2 = (float)(A.k * A.k * A.h * A.h);
  F.h2 = (float)(A.h * A.h);
  F.zfast2 = (A.zfast < 1e18) ? (float)(A.zfast * A.zfast) : INFINITY;
  F.k_hi = (float)A.k;
  F.k_lo = (float)(A.k - (double)F.k_hi);
  // FP64 factors of the reduced FP32 sums (see pair_fast_f)
  const std::complex<double> I4(0.0, 0.25);
  const double ampk = std::sqrt(2.0 / (WCS_PI * A.k)), h2 = A.h * A.h;
  const std::complex<double> fS = I4 * ck * h2, fD = I4 * ampk * A.k * h2, fDt = I4 * kt * ck * h2, fN = I4 * ampk;
  A.fS = mkz(fS.real(), fS.imag());
  A.fD = mkz(fD.real(), fD.imag());
  A.fDt = mkz(fDt.real(), fDt.imag());
  A.fN = mkz(fN.real(), fN.imag());
  A.kk2h2 = A.k * A.k * h2;
  const double tp = 2.0 * WCS_PI;   // 2 pi to ~72 bits: double plus its float-float residual
  const double tp_lo = 2.4492935982947064e-16;
  F.twopi[0] = (float)tp;
  F.twopi[1] = (float)(tp - (double)F.twopi[0]);
  F.twopi[2] = (float)((tp - (double)F.twopi[0] - (double)F.twopi[1]) + tp_lo);
}

__global__ void k_geom_sample_dummy() {}

int wcs_geometry_sample(wcs_ctx* c, int64_t count, const double* s_host, double* out_host) {
  if (!c || !s_host || !out_host || count < 0) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("no mesh yet"); return WCS_ERR_STATE; }
  if (count == 0) return WCS_OK;
  // treat each sample as element e = 0 with xi = s / h (points_build evaluates (e + xi) h)
  DevBuf sb, pb;
  TRY(sb.ensure(sizeof(double) * count));
  TRY(pb.ensure(sizeof(double) * count * 5));
  std::vector<double> xi(count);
  for (int64_t i = 0; i < count; ++i) xi[i] = s_host[i] / c->h;
  cudaMemcpyAsync(sb.p, xi.data(), sizeof(double) * count, cudaMemcpyHostToDevice, c->s);
  Points P;
  double* b = pb.d();
  P.x = b; P.y = b + count; P.nx = b + 2 * count; P.ny = b + 3 * count; P.kappa = b + 4 * count;
  P.n = count;
  // one "element" with count local nodes
  const int64_t savedN = c->N;
  int r = points_build(c->contour, c->arc, 1, c->h, sb.d(), (int)count, P, c->s);
  (void)savedN;
  if (r) { sb.release(); pb.release(); return r; }
  cudaMemcpyAsync(out_host, pb.p, sizeof(double) * count * 5, cudaMemcpyDeviceToHost, c->s);
  r = sync(c);
  sb.release();
  pb.release();
  return r;
}

int wcs_assemble(wcs_ctx* c) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("mesh first"); return WCS_ERR_STATE; }
  const int64_t N = c->N, ld = c->ld;
  if (!c->mixed) {
    TRY(c->ops.ensure(sizeof(zd) * 4 * N * ld));
    c->S = c->ops.z(); c->D = c->S + N * ld; c->Dt = c->D + N * ld; c->Nk = c->Dt + N * ld;
    AsmArgs A = asm_args(c, false);
    A.S = c->S; A.D = c->D; A.Dt = c->Dt; A.Nk = c->Nk;
    ProfScope ps(c, CAT_ASSEMBLY, (double)N * N * c->opt.q_far * c->opt.q_far, 0.0);
    TRY(assemble_dense(A, c->s));
  } else {
    c->ldp = ((2 * N + 63) / 64) * 64;
    TRY(c->opplanes.ensure(sizeof(uint16_t) * (size_t)8 * c->planes * N * c->ldp));
    if (c->ldp != 2 * N) cudaMemsetAsync(c->opplanes.p, 0, c->opplanes.bytes, c->s);   // zero the padding columns
    // element centres (xi = 1/2) and FP32 offsets of the far points
    const int qf = c->opt.q_far;
    TRY(c->centres.ensure(sizeof(double) * 6 * N));
    double* half = c->centres.d() + 5 * N;
    const double hv = 0.5;
    cudaMemcpyAsync(half, &hv, sizeof(double), cudaMemcpyHostToDevice, c->s);
    Points cp;
    cp.x = c->centres.d(); cp.y = cp.x + N; cp.nx = cp.y + N; cp.ny = cp.nx + N; cp.kappa = nullptr; cp.n = N;
    TRY(points_build(c->contour, c->arc, N, c->h, half, 1, cp, c->s));
    const int64_t cff_off = ((8 * N * qf + 3) / 4) * 4;   // floats; float4 table 16-byte aligned
    TRY(c->offs.ensure(sizeof(float) * cff_off + sizeof(float4) * N));
    float* of = (float*)c->offs.p;
    float4* cff = (float4*)(of + cff_off);
    TRY(far_offsets(c->far, cp.x, cp.y, N, qf, of, of + N * qf, of + 2 * N * qf, of + 3 * N * qf, of + 4 * N * qf,
                    of + 5 * N * qf, of + 6 * N * qf, of + 7 * N * qf, cff, c->s));
    AsmArgs A = asm_args(c, false);
    A.mixed = 1;
    A.planes = c->planes;
    A.ldp = c->ldp;
    for (int op = 0; op < 4; ++op)
      for (int l = 0; l < 2; ++l)
        for (int p = 0; p < 3; ++p) A.P[op][l][p] = (p < c->planes) ? plane_ptr(c, op, l, p) : nullptr;
    A.cx = cp.x; A.cy = cp.y;
    A.ox = of; A.oy = of + N * qf; A.nxf = of + 2 * N * qf; A.nyf = of + 3 * N * qf;
    A.nxl = of + 4 * N * qf; A.nyl = of + 5 * N * qf;
    A.oxl = of + 6 * N * qf; A.oyl = of + 7 * N * qf;
    A.cff = cff;
    // zfast <= 0: every pair in FP64 (the FP32 path is off)
    A.zfast = (c->opt.zfast > 0.0) ? c->opt.zfast + 2.0 * c->k * c->h : 1e300;
    set_fast_consts(A);
    if (!c->profile) {
      TRY(assemble_planes(A, c->s));
    } else {
      // two records: the FP32 far-pair kernel, then the FP64 kernel over the
      // remaining tiles; units: element pairs of each kernel's tiles x q_far^2
      cudaEvent_t a0, mid[2], b0;
      cudaEventCreate(&a0);
      cudaEventCreate(&mid[0]);
      cudaEventCreate(&mid[1]);
      cudaEventCreate(&b0);
      cudaEventRecord(a0, c->s);
      int64_t nf64 = 0, nt = 0;
      TRY(assemble_planes(A, c->s, mid, &nf64, &nt));
      cudaEventRecord(b0, c->s);
      const double per_tile = 33.0 * 33.0 * qf * qf;
      c->recs.push_back({CAT_ASSEMBLY_FAST, a0, mid[0], per_tile * (double)(nt - nf64), 0.0});
      c->recs.push_back({CAT_ASSEMBLY, mid[1], b0, per_tile * (double)nf64, 0.0});
    }
  }
  // circle: first rows -> eigenvalues
  TRY(c->mu.ensure(sizeof(zd) * 6 * N));
  AsmArgs B = asm_args(c, true);
  B.S = mu_ptr(c, MU_S); B.D = mu_ptr(c, MU_D); B.Dt = mu_ptr(c, MU_DT); B.Nk = mu_ptr(c, MU_N);
  TRY(assemble_circle_row(B, c->s));
  // mu_X(m) = sum_j X_0j e^{+2 pi i m j / N}
  TRY(fft_columns(c->fft, mu_ptr(c, MU_S), N, 4, +1, c->s));
  k_mu_finish<<<(unsigned)((N + 255) / 256), 256, 0, c->s>>>(c->mu.z(), N, c->h);
  note_launch();
  c->circ.ready = false;   // the FP32 circulant tables follow mu_C
  TRY(c->small.ensure(sizeof(double) * 8));
  k_absmax<<<1, 256, 0, c->s>>>(mu_ptr(c, MU_C), N, c->small.d());
  note_launch();
  cudaMemcpyAsync(&c->norm_cc, c->small.p, sizeof(double), cudaMemcpyDeviceToHost, c->s);
  TRY(sync(c));
  c->U.release(); c->Vw.release(); c->Wt.release(); c->Kinv.release(); c->Wa.release();
  c->rank = -1;
  c->stage = ST_ASSEMBLED;
  return WCS_OK;
}

int wcs_operator_entries(wcs_ctx* c, int64_t count, const int64_t* rows, const int64_t* cols,
                         double* out) {
  if (!c || count < 0 || (count > 0 && (!rows || !cols || !out))) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("mesh first"); return WCS_ERR_STATE; }
  if (count == 0) return WCS_OK;
  for (int64_t t = 0; t < count; ++t)
    if (rows[t] < 0 || rows[t] >= c->N || cols[t] < 0 || cols[t] >= c->N) { set_error("index out of range"); return WCS_ERR_ARG; }
  DevBuf idx, res;
  TRY(idx.ensure(sizeof(int64_t) * 2 * count));
  TRY(res.ensure(sizeof(zd) * 4 * count));
  cudaMemcpyAsync(idx.p, rows, sizeof(int64_t) * count, cudaMemcpyHostToDevice, c->s);
  cudaMemcpyAsync((int64_t*)idx.p + count, cols, sizeof(int64_t) * count, cudaMemcpyHostToDevice, c->s);
  AsmArgs A = asm_args(c, false);
  int r = assemble_entries(A, count, (int64_t*)idx.p, (int64_t*)idx.p + count, res.z(), c->s);
  if (!r) {
    cudaMemcpyAsync(out, res.p, sizeof(zd) * 4 * count, cudaMemcpyDeviceToHost, c->s);
    r = sync(c);
  }
  idx.release();
  res.release();
  return r;
}

int wcs_circulant_eigs(wcs_ctx* c, int op, double* out) {
  if (!c || !out) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_ASSEMBLED) { set_error("assemble first"); return WCS_ERR_STATE; }
  int w;
  switch (op) {
    case WCS_OP_G: w = MU_G; break;
    case WCS_OP_S: w = MU_S; break;
    case WCS_OP_D: w = MU_D; break;
    case WCS_OP_DT: w = MU_DT; break;
    case WCS_OP_N: w = MU_N; break;
    case WCS_OP_CC: w = MU_C; break;
    default: set_error("operator has no circulant eigenvalues"); return WCS_ERR_ARG;
  }
  cudaError_t e = cudaMemcpyAsync(out, mu_ptr(c, w), sizeof(zd) * c->N, cudaMemcpyDeviceToDevice, c->s);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  return WCS_OK;
}

// Plane-wave angles are host arrays: reject non-finite ones before any work.
static int check_angles(int64_t B, const double* a, const char* what) {
  for (int64_t i = 0; i < B; ++i)
    if (!std::isfinite(a[i])) {
      set_error(std::string(what) + ": angle " + std::to_string(i) + " is not finite");
      return WCS_ERR_ARG;
    }
  return 0;
}

static int check_block(wcs_ctx* c, int64_t B, const void* p, int64_t ld) {
  if (B < 0 || (B > 0 && (!p || ld < c->N))) { set_error("bad block argument (pointer or ld < N)"); return WCS_ERR_ARG; }
  return 0;
}

int wcs_apply(wcs_ctx* c, int op, int64_t B, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_ASSEMBLED) { set_error("assemble first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, X, ldx));
  TRY(check_block(c, B, Y, ldy));
  if (B == 0) return WCS_OK;
  const int64_t N = c->N;
  const zd* x = (const zd*)X;
  zd* y = (zd*)Y;
  const int64_t chunk = c->opt.rhs_chunk;
  TRY(ensure_work(c, std::min(B, chunk)));
  for (int64_t c0 = 0; c0 < B; c0 += chunk) {
    const int64_t cc = std::min(chunk, B - c0);
    const zd* xc = x + c0 * ldx;
    zd* yc = y + c0 * ldy;
    switch (op) {
      case WCS_OP_C: TRY(apply_C(c, xc, ldx, yc, ldy, cc, false, PREC_ACCURATE)); break;
      case WCS_OP_CH: TRY(apply_C(c, xc, ldx, yc, ldy, cc, true, PREC_ACCURATE)); break;
      case WCS_OP_CC: TRY(apply_Cc(c, xc, ldx, yc, ldy, cc, 0)); break;
      case WCS_OP_CCH: TRY(apply_Cc(c, xc, ldx, yc, ldy, cc, 1)); break;
      case WCS_OP_CC_INV: TRY(apply_Cc(c, xc, ldx, yc, ldy, cc, 2)); break;
      case WCS_OP_CCH_INV: TRY(apply_Cc(c, xc, ldx, yc, ldy, cc, 3)); break;
      case WCS_OP_S:
      case WCS_OP_D:
      case WCS_OP_DT:
      case WCS_OP_N:
        if (c->mixed) {
          const int which = op - WCS_OP_S;
          TRY(ensure_stage(c, cc));
          TRY(stage(c, c->stage0, xc, ldx, cc, 0));
          TRY(tc_apply(c, which, false, c->stage0, cc, mkz(1.0), mkz(0.0), yc, ldy, PREC_ACCURATE));
          break;
        }
        if (op != WCS_OP_S) goto fp64_ops;
        TRY(zgemm(N, cc, N, mkz(1.0), op_view(c->S, c->ld, false), blk(xc, ldx), mkz(0.0), yc, ldy, c->s)); break;
      fp64_ops:
        if (op == WCS_OP_D) { TRY(zgemm(N, cc, N, mkz(1.0), op_view(c->D, c->ld, false), blk(xc, ldx), mkz(0.0), yc, ldy, c->s)); break; }
        if (op == WCS_OP_DT) { TRY(zgemm(N, cc, N, mkz(1.0), op_view(c->Dt, c->ld, false), blk(xc, ldx), mkz(0.0), yc, ldy, c->s)); break; }
        TRY(zgemm(N, cc, N, mkz(1.0), op_view(c->Nk, c->ld, false), blk(xc, ldx), mkz(0.0), yc, ldy, c->s));
        break;
      case WCS_OP_G: TRY(gram_apply(xc, ldx, yc, ldy, N, cc, c->h, 1.0, 0.0, c->s)); break;
      case WCS_OP_GINV: TRY(ginv(c, xc, ldx, yc, ldy, cc)); break;
      case WCS_OP_SKEL: {
        if (c->stage < ST_SKELETON) { set_error("skeleton first"); return WCS_ERR_STATE; }
        const int64_t r = std::max(c->rank, 0);
        if (r == 0) { TRY(axpby(N, cc, mkz(0.0), xc, ldx, mkz(0.0), yc, ldy, c->s)); break; }
        TRY(c->small.ensure(sizeof(zd) * r * cc));
        // U V^T x = Q (Vw^H x)
        TRY(cgemm(c, r, cc, N, mkz(1.0), blkH(c->Vw.z(), N), xc, ldx, mkz(0.0), c->small.z(), r));
        TRY(cgemm(c, N, cc, r, mkz(1.0), blk(c->U.z(), N), c->small.z(), r, mkz(0.0), yc, ldy));
        break;
      }
      default: set_error("unknown operator"); return WCS_ERR_ARG;
    }
  }
  if (c->mixed) TRY(check_tc(c));
  return WCS_OK;
}

int wcs_skeleton(wcs_ctx* c, double tol, int max_rank, uint64_t seed, int* rank_out) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_ASSEMBLED) { set_error("assemble first"); return WCS_ERR_STATE; }
  if (!(tol >= 0)) { set_error("tolerance must be >= 0"); return WCS_ERR_ARG; }
  const int64_t N = c->N;
  const int64_t cap = (max_rank <= 0 || max_rank > N) ? N : max_rank;
  const int b = c->opt.block;
  ProfScope whole(c, CAT_SKELETON, 0.0, 0.0);
  // samples are drawn SB = 8b columns per pass over the operators (wide
  // products fill the GPU in whole waves) and orthonormalised b columns at a
  // time; Y is linear in Omega and Omega's columns come from one counter
  // stream, so the basis is the one of the b-column loop
  const int64_t SB = std::min<int64_t>(8 * (int64_t)b, ((cap + b - 1) / b) * b);
  TRY(ensure_work(c, SB));
  TRY(c->U.ensure(sizeof(zd) * N * (cap + b)));
  zd* Q = c->U.z();
  const double thr = tol * c->norm_cc / (10.0 * std::sqrt(2.0 / WCS_PI));
  // small scratch: Z (cap x b), Gram (b x b), perm, rank, norms
  DevBuf Zb, Gb, Ib, Nb, GW;
  TRY(GW.ensure(sizeof(zd) * ((N + 255) / 256) * b * b));
  TRY(Zb.ensure(sizeof(zd) * (cap + b) * b));
  TRY(Gb.ensure(sizeof(zd) * 2 * b * b));   // Gram / Cholesky factor, then R^{-1}
  TRY(Ib.ensure(sizeof(int) * (b + 1)));
  TRY(Nb.ensure(sizeof(double) * b));
  int64_t ell = 0;
  uint64_t offset = 0;
  int status = WCS_OK;
  std::vector<double> norms(b);
  zd* Om = c->w4.z();
  zd* Ys = c->w5.z();
  int64_t batch_cols = 0, batch_used = 0;
  const zd one = mkz(1.0), mone = mkz(-1.0), zero = mkz(0.0);
  // mixed form: the accepted basis also lives as resident split-bf16 planes,
  // rows conj(q_i) (for Q^H X) and rows of Q (for Q Z), staged once per block
  const int64_t ldqh = ((2 * N + 63) / 64) * 64, ldqt = ((2 * (cap + b) + 63) / 64) * 64;
  uint16_t *QH[2] = {nullptr, nullptr}, *QT[2] = {nullptr, nullptr};
  if (c->mixed) {
    TRY(c->qh.ensure(sizeof(uint16_t) * 2 * (size_t)(cap + b) * ldqh));
    TRY(c->qt.ensure(sizeof(uint16_t) * 2 * (size_t)N * ldqt));
    for (int p = 0; p < 2; ++p) {
      QH[p] = (uint16_t*)c->qh.p + (int64_t)p * (cap + b) * ldqh;
      QT[p] = (uint16_t*)c->qt.p + (int64_t)p * N * ldqt;
    }
  }
  while (true) {
    if (ell >= cap) { status = (ell < N) ? WCS_ERR_RANK_CAP : WCS_OK; break; }
    if (batch_used == batch_cols) {
      ProfScope ps(c, CAT_SAMPLE, 0.0, 0.0);
      batch_cols = std::min<int64_t>(SB, ((cap - ell + b - 1) / b) * b);
      batch_used = 0;
      TRY(gaussian_fill(Om, N, N, batch_cols, seed, offset, c->s));
      TRY(dbg_check(c, Om, N, batch_cols, N, "gaussian"));
      offset += (uint64_t)N * batch_cols;
      TRY(apply_remainder(c, Om, N, Ys, N, batch_cols, false,
                          (c->mixed && c->opt.sample_planes == 1) ? PREC_FAST1 : PREC_PERIODIC));
      TRY(dbg_check(c, Ys, N, batch_cols, N, "sample"));
    }
    zd* Y = Ys + batch_used * N;
    batch_used += b;
    {
      ProfScope ps_proj(c, CAT_PROJECT, 0.0, 0.0);
      for (int pass = 0; pass < 2 && ell > 0; ++pass) {
        TRY(cgemm_planes(c, ell, b, N, one, QH[0], QH[1], ldqh, blkH(Q, N), Y, N, zero, Zb.z(), ell));
        TRY(dbg_check(c, Zb.z(), ell, b, ell, "projection coefficients"));
        TRY(cgemm_planes(c, N, b, ell, mone, QT[0], QT[1], ldqt, blk(Q, N), Zb.z(), ell, one, Y, N));
        TRY(dbg_check(c, Y, N, b, N, "projection"));
      }
    }
    TRY(column_norms(Y, N, N, b, Nb.d(), c->s));
    cudaMemcpyAsync(norms.data(), Nb.p, sizeof(double) * b, cudaMemcpyDeviceToHost, c->s);
    TRY(sync(c));
    double mx = 0;
    for (int j = 0; j < b; ++j) {
      if (!std::isfinite(norms[j])) { set_error("skeleton: non-finite sample (block at rank " + std::to_string(ell) + ")"); return WCS_ERR_CUDA; }
      mx = std::max(mx, norms[j]);
    }
    if (c->mixed) TRY(check_tc(c));
    if (mx <= thr) break;
    // orthonormalise the block twice (pivoted CholeskyQR)
    ProfScope ps_orth(c, CAT_ORTH, 0.0, 0.0);
    int rk = b;
    const zd* src = Y;
    for (int pass = 0; pass < 2; ++pass) {
      const int cols = (pass == 0) ? b : rk;
      TRY(gram_matrix(src, N, N, cols, Gb.z(), GW.z(), c->s));
      TRY(dbg_check(c, Gb.z(), cols, cols, cols, "gram"));
      TRY(pivoted_cholesky(Gb.z(), cols, 1e-7, (int*)Ib.p, (int*)Ib.p + b, c->s));
      int rk_new = 0;
      cudaMemcpyAsync(&rk_new, (int*)Ib.p + b, sizeof(int), cudaMemcpyDeviceToHost, c->s);
      TRY(sync(c));
      if (rk_new == 0) { rk = 0; break; }
      zd* dst = (pass == 0) ? c->w3.z() : Q + ell * N;
      TRY(dbg_check(c, Gb.z(), cols, cols, cols, "cholesky"));
      TRY(trsm_right_upper(src, N, N, Gb.z(), cols, (int*)Ib.p, (int*)Ib.p + b, rk_new, dst, N, Gb.z() + b * b,
                           c->s));
      TRY(dbg_check(c, dst, N, rk_new, N, "trsm"));
      rk = rk_new;
      if (pass == 0) {
        // re-orthogonalise against the accepted basis before the second pass
        if (ell > 0) {
          TRY(cgemm_planes(c, ell, rk, N, one, QH[0], QH[1], ldqh, blkH(Q, N), c->w3.z(), N, zero, Zb.z(), ell));
          TRY(cgemm_planes(c, N, rk, ell, mone, QT[0], QT[1], ldqt, blk(Q, N), Zb.z(), ell, one, c->w3.z(), N));
          TRY(dbg_check(c, c->w3.z(), N, rk, N, "re-orthogonalisation"));
        }
        src = c->w3.z();
      }
    }
    if (rk == 0) break;
    if (c->mixed) {
      uint16_t* ph[3] = {QH[0] + ell * ldqh, QH[1] + ell * ldqh, nullptr};
      TRY(stage_view(Q + ell * N, rk, N, N, 1, 1, 2, ph, ldqh, c->s));   // rows conj(q_i)
      uint16_t* pt[3] = {QT[0] + 2 * ell, QT[1] + 2 * ell, nullptr};
      TRY(stage_view(Q + ell * N, N, rk, 1, N, 0, 2, pt, ldqt, c->s));   // row p: Q[p, ell + j]
    }
    ell += rk;
    if (ell > cap) ell = cap;
  }
  c->qh.release();
  c->qt.release();
  c->rank = (int)ell;
  // V^T = Q^H (C - C_c)  <=>  Vw = (C - C_c)^H Q  (V = conj(Vw))
  TRY(c->Vw.ensure(sizeof(zd) * N * std::max<int64_t>(ell, 1)));
  ProfScope ps_vw(c, CAT_VW, 0.0, 0.0);
  const int64_t wide = std::max<int64_t>(b, std::min<int64_t>(c->opt.rhs_chunk, 1024));
  TRY(ensure_work(c, wide));
  for (int64_t c0 = 0; c0 < ell; c0 += wide) {
    const int64_t cc = std::min<int64_t>(wide, ell - c0);
    TRY(apply_remainder(c, Q + c0 * N, N, c->Vw.z() + c0 * N, N, cc, true, PREC_PERIODIC));
  }
  TRY(sync(c));
  if (rank_out) *rank_out = (int)ell;
  c->Wt.release(); c->Kinv.release(); c->Wa.release();
  c->stage = ST_SKELETON;
  return status;
}

// Y = A X for r x r complex A and r x cols complex X (column-major, ld r),
// exact up to the FP64 sums of the scaled integer partials (exact.cu): the
// rows of A as fixed-point slices, X as slices of a right-hand block.
static int exact_square(wcs_ctx* c, const zd* A, int64_t r, const zd* X, int64_t cols, zd* Y) {
  TRY(ensure_tcerr(c));
  DevBuf At, pa, pb, ws;
  TRY(At.ensure(sizeof(zd) * r * r));
  k_transpose_z<<<(unsigned)((r * r + 255) / 256), 256, 0, c->s>>>(A, r, At.z());
  note_launch();
  int64_t lda = 0, ncha = 0, ldb = 0, nchb = 0;
  size_t sa = 0, ea = 0, sb = 0, eb = 0;
  // columns per pass: wide passes keep the 21 slice-pair launches large
  // (the FP32 partials take nchunks x 2G x r floats, 268 MB at r = 4096)
  const int64_t G = std::min<int64_t>(1024, std::max<int64_t>(cols, 1));
  exact_operand_alloc_bytes(r, 2 * r, &lda, &ncha, &sa, &ea);
  exact_operand_alloc_bytes(2 * G, 2 * r, &ldb, &nchb, &sb, &eb);
  const size_t sa2 = ((sa + 255) / 256) * 256, sb2 = ((sb + 255) / 256) * 256;
  TRY(pa.ensure(EX_SLICES * sa2 + ea + 256));
  TRY(pb.ensure(EX_SLICES * sb2 + eb + 256));
  const int64_t ws_elems = nchb * 2 * G * r;
  TRY(ws.ensure(sizeof(float) * (size_t)ws_elems));
  ExactOperand oa, ob;
  oa.ld = lda;
  oa.nchunks = ncha;
  ob.ld = ldb;
  ob.nchunks = nchb;
  for (int q = 0; q < EX_SLICES; ++q) {
    oa.slice[q] = (uint16_t*)((char*)pa.p + q * sa2);
    ob.slice[q] = (uint16_t*)((char*)pb.p + q * sb2);
  }
  oa.expo = (int16_t*)((char*)pa.p + EX_SLICES * sa2);
  ob.expo = (int16_t*)((char*)pb.p + EX_SLICES * sb2);
  TRY(exact_slice_real((const double*)At.p, r, 2 * r, 2 * r, oa, c->s));
  ProfScope ps(c, CAT_GEMM_EXACT, 2.0 * r * (2.0 * cols) * (2.0 * r), 0.0);
  for (int64_t c0 = 0; c0 < cols; c0 += G) {
    const int64_t cc = std::min(G, cols - c0);
    TRY(exact_slice_rhs(X + c0 * r, r, cc, r, 0, ob, c->s));
    TRY(exact_product(oa, (int)r, ob, (int)cc, (int)(2 * r), mkz(1.0), mkz(0.0), 0, Y + c0 * r, r,
                      (float*)ws.p, ws_elems, (int*)c->tcerr.p, c->s));
  }
  return check_tc(c);
}

int wcs_factor(wcs_ctx* c) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_SKELETON) { set_error("skeleton first"); return WCS_ERR_STATE; }
  const int64_t N = c->N, r = c->rank;
  c->kinv_res = -1.0;
  ProfScope whole(c, CAT_FACTOR, 8.0 / 3.0 * r * (double)r * r, 0.0);
  if (r > 0) {
    TRY(c->Wt.ensure(sizeof(zd) * N * r));
    // W = C_c^{-1} U  (held in Wt until the inverse is applied)
    DevBuf Wb, Kb, info;
    DevBuf& Kinv = c->Kinv;   // kept for adjoint solves
    c->Wa.release();
    TRY(Wb.ensure(sizeof(zd) * N * r));
    TRY(apply_Cc(c, c->U.z(), N, Wb.z(), N, r, 2));
    // K = I + V^T W = I + Vw^H W
    TRY(Kb.ensure(sizeof(zd) * r * r));
    TRY(Kinv.ensure(sizeof(zd) * r * r));
    TRY(cgemm(c, r, r, N, mkz(1.0), blkH(c->Vw.z(), N), Wb.z(), N, mkz(0.0), Kb.z(), r));
    k_add_identity<<<(unsigned)((r + 255) / 256), 256, 0, c->s>>>(Kb.z(), r);
    note_launch();
    TRY(info.ensure(sizeof(int) + sizeof(double) * 2));
    int* infod = (int*)info.p;
    double* minpiv = (double*)((char*)info.p + 8);
    if (!c->mixed || r < 256) {
      ProfScope ps(c, CAT_INVERSE, 8.0 * r * (double)r * r, 0.0);
      TRY(lu_inverse(Kb.z(), r, Kinv.z(), nullptr, infod, minpiv, c->s));
      int infoh = 0;
      double mp = 0;
      cudaMemcpyAsync(&infoh, infod, sizeof(int), cudaMemcpyDeviceToHost, c->s);
      cudaMemcpyAsync(&mp, minpiv, sizeof(double), cudaMemcpyDeviceToHost, c->s);
      TRY(sync(c));
      if (infoh != 0 || !(mp > 1e-14)) {
        set_error("capacitance matrix is singular (rank " + std::to_string(r) + ", smallest pivot " +
                  std::to_string(mp) + ", first zero pivot at step " + std::to_string(infoh) + ")");
        return WCS_ERR_SINGULAR;
      }
    } else {
      // Newton-Schulz: X <- X (2I - K X) from X0 = K^H / (||K||_1 ||K||_inf),
      // which converges for any nonsingular K; products on the tensor cores
      ProfScope ps(c, CAT_INVERSE, 16.0 * r * (double)r * r, 0.0);
      DevBuf T, sums;
      TRY(T.ensure(sizeof(zd) * r * r));
      TRY(sums.ensure(sizeof(double) * (3 * r + 2 + EYE_BLOCKS)));
      double* cs = sums.d();
      k_col_abs_sums<<<(unsigned)r, 256, 0, c->s>>>(Kb.z(), r, cs);
      note_launch();
      k_row_abs_sums<<<(unsigned)((r + 127) / 128), 128, 0, c->s>>>(Kb.z(), r, cs + r);
      note_launch();
      k_scaled_adjoint<<<1024, 256, 0, c->s>>>(Kb.z(), r, cs, cs + r, Kinv.z());
      note_launch();
      DevBuf X2;
      TRY(X2.ensure(sizeof(zd) * r * r));
      zd* X = Kinv.z();
      zd* Xn = X2.z();
      double res = 1e300, prev = 1e300;
      const double target = 1e-4 * std::sqrt((double)r);   // ||I - K X||_F, i.e. ~1e-4 per direction
      for (int it = 0; it < 120; ++it) {
        // T = K X
        TRY(cgemm(c, r, r, r, mkz(1.0), blk(Kb.z(), r), X, r, mkz(0.0), T.z(), r));
        if ((it & 3) == 3) {
          k_eye_partial<<<EYE_BLOCKS, 256, 0, c->s>>>(T.z(), r, cs + 3 * r);
          note_launch();
          k_eye_finish<<<1, 256, 0, c->s>>>(cs + 3 * r, EYE_BLOCKS, cs + 2 * r);
          note_launch();
          cudaMemcpyAsync(&res, cs + 2 * r, sizeof(double), cudaMemcpyDeviceToHost, c->s);
          TRY(sync(c));
          if (!(res == res)) { set_error("capacitance iteration diverged"); return WCS_ERR_SINGULAR; }
          // converged, or stalled at the contraction's rounding level
          if (res < target || (res < 0.1 * std::sqrt((double)r) && res > 0.8 * prev)) break;
          prev = res;
        }
        // X <- X (2I - T)
        k_two_minus<<<(unsigned)((r * r + 255) / 256), 256, 0, c->s>>>(T.z(), r);
        note_launch();
        TRY(cgemm(c, r, r, r, mkz(1.0), blk(X, r), T.z(), r, mkz(0.0), Xn, r));
        std::swap(X, Xn);
      }
      if (!(res < 0.1 * std::sqrt((double)r))) { set_error("capacitance iteration did not converge"); return WCS_ERR_SINGULAR; }
      // The two-plane iteration stalls near 1e-4 per direction.  One step with
      // the drained three-plane product (~1e-7) and then exact steps (each
      // squares the residual; the exact products carry 42 bits below each
      // chunk's scale, ~1e-11 per direction) close it: an exact product
      // measures ||I - K X||_F after every exact step, and a step is added
      // while that is above 1e-10 per direction (at most three).
      auto eye_residual = [&](double& out) -> int {
        k_eye_partial<<<EYE_BLOCKS, 256, 0, c->s>>>(T.z(), r, cs + 3 * r);
        note_launch();
        k_eye_finish<<<1, 256, 0, c->s>>>(cs + 3 * r, EYE_BLOCKS, cs + 2 * r);
        note_launch();
        cudaMemcpyAsync(&out, cs + 2 * r, sizeof(double), cudaMemcpyDeviceToHost, c->s);
        return sync(c);
      };
      {
        TRY(cgemm(c, r, r, r, mkz(1.0), blk(Kb.z(), r), X, r, mkz(0.0), T.z(), r, true));   // T = K X
        k_two_minus<<<(unsigned)((r * r + 255) / 256), 256, 0, c->s>>>(T.z(), r);
        note_launch();
        TRY(cgemm(c, r, r, r, mkz(1.0), blk(X, r), T.z(), r, mkz(0.0), Xn, r, true));    // X <- X (2I - K X)
        std::swap(X, Xn);
        TRY(exact_square(c, Kb.z(), r, X, r, T.z()));
        for (int it = 0; it < 3; ++it) {
          k_two_minus<<<(unsigned)((r * r + 255) / 256), 256, 0, c->s>>>(T.z(), r);
          note_launch();
          TRY(exact_square(c, X, r, T.z(), r, Xn));             // X <- X (2I - K X)
          std::swap(X, Xn);
          TRY(exact_square(c, Kb.z(), r, X, r, T.z()));          // T = K X
          TRY(eye_residual(res));
          c->kinv_res = res / std::sqrt((double)r);
          if (!(c->kinv_res >= 1e-10)) break;
        }
        if (!(c->kinv_res < 1e-6)) { set_error("capacitance iteration did not reach FP64 accuracy"); return WCS_ERR_SINGULAR; }
      }
      if (X != Kinv.z())
        cudaMemcpyAsync(Kinv.p, X, sizeof(zd) * r * r, cudaMemcpyDeviceToDevice, c->s);
    }
    // Wt = W K^{-1}
    TRY(cgemm(c, N, r, r, mkz(1.0), blk(Wb.z(), N), Kinv.z(), r, mkz(0.0), c->Wt.z(), N));
    TRY(sync(c));
  }
  c->stage = ST_FACTORED;
  return WCS_OK;
}

// ---------------------------------------------------------------- checkpoint
// Binary file (little-endian, as both supported hosts are):
//   CkptHeader                magic, version, rank, N, k, options, contour
//   CkptExt (version >= 3)    flags: bit 0 = the capacitance inverse follows
//   U, V_w, W~                N x rank complex FP64 each, column by column
//   K^-1 (version 2; version 3 with flag bit 0)   rank x rank complex FP64
//   trailer (version >= 3)    tag "WCSFNV64" and a 64-bit FNV-1a checksum of
//                             every byte before the trailer
// The operators are not stored: loading re-runs the mesh and the assembly,
// which are deterministic, and which the refinement needs anyway.  Version 3
// files are checked (size and checksum) before any device work.
struct CkptHeader {
  char magic[8];
  int32_t version;
  int32_t rank;
  int64_t N;
  double k;
  wcs_options opt;
  Contour contour;
};
struct CkptExt {
  uint32_t flags;
  uint32_t reserved;
};
static const char kCkptMagic[8] = {'W', 'C', 'S', 'C', 'K', 'P', 'T', '1'};
static const char kCkptTag[8] = {'W', 'C', 'S', 'F', 'N', 'V', '6', '4'};
constexpr int kCkptVersion = 3;

// FNV-1a (64-bit offset basis and prime) over 8-byte little-endian words; a
// final partial word is hashed byte by byte.  Streaming: add() any split.
struct Fnv64 {
  uint64_t h = 14695981039346656037ull;
  unsigned char pend[8];
  int np = 0;
  static constexpr uint64_t kPrime = 1099511628211ull;
  void word(const unsigned char* b) {
    uint64_t w = 0;
    for (int i = 7; i >= 0; --i) w = (w << 8) | b[i];
    h = (h ^ w) * kPrime;
  }
  void add(const void* data, size_t n) {
    const unsigned char* p = (const unsigned char*)data;
    while (n > 0 && np > 0) {
      pend[np++] = *p++;
      --n;
      if (np == 8) { word(pend); np = 0; }
    }
    for (; n >= 8; n -= 8, p += 8) word(p);
    while (n > 0) { pend[np++] = *p++; --n; }
  }
  uint64_t finish() {
    for (int i = 0; i < np; ++i) h = (h ^ pend[i]) * kPrime;
    np = 0;
    return h;
  }
};

// Reads and writes that keep the running checksum.
struct CkptIO {
  FILE* f;
  Fnv64 sum;
  bool write;
  bool io(void* p, size_t bytes) {
    const bool ok = write ? (fwrite(p, 1, bytes, f) == bytes) : (fread(p, 1, bytes, f) == bytes);
    if (ok) sum.add(p, bytes);
    return ok;
  }
};

static int ckpt_arrays(wcs_ctx* c, CkptIO& io) {
  const int64_t N = c->N, r = c->rank;
  if (r <= 0) return 0;
  zd* arrs[3] = {c->U.z(), c->Vw.z(), c->Wt.z()};
  const int64_t chunk = std::max<int64_t>(1, ((int64_t)64 << 20) / (int64_t)(sizeof(zd) * N));   // columns
  std::vector<zd> host((size_t)N * std::min(chunk, r));
  for (int a = 0; a < 3; ++a) {
    for (int64_t c0 = 0; c0 < r; c0 += chunk) {
      const int64_t cc = std::min(chunk, r - c0);
      const size_t n = (size_t)N * cc;
      if (io.write) {
        cudaMemcpyAsync(host.data(), arrs[a] + c0 * N, sizeof(zd) * n, cudaMemcpyDeviceToHost, c->s);
        TRY(sync(c));
        if (!io.io(host.data(), sizeof(zd) * n)) { set_error("checkpoint: write failed"); return WCS_ERR_ARG; }
      } else {
        if (!io.io(host.data(), sizeof(zd) * n)) { set_error("checkpoint: file is truncated"); return WCS_ERR_ARG; }
        cudaMemcpyAsync(arrs[a] + c0 * N, host.data(), sizeof(zd) * n, cudaMemcpyHostToDevice, c->s);
        TRY(sync(c));
      }
    }
  }
  return 0;
}

// The r x r capacitance inverse (adjoint solves need it).
static int ckpt_kinv(wcs_ctx* c, CkptIO& io) {
  const int64_t r = c->rank;
  if (r <= 0) return 0;
  const size_t n = (size_t)r * r;
  std::vector<zd> host(n);
  if (io.write) {
    cudaMemcpyAsync(host.data(), c->Kinv.p, sizeof(zd) * n, cudaMemcpyDeviceToHost, c->s);
    TRY(sync(c));
    if (!io.io(host.data(), sizeof(zd) * n)) { set_error("checkpoint: write failed"); return WCS_ERR_ARG; }
    return 0;
  }
  if (!io.io(host.data(), sizeof(zd) * n)) { set_error("checkpoint: file is truncated"); return WCS_ERR_ARG; }
  TRY(c->Kinv.ensure(sizeof(zd) * n));
  cudaMemcpyAsync(c->Kinv.p, host.data(), sizeof(zd) * n, cudaMemcpyHostToDevice, c->s);
  return sync(c);
}

static bool ckpt_seek(FILE* f, int64_t off, int whence) {
#if defined(_WIN32)
  return _fseeki64(f, off, whence) == 0;
#else
  return fseeko(f, (off_t)off, whence) == 0;
#endif
}
static int64_t ckpt_tell(FILE* f) {
#if defined(_WIN32)
  return _ftelli64(f);
#else
  return (int64_t)ftello(f);
#endif
}

// Version 3: the file must be exactly as long as its header says, and the
// checksum over everything before the trailer must match.  Leaves f at the
// first byte after the header and extension.
static int ckpt_verify(FILE* f, const CkptHeader& hd, const CkptExt& ext) {
  const int64_t r = hd.rank, N = hd.N;
  const int64_t body = (int64_t)sizeof(CkptHeader) + (int64_t)sizeof(CkptExt);
  const int64_t payload = 3 * N * r * (int64_t)sizeof(zd) + ((ext.flags & 1u) ? r * r * (int64_t)sizeof(zd) : 0);
  const int64_t expect = body + payload + 16;
  if (!ckpt_seek(f, 0, SEEK_END)) { set_error("checkpoint: cannot seek"); return WCS_ERR_ARG; }
  const int64_t size = ckpt_tell(f);
  if (size < expect) { set_error("checkpoint: file is truncated"); return WCS_ERR_ARG; }
  if (size > expect) { set_error("checkpoint: unexpected bytes after the trailer"); return WCS_ERR_ARG; }
  if (!ckpt_seek(f, 0, SEEK_SET)) { set_error("checkpoint: cannot seek"); return WCS_ERR_ARG; }
  Fnv64 sum;
  std::vector<unsigned char> buf((size_t)64 << 20);
  for (int64_t left = size - 16; left > 0;) {
    const size_t n = (size_t)std::min<int64_t>(left, (int64_t)buf.size());
    if (fread(buf.data(), 1, n, f) != n) { set_error("checkpoint: read failed"); return WCS_ERR_ARG; }
    sum.add(buf.data(), n);
    left -= (int64_t)n;
  }
  unsigned char tr[16];
  if (fread(tr, 1, 16, f) != 16) { set_error("checkpoint: file is truncated"); return WCS_ERR_ARG; }
  uint64_t stored = 0;
  for (int i = 15; i >= 8; --i) stored = (stored << 8) | tr[i];
  if (std::memcmp(tr, kCkptTag, 8) != 0 || stored != sum.finish()) {
    set_error("checkpoint: checksum mismatch (the file is corrupted)");
    return WCS_ERR_ARG;
  }
  if (!ckpt_seek(f, body, SEEK_SET)) { set_error("checkpoint: cannot seek"); return WCS_ERR_ARG; }
  return 0;
}

int wcs_save(wcs_ctx* c, const char* path) {
  if (!c || !path) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  FILE* f = fopen(path, "wb");
  if (!f) { set_error(std::string("checkpoint: cannot open ") + path); return WCS_ERR_ARG; }
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.rank = c->rank;
  hd.N = c->N;
  hd.k = c->k;
  hd.opt = c->opt;
  hd.contour = c->contour;
  CkptExt ext{(c->rank > 0 && c->Kinv.p) ? 1u : 0u, 0u};
  CkptIO io{f, Fnv64{}, true};
  int r = (io.io(&hd, sizeof(hd)) && io.io(&ext, sizeof(ext))) ? 0 : WCS_ERR_ARG;
  if (r) set_error("checkpoint: write failed");
  if (!r) r = ckpt_arrays(c, io);
  if (!r && (ext.flags & 1u)) r = ckpt_kinv(c, io);
  if (!r) {
    unsigned char tr[16];
    std::memcpy(tr, kCkptTag, 8);
    uint64_t v = io.sum.finish();
    for (int i = 8; i < 16; ++i) { tr[i] = (unsigned char)(v & 0xFF); v >>= 8; }
    if (fwrite(tr, 1, 16, f) != 16) { set_error("checkpoint: write failed"); r = WCS_ERR_ARG; }
  }
  if (fclose(f) != 0 && !r) { set_error("checkpoint: write failed"); r = WCS_ERR_ARG; }
  return r;
}

int wcs_load(wcs_ctx* c, const char* path) {
  if (!c || !path) { set_error("bad argument"); return WCS_ERR_ARG; }
  FILE* f = fopen(path, "rb");
  if (!f) { set_error(std::string("checkpoint: cannot open ") + path); return WCS_ERR_ARG; }
  CkptHeader hd;
  CkptExt ext{0u, 0u};
  int r = 0;
  if (fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, kCkptMagic, 8) != 0 ||
      hd.version < 1 || hd.version > kCkptVersion) {
    set_error("checkpoint: not a checkpoint of this library");
    r = WCS_ERR_ARG;
  }
  if (!r && hd.version >= 3 && fread(&ext, sizeof(ext), 1, f) != 1) {
    set_error("checkpoint: file is truncated");
    r = WCS_ERR_ARG;
  }
  if (!r && (hd.N < 12 || hd.N > ((int64_t)1 << 22) || hd.rank < 0 || hd.rank > hd.N)) {
    set_error("checkpoint: bad sizes");
    r = WCS_ERR_ARG;
  }
  if (!r && hd.version >= 3) r = ckpt_verify(f, hd, ext);
  const bool has_kinv = (hd.version == 2) || (hd.version >= 3 && (ext.flags & 1u));
  // the factors only fit operators assembled the same way
  const wcs_options& o = c->opt;
  if (!r && (hd.opt.precision != o.precision || hd.opt.q_far != o.q_far || hd.opt.q_near != o.q_near ||
             hd.opt.near_band != o.near_band || hd.opt.mixed_planes != o.mixed_planes ||
             hd.opt.rhs_planes != o.rhs_planes || hd.opt.zfast != o.zfast)) {
    set_error("checkpoint: made with other precision or quadrature options than this context");
    r = WCS_ERR_ARG;
  }
  if (!r) r = set_contour(c, hd.contour);
  if (!r) r = wcs_mesh(c, hd.N, hd.k);
  if (!r) r = wcs_assemble(c);
  if (!r && hd.rank > 0) {
    const size_t b = sizeof(zd) * (size_t)hd.N * hd.rank;
    r = c->U.ensure(b);
    if (!r) r = c->Vw.ensure(b);
    if (!r) r = c->Wt.ensure(b);
  }
  if (!r) {
    c->rank = hd.rank;
    CkptIO io{f, Fnv64{}, false};
    r = ckpt_arrays(c, io);
    if (!r && has_kinv) r = ckpt_kinv(c, io);
  }
  fclose(f);
  if (r) return r;
  c->stage = ST_FACTORED;
  return WCS_OK;
}

int wcs_woodbury_apply(wcs_ctx* c, int64_t B, const double* b, int64_t ldb, double* x, int64_t ldx) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, b, ldb));
  TRY(check_block(c, B, x, ldx));
  const int64_t chunk = c->opt.rhs_chunk;
  TRY(ensure_work(c, std::min(B, chunk)));
  for (int64_t c0 = 0; c0 < B; c0 += chunk) {
    const int64_t cc = std::min(chunk, B - c0);
    TRY(woodbury(c, (const zd*)b + c0 * ldb, ldb, (zd*)x + c0 * ldx, ldx, cc));
  }
  return WCS_OK;
}

int wcs_planewave_rhs(wcs_ctx* c, int64_t B, const double* angles, double* e, double* hv, int64_t ld) {
  if (!c || (B > 0 && !angles)) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("mesh first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, e, ld));
  TRY(check_block(c, B, hv, ld));
  if (B == 0) return WCS_OK;
  TRY(check_angles(B, angles, "planewave_rhs"));
  DevBuf ang;
  TRY(ang.ensure(sizeof(double) * B));
  cudaMemcpyAsync(ang.p, angles, sizeof(double) * B, cudaMemcpyHostToDevice, c->s);
  int r = planewave_rhs(c->near, c->quad.wn, c->quad.xn, c->opt.q_near, c->N, c->h, c->k, ang.d(),
                        (int)B, (zd*)e, (zd*)hv, ld, c->s);
  if (!r) r = sync(c);
  ang.release();
  return r;
}

// b = -i k S~ G^{-1} e - (G/2 + D~) G^{-1} h  (Eq. 5), cc columns.
static int precondition(wcs_ctx* c, const zd* e, const zd* hv, int64_t ld, zd* b, int64_t ldb, int64_t cc,
                        int mode = PREC_ACCURATE) {
  const int64_t N = c->N;
  zd* T1 = c->w1.z();
  zd* T2 = c->w2.z();
  TRY(ginv(c, e, ld, T1, N, cc));
  TRY(ginv(c, hv, ld, T2, N, cc));
  if (c->mixed) {
    TRY(ensure_stage(c, cc));
    TRY(stage(c, c->stage1, T1, N, cc, 0));
    TRY(stage(c, c->stage2, T2, N, cc, 0));
    TRY(tc_apply(c, 0, false, c->stage1, cc, mkz(0.0, -c->k), mkz(0.0), b, ldb, mode));
    TRY(tc_apply(c, 2, false, c->stage2, cc, mkz(-1.0), mkz(1.0), b, ldb, mode));
  } else {
    TRY(zgemm(N, cc, N, mkz(0.0, -c->k), op_view(c->S, c->ld, false), blk(T1, N), mkz(0.0), b, ldb, c->s));
    TRY(zgemm(N, cc, N, mkz(-1.0), op_view(c->Dt, c->ld, false), blk(T2, N), mkz(1.0), b, ldb, c->s));
  }
  TRY(gram_apply(T2, N, b, ldb, N, cc, c->h, -0.5, 1.0, c->s));
  return 0;
}

// Mixed form: R = b - C x with b of Eq. (5) left implicit,
//   R = -(G/2 + D~) G^{-1} (h + (G/2 - D) x) - S~ G^{-1} (i k e + N x),
// i.e. the four products of C x and no product for b.  Uses w1, w2.
static int residual_rhs_mixed(wcs_ctx* c, const zd* e, const zd* hv, int64_t ld, const zd* x, int64_t ldx,
                              zd* R, int64_t cc, int mode) {
  const int64_t N = c->N;
  zd* T1 = c->w1.z();
  zd* T2 = c->w2.z();
  const zd one = mkz(1.0), zero = mkz(0.0), mone = mkz(-1.0);
  if (mode == PREC_EXACT) {
    TRY(ex_apply(c, 1, x, ldx, cc, mone, zero, T1, N));                 // -D x
    TRY(ex_apply(c, 3, x, ldx, cc, one, zero, T2, N));                  // N x
    TRY(gram_apply(x, ldx, T1, N, N, cc, c->h, 0.5, 1.0, c->s));        // + G x / 2
    TRY(axpby(N, cc, one, hv, ld, one, T1, N, c->s));                   // + h
    TRY(axpby(N, cc, mkz(0.0, c->k), e, ld, one, T2, N, c->s));         // + i k e
    TRY(ginv(c, T1, N, T1, N, cc));
    TRY(ginv(c, T2, N, T2, N, cc));
    TRY(ex_apply(c, 2, T1, N, cc, mone, zero, R, N));                   // -D~ T1
    TRY(ex_apply(c, 0, T2, N, cc, mone, one, R, N));                    // - S~ T2
    TRY(gram_apply(T1, N, R, N, N, cc, c->h, -0.5, 1.0, c->s));         // - G T1 / 2
    return 0;
  }
  TRY(ensure_stage(c, cc));
  TRY(stage(c, c->stage0, x, ldx, cc, 0));
  TRY(tc_apply(c, 1, false, c->stage0, cc, mone, zero, T1, N, mode));   // -D x
  TRY(tc_apply(c, 3, false, c->stage0, cc, one, zero, T2, N, mode));    // N x
  TRY(gram_apply(x, ldx, T1, N, N, cc, c->h, 0.5, 1.0, c->s));          // + G x / 2
  TRY(axpby(N, cc, one, hv, ld, one, T1, N, c->s));                     // + h
  TRY(axpby(N, cc, mkz(0.0, c->k), e, ld, one, T2, N, c->s));           // + i k e
  TRY(ginv(c, T1, N, T1, N, cc));
  TRY(ginv(c, T2, N, T2, N, cc));
  TRY(stage(c, c->stage1, T1, N, cc, 0));
  TRY(stage(c, c->stage2, T2, N, cc, 0));
  TRY(tc_apply(c, 2, false, c->stage1, cc, mone, zero, R, N, mode));    // -D~ T1
  TRY(tc_apply(c, 0, false, c->stage2, cc, mone, one, R, N, mode));     // - S~ T2
  TRY(gram_apply(T1, N, R, N, N, cc, c->h, -0.5, 1.0, c->s));           // - G T1 / 2
  return 0;
}

// x = C^{-1} b with Woodbury + iterative refinement on the exact operator.
// Mixed form with e, hv given: b only seeds x and scales the residual norm;
// every residual is formed from e and hv directly (residual_rhs_mixed).
// acc gathers the statistics over the blocks of one call: steps and final
// residual (max over blocks) and the residual history (see wcs_solve_info).
static int solve_block(wcs_ctx* c, const zd* b, int64_t ldb, zd* x, int64_t ldx, int64_t cc,
                       wcs_solve_info* acc, const zd* e = nullptr, const zd* hv = nullptr,
                       int64_t ld_eh = 0, bool adj = false) {
  const int64_t N = c->N;
  // adj: solve C^H x = b (the adjoint Woodbury and C^H in every residual)
  auto approx_inverse = [&](const zd* B, int64_t ldb_, zd* X, int64_t ldx_) -> int {
    return adj ? woodbury_adj(c, B, ldb_, X, ldx_, cc) : woodbury(c, B, ldb_, X, ldx_, cc);
  };
  TRY(approx_inverse(b, ldb, x, ldx));
  DevBuf nb;
  TRY(nb.ensure(sizeof(double) * 2 * cc));
  std::vector<double> bn(cc), rn(cc);
  TRY(column_norms(b, ldb, N, cc, nb.d(), c->s));
  cudaMemcpyAsync(bn.data(), nb.p, sizeof(double) * cc, cudaMemcpyDeviceToHost, c->s);
  zd* R = c->w4.z();
  zd* dx = c->w5.z();
  zd* T = c->w3.z();
  int it = 0;
  // residual after each refinement step of this block (the last evaluation
  // at a step wins: a recomputed residual replaces the carried one)
  double hist[WCS_HISTORY];
  int hlen = 0;
  auto finish = [&](double final_res) {
    acc->refine_steps = std::max(acc->refine_steps, it);
    acc->rel_residual = std::max(acc->rel_residual, final_res);
    if (hlen == 0) { hist[0] = final_res; hlen = 1; }
    for (int i = 0; i < WCS_HISTORY; ++i) {
      const double v = hist[std::min(i, hlen - 1)];   // a block that stopped keeps its last value
      acc->history[i] = std::max(acc->history[i], v);
    }
    acc->history_len = std::max(acc->history_len, hlen);
  };
  // largest relative residual over the block's columns.  A right-hand side
  // that is not finite is the caller's error (WCS_ERR_ARG); a residual that
  // is not finite for a finite right-hand side ends the solve as not
  // converged (the refinement cannot recover from it).
  auto worst_of = [&](double& worst) -> int {
    TRY(column_norms(R, N, N, cc, nb.d() + cc, c->s));
    cudaMemcpyAsync(rn.data(), nb.d() + cc, sizeof(double) * cc, cudaMemcpyDeviceToHost, c->s);
    TRY(sync(c));
    worst = 0;
    for (int64_t j = 0; j < cc; ++j) {
      if (!std::isfinite(bn[j])) {
        set_error("right-hand side column " + std::to_string(j) + " of the block is not finite");
        return WCS_ERR_ARG;
      }
      if (!std::isfinite(rn[j])) {
        set_error("solve: the residual of column " + std::to_string(j) + " of the block is not finite");
        finish(INFINITY);
        return WCS_ERR_NOT_CONVERGED;
      }
      worst = std::max(worst, bn[j] > 0 ? rn[j] / bn[j] : rn[j]);
    }
    if (it < WCS_HISTORY) {
      hist[it] = worst;
      hlen = std::max(hlen, it + 1);
    }
    return 0;
  };
  // R = b - C x with the given precision
  auto residual = [&](int mode, double& worst) -> int {
    if (c->mixed && e && hv && !adj) {
      TRY(residual_rhs_mixed(c, e, hv, ld_eh, x, ldx, R, cc, mode));
    } else {
      TRY(apply_C(c, x, ldx, R, N, cc, adj, mode));
      TRY(axpby(N, cc, mkz(1.0), b, ldb, mkz(-1.0), R, N, c->s));
    }
    return worst_of(worst);
  };
  // After an update, the contraction of the previous one (carried residual
  // upd after prev_upd) predicts the next carried residual.  When that is far
  // below the target the round ends without carrying the residual: the
  // recomputed residual that closes every round replaces it anyway, so the
  // product R <- R - C dx would be spent only to be overwritten.  The round's
  // first update has no contraction yet and always carries.  A wrong
  // prediction costs nothing but another round.
  auto ends_round = [&](double& upd, double prev_upd) -> bool {
    if (!(prev_upd < 1e299) || !(upd > 0.0)) return false;
    const double pred = upd * (upd / prev_upd);
    if (!(pred < 0.01 * c->opt.refine_tol)) return false;
    upd = pred;
    return true;
  };
  double worst = 0;
  if (!c->mixed) {
    // FP64 form: plain refinement on the exact residual
    TRY(residual(PREC_ACCURATE, worst));
    while (worst > c->opt.refine_tol && it < c->opt.max_refine) {
      TRY(approx_inverse(R, N, dx, N));
      TRY(axpby(N, cc, mkz(1.0), dx, N, mkz(1.0), x, ldx, c->s));
      ++it;
      TRY(residual(PREC_ACCURATE, worst));
    }
  } else if (c->opt.exact_residual && !adj) {
    // Mixed form with exact residuals.  Every true residual is exact; the
    // updates R <- R - C dx use the cheapest product whose error (relative to
    // |C dx| ~ the carried residual) stays below ~1e-11 of |b|: exact while
    // the carried residual is above 5e-5, the drained product (~2e-7) down to
    // 5e-7, the periodic drain (~2e-5) below.  Rounds end with a recomputed
    // residual, as in the other branch.
    TRY(residual(PREC_EXACT, worst));
    double prev_true = 1e300;
    bool floor = false;
    while (worst > c->opt.refine_tol && it < c->opt.max_refine && worst < 0.5 * prev_true && !floor) {
      prev_true = worst;
      double upd = worst, prev_upd = 1e300;
      while (upd > 0.1 * c->opt.refine_tol && it < c->opt.max_refine && upd < 0.7 * prev_upd) {
        TRY(approx_inverse(R, N, dx, N));
        TRY(axpby(N, cc, mkz(1.0), dx, N, mkz(1.0), x, ldx, c->s));
        ++it;
        if (ends_round(upd, prev_upd)) break;
        const int m = (upd > 5e-5) ? PREC_EXACT : (upd > 5e-7 ? PREC_ACCURATE : PREC_PERIODIC);
        TRY(apply_C(c, dx, N, T, N, cc, adj, m));
        TRY(axpby(N, cc, mkz(-1.0), T, N, mkz(1.0), R, N, c->s));
        prev_upd = upd;
        TRY(worst_of(upd));
      }
      TRY(residual(PREC_EXACT, worst));
      floor = worst > 10.0 * upd;
    }
  } else {
    // Mixed form.  The first residual is formed with the drained accumulation
    // (~1e-7) and then carried forward by updates R <- R - C dx in the
    // periodic-drain precision (~2e-5 of |C dx|, far below the residual once
    // |dx| is small) or, while |C dx| is large, the drained one.  Each round ends with a recomputed
    // residual, so the reported residual is the true one; rounds stop when it
    // reaches refine_tol or stops decreasing (its floor is the accuracy of
    // the drained product).
    TRY(residual(PREC_ACCURATE, worst));
    double prev_true = 1e300;
    bool floor = false;   // a round ended with the true residual far above the carried one
    while (worst > c->opt.refine_tol && it < c->opt.max_refine && worst < 0.5 * prev_true && !floor) {
      prev_true = worst;
      double upd = worst, prev_upd = 1e300;
      // updates until the carried residual is well below the target
      while (upd > 0.1 * c->opt.refine_tol && it < c->opt.max_refine && upd < 0.7 * prev_upd) {
        TRY(approx_inverse(R, N, dx, N));
        TRY(axpby(N, cc, mkz(1.0), dx, N, mkz(1.0), x, ldx, c->s));
        ++it;
        if (ends_round(upd, prev_upd)) break;
        // the update's error is ~2e-5 of |C dx| ~ the carried residual in the
        // periodic drain: while that would exceed a tenth of the target (a
        // poor approximate inverse, a large residual), the drained product
        // (~2e-7) carries it instead, so the carried residual does not drift
        // from the true one
        const int m = (2e-5 * upd <= 0.1 * c->opt.refine_tol) ? PREC_PERIODIC : PREC_ACCURATE;
        TRY(apply_C(c, dx, N, T, N, cc, adj, m));
        TRY(axpby(N, cc, mkz(-1.0), T, N, mkz(1.0), R, N, c->s));
        prev_upd = upd;
        TRY(worst_of(upd));
      }
      TRY(residual(PREC_ACCURATE, worst));
      // the gap is the evaluation floor of the drained product: another round
      // would start from (and return to) the same floor
      floor = worst > 10.0 * upd;
    }
  }
  nb.release();
  finish(worst);
  return (worst <= c->opt.refine_tol) ? 0 : WCS_ERR_NOT_CONVERGED;
}

int wcs_solve_rhs(wcs_ctx* c, int64_t B, const double* e, const double* hv, int64_t ld, double* j,
                  int64_t ldj, wcs_solve_info* info) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, e, ld));
  TRY(check_block(c, B, hv, ld));
  TRY(check_block(c, B, j, ldj));
  const int64_t chunk = c->opt.rhs_chunk, N = c->N;
  TRY(ensure_work(c, std::min(B, chunk)));
  DevBuf bb;
  TRY(bb.ensure(sizeof(zd) * N * std::min(B, chunk)));
  int status = WCS_OK;
  wcs_solve_info acc{};
  for (int64_t c0 = 0; c0 < B; c0 += chunk) {
    const int64_t cc = std::min(chunk, B - c0);
    // mixed form: b only seeds the solution (residuals are formed from e, h)
    const zd* ec = (const zd*)e + c0 * ld;
    const zd* hc = (const zd*)hv + c0 * ld;
    TRY(precondition(c, ec, hc, ld, bb.z(), N, cc, c->mixed ? PREC_PERIODIC : PREC_ACCURATE));
    int r = solve_block(c, bb.z(), N, (zd*)j + c0 * ldj, ldj, cc, &acc, ec, hc, ld);
    if (r == WCS_ERR_NOT_CONVERGED) status = r;
    else if (r) return r;
  }
  bb.release();
  if (info) *info = acc;
  if (status) set_error("iterative refinement did not reach refine_tol");
  return status;
}

// C x = b (adj: C^H x = b) for B general right-hand sides, chunked.
static int solve_general(wcs_ctx* c, int64_t B, const double* b, int64_t ldb, double* x, int64_t ldx,
                         wcs_solve_info* info, bool adj) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, b, ldb));
  TRY(check_block(c, B, x, ldx));
  if (B == 0) return WCS_OK;
  const int64_t chunk = c->opt.rhs_chunk;
  TRY(ensure_work(c, std::min(B, chunk)));
  int status = WCS_OK;
  wcs_solve_info acc{};
  for (int64_t c0 = 0; c0 < B; c0 += chunk) {
    const int64_t cc = std::min(chunk, B - c0);
    int r = solve_block(c, (const zd*)b + c0 * ldb, ldb, (zd*)x + c0 * ldx, ldx, cc, &acc, nullptr,
                        nullptr, 0, adj);
    if (r == WCS_ERR_NOT_CONVERGED) status = r;
    else if (r) return r;
  }
  if (info) *info = acc;
  if (status) set_error("iterative refinement did not reach refine_tol");
  return status;
}

int wcs_solve(wcs_ctx* c, int64_t B, const double* b, int64_t ldb, double* x, int64_t ldx,
              wcs_solve_info* info) {
  return solve_general(c, B, b, ldb, x, ldx, info, false);
}

int wcs_solve_adjoint(wcs_ctx* c, int64_t B, const double* b, int64_t ldb, double* x, int64_t ldx,
                      wcs_solve_info* info) {
  return solve_general(c, B, b, ldb, x, ldx, info, true);
}

}  // extern "C"

// ---------------------------------------------------------------- shape derivatives
// The contour of parameter i at offset d: the current contour with the Fourier
// perturbation alpha_i (i < M) or beta_{i-M+1} moved by d.
static Contour perturbed_contour(const Contour& base, int M, int i, double d) {
  Contour k = base;
  if (k.np == 0)
    for (int m = 0; m < kMaxPerturb; ++m) { k.pc[m] = 0.0; k.ps[m] = 0.0; }
  k.np = std::max(k.np, M + 1);
  if (i < M) k.pc[i] += d;
  else k.ps[i - M + 1] += d;
  return k;
}

struct CtxGuard {
  wcs_ctx* t = nullptr;
  ~CtxGuard() { if (t) wcs_destroy(t); }
};

// Scratch context meshing the perturbed contours (geometry only, no assembly):
// same N, k and quadrature rules as c.
static int make_scratch(wcs_ctx* c, CtxGuard& g) {
  wcs_options o = c->opt;
  o.precision = WCS_PREC_FP64;
  o.zfast = 0.0;
  o.exact_residual = 0;
  return wcs_create(&g.t, &o, (void*)c->s);
}

__global__ void k_geo_dot(const double* Gr, const double* Gn, Points pp, Points pm, int64_t n, double* part) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double re = 0.0, im = 0.0;
  if (t < n) {
    const double dr[2] = {pp.x[t] - pm.x[t], pp.y[t] - pm.y[t]};
    const double dn[2] = {pp.nx[t] - pm.nx[t], pp.ny[t] - pm.ny[t]};
    const double* g = Gr + 4 * t;
    const double* h = Gn + 4 * t;
    re = g[0] * dr[0] + g[2] * dr[1] + h[0] * dn[0] + h[2] * dn[1];
    im = g[1] * dr[0] + g[3] * dr[1] + h[1] * dn[0] + h[3] * dn[1];
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = re; red[1][threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) { a += red[0][w]; b += red[1][w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// Sum of `n` partial (re, im) pairs in device memory, in a fixed order on the host.
static int sum_parts(wcs_ctx* c, const double* part, int n, zd* out) {
  std::vector<double> h(2 * (size_t)n);
  cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->s);
  TRY(sync(c));
  double re = 0.0, im = 0.0;
  for (int i = 0; i < n; ++i) { re += h[2 * i]; im += h[2 * i + 1]; }
  *out = mkz(re, im);
  return 0;
}

// One assembled operator applied alone: Y = op X or op^H X (0 S~, 1 D, 2 D~, 3 N).
static int op_apply(wcs_ctx* c, int which, bool adj, const zd* X, int64_t ldx, int64_t cols, zd* Y, int64_t ldy) {
  if (!c->mixed) {
    const zd* ops[4] = {c->S, c->D, c->Dt, c->Nk};
    return zgemm(c->N, cols, c->N, mkz(1.0), op_view(ops[which], c->ld, adj), blk(X, ldx), mkz(0.0), Y, ldy, c->s);
  }
  TRY(ensure_stage(c, cols));
  TRY(stage(c, c->stage0, X, ldx, cols, adj ? 1 : 0));
  return tc_apply(c, which, adj, c->stage0, cols, mkz(1.0), mkz(0.0), Y, ldy, PREC_ACCURATE);
}

// T_i = sum_X sum_ij W[X]_ij dX_ij / dp_i for parameters i0 <= i < i1 (out[i - i0]):
// the far pairs by the one-pass derivative kernel (per-point gradients
// contracted with the point motion, k~ and h^2 terms), the near band by
// central differences of its pair integrals (step delta).  W: four row-major
// N x N device matrices (S~, D, D~, N); points move as the arc-length mesh
// of the perturbed contour dictates (central differences of the geometry).
// Scratch contexts tp, tm are meshed on the perturbed contours of parameter i
// and left there for the caller (per_param is called after each).
template <typename F>
static int shape_forms(wcs_ctx* c, const zd* const* W, int M, int i0, int i1, double delta, zd* out, CtxGuard& tp,
                       CtxGuard& tm, F per_param) {
  const int64_t N = c->N, nq = N * c->opt.q_far;
  DevBuf gr, gn, sc, part;
  TRY(gr.ensure(sizeof(double) * 4 * nq));
  TRY(gn.ensure(sizeof(double) * 4 * nq));
  TRY(sc.ensure(sizeof(double) * 4));
  const int64_t nblk_geo = (nq + 255) / 256, nblk_near = (N * (2 * c->opt.near_band + 1) + 127) / 128;
  TRY(part.ensure(sizeof(double) * 2 * std::max(nblk_geo, nblk_near)));
  cudaMemsetAsync(gr.p, 0, gr.bytes, c->s);
  cudaMemsetAsync(gn.p, 0, gn.bytes, c->s);
  cudaMemsetAsync(sc.p, 0, sc.bytes, c->s);
  ShapeArgs sa;
  sa.A = asm_args(c, false);
  for (int X = 0; X < 4; ++X) sa.W[X] = W[X];
  sa.Gr = gr.d();
  sa.Gn = gn.d();
  sa.scal = sc.d();
  {
    ProfScope ps(c, CAT_ASSEMBLY, (double)N * N * c->opt.q_far * c->opt.q_far, 0.0);
    TRY(shape_far_forms(sa, c->s));
  }
  double scal[4];
  cudaMemcpyAsync(scal, sc.p, sizeof(scal), cudaMemcpyDeviceToHost, c->s);
  TRY(sync(c));
  const zd s_kt = mkz(scal[0], scal[1]), s_h2 = mkz(scal[2], scal[3]);
  for (int i = i0; i < i1; ++i) {
    TRY(set_contour(tp.t, perturbed_contour(c->contour, M, i, delta)));
    TRY(wcs_mesh(tp.t, N, c->k));
    TRY(set_contour(tm.t, perturbed_contour(c->contour, M, i, -delta)));
    TRY(wcs_mesh(tm.t, N, c->k));
    zd geo, np_, nm_;
    k_geo_dot<<<(unsigned)nblk_geo, 256, 0, c->s>>>(gr.d(), gn.d(), tp.t->far, tm.t->far, nq, part.d());
    note_launch();
    TRY(sum_parts(c, part.d(), (int)nblk_geo, &geo));
    int nb = 0;
    TRY(shape_near_forms(asm_args(tp.t, false), W, part.d(), &nb, c->s));
    TRY(sum_parts(c, part.d(), nb, &np_));
    TRY(shape_near_forms(asm_args(tm.t, false), W, part.d(), &nb, c->s));
    TRY(sum_parts(c, part.d(), nb, &nm_));
    const double dL = (tp.t->L - tm.t->L) / (2.0 * delta);
    const zd dkt = (1.0 / (2.0 * delta)) * (tp.t->kt - tm.t->kt);
    const zd far = (1.0 / (2.0 * delta)) * geo + s_kt * dkt + (2.0 * dL / c->L) * s_h2;
    const zd near = (1.0 / (2.0 * delta)) * (np_ - nm_);
    out[i - i0] = far + near;
    TRY(per_param(i, dL));
  }
  return 0;
}

extern "C" {

// Far-field shape gradient by the adjoint route.  With j = C^-1 b (forward
// solve), F = E j and lam = C^-H E^H F (one adjoint solve),
//   dJ/dp = 2 Re sum_b [F_b^H dE j_b + lam_b^H dR_b],  R = b - C j,
// and R = -(G/2 + D~) q1 - S~ q2 with q1 = G^-1 (h + (G/2 - D) j),
// q2 = G^-1 (i k e + N j) (Eq. 5 with C of Eq. 6), so with
// w1 = G^-1 (G/2 + D~)^H lam, w2 = G^-1 S~^H lam and dG = (dL/L) G,
//   lam^H dR = -lam^H dD~ q1 - lam^H dS~ q2 + w1^H dD j - w2^H dN j
//              + (dL/L) [-lam^H G q1 / 2 - w1^H G j / 2 + w1^H G q1 + w2^H G q2]
//              - w1^H dh - i k w2^H de.
// The operator terms come from shape_forms (one pass over the far pairs for
// every parameter); dE, de, dh (O(N) per parameter) are central differences.
int wcs_shape_gradient_range(wcs_ctx* c, int64_t B, const double* angles, int nphi, const double* phi, int M,
                             double delta, int i0, int i1, double* J_out, double* grad) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  if (B < 1 || nphi < 1 || !angles || !phi || !J_out || M < 0 || M > kMaxPerturb - 1 || i0 < 0 ||
      i1 < i0 || i1 > 2 * M || (i1 > i0 && !grad)) {
    set_error("shape gradient: bad argument");
    return WCS_ERR_ARG;
  }
  TRY(check_angles(B, angles, "shape_gradient (incidences)"));
  TRY(check_angles(nphi, phi, "shape_gradient (observation angles)"));
  if (!(delta > 0)) delta = 1e-6;
  const int64_t N = c->N;
  DevBuf j, lam, E, F, G, ang, phd, dots;
  TRY(j.ensure(sizeof(zd) * N * B));
  TRY(lam.ensure(sizeof(zd) * N * B));
  TRY(G.ensure(sizeof(zd) * N * B));
  TRY(E.ensure(sizeof(zd) * N * nphi));
  TRY(F.ensure(sizeof(zd) * nphi * B));
  TRY(ang.ensure(sizeof(double) * B));
  TRY(phd.ensure(sizeof(double) * nphi));
  TRY(dots.ensure(sizeof(zd) * 4 * B));
  cudaMemcpyAsync(ang.p, angles, sizeof(double) * B, cudaMemcpyHostToDevice, c->s);
  cudaMemcpyAsync(phd.p, phi, sizeof(double) * nphi, cudaMemcpyHostToDevice, c->s);
  // forward: j, F = E j, J
  int status = WCS_OK;
  wcs_solve_info si{};
  int r = wcs_solve_planewaves(c, B, angles, j.d(), N, &si);
  if (r == WCS_ERR_NOT_CONVERGED) status = r;
  else if (r) return r;
  TRY(farfield_matrix(c->near, c->quad.wn, c->quad.xn, c->opt.q_near, N, c->h, c->k, phd.d(), nphi, E.z(),
                      nphi, c->s));
  TRY(zgemm(nphi, B, N, mkz(1.0), ZView{E.z(), 1, nphi, false}, blk(j.z(), N), mkz(0.0), F.z(), nphi, c->s));
  std::vector<zd> hd(4 * B);
  TRY(column_dotc(F.z(), nphi, F.z(), nphi, nphi, B, dots.z(), c->s));
  cudaMemcpyAsync(hd.data(), dots.p, sizeof(zd) * B, cudaMemcpyDeviceToHost, c->s);
  TRY(sync(c));
  double J = 0.0;
  for (int64_t b = 0; b < B; ++b) J += hd[b].x;
  *J_out = J;
  if (i1 == i0) return status;
  // adjoint: lam = C^-H E^H F
  TRY(zgemm(N, B, nphi, mkz(1.0), ZView{E.z(), nphi, 1, true}, blk(F.z(), nphi), mkz(0.0), G.z(), N, c->s));
  r = solve_general(c, B, G.d(), N, lam.d(), N, &si, true);
  if (r == WCS_ERR_NOT_CONVERGED) status = r;
  else if (r) return r;
  // q1, q2, w1, w2 of the base contour
  DevBuf eb, hb, q1, q2, w1, w2, T, gq;
  for (DevBuf* b : {&eb, &hb, &q1, &q2, &w1, &w2, &T, &gq}) TRY(b->ensure(sizeof(zd) * N * B));
  TRY(planewave_rhs(c->near, c->quad.wn, c->quad.xn, c->opt.q_near, N, c->h, c->k, ang.d(), (int)B, eb.z(), hb.z(),
                    N, c->s));
  TRY(op_apply(c, 1, false, j.z(), N, B, T.z(), N));                         // D j
  TRY(axpby(N, B, mkz(1.0), hb.z(), N, mkz(-1.0), T.z(), N, c->s));         // h - D j
  TRY(gram_apply(j.z(), N, T.z(), N, N, B, c->h, 0.5, 1.0, c->s));          // + G j / 2
  TRY(ginv(c, T.z(), N, q1.z(), N, B));
  TRY(op_apply(c, 3, false, j.z(), N, B, T.z(), N));                         // N j
  TRY(axpby(N, B, mkz(0.0, c->k), eb.z(), N, mkz(1.0), T.z(), N, c->s));    // + i k e
  TRY(ginv(c, T.z(), N, q2.z(), N, B));
  TRY(op_apply(c, 2, true, lam.z(), N, B, T.z(), N));                        // D~^H lam
  TRY(gram_apply(lam.z(), N, T.z(), N, N, B, c->h, 0.5, 1.0, c->s));        // + G lam / 2
  TRY(ginv(c, T.z(), N, w1.z(), N, B));
  TRY(op_apply(c, 0, true, lam.z(), N, B, T.z(), N));                        // S~^H lam
  TRY(ginv(c, T.z(), N, w2.z(), N, B));
  // Gram term: -lam^H G q1 / 2 - w1^H G j / 2 + w1^H G q1 + w2^H G q2
  zd gam = mkz(0.0);
  {
    const zd* pairs[4][2] = {{lam.z(), q1.z()}, {w1.z(), j.z()}, {w1.z(), q1.z()}, {w2.z(), q2.z()}};
    const double wts[4] = {-0.5, -0.5, 1.0, 1.0};
    for (int t = 0; t < 4; ++t) {
      TRY(gram_apply(pairs[t][1], N, gq.z(), N, N, B, c->h, 1.0, 0.0, c->s));
      TRY(column_dotc(pairs[t][0], N, gq.z(), N, N, B, dots.z(), c->s));
      cudaMemcpyAsync(hd.data(), dots.p, sizeof(zd) * B, cudaMemcpyDeviceToHost, c->s);
      TRY(sync(c));
      for (int64_t b = 0; b < B; ++b) gam += wts[t] * hd[b];
    }
  }
  // node-pair coefficients W (row-major): W_S = -sum conj(lam) q2^T, W_D~ =
  // -sum conj(lam) q1^T, W_D = sum conj(w1) j^T, W_N = -sum conj(w2) j^T
  DevBuf Wb;
  TRY(Wb.ensure(sizeof(zd) * 4 * N * N));
  const zd* W[4];
  {
    const zd* U[4] = {lam.z(), w1.z(), lam.z(), w2.z()};
    const zd* V[4] = {q2.z(), j.z(), q1.z(), j.z()};
    const double sgn[4] = {-1.0, 1.0, -1.0, -1.0};
    for (int X = 0; X < 4; ++X) {
      zd* Wx = Wb.z() + (int64_t)X * N * N;
      TRY(zgemm(N, N, B, mkz(sgn[X]), ZView{V[X], 1, N, false}, ZView{U[X], N, 1, true}, mkz(0.0), Wx, N, c->s));
      W[X] = Wx;
    }
  }
  eb.release(); hb.release(); T.release(); gq.release(); G.release();
  // per parameter: the operator terms (shape_forms) plus the O(N) terms
  CtxGuard tp, tm;
  TRY(make_scratch(c, tp));
  TRY(make_scratch(c, tm));
  DevBuf ep, hp, em, hm, Wf;
  for (DevBuf* b : {&ep, &hp, &em, &hm}) TRY(b->ensure(sizeof(zd) * N * B));
  TRY(Wf.ensure(sizeof(zd) * nphi * B));
  std::vector<zd> T_ops(i1 - i0);
  auto per_param = [&](int i, double dL) -> int {
    // far field: F^H (E+ - E-) j
    zd ff = mkz(0.0);
    for (int sgn = 0; sgn < 2; ++sgn) {
      wcs_ctx* t = sgn == 0 ? tp.t : tm.t;
      TRY(farfield_matrix(t->near, t->quad.wn, t->quad.xn, t->opt.q_near, N, t->h, t->k, phd.d(), nphi, E.z(),
                          nphi, c->s));
      TRY(zgemm(nphi, B, N, mkz(1.0), ZView{E.z(), 1, nphi, false}, blk(j.z(), N), mkz(0.0), Wf.z(), nphi, c->s));
      TRY(column_dotc(F.z(), nphi, Wf.z(), nphi, nphi, B, dots.z(), c->s));
      cudaMemcpyAsync(hd.data(), dots.p, sizeof(zd) * B, cudaMemcpyDeviceToHost, c->s);
      TRY(sync(c));
      for (int64_t b = 0; b < B; ++b) ff += (sgn == 0 ? 1.0 : -1.0) * hd[b];
    }
    // right-hand sides: w1^H (h+ - h-) + i k w2^H (e+ - e-)
    TRY(planewave_rhs(tp.t->near, tp.t->quad.wn, tp.t->quad.xn, tp.t->opt.q_near, N, tp.t->h, tp.t->k, ang.d(),
                      (int)B, ep.z(), hp.z(), N, c->s));
    TRY(planewave_rhs(tm.t->near, tm.t->quad.wn, tm.t->quad.xn, tm.t->opt.q_near, N, tm.t->h, tm.t->k, ang.d(),
                      (int)B, em.z(), hm.z(), N, c->s));
    TRY(axpby(N, B, mkz(-1.0), hm.z(), N, mkz(1.0), hp.z(), N, c->s));
    TRY(axpby(N, B, mkz(-1.0), em.z(), N, mkz(1.0), ep.z(), N, c->s));
    TRY(column_dotc(w1.z(), N, hp.z(), N, N, B, dots.z(), c->s));
    TRY(column_dotc(w2.z(), N, ep.z(), N, N, B, dots.z() + B, c->s));
    cudaMemcpyAsync(hd.data(), dots.p, sizeof(zd) * 2 * B, cudaMemcpyDeviceToHost, c->s);
    TRY(sync(c));
    zd rhs = mkz(0.0);
    for (int64_t b = 0; b < B; ++b) rhs += hd[b] + mkz(0.0, c->k) * hd[B + b];
    const double inv = 1.0 / (2.0 * delta);
    const zd total = inv * ff + T_ops[i - i0] + (dL / c->L) * gam - inv * rhs;
    grad[i - i0] = 2.0 * total.x;
    return 0;
  };
  TRY(shape_forms(c, W, M, i0, i1, delta, T_ops.data(), tp, tm, per_param));
  return status;
}

// T_i = sum_b u_b^H (dX / dp_i) v_b for one operator X (0 S~, 1 D, 2 D~, 3 N).
int wcs_shape_operator_forms(wcs_ctx* c, int op, int64_t B, const double* u_dev, const double* v_dev, int64_t ld,
                             int M, double delta, int i0, int i1, double* out_host) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  if (c->stage < ST_ASSEMBLED) { set_error("assemble first"); return WCS_ERR_STATE; }
  if (op < 0 || op > 3 || B < 1 || !u_dev || !v_dev || ld < c->N || M < 0 || M > kMaxPerturb - 1 || i0 < 0 ||
      i1 < i0 || i1 > 2 * M || (i1 > i0 && !out_host)) {
    set_error("shape operator forms: bad argument");
    return WCS_ERR_ARG;
  }
  if (!(delta > 0)) delta = 1e-6;
  const int64_t N = c->N;
  DevBuf Wb;
  TRY(Wb.ensure(sizeof(zd) * 4 * N * N));
  cudaMemsetAsync(Wb.p, 0, Wb.bytes, c->s);
  const zd* W[4];
  for (int X = 0; X < 4; ++X) W[X] = Wb.z() + (int64_t)X * N * N;
  TRY(zgemm(N, N, B, mkz(1.0), ZView{(const zd*)v_dev, 1, ld, false}, ZView{(const zd*)u_dev, ld, 1, true}, mkz(0.0),
            Wb.z() + (int64_t)op * N * N, N, c->s));
  CtxGuard tp, tm;
  TRY(make_scratch(c, tp));
  TRY(make_scratch(c, tm));
  std::vector<zd> T(i1 - i0);
  TRY(shape_forms(c, W, M, i0, i1, delta, T.data(), tp, tm, [](int, double) { return 0; }));
  for (int i = 0; i < i1 - i0; ++i) { out_host[2 * i] = T[i].x; out_host[2 * i + 1] = T[i].y; }
  return WCS_OK;
}

int wcs_shape_gradient(wcs_ctx* c, int64_t B, const double* angles, int nphi, const double* phi, int M,
                       double delta, double* J_out, double* grad) {
  return wcs_shape_gradient_range(c, B, angles, nphi, phi, M, delta, 0, 2 * M, J_out, grad);
}

int wcs_solve_planewaves(wcs_ctx* c, int64_t B, const double* angles, double* j, int64_t ldj,
                         wcs_solve_info* info) {
  if (!c || (B > 0 && !angles)) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_FACTORED) { set_error("factor first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, j, ldj));
  if (B == 0) return WCS_OK;
  TRY(check_angles(B, angles, "solve_planewaves"));
  const int64_t chunk = c->opt.rhs_chunk, N = c->N;
  TRY(ensure_work(c, std::min(B, chunk)));
  DevBuf &eb = c->sol_e, &hb = c->sol_h, &bb = c->sol_b, &ang = c->sol_ang;
  const int64_t cmax = std::min(B, chunk);
  TRY(eb.ensure(sizeof(zd) * N * cmax));
  TRY(hb.ensure(sizeof(zd) * N * cmax));
  TRY(bb.ensure(sizeof(zd) * N * cmax));
  TRY(ang.ensure(sizeof(double) * B));
  cudaMemcpyAsync(ang.p, angles, sizeof(double) * B, cudaMemcpyHostToDevice, c->s);
  int status = WCS_OK;
  wcs_solve_info acc{};
  for (int64_t c0 = 0; c0 < B; c0 += chunk) {
    const int64_t cc = std::min(chunk, B - c0);
    TRY(planewave_rhs(c->near, c->quad.wn, c->quad.xn, c->opt.q_near, N, c->h, c->k, ang.d() + c0,
                      (int)cc, eb.z(), hb.z(), N, c->s, c->mixed));
    TRY(precondition(c, eb.z(), hb.z(), N, bb.z(), N, cc, c->mixed ? PREC_PERIODIC : PREC_ACCURATE));
    int r = solve_block(c, bb.z(), N, (zd*)j + c0 * ldj, ldj, cc, &acc, eb.z(), hb.z(), N);
    if (r == WCS_ERR_NOT_CONVERGED) status = r;
    else if (r) return r;
  }
  if (info) *info = acc;
  if (status) set_error("iterative refinement did not reach refine_tol");
  return status;
}

int wcs_solve_planewaves_host(wcs_ctx* c, int64_t B, const double* angles, double* j_host,
                              int64_t ldj, wcs_solve_info* info) {
  if (!c || (B > 0 && (!angles || !j_host)) || ldj < (c ? c->N : 0)) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (B == 0) return WCS_OK;
  DevBuf& jd = c->sol_j;
  TRY(jd.ensure(sizeof(zd) * c->N * B));
  int r = wcs_solve_planewaves(c, B, angles, jd.d(), c->N, info);
  if (r && r != WCS_ERR_NOT_CONVERGED) return r;
  cudaMemcpy2DAsync(j_host, sizeof(zd) * ldj, jd.p, sizeof(zd) * c->N, sizeof(zd) * c->N, B,
                    cudaMemcpyDeviceToHost, c->s);
  int r2 = sync(c);
  return r2 ? r2 : r;
}

int wcs_farfield(wcs_ctx* c, int64_t B, const double* j, int64_t ldj, int nphi, const double* phi,
                 double* F, int64_t ldf) {
  if (!c || nphi < 0 || (nphi > 0 && (!phi || !F)) || ldf < nphi) { set_error("bad argument"); return WCS_ERR_ARG; }
  if (c->stage < ST_MESH) { set_error("mesh first"); return WCS_ERR_STATE; }
  TRY(check_block(c, B, j, ldj));
  if (B == 0 || nphi == 0) return WCS_OK;
  TRY(check_angles(nphi, phi, "farfield"));
  DevBuf E, ang;
  TRY(E.ensure(sizeof(zd) * (int64_t)nphi * c->N));
  TRY(ang.ensure(sizeof(double) * nphi));
  cudaMemcpyAsync(ang.p, phi, sizeof(double) * nphi, cudaMemcpyHostToDevice, c->s);
  TRY(farfield_matrix(c->near, c->quad.wn, c->quad.xn, c->opt.q_near, c->N, c->h, c->k, ang.d(),
                      nphi, E.z(), nphi, c->s));
  TRY(zgemm(nphi, B, c->N, mkz(1.0), ZView{E.z(), 1, nphi, false}, blk((const zd*)j, ldj), mkz(0.0),
            (zd*)F, ldf, c->s));
  int r = sync(c);
  E.release();
  ang.release();
  return r;
}

static int gemm_split_impl(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                           int64_t ldb, int planes, int accurate, double* D, int64_t ldd, void* stream);

int wcs_gemm_split_bf16(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                        int64_t ldb, int planes, double* D, int64_t ldd, void* stream) {
  return gemm_split_impl(M, Nc, K, A, lda, B, ldb, planes, 0, D, ldd, stream);
}

int wcs_gemm_split_bf16_ex(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                           int64_t ldb, int planes, int accurate, double* D, int64_t ldd, void* stream) {
  return gemm_split_impl(M, Nc, K, A, lda, B, ldb, planes, accurate, D, ldd, stream);
}

static int gemm_split_impl(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                           int64_t ldb, int planes, int accurate, double* D, int64_t ldd, void* stream) {
  if (accurate < 0 || (accurate && planes < 2)) { set_error("accurate contraction needs 2 or 3 planes"); return WCS_ERR_ARG; }
  if (M < 0 || Nc < 0 || K < 0 || planes < 1 || planes > 3 || (M > 0 && (lda < K || (K > 0 && !A))) ||
      (Nc > 0 && (ldb < K || (K > 0 && !B))) || (M > 0 && Nc > 0 && (!D || ldd < Nc))) {
    set_error("bad argument");
    return WCS_ERR_ARG;
  }
  if (M == 0 || Nc == 0) return WCS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0) {   // an empty contraction: D = 0
    cudaError_t e = cudaMemset2DAsync(D, sizeof(double) * ldd, 0, sizeof(double) * Nc, M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
    return WCS_OK;
  }
  const int64_t ldp = ((K + 63) / 64) * 64;
  DevBuf pa, pb, err, ws;
  TRY(pa.ensure(sizeof(uint16_t) * ldp * M * planes));
  TRY(pb.ensure(sizeof(uint16_t) * ldp * Nc * planes));
  TRY(err.ensure(sizeof(int)));
  int64_t ws_need = 0;
  if (!accurate) gemm_tc_split_plan((int)M, (int)Nc, (int)K, planes, planes, EPI_RAW_F64, &ws_need);
  if (ws_need > 0) TRY(ws.ensure(sizeof(float) * (size_t)ws_need));
  {
    cudaError_t e = cudaMemsetAsync(pa.p, 0, pa.bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pb.p, 0, pb.bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
    if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  }
  uint16_t* PA[3];
  uint16_t* PB[3];
  for (int p = 0; p < 3; ++p) {
    PA[p] = (uint16_t*)pa.p + (int64_t)p * ldp * M;
    PB[p] = (uint16_t*)pb.p + (int64_t)p * ldp * Nc;
  }
  TRY(split_real_f64(A, M, K, lda, planes, PA, ldp, s));
  TRY(split_real_f64(B, Nc, K, ldb, planes, PB, ldp, s));
  TcOperand oa, ob;
  oa.planes = ob.planes = planes;
  oa.ld = ob.ld = ldp;
  for (int p = 0; p < planes; ++p) { oa.plane[p] = PA[p]; ob.plane[p] = PB[p]; }
  TcArgs t;
  t.M = (int)M; t.Nc = (int)Nc; t.K = (int)K;
  tc_products(planes, t);
  t.epi = EPI_RAW_F64;
  t.out = D;
  t.ldo = ldd;
  t.err = (int*)err.p;
  t.ws = (float*)ws.p;
  t.ws_elems = (int64_t)(ws.bytes / sizeof(float));
  t.drain = accurate;
  TRY(accurate ? gemm_tc_accurate(oa, ob, t, s) : gemm_tc(oa, ob, t, s));
  int errh = 0;
  cudaMemcpyAsync(&errh, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  pa.release(); pb.release(); err.release(); ws.release();
  if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  if (errh) { set_error("tensor-core contraction: a bounded wait expired"); return WCS_ERR_TIMEOUT; }
  return WCS_OK;
}

int wcs_gemm_exact(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
                   double* D, int64_t ldd, void* stream) {
  if (M < 0 || Nc < 0 || K < 0 || (M > 0 && (lda < K || (K > 0 && !A))) || (Nc > 0 && (ldb < K || (K > 0 && !B))) ||
      (M > 0 && Nc > 0 && (!D || ldd < Nc)) || M > 65535 * 128 || Nc > 65535 * 256) {
    set_error("bad argument");
    return WCS_ERR_ARG;
  }
  if (M == 0 || Nc == 0) return WCS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0) {
    cudaError_t e = cudaMemset2DAsync(D, sizeof(double) * ldd, 0, sizeof(double) * Nc, M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
    return WCS_OK;
  }
  int64_t ld = 0, nch = 0;
  size_t sa = 0, ea = 0, sb = 0, eb = 0;
  exact_operand_alloc_bytes(M, K, &ld, &nch, &sa, &ea);
  exact_operand_alloc_bytes(Nc, K, &ld, &nch, &sb, &eb);
  const size_t sa2 = ((sa + 255) / 256) * 256, sb2 = ((sb + 255) / 256) * 256;
  DevBuf pa, pb, ea_b, eb_b, ws, err;
  TRY(pa.ensure(EX_SLICES * sa2));
  TRY(pb.ensure(EX_SLICES * sb2));
  TRY(ea_b.ensure(ea));
  TRY(eb_b.ensure(eb));
  const int64_t ws_elems = nch * Nc * M;
  TRY(ws.ensure(sizeof(float) * (size_t)ws_elems));
  TRY(err.ensure(sizeof(int)));
  ExactOperand oa, ob;
  oa.ld = ob.ld = ld;
  oa.nchunks = ob.nchunks = nch;
  for (int q = 0; q < EX_SLICES; ++q) {
    oa.slice[q] = (uint16_t*)((char*)pa.p + q * sa2);
    ob.slice[q] = (uint16_t*)((char*)pb.p + q * sb2);
  }
  oa.expo = (int16_t*)ea_b.p;
  ob.expo = (int16_t*)eb_b.p;
  cudaError_t e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  TRY(exact_slice_real(A, M, K, lda, oa, s));
  TRY(exact_slice_real(B, Nc, K, ldb, ob, s));
  TRY(exact_product_real(oa, (int)M, ob, (int)Nc, (int)K, D, ldd, (float*)ws.p, ws_elems, (int*)err.p, s));
  int errh = 0;
  e = cudaMemcpyAsync(&errh, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  if (errh) { set_error("tensor-core contraction: a bounded wait expired"); return WCS_ERR_TIMEOUT; }
  return WCS_OK;
}

uint64_t wcs_launch_count(void) { return (uint64_t)g_launches; }

int wcs_profile(wcs_ctx* c, int enable) {
  if (!c) { set_error("null context"); return WCS_ERR_ARG; }
  c->profile = enable != 0;
  return WCS_OK;
}

int wcs_profile_read(wcs_ctx* c, int reset, double* out_host) {
  if (!c || !out_host) { set_error("bad argument"); return WCS_ERR_ARG; }
  TRY(sync(c));
  for (int k = 0; k < 4 * CAT_COUNT; ++k) out_host[k] = 0.0;
  for (auto& r : c->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    out_host[4 * r.cat + 0] += 1.0;
    out_host[4 * r.cat + 1] += ms;
    out_host[4 * r.cat + 2] += r.flops;
    out_host[4 * r.cat + 3] += r.bytes;
  }
  if (reset) {
    for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    c->recs.clear();
  }
  return WCS_OK;
}

int wcs_quadrature_tables(int q, double* out) {
  if (q < 2 || q > 16 || !out) { set_error("bad argument"); return WCS_ERR_ARG; }
  QuadTables t;
  t.q_near = q;
  t.q_far = q;
  build_quad_tables(t);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < q * q; ++i) out[k * q * q + i] = t.wlog[k][i];
  return WCS_OK;
}

}  // extern "C"
