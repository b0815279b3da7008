// Tensor-core (tcgen05) contraction used by the mixed-precision form.
#pragma once
#include <cstring>

#include "internal.h"

namespace wcs {

// bf16 planes of one operand (split-bf16: value = sum of planes), each a
// row-major matrix with K contiguous and leading dimension ld (elements).
struct TcOperand {
  const void* plane[3] = {nullptr, nullptr, nullptr};
  int planes = 0;
  int64_t ld = 0;
};

enum TcEpilogue {
  EPI_RAW_F64 = 0,       // out (double, row-major M x Nc, ldo) = alpha.x * D + beta.x * out
  EPI_CPLX_F64 = 1,      // complex column-major: out[j*ldo + i] (zd) = alpha * (D[i,2j], D[i,2j+1]) + beta * out
  EPI_CPLX_F32 = 2,      // same with zf output
};

struct TcArgs {
  int M = 0, Nc = 0, K = 0;
  int nprod = 0;
  int ia[6] = {0, 0, 0, 0, 0, 0}, ib[6] = {0, 0, 0, 0, 0, 0};
  int epi = EPI_RAW_F64;
  int conj_out = 0;      // complex epilogues: negate the imaginary part of the product first
  void* out = nullptr;
  int64_t ldo = 0;
  zd alpha = {1.0, 0.0}, beta = {0.0, 0.0};
  int* err = nullptr;    // device flag set to 1 when a bounded wait expires
  // optional FP32 workspace for split-K (complex epilogue only); gemm_tc
  // splits K when the output tiles cannot fill the GPU and ws_elems allows
  float* ws = nullptr;
  int64_t ws_elems = 0;
  int kper = 0;          // set by gemm_tc: k-blocks per split (0: no split)
  // exact products: split K into chunks of force_kper k-blocks whatever the
  // shape (ws must hold splits * Nc * M floats), and leave the FP32 partials
  // in ws for the caller's own reduction (no epilogue, no reduce)
  int force_kper = 0;
  int no_reduce = 0;
  // gemm_tc_accurate: K = 16 steps accumulated in tensor memory before each
  // drain into FP32 registers (1: every step, error ~1e-7; 4: once per K = 64
  // stage, products issued smallest first across it, error ~1e-7; 64: error
  // ~1e-5 at close to the speed of gemm_tc)
  int drain = 1;
};

#define TRY_TC(x)          \
  do {                     \
    int _r = (x);          \
    if (_r) return _r;     \
  } while (0)

// float -> double from the bits (exact), off GB300's FP64 pipe; zeros, FP32
// denormals, infinities and NaN take the hardware conversion
__device__ __forceinline__ double epi_f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;
  const unsigned m = u & 0x7fffffu;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3)), (int)((m & 7u) << 29));
}

__device__ __forceinline__ void epilogue_store(const TcArgs& a, int row, int col0, const float (&v)[32]) {
  if (row >= a.M) return;
  if (a.epi == EPI_CPLX_F64 && a.alpha.y == 0.0 && (a.alpha.x == 1.0 || a.alpha.x == -1.0) && a.beta.y == 0.0 &&
      (a.beta.x == 0.0 || a.beta.x == 1.0)) {
    // alpha = +-1, beta = 0 or 1 (the operator products of the solver): the
    // same values as the general complex arithmetic below (up to the sign of
    // a zero) with two exact conversions and at most two FP64 additions per
    // entry instead of ~10 FP64 operations, which on GB300's FP64 pipe cost
    // each tile's epilogue tens of microseconds
    const float sr = (a.alpha.x < 0.0) ? -1.f : 1.f, si = a.conj_out ? -sr : sr;
    const bool add = (a.beta.x == 1.0);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int j = (col0 >> 1) + c;
      if (2 * j >= a.Nc) break;
      zd p = mkz(epi_f32_to_f64(sr * v[2 * c]), epi_f32_to_f64(si * v[2 * c + 1]));
      zd* o = (zd*)a.out + (int64_t)j * a.ldo + row;
      if (add) {
        const zd q = *o;
        p.x += q.x;
        p.y += q.y;
      }
      *o = p;
    }
    return;
  }
  if (a.epi == EPI_RAW_F64) {
    double* o = (double*)a.out + (int64_t)row * a.ldo;
    const bool b0 = (a.beta.x == 0.0);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int c = col0 + i;
      if (c < a.Nc) o[c] = a.alpha.x * (double)v[i] + (b0 ? 0.0 : a.beta.x * o[c]);
    }
    return;
  }
  const bool b0 = (a.beta.x == 0.0 && a.beta.y == 0.0);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int j = (col0 >> 1) + c;
    if (2 * j >= a.Nc) break;
    zd p = mkz((double)v[2 * c], a.conj_out ? -(double)v[2 * c + 1] : (double)v[2 * c + 1]);
    p = a.alpha * p;
    if (a.epi == EPI_CPLX_F64) {
      zd* o = (zd*)a.out + (int64_t)j * a.ldo + row;
      if (!b0) p += a.beta * (*o);
      *o = p;
    } else {
      zf* o = (zf*)a.out + (int64_t)j * a.ldo + row;
      if (!b0) { zf q = *o; p += a.beta * mkz(q.x, q.y); }
      zf r; r.x = (float)p.x; r.y = (float)p.y;
      *o = r;
    }
  }
}

int gemm_tc(const TcOperand& A, const TcOperand& B, TcArgs args, cudaStream_t s);
// Split-K plan of gemm_tc for a shape: k-blocks per split (0: no split) and
// the FP32 workspace it needs.  gemm_tc splits exactly when args.ws is set
// and args.ws_elems >= that need, so two callers that provide the need get
// identical results.
int gemm_tc_split_plan(int M, int Nc, int K, int planesA, int planesB, int epi, int64_t* ws_elems);
// Same contraction with the accumulator drained into two-level FP32 register
// sums every args.drain K = 16 steps (accuracy ~1e-7 independent of K for
// drain 1, and for drain 4, where each K = 64 stage is one group issued
// product-major).
int gemm_tc_accurate(const TcOperand& A, const TcOperand& B, TcArgs args, cudaStream_t s);

// Product lists for 1, 2 or 3 planes per operand (terms of order <= planes-1),
// smallest first: the accumulator truncates each addition relative to its
// current magnitude, so the dominant hi*hi term is added last.
inline void tc_products(int planes, TcArgs& a) {
  if (planes == 1) { a.nprod = 1; a.ia[0] = 0; a.ib[0] = 0; return; }
  if (planes == 2) {
    const int ia[3] = {1, 0, 0}, ib[3] = {0, 1, 0};
    a.nprod = 3;
    for (int i = 0; i < 3; ++i) { a.ia[i] = ia[i]; a.ib[i] = ib[i]; }
    return;
  }
  const int ia[6] = {2, 1, 0, 1, 0, 0}, ib[6] = {0, 1, 2, 0, 1, 0};
  a.nprod = 6;
  for (int i = 0; i < 6; ++i) { a.ia[i] = ia[i]; a.ib[i] = ib[i]; }
}

// ---- split / staging kernels (mixed.cu)
// Split a real FP64 matrix (rows x cols, row-major, ld) into bf16 planes (ldp).
int split_real_f64(const double* X, int64_t rows, int64_t cols, int64_t ld, int planes, uint16_t* const* P,
                   int64_t ldp, cudaStream_t s);
// Complex matrix (rows x cols complex, row-major, ld complex) -> real rows x 2cols planes.
int split_complex_rows(const zd* X, int64_t rows, int64_t cols, int64_t ld, int planes, uint16_t* const* P,
                       int64_t ldp, cudaStream_t s);
// Right-hand block for the complex apply: X (n x B complex, column-major ldx)
// -> planes of B' (2B x 2n): row 2j = conj(x_j) interleaved, row 2j+1 =
// i conj(x_j) interleaved (with conj_in: use conj(x) in place of x).
int stage_rhs(const zd* X, int64_t n, int64_t B, int64_t ldx, int conj_in, int planes, uint16_t* const* P,
              int64_t ldp, cudaStream_t s);

// Stage a strided complex matrix view (element (i, j) at X[i*rs + j*cs],
// optionally conjugated) as real rows x 2cols bf16 planes (K-major A operand).
int stage_view(const zd* X, int64_t rows, int64_t cols, int64_t rs, int64_t cs, int conj, int planes,
               uint16_t* const* P, int64_t ldp, cudaStream_t s);

}  // namespace wcs
