// Exact operator products for the refinement residual of the mixed form.
//
// Iterative refinement converges to the operator that its residual evaluates
// (Eq. 5 solved through Eq. 9 as an approximate inverse), and a split-bf16
// product accumulated in FP32 carries ~1e-7 relative error, so the residual
// b - C x of the mixed form stalls there.  This file evaluates the operator
// products of C (Eq. 6) without rounding error on the same tensor cores:
//
//  * every row of an operand is cut into chunks of EX_CHUNK consecutive K
//    elements; each chunk gets a power-of-two scale 2^E (its largest entry
//    below 2^E), and the scaled entries, all in (-1, 1), are written as
//    EX_SLICES fixed-point slices of 7 bits, y = sum_s y_s 2^-7(s+1) with
//    integers |y_0| <= 128 and |y_s| <= 64, each exact in bf16;
//  * a product of two slices is a sum of integer products (<= 2^14 each);
//    over one chunk of 1024 terms it stays below 2^24, where the tensor core's
//    FP32 accumulation is exact, so the contraction runs split-K with one
//    split per chunk and returns exact integer partial sums;
//  * the partials are scaled by 2^(E_A + E_B) and summed over the chunks in
//    float-float (an exact integer below 2^24 times a power of two is exact
//    in FP32, and TwoSum keeps ~48 bits of the running sum on the FP32 pipe,
//    which runs at 64 times the FP64 rate of this GPU); each pair's sum, times
//    2^-7(s+t+2), is added to the FP64 output.
//
// Pairs with s + t < EX_LEVELS are formed (21 of the 36); the dropped ones are
// below 2^-56 of the chunk scales.  The operator's slices describe its
// split-bf16 planes (the operator of the rest of the mixed form) to ~2^-42 of
// each chunk's largest entry.  With five slices the chunk that holds the
// log-singular diagonal left its ~500 far entries at ~2^-35 of the diagonal,
// a residual floor near 7e-10 at N = 32768; six put it below 1e-11.
#include <cuda_bf16.h>

#include "gemm_tc.h"
#include "exact.h"

namespace wcs {

__device__ __forceinline__ uint16_t int_bf16(double v) {
  return __bfloat16_as_ushort(__double2bfloat16(v));   // exact for integers |v| <= 256
}

constexpr int EX_PER = EX_CHUNK / 256;   // values per thread of a 256-thread block

// 2^e as a float for the normal range (e in [-126, 127]); scaled partials of
// the residual products stay far inside it (operator entries and currents
// between ~1e-12 and ~1e3, partial sums below 2^24)
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}

// (hi, lo) += v with TwoSum (Knuth): hi + lo carries the sum to ~2^-48
__device__ __forceinline__ void ff_acc(float2& a, float v) {
  const float s = a.x + v;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (v - bb);
  a.x = s;
  a.y += err;
}

// Exponent E of a chunk held by the block (EX_PER values per thread):
// max |v| < 2^E, or 0 for an all-zero chunk.  Written to *expo by thread 0.
__device__ __forceinline__ int chunk_exponent(const double (&m)[EX_PER], int16_t* expo) {
  __shared__ double red[8];
  __shared__ int eshared;
  double x = 0.0;
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) x = fmax(x, m[t]);
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < 8; ++w) mm = fmax(mm, red[w]);
    eshared = (mm > 0.0) ? ilogb(mm) + 1 : 0;   // mm < 2^E
    *expo = (int16_t)eshared;
  }
  __syncthreads();
  return eshared;
}

// The EX_SLICES fixed-point slices of v / 2^E at offset `off` of each slice plane.
__device__ __forceinline__ void write_slices(double v, int E, uint16_t* const* slice, int64_t off) {
  double r = ldexp(v, 7 - E);   // in (-128, 128); exact scaling
#pragma unroll
  for (int q = 0; q < EX_SLICES; ++q) {
    const double y = rint(r);
    slice[q][off] = int_bf16(y);
    r = (r - y) * 128.0;          // exact: r - y in [-1/2, 1/2], 7 more bits
  }
}

// Operator rows from their split-bf16 planes (row-major, ld elements, K
// valid columns): one block per (row, chunk).
__global__ void __launch_bounds__(256) k_slice_planes(const uint16_t* p0, const uint16_t* p1, const uint16_t* p2,
                                                      int planes, int64_t K, int64_t ld, ExactOperand out) {
  const int64_t row = blockIdx.y, c = blockIdx.x;
  double v[EX_PER], m[EX_PER];
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;
    const int64_t o = row * ld + k;
    double x = 0.0;
    if (k < K) {
      x = (double)__bfloat162float(__ushort_as_bfloat16(p0[o]));
      if (planes > 1) x += (double)__bfloat162float(__ushort_as_bfloat16(p1[o]));
      if (planes > 2) x += (double)__bfloat162float(__ushort_as_bfloat16(p2[o]));
    }
    v[t] = x;
    m[t] = fabs(x);
  }
  const int E = chunk_exponent(m, out.expo + row * out.nchunks + c);
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;
    if (k < out.ld) write_slices(v[t], E, out.slice, row * out.ld + k);
  }
}

// Right-hand block X (n x B complex, column-major ldx) as the real K-major
// operand B' (2B x 2n) of the complex product: row 2j = (Re x, -Im x)
// interleaved, row 2j+1 = (Im x, Re x) (x conjugated first when conj_in).
// Both rows hold the same magnitudes, so they share the chunk exponent,
// stored once per column j.  One block per (column, chunk) writes both rows.
__global__ void __launch_bounds__(256) k_slice_rhs(const zd* X, int64_t n, int64_t ldx, int conj_in,
                                                   ExactOperand out) {
  const int64_t j = blockIdx.y, c = blockIdx.x;
  double v[EX_PER], w[EX_PER], m[EX_PER];
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;   // real K index: node k / 2, part k % 2
    const int64_t i = k >> 1;
    double a = 0.0, b = 0.0;
    if (i < n) {
      zd x = X[j * ldx + i];
      if (conj_in) x.y = -x.y;
      a = (k & 1) ? -x.y : x.x;    // row 2j
      b = (k & 1) ? x.x : x.y;     // row 2j + 1
    }
    v[t] = a;
    w[t] = b;
    m[t] = fmax(fabs(a), fabs(b));
  }
  const int E = chunk_exponent(m, out.expo + j * out.nchunks + c);
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;
    if (k < out.ld) {
      write_slices(v[t], E, out.slice, (2 * j) * out.ld + k);
      write_slices(w[t], E, out.slice, (2 * j + 1) * out.ld + k);
    }
  }
}

// Real FP64 rows (row-major, ld): one block per (row, chunk).
__global__ void __launch_bounds__(256) k_slice_real(const double* X, int64_t K, int64_t ld, ExactOperand out) {
  const int64_t row = blockIdx.y, c = blockIdx.x;
  double v[EX_PER], m[EX_PER];
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;
    v[t] = (k < K) ? X[row * ld + k] : 0.0;
    m[t] = fabs(v[t]);
  }
  const int E = chunk_exponent(m, out.expo + row * out.nchunks + c);
#pragma unroll
  for (int t = 0; t < EX_PER; ++t) {
    const int64_t k = c * EX_CHUNK + t * 256 + threadIdx.x;
    if (k < out.ld) write_slices(v[t], E, out.slice, row * out.ld + k);
  }
}

// D (M x Nc, row-major ldd) op= weight * sum_c 2^(EA(i,c) + EB(j,c)) P[c][j][i].
__global__ void k_exact_reduce_real(const float* __restrict__ P, int splits, int M, int Nc, const int16_t* EA,
                                    const int16_t* EB, int64_t nchunks, double weight, int first, double* D,
                                    int64_t ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * Nc) return;
  const int i = (int)(t % M), j = (int)(t / M);
  const int64_t plane = (int64_t)Nc * M;
  float2 sum = make_float2(0.f, 0.f);
  for (int c = 0; c < splits; ++c) {
    const float sc = pow2f((int)EA[(int64_t)i * nchunks + c] + (int)EB[(int64_t)j * nchunks + c]);
    ff_acc(sum, P[c * plane + (int64_t)j * M + i] * sc);
  }
  const double acc = (double)sum.x + (double)sum.y;
  double* o = D + (int64_t)i * ldd + j;
  *o = first ? weight * acc : *o + weight * acc;
}

// out (complex, column-major ldo, M rows, ncols columns) op= alpha * weight *
// sum_c 2^(EA(i,c) + EB(j,c)) (P[c][2j][i] + i P[c][2j+1][i]); first: out =
// beta * out + ..., else out += ...  (conj_out: conjugate the product first).
__global__ void k_exact_reduce(const float* __restrict__ P, int splits, int M, int ncols, const int16_t* EA,
                               const int16_t* EB, int64_t nchunks, double weight, zd alpha, zd beta, int first,
                               int conj_out, zd* out, int64_t ldo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * ncols) return;
  const int i = (int)(t % M), j = (int)(t / M);
  const int64_t plane = (int64_t)2 * ncols * M;
  float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
  for (int c = 0; c < splits; ++c) {
    const float sc = pow2f((int)EA[(int64_t)i * nchunks + c] + (int)EB[(int64_t)j * nchunks + c]);
    ff_acc(re, P[c * plane + (int64_t)(2 * j) * M + i] * sc);
    ff_acc(im, P[c * plane + (int64_t)(2 * j + 1) * M + i] * sc);
  }
  const double dre = (double)re.x + (double)re.y, dim = (double)im.x + (double)im.y;
  zd p = mkz(weight * dre, weight * (conj_out ? -dim : dim));
  p = alpha * p;
  zd* o = out + (int64_t)j * ldo + i;
  if (first) {
    if (!(beta.x == 0.0 && beta.y == 0.0)) p += beta * (*o);
  } else {
    p += *o;
  }
  *o = p;
}

int exact_operand_alloc_bytes(int64_t rows, int64_t K, int64_t* ld, int64_t* nchunks, size_t* slice_bytes,
                              size_t* expo_bytes) {
  *ld = ((K + 63) / 64) * 64;
  *nchunks = (K + EX_CHUNK - 1) / EX_CHUNK;
  *slice_bytes = sizeof(uint16_t) * (size_t)rows * (size_t)(*ld);
  *expo_bytes = sizeof(int16_t) * (size_t)rows * (size_t)(*nchunks);
  return 0;
}

int exact_slice_planes(const uint16_t* const* planes, int nplanes, int64_t rows, int64_t K, int64_t ld_planes,
                       const ExactOperand& out, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
    const int64_t rr = std::min<int64_t>(65535, rows - r0);
    ExactOperand o = out;
    for (int q = 0; q < EX_SLICES; ++q) o.slice[q] = out.slice[q] + r0 * out.ld;
    o.expo = out.expo + r0 * out.nchunks;
    dim3 g((unsigned)out.nchunks, (unsigned)rr);
    k_slice_planes<<<g, 256, 0, s>>>(planes[0] + r0 * ld_planes, nplanes > 1 ? planes[1] + r0 * ld_planes : nullptr,
                                     nplanes > 2 ? planes[2] + r0 * ld_planes : nullptr, nplanes, K, ld_planes, o);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("exact slices: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

int exact_slice_rhs(const zd* X, int64_t n, int64_t cols, int64_t ldx, int conj_in, const ExactOperand& out,
                    cudaStream_t s) {
  for (int64_t j0 = 0; j0 < cols; j0 += 32768) {
    const int64_t jj = std::min<int64_t>(32768, cols - j0);
    ExactOperand o = out;
    for (int q = 0; q < EX_SLICES; ++q) o.slice[q] = out.slice[q] + 2 * j0 * out.ld;
    o.expo = out.expo + j0 * out.nchunks;
    dim3 g((unsigned)out.nchunks, (unsigned)jj);
    k_slice_rhs<<<g, 256, 0, s>>>(X + j0 * ldx, n, ldx, conj_in, o);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("exact rhs slices: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

int exact_product(const ExactOperand& A, int M, const ExactOperand& B, int ncols, int K, zd alpha, zd beta,
                  int conj_out, zd* out, int64_t ldo, float* ws, int64_t ws_elems, int* err, cudaStream_t s) {
  if (M <= 0 || ncols <= 0) return 0;
  const int kper = EX_CHUNK / 64;   // k-blocks of the tensor-core kernel per chunk
  bool first = true;
  // largest levels first, the dominant pair last
  for (int lev = EX_LEVELS - 1; lev >= 0; --lev) {
    for (int sa = 0; sa <= lev; ++sa) {
      const int sb = lev - sa;
      if (sa >= EX_SLICES || sb >= EX_SLICES) continue;
      TcOperand oa, ob;
      oa.planes = ob.planes = 1;
      oa.ld = A.ld;
      ob.ld = B.ld;
      oa.plane[0] = A.slice[sa];
      ob.plane[0] = B.slice[sb];
      TcArgs t;
      t.M = M;
      t.Nc = 2 * ncols;
      t.K = K;
      tc_products(1, t);
      t.epi = EPI_CPLX_F64;
      t.err = err;
      t.ws = ws;
      t.ws_elems = ws_elems;
      t.force_kper = kper;
      t.no_reduce = 1;
      TRY_TC(gemm_tc(oa, ob, t, s));
      const int splits = (int)A.nchunks;
      const int64_t n = (int64_t)M * ncols;
      k_exact_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ws, splits, M, ncols, A.expo, B.expo, A.nchunks,
                                                                 ldexp(1.0, -7 * (lev + 2)), alpha, beta,
                                                                 first ? 1 : 0, conj_out, out, ldo);
      note_launch();
      first = false;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("exact product: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

}  // namespace wcs

namespace wcs {

int exact_slice_real(const double* X, int64_t rows, int64_t K, int64_t ld, const ExactOperand& out, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
    const int64_t rr = std::min<int64_t>(65535, rows - r0);
    ExactOperand o = out;
    for (int q = 0; q < EX_SLICES; ++q) o.slice[q] = out.slice[q] + r0 * out.ld;
    o.expo = out.expo + r0 * out.nchunks;
    dim3 g((unsigned)out.nchunks, (unsigned)rr);
    k_slice_real<<<g, 256, 0, s>>>(X + r0 * ld, K, ld, o);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("exact slices: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

int exact_product_real(const ExactOperand& A, int M, const ExactOperand& B, int Nc, int K, double* D, int64_t ldd,
                       float* ws, int64_t ws_elems, int* err, cudaStream_t s) {
  if (M <= 0 || Nc <= 0) return 0;
  bool first = true;
  for (int lev = EX_LEVELS - 1; lev >= 0; --lev) {
    for (int sa = 0; sa <= lev; ++sa) {
      const int sb = lev - sa;
      if (sa >= EX_SLICES || sb >= EX_SLICES) continue;
      TcOperand oa, ob;
      oa.planes = ob.planes = 1;
      oa.ld = A.ld;
      ob.ld = B.ld;
      oa.plane[0] = A.slice[sa];
      ob.plane[0] = B.slice[sb];
      TcArgs t;
      t.M = M;
      t.Nc = Nc;
      t.K = K;
      tc_products(1, t);
      t.epi = EPI_RAW_F64;
      t.err = err;
      t.ws = ws;
      t.ws_elems = ws_elems;
      t.force_kper = EX_CHUNK / 64;
      t.no_reduce = 1;
      TRY_TC(gemm_tc(oa, ob, t, s));
      const int64_t n = (int64_t)M * Nc;
      k_exact_reduce_real<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ws, (int)A.nchunks, M, Nc, A.expo, B.expo,
                                                                      A.nchunks, ldexp(1.0, -7 * (lev + 2)),
                                                                      first ? 1 : 0, D, ldd);
      note_launch();
      first = false;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("exact product: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

}  // namespace wcs
