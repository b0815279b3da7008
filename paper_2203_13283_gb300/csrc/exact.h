// Exact (fixed-point sliced) operator products for the refinement residual
// of the mixed form (exact.cu).
#pragma once
#include "internal.h"

namespace wcs {

constexpr int EX_SLICES = 6;      // 7-bit slices per value (43 bits below each chunk's scale)
constexpr int EX_CHUNK = 1024;    // K elements per scale chunk and per split of the contraction
constexpr int EX_LEVELS = 6;      // slice pairs (s, t) with s + t < EX_LEVELS are formed

// A K-major real operand (rows x K, leading dimension ld) as EX_SLICES bf16
// planes of integers plus a power-of-two exponent per (row, chunk); for a
// right-hand block the exponent is stored once per complex column (rows 2j
// and 2j + 1 of the real view share it).
struct ExactOperand {
  uint16_t* slice[EX_SLICES] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t ld = 0;
  int16_t* expo = nullptr;
  int64_t nchunks = 0;
};

// Leading dimension, chunk count and bytes of one slice plane and of the
// exponent table for `rows` rows of K values.
int exact_operand_alloc_bytes(int64_t rows, int64_t K, int64_t* ld, int64_t* nchunks, size_t* slice_bytes,
                              size_t* expo_bytes);
// Slices of an operator held as split-bf16 planes (row-major, ld_planes).
int exact_slice_planes(const uint16_t* const* planes, int nplanes, int64_t rows, int64_t K, int64_t ld_planes,
                       const ExactOperand& out, cudaStream_t s);
// Slices of a right-hand block X (n x cols complex, column-major ldx) in the
// real K-major layout of the complex product (see stage_rhs).
int exact_slice_rhs(const zd* X, int64_t n, int64_t cols, int64_t ldx, int conj_in, const ExactOperand& out,
                    cudaStream_t s);
// out = beta * out + alpha * (A x) for the ncols complex columns of B, exact
// up to the FP64 sums of the scaled integer partials.  ws: FP32 workspace of
// nchunks * 2 ncols * M values.
int exact_product(const ExactOperand& A, int M, const ExactOperand& B, int ncols, int K, zd alpha, zd beta,
                  int conj_out, zd* out, int64_t ldo, float* ws, int64_t ws_elems, int* err, cudaStream_t s);

// Real rows (rows x K, row-major FP64, ld) as slices; and the exact real
// product D (M x Nc, row-major FP64, ldd) = A B^T (ws: nchunks * Nc * M floats).
int exact_slice_real(const double* X, int64_t rows, int64_t K, int64_t ld, const ExactOperand& out, cudaStream_t s);
int exact_product_real(const ExactOperand& A, int M, const ExactOperand& B, int Nc, int K, double* D, int64_t ldd,
                       float* ws, int64_t ws_elems, int* err, cudaStream_t s);

}  // namespace wcs
