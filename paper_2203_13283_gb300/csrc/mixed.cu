// Staging of FP64 data into split-bf16 planes for the tensor-core contraction
// (split.cuh: x = p0 + p1 (+ p2), each plane the exact remainder rounded to
// nearest, formed with integer operations so that staging runs at memory
// speed rather than at GB300's FP64 rate).
#include "gemm_tc.h"
#include "split.cuh"

namespace wcs {

__global__ void k_split_real(const double* X, int64_t rows, int64_t cols, int64_t ld, int planes,
                             uint16_t* p0, uint16_t* p1, uint16_t* p2, int64_t ldp) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = blockIdx.y;
  if (c >= cols) return;
  const int64_t o = r * ldp + c;
  uint16_t d1, d2;
  split3_bits(X[r * ld + c], planes, p0 + o, planes > 1 ? p1 + o : &d1, planes > 2 ? p2 + o : &d2);
}

int split_real_f64(const double* X, int64_t rows, int64_t cols, int64_t ld, int planes, uint16_t* const* P,
                   int64_t ldp, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
    const int64_t rr = std::min<int64_t>(65535, rows - r0);
    dim3 g((unsigned)((cols + 255) / 256), (unsigned)rr);
    k_split_real<<<g, 256, 0, s>>>(X + r0 * ld, rr, cols, ld, planes, P[0] + r0 * ldp,
                                   planes > 1 ? P[1] + r0 * ldp : nullptr, planes > 2 ? P[2] + r0 * ldp : nullptr, ldp);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("split: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

int split_complex_rows(const zd* X, int64_t rows, int64_t cols, int64_t ld, int planes, uint16_t* const* P,
                       int64_t ldp, cudaStream_t s) {
  return split_real_f64((const double*)X, rows, 2 * cols, 2 * ld, planes, P, ldp, s);
}

__global__ void k_stage_rhs(const zd* X, int64_t n, int64_t B, int64_t ldx, int conj_in, int planes,
                            uint16_t* p0, uint16_t* p1, uint16_t* p2, int64_t ldp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= n) return;
  zd x = X[j * ldx + i];
  if (conj_in) x.y = -x.y;
  // row 2j: (Re x, -Im x); row 2j+1: (Im x, Re x), each pair one 32-bit store
  // (ldp and 2 i are even)
  uint16_t re[3] = {0, 0, 0}, im[3] = {0, 0, 0}, nim[3] = {0, 0, 0};
  split3_bits(x.x, planes, &re[0], &re[1], &re[2]);
  split3_bits(x.y, planes, &im[0], &im[1], &im[2]);
  split3_bits(-x.y, planes, &nim[0], &nim[1], &nim[2]);
  uint16_t* P[3] = {p0, p1, p2};
  const int64_t o0 = (2 * j) * ldp + 2 * i, o1 = (2 * j + 1) * ldp + 2 * i;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t >= planes) break;
    *(uint32_t*)(P[t] + o0) = (uint32_t)re[t] | ((uint32_t)nim[t] << 16);
    *(uint32_t*)(P[t] + o1) = (uint32_t)im[t] | ((uint32_t)re[t] << 16);
  }
}

int stage_rhs(const zd* X, int64_t n, int64_t B, int64_t ldx, int conj_in, int planes, uint16_t* const* P,
              int64_t ldp, cudaStream_t s) {
  for (int64_t b0 = 0; b0 < B; b0 += 32768) {
    const int64_t bb = std::min<int64_t>(32768, B - b0);
    dim3 g((unsigned)((n + 255) / 256), (unsigned)bb);
    k_stage_rhs<<<g, 256, 0, s>>>(X + b0 * ldx, n, bb, ldx, conj_in, planes, P[0] + 2 * b0 * ldp,
                                  planes > 1 ? P[1] + 2 * b0 * ldp : nullptr,
                                  planes > 2 ? P[2] + 2 * b0 * ldp : nullptr, ldp);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("stage_rhs: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

__global__ void k_stage_view(const zd* X, int64_t rows, int64_t cols, int64_t rs, int64_t cs, int conj,
                             int planes, uint16_t* p0, uint16_t* p1, uint16_t* p2, int64_t ldp) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= cols) return;
  const zd x = X[i * rs + j * cs];
  // (Re x, Im x) adjacent: one 32-bit store per plane (ldp and 2 j are even)
  uint16_t re[3] = {0, 0, 0}, im[3] = {0, 0, 0};
  split3_bits(x.x, planes, &re[0], &re[1], &re[2]);
  split3_bits(conj ? -x.y : x.y, planes, &im[0], &im[1], &im[2]);
  uint16_t* P[3] = {p0, p1, p2};
  const int64_t o = i * ldp + 2 * j;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t >= planes) break;
    *(uint32_t*)(P[t] + o) = (uint32_t)re[t] | ((uint32_t)im[t] << 16);
  }
}

int stage_view(const zd* X, int64_t rows, int64_t cols, int64_t rs, int64_t cs, int conj, int planes,
               uint16_t* const* P, int64_t ldp, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
    const int64_t rr = std::min<int64_t>(65535, rows - r0);
    dim3 g((unsigned)((cols + 255) / 256), (unsigned)rr);
    k_stage_view<<<g, 256, 0, s>>>(X + r0 * rs, rr, cols, rs, cs, conj, planes, P[0] + r0 * ldp,
                                   planes > 1 ? P[1] + r0 * ldp : nullptr, planes > 2 ? P[2] + r0 * ldp : nullptr,
                                   ldp);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("stage_view: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

}  // namespace wcs
