// Allocation-free variant of the split-bf16 tensor-core contraction
// (wcs_gemm_split_bf16_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is
// frozen for real-time work, plug-ins whose host application owns every
// device allocation, or processes that must not allocate between two
// synchronisation points.  For them this entry point keeps its staging
// buffers (the bf16 planes of both operands and the error flag) in one
// file-scope device array of fixed size, so a call allocates nothing: the
// caller passes inputs and the output, and the library passes the array to
// its kernels.  Every GPU that loads the library holds the array until the
// process exits.
#include "../../include/wcs.h"
#include "gemm_tc.h"

namespace wcs {

// Capacity of the shared scratch array: 32 MiB.
constexpr size_t kNoAllocBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device (host code cannot use the
// symbol itself: in host code it names a host-side shadow, not device memory).
static void* g_noalloc_addr[64] = {nullptr};

static int noalloc_setup(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  if (dev < 0 || dev >= 64) { set_error("device index out of range"); return WCS_ERR_ARG; }
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return WCS_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return WCS_OK;
}

}  // namespace wcs

using namespace wcs;

extern "C" int wcs_gemm_split_bf16_noalloc(int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda,
                                           const double* B, int64_t ldb, int planes, double* D, int64_t ldd,
                                           void* stream) {
  if (M < 0 || Nc < 0 || K < 0 || planes < 1 || planes > 3 || (M > 0 && (lda < K || (K > 0 && !A))) ||
      (Nc > 0 && (ldb < K || (K > 0 && !B))) || (M > 0 && Nc > 0 && (!D || ldd < Nc))) {
    set_error("bad argument");
    return WCS_ERR_ARG;
  }
  if (M == 0 || Nc == 0) return WCS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (K == 0) {   // an empty contraction: D = 0
    e = cudaMemset2DAsync(D, sizeof(double) * ldd, 0, sizeof(double) * Nc, M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
    return WCS_OK;
  }
  const int64_t ldp = ((K + 63) / 64) * 64;
  const size_t bytesA = sizeof(uint16_t) * (size_t)ldp * M * planes;
  const size_t bytesB = sizeof(uint16_t) * (size_t)ldp * Nc * planes;
  // the same split-K plan as the allocating entry point (identical results)
  int64_t ws_elems = 0;
  gemm_tc_split_plan((int)M, (int)Nc, (int)K, planes, planes, EPI_RAW_F64, &ws_elems);
  const size_t bytesW = sizeof(float) * (size_t)ws_elems;
  const size_t offB = ((bytesA + 255) / 256) * 256, offE = offB + ((bytesB + 255) / 256) * 256;
  const size_t offW = offE + 256;
  const size_t need = offW + bytesW;
  if (need > kNoAllocBytes) {
    set_error("wcs_gemm_split_bf16_noalloc: (M + Nc) * ceil64(K) * planes * 2 bytes plus the split-K "
              "partials exceed the 32 MiB scratch; use wcs_gemm_split_bf16");
    return WCS_ERR_ARG;
  }
  void* base = nullptr;
  int r = noalloc_setup(&base);
  if (r) return r;
  unsigned char* p = (unsigned char*)base;
  uint16_t* pa = (uint16_t*)p;
  uint16_t* pb = (uint16_t*)(p + offB);
  int* err = (int*)(p + offE);
  float* ws = (float*)(p + offW);
  // the array keeps the previous call's contents: clear the planes (their
  // K padding must read as zero) and the error flag
  e = cudaMemsetAsync(pa, 0, bytesA, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pb, 0, bytesB, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) { set_error(std::string("gemm: clearing the scratch: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  uint16_t* PA[3];
  uint16_t* PB[3];
  for (int q = 0; q < 3; ++q) {
    PA[q] = pa + (int64_t)q * ldp * M;
    PB[q] = pb + (int64_t)q * ldp * Nc;
  }
  if ((r = split_real_f64(A, M, K, lda, planes, PA, ldp, s))) return r;
  if ((r = split_real_f64(B, Nc, K, ldb, planes, PB, ldp, s))) return r;
  TcOperand oa, ob;
  oa.planes = ob.planes = planes;
  oa.ld = ob.ld = ldp;
  for (int q = 0; q < planes; ++q) { oa.plane[q] = PA[q]; ob.plane[q] = PB[q]; }
  TcArgs t;
  t.M = (int)M; t.Nc = (int)Nc; t.K = (int)K;
  tc_products(planes, t);
  t.epi = EPI_RAW_F64;
  t.out = D;
  t.ldo = ldd;
  t.err = err;
  if (ws_elems > 0) { t.ws = ws; t.ws_elems = ws_elems; }
  if ((r = gemm_tc(oa, ob, t, s))) return r;
  int errh = 0;
  e = cudaMemcpyAsync(&errh, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { set_error(std::string("gemm: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  if (errh) { set_error("tensor-core contraction: a bounded wait expired"); return WCS_ERR_TIMEOUT; }
  return WCS_OK;
}
