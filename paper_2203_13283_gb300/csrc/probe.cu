// Issue-rate probes of the FMA pipes (FP64 and FP32), for the rooflines of
// the point-pair integration kernels: the measured-peaks file of the machine
// holds copy bandwidth and tensor-core throughput only.
//
// Each thread runs `chains` independent FMA chains (enough to hide the pipe
// latency) for `iters` rounds; the result is stored so nothing is elided.
// The grid fills every SM several times over.  Timed with CUDA events on the
// given stream; flops are counted as 2 per FMA.
#include "../../include/wcs.h"
#include "internal.h"

namespace wcs {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_stream(T* out, int iters, T a, T b) {
  constexpr int CH = 8;
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int fma_rate(int iters, cudaStream_t s, double* flops_per_s) {
  int dev = 0, sms = 0;
  WCS_CUDA_TRY(cudaGetDevice(&dev));
  WCS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  WCS_CUDA_TRY(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a, b keep the chains bounded (|x| converges to b / (1 - a))
  k_fma_stream<T><<<blocks, threads, 0, s>>>(out, 16, (T)0.999, (T)0.001);   // warm-up
  note_launch();
  cudaEventRecord(e0, s);
  k_fma_stream<T><<<blocks, threads, 0, s>>>(out, iters, (T)0.999, (T)0.001);
  note_launch();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) { set_error(std::string("fma probe: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (1e-3 * (double)ms);
  return WCS_OK;
}

}  // namespace wcs

using namespace wcs;

extern "C" int wcs_fma_rate(int precision, int iters, void* stream, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || (precision != 32 && precision != 64)) {
    set_error("wcs_fma_rate: precision 32 or 64, iters >= 1, output pointer");
    return WCS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return precision == 64 ? fma_rate<double>(iters, s, flops_per_s) : fma_rate<float>(iters, s, flops_per_s);
}
