// Batched complex FP64 FFT along columns, for the circulant algebra on the
// equivalent circle (Sec. V: every operation on gamma_c is done by FFT).
//
// Power-of-two lengths n <= 4096: one pass, each CTA transforms whole columns
// in shared memory (bit-reversed load, in-place radix-2 butterflies).
// Longer power-of-two lengths: four-step (n = n1 n2): length-n2 transforms of
// the n1 interleaved subsequences (with the twiddles W_n^{j1 k2} applied on
// the way out to a scratch buffer), then length-n1 transforms writing the
// natural order back.  Each CTA handles several adjacent subsequences so
// global accesses come in contiguous runs.
// Other lengths: Bluestein's chirp-z convolution with a power-of-two FFT.
#include <vector>

#include "internal.h"

namespace wcs {

constexpr int FFT_SMEM_MAX = 4096;  // complex doubles held in shared memory per CTA

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// Transform `nseq` sequences of length L (power of two) held by one CTA.
// Element t of sequence s (global index sg = blockIdx.x * nseq + s) in column c:
//   in [c * in_cs + sg * in_ss + t * in_es]  ->  out [c * out_cs + sg * out_ss + t * out_es]
// tw: table of e^{-2 pi i j / Ltw} (j < Ltw), Ltw a multiple of L.
// post (optional): multiply output (t, sg) by W_{npost}^{sg * t} from table twn (length npost).
__global__ void k_fft_tile(const zd* __restrict__ in, int64_t in_es, int64_t in_ss, int64_t in_cs,
                           zd* __restrict__ out, int64_t out_es, int64_t out_ss, int64_t out_cs,
                           int L, int logL, int nseq, int64_t nseq_total, const zd* __restrict__ tw,
                           int64_t Ltw, int sign, const zd* __restrict__ twn, int64_t npost) {
  extern __shared__ zd buf[];  // [nseq][L]
  const int64_t c = blockIdx.y;
  const int64_t s0 = (int64_t)blockIdx.x * nseq;
  const int total = nseq * L;
  // load: consecutive threads walk the sequence index first (adjacent in memory
  // when in_ss == 1), then the element index
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    int s, t;
    if (in_ss == 1) { s = u % nseq; t = u / nseq; } else { t = u % L; s = u / L; }
    int64_t sg = s0 + s;
    zd v = mkz(0.0);
    if (sg < nseq_total) v = in[c * in_cs + sg * in_ss + (int64_t)t * in_es];
    buf[s * L + bitrev((unsigned)t, logL)] = v;
  }
  __syncthreads();
  const int64_t tstride = Ltw / L;
  for (int m = 1; m < L; m <<= 1) {
    // butterflies of span 2m; twiddle W_{2m}^j = W_L^{j L/(2m)}
    const int half = total >> 1;
    for (int u = threadIdx.x; u < half; u += blockDim.x) {
      const int s = u / (L >> 1);
      const int b = u - s * (L >> 1);
      const int grp = b / m, j = b - grp * m;
      const int i0 = s * L + grp * 2 * m + j;
      const int i1 = i0 + m;
      zd w = tw[(int64_t)j * (L / (2 * m)) * tstride];
      if (sign > 0) w.y = -w.y;
      zd x1 = buf[i1] * w;
      zd x0 = buf[i0];
      buf[i0] = x0 + x1;
      buf[i1] = x0 - x1;
    }
    __syncthreads();
  }
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    int s, t;
    if (out_ss == 1) { s = u % nseq; t = u / nseq; } else { t = u % L; s = u / L; }
    int64_t sg = s0 + s;
    if (sg >= nseq_total) continue;
    zd v = buf[s * L + t];
    if (twn) {
      zd w = twn[(sg * (int64_t)t) % npost];
      if (sign > 0) w.y = -w.y;
      v = v * w;
    }
    out[c * out_cs + sg * out_ss + (int64_t)t * out_es] = v;
  }
}

__global__ void k_twiddles(zd* tw, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)n, &s, &c);
  tw[j] = mkz(c, s);
}

// Bluestein chirp c_j = exp(-i pi j^2 / n), j^2 reduced mod 2n exactly
__global__ void k_chirp(zd* chirp, int64_t n) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t q = (int64_t)(((unsigned __int128)j * (unsigned __int128)j) % (unsigned __int128)(2 * n));
  double s, c;
  sincospi(-(double)q / (double)n, &s, &c);
  chirp[j] = mkz(c, s);
}

// filter b_j = conj(c_j) for j < n and b_{m-j} = conj(c_j) for 1 <= j < n
__global__ void k_bluestein_filter(const zd* chirp, int64_t n, int64_t m, zd* b) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  zd v = mkz(0.0);
  if (j < n) v = conj(chirp[j]);
  else if (m - j < n) v = conj(chirp[m - j]);
  b[j] = v;
}

// work[:, c] = x[:, c] * chirp, zero padded to m.  The inverse transform is
// taken as conj(DFT(conj(x))), so for sign > 0 the input is conjugated here
// and the output in k_bluestein_post.
__global__ void k_bluestein_pre(const zd* x, int64_t ld, int64_t n, int64_t m, const zd* chirp,
                                int sign, zd* work) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = blockIdx.y;
  if (j >= m) return;
  zd v = mkz(0.0);
  if (j < n) {
    zd xv = x[c * ld + j];
    if (sign > 0) xv.y = -xv.y;
    v = xv * chirp[j];
  }
  work[c * m + j] = v;
}

__global__ void k_pointwise(zd* work, int64_t m, const zd* bhat, int conj_b) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = blockIdx.y;
  if (j >= m) return;
  zd b = bhat[j];
  if (conj_b) b.y = -b.y;
  work[c * m + j] = work[c * m + j] * b;
}

__global__ void k_bluestein_post(const zd* work, int64_t n, int64_t m, const zd* chirp, int sign,
                                 zd* x, int64_t ld) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = blockIdx.y;
  if (j >= n) return;
  zd v = (1.0 / (double)m) * (work[c * m + j] * chirp[j]);
  if (sign > 0) v.y = -v.y;
  x[c * ld + j] = v;
}

__global__ void k_scale_columns(zd* x, int64_t n, int64_t ld, const zd* mu, int divide,
                                int conj_mu, double extra) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = blockIdx.y;
  if (j >= n) return;
  zd m = mu[j];
  if (conj_mu) m.y = -m.y;
  zd v = x[c * ld + j];
  v = divide ? zdiv(v, m) : v * m;
  x[c * ld + j] = extra * v;
}

static int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t)1 << l < n) ++l;
  return l;
}

// ---- power-of-two transform of `cols` columns (ld), in place, using scratch when n > 4096
struct Pow2 {
  int64_t n;
  zd* tw = nullptr;       // e^{-2 pi i j / n}, j < n
  zd* scratch = nullptr;  // n * scratch_cols
  int64_t scratch_cols = 0;
};

static int launch_tile(const zd* in, int64_t in_es, int64_t in_ss, int64_t in_cs, zd* out,
                       int64_t out_es, int64_t out_ss, int64_t out_cs, int64_t L, int64_t nseq_total,
                       int64_t cols, const zd* tw, int64_t Ltw, int sign, const zd* twn,
                       int64_t npost, cudaStream_t s) {
  int nseq = (int)std::max<int64_t>(1, std::min<int64_t>(nseq_total, FFT_SMEM_MAX / L));
  if (nseq > 16) nseq = 16;
  if (in_ss != 1 && out_ss != 1) nseq = 1;
  size_t smem = sizeof(zd) * nseq * L;
  static DeviceOnce attr;
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(zd) * FFT_SMEM_MAX));
    if (e != cudaSuccess) { set_error(std::string("fft: shared-memory opt-in: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  int threads = (int)std::min<int64_t>(512, std::max<int64_t>(32, nseq * L / 2));
  for (int64_t c0 = 0; c0 < cols; c0 += 65535) {
    int64_t cc = std::min<int64_t>(65535, cols - c0);
    dim3 grid((unsigned)((nseq_total + nseq - 1) / nseq), (unsigned)cc);
    k_fft_tile<<<grid, threads, smem, s>>>(in + c0 * in_cs, in_es, in_ss, in_cs, out + c0 * out_cs,
                                           out_es, out_ss, out_cs, (int)L, ilog2(L), nseq,
                                           nseq_total, tw, Ltw, sign, twn, npost);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("fft: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

static int pow2_transform(Pow2& P, zd* x, int64_t ld, int64_t cols, int sign, cudaStream_t s) {
  const int64_t n = P.n;
  if (n <= FFT_SMEM_MAX) {
    return launch_tile(x, 1, ld, ld, x, 1, ld, ld, n, 1, cols, P.tw, n, sign, nullptr, 0, s);
  }
  // four-step: n = n1 * n2, j = j1 + n1 j2, k = k2 + n2 k1
  int lg = ilog2(n);
  int64_t n2 = (int64_t)1 << (lg / 2);
  int64_t n1 = n / n2;
  if (n1 > FFT_SMEM_MAX || n2 > FFT_SMEM_MAX) { set_error("fft length too large"); return 1; }
  for (int64_t c0 = 0; c0 < cols; c0 += P.scratch_cols) {
    int64_t cc = std::min(P.scratch_cols, cols - c0);
    zd* xc = x + c0 * ld;
    // step 1: sequences j1 (stride 1), elements j2 (stride n1): length n2 -> scratch[j1 n2 + k2]
    int r = launch_tile(xc, n1, 1, ld, P.scratch, 1, n2, n, n2, n1, cc, P.tw, n, sign, P.tw, n, s);
    if (r) return r;
    // step 2: sequences k2 (stride 1 in scratch), elements j1 (stride n2): length n1 -> x[k2 + n2 k1]
    r = launch_tile(P.scratch, n2, 1, n, xc, n2, 1, ld, n1, n2, cc, P.tw, n, sign, nullptr, 0, s);
    if (r) return r;
  }
  return 0;
}

struct PlanImpl {
  Pow2 main;   // length n (pow2) or m (Bluestein)
};

int fft_plan_create(FFTPlan& p, int64_t n, cudaStream_t s) {
  p.n = n;
  p.pow2 = (n & (n - 1)) == 0;
  int64_t len = n;
  if (!p.pow2) {
    int64_t m = 1;
    while (m < 2 * n - 1) m <<= 1;
    p.m = m;
    len = m;
  }
  if (cudaMalloc(&p.twiddle, sizeof(zd) * len) != cudaSuccess) { set_error("oom (fft)"); return 4; }
  k_twiddles<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(p.twiddle, len);
  note_launch();
  p.work_cols = std::max<int64_t>(1, std::min<int64_t>(256, (int64_t(1) << 27) / len));
  if (cudaMalloc(&p.work, sizeof(zd) * len * p.work_cols * (p.pow2 ? 1 : 2)) != cudaSuccess) {
    set_error("oom (fft work)");
    return 4;
  }
  if (!p.pow2) {
    const int64_t m = p.m;
    if (cudaMalloc(&p.chirp, sizeof(zd) * n) != cudaSuccess ||
        cudaMalloc(&p.chirp_hat, sizeof(zd) * m) != cudaSuccess) {
      set_error("oom (bluestein)");
      return 4;
    }
    k_chirp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.chirp, n);
    note_launch();
    k_bluestein_filter<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.chirp, n, m, p.chirp_hat);
    note_launch();
    Pow2 P{m, p.twiddle, p.work + m * p.work_cols, p.work_cols};
    int r = pow2_transform(P, p.chirp_hat, m, 1, -1, s);
    if (r) return r;
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

void fft_plan_destroy(FFTPlan& p) {
  cudaFree(p.twiddle);
  cudaFree(p.chirp);
  cudaFree(p.chirp_hat);
  cudaFree(p.work);
  p = FFTPlan();
}

int fft_columns(FFTPlan& p, zd* x, int64_t ld, int64_t cols, int sign, cudaStream_t s) {
  if (cols <= 0) return 0;
  if (p.pow2) {
    Pow2 P{p.n, p.twiddle, p.work, p.work_cols};
    return pow2_transform(P, x, ld, cols, sign, s);
  }
  const int64_t n = p.n, m = p.m;
  zd* work = p.work;
  zd* scratch = p.work + m * p.work_cols;
  for (int64_t c0 = 0; c0 < cols; c0 += p.work_cols) {
    int64_t cc = std::min(p.work_cols, cols - c0);
    dim3 gm((unsigned)((m + 255) / 256), (unsigned)cc), gn((unsigned)((n + 255) / 256), (unsigned)cc);
    k_bluestein_pre<<<gm, 256, 0, s>>>(x + c0 * ld, ld, n, m, p.chirp, sign, work);
    note_launch();
    Pow2 P{m, p.twiddle, scratch, p.work_cols};
    int r = pow2_transform(P, work, m, cc, -1, s);
    if (r) return r;
    k_pointwise<<<gm, 256, 0, s>>>(work, m, p.chirp_hat, 0);
    note_launch();
    r = pow2_transform(P, work, m, cc, +1, s);
    if (r) return r;
    k_bluestein_post<<<gn, 256, 0, s>>>(work, n, m, p.chirp, sign, x + c0 * ld, ld);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

int scale_columns(zd* x, int64_t n, int64_t ld, int64_t cols, const zd* mu, bool divide,
                  bool conj_mu, double extra, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < cols; c0 += 65535) {
    int64_t cc = std::min<int64_t>(65535, cols - c0);
    dim3 g((unsigned)((n + 255) / 256), (unsigned)cc);
    k_scale_columns<<<g, 256, 0, s>>>(x + c0 * ld, n, ld, mu, divide, conj_mu, extra);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

}  // namespace wcs
