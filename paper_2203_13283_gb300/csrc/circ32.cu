// Circulant applies of the mixed form in FP32: y = F^-1 diag(s) F x for the
// equivalent circle's operator C_c (Sec. V: C_c is diagonalised by the DFT,
// its eigenvalues mu_C; s = mu_C, conj(mu_C), 1/mu_C or 1/conj(mu_C)).
//
// In the mixed form C_c^-1 serves the Woodbury approximate inverse (Eq. 9)
// that iterative refinement corrects, and C_c the sampling of C - C_c; an
// FP32 transform (relative error ~1e-6) is far below the accuracy those
// need, while GB300's FP64 pipe (1/64 of FP32) made the FP64 transform
// arithmetic-bound.  The eigenvalues themselves stay FP64 (the FP64
// transform computes them; this file only reads them).
//
// Power-of-two n = n1 n2 (n1 = 32 R1, n2 = 32 R2, 1024 <= n <= 65536), in
// three passes over each column, x[j1 + n1 j2] -> y:
//   1. for each j1, a length-n2 DFT over j2, times W_n^{j1 k2}   -> S[k2 n1 + j1]
//   2. for each k2, a length-n1 DFT over j1 (giving X[k2 + n2 k1]), times
//      s[k2 + n2 k1] / n, the inverse length-n1 DFT over k1, times
//      W_n^{-j1 k2}                                               -> S[k2 n1 + j1]
//   3. for each j1, the inverse length-n2 DFT over k2              -> y[j1 + n1 j2]
// (the four-step factorisation W_n^{jk} = W_n^{j1 k2} W_n1^{j1 k1} W_n2^{j2 k2}
// for j = j1 + n1 j2, k = k2 + n2 k1, applied forward and then backward, with
// the diagonal and the middle steps of both transforms fused into pass 2).
// x and y are FP64 in HBM, S is FP32: 24 + 16 + 24 bytes per element.
//
// One warp transforms one sequence of L = 32 R points: lane l holds points
// l + 32 m (m < R) in registers; a radix-2 DIF over the R registers, the
// twiddles W_L^{l a}, and a radix-2 DIF across the 32 lanes by xor shuffles
// leave X[a + R brev5(l)] in register brev_R(a).  The inverse runs the adjoint
// of each step in reverse order and returns natural order.  Passes 1 and 3
// move sequences that are strided in memory through a shared-memory tile of
// 16 sequences (rows of 16 x 8 bytes, XOR-swizzled so that both the natural
// and the bit-reversed lane patterns are free of bank conflicts).
#include "../../include/wcs.h"
#include "internal.h"

namespace wcs {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int CG = 16;   // sequences per CTA in passes 1 and 3 (one warp each)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 shfl_x(float2 v, int m) {
  return make_float2(__shfl_xor_sync(FULL, v.x, m), __shfl_xor_sync(FULL, v.y, m));
}

// e^{sign 2 pi i q / n} in FP32 for n = 2^lg: q reduced mod n exactly and
// 2 q / n formed exactly (a power-of-two scale), so only sincospif rounds.
// Integer arguments stay 32-bit: 64-bit integer conversions, like every
// conversion involving FP64, run on the FP64 pipe (1/64 of the FP32 rate).
__device__ __forceinline__ float2 twf(int q, int lg, int sign) {
  q &= (1 << lg) - 1;
  float s, c;
  sincospif((float)q * __int_as_float((128 - lg) << 23), &s, &c);
  return make_float2(c, sign > 0 ? s : -s);
}

// FP64 <-> FP32 by integer operations (the hardware conversions run on the
// FP64 pipe).  f64_to_f32 rounds to nearest even; magnitudes below the FP32
// normal range flush to zero, above it become infinite; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned sign = hi & 0x80000000u;
  const int ed = (int)((hi >> 20) & 0x7ffu);
  if (ed == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
  const int e = ed - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned f = sign | ((unsigned)e << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) f += 1u;   // a carry moves into the exponent
  return __uint_as_float(f);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi;
  if (e == 0) hi = sign;                                     // zero (FP32 denormals flush)
  else if (e == 255) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else hi = sign | ((e + 896u) << 20) | (m >> 3);
  const unsigned lo = (e == 0) ? 0u : (m & 7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

template <int R>
__host__ __device__ constexpr int brev_r(int r) {
  int out = 0;
  for (int b = 1, t = R >> 1; b < R; b <<= 1, t >>= 1)
    if (r & b) out |= t;
  return out;
}

template <int R>
struct WarpTw {
  float2 reg[R > 1 ? R / 2 : 1];   // W_R^t, t < R/2
  float2 lane[R];                  // W_L^{l a}, a < R
  float2 net[5];                   // W_{2s}^{l mod s}, s = 16, 8, 4, 2, 1
};

__host__ __device__ constexpr int log2c(int v) { return v <= 1 ? 0 : 1 + log2c(v >> 1); }

template <int R>
__device__ __forceinline__ void warp_tw_init(WarpTw<R>& w, int lane) {
#pragma unroll
  for (int t = 0; t < (R > 1 ? R / 2 : 1); ++t) w.reg[t] = twf(t, R > 1 ? log2c(R) : 1, -1);
#pragma unroll
  for (int a = 0; a < R; ++a) w.lane[a] = twf(lane * a, log2c(32 * R), -1);
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int s = 16 >> st;
    w.net[st] = twf(lane & (s - 1), log2c(2 * s), -1);
  }
}

// radix-2 DIF over the registers: natural order in, bit-reversed out
template <int R>
__device__ __forceinline__ void reg_dif(float2 (&v)[R], const float2* tw) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1)
#pragma unroll
    for (int b0 = 0; b0 < R; b0 += 2 * half)
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 a = v[b0 + j], b = v[b0 + j + half];
        v[b0 + j] = cadd(a, b);
        const float2 d = csub(a, b);
        v[b0 + j + half] = (j == 0) ? d : cmulf(d, tw[j * (R / (2 * half))]);
      }
}

// its adjoint: each stage (a, b) -> (a + b, (a - b) w) becomes
// (x, y) -> (x + conj(w) y, x - conj(w) y), stages in reverse order
template <int R>
__device__ __forceinline__ void reg_dif_adj(float2 (&v)[R], const float2* tw) {
#pragma unroll
  for (int half = 1; half <= R / 2; half <<= 1)
#pragma unroll
    for (int b0 = 0; b0 < R; b0 += 2 * half)
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 x = v[b0 + j];
        const float2 y = (j == 0) ? v[b0 + j + half] : cmulc(v[b0 + j + half], tw[j * (R / (2 * half))]);
        v[b0 + j] = cadd(x, y);
        v[b0 + j + half] = csub(x, y);
      }
}

// radix-2 DIF across the lanes (length 32): lane l ends with X[brev5(l)]
__device__ __forceinline__ float2 lane_dif(float2 v, const float2 (&net)[5], int lane) {
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int s = 16 >> st;
    const float2 o = shfl_x(v, s);
    v = (lane & s) ? cmulf(csub(o, v), net[st]) : cadd(v, o);
  }
  return v;
}

__device__ __forceinline__ float2 lane_dif_adj(float2 v, const float2 (&net)[5], int lane) {
#pragma unroll
  for (int st = 4; st >= 0; --st) {
    const int s = 16 >> st;
    const float2 o = shfl_x(v, s);
    v = (lane & s) ? csub(o, cmulc(v, net[st])) : cadd(v, cmulc(o, net[st]));
  }
  return v;
}

// length 32 R: v[m] = point l + 32 m in; register brev_R(a) = X[a + R brev5(l)] out
template <int R>
__device__ __forceinline__ void warp_fft(float2 (&v)[R], const WarpTw<R>& w, int lane) {
  if (R > 1) reg_dif<R>(v, w.reg);
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (brev_r<R>(r) != 0) v[r] = cmulf(v[r], w.lane[brev_r<R>(r)]);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = lane_dif(v[r], w.net, lane);
}

// the adjoint (the unnormalised inverse DFT): layouts swapped
template <int R>
__device__ __forceinline__ void warp_fft_adj(float2 (&v)[R], const WarpTw<R>& w, int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = lane_dif_adj(v[r], w.net, lane);
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (brev_r<R>(r) != 0) v[r] = cmulc(v[r], w.lane[brev_r<R>(r)]);
  if (R > 1) reg_dif_adj<R>(v, w.reg);
}

// shared-memory tile of CG sequences: element (row, g) at row * CG + (g ^ h(row)),
// h(row) = (row ^ (row >> (log2 R + 1))) mod 16.  A half-warp touching rows
// l + 32 m (natural) or a + R brev5(l) (after the transform) hits 16
// different columns, i.e. all 32 banks once.
template <int R>
__device__ __forceinline__ int tile_at(int row, int g) {
  constexpr int sh = (R == 1) ? 1 : (R == 2) ? 2 : (R == 4) ? 3 : 4;
  return row * CG + (g ^ ((row ^ (row >> sh)) & (CG - 1)));
}

constexpr int P13_WARPS = 4;           // passes 1, 3: 4 warps, CG / 4 sequences each
constexpr int P2_WARPS = 8, P2_SEQ = 4;  // pass 2: 8 warps, 4 sequences each

// pass 1: x (FP64, column c at x + c ld) -> S (FP32, column c at S + c n)
template <int R2>
__global__ void __launch_bounds__(32 * P13_WARPS) k_circ_pass1(const zd* __restrict__ x, int64_t ld,
                                                               float2* __restrict__ S, int n1, int lgn) {
  constexpr int n2 = 32 * R2;
  __shared__ float2 tile[n2 * CG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.y, n = (int64_t)1 << lgn;
  const int j1b = blockIdx.x * CG;
  const zd* xc = x + c * ld;
  for (int u = threadIdx.x; u < n2 * CG; u += blockDim.x) {
    const int g = u & (CG - 1), j2 = u / CG;
    const zd v = xc[j1b + g + (int64_t)n1 * j2];
    tile[tile_at<R2>(j2, g)] = make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
  }
  WarpTw<R2> w;
  warp_tw_init<R2>(w, lane);
  const int b = (int)(__brev((unsigned)lane) >> 27);
  __syncthreads();
  float2 v[CG / P13_WARPS][R2];
#pragma unroll
  for (int i = 0; i < CG / P13_WARPS; ++i) {
    const int g = warp + P13_WARPS * i;
#pragma unroll
    for (int m = 0; m < R2; ++m) v[i][m] = tile[tile_at<R2>(lane + 32 * m, g)];
    warp_fft<R2>(v[i], w, lane);
    // W_n^{j1 k2}, k2 = a + R2 b: W^{j1 R2 b} W^{j1 a}
    const int j1 = j1b + g;
    const float2 step = twf(j1, lgn, -1);
    float2 p = twf(j1 * R2 * b, lgn, -1), t[R2];
#pragma unroll
    for (int a = 0; a < R2; ++a) { t[a] = p; p = cmulf(p, step); }
#pragma unroll
    for (int r = 0; r < R2; ++r) v[i][r] = cmulf(v[i][r], t[brev_r<R2>(r)]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CG / P13_WARPS; ++i)
#pragma unroll
    for (int r = 0; r < R2; ++r) tile[tile_at<R2>(brev_r<R2>(r) + R2 * b, warp + P13_WARPS * i)] = v[i][r];
  __syncthreads();
  float2* sc = S + c * n;
  for (int u = threadIdx.x; u < n2 * CG; u += blockDim.x) {
    const int gg = u & (CG - 1), k2 = u / CG;
    sc[(int64_t)k2 * n1 + j1b + gg] = tile[tile_at<R2>(k2, gg)];
  }
}

// pass 2: in place on S; scale: [k2][r][l] = s[k2 + n2 (brev_R1(r) + R1 brev5(l))] / n
template <int R1>
__global__ void __launch_bounds__(32 * P2_WARPS) k_circ_pass2(float2* __restrict__ S, const float2* __restrict__ scale,
                                                              int n2, int lgn) {
  constexpr int n1 = 32 * R1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpTw<R1> w;
  warp_tw_init<R1>(w, lane);
  const int64_t n = (int64_t)1 << lgn;
  for (int i = 0; i < P2_SEQ; ++i) {
    const int k2 = (blockIdx.x * P2_WARPS + warp) * P2_SEQ + i;
    if (k2 >= n2) break;
    float2* s = S + (int64_t)blockIdx.y * n + (int64_t)k2 * n1;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = s[lane + 32 * m];
    warp_fft<R1>(v, w, lane);
    const float2* sc = scale + (int64_t)k2 * n1;
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = cmulf(v[r], sc[32 * r + lane]);
    warp_fft_adj<R1>(v, w, lane);
    // W_n^{-j1 k2}, j1 = l + 32 m
    const float2 step = twf(32 * k2, lgn, +1);
    float2 p = twf(lane * k2, lgn, +1);
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      s[lane + 32 * m] = cmulf(v[m], p);
      p = cmulf(p, step);
    }
  }
}

// pass 3: S -> y (FP64, column c at y + c ld)
template <int R2>
__global__ void __launch_bounds__(32 * P13_WARPS) k_circ_pass3(const float2* __restrict__ S, zd* __restrict__ y,
                                                               int64_t ld, int n1, int lgn) {
  constexpr int n2 = 32 * R2;
  __shared__ float2 tile[n2 * CG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.y, n = (int64_t)1 << lgn;
  const int j1b = blockIdx.x * CG;
  const float2* sc = S + c * n;
  for (int u = threadIdx.x; u < n2 * CG; u += blockDim.x) {
    const int g = u & (CG - 1), k2 = u / CG;
    tile[tile_at<R2>(k2, g)] = sc[(int64_t)k2 * n1 + j1b + g];
  }
  WarpTw<R2> w;
  warp_tw_init<R2>(w, lane);
  const int b = (int)(__brev((unsigned)lane) >> 27);
  __syncthreads();
  float2 v[CG / P13_WARPS][R2];
#pragma unroll
  for (int i = 0; i < CG / P13_WARPS; ++i) {
    const int g = warp + P13_WARPS * i;
#pragma unroll
    for (int r = 0; r < R2; ++r) v[i][r] = tile[tile_at<R2>(brev_r<R2>(r) + R2 * b, g)];
    warp_fft_adj<R2>(v[i], w, lane);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CG / P13_WARPS; ++i)
#pragma unroll
    for (int m = 0; m < R2; ++m) tile[tile_at<R2>(lane + 32 * m, warp + P13_WARPS * i)] = v[i][m];
  __syncthreads();
  zd* yc = y + c * ld;
  for (int u = threadIdx.x; u < n2 * CG; u += blockDim.x) {
    const int gg = u & (CG - 1), j2 = u / CG;
    const float2 t = tile[tile_at<R2>(j2, gg)];
    yc[j1b + gg + (int64_t)n1 * j2] = mkz(f32_to_f64(t.x), f32_to_f64(t.y));
  }
}

// scale tables for the four modes, permuted to pass 2's register layout
__global__ void k_circ_scale(const zd* __restrict__ mu, int64_t n, int n1, int n2, int R1, float2* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k2 = (int)(t / n1), rem = (int)(t % n1), r = rem / 32, l = rem % 32;
  int a = 0;
  for (int bit = 1, hi = R1 >> 1; bit < R1; bit <<= 1, hi >>= 1)
    if (r & bit) a |= hi;
  const int k1 = a + R1 * (int)(__brev((unsigned)l) >> 27);
  const zd m = mu[k2 + (int64_t)n2 * k1];
  const double inv_n = 1.0 / (double)n;
  const zd cm = mkz(m.x, -m.y);
  const zd v[4] = {inv_n * m, inv_n * cm, zdiv(mkz(inv_n, 0.0), m), zdiv(mkz(inv_n, 0.0), cm)};
  for (int mode = 0; mode < 4; ++mode) out[mode * n + t] = make_float2((float)v[mode].x, (float)v[mode].y);
}

int log2i(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return l;
}

template <int R2>
void launch_p1(const zd* x, int64_t ld, float2* S, int n1, int lgn, int64_t cols, cudaStream_t s) {
  k_circ_pass1<R2><<<dim3((unsigned)(n1 / CG), (unsigned)cols), 32 * P13_WARPS, 0, s>>>(x, ld, S, n1, lgn);
}
template <int R2>
void launch_p3(const float2* S, zd* y, int64_t ld, int n1, int lgn, int64_t cols, cudaStream_t s) {
  k_circ_pass3<R2><<<dim3((unsigned)(n1 / CG), (unsigned)cols), 32 * P13_WARPS, 0, s>>>(S, y, ld, n1, lgn);
}
template <int R1>
void launch_p2(float2* S, const float2* scale, int n2, int lgn, int64_t cols, cudaStream_t s) {
  const unsigned gx = (unsigned)((n2 + P2_WARPS * P2_SEQ - 1) / (P2_WARPS * P2_SEQ));
  k_circ_pass2<R1><<<dim3(gx, (unsigned)cols), 32 * P2_WARPS, 0, s>>>(S, scale, n2, lgn);
}

}  // namespace

bool circ32_supported(int64_t n) { return n >= 1024 && n <= 65536 && (n & (n - 1)) == 0; }

int circ32_prepare(Circ32& p, const zd* mu, int64_t n, cudaStream_t s) {
  if (!circ32_supported(n)) { set_error("circ32: unsupported length"); return WCS_ERR_ARG; }
  const int lg = log2i(n);
  p.n = n;
  p.n2 = 1 << (lg / 2);
  p.n1 = (int)(n / p.n2);
  if (p.scale == nullptr || p.scale_n < n) {
    cudaFree(p.scale);
    p.scale = nullptr;
    p.scale_n = 0;
    if (cudaMalloc(&p.scale, sizeof(float2) * 4 * n) != cudaSuccess) { set_error("oom (circ32 scale)"); return WCS_ERR_OOM; }
    p.scale_n = n;
  }
  k_circ_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mu, n, p.n1, p.n2, p.n1 / 32, p.scale);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("circ32 scale: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  p.ready = true;
  return WCS_OK;
}

int circ32_apply(Circ32& p, const zd* x, int64_t ldx, zd* y, int64_t ldy, int64_t cols, int mode, cudaStream_t s) {
  if (!p.ready || mode < 0 || mode > 3) { set_error("circ32: not prepared"); return WCS_ERR_STATE; }
  if (cols <= 0) return WCS_OK;
  const int64_t n = p.n;
  const int n1 = p.n1, n2 = p.n2, lg = log2i(n);
  // scratch: up to 2^28 bytes of FP32 columns per chunk
  const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(cols, ((int64_t)1 << 25) / n));
  if (p.work == nullptr || p.work_elems < n * cap) {
    cudaFree(p.work);
    p.work = nullptr;
    p.work_elems = 0;
    if (cudaMalloc(&p.work, sizeof(float2) * n * cap) != cudaSuccess) { set_error("oom (circ32 work)"); return WCS_ERR_OOM; }
    p.work_elems = n * cap;
  }
  float2* S = p.work;
  const float2* sc = p.scale + (int64_t)mode * n;
  for (int64_t c0 = 0; c0 < cols; c0 += cap) {
    const int64_t cc = std::min(cap, cols - c0);
    const zd* xc = x + c0 * ldx;
    zd* yc = y + c0 * ldy;
    switch (n2 / 32) {
      case 1: launch_p1<1>(xc, ldx, S, n1, lg, cc, s); break;
      case 2: launch_p1<2>(xc, ldx, S, n1, lg, cc, s); break;
      case 4: launch_p1<4>(xc, ldx, S, n1, lg, cc, s); break;
      default: launch_p1<8>(xc, ldx, S, n1, lg, cc, s); break;
    }
    switch (n1 / 32) {
      case 1: launch_p2<1>(S, sc, n2, lg, cc, s); break;
      case 2: launch_p2<2>(S, sc, n2, lg, cc, s); break;
      case 4: launch_p2<4>(S, sc, n2, lg, cc, s); break;
      default: launch_p2<8>(S, sc, n2, lg, cc, s); break;
    }
    switch (n2 / 32) {
      case 1: launch_p3<1>(S, yc, ldy, n1, lg, cc, s); break;
      case 2: launch_p3<2>(S, yc, ldy, n1, lg, cc, s); break;
      case 4: launch_p3<4>(S, yc, ldy, n1, lg, cc, s); break;
      default: launch_p3<8>(S, yc, ldy, n1, lg, cc, s); break;
    }
    note_launch();
    note_launch();
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("circ32: ") + cudaGetErrorString(e)); return WCS_ERR_CUDA; }
  return WCS_OK;
}

void circ32_release(Circ32& p) {
  cudaFree(p.scale);
  cudaFree(p.work);
  p = Circ32();
}

}  // namespace wcs
