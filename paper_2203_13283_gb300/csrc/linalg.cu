// Dense complex FP64 linear algebra for the solver: operator applies
// (Eq. 6), randomized range finding for the skeleton (Eq. 7) and the
// capacitance matrix of the Woodbury identity (Eq. 9).
#include <algorithm>
#include <climits>
#include <vector>

#include "internal.h"

namespace wcs {

// =========================================================================== ZGEMM (FP64 FMA pipe)
// C (m x n, column-major) = alpha * A * B + beta * C; A (m x k), B (k x n) are
// strided views (element (i, j) at p[i*rs + j*cs], optionally conjugated).
// 256 threads as a TY x TX grid, each computing TM x TN outputs: tiles of
// (TY TM) x (TX TN).  The FP64 pipe is the bound (GB300 issues ~2 DFMA per
// clock per SM), so the tile width follows n: a block of a few right-hand
// sides must not pay for 64 columns of zeros.
constexpr int GB_K = 16;

template <int TY, int TX, int TM, int TN>
__global__ void __launch_bounds__(256) k_zgemm(int64_t m, int64_t n, int64_t k, zd alpha, ZView A,
                                               ZView B, zd beta, zd* __restrict__ C, int64_t ldc) {
  static_assert(TY * TX == 256, "256 threads");
  constexpr int BM = TY * TM, BN = TX * TN;
  __shared__ zd As[GB_K][BM + 1];
  __shared__ zd Bs[GB_K][BN + 1];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  zd acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mkz(0.0);
  const bool a_kfast = (A.cs == 1);  // walk k first when it is the contiguous index
  const bool b_kfast = (B.rs == 1);
  for (int64_t k0 = 0; k0 < k; k0 += GB_K) {
    for (int u = threadIdx.x; u < BM * GB_K; u += 256) {
      int ii, kk;
      if (a_kfast) { kk = u % GB_K; ii = u / GB_K; } else { ii = u % BM; kk = u / BM; }
      const int64_t gi = m0 + ii, gk = k0 + kk;
      zd v = mkz(0.0);
      if (gi < m && gk < k) {
        v = A.p[gi * A.rs + gk * A.cs];
        if (A.conj) v.y = -v.y;
      }
      As[kk][ii] = v;
    }
    for (int u = threadIdx.x; u < BN * GB_K; u += 256) {
      int jj, kk;
      if (b_kfast) { kk = u % GB_K; jj = u / GB_K; } else { jj = u % BN; kk = u / BN; }
      const int64_t gj = n0 + jj, gk = k0 + kk;
      zd v = mkz(0.0);
      if (gj < n && gk < k) {
        v = B.p[gk * B.rs + gj * B.cs];
        if (B.conj) v.y = -v.y;
      }
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GB_K; ++kk) {
      zd a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) zfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const bool beta0 = (beta.x == 0.0 && beta.y == 0.0);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gi = m0 + ty + TY * i, gj = n0 + tx + TX * j;
      if (gi < m && gj < n) {
        zd r = alpha * acc[i][j];
        if (!beta0) r += beta * C[gj * ldc + gi];
        C[gj * ldc + gi] = r;
      }
    }
}

template <int TY, int TX, int TM, int TN>
static int launch_zgemm(int64_t m, int64_t n, int64_t k, zd alpha, ZView A, ZView B, zd beta, zd* C, int64_t ldc,
                        cudaStream_t s) {
  constexpr int BM = TY * TM, BN = TX * TN;
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM));
  if (grid.y > 65535) { set_error("zgemm: m too large"); return 1; }
  k_zgemm<TY, TX, TM, TN><<<grid, 256, 0, s>>>(m, n, k, alpha, A, B, beta, C, ldc);
  note_launch();
  return 0;
}

int zgemm(int64_t m, int64_t n, int64_t k, zd alpha, ZView A, ZView B, zd beta, zd* C, int64_t ldc,
          cudaStream_t s) {
  if (m <= 0 || n <= 0) return 0;
  int r;
  if (n <= 8) r = launch_zgemm<32, 8, 4, 1>(m, n, k, alpha, A, B, beta, C, ldc, s);          // 128 x 8 tiles
  else if (n <= 16) r = launch_zgemm<16, 16, 4, 1>(m, n, k, alpha, A, B, beta, C, ldc, s);   // 64 x 16
  else if (n <= 32) r = launch_zgemm<16, 16, 4, 2>(m, n, k, alpha, A, B, beta, C, ldc, s);   // 64 x 32
  else r = launch_zgemm<16, 16, 4, 4>(m, n, k, alpha, A, B, beta, C, ldc, s);                // 64 x 64
  if (r) return r;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("zgemm: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

// =========================================================================== Gram matrix
// G = (h/6) circ(1, 4, 1).  With rho = sqrt(3) - 2 (root of rho^2 + 4 rho + 1):
// circ(1,4,1) = (-1/rho) (1 - rho S)(1 - rho S^-1), S the cyclic down-shift,
// so G^{-1} x = (6/h)(-rho) z with u_i = x_i + rho u_{i-1} (forward) and
// z_i = u_i + rho z_{i+1} (backward).  Each thread filters a chunk of CH
// outputs starting WARM samples early; |rho|^WARM < 1e-23 makes the cyclic
// wrap-around exact to rounding.
constexpr int GI_CH = 64, GI_WARM = 40;

__global__ void k_gram_fwd(const zd* __restrict__ X, int64_t ldx, zd* __restrict__ U, int64_t n,
                           int64_t cols, double rho) {
  const int64_t chunks = (n + GI_CH - 1) / GI_CH;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= chunks * cols) return;
  const int64_t c = t / chunks, i0 = (t - c * chunks) * GI_CH;
  const int64_t i1 = min(n, i0 + GI_CH);
  const zd* x = X + c * ldx;
  zd* u = U + c * n;
  zd acc = mkz(0.0);
  const int64_t warm = GI_WARM;  // the input is periodic: wrapping more than once is fine
  int64_t ii = ((i0 - warm) % n + n) % n;   // index mod n, advanced with a compare (no division per step)
  for (int64_t i = i0 - warm; i < i1; ++i) {
    acc = x[ii] + rho * acc;
    if (i >= i0) u[ii] = acc;
    if (++ii == n) ii = 0;
  }
}

__global__ void k_gram_bwd(const zd* __restrict__ U, zd* __restrict__ Y, int64_t ldy, int64_t n,
                           int64_t cols, double rho, double scale) {
  const int64_t chunks = (n + GI_CH - 1) / GI_CH;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= chunks * cols) return;
  const int64_t c = t / chunks, i0 = (t - c * chunks) * GI_CH;
  const int64_t i1 = min(n, i0 + GI_CH);
  const zd* u = U + c * n;
  zd* y = Y + c * ldy;
  zd acc = mkz(0.0);
  const int64_t warm = GI_WARM;
  int64_t ii = (i1 - 1 + warm) % n;
  for (int64_t i = i1 - 1 + warm; i >= i0; --i) {
    acc = u[ii] + rho * acc;
    if (i < i1) y[ii] = scale * acc;
    if (--ii < 0) ii = n - 1;
  }
}

int gram_inverse(const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t n, int64_t cols, double h,
                 zd* work, cudaStream_t s) {
  if (cols <= 0) return 0;
  if (!work) { set_error("gram: no work buffer"); return 1; }
  const double rho = sqrt(3.0) - 2.0;
  const int64_t tasks = ((n + GI_CH - 1) / GI_CH) * cols;
  const unsigned blocks = (unsigned)((tasks + 127) / 128);
  k_gram_fwd<<<blocks, 128, 0, s>>>(X, ldx, work, n, cols, rho);
  note_launch();
  k_gram_bwd<<<blocks, 128, 0, s>>>(work, Y, ldy, n, cols, rho, -rho * 6.0 / h);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("gram: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

__global__ void k_gram_apply(const zd* __restrict__ X, int64_t ldx, zd* __restrict__ Y, int64_t ldy,
                             int64_t n, double a6, double a4, double beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= n) return;
  const zd* x = X + c * ldx;
  const zd xm = x[i == 0 ? n - 1 : i - 1], x0 = x[i], xp = x[i == n - 1 ? 0 : i + 1];
  zd r = a6 * (xm + xp) + a4 * x0;
  zd* y = Y + c * ldy;
  if (beta != 0.0) r += beta * y[i];
  y[i] = r;
}

int gram_apply(const zd* X, int64_t ldx, zd* Y, int64_t ldy, int64_t n, int64_t cols, double h,
               double alpha, double beta, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < cols; c0 += 65535) {
    int64_t cc = std::min<int64_t>(65535, cols - c0);
    dim3 g((unsigned)((n + 255) / 256), (unsigned)cc);
    k_gram_apply<<<g, 256, 0, s>>>(X + c0 * ldx, ldx, Y + c0 * ldy, ldy, n, alpha * h / 6.0,
                                   alpha * 4.0 * h / 6.0, beta);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("gram_apply: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

// =========================================================================== small kernels
__global__ void k_colnorm(const zd* X, int64_t ld, int64_t m, double* out) {
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
  if (threadIdx.x == 0) out[c] = sqrt(red[0]);
}

__global__ void k_coldotc(const zd* X, int64_t ldx, const zd* Y, int64_t ldy, int64_t m, zd* out) {
  __shared__ double re[256], im[256];
  const int64_t c = blockIdx.x;
  zd s = mkz(0.0);
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += conj(X[c * ldx + i]) * Y[c * ldy + i];
  re[threadIdx.x] = s.x;
  im[threadIdx.x] = s.y;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      re[threadIdx.x] += re[threadIdx.x + o];
      im[threadIdx.x] += im[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = mkz(re[0], im[0]);
}

int column_dotc(const zd* X, int64_t ldx, const zd* Y, int64_t ldy, int64_t m, int64_t n, zd* out,
                cudaStream_t s) {
  for (int64_t c0 = 0; c0 < n; c0 += 65535) {
    const int64_t cc = std::min<int64_t>(65535, n - c0);
    k_coldotc<<<(unsigned)cc, 256, 0, s>>>(X + c0 * ldx, ldx, Y + c0 * ldy, ldy, m, out + c0);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

int column_norms(const zd* X, int64_t ld, int64_t m, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return 0;
  k_colnorm<<<(unsigned)n, 256, 0, s>>>(X, ld, m, out);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
__device__ __forceinline__ uint4 philox4x32(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
  // 53-bit uniform in (0, 1]
  const uint64_t v = ((uint64_t)a << 21) ^ (uint64_t)b;
  return ((double)(v & ((1ull << 53) - 1)) + 1.0) * (1.0 / 9007199254740992.0);
}

__global__ void k_gauss(zd* X, int64_t ld, int64_t m, int64_t n, uint64_t seed, uint64_t offset) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t c = t / m, i = t - c * m;
  const uint64_t ctr = offset + (uint64_t)t;
  uint4 r = philox4x32(make_uint4((uint32_t)ctr, (uint32_t)(ctr >> 32), 0x57435331u, 0u),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double u1 = u01(r.x, r.y), u2 = u01(r.z, r.w);
  const double rad = sqrt(-log(u1));  // E|z|^2 = 1
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  X[c * ld + i] = mkz(rad * cs, rad * sn);
}

int gaussian_fill(zd* X, int64_t ld, int64_t m, int64_t n, uint64_t seed, uint64_t offset,
                  cudaStream_t s) {
  const int64_t tot = m * n;
  if (tot <= 0) return 0;
  k_gauss<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ld, m, n, seed, offset);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

__global__ void k_axpby(int64_t m, zd a, const zd* X, int64_t ldx, zd b, zd* Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= m) return;
  zd y = mkz(0.0);
  if (b.x != 0.0 || b.y != 0.0) y = b * Y[c * ldy + i];
  Y[c * ldy + i] = y + a * X[c * ldx + i];
}

int axpby(int64_t m, int64_t n, zd a, const zd* X, int64_t ldx, zd b, zd* Y, int64_t ldy,
          cudaStream_t s) {
  for (int64_t c0 = 0; c0 < n; c0 += 65535) {
    int64_t cc = std::min<int64_t>(65535, n - c0);
    dim3 g((unsigned)((m + 255) / 256), (unsigned)cc);
    k_axpby<<<g, 256, 0, s>>>(m, a, X + c0 * ldx, ldx, b, Y + c0 * ldy, ldy);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

// =========================================================================== Gram matrix X^H X
// Tall-skinny X (m x b, b <= 64): CTAs take row chunks and write partial
// b x b Grams, a second kernel sums the partials (fixed order: deterministic).
constexpr int GRAM_ROWS = 256;

// Partial Gram sums over GRAM_ROWS rows: only the upper triangle i <= j of the
// Hermitian b x b result is formed (pair index p -> column j = row of the
// triangular numbers, row i = p - j (j + 1) / 2); both halves are written.
__global__ void k_gram_partial(const zd* X, int64_t ld, int64_t m, int b, zd* part) {
  __shared__ zd xs[64][33];
  const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
  const int tid = threadIdx.x;                  // 256 threads: up to 9 pairs each
  const int npairs = b * (b + 1) / 2;
  int ii[9], jj[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int p = tid + 256 * t;
    int j = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while (j * (j + 1) / 2 > p) --j;
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    ii[t] = (p < npairs) ? p - j * (j + 1) / 2 : -1;
    jj[t] = j;
  }
  zd acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = mkz(0.0);
  for (int64_t rr = r0; rr < min(m, r0 + GRAM_ROWS); rr += 32) {
    __syncthreads();
    for (int u = tid; u < 32 * b; u += blockDim.x) {
      const int c = u / 32, r = u % 32;
      xs[c][r] = (rr + r < m) ? X[(int64_t)c * ld + rr + r] : mkz(0.0);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      if (ii[t] >= 0) {
        const int i = ii[t], j = jj[t];
        for (int r = 0; r < 32; ++r) zfma(acc[t], conj(xs[i][r]), xs[j][r]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    if (ii[t] < 0) continue;
    const int i = ii[t], j = jj[t];
    zd* P = part + (int64_t)blockIdx.x * b * b;
    P[j * b + i] = acc[t];
    if (i != j) P[i * b + j] = conj(acc[t]);
  }
}

__global__ void k_gram_reduce(const zd* part, int nparts, int b, zd* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b * b) return;
  zd s = mkz(0.0);
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * b * b + t];
  G[t] = s;
}

int gram_matrix(const zd* X, int64_t ld, int64_t m, int b, zd* G, zd* work, cudaStream_t s) {
  if (b > 64) { set_error("gram_matrix: b <= 64"); return 1; }
  const int nparts = (int)((m + GRAM_ROWS - 1) / GRAM_ROWS);
  k_gram_partial<<<nparts, 256, 0, s>>>(X, ld, m, b, work);
  note_launch();
  k_gram_reduce<<<(b * b + 255) / 256, 256, 0, s>>>(work, nparts, b, G);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("gram: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

// =========================================================================== pivoted Cholesky
// On a Hermitian b x b matrix (column-major, ld = b, b <= 64), one CTA, the
// matrix held in shared memory.  After return: rank r, perm[0:b], and R
// (upper, row j holds R[j, j..b-1] in permuted order) in Gm's upper triangle.
// Pivot: the largest remaining diagonal entry, the first of equal ones; the
// factorisation stops when it is <= rel_tol^2 times the first pivot (or <= 0).
__global__ void k_pchol(zd* Gm, int b, double rel_tol, int* perm, int* rank_out) {
  extern __shared__ zd G[];
  __shared__ double best_s, dmax_s, rjj_s, rinv_s;
  __shared__ int piv_s, perm_s[64];
  const int tid = threadIdx.x;
  for (int u = tid; u < b * b; u += blockDim.x) G[u] = Gm[u];
  for (int i = tid; i < b; i += blockDim.x) perm_s[i] = i;
  __syncthreads();
  int rank = b;
  for (int j = 0; j < b; ++j) {
    if (tid < 32) {
      // warp argmax over the remaining diagonal; ties go to the lower index
      double v = -1.0;
      int p = INT_MAX;
      for (int i = j + tid; i < b; i += 32) {
        const double d = G[i * b + i].x;
        if (d > v) { v = d; p = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, v, o);
        const int p2 = __shfl_down_sync(0xffffffffu, p, o);
        if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
      }
      if (tid == 0) {
        if (p == INT_MAX) { p = j; v = -1.0; }
        if (j == 0) dmax_s = v;
        piv_s = p;
        best_s = v;
      }
    }
    __syncthreads();
    const double best = best_s;
    if (best <= rel_tol * rel_tol * dmax_s || best <= 0.0) { rank = j; break; }
    const int p = piv_s;
    if (p != j) {
      // symmetric swap of rows/columns j and p
      for (int i = tid; i < b; i += blockDim.x) {
        zd t = G[j * b + i]; G[j * b + i] = G[p * b + i]; G[p * b + i] = t;  // columns
      }
      __syncthreads();
      for (int i = tid; i < b; i += blockDim.x) {
        zd t = G[i * b + j]; G[i * b + j] = G[i * b + p]; G[i * b + p] = t;  // rows
      }
      if (tid == 0) { int t = perm_s[j]; perm_s[j] = perm_s[p]; perm_s[p] = t; }
      __syncthreads();
    }
    // sqrt and reciprocal once: on the FP64 pipe of one SM, 512 copies of
    // them would cost more than the whole Schur update of the step
    if (tid == 0) {
      rjj_s = sqrt(G[j * b + j].x);
      rinv_s = 1.0 / rjj_s;
    }
    __syncthreads();
    const double rjj = rjj_s, rinv = rinv_s;
    // row j of R: R[j, i] = G[j, i] / rjj  (G[j, i] at column i, row j)
    for (int i = tid; i < b; i += blockDim.x) {
      if (i > j) G[i * b + j] = rinv * G[i * b + j];
      if (i == j) G[j * b + j] = mkz(rjj);
    }
    __syncthreads();
    // Schur complement: G[l, i] -= conj(R[j, l]) R[j, i] for j < l <= i
    // (warp w: columns i = j + 1 + w + 16 t; lanes: rows l), mirrored into
    // the lower triangle, which the pivot swaps read
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int i = j + 1 + warp; i < b; i += nw) {
      const zd rji = G[i * b + j];
      for (int l = j + 1 + lane; l <= i; l += 32) {
        const zd v = G[i * b + l] - conj(G[l * b + j]) * rji;
        G[i * b + l] = v;
        if (l < i) G[l * b + i] = conj(v);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int u = tid; u < b * b; u += blockDim.x) Gm[u] = G[u];
  for (int i = tid; i < b; i += blockDim.x) perm[i] = perm_s[i];
  if (tid == 0) *rank_out = rank;
}

int pivoted_cholesky(zd* Gm, int b, double rel_tol, int* perm, int* rank_dev, cudaStream_t s) {
  if (b < 1 || b > 64) { set_error("pivoted_cholesky: 1 <= b <= 64"); return 1; }
  const int smem = (int)sizeof(zd) * b * b;
  static DeviceOnce attr;
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(k_pchol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(zd) * 64 * 64);
    if (e != cudaSuccess) { set_error(std::string("pivoted_cholesky: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  k_pchol<<<1, 512, smem, s>>>(Gm, b, rel_tol, perm, rank_dev);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

// Y(i, 0:r) = X(i, perm[0:r]) R^{-1}, R the r x r upper factor of k_pchol
// (R[i][l] at R[l * b + i]).  Two kernels: Z = R^{-1} column by column (CTA c
// solves R z = e_c by back substitution, the update of each finished entry
// spread over the threads), then Y = X_perm Z over row tiles, where each row
// is independent: no dependency chain through memory, so the FP64 pipe is
// the bound.
__global__ void k_tri_inv(const zd* R, int b, const int* rank_dev, zd* Z) {
  extern __shared__ zd Rs[];   // R[0:c+1, 0:c+1], column-major, ld c + 1 (64 KB at c = 63)
  __shared__ zd dinv[64], zl_s;
  const int r = *rank_dev, c = blockIdx.x, i = threadIdx.x, n = c + 1;
  if (c >= r) return;
  for (int u = i; u < n * n; u += blockDim.x) {
    const int row = u % n, col = u / n;
    Rs[u] = (row <= col) ? R[col * b + row] : mkz(0.0);
  }
  if (i < n) dinv[i] = zrecip(R[i * b + i]);
  __syncthreads();
  zd s = mkz(i == c ? 1.0 : 0.0);
  for (int l = c; l >= 0; --l) {
    if (i == l) {
      zl_s = s * dinv[l];
      Z[c * r + l] = zl_s;
    }
    __syncthreads();
    const zd z = zl_s;
    if (i < l) s -= Rs[l * n + i] * z;
    __syncthreads();
  }
  for (int u = c + 1 + i; u < r; u += blockDim.x) Z[c * r + u] = mkz(0.0);
}

constexpr int TRSM_ROWS = 32;   // rows per CTA

// 4 warps: warp g forms columns g, g + 4, ..., g + 60 of 32 rows (interleaved,
// so the triangle's work is even over the warps), each column over its own
// l <= c only (a predicated-off FP64 FMA still takes its issue slot in the
// FP64 pipe); X tile and Z in shared memory (Z read as broadcasts, X
// row-consecutive across the lanes).
__global__ void __launch_bounds__(128) k_trsm_apply(const zd* X, int64_t ldx, int64_t m, const zd* Z,
                                                    const int* perm, const int* rank_dev, zd* Y,
                                                    int64_t ldy) {
  extern __shared__ zd sm[];
  const int r = *rank_dev;
  zd* Zs = sm;                 // r x r, column-major
  zd* xs = sm + r * r;         // r x TRSM_ROWS
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * TRSM_ROWS;
  for (int u = tid; u < r * r; u += blockDim.x) Zs[u] = Z[u];
  for (int u = tid; u < r * TRSM_ROWS; u += blockDim.x) {
    const int l = u / TRSM_ROWS, rr = u % TRSM_ROWS;
    xs[u] = (row0 + rr < m) ? X[(int64_t)perm[l] * ldx + row0 + rr] : mkz(0.0);
  }
  __syncthreads();
  const int64_t i = row0 + lane;
  for (int c = g; c < r; c += 4) {
    // two partial sums (even and odd l) for two independent FMA chains
    zd a0 = mkz(0.0), a1 = mkz(0.0);
    const zd* zc = Zs + c * r;
    int l = 0;
    for (; l + 1 <= c; l += 2) {
      zfma(a0, xs[l * TRSM_ROWS + lane], zc[l]);
      zfma(a1, xs[(l + 1) * TRSM_ROWS + lane], zc[l + 1]);
    }
    if (l == c) zfma(a0, xs[l * TRSM_ROWS + lane], zc[l]);
    if (i < m) Y[(int64_t)c * ldy + i] = a0 + a1;
  }
}

int trsm_right_upper(const zd* X, int64_t ldx, int64_t m, const zd* R, int b, const int* perm,
                     const int* rank_dev, int rank_host, zd* Y, int64_t ldy, zd* work, cudaStream_t s) {
  if (b > 64 || rank_host > b) { set_error("trsm: block too wide"); return 1; }
  if (rank_host <= 0) return 0;
  static DeviceOnce attr;
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(k_trsm_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(zd) * (64 * 64 + 64 * TRSM_ROWS)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tri_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(zd) * 64 * 64));
    if (e != cudaSuccess) { set_error(std::string("trsm: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  k_tri_inv<<<(unsigned)rank_host, 64, sizeof(zd) * rank_host * rank_host, s>>>(R, b, rank_dev, work);
  note_launch();
  const size_t smem = sizeof(zd) * ((size_t)rank_host * rank_host + (size_t)rank_host * TRSM_ROWS);
  k_trsm_apply<<<(unsigned)((m + TRSM_ROWS - 1) / TRSM_ROWS), 128, smem, s>>>(X, ldx, m, work, perm, rank_dev,
                                                                                Y, ldy);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("trsm: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

// =========================================================================== Gauss-Jordan inverse
// M = [A | I] (n x 2n, column-major, ld = n).  Step j: pick the pivot row in
// column j, swap, scale the pivot row, eliminate column j from every other row.
__global__ void k_gj_pivot(zd* M, int64_t n, int64_t j, zd* colj, zd* rowj, int* info,
                           double* minpiv) {
  __shared__ double best[512];
  __shared__ int bidx[512];
  const int tid = threadIdx.x;
  double b = -1.0;
  int bi = (int)j;
  for (int64_t i = j + tid; i < n; i += blockDim.x) {
    double v = abs2(M[j * n + i]);
    if (v > b) { b = v; bi = (int)i; }
  }
  best[tid] = b;
  bidx[tid] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o && best[tid + o] > best[tid]) { best[tid] = best[tid + o]; bidx[tid] = bidx[tid + o]; }
    __syncthreads();
  }
  const int64_t p = bidx[0];
  const double pv = sqrt(best[0]);
  if (tid == 0) {
    if (pv < *minpiv) *minpiv = pv;
    if (!(pv > 0.0)) *info = (int)j + 1;
  }
  // swap rows j and p over all 2n columns
  if (p != j)
    for (int64_t c = tid; c < 2 * n; c += blockDim.x) {
      zd t = M[c * n + j]; M[c * n + j] = M[c * n + p]; M[c * n + p] = t;
    }
  __syncthreads();
  const zd inv = (pv > 0.0) ? zrecip(M[j * n + j]) : mkz(0.0);
  for (int64_t i = tid; i < n; i += blockDim.x) colj[i] = M[j * n + i];
  for (int64_t c = tid; c < 2 * n; c += blockDim.x) rowj[c] = M[c * n + j] * inv;
}

__global__ void k_gj_update(zd* M, int64_t n, int64_t j, int64_t cbase, const zd* colj,
                            const zd* rowj) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = cbase + blockIdx.y;
  if (i >= n || c >= 2 * n) return;
  if (i == j) M[c * n + i] = rowj[c];
  else M[c * n + i] -= colj[i] * rowj[c];
}

__global__ void k_identity(zd* M, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) M[i * n + i] = mkz(1.0);
}

int lu_inverse(zd* A, int64_t n, zd* Ainv, int* piv, int* info_dev, double* minpiv_dev,
               cudaStream_t s) {
  (void)piv;
  zd *M = nullptr, *colj = nullptr, *rowj = nullptr;
  if (cudaMalloc(&M, sizeof(zd) * n * 2 * n) != cudaSuccess ||
      cudaMalloc(&colj, sizeof(zd) * n) != cudaSuccess ||
      cudaMalloc(&rowj, sizeof(zd) * 2 * n) != cudaSuccess) {
    cudaFree(M); cudaFree(colj); cudaFree(rowj);
    set_error("oom (capacitance inverse)");
    return 4;
  }
  cudaMemcpy2DAsync(M, sizeof(zd) * n, A, sizeof(zd) * n, sizeof(zd) * n, n, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(M + n * n, 0, sizeof(zd) * n * n, s);
  k_identity<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M + n * n, n);
  note_launch();
  const double big = 1e300;
  cudaMemcpyAsync(minpiv_dev, &big, sizeof(double), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(info_dev, 0, sizeof(int), s);
  for (int64_t j = 0; j < n; ++j) {
    k_gj_pivot<<<1, 512, 0, s>>>(M, n, j, colj, rowj, info_dev, minpiv_dev);
    note_launch();
    const int64_t ncols = 2 * n - j;
    for (int64_t c0 = 0; c0 < ncols; c0 += 65535) {
      dim3 g((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(65535, ncols - c0));
      k_gj_update<<<g, 256, 0, s>>>(M, n, j, j + c0, colj, rowj);
      note_launch();
    }
  }
  cudaMemcpy2DAsync(Ainv, sizeof(zd) * n, M + n * n, sizeof(zd) * n, sizeof(zd) * n, n,
                    cudaMemcpyDeviceToDevice, s);
  cudaError_t err = cudaStreamSynchronize(s);
  cudaFree(M); cudaFree(colj); cudaFree(rowj);
  if (err != cudaSuccess) { set_error(std::string("inverse: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

}  // namespace wcs
