// Galerkin assembly of the operators of Eq. (4) and Eq. (5):
//   S~ = <l_i, S^k~ l_j>   kernel g_k~ = (i/4) H0(k~ R)
//   D  = <l_i, D^k  l_j>   kernel dg_k/dn' = (i k/4) H1(k R) (r - r').n' / R
//   D~ = <l_i, D^k~ l_j>
//   N  = <l_i, N^k  l_j>   Maue form: [l_i' l_j' - k^2 (n.n') l_i l_j] g_k
// with piecewise-linear hats on the arc-length-uniform mesh (Sec. V).
//
// Element pair (e, f) contributes a 2x2 block to node pairs (e+a, f+b).  One
// CTA owns a 32 x 32 tile of node pairs and evaluates the 33 x 33 element
// pairs that touch it (one Hankel evaluation per point pair and wavenumber is
// shared by all four operators), accumulating in shared memory in four
// conflict-free phases (a, b), so the result is deterministic.
//
// Quadrature by periodic element distance d: d > near_band tensor Gauss
// (q_far); 2 <= d <= near_band tensor Gauss (q_near); d <= 1 the same q_near
// grid with the log|s - s'| part of each kernel integrated by product
// weights (split K = A log|s - s'| + B, A = -(1/2pi) J0 or -(kappa/2pi) J1 g).
#include "hankel.cuh"
#include "internal.h"

namespace wcs {

__constant__ double c_xf[16], c_wf[16], c_xn[16], c_wn[16];

struct PairOut {
  zd v[4][4];  // [operator S~, D, D~, N][a * 2 + b]
};

__device__ __forceinline__ int periodic_dist(int64_t e, int64_t f, int64_t N) {
  int64_t d = e - f;
  if (d < 0) d = -d;
  if (N - d < d) d = N - d;
  return (int)d;
}

// i/4 * H
__device__ __forceinline__ zd i4(zd H) { return mkz(-0.25 * H.y, 0.25 * H.x); }

__device__ void pair_integrals(const AsmArgs& A, int64_t e, int64_t f, PairOut& o) {
#pragma unroll
  for (int op = 0; op < 4; ++op)
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[op][j] = mkz(0.0);
  const int64_t N = A.N;
  const int d = periodic_dist(e, f, N);
  const double h = A.h, k = A.k, kk2h2 = k * k * h * h;
  const zd kt = A.kt;
  if (d > A.near_band) {
    const int q = A.q_far;
    for (int p = 0; p < q; ++p) {
      const int64_t ip = e * q + p;
      const double xt = A.far.x[ip], yt = A.far.y[ip], nxt = A.far.nx[ip], nyt = A.far.ny[ip];
      const double xip = c_xf[p], wp = c_wf[p];
      for (int r = 0; r < q; ++r) {
        const int64_t ir = f * q + r;
        const double dx = xt - A.far.x[ir], dy = yt - A.far.y[ir];
        const double nxs = A.far.nx[ir], nys = A.far.ny[ir];
        const double R = sqrt(dx * dx + dy * dy);
        const double gg = (dx * nxs + dy * nys) / R;
        const double nd = nxt * nxs + nyt * nys;
        Hankel01 Hk = hankel01(mkz(k * R));
        Hankel01 Ht = hankel01(kt * R);
        const zd gk = i4(Hk.H0);
        const zd gt = i4(Ht.H0);
        const zd dgk = (k * gg) * i4(Hk.H1);
        const zd dgt = gg * (kt * i4(Ht.H1));
        const double w = wp * c_wf[r];
        const double xir = c_xf[r];
        const double ph[2] = {1.0 - xip, xip}, ps[2] = {1.0 - xir, xir};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const double c = w * ph[a] * ps[b];
            const double cn = w * ((a == b) ? 1.0 : -1.0) - kk2h2 * nd * c;
            zfmas(o.v[0][a * 2 + b], c, gt);
            zfmas(o.v[1][a * 2 + b], c, dgk);
            zfmas(o.v[2][a * 2 + b], c, dgt);
            zfmas(o.v[3][a * 2 + b], cn, gk);
          }
      }
    }
  } else {
    const int q = A.q_near;
    int kind = -1;
    if (d == 0) kind = 0;
    else if (d == 1) kind = (((e + 1) % N) == f) ? 1 : 2;
    const double* wl = (kind >= 0) ? (A.wlog + kind * q * q) : nullptr;
    const double lh = log(h);
    const zd logkt2 = zlog(0.5 * kt);
    const double logk2 = log(0.5 * k);
    for (int p = 0; p < q; ++p) {
      const int64_t ip = e * q + p;
      const double xt = A.near.x[ip], yt = A.near.y[ip], nxt = A.near.nx[ip], nyt = A.near.ny[ip];
      const double kap = A.near.kappa[ip];
      const double xip = c_xn[p], wp = c_wn[p];
      for (int r = 0; r < q; ++r) {
        const int64_t ir = f * q + r;
        const double xir = c_xn[r];
        const double dx = xt - A.near.x[ir], dy = yt - A.near.y[ir];
        const double nxs = A.near.nx[ir], nys = A.near.ny[ir];
        const double nd = nxt * nxs + nyt * nys;
        const double w = wp * c_wn[r];
        zd kS, kD, kDt, kN;       // smooth parts (full kernels for regular pairs)
        zd aS = mkz(0.0), aD = mkz(0.0), aDt = mkz(0.0), aN = mkz(0.0);  // log coefficients
        double lw = 0.0;          // weight of the log part
        if (kind == 0 && p == r) {
          // coincident points: limits of B = K - A log|s - s'| at R = 0
          kS = mkz(0.0, 0.25) - (1.0 / (2.0 * WCS_PI)) * (logkt2 + mkz(WCS_EULER_GAMMA));
          kN = mkz(-(1.0 / (2.0 * WCS_PI)) * (logk2 + WCS_EULER_GAMMA), 0.25);
          kD = mkz(-kap / (4.0 * WCS_PI));
          kDt = kD;
          aS = mkz(-1.0 / (2.0 * WCS_PI));
          aN = aS;
          lw = wl[p * q + r] + w * lh;
        } else {
          const double R = sqrt(dx * dx + dy * dy);
          const double gg = (dx * nxs + dy * nys) / R;
          Hankel01 Hk = hankel01(mkz(k * R));
          Hankel01 Ht = hankel01(kt * R);
          kN = i4(Hk.H0);
          kS = i4(Ht.H0);
          kD = (k * gg) * i4(Hk.H1);
          kDt = gg * (kt * i4(Ht.H1));
          if (kind >= 0) {
            double dl = (kind == 0) ? fabs(xip - xir) : ((kind == 1) ? (1.0 - xip + xir) : (xip + 1.0 - xir));
            const double lg = lh + log(dl);  // log |s - s'|
            aS = (-1.0 / (2.0 * WCS_PI)) * Ht.J0;
            aN = (-1.0 / (2.0 * WCS_PI)) * Hk.J0;
            aD = (-(k * gg) / (2.0 * WCS_PI)) * Hk.J1;
            aDt = (-gg / (2.0 * WCS_PI)) * (kt * Ht.J1);
            kS -= lg * aS;
            kN -= lg * aN;
            kD -= lg * aD;
            kDt -= lg * aDt;
            lw = wl[p * q + r] + w * lh;
          }
        }
        const double ph[2] = {1.0 - xip, xip}, ps[2] = {1.0 - xir, xir};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const double pp = ph[a] * ps[b];
            const double sab = (a == b) ? 1.0 : -1.0;
            const double c = w * pp;
            const double cn = w * sab - kk2h2 * nd * c;
            zfmas(o.v[0][a * 2 + b], c, kS);
            zfmas(o.v[1][a * 2 + b], c, kD);
            zfmas(o.v[2][a * 2 + b], c, kDt);
            zfmas(o.v[3][a * 2 + b], cn, kN);
            if (kind >= 0) {
              const double cl = lw * pp;
              const double cln = lw * (sab - kk2h2 * nd * pp);
              zfmas(o.v[0][a * 2 + b], cl, aS);
              zfmas(o.v[1][a * 2 + b], cl, aD);
              zfmas(o.v[2][a * 2 + b], cl, aDt);
              zfmas(o.v[3][a * 2 + b], cln, aN);
            }
          }
      }
    }
  }
  const double h2 = h * h;
#pragma unroll
  for (int op = 0; op < 3; ++op)
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[op][j] = h2 * o.v[op][j];
}

constexpr int TILE = 32;
constexpr int ASM_THREADS = 256;

__global__ void __launch_bounds__(ASM_THREADS) k_assemble(AsmArgs A) {
  extern __shared__ zd acc[];  // [4][TILE][TILE]
  const int64_t N = A.N;
  const int64_t i0 = (int64_t)blockIdx.y * TILE, j0 = (int64_t)blockIdx.x * TILE;
  for (int t = threadIdx.x; t < 4 * TILE * TILE; t += blockDim.x) acc[t] = mkz(0.0);
  __syncthreads();
  const int span = TILE + 1;
  const int npairs = span * span;
  for (int base = 0; base < npairs; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const int el = idx / span, fl = idx - (idx / span) * span;
    bool valid = idx < npairs;
    // element row e = i0 - 1 + el touches node rows i0 - 1 + el + a, a in {0,1}
    // element row i0 - 1 + el feeds tile rows el - 1 (a = 1) and el (a = 0)
    const bool rowok = valid && ((el >= 1 && i0 + el - 1 < N) || (el < TILE && i0 + el < N));
    const bool colok = valid && ((fl >= 1 && j0 + fl - 1 < N) || (fl < TILE && j0 + fl < N));
    PairOut o;
    if (rowok && colok) {
      const int64_t e = ((i0 - 1 + el) % N + N) % N;
      const int64_t f = ((j0 - 1 + fl) % N + N) % N;
      pair_integrals(A, e, f, o);
    }
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) {
      const int a = ph >> 1, b = ph & 1;
      if (rowok && colok) {
        const int li = el - 1 + a, lj = fl - 1 + b;
        if (li >= 0 && li < TILE && lj >= 0 && lj < TILE && i0 + li < N && j0 + lj < N) {
#pragma unroll
          for (int op = 0; op < 4; ++op) acc[(op * TILE + li) * TILE + lj] += o.v[op][ph];
        }
      }
      __syncthreads();
    }
  }
  zd* outs[4] = {A.S, A.D, A.Dt, A.Nk};
  for (int t = threadIdx.x; t < 4 * TILE * TILE; t += blockDim.x) {
    const int op = t / (TILE * TILE), rem = t - op * TILE * TILE;
    const int li = rem / TILE, lj = rem - (rem / TILE) * TILE;
    if (i0 + li < N && j0 + lj < N) outs[op][(i0 + li) * A.ld + j0 + lj] = acc[t];
  }
}

// Row 0 of the four operators: thread per column j; node 0 gets element
// N-1 (a = 1) and element 0 (a = 0); column j gets elements j-1 (b = 1), j (b = 0).
__global__ void k_circle_row(AsmArgs A) {
  const int64_t N = A.N;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  zd sum[4] = {mkz(0.0), mkz(0.0), mkz(0.0), mkz(0.0)};
  const int64_t es[2] = {N - 1, 0};
  const int as_[2] = {1, 0};
  const int64_t fs[2] = {(j - 1 + N) % N, j};
  const int bs[2] = {1, 0};
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      PairOut o;
      pair_integrals(A, es[u], fs[v], o);
      for (int op = 0; op < 4; ++op) sum[op] += o.v[op][as_[u] * 2 + bs[v]];
    }
  A.S[j] = sum[0];
  A.D[j] = sum[1];
  A.Dt[j] = sum[2];
  A.Nk[j] = sum[3];
}

// Entries (row i, col j): sum of the four element pairs (i-1|i) x (j-1|j).
__global__ void k_entries(AsmArgs A, int64_t count, const int64_t* rows, const int64_t* cols,
                          zd* out4) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t N = A.N, i = rows[t], j = cols[t];
  zd sum[4] = {mkz(0.0), mkz(0.0), mkz(0.0), mkz(0.0)};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int64_t e = (i - a + N) % N, f = (j - b + N) % N;
      PairOut o;
      pair_integrals(A, e, f, o);
      for (int op = 0; op < 4; ++op) sum[op] += o.v[op][a * 2 + b];
    }
  for (int op = 0; op < 4; ++op) out4[op * count + t] = sum[op];
}

static int upload_rules(const AsmArgs& A) {
  double xf[16], wf[16], xn[16], wn[16];
  gauss_legendre01(A.q_far, xf, wf);
  gauss_legendre01(A.q_near, xn, wn);
  if (cudaMemcpyToSymbol(c_xf, xf, sizeof(double) * A.q_far) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_wf, wf, sizeof(double) * A.q_far) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_xn, xn, sizeof(double) * A.q_near) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_wn, wn, sizeof(double) * A.q_near) != cudaSuccess) return 3;
  return 0;
}

int assemble_dense(const AsmArgs& A, cudaStream_t s) {
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  const size_t smem = sizeof(zd) * 4 * TILE * TILE;
  cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t nt = (A.N + TILE - 1) / TILE;
  dim3 grid((unsigned)nt, (unsigned)nt);
  k_assemble<<<grid, ASM_THREADS, smem, s>>>(A);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("assemble: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int assemble_circle_row(const AsmArgs& A, cudaStream_t s) {
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  k_circle_row<<<(unsigned)((A.N + 63) / 64), 64, 0, s>>>(A);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("circle row: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int assemble_entries(const AsmArgs& A, int64_t count, const int64_t* rows, const int64_t* cols,
                     zd* out4, cudaStream_t s) {
  if (count <= 0) return 0;
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  k_entries<<<(unsigned)((count + 63) / 64), 64, 0, s>>>(A, count, rows, cols, out4);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("entries: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

}  // namespace wcs
