// Contour geometry and arc-length mesh (Sec. II, Sec. V of the paper).
//
// gamma is star-shaped, r(theta) = rho(theta)(cos theta, sin theta).  The
// mesh is uniform in arc length (Sec. V): node i sits at s_i = i h, h = L/N,
// node 0 at theta = 0.  Arc length s(theta) is tabulated on P uniform theta
// panels (16-point Gauss-Legendre each, compensated prefix sum); theta(s) is
// found by Newton inside the panel.  Derivatives of rho are analytic per
// family.  Outward normal n = (t_y, -t_x) for counter-clockwise traversal.
#include "internal.h"

namespace wcs {

__constant__ double c_gl16x[16];
__constant__ double c_gl16w[16];

__device__ __forceinline__ void rho_base(const Contour& c, double th, double& r0, double& r1,
                                         double& r2) {
  double sn, cs;
  sincos(th, &sn, &cs);
  switch (c.family) {
    case FAM_CIRCLE:
      r0 = c.a; r1 = 0.0; r2 = 0.0;
      return;
    case FAM_ELLIPSE: {
      // u = cos^2/ax^2 + sin^2/ay^2, rho = u^{-1/2}
      double A = 1.0 / (c.ax * c.ax), B = 1.0 / (c.ay * c.ay);
      double u = A * cs * cs + B * sn * sn;
      double u1 = 2.0 * sn * cs * (B - A);
      double u2 = 2.0 * (cs * cs - sn * sn) * (B - A);
      double r = rsqrt(u);
      r0 = r;
      r1 = -0.5 * r / u * u1;
      r2 = 0.75 * r / (u * u) * u1 * u1 - 0.5 * r / u * u2;
      return;
    }
    case FAM_SUPERELLIPSE: {
      // u = |cos/ax|^p + |sin/ay|^p, rho = u^{-1/p}  (p >= 2)
      double p = c.p;
      double ca = fabs(cs) / c.ax, sa = fabs(sn) / c.ay;
      double cp2 = pow(ca, p - 2.0), sp2 = pow(sa, p - 2.0);
      double cpp = cp2 * ca * ca, spp = sp2 * sa * sa;
      double u = cpp + spp;
      // d/dth |cos/ax|^p = -p sin cos |cos/ax|^{p-2} / ax^2 ; same pattern for sin
      double u1 = p * sn * cs * (-cp2 / (c.ax * c.ax) + sp2 / (c.ay * c.ay));
      double u2 = p * (p - 1.0) * (sn * sn * cp2 / (c.ax * c.ax) + cs * cs * sp2 / (c.ay * c.ay)) -
                  p * u;
      double ip = 1.0 / p;
      double r = pow(u, -ip);
      r0 = r;
      r1 = -ip * r / u * u1;
      r2 = ip * (ip + 1.0) * r / (u * u) * u1 * u1 - ip * r / u * u2;
      return;
    }
    default: {
      // rho = sum c_m cos(m th) + s_m sin(m th), angle-addition recurrence
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      double cm = 1.0, sm = 0.0;
      for (int m = 0; m < c.nf; ++m) {
        double fc = c.fc[m], fsn = c.fs[m];
        a0 += fc * cm + fsn * sm;
        a1 += m * (-fc * sm + fsn * cm);
        a2 -= (double)m * m * (fc * cm + fsn * sm);
        double cn = cm * cs - sm * sn;
        sm = sm * cs + cm * sn;
        cm = cn;
      }
      r0 = a0; r1 = a1; r2 = a2;
      return;
    }
  }
}

// rho and its first two theta-derivatives: the family's own plus the shape
// perturbation sum_m pc_m cos(m th) + ps_m sin(m th) (angle-addition recurrence)
__device__ __forceinline__ void rho_derivs(const Contour& c, double th, double& r0, double& r1,
                                           double& r2) {
  rho_base(c, th, r0, r1, r2);
  if (c.np == 0) return;
  double sn, cs;
  sincos(th, &sn, &cs);
  double cm = 1.0, sm = 0.0;
  for (int m = 0; m < c.np; ++m) {
    const double a = c.pc[m], b = c.ps[m];
    r0 += a * cm + b * sm;
    r1 += m * (-a * sm + b * cm);
    r2 -= (double)m * m * (a * cm + b * sm);
    const double cn = cm * cs - sm * sn;
    sm = sm * cs + cm * sn;
    cm = cn;
  }
}

__device__ __forceinline__ double speed(const Contour& c, double th) {
  double r0, r1, r2;
  rho_derivs(c, th, r0, r1, r2);
  return sqrt(r0 * r0 + r1 * r1);
}

__device__ __forceinline__ double arc_int(const Contour& c, double a, double b) {
  double s = 0.0;
#pragma unroll 4
  for (int g = 0; g < 16; ++g) s += c_gl16w[g] * speed(c, a + (b - a) * c_gl16x[g]);
  return s * (b - a);
}

__global__ void k_panel_lengths(Contour c, int P, double* len) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  double dth = 2.0 * WCS_PI / P;
  len[j] = arc_int(c, j * dth, (j + 1) * dth);
}

__global__ void k_prefix_kahan(const double* len, int P, double* cum) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0, comp = 0.0;
  cum[0] = 0.0;
  for (int j = 0; j < P; ++j) {
    double y = len[j] - comp;
    double t = s + y;
    comp = (t - s) - y;
    s = t;
    cum[j + 1] = s;
  }
}

__device__ void point_at(const Contour& c, const double* cum, int P, double L, double s,
                         double& x, double& y, double& nx, double& ny, double& kap) {
  double th;
  if (c.family == FAM_CIRCLE && c.np == 0) {
    th = s / c.a;
  } else {
    s = s - floor(s / L) * L;
    int lo = 0, hi = P;  // find panel j with cum[j] <= s < cum[j+1]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (cum[mid] <= s) lo = mid; else hi = mid;
    }
    double dth = 2.0 * WCS_PI / P;
    double t0 = lo * dth;
    double ds = s - cum[lo];
    double plen = cum[lo + 1] - cum[lo];
    th = t0 + dth * ds / plen;
    for (int it = 0; it < 8; ++it) {
      double F = arc_int(c, t0, th) - ds;
      double d = F / speed(c, th);
      th -= d;
      if (fabs(d) < 1e-16) break;
    }
  }
  double r0, r1, r2;
  rho_derivs(c, th, r0, r1, r2);
  double sn, cs;
  sincos(th, &sn, &cs);
  x = r0 * cs;
  y = r0 * sn;
  double dx = r1 * cs - r0 * sn, dy = r1 * sn + r0 * cs;
  double sp = sqrt(dx * dx + dy * dy);
  nx = dy / sp;
  ny = -dx / sp;
  kap = (r0 * r0 + 2.0 * r1 * r1 - r0 * r2) / (sp * sp * sp);
}

__global__ void k_points(Contour c, const double* cum, int P, double L, int64_t N, double h,
                         const double* xi, int nq, Points out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * nq) return;
  int64_t e = idx / nq;
  int g = (int)(idx - e * nq);
  double s = ((double)e + xi[g]) * h;
  double x, y, nx, ny, kap;
  point_at(c, cum, P, L, s, x, y, nx, ny, kap);
  out.x[idx] = x; out.y[idx] = y; out.nx[idx] = nx; out.ny[idx] = ny;
  if (out.kappa) out.kappa[idx] = kap;
}

__global__ void k_min_curv(Contour c, const double* cum, int P, double L, int64_t M, double* kmin) {
  __shared__ double red[256];
  double m = 1e300;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    // a dense uniform grid in theta covers the curve as well as one in arc
    // length and needs no arc-length inversion
    const double th = 2.0 * WCS_PI * (double)i / (double)M;
    double r0, r1, r2;
    rho_derivs(c, th, r0, r1, r2);
    const double sp2 = r0 * r0 + r1 * r1;
    m = fmin(m, (r0 * r0 + 2.0 * r1 * r1 - r0 * r2) / (sp2 * sqrt(sp2)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) kmin[blockIdx.x] = red[0];
}

static DeviceOnce g_gl16_ready;   // __constant__ tables are per device

static int ensure_gl16() {
  if (!g_gl16_ready.need()) return 0;
  double x[16], w[16];
  gauss_legendre01(16, x, w);
  if (cudaMemcpyToSymbol(c_gl16x, x, sizeof(x)) != cudaSuccess) return 1;
  if (cudaMemcpyToSymbol(c_gl16w, w, sizeof(w)) != cudaSuccess) return 1;
  g_gl16_ready.done();
  return 0;
}

int arc_table_build(const Contour& c, ArcTable& t, cudaStream_t s) {
  if (ensure_gl16()) { set_error("uploading Gauss-Legendre table failed"); return 3; }
  t.P = 8192;
  double* len = nullptr;
  if (cudaMalloc(&len, sizeof(double) * t.P) != cudaSuccess ||
      cudaMalloc(&t.cum, sizeof(double) * (t.P + 1)) != cudaSuccess) {
    set_error("out of device memory (arc table)");
    return 4;
  }
  k_panel_lengths<<<(t.P + 127) / 128, 128, 0, s>>>(c, t.P, len);
  note_launch();
  k_prefix_kahan<<<1, 32, 0, s>>>(len, t.P, t.cum);
  note_launch();
  double L = 0.0;
  cudaMemcpyAsync(&L, t.cum + t.P, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaError_t err = cudaStreamSynchronize(s);
  cudaFree(len);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  t.L = L;
  return 0;
}

int points_build(const Contour& c, const ArcTable& t, int64_t N, double h, const double* xi_dev,
                 int nq, Points& out, cudaStream_t s) {
  int64_t n = N * nq;
  k_points<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c, t.cum, t.P, t.L, N, h, xi_dev, nq, out);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  return 0;
}

int min_curvature(const Contour& c, const ArcTable& t, int64_t samples, double* kmin,
                  cudaStream_t s) {
  const int blocks = 304;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks) != cudaSuccess) { set_error("oom"); return 4; }
  k_min_curv<<<blocks, 256, 0, s>>>(c, t.cum, t.P, t.L, samples, d);
  note_launch();
  double h[blocks];
  cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t err = cudaStreamSynchronize(s);
  cudaFree(d);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return 3; }
  double m = 1e300;
  for (int i = 0; i < blocks; ++i) m = fmin(m, h[i]);
  *kmin = m;
  return 0;
}

}  // namespace wcs
