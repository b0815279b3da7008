// Plane-wave right-hand sides (Sec. II, Eq. 4) and the far-field map.
//
// exp(-i w t) convention; plane wave of propagation angle phi, d = (cos phi,
// sin phi), phase reference at the origin: H_z^inc = exp(i k d.r) and
// E_t^inc / eta = (d.n) exp(i k d.r).  [h]_i = int l_i H_z^inc,
// [e/eta]_i = int l_i E_t^inc / eta by q-point Gauss on the two elements of
// hat i.  Far field H^s ~ F(phi_o) e^{i k rho} / sqrt(rho),
// F = (i k e^{i pi/4} / sqrt(8 pi k)) int (x.n') e^{-i k x.r'} j ds'.
// Phases are formed and reduced in FP64 (k |r| reaches ~1e4).
#include "internal.h"

namespace wcs {

__constant__ double c_rx[16], c_rw[16];

__global__ void k_planewave(Points P, int q, int64_t N, double h, double k, const double* angles,
                            int B, zd* e, zd* hv, int64_t ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= N) return;
  double ds, dc;
  sincos(angles[b], &ds, &dc);
  zd se = mkz(0.0), sh = mkz(0.0);
  for (int a = 0; a < 2; ++a) {
    const int64_t el = (a == 1) ? (i - 1 + N) % N : i;  // a = 1: hat i is xi on element i-1
    for (int g = 0; g < q; ++g) {
      const int64_t ip = el * q + g;
      const double phi = (a == 1) ? c_rx[g] : 1.0 - c_rx[g];
      const double w = h * c_rw[g] * phi;
      double s, c;
      sincos(k * (dc * P.x[ip] + ds * P.y[ip]), &s, &c);
      const double dn = dc * P.nx[ip] + ds * P.ny[ip];
      sh += mkz(w * c, w * s);
      se += mkz(w * dn * c, w * dn * s);
    }
  }
  e[(int64_t)b * ld + i] = se;
  hv[(int64_t)b * ld + i] = sh;
}

// Mixed form: the phase k d.r is split at a reference point r0 of hat i (its
// first Gauss point on element i): exp(i k d.r0) in FP64, once per angle, and
// exp(i k d.(r - r0)) in FP32, where |k d.(r - r0)| <= 2 k h stays small
// (~1e-7 absolute error).  A thread walks the 2q points of its hat once for
// PW_ANGLES angles.
constexpr int PW_ANGLES = 8;
__global__ void k_planewave_split(Points P, int q, int64_t N, double h, double k, const double* angles,
                                  int B, zd* e, zd* hv, int64_t ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b0 = blockIdx.y * PW_ANGLES;
  if (i >= N) return;
  const int nb = min(PW_ANGLES, B - b0);
  const double x0 = P.x[i * q], y0 = P.y[i * q];
  float dcf[PW_ANGLES], dsf[PW_ANGLES];
  float shr[PW_ANGLES], shi[PW_ANGLES], ser[PW_ANGLES], sei[PW_ANGLES];
#pragma unroll
  for (int a = 0; a < PW_ANGLES; ++a) {
    double sn = 0.0, cs = 1.0;
    if (a < nb) sincos(angles[b0 + a], &sn, &cs);
    dcf[a] = (float)cs;
    dsf[a] = (float)sn;
    shr[a] = shi[a] = ser[a] = sei[a] = 0.f;
  }
  const float kf = (float)k;
  for (int side = 0; side < 2; ++side) {
    const int64_t el = (side == 1) ? (i - 1 + N) % N : i;   // side 1: hat i is xi on element i-1
    for (int g = 0; g < q; ++g) {
      const int64_t ip = el * q + g;
      const float dx = (float)(P.x[ip] - x0), dy = (float)(P.y[ip] - y0);
      const float nx = (float)P.nx[ip], ny = (float)P.ny[ip];
      const float lam = (side == 1) ? (float)c_rx[g] : (float)(1.0 - c_rx[g]);
      const float w = (float)(h * c_rw[g]) * lam;
#pragma unroll
      for (int a = 0; a < PW_ANGLES; ++a) {
        float sn, cs;
        sincosf(kf * (dcf[a] * dx + dsf[a] * dy), &sn, &cs);
        const float dn = w * (dcf[a] * nx + dsf[a] * ny);
        shr[a] = fmaf(w, cs, shr[a]);
        shi[a] = fmaf(w, sn, shi[a]);
        ser[a] = fmaf(dn, cs, ser[a]);
        sei[a] = fmaf(dn, sn, sei[a]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < PW_ANGLES; ++a) {
    if (a >= nb) break;
    double sn, cs;
    sincos(angles[b0 + a], &sn, &cs);
    double ps, pc;
    sincos(k * (cs * x0 + sn * y0), &ps, &pc);
    const zd ph = mkz(pc, ps);
    e[(int64_t)(b0 + a) * ld + i] = ph * mkz((double)ser[a], (double)sei[a]);
    hv[(int64_t)(b0 + a) * ld + i] = ph * mkz((double)shr[a], (double)shi[a]);
  }
}

__global__ void k_farfield_matrix(Points P, int q, int64_t N, double h, double k, const double* phi,
                                  int nphi, zd* E, int64_t lde) {
  const int o = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double os, oc;
  sincos(phi[o], &os, &oc);
  zd acc = mkz(0.0);
  for (int a = 0; a < 2; ++a) {
    const int64_t el = (a == 1) ? (i - 1 + N) % N : i;
    for (int g = 0; g < q; ++g) {
      const int64_t ip = el * q + g;
      const double lam = (a == 1) ? c_rx[g] : 1.0 - c_rx[g];
      const double w = h * c_rw[g] * lam * (oc * P.nx[ip] + os * P.ny[ip]);
      double s, c;
      sincos(-k * (oc * P.x[ip] + os * P.y[ip]), &s, &c);
      acc += mkz(w * c, w * s);
    }
  }
  // i k e^{i pi/4} / sqrt(8 pi k)
  const double amp = k / sqrt(8.0 * WCS_PI * k);
  const zd pre = mkz(-amp * sqrt(0.5), amp * sqrt(0.5));
  E[i * lde + o] = pre * acc;
}

static int upload(const double* xn, const double* wn, int q) {
  if (cudaMemcpyToSymbol(c_rx, xn, sizeof(double) * q) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_rw, wn, sizeof(double) * q) != cudaSuccess) return 3;
  return 0;
}

int planewave_rhs(const Points& near, const double* wn, const double* xn, int q, int64_t N,
                  double h, double k, const double* angles, int B, zd* e, zd* hv, int64_t ld,
                  cudaStream_t s, bool split_phase) {
  if (upload(xn, wn, q)) { set_error("upload rule"); return 3; }
  if (split_phase) {
    for (int b0 = 0; b0 < B; b0 += 65535 * PW_ANGLES) {
      const int bb = std::min(65535 * PW_ANGLES, B - b0);
      dim3 g((unsigned)((N + 127) / 128), (unsigned)((bb + PW_ANGLES - 1) / PW_ANGLES));
      k_planewave_split<<<g, 128, 0, s>>>(near, q, N, h, k, angles + b0, bb, e + (int64_t)b0 * ld,
                                          hv + (int64_t)b0 * ld, ld);
      note_launch();
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) { set_error(std::string("rhs: ") + cudaGetErrorString(err)); return 3; }
    return 0;
  }
  for (int b0 = 0; b0 < B; b0 += 65535) {
    int bb = std::min(65535, B - b0);
    dim3 g((unsigned)((N + 127) / 128), (unsigned)bb);
    k_planewave<<<g, 128, 0, s>>>(near, q, N, h, k, angles + b0, bb, e + (int64_t)b0 * ld,
                                  hv + (int64_t)b0 * ld, ld);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("rhs: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int farfield_matrix(const Points& near, const double* wn, const double* xn, int q, int64_t N,
                    double h, double k, const double* phi, int nphi, zd* E, int64_t lde,
                    cudaStream_t s) {
  if (upload(xn, wn, q)) { set_error("upload rule"); return 3; }
  for (int o0 = 0; o0 < nphi; o0 += 65535) {
    int oo = std::min(65535, nphi - o0);
    dim3 g((unsigned)((N + 127) / 128), (unsigned)oo);
    k_farfield_matrix<<<g, 128, 0, s>>>(near, q, N, h, k, phi + o0, oo, E + o0, lde);
    note_launch();
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("farfield: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

}  // namespace wcs
