// Hankel functions H0^(1), H1^(1) and Bessel J0, J1 for real or complex argument.
//
// Sec. II of the paper fixes the kernel g_k = (i/4) H0^(1)(k |r - r'|); its
// normal derivative needs H1^(1).  The preconditioner of Eq. (5) evaluates the
// same kernels at the complex wavenumber k~ of Sec. III.  Written from the
// published formulas (NIST DLMF):
//   |z| <= 2 : ascending series of J0, J1, Y0, Y1 (DLMF 10.8.1-10.8.3);
//   |z| <= 17: Miller backward recurrence for J_n normalised by
//              J0 + 2 sum J_2k = 1 (DLMF 10.12.4, 3.6), Neumann series for Y0
//              (DLMF 10.23.9) and its derivative for Y1;
//   |z| > 17 : Hankel asymptotic expansion (DLMF 10.17.5), summed until the
//              smallest term.
// Crossovers were chosen so every branch is within ~2e-13 of reference
// values for |arg z| small (the wavenumbers here have Im k~ << Re k~).
#pragma once
#include "common.cuh"

namespace wcs {

struct Hankel01 {
  zd H0, H1;   // H0^(1)(z), H1^(1)(z)
  zd J0, J1;   // J0(z), J1(z)
};

__device__ __forceinline__ zd zexpi_damped(zd z) {
  // exp(i z) = exp(i x) exp(-y); the phase keeps full double accuracy
  double s, c;
  sincos(z.x, &s, &c);
  double m = exp(-z.y);
  return mkz(m * c, m * s);
}

__device__ inline Hankel01 hankel01_series(zd z) {
  // J0 = sum q^m/(m!)^2, J1 = z/2 sum q^m/(m!(m+1)!), q = -z^2/4
  // Y0 = (2/pi)[(log(z/2)+gamma) J0 - sum H_m q^m/(m!)^2]
  // Y1 = -2/(pi z) + (2/pi) log(z/2) J1 - (1/pi)(z/2) sum (psi(m+1)+psi(m+2)) q^m/(m!(m+1)!)
  zd q = -0.25 * (z * z);
  zd t0 = mkz(1.0), t1 = mkz(1.0);
  zd J0 = t0, J1s = t1, S0 = mkz(0.0), T1 = (1.0 - 2.0 * WCS_EULER_GAMMA) * t1;
  double H = 0.0;
  for (int m = 1; m < 40; ++m) {
    t0 = t0 * q * (1.0 / ((double)m * m));
    t1 = t1 * q * (1.0 / ((double)m * (m + 1)));
    H += 1.0 / m;
    J0 += t0;
    J1s += t1;
    S0 -= H * t0;
    T1 += (2.0 * H + 1.0 / (m + 1) - 2.0 * WCS_EULER_GAMMA) * t1;
    if (abs2(t0) < 1e-36 * abs2(J0) && abs2(t1) < 1e-36 * abs2(J1s)) break;
  }
  zd hz = 0.5 * z;
  zd J1 = hz * J1s;
  zd lz = zlog(hz);
  zd Y0 = (2.0 / WCS_PI) * ((lz + mkz(WCS_EULER_GAMMA)) * J0 + S0);
  zd Y1 = (-2.0 / WCS_PI) * zrecip(z) + (2.0 / WCS_PI) * (lz * J1) - (1.0 / WCS_PI) * (hz * T1);
  Hankel01 r;
  r.J0 = J0; r.J1 = J1;
  r.H0 = mkz(J0.x - Y0.y, J0.y + Y0.x);
  r.H1 = mkz(J1.x - Y1.y, J1.y + Y1.x);
  return r;
}

__device__ inline Hankel01 hankel01_miller(zd z) {
  // start index: |z| + 25 is within 1e-14 for |z| < 12, |z| + 45 above
  const double az = zabs(z);
  int n0 = (int)(az + (az < 12.0 ? 25.0 : 45.0));
  n0 += (n0 & 1);
  zd iz2 = 2.0 * zrecip(z);           // 2/z
  zd jp1 = mkz(0.0), j = mkz(1e-30);
  zd norm = mkz(0.0);                 // J0 + 2 sum J_2k (unnormalised)
  zd s0 = mkz(0.0);                   // sum (-1)^k J_2k / k
  zd s1 = mkz(0.0);                   // sum (-1)^k (J_2k-1 - J_2k+1) / k
  zd Jn1 = mkz(0.0);                  // J_{n+1} bookkeeping for s1
  // walk n from n0 down to 0; at each step j = J_n, jp1 = J_{n+1}
  zd J1 = mkz(0.0);
  for (int n = n0; n >= 0; --n) {
    if (n > 0 && (n & 1) == 0) {
      int k = n >> 1;
      double sg = (k & 1) ? -1.0 : 1.0;
      norm += 2.0 * j;
      s0 += (sg / k) * j;
    }
    if ((n & 1) == 1) {
      // J_n with n = 2k-1 contributes (+) to term k = (n+1)/2 and J_n with
      // n = 2k+1 contributes (-) to term k = (n-1)/2
      int kp = (n + 1) >> 1, km = (n - 1) >> 1;
      double sp = (kp & 1) ? -1.0 : 1.0;
      s1 += (sp / kp) * j;
      if (km >= 1) {
        double sm = (km & 1) ? -1.0 : 1.0;
        s1 -= (sm / km) * j;
      }
    }
    if (n == 1) J1 = j;
    if (n == 0) break;
    zd jm = ((double)n * iz2) * j - jp1;
    jp1 = j;
    j = jm;
  }
  (void)Jn1;
  norm += j;                          // + J0
  zd inv = zrecip(norm);
  zd J0 = j * inv;
  J1 = J1 * inv;
  s0 = s0 * inv;
  s1 = s1 * inv;
  zd lz = zlog(0.5 * z) + mkz(WCS_EULER_GAMMA);
  zd Y0 = (2.0 / WCS_PI) * (lz * J0 - 2.0 * s0);
  zd Y1 = (2.0 / WCS_PI) * (lz * J1 - J0 * zrecip(z) + s1);
  Hankel01 r;
  r.J0 = J0; r.J1 = J1;
  r.H0 = mkz(J0.x - Y0.y, J0.y + Y0.x);
  r.H1 = mkz(J1.x - Y1.y, J1.y + Y1.x);
  return r;
}

__device__ inline Hankel01 hankel01_asymptotic(zd z) {
  // H_nu(z) ~ sqrt(2/(pi z)) exp(i(z - nu pi/2 - pi/4)) sum_k (i/z)^k a_k(nu),
  // a_k(nu) = a_{k-1}(nu) (4 nu^2 - (2k-1)^2) / (8k)
  zd w = zrecip(z);
  w = mkz(-w.y, w.x);                 // i / z
  zd s0 = mkz(1.0), s1 = mkz(1.0), t0 = mkz(1.0), t1 = mkz(1.0);
  bool run0 = true, run1 = true;
  for (int k = 1; k < 48 && (run0 || run1); ++k) {
    double o = (double)(2 * k - 1);
    if (run0) {
      zd tn = t0 * w * ((-o * o) / (8.0 * k));
      if (abs2(tn) > abs2(t0)) run0 = false;
      else { t0 = tn; s0 += tn; if (abs2(tn) < 1e-36 * abs2(s0)) run0 = false; }
    }
    if (run1) {
      zd tn = t1 * w * ((4.0 - o * o) / (8.0 * k));
      if (abs2(tn) > abs2(t1)) run1 = false;
      else { t1 = tn; s1 += tn; if (abs2(tn) < 1e-36 * abs2(s1)) run1 = false; }
    }
  }
  // common factor sqrt(2/(pi z)) exp(i (z - pi/4))
  zd amp = zsqrt((2.0 / WCS_PI) * zrecip(z));
  zd e = zexpi_damped(z - mkz(0.25 * WCS_PI));
  zd f = amp * e;
  Hankel01 r;
  r.H0 = f * s0;
  zd h1 = f * s1;
  r.H1 = mkz(h1.y, -h1.x);            // extra factor exp(-i pi/2) = -i
  // J = (H^(1) + H^(2)) / 2 is not needed in this regime
  r.J0 = mkz(0.0); r.J1 = mkz(0.0);
  return r;
}

// Full evaluation.  want_J: also return J0, J1 (only used for small |z|,
// where the log-singular split of the near-field quadrature needs them).
__device__ inline Hankel01 hankel01(zd z) {
  double az = zabs(z);
  if (az <= 2.0) return hankel01_series(z);
  if (az <= 17.0) return hankel01_miller(z);
  return hankel01_asymptotic(z);
}

}  // namespace wcs
