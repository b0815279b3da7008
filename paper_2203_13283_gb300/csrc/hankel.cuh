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

// ---------------------------------------------------------------------------
// Both wavenumbers of a point pair from one real evaluation.  k~ = k + i beta
// (Sec. III) has Re k~ = k, so the two arguments are x = k R and x (1 + i t)
// with t = beta / k.  J0, J1, Y0, Y1 are evaluated at the real x in real
// arithmetic and carried to x + i y (y = x t) by their Taylor series in i y.
// The derivatives follow from Bessel's equation (DLMF 10.2.1) differentiated
// m times,
//     x f^(m+2) = -(m+1) f^(m+1) - x f^(m) - m f^(m-1)      (f = J0 or Y0),
// with J1 = -J0', Y1 = -Y0' (DLMF 10.6.3).  The terms fall like t^m for every
// x (Y0's branch point is at distance x), so the form is used for t <= 0.1.
// Large x uses the Hankel expansion of both with one shared sincos.
// ---------------------------------------------------------------------------
__constant__ double c_recip[72] = {
    0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7,
    1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15,
    1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23,
    1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31,
    1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39,
    1.0 / 40, 1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47,
    1.0 / 48, 1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55,
    1.0 / 56, 1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63,
    1.0 / 64, 1.0 / 65, 1.0 / 66, 1.0 / 67, 1.0 / 68, 1.0 / 69, 1.0 / 70, 1.0 / 71,
};

struct Bessel01 {
  double J0, J1, Y0, Y1;
};

__device__ inline Bessel01 bessel01_series_real(double x) {
  // the ascending series of hankel01_series for real x
  const double q = -0.25 * x * x;
  double t0 = 1.0, t1 = 1.0, J0 = 1.0, J1s = 1.0, S0 = 0.0, T1 = 1.0 - 2.0 * WCS_EULER_GAMMA, H = 0.0;
  for (int m = 1; m < 40; ++m) {
    const double rm = c_recip[m], rm1 = c_recip[m + 1];
    t0 *= q * (rm * rm);
    t1 *= q * (rm * rm1);
    H += rm;
    J0 += t0;
    J1s += t1;
    S0 -= H * t0;
    T1 += (2.0 * H + rm1 - 2.0 * WCS_EULER_GAMMA) * t1;
    if (fabs(t0) < 1e-18 * fabs(J0) && fabs(t1) < 1e-18 * fabs(J1s)) break;
  }
  const double hz = 0.5 * x, lz = log(hz);
  Bessel01 b;
  b.J0 = J0;
  b.J1 = hz * J1s;
  b.Y0 = (2.0 / WCS_PI) * ((lz + WCS_EULER_GAMMA) * J0 + S0);
  b.Y1 = (-2.0 / WCS_PI) / x + (2.0 / WCS_PI) * lz * b.J1 - (1.0 / WCS_PI) * hz * T1;
  return b;
}

__device__ inline Bessel01 bessel01_miller_real(double x) {
  // the backward recurrence of hankel01_miller for real x; the threads that
  // run this branch together start at their largest index, which keeps the
  // loop (and the reciprocal-table reads) uniform across the warp
  int n0 = (int)(x + (x < 12.0 ? 25.0 : 45.0));
  n0 += (n0 & 1);
  n0 = __reduce_max_sync(__activemask(), n0);
  const double iz2 = 2.0 / x;
  double jp1 = 0.0, j = 1e-30, norm = 0.0, s0 = 0.0, s1 = 0.0, J1 = 0.0;
  for (int n = n0; n > 0; --n) {
    if ((n & 1) == 0) {
      const int k = n >> 1;
      const double r = (k & 1) ? -c_recip[k] : c_recip[k];
      norm += 2.0 * j;
      s0 += r * j;
    } else {
      const int kp = (n + 1) >> 1, km = (n - 1) >> 1;
      s1 += ((kp & 1) ? -c_recip[kp] : c_recip[kp]) * j;
      if (km >= 1) s1 -= ((km & 1) ? -c_recip[km] : c_recip[km]) * j;
      if (n == 1) J1 = j;
    }
    const double jm = ((double)n * iz2) * j - jp1;
    jp1 = j;
    j = jm;
  }
  norm += j;
  const double inv = 1.0 / norm;
  Bessel01 b;
  b.J0 = j * inv;
  b.J1 = J1 * inv;
  const double lz = log(0.5 * x) + WCS_EULER_GAMMA;
  b.Y0 = (2.0 / WCS_PI) * (lz * b.J0 - 2.0 * (s0 * inv));
  b.Y1 = (2.0 / WCS_PI) * (lz * b.J1 - b.J0 * (0.5 * iz2) + s1 * inv);
  return b;
}

// J0, J1, Y0, Y1 at z = x + i y from their values at x (Taylor series in i y)
__device__ inline Hankel01 bessel01_shift(double x, double y, const Bessel01& b) {
  const double ix = 1.0 / x;
  double fm1 = 0.0, f0 = b.J0, f1 = -b.J1;   // J0^(m-1), J0^(m), J0^(m+1)
  double gm1 = 0.0, g0 = b.Y0, g1 = -b.Y1;   // same for Y0
  zd J0 = mkz(b.J0), J1 = mkz(b.J1), Y0 = mkz(b.Y0), Y1 = mkz(b.Y1);
  zd c = mkz(1.0);                           // (i y)^(m+1) / (m+1)! after the update
  for (int m = 0; m < 64; ++m) {
    const double f2 = -((double)(m + 1) * f1 + x * f0 + (double)m * fm1) * ix;
    const double g2 = -((double)(m + 1) * g1 + x * g0 + (double)m * gm1) * ix;
    c = mkz(-c.y * y, c.x * y) * c_recip[m + 1];
    J0 += c * f1;
    Y0 += c * g1;
    J1 -= c * f2;
    Y1 -= c * g2;
    fm1 = f0; f0 = f1; f1 = f2;
    gm1 = g0; g0 = g1; g1 = g2;
    const double tm = (fabs(c.x) + fabs(c.y)) * (fabs(f0) + fabs(g0) + fabs(f1) + fabs(g1));
    const double vm = fabs(J0.x) + fabs(J0.y) + fabs(Y0.x) + fabs(Y0.y) + fabs(J1.x) + fabs(J1.y) +
                      fabs(Y1.x) + fabs(Y1.y);
    if (m >= 1 && tm < 1e-17 * vm) break;
  }
  Hankel01 r;
  r.J0 = J0; r.J1 = J1;
  r.H0 = mkz(J0.x - Y0.y, J0.y + Y0.x);
  r.H1 = mkz(J1.x - Y1.y, J1.y + Y1.x);
  return r;
}

// Hankel expansion (DLMF 10.17.5) at x and at x (1 + i t) sharing sin/cos of
// x - pi/4: exp(i(z - pi/4)) = exp(i(x - pi/4)) exp(-x t),
// sqrt(2/(pi z)) = sqrt(2/(pi x)) (1 + i t)^(-1/2), i/z = (i/x) / (1 + i t).
__device__ inline void hankel01_asymptotic_pair(double x, const KtPair& kp, Hankel01& hk, Hankel01& ht) {
  const double ix = 1.0 / x;
  const zd w = mkz(0.0, ix);                          // i / x
  const zd wt = mkz(-kp.c1.y * ix, kp.c1.x * ix);     // i / z
  zd s0 = mkz(1.0), s1 = mkz(1.0), t0 = mkz(1.0), t1 = mkz(1.0);
  zd u0 = mkz(1.0), u1 = mkz(1.0), v0 = mkz(1.0), v1 = mkz(1.0);
  bool r0 = true, r1 = true, q0 = true, q1 = true;
  for (int k = 1; k < 48 && (r0 || r1 || q0 || q1); ++k) {
    const double o = (double)(2 * k - 1);
    const double a0 = (-o * o) * (0.125 * c_recip[k]), a1 = (4.0 - o * o) * (0.125 * c_recip[k]);
    if (r0) {
      const zd tn = t0 * w * a0;
      if (abs2(tn) > abs2(t0)) r0 = false;
      else { t0 = tn; s0 += tn; if (abs2(tn) < 1e-36 * abs2(s0)) r0 = false; }
    }
    if (r1) {
      const zd tn = t1 * w * a1;
      if (abs2(tn) > abs2(t1)) r1 = false;
      else { t1 = tn; s1 += tn; if (abs2(tn) < 1e-36 * abs2(s1)) r1 = false; }
    }
    if (q0) {
      const zd tn = v0 * wt * a0;
      if (abs2(tn) > abs2(v0)) q0 = false;
      else { v0 = tn; u0 += tn; if (abs2(tn) < 1e-36 * abs2(u0)) q0 = false; }
    }
    if (q1) {
      const zd tn = v1 * wt * a1;
      if (abs2(tn) > abs2(v1)) q1 = false;
      else { v1 = tn; u1 += tn; if (abs2(tn) < 1e-36 * abs2(u1)) q1 = false; }
    }
  }
  double sn, cs;
  sincos(x - 0.25 * WCS_PI, &sn, &cs);
  const double amp = sqrt((2.0 / WCS_PI) * ix);
  const zd f = mkz(amp * cs, amp * sn);
  const zd ft = (f * kp.c2) * exp(-x * kp.t);
  hk.H0 = f * s0;
  zd h1 = f * s1;
  hk.H1 = mkz(h1.y, -h1.x);
  ht.H0 = ft * u0;
  h1 = ft * u1;
  ht.H1 = mkz(h1.y, -h1.x);
  hk.J0 = hk.J1 = ht.J0 = ht.J1 = mkz(0.0);
}

// The same expansion with a fixed number of terms for x >= 20, where 20
// terms (k = 0..19) leave a relative truncation error below 4e-16 for both
// orders and both arguments.  Even and odd powers of u = 1/x are summed by
// Horner's rule in u^2 with per-run coefficient tables: (-1)^m a_k(nu) for the
// real argument and (-1)^m a_k(nu) (1 + i t)^-k for x (1 + i t).  The first
// omitted term of a sum of 2M terms is a_2M(nu) / x^2M, so larger x needs
// fewer terms: KtPair::xth[] holds, for M = 2, 3, 4, 5, 7, the smallest x at
// which that term is below the run's tolerance (1e-16 for the FP64 form, 1e-13
// for the mixed form, whose entries are stored to 24 bits).

template <int M>
__device__ __forceinline__ void asym_sums(double u, double u2, const KtPair& kp, zd (&S)[2], zd (&St)[2]) {
#pragma unroll
  for (int nu = 0; nu < 2; ++nu) {
    double e = kp.asym.re[nu][M - 1], o = kp.asym.ro[nu][M - 1];
    zd ce = kp.asym.ce[nu][M - 1], co = kp.asym.co[nu][M - 1];
#pragma unroll
    for (int m = M - 2; m >= 0; --m) {
      e = fma(e, u2, kp.asym.re[nu][m]);
      o = fma(o, u2, kp.asym.ro[nu][m]);
      ce = mkz(fma(ce.x, u2, kp.asym.ce[nu][m].x), fma(ce.y, u2, kp.asym.ce[nu][m].y));
      co = mkz(fma(co.x, u2, kp.asym.co[nu][m].x), fma(co.y, u2, kp.asym.co[nu][m].y));
    }
    S[nu] = mkz(e, u * o);                             // sum a_k (i u)^k
    St[nu] = mkz(ce.x - u * co.y, ce.y + u * co.x);    // sum a_k (i u / (1 + i t))^k
  }
}

__device__ inline void hankel01_asymptotic_fixed(double x, const KtPair& kp, Hankel01& hk, Hankel01& ht) {
  const double u = 1.0 / x, u2 = u * u;
  zd S[2], St[2];
  if (x >= kp.xth[0]) asym_sums<2>(u, u2, kp, S, St);
  else if (x >= kp.xth[1]) asym_sums<3>(u, u2, kp, S, St);
  else if (x >= kp.xth[2]) asym_sums<4>(u, u2, kp, S, St);
  else if (x >= kp.xth[3]) asym_sums<5>(u, u2, kp, S, St);
  else if (x >= kp.xth[4]) asym_sums<7>(u, u2, kp, S, St);
  else asym_sums<ASYM_M>(u, u2, kp, S, St);
  double sn, cs;
  sincos(x - 0.25 * WCS_PI, &sn, &cs);
  const double amp = sqrt((2.0 / WCS_PI) * u);
  const zd f = mkz(amp * cs, amp * sn);
  const zd ft = (f * kp.c2) * exp(-x * kp.t);
  hk.H0 = f * S[0];
  zd h1 = f * S[1];
  hk.H1 = mkz(h1.y, -h1.x);
  ht.H0 = ft * St[0];
  h1 = ft * St[1];
  ht.H1 = mkz(h1.y, -h1.x);
  hk.J0 = hk.J1 = ht.J0 = ht.J1 = mkz(0.0);
}

// The same expansion for the point pairs of one far element pair whose phase
// and damping were evaluated once at a reference argument x0 (the element
// reference points): exp(i(x - pi/4)) = exp(i(x0 - pi/4)) exp(i dl) and
// exp(-x t) = exp(-x0 t) exp(-dl t) with dl = x - x0, |dl| <= 1.05 (the caller
// takes this route only when k h <= 1.2 and t <= 0.019); exp(i dl) by its
// Taylor series to dl^19 (first omitted term below 2e-17), exp(-dl t) by its
// series to (dl t)^8 (|dl t| <= 0.02, omitted term below 1e-21).  rs = x^-1/2
// supplies both u = 1/x and the amplitude.
__device__ inline void hankel01_asymptotic_rot(double x, double rs, double x0, zd ph0, double damp0,
                                               const KtPair& kp, Hankel01& hk, Hankel01& ht) {
  const double u = rs * rs, u2 = u * u;
  zd S[2], St[2];
  if (x >= kp.xth[0]) asym_sums<2>(u, u2, kp, S, St);
  else if (x >= kp.xth[1]) asym_sums<3>(u, u2, kp, S, St);
  else if (x >= kp.xth[2]) asym_sums<4>(u, u2, kp, S, St);
  else if (x >= kp.xth[3]) asym_sums<5>(u, u2, kp, S, St);
  else if (x >= kp.xth[4]) asym_sums<7>(u, u2, kp, S, St);
  else asym_sums<ASYM_M>(u, u2, kp, S, St);
  const double dl = x - x0, d2 = dl * dl;
  double c = -1.5619206968586225e-16;
  c = fma(c, d2, 4.779477332387385e-14);
  c = fma(c, d2, -1.1470745597729725e-11);
  c = fma(c, d2, 2.08767569878681e-09);
  c = fma(c, d2, -2.755731922398589e-07);
  c = fma(c, d2, 2.48015873015873e-05);
  c = fma(c, d2, -0.001388888888888889);
  c = fma(c, d2, 0.041666666666666664);
  c = fma(c, d2, -0.5);
  c = fma(c, d2, 1.0);
  double sn = 2.8114572543455206e-15;
  sn = fma(sn, d2, -7.647163731819816e-13);
  sn = fma(sn, d2, 1.6059043836821613e-10);
  sn = fma(sn, d2, -2.505210838544172e-08);
  sn = fma(sn, d2, 2.7557319223985893e-06);
  sn = fma(sn, d2, -0.0001984126984126984);
  sn = fma(sn, d2, 0.008333333333333333);
  sn = fma(sn, d2, -0.16666666666666666);
  sn = fma(sn, d2, 1.0);
  sn *= dl;
  const zd ph = ph0 * mkz(c, sn);
  const double amp = 0.79788456080286541 * rs;          // sqrt(2 / pi) x^-1/2
  const zd f = mkz(amp * ph.x, amp * ph.y);
  const double z = -dl * kp.t;   // |z| <= 0.02: sum z^j / j! to j = 8 (omitted term < 1e-21)
  double e = 2.48015873015873e-05;
  e = fma(e, z, 0.0001984126984126984);
  e = fma(e, z, 0.001388888888888889);
  e = fma(e, z, 0.008333333333333333);
  e = fma(e, z, 0.041666666666666664);
  e = fma(e, z, 0.16666666666666666);
  e = fma(e, z, 0.5);
  e = fma(e, z, 1.0);
  e = fma(e, z, 1.0);
  const double dmp = damp0 * e;
  const zd ft = (f * kp.c2) * dmp;
  hk.H0 = f * S[0];
  zd h1 = f * S[1];
  hk.H1 = mkz(h1.y, -h1.x);
  ht.H0 = ft * St[0];
  h1 = ft * St[1];
  ht.H1 = mkz(h1.y, -h1.x);
  hk.J0 = hk.J1 = ht.J0 = ht.J1 = mkz(0.0);
}

// H0, H1 (and J0, J1 below the expansion range) at k R = x and at k~ R
__device__ inline void hankel01_pair(double x, const KtPair& kp, Hankel01& hk, Hankel01& ht) {
  if (x >= 20.0) { hankel01_asymptotic_fixed(x, kp, hk, ht); return; }
  if (x > 17.0) { hankel01_asymptotic_pair(x, kp, hk, ht); return; }
  const Bessel01 b = (x <= 2.0) ? bessel01_series_real(x) : bessel01_miller_real(x);
  hk.J0 = mkz(b.J0);
  hk.J1 = mkz(b.J1);
  hk.H0 = mkz(b.J0, b.Y0);
  hk.H1 = mkz(b.J1, b.Y1);
  ht = bessel01_shift(x, x * kp.t, b);
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
