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
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

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

// Hankel functions at k R and k~ R
__device__ __forceinline__ void hankel_k_kt(const AsmArgs& A, double R, Hankel01& Hk, Hankel01& Ht) {
  if (A.kt_pair) {
    hankel01_pair(A.k * R, A.ktp, Hk, Ht);
  } else {
    Hk = hankel01(mkz(A.k * R));
    Ht = hankel01(A.kt * R);
  }
}

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
    // Element pairs whose point pairs all lie in the expansion range share
    // the phase and damping of the expansion, evaluated once at the
    // reference argument x0 = k |c_e - c_f| (c: mean of the element's
    // points, every point within 0.45 h of it, so |k R - x0| <= 0.9 k h).
    bool rot = false;
    double x0 = 0.0, damp0 = 0.0;
    zd ph0 = mkz(0.0);
    if (A.kt_pair && A.rot_ok) {
      double cex = 0.0, cey = 0.0, cfx = 0.0, cfy = 0.0;
      for (int p = 0; p < q; ++p) {
        cex += A.far.x[e * q + p];
        cey += A.far.y[e * q + p];
        cfx += A.far.x[f * q + p];
        cfy += A.far.y[f * q + p];
      }
      const double iq = 1.0 / (double)q;
      const double ddx = (cex - cfx) * iq, ddy = (cey - cfy) * iq;
      x0 = k * sqrt(ddx * ddx + ddy * ddy);
      if (x0 >= 20.0 + k * h) {
        rot = true;
        double s0, c0;
        sincos(x0 - 0.25 * WCS_PI, &s0, &c0);
        ph0 = mkz(c0, s0);
        damp0 = exp(-x0 * A.ktp.t);
      }
    }
    for (int p = 0; p < q; ++p) {
      const int64_t ip = e * q + p;
      const double xt = A.far.x[ip], yt = A.far.y[ip], nxt = A.far.nx[ip], nyt = A.far.ny[ip];
      const double xip = c_xf[p], wp = c_wf[p];
      for (int r = 0; r < q; ++r) {
        const int64_t ir = f * q + r;
        const double dx = xt - A.far.x[ir], dy = yt - A.far.y[ir];
        const double nxs = A.far.nx[ir], nys = A.far.ny[ir];
        const double nd = nxt * nxs + nyt * nys;
        Hankel01 Hk, Ht;
        double R, gg;
        if (rot) {
          // one reciprocal square root each for 1/R and for (k R)^-1/2
          const double R2 = dx * dx + dy * dy;
          const double ri = rsqrt(R2);
          R = R2 * ri;
          gg = (dx * nxs + dy * nys) * ri;
          const double x = k * R;
          hankel01_asymptotic_rot(x, rsqrt(x), x0, ph0, damp0, A.ktp, Hk, Ht);
        } else {
          R = sqrt(dx * dx + dy * dy);
          gg = (dx * nxs + dy * nys) / R;
          hankel_k_kt(A, R, Hk, Ht);
        }
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
          Hankel01 Hk, Ht;
          hankel_k_kt(A, R, Hk, Ht);
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


// ---------------------------------------------------------------------------
// Far element pairs in the mixed form.  With element centres c_e, c_f and
// point offsets o = r - c (|o| < h), R = |d0 + o_p - o_r| with d0 = c_e - c_f:
// R0 = |d0| and the phase k R0 mod 2 pi are formed in float-float once per
// pair; R - R0 = (2 d0.(o_p - o_r) + |o_p - o_r|^2) / (R + R0) is small, so
// the phase k R = (k R0 mod 2 pi) + k (R - R0) keeps ~1e-7 absolute accuracy
// even for k R ~ 1e4.  The Hankel functions use the large-argument expansion
// (DLMF 10.17.5) with ten terms (z >= 9 gives < 1e-7), for k and for
// k~ = k + i beta (exp(i k~ R) = exp(i k R - beta R)).
//
// Roundings that repeat identically in every element pair act like one
// perturbation of the whole operator and are not averaged out: the products
// of quadrature weights and hat values, the wavenumber constants, the point
// offsets and the normals.  So the weights come from float-float tables
// (the tensor rule is separable: an inner sum over the source points r with
// weights w_r phi_b(xi_r), an outer sum over the target points p with
// w_p phi_a(xi_p)), offsets and normals carry float-float tails, and every
// constant factor of a kernel is left out of the FP32 sums and applied in
// FP64 when the entry is stored (AsmArgs::fS .. fN, kk2h2).  What remains in
// FP32 varies from pair to pair (the rounding of R, the Hankel series, the
// sums), so its effect on the solution averages down.
// ---------------------------------------------------------------------------
__constant__ float c_a0[10], c_a1[10];   // a_k(0), a_k(1) of the Hankel expansion
__constant__ float c_fwt[2][16][2];      // w_r phi_b(xi_r) as float-float [b][r][hi, lo]
__constant__ float c_fw[16][2];          // w_r as float-float

struct cf {
  float x, y;
};
__device__ __forceinline__ cf cmul(cf a, cf b) { return {fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)}; }
__device__ __forceinline__ cf cscale(cf a, float s) { return {a.x * s, a.y * s}; }
// acc += (hi + lo) v, the small term first
__device__ __forceinline__ void cfma2(cf& acc, float hi, float lo, cf v) {
  acc.x = fmaf(hi, v.x, fmaf(lo, v.x, acc.x));
  acc.y = fmaf(hi, v.y, fmaf(lo, v.y, acc.y));
}
__device__ __forceinline__ void cadd(cf& acc, cf v) { acc.x += v.x; acc.y += v.y; }

// Reduced sums of one element pair, [a * 2 + b]:
//   0  S~ / fS     1  D / fD     2  D~ / fD~
//   3  N, k^2 h^2 (n.n') part     4  N, derivative part (signs s_a s_b applied)
// with N = fN (v[4] - k^2 h^2 v[3]).
struct PairOutF {
  cf v[5][4];
};

__device__ void pair_fast_f(const AsmArgs& A, int64_t e, int64_t f, PairOutF& out);

__device__ __forceinline__ zd zf2d(cf a) { return mkz((double)a.x, (double)a.y); }

// The four operators of a far pair from the reduced FP32 sums (FP64 factors).
__device__ void pair_fast(const AsmArgs& A, int64_t e, int64_t f, PairOut& out) {
  PairOutF o;
  pair_fast_f(A, e, f, o);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    out.v[0][j] = A.fS * zf2d(o.v[0][j]);
    out.v[1][j] = A.fD * zf2d(o.v[1][j]);
    out.v[2][j] = A.fDt * zf2d(o.v[2][j]);
    out.v[3][j] = A.fN * (zf2d(o.v[4][j]) - A.kk2h2 * zf2d(o.v[3][j]));
  }
}

// Float-float arithmetic (value = hi + lo, ~48 bits; Dekker/Knuth error-free
// transformations).  The far-pair phase k |c_e - c_f| mod 2 pi needs ~1e-7
// absolute accuracy at k R ~ 2e4; float-float gives ~1e-10 without touching
// the FP64 pipe, which runs at 1/64 of the FP32 rate on this GPU.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_quick(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_quick(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  return ff_quick(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  // one Newton step from the FP32 root: x + (a - x^2) / (2x)
  const float x = sqrtf(a.hi);
  const ff d = ff_add(a, ff_neg(ff_two_prod(x, x)));
  return ff_quick(x, d.hi * (0.5f / x));
}

__device__ void pair_fast_f(const AsmArgs& A, int64_t e, int64_t f, PairOutF& out) {
  const int q = A.q_far;
  const FastConsts& F = A.fk;
  const float4 ce = A.cff[e], cf_ = A.cff[f];   // (x hi, x lo, y hi, y lo)
  const ff dx = ff_add(ff_two_sum(ce.x, -cf_.x), ff_two_sum(ce.y, -cf_.y));
  const ff dy = ff_add(ff_two_sum(ce.z, -cf_.z), ff_two_sum(ce.w, -cf_.w));
  const ff R0 = ff_sqrt(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)));
  const ff kR0 = ff_mul({F.k_hi, F.k_lo}, R0);
  // kR0 - n 2pi with 2pi = t1 + t2 + t3 (24 + 24 + 24 bits); n < 2^13 so n t1, n t2 are exact products
  const float n = rintf(kR0.hi * 0.15915494309189535f);
  ff t = ff_add(kR0, ff_neg(ff_two_prod(n, F.twopi[0])));
  t = ff_add(t, ff_neg(ff_two_prod(n, F.twopi[1])));
  // ph0 = k R0 - pi/4 reduced, kept in float-float (|ph0| <= 5 pi / 4);
  // -pi/4 = -0.785398185 + 2.18556941e-8 (float head, float tail)
  const ff ph0 = ff_add(ff_add(t, {-n * F.twopi[2], 0.f}), {-0.785398185f, 2.18556941e-08f});
  const float fdx0 = dx.hi, fdy0 = dy.hi, fR0 = R0.hi;
  const ff twoR0 = {2.f * R0.hi, 2.f * R0.lo};
  const ff kff = {F.k_hi, F.k_lo};
  const float ldx0 = dx.lo, ldy0 = dy.lo;
  const float k = F.kf, beta = F.beta, beta_lo = F.beta_lo;
  const cf ik = {F.ik[0], F.ik[1]};      // i / k~
  cf vS[4], vD[4], vDt[4], vNb[4], vNd = {0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 4; ++j) vS[j] = vD[j] = vDt[j] = vNb[j] = cf{0.f, 0.f};
  for (int p = 0; p < q; ++p) {
    const int64_t ip = e * q + p;
    const float oxp = A.ox[ip], oyp = A.oy[ip], oxlp = A.oxl[ip], oylp = A.oyl[ip];
    const float nxt = A.nxf[ip], nyt = A.nyf[ip], nxtl = A.nxl[ip], nytl = A.nyl[ip];
    cf uS[2], uD[2], uDt[2], uNb[2], uNd = {0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 2; ++b) uS[b] = uD[b] = uDt[b] = uNb[b] = cf{0.f, 0.f};
    for (int r = 0; r < q; ++r) {
      const int64_t ir = f * q + r;
      // D = o_p - o_r in float-float (the offsets' tails included)
      ff Dx = ff_two_sum(oxp, -A.ox[ir]), Dy = ff_two_sum(oyp, -A.oy[ir]);
      Dx = ff_quick(Dx.hi, Dx.lo + (oxlp - A.oxl[ir]));
      Dy = ff_quick(Dy.hi, Dy.lo + (oylp - A.oyl[ir]));
      const float nxs = A.nxf[ir], nys = A.nyf[ir], nxsl = A.nxl[ir], nysl = A.nyl[ir];
      const float a = 2.f * (fdx0 * Dx.hi + fdy0 * Dy.hi) + Dx.hi * Dx.hi + Dy.hi * Dy.hi;
      const float R = sqrtf(fR0 * fR0 + a);
      const float iR = 1.f / R;
      // n . n' with the normals' tails (a rounded normal would repeat in every pair of its point)
      const float nd = fmaf(nxt, nxs, nyt * nys) + (fmaf(nxtl, nxs, nxt * nxsl) + fmaf(nytl, nys, nyt * nysl));
      // phase k R - pi/4 = ph0 + k (R - R0) in float-float: R - R0 = a / (2 R0 + (R - R0))
      // with a = 2 d0.D + |D|^2 from error-free products; the denominator
      // takes the FP32 estimate of R - R0, whose error enters only relative to 2 R0
      // (r - r').n' in float-float: on the flat parts of a contour it cancels to
      // ~curvature R^2, far below the FP32 rounding of its terms (~6e-8 R)
      const ff rx = ff_add(ff{fdx0, ldx0}, Dx), ry = ff_add(ff{fdy0, ldy0}, Dy);
      const ff dn = ff_add(ff_mul(rx, ff{nxs, nxsl}), ff_mul(ry, ff{nys, nysl}));
      const float gg = (dn.hi + dn.lo) * iR;
      const ff a_ff = ff_add(ff_add(ff_add(ff_two_prod(2.f * Dx.hi, fdx0), ff_two_prod(2.f * Dy.hi, fdy0)),
                                    ff_add(ff_two_prod(Dx.hi, Dx.hi), ff_two_prod(Dy.hi, Dy.hi))),
                             ff{2.f * (Dx.hi * ldx0 + Dy.hi * ldy0 + Dx.lo * (fdx0 + Dx.hi) + Dy.lo * (fdy0 + Dy.hi)),
                                0.f});
      const ff den = ff_add(twoR0, ff{a / (fR0 + R), 0.f});
      const float q0 = a_ff.hi / den.hi;
      const ff rem = ff_add(a_ff, ff_neg(ff_mul(ff{q0, 0.f}, den)));
      const ff th = ff_add(ph0, ff_mul(kff, ff_quick(q0, rem.hi / den.hi)));
      float sn, cs;
      sincosf(th.hi, &sn, &cs);
      const float sq = sqrtf(iR);
      // e^{i(kR - pi/4)} / sqrt(R)
      const cf E1 = {fmaf(-sn, th.lo, cs) * sq, fmaf(cs, th.lo, sn) * sq};
      // real wavenumber: P + iQ = sum (i t)^k a_k, t = 1/(kR)
      const float tt = iR / k, t2 = tt * tt;
      float P0 = c_a0[8], Q0 = c_a0[9], P1 = c_a1[8], Q1 = c_a1[9];
#pragma unroll
      for (int m = 3; m >= 0; --m) {
        P0 = fmaf(-t2, P0, c_a0[2 * m]);
        Q0 = fmaf(-t2, Q0, c_a0[2 * m + 1]);
        P1 = fmaf(-t2, P1, c_a1[2 * m]);
        Q1 = fmaf(-t2, Q1, c_a1[2 * m + 1]);
      }
      Q0 *= tt;
      Q1 *= tt;
      const cf H0 = cmul(E1, {P0, Q0});                         // H0(kR) / sqrt(2 / (pi k))
      const cf H1g = cscale(cmul(E1, {Q1, -P1}), gg);           // H1(kR) gg / sqrt(2 / (pi k))
      // complex wavenumber: w = i/(k~ R)
      const cf w = cscale(ik, iR);
      cf s0 = {c_a0[9], 0.f}, s1 = {c_a1[9], 0.f};
#pragma unroll
      for (int m = 8; m >= 0; --m) {
        s0 = cmul(s0, w); s0.x += c_a0[m];
        s1 = cmul(s1, w); s1.x += c_a1[m];
      }
      // exp(-Im k~ R); expf, not the fast intrinsic: its error grows with |beta R| (up to ~12 here)
      const float damp = expf(-beta * R) * fmaf(-beta_lo, R, 1.f);
      const cf Et = cscale(E1, damp);
      const cf Ht0 = cmul(Et, s0);                              // H0(k~R) / sqrt(2 / (pi k~))
      const cf Ht1g = cscale(cmul(Et, {s1.y, -s1.x}), gg);      // H1(k~R) gg / sqrt(2 / (pi k~))
      const cf HN = cscale(H0, nd);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float wh = c_fwt[b][r][0], wl = c_fwt[b][r][1];
        cfma2(uS[b], wh, wl, Ht0);
        cfma2(uD[b], wh, wl, H1g);
        cfma2(uDt[b], wh, wl, Ht1g);
        cfma2(uNb[b], wh, wl, HN);
      }
      cfma2(uNd, c_fw[r][0], c_fw[r][1], H0);
    }
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      const float wh = c_fwt[aa][p][0], wl = c_fwt[aa][p][1];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        cfma2(vS[aa * 2 + b], wh, wl, uS[b]);
        cfma2(vD[aa * 2 + b], wh, wl, uD[b]);
        cfma2(vDt[aa * 2 + b], wh, wl, uDt[b]);
        cfma2(vNb[aa * 2 + b], wh, wl, uNb[b]);
      }
    }
    cfma2(vNd, c_fw[p][0], c_fw[p][1], uNd);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    out.v[0][j] = vS[j];
    out.v[1][j] = vD[j];
    out.v[2][j] = vDt[j];
    out.v[3][j] = vNb[j];
    // derivative part of the Maue form: phi_a' phi_b' h^2 = s_a s_b, + on the diagonal of the 2x2 block
    out.v[4][j] = (j == 0 || j == 3) ? vNd : cf{-vNd.x, -vNd.y};
  }
}

__device__ __forceinline__ bool fast_ok(const AsmArgs& A, int64_t e, int64_t f) {
  if (periodic_dist(e, f, A.N) <= A.near_band) return false;
  const float4 ce = A.cff[e], cf_ = A.cff[f];
  const float dx0 = ce.x - cf_.x, dy0 = ce.z - cf_.z;
  return A.fk.kf * A.fk.kf * (dx0 * dx0 + dy0 * dy0) >= A.fk.zfast2;
}

__device__ __forceinline__ void pair_any(const AsmArgs& A, int64_t e, int64_t f, PairOut& o) {
  if (A.mixed && fast_ok(A, e, f)) { pair_fast(A, e, f, o); return; }
  pair_integrals(A, e, f, o);
}

__device__ __forceinline__ void split_store(double x, int planes, uint16_t* const* P, int64_t off);

constexpr int TILE = 32;
constexpr int ASM_THREADS = 256;

template <int MIXED>
__global__ void __launch_bounds__(ASM_THREADS) k_assemble(AsmArgs A) {
  extern __shared__ zd acc[];  // [4][TILE][TILE]
  const int64_t N = A.N;
  const int64_t i0 = (int64_t)blockIdx.y * TILE, j0 = (int64_t)blockIdx.x * TILE;
  if (MIXED && A.tile_flags && !A.tile_flags[(int64_t)blockIdx.y * gridDim.x + blockIdx.x]) return;
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
      if (MIXED) pair_any(A, e, f, o); else pair_integrals(A, e, f, o);
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
  if constexpr (!MIXED) {
    zd* outs[4] = {A.S, A.D, A.Dt, A.Nk};
    for (int t = threadIdx.x; t < 4 * TILE * TILE; t += blockDim.x) {
      const int op = t / (TILE * TILE), rem = t - op * TILE * TILE;
      const int li = rem / TILE, lj = rem - (rem / TILE) * TILE;
      if (i0 + li < N && j0 + lj < N) outs[op][(i0 + li) * A.ld + j0 + lj] = acc[t];
    }
  } else {
  // planes: layout 0 row i0+li holds (re, im) of column j0+lj at 2(j0+lj);
  // layout 1 (transpose) row j0+lj holds entry (i0+li, j0+lj) at 2(i0+li)
  for (int t = threadIdx.x; t < 4 * TILE * TILE * 2; t += blockDim.x) {
    const int comp = t & 1;
    const int u = t >> 1;
    const int op = u / (TILE * TILE), rem = u - op * TILE * TILE;
    const int li = rem / TILE, lj = rem - (rem / TILE) * TILE;
    if (i0 + li < N && j0 + lj < N) {
      const zd v = acc[(op * TILE + li) * TILE + lj];
      const double x = comp ? v.y : v.x;
      split_store(x, A.planes, A.P[op][0], (i0 + li) * A.ldp + 2 * (j0 + lj) + comp);
    }
  }
  for (int t = threadIdx.x; t < 4 * TILE * TILE * 2; t += blockDim.x) {
    const int comp = t & 1;
    const int u = t >> 1;
    const int op = u / (TILE * TILE), rem = u - op * TILE * TILE;
    const int lj = rem / TILE, li = rem - (rem / TILE) * TILE;   // consecutive threads walk i
    if (i0 + li < N && j0 + lj < N) {
      const zd v = acc[(op * TILE + li) * TILE + lj];
      const double x = comp ? v.y : v.x;
      split_store(x, A.planes, A.P[op][1], (j0 + lj) * A.ldp + 2 * (i0 + li) + comp);
    }
  }
  }
}

// Row 0 of the four operators: node 0 gets element N-1 (a = 1) and element 0
// (a = 0); column j gets elements j-1 (b = 1) and j (b = 0).  One thread per
// (column, element pair); the four partial values are summed in fixed order.
__global__ void k_circle_row_part(AsmArgs A, zd* part) {
  const int64_t N = A.N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * N) return;
  const int64_t j = t >> 2;
  const int u = (int)((t >> 1) & 1), v = (int)(t & 1);
  const int64_t e = u ? 0 : N - 1;
  const int a = u ? 0 : 1;
  const int64_t f = v ? j : (j - 1 + N) % N;
  const int b = v ? 0 : 1;
  PairOut o;
  pair_integrals(A, e, f, o);
  for (int op = 0; op < 4; ++op) part[(int64_t)op * 4 * N + t] = o.v[op][a * 2 + b];
}

__global__ void k_circle_row_sum(AsmArgs A, const zd* part) {
  const int64_t N = A.N;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  zd* outs[4] = {A.S, A.D, A.Dt, A.Nk};
  for (int op = 0; op < 4; ++op) {
    const zd* p = part + (int64_t)op * 4 * N + 4 * j;
    outs[op][j] = ((p[0] + p[1]) + p[2]) + p[3];
  }
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

// Coefficient tables of hankel01_asymptotic_fixed for k~ = k (1 + i t), and
// the x above which 2M terms (M = 2, 3, 4, 5, 7) meet the relative tolerance
// tol: the first omitted term max_nu |a_2M(nu)| / x^2M (|1 + i t|^-2M <= 1),
// with 10% margin on x and never below 20, where the expansion starts
void fill_asymptotic(KtPair& kp, double tol) {
  AsymCoef& h = kp.asym;
  std::memset(&h, 0, sizeof(h));
  const std::complex<double> c1 = std::complex<double>(1.0, 0.0) / std::complex<double>(1.0, kp.t);
  for (int nu = 0; nu < 2; ++nu) {
    double a = 1.0;
    std::complex<double> cp = 1.0;   // c1^k
    for (int k = 0; k < 2 * ASYM_M; ++k) {
      if (k > 0) {
        a *= (4.0 * nu * nu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
        cp *= c1;
      }
      const int m = k / 2;
      const double sg = (m & 1) ? -1.0 : 1.0;
      const std::complex<double> b = sg * a * cp;
      if ((k & 1) == 0) { h.re[nu][m] = sg * a; h.ce[nu][m] = mkz(b.real(), b.imag()); }
      else { h.ro[nu][m] = sg * a; h.co[nu][m] = mkz(b.real(), b.imag()); }
    }
  }
  const int Ms[5] = {2, 3, 4, 5, 7};
  for (int i = 0; i < 5; ++i) {
    const int k2 = 2 * Ms[i];
    double need = 20.0;
    for (int nu = 0; nu < 2; ++nu) {
      double a = 1.0;
      for (int k = 1; k <= k2; ++k) a *= (4.0 * nu * nu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
      need = std::max(need, 1.1 * std::pow(std::fabs(a) / tol, 1.0 / k2));
    }
    kp.xth[i] = need;
  }
}

static int upload_rules(const AsmArgs& A) {
  double xf[16], wf[16], xn[16], wn[16];
  gauss_legendre01(A.q_far, xf, wf);
  gauss_legendre01(A.q_near, xn, wn);
  if (cudaMemcpyToSymbol(c_xf, xf, sizeof(double) * A.q_far) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_wf, wf, sizeof(double) * A.q_far) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_xn, xn, sizeof(double) * A.q_near) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_wn, wn, sizeof(double) * A.q_near) != cudaSuccess) return 3;
  // float-float weights of the FP32 far path: w_r phi_b(xi_r) and w_r
  float fwt[2][16][2], fw[16][2];
  std::memset(fwt, 0, sizeof(fwt));
  std::memset(fw, 0, sizeof(fw));
  for (int i = 0; i < A.q_far; ++i) {
    const double v[3] = {wf[i] * (1.0 - xf[i]), wf[i] * xf[i], wf[i]};
    float* dst[3] = {fwt[0][i], fwt[1][i], fw[i]};
    for (int t = 0; t < 3; ++t) {
      dst[t][0] = (float)v[t];
      dst[t][1] = (float)(v[t] - (double)dst[t][0]);
    }
  }
  if (cudaMemcpyToSymbol(c_fwt, fwt, sizeof(fwt)) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_fw, fw, sizeof(fw)) != cudaSuccess) return 3;
  return 0;
}

int assemble_dense(const AsmArgs& A, cudaStream_t s) {
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  const size_t smem = sizeof(zd) * 4 * TILE * TILE;
  cudaFuncSetAttribute(k_assemble<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t nt = (A.N + TILE - 1) / TILE;
  dim3 grid((unsigned)nt, (unsigned)nt);
  k_assemble<0><<<grid, ASM_THREADS, smem, s>>>(A);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("assemble: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

__device__ __forceinline__ void split_store(double x, int planes, uint16_t* const* P, int64_t off) {
  __nv_bfloat16 h0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(h0);
  P[0][off] = __bfloat16_as_ushort(h0);
  if (planes > 1) {
    __nv_bfloat16 h1 = __double2bfloat16(r);
    r -= (double)__bfloat162float(h1);
    P[1][off] = __bfloat16_as_ushort(h1);
    if (planes > 2) P[2][off] = __bfloat16_as_ushort(__double2bfloat16(r));
  }
}

// FP32 values: x - hi and (x - hi) - mid are exact in FP32, so the planes
// equal those of split_store((double)x)
__device__ __forceinline__ void split_store_f(float x, int planes, uint16_t* const* P, int64_t off) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(h0);
  P[0][off] = __bfloat16_as_ushort(h0);
  if (planes > 1) {
    const __nv_bfloat16 h1 = __float2bfloat16_rn(r);
    r -= __bfloat162float(h1);
    P[1][off] = __bfloat16_as_ushort(h1);
    if (planes > 2) P[2][off] = __bfloat16_as_ushort(__float2bfloat16_rn(r));
  }
}

static int upload_hankel_coefficients() {
  float a0[10], a1[10];
  double t0 = 1.0, t1 = 1.0;
  a0[0] = 1.f;
  a1[0] = 1.f;
  for (int kk = 1; kk < 10; ++kk) {
    const double o = 2.0 * kk - 1.0;
    t0 *= (0.0 - o * o) / (8.0 * kk);
    t1 *= (4.0 - o * o) / (8.0 * kk);
    a0[kk] = (float)t0;
    a1[kk] = (float)t1;
  }
  if (cudaMemcpyToSymbol(c_a0, a0, sizeof(a0)) != cudaSuccess) return 3;
  if (cudaMemcpyToSymbol(c_a1, a1, sizeof(a1)) != cudaSuccess) return 3;
  return 0;
}

// flag[t] = 1 when tile t holds an element pair outside the FP32 fast path
__global__ void k_tile_flags(AsmArgs A, int64_t nt, uint8_t* flag) {
  const int64_t t = blockIdx.x;
  const int64_t ti = t / nt, tj = t - (t / nt) * nt;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int span = TILE + 1;
  for (int u = threadIdx.x; u < span * span; u += blockDim.x) {
    const int el = u / span, fl = u - (u / span) * span;
    const int64_t e = ((ti * TILE - 1 + el) % A.N + A.N) % A.N;
    const int64_t f = ((tj * TILE - 1 + fl) % A.N + A.N) % A.N;
    if (!fast_ok(A, e, f)) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) flag[t] = (uint8_t)any;
}

// Tiles whose element pairs all take the FP32 path: the reduced sums of
// pair_fast_f accumulated per node pair in shared memory (FP32, four
// conflict-free phases), then scaled by their FP64 factors, combined (N) and
// written as split-bf16 planes.
// float-float helpers for the epilogue of k_assemble_fast
struct ff2 {
  ff r, i;
};
__device__ __forceinline__ ff ff_of(double x) {
  const float h = (float)x;
  return ff{h, (float)(x - (double)h)};
}
__device__ __forceinline__ ff2 ff2_of(zd z) { return ff2{ff_of(z.x), ff_of(z.y)}; }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const ff p = ff_two_prod(a.hi, b);
  return ff_quick(p.hi, fmaf(a.lo, b, p.lo));
}
// bf16 planes of a float-float value: hi - bf16(hi) is exact in FP32, so the
// second residual carries the value to ~2^-24 of the first plane's scale
__device__ __forceinline__ void ff_planes(ff x, uint16_t (&p)[3]) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x.hi);
  const float r1 = (x.hi - __bfloat162float(h0)) + x.lo;
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);
  p[0] = __bfloat16_as_ushort(h0);
  p[1] = __bfloat16_as_ushort(h1);
  p[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}
// (re, im) as adjacent bf16 pairs, one 32-bit store per plane (off even)
__device__ __forceinline__ void split_store_ff2(ff re, ff im, int planes, uint16_t* const* P, int64_t off) {
  uint16_t a[3], b[3];
  ff_planes(re, a);
  ff_planes(im, b);
  for (int q = 0; q < planes; ++q) *(uint32_t*)(P[q] + off) = (uint32_t)a[q] | ((uint32_t)b[q] << 16);
}

__global__ void __launch_bounds__(ASM_THREADS) k_assemble_fast(AsmArgs A, int64_t nt, const uint8_t* flag) {
  const int64_t ti = blockIdx.y, tj = blockIdx.x;
  if (flag[ti * nt + tj]) return;
  __shared__ cf acc[5 * TILE * TILE];
  const int64_t N = A.N;
  const int64_t i0 = ti * TILE, j0 = tj * TILE;
  for (int t = threadIdx.x; t < 5 * TILE * TILE; t += blockDim.x) acc[t] = {0.f, 0.f};
  __syncthreads();
  const int span = TILE + 1;
  const int npairs = span * span;
  for (int base = 0; base < npairs; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const int el = idx / span, fl = idx - (idx / span) * span;
    const bool valid = idx < npairs;
    const bool rowok = valid && ((el >= 1 && i0 + el - 1 < N) || (el < TILE && i0 + el < N));
    const bool colok = valid && ((fl >= 1 && j0 + fl - 1 < N) || (fl < TILE && j0 + fl < N));
    PairOutF o;
    if (rowok && colok) {
      const int64_t e = ((i0 - 1 + el) % N + N) % N;
      const int64_t f = ((j0 - 1 + fl) % N + N) % N;
      pair_fast_f(A, e, f, o);
    }
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) {
      const int a = ph >> 1, b = ph & 1;
      if (rowok && colok) {
        const int li = el - 1 + a, lj = fl - 1 + b;
        if (li >= 0 && li < TILE && lj >= 0 && lj < TILE && i0 + li < N && j0 + lj < N) {
#pragma unroll
          for (int op = 0; op < 5; ++op) cadd(acc[(op * TILE + li) * TILE + lj], o.v[op][ph]);
        }
      }
      __syncthreads();
    }
  }
  // Entries: the FP64 run factors times the FP32 tile sums, in float-float
  // on the FP32 pipe (the factors as hi + lo; products by TwoProd), split
  // into bf16 planes from the float-float value.  The result carries ~44
  // bits, far beyond the 24 of the FP32 sums, without touching the FP64
  // pipe (64 times slower), which the FP64 form of this epilogue saturated.
  const ff2 fS = ff2_of(A.fS), fD = ff2_of(A.fD), fDt = ff2_of(A.fDt), fN = ff2_of(A.fN);
  const ff kk = ff_of(A.kk2h2);
  auto entry = [&](int op, int t, ff& re, ff& im) {
    if (op == 3) {
      // N = fN (Nd - k^2 h^2 Nb)
      const cf nb = acc[3 * TILE * TILE + t], nd = acc[4 * TILE * TILE + t];
      const ff dr = ff_add(ff{nd.x, 0.f}, ff_neg(ff_mul_f(kk, nb.x)));
      const ff di = ff_add(ff{nd.y, 0.f}, ff_neg(ff_mul_f(kk, nb.y)));
      re = ff_add(ff_mul(fN.r, dr), ff_neg(ff_mul(fN.i, di)));
      im = ff_add(ff_mul(fN.r, di), ff_mul(fN.i, dr));
      return;
    }
    const ff2& f = (op == 0) ? fS : (op == 1) ? fD : fDt;
    const cf a = acc[op * TILE * TILE + t];
    re = ff_add(ff_mul_f(f.r, a.x), ff_neg(ff_mul_f(f.i, a.y)));
    im = ff_add(ff_mul_f(f.r, a.y), ff_mul_f(f.i, a.x));
  };
  // layout 0: rows i (consecutive threads along j); layout 1: rows j
  for (int lay = 0; lay < 2; ++lay) {
    for (int u = threadIdx.x; u < 4 * TILE * TILE; u += blockDim.x) {
      const int op = u / (TILE * TILE), rem = u - op * TILE * TILE;
      const int a = rem / TILE, b = rem - (rem / TILE) * TILE;
      const int li = lay ? b : a, lj = lay ? a : b;
      if (i0 + li < N && j0 + lj < N) {
        ff re, im;
        entry(op, li * TILE + lj, re, im);
        const int64_t off = lay ? (j0 + lj) * A.ldp + 2 * (i0 + li) : (i0 + li) * A.ldp + 2 * (j0 + lj);
        split_store_ff2(re, im, A.planes, A.P[op][lay], off);
      }
    }
  }
}

int assemble_planes(const AsmArgs& A, cudaStream_t s, cudaEvent_t* mid, int64_t* fp64_tiles, int64_t* tiles) {
  if (upload_rules(A) || upload_hankel_coefficients()) { set_error("uploading quadrature rules failed"); return 3; }
  const size_t smem = sizeof(zd) * 4 * TILE * TILE;
  cudaFuncSetAttribute(k_assemble<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t nt = (A.N + TILE - 1) / TILE;
  uint8_t* flag = nullptr;
  if (cudaMalloc(&flag, nt * nt) != cudaSuccess) { set_error("oom (tile flags)"); return 4; }
  k_tile_flags<<<(unsigned)(nt * nt), 256, 0, s>>>(A, nt, flag);
  note_launch();
  dim3 grid((unsigned)nt, (unsigned)nt);
  k_assemble_fast<<<grid, ASM_THREADS, 0, s>>>(A, nt, flag);
  note_launch();
  if (mid) { cudaEventRecord(mid[0], s); cudaEventRecord(mid[1], s); }
  AsmArgs B = A;
  B.tile_flags = flag;
  k_assemble<1><<<grid, ASM_THREADS, smem, s>>>(B);
  note_launch();
  if (fp64_tiles) {   // the tiles that took the FP64 kernel (for the work count of each kernel)
    std::vector<uint8_t> h((size_t)(nt * nt));
    cudaMemcpyAsync(h.data(), flag, h.size(), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int64_t n = 0;
    for (uint8_t v : h) n += v;
    *fp64_tiles = n;
    *tiles = nt * nt;
  }
  cudaStreamSynchronize(s);
  cudaFree(flag);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("assemble (planes): ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

__global__ void k_far_offsets(Points far, const double* cx, const double* cy, int64_t N, int q, float* ox,
                              float* oy, float* nxf, float* nyf, float* nxl, float* nyl, float* oxl, float* oyl) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * q) return;
  const int64_t e = t / q;
  const double dxo = far.x[t] - cx[e], dyo = far.y[t] - cy[e];
  ox[t] = (float)dxo;
  oy[t] = (float)dyo;
  oxl[t] = (float)(dxo - (double)ox[t]);   // float-float tails of the offsets
  oyl[t] = (float)(dyo - (double)oy[t]);
  nxf[t] = (float)far.nx[t];
  nyf[t] = (float)far.ny[t];
  nxl[t] = (float)(far.nx[t] - (double)nxf[t]);   // float-float tails of the normals
  nyl[t] = (float)(far.ny[t] - (double)nyf[t]);
}

__global__ void k_centres_ff(const double* cx, const double* cy, int64_t N, float4* cff) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const float xh = (float)cx[e], yh = (float)cy[e];
  cff[e] = make_float4(xh, (float)(cx[e] - (double)xh), yh, (float)(cy[e] - (double)yh));
}

int far_offsets(const Points& far, const double* cx, const double* cy, int64_t N, int q, float* ox,
                float* oy, float* nxf, float* nyf, float* nxl, float* nyl, float* oxl, float* oyl, float4* cff,
                cudaStream_t s) {
  k_far_offsets<<<(unsigned)((N * q + 255) / 256), 256, 0, s>>>(far, cx, cy, N, q, ox, oy, nxf, nyf, nxl, nyl,
                                                                oxl, oyl);
  note_launch();
  k_centres_ff<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(cx, cy, N, cff);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("far offsets: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int assemble_circle_row(const AsmArgs& A, cudaStream_t s) {
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  zd* part = nullptr;
  if (cudaMalloc(&part, sizeof(zd) * 16 * A.N) != cudaSuccess) { set_error("oom (circle row)"); return 4; }
  k_circle_row_part<<<(unsigned)((4 * A.N + 63) / 64), 64, 0, s>>>(A, part);
  note_launch();
  k_circle_row_sum<<<(unsigned)((A.N + 127) / 128), 128, 0, s>>>(A, part);
  cudaStreamSynchronize(s);
  cudaFree(part);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("circle row: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int assemble_entries(const AsmArgs& A, int64_t count, const int64_t* rows, const int64_t* cols,
                     zd* out4, cudaStream_t s) {
  if (count <= 0) return 0;
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  k_entries<<<(unsigned)((count + 63) / 64), 64, 0, s>>>(A, count, rows, cols, out4);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("entries: ") + cudaGetErrorString(err)); return 3; }
  return 0;
}


// ---------------------------------------------------------------------------
// Shape derivatives of the Galerkin entries (differentiation of Sec. II Eq. 4
// with respect to the contour).  A far entry is h^2 sum w_p w_r phi_a phi_b K
// over point pairs; moving the contour moves the points (r, r'), turns the
// normals (n, n'), changes k~ through a = L / 2 pi (Sec. III) and scales h^2.
// For the forms T = sum_ij W_ij X_ij the derivative with respect to any
// parameter is therefore
//   sum_P (dT/dr_P . dr_P/dp + dT/dn_P . dn_P/dp) + dT/dk~ dk~/dp + 2 (dh/h) T_h2,
// and one pass over the point pairs gathers dT/dr_P, dT/dn_P (per point),
// dT/dk~ and T_h2 for all parameters at once.  Kernel derivatives, with
// d = r - r', R = |d|, d^ = d / R, g = d.n' / R, z = kappa R,
// H1'(z) = H0(z) - H1(z) / z:
//   S~ = (i/4) H0(k~R):      d/dd = -(i/4) k~ H1 d^,   d/dk~ = -(i/4) R H1
//   D  = (i k/4) H1(kR) g:   d/dd = (i k/4) [k H1' g d^ + H1 (n' - g d^) / R],
//                            d/dn' = (i k/4) H1 d^
//   D~ likewise with k~, and d/dk~ = (i/4) k~ R H0(k~R) g
//   N  (Maue form): [s_a s_b - k^2 h^2 (n.n') phi_a phi_b] (i/4) H0(kR):
//                            d/dd = -(i/4) k H1 d^ (both parts),
//                            d/dn = (i/4) H0 n' and d/dn' = (i/4) H0 n (second part)
// Only far pairs are differentiated here; the near band keeps its singular
// product rules and is differenced (shape_near_forms).
// ---------------------------------------------------------------------------
constexpr int SH_E = 8;       // element rows per block
constexpr int SH_F = 256;     // element columns per block (8 warps x 32 lanes)

__device__ __forceinline__ zd i4(double s, zd H) { return mkz(-0.25 * s * H.y, 0.25 * s * H.x); }   // (i/4) s H

__global__ void __launch_bounds__(256) k_shape_far(ShapeArgs S) {
  const AsmArgs& A = S.A;
  const int64_t N = A.N;
  const int q = A.q_far;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e0 = (int64_t)blockIdx.y * SH_E;
  const int64_t f = (int64_t)blockIdx.x * SH_F + warp * 32 + lane;
  const bool fvalid = f < N;
  __shared__ double rowacc[SH_E][16][8];
  __shared__ double red[8][4];
  for (int t = threadIdx.x; t < SH_E * 16 * 8; t += blockDim.x) (&rowacc[0][0][0])[t] = 0.0;
  __syncthreads();
  const double h = A.h, k = A.k, h2 = h * h, kk2h2 = k * k * h2;
  const zd kt = A.kt;
  double sc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t f1 = fvalid ? (f + 1) % N : 0;
  for (int r = 0; r < q; ++r) {
    double col[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t iq = fvalid ? f * q + r : 0;
    const double xq = A.far.x[iq], yq = A.far.y[iq], nxq = A.far.nx[iq], nyq = A.far.ny[iq];
    const double eta = c_xf[r], wr = c_wf[r];
    const double pb0 = 1.0 - eta, pb1 = eta;
    for (int el = 0; el < SH_E; ++el) {
      const int64_t e = e0 + el;
      const bool ok = fvalid && e < N && periodic_dist(e, f, N) > A.near_band;
      // per operator: sum_b W(e + a, f + b) phi_b(eta_r) for a = 0, 1; and for
      // the derivative part of N, sum_b s_b W_N(e + a, f + b)
      zd cw[4][2], cwd[2];
      if (ok) {
        const int64_t ea[2] = {e, (e + 1) % N};
#pragma unroll
        for (int X = 0; X < 4; ++X)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const zd w0 = S.W[X][ea[a] * N + f], w1 = S.W[X][ea[a] * N + f1];
            cw[X][a] = pb0 * w0 + pb1 * w1;
            if (X == 3) cwd[a] = w1 - w0;          // s_0 = -1, s_1 = +1
          }
      } else {
#pragma unroll
        for (int X = 0; X < 4; ++X) cw[X][0] = cw[X][1] = mkz(0.0);
        cwd[0] = cwd[1] = mkz(0.0);
      }
      for (int p = 0; p < q; ++p) {
        double rowc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (ok) {
          const int64_t ip = e * q + p;
          const double xp = A.far.x[ip], yp = A.far.y[ip], nxp = A.far.nx[ip], nyp = A.far.ny[ip];
          const double xi = c_xf[p], ww = c_wf[p] * wr;
          const double pa0 = 1.0 - xi, pa1 = xi;
          // point-pair coefficients of the four operators
          const zd cS = (h2 * ww) * (pa0 * cw[0][0] + pa1 * cw[0][1]);
          const zd cD = (h2 * ww) * (pa0 * cw[1][0] + pa1 * cw[1][1]);
          const zd cDt = (h2 * ww) * (pa0 * cw[2][0] + pa1 * cw[2][1]);
          const zd cNn = (-kk2h2 * ww) * (pa0 * cw[3][0] + pa1 * cw[3][1]);
          const zd cNd = ww * (cwd[1] - cwd[0]);   // s_a: -1 for a = 0, +1 for a = 1
          const double dx = xp - xq, dy = yp - yq;
          const double R = sqrt(dx * dx + dy * dy), iR = 1.0 / R;
          const double ux = dx * iR, uy = dy * iR;
          const double g = (dx * nxq + dy * nyq) * iR;
          const double nd = nxp * nxq + nyp * nyq;
          Hankel01 Hk, Ht;
          hankel_k_kt(A, R, Hk, Ht);
          const double z = k * R;
          const zd zt = kt * R;
          const zd H1pk = Hk.H0 - (1.0 / z) * Hk.H1;              // H1'(kR)
          const zd H1pt = Ht.H0 - zdiv(Ht.H1, zt);               // H1'(k~R)
          // S~
          const zd aS = cS * i4(-1.0, kt * Ht.H1);               // coefficient of d^ in dK/dd
          // D: (ik/4)[k H1' g d^ + H1 (n' - g d^)/R]
          const zd Dd = cD * i4(k, k * g * H1pk - (g * iR) * Hk.H1);   // along d^
          const zd Dn = cD * i4(k * iR, Hk.H1);                  // along n'
          // D~
          const zd Dtd = cDt * (i4(1.0, kt) * (kt * g * H1pt - (g * iR) * Ht.H1));
          const zd Dtn = cDt * (i4(iR, kt) * Ht.H1);
          // N
          const zd cN = cNd + nd * cNn;
          const zd aN = cN * i4(-k, Hk.H1);
          const zd uR = aS + Dd + Dtd + aN;                       // dT/dd = uR d^ + (Dn + Dtn) n'
          const zd un = Dn + Dtn;
          const double gdx[4] = {uR.x * ux + un.x * nxq, uR.y * ux + un.y * nxq,
                                 uR.x * uy + un.x * nyq, uR.y * uy + un.y * nyq};
          // dT/dn' = (D + D~ terms) d^ + N: cNn (i/4) H0 n ; dT/dn = cNn (i/4) H0 n'
          const zd vq = cD * i4(k, Hk.H1) + cDt * (i4(1.0, kt) * Ht.H1);
          const zd wn = cNn * i4(1.0, Hk.H0);
          // d/dk~: S~ and D~
          const zd dkt = cS * i4(-R, Ht.H1) + cDt * (i4(R, kt) * (Ht.H0 * g));
          // h^2-scaled part of T (all of S~, D, D~ and the k^2 h^2 part of N)
          const zd val = cS * i4(1.0, Ht.H0) + cD * i4(k * g, Hk.H1) + cDt * (i4(g, kt) * Ht.H1) +
                         nd * (cNn * i4(1.0, Hk.H0));
          rowc[0] = gdx[0]; rowc[1] = gdx[1]; rowc[2] = gdx[2]; rowc[3] = gdx[3];
          rowc[4] = wn.x * nxq; rowc[5] = wn.y * nxq; rowc[6] = wn.x * nyq; rowc[7] = wn.y * nyq;
          col[0] -= gdx[0]; col[1] -= gdx[1]; col[2] -= gdx[2]; col[3] -= gdx[3];
          col[4] += vq.x * ux + wn.x * nxp;
          col[5] += vq.y * ux + wn.y * nxp;
          col[6] += vq.x * uy + wn.x * nyp;
          col[7] += vq.y * uy + wn.y * nyp;
          sc[0] += dkt.x; sc[1] += dkt.y; sc[2] += val.x; sc[3] += val.y;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
          for (int o = 16; o > 0; o >>= 1) rowc[i] += __shfl_xor_sync(0xffffffffu, rowc[i], o);
        if (lane == 0) {
#pragma unroll
          for (int i = 0; i < 8; ++i) atomicAdd(&rowacc[el][p][i], rowc[i]);
        }
      }
    }
    if (fvalid) {
      double* gr = S.Gr + 4 * iq;
      double* gn = S.Gn + 4 * iq;
#pragma unroll
      for (int i = 0; i < 4; ++i) { atomicAdd(gr + i, col[i]); atomicAdd(gn + i, col[4 + i]); }
    }
  }
  // block sums of the scalars, then the row accumulators
#pragma unroll
  for (int i = 0; i < 4; ++i)
    for (int o = 16; o > 0; o >>= 1) sc[i] += __shfl_xor_sync(0xffffffffu, sc[i], o);
  if (lane == 0)
    for (int i = 0; i < 4; ++i) red[warp][i] = sc[i];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    atomicAdd(S.scal + threadIdx.x, t);
  }
  for (int t = threadIdx.x; t < SH_E * q * 8; t += blockDim.x) {
    const int el = t / (q * 8), rem = t - el * q * 8, p = rem / 8, i = rem - p * 8;
    const int64_t e = e0 + el;
    if (e < N) atomicAdd((i < 4 ? S.Gr : S.Gn) + 4 * (e * q + p) + (i & 3), rowacc[el][p][i]);
  }
}

// Near band: sum over element pairs with distance <= near_band of the W-weighted
// pair integrals of A's geometry (one thread per pair, block partial sums).
__global__ void __launch_bounds__(128) k_shape_near(AsmArgs A, const zd* W0, const zd* W1, const zd* W2,
                                                    const zd* W3, double* part) {
  const int64_t N = A.N;
  const int span = 2 * A.near_band + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  zd acc = mkz(0.0);
  if (t < N * span) {
    const int64_t e = t / span;
    const int64_t f = ((e + (t - e * span) - A.near_band) % N + N) % N;
    PairOut o;
    pair_integrals(A, e, f, o);
    const zd* W[4] = {W0, W1, W2, W3};
#pragma unroll
    for (int X = 0; X < 4; ++X)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc += W[X][((e + a) % N) * N + (f + b) % N] * o.v[X][a * 2 + b];
  }
  __shared__ double red[2][4];
  double v[2] = {acc.x, acc.y};
  for (int i = 0; i < 2; ++i)
    for (int o2 = 16; o2 > 0; o2 >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o2);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = v[0]; red[1][threadIdx.x >> 5] = v[1]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
    part[2 * blockIdx.x + 1] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
  }
}

int shape_far_forms(const ShapeArgs& a, cudaStream_t s) {
  if (a.A.q_far > 16) { set_error("shape derivative: q_far <= 16"); return 1; }
  if (upload_rules(a.A)) { set_error("uploading quadrature rules failed"); return 3; }
  dim3 grid((unsigned)((a.A.N + SH_F - 1) / SH_F), (unsigned)((a.A.N + SH_E - 1) / SH_E));
  k_shape_far<<<grid, 256, 0, s>>>(a);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("shape (far): ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

int shape_near_forms(const AsmArgs& A, const zd* const* W, double* part, int* nparts, cudaStream_t s) {
  if (upload_rules(A)) { set_error("uploading quadrature rules failed"); return 3; }
  const int64_t n = A.N * (2 * A.near_band + 1);
  const unsigned blocks = (unsigned)((n + 127) / 128);
  k_shape_near<<<blocks, 128, 0, s>>>(A, W[0], W[1], W[2], W[3], part);
  note_launch();
  *nparts = (int)blocks;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) { set_error(std::string("shape (near): ") + cudaGetErrorString(err)); return 3; }
  return 0;
}

}  // namespace wcs
