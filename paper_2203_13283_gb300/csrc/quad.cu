// Host-side quadrature tables for the Galerkin integrals of Eq. (4).
//
// Regular element pairs use tensor Gauss-Legendre rules.  For element pairs
// that coincide or share a vertex the kernels carry a log|s - s'| singularity;
// there the log part is integrated by product integration on the same tensor
// grid: W_pq = int int l_p(xi) l_q(eta) log d(xi, eta), with l_p the Lagrange
// polynomials on the Gauss nodes, so that sum_pq W_pq F(xi_p, eta_q) is exact
// for every F that is a polynomial of degree < n in each variable.  W is
// computed exactly from the shifted-Legendre log moments
// int_0^1 P~_j(t) log t dt = -1 (j = 0), (-1)^{j+1} / (j (j+1)) (j >= 1).
#include <cmath>
#include <vector>

#include "internal.h"

namespace wcs {

typedef long double ld_t;

static void gl_ld(int n, std::vector<ld_t>& x, std::vector<ld_t>& w) {
  // Gauss-Legendre on [-1, 1] by Newton on P_n
  x.resize(n);
  w.resize(n);
  const ld_t pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    ld_t z = cosl(pi * (i + 0.75L) / (n + 0.5L)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      ld_t p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        ld_t p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1; }
      pp = n * (z * p1 - p0) / (z * z - 1);
      ld_t dz = p1 / pp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    // recompute derivative at the converged node
    ld_t p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      ld_t p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    pp = n * (z * p1 - p0) / (z * z - 1);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2 / ((1 - z * z) * pp * pp);
  }
}

void gauss_legendre01(int n, double* x, double* w) {
  std::vector<ld_t> X, W;
  gl_ld(n, X, W);
  for (int i = 0; i < n; ++i) {
    x[i] = (double)((X[i] + 1) / 2);
    w[i] = (double)(W[i] / 2);
  }
}

// Lagrange basis polynomial l_p on nodes xs evaluated at t
static ld_t lagrange(const std::vector<ld_t>& xs, int p, ld_t t) {
  ld_t v = 1;
  for (size_t j = 0; j < xs.size(); ++j)
    if ((int)j != p) v *= (t - xs[j]) / (xs[p] - xs[j]);
  return v;
}

// shifted Legendre P~_j(t), t in [0, 1], for j = 0..J-1
static void shifted_legendre(int J, ld_t t, std::vector<ld_t>& out) {
  out.assign(J, 0);
  ld_t z = 2 * t - 1;
  out[0] = 1;
  if (J > 1) out[1] = z;
  for (int k = 2; k < J; ++k) out[k] = ((2 * k - 1) * z * out[k - 1] - (k - 1) * out[k - 2]) / k;
}

// int_0^1 log(t) P(t) dt for a polynomial P of degree < J given by samples on
// the J-point Gauss rule (tg, wg) of [0, 1]
static ld_t log_moment_integral(const std::vector<ld_t>& tg, const std::vector<ld_t>& wg,
                                const std::vector<ld_t>& vals) {
  int J = (int)tg.size();
  std::vector<ld_t> pl;
  ld_t total = 0;
  std::vector<ld_t> coef(J, 0);
  for (int m = 0; m < J; ++m) {
    shifted_legendre(J, tg[m], pl);
    for (int j = 0; j < J; ++j) coef[j] += wg[m] * vals[m] * pl[j];
  }
  for (int j = 0; j < J; ++j) {
    ld_t c = (2 * j + 1) * coef[j];
    ld_t mom = (j == 0) ? -1.0L : ((j % 2 == 1) ? 1.0L : -1.0L) / ((ld_t)j * (j + 1));
    total += c * mom;
  }
  return total;
}

void build_quad_tables(QuadTables& q) {
  gauss_legendre01(q.q_far, q.xf, q.wf);
  gauss_legendre01(q.q_near, q.xn, q.wn);
  const int n = q.q_near;
  std::vector<ld_t> X, W;
  gl_ld(n, X, W);
  std::vector<ld_t> xs(n);
  for (int i = 0; i < n; ++i) xs[i] = (X[i] + 1) / 2;
  // Gauss rule with J = 2n + 2 nodes on [0,1] for polynomials of degree <= 2n - 1
  const int J = 2 * n + 2;
  std::vector<ld_t> TJ, WJ;
  gl_ld(J, TJ, WJ);
  std::vector<ld_t> tg(J), wg(J);
  for (int i = 0; i < J; ++i) { tg[i] = (TJ[i] + 1) / 2; wg[i] = WJ[i] / 2; }
  // inner rule for polynomial integrals of degree <= 2n - 2
  std::vector<ld_t> IX, IW;
  gl_ld(n + 1, IX, IW);

  // --- self: d = |xi - eta|.  W_pq = int_0^1 log t Q_pq(t) dt,
  //     Q_pq(t) = int_0^{1-t} [l_p(y + t) l_q(y) + l_p(y) l_q(y + t)] dy
  q.wlog[0].assign(n * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int r = 0; r < n; ++r) {
      std::vector<ld_t> vals(J);
      for (int m = 0; m < J; ++m) {
        ld_t t = tg[m], L = 1 - t, acc = 0;
        for (int g = 0; g < n + 1; ++g) {
          ld_t y = L * (IX[g] + 1) / 2, wy = L * IW[g] / 2;
          acc += wy * (lagrange(xs, p, y + t) * lagrange(xs, r, y) +
                       lagrange(xs, p, y) * lagrange(xs, r, y + t));
        }
        vals[m] = acc;
      }
      q.wlog[0][p * n + r] = (double)log_moment_integral(tg, wg, vals);
    }

  // --- touching: V_ij = int int l_i(a) l_j(b) log(a + b), a, b in [0, 1].
  //     With v = a + b: on v in [0,1] Q(v) = int_0^v l_i(a) l_j(v - a) da (log moments),
  //     on v in [1,2] log v is smooth (plain Gauss with J nodes).
  std::vector<ld_t> V(n * n, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      std::vector<ld_t> vals(J);
      for (int m = 0; m < J; ++m) {
        ld_t v = tg[m], acc = 0;
        for (int g = 0; g < n + 1; ++g) {
          ld_t a = v * (IX[g] + 1) / 2, wa = v * IW[g] / 2;
          acc += wa * lagrange(xs, i, a) * lagrange(xs, j, v - a);
        }
        vals[m] = acc;
      }
      ld_t part1 = log_moment_integral(tg, wg, vals);
      ld_t part2 = 0;
      for (int m = 0; m < J; ++m) {
        ld_t v = 1 + tg[m], acc = 0;   // a in [v - 1, 1]
        ld_t lo = v - 1, L = 1 - lo;
        for (int g = 0; g < n + 1; ++g) {
          ld_t a = lo + L * (IX[g] + 1) / 2, wa = L * IW[g] / 2;
          acc += wa * lagrange(xs, i, a) * lagrange(xs, j, v - a);
        }
        part2 += wg[m] * logl(v) * acc;
      }
      V[i * n + j] = part1 + part2;
    }
  // f = e + 1: a = 1 - xi (node index mirrored), b = eta
  // f = e - 1: a = xi, b = 1 - eta
  q.wlog[1].assign(n * n, 0.0);
  q.wlog[2].assign(n * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int r = 0; r < n; ++r) {
      q.wlog[1][p * n + r] = (double)V[(n - 1 - p) * n + r];
      q.wlog[2][p * n + r] = (double)V[p * n + (n - 1 - r)];
    }
}

}  // namespace wcs
