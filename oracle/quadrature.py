"""Quadrature rules of the oracle (test infrastructure only).

All rules are Gauss-Legendre based.  Singular element pairs are integrated with
geometrically graded composite Gauss-Legendre panels after a Duffy-type change
of variables, which converges exponentially for the logarithmic singularity of
the 2D Helmholtz Green's function (Sec. II, g_k = (i/4) H0(k|r - r'|)).
"""

import numpy as np


def gauss_legendre01(n):
    """n-point Gauss-Legendre rule on [0, 1] (nodes, weights)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def composite(breaks, n):
    """Composite n-point Gauss-Legendre rule over consecutive [breaks[i], breaks[i+1]]."""
    x0, w0 = gauss_legendre01(n)
    xs, ws = [], []
    for a, b in zip(breaks[:-1], breaks[1:]):
        xs.append(a + (b - a) * x0)
        ws.append((b - a) * w0)
    return np.concatenate(xs), np.concatenate(ws)


def graded01(n=16, ratio=0.25, t_min=1e-13):
    """Rule on [0, 1] geometrically graded toward 0 (for log t and t log t).

    Panels [r^{j+1}, r^j] for j = 0.. until r^j < t_min, then [0, r^J].
    With ratio 0.25 and 16 nodes per panel each panel integrates log t to
    ~1e-16 relative (the singularity sits one third of a panel length away).
    """
    breaks = [1.0]
    while breaks[-1] > t_min:
        breaks.append(breaks[-1] * ratio)
    breaks.append(0.0)
    return composite(np.array(breaks[::-1]), n)


def panels01(n=16, breaks=(0.0, 0.004, 0.02, 0.1, 0.4, 1.0)):
    """Mildly graded rule on [0, 1] for bounded integrands with t^2 log t terms."""
    return composite(np.array(breaks), n)


# ---------------------------------------------------------------------------
# Rules on the unit square [0,1]^2 for an element pair (xi on e, eta on f).
# Each returns (xi, eta, w) flat arrays; Jacobians are folded into w.
# ---------------------------------------------------------------------------

def tensor_rule(n):
    x, w = gauss_legendre01(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    return X.ravel(), Y.ravel(), W.ravel()


def self_rule(t_rule, n_u=16):
    """Coincident element pair: singular on the diagonal xi = eta.

    Triangle xi > eta: t = xi - eta in (0,1), xi = t + (1-t) u, eta = (1-t) u,
    Jacobian (1 - t); the other triangle by symmetry.  The t rule carries the
    grading toward the singular line t = 0.
    """
    t, wt = t_rule
    u, wu = gauss_legendre01(n_u)
    T, U = np.meshgrid(t, u, indexing="ij")
    W = np.outer(wt, wu) * (1.0 - T)
    xi = T + (1.0 - T) * U
    eta = (1.0 - T) * U
    xi, eta, W = xi.ravel(), eta.ravel(), W.ravel()
    return (np.concatenate([xi, eta]), np.concatenate([eta, xi]),
            np.concatenate([W, W]))


def touching_rule(rho_rule, n_v=16, shared="e_end"):
    """Element pair sharing one vertex; Duffy map centred on that vertex.

    shared == "e_end": the shared vertex is xi = 1 (end of e) = eta = 0 (start
    of f), i.e. f = e + 1.  Local distances a = 1 - xi, b = eta.
    shared == "e_start": xi = 0 = eta = 1, i.e. f = e - 1; a = xi, b = 1 - eta.
    Triangles a >= b: (a, b) = (rho, rho v); b > a: (a, b) = (rho v, rho);
    Jacobian rho.
    """
    r, wr = rho_rule
    v, wv = gauss_legendre01(n_v)
    R, V = np.meshgrid(r, v, indexing="ij")
    W = (np.outer(wr, wv) * R).ravel()
    R, V = R.ravel(), V.ravel()
    a = np.concatenate([R, R * V])
    b = np.concatenate([R * V, R])
    W = np.concatenate([W, W])
    if shared == "e_end":
        return 1.0 - a, b, W
    return a, 1.0 - b, W


# ---------------------------------------------------------------------------
# Exact integrals of polynomial x logarithm over the unit square, used to take
# the log singularity of g out of the coincident and touching element pairs.
# The integrands reduce to int_0^1 P(t) log t dt with P a cubic polynomial
# (exact through the moments int_0^1 t^n log t dt = -1/(n+1)^2) plus, for
# the touching case, int_1^2 P(v) log v dv with log v analytic there.
# ---------------------------------------------------------------------------

_LOG_CACHE = {}


def _poly_log_moment(fun, deg=3):
    """int_0^1 fun(t) log t dt for a polynomial fun of degree <= deg."""
    t, _ = gauss_legendre01(deg + 3)
    V = np.vander(t, deg + 1, increasing=True)
    c = np.linalg.lstsq(V, fun(t), rcond=None)[0]
    return sum(cn * (-1.0 / (n + 1) ** 2) for n, cn in enumerate(c))


def log_integrals(kind):
    """Exact I[a][b] = int_0^1 int_0^1 phi_a(xi) phi_b(eta) log(d(xi, eta)) and
    I1 = int int log(d), with phi_0 = 1 - x, phi_1 = x and

      kind "self":   d = |xi - eta|
      kind "e_end":  d = (1 - xi) + eta     (shared vertex xi = 1, eta = 0)
      kind "e_start": d = xi + (1 - eta)    (shared vertex xi = 0, eta = 1)
    """
    if kind in _LOG_CACHE:
        return _LOG_CACHE[kind]
    phi = (lambda x: 1.0 - x, lambda x: x)
    one = lambda x: np.ones_like(x)
    yg, wg = gauss_legendre01(6)      # exact for the cubic inner integrands
    vg, wv = gauss_legendre01(40)     # log v on [1, 2]

    def integ(f, g):
        if kind == "self":
            # int int f(x) g(y) log|x - y| = int_0^1 log t P(t) dt,
            # P(t) = int_0^{1-t} f(y+t) g(y) + f(y) g(y+t) dy
            def P(t):
                y = (1.0 - t)[:, None] * yg[None, :]
                w = (1.0 - t)[:, None] * wg[None, :]
                return np.sum(w * (f(y + t[:, None]) * g(y) + f(y) * g(y + t[:, None])), axis=1)
            return _poly_log_moment(P)
        # touching: with a, b the distances from the shared vertex, d = a + b;
        # F(a, b) is the integrand in those coordinates
        if kind == "e_end":
            F = lambda a, b: f(1.0 - a) * g(b)
        else:
            F = lambda a, b: f(a) * g(1.0 - b)

        def Q(v):  # int over a of F(a, v - a), a in [max(0, v-1), min(1, v)]
            lo, hi = np.maximum(0.0, v - 1.0), np.minimum(1.0, v)
            a = lo[:, None] + (hi - lo)[:, None] * yg[None, :]
            w = (hi - lo)[:, None] * wg[None, :]
            return np.sum(w * F(a, v[:, None] - a), axis=1)
        part1 = _poly_log_moment(Q)
        v = 1.0 + vg
        part2 = np.sum(wv * np.log(v) * Q(v))
        return part1 + part2

    I = np.array([[integ(phi[a], phi[b]) for b in range(2)] for a in range(2)])
    I1 = integ(one, one)
    _LOG_CACHE[kind] = (I, I1)
    return I, I1
