"""Pins of the oracle's geometry and quadrature against closed forms (CPU)."""

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from oracle import assembly, geometry, quadrature


def test_ellipse_perimeter_closed_form():
    # perimeter of an ellipse: 4 a E(1 - b^2/a^2) (complete elliptic integral)
    for ax, ay in [(1.0, 0.5), (1.0, 0.7), (2.0, 1.0)]:
        cur = geometry.Contour("ellipse", {"ax": ax, "ay": ay})
        ref = 4.0 * ax * sp.ellipe(1.0 - (ay / ax) ** 2)
        assert abs(cur.L - ref) < 1e-13 * ref


def test_superellipse_perimeter_polygon_richardson():
    # independent: inscribed polygons in the polar angle, Richardson-extrapolated
    cur = geometry.Contour("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0})
    rho = geometry.rho_function("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0})

    def poly(M):
        th = 2 * np.pi * np.arange(M + 1) / M
        x, y = rho(th) * np.cos(th), rho(th) * np.sin(th)
        return np.sum(np.hypot(np.diff(x), np.diff(y)))

    p1, p2, p3 = poly(4000), poly(8000), poly(16000)
    r1 = (4 * p2 - p1) / 3
    r2 = (4 * p3 - p2) / 3
    ref = (16 * r2 - r1) / 15
    assert abs(cur.L - ref) < 1e-11
    assert abs(cur.L - 5.6527241628) < 1e-9


def test_ellipse_curvature_and_normals():
    ax, ay = 1.0, 0.5
    cur = geometry.Contour("ellipse", {"ax": ax, "ay": ay})
    s = np.linspace(0.0, cur.L, 97)[:-1]
    P = cur.points(s)
    # closed form curvature at a point (x, y): a b / (b^4 x^2/a^2 ... ) via parametric t
    t = np.arctan2(P["y"] / ay, P["x"] / ax)
    kap = ax * ay / (ax ** 2 * np.sin(t) ** 2 + ay ** 2 * np.cos(t) ** 2) ** 1.5
    assert np.max(np.abs(P["kappa"] - kap)) < 1e-12
    # outward unit normal: gradient of x^2/a^2 + y^2/b^2
    gx, gy = P["x"] / ax ** 2, P["y"] / ay ** 2
    gn = np.hypot(gx, gy)
    assert np.max(np.abs(P["nx"] - gx / gn)) < 1e-13
    assert np.max(np.abs(P["ny"] - gy / gn)) < 1e-13
    # points lie on the ellipse, and arc length between them is uniform
    assert np.max(np.abs((P["x"] / ax) ** 2 + (P["y"] / ay) ** 2 - 1)) < 1e-14


def test_arc_length_by_adaptive_quadrature():
    cur = geometry.Contour("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0})
    rho = geometry.rho_function("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0})
    d = 1e-6

    def speed(t):
        r = rho(t)
        dr = (rho(t + d) - rho(t - d)) / (2 * d)
        return np.hypot(r, dr)

    for th in [0.3, 1.1, 2.5]:
        ref = si.quad(speed, 0.0, th, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
        assert abs(cur.s_of_theta(np.array([th]))[0] - ref) < 1e-8


def test_element_interpolation_matches_direct():
    cur = geometry.Contour("ellipse", {"ax": 1.0, "ay": 0.5})
    N = 64
    geo = assembly.ElementGeometry(cur, N)
    rng = np.random.default_rng(0)
    e = rng.integers(0, N, 20)
    xi = rng.random(7)
    P = geo.at(e, xi)
    Q = cur.points((e[:, None] + xi[None, :]) * geo.h)
    for f in ("x", "y", "nx", "ny", "kappa"):
        assert np.max(np.abs(P[f] - Q[f])) < 1e-13


def test_quadrature_rules():
    x, w = quadrature.gauss_legendre01(6)
    for n in range(12):
        assert abs(np.sum(w * x ** n) - 1.0 / (n + 1)) < 1e-15
    t, wt = quadrature.panels01(12)
    # int_0^1 t^2 log t = -1/9 ; int_0^1 log(t) t^0 on the mild panels is not exact
    assert abs(np.sum(wt * t ** 2 * np.log(t)) + 1.0 / 9.0) < 1e-13
    # self rule: int int |xi - eta|^2 log|xi - eta| over the square = 2 * (-7/144)
    xi, eta, W = quadrature.self_rule(quadrature.panels01(12), 12)
    d = np.abs(xi - eta)
    assert abs(np.sum(W * d ** 2 * np.log(d)) - 2 * (-7.0 / 144.0)) < 1e-12
    assert abs(np.sum(W) - 1.0) < 1e-14


@pytest.mark.parametrize("kind", ["self", "e_end", "e_start"])
def test_log_integrals_numeric(kind):
    I, I1 = quadrature.log_integrals(kind)
    f = {"self": lambda x, y: np.log(abs(x - y)),
         "e_end": lambda x, y: np.log((1 - x) + y),
         "e_start": lambda x, y: np.log(x + 1 - y)}[kind]
    phi = (lambda x: 1 - x, lambda x: x)
    for a in range(2):
        for b in range(2):
            g = lambda y, x: phi[a](x) * phi[b](y) * f(x, y)
            if kind == "self":   # split along the singular diagonal
                ref = (si.dblquad(g, 0, 1, 0, lambda x: x, epsabs=1e-11, epsrel=1e-11)[0]
                       + si.dblquad(g, 0, 1, lambda x: x, 1, epsabs=1e-11, epsrel=1e-11)[0])
            else:
                ref = si.dblquad(g, 0, 1, 0, 1, epsabs=1e-11, epsrel=1e-11)[0]
            assert abs(I[a, b] - ref) < 1e-8
    if kind == "self":
        assert abs(I1 + 1.5) < 1e-14
    else:
        assert abs(I1 - (2 * np.log(2) - 1.5)) < 1e-14
