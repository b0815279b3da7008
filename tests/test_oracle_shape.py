"""Pins of the oracle's shape gradient (oracle/shape.py), CPU only.

1. On the unit circle the alpha_0 perturbation is a change of radius, so J
   and dJ/d alpha_0 follow from the closed-form discrete solution and far
   field (no quadrature, no assembly).
2. The adjoint formula agrees with central differences of J itself.
3. Symmetries of the ellipse with incidence and observation sets closed under
   y -> -y and rotation by pi: J(beta) = J(-beta) and J(alpha_odd) =
   J(-alpha_odd), so those derivatives vanish; a swapped cos/sin index or a
   wrong parameter map fails here.
4. Rotation covariance on the circle: turning the whole configuration by
   psi = -pi / (2m) maps the perturbation sin(m theta) onto cos(m theta), so
   dJ/d beta_m at incidence and observation sets (I, O) equals dJ/d alpha_m at
   (I + psi, O + psi).  This pins the sine map by itself (an index off by one
   changes the value by ~100%, a sign slip by 200%), independently of the
   finite-difference and adjoint routes, which share the parameter map.
5. The adjoint route against central differences at a point without
   symmetry (alpha_3 = beta_2 = 0.01 breaks both mirrors and the half turn),
   on sine parameters whose derivative is not zero.
"""

import numpy as np
import pytest

import closed_form_circle as cf
import workloads
from oracle import geometry, shape

M = workloads.WORKLOADS["ellipse_n8192"]["shape_modes"]
N = 64
INC = workloads.WORKLOADS["ellipse_n8192"]["angles"]                # 16 incidences, 22.5 degrees apart
OBS = workloads.WORKLOADS["ellipse_n8192"]["observation_angles"]    # 90 observation angles, 4 degrees apart


def _circle_J(a, k):
    kt = k + 0.4j * k ** (1.0 / 3.0) * a ** (-2.0 / 3.0)     # Sec. III with a = L / 2 pi
    J = 0.0
    for phi in INC:
        j = cf.discrete_solution(a, N, k, kt, phi)
        J += np.sum(np.abs(cf.discrete_farfield(a, N, k, j, OBS)) ** 2)
    return J


def test_circle_radius_derivative_closed_form():
    k = 8.0
    p = np.zeros(2 * M)
    J, _ = shape.objective("circle", {"a": 1.0}, p, M, N, k, INC, OBS)
    assert abs(J - _circle_J(1.0, k)) <= 1e-10 * J
    d = 1e-5
    g_ref = (_circle_J(1.0 + d, k) - _circle_J(1.0 - d, k)) / (2 * d)
    g_fd = shape.gradient_fd("circle", {"a": 1.0}, p, M, N, k, INC, OBS, [0], delta=d)[0]
    _, g_adj = shape.gradient_adjoint("circle", {"a": 1.0}, p, M, N, k, INC, OBS, [0], delta=1e-6)
    assert abs(g_fd - g_ref) <= 1e-7 * abs(g_ref)
    assert abs(g_adj[0] - g_ref) <= 1e-7 * abs(g_ref)


@pytest.fixture(scope="module")
def ellipse():
    w = workloads.WORKLOADS["ellipse_n8192"]
    L = geometry.Contour(w["family"], w["params"]).L
    k = 2.0 * np.pi * (N / 10.0) / L
    return w["family"], w["params"], k


def test_adjoint_matches_central_differences(ellipse):
    fam, base, k = ellipse
    p = np.zeros(2 * M)
    p[2] = 0.01                       # away from the symmetric point as well
    idx = [0, 2]                      # two parameters with a non-zero derivative
    _, g_adj = shape.gradient_adjoint(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    g_fd = shape.gradient_fd(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    scale = np.max(np.abs(g_fd))
    assert np.max(np.abs(g_adj - g_fd)) <= 1e-8 * scale


def test_symmetric_parameters_have_zero_derivative(ellipse):
    fam, base, k = ellipse
    p = np.zeros(2 * M)
    J, g = shape.gradient_adjoint(fam, base, p, M, N, k, INC, OBS, [0, 3, M + 1], delta=1e-6)
    assert abs(g[0]) > 1e-2 * J                       # alpha_0: a real effect
    assert np.max(np.abs(g[1:])) <= 1e-10 * J         # alpha_3, beta_2


def test_product_rule_bilinear_forms(ellipse):
    # the product-rule expansion of lam^H dC j over Eq. (6) reproduces the
    # adjoint gradient, and the Gram derivative is dG = (dh / h) G
    fam, base, k = ellipse
    p = np.zeros(2 * M)
    p[2] = 0.01
    idx = [2]
    J, g_bil, terms = shape.gradient_bilinear(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    _, g_adj = shape.gradient_adjoint(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    assert np.max(np.abs(g_bil - g_adj)) <= 1e-9 * np.max(np.abs(g_adj))
    ops, _, _, L = shape.operators_at(fam, base, p, M, N, k, INC, OBS)
    ops_p, _, _, L_p = shape.operators_at(fam, base, p + 1e-6 * np.eye(2 * M)[0], M, N, k, INC, OBS)
    dG = (ops_p["G"] - ops["G"]) / 1e-6
    assert np.max(np.abs(dG - (L_p - L) / (1e-6 * L) * ops["G"])) <= 1e-12 * np.max(np.abs(ops["G"])) / 1e-6
    for t in terms:
        assert all(np.isfinite(t[key]) for key in ("Dt", "D", "S", "N"))


def test_beta_rotation_identity_on_circle():
    Mr, Nr, k = 4, 64, 8.0
    inc = np.array([0.3, 1.7, 4.0])
    obs = np.deg2rad(np.arange(0.0, 360.0, 20.0))
    p = np.zeros(2 * Mr)
    for m in (2, 3):
        psi = -np.pi / (2 * m)
        _, gb = shape.gradient_adjoint("circle", {"a": 1.0}, p, Mr, Nr, k, inc, obs, [Mr + m - 1], delta=1e-6)
        ga = shape.gradient_fd("circle", {"a": 1.0}, p, Mr, Nr, k, inc + psi, obs + psi, [m], delta=1e-5)[0]
        assert abs(ga) > 1e-2
        assert abs(gb[0] - ga) <= 1e-8 * abs(ga), (m, gb[0], ga)


def test_adjoint_matches_central_differences_beta(ellipse):
    fam, base, k = ellipse
    p = np.zeros(2 * M)
    p[3] = 0.01                       # alpha_3: breaks the y-axis mirror and the half turn
    p[M + 1] = 0.01                   # beta_2: breaks the x-axis mirror
    idx = [M + 1, M + 2, M + 4]       # beta_2, beta_3, beta_5
    _, g_adj = shape.gradient_adjoint(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    g_fd = shape.gradient_fd(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    scale = np.max(np.abs(g_fd))
    assert np.min(np.abs(g_fd)) > 1e-3 * scale      # all three are genuinely non-zero
    assert np.max(np.abs(g_adj - g_fd)) <= 1e-8 * scale
