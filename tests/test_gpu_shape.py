"""GPU parity of the far-field shape gradient (wcs_shape_gradient) and of
perturbed contours (wcs_contour_perturb) against the oracle (oracle/shape.py):
J to 1e-9, the gradient to 1e-6 of its largest entry against central
differences of the oracle's J, and the derivatives that the ellipse's
symmetries force to zero."""

import numpy as np
import pytest

import workloads
from gpu_common import built
from oracle import geometry, shape

pytestmark = pytest.mark.gpu

M = workloads.WORKLOADS["ellipse_n8192"]["shape_modes"]
N = 64
INC = workloads.WORKLOADS["ellipse_n8192"]["angles"]                # 16 incidences, 22.5 degrees apart
OBS = workloads.WORKLOADS["ellipse_n8192"]["observation_angles"]    # 90 observation angles, 4 degrees apart


def test_shape_gradient_vs_oracle():
    built()
    from paper_2203_13283_gb300 import Solver
    w = workloads.WORKLOADS["ellipse_n8192"]
    fam, base = w["family"], w["params"]
    k = 2.0 * np.pi * (N / 10.0) / geometry.Contour(fam, base).L
    p = np.zeros(2 * M)
    p[2] = 0.01                                    # alpha_2: keeps both symmetries
    s = Solver(refine_tol=1e-12, max_refine=16)
    s.contour(fam, **base).perturb(p[:M], p[M:]).mesh(N, k).assemble()
    s.skeleton(1e-10, max_rank=N // 2, seed=1, allow_cap=True)
    s.factor()
    J, g = s.shape_gradient(INC, OBS, M)
    J_ref, _ = shape.objective(fam, base, p, M, N, k, INC, OBS)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    idx = [0, 2, 4, 6]
    g_ref = shape.gradient_fd(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g[idx] - g_ref)) <= 1e-6 * scale
    odd = [m for m in range(M) if m % 2 == 1] + list(range(M, 2 * M))
    assert np.max(np.abs(g[odd])) <= 1e-6 * scale
    s.close()


def test_shape_objective_autograd():
    # the autograd wrapper returns wcs_shape_gradient's J and, through
    # backward, its gradient scaled by the incoming gradient
    built()
    import torch
    from paper_2203_13283_gb300 import Solver, autograd
    w = workloads.WORKLOADS["ellipse_n8192"]
    fam, base = w["family"], w["params"]
    k = 2.0 * np.pi * (N / 10.0) / geometry.Contour(fam, base).L
    m = 2
    p = torch.zeros(2 * m, dtype=torch.float64)
    p[0] = 0.003
    p.requires_grad_(True)
    J = autograd.shape_objective(p, fam, base, N, k, INC, OBS, refine_tol=1e-12, max_refine=16)
    (3.0 * J).backward()
    s = Solver(refine_tol=1e-12, max_refine=16)
    pv = p.detach().numpy()
    s.contour(fam, **base).perturb(pv[:m], pv[m:]).mesh(N, k).assemble()
    s.skeleton(1e-10, seed=1, allow_cap=True)
    s.factor()
    J_ref, g_ref = s.shape_gradient(INC, OBS, m)
    s.close()
    assert abs(J.item() - J_ref) <= 1e-12 * J_ref
    assert np.max(np.abs(p.grad.numpy() - 3.0 * g_ref)) <= 1e-10 * np.max(np.abs(g_ref))


def _factored(fam, base, p, Mp, k):
    from paper_2203_13283_gb300 import Solver
    s = Solver(refine_tol=1e-12, max_refine=16)
    s.contour(fam, **base).perturb(p[:Mp], p[Mp:]).mesh(N, k).assemble()
    s.skeleton(1e-10, max_rank=N // 2, seed=1, allow_cap=True)
    s.factor()
    return s


def test_shape_gradient_beta_vs_oracle():
    # sine parameters at a point without any symmetry (alpha_3 = beta_2 =
    # 0.01), where their derivatives are genuinely non-zero
    built()
    w = workloads.WORKLOADS["ellipse_n8192"]
    fam, base = w["family"], w["params"]
    k = 2.0 * np.pi * (N / 10.0) / geometry.Contour(fam, base).L
    p = np.zeros(2 * M)
    p[3] = 0.01
    p[M + 1] = 0.01
    s = _factored(fam, base, p, M, k)
    J, g = s.shape_gradient(INC, OBS, M)
    s.close()
    idx = [M + 1, M + 2, M + 4]                    # beta_2, beta_3, beta_5
    g_ref = shape.gradient_fd(fam, base, p, M, N, k, INC, OBS, idx, delta=1e-6)
    scale = np.max(np.abs(g_ref))
    assert np.min(np.abs(g_ref)) > 1e-3 * scale
    assert np.max(np.abs(g[idx] - g_ref)) <= 1e-6 * scale


def test_shape_gradient_beta_rotation_identity():
    # on the circle, turning everything by psi = -pi / (2m) maps sin(m theta)
    # onto cos(m theta): dJ/d beta_m at (I, O) = dJ/d alpha_m at (I + psi, O + psi)
    built()
    Mr, k = 4, 8.0
    inc = np.array([0.3, 1.7, 4.0])
    obs = np.deg2rad(np.arange(0.0, 360.0, 20.0))
    p = np.zeros(2 * Mr)
    for m in (2, 3):
        psi = -np.pi / (2 * m)
        s = _factored("circle", {"a": 1.0}, p, Mr, k)
        _, gb = s.shape_gradient(inc, obs, Mr)
        _, ga = s.shape_gradient(inc + psi, obs + psi, Mr)
        s.close()
        assert abs(ga[m]) > 1e-2
        assert abs(gb[Mr + m - 1] - ga[m]) <= 1e-6 * abs(ga[m]), (m, gb[Mr + m - 1], ga[m])


@pytest.fixture(scope="module")
def oracle_operator_derivatives():
    # central differences (delta 1e-6) of the oracle's dense operators at an
    # asymmetric point of the ellipse, for 3 cosine and 3 sine parameters
    w = workloads.WORKLOADS["ellipse_n8192"]
    fam, base = w["family"], w["params"]
    k = 2.0 * np.pi * (N / 10.0) / geometry.Contour(fam, base).L
    Mp = 3
    p = np.zeros(2 * Mp)
    p[2] = 0.01                   # alpha_2
    p[Mp + 1] = 0.01              # beta_2
    d = 1e-6
    dX = []
    for i in range(2 * Mp):
        e = np.zeros(2 * Mp)
        e[i] = d
        op_p, _, _, _ = shape.operators_at(fam, base, p + e, Mp, N, k, INC[:1], OBS[:1])
        op_m, _, _, _ = shape.operators_at(fam, base, p - e, Mp, N, k, INC[:1], OBS[:1])
        dX.append({key: (op_p[key] - op_m[key]) / (2 * d) for key in ("S", "D", "Dt", "N")})
    return fam, base, k, Mp, p, dX


@pytest.mark.parametrize("op", ["S", "D", "Dt", "N"])
def test_operator_shape_derivative_forms_vs_oracle(oracle_operator_derivatives, op):
    # the one-pass derivative kernel (far pairs) plus the differenced near band,
    # per operator: sum_b u_b^H dX/dp_i v_b against the oracle's differenced
    # dense operators, for every parameter
    built()
    from paper_2203_13283_gb300 import Solver
    fam, base, k, Mp, p, dX = oracle_operator_derivatives
    g = np.random.default_rng(7)
    u = g.standard_normal((N, 3)) + 1j * g.standard_normal((N, 3))
    v = g.standard_normal((N, 3)) + 1j * g.standard_normal((N, 3))
    s = Solver(precision=0)
    s.contour(fam, **base).perturb(p[:Mp], p[Mp:]).mesh(N, k).assemble()
    T = s.shape_operator_forms(op, u, v, Mp)
    s.close()
    ref = np.array([np.sum(u.conj() * (d[op] @ v)) for d in dX])
    print(op, np.max(np.abs(T - ref)) / np.max(np.abs(ref)))
    assert np.max(np.abs(T - ref)) <= 1e-8 * np.max(np.abs(ref)), (T, ref)


def test_operator_shape_derivative_forms_in_expansion_range():
    # N = 256 (k = 29.9): element pairs farther than R = 20 / k ~ 0.67 take the
    # Hankel expansion branch of the derivative kernel, which N = 64 never
    # reaches; one cosine and one sine parameter at the asymmetric point,
    # all four operators against the oracle's differenced dense operators
    built()
    from paper_2203_13283_gb300 import Solver
    w = workloads.WORKLOADS["ellipse_n8192"]
    fam, base = w["family"], w["params"]
    n = 256
    k = 2.0 * np.pi * (n / 10.0) / geometry.Contour(fam, base).L
    Mp = 4
    p = np.zeros(2 * Mp)
    p[3] = 0.01                   # alpha_3
    p[Mp + 1] = 0.01              # beta_2
    params = [2, Mp + 2]          # alpha_2, beta_3
    d = 1e-6
    dX = []
    for i in params:
        e = np.zeros(2 * Mp)
        e[i] = d
        op_p, _, _, _ = shape.operators_at(fam, base, p + e, Mp, n, k, INC[:1], OBS[:1])
        op_m, _, _, _ = shape.operators_at(fam, base, p - e, Mp, n, k, INC[:1], OBS[:1])
        dX.append({key: (op_p[key] - op_m[key]) / (2 * d) for key in ("S", "D", "Dt", "N")})
    g = np.random.default_rng(11)
    u = g.standard_normal((n, 2)) + 1j * g.standard_normal((n, 2))
    v = g.standard_normal((n, 2)) + 1j * g.standard_normal((n, 2))
    s = Solver(precision=0)
    s.contour(fam, **base).perturb(p[:Mp], p[Mp:]).mesh(n, k).assemble()
    for op in ("S", "D", "Dt", "N"):
        T = s.shape_operator_forms(op, u, v, Mp, params=(params[0], params[0] + 1))
        T2 = s.shape_operator_forms(op, u, v, Mp, params=(params[1], params[1] + 1))
        got = np.array([T[0], T2[0]])
        ref = np.array([np.sum(u.conj() * (dd[op] @ v)) for dd in dX])
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        print(op, f"{err:.1e}")
        assert err <= 1e-8, (op, got, ref)
    s.close()
