"""GPU parity: every step of the CUDA path against the CPU oracle (small
workloads, full matrices) and against closed forms on the circle.

Tolerances: operator entries and circle eigenvalues 2e-12 relative to the
largest entry (both quadratures converge to ~1e-13); solutions and far fields
1e-10 relative per column, the FP64 bar of the method."""

import numpy as np
import pytest
import torch

import closed_form_circle as cf
import workloads
from gpu_common import colrel, make_solver, rel, to_np
from oracle import assembly, geometry, solver as osolver
from oracle_cache import curve_of, solved

pytestmark = pytest.mark.gpu

SMALL = ["circle_n64", "ellipse_n200", "superellipse_n320", "star_n200"]


@pytest.mark.parametrize("name", ["ellipse_n256", "superellipse_n320", "star_n200"])
def test_geometry_vs_oracle(name):
    w = workloads.SMALL[name]
    s = make_solver(w)
    cur = curve_of(w)
    L = s.info()["L"]
    assert abs(L - cur.L) < 1e-13 * cur.L
    rng = np.random.default_rng(1)
    sv = np.concatenate([rng.random(64) * L, [0.0, L / 3, 0.5 * L]])
    G = s.geometry_sample(sv)
    O = cur.points(sv)
    for f in ("x", "y", "nx", "ny"):
        assert np.max(np.abs(G[f] - O[f])) < 1e-13, f
    assert np.max(np.abs(G["kappa"] - O["kappa"])) < 1e-10 * np.max(np.abs(O["kappa"]))
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_operators_vs_oracle(name):
    r = solved(name)
    s = make_solver(r["w"])
    info = s.info()
    assert abs(info["k"] - r["k"]) < 1e-12 * r["k"]
    assert abs(complex(info["kt_re"], info["kt_im"]) - r["kt"]) < 1e-12 * abs(r["kt"])
    s.assemble()
    N = r["w"]["N"]
    I = torch.eye(N, dtype=torch.complex128, device="cuda")
    for op, key in (("S", "S"), ("D", "D"), ("DT", "Dt"), ("N", "N")):
        X = to_np(s.apply(op, I))
        assert rel(X, r["M"][key]) < 2e-12, (op, rel(X, r["M"][key]))
    # circle eigenvalues against the oracle's dense circle operators
    for op, key in (("S", "S"), ("D", "D"), ("DT", "Dt"), ("N", "N"), ("G", "G")):
        mu = to_np(s.circulant_eigs(op))
        row = r["Mc"][key][0]
        ref = np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) @ row
        assert rel(mu, ref) < 2e-12, op
    s.close()


@pytest.mark.parametrize("name", ["circle_n256", "ellipse_n200"])
def test_circle_eigenvalues_closed_form(name):
    # pin independent of the oracle: aliasing sums of the Bessel symbols
    w = workloads.SMALL[name]
    s = make_solver(w)
    s.assemble()
    info = s.info()
    mu = cf.galerkin_eigs(info["a"], w["N"], info["k"], complex(info["kt_re"], info["kt_im"]))
    for op, key in (("S", "S"), ("D", "D"), ("DT", "Dt"), ("N", "N"), ("G", "G")):
        assert rel(to_np(s.circulant_eigs(op)), mu[key]) < 2e-12, op
    assert rel(to_np(s.circulant_eigs("CC")), cf.c_eigs(mu)) < 2e-12
    s.close()


@pytest.mark.parametrize("name", ["ellipse_n200", "star_n200"])
def test_operator_applies_vs_oracle(name):
    r = solved(name)
    s = make_solver(r["w"])
    s.assemble()
    N = r["w"]["N"]
    rng = np.random.default_rng(5)
    X = rng.standard_normal((N, 7)) + 1j * rng.standard_normal((N, 7))
    Xt = torch.tensor(X, device="cuda")
    C, Cc = r["C"], r["Cc"]
    assert colrel(to_np(s.apply("C", Xt)), C @ X) < 1e-11
    assert colrel(to_np(s.apply("CH", Xt)), C.conj().T @ X) < 1e-11
    assert colrel(to_np(s.apply("CC", Xt)), Cc @ X) < 1e-11
    assert colrel(to_np(s.apply("CCH", Xt)), Cc.conj().T @ X) < 1e-11
    assert colrel(to_np(s.apply("CC_INV", Xt)), np.linalg.solve(Cc, X)) < 1e-11
    assert colrel(to_np(s.apply("G", Xt)), r["M"]["G"] @ X) < 1e-14
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_rhs_vs_oracle(name):
    r = solved(name)
    s = make_solver(r["w"])
    e, hv = s.planewave_rhs(r["w"]["angles"])
    assert colrel(to_np(e), r["e"]) < 1e-13
    assert colrel(to_np(hv), r["h"]) < 1e-13
    s.close()


@pytest.mark.parametrize("name", SMALL)
def test_solve_vs_oracle_tight_skeleton(name):
    # skeleton at 1e-10 (Eq. 7), Woodbury (Eq. 9) and refinement to 1e-12
    r = solved(name)
    w = r["w"]
    s = make_solver(w)
    s.assemble()
    rank = s.skeleton(1e-10, seed=7)
    s.factor()
    if w["family"] == "circle":
        assert rank == 0
    j = to_np(s.solve_planewaves(w["angles"]))
    assert colrel(j, r["j"]) < 1e-10
    # Woodbury alone is already at the skeleton tolerance
    x = to_np(s.woodbury_apply(torch.tensor(r["b"], device="cuda")))
    assert colrel(x, r["j"]) < 1e-8
    # far field
    phi = np.linspace(0, 2 * np.pi, 37)
    F = to_np(s.farfield(torch.tensor(j, device="cuda"), phi))
    Fo = osolver.farfield(r["curve"], w["N"], r["k"], r["j"], phi)
    assert colrel(F, Fo) < 1e-10
    s.close()


@pytest.mark.parametrize("tol", [3e-2, 3e-3])
def test_loose_skeleton_plus_refinement(tol):
    r = solved("superellipse_n320")
    w = r["w"]
    s = make_solver(w)
    s.assemble()
    rank = s.skeleton(tol, seed=11)
    assert 0 < rank <= w["N"]
    s.factor()
    x = to_np(s.woodbury_apply(torch.tensor(r["b"], device="cuda")))
    err_w = colrel(x, r["j"])
    assert err_w < 50 * tol
    j = to_np(s.solve_planewaves(w["angles"]))
    assert s.last_solve["rel_residual"] <= 1e-12
    assert colrel(j, r["j"]) < 1e-10
    s.close()


def test_circle_config_closed_form_and_mie():
    # unit circle, k = 16, N = 256, one plane wave at 0 deg: rank 0 and the exact
    # discrete solution of Eq. (5) from the circle closed forms
    w = workloads.WORKLOADS["circle_n256"]
    s = make_solver(w)
    s.assemble()
    assert s.skeleton(1e-10) == 0
    s.factor()
    j = to_np(s.solve_planewaves(w["angles"]))[:, 0]
    info = s.info()
    jc = cf.discrete_solution(1.0, 256, 16.0, complex(info["kt_re"], info["kt_im"]), 0.0)
    assert np.linalg.norm(j - jc) / np.linalg.norm(jc) < 1e-10
    th = 2 * np.pi * np.arange(256) / 256
    jm = cf.mie_current(1.0, 16.0, 0.0, th)
    assert np.linalg.norm(j - jm) / np.linalg.norm(jm) < 0.01  # O(h^2) discretisation error
    s.close()


def test_state_and_argument_errors():
    from paper_2203_13283_gb300 import Solver, WCSError
    s = Solver()
    with pytest.raises(WCSError) as ei:
        s.assemble()
    assert "STATE" in str(ei.value)
    with pytest.raises(WCSError):
        s.contour("ellipse", ax=-1.0, ay=1.0)
    # a non-convex star is rejected at meshing
    s.contour("fourier", cos=[1.0, 0.0, 0.0, 0.3], sin=[0.0] * 4)
    with pytest.raises(WCSError) as ei:
        s.mesh(256)
    assert "NOT_CONVEX" in str(ei.value)
    s.close()
