"""Pins of the oracle on the circle: closed-form Galerkin eigenvalues, exact
discrete solution and its far field, Mie series (CPU)."""

import numpy as np
import pytest

import closed_form_circle as cf
from oracle import assembly, geometry, solver
from oracle_cache import solved


def _eig(X):
    N = X.shape[0]
    return np.exp(2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) @ X[0]


@pytest.mark.parametrize("name", ["circle_n64", "circle_n256"])
def test_circle_galerkin_eigenvalues(name):
    r = solved(name)
    N = r["w"]["N"]
    mu = cf.galerkin_eigs(r["a"], N, r["k"], r["kt"])
    for key in ("G", "S", "D", "Dt", "N"):
        X = r["M"][key]
        ev = _eig(X)
        assert np.max(np.abs(ev - mu[key])) < 1e-11 * np.max(np.abs(mu[key])), key
        # circulant structure
        assert np.max(np.abs(X - np.roll(np.roll(X, 1, 0), 1, 1))) < 1e-12 * np.max(np.abs(X)), key


def test_circle_symbol_limits():
    # halved identity away from the resonance: 1/2 - D -> 1/2, mu_C -> mu_G / 4
    a, k = 1.0, 16.0
    kt = geometry.wavenumbers(2 * np.pi, 256, k)[1]
    sig = cf.symbols(a, k, kt, 4000)
    assert abs(sig["D"][4000]) < 1e-6
    # Calderon identity S N = 1/4 - D^2 holds for equal wavenumbers
    sk = cf.symbols(a, k, k, 300)
    n = np.arange(301)
    lhs = sk["S"] * sk["N"]
    rhs = 0.25 - sk["D"] ** 2
    assert np.max(np.abs(lhs - rhs)[n > 0]) < 1e-11


@pytest.mark.parametrize("name", ["circle_n64", "circle_n256"])
def test_circle_rhs_and_discrete_solution(name):
    r = solved(name)
    w = r["w"]
    N = w["N"]
    for col, phi in enumerate(w["angles"]):
        ec, hc = cf.planewave_rhs(r["a"], N, r["k"], phi)
        assert np.max(np.abs(r["e"][:, col] - ec)) < 1e-13 * np.max(np.abs(ec))
        assert np.max(np.abs(r["h"][:, col] - hc)) < 1e-13 * np.max(np.abs(hc))
        jc = cf.discrete_solution(r["a"], N, r["k"], r["kt"], phi)
        assert np.linalg.norm(r["j"][:, col] - jc) < 1e-11 * np.linalg.norm(jc)


@pytest.mark.parametrize("name", ["circle_n64", "circle_n256"])
def test_circle_discrete_farfield_closed_form(name):
    # the far field of the discrete solution, in closed form (Jacobi-Anger
    # and the hat transform), against the oracle's Gauss quadrature of a11
    r = solved(name)
    w = r["w"]
    N = w["N"]
    obs = np.deg2rad(np.arange(0.0, 360.0, 7.0))
    F = solver.farfield(r["curve"], N, r["k"], r["j"], obs)
    for col, phi in enumerate(w["angles"]):
        jc = cf.discrete_solution(r["a"], N, r["k"], r["kt"], phi)
        Fc = cf.discrete_farfield(r["a"], N, r["k"], jc, obs)
        assert np.max(np.abs(F[:, col] - Fc)) < 1e-11 * np.max(np.abs(Fc))


def test_circle_mie_convergence():
    # discrete current converges to the Mie current at O(h^2); far field too
    a, k = 1.0, 8.0
    errs, ferrs = [], []
    for N in (32, 64, 128):
        circ = geometry.Circle(2 * np.pi * a)
        kk, kt, _ = geometry.wavenumbers(circ.L, N, k)
        M = assembly.assemble(circ, N, kk, kt)
        e, hv = solver.planewave_rhs(circ, N, kk, [0.3])
        j, _, _ = solver.dense_solve(M, kk, e, hv)
        th = 2 * np.pi * np.arange(N) / N
        jm = cf.mie_current(a, kk, 0.3, th)
        errs.append(np.linalg.norm(j[:, 0] - jm) / np.linalg.norm(jm))
        po = np.linspace(0, 2 * np.pi, 19)
        F = solver.farfield(circ, N, kk, j, po)
        Fm = cf.mie_farfield(a, kk, 0.3, po)
        ferrs.append(np.linalg.norm(F[:, 0] - Fm) / np.linalg.norm(Fm))
    assert errs[-1] < 0.01
    for e1, e2 in zip(errs[:-1], errs[1:]):
        assert 3.0 < e1 / e2 < 5.0
    assert ferrs[-1] < 2e-3
    assert ferrs[0] / ferrs[-1] > 12.0


def test_generic_contour_path_on_circle_is_circulant_counterpart():
    # the unit circle through the generic (Fourier, Newton, interpolation) path
    # must reproduce the dedicated circle: C - C_c = 0, skeleton rank 0 (Eq. 7)
    N = 64
    cur = geometry.Contour("fourier", {"cos": [1.0]})
    assert abs(cur.L - 2 * np.pi) < 1e-14
    k, kt, _ = geometry.wavenumbers(cur.L, N, 8.0)
    C = assembly.preconditioned(assembly.assemble(cur, N, k, kt))
    Cc = solved("circle_n64")["Cc"]
    assert np.max(np.abs(C - Cc)) < 1e-12 * np.max(np.abs(Cc))
    U, V = solver.reference_skeleton(C, Cc, 1e-10)
    assert U.shape[1] == 0


def test_mie_optical_theorem():
    # the normalisation of the optical theorem used on non-circles, checked
    # on the exact Mie far field
    a, k, phi = 1.0, 8.0, 0.3
    n_obs = 2048
    po = 2.0 * np.pi * np.arange(n_obs) / n_obs
    power = np.sum(np.abs(cf.mie_farfield(a, k, phi, po)) ** 2) * 2.0 * np.pi / n_obs
    Ff = cf.mie_farfield(a, k, phi, np.array([phi]))[0]
    ext = -np.sqrt(8.0 * np.pi / k) * np.real(np.exp(0.25j * np.pi) * Ff)
    assert abs(power - ext) < 1e-12 * power
