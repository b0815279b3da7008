"""Pins of the oracle's solver pieces: brute-force Woodbury, invariants, energy balance (CPU)."""

import numpy as np
import pytest

from oracle import assembly, geometry, solver
from oracle_cache import solved


def test_woodbury_equals_dense_inverse_full_rank():
    r = solved("ellipse_n200")
    C, Cc, b = r["C"], r["Cc"], r["b"]
    U, V = solver.reference_skeleton(C, Cc, 0.0)
    assert U.shape[1] == C.shape[0]
    x = solver.woodbury_solve(Cc, U, V, b)
    assert np.linalg.norm(x - r["j"]) < 1e-10 * np.linalg.norm(r["j"])


def test_woodbury_truncated_error_tracks_tolerance():
    r = solved("ellipse_n200")
    C, Cc, b = r["C"], r["Cc"], r["b"]
    prev = None
    for tol in (1e-4, 1e-7, 1e-10):
        U, V = solver.reference_skeleton(C, Cc, tol)
        x = solver.woodbury_solve(Cc, U, V, b)
        err = np.linalg.norm(x - r["j"]) / np.linalg.norm(r["j"])
        # ||C^-1|| ||C - C_c - U V^T|| bound (C well conditioned)
        assert err < 100 * tol
        if prev is not None:
            assert U.shape[1] >= prev
        prev = U.shape[1]
    # at the paper's compression parameter (Sec. IV, Fig. 3) the skeleton is
    # well below full rank
    U, V = solver.reference_skeleton(C, Cc, 0.015)
    assert U.shape[1] < 0.5 * C.shape[0]


def test_ellipse_mirror_symmetry():
    # ellipse symmetric under y -> -y; node i <-> node N - i; incidence at 0 deg
    r = solved("ellipse_n256")
    j = r["j"][:, 0]
    N = len(j)
    jm = j[(-np.arange(N)) % N]
    assert np.max(np.abs(j - jm)) < 1e-10 * np.max(np.abs(j))


def test_reciprocity_farfield():
    # F(phi_o; phi_i) = F(phi_i + pi; phi_o + pi), up to discretisation error
    r = solved("superellipse_n320")
    cur, k = r["curve"], r["k"]
    N = r["w"]["N"]
    M, C = r["M"], r["C"]
    pi_, po = 0.4, 2.1
    e, hv = solver.planewave_rhs(cur, N, k, [pi_, po + np.pi])
    b = solver.preconditioned_rhs(M, k, e, hv)
    j = np.linalg.solve(C, b)
    F1 = solver.farfield(cur, N, k, j[:, :1], [po])[0, 0]
    F2 = solver.farfield(cur, N, k, j[:, 1:], [pi_ + np.pi])[0, 0]
    assert abs(F1 - F2) < 2e-3 * abs(F1)


@pytest.mark.parametrize("name", ["ellipse_n200", "star_n200", "superellipse_n320"])
def test_optical_theorem(name):
    # energy balance of a lossless scatterer: the scattered power equals the
    # extinction read off the forward far field,
    #   int |F|^2 dphi = -sqrt(8 pi / k) Re(e^{i pi/4} F(phi_inc)),
    # exact for the Mie series (normalisation and signs), O(h^2) here; a sign
    # slip in an operator or the right-hand side breaks it at O(1)
    r = solved(name)
    w = r["w"]
    n_obs = 720                                        # trapezoid on a periodic, band-limited F
    po = 2.0 * np.pi * np.arange(n_obs) / n_obs
    F = solver.farfield(r["curve"], w["N"], r["k"], r["j"], np.concatenate([po, w["angles"]]))
    power = np.sum(np.abs(F[:n_obs]) ** 2, axis=0) * 2.0 * np.pi / n_obs
    for b in range(len(w["angles"])):
        ext = -np.sqrt(8.0 * np.pi / r["k"]) * np.real(np.exp(0.25j * np.pi) * F[n_obs + b, b])
        assert abs(power[b] - ext) < 1e-3 * power[b]


def test_quadrature_order_convergence():
    # entries agree when every rule is refined (Sec. II integrals are converged)
    cur = geometry.Contour("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0})
    N = 96
    k, kt, _ = geometry.wavenumbers(cur.L, N)
    M1 = assembly.assemble(cur, N, k, kt)
    M2 = assembly.assemble(cur, N, k, kt, rules=assembly.Rules(q_far=9, q_near=24, n_sing=16))
    for key in ("S", "D", "Dt", "N"):
        assert np.max(np.abs(M1[key] - M2[key])) < 2e-12 * np.max(np.abs(M2[key])), key
