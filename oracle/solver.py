"""Right-hand sides, dense solves, reference Woodbury and far field (test infrastructure only).

Time convention exp(-i w t).  Plane wave of propagation angle phi,
d = (cos phi, sin phi), phase reference at the origin:
    H_z^inc = exp(i k d . r),   E_t^inc / eta = (d . n) exp(i k d . r)
(E = (i / (w eps)) curl(z H_z) gives E_t / eta = -(i/k) dH_z/dn).

Sec. II, Eq. (4): [e]_i = int lambda_i E_t^inc, [h]_i = int lambda_i H_z^inc;
only e / eta enters, so eta = 1 is used throughout.
Sec. III, Eq. (5): b = -i k S~ G^{-1} (e/eta) - (G/2 + D~) G^{-1} h.
Sec. V, Eq. (9): C^{-1} = C_c^{-1} - C_c^{-1} U (I + V^T C_c^{-1} U)^{-1} V^T C_c^{-1}.

Far field: H^s(rho, phi_o) ~ F(phi_o) e^{i k rho} / sqrt(rho) with
F(phi_o) = (i k e^{i pi/4} / sqrt(8 pi k)) int (x^ . n') e^{-i k x^ . r'} j(s') ds',
x^ = (cos phi_o, sin phi_o), obtained from H^s = -D^k[j] in the far zone.
"""

import numpy as np

from . import quadrature as qd
from .assembly import ElementGeometry, preconditioned


def planewave_rhs(curve, N, k, angles, q=16):
    """Galerkin projections (e/eta, h) of plane waves, arrays of shape (N, B)."""
    geo = ElementGeometry(curve, N)
    h = geo.h
    xg, wg = qd.gauss_legendre01(q)
    P = geo.at(np.arange(N), xg)                      # (N, q)
    angles = np.atleast_1d(np.asarray(angles, float))
    dx, dy = np.cos(angles), np.sin(angles)           # (B,)
    phase = k * (P["x"][..., None] * dx + P["y"][..., None] * dy)
    Hz = np.exp(1j * phase)                           # (N, q, B)
    Et = (P["nx"][..., None] * dx + P["ny"][..., None] * dy) * Hz
    e = np.zeros((N, len(angles)), complex)
    hv = np.zeros_like(e)
    for a, phi in enumerate((1.0 - xg, xg)):
        wq = h * wg * phi
        rows = (np.arange(N) + a) % N
        np.add.at(e, rows, np.einsum("q,nqb->nb", wq, Et))
        np.add.at(hv, rows, np.einsum("q,nqb->nb", wq, Hz))
    return e, hv


def preconditioned_rhs(M, k, e, hv):
    """b of Eq. (5) for e/eta and h."""
    G = M["G"]
    return -1j * k * (M["S"] @ np.linalg.solve(G, e)) - (0.5 * G + M["Dt"]) @ np.linalg.solve(G, hv)


def dense_solve(M, k, e, hv):
    """Plain-definition solution j of Eq. (5) by dense LU; returns (j, C, b)."""
    C = preconditioned(M)
    b = preconditioned_rhs(M, k, e, hv)
    return np.linalg.solve(C, b), C, b


def spectral_norm_circulant(Cc):
    """||C_c||_2 = max |eigenvalue| of the (normal) circulant C_c."""
    return np.max(np.abs(np.fft.fft(Cc[0])))


def reference_skeleton(C, Cc, tol):
    """Truncated SVD of C - C_c (Eq. 7): keep sigma_i > tol * ||C_c||_2.

    Returns (U, V) with C - C_c ~= U V^T.
    """
    W, s, Zh = np.linalg.svd(C - Cc)
    thr = tol * spectral_norm_circulant(Cc)
    r = int(np.sum(s > thr))
    U = W[:, :r] * s[:r]
    V = Zh[:r].T.copy()                      # V^T = Zh[:r]
    return U, V


def woodbury_solve(Cc, U, V, b):
    """Eq. (9) with dense solves against C_c (no FFT): returns C^{-1} b."""
    Y = np.linalg.solve(Cc, b)
    if U.shape[1] == 0:
        return Y
    W = np.linalg.solve(Cc, U)
    K = np.eye(U.shape[1]) + V.T @ W
    return Y - W @ np.linalg.solve(K, V.T @ Y)


def farfield(curve, N, k, j, phi_obs, q=16):
    """F(phi_o) for each column of j (hat coefficients); returns (n_phi, B)."""
    geo = ElementGeometry(curve, N)
    h = geo.h
    xg, wg = qd.gauss_legendre01(q)
    P = geo.at(np.arange(N), xg)
    phi_obs = np.atleast_1d(np.asarray(phi_obs, float))
    ox, oy = np.cos(phi_obs), np.sin(phi_obs)
    j = np.asarray(j).reshape(N, -1)
    jq = (1.0 - xg)[None, :, None] * j[:, None, :] + xg[None, :, None] * np.roll(j, -1, axis=0)[:, None, :]
    ker = ((P["nx"][..., None] * ox + P["ny"][..., None] * oy)
           * np.exp(-1j * k * (P["x"][..., None] * ox + P["y"][..., None] * oy)))   # (N, q, n_phi)
    integral = h * np.einsum("q,nqo,nqb->ob", wg, ker, jq)
    return 1j * k * np.exp(0.25j * np.pi) / np.sqrt(8.0 * np.pi * k) * integral
