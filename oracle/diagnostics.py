"""Spectral diagnostics of Sec. IV-V (test infrastructure only).

Sec. IV: the spectrum of the preconditioned operator C of Eq. (5) is largest
around the surface resonance, where the spatial frequency m of a singular
vector matches k a; elsewhere it is close to the halved identity, but the
discretisation leaves a constant offset in that (elliptic) part.  Sec. V:
for C - C_c the elliptic part decays at high spatial frequencies, which is
what makes the skeleton of Eq. (7) small; the rank at a fixed compression
parameter is reported as a function of k together with the accuracy of the
compressed solve.

Galerkin matrices carry the element size, so the spectra here are those of
G^-1 C and G^-1 (C - C_c) (the halved identity is then 1/2); the rank uses
the same rule as the skeleton (singular values of C - C_c above
eps * ||C_c||_2).  Dense SVDs, CPU only.
"""

import numpy as np

from . import assembly, geometry, solver


def operators(curve, N, k=None):
    """(C, C_c, G, k, a) for the contour at N elements (k: 10 per wavelength if None)."""
    k, kt, a = geometry.wavenumbers(curve.L, N, k)
    M = assembly.assemble(curve, N, k, kt)
    Mc = assembly.assemble(geometry.Circle(curve.L), N, k, kt)
    return assembly.preconditioned(M), assembly.preconditioned(Mc), M["G"], k, a, M


def spectrum_by_frequency(X, G):
    """Singular values of G^-1 X and the spatial frequency |m| (0..N/2) that
    dominates each right singular vector, sorted by that frequency."""
    N = X.shape[0]
    _, s, Vh = np.linalg.svd(np.linalg.solve(G, X))
    f = np.abs(np.fft.fft(Vh.conj().T, axis=0))
    m = np.argmax(f, axis=0)
    m = np.minimum(m, N - m)
    order = np.argsort(m, kind="stable")
    return m[order], s[order]


def rank_and_error(curve, N, eps, angles, k=None):
    """Skeleton rank at compression parameter eps and the relative error of
    the compressed (Woodbury, Eq. 9) solve against the dense solve."""
    C, Cc, _, k, a, M = operators(curve, N, k)
    U, V = solver.reference_skeleton(C, Cc, eps)
    e, hv = solver.planewave_rhs(curve, N, k, angles)
    b = solver.preconditioned_rhs(M, k, e, hv)
    j = np.linalg.solve(C, b)
    jw = solver.woodbury_solve(Cc, U, V, b)
    err = float(np.max(np.linalg.norm(jw - j, axis=0) / np.linalg.norm(j, axis=0)))
    return U.shape[1], err, k


def frequency_response(X, G):
    """||G^-1 X v_m|| for the unit Fourier vectors v_m(j) = e^{2 pi i m j / N} / sqrt(N),
    m = 0..N-1: how strongly X acts at each spatial frequency (Sec. IV-V).
    For a circulant X (the circle) this is |mu_X(m) / mu_G(m)| exactly."""
    N = X.shape[0]
    j = np.arange(N)
    V = np.exp(2j * np.pi * np.outer(j, np.arange(N)) / N) / np.sqrt(N)
    return np.linalg.norm(np.linalg.solve(G, X @ V), axis=0)
