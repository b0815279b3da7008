"""Spectral diagnostics of Sec. IV-V computed by the library on the GPU.

* circle_spectrum: the spectrum of the preconditioned operator of Eq. (5) on a
  circle, |mu_C / mu_G| per Fourier index, from the circulant eigenvalues
  (the paper's first figure).
* frequency_response: ||G^-1 X v_m|| for the unit Fourier vectors v_m and
  X = C or C - C_c: where the operator acts strongly (up to the resonance
  |m| ~ k a) and how the remainder C - C_c dies off at high frequency, which
  is what keeps the skeleton of Eq. (7) small.
* rank_sweep: the skeleton rank at a compression parameter eps and the error
  of the compressed (Woodbury, Eq. 9) solve against the refined solve, for a
  sequence of mesh sizes at 10 elements per wavelength (k grows with N).

Every number comes from libwcs calls; torch only holds the blocks.
"""

import numpy as np
import torch

from .solver import Solver


def circle_spectrum(N, k, a=1.0, **options):
    """|mu_C(m) / mu_G(m)|, m = 0..N-1, on the circle of radius a (FP64 form)."""
    s = Solver(precision=0, **options)
    try:
        s.contour("circle", a=a).mesh(N, k).assemble()
        muC = s.circulant_eigs("CC").cpu().numpy()
        muG = s.circulant_eigs("G").cpu().numpy()
    finally:
        s.close()
    return np.abs(muC / muG)


def frequency_response(solver, which="C", chunk=256):
    """||G^-1 X v_m|| for m = 0..N-1 with X = C ("C") or C - C_c ("C-Cc");
    solver is an assembled Solver (FP64 form for full accuracy)."""
    N = solver.N
    j = torch.arange(N, dtype=torch.float64, device=solver.device)
    out = np.empty(N)
    for m0 in range(0, N, chunk):
        m = torch.arange(m0, min(N, m0 + chunk), dtype=torch.float64, device=solver.device)
        V = torch.exp(2j * np.pi * torch.outer(j, m) / N) / np.sqrt(N)
        Y = solver.apply("C", V)
        if which == "C-Cc":
            Y = Y - solver.apply("CC", V)
        Y = solver.apply("GINV", Y)
        out[m0:m0 + V.shape[1]] = torch.linalg.vector_norm(Y, dim=0).cpu().numpy()
    return out


def rank_sweep(family, params, Ns, eps=0.015, angles=(0.0, 1.0), seed=1):
    """[(N, k, rank, compressed-solve error)] at 10 elements per wavelength,
    FP64 form: the rank of the skeleton of C - C_c whose range finder stops
    once every new projected sample is below eps ||C_c||_2 (wcs_skeleton's
    tolerance eps * 10 sqrt(2 / pi)), and the relative error of the Woodbury
    solve of Eq. (9) alone against the solve refined to 1e-12."""
    rows = []
    tol = eps * 10.0 * np.sqrt(2.0 / np.pi)
    for N in Ns:
        s = Solver(precision=0, refine_tol=1e-12, max_refine=60, rhs_chunk=64)
        try:
            s.contour(family, **params).mesh(N).assemble()
            r = s.skeleton(tol, seed=seed)
            s.factor()
            j = s.solve_planewaves(np.asarray(angles, float))
            b = s.apply("C", j)
            jw = s.woodbury_apply(b)
            err = (torch.linalg.vector_norm(jw - j, dim=0) / torch.linalg.vector_norm(j, dim=0)).max().item()
            rows.append((int(N), float(s.info()["k"]), int(r), float(err)))
        finally:
            s.close()
    return rows
