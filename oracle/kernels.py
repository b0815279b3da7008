"""Point-pair kernels of the oracle (test infrastructure only).

Sec. II: g_k(r, r') = (i/4) H0^(1)(k |r - r'|).  The double-layer kernel is
d g_k / d n' = (i k / 4) H1^(1)(k R) ((r - r') . n') / R, with R = |r - r'|.
Hankel functions come from scipy (AMOS for complex argument, Cephes Bessel
functions for real argument).
"""

import numpy as np
import scipy.special as sp


def hankel01(kappa, z):
    """H0^(1)(z), H1^(1)(z) for z = kappa * R (kappa real or complex)."""
    if np.imag(kappa) == 0.0:
        z = np.real(z)
        return sp.j0(z) + 1j * sp.y0(z), sp.j1(z) + 1j * sp.y1(z)
    return sp.hankel1(0, z), sp.hankel1(1, z)


def pair_kernels(P, Q, kappa):
    """Kernels between target points P and source points Q (dicts of arrays).

    Returns g = (i/4) H0(kappa R), dgdn = d g / d n' (source normal), and
    ndot = n . n'.
    """
    dx, dy = P["x"] - Q["x"], P["y"] - Q["y"]
    R = np.sqrt(dx * dx + dy * dy)
    H0, H1 = hankel01(kappa, kappa * R)
    g = 0.25j * H0
    dgdn = 0.25j * kappa * H1 * (dx * Q["nx"] + dy * Q["ny"]) / R
    ndot = P["nx"] * Q["nx"] + P["ny"] * Q["ny"]
    return g, dgdn, ndot
