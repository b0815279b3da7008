"""Per-process cache of oracle results for the small workloads (tests only)."""

import functools

import numpy as np

import workloads
from oracle import assembly, geometry, solver


def curve_of(w):
    if w["family"] == "circle":
        return geometry.Circle(2.0 * np.pi * w["params"]["a"])
    return geometry.Contour(w["family"], w["params"])


@functools.lru_cache(maxsize=None)
def solved(name):
    """Oracle matrices, C, C_c, RHS and dense solution for workloads.SMALL[name]."""
    w = workloads.SMALL[name]
    cur = curve_of(w)
    N = w["N"]
    k, kt, a = geometry.wavenumbers(cur.L, N, w["k"])
    M = assembly.assemble(cur, N, k, kt)
    Mc = assembly.assemble(geometry.Circle(cur.L), N, k, kt)
    e, hv = solver.planewave_rhs(cur, N, k, w["angles"])
    j, C, b = solver.dense_solve(M, k, e, hv)
    Cc = assembly.preconditioned(Mc)
    return dict(w=w, curve=cur, k=k, kt=kt, a=a, M=M, Mc=Mc, C=C, Cc=Cc, e=e, h=hv, b=b, j=j)
