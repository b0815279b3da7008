"""Helpers shared by the GPU tests: build the library once, make solvers for
the seeded workloads."""

import functools

import numpy as np

import workloads


@functools.lru_cache(maxsize=None)
def built():
    from paper_2203_13283_gb300 import build
    return build.build()


def make_solver(w, **options):
    built()
    from paper_2203_13283_gb300 import Solver
    s = Solver(**options)
    s.contour(w["family"], **w["params"])
    s.mesh(w["N"], w["k"])
    return s


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def colrel(a, b):
    """max over columns of ||a - b|| / ||b||"""
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


def to_np(t):
    return t.detach().cpu().numpy()
