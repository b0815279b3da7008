"""GB300-native Woodbury-circulant fast direct solver for the preconditioned
TE combined-field integral equation on convex 2D PEC contours
(arXiv 2203.13283).  The compute path is libwcs.so (CUDA, sm_103a) behind the
C ABI in include/wcs.h; ``Solver`` marshals torch buffers into it."""

from ._lib import WCSError, load  # noqa: F401


def __getattr__(name):
    if name in ("Solver", "default_options", "quadrature_tables"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
