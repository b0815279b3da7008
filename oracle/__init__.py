"""CPU FP64 oracle for the preconditioned TE-CFIE Woodbury-circulant solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or calls this package.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it.

What it computes is the *plain definition* of the discrete problem of the paper
(Consoli et al., "On the Fast Direct Solution of a Preconditioned
Electromagnetic Integral Equation", arXiv 2203.13283):

* the Galerkin matrices of Sec. II, Eq. (4), with piecewise-linear hat
  functions on a mesh that is uniform in arc length (Sec. V), assembled densely
  with converged quadrature (graded composite Gauss-Legendre + Duffy maps near
  the log singularity -- a different rule family from the CUDA path);
* the preconditioned operator C of Eq. (6) and the right-hand side of Eq. (5);
* the dense LU solution of C j = b (no circulant or Woodbury shortcut);
* the circle counterpart C_c and, for small N, a reference Woodbury inverse
  (Eq. 9) built from a truncated full SVD of C - C_c (Eq. 7);
* plane-wave right-hand sides and the far field.

Readings of points the paper leaves open:
S^k~ is the Galerkin single layer with kernel (i/4) H0(k~ R); the hypersingular
operator is assembled in Maue's form; the "suitable average radius" a is
L / (2 pi); C_c uses the same k and k~ as C; exp(-i w t) time convention,
counter-clockwise traversal, outward normal.

Parity pins for this package live in ``tests/test_oracle_*.py`` (closed forms on
the unit circle, Mie series, brute force at tiny N, perimeter closed forms).
"""

from . import quadrature, geometry, kernels, assembly, solver  # noqa: F401
