"""Writes ellipse_n4096_oracle.npz: the oracle's dense solution of Eq. (5) for
the ellipse 1.0 x 0.5 at N = 4096 (10 elements per wavelength) and the far
field of each current at 360 observation angles, for four of the 360
plane-wave incidences of that workload.

Calls only oracle/ (dense FP64 assembly of Sec. II Eq. (4), C of Eq. (6),
LU solve of Eq. (5), far field) and the input descriptions in workloads.py.
Run from the repository root:  python tests/golden/make_ellipse_n4096.py
(about 20 minutes on 8 cores)."""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import assembly, geometry, solver  # noqa: E402

# incidences (degrees) taken from the workload's 1-degree grid: along each
# symmetry axis, and two oblique ones
INCIDENCES_DEG = (0, 37, 90, 211)


def main():
    w = workloads.WORKLOADS["ellipse_n4096"]
    N = w["N"]
    cur = geometry.Contour(w["family"], w["params"])
    k, kt, a = geometry.wavenumbers(cur.L, N, w["k"])
    angles = w["angles"][list(INCIDENCES_DEG)]
    t0 = time.time()
    M = assembly.assemble(cur, N, k, kt)
    t1 = time.time()
    e, hv = solver.planewave_rhs(cur, N, k, angles)
    j, C, b = solver.dense_solve(M, k, e, hv)
    res = np.linalg.norm(C @ j - b, axis=0) / np.linalg.norm(b, axis=0)
    phi = np.deg2rad(np.arange(360.0))
    F = solver.farfield(cur, N, k, j, phi)
    t2 = time.time()
    out = os.path.join(HERE, "ellipse_n4096_oracle.npz")
    np.savez(out, N=N, k=k, kt=kt, L=cur.L, angles=angles, incidences_deg=np.array(INCIDENCES_DEG),
             j=j, phi_obs=phi, F=F, residual=res)
    print(f"wrote {out}: assembly {t1 - t0:.0f} s, solve + far field {t2 - t1:.0f} s, "
          f"LU residual {res.max():.1e}")


if __name__ == "__main__":
    main()
