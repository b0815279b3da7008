"""The ellipse 1.0 x 0.5 at N = 4096 (10 elements per wavelength, skeleton
tolerance 1e-10) against the oracle's dense LU solution of Eq. (5) at the
same size, stored by tests/golden/make_ellipse_n4096.py (which calls only
oracle/): four of the workload's 360 incidences (0, 37, 90 and 211 degrees),
their currents and far fields at 360 observation angles.

FP64 form: relative 2-norm error <= 1e-10 per column in the current and in the
far field.  Mixed form: <= 1e-6 per column."""

import os

import numpy as np
import pytest
import torch

import workloads
from gpu_common import make_solver, to_np

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ellipse_n4096_oracle.npz")


@pytest.fixture(scope="module")
def golden():
    return dict(np.load(GOLDEN))


def _colrel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_ellipse4096_vs_oracle_golden(golden, precision):
    w = workloads.WORKLOADS["ellipse_n4096"]
    assert int(golden["N"]) == w["N"]
    if precision == 0:
        s = make_solver(w, precision=0, refine_tol=1e-12, max_refine=20)
        s.assemble()
        s.skeleton(w["tol"], seed=1)                 # tolerance 1e-10 of the workload
    else:
        s = make_solver(w, precision=1, refine_tol=1e-7, max_refine=12, rhs_chunk=64, block=64)
        s.assemble()
        s.skeleton(1e-6, max_rank=w["N"] // 8, seed=1, allow_cap=True)
    s.factor()
    info = s.info()
    assert abs(info["k"] - float(golden["k"])) <= 1e-12 * float(golden["k"])
    ang = golden["angles"]
    assert np.allclose(ang, w["angles"][golden["incidences_deg"]])
    j = to_np(s.solve_planewaves(ang, allow_unconverged=(precision == 1)))
    F = to_np(s.farfield(torch.tensor(j, device="cuda"), golden["phi_obs"]))
    s.close()
    ej, eF = _colrel(j, golden["j"]), _colrel(F, golden["F"])
    print(f"precision {precision}: current {ej}, far field {eF}")
    tol = 1e-10 if precision == 0 else 1e-6
    assert np.all(ej <= tol), ej
    assert np.all(eF <= tol), eF
