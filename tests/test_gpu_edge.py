"""Edge cases of the solve entry points: an empty batch, batches split into
ragged chunks (the chunk loop must not change any column), and right-hand
sides given directly (wcs_solve_rhs) against the plane-wave path."""

import numpy as np
import pytest
import torch

import workloads
from gpu_common import make_solver, to_np

pytestmark = pytest.mark.gpu


def _factored(w, **opt):
    s = make_solver(w, **opt)
    s.assemble()
    s.skeleton(1e-8, seed=2)
    s.factor()
    return s


def test_empty_batch():
    w = workloads.SMALL["ellipse_n200"]
    s = _factored(w)
    j = s.solve_planewaves(np.zeros(0))
    assert tuple(j.shape) == (w["N"], 0)
    Y = s.apply("C", torch.zeros((w["N"], 0), dtype=torch.complex128, device="cuda"))
    assert tuple(Y.shape) == (w["N"], 0)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_chunks_match_one_chunk(precision):
    w = workloads.SMALL["ellipse_n200"]
    ang = np.linspace(0.0, 2.0 * np.pi, 7, endpoint=False)
    opt = dict(precision=precision, refine_tol=1e-10 if precision == 0 else 1e-7)
    a = _factored(w, rhs_chunk=256, **opt)
    ja = to_np(a.solve_planewaves(ang, allow_unconverged=True))
    a.close()
    b = _factored(w, rhs_chunk=3, **opt)     # chunks of 3, 3, 1 columns
    jb = to_np(b.solve_planewaves(ang, allow_unconverged=True))
    b.close()
    tol = 1e-12 if precision == 0 else 1e-6
    assert np.max(np.abs(ja - jb)) <= tol * np.max(np.abs(ja))


def test_solve_rhs_matches_planewaves():
    w = workloads.SMALL["superellipse_n320"]
    s = _factored(w, refine_tol=1e-11)
    ang = np.array([0.0, 0.7, 2.0])
    j1 = to_np(s.solve_planewaves(ang))
    e, hv = s.planewave_rhs(ang)
    j2 = to_np(s.solve_rhs(e, hv))
    assert np.max(np.abs(j1 - j2)) <= 1e-11 * np.max(np.abs(j1))
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_inputs_are_rejected(precision):
    # a NaN injected on the host into an angle, a general right-hand side or
    # the Galerkin data e/eta must give WCS_ERR_ARG (not a "converged" NaN
    # current), and the context must solve normally afterwards
    from paper_2203_13283_gb300._lib import WCS_ERR_ARG, WCSError
    w = workloads.SMALL["ellipse_n200"]
    s = _factored(w, precision=precision, refine_tol=1e-10 if precision == 0 else 1e-7)
    ang = np.array([0.0, 0.5, 1.0])
    good = to_np(s.solve_planewaves(ang, allow_unconverged=True))
    bad = ang.copy()
    bad[1] = np.nan
    with pytest.raises(WCSError) as ei:
        s.solve_planewaves(bad)
    assert ei.value.status == WCS_ERR_ARG and "angle 1" in str(ei.value)
    b = np.ones((w["N"], 2), dtype=complex)
    b[17, 1] = np.inf
    with pytest.raises(WCSError) as ei:
        s.solve(b)
    assert ei.value.status == WCS_ERR_ARG and "not finite" in str(ei.value)
    with pytest.raises(WCSError) as ei:
        s.solve_adjoint(b)
    assert ei.value.status == WCS_ERR_ARG
    e, hv = s.planewave_rhs(ang)
    e = e.clone()
    e[5, 2] = complex(float("nan"), 0.0)
    with pytest.raises(WCSError) as ei:
        s.solve_rhs(e, hv)
    assert ei.value.status == WCS_ERR_ARG
    again = to_np(s.solve_planewaves(ang, allow_unconverged=True))
    assert np.array_equal(good, again)
    s.close()
