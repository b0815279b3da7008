"""Batched form (wcs_batch_solve_fourier): several star contours of the
batched workload's family (r = 1 + sum a_m cos(m theta + phi_m), seeded), at
sizes the dense oracle finishes in seconds (including N that are not powers
of two, which take the Bluestein transform), solved in one batch call by two
workers on their own streams.  Each contour's current is checked against the
oracle's dense LU solution (FP64 form 1e-10, mixed form 1e-6) and against a
single-context solve of the same contour (the batch changes nothing but the
scheduling)."""

import numpy as np
import pytest

import workloads
from gpu_common import built, colrel, make_solver, to_np
from oracle import assembly, geometry, solver as osolver

pytestmark = pytest.mark.gpu

SIZES = [320, 200, 256, 150]


@pytest.fixture(scope="module")
def stars():
    base = workloads.star_contours(count=len(SIZES))
    out = []
    for w, N in zip(base, SIZES):
        w = dict(w, N=N, angles=workloads.uniform_angles(4))
        cur = geometry.Contour(w["family"], w["params"])
        k, kt, _ = geometry.wavenumbers(cur.L, N, None)
        M = assembly.assemble(cur, N, k, kt)
        e, hv = osolver.planewave_rhs(cur, N, k, w["angles"])
        j, _, _ = osolver.dense_solve(M, k, e, hv)
        out.append((w, j))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_vs_oracle_and_single_context(stars, precision):
    built()
    from paper_2203_13283_gb300.solver import batch_solve_fourier
    ang = stars[0][0]["angles"]
    contours = [{"cos": w["params"]["cos"], "sin": w["params"]["sin"], "N": w["N"]} for w, _ in stars]
    opts = dict(precision=precision, refine_tol=1e-12 if precision == 0 else 1e-7, max_refine=20)
    tol = 1e-10 if precision == 0 else 1e-6
    js, st = batch_solve_fourier(contours, ang, tol=tol, rank_div=4, seed=5, workers=2,
                                 allow_unconverged=(precision == 1), **opts)
    assert sorted({s["worker"] for s in st}) == [0, 1]
    for (w, jo), j, s in zip(stars, js, st):
        assert s["status"] in (0, 7), s
        err = colrel(j, jo)
        print(w["N"], s, err)
        assert err <= (1e-10 if precision == 0 else 1e-6), (w["N"], err)
        one = make_solver(w, **opts)
        one.assemble()
        one.skeleton(tol, max_rank=w["N"] // 4, seed=5, allow_cap=True)
        one.factor()
        j1 = to_np(one.solve_planewaves(ang, allow_unconverged=True))
        one.close()
        assert np.max(np.abs(j - j1)) <= 1e-13 * np.max(np.abs(j1))


def test_batch_rejects_bad_arguments():
    built()
    from paper_2203_13283_gb300._lib import WCSError
    from paper_2203_13283_gb300.solver import batch_solve_fourier
    with pytest.raises(WCSError):
        batch_solve_fourier([{"cos": [1.0], "N": 8}], [0.0])                 # N < 12
    with pytest.raises(WCSError):
        batch_solve_fourier([{"cos": [-1.0], "N": 64}], [0.0])               # negative mean radius
    with pytest.raises(WCSError):
        batch_solve_fourier([{"cos": [1.0], "N": 64}], [0.0], workers=9)


def test_batch_mid_size_matches_single_contexts():
    # star contours at N = 2048, 1500 (Bluestein) and 1024 in the mixed form:
    # the FP32 circulant transform (powers of two), the shared reference
    # phase of the FP64 far pairs and the FP32 far-pair kernel all run in
    # three concurrent contexts; each contour must equal its single-context
    # solve and meet the residual target
    built()
    from paper_2203_13283_gb300.solver import batch_solve_fourier
    base = workloads.star_contours(count=3, seed=7)
    sizes = [2048, 1500, 1024]
    ang = workloads.uniform_angles(8)
    contours = [{"cos": w["params"]["cos"], "sin": w["params"]["sin"], "N": n} for w, n in zip(base, sizes)]
    opts = dict(precision=1, refine_tol=5e-7, max_refine=12)
    js, st = batch_solve_fourier(contours, ang, tol=1e-6, rank_div=8, seed=3, workers=3, **opts)
    assert sorted({s["worker"] for s in st}) == [0, 1, 2]
    for w, n, j, s in zip(base, sizes, js, st):
        assert s["status"] == 0 and s["rel_residual"] <= 5e-7, s
        one = make_solver(dict(w, N=n), **opts)
        one.assemble()
        one.skeleton(1e-6, max_rank=n // 8, seed=3, allow_cap=True)
        one.factor()
        j1 = to_np(one.solve_planewaves(ang))
        one.close()
        err = np.max(np.abs(j - j1)) / np.max(np.abs(j1))
        print(n, s, f"{err:.1e}")
        assert err <= 1e-13, (n, err)
