"""Checkpoint of a factored context (wcs_save / wcs_load).

A context restored from the file rebuilds its mesh and operators and takes
the saved skeleton (Eq. 7) and Woodbury factors (Eq. 9); its solves must be
identical to those of the context that wrote the file, for both forms."""

import pytest
import torch

import workloads
from gpu_common import built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,name", [(0, "ellipse_n200"), (1, "superellipse_n320")])
def test_save_load_gives_identical_solves(tmp_path, precision, name):
    built()
    from paper_2203_13283_gb300 import Solver
    w = workloads.SMALL[name]
    opts = dict(precision=precision, refine_tol=1e-10 if precision == 0 else 1e-7)
    a = Solver(**opts)
    a.contour(w["family"], **w["params"]).mesh(w["N"], w["k"]).assemble()
    rank = a.skeleton(1e-8 if precision == 0 else 1e-6, max_rank=w["N"] // 4, seed=7, allow_cap=True)
    a.factor()
    ang = w["angles"][:4]
    ja = a.solve_planewaves(ang, allow_unconverged=True).clone()
    g = torch.Generator().manual_seed(3)
    rhs = torch.randn(w["N"], 2, dtype=torch.complex128, generator=g)
    xa = a.solve_adjoint(rhs, allow_unconverged=True).clone()
    path = tmp_path / "ctx.wcs"
    a.save(path)
    a.close()
    b = Solver(**opts)
    b.load(path)
    assert b.info()["rank"] == rank
    jb = b.solve_planewaves(ang, allow_unconverged=True)
    xb = b.solve_adjoint(rhs, allow_unconverged=True)
    torch.cuda.synchronize()
    assert torch.equal(ja, jb)
    # the capacitance inverse travels with the file: adjoint solves match too
    assert torch.equal(xa, xb)
    b.close()


def test_load_rejects_other_options(tmp_path):
    built()
    from paper_2203_13283_gb300 import Solver
    from paper_2203_13283_gb300._lib import WCSError
    w = workloads.SMALL["ellipse_n200"]
    a = Solver(precision=0)
    a.contour(w["family"], **w["params"]).mesh(w["N"], w["k"]).assemble()
    a.skeleton(1e-6, seed=1)
    a.factor()
    path = tmp_path / "ctx.wcs"
    a.save(path)
    a.close()
    b = Solver(precision=0, q_near=10)
    with pytest.raises(WCSError):
        b.load(path)
    with pytest.raises(WCSError):
        b.load(tmp_path / "missing.wcs")
    b.close()


def test_load_rejects_corrupted_or_truncated_file_and_keeps_context(tmp_path):
    # a real checkpoint with one payload byte flipped, and one cut short: both
    # rejected (WCS_ERR_ARG) before any device work; the context that refused
    # them still solves exactly as before, and the intact file still loads
    built()
    from paper_2203_13283_gb300 import Solver
    from paper_2203_13283_gb300._lib import WCS_ERR_ARG, WCSError
    w = workloads.SMALL["ellipse_n200"]
    a = Solver(precision=0, refine_tol=1e-10)
    a.contour(w["family"], **w["params"]).mesh(w["N"], w["k"]).assemble()
    a.skeleton(1e-8, seed=4)
    a.factor()
    ang = w["angles"][:3]
    ja = a.solve_planewaves(ang).clone()
    path = tmp_path / "ctx.wcs"
    a.save(path)
    data = path.read_bytes()
    bad = bytearray(data)
    bad[len(data) // 2] ^= 0x01
    (tmp_path / "flip.wcs").write_bytes(bytes(bad))
    (tmp_path / "cut.wcs").write_bytes(data[:-1000])
    for name, word in (("flip.wcs", "checksum"), ("cut.wcs", "truncated")):
        with pytest.raises(WCSError) as ei:
            a.load(tmp_path / name)
        assert ei.value.status == WCS_ERR_ARG and word in str(ei.value), str(ei.value)
    assert torch.equal(a.solve_planewaves(ang), ja)
    a.close()
    b = Solver(precision=0, refine_tol=1e-10)
    b.load(path)
    assert torch.equal(b.solve_planewaves(ang), ja)
    b.close()
