"""GPU parity of the mixed-precision form (tensor-core products; far pairs in
FP64 by default, or in FP32 with zfast > 0): against the CPU oracle on small
workloads and against the FP64 form (itself pinned to the oracle) at N = 4096.
The bar is the mixed form's target, 1e-6 relative per column in the surface
current."""

import numpy as np
import pytest
import torch

import workloads
from gpu_common import colrel, make_solver, to_np
from oracle_cache import solved

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("zfast", [0.0, 9.0])
@pytest.mark.parametrize("name", ["ellipse_n200", "superellipse_n320", "star_n200"])
def test_mixed_solve_vs_oracle(name, zfast):
    r = solved(name)
    w = r["w"]
    s = make_solver(w, precision=1, refine_tol=1e-8, max_refine=12, zfast=zfast)
    s.assemble()
    s.skeleton(1e-6, max_rank=w["N"] // 4, seed=5, allow_cap=True)
    s.factor()
    j = to_np(s.solve_planewaves(w["angles"], allow_unconverged=True))
    assert colrel(j, r["j"]) < 1e-6
    s.close()


@pytest.fixture(scope="module")
def pair4096():
    w = dict(workloads.WORKLOADS["superellipse_n32768"])
    w["N"] = 4096
    s64 = make_solver(w)
    s64.assemble()
    sm = make_solver(w, precision=1, refine_tol=1e-8, max_refine=16)
    sm.assemble()
    yield w, s64, sm
    s64.close()
    sm.close()


def test_mixed_operator_products(pair4096):
    w, s64, sm = pair4096
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(w["N"], 40, dtype=torch.complex128, device="cuda", generator=g)
    for op in ("S", "D", "DT", "N", "C", "CH"):
        err = colrel(to_np(sm.apply(op, X)), to_np(s64.apply(op, X)))
        assert err < 2e-6, (op, err)


def test_mixed_solve_vs_fp64_capacitance_iteration(pair4096):
    # rank 512 >= 256: the mixed form inverts the capacitance matrix by
    # Newton-Schulz on the tensor cores, closed by two steps with exact
    # products; their residual ||I - K K^-1||_F / sqrt(r), measured with an
    # exact product, is set by those products: six 7-bit slices keep 42 bits
    # below each chunk's scale, so each entry of K X carries ~2^-42 sqrt(r)
    # (~5e-12 at r = 512) of its terms' size; 1e-10 allows for ||K^-1||
    w, s64, sm = pair4096
    ang = workloads.uniform_angles(48)
    s64.skeleton(1e-2, seed=2)
    s64.factor()
    j64 = to_np(s64.solve_planewaves(ang))
    rank = sm.skeleton(1e-6, max_rank=512, seed=2, allow_cap=True)
    assert rank == 512
    sm.factor()
    kres = sm.info()["capacitance_residual"]
    print("capacitance residual", kres)
    assert 0.0 <= kres <= 1e-10
    jm = to_np(sm.solve_planewaves(ang, allow_unconverged=True))
    assert colrel(jm, j64) < 1e-6
    assert sm.last_solve["rel_residual"] < 1e-6
