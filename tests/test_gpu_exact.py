"""Exact tensor-core products (exact.cu) and the mixed form's exact refinement
residual (wcs_options.exact_residual).

* wcs_gemm_exact against the FP64 product, entry by entry.  The slices of a
  value are exact to 2^-42 of the largest entry of its chunk of 1024 (cmax),
  and the dropped slice pairs are below 2^-42 cmax_A cmax_B per term, so the
  error of D_ij is bounded by 2^-40 sum_k (cmax_A |B_jk| + |A_ik| cmax_B +
  cmax_A cmax_B); for data without a wide range inside a chunk that is
  within 2^-38 (|A| |B|^T).  Both are checked, with entries spanning eight
  decades across chunks and within chunks, and K not a multiple of 1024.
  The drained split-bf16 product of the same inputs is ~1e-7 off.
* The mixed form with exact residuals refines to 1e-11 against its stored
  operator, where the drained residual stalls near 2e-7, and its solutions
  stay within 1e-6 of the dense FP64 oracle (the operator's own accuracy)."""

import numpy as np
import pytest
import torch

import workloads
from gpu_common import built, colrel, make_solver, to_np
from oracle_cache import solved

pytestmark = pytest.mark.gpu


def _chunk_max(X, chunk=1024):
    K = X.shape[1]
    out = np.empty_like(X)
    for c0 in range(0, K, chunk):
        out[:, c0:c0 + chunk] = np.max(np.abs(X[:, c0:c0 + chunk]), axis=1, keepdims=True)
    return out


@pytest.mark.parametrize("M,Nc,K,within", [(300, 70, 3000, False), (1024, 512, 4096, False),
                                           (300, 70, 3000, True)])
def test_gemm_exact_componentwise(M, Nc, K, within):
    built()
    from paper_2203_13283_gb300.solver import gemm_exact, gemm_split_bf16
    g = np.random.default_rng(M + K + within)
    if within:      # magnitudes over eight decades inside every chunk
        scale = 10.0 ** g.uniform(-4, 4, size=K)
    else:           # eight decades across chunks, smooth inside
        scale = np.repeat(10.0 ** g.uniform(-4, 4, size=(K + 1023) // 1024), 1024)[:K]
    A = g.standard_normal((M, K)) * scale * 10.0 ** g.uniform(-1.5, 1.5, size=(M, 1))
    B = g.standard_normal((Nc, K)) / np.sqrt(scale)
    ref = A @ B.T
    D = to_np(gemm_exact(A, B))
    cA, cB = _chunk_max(A), _chunk_max(B)
    chunked = 2.0 ** -40 * (cA @ np.abs(B).T + np.abs(A) @ cB.T + cA @ cB.T)
    assert np.all(np.abs(D - ref) <= chunked), np.max(np.abs(D - ref) / chunked)
    plain = np.abs(A) @ np.abs(B).T
    err = np.max(np.abs(D - ref) / plain)
    acc = to_np(gemm_split_bf16(A, B, planes=3, accurate=True))
    err_acc = np.max(np.abs(acc - ref) / plain)
    print(f"within={within}: exact {err:.1e}, drained split-bf16 {err_acc:.1e}")
    if not within:
        assert err <= 2.0 ** -38, err
        assert err_acc > 100 * err


@pytest.mark.parametrize("name", ["ellipse_n200", "superellipse_n320"])
def test_exact_residual_refines_below_the_drained_floor(name):
    d = solved(name)
    w = d["w"]
    opts = dict(precision=1, max_refine=30, rhs_chunk=256)
    s = make_solver(w, exact_residual=1, refine_tol=1e-11, **opts)
    s.assemble()
    s.skeleton(1e-4, max_rank=w["N"] // 8, seed=2, allow_cap=True)
    s.factor()
    j = to_np(s.solve_planewaves(w["angles"]))
    st = s.last_solve
    s.close()
    print(name, st)
    assert st["rel_residual"] <= 1e-11
    assert colrel(j, d["j"]) <= 1e-6
    # the drained residual of the same context cannot get there
    t = make_solver(w, exact_residual=0, refine_tol=1e-11, **opts)
    t.assemble()
    t.skeleton(1e-4, max_rank=w["N"] // 8, seed=2, allow_cap=True)
    t.factor()
    jt = to_np(t.solve_planewaves(w["angles"], allow_unconverged=True))
    stt = t.last_solve
    t.close()
    assert stt["rel_residual"] > 1e-9
    # both describe the same stored operator: their solutions agree to its accuracy
    assert colrel(jt, j) <= 1e-6


def test_exact_residual_ellipse4096_golden():
    # the N = 4096 ellipse of the golden file with exact residuals: refined to
    # 1e-10, within 1e-6 of the oracle's dense LU solution
    import os
    w = workloads.WORKLOADS["ellipse_n4096"]
    gd = dict(np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ellipse_n4096_oracle.npz")))
    s = make_solver(w, precision=1, exact_residual=1, refine_tol=1e-10, max_refine=30, rhs_chunk=64, block=64)
    s.assemble()
    s.skeleton(1e-6, max_rank=w["N"] // 8, seed=1, allow_cap=True)
    s.factor()
    j = to_np(s.solve_planewaves(gd["angles"]))
    st = s.last_solve
    s.close()
    print(st)
    assert st["rel_residual"] <= 1e-10
    assert colrel(j, gd["j"]) <= 1e-6
