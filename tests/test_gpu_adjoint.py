"""GPU parity of the adjoint solve C^H x = b (the conjugate transpose of the
preconditioned operator of Eq. 5, approximate inverse the adjoint of Eq. 9)
against a dense solve with the oracle's C, and the duality identity
<C^-H c, b> = <c, C^-1 b> between adjoint and forward solves."""

import numpy as np
import pytest
import torch

from gpu_common import colrel, make_solver, to_np
from oracle_cache import solved

pytestmark = pytest.mark.gpu


def _rhs(N, B, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((N, B)) + 1j * g.standard_normal((N, B))


@pytest.mark.parametrize("precision,name,tol", [(0, "ellipse_n200", 1e-10), (0, "superellipse_n320", 1e-10),
                                                (1, "superellipse_n320", 1e-6)])
def test_adjoint_vs_oracle(precision, name, tol):
    r = solved(name)
    w = r["w"]
    N = w["N"]
    s = make_solver(w, precision=precision, refine_tol=1e-12 if precision == 0 else 1e-8, max_refine=16)
    s.assemble()
    s.skeleton(1e-8 if precision == 0 else 1e-6, max_rank=N // 4, seed=3, allow_cap=True)
    s.factor()
    b = _rhs(N, 5, 11)
    x = to_np(s.solve_adjoint(torch.from_numpy(b), allow_unconverged=precision == 1))
    x_ref = np.linalg.solve(r["C"].conj().T, b)
    assert colrel(x, x_ref) < tol
    s.close()


def test_adjoint_duality_and_chunks():
    # forward j = C^-1 b and adjoint x = C^-H c satisfy c^H j = x^H b; columns
    # split over several chunks (rhs_chunk 3, 7 columns) give the same answer
    r = solved("ellipse_n200")
    w = r["w"]
    N = w["N"]
    s = make_solver(w, rhs_chunk=3, refine_tol=1e-12, max_refine=16)
    s.assemble()
    s.skeleton(1e-8, max_rank=N // 4, seed=3, allow_cap=True)
    s.factor()
    b, cvec = _rhs(N, 7, 1), _rhs(N, 7, 2)
    x = to_np(s.solve_adjoint(torch.from_numpy(cvec)))
    x1 = to_np(s.solve_adjoint(torch.from_numpy(cvec[:, 2:3])))
    assert np.max(np.abs(x[:, 2:3] - x1)) <= 1e-12 * np.max(np.abs(x1))
    # the dense forward solve with the oracle's C
    j = np.linalg.solve(r["C"], b)
    lhs = np.einsum("ij,ij->j", cvec.conj(), j)
    rhs = np.einsum("ij,ij->j", x.conj(), b)
    assert np.max(np.abs(lhs - rhs) / np.abs(lhs)) < 1e-10
    # the operator product C^H of the library agrees with the oracle's C^H
    y = to_np(s.apply("CH", torch.from_numpy(x)))
    assert colrel(y, cvec) < 1e-10
    s.close()


def test_general_solve_and_autograd():
    # wcs_solve on a general b against the oracle's dense solve; the autograd
    # wrapper's backward is the adjoint solve: for L = Re(c^H x), x = C^-1 b,
    # dL/db (PyTorch convention) = C^-H c
    from paper_2203_13283_gb300 import autograd
    r = solved("superellipse_n320")
    w = r["w"]
    N = w["N"]
    s = make_solver(w, refine_tol=1e-12, max_refine=16)
    s.assemble()
    s.skeleton(1e-8, max_rank=N // 4, seed=3, allow_cap=True)
    s.factor()
    b = _rhs(N, 3, 21)
    cvec = _rhs(N, 3, 22)
    x = to_np(s.solve(torch.from_numpy(b)))
    assert colrel(x, np.linalg.solve(r["C"], b)) < 1e-10
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    ct = torch.from_numpy(cvec).cuda()
    xt = autograd.solve(s, bt)
    loss = torch.real(torch.sum(ct.conj() * xt))
    loss.backward()
    g_ref = np.linalg.solve(r["C"].conj().T, cvec)
    assert colrel(to_np(bt.grad), g_ref) < 1e-10
    # single column (1-D) input
    b1 = torch.from_numpy(b[:, 0].copy()).cuda().requires_grad_(True)
    x1 = autograd.solve(s, b1)
    assert x1.shape == (N,)
    torch.real(torch.sum(ct[:, 0].conj() * x1)).backward()
    assert colrel(to_np(b1.grad), g_ref[:, 0]) < 1e-10
    s.close()
