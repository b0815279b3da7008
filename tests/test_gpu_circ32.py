"""FP32 circulant applies of the mixed form (Sec. V: C_c = F^-1 diag(mu_C) F).

In the mixed form, for power-of-two N in [1024, 65536], C_c, C_c^H, C_c^-1 and
C_c^-H are applied by a three-pass FP32 transform with the FP64 eigenvalues
(these applies serve the Woodbury approximate inverse of Eq. 9 and the
sampling of C - C_c, which refinement corrects).  Each is compared with
numpy.fft in FP64 using the library's own mu_C, column by column in the
relative 2-norm.

Bound: the input, each of the 2 log2 N radix-2 stages and the twiddles round
to FP32 (u = 2^-24 ~ 6e-8) with a relative error of a few u per complex
multiply-add; the errors of different stages are independent, so the 2-norm
error grows like c u sqrt(2 log2 N) ~ 3 * 6e-8 * 5.5 = 1e-6 at N = 32768.  The
test allows 5e-6, and checks that the error is above 1e-9 (the FP32 transform
ran, not the FP64 one).  Lengths: 1024 (32 x 32), 4096, 8192 (the
shape-gradient ellipse, 128 x 64) and 32768 (the benchmark superellipse,
256 x 128).  N = 5000 is not a power of two and keeps the FP64 transform in
the mixed form too (2e-12)."""

import numpy as np
import pytest
import torch

from gpu_common import make_solver, to_np

pytestmark = pytest.mark.gpu

CASES = [
    ("ellipse", {"ax": 1.0, "ay": 0.5}, 1024),
    ("ellipse", {"ax": 1.0, "ay": 0.5}, 4096),
    ("ellipse", {"ax": 1.0, "ay": 0.7}, 8192),
    ("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0}, 32768),
    ("ellipse", {"ax": 1.0, "ay": 0.5}, 5000),
]


@pytest.mark.parametrize("family,params,N", CASES, ids=[f"{c[0]}_n{c[2]}" for c in CASES])
def test_mixed_circulant_applies(family, params, N):
    w = dict(family=family, params=params, N=N, k=None)
    s = make_solver(w, precision=1, rhs_chunk=64)
    s.assemble()
    mu = to_np(s.circulant_eigs("CC"))
    g = np.random.default_rng(N + 1)
    X = g.standard_normal((N, 5)) + 1j * g.standard_normal((N, 5))
    X[:, 4] *= 1e-6                     # columns of very different size
    Xt = torch.tensor(X, device="cuda")
    Xh = np.fft.fft(X, axis=0)
    pow2 = (N & (N - 1)) == 0
    for op, d in (("CC", mu), ("CCH", np.conj(mu)), ("CC_INV", 1.0 / mu), ("CCH_INV", 1.0 / np.conj(mu))):
        ref = np.fft.ifft(Xh * d[:, None], axis=0)
        Y = to_np(s.apply(op, Xt))
        e = np.max(np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0))
        print(N, op, f"{e:.2e}")
        if pow2:
            assert 1e-9 < e <= 5e-6, (op, e)
        else:
            assert e <= 2e-12, (op, e)
    s.close()


def test_mixed_woodbury_with_fp32_circulant_refines():
    # the approximate inverse built on the FP32 transform still drives the
    # refinement of the mixed form to its usual residual at N = 4096
    w = dict(family="ellipse", params={"ax": 1.0, "ay": 0.5}, N=4096, k=None)
    s = make_solver(w, precision=1, refine_tol=5e-7, max_refine=12, rhs_chunk=64)
    s.assemble()
    s.skeleton(1e-6, max_rank=512, seed=1, allow_cap=True)
    s.factor()
    s.solve_planewaves(np.linspace(0.0, 6.0, 8))
    st = s.last_solve
    print(st)
    assert st["rel_residual"] <= 5e-7
    s.close()
