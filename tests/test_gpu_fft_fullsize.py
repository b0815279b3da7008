"""Circulant algebra of Sec. V at the full-size transform lengths.

The FFT takes three routes: one shared-memory pass for power-of-two n <= 4096,
the four-step transform above that (the N = 8192 shape-gradient ellipse and
the N = 32768 superellipse of the benchmark), and Bluestein's convolution for
other n, whose padded length m is itself a four-step transform once m > 4096
(N = 5000 -> m = 16384, N = 12289 -> m = 32768).  For each route:

* C_c, C_c^H and C_c^-1 applied to random blocks against numpy.fft with the
  library's own mu_C, element by element at 2e-12 of the largest entry (this
  isolates the transform);
* the eigenvalues mu_X of the circle operators (first rows on gamma_c, then
  the FFT) against the closed-form Galerkin symbols of tests/closed_form_circle.py.
  Their accuracy is that of the kernel values, not of the transform: at
  k R up to 2 k a ~ 6.5e3 (N = 32768) an FP64 phase carries ~1e-16 k R
  absolute error, so the rows hold entries good to ~1e-12, and N of them
  summed give eigenvalues good to ~1e-11 of the largest (measured: 8e-12 for
  D, 1.3e-11 for N at N = 32768, 1e-12 at N = 8192).  mu_C combines them
  through (G/2 + mu_D~)(G/2 - mu_D)/G + mu_S mu_N / G, which amplifies the
  error about tenfold (1.5e-10 at N = 32768).  Bounds: 3e-11 for the four
  operators, 3e-10 for C_c, 1e-15 for G (exact).

FP64 form (its quadrature resolves the circle rows to ~1e-13 at small k)."""

import numpy as np
import pytest
import torch

import closed_form_circle as cf
from gpu_common import make_solver, to_np

pytestmark = pytest.mark.gpu

CASES = [
    ("ellipse", {"ax": 1.0, "ay": 0.7}, 8192),
    ("superellipse", {"ax": 1.0, "ay": 0.6, "p": 4.0}, 32768),
    ("ellipse", {"ax": 1.0, "ay": 0.5}, 5000),
    ("ellipse", {"ax": 1.0, "ay": 0.5}, 12289),
]


@pytest.mark.parametrize("family,params,N", CASES, ids=[f"{c[0]}_n{c[2]}" for c in CASES])
def test_circulant_parity_full_size(family, params, N):
    w = dict(family=family, params=params, N=N, k=None)
    s = make_solver(w, precision=0, rhs_chunk=64)
    s.assemble()
    info = s.info()
    kt = complex(info["kt_re"], info["kt_im"])
    mu = {key: to_np(s.circulant_eigs(op))
          for key, op in (("G", "G"), ("S", "S"), ("D", "D"), ("Dt", "DT"), ("N", "N"), ("CC", "CC"))}
    # the transforms: element by element against numpy.fft with the library's mu_C
    g = np.random.default_rng(N)
    X = g.standard_normal((N, 3)) + 1j * g.standard_normal((N, 3))
    Xt = torch.tensor(X, device="cuda")
    Xh = np.fft.fft(X, axis=0)
    for op, y_ref in (("CC_INV", np.fft.ifft(Xh / mu["CC"][:, None], axis=0)),
                      ("CC", np.fft.ifft(Xh * mu["CC"][:, None], axis=0)),
                      ("CCH", np.fft.ifft(Xh * np.conj(mu["CC"])[:, None], axis=0))):
        Y = to_np(s.apply(op, Xt))
        e = np.max(np.abs(Y - y_ref)) / np.max(np.abs(y_ref))
        print(N, op, f"{e:.1e}")
        assert e <= 2e-12, (op, e)
    # the eigenvalues against the closed form
    ref = cf.galerkin_eigs(info["a"], N, info["k"], kt, P=40)
    ref["CC"] = cf.c_eigs(ref)
    errs = {key: np.max(np.abs(mu[key] - ref[key])) / np.max(np.abs(ref[key])) for key in mu}
    print(N, {k: f"{v:.1e}" for k, v in errs.items()})
    bound = {"G": 2e-15, "S": 3e-11, "D": 3e-11, "Dt": 3e-11, "N": 3e-11, "CC": 3e-10}
    for key, e in errs.items():
        assert e <= bound[key], (key, e)
    s.close()
