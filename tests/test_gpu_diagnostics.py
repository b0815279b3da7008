"""GPU diagnostics of Sec. IV-V (paper_2203_13283_gb300/diagnostics.py)
against the oracle and the closed forms.

* Circle: the spectrum of Eq. (5), |mu_C / mu_G| from the library's circulant
  eigenvalues, element by element against the closed-form Galerkin symbols,
  and the trends the paper shows for it (peak just below the surface
  resonance m = k a, moving towards it as k grows; a high-frequency offset
  above the halved identity that does not shrink with h).
* 2 x 1 ellipse (the paper's test contour): the response of G^-1 C and of
  G^-1 (C - C_c) to every Fourier vector against the oracle's dense matrices,
  and the skeleton rank at eps = 0.015 with the error of the compressed
  solve against the oracle's SVD-truncated skeleton."""

import numpy as np
import pytest

import closed_form_circle as cf
from gpu_common import built
from oracle import diagnostics as odiag
from oracle import geometry

pytestmark = pytest.mark.gpu

ELLIPSE = ("ellipse", {"ax": 2.0, "ay": 1.0})


def test_circle_spectrum_of_eq5_vs_closed_form():
    built()
    from paper_2203_13283_gb300 import diagnostics
    peaks, offsets = [], []
    for k, N in ((16.0, 256), (64.0, 1024), (200.0, 4096)):
        lam = diagnostics.circle_spectrum(N, k)
        kt = k + 0.4j * k ** (1.0 / 3.0)
        mu = cf.galerkin_eigs(1.0, N, k, kt)
        ref = np.abs(cf.c_eigs(mu) / mu["G"])
        assert np.max(np.abs(lam - ref)) <= 1e-10 * np.max(ref), (k, N)
        m = np.minimum(np.arange(N), N - np.arange(N))
        peaks.append(m[np.argmax(lam)] / k)
        hi = m > 2 * k
        assert np.all(lam[hi] > 0.5)
        offsets.append(np.max(lam[hi] - 0.5))
    assert 0.75 < peaks[0] < peaks[1] < peaks[2] <= 1.0
    assert max(offsets) < 1.1 * min(offsets)


@pytest.mark.parametrize("N", [64, 128])
def test_frequency_response_vs_oracle(N):
    built()
    from paper_2203_13283_gb300 import Solver, diagnostics
    curve = geometry.Contour(*ELLIPSE)
    C, Cc, G, k, a, _ = odiag.operators(curve, N)
    s = Solver(precision=0)
    s.contour(ELLIPSE[0], **ELLIPSE[1]).mesh(N).assemble()
    rC = diagnostics.frequency_response(s, "C")
    rR = diagnostics.frequency_response(s, "C-Cc")
    s.close()
    oC = odiag.frequency_response(C, G)
    oR = odiag.frequency_response(C - Cc, G)
    assert np.max(np.abs(rC - oC)) <= 1e-10 * np.max(oC)
    assert np.max(np.abs(rR - oR)) <= 1e-10 * np.max(oC)
    m = np.minimum(np.arange(N), N - np.arange(N))
    ka = k * a
    # the remainder dies off at high frequency (N = 64: 4.5e-3 of its peak
    # just above 2 k a, 2e-3 beyond 3 k a), and monotonically so
    assert np.max(rR[m > 2 * ka]) < 3e-2 * np.max(rR)
    assert np.max(rR[m > 3 * ka]) < 5e-3 * np.max(rR)
    tail = [np.max(rR[m == mm]) for mm in range(int(np.ceil(2 * ka)) + 1, N // 2 + 1)]
    assert all(b <= a * (1 + 1e-9) for a, b in zip(tail, tail[1:]))
    assert m[np.argmax(rC)] <= 1.2 * ka                        # C is strongest up to the resonance


def test_rank_sweep_vs_oracle():
    built()
    from paper_2203_13283_gb300 import diagnostics
    curve = geometry.Contour(*ELLIPSE)
    rows = diagnostics.rank_sweep(*ELLIPSE, [64, 128, 256], eps=0.015)
    ranks = []
    for (N, k, r, err) in rows:
        r_or, e_or, k_or = odiag.rank_and_error(curve, N, 0.015, [0.0, 1.0])
        assert abs(k - k_or) <= 1e-12 * k
        # the range finder stops when its projected samples, which measure the
        # Frobenius norm of the remainder, drop below eps ||C_c||; the SVD rule
        # counts singular values above it, so the GPU keeps at least that rank
        print(N, k, "rank", r, "oracle", r_or, "error", err, "oracle", e_or)
        assert r_or <= r <= 3 * r_or, (N, r, r_or)
        assert err <= 2.0 * e_or + 1e-4, (N, err, e_or)
        ranks.append(r)
    assert ranks[0] < ranks[1] < ranks[2]
