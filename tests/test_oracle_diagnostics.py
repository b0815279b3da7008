"""Trend checks of the spectral statements of Sec. IV-V, at 10 elements per
wavelength (CPU).

Circle (closed-form eigenvalues of Eq. 5, the spectrum the paper plots first):
the largest |mu_C / mu_G| sits just below the surface resonance m = k a and
moves towards it as k grows; at high frequency (|m| > 2 k a) the values sit
above the halved identity 1/2 by an offset that does not shrink with h.

2 x 1 ellipse of the paper's experiments (oracle):
* G^-1 C: the largest singular values belong to singular vectors of spatial
  frequency up to about k a; the high-frequency ones again sit just above 1/2
  with an offset that does not shrink as N doubles.
* G^-1 (C - C_c): the high-frequency part has decayed to ~0.
* The rank at eps = 0.015 grows with k, more slowly than k itself.
"""

import numpy as np
import pytest

import closed_form_circle as cf
from oracle import diagnostics, geometry


def test_circle_spectrum_peak_and_offset():
    peaks, offsets = [], []
    for k, N in ((16.0, 256), (64.0, 1024), (200.0, 4096)):
        a = 1.0
        kt = k + 0.4j * k ** (1.0 / 3.0) * a ** (-2.0 / 3.0)
        mu = cf.galerkin_eigs(a, N, k, kt)
        lam = np.abs(cf.c_eigs(mu) / mu["G"])
        m = np.minimum(np.arange(N), N - np.arange(N))
        peaks.append(m[np.argmax(lam)] / (k * a))
        hi = m > 2 * k * a
        assert np.all(lam[hi] > 0.5)
        offsets.append(np.max(lam[hi] - 0.5))
    assert 0.75 < peaks[0] < peaks[1] < peaks[2] <= 1.0
    assert max(offsets) < 1.1 * min(offsets)          # constant in h at fixed k h

CURVE = geometry.Contour("ellipse", {"ax": 2.0, "ay": 1.0})


@pytest.fixture(scope="module")
def ops():
    return {N: diagnostics.operators(CURVE, N) for N in (64, 128)}


def test_resonance_and_elliptic_offset(ops):
    offsets = []
    for N, (C, Cc, G, k, a, _) in ops.items():
        m, s = diagnostics.spectrum_by_frequency(C, G)
        ka = k * a
        top = np.argsort(-s)[:5]
        assert np.all(m[top] <= 1.2 * ka)                      # strength up to the resonance
        hi = m > 2 * ka
        assert hi.sum() > N // 8
        dev = s[hi] - 0.5
        assert np.all(dev > 0) and np.max(dev) < 0.05           # near, not at, the halved identity
        offsets.append(np.max(dev))
    # a constant discretisation offset: it does not shrink with h
    assert abs(offsets[1] - offsets[0]) < 0.3 * offsets[0]


def test_extracted_part_decays_at_high_frequency(ops):
    for N, (C, Cc, G, k, a, _) in ops.items():
        m, s = diagnostics.spectrum_by_frequency(C - Cc, G)
        hi = m > 2 * k * a
        assert np.max(s[hi]) < 1e-2 * np.max(s)


def test_rank_grows_slower_than_k():
    r64, e64, k64 = diagnostics.rank_and_error(CURVE, 64, 0.015, [0.0, 1.0])
    r128, e128, k128 = diagnostics.rank_and_error(CURVE, 128, 0.015, [0.0, 1.0])
    assert 0 < r64 < r128 < (k128 / k64) * r64
    assert max(e64, e128) < 1e-2       # eps = 0.015 of ||C_c||: a percent-level solve


def test_frequency_response_is_the_eigenvalue_ratio_on_the_circle():
    # pin of diagnostics.frequency_response: on the circle G^-1 C is circulant,
    # so its response to the Fourier vector of frequency m is |mu_C / mu_G|
    # (closed form, no quadrature)
    N, k = 128, 8.0
    C, Cc, G, k, a, _ = diagnostics.operators(geometry.Circle(2.0 * np.pi), N, k)
    mu = cf.galerkin_eigs(1.0, N, k, k + 0.4j * k ** (1.0 / 3.0))
    ref = np.abs(cf.c_eigs(mu) / mu["G"])
    resp = diagnostics.frequency_response(C, G)
    assert np.max(np.abs(resp - ref)) <= 1e-10 * np.max(ref)
    assert np.max(diagnostics.frequency_response(C - Cc, G)) <= 1e-10 * np.max(ref)
