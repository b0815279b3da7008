"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle runs.

This module holds only input descriptions (contour families and parameters,
mesh sizes, incidence angles, seeds).  It contains none of the solver's
arithmetic: each side (CUDA library, CPU oracle) derives k, k~, the mesh and
everything else from these descriptions with its own code.

The paper (arXiv 2203.13283, Sec. VI) tests an ellipse and reports no data set;
all workloads here are synthetic contours with the shapes of that section and
of the solver's intended use (many plane-wave incidences per contour).
"""

import math

import numpy as np

# elements per wavelength used when k is not given: k = 2 pi (N / 10) / L
ELEMENTS_PER_WAVELENGTH = 10.0


def uniform_angles(B):
    """B plane-wave propagation angles 2 pi j / B, j = 0..B-1."""
    return 2.0 * math.pi * np.arange(B) / B


def degree_angles(B):
    """B angles at 1-degree steps starting at 0."""
    return np.deg2rad(np.arange(B, dtype=float))


WORKLOADS = {
    # unit circle, k = 16, N = 256, one plane wave at 0 degrees
    "circle_n256": dict(family="circle", params={"a": 1.0}, N=256, k=16.0,
                        angles=np.array([0.0]), tol=1e-10),
    # ellipse 1.0 x 0.5, 10 elements per wavelength, 360 angles at 1-degree steps
    "ellipse_n4096": dict(family="ellipse", params={"ax": 1.0, "ay": 0.5}, N=4096, k=None,
                          angles=degree_angles(360), tol=1e-10),
    # superellipse |x|^4 + |y/0.6|^4 = 1, 10 elements per wavelength, 1024 angles
    "superellipse_n32768": dict(family="superellipse", params={"ax": 1.0, "ay": 0.6, "p": 4.0},
                                N=32768, k=None, angles=uniform_angles(1024), tol=1e-7),
    # ellipse 1.0 x 0.7 (shape-derivative workload), 16 angles 22.5 degrees apart
    "ellipse_n8192": dict(family="ellipse", params={"ax": 1.0, "ay": 0.7}, N=8192, k=None,
                          angles=uniform_angles(16), tol=1e-10,
                          shape_modes=16, observation_angles=np.deg2rad(np.arange(0.0, 360.0, 4.0))),
}

# small cases of the same families, sized so the CPU oracle runs in seconds
SMALL = {
    "circle_n64": dict(family="circle", params={"a": 1.0}, N=64, k=8.0,
                       angles=np.array([0.0, 1.0]), tol=1e-10),
    "circle_n256": WORKLOADS["circle_n256"],
    "ellipse_n256": dict(family="ellipse", params={"ax": 1.0, "ay": 0.5}, N=256, k=None,
                         angles=degree_angles(360)[::45], tol=1e-10),
    "superellipse_n320": dict(family="superellipse", params={"ax": 1.0, "ay": 0.6, "p": 4.0},
                              N=320, k=None, angles=uniform_angles(8), tol=1e-10),
    "star_n200": None,  # filled below from the star generator
}


def star_contours(count=64, seed=2203_13283, modes=range(2, 9), n_range=(512, 16384)):
    """Random convex star contours r(theta) = 1 + sum_m a_m cos(m theta + phi_m).

    a_m ~ U(0, 0.02 / m^2), phi_m ~ U(0, 2 pi), N ~ U{n_range}; drawn in that
    order per contour from numpy's default_rng(seed).  Returned as Fourier
    coefficients (cos, sin) of r(theta), so a_m cos(m t + phi) =
    a_m cos(phi) cos(m t) - a_m sin(phi) sin(m t).
    """
    rng = np.random.default_rng(seed)
    out = []
    modes = list(modes)
    mmax = max(modes)
    for _ in range(count):
        a = np.array([rng.uniform(0.0, 0.02 / m ** 2) for m in modes])
        ph = np.array([rng.uniform(0.0, 2.0 * math.pi) for _ in modes])
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        c = np.zeros(mmax + 1)
        s = np.zeros(mmax + 1)
        c[0] = 1.0
        for am, pm, m in zip(a, ph, modes):
            c[m] += am * math.cos(pm)
            s[m] -= am * math.sin(pm)
        out.append(dict(family="fourier", params={"cos": c.tolist(), "sin": s.tolist()}, N=N,
                        k=None, angles=uniform_angles(64), tol=1e-7))
    return out


_star = star_contours(count=1)[0]
SMALL["star_n200"] = dict(_star, N=200, angles=uniform_angles(4), tol=1e-10)
SMALL["ellipse_n200"] = dict(SMALL["ellipse_n256"], N=200)
