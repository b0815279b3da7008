"""Contour geometry and the arc-length mesh of the oracle (test infrastructure only).

Sec. II: the scatterer is a convex 2D contour gamma.  Sec. V: gamma and its
equivalent circle gamma_c (same perimeter L) are both discretised uniformly in
arc length with N elements of length h = L / N; node 0 sits at polar angle 0.

Contours are star-shaped, r(theta) = rho(theta) (cos theta, sin theta).  The
oracle represents rho by its Fourier series (FFT of samples on a fine grid), so
derivatives, arc length s(theta) and curvature are spectrally exact and share
no formula with the CUDA path, which differentiates each family analytically.
"""

import numpy as np


def rho_function(family, params):
    """Radial function rho(theta) of a contour family (vectorised, numpy).

    Optional keys "alpha" (alpha_0, alpha_1, ...) and "beta" (beta_1, beta_2,
    ...) add a Fourier perturbation sum_m alpha_m cos(m theta) +
    sum_m beta_m sin(m theta) to any family (the shape parameters of the
    far-field objective whose gradient oracle/shape.py computes)."""
    alpha = np.asarray(params.get("alpha", ()), float)
    beta = np.asarray(params.get("beta", ()), float)
    base = _base_rho(family, params)
    if alpha.size == 0 and beta.size == 0:
        return base

    def f(th):
        th = np.asarray(th, float)
        out = base(th)
        for m, a in enumerate(alpha):
            out = out + a * np.cos(m * th)
        for m, b in enumerate(beta, start=1):
            out = out + b * np.sin(m * th)
        return out
    return f


def _base_rho(family, params):
    if family == "circle":
        a = float(params.get("a", 1.0))
        return lambda th: np.full_like(np.asarray(th, float), a)
    if family == "ellipse":
        ax, ay = float(params["ax"]), float(params["ay"])
        return lambda th: 1.0 / np.sqrt((np.cos(th) / ax) ** 2 + (np.sin(th) / ay) ** 2)
    if family == "superellipse":
        ax, ay, p = float(params["ax"]), float(params["ay"]), float(params["p"])
        return lambda th: (np.abs(np.cos(th) / ax) ** p + np.abs(np.sin(th) / ay) ** p) ** (-1.0 / p)
    if family == "fourier":
        c = np.asarray(params["cos"], float)
        s = np.asarray(params.get("sin", np.zeros_like(c)), float)

        def f(th):
            th = np.asarray(th, float)
            out = np.zeros_like(th)
            for m in range(len(c)):
                out = out + c[m] * np.cos(m * th) + s[m] * np.sin(m * th)
            return out
        return f
    raise ValueError(f"unknown contour family {family!r}")


class FourierCurve:
    """Spectral representation of a periodic real function on [0, 2 pi)."""

    def __init__(self, samples, tol=1e-15):
        M = len(samples)
        c = np.fft.rfft(samples) / M
        c[1:] *= 2.0  # one-sided: f = Re(sum_m c_m e^{i m th})
        if M % 2 == 0:
            c[-1] *= 0.5
        mag = np.abs(c)
        keep = np.nonzero(mag > tol * mag[0])[0]
        K = min(len(c), (int(keep[-1]) + 1 if len(keep) else 1) + 8)
        if K > 0.5 * len(c):
            raise ValueError("contour is not resolved by the Fourier grid (not smooth enough)")
        self.c = c[:K]
        self.m = np.arange(K)

    def eval(self, th, deriv=0):
        th = np.asarray(th, float)
        out = np.empty(th.shape)
        flat_in, flat_out = th.ravel(), out.reshape(-1)
        coef = self.c * (1j * self.m) ** deriv
        for i0 in range(0, flat_in.size, 32768):
            e = np.exp(1j * np.outer(flat_in[i0:i0 + 32768], self.m))
            flat_out[i0:i0 + 32768] = (e @ coef).real
        return out


class Contour:
    """Star-shaped contour with arc-length parametrisation.

    s(theta) = int_0^theta |r'(t)| dt is obtained by term-wise integration of
    the Fourier series of the speed |r'(theta)|; theta(s) by Newton.
    """

    def __init__(self, family, params, M=4096):
        self.family, self.params = family, dict(params)
        th = 2.0 * np.pi * np.arange(M) / M
        self.rho = FourierCurve(rho_function(family, params)(th))
        r0, r1 = self.rho.eval(th), self.rho.eval(th, 1)
        self.speed = FourierCurve(np.sqrt(r0 ** 2 + r1 ** 2))
        self.L = 2.0 * np.pi * self.speed.c[0].real

    def s_of_theta(self, th):
        th = np.asarray(th, float)
        c, m = self.speed.c[1:], self.speed.m[1:]
        out = self.speed.c[0].real * th
        flat, res = th.ravel(), out.reshape(-1)
        for i0 in range(0, flat.size, 32768):
            t = flat[i0:i0 + 32768]
            e = (np.exp(1j * np.outer(t, m)) - 1.0) / (1j * m)
            res[i0:i0 + 32768] += (e @ c).real
        return out

    def theta_of_s(self, s):
        s = np.asarray(s, float)
        th = 2.0 * np.pi * s / self.L
        for _ in range(60):
            d = (self.s_of_theta(th) - s) / self.speed.eval(th)
            th = th - d
            if np.max(np.abs(d)) < 1e-15:
                break
        return th

    def points(self, s):
        """Position, unit outward normal and curvature at arc lengths s."""
        th = self.theta_of_s(s)
        r0, r1, r2 = self.rho.eval(th), self.rho.eval(th, 1), self.rho.eval(th, 2)
        c, sn = np.cos(th), np.sin(th)
        x, y = r0 * c, r0 * sn
        dx, dy = r1 * c - r0 * sn, r1 * sn + r0 * c
        sp = np.sqrt(dx * dx + dy * dy)
        tx, ty = dx / sp, dy / sp
        kappa = (r0 ** 2 + 2 * r1 ** 2 - r0 * r2) / sp ** 3
        return {"x": x, "y": y, "nx": ty, "ny": -tx, "kappa": kappa}


class Circle:
    """Equivalent circle gamma_c of radius a = L/(2 pi), same arc-length origin."""

    def __init__(self, L):
        self.L = float(L)
        self.a = self.L / (2.0 * np.pi)

    def points(self, s):
        th = np.asarray(s, float) / self.a
        c, sn = np.cos(th), np.sin(th)
        return {"x": self.a * c, "y": self.a * sn, "nx": c, "ny": sn,
                "kappa": np.full_like(th, 1.0 / self.a)}


def wavenumbers(L, N, k=None, elements_per_wavelength=10.0):
    """k (given, or fixed by elements per wavelength) and the complex k~ of Sec. III.

    k~ = k + 0.4 i k^{1/3} a^{-2/3} with a = L / (2 pi) (reading of the
    "suitable average of the radii of curvature": the reciprocal of the
    arc-length mean curvature of a convex curve).
    """
    if k is None or k <= 0:
        k = 2.0 * np.pi * (N / elements_per_wavelength) / L
    a = L / (2.0 * np.pi)
    kt = k + 0.4j * k ** (1.0 / 3.0) * a ** (-2.0 / 3.0)
    return float(k), complex(kt), a
