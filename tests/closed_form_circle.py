"""Closed forms on the circle, used to pin the oracle and the CUDA path.

On a circle of radius a every operator of Sec. II is diagonal in the Fourier
basis e^{i n theta}, with symbols (x = kappa a, Graf's addition theorem)

    S^kappa:        (i pi a / 2) J_n(x) H_n(x)
    1/2 - D^kappa:  -(i pi x / 2) J_n(x) H_n'(x)
    N^k:            -(i pi k^2 a / 2) J_n'(ka) H_n'(ka)

and the hat-function Galerkin matrices on the uniform mesh of N elements are
circulant with eigenvalues (m = 0..N-1, h = 2 pi a / N)

    mu_X(m) = h sum_{p in Z} sinc^4(pi (m + pN) / N) sigma_X(m + pN).

This module shares no code with the oracle or the CUDA library.  Products of
Bessel functions at large order are computed from stable ratio recurrences
(backward for J_n / J_{n-1}, forward for Y_{n-1} / Y_n) and the Wronskian, so
nothing over- or underflows; the algebraic tails of the S and N sums beyond
|p| > P are summed with Hurwitz zeta functions.

The discrete right-hand sides follow from the Jacobi-Anger expansion, the Mie
series give the exact surface current and far field of the continuous problem.
"""

import numpy as np
import scipy.special as sp


def _products(z, nmax, n_direct=None):
    """J_n H_n, J_n H_n', J_n' H_n', for n = 0..nmax at argument z (complex ok).

    Direct scipy evaluation for n <= n_direct (about |z| + 40, where Y_n is
    still far from overflow); for larger n, from ratios: rho_n = J_n / J_{n-1}
    by backward recurrence, tau_n = Y_{n-1} / Y_n by forward recurrence, the
    Wronskian J_n Y_{n-1} - J_{n-1} Y_n = 2 / (pi z) for the products J Y, and
    J_{n-1}^2 continued from the last direct value by the product of the
    rho's (in logarithms, so it underflows gracefully to 0 far above |z|).
    """
    z = complex(z)
    if n_direct is None:
        n_direct = int(min(nmax, max(40, abs(z) + 40)))
    n = np.arange(n_direct + 1)
    J = sp.jv(n, z)
    H = sp.hankel1(n, z)
    Jp = sp.jvp(n, z)
    Hp = sp.h1vp(n, z)
    JH, JHp, JpHp = [np.empty(nmax + 1, complex) for _ in range(3)]
    JH[:n_direct + 1], JHp[:n_direct + 1], JpHp[:n_direct + 1] = J * H, J * Hp, Jp * Hp
    if nmax <= n_direct:
        return JH, JHp, JpHp
    # rho_n = J_n / J_{n-1} by backward recurrence from far above nmax
    top = nmax + 200
    rho = np.empty(top + 2, complex)
    rho[top + 1] = z / (2.0 * (top + 1))
    for m in range(top, 0, -1):
        rho[m] = 1.0 / (2.0 * m / z - rho[m + 1])
    # tau_n = Y_{n-1} / Y_n by forward recurrence from scipy's Y_0 / Y_1
    tau = np.empty(nmax + 1, complex)
    tau[1] = sp.yv(0, z) / sp.yv(1, z)
    for m in range(1, nmax):
        tau[m + 1] = 1.0 / (2.0 * m / z - tau[m])
    m = np.arange(n_direct + 1, nmax + 1)
    r, t = rho[m], tau[m]
    base = 2.0 / (np.pi * z * (r * t - 1.0))        # J_{n-1} Y_n
    Jp_over = 1.0 - m * r / z                        # J_n' / J_{n-1}
    Yp_over = t - m / z                              # Y_n' / Y_n
    # J_{n-1}^2 for n = n_direct + 1 .. nmax
    logJ = np.log(complex(J[n_direct])) + np.concatenate([[0.0], np.cumsum(np.log(r[:-1]))])
    J2 = np.exp(2.0 * logJ)
    JH[m] = r * r * J2 + 1j * (r * base)
    JHp[m] = r * J2 * Jp_over + 1j * (r * base * Yp_over)
    JpHp[m] = J2 * Jp_over * Jp_over + 1j * (base * Jp_over * Yp_over)
    return JH, JHp, JpHp


def symbols(a, k, kt, nmax):
    """sigma_X(n), n = 0..nmax, for X in (S~, D, D~, N); all even in n."""
    JHt, JHpt, _ = _products(kt * a, nmax)
    _, JHp, JpHp = _products(k * a, nmax)
    S = 0.5j * np.pi * a * JHt
    D = 0.5 + 0.5j * np.pi * (k * a) * JHp
    Dt = 0.5 + 0.5j * np.pi * (kt * a) * JHpt
    Nk = -0.5j * np.pi * k * k * a * JpHp
    return {"S": S, "D": D, "Dt": Dt, "N": Nk}


def galerkin_eigs(a, N, k, kt, P=200):
    """mu_X(m), m = 0..N-1, for X in (G, S~, D, D~, N) on the circle of radius a."""
    h = 2.0 * np.pi * a / N
    m = np.arange(N)
    p = np.arange(-P, P + 1)
    n = m[:, None] + p[None, :] * N                 # (N, 2P+1)
    nabs = np.abs(n)
    sig = symbols(a, k, kt, int(nabs.max()))
    s4 = np.sinc(n / N) ** 4                         # numpy sinc(x) = sin(pi x)/(pi x)
    out = {"G": h * (2.0 + np.cos(2.0 * np.pi * m / N)) / 3.0}
    # algebraic tails beyond |p| > P: sinc^4 = sin^4(pi m / N) (N / (pi n))^4
    c4 = np.sin(np.pi * m / N) ** 4 * (N / np.pi) ** 4
    z3 = (sp.zeta(3, P + 1 + m / N) + sp.zeta(3, P + 1 - m / N)) / N ** 3
    z5 = (sp.zeta(5, P + 1 + m / N) + sp.zeta(5, P + 1 - m / N)) / N ** 5
    for key in ("S", "D", "Dt", "N"):
        mu = h * np.sum(s4 * sig[key][nabs], axis=1)
        if key == "S":      # sigma_S ~ a / (2|n|) (1 + kt^2 a^2 / (2 n^2) + ...)
            mu += h * c4 * (a / 2.0) * z5
        if key == "N":      # sigma_N ~ |n| / (2a) - k^2 a / (4 |n|) + ...
            mu += h * c4 * ((1.0 / (2.0 * a)) * z3 - (k * k * a / 4.0) * z5)
        out[key] = mu
    return out


def c_eigs(mu, k=None):
    """Eigenvalues of C (Eq. 6) from the operator eigenvalues."""
    G = mu["G"]
    return (G / 2 + mu["Dt"]) * (G / 2 - mu["D"]) / G + mu["S"] * mu["N"] / G


def planewave_rhs(a, N, k, phi, nmax=None):
    """Closed-form Galerkin projections (e/eta, h) of one plane wave on the circle."""
    h = 2.0 * np.pi * a / N
    if nmax is None:
        nmax = int(abs(k * a) + 60)
    n = np.arange(-nmax, nmax + 1)
    J = sp.jv(n, k * a)
    Jp = sp.jvp(n, k * a)
    s2 = np.sinc(n / N) ** 2
    ch = (1j ** n) * J * np.exp(-1j * n * phi) * h * s2
    ce = -1j * (1j ** n) * Jp * np.exp(-1j * n * phi) * h * s2
    hh = np.zeros(N, complex)
    ee = np.zeros(N, complex)
    np.add.at(hh, n % N, ch)
    np.add.at(ee, n % N, ce)
    # coefficient c at Fourier index m multiplies e^{2 pi i m i / N}
    return np.fft.ifft(ee) * N, np.fft.ifft(hh) * N


def discrete_solution(a, N, k, kt, phi, P=200):
    """Exact discrete solution of Eq. (5) on the circle (node coefficients)."""
    mu = galerkin_eigs(a, N, k, kt, P)
    e, hv = planewave_rhs(a, N, k, phi)
    eh, hh = np.fft.fft(e), np.fft.fft(hv)
    bh = -1j * k * mu["S"] * eh / mu["G"] - (mu["G"] / 2 + mu["Dt"]) * hh / mu["G"]
    return np.fft.ifft(bh / c_eigs(mu))


def mie_current(a, k, phi, theta, nmax=None):
    """Exact surface current j = -H_z^tot of the continuous TE PEC circle problem."""
    if nmax is None:
        nmax = int(k * a + 60)
    n = np.arange(-nmax, nmax + 1)
    coef = (1j ** n) * (2j / (np.pi * k * a)) / sp.h1vp(n, k * a)
    return -np.exp(1j * np.outer(np.asarray(theta) - phi, n)) @ coef


def mie_farfield(a, k, phi, phi_obs, nmax=None):
    """Exact far-field pattern F(phi_o), H^s ~ F e^{ik rho} / sqrt(rho)."""
    if nmax is None:
        nmax = int(k * a + 60)
    n = np.arange(-nmax, nmax + 1)
    coef = sp.jvp(n, k * a) / sp.h1vp(n, k * a)
    return -np.sqrt(2.0 / (np.pi * k)) * np.exp(-0.25j * np.pi) * (
        np.exp(1j * np.outer(np.asarray(phi_obs) - phi, n)) @ coef)


def discrete_farfield(a, N, k, j, phi_obs, nmax=None):
    """Far field F(phi_o) of hat coefficients j on the circle of radius a, in
    closed form: with psi = theta - phi_o, (x^.n) e^{-i k x^.r} = cos psi
    e^{-i ka cos psi} = i sum_n (-i)^n J_n'(ka) e^{i n psi}, and a hat of
    width 2h centred at theta_i integrates e^{i n theta} to
    h sinc^2(pi n / N) e^{i n theta_i}."""
    h = 2.0 * np.pi * a / N
    if nmax is None:
        nmax = int(abs(k * a) + 60)
    n = np.arange(-nmax, nmax + 1)
    jhat = np.fft.ifft(np.asarray(j)) * N                 # sum_i j_i e^{2 pi i n i / N} at n mod N
    coef = 1j * (-1j) ** n * sp.jvp(n, k * a) * h * np.sinc(n / N) ** 2 * jhat[n % N]
    integral = np.exp(-1j * np.outer(np.atleast_1d(phi_obs), n)) @ coef
    return 1j * k * np.exp(0.25j * np.pi) / np.sqrt(8.0 * np.pi * k) * integral
