"""Shape gradient of the far-field objective (test infrastructure only).

The contour is a base family plus a Fourier perturbation of its radial
function, rho = rho_base + sum_{m<M} alpha_m cos(m theta) + sum_{m=1..M}
beta_m sin(m theta), with parameter vector p = (alpha_0..alpha_{M-1},
beta_1..beta_M).  For fixed N and k the discrete problem of Sec. II-V (mesh
uniform in arc length, k~ from a = L / 2 pi, preconditioned system of
Eq. 5) gives j(p) = C(p)^-1 b(p) for each incidence angle and the far field
F(p) = E(p) j(p) at the observation angles; the objective is
J(p) = sum over incidences and observation angles of |F|^2.

gradient_fd is the plain definition: central differences of J.
gradient_adjoint takes the adjoint route.  With lam_b = C^-H E^H F_b,

    dJ/dp = 2 Re sum_b [ F_b^H (dE j_b) + lam_b^H (db_b - dC j_b) ],

where dE, db, dC are central differences of the far-field map, the
right-hand side and the operator at fixed j (one adjoint solve instead of a
solve per parameter).  gradient_bilinear is the same gradient with dC
expanded by the product rule into bilinear forms of the individual operators
(the reference for a one-pass derivative kernel).  All use dense LU;
nothing here is shared with the CUDA path.
"""

import numpy as np

from . import assembly, geometry, solver


def shape_params(base_params, p, M):
    """Contour parameters of the base family with the perturbation p added."""
    p = np.asarray(p, float)
    d = dict(base_params)
    d["alpha"] = p[:M].tolist()
    d["beta"] = p[M:2 * M].tolist()
    return d


def system(family, base_params, p, M, N, k, inc, obs):
    """(C, b, E) of the perturbed contour: Eq. (5) operator and right-hand
    sides for the incidence angles, far-field map (n_obs x N)."""
    cur = geometry.Contour(family, shape_params(base_params, p, M))
    _, kt, _ = geometry.wavenumbers(cur.L, N, k)
    ops = assembly.assemble(cur, N, k, kt)
    C = assembly.preconditioned(ops)
    e, hv = solver.planewave_rhs(cur, N, k, inc)
    b = solver.preconditioned_rhs(ops, k, e, hv)
    E = solver.farfield(cur, N, k, np.eye(N), obs)
    return C, b, E


def operators_at(family, base_params, p, M, N, k, inc, obs):
    """Galerkin operators (S~, D, D~, N, G), the Eq. (5) right-hand side b and
    the far-field map E of the perturbed contour."""
    cur = geometry.Contour(family, shape_params(base_params, p, M))
    _, kt, _ = geometry.wavenumbers(cur.L, N, k)
    ops = assembly.assemble(cur, N, k, kt)
    e, hv = solver.planewave_rhs(cur, N, k, inc)
    b = solver.preconditioned_rhs(ops, k, e, hv)
    E = solver.farfield(cur, N, k, np.eye(N), obs)
    return ops, b, E, cur.L


def objective(family, base_params, p, M, N, k, inc, obs):
    """J(p) and the forward quantities (j, F, C, b, E)."""
    C, b, E = system(family, base_params, p, M, N, k, inc, obs)
    j = np.linalg.solve(C, b)
    F = E @ j
    return float(np.sum(np.abs(F) ** 2)), dict(j=j, F=F, C=C, b=b, E=E)


def _unit(p, i, M):
    d = np.zeros(2 * M)
    d[i] = 1.0
    return d


def gradient_fd(family, base_params, p, M, N, k, inc, obs, idx, delta=1e-4):
    """dJ/dp_i for i in idx by central differences of J."""
    p = np.asarray(p, float)
    out = []
    for i in idx:
        u = _unit(p, i, M)
        jp, _ = objective(family, base_params, p + delta * u, M, N, k, inc, obs)
        jm, _ = objective(family, base_params, p - delta * u, M, N, k, inc, obs)
        out.append((jp - jm) / (2.0 * delta))
    return np.array(out)


def gradient_adjoint(family, base_params, p, M, N, k, inc, obs, idx, delta=1e-4):
    """dJ/dp_i for i in idx by the adjoint formula (operators differenced at fixed j)."""
    p = np.asarray(p, float)
    J, f = objective(family, base_params, p, M, N, k, inc, obs)
    j, F, C, E = f["j"], f["F"], f["C"], f["E"]
    lam = np.linalg.solve(C.conj().T, E.conj().T @ F)
    out = []
    for i in idx:
        u = _unit(p, i, M)
        Cp, bp, Ep = system(family, base_params, p + delta * u, M, N, k, inc, obs)
        Cm, bm, Em = system(family, base_params, p - delta * u, M, N, k, inc, obs)
        dE = (Ep - Em) / (2.0 * delta)
        db = (bp - bm) / (2.0 * delta)
        dC = (Cp - Cm) / (2.0 * delta)
        g = np.sum(F.conj() * (dE @ j)) + np.sum(lam.conj() * (db - dC @ j))
        out.append(2.0 * g.real)
    return J, np.array(out)


def gradient_bilinear(family, base_params, p, M, N, k, inc, obs, idx, delta=1e-6):
    """The adjoint gradient with dC expanded by the product rule over Eq. (6),
    the form a one-pass derivative kernel evaluates.  With
    t1 = G^-1 (G/2 - D) j, t2 = G^-1 N j, s1 = G^-H (G/2 + D~)^H lam and
    s2 = G^-H S~^H lam:

        lam^H dC j = lam^H (dG/2 + dD~) t1 + s1^H (dG/2 - dD) j - s1^H dG t1
                     + lam^H dS~ t2 + s2^H dN j - s2^H dG t2.

    Each operator derivative is a central difference of that operator alone.
    Returns (J, grad, terms), terms[i] holding the four operator bilinear
    forms lam^H dD~ t1, s1^H dD j, lam^H dS~ t2, s2^H dN j (summed over the
    incidences) and dh / h of parameter i (dG = (dh / h) G on a mesh uniform
    in arc length)."""
    p = np.asarray(p, float)
    ops, b, E, L0 = operators_at(family, base_params, p, M, N, k, inc, obs)
    G = ops["G"]
    C = assembly.preconditioned(ops)
    j = np.linalg.solve(C, b)
    F = E @ j
    J = float(np.sum(np.abs(F) ** 2))
    lam = np.linalg.solve(C.conj().T, E.conj().T @ F)
    t1 = np.linalg.solve(G, 0.5 * G @ j - ops["D"] @ j)
    t2 = np.linalg.solve(G, ops["N"] @ j)
    s1 = np.linalg.solve(G.T, (0.5 * G + ops["Dt"]).conj().T @ lam)
    s2 = np.linalg.solve(G.T, ops["S"].conj().T @ lam)

    def form(u, X, w):
        return np.sum(u.conj() * (X @ w))

    grads, terms = [], []
    for i in idx:
        u = _unit(p, i, M)
        op_p, b_p, E_p, L_p = operators_at(family, base_params, p + delta * u, M, N, k, inc, obs)
        op_m, b_m, E_m, L_m = operators_at(family, base_params, p - delta * u, M, N, k, inc, obs)
        d = {key: (op_p[key] - op_m[key]) / (2.0 * delta) for key in ("S", "D", "Dt", "N", "G")}
        db = (b_p - b_m) / (2.0 * delta)
        dE = (E_p - E_m) / (2.0 * delta)
        dGt = form(lam, 0.5 * d["G"], t1) - form(s1, d["G"], t1) + form(s1, 0.5 * d["G"], j) \
            - form(s2, d["G"], t2)
        fDt, fD = form(lam, d["Dt"], t1), form(s1, d["D"], j)
        fS, fN = form(lam, d["S"], t2), form(s2, d["N"], j)
        dCj = dGt + fDt - fD + fS + fN
        g = np.sum(F.conj() * (dE @ j)) + np.sum(lam.conj() * db) - dCj
        grads.append(2.0 * g.real)
        terms.append(dict(Dt=fDt, D=fD, S=fS, N=fN, dh_over_h=(L_p - L_m) / (2.0 * delta * L0)))
    return J, np.array(grads), terms
