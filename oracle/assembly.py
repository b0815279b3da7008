"""Dense Galerkin assembly of the oracle (test infrastructure only).

Sec. II, Eq. (4): with piecewise-linear hat functions lambda_i on a mesh
uniform in arc length (Sec. V),

    [G]_ij   = <lambda_i, lambda_j>
    [D^k]_ij = <lambda_i, D^k lambda_j>,  D^k kernel  d g_k / d n'
    [N^k]_ij = <lambda_i, N^k lambda_j>,  N^k = -d/dn int d/dn' g_k
    [S^k~]_ij = <lambda_i, S^k~ lambda_j>, kernel g_k~ (reading of Eq. 5)

N^k is integrated in Maue's form (integration by parts on the closed curve):
<lambda_i, N^k lambda_j> = int int [lambda_i' lambda_j' - k^2 (n . n')
lambda_i lambda_j] g_k ds' ds.

Element e spans arc lengths [e h, (e+1) h]; on it hat e is 1 - xi and hat
e + 1 is xi.  Every element pair (e, f) contributes a 2x2 block to the node
pairs (e + a, f + b), a, b in {0, 1}, indices mod N.

Quadrature (chosen by periodic element distance d = |e - f| mod N):
  d = 0     split along the diagonal, panels graded toward it;
  d = 1     Duffy map centred on the shared vertex, panels graded radially;
  for d <= 1 the log singularity -(1/2 pi) log|s - s'| of g is subtracted
  and integrated exactly against the hat-function products;
  2..near   tensor Gauss-Legendre with q_near points per element;
  > near    tensor Gauss-Legendre with q_far points per element.
"""

import numpy as np

from . import quadrature as qd
from .kernels import pair_kernels
from .geometry import Circle


class ElementGeometry:
    """Geometry at arbitrary local coordinates xi of each element.

    Exact points (Newton on the arc length) are taken at n_cheb Chebyshev
    nodes per element and evaluated elsewhere by barycentric interpolation;
    the map xi -> geometry is analytic, so this is exact to rounding for the
    smooth contours used here (checked against direct evaluation in tests).
    """

    FIELDS = ("x", "y", "nx", "ny", "kappa")

    def __init__(self, curve, N, n_cheb=32, elements=None):
        """elements: optional subset of element indices to prepare (the only
        ones at() may then be asked for); by default all N."""
        self.curve, self.N = curve, N
        self.h = curve.L / N
        self.exact = isinstance(curve, Circle)
        if self.exact:
            return
        j = np.arange(n_cheb)
        self.xc = 0.5 * (1.0 - np.cos(np.pi * (j + 0.5) / n_cheb))
        self.bw = (-1.0) ** j * np.sin((2 * j + 1) * np.pi / (2 * n_cheb))
        el = np.arange(N) if elements is None else np.unique(np.asarray(elements) % N)
        self.row = np.full(N, -1, np.int64)
        self.row[el] = np.arange(len(el))
        s = (el[:, None] + self.xc[None, :]) * self.h
        pts = curve.points(s)
        self.vals = {f: pts[f] for f in self.FIELDS}

    def _bary(self, xi):
        d = xi[:, None] - self.xc[None, :]
        hit = d == 0.0
        d[hit] = 1.0
        W = self.bw[None, :] / d
        rows = np.nonzero(hit.any(axis=1))[0]
        W[rows] = hit[rows].astype(float)
        return W / W.sum(axis=1, keepdims=True)

    def at(self, e, xi):
        """Points at local coordinate xi (shape (Q,)) of elements e (shape (P,))."""
        e = np.asarray(e) % self.N
        xi = np.asarray(xi, float)
        if self.exact:
            return self.curve.points((e[:, None] + xi[None, :]) * self.h)
        W = self._bary(xi)
        r = self.row[e]
        if np.any(r < 0):
            raise ValueError("element geometry not prepared for these elements")
        return {f: self.vals[f][r] @ W.T for f in self.FIELDS}


def _locals(geo, e, f, rule, k, kt, log_kind=None):
    """2x2 local integrals of (S~, D, D~, N) for element pairs (e, f) with one rule.

    log_kind (None, "self", "e_end", "e_start") marks a singular pair: the
    log singularity -(1/2pi) log|s - s'| of g is then subtracted from the S~
    and N integrands, integrated exactly (quadrature.log_integrals) and the
    bounded remainder integrated with the rule.  D and D~ have bounded kernels
    and use the rule directly.  Returns an array of shape (4, 2, 2, P).
    """
    xi, eta, w = rule
    h = geo.h
    P = geo.at(e, xi)
    Q = geo.at(f, eta)
    phi = (1.0 - xi, xi)
    psi = (1.0 - eta, eta)
    sgn = (-1.0, 1.0)
    gk, dgk, ndot = pair_kernels(P, Q, k)
    gt, dgt, _ = pair_kernels(P, Q, kt)
    if log_kind is not None:
        dloc = {"self": np.abs(xi - eta), "e_end": (1.0 - xi) + eta,
                "e_start": xi + (1.0 - eta)}[log_kind]
        logd = np.log(h * dloc)
        Ilog, I1 = qd.log_integrals(log_kind)
        lh = np.log(h)
    c2 = 0.5 / np.pi
    out = np.zeros((4, 2, 2, len(e)), complex)
    for a in range(2):
        for b in range(2):
            pab = phi[a] * psi[b]
            wab = w * pab
            out[1, a, b] = h * h * (dgk @ wab)
            out[2, a, b] = h * h * (dgt @ wab)
            cN = sgn[a] * sgn[b] - k * k * h * h * ndot * pab
            if log_kind is None:
                out[0, a, b] = h * h * (gt @ wab)
                out[3, a, b] = (gk * cN) @ w
            else:
                polyN = sgn[a] * sgn[b] - k * k * h * h * pab
                out[0, a, b] = (h * h * ((gt + c2 * logd) @ wab)
                                - c2 * h * h * (0.25 * lh + Ilog[a, b]))
                out[3, a, b] = ((gk * cN + c2 * polyN * logd) @ w
                                - c2 * (sgn[a] * sgn[b] * (lh + I1)
                                        - k * k * h * h * (0.25 * lh + Ilog[a, b])))
    return out


def _scatter(X, e, f, loc, N):
    for a in range(2):
        for b in range(2):
            np.add.at(X, ((e + a) % N, (f + b) % N), loc[a, b])


def gram(N, h):
    """Gram matrix <lambda_i, lambda_j>: 2h/3 on the diagonal, h/6 beside it (cyclic)."""
    G = np.zeros((N, N))
    i = np.arange(N)
    G[i, i] = 2.0 * h / 3.0
    G[i, (i + 1) % N] = h / 6.0
    G[i, (i - 1) % N] = h / 6.0
    return G


class Rules:
    def __init__(self, q_far=6, q_near=16, near=4, n_sing=12):
        self.q_far, self.q_near, self.near = q_far, q_near, near
        panels = qd.panels01(n_sing)
        self.self_rule = qd.self_rule(panels, n_sing)
        self.touch_next = qd.touching_rule(panels, n_sing, "e_end")
        self.touch_prev = qd.touching_rule(panels, n_sing, "e_start")
        self.near_rule = qd.tensor_rule(q_near)


def assemble(curve, N, k, kt, rules=None, chunk=96):
    """Dense (G, S~, D, D~, N) on a curve discretised with N elements.

    curve: oracle.geometry.Contour or Circle.  k real, kt complex.
    Returns a dict of complex (N, N) arrays (G real).
    """
    rules = rules or Rules()
    if N < 2 * rules.near + 2:
        raise ValueError("N too small for the near-field band")
    geo = ElementGeometry(curve, N)
    h = geo.h
    ops = np.zeros((4, N, N), complex)

    # far pairs: tensor Gauss-Legendre, evaluated as point-by-point matrices
    xg, wg = qd.gauss_legendre01(rules.q_far)
    allp = geo.at(np.arange(N), xg)
    flat = {f: v.reshape(-1) for f, v in allp.items()}
    phiw = np.stack([wg * (1.0 - xg), wg * xg])          # (2, q)
    sgnw = np.stack([-wg, wg])                           # derivative weights * h
    q = rules.q_far
    dist = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :])
    dist = np.minimum(dist, N - dist)
    farmask = dist > rules.near
    for r0 in range(0, N, chunk):
        r1 = min(N, r0 + chunk)
        P = {f: v[r0 * q:r1 * q, None] for f, v in flat.items()}
        Q = {f: v[None, :] for f, v in flat.items()}
        with np.errstate(divide="ignore", invalid="ignore"):
            gk, dgk, ndot = pair_kernels(P, Q, k)
            gt, dgt, _ = pair_kernels(P, Q, kt)
        shp = (r1 - r0, q, N, q)
        gk, dgk, ndot, gt, dgt = (t.reshape(shp) for t in (gk, dgk, ndot, gt, dgt))
        m = farmask[r0:r1]
        for a in range(2):
            for b in range(2):
                with np.errstate(invalid="ignore"):
                    Ls = h * h * np.einsum("p,epfr,r->ef", phiw[a], gt, phiw[b])
                Ld = h * h * np.einsum("p,epfr,r->ef", phiw[a], dgk, phiw[b])
                Ldt = h * h * np.einsum("p,epfr,r->ef", phiw[a], dgt, phiw[b])
                Ln = (np.einsum("p,epfr,r->ef", sgnw[a], gk, sgnw[b])
                      - k * k * h * h * np.einsum("p,epfr,r->ef", phiw[a], gk * ndot, phiw[b]))
                rows = (np.arange(r0, r1) + a) % N
                for o, Lx in enumerate((Ls, Ld, Ldt, Ln)):
                    Lx = np.where(m, Lx, 0.0)
                    ops[o, rows, :] += np.roll(Lx, b, axis=1)

    e = np.arange(N)
    # near pairs
    for d in range(2, rules.near + 1):
        for sgn in (1, -1):
            f = (e + sgn * d) % N
            _scatter_all(ops, e, f, _locals(geo, e, f, rules.near_rule, k, kt), N)
    # touching pairs: f = e + 1 (shared vertex at the end of e) and f = e - 1
    _scatter_all(ops, e, (e + 1) % N,
                 _locals(geo, e, (e + 1) % N, rules.touch_next, k, kt, "e_end"), N)
    _scatter_all(ops, e, (e - 1) % N,
                 _locals(geo, e, (e - 1) % N, rules.touch_prev, k, kt, "e_start"), N)
    # coincident pairs
    _scatter_all(ops, e, e, _locals(geo, e, e, rules.self_rule, k, kt, "self"), N)

    return {"G": gram(N, h), "S": ops[0], "D": ops[1], "Dt": ops[2], "N": ops[3], "h": h}


def _scatter_all(ops, e, f, loc, N):
    for o in range(4):
        _scatter(ops[o], e, f, loc[o], N)


def preconditioned(M):
    """C of Eq. (6): (G/2 + D~) G^{-1} (G/2 - D) + S~ G^{-1} N, formed densely."""
    G = M["G"]
    A1 = np.linalg.solve(G, 0.5 * G - M["D"])
    A2 = np.linalg.solve(G, M["N"])
    return (0.5 * G + M["Dt"]) @ A1 + M["S"] @ A2


def entries(curve, N, k, kt, rows, cols, rules=None):
    """Entries (rows[t], cols[t]) of (S~, D, D~, N), one element pair at a time.

    Same definition and rules as assemble(); used for sampled checks at sizes
    where the dense oracle would be too slow.  Returns a dict of complex arrays.
    """
    rules = rules or Rules()
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    # only the elements touching the requested node pairs (e = i - a, f = j - b)
    geo = ElementGeometry(curve, N, elements=np.concatenate([rows, rows - 1, cols, cols - 1]))
    out = np.zeros((4, len(rows)), complex)
    xg, wg = qd.gauss_legendre01(rules.q_far)
    far_rule = qd.tensor_rule(rules.q_far)
    for a in range(2):
        for b in range(2):
            e = (rows - a) % N
            f = (cols - b) % N
            d = np.abs(e - f)
            d = np.minimum(d, N - d)
            groups = [(d > rules.near, far_rule, None),
                      ((d >= 2) & (d <= rules.near), rules.near_rule, None),
                      ((d == 1) & ((e + 1) % N == f), rules.touch_next, "e_end"),
                      ((d == 1) & ((e - 1) % N == f) & ((e + 1) % N != f), rules.touch_prev, "e_start"),
                      (d == 0, rules.self_rule, "self")]
            for mask, rule, kind in groups:
                idx = np.nonzero(mask)[0]
                if len(idx) == 0:
                    continue
                loc = _locals(geo, e[idx], f[idx], rule, k, kt, kind)
                out[:, idx] += loc[:, a, b, :]
    return {"S": out[0], "D": out[1], "Dt": out[2], "N": out[3]}
