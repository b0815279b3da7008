"""Python binding of the solver library: marshals torch/numpy buffers into the
C ABI of include/wcs.h.  Every computation runs in libwcs.so on the GPU;
torch only provides device memory and the stream."""

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import OPS, Info, Options, SolveInfo, check, load


def default_options(**overrides):
    o = Options()
    check(load().wcs_default_options(C.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _solve_stats(si):
    return {"refine_steps": si.refine_steps, "rel_residual": si.rel_residual,
            "history": [si.history[i] for i in range(si.history_len)]}


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


class Solver:
    """One contour, its mesh, operators, skeleton and factorisation (one CUDA device)."""

    def __init__(self, device=None, stream=None, **options):
        self.lib = load()
        self.device = torch.device(device or "cuda")
        if self.device.type != "cuda":
            raise ValueError("the solver runs on a CUDA device only")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.opt = default_options(**options)
        h = C.c_void_p()
        check(self.lib.wcs_create(C.byref(h), C.byref(self.opt), C.c_void_p(self.stream.cuda_stream)))
        self.h = h
        self.N = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.wcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- contour and mesh
    def contour(self, family, **p):
        if family == "circle":
            check(self.lib.wcs_contour_circle(self.h, float(p.get("a", 1.0))))
        elif family == "ellipse":
            check(self.lib.wcs_contour_ellipse(self.h, float(p["ax"]), float(p["ay"])))
        elif family == "superellipse":
            check(self.lib.wcs_contour_superellipse(self.h, float(p["ax"]), float(p["ay"]), float(p["p"])))
        elif family == "fourier":
            cc, pc = _host(p["cos"], np.float64)
            ss, ps = _host(p.get("sin", np.zeros(len(cc))), np.float64)
            check(self.lib.wcs_contour_fourier(self.h, len(cc), pc, ps))
        else:
            raise ValueError(family)
        return self

    def perturb(self, alpha, beta):
        """Add sum alpha_m cos(m theta) + sum beta_m sin(m theta) (m from 0 and
        from 1) to the contour's radial function; len(alpha) == len(beta)."""
        a, pa = _host(alpha, np.float64)
        b, pb = _host(beta, np.float64)
        if len(a) != len(b):
            raise ValueError("alpha and beta need the same length")
        check(self.lib.wcs_contour_perturb(self.h, len(a), pa, pb))
        return self

    def mesh(self, N, k=None):
        check(self.lib.wcs_mesh(self.h, int(N), float(k) if k else 0.0))
        self.N = int(N)
        return self

    def info(self):
        i = Info()
        check(self.lib.wcs_query(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def geometry_sample(self, s):
        s, ps = _host(s, np.float64)
        out = np.empty(5 * len(s))
        check(self.lib.wcs_geometry_sample(self.h, len(s), ps, out.ctypes.data_as(C.c_void_p)))
        out = out.reshape(5, len(s))
        return dict(zip(("x", "y", "nx", "ny", "kappa"), out))

    # ---- setup
    def assemble(self):
        check(self.lib.wcs_assemble(self.h))
        return self

    def skeleton(self, tol, max_rank=0, seed=0, allow_cap=False):
        r = C.c_int(0)
        allow = (_lib.WCS_ERR_RANK_CAP,) if allow_cap else ()
        check(self.lib.wcs_skeleton(self.h, float(tol), int(max_rank), int(seed), C.byref(r)), allow)
        return r.value

    def factor(self):
        check(self.lib.wcs_factor(self.h))
        return self

    def save(self, path):
        """Write the skeleton and Woodbury factors (host file; see wcs_save)."""
        check(self.lib.wcs_save(self.h, str(path).encode()))
        return self

    def load(self, path):
        """Rebuild mesh and operators and restore the factors written by save()."""
        check(self.lib.wcs_load(self.h, str(path).encode()))
        info = self.info()
        self.N = int(info["N"])
        return self

    # ---- blocks: (N, B) views of column-major storage
    def _block(self, B):
        return torch.empty((B, self.N), dtype=torch.complex128, device=self.device)

    def _as_cols(self, X):
        X = torch.as_tensor(X, dtype=torch.complex128, device=self.device)
        if X.dim() == 1:
            X = X[:, None]
        return X.t().contiguous()  # (B, N) row-major == N x B column-major

    def apply(self, op, X):
        Xc = self._as_cols(X)
        B = Xc.shape[0]
        Y = self._block(B)
        check(self.lib.wcs_apply(self.h, OPS[op], B, _ptr(Xc), self.N, _ptr(Y), self.N))
        return Y.t()

    def circulant_eigs(self, op):
        out = torch.empty(self.N, dtype=torch.complex128, device=self.device)
        check(self.lib.wcs_circulant_eigs(self.h, OPS[op], _ptr(out)))
        return out

    def operator_entries(self, rows, cols):
        r, pr = _host(rows, np.int64)
        c, pc = _host(cols, np.int64)
        out = np.empty(4 * len(r), dtype=np.complex128)
        check(self.lib.wcs_operator_entries(self.h, len(r), pr, pc, out.ctypes.data_as(C.c_void_p)))
        return dict(zip(("S", "D", "Dt", "N"), out.reshape(4, len(r))))

    def planewave_rhs(self, angles):
        a, pa = _host(angles, np.float64)
        e, hv = self._block(len(a)), self._block(len(a))
        check(self.lib.wcs_planewave_rhs(self.h, len(a), pa, _ptr(e), _ptr(hv), self.N))
        return e.t(), hv.t()

    def woodbury_apply(self, b):
        bc = self._as_cols(b)
        x = self._block(bc.shape[0])
        check(self.lib.wcs_woodbury_apply(self.h, bc.shape[0], _ptr(bc), self.N, _ptr(x), self.N))
        return x.t()

    def solve_planewaves(self, angles, out=None, allow_unconverged=False):
        a, pa = _host(angles, np.float64)
        j = out if out is not None else self._block(len(a))
        si = SolveInfo()
        allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        check(self.lib.wcs_solve_planewaves(self.h, len(a), pa, _ptr(j), self.N, C.byref(si)), allow)
        self.last_solve = _solve_stats(si)
        return j.t()

    def solve_planewaves_host(self, angles, allow_unconverged=False, out=None):
        """Solve with host buffers: angles read from host memory, the (N, B)
        current written to host memory.  angles and out may be CPU torch
        tensors (pinned for full copy speed); out has shape (B, N), complex128."""
        if isinstance(angles, torch.Tensor):
            a = angles.to(torch.float64).contiguous()
            pa, na = C.c_void_p(a.data_ptr()), a.numel()
        else:
            a, pa = _host(angles, np.float64)
            na = len(a)
        if out is None:
            out = np.empty((na, self.N), dtype=np.complex128)
        pj = C.c_void_p(out.data_ptr()) if isinstance(out, torch.Tensor) else out.ctypes.data_as(C.c_void_p)
        si = SolveInfo()
        allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        check(self.lib.wcs_solve_planewaves_host(self.h, na, pa, pj, self.N, C.byref(si)), allow)
        self.last_solve = _solve_stats(si)
        return out.T

    def solve_rhs(self, e, hv, allow_unconverged=False):
        ec, hc = self._as_cols(e), self._as_cols(hv)
        j = self._block(ec.shape[0])
        si = SolveInfo()
        allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        check(self.lib.wcs_solve_rhs(self.h, ec.shape[0], _ptr(ec), _ptr(hc), self.N, _ptr(j), self.N,
                                     C.byref(si)), allow)
        self.last_solve = _solve_stats(si)
        return j.t()

    def _solve_general(self, fn, b, allow_unconverged):
        bc = self._as_cols(b)
        x = self._block(bc.shape[0])
        si = SolveInfo()
        allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        check(fn(self.h, bc.shape[0], _ptr(bc), self.N, _ptr(x), self.N, C.byref(si)), allow)
        self.last_solve = _solve_stats(si)
        return x.t()

    def solve(self, b, allow_unconverged=False):
        """x with C x = b (N x B or N, complex128): Eq. (9) plus refinement."""
        return self._solve_general(self.lib.wcs_solve, b, allow_unconverged)

    def solve_adjoint(self, b, allow_unconverged=False):
        """x with C^H x = b (N x B or N, complex128) through the adjoint factors."""
        return self._solve_general(self.lib.wcs_solve_adjoint, b, allow_unconverged)

    def shape_gradient(self, angles, phi_obs, M, delta=1e-6, allow_unconverged=False, params=None):
        """(J, grad): J = sum |F|^2 over incidences and observation angles and
        its gradient in (alpha_0..alpha_{M-1}, beta_1..beta_M); params = (i0, i1)
        restricts grad to those parameters (a rank's share of a sharded job)."""
        a, pa = _host(angles, np.float64)
        p, pp = _host(phi_obs, np.float64)
        i0, i1 = (0, 2 * int(M)) if params is None else (int(params[0]), int(params[1]))
        J = np.zeros(1)
        g = np.zeros(max(i1 - i0, 1))
        allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
        check(self.lib.wcs_shape_gradient_range(self.h, len(a), pa, len(p), pp, int(M), float(delta), i0, i1,
                                                J.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p)),
              allow)
        return float(J[0]), g[:i1 - i0]

    def shape_operator_forms(self, op, u, v, M, delta=1e-6, params=None):
        """sum_b u_b^H (dX/dp_i) v_b for operator op in ("S", "D", "DT", "N") and
        the shape parameters i (all 2M, or range params = (i0, i1)); u, v: N x B."""
        which = {"S": 0, "D": 1, "DT": 2, "Dt": 2, "N": 3}[op]
        uc, vc = self._as_cols(u), self._as_cols(v)
        i0, i1 = (0, 2 * int(M)) if params is None else (int(params[0]), int(params[1]))
        out = np.zeros(2 * max(i1 - i0, 1))
        check(self.lib.wcs_shape_operator_forms(self.h, which, uc.shape[0], _ptr(uc), _ptr(vc), self.N, int(M),
                                                float(delta), i0, i1, out.ctypes.data_as(C.c_void_p)))
        return (out[0::2] + 1j * out[1::2])[:i1 - i0]

    PROFILE_CATS = ("gemm_tc", "assembly", "fft", "zgemm", "skeleton", "factor", "solve", "gemm_tc_acc",
                    "sample", "project", "orth", "vw", "inverse", "gemm_exact", "assembly_fast", "gemm_tc_per")

    def profile(self, enable=True):
        check(self.lib.wcs_profile(self.h, 1 if enable else 0))

    def profile_read(self, reset=True):
        out = np.zeros(4 * len(self.PROFILE_CATS))
        check(self.lib.wcs_profile_read(self.h, 1 if reset else 0, out.ctypes.data_as(C.c_void_p)))
        out = out.reshape(-1, 4)
        return {c: {"launches": int(r[0]), "ms": r[1], "work": r[2], "bytes": r[3]}
                for c, r in zip(self.PROFILE_CATS, out)}

    def farfield(self, j, phi):
        jc = self._as_cols(j)
        p, pp = _host(phi, np.float64)
        F = torch.empty((jc.shape[0], len(p)), dtype=torch.complex128, device=self.device)
        check(self.lib.wcs_farfield(self.h, jc.shape[0], _ptr(jc), self.N, len(p), pp, _ptr(F), len(p)))
        return F.t()


def quadrature_tables(q):
    out = np.empty(3 * q * q)
    check(load().wcs_quadrature_tables(int(q), out.ctypes.data_as(C.c_void_p)))
    return out.reshape(3, q, q)


def gemm_split_bf16(A, B, planes=2, accurate=False):
    """D = A @ B.T on the tensor cores with split-bf16 operands (FP64 in/out, cuda).

    accurate: False/0 one accumulator over all of K; True/1 accumulator
    drained every K = 16 step; an int n > 1 drains every n steps (4: once per
    K = 64 stage, products issued smallest first across it)."""
    A = torch.as_tensor(A, dtype=torch.float64, device="cuda").contiguous()
    B = torch.as_tensor(B, dtype=torch.float64, device="cuda").contiguous()
    M, K = A.shape
    Nc = B.shape[0]
    D = torch.empty((M, Nc), dtype=torch.float64, device=A.device)
    st = torch.cuda.current_stream(A.device)
    check(load().wcs_gemm_split_bf16_ex(M, Nc, K, _ptr(A), K, _ptr(B), K, int(planes), int(accurate),
                                        _ptr(D), Nc, C.c_void_p(st.cuda_stream)))
    return D


def gemm_exact(A, B):
    """D = A @ B.T, exact up to ~2^-35 |A| |B|^T per entry, on the tensor cores
    (fixed-point bf16 slices, integer products, FP64 sums); FP64 in/out, cuda."""
    A = torch.as_tensor(A, dtype=torch.float64, device="cuda").contiguous()
    B = torch.as_tensor(B, dtype=torch.float64, device="cuda").contiguous()
    M, K = A.shape
    Nc = B.shape[0]
    D = torch.empty((M, Nc), dtype=torch.float64, device=A.device)
    st = torch.cuda.current_stream(A.device)
    check(load().wcs_gemm_exact(M, Nc, K, _ptr(A), K, _ptr(B), K, _ptr(D), Nc, C.c_void_p(st.cuda_stream)))
    return D


def batch_solve_fourier(contours, angles, tol=1e-6, rank_div=8, seed=1, workers=2, allow_unconverged=False,
                        **options):
    """Batched form: contours is a list of dicts {"cos": [...], "sin": [...], "N": int, "k": float or None}
    (Fourier radial functions); every contour is solved for the same plane waves.
    Returns (list of N_c x B complex128 host arrays, list of per-contour stats dicts)."""
    lib = load()
    opt = default_options(**options)
    nf = max(len(c["cos"]) for c in contours)
    count = len(contours)
    cs = np.zeros((count, nf))
    sn = np.zeros((count, nf))
    for i, c in enumerate(contours):
        cs[i, :len(c["cos"])] = c["cos"]
        sn[i, :len(c.get("sin", []))] = c.get("sin", [])
    Ns = np.array([int(c["N"]) for c in contours], dtype=np.int64)
    ks = np.array([float(c.get("k") or 0.0) for c in contours])
    a = np.ascontiguousarray(angles, dtype=np.float64)
    B = len(a)
    out = np.zeros(int(Ns.sum()) * B, dtype=np.complex128)
    stats = (_lib.BatchStats * max(count, 1))()
    allow = (_lib.WCS_ERR_NOT_CONVERGED,) if allow_unconverged else ()
    check(lib.wcs_batch_solve_fourier(C.byref(opt), count, nf, cs.ctypes.data_as(C.c_void_p),
                                      sn.ctypes.data_as(C.c_void_p), Ns.ctypes.data_as(C.c_void_p),
                                      ks.ctypes.data_as(C.c_void_p), B, a.ctypes.data_as(C.c_void_p), float(tol),
                                      int(rank_div), int(seed), int(workers), out.ctypes.data_as(C.c_void_p),
                                      stats), allow)
    js, o = [], 0
    for n in Ns:
        js.append(out[o:o + n * B].reshape(B, n).T)
        o += n * B
    st = [{f: getattr(stats[i], f) for f, _ in _lib.BatchStats._fields_} for i in range(count)]
    return js, st
