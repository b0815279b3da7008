"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-side quadrature tables are exact (no GPU needed)."""

import os
import re

import numpy as np
import pytest
import scipy.integrate as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_13283_gb300 import build
    build.build()
    from paper_2203_13283_gb300 import _lib
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wcs.h")).read()
    return sorted(set(re.findall(r"\b(wcs_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    import ctypes
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each of them
    from paper_2203_13283_gb300 import _lib
    assert set(names) == set(_lib.SIGNATURES)
    assert b"sm_103a" in lib.wcs_version()
    del ctypes


def test_options_defaults(lib):
    from paper_2203_13283_gb300.solver import default_options
    o = default_options()
    assert (o.q_far, o.q_near, o.near_band, o.precision, o.sample_planes) == (0, 0, 4, 0, 0)
    assert (o.zfast, o.exact_residual) == (-1.0, 0)


@pytest.mark.parametrize("q", [8, 12])
def test_product_integration_weights_exact_on_polynomials(lib, q):
    from paper_2203_13283_gb300.solver import quadrature_tables
    W = quadrature_tables(q)
    x, _ = np.polynomial.legendre.leggauss(q)
    x = 0.5 * (x + 1)
    logs = {0: lambda a, b: np.log(abs(a - b)), 1: lambda a, b: np.log(1 - a + b),
            2: lambda a, b: np.log(a + 1 - b)}
    for kind in range(3):
        for (pa, pb) in [(0, 0), (1, 0), (2, 3), (q - 1, 1)]:
            F = np.outer(x ** pa, x ** pb)
            approx = np.sum(W[kind] * F)
            g = lambda b, a: a ** pa * b ** pb * logs[kind](a, b)
            if kind == 0:
                ref = (si.dblquad(g, 0, 1, 0, lambda a: a, epsabs=1e-12, epsrel=1e-12)[0]
                       + si.dblquad(g, 0, 1, lambda a: a, 1, epsabs=1e-12, epsrel=1e-12)[0])
            else:
                ref = si.dblquad(g, 0, 1, 0, 1, epsabs=1e-12, epsrel=1e-12)[0]
            assert abs(approx - ref) < 1e-9, (kind, pa, pb, approx, ref)
    assert abs(W[0].sum() + 1.5) < 1e-13
    assert abs(W[1].sum() - (2 * np.log(2) - 1.5)) < 1e-13


def test_product_weights_symmetry(lib):
    from paper_2203_13283_gb300.solver import quadrature_tables
    W = quadrature_tables(12)
    assert np.max(np.abs(W[0] - W[0].T)) < 1e-14
    # log(xi + 1 - eta) is log(1 - xi' + eta') with the roles of xi and eta swapped
    assert np.max(np.abs(W[2] - W[1].T)) < 1e-14


def test_checkpoint_rejects_null_arguments(lib):
    """wcs_save / wcs_load validate their arguments before touching a device."""
    from paper_2203_13283_gb300._lib import WCS_ERR_ARG
    assert lib.wcs_save(None, b"/nonexistent/ckpt") == WCS_ERR_ARG
    assert lib.wcs_load(None, b"/nonexistent/ckpt") == WCS_ERR_ARG


def test_differentiation_entry_points_validate_before_device_work(lib):
    """wcs_contour_perturb, wcs_solve, wcs_solve_adjoint and wcs_shape_gradient
    check their arguments and the call order on the host."""
    import ctypes as C
    WCS_ERR_ARG, WCS_ERR_STATE = 1, 9
    h = C.c_void_p()
    assert lib.wcs_create(C.byref(h), None, None) == 0
    z = np.zeros(40)
    pz = z.ctypes.data_as(C.c_void_p)
    assert lib.wcs_contour_perturb(h, 0, None, None) == WCS_ERR_STATE      # no contour yet
    assert lib.wcs_contour_ellipse(h, 1.0, 0.7) == 0
    assert lib.wcs_contour_perturb(h, 33, pz, pz) == WCS_ERR_ARG           # M <= 32
    assert lib.wcs_contour_perturb(h, 2, None, None) == WCS_ERR_ARG
    assert lib.wcs_contour_perturb(h, 2, pz, pz) == 0
    J, g = np.zeros(1), np.zeros(4)
    assert lib.wcs_shape_gradient(h, 1, pz, 1, pz, 2, 1e-6, J.ctypes.data_as(C.c_void_p),
                                  g.ctypes.data_as(C.c_void_p)) == WCS_ERR_STATE   # not factored
    assert lib.wcs_solve(h, 1, pz, 40, pz, 40, None) == WCS_ERR_STATE
    assert lib.wcs_solve_adjoint(h, 1, pz, 40, pz, 40, None) == WCS_ERR_STATE
    assert lib.wcs_solve(None, 1, pz, 40, pz, 40, None) == WCS_ERR_ARG
    assert lib.wcs_shape_gradient(None, 1, pz, 1, pz, 2, 1e-6, None, None) == WCS_ERR_ARG
    assert lib.wcs_shape_gradient_range(None, 1, pz, 1, pz, 2, 1e-6, 0, 4, None, None) == WCS_ERR_ARG
    assert lib.wcs_shape_gradient_range(h, 1, pz, 1, pz, 2, 1e-6, 0, 4, J.ctypes.data_as(C.c_void_p),
                                        g.ctypes.data_as(C.c_void_p)) == WCS_ERR_STATE
    assert lib.wcs_destroy(h) == 0


def test_header_is_plain_c(tmp_path):
    """include/wcs.h is a C-ABI header: it compiles as strict C99 and as C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_header.c"
    src.write_text('#include "wcs.h"\n'
                   'int main(void) {\n'
                   '  int (*f)(wcs_options*) = wcs_default_options;\n'
                   '  int (*g)(wcs_ctx*, int64_t, const double*, int64_t, double*, int64_t, wcs_solve_info*) =\n'
                   '      wcs_solve_adjoint;\n'
                   '  return (int)(sizeof(wcs_options) == 0) + (f == 0) + (g == 0);\n'
                   '}\n')
    inc = os.path.join(ROOT, "include")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc,
                    str(src)], check=True)
    gxx = shutil.which("g++")
    if gxx:
        subprocess.run([gxx, "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, "-x", "c++", str(src)],
                       check=True)


# ---- checkpoint file format (version 3), checked on the host ------------------
def _ckpt_structs():
    import ctypes as C
    from paper_2203_13283_gb300._lib import Options

    class Contour(C.Structure):
        _fields_ = [("family", C.c_int), ("a", C.c_double), ("ax", C.c_double), ("ay", C.c_double),
                    ("p", C.c_double), ("nf", C.c_int), ("fc", C.c_double * 64), ("fs", C.c_double * 64),
                    ("np", C.c_int), ("pc", C.c_double * 33), ("ps", C.c_double * 33)]

    class Header(C.Structure):
        _fields_ = [("magic", C.c_char * 8), ("version", C.c_int32), ("rank", C.c_int32), ("N", C.c_int64),
                    ("k", C.c_double), ("opt", Options), ("contour", Contour)]

    return Header


def _fnv64_words(data):
    """FNV-1a, 64-bit basis and prime, over 8-byte little-endian words; the
    final partial word byte by byte (the checkpoint trailer's checksum)."""
    h, prime, mask = 14695981039346656037, 1099511628211, (1 << 64) - 1
    n8 = len(data) // 8
    for w in np.frombuffer(data[:8 * n8], dtype="<u8").tolist():
        h = ((h ^ w) * prime) & mask
    for b in data[8 * n8:]:
        h = ((h ^ b) * prime) & mask
    return h


def _write_ckpt(path, lib, N=16, rank=2, kinv=True, corrupt_at=None, cut=0):
    import ctypes as C
    from paper_2203_13283_gb300.solver import default_options
    Header = _ckpt_structs()
    hd = Header()
    hd.magic = b"WCSCKPT1"
    hd.version, hd.rank, hd.N, hd.k = 3, rank, N, 4.0
    hd.opt = default_options()
    lib.wcs_default_options(C.byref(hd.opt))
    hd.opt.q_far, hd.opt.q_near = 6, 12          # as wcs_create resolves the automatic choice
    hd.opt.sample_planes = 2
    hd.opt.zfast = 0.0                            # resolved value of the FP64 form
    hd.contour.family, hd.contour.ax, hd.contour.ay = 1, 1.0, 0.5
    ext = np.array([1 if kinv else 0, 0], dtype="<u4").tobytes()
    rng = np.random.default_rng(5)
    payload = rng.standard_normal(2 * (3 * N * rank + (rank * rank if kinv else 0))).tobytes()
    body = bytes(hd) + ext + payload
    data = bytearray(body + b"WCSFNV64" + _fnv64_words(body).to_bytes(8, "little"))
    if corrupt_at is not None:
        data[corrupt_at] ^= 0x10
    if cut:
        data = data[:-cut]
    path.write_bytes(bytes(data))
    return len(bytes(hd)) + len(ext)


def test_checkpoint_checksum_and_size_are_checked_before_device_work(lib, tmp_path):
    """Version-3 checkpoints carry an FNV-1a checksum; wcs_load rejects a
    corrupted or truncated file with WCS_ERR_ARG before any device work (a
    valid file gets past the check and fails later, here for want of a GPU)."""
    import ctypes as C
    from paper_2203_13283_gb300._lib import WCS_ERR_ARG
    h = C.c_void_p()
    assert lib.wcs_create(C.byref(h), None, None) == 0
    good = tmp_path / "good.wcs"
    off = _write_ckpt(good, lib)
    cases = {"corrupt": dict(corrupt_at=off + 100), "header": dict(corrupt_at=12),
             "truncated": dict(cut=9), "no_kinv_flag_mismatch": dict(kinv=False, cut=0)}
    for name, kw in cases.items():
        p = tmp_path / f"{name}.wcs"
        _write_ckpt(p, lib, **kw)
        if name == "no_kinv_flag_mismatch":
            # flip the flag word without fixing the checksum
            d = bytearray(p.read_bytes())
            d[off - 8] ^= 1
            p.write_bytes(bytes(d))
        st = lib.wcs_load(h, str(p).encode())
        assert st == WCS_ERR_ARG, name
        msg = lib.wcs_last_error().decode()
        assert ("checksum" in msg) or ("truncated" in msg) or ("bad sizes" in msg) or ("after the trailer" in msg), \
            (name, msg)
    garbage = tmp_path / "garbage.wcs"
    garbage.write_bytes(b"not a checkpoint at all" * 10)
    assert lib.wcs_load(h, str(garbage).encode()) == WCS_ERR_ARG
    st = lib.wcs_load(h, str(good).encode())
    msg = lib.wcs_last_error().decode()
    assert "checksum" not in msg and "truncated" not in msg, msg
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        assert st != 0           # got past the file checks, then needed a device
    assert lib.wcs_destroy(h) == 0
