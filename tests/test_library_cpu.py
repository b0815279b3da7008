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
