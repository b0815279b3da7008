"""The allocation-free contraction entry point (wcs_gemm_split_bf16_noalloc).

It exists for callers that cannot allocate device memory (frozen memory
pools, plug-ins whose host owns all device memory): it keeps its staging in a
fixed device array instead.  Its results must match the allocating entry
point wcs_gemm_split_bf16 on the same inputs, on consecutive calls (the shared
array keeps the previous call's contents, which must not leak into the next).
This file is collected last on purpose."""

import ctypes as C

import pytest
import torch

from gpu_common import built

pytestmark = pytest.mark.gpu


def _call(fn, A, B, planes):
    M, K = A.shape
    Nc = B.shape[0]
    D = torch.full((M, Nc), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    from paper_2203_13283_gb300._lib import check
    check(fn(M, Nc, K, C.c_void_p(A.data_ptr()), K, C.c_void_p(B.data_ptr()), K, planes,
             C.c_void_p(D.data_ptr()), Nc, C.c_void_p(st)))
    return D


def test_noalloc_matches_allocating_entry_point_twice():
    built()
    from paper_2203_13283_gb300._lib import load
    lib = load()
    g = torch.Generator(device="cpu").manual_seed(11)
    # two calls in a row with different shapes and data: the second must not
    # see the first call's planes (K padding, stale columns)
    for (M, Nc, K, planes) in [(300, 200, 1000, 3), (130, 70, 200, 2)]:
        A = torch.randn(M, K, generator=g, dtype=torch.float64).cuda()
        B = torch.randn(Nc, K, generator=g, dtype=torch.float64).cuda()
        ref = _call(lib.wcs_gemm_split_bf16, A, B, planes)
        out = _call(lib.wcs_gemm_split_bf16_noalloc, A, B, planes)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        scale = (A.abs() @ B.abs().T).max()
        assert ((out - ref).abs().max() / scale).item() < 1e-12
        exact = A @ B.T
        bound = {2: 6e-5, 3: 1e-5}[planes]
        assert ((out - exact).abs().max() / scale).item() < bound


def test_noalloc_rejects_oversize():
    built()
    from paper_2203_13283_gb300._lib import WCSError, check, load
    lib = load()
    A = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    with pytest.raises(WCSError) as ei:
        check(lib.wcs_gemm_split_bf16_noalloc(4096, 4096, 4096, C.c_void_p(A.data_ptr()), 4096,
                                              C.c_void_p(A.data_ptr()), 4096, 3, C.c_void_p(A.data_ptr()),
                                              4096, C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    assert "32 MiB" in str(ei.value)


def test_noalloc_empty_contraction_zeroes_output():
    # K = 0: D = A B^T is the zero matrix; the call must write it (the output
    # buffer starts as NaN) for both entry points, twice in a row
    built()
    from paper_2203_13283_gb300._lib import load
    lib = load()
    A = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    for fn in (lib.wcs_gemm_split_bf16_noalloc, lib.wcs_gemm_split_bf16, lib.wcs_gemm_split_bf16_noalloc):
        D = _call(fn, A[:, :0].expand(37, 0), A[:, :0].expand(19, 0), 2)
        torch.cuda.synchronize()
        assert D.shape == (37, 19)
        assert (D == 0).all()
