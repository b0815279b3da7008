"""Host logic of bench.py: the per-kernel roofline entries it builds from the
run's CUDA-event profile and the per-unit figures of the ncu summaries in
profiles/.  Every figure the bench reads must be present and parse, and each
entry must be consistent (frac = achieved / peak, issued fraction = products
x useful fraction, traffic = figure x units)."""

import pytest

import bench

FIGURES = [
    ("k_gemm_tc_ellipse_n4096_mixed.md", "dram_bytes_per_algorithmic_byte"),
    ("k_gemm_tc_acc_ellipse_n4096_mixed.md", "dram_bytes_per_algorithmic_byte"),
    ("k_gemm_tc_per_superellipse_n4096_mixed.md", "dram_bytes_per_algorithmic_byte"),
    ("k_circ_pass_superellipse_n32768_mixed.md", "dram_bytes_per_algorithmic_byte"),
    ("k_assemble_fp64_superellipse_n4096_mixed.md", "fp64_flops_per_far_point_pair"),
    ("k_assemble_fp64_superellipse_n4096_mixed.md", "dram_bytes_per_far_point_pair"),
    ("k_assemble_fp64_superellipse_n4096_mixed.md", "pipe_active_frac"),
    ("k_assemble_fast_superellipse_n4096_zfast9.md", "fp32_flops_per_far_point_pair"),
    ("k_assemble_fast_superellipse_n4096_zfast9.md", "dram_bytes_per_far_point_pair"),
    ("k_assemble_fast_superellipse_n4096_zfast9.md", "pipe_active_frac"),
]


@pytest.mark.parametrize("name,key", FIGURES)
def test_profile_figures_present(name, key):
    v, src = bench.profile_figure(name, key)
    assert v is not None and v > 0, (name, key)
    assert src == "profiles/" + name
    if key == "pipe_active_frac":
        assert v <= 1.0


def test_missing_figure_is_none():
    assert bench.profile_figure("no_such_profile.md", "x") == (None, None)
    assert bench.profile_figure("k_gemm_tc_ellipse_n4096_mixed.md", "no_such_key")[0] is None


HBM, BF16, FMA = 6763.3, 1701.9, {64: 1.25e12, 32: 78.0e12}


def _prof(cat, launches, ms, work, nbytes):
    return {cat: {"launches": launches, "ms": ms, "work": work, "bytes": nbytes}}


@pytest.mark.parametrize("cat,nprod", [("gemm_tc", 3), ("gemm_tc_acc", 6), ("gemm_tc_per", 3)])
def test_tensor_entry(cat, nprod):
    work, nbytes = 8.0e13, 2.0e10
    r = bench.roofline_entry(cat, _prof(cat, 4, 100.0, work, nbytes), HBM, BF16, FMA)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(work / 0.1 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / BF16)
    assert r["issued_frac"] == pytest.approx(nprod * r["frac"])
    name = r["traffic_source"].split("/")[-1]
    ratio, _ = bench.profile_figure(name, "dram_bytes_per_algorithmic_byte")
    changed, _ = bench.profile_figure(name, "kernel_changed_since_capture")
    if changed:
        # counters older than the kernel: no traffic figure, and a note says why
        assert r["traffic"] is None and r["traffic_note"]
    else:
        assert r["traffic"] == pytest.approx(ratio * nbytes / 4)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(nbytes / 4)


def test_fft_entry():
    nbytes = 1.0e11
    r = bench.roofline_entry("fft", _prof("fft", 48, 30.0, 0.0, nbytes), HBM, BF16, FMA)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(nbytes / 0.03 / 1e9 / HBM)
    assert r["traffic"] is not None


@pytest.mark.parametrize("cat,bits", [("assembly", 64), ("assembly_fast", 32)])
def test_assembly_entry(cat, bits):
    pairs, launches, ms = 1.8e9 * 3, 3, 3600.0
    r = bench.roofline_entry(cat, _prof(cat, launches, ms, pairs, 0.0), HBM, BF16, FMA)
    key = "fp64_flops_per_far_point_pair" if bits == 64 else "fp32_flops_per_far_point_pair"
    fpu, _ = bench.profile_figure(r["figures_source"].split("/")[-1], key)
    per_launch = pairs / launches
    assert r["achieved"] == pytest.approx(fpu * per_launch / (ms / 1e3 / launches) / 1e12)
    assert r["peak"] == pytest.approx(FMA[bits] / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert 0 < r["pipe_active_frac"] <= 1.0
    assert r["traffic"] > 0


def test_empty_category_has_no_entry():
    assert bench.roofline_entry("gemm_tc", _prof("gemm_tc", 0, 0.0, 0.0, 0.0), HBM, BF16, FMA) is None
