"""The integer bf16 split of the staging kernels (csrc/split.cuh) against the
FP64 split it replaces, compiled for the host: every plane must agree bit for
bit (random values across the exponent window and beyond it, constructed
round-to-nearest ties in each plane, zeros, subnormals, infinities, NaN)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_integer_split_matches_fp64_split(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "split_bits_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "split_bits_check.cu")], check=True,
                   capture_output=True, timeout=300)
    r = subprocess.run([exe, "2000000"], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "mismatching planes 0" in r.stdout
