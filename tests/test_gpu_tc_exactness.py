"""The property that exact (fixed-point sliced) products rest on: the
tensor core's FP32 accumulation of bf16 products whose values are integers
is exact as long as every partial sum stays below 2^24 in magnitude.

Integers |a|, |b| <= 128 are exact in bf16 and their products (<= 2^14)
exact in FP32; over K terms the sum is bounded by K 2^14.  One bf16 plane
per operand (a single product, accumulated over all of K in tensor memory)
is compared with the exact integer product computed on the host."""

import numpy as np
import pytest
import torch

from gpu_common import built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [64, 512, 1024])
def test_integer_bf16_products_accumulate_exactly(K):
    built()
    from paper_2203_13283_gb300.solver import gemm_split_bf16
    rng = np.random.default_rng(K)
    M, Nc = 2560, 2048            # 20 x 8 = 160 output tiles: no split of K
    A = rng.integers(-128, 129, size=(M, K))
    B = rng.integers(-128, 129, size=(Nc, K))
    # worst case for the accumulator: all products of one sign in some rows
    A[:8] = 128
    B[:8] = 128
    A[8:16] = -128
    exact = A.astype(np.float64) @ B.astype(np.float64).T     # exact: |partial sums| < 2^53
    assert np.max(np.abs(exact)) <= K * 2 ** 14 <= 2 ** 24
    D = gemm_split_bf16(torch.tensor(A, dtype=torch.float64), torch.tensor(B, dtype=torch.float64),
                        planes=1).cpu().numpy()
    assert np.array_equal(D, exact), np.max(np.abs(D - exact))
