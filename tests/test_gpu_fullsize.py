"""Full-size checks of the FP64 path: ellipse 1.0 x 0.5, N = 4096,
10 elements per wavelength, 360 plane waves at 1-degree steps.

The dense oracle is too slow at this size, so the operator is checked on
sampled entries computed one by one by the oracle, and the solution through
properties that hold at any size: mirror symmetry of the current for
incidence along the symmetry axis, far-field reciprocity (to discretisation
error), and the refinement residual."""

import numpy as np
import pytest
import torch

import workloads
from gpu_common import make_solver, to_np
from oracle import assembly
from oracle_cache import curve_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ellipse4096():
    w = workloads.WORKLOADS["ellipse_n4096"]
    s = make_solver(w)
    s.assemble()
    yield w, s
    s.close()


def test_sampled_entries_vs_oracle(ellipse4096):
    w, s = ellipse4096
    N = w["N"]
    info = s.info()
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.integers(0, N, 120), np.arange(0, N, 512)])
    cols = np.concatenate([rng.integers(0, N, 120), (np.arange(0, N, 512) + rng.integers(-3, 4, 8)) % N])
    rows = np.concatenate([rows, [0, 0, N - 1, 5, 4095]])
    cols = np.concatenate([cols, [0, N - 1, 0, 7, 4093]])
    G = s.operator_entries(rows, cols)
    cur = curve_of(w)
    O = assembly.entries(cur, N, info["k"], complex(info["kt_re"], info["kt_im"]), rows, cols)
    # the same entries read back from the assembled dense operators
    I = torch.zeros((N, 1), dtype=torch.complex128, device="cuda")
    # scale: operators enter C of Eq. (6) next to G/2, whose entries are O(h);
    # nearly coincident points carry an absolute rounding floor ~1e-17 in the
    # double-layer kernel ((r - r').n' / R^2), on both sides
    h = info["h"]
    for key in ("S", "D", "Dt"):
        assert np.max(np.abs(G[key] - O[key])) < 1e-12 * h, key
    assert np.max(np.abs(G["N"] - O["N"])) < 1e-12 * np.max(np.abs(O["N"]))
    for c in np.unique(cols)[:4]:
        I.zero_()
        I[c, 0] = 1.0
        for key, op in (("S", "S"), ("N", "N")):
            col = to_np(s.apply(op, I))[:, 0]
            sel = cols == c
            assert np.max(np.abs(col[rows[sel]] - G[key][sel])) < 1e-13 * np.max(np.abs(G[key]))


def test_solution_invariants(ellipse4096):
    w, s = ellipse4096
    N = w["N"]
    rank = s.skeleton(w["tol"], seed=1)
    assert rank > 0
    s.factor()
    j = to_np(s.solve_planewaves(w["angles"]))
    assert s.last_solve["rel_residual"] <= 1e-12
    # mirror symmetry of the ellipse about the x axis, incidence at 0 degrees
    j0 = j[:, 0]
    assert np.max(np.abs(j0 - j0[(-np.arange(N)) % N])) < 1e-10 * np.max(np.abs(j0))
    # incidence at 90 degrees: symmetric about the y axis, node i <-> N/2 - i
    j90 = j[:, 90]
    assert np.max(np.abs(j90 - j90[(N // 2 - np.arange(N)) % N])) < 1e-10 * np.max(np.abs(j90))
    # reciprocity F(po; pi) = F(pi + pi; po + pi) to discretisation error
    phi = np.deg2rad(np.arange(360.0))
    F = to_np(s.farfield(torch.tensor(j, device="cuda"), phi))   # (n_obs, n_inc)
    for pi_, po in [(10, 250), (33, 100), (0, 180)]:
        a = F[po, pi_]
        b = F[(pi_ + 180) % 360, (po + 180) % 360]
        assert abs(a - b) < 1e-3 * abs(a)
