"""Split-precision (BF16 hi + lo on the tensor cores) BF apply and refinement.

Tolerance of the split path: rel-l2 <= 1e-4 against the oracle's apply of the
same factors.  Refinement forms its residuals with the FP32 applies, so one
step must bring the solve error far below the HSS tolerance band.
"""
import numpy as np
import pytest
import torch

from fio_inputs import crandn
from oracle.butterfly import Butterfly1D
from oracle.problem import K_rows, Phase
from oracle.solver import FIOSolver
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n", [1 << 12, 1 << 13, 1 << 14])
@pytest.mark.parametrize("k", [1, 5, 16])
def test_split_apply_matches_oracle(n, k):
    from paper_2609_11520_b300 import BF
    ob = Butterfly1D(Phase("cabs", 0.8), n, 16)
    gb = BF(n, 16, "cabs", 0.8).set_precision("split_bf16")
    f = crandn(n, k, seed=n + k)
    e_fwd = rel(to_np(gb.apply(to_dev(f))), ob.apply(f))
    e_adj = rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f))
    assert e_fwd < TOL_SPLIT and e_adj < TOL_SPLIT, (e_fwd, e_adj)
    assert e_fwd > 1e-8   # it really is a different arithmetic than FP32


@pytest.mark.parametrize("n", [1 << 16, 1 << 17, 1 << 18])
def test_split_apply_full_size_sampled_rows(n):
    from paper_2609_11520_b300 import BF
    gb = BF(n, 16).set_precision("split_bf16")
    f = crandn(n, 2, seed=7)
    y = to_np(gb.apply(to_dev(f)))
    rows = np.random.default_rng(1).choice(n, 128, replace=False)
    assert rel(y[rows], K_rows(Phase("cabs"), n, rows) @ f) < TOL_SPLIT
    g = crandn(n, 1, seed=8)[:, 0]
    lhs = np.vdot(g, y[:, 0])
    rhs = np.vdot(to_np(gb.adjoint(to_dev(g))), f[:, 0])
    assert abs(lhs - rhs) / abs(lhs) < TOL_SPLIT


def test_split_rejected_where_unsupported():
    from paper_2609_11520_b300 import BF, FioError
    with pytest.raises(FioError):
        BF(1024, 16).set_precision("split_bf16")


def test_split_solve_and_refinement():
    """N = 4096, tol 1e-3: split solve within 2x the oracle's error; one FP32-residual refinement
    step gains more than an order of magnitude (the iteration contracts by about tol per step)."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    n, leaf, p, tol, seed = 4096, 128, 10, 1e-3, 1
    S = FIOSolver(Phase("cabs"), n, 16, leaf, p, tol, seed)
    f = crandn(n, 4, seed=0)
    u = S.bf.apply(f)
    e_oracle = rel(S.solve(u), f)
    bf = BF(n, 16)
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed).factor()
    U = to_dev(u)
    e32 = rel(to_np(fio_solve(bf, g, U)), f)
    bf.set_precision("split_bf16")
    e_split = rel(to_np(fio_solve(bf, g, U)), f)
    e_ref = rel(to_np(fio_solve(bf, g, U, refine_steps=1)), f)
    e_ref2 = rel(to_np(fio_solve(bf, g, U, refine_steps=2)), f)
    assert e_split <= 2 * e_oracle, (e_split, e_oracle)
    assert abs(e_split - e32) < 0.1 * e32
    assert e_ref < 0.1 * e_split, (e_ref, e_split)
    assert e_ref2 <= e_ref * 1.01 + 1e-6


@pytest.mark.parametrize("k", [16, 40])
def test_split_solve_with_tensor_core_hss_products(k):
    """Split precision on the HSS products too: the ULV node products of k > 8 columns on the
    tensor cores with BF16 hi/lo parts (solve path 1 under a split-precision BF handle).  The
    solve error stays within 2x the oracle's (the HSS tolerance dominates BF16 hi/lo rounding) and
    one FP32-residual refinement step still gains an order of magnitude."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    n, leaf, p, tol, seed = 4096, 128, 10, 1e-3, 1
    S = FIOSolver(Phase("cabs"), n, 16, leaf, p, tol, seed)
    f = crandn(n, k, seed=3)
    u = S.bf.apply(f)
    e_oracle = rel(S.solve(u), f)
    bf = BF(n, 16).set_precision("split_bf16")
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed).factor()
    U = to_dev(u)
    e_cc = rel(to_np(fio_solve(bf, g, U)), f)
    g.set_solve_path("tensor_cores")
    e_tc = rel(to_np(fio_solve(bf, g, U)), f)
    e_ref = rel(to_np(fio_solve(bf, g, U, refine_steps=1)), f)
    assert e_tc <= 2 * e_oracle, (e_tc, e_oracle)
    assert abs(e_tc - e_cc) < 0.1 * e_cc
    assert e_ref < 0.1 * e_tc, (e_ref, e_tc)
