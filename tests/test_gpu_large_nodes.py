"""Large-node kernels (level-3 formulations for HSS levels with few, large nodes:
FP32 bulk products at tol >= 1e-4, FP64 node pass below it, FP64 Gram/pivoted
Cholesky, root, eliminated-block Cholesky and merge) against the same
references as the one-CTA kernels.

The threshold is lowered to 2 so that the large-node path runs on small cases
whose exact answers are known: generator-built HSS matrices (matvec, ULV solve
against the oracle and dense solves), the black-box construction on exact HSS
matrices (ranks recovered, G~ = H), and the 1D and 2D online solves against
the oracle.  The natural case (2D, n = 64, leaf 256: levels 1-3 have 930..1560
unknowns per node) is compared with the oracle's stored error.
"""
import os

import numpy as np
import pytest
import torch

from fio_inputs import crandn
from tests import test_gpu_bf2d as t2d
from tests import test_gpu_hss as base
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "solve2d_n64.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture
def large():
    from paper_2609_11520_b300 import set_large_node
    set_large_node(2)
    yield
    set_large_node(384)


@pytest.mark.parametrize("N,leaf,ranks", base.CASES)
def test_ulv_large_matches_oracle(large, N, leaf, ranks):
    base.test_ulv_solve_matches_oracle(N, leaf, ranks)


def test_ulv_large_rejects_indefinite(large):
    base.test_ulv_rejects_indefinite()


@pytest.mark.parametrize("N,leaf,ranks", [(512, 32, [0, 6, 5, 5, 4]), (1024, 64, [0, 10, 9, 8, 7]),
                                          (256, 32, [0, 0, 2, 3])])
def test_blackbox_large_recovers_exact_hss(large, N, leaf, ranks):
    base.test_blackbox_recovers_exact_hss(N, leaf, ranks)


@pytest.mark.parametrize("tol", [1e-4, 3e-3])
def test_fio_pipeline_large(large, tol):
    """1D, N = 1024, leaf 64, every level on the large-node kernels.  The large-node path reveals
    ranks with a random orthonormal null basis instead of the oracle's Householder one, so a pivot
    that lies close to the truncation threshold can fall on either side of it.  At tol 1e-3 some
    pivots of this operator lie within 0.9..1.4 x the threshold; at the two tolerances used here
    none lies within 0.7..1.6 x (oracle pivots, ranks 4 and 2 per level), so the ranks are
    decided the same way on both sides and the bound is the benchmark spec's 2x."""
    from oracle.problem import Phase
    from oracle.solver import FIOSolver
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    n, leaf, p, seed = 1024, 64, 10, 1
    S = FIOSolver(Phase("cabs"), n, 16, leaf, p, tol, seed)
    bf = BF(n, 16)
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed)
    assert g.info()["ranks"] == S.hss.ranks, (g.info()["ranks"], S.hss.ranks)
    x = crandn(n, 2, seed=3)
    GKx = S.bf.adjoint(S.bf.apply(x))
    e_hss_o = rel(S.hss.matvec(x), GKx)
    e_hss_g = rel(to_np(g.matvec(to_dev(x))), GKx)
    assert e_hss_g <= 2 * e_hss_o + 1e-5, (e_hss_g, e_hss_o, g.info()["ranks"], S.stats["ranks"])
    g.factor()
    f = crandn(n, 4, seed=0)
    u = S.bf.apply(f)
    e_o = rel(S.solve(u), f)
    e_g = rel(to_np(fio_solve(bf, g, to_dev(u))), f)
    assert e_g <= 2 * e_o + 1e-5, (e_g, e_o)
    e_r = rel(to_np(fio_solve(bf, g, to_dev(u), refine_steps=2)), f)
    assert e_r <= 2 * e_o + 1e-5, (e_r, e_o)


def test_solve2d_large(large):
    t2d.test_solve2d_matches_oracle(check_ranks=False)


def test_solve2d_n64_natural():
    """n = 64 (N = 4096), leaf 256, default threshold: the top levels take the large-node
    path by themselves.  Error against f_true within 2x the oracle's stored value."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    vals = dict(line.split()[:2] for line in open(GOLDEN) if not line.startswith("#"))
    e_oracle = float(vals["e_direct"])
    n = 64
    bf = BF(n, 25, "elliptic2d")
    g = HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=1).factor()
    f = crandn(n * n, 2, seed=0)
    u = bf.apply(to_dev(f))
    e = rel(to_np(fio_solve(bf, g, u)), f)
    assert e <= 2 * e_oracle, (e, e_oracle, g.info()["ranks"])
    e1 = rel(to_np(fio_solve(bf, g, u, refine_steps=1)), f)
    assert e1 < e
