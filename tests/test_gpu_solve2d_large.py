"""The 2D end-to-end solve at the sizes of Section 5.2's table (n = 128 and n = 256, N = 2^14 and
2^16) on the 7 x 7 Chebyshev grid (r = 49; at 5 x 5 the BF error lies above the HSS tolerance and
the HSS ranks outgrow the offline budget).

n = 64, 128: the GPU solve error against f_true is no worse than 2x the stored oracle error
(tests/golden/solve2d_n{64,128}_r49.txt, same seeds).  n = 256: the oracle does not finish
there, so the checks are properties that hold at any size: the HSS of G~ = K~^* K~ reproduces
K~^* K~ on random vectors to about its tolerance, the solve error lies in the band of the largest
stored oracle error (the HSS tolerance sets it), one refinement step lowers it by more than an
order, and the top HSS rank grows like sqrt(N) (2x per doubling of n).
"""
import os

import numpy as np
import pytest
import torch

from fio_inputs import crandn
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _golden_path(n):
    return os.path.join(GOLDEN, "solve2d_n%d_r49.txt" % n)


def _golden(n):
    with open(_golden_path(n)) as fh:
        vals = dict(line.split(None, 1) for line in fh if not line.startswith("#"))
    return float(vals["e_direct"]), [int(x) for x in vals["ranks"].split()]


# the stored oracle runs (n = 128 takes the oracle about two hours on 8 cores)
STORED = [n for n in (64, 128) if os.path.exists(_golden_path(n))]


def _solve(n, seed_f=0, k=2):
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    bf = BF(n, 49, "elliptic2d")
    g = HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=1).factor()
    f = crandn(n * n, k, seed=seed_f)
    F = to_dev(f)
    U = bf.apply(F)
    e = float(torch.linalg.norm(fio_solve(bf, g, U) - F) / torch.linalg.norm(F))
    e1 = float(torch.linalg.norm(fio_solve(bf, g, U, refine_steps=1) - F) / torch.linalg.norm(F))
    return bf, g, e, e1


@pytest.mark.parametrize("n", STORED)
def test_solve2d_r49_matches_oracle_golden(n):
    e_or, ranks_or = _golden(n)
    _, g, e, e1 = _solve(n)
    assert e <= 2 * e_or, (e, e_or)
    assert e1 < e / 10
    ranks = g.info()["ranks"]
    assert len(ranks) == len(ranks_or)
    assert all(abs(a - b) <= max(8, b // 5) for a, b in zip(ranks[1:], ranks_or[1:])), (ranks, ranks_or)


def test_solve2d_n256_r49():
    from oracle.problem import morton_order
    nref = max(STORED)
    eref, ranks_ref = _golden(nref)
    bf, g, e, e1 = _solve(256, k=4)
    assert 0.25 * eref < e < 2 * eref, (e, eref)
    assert e1 < e / 30
    n = 256
    perm = torch.from_numpy(morton_order(n)).cuda()
    X = to_dev(crandn(n * n, 4, seed=9))                 # Morton order
    Xl = torch.empty_like(X)
    Xl[:, perm] = X
    ref = bf.adjoint(bf.apply(Xl))[:, perm]
    got = g.matvec(X)
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) < 2e-2
    grow = max(g.info()["ranks"]) / max(ranks_ref)     # ~ sqrt(N) ratio = 256 / nref
    assert 0.7 * 256 / nref < grow < 1.4 * 256 / nref, (g.info()["ranks"], ranks_ref)
