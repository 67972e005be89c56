"""Full-size online stage (N = 2^16, complex64).

Against the oracle: the error against f_true is at most 2x the oracle's stored
e_direct for the same operator, seeds and f_true (the oracle's construction
at this size takes about 20 minutes on 8 cores, so its value is stored).
Properties that hold at any size: the solve inverts the constructed G~
(residual through hss_matvec), one RHS alone equals the same RHS inside a
64-wide block, and refinement does not increase the error.
"""
import numpy as np
import pytest
import torch

from fio_inputs import WORKLOADS, crandn
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, HSS
    w = WORKLOADS["large1d"]
    bf = BF(w["n"], w["r"], w["phase"], w["s"])
    g = HSS.from_samples(bf=bf, leaf=w["leaf"], oversample=w["p"], tol=w["tol"], seed=w["seed_omega"])
    g.factor()
    return w, bf, g


def test_large_solve_against_stored_oracle(large):
    """N = 2^16: error against f_true at most 2x the oracle's e_direct for the same f_true
    (tests/golden/solve1d_N65536.txt, written by make_solve_golden.py from oracle/ only;
    the oracle's HSS ranks are those of the GPU construction)."""
    import os
    from paper_2609_11520_b300 import fio_solve
    w, bf, g = large
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "solve1d_N65536.txt")
    vals = dict(line.split(maxsplit=1) for line in open(path) if not line.startswith("#"))
    e_oracle = float(vals["e_direct"])
    assert g.info()["ranks"] == [int(v) for v in vals["ranks"].split()]
    f = crandn(w["n"], 2, seed=3)
    F = to_dev(f)
    U = bf.apply(F)                                   # u = K~ f_true (Section 5)
    e = rel(to_np(fio_solve(bf, g, U)), f)
    assert e <= 2 * e_oracle, (e, e_oracle)


def test_large_solve(large):
    from paper_2609_11520_b300 import fio_solve
    w, bf, g = large
    n = w["n"]
    f = crandn(n, 64, seed=w["seed_f"])
    F = to_dev(f)
    U = bf.apply(F)
    out = fio_solve(bf, g, U)
    e = rel(to_np(out), f)
    assert 1e-7 < e < 5e-3, e
    # G~ f^ = K~^* u
    rhs = bf.adjoint(U)
    assert rel(to_np(g.matvec(out)), to_np(rhs)) < 1e-4
    # one column alone equals the same column inside the block
    one = fio_solve(bf, g, U[5:6].clone())
    assert rel(to_np(one)[:, 0], to_np(out)[:, 5]) < 1e-6
    # refinement
    out2 = fio_solve(bf, g, U, refine_steps=1)
    assert rel(to_np(out2), f) <= e * 1.01
