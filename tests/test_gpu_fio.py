"""Full-size online stage (N = 2^16, complex64): properties that hold at any size.

The oracle's HSS construction at N = 2^16 would take hours, so here the checks
are: the solve inverts the constructed G~ (residual through hss_matvec), the
error against f_true for u = K~ f_true stays in the tolerance band of the
HSS construction, one RHS alone equals the same RHS inside a 64-wide block,
and refinement does not increase the error.
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
