"""fio_pcg: CG on the approximate normal equation K~^* K~ f = K~^* u preconditioned by the
ULV factorization of G~ (Section 4.1, Eq. 4.3), against the oracle's PCG (oracle/pcg.py,
pinned against SciPy's CG and dense solves) on the same operator, HSS seeds and right-hand
sides.  The GPU iterates in complex64 (FP64 inner products), so tolerances are >= 1e-6; at
those tolerances the iteration count must match the oracle's within one, and the error
against f_true must be within 2x the oracle's at the same tolerance (plus the FP32 floor)."""
import numpy as np
import pytest
import torch

from fio_inputs import WORKLOADS, crandn
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def case4096():
    from oracle.problem import Phase
    from oracle.solver import FIOSolver
    from paper_2609_11520_b300 import BF, HSS
    n, leaf, p, tol, seed = 4096, 128, 10, 1e-3, 1
    S = FIOSolver(Phase("cabs"), n, 16, leaf, p, tol, seed)
    bf = BF(n, 16)
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed).factor()
    f = crandn(n, 3, seed=0)
    u = S.bf.apply(f)
    return S, bf, g, f, u


@pytest.mark.parametrize("tol", [1e-5, 1e-6])
def test_pcg_matches_oracle(case4096, tol):
    from oracle.pcg import fio_pcg as oracle_pcg
    from paper_2609_11520_b300 import fio_pcg
    S, bf, g, f, u = case4096
    xo, ito, rro = oracle_pcg(S, u, tol=tol)
    F, it, rr = fio_pcg(bf, g, to_dev(u), tol=tol, maxit=30)
    assert abs(it - int(ito.max())) <= 1, (it, ito)
    assert max(rr) <= tol, rr
    e_o, e_g = rel(xo, f), rel(to_np(F), f)
    assert e_g <= 2 * e_o + 2e-6, (e_g, e_o)


def test_pcg_improves_on_direct_solve(case4096):
    """PCG converges past the direct solve's HSS-tolerance error (Tables 5.1 vs 5.2)."""
    from paper_2609_11520_b300 import fio_pcg, fio_solve
    S, bf, g, f, u = case4096
    U = to_dev(u)
    e_direct = rel(to_np(fio_solve(bf, g, U)), f)
    F, it, _ = fio_pcg(bf, g, U, tol=1e-6, maxit=30)
    assert rel(to_np(F), f) < e_direct / 10, (rel(to_np(F), f), e_direct)
    assert it <= 5


def test_pcg_full_size():
    """N = 2^16 (the served operator): a few iterations to 1e-5 and an error well below the direct
    solve's; the unpreconditioned count at the same tolerance is several times larger."""
    from paper_2609_11520_b300 import BF, HSS, fio_pcg, fio_solve
    w = WORKLOADS["large1d"]
    bf = BF(w["n"], w["r"], w["phase"], w["s"])
    g = HSS.from_samples(bf=bf, leaf=w["leaf"], oversample=w["p"], tol=w["tol"], seed=w["seed_omega"]).factor()
    f = crandn(w["n"], 4, seed=w["seed_f"])
    U = bf.apply(to_dev(f))
    e_direct = rel(to_np(fio_solve(bf, g, U)), f)
    F, it, rr = fio_pcg(bf, g, U, tol=1e-5, maxit=30)
    e = rel(to_np(F), f)
    assert it <= 4 and max(rr) <= 1e-5, (it, rr)
    assert e < e_direct / 5, (e, e_direct)


def test_pcg_2d():
    """2D (elliptic phase, n = 32, leaf 256): the iteration runs in the HSS's quadtree order and
    returns lexicographic vectors."""
    from paper_2609_11520_b300 import BF, HSS, fio_pcg, fio_solve
    n = 32
    bf = BF(n, 25, "elliptic2d")
    g = HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=1).factor()
    f = crandn(n * n, 2, seed=0)
    U = bf.apply(to_dev(f))
    e_direct = rel(to_np(fio_solve(bf, g, U)), f)
    F, it, rr = fio_pcg(bf, g, U, tol=1e-5, maxit=40)
    assert max(rr) <= 1e-5 and rel(to_np(F), f) < e_direct / 5, (it, rr, rel(to_np(F), f), e_direct)


def test_pcg_zero_column_and_errors(case4096):
    from paper_2609_11520_b300 import BF, HSS, FioError, fio_pcg
    S, bf, g, f, u = case4096
    U = to_dev(u)
    U[1].zero_()
    F, it, rr = fio_pcg(bf, g, U, tol=1e-5)
    assert rr[1] == 0.0 and float(torch.linalg.norm(F[1])) == 0.0
    assert it >= 1
    g2 = HSS.from_samples(bf=bf, leaf=128, oversample=10, tol=1e-3, seed=5)   # not factored
    with pytest.raises(FioError):
        fio_pcg(bf, g2, U)
