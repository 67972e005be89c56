"""Pins of the oracle's preconditioned CG (Section 4.1, Eq. 4.3) against facts fixed
outside it: the dense solve, SciPy's CG (a library routine) on the same system,
preconditioner and stopping rule, finite termination, the exact preconditioner,
and the paper's observation (Section 5.1, Table 5.2) that the ULV factorization
of the HSS approximation brings CG on the approximate normal equation down to a
handful of iterations at a 1e-12 relative residual."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from fio_inputs import crandn
from oracle.pcg import fio_pcg, pcg


def _hpd(n, cond, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    d = np.geomspace(1.0, cond, n)
    return (q * d) @ q.conj().T


def test_pcg_matches_dense_solve():
    A = _hpd(60, 1e3, 0)
    b = crandn(60, 3, seed=1)
    x, it, rr = pcg(lambda v: A @ v, b, tol=1e-12, maxit=1000)
    assert np.all(rr <= 1e-12)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(np.linalg.solve(A, b)) < 1e-9


@pytest.mark.parametrize("precond", [False, True])
def test_pcg_iterations_match_scipy_cg(precond):
    A = _hpd(80, 1e4, 2)
    P = _hpd(80, 10.0, 3)
    Minv = np.linalg.inv(A + 0.3 * P)          # an approximate inverse
    b = crandn(80, 1, seed=4)[:, 0]
    counts = []
    x_ref, info = spla.cg(A, b, rtol=1e-10, atol=0.0, maxiter=2000, M=(Minv if precond else None),
                          callback=lambda xk: counts.append(1))
    assert info == 0
    x, it, rr = pcg(lambda v: A @ v, b, (lambda v: Minv @ v) if precond else None, tol=1e-10, maxit=2000)
    assert abs(int(it[0]) - len(counts)) <= 1, (it, len(counts))
    assert np.linalg.norm(x[:, 0] - x_ref) / np.linalg.norm(x_ref) < 1e-8


def test_pcg_finite_termination_and_exact_preconditioner():
    A = _hpd(8, 50.0, 5)
    b = crandn(8, 2, seed=6)
    _, it, rr = pcg(lambda v: A @ v, b, tol=1e-10, maxit=100)
    assert np.all(it <= 9) and np.all(rr <= 1e-10)       # n steps in exact arithmetic
    Ainv = np.linalg.inv(A)
    _, it1, _ = pcg(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-10, maxit=100)
    assert np.all(it1 == 1)


def test_fio_pcg_few_iterations():
    """N = 1024, HSS tol 1e-3 (the paper's setting): preconditioned CG reaches the paper's 1e-12
    relative residual in a handful of iterations (4-5 in Table 5.2), several times fewer than
    plain CG, and recovers f_true of u = K~ f_true."""
    from oracle.problem import Phase
    from oracle.solver import FIOSolver
    S = FIOSolver(Phase("cabs"), 1024, 16, 64, 10, 1e-3, 1)
    f = crandn(1024, 2, seed=0)
    u = S.bf.apply(f)
    x, it, rr = fio_pcg(S, u, tol=1e-12)
    assert np.all(rr <= 1e-12)
    assert np.all((3 <= it) & (it <= 7)), it
    assert np.linalg.norm(x - f) / np.linalg.norm(f) < 1e-9
    _, it0, _ = fio_pcg(S, u, tol=1e-12, precondition=False)
    assert np.all(it0 >= 3 * it), (it0, it)
