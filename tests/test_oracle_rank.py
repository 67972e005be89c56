"""Oracle of the adaptive BF rank (oracle/rank.py) against what fixes it independently: the dense
Frobenius error of the whole matrix (every entry sampled), Eq. 1.2 entry by entry through the dense
K builders, the decrease of the Chebyshev interpolation error with the rank, and the statistics of
a random sample."""
import numpy as np
import pytest

from fio_inputs import bump_centers, sample_entries
from oracle.butterfly import Butterfly1D
from oracle.butterfly2d import Butterfly2D
from oracle.problem import Amplitude, Phase, dense_K, dense_K2
from oracle.rank import choose_rank, exact_entries, sampled_bf_entries, sampled_error


def _all_pairs(N):
    i, j = np.divmod(np.arange(N * N), N)
    return i, j


@pytest.mark.parametrize("r", [3, 6])
def test_full_sample_is_the_dense_frobenius_error_1d(r):
    n = 64
    ph = Phase("cabs")
    bf = Butterfly1D(ph, n, r)
    rows, cols = _all_pairs(n)
    e = sampled_error(sampled_bf_entries(bf, n, rows, cols), exact_entries(ph, n, 1, rows, cols))
    Kt, K = bf.dense(), dense_K(ph, n)
    assert e == pytest.approx(np.linalg.norm(Kt - K) / np.linalg.norm(K), rel=1e-12)


def test_full_sample_is_the_dense_frobenius_error_2d():
    n = 8
    ph = Phase("elliptic2d")
    bf = Butterfly2D(ph, n, 3)
    rows, cols = _all_pairs(n * n)
    e = sampled_error(sampled_bf_entries(bf, n * n, rows, cols), exact_entries(ph, n, 2, rows, cols))
    Kt, K = bf.dense(), dense_K2(ph, n)
    assert e == pytest.approx(np.linalg.norm(Kt - K) / np.linalg.norm(K), rel=1e-12)


def test_exact_entries_match_the_dense_builders():
    n = 32
    rows, cols = sample_entries(n, 50, seed=1)
    ph = Phase("cabs8")
    amp = Amplitude("bumps", bump_centers(n), 0.1, N=n)
    assert np.allclose(exact_entries(ph, n, 1, rows, cols, amp), dense_K(ph, n, amp)[rows, cols], atol=1e-14)
    ph2 = Phase("iso2d")
    amp2 = Amplitude("hankel", phase=ph2)
    r2, c2 = sample_entries(n * n, 50, seed=2)
    c2[c2 == (n // 2) * n + n // 2] = 0          # keep xi = 0 out (infinite amplitude)
    assert np.allclose(exact_entries(ph2, n, 2, r2, c2, amp2), dense_K2(ph2, n, amp2)[r2, c2], atol=1e-12)


def test_error_falls_with_rank_and_choice_is_the_first_below_tol():
    n = 256
    ph = Phase("cabs")
    rows, cols = sample_entries(n, 400, seed=3)
    k = exact_entries(ph, n, 1, rows, cols)
    errs = [sampled_error(sampled_bf_entries(Butterfly1D(ph, n, r), n, rows, cols), k) for r in range(4, 17, 2)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs       # Chebyshev interpolation of an analytic kernel
    assert errs[0] > 1e-3 and errs[-1] < 1e-10, errs
    tol = np.sqrt(errs[2] * errs[3])                               # strictly between r = 8 and r = 10
    r, e = choose_rank(lambda rr: Butterfly1D(ph, n, rr), list(range(4, 17, 2)), tol, n, k, rows, cols)
    assert r == 10 and e == pytest.approx(errs[3])
    r, e = choose_rank(lambda rr: Butterfly1D(ph, n, rr), [4, 6], 1e-30, n, k, rows, cols)
    assert r == 6 and e == pytest.approx(errs[1])                  # none reaches tol: the largest


def test_random_sample_estimates_the_frobenius_error():
    n = 512
    ph = Phase("cabs")
    bf = Butterfly1D(ph, n, 6)
    full = np.linalg.norm(bf.dense() - dense_K(ph, n)) / np.sqrt(n * n)
    rows, cols = sample_entries(n, 4000, seed=4)
    e = sampled_error(sampled_bf_entries(bf, n, rows, cols), exact_entries(ph, n, 1, rows, cols))
    assert 0.8 < e / full < 1.25
