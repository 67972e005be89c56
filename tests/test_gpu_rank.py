"""Sampled FP64 entries of K~ (bf_entries), their error (bf_entry_error) and the adaptive rank
(bf_build_tol) against the oracle (oracle/rank.py).

The GPU evaluates each sampled entry of K~ along its single chain of factor blocks in FP64; the
oracle applies its FP64 BF to unit vectors.  Both are FP64 evaluations of the same factorization,
so the entries agree to rounding; the exact entries of K likewise.  The rounding is that of the FP64
phases, |Phi| <= N in 1D (n^2 in 2D), so the bound on entries of modulus ~1 is 64 eps max|Phi|, at
least 1e-10 for K~ (its r^2 products per level) and 1e-12 for K.  The sampled errors agree to 1e-6
relative and the chosen ranks exactly.
"""
import numpy as np
import pytest
import torch

from fio_inputs import bump_centers, crandn, sample_entries
from oracle.butterfly import Butterfly1D
from oracle.butterfly2d import Butterfly2D
from oracle.problem import Amplitude, Phase
from oracle.rank import choose_rank, exact_entries, sampled_bf_entries, sampled_error
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _bounds(phi_max, scale):
    """(K~ bound, K bound) on absolute entry differences for phases up to phi_max."""
    ph = 64 * EPS * phi_max
    return max(1e-10, ph) * scale, max(1e-12, ph) * scale


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES_1D = [   # (N, r, phase, amplitude)
    (1024, 4, "cabs", None), (1024, 9, "cabs", None), (1024, 16, "cabs", None),
    (1024, 8, "cabs8", "bumps"), (4096, 6, "dft", None), (65536, 16, "cabs", None),
]


@pytest.mark.parametrize("N,r,phase,amp", CASES_1D)
def test_entries_1d_match_oracle(N, r, phase, amp):
    """N = 1024: two C and two B levels; 2^16: five of each (a few distinct columns)."""
    from paper_2609_11520_b300 import BF
    ph = Phase(phase)
    oamp = gamp = None
    if amp == "bumps":
        c = bump_centers(N)
        oamp, gamp = Amplitude("bumps", c, 0.1, N=N), ("bumps", c, 0.1)
    rows, cols = sample_entries(N, 64, seed=N + r, ncols=4 if N > 4096 else None)
    got = BF(N, r, phase, amp=gamp).entries(rows, cols)
    want_t = sampled_bf_entries(Butterfly1D(ph, N, r, amp=oamp), N, rows, cols)
    want_k = exact_entries(ph, N, 1, rows, cols, oamp)
    bt, bk = _bounds(N, max(1.0, np.max(np.abs(want_k))))
    assert np.max(np.abs(got[:, 0] - want_t)) < bt
    assert np.max(np.abs(got[:, 1] - want_k)) < bk


CASES_2D = [   # (n, r1, phase, amplitude, distinct columns)
    (16, 3, "elliptic2d", None, None), (32, 5, "elliptic2d", None, None), (32, 7, "elliptic2d", None, None),
    (16, 4, "iso2d", "hankel", None), (128, 6, "elliptic2d", None, 4), (256, 3, "elliptic2d", None, 3),
]


@pytest.mark.parametrize("n,r1,phase,amp,ncols", CASES_2D)
def test_entries_2d_match_oracle(n, r1, phase, amp, ncols):
    """n <= 64 have no transfer level, 128 one B level, 256 one C and one B level."""
    from paper_2609_11520_b300 import BF
    ph = Phase(phase)
    oamp = Amplitude("hankel", phase=ph) if amp else None
    N = n * n
    rows, cols = sample_entries(N, 48, seed=n + r1, ncols=ncols)
    if amp:
        cols[cols == (n // 2) * n + n // 2] = 0      # xi = 0: infinite amplitude
    got = BF(n, r1 * r1, phase, amp=amp).entries(rows, cols)
    want_t = sampled_bf_entries(Butterfly2D(ph, n, r1, amp=oamp), N, rows, cols)
    want_k = exact_entries(ph, n, 2, rows, cols, oamp)
    bt, bk = _bounds(N, max(1.0, np.max(np.abs(want_k))))
    assert np.max(np.abs(got[:, 0] - want_t)) < bt
    assert np.max(np.abs(got[:, 1] - want_k)) < bk


def test_entry_error_matches_oracle():
    from paper_2609_11520_b300 import entry_error
    N = 1024
    ph = Phase("cabs")
    rows, cols = sample_entries(N, 500, seed=21)
    k = exact_entries(ph, N, 1, rows, cols)
    for r in (4, 8, 12):
        want = sampled_error(sampled_bf_entries(Butterfly1D(ph, N, r), N, rows, cols), k)
        assert entry_error(N, r, rows, cols, "cabs") == pytest.approx(want, rel=1e-6)
    n = 32
    ph2 = Phase("elliptic2d")
    r2, c2 = sample_entries(n * n, 300, seed=22)
    k2 = exact_entries(ph2, n, 2, r2, c2)
    for r1 in (3, 6):
        want = sampled_error(sampled_bf_entries(Butterfly2D(ph2, n, r1), n * n, r2, c2), k2)
        assert entry_error(n, r1 * r1, r2, c2, "elliptic2d") == pytest.approx(want, rel=1e-6)


def test_adaptive_rank_1d_matches_oracle_and_applies():
    """tol 1e-8 (the paper's BF tolerance) at N = 1024: the same rank as the oracle's choice; the
    built handle has that rank and matches the oracle's apply at it."""
    from paper_2609_11520_b300 import BF
    N, tol = 1024, 1e-8
    ph = Phase("cabs")
    rows, cols = sample_entries(N, 800, seed=23)
    k = exact_entries(ph, N, 1, rows, cols)
    r_or, e_or = choose_rank(lambda r: Butterfly1D(ph, N, r), list(range(4, 17, 2)), tol, N, k, rows, cols)
    bf = BF.with_tol(N, tol, rows, cols, "cabs")
    assert bf.r == r_or and bf.entry_error == pytest.approx(e_or, rel=1e-6) and bf.entry_error <= tol
    assert bf.info()["r"] == r_or
    f = crandn(N, 3, seed=24)
    assert rel(to_np(bf.apply(to_dev(f))), Butterfly1D(ph, N, r_or).apply(f)) < 1e-5


def test_adaptive_rank_2d_matches_oracle():
    """2D n = 32, tol 1e-2: the grid r1 x r1 of the oracle's choice."""
    from paper_2609_11520_b300 import BF
    n, tol = 32, 1e-2
    ph = Phase("elliptic2d")
    rows, cols = sample_entries(n * n, 600, seed=25)
    k = exact_entries(ph, n, 2, rows, cols)
    r1_or, e_or = choose_rank(lambda r1: Butterfly2D(ph, n, r1), [3, 4, 5, 6, 7], tol, n * n, k, rows, cols)
    bf = BF.with_tol(n, tol, rows, cols, "elliptic2d")
    assert bf.r == r1_or * r1_or and bf.entry_error == pytest.approx(e_or, rel=1e-6)


def test_adaptive_rank_rejections():
    from paper_2609_11520_b300 import BF, FioError, entry_error
    rows, cols = sample_entries(1024, 10, seed=26)
    with pytest.raises(FioError):
        BF.with_tol(1024, 0.0, rows, cols, "cabs")             # tol must be positive
    with pytest.raises(FioError):
        entry_error(1024, 8, rows + 1024, cols, "cabs")        # index out of range
    with pytest.raises(FioError):
        entry_error(1024, 8, rows[:0], cols[:0], "cabs")       # no sample
    with pytest.raises(FioError):
        entry_error(32, 20, rows % 1024, cols % 1024, "elliptic2d")   # 2D rank must be a square
