"""Adaptive butterfly rank (Section 5: the BF is built to a prescribed accuracy, 1e-8 in the
experiments, instead of a fixed rank).

Test infrastructure only: nothing on the product path imports this module.

Error measure on sampled index pairs (i_e, j_e):
    e = sqrt( sum_e |K~(i_e, j_e) - K(i_e, j_e)|^2 / sum_e |K(i_e, j_e)|^2 ),
the sampled estimate of ||K~ - K||_F / ||K||_F.  For a random vector f with independent
standard entries, E ||(K~ - K) f||^2 = ||K~ - K||_F^2 over the rows, so this is also the estimate
of the relative sampled-row error e_cBF that Section 5 reports.  The adaptive rank is the
smallest candidate rank whose e is at most the tolerance.

K~ entries come from the oracle's own apply of unit vectors (one apply per distinct sampled
column); K entries from Eq. 1.2.  A sample where the amplitude is infinite (the Hankel amplitude
at xi = 0) contributes to neither sum.
"""
import numpy as np

from .problem import freq_grid_1d, freq_grid_2d, space_grid_1d, space_grid_2d


def sampled_bf_entries(bf, N, rows, cols):
    """K~(rows[e], cols[e]) through bf.apply on the unit vectors of the distinct columns."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    uniq, inv = np.unique(cols, return_inverse=True)
    E = np.zeros((N, uniq.size), dtype=np.complex128)
    E[uniq, np.arange(uniq.size)] = 1.0
    Y = bf.apply(E)
    return Y[rows, inv]


def exact_entries(phase, n, d, rows, cols, amp=None):
    """K(rows[e], cols[e]) = a(x, xi) e^{2 pi i Phi(x, xi)} (Eq. 1.2); n points per dimension,
    lexicographic indices in 2D."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if d == 1:
        x, xi = space_grid_1d(n)[rows], freq_grid_1d(n)[cols]
    else:
        x, xi = space_grid_2d(n)[rows], freq_grid_2d(n)[cols]
    a = 1.0 if amp is None else amp(x, xi)
    return a * np.exp(2j * np.pi * phase(x, xi))


def sampled_error(kt, k):
    """sqrt(sum |kt - k|^2 / sum |k|^2) over the samples where k is finite."""
    ok = np.isfinite(k)
    return float(np.sqrt(np.sum(np.abs(kt[ok] - k[ok]) ** 2) / np.sum(np.abs(k[ok]) ** 2)))


def choose_rank(build, candidates, tol, N, k_exact, rows, cols):
    """Smallest r in `candidates` (ascending) with sampled_error <= tol, and its error; the
    largest candidate and its error when none reaches tol.  build(r) returns a BF with .apply."""
    r, e = None, None
    for r in candidates:
        e = sampled_error(sampled_bf_entries(build(r), N, rows, cols), k_exact)
        if e <= tol:
            break
    return r, e
