"""Pins for the oracle's butterfly factorization (CPU only).

Each check is anchored in something other than the oracle itself: the DFT
closed form evaluated by numpy's FFT, dense K from Eq. 1.2, the adjoint
identity, Chebyshev/Lagrange invariants, and the factor counts of Section 5.2.
"""
import numpy as np
import pytest

from oracle.butterfly import Butterfly1D, cheb_nodes, lagrange
from oracle.problem import K_rows, Phase, dense_K

RNG = np.random.default_rng(1234)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ---- P4: interpolation invariants -----------------------------------------

@pytest.mark.parametrize("r", [4, 9, 16, 25])
def test_chebyshev_nodes_are_roots_of_T_r(r):
    t = cheb_nodes(r)
    assert np.max(np.abs(np.cos(r * np.arccos(t)))) < 1e-13
    assert len(np.unique(np.round(t, 14))) == r


@pytest.mark.parametrize("r", [5, 16])
def test_lagrange_partition_of_unity_and_polynomial_reproduction(r):
    lo, w = 0.37, 1.0 / 64
    nodes = lo + w / 2 * (1 + cheb_nodes(r))
    x = lo + w * RNG.random(50)
    P = lagrange(nodes, x)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    # exact reproduction of every polynomial of degree < r (in box coordinates)
    for deg in range(r):
        f = lambda s: ((s - lo) / w - 0.3) ** deg
        assert np.allclose(P @ f(nodes), f(x), atol=1e-10)
    # Kronecker property at the nodes
    assert np.allclose(lagrange(nodes, nodes), np.eye(r), atol=1e-12)


# ---- levels of Section 5.2 ----------------------------------------------------

@pytest.mark.parametrize("L,nB", [(6, 0), (8, 1), (10, 2), (12, 3), (16, 5)])
def test_practical_top_level_even_L(L, nB):
    """Section 5.2: outermost factors at max(L-3, h); #B = #C = max(L/2 - 3, 0)."""
    bf = Butterfly1D(Phase("cabs"), 2 ** L, 4)
    assert bf.sU == max(L - 3, L // 2)
    assert bf.sU - bf.h == nB
    assert bf.h - bf.sV == nB


@pytest.mark.parametrize("L", [5, 7, 9, 13, 17])
def test_practical_top_level_odd_L(L):
    """Odd L (the paper assumes L even): h = floor(L/2), pairs stay complementary."""
    bf = Butterfly1D(Phase("cabs"), 2 ** L, 4)
    assert bf.sV <= bf.h <= bf.sU
    assert bf.sU == max(L - 3, L // 2) and bf.sV == min(3, L // 2)


# ---- P1: DFT closed form --------------------------------------------------------

def dft_apply(f):
    """(K f)_i = sum_j e^{2 pi i x_i xi_j} f_j = n * ifft(ifftshift(f))_i."""
    n = f.shape[0]
    return n * np.fft.ifft(np.fft.ifftshift(f, axes=0), axis=0)


def dft_adjoint(g):
    """(K^* g)_j = sum_i e^{-2 pi i x_i xi_j} g_i = fftshift(fft(g))_j."""
    return np.fft.fftshift(np.fft.fft(g, axis=0), axes=0)


@pytest.mark.parametrize("n", [64, 1024, 4096])
def test_dft_closed_form(n):
    bf = Butterfly1D(Phase("dft"), n, 16)
    f = crandn(n, 2)
    y = bf.apply(f)
    assert np.linalg.norm(y - dft_apply(f)) / np.linalg.norm(y) < 1e-12
    g = crandn(n, 2)
    assert np.linalg.norm(bf.adjoint(g) - dft_adjoint(g)) / np.linalg.norm(g) / np.sqrt(n) < 1e-12


# ---- P2: brute force against dense K ----------------------------------------------

@pytest.mark.parametrize("kind", ["dft", "cabs"])
@pytest.mark.parametrize("n", [16, 64, 256, 1024])
def test_bf_matches_dense_K(kind, n):
    ph = Phase(kind)
    K = dense_K(ph, n)
    Kt = Butterfly1D(ph, n, 16).dense()
    assert np.linalg.norm(Kt - K) / np.linalg.norm(K) < 1e-10


def test_bf_error_decreases_with_rank():
    ph = Phase("cabs")
    n = 256
    K = dense_K(ph, n)
    errs = [np.linalg.norm(Butterfly1D(ph, n, r).dense() - K) / np.linalg.norm(K) for r in (6, 10, 14)]
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    assert errs[0] > 1e-6  # low rank really is approximate


def test_bf_sampled_rows_at_4096():
    """e_cBF estimated from sampled rows of K (Section 5)."""
    n = 4096
    ph = Phase("cabs", s=0.7)
    bf = Butterfly1D(ph, n, 16)
    f = crandn(n)
    rows = RNG.choice(n, 64, replace=False)
    ref = K_rows(ph, n, rows) @ f
    assert np.linalg.norm(bf.apply(f)[rows] - ref) / np.linalg.norm(ref) < 1e-10


# ---- P3: adjoint identity ------------------------------------------------------------

@pytest.mark.parametrize("n", [64, 512, 2048])
def test_adjoint_identity(n):
    bf = Butterfly1D(Phase("cabs"), n, 16)
    x, y = crandn(n, 3), crandn(n, 3)
    lhs = np.vdot(y, bf.apply(x))
    rhs = np.vdot(bf.adjoint(y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_column_blocks_are_independent():
    bf = Butterfly1D(Phase("cabs"), 256, 16)
    X = crandn(256, 5)
    Y = bf.apply(X)
    for j in range(5):
        assert np.allclose(Y[:, j], bf.apply(X[:, j]), rtol=0, atol=1e-12 * np.abs(Y).max())
