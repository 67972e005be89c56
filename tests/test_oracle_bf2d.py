"""Pins of the 2D oracle (quadtree BF, Morton order, 2D solver) against the
mathematics: a separable phase reduces the 2D BF to a Kronecker product of the
pinned 1D BF, brute force against dense K, adjoint identity, the DFT closed
form through numpy's FFT, tensor interpolation invariants, and a dense solve."""
import numpy as np
import pytest

from fio_inputs import crandn
from oracle.butterfly import Butterfly1D
from oracle.butterfly2d import Butterfly2D, _tensor_lagrange
from oracle.problem import Phase, dense_K2, morton_order
from oracle.solver import FIOSolver2D, rel_err


@pytest.mark.parametrize("n,levels", [(16, None), (16, (2, 3, 1)), (32, (2, 4, 1)), (32, (1, 4, 0))])
def test_dft_2d_is_kron_of_1d(n, levels):
    """Phi = x.xi: every 2D factor is the Kronecker product of the 1D factors on the same
    levels, so K~_2 = K~_1 (x) K~_1 (lexicographic order) to rounding.  The level overrides
    put C and B transfer levels into small sizes (every factor kind is exercised)."""
    b2 = Butterfly2D(Phase("dft", d=2), n, 5, levels=levels)
    b1 = Butterfly1D(Phase("dft"), n, 5, levels=levels)
    D1 = b1.dense()
    f = crandn(n * n, 3, seed=n)
    F = f.reshape(n, n, 3)
    ref = np.einsum("ia,abk,jb->ijk", D1, F, D1).reshape(n * n, 3)
    assert rel_err(b2.apply(f), ref) < 1e-12
    refa = np.einsum("ai,abk,bj->ijk", D1.conj(), F, D1.conj()).reshape(n * n, 3)
    assert rel_err(b2.adjoint(f), refa) < 1e-12


def test_dense_2d_equals_kron_full():
    b2 = Butterfly2D(Phase("dft", d=2), 16, 5, levels=(2, 3, 1))
    b1 = Butterfly1D(Phase("dft"), 16, 5, levels=(2, 3, 1))
    D1 = b1.dense()
    assert rel_err(b2.dense(), np.kron(D1, D1)) < 1e-12


@pytest.mark.parametrize("n", [32, 64])
def test_elliptic_brute_force(n):
    """e_cBF against dense K falls with the interpolation rank (r1 = 5 -> 7)."""
    K = dense_K2(Phase("elliptic2d"), n)
    f = crandn(n * n, 2, seed=1)
    ref = K @ f
    e5 = rel_err(Butterfly2D(Phase("elliptic2d"), n, 5).apply(f), ref)
    e7 = rel_err(Butterfly2D(Phase("elliptic2d"), n, 7).apply(f), ref)
    assert e5 < 1e-2 and e7 < 1e-3 and e7 < e5 / 10, (e5, e7)


def test_elliptic_levels_brute_force():
    """With transfer levels forced in (h, sU, sV) = (2, 4, 1) the BF still tracks dense K."""
    n = 32
    K = dense_K2(Phase("elliptic2d"), n)
    f = crandn(n * n, 2, seed=2)
    e = rel_err(Butterfly2D(Phase("elliptic2d"), n, 7, levels=(2, 4, 1)).apply(f), K @ f)
    assert e < 5e-3, e


def test_adjoint_identity():
    b = Butterfly2D(Phase("elliptic2d"), 64, 5)
    x = crandn(64 * 64, 1, seed=3)[:, 0]
    y = crandn(64 * 64, 1, seed=4)[:, 0]
    lhs = np.vdot(y, b.apply(x))
    rhs = np.vdot(b.adjoint(y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_dft_closed_form_fft():
    """K f = (-1)^(i1+i2) n^2 ifft2(F) for Phi = x.xi (x = i/n, xi = j - n/2), within the
    r1 = 5 interpolation error of the BF (the 1D r = 5 BF's error, squared into 2D)."""
    n = 64
    b = Butterfly2D(Phase("dft", d=2), n, 5)
    f = crandn(n * n, 1, seed=5)[:, 0]
    i1, i2 = np.divmod(np.arange(n * n), n)
    ref = ((-1.0) ** (i1 + i2)) * (n * n * np.fft.ifft2(f.reshape(n, n))).reshape(-1)
    e1 = rel_err(Butterfly1D(Phase("dft"), n, 5).apply(crandn(n, 1, seed=6)[:, 0]),
                 ((-1.0) ** np.arange(n)) * n * np.fft.ifft(crandn(n, 1, seed=6)[:, 0]))
    assert rel_err(b.apply(f), ref) < 3 * e1 + 1e-12


def test_tensor_lagrange_invariants():
    nodes = np.cos((2 * np.arange(5) + 1) * np.pi / 10)
    p = np.random.default_rng(0).uniform(-1, 1, size=(40, 2))
    Lt = _tensor_lagrange(nodes, nodes, p[:, 0], p[:, 1])          # (40, 25)
    assert np.allclose(Lt.sum(axis=1), 1.0, atol=1e-12)
    g1 = np.repeat(nodes, 5)
    g2 = np.tile(nodes, 5)
    for a in range(5):
        for c in range(5):
            assert np.allclose(Lt @ (g1 ** a * g2 ** c), p[:, 0] ** a * p[:, 1] ** c, atol=1e-11)


def test_morton_order_boxes_contiguous():
    n = 32
    perm = morton_order(n)
    assert np.array_equal(np.sort(perm), np.arange(n * n))
    j1, j2 = np.divmod(perm, n)
    for lev in range(1, 6):
        w = n >> lev
        box = (j1 // w) * (1 << lev) + (j2 // w)
        size = w * w
        blocks = box.reshape(-1, size)
        assert np.all(blocks == blocks[:, :1])                    # each run of w^2 positions is one box
        assert len(np.unique(blocks[:, 0])) == 4 ** lev


def test_solver2d_against_dense_lu():
    """n = 16 (N = 256), leaf 16: f^ = P^T F~ P K~^* u tracks f_true and the dense LU solve of K."""
    n = 16
    S = FIOSolver2D(Phase("elliptic2d"), n, 5, 16, 10, 1e-6, 1)
    f = crandn(n * n, 2, seed=7)
    K = dense_K2(Phase("elliptic2d"), n)
    u = K @ f
    f_lu = np.linalg.solve(K, u)
    fh = S.solve(u)
    assert rel_err(f_lu, f) < 1e-8
    eb = rel_err(S.bf.apply(f), u)                 # BF error of this size
    assert rel_err(fh, f) < 50 * eb + 1e-6, (rel_err(fh, f), eb)
