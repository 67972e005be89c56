"""Pins of the oracle's phase functions and dense K against values worked out by hand.

Every other oracle test builds K and K~ from the same Phase object, so a
misread constant there (/8 for /16, sin(pi x) for sin(2 pi x), c1 and c2
exchanged, a dropped |xi|) would pass them all.  The values below follow the
phase formulas of Section 5 directly:

  1D (Section 5.1 form, workload constants):  Phi = x xi + c(x) |xi|,
      c(x) = (2 + s sin 2 pi x) / 16
  2D (Section 5.2):  Phi = x . xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2),
      c1 = (2 + sin 2 pi x1 sin 2 pi x2) / 16,  c2 = (2 + cos 2 pi x1 cos 2 pi x2) / 16

with the grids of Eq. 1.1 (x_i = i/n, xi_j = j - n/2, lexicographic with the
first coordinate slow in 2D).
"""
import numpy as np
import pytest

from oracle.problem import K2_rows, K_rows, Phase, dense_K, dense_K2


@pytest.mark.parametrize("x,xi,s,want", [
    (0.25, -8.0, 1.0, -0.5),      # c = 3/16: -2 + 3/2
    (0.0, 5.0, 1.0, 0.625),       # c = 1/8: 5/8
    (0.75, 4.0, 0.5, 3.375),      # c = (2 - 1/2)/16 = 3/32: 3 + 3/8
    (0.5, -16.0, 1.0, -6.0),      # c = 1/8: -8 + 2
    (0.125, 0.0, 1.0, 0.0),       # |xi| = 0
])
def test_cabs_values(x, xi, s, want):
    assert Phase("cabs", s=s)(np.float64(x), np.float64(xi)) == pytest.approx(want, abs=1e-14)


def test_cabs_c_is_even_in_xi_and_periodic_in_x():
    ph = Phase("cabs")
    x = np.linspace(0, 1, 17)
    xi = 7.0
    # Phi(x, xi) - Phi(x, -xi) = 2 x xi (the |xi| term cancels)
    assert np.allclose(ph(x, xi) - ph(x, -xi), 2 * x * xi, atol=1e-13)
    # c(x + 1) = c(x)
    assert np.allclose(ph.c(x + 1.0), ph.c(x), atol=1e-14)
    # c ranges over [1/16, 3/16] with s = 1
    xs = np.linspace(0, 1, 4001)
    assert ph.c(xs).min() == pytest.approx(1 / 16, abs=1e-7) and ph.c(xs).max() == pytest.approx(3 / 16, abs=1e-7)


@pytest.mark.parametrize("x,xi,want", [
    ((0.25, 0.25), (16.0, 32.0), 17.0),                 # c1 = 3/16, c2 = 1/8: 12 + sqrt(9 + 16)
    ((0.0, 0.0), (-24.0, 16.0), 3.0 * np.sqrt(2.0)),    # c1 = 1/8, c2 = 3/16: sqrt(9 + 9)
    ((0.5, 0.0), (-8.0, 48.0), -4.0 + np.sqrt(10.0)),   # c1 = 1/8, c2 = 1/16: -4 + sqrt(1 + 9)
    ((0.25, 0.75), (8.0, 0.0), 2.5),                   # c1 = (2 - 1)/16: 2 + 1/2
])
def test_elliptic_values(x, xi, want):
    ph = Phase("elliptic2d")
    got = ph(np.array(x, dtype=np.float64), np.array(xi, dtype=np.float64))
    assert float(got) == pytest.approx(want, abs=1e-13)


def test_elliptic_reduces_to_dft_plus_norm_on_axes():
    """On xi = (k, 0): Phi = x1 k + c1(x) |k|; on xi = (0, k): Phi = x2 k + c2(x) |k|."""
    ph = Phase("elliptic2d")
    rng = np.random.default_rng(0)
    x = rng.random((20, 2))
    k = rng.integers(-64, 64, 20).astype(np.float64)
    c1 = (2 + np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1])) / 16
    c2 = (2 + np.cos(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])) / 16
    z = np.zeros_like(k)
    assert np.allclose(ph(x, np.stack([k, z], -1)), x[:, 0] * k + c1 * np.abs(k), atol=1e-12)
    assert np.allclose(ph(x, np.stack([z, k], -1)), x[:, 1] * k + c2 * np.abs(k), atol=1e-12)


def test_dense_K_entries():
    """K_ij = exp(2 pi i Phi(i/n, j - n/2)) at hand-picked entries."""
    K = dense_K(Phase("cabs"), 16)
    assert K[4, 0] == pytest.approx(-1.0, abs=1e-13)                # x = 1/4, xi = -8: Phi = -1/2
    assert K[0, 13] == pytest.approx(np.exp(2j * np.pi * 0.625), abs=1e-13)   # x = 0, xi = 5
    # the DFT: K_ij = exp(2 pi i (i/n)(j - n/2))
    Kd = dense_K(Phase("dft"), 8)
    assert Kd[3, 1] == pytest.approx(np.exp(2j * np.pi * 3 / 8 * -3), abs=1e-13)
    R = K_rows(Phase("cabs", s=0.5), 64, [48])                      # x = 3/4
    assert R[0, 36] == pytest.approx(np.exp(2j * np.pi * 3.375), abs=1e-13)   # xi = 4


def test_dense_K2_entries():
    """2D, lexicographic i = i1 n + i2, j = j1 n + j2 with xi = (j1 - n/2, j2 - n/2)."""
    K = dense_K2(Phase("elliptic2d"), 16)
    # x = (4/16, 4/16): c1 = 3/16; xi = (-8, 0): Phi = -2 + 3/2 = -1/2
    assert K[4 * 16 + 4, 0 * 16 + 8] == pytest.approx(-1.0, abs=1e-13)
    # x = (0, 0): c1 = 1/8, c2 = 3/16; xi = (-8, -8) -> Phi = sqrt(1 + 9/4)
    assert K[0, 0] == pytest.approx(np.exp(2j * np.pi * np.sqrt(1.0 + 2.25)), abs=1e-13)
    # n = 64: x = (1/4, 1/4), xi = (8, 0): Phi = 2 + 3/2 = 7/2
    R = K2_rows(Phase("elliptic2d"), 64, [16 * 64 + 16])
    assert R[0, 40 * 64 + 32] == pytest.approx(-1.0, abs=1e-12)
    # the first coordinate is the slow index: x = (0, 1/2) differs from x = (1/2, 0)
    R2 = K2_rows(Phase("elliptic2d"), 64, [32, 32 * 64])
    j = (32 - 8) * 64 + (32 + 48 - 32)   # xi = (-8, 16)
    # x = (0, 1/2): c1 = 1/8, c2 = (2 - 1)/16; Phi = 8 + sqrt(1 + 1)
    assert R2[0, j] == pytest.approx(np.exp(2j * np.pi * (8.0 + np.sqrt(2.0))), abs=1e-12)
    # x = (1/2, 0): c1 = 1/8, c2 = 1/16; Phi = -4 + sqrt(1 + 1)
    assert R2[1, j] == pytest.approx(np.exp(2j * np.pi * (-4.0 + np.sqrt(2.0))), abs=1e-12)
