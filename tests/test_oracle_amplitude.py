"""Pins of the variable-amplitude operators (Section 5.1: Gaussian bumps with the /8 phase;
Section 5.3: the Hankel amplitude with the isotropic 2D phase), and of the BF with an
amplitude, which enters only the middle factor M = a(z, gamma) e^{2 pi i Phi(z, gamma)}
(Section 2.2): hand-worked values, SciPy's J0/Y0 (library routines other than the Hankel
function the oracle calls), the kernel identity a e^{2 pi i Phi} = H0(2 pi phi) e^{2 pi i x.xi},
brute force against dense K, and the adjoint identity."""
import numpy as np
import pytest
from scipy.special import j0, y0

from fio_inputs import bump_centers, crandn
from oracle.butterfly import Butterfly1D
from oracle.butterfly2d import Butterfly2D
from oracle.problem import Amplitude, Phase, dense_K, dense_K2, freq_grid_2d, space_grid_2d


def test_phase_values_of_the_variable_amplitude_examples():
    # 'cabs8' (Section 5.1): c(1/4) = (2 + 1)/8; Phi(1/4, -8) = -2 + 3 = 1
    assert Phase("cabs8")(np.float64(0.25), np.float64(-8.0)) == pytest.approx(1.0, abs=1e-14)
    # 'iso2d' (Section 5.3): c = (3 + 1)/8 at x = (1/4, 1/4); xi = (3, 4): 3/4 + 1 + (1/2) 5
    ph = Phase("iso2d")
    assert float(ph(np.array([0.25, 0.25]), np.array([3.0, 4.0]))) == pytest.approx(4.25, abs=1e-13)
    assert float(ph.nonlinear(np.array([0.25, 0.75]), np.array([0.0, -8.0]))) == pytest.approx(2.0 / 8 * 8, abs=1e-13)


def test_bump_amplitude_values():
    a = Amplitude("bumps", centers=[[0.5, 100.0], [0.2, -300.0]], sigma2=0.1, N=1000.0)
    # at the first centre: 1 + exp(-((0.3)^2 + (0.4)^2)/0.1) = 1 + exp(-2.5)
    assert a(np.float64(0.5), np.float64(100.0)) == pytest.approx(1.0 + np.exp(-2.5), abs=1e-14)
    # x offset 0.1 and frequency offset 0.1 N from the first centre
    v = a(np.float64(0.6), np.float64(200.0))
    want = np.exp(-(0.01 + 0.01) / 0.1) + np.exp(-(0.16 + 0.25) / 0.1)
    assert v == pytest.approx(want, abs=1e-14)
    assert np.all(np.abs(a(np.linspace(0, 1, 7), 0.0).imag) == 0)


def test_hankel_amplitude_against_bessel_functions():
    ph = Phase("iso2d")
    amp = Amplitude("hankel", phase=ph)
    rng = np.random.default_rng(0)
    x = rng.random((30, 2))
    xi = rng.integers(-40, 40, (30, 2)).astype(np.float64)
    xi[xi.sum(axis=1) == 0] += 1.0
    phi = ph.nonlinear(x, xi)
    want = (j0(2 * np.pi * phi) + 1j * y0(2 * np.pi * phi)) * np.exp(-2j * np.pi * phi)
    assert np.allclose(amp(x, xi), want, rtol=1e-12, atol=1e-14)
    # the kernel: a e^{2 pi i Phi} = H0(2 pi phi) e^{2 pi i x.xi} (the e^{-2 pi i phi} cancels)
    n = 8
    K = dense_K2(ph, n, amp)
    X, XI = space_grid_2d(n), freq_grid_2d(n)
    phi_g = ph.nonlinear(X[:, None, :], XI[None, :, :])
    with np.errstate(all="ignore"):
        K2 = (j0(2 * np.pi * phi_g) + 1j * y0(2 * np.pi * phi_g)) * np.exp(2j * np.pi * (X @ XI.T))
    ok = np.isfinite(K2)
    assert np.allclose(K[ok], K2[ok], rtol=1e-11, atol=1e-13)
    assert not ok[:, (n // 2) * n + n // 2].any()          # xi = 0: phi = 0, Y0 infinite


@pytest.mark.parametrize("n", [64, 256])
def test_bf_with_bump_amplitude_matches_dense(n):
    ph = Phase("cabs8")
    amp = Amplitude("bumps", centers=bump_centers(n), sigma2=0.1, N=n)
    bf = Butterfly1D(ph, n, 16, amp=amp)
    f = crandn(n, 2, seed=1)
    K = dense_K(ph, n, amp)
    assert np.linalg.norm(bf.apply(f) - K @ f) / np.linalg.norm(K @ f) < 1e-8
    g = crandn(n, 2, seed=2)
    assert np.linalg.norm(bf.adjoint(g) - K.conj().T @ g) / np.linalg.norm(K.conj().T @ g) < 1e-8
    # with a = 1 the operator differs: the amplitude is really applied
    assert np.linalg.norm(Butterfly1D(ph, n, 16).apply(f) - K @ f) > 0.1 * np.linalg.norm(K @ f)


def test_bf_with_hankel_amplitude_2d():
    """n = 32: K~ against dense K on vectors without the xi = 0 entry (where a is infinite); the
    interpolation error falls with r1, and the adjoint identity holds to rounding."""
    n = 32
    ph = Phase("iso2d")
    amp = Amplitude("hankel", phase=ph)
    K = dense_K2(ph, n, amp)
    zero = (n // 2) * n + n // 2
    K[:, zero] = 0.0
    f = crandn(n * n, 2, seed=3)
    f[zero] = 0.0
    errs = []
    for r1 in (5, 7):
        bf = Butterfly2D(ph, n, r1, amp=amp)
        errs.append(np.linalg.norm(bf.apply(f) - K @ f) / np.linalg.norm(K @ f))
    assert errs[1] < errs[0] < 5e-2, errs
    bf = Butterfly2D(ph, n, 5, amp=amp)
    g = crandn(n * n, 1, seed=4)[:, 0]
    lhs = np.vdot(g, bf.apply(f[:, 0]))
    rhs = np.vdot(bf.adjoint(g), f[:, 0])
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
