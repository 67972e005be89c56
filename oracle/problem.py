"""Discrete FIO problem definition: grids, phase functions, dense K.

Test infrastructure only: nothing on the product path imports this module.

Eq. 1.1-1.2: K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)) with
x_i = i/n on [0,1)^d and integer frequencies xi_j in [-n/2, n/2)^d, N = n^d.
The main workloads have amplitude a = 1; Amplitude gives the variable
amplitudes of Sections 5.1 and 5.3.

Phase families:
  'dft'        Phi = x . xi                      (K^* K = N I exactly)
  'cabs'       Phi = x xi + c(x) |xi|,  c(x) = (2 + s sin 2 pi x) / 16   (1D)
  'cabs8'      Phi = x xi + c(x) |xi|,  c(x) = (2 + s sin 2 pi x) / 8    (1D, Section 5.1)
  'elliptic2d' Phi = x . xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2),
               c1 = (2 + sin 2 pi x1 sin 2 pi x2) / 16,
               c2 = (2 + cos 2 pi x1 cos 2 pi x2) / 16          (Section 5.2)
  'iso2d'      Phi = x . xi + c(x) ||xi||,
               c = (3 + s sin 2 pi x1 sin 2 pi x2) / 8             (Section 5.3)
"""
import numpy as np
from scipy.special import hankel1


class Phase:
    """Phase function of one workload family.  d is the dimension: 1 for
    'cabs', 2 for 'elliptic2d', either for 'dft' (default 1)."""

    def __init__(self, kind="cabs", s=1.0, d=None):
        if kind not in ("dft", "cabs", "cabs8", "elliptic2d", "iso2d"):
            raise ValueError(kind)
        self.kind = kind
        self.s = float(s)
        self.d = 2 if kind in ("elliptic2d", "iso2d") else (1 if d is None else int(d))
        if (kind in ("cabs", "cabs8") and self.d != 1) or self.d not in (1, 2):
            raise ValueError("phase %s has no %d-dimensional form" % (kind, self.d))

    def c(self, x):
        """c(x) of the 1D families."""
        return (2.0 + self.s * np.sin(2.0 * np.pi * x)) / (8.0 if self.kind == "cabs8" else 16.0)

    def nonlinear(self, x, xi):
        """Phi(x, xi) - x . xi (the part that is not the DFT)."""
        if self.d == 1:
            return self(x, xi) - x * xi
        return self(x, xi) - np.sum(x * xi, axis=-1)

    def __call__(self, x, xi):
        """Phi(x, xi), broadcasting.  1D: scalars arrays.  2D: trailing axis 2."""
        if self.kind == "dft":
            if self.d == 1:
                return x * xi
            return np.sum(x * xi, axis=-1)
        if self.kind in ("cabs", "cabs8"):
            return x * xi + self.c(x) * np.abs(xi)
        x1, x2 = x[..., 0], x[..., 1]
        k1, k2 = xi[..., 0], xi[..., 1]
        if self.kind == "iso2d":
            c = (3.0 + self.s * np.sin(2 * np.pi * x1) * np.sin(2 * np.pi * x2)) / 8.0
            return x1 * k1 + x2 * k2 + c * np.sqrt(k1 * k1 + k2 * k2)
        c1 = (2.0 + np.sin(2 * np.pi * x1) * np.sin(2 * np.pi * x2)) / 16.0
        c2 = (2.0 + np.cos(2 * np.pi * x1) * np.cos(2 * np.pi * x2)) / 16.0
        return x1 * k1 + x2 * k2 + np.sqrt(c1 * c1 * k1 * k1 + c2 * c2 * k2 * k2)


class Amplitude:
    """Amplitude a(x, xi) of Eq. 1.2 (returned complex, broadcasting like Phase).

    'one'     a = 1.
    'bumps'   Section 5.1: a = sum_k exp(-((x - x_k)^2 + ((xi - xi_k) / N)^2) / sigma2), with the
              centres (x_k, xi_k) given as an (m, 2) array and N the vector length.
    'hankel'  Section 5.3: a = H0^(1)(2 pi phi) exp(-2 pi i phi), phi = Phi(x, xi) - x . xi of the
              given 2D phase (infinite where phi = 0, i.e. at xi = 0).
    """

    def __init__(self, kind="one", centers=None, sigma2=0.1, N=None, phase=None):
        if kind not in ("one", "bumps", "hankel"):
            raise ValueError(kind)
        self.kind = kind
        if kind == "bumps":
            self.centers = np.asarray(centers, dtype=np.float64).reshape(-1, 2)
            self.sigma2, self.N = float(sigma2), float(N)
        if kind == "hankel":
            if phase is None or phase.d != 2:
                raise ValueError("the Hankel amplitude needs its 2D phase")
            self.phase = phase

    def __call__(self, x, xi):
        if self.kind == "one":
            return np.ones(np.broadcast_shapes(np.shape(x), np.shape(xi)), dtype=np.complex128)
        if self.kind == "bumps":
            x = np.asarray(x, dtype=np.float64)[..., None]
            xi = np.asarray(xi, dtype=np.float64)[..., None]
            xk, fk = self.centers[:, 0], self.centers[:, 1]
            e = ((x - xk) ** 2 + ((xi - fk) / self.N) ** 2) / self.sigma2
            return np.sum(np.exp(-e), axis=-1).astype(np.complex128)
        ph = self.phase.nonlinear(np.asarray(x, dtype=np.float64), np.asarray(xi, dtype=np.float64))
        with np.errstate(all="ignore"):
            return hankel1(0, 2 * np.pi * ph) * np.exp(-2j * np.pi * ph)


def _amp(amp, x, xi):
    return 1.0 if amp is None else amp(x, xi)


def space_grid_1d(n):
    """x_i = i/n, i = 0..n-1 (Eq. 1.1)."""
    return np.arange(n, dtype=np.float64) / n


def freq_grid_1d(n):
    """xi_j = j - n/2, j = 0..n-1 (Eq. 1.1)."""
    return np.arange(n, dtype=np.float64) - n / 2


def dense_K(phase, n, amp=None):
    """Dense K (1D), Eq. 1.2 (a = 1 unless an Amplitude is given).  Only for small n."""
    x = space_grid_1d(n)
    xi = freq_grid_1d(n)
    return _amp(amp, x[:, None], xi[None, :]) * np.exp(2j * np.pi * phase(x[:, None], xi[None, :]))


def K_rows(phase, n, rows, amp=None):
    """Selected rows of K (1D), evaluated one entry at a time from Eq. 1.2."""
    x = space_grid_1d(n)[np.asarray(rows)]
    xi = freq_grid_1d(n)
    return _amp(amp, x[:, None], xi[None, :]) * np.exp(2j * np.pi * phase(x[:, None], xi[None, :]))


def space_grid_2d(n):
    """x_i = (i1/n, i2/n) for the lexicographic index i = i1 n + i2 (i1 slow), shape (n^2, 2)."""
    i1, i2 = np.divmod(np.arange(n * n), n)
    return np.stack([i1 / n, i2 / n], axis=-1).astype(np.float64)


def freq_grid_2d(n):
    """xi_j = (j1 - n/2, j2 - n/2) for j = j1 n + j2 (j1 slow), shape (n^2, 2)."""
    j1, j2 = np.divmod(np.arange(n * n), n)
    return np.stack([j1 - n / 2, j2 - n / 2], axis=-1).astype(np.float64)


def dense_K2(phase, n, amp=None):
    """Dense K (2D), Eq. 1.2, lexicographic rows and columns.  Small n only."""
    x = space_grid_2d(n)
    xi = freq_grid_2d(n)
    return _amp(amp, x[:, None, :], xi[None, :, :]) * np.exp(2j * np.pi * phase(x[:, None, :], xi[None, :, :]))


def K2_rows(phase, n, rows, amp=None):
    """Selected rows of the 2D K, entry by entry from Eq. 1.2."""
    x = space_grid_2d(n)[np.asarray(rows)]
    xi = freq_grid_2d(n)
    return _amp(amp, x[:, None, :], xi[None, :, :]) * np.exp(2j * np.pi * phase(x[:, None, :], xi[None, :, :]))


def morton_order(n):
    """Quadtree (Morton) order of the n x n frequency grid: perm[m] is the
    lexicographic index j = j1 n + j2 at Morton position m, where m interleaves
    the bits of j1 (odd positions, more significant) and j2 (even positions).
    Every quadtree box is then a contiguous range of positions."""
    L = int(round(np.log2(n)))
    m = np.arange(n * n)
    j1 = np.zeros_like(m)
    j2 = np.zeros_like(m)
    for k in range(L):
        j2 |= ((m >> (2 * k)) & 1) << k
        j1 |= ((m >> (2 * k + 1)) & 1) << k
    return j1 * n + j2
