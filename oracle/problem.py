"""Discrete FIO problem definition: grids, phase functions, dense K.

Test infrastructure only: nothing on the product path imports this module.

Eq. 1.1-1.2: K_ij = a(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)) with
x_i = i/n on [0,1)^d and integer frequencies xi_j in [-n/2, n/2)^d, N = n^d.
Every workload here has amplitude a = 1.

Phase families:
  'dft'        Phi = x . xi                      (K^* K = N I exactly)
  'cabs'       Phi = x xi + c(x) |xi|,  c(x) = (2 + s sin 2 pi x) / 16   (1D)
               (Section 5.1 uses the same form with /8 and a variable amplitude)
  'elliptic2d' Phi = x . xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2),
               c1 = (2 + sin 2 pi x1 sin 2 pi x2) / 16,
               c2 = (2 + cos 2 pi x1 cos 2 pi x2) / 16          (Section 5.2)
"""
import numpy as np


class Phase:
    """Phase function of one workload family.  d is the dimension: 1 for
    'cabs', 2 for 'elliptic2d', either for 'dft' (default 1)."""

    def __init__(self, kind="cabs", s=1.0, d=None):
        if kind not in ("dft", "cabs", "elliptic2d"):
            raise ValueError(kind)
        self.kind = kind
        self.s = float(s)
        self.d = 2 if kind == "elliptic2d" else (1 if d is None else int(d))
        if (kind == "cabs" and self.d != 1) or self.d not in (1, 2):
            raise ValueError("phase %s has no %d-dimensional form" % (kind, self.d))

    def c(self, x):
        """c(x) of the 1D family."""
        return (2.0 + self.s * np.sin(2.0 * np.pi * x)) / 16.0

    def __call__(self, x, xi):
        """Phi(x, xi), broadcasting.  1D: scalars arrays.  2D: trailing axis 2."""
        if self.kind == "dft":
            if self.d == 1:
                return x * xi
            return np.sum(x * xi, axis=-1)
        if self.kind == "cabs":
            return x * xi + self.c(x) * np.abs(xi)
        x1, x2 = x[..., 0], x[..., 1]
        k1, k2 = xi[..., 0], xi[..., 1]
        c1 = (2.0 + np.sin(2 * np.pi * x1) * np.sin(2 * np.pi * x2)) / 16.0
        c2 = (2.0 + np.cos(2 * np.pi * x1) * np.cos(2 * np.pi * x2)) / 16.0
        return x1 * k1 + x2 * k2 + np.sqrt(c1 * c1 * k1 * k1 + c2 * c2 * k2 * k2)


def space_grid_1d(n):
    """x_i = i/n, i = 0..n-1 (Eq. 1.1)."""
    return np.arange(n, dtype=np.float64) / n


def freq_grid_1d(n):
    """xi_j = j - n/2, j = 0..n-1 (Eq. 1.1)."""
    return np.arange(n, dtype=np.float64) - n / 2


def dense_K(phase, n):
    """Dense K (1D), Eq. 1.2 with a = 1.  Only for small n."""
    x = space_grid_1d(n)
    xi = freq_grid_1d(n)
    return np.exp(2j * np.pi * phase(x[:, None], xi[None, :]))


def K_rows(phase, n, rows):
    """Selected rows of K (1D), evaluated one entry at a time from Eq. 1.2."""
    x = space_grid_1d(n)[np.asarray(rows)]
    xi = freq_grid_1d(n)
    return np.exp(2j * np.pi * phase(x[:, None], xi[None, :]))


def space_grid_2d(n):
    """x_i = (i1/n, i2/n) for the lexicographic index i = i1 n + i2 (i1 slow), shape (n^2, 2)."""
    i1, i2 = np.divmod(np.arange(n * n), n)
    return np.stack([i1 / n, i2 / n], axis=-1).astype(np.float64)


def freq_grid_2d(n):
    """xi_j = (j1 - n/2, j2 - n/2) for j = j1 n + j2 (j1 slow), shape (n^2, 2)."""
    j1, j2 = np.divmod(np.arange(n * n), n)
    return np.stack([j1 - n / 2, j2 - n / 2], axis=-1).astype(np.float64)


def dense_K2(phase, n):
    """Dense K (2D), Eq. 1.2 with a = 1, lexicographic rows and columns.  Small n only."""
    x = space_grid_2d(n)
    xi = freq_grid_2d(n)
    return np.exp(2j * np.pi * phase(x[:, None, :], xi[None, :, :]))


def K2_rows(phase, n, rows):
    """Selected rows of the 2D K, entry by entry from Eq. 1.2."""
    x = space_grid_2d(n)[np.asarray(rows)]
    xi = freq_grid_2d(n)
    return np.exp(2j * np.pi * phase(x[:, None, :], xi[None, :, :]))


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
