"""Two-stage approximate inverse of the discrete FIO (Algorithm 1, Eq. 4.1-4.3).

Test infrastructure only: nothing on the product path imports this module.

Offline: BF K~ of K (Section 2.2); black-box HSS G~ of G = K^* K sampled
through K~^* K~ (Section 3, Section 4.1); ULV factorization F~ of G~
(Section 2.4).  Online: f^ = F~ K~^* u (Eq. 4.2, direct solver on the
approximate normal equation Eq. 4.3).
"""
import numpy as np

from .butterfly import Butterfly1D
from .hss import ULV, build_blackbox


class FIOSolver:
    def __init__(self, phase, n, r, leaf, p, tol, seed, rank_frac=0.5, amp=None):
        self.bf = Butterfly1D(phase, n, r, amp=amp)
        self.stats = {}
        self.hss = build_blackbox(lambda X: self.bf.adjoint(self.bf.apply(X)),
                                  n, leaf, p, tol, seed, rank_frac=rank_frac, stats=self.stats)
        self.ulv = ULV(self.hss)

    def solve(self, u):
        """f^ = F~ (K~^* u)."""
        return self.ulv.solve(self.bf.adjoint(u))


class FIOSolver2D:
    """Algorithm 1 in 2D: the HSS of G~ = K~^* K~ is built over the frequency
    index in quadtree (Morton) order, so that HSS leaves and nodes are
    quadtree boxes and their concatenations (a binary tree whose levels
    alternate the split direction); f^ = P^T F~ P K~^* u."""

    def __init__(self, phase, n, r1, leaf, p, tol, seed, rank_frac=0.5, amp=None):
        from .butterfly2d import Butterfly2D
        from .problem import morton_order
        self.bf = Butterfly2D(phase, n, r1, amp=amp)
        self.perm = morton_order(n)
        self.stats = {}
        N = n * n

        def apply_H(X):   # P K~^* K~ P^T X, 64 columns at a time (bounded coefficient states)
            out = np.empty_like(X)
            for c0 in range(0, X.shape[1], 64):
                Y = np.empty_like(X[:, c0:c0 + 64])
                Y[self.perm] = X[:, c0:c0 + 64]
                out[:, c0:c0 + 64] = self.bf.adjoint(self.bf.apply(Y))[self.perm]
            return out

        self.hss = build_blackbox(apply_H, N, leaf, p, tol, seed, rank_frac=rank_frac, stats=self.stats)
        self.ulv = ULV(self.hss)

    def solve(self, u):
        z = self.ulv.solve(self.bf.adjoint(u)[self.perm])
        f = np.empty_like(z)
        f[self.perm] = z
        return f


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
