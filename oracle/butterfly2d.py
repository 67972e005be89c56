"""Butterfly factorization (BF) of a 2D discrete FIO, built from its definitions.

Test infrastructure only: nothing on the product path imports this module.

Section 2.2 with d = 2 (Section 5.2): the same factorization as Eq. 2.1,
    K ~ K~ = U^[T] B^[T] ... B^[h+1] M^[h] C^[h+1] ... C^[T] V^[T],
over quadtrees instead of binary trees.  Notation (per dimension as in 1D):

* n points per dimension, N = n^2, L = log2 n, h = floor(L/2), sU = max(L-3, h),
  sV = min(3, h).  Vectors are lexicographic: x_i = (i1/n, i2/n) for
  i = i1 n + i2, xi_j = (j1 - n/2, j2 - n/2) for j = j1 n + j2.
* A box at level s is (a1, a2), 0 <= a1, a2 < 2^s, with id a = a1 2^s + a2; it
  is the tensor product of the 1D boxes a1 and a2.  Its four children are
  (2 a1 + c1, 2 a2 + c2), child number c = 2 c1 + c2.
* Chebyshev grid of a box: the tensor product of the 1D first-kind points,
  node t = t1 r1 + t2 (r = r1^2 nodes), and the tensor Lagrange basis
  p_t(x) = p_t1(x1) p_t2(x2).
* A pair at space level s is (tau at space level s, sigma at frequency
  level L - s) with index a 4^(L-s) + b: there are 4^L = N pairs per level.

Factor entries are those of the 1D definitions with vector arguments and
products of dot-products in Phi (Section 2.2):
  V[(tau,sigma,j), xi] = e^{2 pi i (Phi(y_tau, xi) - Phi(y_tau, gamma_sigma_j))} q_sigma_j(xi)
  C[(tau',sigma',j), (tau,beta,t)] = e^{2 pi i (Phi(y_tau', gamma_beta_t) - Phi(y_tau', gamma_sigma'_j))} q_sigma'_j(gamma_beta_t)
  M[(tau,sigma,i), (tau,sigma,j)] = e^{2 pi i Phi(z_tau_i, gamma_sigma_j)}
  B[(tau,sigma,i), (alpha,beta,t)] = e^{2 pi i (Phi(z_tau_i, eta_beta) - Phi(z_alpha_t, eta_beta))} p_alpha_t(z_tau_i)
  U[x, (tau,sigma,i)] = e^{2 pi i (Phi(x, eta_sigma) - Phi(z_tau_i, eta_sigma))} p_tau_i(x)
with tau' a child of tau and beta a child of sigma' in C, tau a child of alpha
and beta a child of sigma in B.  The adjoint applies the conjugate transposes
in reverse order.
"""
import numpy as np

from .butterfly import cheb_nodes, lagrange

TWO_PI_I = 2j * np.pi


def _tensor_lagrange(n1, n2, p1, p2):
    """Tensor Lagrange basis.  n1, n2: (..., r1) 1D nodes; p1, p2: (..., m) point
    coordinates -> (..., m, r1^2) with column t1 r1 + t2 = l_t1(p1) l_t2(p2)."""
    l1 = lagrange(n1, p1)
    l2 = lagrange(n2, p2)
    out = l1[..., :, :, None] * l2[..., :, None, :]
    return out.reshape(out.shape[:-2] + (-1,))


class Butterfly2D:
    """BF of the 2D FIO, r = r1^2 tensor Chebyshev nodes per box; the amplitude (default a = 1)
    enters only the middle factor M (Section 2.2)."""

    def __init__(self, phase, n, r1, max_block_elems=1 << 23, levels=None, amp=None):
        self.amp = amp
        L = int(round(np.log2(n)))
        if 2 ** L != n or L < 2:
            raise ValueError("n must be a power of two >= 4")
        if phase.d != 2:
            raise ValueError("Butterfly2D needs a 2D phase")
        self.phase, self.n, self.r1, self.r, self.L = phase, n, r1, r1 * r1, L
        self.N = n * n
        self.h = L // 2
        self.sU = max(L - 3, self.h)
        self.sV = min(3, self.h)
        if levels is not None:   # (h, sU, sV) other than Section 5.2's choice, 0 <= sV <= h <= sU <= L
            self.h, self.sU, self.sV = levels
            if not 0 <= self.sV <= self.h <= self.sU <= L:
                raise ValueError("levels must satisfy 0 <= sV <= h <= sU <= L")
        self.t = cheb_nodes(r1)
        self.max_block_elems = max_block_elems

    # ---- quadtree geometry -----------------------------------------------
    @staticmethod
    def split(s, a):
        """box id -> (a1, a2) at level s."""
        a = np.asarray(a)
        return a >> s, a & ((1 << s) - 1)

    @staticmethod
    def child(s, a, c):
        """id at level s + 1 of child c of box a at level s."""
        a1, a2 = Butterfly2D.split(s, a)
        c = np.asarray(c)
        return ((2 * a1 + (c >> 1)) << (s + 1)) + 2 * a2 + (c & 1)

    @staticmethod
    def parent(s, a):
        """id at level s - 1 of the parent of box a at level s."""
        a1, a2 = Butterfly2D.split(s, a)
        return ((a1 >> 1) << (s - 1)) + (a2 >> 1)

    def space_center(self, s, a):
        a1, a2 = self.split(s, a)
        return np.stack([(a1 + 0.5) / 2.0 ** s, (a2 + 0.5) / 2.0 ** s], axis=-1)

    def space_nodes_1d(self, s, a):
        """(..., 2, r1): 1D Chebyshev points of the box in each dimension."""
        y = self.space_center(s, a)
        return y[..., :, None] + (0.5 / 2.0 ** s) * self.t

    def space_nodes(self, s, a):
        """(..., r, 2): tensor nodes z_t, t = t1 r1 + t2."""
        nd = self.space_nodes_1d(s, a)
        g1 = np.repeat(nd[..., 0, :], self.r1, axis=-1)
        g2 = np.tile(nd[..., 1, :], self.r1)
        return np.stack([g1, g2], axis=-1)

    def space_points(self, s, a):
        """(..., m^2, 2) points of the box (local index l1 m + l2) and (..., m^2) lexicographic indices."""
        m = self.n >> s
        a1, a2 = self.split(s, a)
        l1, l2 = np.divmod(np.arange(m * m), m)
        i1 = a1[..., None] * m + l1
        i2 = a2[..., None] * m + l2
        return np.stack([i1 / self.n, i2 / self.n], axis=-1), i1 * self.n + i2

    def freq_center(self, l, b):
        b1, b2 = self.split(l, b)
        w = self.n / 2.0 ** l
        return np.stack([-self.n / 2 + (b1 + 0.5) * w, -self.n / 2 + (b2 + 0.5) * w], axis=-1)

    def freq_nodes_1d(self, l, b):
        w = self.n / 2.0 ** l
        return self.freq_center(l, b)[..., :, None] + (w / 2) * self.t

    def freq_nodes(self, l, b):
        nd = self.freq_nodes_1d(l, b)
        g1 = np.repeat(nd[..., 0, :], self.r1, axis=-1)
        g2 = np.tile(nd[..., 1, :], self.r1)
        return np.stack([g1, g2], axis=-1)

    def freq_points(self, l, b):
        """(..., m^2, 2) integer frequencies of the box and (..., m^2) lexicographic indices."""
        m = self.n >> l
        b1, b2 = self.split(l, b)
        l1, l2 = np.divmod(np.arange(m * m), m)
        j1 = b1[..., None] * m + l1
        j2 = b2[..., None] * m + l2
        return np.stack([j1 - self.n / 2, j2 - self.n / 2], axis=-1).astype(np.float64), j1 * self.n + j2

    def _chunks(self, count, per_item, multiple=1):
        step = max(multiple, self.max_block_elems // max(1, per_item))
        step -= step % multiple
        for lo in range(0, count, step):
            yield lo, min(count, lo + step)

    # ---- factor blocks (entries straight from the definitions) -------------
    def V_block(self, a):
        """[a, b, j, q]: space boxes a at level sV, every frequency leaf b (level L - sV)."""
        L, s = self.L, self.sV
        b = np.arange(4 ** (L - s))
        gn = self.freq_nodes_1d(L - s, b)                        # (nb, 2, r1)
        gam = self.freq_nodes(L - s, b)                          # (nb, r, 2)
        xi, _ = self.freq_points(L - s, b)                       # (nb, ls, 2)
        q = _tensor_lagrange(gn[:, 0], gn[:, 1], xi[..., 0], xi[..., 1])   # (nb, ls, r)
        y = self.space_center(s, a)[:, None, None, None, :]
        ph = self.phase(y, xi[None, :, None, :, :]) - self.phase(y, gam[None, :, :, None, :])
        return np.exp(TWO_PI_I * ph) * np.swapaxes(q, 1, 2)[None]

    def C_block(self, s, a_out):
        """[a', b', j, c, t] of C (pair level s -> s+1): a' at space level s+1,
        b' at frequency level L-s-1, input frequency boxes beta_c = child c of b'."""
        L = self.L
        b_out = np.arange(4 ** (L - s - 1))
        y = self.space_center(s + 1, a_out)[:, None, None, None, None, :]
        gn_out = self.freq_nodes_1d(L - s - 1, b_out)            # (nb, 2, r1)
        gam_out = self.freq_nodes(L - s - 1, b_out)              # (nb, r, 2)
        b_in = self.child(L - s - 1, b_out[:, None], np.arange(4)[None, :])   # (nb, 4)
        gam_in = self.freq_nodes(L - s, b_in)                    # (nb, 4, r, 2)
        # q_{b', j}(gamma_{beta_c, t}) -> (nb, 4, r_t, r_j)
        qv = _tensor_lagrange(gn_out[:, None, 0], gn_out[:, None, 1], gam_in[..., 0], gam_in[..., 1])
        ph = (self.phase(y, gam_in[None, :, None, :, :, :])
              - self.phase(y, gam_out[None, :, :, None, None, :]))
        return np.exp(TWO_PI_I * ph) * np.transpose(qv, (0, 3, 1, 2))[None]

    def M_block(self, a):
        """[a, b, i, j] = a(z_a_i, gamma_b_j) e^{2 pi i Phi(z_a_i, gamma_b_j)} at the middle level h."""
        L, h = self.L, self.h
        b = np.arange(4 ** (L - h))
        z = self.space_nodes(h, a)[:, None, :, None, :]
        gam = self.freq_nodes(L - h, b)[None, :, None, :, :]
        m = np.exp(TWO_PI_I * self.phase(z, gam))
        return m if self.amp is None else self.amp(z, gam) * m

    def B_block(self, s, a_out):
        """[a', b', i, c, t] of B (pair level s -> s+1): a' at space level s+1 with
        parent alpha, b' at frequency level L-s-1 with children beta_c."""
        L = self.L
        b_out = np.arange(4 ** (L - s - 1))
        al = self.parent(s + 1, a_out)
        z_out = self.space_nodes(s + 1, a_out)                   # (na, r, 2)
        z_in = self.space_nodes(s, al)                           # (na, r, 2)
        an = self.space_nodes_1d(s, al)                          # (na, 2, r1)
        pv = _tensor_lagrange(an[:, 0], an[:, 1], z_out[..., 0], z_out[..., 1])   # (na, r_i, r_t)
        b_in = self.child(L - s - 1, b_out[:, None], np.arange(4)[None, :])
        eta = self.freq_center(L - s, b_in)                      # (nb, 4, 2)
        zo = z_out[:, None, :, None, None, :]
        zi = z_in[:, None, None, None, :, :]
        e = eta[None, :, None, :, None, :]
        ph = self.phase(zo, e) - self.phase(zi, e)
        return np.exp(TWO_PI_I * ph) * pv[:, None, :, None, :]

    def U_block(self, a):
        """[a, l, b, i]: space leaves a (level sU), point l of the leaf, frequency boxes b (level L-sU)."""
        L, s = self.L, self.sU
        b = np.arange(4 ** (L - s))
        x, _ = self.space_points(s, a)                           # (na, ls, 2)
        z = self.space_nodes(s, a)                               # (na, r, 2)
        an = self.space_nodes_1d(s, a)
        p = _tensor_lagrange(an[:, 0], an[:, 1], x[..., 0], x[..., 1])   # (na, ls, r)
        eta = self.freq_center(L - s, b)                         # (nb, 2)
        ph = (self.phase(x[:, :, None, None, :], eta[None, None, :, None, :])
              - self.phase(z[:, None, None, :, :], eta[None, None, :, None, :]))
        return np.exp(TWO_PI_I * ph) * p[:, :, None, :]

    # ---- stages --------------------------------------------------------------
    def _V(self, f, adjoint=False):
        L, s, r = self.L, self.sV, self.r
        na, nb = 4 ** s, 4 ** (L - s)
        _, idx = self.freq_points(L - s, np.arange(nb))          # (nb, ls)
        ls = idx.shape[1]
        if not adjoint:
            F = f[idx]                                           # (nb, ls, k)
            c = np.empty((na, nb, r, f.shape[-1]), dtype=np.complex128)
            for lo, hi in self._chunks(na, nb * r * ls):
                c[lo:hi] = np.matmul(self.V_block(np.arange(lo, hi)), F[None])
            return c.reshape(na * nb, r, -1)
        C = f.reshape(na, nb, r, -1)
        acc = np.zeros((nb, ls, C.shape[-1]), dtype=np.complex128)
        for lo, hi in self._chunks(na, nb * r * ls):
            Vh = np.swapaxes(self.V_block(np.arange(lo, hi)).conj(), -1, -2)
            acc += np.matmul(Vh, C[lo:hi]).sum(axis=0)
        out = np.zeros((self.N, C.shape[-1]), dtype=np.complex128)
        out[idx.reshape(-1)] = acc.reshape(nb * ls, -1)
        return out

    def _transfer(self, block_fn, s, x, adjoint=False):
        """One transfer factor (B or C) between pair levels s and s+1: output pair
        (a', b') couples to the inputs (parent(a'), child_c(b')), c = 0..3; a block
        is r x 4r."""
        L, r = self.L, self.r
        na_in, nb_in = 4 ** s, 4 ** (L - s)
        na_out, nb_out = 4 ** (s + 1), 4 ** (L - s - 1)
        k = x.shape[-1]
        kids = self.child(L - s - 1, np.arange(nb_out)[:, None], np.arange(4)[None, :])   # (nb_out, 4)
        xin = x.reshape(na_in, nb_in, r, k)
        if not adjoint:
            out = np.empty((na_out, nb_out, r, k), dtype=np.complex128)
            for lo, hi in self._chunks(na_out, nb_out * 4 * r * r):
                a = np.arange(lo, hi)
                blk = block_fn(s, a).reshape(hi - lo, nb_out, r, 4 * r)
                g = xin[self.parent(s + 1, a)[:, None, None], kids[None]]            # (na, nb_out, 4, r, k)
                out[lo:hi] = np.matmul(blk, g.reshape(hi - lo, nb_out, 4 * r, k))
            return out.reshape(na_out * nb_out, r, k)
        xout = x.reshape(na_out, nb_out, r, k)
        res = np.zeros((na_in, nb_in, r, k), dtype=np.complex128)
        for lo, hi in self._chunks(na_out, nb_out * 4 * r * r):
            a = np.arange(lo, hi)
            blk = block_fn(s, a).reshape(hi - lo, nb_out, r, 4 * r)
            contrib = np.matmul(np.swapaxes(blk.conj(), -1, -2), xout[lo:hi])        # (na, nb_out, 4r, k)
            contrib = contrib.reshape(hi - lo, nb_out, 4, r, k)
            np.add.at(res, (self.parent(s + 1, a)[:, None, None], kids[None]), contrib)
        return res.reshape(na_in * nb_in, r, k)

    def _M(self, c, adjoint=False):
        L, h, r = self.L, self.h, self.r
        na, nb = 4 ** h, 4 ** (L - h)
        x = c.reshape(na, nb, r, -1)
        out = np.empty_like(x)
        for lo, hi in self._chunks(na, nb * r * r):
            Mb = self.M_block(np.arange(lo, hi))
            if adjoint:
                Mb = np.swapaxes(Mb.conj(), -1, -2)
            out[lo:hi] = np.matmul(Mb, x[lo:hi])
        return out.reshape(na * nb, r, -1)

    def _U(self, d, adjoint=False):
        L, s, r = self.L, self.sU, self.r
        na, nb = 4 ** s, 4 ** (L - s)
        _, idx = self.space_points(s, np.arange(na))             # (na, ls)
        ls = idx.shape[1]
        if not adjoint:
            D = d.reshape(na, nb * r, -1)
            y = np.zeros((self.N, D.shape[-1]), dtype=np.complex128)
            for lo, hi in self._chunks(na, ls * nb * r):
                Ub = self.U_block(np.arange(lo, hi)).reshape(hi - lo, ls, nb * r)
                y[idx[lo:hi].reshape(-1)] = np.matmul(Ub, D[lo:hi]).reshape((hi - lo) * ls, -1)
            return y
        G = d[idx]                                               # (na, ls, k)
        out = np.empty((na, nb * r, G.shape[-1]), dtype=np.complex128)
        for lo, hi in self._chunks(na, ls * nb * r):
            Ub = self.U_block(np.arange(lo, hi)).reshape(hi - lo, ls, nb * r)
            out[lo:hi] = np.matmul(np.swapaxes(Ub.conj(), -1, -2), G[lo:hi])
        return out.reshape(na * nb, r, -1)

    # ---- public ----------------------------------------------------------------
    def apply(self, f):
        """K~ f for lexicographic f of shape (N,) or (N, k)."""
        f = np.asarray(f, dtype=np.complex128)
        vec = f.ndim == 1
        x = f.reshape(self.N, -1)
        c = self._V(x)
        for s in range(self.sV, self.h):
            c = self._transfer(self.C_block, s, c)
        d = self._M(c)
        for s in range(self.h, self.sU):
            d = self._transfer(self.B_block, s, d)
        y = self._U(d)
        return y[:, 0] if vec else y

    def adjoint(self, g):
        """K~^* g: conjugate transposes of the factors in reverse order."""
        g = np.asarray(g, dtype=np.complex128)
        vec = g.ndim == 1
        x = g.reshape(self.N, -1)
        d = self._U(x, adjoint=True)
        for s in reversed(range(self.h, self.sU)):
            d = self._transfer(self.B_block, s, d, adjoint=True)
        c = self._M(d, adjoint=True)
        for s in reversed(range(self.sV, self.h)):
            c = self._transfer(self.C_block, s, c, adjoint=True)
        f = self._V(c, adjoint=True)
        return f[:, 0] if vec else f

    def dense(self):
        """K~ as a dense matrix (small n only)."""
        return self.apply(np.eye(self.N, dtype=np.complex128))
