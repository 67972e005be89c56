"""Butterfly factorization (BF) of a 1D discrete FIO, built from its definitions.

Test infrastructure only: nothing on the product path imports this module.

Section 2.2 and Eq. 2.1:
    K ~ K~ = U^[T] B^[T] ... B^[h+1] M^[h] C^[h+1] ... C^[T] V^[T],
with Chebyshev interpolation of rank r in every box.  Notation:

* Space tree: box (s, a) = [a/2^s, (a+1)/2^s], holding x_i = i/n for
  i in [a n/2^s, (a+1) n/2^s).  Frequency tree: box (l, b) =
  [-n/2 + b n/2^l, -n/2 + (b+1) n/2^l], holding the integer frequencies
  xi_j = j - n/2 inside it.  Centre = midpoint.
* Chebyshev points of the first kind on the closed box interval,
  z = centre + (w/2) cos((2k+1) pi / (2r)), k = 0..r-1, and the Lagrange
  polynomials p (space) and q (frequency) on them.
* A "pair" at space level s is (tau at space level s, sigma at frequency
  level L-s) -- the complementary low-rank blocks.  Pair index
  p = a * 2^(L-s) + b.
* L = log2 n, h = floor(L/2) (the middle level).  Outermost factors follow the
  practical top level of Section 5.2: the space leaves of U sit at level
  T = max(L-3, h); the frequency leaves of V sit at level max(L-3, L-h), i.e.
  the V pairs have space level sV = min(3, h).  #C = h - sV, #B = T - h.

Factor entries (Section 2.2, phase-modulated interpolation functions u, v):
  V[(tau,sigma,j), xi] = e^{2 pi i (Phi(y_tau, xi) - Phi(y_tau, gamma_sigma_j))} q_sigma_j(xi)
  C[(tau',sigma',j), (tau,beta,t)] = v_{tau',sigma';j}(gamma_beta_t)
        = e^{2 pi i (Phi(y_tau', gamma_beta_t) - Phi(y_tau', gamma_sigma'_j))} q_sigma'_j(gamma_beta_t)
        (tau' a child of tau, beta a child of sigma': right transfer, roles of
         x and xi exchanged with respect to B)
  M[(tau,sigma,i), (tau,sigma,j)] = k(z_tau_i, gamma_sigma_j) = e^{2 pi i Phi(z_tau_i, gamma_sigma_j)}
  B[(tau,sigma,i), (alpha,beta,t)] = u_{alpha,beta;t}(z_tau_i)
        = e^{2 pi i (Phi(z_tau_i, eta_beta) - Phi(z_alpha_t, eta_beta))} p_alpha_t(z_tau_i)
        (tau a child of alpha, beta a child of sigma: Eq. 2.4-2.6)
  U[x, (tau,sigma,i)] = e^{2 pi i (Phi(x, eta_sigma) - Phi(z_tau_i, eta_sigma))} p_tau_i(x)

The adjoint (Section 2.2, last paragraph) applies the conjugate transposes of
the factors in reverse order.
"""
import numpy as np

TWO_PI_I = 2j * np.pi


def cheb_nodes(r):
    """Chebyshev points of the first kind on [-1, 1]."""
    k = np.arange(r, dtype=np.float64)
    return np.cos((2 * k + 1) * np.pi / (2 * r))


def lagrange(nodes, x):
    """Lagrange basis on `nodes` evaluated at `x`.

    nodes: (..., r); x: (..., m)  ->  (..., m, r) with
    out[..., q, k] = prod_{k' != k} (x_q - nodes_k') / (nodes_k - nodes_k').
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = nodes.shape[-1]
    diff = x[..., :, None] - nodes[..., None, :]            # (..., m, r)
    out = np.empty(diff.shape, dtype=np.float64)
    for k in range(r):
        others = [kk for kk in range(r) if kk != k]
        num = np.prod(diff[..., others], axis=-1)          # (..., m)
        den = np.prod(nodes[..., k:k + 1] - nodes[..., others], axis=-1)  # (...,)
        out[..., k] = num / den[..., None]
    return out


class Butterfly1D:
    """BF of the 1D FIO (Eq. 2.1), applied block by block.  The amplitude (default a = 1) enters
    only the middle factor, M = k(z_i, gamma_j) = a(z_i, gamma_j) e^{2 pi i Phi(z_i, gamma_j)}
    (Section 2.2); the interpolation factors are amplitude-free."""

    def __init__(self, phase, n, r, max_block_elems=1 << 23, cache=None, levels=None, amp=None):
        self.amp = amp
        L = int(round(np.log2(n)))
        if 2 ** L != n or L < 2:
            raise ValueError("n must be a power of two >= 4")
        self.phase, self.n, self.r, self.L = phase, n, r, L
        self.h = L // 2
        self.sU = max(L - 3, self.h)
        self.sV = min(3, self.h)
        if levels is not None:   # (h, sU, sV) other than Section 5.2's choice, 0 <= sV <= h <= sU <= L
            self.h, self.sU, self.sV = levels
            if not 0 <= self.sV <= self.h <= self.sU <= L:
                raise ValueError("levels must satisfy 0 <= sV <= h <= sU <= L")
        self.t = cheb_nodes(r)
        self.max_block_elems = max_block_elems
        # Factor blocks are pure functions of (factor, level, chunk); keeping
        # them avoids rebuilding them for every product (small n only).
        self.cache = (n <= 1 << 13) if cache is None else cache
        self._blocks = {}

    def _blk(self, fn, *args):
        if not self.cache:
            return fn(*args)
        key = (fn.__name__,) + tuple(a if np.isscalar(a) else (int(a[0]), int(a[-1]) + 1) for a in args)
        if key not in self._blocks:
            self._blocks[key] = fn(*args)
        return self._blocks[key]

    # ---- tree geometry -------------------------------------------------
    def space_center(self, s, a):
        return (np.asarray(a, dtype=np.float64) + 0.5) / 2.0 ** s

    def space_nodes(self, s, a):
        y = self.space_center(s, a)
        return y[..., None] + (0.5 / 2.0 ** s) * self.t

    def space_points(self, s, a):
        m = self.n >> s
        a = np.asarray(a)
        return (a[..., None] * m + np.arange(m)) / self.n

    def freq_center(self, l, b):
        w = self.n / 2.0 ** l
        return -self.n / 2 + (np.asarray(b, dtype=np.float64) + 0.5) * w

    def freq_nodes(self, l, b):
        w = self.n / 2.0 ** l
        return self.freq_center(l, b)[..., None] + (w / 2) * self.t

    def freq_points(self, l, b):
        m = self.n >> l
        b = np.asarray(b)
        return (b[..., None] * m + np.arange(m)).astype(np.float64) - self.n / 2

    def _chunks(self, count, per_item, even=False):
        step = max(1, self.max_block_elems // max(1, per_item))
        if even:
            step = max(2, step - step % 2)
        for lo in range(0, count, step):
            yield lo, min(count, lo + step)

    # ---- factor blocks (entries straight from the definitions) -----------
    def V_block(self, a):
        """v[a, b, j, q] for space boxes a (level sV), all frequency leaves b."""
        L, s = self.L, self.sV
        b = np.arange(2 ** (L - s))
        gam = self.freq_nodes(L - s, b)                 # (nb, r)
        xi = self.freq_points(L - s, b)                 # (nb, ls)
        q = lagrange(gam, xi)                           # (nb, ls, r)
        y = self.space_center(s, a)[:, None, None, None]
        ph = self.phase(y, xi[None, :, None, :]) - self.phase(y, gam[None, :, :, None])
        return np.exp(TWO_PI_I * ph) * np.transpose(q, (0, 2, 1))[None]

    def C_block(self, s, a_out):
        """Block [a', b', j, beta, t] of C (pair level s -> s+1), a' at level s+1."""
        L = self.L
        b_out = np.arange(2 ** (L - s - 1))
        y = self.space_center(s + 1, a_out)[:, None, None, None, None]
        gam_out = self.freq_nodes(L - s - 1, b_out)                       # (nb, r)
        b_in = 2 * b_out[:, None] + np.arange(2)[None, :]                 # (nb, 2)
        gam_in = self.freq_nodes(L - s, b_in)                             # (nb, 2, r)
        # q_{b', j}(gamma_{beta, t}) -> (nb, 2, r_t, r_j)
        qv = lagrange(gam_out[:, None, :], gam_in)
        ph = (self.phase(y, gam_in[None, :, None, :, :])
              - self.phase(y, gam_out[None, :, :, None, None]))
        return np.exp(TWO_PI_I * ph) * np.transpose(qv, (0, 3, 1, 2))[None]

    def M_block(self, a):
        """M[a, b, i, j] = a(z_a_i, gamma_b_j) e^{2 pi i Phi(z_a_i, gamma_b_j)} at the middle level h."""
        L, h = self.L, self.h
        b = np.arange(2 ** (L - h))
        z = self.space_nodes(h, a)[:, None, :, None]
        gam = self.freq_nodes(L - h, b)[None, :, None, :]
        m = np.exp(TWO_PI_I * self.phase(z, gam))
        return m if self.amp is None else self.amp(z, gam) * m

    def B_block(self, s, a_out):
        """Block [a', b', i, beta, t] of B (pair level s -> s+1), a' at level s+1."""
        L = self.L
        b_out = np.arange(2 ** (L - s - 1))
        z_out = self.space_nodes(s + 1, a_out)                            # (na, r)
        z_in = self.space_nodes(s, np.asarray(a_out) // 2)                # (na, r)
        pv = lagrange(z_in, z_out)                                        # (na, r_i, r_t)
        b_in = 2 * b_out[:, None] + np.arange(2)[None, :]
        eta = self.freq_center(L - s, b_in)                               # (nb, 2)
        zo = z_out[:, None, :, None, None]
        zi = z_in[:, None, None, None, :]
        e = eta[None, :, None, :, None]
        ph = self.phase(zo, e) - self.phase(zi, e)
        return np.exp(TWO_PI_I * ph) * pv[:, None, :, None, :]

    def U_block(self, a):
        """U[a, q, b, i] for space leaves a (level sU), frequency boxes b (level L-sU)."""
        L, s = self.L, self.sU
        b = np.arange(2 ** (L - s))
        x = self.space_points(s, a)                     # (na, ls)
        z = self.space_nodes(s, a)                      # (na, r)
        p = lagrange(z, x)                              # (na, ls, r)
        eta = self.freq_center(L - s, b)
        ph = (self.phase(x[:, :, None, None], eta[None, None, :, None])
              - self.phase(z[:, None, None, :], eta[None, None, :, None]))
        return np.exp(TWO_PI_I * ph) * p[:, :, None, :]

    # ---- stages ---------------------------------------------------------
    def _V(self, f, adjoint=False):
        L, s, r, n = self.L, self.sV, self.r, self.n
        na, nb, ls = 2 ** s, 2 ** (L - s), n >> (L - s)
        if not adjoint:
            F = f.reshape(nb, ls, -1)
            c = np.empty((na, nb, r, F.shape[-1]), dtype=np.complex128)
            for lo, hi in self._chunks(na, nb * r * ls):
                c[lo:hi] = np.matmul(self._blk(self.V_block, np.arange(lo, hi)), F[None])
            return c.reshape(na * nb, r, -1)
        C = f.reshape(na, nb, r, -1)
        out = np.zeros((nb, ls, C.shape[-1]), dtype=np.complex128)
        for lo, hi in self._chunks(na, nb * r * ls):
            Vh = np.swapaxes(self._blk(self.V_block, np.arange(lo, hi)).conj(), -1, -2)
            out += np.matmul(Vh, C[lo:hi]).sum(axis=0)
        return out.reshape(n, -1)

    def _transfer(self, block_fn, s, x, adjoint=False):
        """One transfer factor (B or C) between pair levels s and s+1.

        Each output pair (a', b') couples to the inputs (a'//2, 2b'+beta),
        beta = 0, 1; a block is r x 2r.  Chunks hold whole sibling pairs.
        """
        L, r = self.L, self.r
        na_out, nb_out = 2 ** (s + 1), 2 ** (L - s - 1)
        k = x.shape[-1]
        if not adjoint:
            xin = x.reshape(2 ** s, nb_out, 2 * r, k)
            out = np.empty((na_out, nb_out, r, k), dtype=np.complex128)
            for lo, hi in self._chunks(na_out, nb_out * 2 * r * r, even=True):
                a = np.arange(lo, hi)
                blk = self._blk(block_fn, s, a).reshape(hi - lo, nb_out, r, 2 * r)
                out[lo:hi] = np.matmul(blk, xin[a // 2])
            return out.reshape(na_out * nb_out, r, k)
        xout = x.reshape(na_out, nb_out, r, k)
        xin = np.zeros((2 ** s, nb_out, 2 * r, k), dtype=np.complex128)
        for lo, hi in self._chunks(na_out, nb_out * 2 * r * r, even=True):
            a = np.arange(lo, hi)
            blk = self._blk(block_fn, s, a).reshape(hi - lo, nb_out, r, 2 * r)
            contrib = np.matmul(np.swapaxes(blk.conj(), -1, -2), xout[lo:hi])
            xin[lo // 2:hi // 2] += contrib.reshape((hi - lo) // 2, 2, nb_out, 2 * r, k).sum(axis=1)
        return xin.reshape(2 ** s * 2 ** (L - s), r, k)

    def _M(self, c, adjoint=False):
        L, h, r = self.L, self.h, self.r
        na, nb = 2 ** h, 2 ** (L - h)
        x = c.reshape(na, nb, r, -1)
        out = np.empty_like(x)
        for lo, hi in self._chunks(na, nb * r * r):
            Mb = self._blk(self.M_block, np.arange(lo, hi))
            if adjoint:
                Mb = np.swapaxes(Mb.conj(), -1, -2)
            out[lo:hi] = np.matmul(Mb, x[lo:hi])
        return out.reshape(na * nb, r, -1)

    def _U(self, d, adjoint=False):
        L, s, r, n = self.L, self.sU, self.r, self.n
        na, nb, ls = 2 ** s, 2 ** (L - s), n >> s
        if not adjoint:
            D = d.reshape(na, nb * r, -1)
            y = np.empty((na, ls, D.shape[-1]), dtype=np.complex128)
            for lo, hi in self._chunks(na, ls * nb * r):
                Ub = self._blk(self.U_block, np.arange(lo, hi)).reshape(hi - lo, ls, nb * r)
                y[lo:hi] = np.matmul(Ub, D[lo:hi])
            return y.reshape(n, -1)
        G = d.reshape(na, ls, -1)
        out = np.empty((na, nb * r, G.shape[-1]), dtype=np.complex128)
        for lo, hi in self._chunks(na, ls * nb * r):
            Ub = self._blk(self.U_block, np.arange(lo, hi)).reshape(hi - lo, ls, nb * r)
            out[lo:hi] = np.matmul(np.swapaxes(Ub.conj(), -1, -2), G[lo:hi])
        return out.reshape(na * nb, r, -1)

    # ---- public ---------------------------------------------------------
    def apply(self, f):
        """K~ f for f of shape (n,) or (n, k) (Eq. 2.1, right to left)."""
        f = np.asarray(f, dtype=np.complex128)
        vec = f.ndim == 1
        x = f.reshape(self.n, -1)
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
        x = g.reshape(self.n, -1)
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
        return self.apply(np.eye(self.n, dtype=np.complex128))
