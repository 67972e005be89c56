"""HSS matrices, randomized black-box construction and ULV factorization.

Test infrastructure only: nothing on the product path imports this module.

* Def. 2.1-2.2: HSS tree (full binary, leaves of size m at level Lh) and
  generators D (leaves), U (leaf bases; transfer matrices at nonleaf nodes),
  B_{alpha2,alpha1} (one per nonleaf node).
* Eq. 2.7-2.8: telescoping factorization, used for the dense reconstruction
  and for the matrix-vector product.
* Section 3.1-3.3: bottom-up construction from samples Y = H Omega with an
  independent Gaussian test matrix per level, then top-down postprocessing.
* Section 2.4, Eq. 2.9-2.12: ULV factorization (QL basis elimination,
  partial Cholesky, merge, root Cholesky) and the bottom-up / top-down solve.

Readings where the paper leaves a choice open (each stated again where it is
used):
  R1  rank per level: Section 3 assumes one rank r_l per level; every node of
      level l keeps the first r_l = max over the level of its truncated rank
      QRCP columns.
  R2  truncation: the QRCP of Y_tau Gamma_tau keeps the columns whose pivot
      satisfies |R_kk| > tol * max_j ||Y_tau(:, j)||_2 (prescribed accuracy
      relative to the sampled row block of H).
  R3  unknown r_l in s_l = r_l + m_l + p: start from a guess rhat = m_l / 2;
      when the truncated rank exceeds rhat the level is sampled again (next
      attempt counter) with rhat doubled, up to m_l.
  R4  Hermitian part: H^[0] and every diagonal block D^[l]_tau of the
      postprocessing are replaced by (A + A^*) / 2 before they are split,
      since the construction assumes H Hermitian.
"""
import numpy as np
import scipy.linalg as sla

from .philox import gaussian_matrix


def herm(a):
    return 0.5 * (a + a.conj().T)


def blockdiag(blocks):
    return sla.block_diag(*blocks) if blocks else np.zeros((0, 0), dtype=np.complex128)


class NotHPD(Exception):
    pass


class HSS:
    """Generators of a Hermitian HSS matrix with one rank per level.

    ranks[l], l = 0..Lh (ranks[0] = 0); U[l][t] is m_l x r_l for l = 1..Lh,
    with m_Lh = leaf and m_l = 2 r_{l+1}; B[l][t] = B_{alpha2,alpha1} of node t
    at level l (r_{l+1} x r_{l+1}), l = 0..Lh-1; D[t] leaf diagonal blocks.
    """

    def __init__(self, N, leaf, ranks, U, B, D):
        self.N, self.leaf = N, leaf
        self.Lh = int(round(np.log2(N // leaf)))
        if leaf << self.Lh != N or self.Lh < 1:
            raise ValueError("N must be leaf * 2^Lh with Lh >= 1")
        self.ranks, self.U, self.B, self.D = list(ranks), U, B, D

    def m(self, l):
        return self.leaf if l == self.Lh else 2 * self.ranks[l + 1]

    def dense(self):
        """Eq. 2.8: H^[0] = B^[0]; H^[l] = U^[l] H^[l-1] U^[l]* + B^[l]; + D at Lh."""
        def bfull(b):
            r = b.shape[0]
            z = np.zeros((r, r), dtype=np.complex128)
            return np.block([[z, b.conj().T], [b, z]])
        H = blockdiag([bfull(b) for b in self.B[0]])
        for l in range(1, self.Lh + 1):
            Ul = blockdiag(self.U[l])
            last = blockdiag(self.D) if l == self.Lh else blockdiag([bfull(b) for b in self.B[l]])
            H = Ul @ H @ Ul.conj().T + last
        return H

    def matvec(self, X):
        """H X through the telescoping factorization (Eq. 2.8), X of shape (N, k)."""
        X = np.asarray(X, dtype=np.complex128).reshape(self.N, -1)
        Lh, leaf = self.Lh, self.leaf
        xs = {Lh: [self.U[Lh][t].conj().T @ X[t * leaf:(t + 1) * leaf] for t in range(2 ** Lh)]}
        for l in range(Lh - 1, 0, -1):
            xs[l] = [self.U[l][t].conj().T @ np.vstack([xs[l + 1][2 * t], xs[l + 1][2 * t + 1]])
                     for t in range(2 ** l)]
        ys = {l: [np.zeros_like(v) for v in xs[l]] for l in xs}
        for l in range(0, Lh):
            for t in range(2 ** l):
                b = self.B[l][t]
                ys[l + 1][2 * t] += b.conj().T @ xs[l + 1][2 * t + 1]
                ys[l + 1][2 * t + 1] += b @ xs[l + 1][2 * t]
        for l in range(1, Lh):
            for t in range(2 ** l):
                v = self.U[l][t] @ ys[l][t]
                r = self.ranks[l + 1]
                ys[l + 1][2 * t] += v[:r]
                ys[l + 1][2 * t + 1] += v[r:]
        out = np.empty_like(X)
        for t in range(2 ** Lh):
            sl = slice(t * leaf, (t + 1) * leaf)
            out[sl] = self.D[t] @ X[sl] + self.U[Lh][t] @ ys[Lh][t]
        return out


# ---------------------------------------------------------------------------
# Section 3: black-box construction
# ---------------------------------------------------------------------------

def _expand(hss_U, ranks, Lh, leaf, X, l):
    """(U^[Lh] ... U^[l+1]) X for X with 2^l m_l rows (Section 3.2)."""
    for j in range(l + 1, Lh + 1):
        r = ranks[j]
        X = np.vstack([hss_U[j][t] @ X[t * r:(t + 1) * r] for t in range(2 ** j)])
    return X


def _compress(hss_U, ranks, Lh, leaf, Z, l):
    """(U^[l+1]* ... U^[Lh]*) Z (Section 3.2)."""
    for j in range(Lh, l, -1):
        m = leaf if j == Lh else 2 * ranks[j + 1]
        Z = np.vstack([hss_U[j][t].conj().T @ Z[t * m:(t + 1) * m] for t in range(2 ** j)])
    return Z


def build_blackbox(apply_H, N, leaf, p, tol, seed, rank_frac=0.5, stats=None):
    """Randomized HSS construction of a Hermitian H from products H X.

    apply_H(X) -> H X for X of shape (N, s).  Returns an HSS.
    """
    Lh = int(round(np.log2(N // leaf)))
    if leaf << Lh != N or Lh < 1:
        raise ValueError("N must be leaf * 2^Lh with Lh >= 1")
    ranks = [0] * (Lh + 1)
    U = [None] * (Lh + 1)
    Dchk = [None] * (Lh + 1)
    samples = 0
    for l in range(Lh, 0, -1):
        m = leaf if l == Lh else 2 * ranks[l + 1]
        nn = 2 ** l
        if m == 0:
            U[l] = [np.zeros((0, 0), dtype=np.complex128)] * nn
            Dchk[l] = [np.zeros((0, 0), dtype=np.complex128)] * nn
            continue
        rhat = max(1, min(m, int(round(rank_frac * m))))            # R3
        attempt = 0
        while True:
            s = rhat + m + p                                         # s_l = r_l + m_l + p
            Om = gaussian_matrix(seed, l, attempt, nn * m, s)
            Y = _compress(U, ranks, Lh, leaf, apply_H(_expand(U, ranks, Lh, leaf, Om, l)), l)
            samples += s
            qs, khat, pinvs = [], [], []
            for t in range(nn):
                Om_t = Om[t * m:(t + 1) * m]
                Y_t = Y[t * m:(t + 1) * m]
                # Gamma: orthonormal null basis of Omega_t from a complete QRCP of Omega_t^*
                Q, _, _ = sla.qr(Om_t.conj().T, pivoting=True)
                Gam = Q[:, m:]
                Qy, Ry, _ = sla.qr(Y_t @ Gam, mode="economic", pivoting=True)
                thr = tol * np.max(np.linalg.norm(Y_t, axis=0))      # R2
                khat.append(int(np.sum(np.abs(np.diag(Ry)) > thr)))
                qs.append(Qy)
                pinvs.append(np.linalg.pinv(Om_t))
            rl = max(khat)                                           # R1
            if rl > rhat and rhat < m:
                rhat = min(m, 2 * rhat)
                attempt += 1
                continue
            break
        ranks[l] = rl
        U[l] = [q[:, :rl] for q in qs]
        Dchk[l] = []
        for t in range(nn):
            Y_t = Y[t * m:(t + 1) * m]
            Ut = U[l][t]
            W = Y_t @ pinvs[t]                                       # (I - UU*) D = (I - UU*) Y Omega^+
            X = W - Ut @ (Ut.conj().T @ W)
            Dchk[l].append(X + Ut @ (Ut.conj().T @ X.conj().T))     # D-check (Section 3.1)
    # root: H^[0] from Y^[0] = H^[0] Omega^[0]
    m0 = 2 * ranks[1]
    if m0 > 0:
        Om0 = gaussian_matrix(seed, 0, 0, m0, m0 + p)
        Y0 = _compress(U, ranks, Lh, leaf, apply_H(_expand(U, ranks, Lh, leaf, Om0, 0)), 0)
        samples += m0 + p
        H0 = herm(Y0 @ np.linalg.pinv(Om0))                          # R4
    else:
        H0 = np.zeros((0, 0), dtype=np.complex128)
    # Section 3.3: top-down postprocessing
    Dcur = [H0]
    B = [None] * Lh
    for l in range(0, Lh):
        rc = ranks[l + 1]
        B[l] = []
        Dnext = []
        for t in range(2 ** l):
            Dt = herm(Dcur[t])                                       # R4
            B[l].append(Dt[rc:, :rc].copy())                         # B_{alpha2,alpha1} = A21
            for c, A in ((0, Dt[:rc, :rc]), (1, Dt[rc:, rc:])):
                a = 2 * t + c
                Ua = U[l + 1][a]
                Dnext.append(Dchk[l + 1][a] + Ua @ A @ Ua.conj().T)  # D_alpha = Dcheck + U A U*
        Dcur = Dnext
    D = [herm(d) for d in Dcur]
    if stats is not None:
        stats["samples"] = samples
        stats["ranks"] = list(ranks)
    return HSS(N, leaf, ranks, U, B, D)


def random_hss(N, leaf, ranks, rng, shift=None):
    """Random Hermitian HSS with given per-level ranks (for exact-recovery pins).

    U's have orthonormal columns; B and D are Gaussian; if `shift` is None the
    leaf blocks get a shift that makes the dense matrix positive definite.
    """
    Lh = int(round(np.log2(N // leaf)))
    ranks = list(ranks)

    def cg(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    U = [None] * (Lh + 1)
    for l in range(1, Lh + 1):
        m = leaf if l == Lh else 2 * ranks[l + 1]
        U[l] = [np.linalg.qr(cg(m, ranks[l]))[0] if ranks[l] else np.zeros((m, 0)) for _ in range(2 ** l)]
    B = [[cg(ranks[l + 1], ranks[l + 1]) for _ in range(2 ** l)] for l in range(Lh)]
    D = [herm(cg(leaf, leaf)) for _ in range(2 ** Lh)]
    hss = HSS(N, leaf, ranks, U, B, D)
    if shift is None:
        lam = np.linalg.eigvalsh(hss.dense())
        shift = max(0.0, -lam[0]) + 0.5 * (lam[-1] - lam[0]) + 1.0
    hss.D = [d + shift * np.eye(leaf) for d in D]
    return hss


# ---------------------------------------------------------------------------
# Section 2.4: ULV factorization and solve
# ---------------------------------------------------------------------------

def ql(Umat):
    """QL factorization: unitary Q with Q^* U = [0; Uh2], Uh2 lower triangular (Eq. 2.9)."""
    m, r = Umat.shape
    Qr, Rr = np.linalg.qr(Umat[::-1, ::-1], mode="complete")
    return Qr[::-1, ::-1], Rr[:r, :r][::-1, ::-1]


def _chol(A):
    try:
        return np.linalg.cholesky(A)
    except np.linalg.LinAlgError as e:
        raise NotHPD(str(e))


class ULV:
    """ULV factorization of a Hermitian positive definite HSS matrix."""

    def __init__(self, hss):
        self.hss = hss
        Lh = hss.Lh
        self.f = {}
        Dc = list(hss.D)
        Uc = list(hss.U[Lh])
        for l in range(Lh, 0, -1):
            Dh22, Uh2 = [], []
            for t in range(2 ** l):
                m, r = Uc[t].shape
                Q, Uh = ql(Uc[t])                                     # basis elimination
                Dq = Q.conj().T @ Dc[t] @ Q
                k = m - r
                L11 = _chol(Dq[:k, :k])                               # partial Cholesky
                Dh21 = sla.solve_triangular(L11, Dq[k:, :k].conj().T, lower=True).conj().T
                Dh22.append(Dq[k:, k:] - Dh21 @ Dh21.conj().T)        # Schur complement
                Uh2.append(Uh)
                self.f[(l, t)] = (Q, L11, Dh21, k)
            # merge into level l-1 (Eq. 2.12)
            Dc, Uc = [], []
            for t in range(2 ** (l - 1)):
                b = hss.B[l - 1][t]
                u1, u2 = Uh2[2 * t], Uh2[2 * t + 1]
                Dc.append(np.block([[Dh22[2 * t], u1 @ b.conj().T @ u2.conj().T],
                                    [u2 @ b @ u1.conj().T, Dh22[2 * t + 1]]]))
                if l - 1 >= 1:
                    Uc.append(blockdiag([u1, u2]) @ hss.U[l - 1][t])
        self.Lroot = _chol(Dc[0]) if Dc[0].size else np.zeros((0, 0), dtype=np.complex128)

    def solve(self, y):
        hss = self.hss
        Lh, leaf = hss.Lh, hss.leaf
        y = np.asarray(y, dtype=np.complex128)
        vec = y.ndim == 1
        y = y.reshape(hss.N, -1)
        yc = [y[t * leaf:(t + 1) * leaf] for t in range(2 ** Lh)]
        bh1 = {}
        for l in range(Lh, 0, -1):
            y2 = []
            for t in range(2 ** l):
                Q, L11, Dh21, k = self.f[(l, t)]
                yh = Q.conj().T @ yc[t]
                b1 = sla.solve_triangular(L11, yh[:k], lower=True)
                bh1[(l, t)] = b1
                y2.append(yh[k:] - Dh21 @ b1)
            yc = [np.vstack([y2[2 * t], y2[2 * t + 1]]) for t in range(2 ** (l - 1))]
        if self.Lroot.size:
            b = sla.solve_triangular(self.Lroot, yc[0], lower=True)
            cc = [sla.solve_triangular(self.Lroot.conj().T, b, lower=False)]
        else:
            cc = [np.zeros((0, y.shape[1]), dtype=np.complex128)]
        for l in range(1, Lh + 1):
            r = hss.ranks[l]
            nxt = []
            for t in range(2 ** l):
                Q, L11, Dh21, k = self.f[(l, t)]
                c2 = cc[t // 2][(t % 2) * r:(t % 2 + 1) * r]
                c1 = sla.solve_triangular(L11.conj().T, bh1[(l, t)] - Dh21.conj().T @ c2, lower=False)
                nxt.append(Q @ np.vstack([c1, c2]))
            cc = nxt
        out = np.vstack(cc)
        return out[:, 0] if vec else out
