"""Pins for the oracle's HSS construction, ULV factorization and FIO solve (CPU).

Anchors: the nested-basis recursion of Def. 2.2 evaluated independently of the
telescoping code (Eq. 2.8), dense linear solves (numpy LAPACK), exact recovery
of HSS matrices built from known generators, the DFT special case K^* K = N I,
and dense LU of K for the end-to-end solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.butterfly import Butterfly1D
from oracle.hss import HSS, ULV, NotHPD, build_blackbox, random_hss
from oracle.philox import gaussian_matrix, philox4x32_10
from oracle.problem import Phase, dense_K
from oracle.solver import FIOSolver, rel_err

RNG = np.random.default_rng(99)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ---- Philox (input generator of the test matrices) ---------------------------

def test_philox_known_answers():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = np.array([int(w, 16) for w in row], dtype=np.uint64).astype(np.uint32)
        out = philox4x32_10(v[:4], v[4:6])
        assert list(out) == list(v[6:10])


def test_gaussian_moments_and_counter_independence():
    om = gaussian_matrix(5, 3, 0, 400, 300)
    for part in (om.real, om.imag):
        assert abs(part.mean()) < 0.01
        assert abs(part.var() - 1.0) < 0.02
    assert abs(np.mean(om.real * om.imag)) < 0.01
    # different level / attempt / seed give unrelated matrices; same counters repeat
    assert np.array_equal(om, gaussian_matrix(5, 3, 0, 400, 300))
    for other in (gaussian_matrix(5, 2, 0, 400, 300), gaussian_matrix(5, 3, 1, 400, 300),
                  gaussian_matrix(6, 3, 0, 400, 300)):
        assert abs(np.vdot(om, other)) / om.size < 0.02
    # a sub-block of a larger matrix is the same matrix (entries depend on (row, col) only)
    assert np.array_equal(gaussian_matrix(5, 3, 0, 10, 7), om[:10, :7])


# ---- Def. 2.2 versus Eq. 2.8 --------------------------------------------------

def dense_by_definition(hss):
    """Def. 2.2: D_tau = [[D1, U1big B^* U2big^*], [U2big B U1big^*, D2]], U_big nested."""
    Lh = hss.Lh
    Dl = list(hss.D)
    Ubig = list(hss.U[Lh])
    for l in range(Lh - 1, -1, -1):
        nD, nU = [], []
        for t in range(2 ** l):
            b = hss.B[l][t]
            u1, u2 = Ubig[2 * t], Ubig[2 * t + 1]
            nD.append(np.block([[Dl[2 * t], u1 @ b.conj().T @ u2.conj().T],
                                [u2 @ b @ u1.conj().T, Dl[2 * t + 1]]]))
            if l > 0:
                nU.append(sla.block_diag(u1, u2) @ hss.U[l][t])
        Dl, Ubig = nD, nU
    return Dl[0]


@pytest.mark.parametrize("ranks", [[0, 3, 4, 5], [0, 0, 2, 1], [0, 5, 5, 6]])
def test_telescoping_equals_definition(ranks):
    hss = random_hss(256, 32, ranks, RNG)
    Hd = hss.dense()
    assert np.linalg.norm(Hd - dense_by_definition(hss)) / np.linalg.norm(Hd) < 1e-14
    assert np.linalg.norm(Hd - Hd.conj().T) < 1e-12 * np.linalg.norm(Hd)
    X = crandn(256, 4)
    assert np.linalg.norm(hss.matvec(X) - Hd @ X) / np.linalg.norm(Hd @ X) < 1e-14


# ---- P5: exact recovery ----------------------------------------------------------

@pytest.mark.parametrize("N,leaf,ranks", [(512, 32, [0, 6, 5, 5, 4]),
                                          (256, 64, [0, 7, 9]),
                                          (256, 32, [0, 0, 2, 3])])
def test_blackbox_recovers_exact_hss(N, leaf, ranks):
    H = random_hss(N, leaf, ranks, RNG)
    Hd = H.dense()
    st = {}
    G = build_blackbox(lambda X: Hd @ X, N, leaf, 10, 1e-10, 11, stats=st)
    assert st["ranks"] == ranks
    assert np.linalg.norm(G.dense() - Hd) / np.linalg.norm(Hd) < 1e-12


def test_blackbox_rank_guess_too_small_is_redone():
    """Leaf rank 22 > initial guess 16 = m/2: the level is sampled again (R3)."""
    N, leaf = 128, 32
    H = random_hss(N, leaf, [0, 10, 22], RNG)
    Hd = H.dense()
    st = {}
    G = build_blackbox(lambda X: Hd @ X, N, leaf, 8, 1e-10, 3, stats=st)
    assert st["ranks"][2] == 22
    assert np.linalg.norm(G.dense() - Hd) / np.linalg.norm(Hd) < 1e-12


def test_blackbox_truncates_to_tolerance():
    """A perturbation below tol * scale is truncated away; the error stays O(tol)."""
    N, leaf = 256, 32
    H = random_hss(N, leaf, [0, 3, 3, 3], RNG)
    Hd = H.dense()
    E = crandn(N, N)
    E = 1e-7 * np.linalg.norm(Hd, 2) * (E + E.conj().T) / np.linalg.norm(E + E.conj().T, 2)
    st = {}
    G = build_blackbox(lambda X: (Hd + E) @ X, N, leaf, 10, 1e-4, 5, stats=st)
    assert st["ranks"] == [0, 3, 3, 3]
    assert np.linalg.norm(G.dense() - Hd) / np.linalg.norm(Hd) < 1e-5


# ---- P6: ULV exactness -------------------------------------------------------------

@pytest.mark.parametrize("N,leaf,ranks", [(512, 32, [0, 6, 5, 5, 4]), (256, 64, [0, 0, 0]),
                                          (128, 16, [0, 8, 8, 16])])
def test_ulv_solve_equals_dense_solve(N, leaf, ranks):
    H = random_hss(N, leaf, ranks, RNG)
    Hd = H.dense()
    Y = crandn(N, 3)
    C = ULV(H).solve(Y)
    ref = np.linalg.solve(Hd, Y)
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(Hd @ C - Y) / np.linalg.norm(Y) < 1e-12


def test_ulv_rejects_indefinite():
    H = random_hss(128, 32, [0, 4, 4], RNG, shift=0.0)
    H.D = [d - 1e3 * np.eye(32) for d in H.D]
    with pytest.raises(NotHPD):
        ULV(H)


def test_ql_elimination():
    from oracle.hss import ql
    U = np.linalg.qr(crandn(40, 7))[0]
    Q, Uh = ql(U)
    Z = Q.conj().T @ U
    assert np.allclose(Q.conj().T @ Q, np.eye(40), atol=1e-13)
    assert np.max(np.abs(Z[:33])) < 1e-13
    assert np.allclose(Z[33:], Uh, atol=1e-13)
    assert np.allclose(np.triu(Uh, 1), 0, atol=1e-13)


# ---- DFT special case: K^* K = N I ------------------------------------------------------

def test_dft_hss_is_block_diagonal_and_solve_is_scaled_adjoint():
    n = 512
    S = FIOSolver(Phase("dft"), n, 16, 64, 10, 1e-3, 4)
    assert S.stats["ranks"] == [0, 0, 0, 0]
    for d in S.hss.D:
        assert np.allclose(d, n * np.eye(64), atol=1e-8 * n)
    f = crandn(n)
    u = dense_K(Phase("dft"), n) @ f
    assert rel_err(S.solve(u), f) < 1e-10


# ---- P7: end to end -------------------------------------------------------------------

def test_fio_solve_config1_shape_tight_tolerance():
    """N = 1024, BF rank 16, leaf 64, tol 1e-8, u = K f_true with dense K."""
    n = 1024
    ph = Phase("cabs")
    S = FIOSolver(ph, n, 16, 64, 10, 1e-8, 1)
    K = dense_K(ph, n)
    f = crandn(n)
    u = K @ f
    fh = S.solve(u)
    f_lu = np.linalg.solve(K, u)
    assert rel_err(f_lu, f) < 1e-10
    assert rel_err(fh, f) < 1e-7
    # G~ is HPD and close to K^* K
    Gd = S.hss.dense()
    assert np.linalg.eigvalsh(0.5 * (Gd + Gd.conj().T))[0] > 0
    KK = K.conj().T @ K
    assert np.linalg.norm(Gd - KK) / np.linalg.norm(KK) < 1e-7


def test_fio_solve_hss_tolerance_band():
    """tol 1e-3: e_cHSS and e_direct of order 1e-4 (Table 5.1 band, different amplitude)."""
    n = 1024
    S = FIOSolver(Phase("cabs"), n, 16, 64, 10, 1e-3, 2)
    f = crandn(n, 2)
    u = S.bf.apply(f)
    e = rel_err(S.solve(u), f)
    assert 1e-6 < e < 2e-3
    x = crandn(n, 2)
    ref = S.bf.adjoint(S.bf.apply(x))
    assert rel_err(S.hss.matvec(x), ref) < 2e-3
