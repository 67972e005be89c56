"""GPU parity of the HSS construction, ULV factorization and solve.

HSS generators are not unique (any orthonormal null basis, QRCP pivot order),
so parity is checked on what is unique: the reconstructed matrix G~ (through
hss_matvec), ranks where the true rank is exact, and solutions.
"""
import numpy as np
import pytest
import torch

from fio_inputs import crandn
from oracle.hss import ULV, build_blackbox, random_hss
from oracle.problem import Phase, dense_K
from oracle.solver import FIOSolver
from tests.gpu_util import hss_to_c_layout, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_11520_b300  # noqa: F401


def gpu_hss_from_oracle(h):
    from paper_2609_11520_b300 import HSS
    ranks, U, B, D = hss_to_c_layout(h)
    return HSS.from_generators(h.N, h.leaf, ranks, U, B, D)


CASES = [(512, 32, [0, 6, 5, 5, 4]), (256, 64, [0, 0, 0]), (128, 16, [0, 8, 8, 16]), (1024, 128, [0, 12, 10, 9])]


@pytest.mark.parametrize("N,leaf,ranks", CASES)
def test_matvec_matches_oracle(N, leaf, ranks):
    h = random_hss(N, leaf, ranks, np.random.default_rng(N))
    g = gpu_hss_from_oracle(h)
    X = crandn(N, 3, seed=1)
    assert rel(to_np(g.matvec(to_dev(X))), h.matvec(X)) < 1e-5


@pytest.mark.parametrize("N,leaf,ranks", CASES)
def test_ulv_solve_matches_oracle(N, leaf, ranks):
    h = random_hss(N, leaf, ranks, np.random.default_rng(N + 1))
    g = gpu_hss_from_oracle(h).factor()
    Y = crandn(N, 5, seed=2)
    ref = ULV(h).solve(Y)
    assert rel(ref, np.linalg.solve(h.dense(), Y)) < 1e-10
    assert rel(to_np(g.solve(to_dev(Y))), ref) < 1e-4


SOLVE_SHAPES = [(2048, 128, [0, 4, 6, 8, 10]),              # upper levels m = 12..20: one fused launch
                (4096, 64, [0, 20, 24, 40, 36, 30, 20]),      # m = 48, 80, 72, 60, 40 and leaves of 64
                (1024, 256, [0, 200, 150])]                   # m = 300, 256 on 2 and 4 nodes: sliced inner index


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 9, 16, 64, 67])
@pytest.mark.parametrize("shape", range(len(SOLVE_SHAPES)))
def test_ulv_solve_every_width(shape, k):
    """Each solve kernel: k <= 8 skinny node products plus the fused upper levels and root
    (m_l <= 64), k > 8 the wide products (m >= 32; few nodes of large m: inner index cut into
    slices summed by a second kernel) or the tiled ones (m < 32); ragged k."""
    N, leaf, ranks = SOLVE_SHAPES[shape]
    h = random_hss(N, leaf, ranks, np.random.default_rng(N + k))
    g = gpu_hss_from_oracle(h).factor()
    Y = crandn(N, k, seed=k)
    assert rel(to_np(g.solve(to_dev(Y))), ULV(h).solve(Y)) < 1e-4


@pytest.mark.parametrize("k", [9, 32, 64, 67])
@pytest.mark.parametrize("shape", [1, 2])
def test_ulv_tensor_core_products_match_cuda_cores(shape, k):
    """k > 8: the tcgen05 node products (FP16 hi/lo parts, power-of-two scales) against the FP32
    CUDA-core products on the same factorization.  Each part product is exact to 2^-22 of its
    row/column scale and an output sums K = 2 m_l (up to 600) of them, so the two paths differ
    by about sqrt(K) 2^-22 ~ 6e-6 relative: bound 2e-5.  Parity with the oracle stays 1e-4."""
    N, leaf, ranks = SOLVE_SHAPES[shape]
    h = random_hss(N, leaf, ranks, np.random.default_rng(7 * N + k))
    g = gpu_hss_from_oracle(h).factor()
    Y = to_dev(crandn(N, k, seed=100 + k))
    b = to_np(g.solve(Y))
    a = to_np(g.set_solve_path("tensor_cores").solve(Y))
    assert rel(a, b) < 2e-5
    assert rel(a, ULV(h).solve(to_np(Y))) < 1e-4


def test_ulv_rejects_indefinite():
    from paper_2609_11520_b300 import FioError
    h = random_hss(128, 32, [0, 4, 4], np.random.default_rng(3), shift=0.0)
    h.D = [d - 1e3 * np.eye(32) for d in h.D]
    g = gpu_hss_from_oracle(h)
    with pytest.raises(FioError, match="FIO_ENOTHPD"):
        g.factor()


@pytest.mark.parametrize("N,leaf,ranks", [(512, 32, [0, 6, 5, 5, 4]), (1024, 64, [0, 10, 9, 8, 7]),
                                          (256, 32, [0, 0, 2, 3])])
def test_blackbox_recovers_exact_hss(N, leaf, ranks):
    """Dense sampler on an exact HSS matrix: ranks recovered, G~ equal to H in FP32."""
    from paper_2609_11520_b300 import HSS
    h = random_hss(N, leaf, ranks, np.random.default_rng(N + 5))
    Hd = h.dense()
    dense = torch.from_numpy(Hd.astype(np.complex64)).cuda()
    g = HSS.from_samples(dense=dense, leaf=leaf, oversample=10, tol=1e-5, seed=9)
    info = g.info()
    assert info["ranks"] == ranks
    X = crandn(N, 4, seed=4)
    assert rel(to_np(g.matvec(to_dev(X))), Hd @ X) < 2e-5
    # the oracle, same sampler, same seed: same ranks, same matrix
    o = build_blackbox(lambda Z: Hd @ Z, N, leaf, 10, 1e-5, 9)
    assert o.ranks == ranks
    g.factor()
    Y = crandn(N, 2, seed=8)
    assert rel(to_np(g.solve(to_dev(Y))), np.linalg.solve(Hd, Y)) < 1e-4


@pytest.mark.parametrize("n,leaf", [(1024, 64), (4096, 128)])
def test_fio_pipeline_matches_oracle(n, leaf):
    """Config-1 shape at tol 1e-3 (FP32 GPU): e_cHSS and e_direct no worse than 2x the oracle's."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    tol, p, seed = 1e-3, 10, 1
    S = FIOSolver(Phase("cabs"), n, 16, leaf, p, tol, seed)
    bf = BF(n, 16)
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed)
    ginfo = g.info()
    f = crandn(n, 4, seed=0)
    u = S.bf.apply(f)                                   # u = K~ f_true (Section 5), oracle-side
    x = crandn(n, 2, seed=3)
    GKx = S.bf.adjoint(S.bf.apply(x))
    e_hss_o = rel(S.hss.matvec(x), GKx)
    e_hss_g = rel(to_np(g.matvec(to_dev(x))), GKx)
    assert e_hss_g <= 2 * e_hss_o + 1e-5, (e_hss_g, e_hss_o, ginfo["ranks"], S.stats["ranks"])
    g.factor()
    e_o = rel(S.solve(u), f)
    fg = to_np(fio_solve(bf, g, to_dev(u)))
    e_g = rel(fg, f)
    assert e_g <= 2 * e_o + 1e-5, (e_g, e_o)
    # refinement does not make it worse
    fr = to_np(fio_solve(bf, g, to_dev(u), refine_steps=2))
    assert rel(fr, f) <= e_g * 1.01 + 1e-6


def test_dft_special_case():
    """Phi = x.xi: K^* K = N I, so G~ truncates to block-diagonal N I and f = K^* u / N."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    n = 2048
    bf = BF(n, 16, "dft")
    g = HSS.from_samples(bf=bf, leaf=64, oversample=10, tol=1e-3, seed=3)
    assert g.info()["ranks"] == [0] * 6
    g.factor()
    f = crandn(n, 2, seed=1)
    u = n * np.fft.ifft(np.fft.ifftshift(f, axes=0), axis=0)   # K f (closed form)
    assert rel(to_np(fio_solve(bf, g, to_dev(u))), f) < 1e-5
