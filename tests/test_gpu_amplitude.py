"""Variable amplitudes on the GPU (bf_build_amp) against the oracle with the same amplitude:
the Gaussian bumps of Section 5.1 (1D, phase with c = (2 + sin 2 pi x)/8) and the Hankel
amplitude of Section 5.3 (2D isotropic phase).  The amplitude enters only the middle factor,
so the apply must match the oracle's apply of the same factors to the FP32 tolerance 1e-5;
the solve (Algorithm 1) and PCG (Section 4.1) must stay within 2x of the oracle's error."""
import numpy as np
import pytest
import torch

from fio_inputs import bump_centers, crandn
from oracle.butterfly import Butterfly1D
from oracle.butterfly2d import Butterfly2D
from oracle.problem import Amplitude, K_rows, Phase
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bumps(n):
    c = bump_centers(n)
    return c, Amplitude("bumps", centers=c, sigma2=0.1, N=n)


@pytest.mark.parametrize("n", [256, 1024, 8192])
def test_bumps_apply_matches_oracle(n):
    from paper_2609_11520_b300 import BF
    c, amp = _bumps(n)
    ob = Butterfly1D(Phase("cabs8"), n, 16, amp=amp)
    gb = BF(n, 16, "cabs8", amp=("bumps", c, 0.1))
    f = crandn(n, 3, seed=n)
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL


def test_bumps_full_size_sampled_rows():
    """N = 2^16 against K itself (Eq. 1.2 with the amplitude) on sampled rows."""
    from paper_2609_11520_b300 import BF
    n = 1 << 16
    c, amp = _bumps(n)
    gb = BF(n, 16, "cabs8", amp=("bumps", c, 0.1))
    f = crandn(n, 2, seed=5)
    y = to_np(gb.apply(to_dev(f)))
    rows = np.random.default_rng(4).choice(n, 128, replace=False)
    assert rel(y[rows], K_rows(Phase("cabs8"), n, rows, amp) @ f) < TOL


@pytest.mark.parametrize("n", [16, 32, 64])
def test_hankel_apply_matches_oracle(n):
    from paper_2609_11520_b300 import BF
    ph = Phase("iso2d")
    ob = Butterfly2D(ph, n, 5, amp=Amplitude("hankel", phase=ph))
    gb = BF(n, 25, "iso2d", amp="hankel")
    f = crandn(n * n, 2, seed=n)
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL


def test_bumps_solve_and_pcg_match_oracle():
    from oracle.pcg import fio_pcg as oracle_pcg
    from oracle.solver import FIOSolver
    from paper_2609_11520_b300 import BF, HSS, fio_pcg, fio_solve
    n, leaf, p, tol, seed = 4096, 128, 10, 1e-3, 1
    c, amp = _bumps(n)
    S = FIOSolver(Phase("cabs8"), n, 16, leaf, p, tol, seed, amp=amp)
    bf = BF(n, 16, "cabs8", amp=("bumps", c, 0.1))
    g = HSS.from_samples(bf=bf, leaf=leaf, oversample=p, tol=tol, seed=seed).factor()
    f = crandn(n, 2, seed=0)
    u = S.bf.apply(f)
    e_o = rel(S.solve(u), f)
    e_g = rel(to_np(fio_solve(bf, g, to_dev(u))), f)
    assert e_g <= 2 * e_o + 1e-5, (e_g, e_o)
    xo, ito, _ = oracle_pcg(S, u, tol=1e-5)
    F, it, rr = fio_pcg(bf, g, to_dev(u), tol=1e-5, maxit=40)
    assert abs(it - int(ito.max())) <= 1 and max(rr) <= 1e-5, (it, ito)
    assert rel(to_np(F), f) <= 2 * rel(xo, f) + 2e-6


def test_hankel_solve_matches_oracle():
    from oracle.solver import FIOSolver2D
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    n = 32
    ph = Phase("iso2d")
    S = FIOSolver2D(ph, n, 5, 256, 10, 1e-3, 1, amp=Amplitude("hankel", phase=ph))
    bf = BF(n, 25, "iso2d", amp="hankel")
    g = HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=1).factor()
    f = crandn(n * n, 2, seed=0)
    u = S.bf.apply(f)
    e_o = rel(S.solve(u), f)
    e_g = rel(to_np(fio_solve(bf, g, to_dev(u))), f)
    assert e_g <= 2 * e_o + 1e-5, (e_g, e_o)


def test_amplitude_rejected_where_undefined():
    from paper_2609_11520_b300 import BF, FioError
    with pytest.raises(FioError):
        BF(64, 25, "elliptic2d", amp="hankel")        # the Hankel amplitude needs the iso phase
    with pytest.raises(FioError):
        BF(32, 25, "iso2d", amp=("bumps", bump_centers(1024), 0.1))   # bumps are 1D
    with pytest.raises(FioError):
        BF(1024, 16, "cabs8", amp=("bumps", bump_centers(1024), -1.0))
