"""GPU parity of bf_build / bf_apply against the FP64 oracle (Section 2.2, Eq. 2.1).

Tolerance: rel-l2 <= 1e-5 for the FP32-complex apply against the oracle's
apply of the same factors (both use the factor definitions of Section 2.2).
"""
import numpy as np
import pytest
import torch

from fio_inputs import crandn
from oracle.butterfly import Butterfly1D
from oracle.problem import K_rows, Phase
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_11520_b300  # noqa: F401  (fails loudly if the library is missing)


@pytest.mark.parametrize("path", ["per_level", "auto"])
@pytest.mark.parametrize("kind,s", [("cabs", 1.0), ("dft", 1.0), ("cabs", 0.6)])
@pytest.mark.parametrize("n", [16, 64, 128, 256, 2048, 8192])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_bf_apply_matches_oracle(kind, s, n, k, path):
    from paper_2609_11520_b300 import BF
    ob = Butterfly1D(Phase(kind, s), n, 16)
    gb = BF(n, 16, kind, s).set_path(path)
    f = crandn(n, k, seed=n + k)
    y_ref = ob.apply(f)
    y = to_np(gb.apply(to_dev(f)))
    assert rel(y, y_ref) < TOL
    g = crandn(n, k, seed=7 * n + k)
    x_ref = ob.adjoint(g)
    x = to_np(gb.adjoint(to_dev(g)))
    assert rel(x, x_ref) < TOL


@pytest.mark.parametrize("r", [4, 9, 16])
def test_bf_apply_other_ranks(r):
    from paper_2609_11520_b300 import BF
    n = 1024
    ob = Butterfly1D(Phase("cabs"), n, r)
    gb = BF(n, r)
    f = crandn(n, 2, seed=r)
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL


@pytest.mark.parametrize("path", ["per_level", "fused"])
def test_bf_apply_column_blocks_with_leading_dimension(path):
    """k ragged (67 columns crosses the 64-column chunk), rows padded to ld > N."""
    from paper_2609_11520_b300 import BF
    n, k, ld = 512, 67, 600
    ob = Butterfly1D(Phase("cabs"), n, 16)
    gb = BF(n, 16).set_path(path)
    f = crandn(n, k, seed=3)
    X = torch.zeros(k, ld, dtype=torch.complex64, device="cuda")
    X[:, :n] = to_dev(f)
    Y = torch.full((k, ld), 7 + 7j, dtype=torch.complex64, device="cuda")
    gb.apply(X[:, :n], out=Y[:, :n])
    assert rel(to_np(Y[:, :n]), ob.apply(f)) < TOL
    assert torch.all(Y[:, n:] == 7 + 7j)   # padding untouched


def test_bf_apply_empty_block():
    from paper_2609_11520_b300 import BF
    gb = BF(256, 16)
    X = torch.zeros(0, 256, dtype=torch.complex64, device="cuda")
    assert gb.apply(X).shape == (0, 256)


@pytest.mark.parametrize("path", ["per_level", "fused", "fused_v2"])
def test_bf_apply_16384_elementwise(path):
    from paper_2609_11520_b300 import BF
    n = 1 << 14
    ob = Butterfly1D(Phase("cabs"), n, 16)
    gb = BF(n, 16).set_path(path)
    f = crandn(n, 1, seed=11)
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL


def test_bf_apply_full_size_sampled_rows_and_dft():
    """N = 2^16 (the benchmark operator): sampled rows of K from Eq. 1.2, DFT closed form."""
    from paper_2609_11520_b300 import BF
    n = 1 << 16
    gb = BF(n, 16)
    f = crandn(n, 2, seed=5)
    y = to_np(gb.apply(to_dev(f)))
    rows = np.random.default_rng(0).choice(n, 256, replace=False)
    ref = K_rows(Phase("cabs"), n, rows) @ f
    assert rel(y[rows], ref) < TOL
    # adjoint: sampled columns of K^* are conjugated rows of K^T; use the identity <K x, y> = <x, K^* y>
    g = crandn(n, 1, seed=6)[:, 0]
    lhs = np.vdot(g, y[:, 0])
    rhs = np.vdot(to_np(gb.adjoint(to_dev(g))), f[:, 0])
    assert abs(lhs - rhs) / abs(lhs) < TOL
    gd = BF(n, 16, "dft")
    yd = to_np(gd.apply(to_dev(f)))
    ref_d = n * np.fft.ifft(np.fft.ifftshift(f, axes=0), axis=0)
    assert rel(yd, ref_d) < TOL
    xd = to_np(gd.adjoint(to_dev(f)))
    assert rel(xd, np.fft.fftshift(np.fft.fft(f, axis=0), axes=0)) < TOL


@pytest.mark.parametrize("n", [1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18])
def test_fused_equals_per_level(n):
    """The kernel paths agree at every size of the batched/serving workloads: the CUDA-core paths
    (per-level, fused_v2, fused_simt) to FP32 rounding (2e-6), the staged fused path with its
    tensor-core transfer levels (FP16 hi + lo parts, 22 significand bits, FP32 accumulation)
    to 5e-6."""
    from paper_2609_11520_b300 import BF
    gb = BF(n, 16)
    X = to_dev(crandn(n, 5, seed=n % 977))
    for adj in (False, True):
        a = to_np(gb.set_path("fused").apply(X, adjoint=adj))
        b = to_np(gb.set_path("per_level").apply(X, adjoint=adj))
        c = to_np(gb.set_path("fused_v2").apply(X, adjoint=adj))
        d = to_np(gb.set_path("fused_simt").apply(X, adjoint=adj))
        assert rel(a, b) < 5e-6
        assert rel(c, b) < 2e-6
        assert rel(d, b) < 2e-6


def test_bf_set_path_rejects_unsupported():
    from paper_2609_11520_b300 import BF, FioError
    with pytest.raises(FioError):
        BF(1024, 9).set_path("fused")


def test_bf_info_levels():
    from paper_2609_11520_b300 import BF
    info = BF(1 << 16, 16).info()
    assert (info["L"], info["h"], info["sU"], info["sV"]) == (16, 8, 13, 3)
    assert info["table_bytes"] > 0
