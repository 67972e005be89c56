"""Tensor-core transfer levels (tcgen05, FP32 accumulation in tensor memory) against the
FP64 oracle and against the CUDA-core FP32 kernels of the same fused pass.

The FP32 setting splits both GEMM operands into FP16 parts (hi*hi + hi*lo + lo*hi, rows
scaled by exact powers of two), which must hold the FP32 tolerance of the BF apply (rel-l2
<= 1e-5 against the oracle's apply of the same factors, Section 2.2 / Eq. 2.1); the split
setting uses BF16 parts (tolerance 1e-4).  Sizes cover every pair count per CTA of the
staged kernels (64 .. 512, odd L included), ragged column counts (the last CTA of a launch
holds fewer columns), inputs scaled far from unit magnitude (the FP16 row scaling), and the
device flag of the bounded MMA waits.
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
TOL_SPLIT = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_11520_b300  # noqa: F401


def _check_device():
    from paper_2609_11520_b300 import device_status
    device_status()


@pytest.mark.parametrize("n", [1 << 12, 1 << 13, 1 << 14, 1 << 15])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("kind,s", [("cabs", 1.0), ("cabs", 0.55), ("dft", 1.0)])
def test_tc_apply_matches_oracle(n, k, kind, s):
    from paper_2609_11520_b300 import BF
    ob = Butterfly1D(Phase(kind, s), n, 16)
    gb = BF(n, 16, kind, s)   # default: staged fused kernels, tensor-core transfer levels
    f = crandn(n, k, seed=n + 3 * k)
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    g = crandn(n, k, seed=n + 5 * k)
    assert rel(to_np(gb.adjoint(to_dev(g))), ob.adjoint(g)) < TOL
    _check_device()


@pytest.mark.parametrize("n", [1 << 16, 1 << 17, 1 << 18])
def test_tc_equals_cuda_core_pass_full_size(n):
    """Same fused pass, transfer levels on the tensor cores vs FP32 FMA, ragged k = 7 (the last
    CTA holds fewer columns).  FP16 hi + lo parts carry 22 of FP32's 24 significand bits and the
    tensor core accumulates in FP32, so the two differ by a few 1e-6 over ten levels (measured
    2.0e-6 at N = 2^16): bound 5e-6, half the FP32 tolerance against the oracle."""
    from paper_2609_11520_b300 import BF
    gb = BF(n, 16)
    gs = BF(n, 16).set_path("fused_simt")
    X = to_dev(crandn(n, 7, seed=11))
    for adj in (False, True):
        a = gb.apply(X, adjoint=adj)
        b = gs.apply(X, adjoint=adj)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < 5e-6, (n, adj)
    _check_device()


@pytest.mark.parametrize("n", [1 << 16, 1 << 17])
def test_tc_full_size_sampled_rows(n):
    """Full size against K itself on sampled rows (the BF error at r = 16 is ~1e-13), and the
    adjoint identity <K~ f, g> = <f, K~^* g>."""
    from paper_2609_11520_b300 import BF
    gb = BF(n, 16)
    f = crandn(n, 3, seed=5)
    y = to_np(gb.apply(to_dev(f)))
    rows = np.random.default_rng(2).choice(n, 192, replace=False)
    assert rel(y[rows], K_rows(Phase("cabs"), n, rows) @ f) < TOL
    g = crandn(n, 1, seed=6)[:, 0]
    lhs = np.vdot(g, y[:, 0])
    rhs = np.vdot(to_np(gb.adjoint(to_dev(g))), f[:, 0])
    assert abs(lhs - rhs) / abs(lhs) < TOL
    _check_device()


@pytest.mark.parametrize("scale", [1e-12, 1e-3, 1e4, 1e12])
def test_tc_row_scaling_far_from_unit(scale):
    """FP16 parts with per-row power-of-two scaling: relative accuracy independent of the input
    magnitude (unscaled FP16 would overflow above 6.5e4 and lose everything below 6e-8)."""
    from paper_2609_11520_b300 import BF
    n = 1 << 13
    ob = Butterfly1D(Phase("cabs"), n, 16)
    gb = BF(n, 16)
    f = crandn(n, 2, seed=9) * scale
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL
    _check_device()


def test_tc_mixed_magnitudes_in_one_vector():
    """Entries spanning 1e-6 .. 1e6 inside one vector: the rel-l2 bound still holds."""
    from paper_2609_11520_b300 import BF
    n = 1 << 14
    ob = Butterfly1D(Phase("cabs"), n, 16)
    gb = BF(n, 16)
    f = crandn(n, 2, seed=10) * np.logspace(-6, 6, n)[:, None]
    assert rel(to_np(gb.apply(to_dev(f))), ob.apply(f)) < TOL
    assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL
    _check_device()


@pytest.mark.parametrize("n", [1 << 12, 1 << 15, 1 << 18])
def test_tc_split_bf16_matches_oracle(n):
    from paper_2609_11520_b300 import BF
    gb = BF(n, 16).set_precision("split_bf16")
    f = crandn(n, 4, seed=12)
    y = to_np(gb.apply(to_dev(f)))
    if n <= 1 << 15:
        ob = Butterfly1D(Phase("cabs"), n, 16)
        assert rel(y, ob.apply(f)) < TOL_SPLIT
        assert rel(to_np(gb.adjoint(to_dev(f))), ob.adjoint(f)) < TOL_SPLIT
    else:
        rows = np.random.default_rng(3).choice(n, 128, replace=False)
        assert rel(y[rows], K_rows(Phase("cabs"), n, rows) @ f) < TOL_SPLIT
    _check_device()
