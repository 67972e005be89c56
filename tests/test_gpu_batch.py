"""Batched online solves over operators of uneven size (grouped launches, CUDA graph).

Each mode must give the same solutions as one fio_solve per operator (same
arithmetic, per-column independent), the graph replay must see in-place
updates of its input buffers, and a new shape must replan.  fio_solve itself
is checked against the oracle in test_gpu_hss.py.
"""
import numpy as np
import pytest
import torch

from fio_inputs import batched_operators, crandn
from tests.gpu_util import rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, HSS
    sizes = [(1 << 12, 0.55), (1 << 13, 0.8), (1 << 14, 0.95), (1 << 12, 0.7), (1 << 15, 0.6), (1 << 17, 1.0),
             (1 << 11, 0.9)]
    out = []
    for i, (n, s) in enumerate(sizes):
        bf = BF(n, 16, "cabs", s)
        h = HSS.from_samples(bf=bf, leaf=128 if n >= 4096 else 64, oversample=10, tol=1e-3, seed=10 + i).factor()
        out.append((bf, h))
    return out


def test_batch_modes_equal_per_operator(ops):
    from paper_2609_11520_b300 import Batch, fio_solve
    ks = [16, 5, 16, 1, 9, 3, 7]
    Us = [to_dev(crandn(bf.n, k, seed=100 + i)) for i, ((bf, _), k) in enumerate(zip(ops, ks))]
    refs = [to_np(fio_solve(bf, h, U)) for (bf, h), U in zip(ops, Us)]
    b = Batch(ops)
    for mode in ("per_operator", "grouped", "graph", "persistent"):
        b.set_mode(mode)
        Fs = [torch.empty_like(U) for U in Us]
        for rep in range(3):   # graph: eager + capture, then replays
            b.solve(Us, Fs)
        torch.cuda.synchronize()
        for F, ref in zip(Fs, refs):
            assert rel(to_np(F), ref) < 1e-5, mode


def test_graph_replay_sees_new_inputs_and_replans(ops):
    from paper_2609_11520_b300 import Batch, fio_solve
    b = Batch(ops).set_mode("graph")
    ks = [4] * len(ops)
    Us = [to_dev(crandn(bf.n, k, seed=200 + i)) for i, ((bf, _), k) in enumerate(zip(ops, ks))]
    Fs = [torch.empty_like(U) for U in Us]
    b.solve(Us, Fs)
    b.solve(Us, Fs)
    for i, U in enumerate(Us):   # new data in the same buffers
        U.copy_(to_dev(crandn(ops[i][0].n, 4, seed=300 + i)))
    b.solve(Us, Fs)
    torch.cuda.synchronize()
    for (bf, h), U, F in zip(ops, Us, Fs):
        assert rel(to_np(F), to_np(fio_solve(bf, h, U))) < 1e-5
    Us2 = [to_dev(crandn(bf.n, 2, seed=400 + i)) for i, (bf, _) in enumerate(ops)]
    Fs2 = b.solve(Us2)
    torch.cuda.synchronize()
    for (bf, h), U, F in zip(ops, Us2, Fs2):
        assert rel(to_np(F), to_np(fio_solve(bf, h, U))) < 1e-5


def test_autotune_reports_every_candidate(ops):
    from paper_2609_11520_b300 import Batch
    b = Batch(ops[:4])
    Us = [to_dev(crandn(bf.n, 8, seed=500 + i)) for i, (bf, _) in enumerate(ops[:4])]
    Fs = [torch.empty_like(U) for U in Us]
    rep = b.autotune(Us, Fs, reps=2)
    assert "grouped launches in a CUDA graph" in rep and "chosen:" in rep
    b.solve(Us, Fs)


def test_batched_workload_operators():
    """The batched workload's operator list: 32 operators, N in 2^12..2^17, s in [0.5, 1]."""
    ops_ = batched_operators()
    assert len(ops_) == 32
    assert {n for n, _ in ops_} <= {1 << e for e in range(12, 18)}
    assert all(0.5 <= s <= 1.0 for _, s in ops_)


@pytest.mark.parametrize("mode", ["grouped", "graph", "persistent"])
def test_batch_matches_oracle(mode):
    """Grouped launches and their graph replay against the FP64 oracle (Algorithm 1 per operator):
    three operators of different N and s, each with its own oracle FIOSolver on the same Philox
    test matrices.  Per operator the batched solve error against f_true is at most 2x the
    oracle's, and the solution equals the GPU ULV solve of the oracle's K~^* u (which checks the
    grouped K~^* half passes element-wise through the linear solve)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.problem import Phase
    from oracle.solver import FIOSolver
    from paper_2609_11520_b300 import BF, HSS, Batch
    cases = [(1 << 11, 0.9, 64, 21), (1 << 12, 0.55, 128, 22), (1 << 13, 0.8, 128, 23)]
    ops, oracles, fs, us = [], [], [], []
    for i, (n, s, leaf, seed) in enumerate(cases):
        S = FIOSolver(Phase("cabs", s=s), n, 16, leaf, 10, 1e-3, seed)
        bf = BF(n, 16, "cabs", s)
        h = HSS.from_samples(bf=bf, leaf=leaf, oversample=10, tol=1e-3, seed=seed).factor()
        f = crandn(n, 3 + 2 * i, seed=600 + i)
        ops.append((bf, h))
        oracles.append(S)
        fs.append(f)
        us.append(S.bf.apply(f))
    b = Batch(ops).set_mode(mode)
    Us = [to_dev(u) for u in us]
    Fs = [torch.empty_like(U) for U in Us]
    for _ in range(3):   # graph: eager + capture, then a replay
        b.solve(Us, Fs)
    torch.cuda.synchronize()
    for (bf, h), S, f, u, F in zip(ops, oracles, fs, us, Fs):
        e_o = rel(S.solve(u), f)
        e_g = rel(to_np(F), f)
        assert e_g <= 2 * e_o + 1e-5, (bf.n, e_g, e_o)
        ref = to_np(h.solve(to_dev(S.bf.adjoint(u))))
        assert rel(to_np(F), ref) < 1e-4, bf.n


def test_persistent_replans_and_sees_new_inputs(ops):
    from paper_2609_11520_b300 import Batch, device_status, fio_solve
    b = Batch(ops).set_mode("persistent")
    Us = [to_dev(crandn(bf.n, 3, seed=700 + i)) for i, (bf, _) in enumerate(ops)]
    Fs = b.solve(Us)
    for i, U in enumerate(Us):
        U.copy_(to_dev(crandn(ops[i][0].n, 3, seed=800 + i)))
    b.solve(Us, Fs)
    torch.cuda.synchronize()
    for (bf, h), U, F in zip(ops, Us, Fs):
        assert rel(to_np(F), to_np(fio_solve(bf, h, U))) < 1e-5
    device_status()   # no dependency wait ran out


def test_persistent_wait_runs_out_and_is_reported():
    """Failure detection without a GPU fault: a work item whose prerequisite never completes must
    end its bounded wait, let the kernel finish, and surface as FIO_ETIMEOUT; the flag clears."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2609_11520_b300 import _lib, device_status
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _lib.lib.fio_selftest_wait_timeout(st) == _lib.FIO_ETIMEOUT
    device_status()   # cleared: raises nothing
    x = torch.ones(4, device="cuda")
    assert float((x + 1).sum()) == 8.0   # the context is still usable
