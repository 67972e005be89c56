"""Serving loop: continuous batching over resident operators.

Every request's result inside a coalesced block must equal the same request
solved alone (columns are independent in every kernel), all requests must
complete under a tight HBM budget, and blocks must actually coalesce.
"""
import numpy as np
import pytest
import torch

from fio_inputs import poisson_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_11520_b300 import BF, HSS
    out = {}
    for i, (n, s) in enumerate([(4096, 1.0), (8192, 0.7), (1 << 14, 0.9)]):
        bf = BF(n, 16, "cabs", s)
        out[f"op{i}"] = (bf, HSS.from_samples(bf=bf, leaf=128, oversample=10, tol=1e-3, seed=20 + i).factor())
    return out


def make_trace(ops, n_req, rate, seed, kmax=8):
    names = sorted(ops)
    t, opi, ks = poisson_requests(n_req, rate, len(names), seed=seed, kmax=kmax)
    rng = np.random.default_rng(seed)
    reqs = []
    for ti, oi, k in zip(t, opi, ks):
        n = ops[names[oi]][0].n
        u = (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))).astype(np.complex64)
        reqs.append((float(ti), names[oi], torch.from_numpy(u).pin_memory()))
    return reqs


def test_mix_equals_alone(ops):
    from paper_2609_11520_b300 import fio_solve
    from paper_2609_11520_b300.serve import Server, latency_stats
    reqs = make_trace(ops, 60, rate=4000.0, seed=1)
    srv = Server(ops, kmax=32, n_slots=3)
    done = srv.run(reqs)
    assert len(done) == len(reqs)
    assert srv.blocks < len(reqs)           # requests were coalesced
    for r, (t, name, u) in zip(done, reqs):
        bf, hss = ops[name]
        alone = fio_solve(bf, hss, u.cuda()).cpu()
        err = float(torch.linalg.norm(r.f - alone) / torch.linalg.norm(alone))
        assert err <= 1e-6, (r.rid, err)
        assert r.t_done >= r.t_admit >= r.t_arrive - 1e-9
    st = latency_stats(done)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_tight_hbm_budget_queues_and_completes(ops):
    from paper_2609_11520_b300.serve import Server
    reqs = make_trace(ops, 30, rate=1e5, seed=2)
    biggest = max(2 * u.numel() * 8 for _, _, u in reqs)
    srv = Server(ops, hbm_budget_bytes=biggest, kmax=16, n_slots=2)   # one request admitted at a time
    done = srv.run(reqs)
    assert len(done) == len(reqs)
    assert srv.in_use == 0
    for r in done:
        assert r.f is not None and torch.isfinite(r.f).all()


def test_pinned_outputs_and_pageable_inputs(ops):
    """Requests that bring pinned output buffers get their solutions there (direct D2H per
    request); pageable inputs go through the slot's staging buffers; both equal solving alone."""
    from paper_2609_11520_b300 import fio_solve
    from paper_2609_11520_b300.serve import Server
    base = make_trace(ops, 40, rate=4000.0, seed=3)
    reqs = []
    for i, (t, name, u) in enumerate(base):
        if i % 2:
            reqs.append((t, name, u.clone(), torch.empty_like(u).pin_memory()))   # pageable in, pinned out
        else:
            reqs.append((t, name, u))
    done = Server(ops, kmax=32, n_slots=2).run(reqs)
    for r, req in zip(done, reqs):
        bf, hss = ops[req[1]]
        if len(req) > 3:
            assert r.f is req[3]
        alone = fio_solve(bf, hss, req[2].cuda()).cpu()
        assert float(torch.linalg.norm(r.f - alone) / torch.linalg.norm(alone)) <= 1e-6


def test_mixed_1d_2d_operators():
    """A 2D operator (n = 32, N = 1024, quadtree BF, Morton-ordered HSS) served beside a 1D one:
    every result equals the same request solved alone."""
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    from paper_2609_11520_b300.serve import Server
    b1 = BF(4096, 16)
    b2 = BF(32, 25, "elliptic2d")
    ops = {"one_d": (b1, HSS.from_samples(bf=b1, leaf=128, oversample=10, tol=1e-3, seed=31).factor()),
           "two_d": (b2, HSS.from_samples(bf=b2, leaf=64, oversample=10, tol=1e-3, seed=32).factor())}
    reqs = make_trace(ops, 40, rate=4000.0, seed=4)
    done = Server(ops, kmax=16, n_slots=2).run(reqs)
    assert len(done) == len(reqs)
    for r, (t, name, u) in zip(done, reqs):
        bf, hss = ops[name]
        alone = fio_solve(bf, hss, u.cuda()).cpu()
        assert float(torch.linalg.norm(r.f - alone) / torch.linalg.norm(alone)) <= 1e-6
