"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds input generation only -- none of the method's arithmetic --
so both the CUDA path and the CPU oracle may draw their inputs from it.

Workloads (all synthetic; the paper uses no dataset):
  small1d    d=1, n=N=1024, Phi = x xi + c(x)|xi|, c = (2 + sin 2 pi x)/16, a = 1,
             BF rank 16, HSS leaf 64, tol 1e-8 (oracle, complex128), one RHS
  large1d    d=1, N=2^16, same phase, complex64 on the GPU; HSS leaf 128,
             oversampling 10, HSS tol 1e-3; solves of 1 and 64 RHS
  batched1d  32 operators, N uniform over {2^12..2^17}, c = (2 + s sin 2 pi x)/16
             with s ~ U[0.5, 1], 16 RHS each
  serving    resident operators, Poisson arrivals, 1..32 RHS per request
Vectors f_true have independent standard normal real and imaginary parts
(Section 5); right-hand sides are u = K f_true.
"""
import numpy as np

WORKLOADS = {
    "small1d": dict(d=1, n=1024, phase="cabs", s=1.0, r=16, leaf=64, p=10, tol=1e-8, k=1,
                    seed_f=0, seed_omega=1),
    "large1d": dict(d=1, n=1 << 16, phase="cabs", s=1.0, r=16, leaf=128, p=10, tol=1e-3, k=64,
                    seed_omega=2, seed_f=3),
}


def crandn(n, k, seed):
    """(n, k) complex128 with iid N(0,1) real and imaginary parts (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))


def bump_centers(N, m=10, seed=7):
    """(m, 2) centres (x_k, xi_k) of the Gaussian-bump amplitude of Section 5.1: x_k ~ U[0, 1],
    xi_k ~ U[-N/2, N/2] (the paper draws them at random without giving the draw)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.0, 1.0, m), rng.uniform(-N / 2, N / 2, m)], axis=1)


def sample_entries(N, S, seed=8, ncols=None):
    """S index pairs (rows, cols) uniform over [0, N) x [0, N) (int64), for the sampled-entry error
    of the adaptive BF rank; with ncols the columns are drawn from ncols distinct values only."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, N, S, dtype=np.int64)
    if ncols is None:
        cols = rng.integers(0, N, S, dtype=np.int64)
    else:
        pool = rng.choice(N, size=ncols, replace=False).astype(np.int64)
        cols = pool[rng.integers(0, ncols, S)]
    return rows, cols


def batched_operators(count=32, seed=4, logs=(12, 13, 14, 15, 16, 17)):
    """(N, s) per operator: N uniform over 2^logs, s ~ U[0.5, 1]."""
    rng = np.random.default_rng(seed)
    ns = [1 << int(rng.choice(logs)) for _ in range(count)]
    ss = [float(rng.uniform(0.5, 1.0)) for _ in range(count)]
    return list(zip(ns, ss))


def poisson_requests(n_requests, rate_per_s, n_ops, seed=5, kmax=32):
    """Arrival times (s), operator ids and RHS counts of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    return np.cumsum(gaps), rng.integers(0, n_ops, n_requests), rng.integers(1, kmax + 1, n_requests)
