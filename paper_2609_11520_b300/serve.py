"""Continuous-batching request loop over resident FIO operators.

A request asks for f = G~^{-1} K~^* u for k right-hand sides of one resident
operator (Eq. 4.2).  The server keeps every operator's BF and ULV factors on
the device and runs a host loop that

* admits arrived requests in arrival order while their device buffers fit
  the HBM budget (inputs + outputs, 16 bytes per RHS entry), and keeps the
  rest queued;
* whenever an execution slot (a CUDA stream with its own staging block) is
  free, takes the operator whose oldest admitted request waited longest and
  coalesces its admitted requests, oldest first, into one block of at most
  kmax columns -- requests that arrive while other blocks run join the next
  block of their operator (continuous batching);
* copies the block's right-hand sides host->device, launches fio_solve on
  the slot's stream, copies the solutions back, and completes the requests
  when the slot's event fires.  A request whose input (and output buffer,
  if it brings one) is in pinned host memory is copied by one asynchronous
  DMA per request straight into (out of) its columns of the block; other
  requests go through the slot's pinned staging buffers.

An operator has at most one block in flight (its handles are used by one
stream at a time); blocks of different operators overlap on the device.
Columns are independent in every kernel, so a request's result does not
depend on which other requests share its block.
"""
import collections
import time

import torch

from .api import fio_solve


class Request:
    __slots__ = ("rid", "op", "k", "u", "f", "out", "t_arrive", "t_admit", "t_done", "nbytes")

    def __init__(self, rid, op, u, t_arrive, out=None):
        self.rid, self.op, self.u, self.t_arrive = rid, op, u, t_arrive
        self.k = u.shape[0]
        self.f = None
        self.out = out
        self.t_admit = self.t_done = None
        self.nbytes = 2 * u.numel() * 8


class _Slot:
    """A CUDA stream with flat staging buffers: a block of k columns of length n
    uses their first k*n entries as contiguous (k, n) views, so every host copy
    is one asynchronous DMA."""

    def __init__(self, kmax, nmax):
        self.stream = torch.cuda.Stream()
        self.U = torch.empty(kmax * nmax, dtype=torch.complex64, device="cuda")
        self.F = torch.empty_like(self.U)
        self.host_in = torch.empty(kmax * nmax, dtype=torch.complex64).pin_memory()
        self.host_out = torch.empty(kmax * nmax, dtype=torch.complex64).pin_memory()
        self.event = torch.cuda.Event()
        self.busy = False
        self.reqs = []
        self.op = None
        self.out = None
        self.direct_out = False


class Server:
    """ops: dict name -> (BF, HSS) with factored HSS."""

    def __init__(self, ops, hbm_budget_bytes=8 << 30, kmax=64, n_slots=4, refine_steps=0):
        self.ops = dict(ops)
        self.kmax, self.refine = int(kmax), int(refine_steps)
        nmax = max(bf.n for bf, _ in self.ops.values())
        self.slots = [_Slot(self.kmax, nmax) for _ in range(n_slots)]
        self.budget = int(hbm_budget_bytes)
        self.in_use = 0
        self.waiting = collections.deque()                       # arrived, not admitted
        self.admitted = {name: collections.deque() for name in self.ops}
        self.op_busy = {name: False for name in self.ops}
        self.done = []
        self.blocks = 0

    # ------------------------------------------------------------------ loop
    def _admit(self):
        # a request larger than the whole budget is admitted alone (when nothing else is held)
        while self.waiting and (self.in_use + self.waiting[0].nbytes <= self.budget or self.in_use == 0):
            r = self.waiting.popleft()
            r.t_admit = time.perf_counter()
            self.in_use += r.nbytes
            self.admitted[r.op].append(r)

    def _complete(self):
        for s in self.slots:
            if s.busy and s.event.query():
                now = time.perf_counter()
                col = 0
                for r in s.reqs:
                    if s.direct_out:
                        r.f = r.out                         # written by the block's D2H copies
                    elif r.out is not None:
                        r.f = r.out.copy_(s.out[col:col + r.k])
                    else:
                        r.f = s.out[col:col + r.k].clone()
                    col += r.k
                    r.t_done = now
                    self.in_use -= r.nbytes
                    self.done.append(r)
                self.op_busy[s.op] = False
                s.busy, s.reqs, s.op = False, [], None

    def _dispatch(self):
        for s in self.slots:
            if s.busy:
                continue
            cands = [(q[0].t_arrive, name) for name, q in self.admitted.items() if q and not self.op_busy[name]]
            if not cands:
                return
            _, name = min(cands)
            bf, hss = self.ops[name]
            q, reqs, k = self.admitted[name], [], 0
            while q and k + q[0].k <= self.kmax:
                r = q.popleft()
                reqs.append(r)
                k += r.k
            if not reqs:   # a request wider than kmax runs alone in its own block
                reqs = [q.popleft()]
                k = reqs[0].k
            n = bf.n
            if k <= self.kmax:
                U, F = s.U[:k * n].view(k, n), s.F[:k * n].view(k, n)
                Hi, H = s.host_in[:k * n].view(k, n), s.host_out[:k * n].view(k, n)
            else:
                U = torch.empty(k, n, dtype=torch.complex64, device="cuda")
                F = torch.empty_like(U)
                Hi = torch.empty(k, n, dtype=torch.complex64).pin_memory()
                H = torch.empty(k, n, dtype=torch.complex64).pin_memory()
            direct_in = all(r.u.is_pinned() for r in reqs)
            direct_out = all(r.out is not None and r.out.is_pinned() for r in reqs)
            if not direct_in:
                col = 0
                for r in reqs:   # gather the block on the host (the slot is idle, so its buffers are free)
                    Hi[col:col + r.k].copy_(r.u)
                    col += r.k
            with torch.cuda.stream(s.stream):
                if direct_in:
                    col = 0
                    for r in reqs:
                        U[col:col + r.k].copy_(r.u, non_blocking=True)
                        col += r.k
                else:
                    U.copy_(Hi, non_blocking=True)
                fio_solve(bf, hss, U, out=F, refine_steps=self.refine, stream=s.stream)
                if direct_out:
                    col = 0
                    for r in reqs:
                        r.out.copy_(F[col:col + r.k], non_blocking=True)
                        col += r.k
                else:
                    H.copy_(F, non_blocking=True)
                s.event.record(s.stream)
            s.out, s.direct_out = H, direct_out
            s.busy, s.reqs, s.op = True, reqs, name
            self.op_busy[name] = True
            self.blocks += 1

    def run(self, requests):
        """Serve `requests` in arrival order: a list of (t_arrive_s, op_name, u) or
        (t_arrive_s, op_name, u, out), u a host tensor (k, N) and out an optional host
        tensor of the same shape that receives the solution.

        Returns the completed Request objects (results in .f, times in seconds
        relative to the start of the run).
        """
        pending = sorted(requests, key=lambda x: x[0])
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or self.waiting or any(self.admitted.values()) or any(s.busy for s in self.slots):
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i][0] <= now:
                t, op, u = pending[i][:3]
                out = pending[i][3] if len(pending[i]) > 3 else None
                self.waiting.append(Request(i, op, u, t0 + t, out))
                i += 1
            self._complete()
            self._admit()
            self._dispatch()
            if not any(s.busy for s in self.slots) and not self.waiting and i < len(pending):
                time.sleep(max(0.0, min(1e-3, pending[i][0] - (time.perf_counter() - t0))))
        for r in self.done:
            r.t_arrive -= t0
            r.t_admit -= t0
            r.t_done -= t0
        return sorted(self.done, key=lambda r: r.rid)


def latency_stats(done):
    """p50 / p99 request latency (arrival to completion) and RHS throughput."""
    lat = sorted(r.t_done - r.t_arrive for r in done)
    pick = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    span = max(r.t_done for r in done) - min(r.t_arrive for r in done)
    nrhs = sum(r.k for r in done)
    return {"p50_ms": 1e3 * pick(0.50), "p99_ms": 1e3 * pick(0.99), "rhs_per_s": nrhs / span, "requests": len(done),
            "rhs": nrhs, "span_s": span}
