"""Benchmark: RHS solves/s of the online stage f = G~^{-1} K~^* u at N = 2^16.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--k 64]

One step = one pass of the online hot path (BF adjoint K~^* + ULV solve of G~)
over one block of k = 64 right-hand sides (the coalesced "served" block) of
the 1D operator Phi = x xi + c(x)|xi|, c = (2 + sin 2 pi x)/16, N = 2^16,
BF rank 16, HSS leaf 128, oversampling 10, HSS tol 1e-3, complex64.  The
offline stage (bf_build, black-box HSS, ULV factor) runs once before timing
and its times are reported in `config`.  The plain path (one RHS per call)
is measured the same way and reported beside it with p50/p99 latencies.

`--impl reference` times the CPU FP64 oracle's online stage on the same
workload (each step one RHS: K~^* apply with the oracle's factor blocks built
beforehand, plus the oracle ULV solve on an HSS of the same tree shape).
Multi-GPU: one process per GPU (torchrun); every rank builds its own replica
of the operators and solves its own blocks (weak scaling, no collective on the
data path); rank 0 prints the line with the max time over ranks.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from fio_inputs import WORKLOADS, crandn  # noqa: E402

METRIC = "RHS solves/s at N=2^16 (Kt^* + HSS ULV) vs plain FP32 path; p50/p99 latency"
UNIT = "RHS/s"
L2_BYTES = 126 * 2 ** 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


def kernel_bytes(name, N, r, kc, binfo, hinfo):
    """Algorithmic HBM bytes of one launch (reads of inputs and tables, writes of outputs)."""
    S = N * r * kc * 8
    vec = N * kc * 8
    tables_quad = 2 * N * r * 8
    lsU = 1 << (binfo["L"] - binfo["sU"])
    nVP = (1 << binfo["sV"]) * N * 8
    if name == "k_U_adj" or name == "k_U_fwd":
        return vec + N * lsU * 8 + S
    if name == "k_V_adj" or name == "k_V_fwd":
        return S + nVP + vec
    if name.startswith("k_quad"):
        return 2 * S + tables_quad
    if name.startswith("k_M"):
        return 2 * S + N * r * r * 8
    nB, nC = binfo["sU"] - binfo["h"], binfo["h"] - binfo["sV"]
    if name.startswith("k_bf_left"):     # U^(*) + B^(*) levels + (M^* for the adjoint) ; middle state
        b = vec + N * lsU * 8 + nB * tables_quad + S
        return b + (N * r * r * 8 if name.endswith("adj") else 0)
    if name.startswith("k_bf_right"):    # V^(*) + C^(*) levels + (M for the forward) ; middle state
        b = vec + nVP + nC * tables_quad + S
        return b + (N * r * r * 8 if name.endswith("fwd") else 0)
    if name in ("k_ulv_up", "k_ulv_down"):
        # average over the Lh launches of one pass: W_l plus the level's vectors
        Lh, leaf, ranks = hinfo["Lh"], hinfo["leaf"], hinfo["ranks"]
        tot = 0
        for l in range(1, Lh + 1):
            m = leaf if l == Lh else 2 * ranks[l + 1]
            tot += (2 ** l) * m * m * 8 + 2 * (2 ** l) * m * kc * 8
        return tot / Lh
    return None


def kernel_fma(name, N, r, kc, binfo):
    """FP32 FMA instructions (per thread-lane) of one launch of a fused half pass, as the kernels issue them.

    Transfer level: per quad and column 2 x 1152 FMA (16 x 16 real Lagrange matrix applied to the
    real and imaginary parts of both halves, plus the complex phase products); middle level:
    r^2 complex MACs (4 FMA) per pair; leaf levels: 8 x (16 x 2 + 4) FMA per pair or point.
    """
    nB, nC = binfo["sU"] - binfo["h"], binfo["h"] - binfo["sV"]
    quad = (N // 2) * 2 * 1152
    leaf = N * 8 * (2 * r + 4)
    mid = N * r * r * 4
    if name.startswith("k_bf_left"):
        return kc * (nB * quad + leaf + (mid if name.endswith("adj") else 0))
    if name.startswith("k_bf_right"):
        return kc * (nC * quad + leaf + (mid if name.endswith("fwd") else 0))
    return None


def fp32_peak_tflops(sm_mhz, sm_count):
    """FP32 FMA peak: SMs (from the device) x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def parse_profile(text):
    out = {}
    for line in text.strip().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


# DRAM bytes (read + write) per launch from one ncu capture of the current kernel build:
# (kernel name, N, columns per launch, transfer-level arithmetic) -> bytes, or absent.
# `python bench.py --profile-case bf_adjoint --n 65536 --k 64 --reps 1` under
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` (one launch of each half pass).
NCU_TRAFFIC = {
    ("k_bf_left_adj", 65536, 64, "tc_f16"): 256577280 + 489624320,
    ("k_bf_right_adj", 65536, 64, "tc_f16"): 625194752 + 31775744,
}


def roofline_entry(name, per_launch_ms, nbytes, nfma, hbm_peak, peak_src, clocks, sm_count, traffic=None):
    """Roofline of the dominant kernel against the measured HBM copy bandwidth.  The fused BF half
    passes move their transfer-level products to the tensor cores, so their ideal time is set by
    the algorithmic HBM bytes; the FP32-FMA equivalent of their arithmetic (what the CUDA-core
    variant issues) is reported beside it for context."""
    hbm_achieved = nbytes / (per_launch_ms / 1e3) / 1e9 if nbytes else None
    out = {"kernel": name, "bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": (hbm_achieved / hbm_peak) if hbm_achieved else None, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
           "bytes_per_launch": nbytes, "ms_per_launch": per_launch_ms, "traffic": traffic}
    if nfma:
        sm_max = clocks.get("sm_max_mhz") or 2032.0
        fp = fp32_peak_tflops(sm_max, sm_count)
        out["fp32_equivalent"] = {"tflops": 2 * nfma / (per_launch_ms / 1e3) / 1e12, "peak_tflops": fp,
                                  "peak_source": "derived: %d SMs (device attribute) x 128 FP32 FMA/clk x 2 x %.0f MHz"
                                                 % (sm_count, sm_max)}
    return out


def operator_ranks(n, leaf):
    """Per-level HSS ranks of the oracle's own construction of the N = 2^16 operator (stored by
    tests/golden/make_solve_golden.py, which calls only oracle/); None if absent or another size."""
    path = os.path.join(ROOT, "tests", "golden", "solve1d_N65536.txt")
    if n != 1 << 16 or leaf != 128 or not os.path.exists(path):
        return None
    vals = dict(line.split(maxsplit=1) for line in open(path) if not line.startswith("#"))
    return [int(v) for v in vals["ranks"].split()]


def cpu_oracle_online(n, steps, warmup, leaf, r, seed=3, threads=None):
    """Oracle online stage, one RHS per step: K~^* u (factor blocks built first) + ULV solve on an
    HSS with the tree and per-level ranks of the operator's own (oracle-built) HSS.  The solve's
    cost depends only on that shape, so its generators are random (building the oracle's HSS at
    N = 2^16 takes about 20 minutes).  threads: BLAS threads; a number runs the measurement in a
    child process whose BLAS libraries start with that many threads (None = this process, all
    cores)."""
    if threads is not None:
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
                   MKL_NUM_THREADS=str(threads))
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-oracle", str(steps), str(warmup),
                              str(threads)], capture_output=True, text=True, env=env, cwd=ROOT)
        if out.returncode != 0:
            raise RuntimeError("CPU oracle child failed: " + out.stderr[-2000:])
        d = json.loads(out.stdout.strip().splitlines()[-1])
        return d["value"], threads, d["sample"], d["times"]
    from oracle.butterfly import Butterfly1D
    from oracle.hss import ULV, random_hss
    from oracle.problem import Phase
    cores = len(os.sched_getaffinity(0))
    Lh = int(np.log2(n // leaf))
    ranks = operator_ranks(n, leaf) or ([0] + [8] * Lh)
    bf = Butterfly1D(Phase("cabs"), n, r, cache=True)
    hss = random_hss(n, leaf, ranks, np.random.default_rng(0), shift=float(n))
    ulv = ULV(hss)
    u = crandn(n, 1, seed)
    t0 = time.perf_counter()
    bf.adjoint(u)                      # builds and keeps the factor blocks (offline part)
    setup = time.perf_counter() - t0
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        ulv.solve(bf.adjoint(crandn(n, 1, seed + 1 + i)))
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    med = statistics.median(times)
    used = int(os.environ.get("OPENBLAS_NUM_THREADS", cores))
    sample = (f"{steps} RHS of the N=2^16 workload, one per step (median {med:.2f} s, {used} BLAS threads): "
              f"oracle K~^* apply (complex128, factor blocks built once beforehand in {setup:.1f} s, excluded) + "
              f"oracle ULV solve on an HSS with the operator's tree and ranks {ranks}")
    return 1.0 / med, used, sample, times


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS["large1d"]
    value, cores, sample, times = cpu_oracle_online(w["n"], args.steps, args.warmup, w["leaf"], w["r"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "large1d: d=1 N=2^16 Phi=x*xi+c(x)|xi| BF r=16 HSS leaf 128 tol 1e-3, 1 RHS/step",
                   "k_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def kernel2d_bytes(name, N, kc, sV, L, sU, R=25):
    """Algorithmic HBM bytes of one 2D kernel launch (kc columns): coefficient states
    N*R*kc complex64 in and out (R = r1^2), the vectors, and each table read once."""
    S = N * R * kc * 8
    vec = N * kc * 8
    if name.startswith("k2_V"):
        return S + vec + (4 ** sV) * N * 8
    if name.startswith("k2_U"):
        return S + vec + N * (4 ** (L - sU)) * 8
    if name.startswith("k2_C") or name.startswith("k2_B"):
        return 2 * S + N * 4 * R * 8
    if name.startswith("k2_M"):
        return 2 * S + N * R * R * 8
    return None


def run_2d(args):
    """2D workload: the K~^* apply of the quadtree BF at n = 256 (N = 2^16, r = r1^2, r1 = --r1-2d,
    default 5) on blocks of k = 16 RHS, and the full online solve at n = --n2d (default 64) with
    its offline stages timed."""
    import torch
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    from paper_2609_11520_b300 import _lib
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n, k = 256, 16
    N = n * n
    R = args.r1_2d ** 2
    bf = BF(n, R, "elliptic2d")
    info = bf.info()
    rng = np.random.default_rng(3)
    X = torch.from_numpy((rng.standard_normal((k, N)) + 1j * rng.standard_normal((k, N))).astype(np.complex64)).cuda()
    Y = torch.empty_like(X)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    with Clocks(0) as clk:
        adj = timed(lambda: bf.apply(X, adjoint=True, out=Y), args.steps, args.warmup)
        fwd = timed(lambda: bf.apply(X, out=Y), args.steps, args.warmup)
    _lib.lib.fio_profile_enable(1)
    for _ in range(args.steps):
        flush.fill_(1.0)
        bf.apply(X, adjoint=True, out=Y)
    torch.cuda.synchronize()
    buf = ctypes.create_string_buffer(1 << 16)
    _lib.check(_lib.lib.fio_profile_report(buf, len(buf)))
    _lib.lib.fio_profile_enable(0)
    prof = parse_profile(buf.value.decode())
    tot = sum(v[1] for v in prof.values())
    peak, peak_src = load_peaks()
    kernels = {}
    for name, (cnt, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        nb = kernel2d_bytes(name, N, k, info["sV"], info["L"], info["sU"], R)
        gbs = nb / (ms / cnt / 1e3) / 1e9 if nb else None
        kernels[name] = {"launches": cnt, "ms_total": round(ms, 4), "share": round(ms / tot, 4),
                         "bytes_per_launch": nb, "achieved_gbs": gbs}
    top = max(prof.items(), key=lambda kv: kv[1][1])
    tb = kernel2d_bytes(top[0], N, k, info["sV"], info["L"], info["sU"], R)
    ach = tb / (top[1][1] / top[1][0] / 1e3) / 1e9
    # full solve at a smaller n
    ns = args.n2d
    t0 = time.perf_counter()
    bs = BF(ns, R, "elliptic2d")
    g = HSS.from_samples(bf=bs, leaf=256, oversample=10, tol=1e-3, seed=1)
    t_hss = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.factor()
    t_fac = time.perf_counter() - t0
    f = crandn(ns * ns, k, seed=0)
    Ft = torch.from_numpy(np.ascontiguousarray(f.T.astype(np.complex64))).cuda()
    U = bs.apply(Ft)
    OUT = torch.empty_like(U)
    sol = timed(lambda: fio_solve(bs, g, U, out=OUT), args.steps, args.warmup)
    e = float(torch.linalg.norm(OUT - Ft) / torch.linalg.norm(Ft))
    fio_solve(bs, g, U, out=OUT, refine_steps=1)
    e1 = float(torch.linalg.norm(OUT - Ft) / torch.linalg.norm(Ft))
    _lib.lib.fio_profile_enable(1)
    for _ in range(args.steps):
        flush.fill_(1.0)
        fio_solve(bs, g, U, out=OUT)
    torch.cuda.synchronize()
    _lib.check(_lib.lib.fio_profile_report(buf, len(buf)))
    _lib.lib.fio_profile_enable(0)
    sprof = parse_profile(buf.value.decode())
    stot = sum(v[1] for v in sprof.values())
    solve_kernels = {nm: {"launches": c, "ms_total": round(ms, 4), "share": round(ms / stot, 4)}
                     for nm, (c, ms) in sorted(sprof.items(), key=lambda kv: -kv[1][1])}
    line = {
        "metric": f"2D K~^* apply RHS/s (n = 256, N = 2^16, quadtree BF r = {R}); 2D online solve", "unit": UNIT,
        "value": k * args.steps / (sum(adj) / 1e3), "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(adj), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"2d: Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), a = 1, n = 256, r = {R}, k = 16 per apply",
                   "l2": "flushed between timed steps (256 MiB write)", "table_bytes": info["table_bytes"]},
        "forward": {"value": k * args.steps / (sum(fwd) / 1e3), "ms_per_step": statistics.mean(fwd)},
        "kernels": kernels,
        "roofline": {"kernel": top[0], "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "peak_source": peak_src, "bytes_per_launch": tb, "traffic": None},
        "solve": {"n": ns, "N": ns * ns, "r": R, "leaf": 256, "tol": 1e-3, "k": k, "hss_build_s": round(t_hss, 2),
                  "ulv_factor_s": round(t_fac, 2), "ranks": g.info()["ranks"], "rhs_per_s": k * args.steps / (sum(sol) / 1e3),
                  "ms_per_solve": statistics.mean(sol), "e_direct_vs_f_true": e, "e_refine1": e1,
                  "kernels": solve_kernels},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def batched_leg(steps, warmup, count=32):
    """Config-4 workload: `count` operators, N uniform over 2^12..2^17 (seed 4), s ~ U[0.5, 1], 16 RHS
    each; one step = one solve of every operator's block.  Times every mode of fio_batch_* after the
    autotuner and returns the summary dict."""
    import torch
    from fio_inputs import batched_operators
    from paper_2609_11520_b300 import BF, HSS, Batch
    t0 = time.perf_counter()
    ops = []
    for i, (n, sdepth) in enumerate(batched_operators(count)):
        bf = BF(n, 16, "cabs", sdepth)
        ops.append((bf, HSS.from_samples(bf=bf, leaf=128, oversample=10, tol=1e-3, seed=40 + i).factor()))
    t_build = time.perf_counter() - t0
    k = 16
    Us = [torch.from_numpy(np.ascontiguousarray(crandn(bf.n, k, 60 + i).T.astype(np.complex64))).cuda()
          for i, (bf, _) in enumerate(ops)]
    Fs = [torch.empty_like(U) for U in Us]
    b = Batch(ops)
    report = b.autotune(Us, Fs, reps=3)
    times = {}
    for mode in ("per_operator", "grouped", "graph"):
        b.set_mode(mode)
        for _ in range(warmup):
            b.solve(Us, Fs)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(steps):
            b.solve(Us, Fs)
        ev[1].record()
        ev[1].synchronize()
        times[mode] = ev[0].elapsed_time(ev[1]) / steps
    best = min(times, key=times.get)
    nrhs = k * len(ops)
    return {"rhs_per_s": nrhs / (times[best] / 1e3), "ms_per_step": times[best], "mode": best,
            "ms_per_step_by_mode": {m: round(v, 4) for m, v in times.items()}, "operators": len(ops),
            "rhs_per_step": nrhs, "offline_build_s": round(t_build, 2),
            "autotune": report.strip().splitlines(),
            "workload": "32 1D operators, N uniform over {2^12..2^17} (seed 4), s ~ U[0.5, 1], BF r 16, "
                        "HSS leaf 128 tol 1e-3, 16 RHS each, device-resident inputs"}


SERVING_1D = [(1 << 14, 1.0), (1 << 15, 1.0), (1 << 16, 1.0), (1 << 16, 0.5), (1 << 17, 1.0), (1 << 18, 1.0)]


def serving_leg(nreq, rates=(0.5, 0.8, 1.0), ops2d=(128, 256), seed=5, r2d=49, prebuilt=None):
    """Config-5 workload through the continuous-batching server: resident operators (the six 1D
    operators of SERVING_1D and 2D elliptic operators with n per dimension in ops2d), Poisson
    arrivals (seed 5) at the given fractions of the measured saturated request rate, 1..32 RHS per
    request from pinned host memory (H2D and D2H inside each request's latency)."""
    import torch
    from fio_inputs import poisson_requests
    from paper_2609_11520_b300 import BF, HSS
    from paper_2609_11520_b300.serve import Server, latency_stats
    t0 = time.perf_counter()
    ops = {}
    for i, (n, sdepth) in enumerate(SERVING_1D):
        bf = BF(n, 16, "cabs", sdepth)
        ops[f"1d_n{n}_s{sdepth}"] = (bf, HSS.from_samples(bf=bf, leaf=128, oversample=10, tol=1e-3, seed=70 + i).factor())
    for i, n2 in enumerate(ops2d):
        if prebuilt and (n2, r2d) in prebuilt:
            ops[f"2d_n{n2}"] = prebuilt[(n2, r2d)]
            continue
        bf = BF(n2, r2d, "elliptic2d")
        ops[f"2d_n{n2}"] = (bf, HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=90 + i).factor())
    t_build = time.perf_counter() - t0
    names = sorted(ops)
    # request inputs: slices of a pinned pool of 64 random columns per operator; solutions land in a
    # pinned output pool per operator
    rng = np.random.default_rng(6)
    pool_in, pool_out = {}, {}
    for nm in names:
        n = ops[nm][0].n
        u = (rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))).astype(np.complex64)
        pool_in[nm] = torch.from_numpy(u).pin_memory()
        pool_out[nm] = torch.empty_like(pool_in[nm]).pin_memory()

    def trace(rate, sd):
        t, oi, ks = poisson_requests(nreq, rate, len(names), seed=sd, kmax=32)
        offs = np.random.default_rng(sd + 1).integers(0, 33, size=len(t))
        return [(float(ti), names[o], pool_in[names[o]][off:off + kk], pool_out[names[o]][off:off + kk])
                for ti, o, kk, off in zip(t, oi, ks, offs)]

    sat_trace = [(0.0,) + tuple(x[1:]) for x in trace(1.0, seed)]
    Server(ops, kmax=64, n_slots=4).run(sat_trace[: min(100, nreq)])   # warm-up
    sat = latency_stats(Server(ops, kmax=64, n_slots=4).run(sat_trace))
    avg_k = float(np.mean([x[2].shape[0] for x in sat_trace]))
    req_rate = sat["rhs_per_s"] / avg_k
    by_rate = {}
    for frac in rates:
        st = latency_stats(Server(ops, kmax=64, n_slots=4).run(trace(frac * req_rate, seed)))
        by_rate[str(frac)] = {k_: round(v, 4) if isinstance(v, float) else v for k_, v in st.items()}
    top = by_rate[str(max(rates))]
    return {"p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"], "rhs_per_s": sat["rhs_per_s"],
            "requests_per_rate": nreq, "saturated": {k_: round(v, 4) if isinstance(v, float) else v for k_, v in sat.items()},
            "by_rate_fraction": by_rate, "offline_build_s": round(t_build, 2), "operators": names,
            "workload": "continuous batching over resident operators (1D N = 2^14, 2^15, 2^16, 2^16 with s = 0.5, "
                        "2^17, 2^18; 2D elliptic n = %s, BF r = %d), Poisson arrivals (seed 5), 1..32 RHS per request, "
                        "kmax 64, 4 streams, pinned host requests (H2D and D2H inside the latency); p50/p99 at the "
                        "highest rate fraction, rhs_per_s saturated" % (", ".join(str(x) for x in ops2d), r2d)}


def c3_leg(steps, warmup, n=256, r1=7, k=16):
    """2D end-to-end solve (n = 256, N = 2^16, HSS leaf 256 = 16 x 16, tol 1e-3, 16 RHS): offline BF,
    HSS construction and ULV timed once; the online f = F~ K~^* u timed on device-resident blocks
    with L2 flushed.  u = K~ f_true.  The BF runs on the r1 x r1 grid (default 7 x 7 = 49): the
    sampled FP64 entry errors of the 5 x 5 and 7 x 7 grids are reported beside it (at 5 x 5 the BF
    error lies above the HSS tolerance and the HSS ranks grow past what fits the offline budget).
    Returns (summary, (bf, hss))."""
    import torch
    from fio_inputs import sample_entries
    from paper_2609_11520_b300 import BF, HSS, entry_error, fio_solve
    N = n * n
    rows, cols = sample_entries(N, 2000, seed=9)
    e_grid = {f"{q}x{q}": entry_error(n, q * q, rows, cols, "elliptic2d") for q in (5, 6, 7)}
    t0 = time.perf_counter()
    bf = BF(n, r1 * r1, "elliptic2d")
    torch.cuda.synchronize()
    t_bf = time.perf_counter() - t0
    t0 = time.perf_counter()
    g = HSS.from_samples(bf=bf, leaf=256, oversample=10, tol=1e-3, seed=1)
    torch.cuda.synchronize()
    t_hss = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.factor()
    torch.cuda.synchronize()
    t_fac = time.perf_counter() - t0
    f = crandn(N, k, seed=0)
    Ft = torch.from_numpy(np.ascontiguousarray(f.T.astype(np.complex64))).cuda()
    U = bf.apply(Ft)
    OUT = torch.empty_like(U)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        fio_solve(bf, g, U, out=OUT)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fio_solve(bf, g, U, out=OUT)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    e = float(torch.linalg.norm(OUT - Ft) / torch.linalg.norm(Ft))
    fio_solve(bf, g, U, out=OUT, refine_steps=1)
    e1 = float(torch.linalg.norm(OUT - Ft) / torch.linalg.norm(Ft))
    ms = statistics.median(ts)
    return ({"rhs_per_s": k / (ms / 1e3), "ms_per_solve": ms, "k": k, "n": n, "N": N, "r": r1 * r1,
             "offline_s": {"bf_build": round(t_bf, 3), "hss_build": round(t_hss, 2), "ulv_factor": round(t_fac, 2)},
             "hss_ranks": g.info()["ranks"], "e_direct_vs_f_true": e, "e_refine1": e1,
             "bf_entry_error_by_grid": e_grid,
             "workload": "2D Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), a = 1, n = 256, BF r1 x r1 = %d x %d, "
                         "HSS leaf 256 (16 x 16), oversample 10, tol 1e-3, 16 RHS per solve, u = K~ f_true, "
                         "L2 flushed between timed solves" % (r1, r1)}, (bf, g))


def run_batched(args):
    """Batched workload alone (one JSON line)."""
    import torch
    torch.cuda.set_device(0)
    b = batched_leg(args.steps, args.warmup)
    line = {"metric": "RHS solves/s, batched workload (32 uneven 1D operators x 16 RHS)", "value": b["rhs_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "batched1d: " + b["workload"]}, "batched": b}
    print(json.dumps(line))


def run_serving(args):
    """Serving workload alone (one JSON line), with the 2D operators of --serve-2d."""
    import torch
    torch.cuda.set_device(0)
    sv = serving_leg(args.requests, ops2d=tuple(int(x) for x in args.serve_2d.split(",") if x))
    line = {"metric": "RHS solves/s served (continuous batching, Poisson arrivals); p50/p99 latency",
            "value": sv["rhs_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.requests, "warmup": 100,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic", "config": {"workload": "serving: " + sv["workload"]}, "served_requests": sv}
    print(json.dumps(line))


def run_profile_case(args):
    """One stage of the online path, repeated between cudaProfilerStart / Stop so that
    `ncu --profile-from-start off` captures only those launches.  Cases: bf_adjoint, bf_forward
    (1D, N = --n, k = --k columns), hss_solve, fio_solve (1D operator with its HSS), bf2d_adjoint,
    bf2d_forward (2D elliptic phase, n = --n per dimension).  --path picks the BF kernels
    (auto, per_level, fused, fused_v2, fused_simt), --precision fp32 or split_bf16.
    Prints the mean CUDA-event time per repetition."""
    import torch
    from paper_2609_11520_b300 import BF, HSS, fio_solve
    torch.cuda.set_device(0)
    case = args.profile_case
    two_d = case.startswith("bf2d")
    n = args.n if args.n else (256 if two_d else 1 << 16)
    bf = BF(n, 25, "elliptic2d") if two_d else BF(n, 16)
    hss = None
    if case in ("hss_solve", "fio_solve"):
        hss = HSS.from_samples(bf=bf, leaf=128, oversample=10, tol=1e-3, seed=2).factor()
    if not two_d:
        bf.set_path(args.path).set_precision(args.precision)
    rng = np.random.default_rng(0)
    X = torch.from_numpy((rng.standard_normal((args.k, bf.n)) + 1j * rng.standard_normal((args.k, bf.n)))
                         .astype(np.complex64)).cuda()
    Y = torch.empty_like(X)

    def run():
        if case in ("bf_adjoint", "bf2d_adjoint"):
            bf.apply(X, adjoint=True, out=Y)
        elif case in ("bf_forward", "bf2d_forward"):
            bf.apply(X, out=Y)
        elif case == "hss_solve":
            hss.solve(X, out=Y)
        else:
            fio_solve(bf, hss, X, out=Y)

    run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    a.record()
    for _ in range(args.reps):
        run()
    b.record()
    torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    print(f"{case} n={n} k={args.k} path={args.path} precision={args.precision}: "
          f"{a.elapsed_time(b) / args.reps:.4f} ms per repetition")


def main():
    if len(sys.argv) == 5 and sys.argv[1] == "--cpu-oracle":   # child of cpu_oracle_online(threads=...)
        w = WORKLOADS["large1d"]
        v, _, sample, times = cpu_oracle_online(w["n"], int(sys.argv[2]), int(sys.argv[3]), w["leaf"], w["r"])
        print(json.dumps({"value": v, "sample": sample, "times": times}))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--workload", default="large1d", choices=["large1d", "batched1d", "serving", "2d"])
    ap.add_argument("--n2d", type=int, default=64)
    ap.add_argument("--r1-2d", type=int, default=5, help="2D tensor grid r1 (rank r1^2) of --workload 2d")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--serve-2d", default="128,256", help="n per dimension of the 2D serving operators (r = 49), comma separated")
    ap.add_argument("--serve-requests", type=int, default=600, help="requests per rate of the default line's serving leg")
    ap.add_argument("--no-legs", action="store_true", help="skip the 2D solve, serving and batched legs of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    choices=["bf_adjoint", "bf_forward", "hss_solve", "fio_solve", "bf2d_adjoint", "bf2d_forward"])
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--path", default="auto")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split_bf16"])
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched1d":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "2d":
        return run_2d(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_2609_11520_b300 import BF, HSS, fio_solve
    from paper_2609_11520_b300 import _lib

    w = WORKLOADS["large1d"]
    n, r, k = w["n"], w["r"], args.k
    stream = torch.cuda.current_stream()

    # ---- offline stage (not timed in `value`) ----
    t0 = time.perf_counter()
    bf = BF(n, r, w["phase"], w["s"])
    t_bf = time.perf_counter() - t0
    t0 = time.perf_counter()
    hss = HSS.from_samples(bf=bf, leaf=w["leaf"], oversample=w["p"], tol=w["tol"], seed=w["seed_omega"] + rank)
    t_hss = time.perf_counter() - t0
    t0 = time.perf_counter()
    hss.factor()
    t_fac = time.perf_counter() - t0
    binfo, hinfo = bf.info(), hss.info()

    # ---- inputs resident in HBM: u = K~ f_true ----
    f_true = crandn(n, k, seed=w["seed_f"] + 100 * rank)
    F_true = torch.from_numpy(np.ascontiguousarray(f_true.T.astype(np.complex64))).cuda()
    U = bf.apply(F_true)
    OUT = torch.empty_like(U)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)                       # L2 flush between timed iterations
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    # ---- served path: one coalesced block of k RHS per step ----
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        served = timed(lambda: fio_solve(bf, hss, U, out=OUT), args.steps, args.warmup)
    torch.cuda.synchronize()
    barrier()
    tot_ms = sum(served)
    if world > 1:
        tt = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tot_ms = float(tt.item())
    value = world * k * args.steps / (tot_ms / 1e3)
    e_direct = float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true))

    # ---- plain path: one RHS per call ----
    U1 = U[:1].clone()
    O1 = torch.empty_like(U1)
    plain = timed(lambda: fio_solve(bf, hss, U1, out=O1), args.steps, args.warmup)
    plain_value = 1e3 / statistics.mean(plain)

    # ---- end to end through the public API with pinned host buffers: every step copies its block of
    # right-hand sides host->device and its solutions device->host; steps are pipelined over two
    # buffers, an H2D stream and a D2H stream, so the copies of step i+1 and i-1 overlap the solve
    # of step i ----
    Uh = [U.cpu().pin_memory() for _ in range(2)]
    Oh = [torch.empty(U.shape, dtype=U.dtype).pin_memory() for _ in range(2)]
    Ud = [torch.empty_like(U) for _ in range(2)]
    Od = [torch.empty_like(U) for _ in range(2)]
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]
    d2h_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(nsteps):
        for i in range(nsteps):
            j = i & 1
            with torch.cuda.stream(h2d_s):
                h2d_s.wait_event(solved[j])              # the solve that last read Ud[j] is done
                Ud[j].copy_(Uh[j], non_blocking=True)
                h2d_done[j].record(h2d_s)
            stream.wait_event(h2d_done[j])
            stream.wait_event(d2h_done[j])               # Od[j] has been copied out
            fio_solve(bf, hss, Ud[j], out=Od[j], stream=stream)
            solved[j].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(solved[j])
                Oh[j].copy_(Od[j], non_blocking=True)
                d2h_done[j].record(d2h_s)

    for j in range(2):
        solved[j].record(stream)
        d2h_done[j].record(d2h_s)
    e2e_run(args.warmup)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    h2d_s.wait_event(ea)
    d2h_s.wait_event(ea)
    e2e_run(args.steps)
    stream.wait_stream(d2h_s)
    eb.record(stream)
    eb.synchronize()
    e2e_ms = ea.elapsed_time(eb)
    e2e_value = world * k * args.steps / (e2e_ms / 1e3)
    e2e_err = float(torch.linalg.norm(Oh[(args.steps - 1) & 1].cuda() - F_true) / torch.linalg.norm(F_true))

    # ---- per-kernel CUDA-event attribution over an identical pass ----
    _lib.lib.fio_profile_enable(1)
    for _ in range(args.steps):
        flush.fill_(1.0)
        fio_solve(bf, hss, U, out=OUT)
    torch.cuda.synchronize()
    buf = ctypes.create_string_buffer(1 << 16)
    _lib.check(_lib.lib.fio_profile_report(buf, len(buf)))
    _lib.lib.fio_profile_enable(0)
    prof = parse_profile(buf.value.decode())
    launches = sum(c for c, _ in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][1])
    kc = min(k, 64)
    peak, peak_src = load_peaks()
    per_launch_ms = top[1][1] / top[1][0]
    nbytes = kernel_bytes(top[0], n, r, kc, binfo, hinfo)
    nfma = kernel_fma(top[0], n, r, kc, binfo)
    kernels = {name: {"launches": c, "ms_total": round(ms, 4), "share": round(ms / sum(v[1] for v in prof.values()), 4)}
               for name, (c, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- the same block with the FP32 transfer levels on the CUDA cores instead of the tensor cores ----
    bf.set_path("fused_simt")
    simt = timed(lambda: fio_solve(bf, hss, U, out=OUT), args.steps, args.warmup)
    bf.set_path("auto")

    # ---- split-precision transfer levels (BF16 hi + lo on the tensor cores), same served block ----
    split = None
    try:
        bf.set_precision("split_bf16")
    except Exception as e:   # operator shape without a split kernel
        split = {"unavailable": str(e)}
    if split is None:
        sp = timed(lambda: fio_solve(bf, hss, U, out=OUT), args.steps, args.warmup)
        e_sp = float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true))
        sp1 = timed(lambda: fio_solve(bf, hss, U, out=OUT, refine_steps=1), args.steps, args.warmup)
        e_sp1 = float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true))
        # split precision on the HSS products too: the ULV node products on the tensor cores (BF16 parts)
        hss.set_solve_path("tensor_cores")
        sph = timed(lambda: fio_solve(bf, hss, U, out=OUT), args.steps, args.warmup)
        e_sph = float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true))
        hss.set_solve_path("cuda_cores")
        bf.set_precision("fp32")
        fp1 = timed(lambda: fio_solve(bf, hss, U, out=OUT, refine_steps=1), args.steps, args.warmup)
        e_fp1 = float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true))
        split = {"value": world * k * args.steps / (sum(sp) / 1e3), "unit": UNIT, "e_direct_vs_f_true": e_sp,
                 "refine1": {"value": world * k * args.steps / (sum(sp1) / 1e3), "e_vs_f_true": e_sp1},
                 "hss_tensor_cores": {"value": world * k * args.steps / (sum(sph) / 1e3), "e_direct_vs_f_true": e_sph},
                 "fp32_refine1": {"value": world * k * args.steps / (sum(fp1) / 1e3), "e_vs_f_true": e_fp1}}

    # ---- preconditioned CG on Eq. 4.3 (Section 4.1), same block, tolerance 1e-5 ----
    from paper_2609_11520_b300 import fio_pcg
    pcg_info = {}

    def pcg_step():
        _, it, rr = fio_pcg(bf, hss, U, out=OUT, tol=1e-5, maxit=30)
        pcg_info.update(iterations=it, max_relres=max(rr))

    pcg_t = timed(pcg_step, max(3, args.steps // 4), 1)
    pcg = {"value": world * k * len(pcg_t) / (sum(pcg_t) / 1e3), "unit": UNIT, "tol": 1e-5,
           "e_vs_f_true": float(torch.linalg.norm(OUT - F_true) / torch.linalg.norm(F_true)), **pcg_info}

    legs = {}
    if rank == 0 and world == 1 and not args.no_legs:
        legs["solve_2d"], op256 = c3_leg(max(3, args.steps // 2), args.warmup)
        legs["served_requests"] = serving_leg(args.serve_requests,
                                              ops2d=tuple(int(x) for x in args.serve_2d.split(",") if x),
                                              prebuilt={(256, 49): op256})
        legs["batched"] = batched_leg(max(3, args.steps // 2), args.warmup)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, cores, sample, _ = cpu_oracle_online(n, 3, 0, w["leaf"], r)
        cv1, _, sample1, _ = cpu_oracle_online(n, 2, 0, w["leaf"], r, threads=1)
        cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "one_thread": {"value": cv1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if rank == 0:
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(served), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {
                "workload": "large1d: d=1, N=2^16, Phi=x*xi+c(x)|xi|, c=(2+sin 2pi x)/16, a=1, BF r=16, "
                            "HSS leaf 128, oversample 10, tol 1e-3; served block of k RHS per step",
                "k_per_step": k, "l2": "flushed between timed steps (256 MiB write)",
                "offline_s": {"bf_build": round(t_bf, 3), "hss_build": round(t_hss, 3), "ulv_factor": round(t_fac, 3)},
                "hss_ranks": hinfo["ranks"], "hss_samples": hinfo["samples"],
                "e_direct_vs_f_true": e_direct, "parallelism": f"replicas x{world}",
                "transfer_levels": "tcgen05 tensor cores, FP16 hi/lo three-term products (FP32 accuracy)",
            },
            "latency_ms": {"served_p50": percentile(served, 50), "served_p99": percentile(served, 99),
                           "plain_p50": percentile(plain, 50), "plain_p99": percentile(plain, 99)},
            "plain": {"value": plain_value, "unit": UNIT, "k_per_call": 1},
            "cuda_core_fp32": {"value": world * k * args.steps / (sum(simt) / 1e3), "unit": UNIT,
                               "ms_per_step": statistics.mean(simt)},
            "split_bf16": split,
            "pcg": pcg,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(U.numel() * 8),
                    "d2h_bytes_per_step": int(U.numel() * 8), "e_vs_f_true": e2e_err,
                    "pipelining": "two buffers; H2D and D2H on their own streams overlap the neighbouring steps' solves"},
            "gpu_launches": int(launches),
            "kernels": kernels,
            "roofline": roofline_entry(top[0], per_launch_ms, nbytes, nfma, peak, peak_src, clk.summary(), sm_count,
                                       NCU_TRAFFIC.get((top[0], n, kc, "tc_f16"))),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        line.update(legs)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
