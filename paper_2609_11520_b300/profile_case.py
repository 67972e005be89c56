"""Run one stage of the online path repeatedly, for profilers.

    python -m paper_2609_11520_b300.profile_case --case fio_solve --n 65536 --k 64 --reps 3

Builds the operator (BF; BF + HSS + ULV for the solve cases) outside the
profiled range, then runs `reps` repetitions of the chosen case between
cudaProfilerStart and cudaProfilerStop, so that `ncu --profile-from-start off`
captures only those launches.  Cases:
  bf_adjoint   Y = K~^* X   (k columns)
  bf_forward   Y = K~ X
  hss_solve    X = G~^{-1} B
  fio_solve    f = G~^{-1} K~^* u   (one online step)
  bf2d_adjoint / bf2d_forward   the 2D quadtree BF (elliptic phase, r = 25), n per dimension
--precision split_bf16 runs the BF applies on the split-precision kernels.
Prints the mean CUDA-event time per repetition.
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2609_11520_b300 import BF, HSS, fio_solve  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="fio_solve",
                    choices=["bf_adjoint", "bf_forward", "hss_solve", "fio_solve", "bf2d_adjoint", "bf2d_forward"])
    ap.add_argument("--n", type=int, default=1 << 16)
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--r", type=int, default=16)
    ap.add_argument("--leaf", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split_bf16"])
    args = ap.parse_args()
    torch.cuda.set_device(0)
    two_d = args.case.startswith("bf2d")
    bf = BF(args.n, 25, "elliptic2d") if two_d else BF(args.n, args.r)
    hss = None
    if args.case in ("hss_solve", "fio_solve"):
        hss = HSS.from_samples(bf=bf, leaf=args.leaf, oversample=10, tol=args.tol, seed=2).factor()
    if not two_d:
        bf.set_precision(args.precision)
    rng = np.random.default_rng(0)
    X = torch.from_numpy((rng.standard_normal((args.k, bf.n)) + 1j * rng.standard_normal((args.k, bf.n)))
                         .astype(np.complex64)).cuda()
    Y = torch.empty_like(X)

    def run():
        if args.case in ("bf_adjoint", "bf2d_adjoint"):
            bf.apply(X, adjoint=True, out=Y)
        elif args.case in ("bf_forward", "bf2d_forward"):
            bf.apply(X, out=Y)
        elif args.case == "hss_solve":
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
    print(f"{args.case} n={args.n} k={args.k}: {a.elapsed_time(b) / args.reps:.4f} ms per repetition")


if __name__ == "__main__":
    main()
