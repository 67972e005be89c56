"""Writes the oracle's end-to-end solve errors for the full-size workloads:

  solve1d_N65536.txt  d = 1, N = 2^16, Phi = x xi + c(x)|xi|, r = 16, HSS leaf 128,
                      oversample 10, tol 1e-3, Philox seed 2, f_true = crandn(N, 2, seed 3)
  solve2d_n128.txt    d = 2, n = 128 (N = 16384), elliptic phase, r = 5 x 5, leaf 256,
                      oversample 10, tol 1e-3, Philox seed 1, f_true = crandn(N, 2, seed 0)

with u = K~ f_true through the oracle's own BF (Section 5) and e_direct =
||f^ - f_true|| / ||f_true||.  Calls only oracle/ and the shared input generator.

    python tests/golden/make_solve_golden.py 1d|2d
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from fio_inputs import crandn  # noqa: E402
from oracle.problem import Phase  # noqa: E402
from oracle.solver import FIOSolver, FIOSolver2D, rel_err  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = {
    "1d": dict(file="solve1d_N65536.txt", d=1, n=1 << 16, r=16, leaf=128, p=10, tol=1e-3, seed=2, seed_f=3),
    "2d": dict(file="solve2d_n128.txt", d=2, n=128, r=5, leaf=256, p=10, tol=1e-3, seed=1, seed_f=0),
}


def main(which):
    c = CASES[which]
    t0 = time.time()
    if c["d"] == 1:
        S = FIOSolver(Phase("cabs"), c["n"], c["r"], c["leaf"], c["p"], c["tol"], c["seed"])
        N = c["n"]
    else:
        S = FIOSolver2D(Phase("elliptic2d"), c["n"], c["r"], c["leaf"], c["p"], c["tol"], c["seed"])
        N = c["n"] ** 2
    t1 = time.time()
    f = crandn(N, 2, seed=c["seed_f"])
    e = rel_err(S.solve(S.bf.apply(f)), f)
    out = os.path.join(HERE, c["file"])
    with open(out, "w") as fh:
        fh.write("# oracle solve, d=%d n=%d r=%d leaf=%d p=%d tol=%g seed=%d f=crandn(%d,2,seed=%d); "
                 "written by make_solve_golden.py (build %.0f s)\n"
                 % (c["d"], c["n"], c["r"], c["leaf"], c["p"], c["tol"], c["seed"], N, c["seed_f"], t1 - t0))
        fh.write("e_direct %.6e\n" % e)
        fh.write("ranks %s\n" % " ".join(str(r) for r in S.hss.ranks))
    print(open(out).read())


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "1d")
