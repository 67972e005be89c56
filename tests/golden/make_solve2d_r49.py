"""Writes solve2d_n{n}_r49.txt: the oracle's e_direct for the 2D solve on the 7 x 7 Chebyshev grid
(r = 49), HSS leaf 256, oversample 10, tol 1e-3, Philox seed 1, f_true = crandn(N, 2, seed 0),
u = K~ f_true with the oracle's BF.  Calls only oracle/ and the shared input generator.

    python tests/golden/make_solve2d_r49.py 128
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from fio_inputs import crandn  # noqa: E402
from oracle.problem import Phase  # noqa: E402
from oracle.solver import FIOSolver2D, rel_err  # noqa: E402


def main(n):
    r1, leaf, p, tol, seed = 7, 256, 10, 1e-3, 1
    S = FIOSolver2D(Phase("elliptic2d"), n, r1, leaf, p, tol, seed)
    f = crandn(n * n, 2, seed=0)
    e = rel_err(S.solve(S.bf.apply(f)), f)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve2d_n%d_r49.txt" % n)
    with open(out, "w") as fh:
        fh.write("# oracle 2D solve, n=%d r1=7 leaf=256 p=10 tol=1e-3 seed=1 f=crandn(%d,2,seed=0); "
                 "written by make_solve2d_r49.py\n" % (n, n * n))
        fh.write("e_direct %.6e\n" % e)
        fh.write("ranks %s\n" % " ".join(str(r) for r in S.hss.ranks))
    print(open(out).read())


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 128)
