"""Writes tests/golden/oracle_iterations_2d_1024.txt: the oracle's own CG
iteration counts for the 1024 x 1024 elliptic workload (32 seeded Gaussians,
seed 0, tol 1e-8, FD preconditioner for alpha >= 1, plain CG below), used
to scale the oracle's timed per-iteration cost to whole solves.

Calls only the oracle and the seeded input generator.  Test infrastructure.
Usage: python -m oracle.iteration_counts
"""

import os
import time

from oracle import solvers
from oracle.operator import Plan
from paper_1802_03770_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "golden", "oracle_iterations_2d_1024.txt")


def main(n=1024, alphas=(0.5, 1.0, 1.5), tol=1e-8):
    f = inputs.gaussian_mixture(n, 2, 32, 0)
    rows = []
    for alpha in alphas:
        p = Plan(2, n, 1.0 / (n + 1), alpha)
        t = time.time()
        _, its, ok, _ = solvers.solve_elliptic(p, f, tol, 4000, alpha >= 1.0)
        assert ok
        rows.append((alpha, its, time.time() - t))
        print(alpha, its, f"{time.time() - t:.1f}s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# FP64 CG iteration counts of the oracle on the 1024 x 1024 elliptic\n"
                 "# workload: 32 seeded Gaussians (seed 0, widths U(0.05, 0.2)),\n"
                 "# tol 1e-8, FD preconditioner for alpha >= 1, none below.\n"
                 "# Written by `python -m oracle.iteration_counts` (oracle only).\n"
                 "# columns: n alpha iterations\n")
        for alpha, its, _ in rows:
            fh.write(f"{n} {alpha:.2f} {its}\n")


if __name__ == "__main__":
    main()
