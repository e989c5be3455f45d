"""Writes table2_iterations_mgrit_large_oracle.txt: the oracle's FGMRES iteration counts for
the two larger rows of Table 2 (Sec. 3.3.1), MGRIT-based columns (Y of Eq. (mgritY), Z of
Eq. (mgritZ), coarse matrix of Eq. (coarsemat)), with the seeded initial state of the other
Table 2 pins (uniform random u_0, generator seed 7), exact coarse solve, mu = 1, theta = 1/2,
C = 0.64, tol 1e-6.  Calls only the oracle; about ten minutes on one CPU core.  Run from the
repository root: python tests/golden/make_table2_mgrit_large_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

ROWS = [(512, 2048), (1024, 8192)]


def main():
    lines = ["# Oracle FGMRES iterations (seeded uniform-random u_0, seed 7) for the two larger",
             "# rows of Table 2 (Sec. 3.3.1), MGRIT-based columns; written by",
             "# make_table2_mgrit_large_oracle.py.",
             "# columns: n_x n_t iters(nu=2) iters(nu=4) iters(nu=8)"]
    for n, nt in ROWS:
        h = 1.0 / (n + 1)
        dt = 0.32 * h * h
        u0 = np.random.default_rng(7).uniform(size=n)
        f = O.assemble_rhs(u0, None, nt, 0.5, dt)
        its = []
        for nu in (2, 4, 8):
            H = O.make_hierarchy(1, n, 1, nt, 1.0, 0.5, dt, (nu,), (False,), (), 0,
                                 mu_mode="one", transfer="mgrit")
            _, info = O.fgmres(H, f, 1e-6, restart=200, maxit=200)
            its.append(info.iterations)
        lines.append(" ".join(str(v) for v in (n, nt, *its)))
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "table2_iterations_mgrit_large_oracle.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
