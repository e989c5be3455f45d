"""Writes table3_iterations_oracle.txt: the oracle's FGMRES iteration counts on the Table 3
workload (Sec. 4.2: 2D 192 x 192, n_t = 2^11, C = 0.16, theta = 1/2, alternate time-space
coarsening with 7..11 levels, 16 decoupled slabs, inner iterations 2 and 1 on the level above
the coarsest, mu = lambda_max, tol 1e-6) with the seeded smooth initial state of the
workload generator (seed 5).  Calls only the oracle and the input generator; about an hour
on one CPU core and up to ~30 GB of memory.  Run from the repository root:
python tests/golden/make_table3_oracle.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    lines = ["# Oracle FGMRES iterations on the Table 3 workload (Sec. 4.2) with the seeded smooth",
             "# initial state; written by make_table3_oracle.py.",
             "# columns: levels iterations"]
    for levels in range(7, 12):
        P = W.heat2d_alternate(levels)
        s = P.schedule
        H = O.make_hierarchy(2, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, s.nu, s.space,
                             s.m_inner, s.n_cgs)
        f = O.assemble_rhs(P.u0, None, P.nt, P.theta, P.dt)
        _, info = O.fgmres(H, f, 1e-6, restart=50, maxit=60)
        lines.append(f"{levels} {info.iterations}")
        print(lines[-1], info.rel_residual, flush=True)
        del H, f
    with open(os.path.join(HERE, "table3_iterations_oracle.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
