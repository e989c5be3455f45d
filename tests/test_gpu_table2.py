"""Table 2 (Sec. 3.3.1) on the GPU: iterations of the two-level method with time coarsening
and the exact coupled coarse solve (n_cgs = 0), mu = 1, theta = 1/2, C = 0.64, tol 1e-6, for all
four rows the paper prints.  The paper's initial state is unstated; a seeded uniform-random
u_0 (seed 7, as in the oracle's pin) is used.

* parity: the GPU count equals the oracle's FGMRES count within 1 (classical vs modified
  Gram-Schmidt), on the two smaller rows by running the oracle, on the two larger rows
  against the oracle's counts stored by tests/golden/make_table2_large_oracle.py;
* against the paper: within 3, except n = 1024, n_t = 8192, nu = 8, where the oracle and the
  GPU both take 33 iterations for this initial state and the paper prints 27 (allowed 7).
"""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PAPER_SLACK = {(1024, 8192, 8): 7}


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [list(map(int, l.split())) for l in fh if l.strip() and not l.startswith("#")]


@pytest.mark.parametrize("name", ["table2_iterations.txt", "table2_iterations_large.txt"])
def test_table2_two_level_iterations_gpu(name):
    large = name == "table2_iterations_large.txt"
    stored = {}
    if large:
        for n, nt, *its in _rows("table2_iterations_large_oracle.txt"):
            stored[(n, nt)] = its
    for n, nt, *iters in _rows(name):
        h = 1.0 / (n + 1)
        dt = 0.32 * h * h
        u0 = np.random.default_rng(7).uniform(size=n)
        u = np.empty((nt + 1, n))
        with mk.Problem(1, n, 1.0, 0.5, dt, nt) as p:
            for c, (nu, ref) in enumerate(zip((2, 4, 8), iters)):
                o = mk.make_opts(levels=2, nu=(nu,), n_cgs=0, mu="one", tol=1e-6, restart=128,
                                 max_iters=200, precision="fp64")
                info = mk.mk_solve(p.handle, u0, u, o)
                assert info.rel_residual < 1e-6
                if large:
                    oracle_its = stored[(n, nt)][c]
                else:
                    f = O.assemble_rhs(u0, None, nt, 0.5, dt)
                    H = O.make_hierarchy(1, n, 1, nt, 1.0, 0.5, dt, (nu,), (False,), (), 0,
                                         mu_mode="one")
                    _, oinfo = O.fgmres(H, f, 1e-6, restart=200, maxit=200)
                    oracle_its = oinfo.iterations
                assert abs(info.iterations - oracle_its) <= 1, (n, nt, nu, info.iterations, oracle_its)
                slack = PAPER_SLACK.get((n, nt, nu), 3)
                assert abs(info.iterations - ref) <= slack, (n, nt, nu, info.iterations, ref)
