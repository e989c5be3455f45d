"""The schedule autotuner (mk_tune) on small seeded problems: it returns options under which
the solve converges to the oracle's solution, never slower than its starting point, within
its trial budget."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")


@pytest.mark.parametrize("levels_flag", [False, True])
def test_tune_picks_converging_options(levels_flag):
    P = W.custom(1, 127, 512, 0.5, 1.0, 1.0, W.Schedule((2, 2, 2), (False,) * 3, (2, 1), 16),
                 seed=51, with_source=True)
    ref = O.theta_march(1, P.nx, 1, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    base = mk.make_opts(levels=4, nu=(2, 2, 2), m_inner=(2, 1), n_cgs=16, tol=1e-9,
                        precision="mixed", max_iters=600)
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, P.g) as p:
        u = np.empty((P.nt + 1, P.nx))
        b_info = mk.mk_solve(p.handle, P.u0, u, base)
        best, info = mk.mk_tune(p.handle, P.u0, base, levels=levels_flag, max_trials=24)
        assert 1 <= info.trials <= 24
        assert info.best_iterations >= 1 and info.best_ms > 0.0 and info.tune_ms >= info.best_ms
        assert best.levels <= 4 and (levels_flag or best.levels == 4)
        assert best.tol == base.tol and best.precision == 1
        i2 = mk.mk_solve(p.handle, P.u0, u, best)
    assert i2.rel_residual < 1e-9
    assert O.max_rel_error(u, ref) <= 1e-8
    # the re-solve rebuilds the hierarchy and re-times its tiles; a different tile choice sums
    # in another order, and FGMRES at this tolerance moves by a few iterations with the
    # rounding (5% of the count, at least 2)
    assert abs(info.best_iterations - i2.iterations) <= max(2, 0.05 * i2.iterations)
    # the starting point is a candidate, so the pick is not slower than it (same device, up
    # to timing noise; its first solve also built the hierarchy)
    assert info.best_ms <= 1.5 * b_info.solve_ms


def test_tune_rejects_bad_arguments():
    P = W.heat1d_small()
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt) as p:
        with pytest.raises(mk.MKError):
            mk.mk_tune(p.handle, None)
