"""FGMRES with recycled corrections (mk_solve_opts.augment = k): the GPU runs the oracle's
algorithm -- the last k slots of every restart cycle after the k-th take the corrections of
earlier cycles -- so in FP64 it needs the oracle's iteration count (within one: classical
against modified Gram-Schmidt) and reaches the unique solution of Eq. (finesys)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")


def _case():
    return W.heat1d_small()


@pytest.mark.parametrize("restart,augment", [(6, 1), (8, 2), (8, 3)])
def test_augmented_counts_match_oracle_fp64(restart, augment):
    P = _case()
    s = P.schedule
    H = O.make_hierarchy(1, P.nx, 1, P.nt, P.tau, P.theta, P.dt, s.nu, s.space, s.m_inner, s.n_cgs)
    f = O.assemble_rhs(P.u0, P.g, P.nt, P.theta, P.dt)
    uo, io = O.fgmres(H, f, 1e-11, restart=restart, augment=augment, maxit=800)
    ref = O.theta_march(1, P.nx, 1, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    o = mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=s.n_cgs,
                     tol=1e-11, restart=restart, precision="fp64", augment=augment, max_iters=800)
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, P.g) as p:
        u = np.empty_like(ref)
        info = mk.mk_solve(p.handle, P.u0, u, o)
    assert abs(info.iterations - io.iterations) <= max(1, io.iterations // 50), (info.iterations, io.iterations)
    assert info.restarts > augment
    assert O.max_rel_error(u, ref) <= 1e-10


@pytest.mark.parametrize("use_graph", [True, False])
def test_augmented_mixed_solution(use_graph):
    """Mixed precision (corrections stored in FP32, w = A x formed in FP64 then kept as
    double-float pairs): the solution within the mixed bound 1e-8, with and without graphs."""
    P = _case()
    s = P.schedule
    ref = O.theta_march(1, P.nx, 1, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    o = mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=s.n_cgs,
                     tol=1e-11, restart=8, precision="mixed", augment=2, max_iters=800,
                     use_graph=use_graph)
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, P.g) as p:
        u = np.empty_like(ref)
        info = mk.mk_solve(p.handle, P.u0, u, o)
    assert info.restarts > 2
    assert O.max_rel_error(u, ref) <= 1e-8, info.iterations


def test_augmented_2d_fp64():
    P = W.custom(2, 15, 32, 0.05, 1.0, 1.0, W.Schedule((2, 2), (True, True), (2,), 4), seed=92, ny=13,
                 with_source=True)
    s = P.schedule
    ref = O.theta_march(2, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    o = mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=s.n_cgs,
                     tol=1e-12, restart=5, precision="fp64", augment=2, max_iters=800)
    with mk.Problem(2, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        u = np.empty_like(ref)
        mk.mk_solve(p.handle, P.u0, u, o)
    assert O.max_rel_error(u, ref) <= 1e-10


def test_augmented_full_size_at_bench_tolerance():
    """The 1D workload (n = 1023, n_t = 8192, 5 levels, mixed), restart 16 with 2 recycled
    corrections: within the metric's 1e-8 of the oracle."""
    P = W.heat1d_large(precision="mixed")
    s = P.schedule
    ref = O.theta_march(1, P.nx, 1, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    o = mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=2,
                     tol=1e-8, restart=16, precision="mixed", orth=0, augment=2)
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, P.g) as p:
        u = np.empty_like(ref)
        info = mk.mk_solve(p.handle, P.u0, u, o)
    assert info.rel_residual < 1e-8
    assert O.max_rel_error(u, ref) <= 1e-8, info.iterations


def test_augment_rejected():
    P = _case()
    s = P.schedule
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, P.g) as p:
        u = np.empty((P.nt + 1, P.nx))
        for aug, restart in ((8, 8), (9, 20), (-1, 8)):
            o = mk.make_opts(levels=s.levels, nu=s.nu, m_inner=s.m_inner, restart=restart, augment=aug)
            with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
                mk.mk_solve(p.handle, P.u0, u, o)
        o = mk.make_opts(levels=s.levels, nu=s.nu, m_inner=s.m_inner, restart=8, augment=2)
        with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
            mk.mk_create_batch([p.handle], [o])
