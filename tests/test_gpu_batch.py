"""Batched solves (mk_create_batch / mk_solve_batch): many independent problems of uneven
size, dimension, theta and tau advanced together by one CUDA graph per restart cycle.

Every member must match the CPU oracle's theta-march (the unique solution of Eq. (finesys))
within the solve tolerances of the single-problem tests (FP64 1e-10, mixed 1e-8 max relative
error); without autotuning a member must reproduce the single-problem mk_solve bit for bit
(same hierarchy, kernels and reduction order, only run on a graph branch).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")


def _opts(P: W.Problem, precision, tol=1e-12, max_iters=2000):
    s = P.schedule
    return mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=s.n_cgs,
                        tol=tol, precision=precision, max_iters=max_iters)


def _members():
    S2 = W.Schedule((2, 2), (False, False), (1,), 8)
    S3 = W.Schedule((2, 2, 2), (False,) * 3, (2, 1), 4)
    TS = W.Schedule((2, 2), (True, True), (1,), 4)
    return [
        W.custom(1, 63, 256, 0.1, 1.0, 0.5, S2, seed=41, with_source=True),
        W.custom(1, 127, 512, 0.5, 2.0, 1.0, S3, seed=42),
        W.custom(1, 100, 64, 0.05, 0.3, 0.5, TS, seed=43, with_source=True),
        W.custom(2, 15, 64, 0.05, 1.0, 1.0, TS, seed=44, ny=13),
        W.custom(1, 255, 128, 0.2, 5.0, 1.0, S2, seed=45),
        W.custom(2, 31, 32, 0.02, 0.5, 0.5, W.Schedule((2,), (True,), (), 4), seed=46, ny=31,
                 with_source=True),
    ]


def _handles(ms):
    return [mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) for P in ms]


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-10), ("mixed", 1e-8), ("mixed32", 1e-8)])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_oracle(precision, bound, autotune):
    ms = _members()
    probs = _handles(ms)
    opts = [_opts(P, precision) for P in ms]
    outs = [np.empty((P.nt + 1,) + P.space_shape()) for P in ms]
    with mk.Batch(probs, opts, autotune=autotune) as b:
        infos = b.solve([P.u0 for P in ms], outs)
    for P, u, info in zip(ms, outs, infos):
        ref = O.theta_march(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
        assert O.max_rel_error(u, ref) <= bound, P.name
        assert info.rel_residual <= 1e-12 * 1.0001
        assert info.iterations > 0 and info.levels == P.schedule.levels
    for p in probs:
        p.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed32"])
def test_batch_equals_single_solves(precision):
    ms = _members()
    probs = _handles(ms)
    opts = [_opts(P, precision) for P in ms]
    single = []
    for P, p, o in zip(ms, probs, opts):
        u = np.empty((P.nt + 1,) + P.space_shape())
        info = mk.mk_solve(p.handle, P.u0, u, o)
        single.append((u, info.iterations))
    outs = [np.empty((P.nt + 1,) + P.space_shape()) for P in ms]
    with mk.Batch(probs, opts, autotune=False) as b:
        infos = b.solve([P.u0 for P in ms], outs)
        # a second solve with the same batch (the graph is replayed from a fresh start)
        outs2 = [np.empty_like(u) for u in outs]
        infos2 = b.solve([P.u0 for P in ms], outs2)
    for (u1, it1), u, info, u2, info2 in zip(single, outs, infos, outs2, infos2):
        assert info.iterations == it1 == info2.iterations
        assert np.array_equal(u, u1)
        assert np.array_equal(u2, u1)
    for p in probs:
        p.close()


def test_batch_member_not_converged():
    ms = _members()[:3]
    probs = _handles(ms)
    opts = [_opts(P, "fp64") for P in ms]
    s1 = ms[1].schedule
    opts[1] = mk.make_opts(levels=s1.levels, nu=s1.nu, space=s1.space, m_inner=s1.m_inner,
                           n_cgs=s1.n_cgs, tol=1e-12, restart=2, max_iters=3)
    outs = [np.empty((P.nt + 1,) + P.space_shape()) for P in ms]
    with mk.Batch(probs, opts) as b:
        with pytest.raises(mk.MKError, match="MK_ERR_NOT_CONVERGED"):
            b.solve([P.u0 for P in ms], outs)
        infos = b.solve([P.u0 for P in ms], outs, allow_not_converged=True)
    assert infos[1].iterations == 4 and infos[1].rel_residual > 1e-12
    for k in (0, 2):
        P = ms[k]
        ref = O.theta_march(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
        assert O.max_rel_error(outs[k], ref) <= 1e-10
    for p in probs:
        p.close()


def test_batch_invalid_arguments():
    ms = _members()[:2]
    probs = _handles(ms)
    with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
        mk.mk_create_batch([probs[0].handle, probs[0].handle])
    with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
        mk.mk_create_batch([])
    bad = [_opts(ms[0], "fp64"), mk.make_opts(levels=3, nu=(3, 3))]   # nt not divisible
    with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
        mk.mk_create_batch([p.handle for p in probs], bad)
    for p in probs:
        p.close()


@pytest.fixture(scope="module")
def uneven_full():
    ms = W.batched_problems(seed=4, count_1d=6, count_2d=2)
    refs = [O.theta_march(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g) for P in ms]
    return ms, refs


@pytest.mark.parametrize("precision", ["mixed", "mixed32"])
def test_batch_uneven_members_full_size(uneven_full, precision):
    """Members of the uneven batched workload at their full sizes (1D: n in 63..2047, n_t in
    256..8192; 2D: side in 63..255, n_t in 128..1024; tau in [0.1, 10], theta in {1/2, 1}; end
    time from a Courant number in the range of its theta; the 3-level 1D and 4-level 2D
    schedules, both mixed modes, tol 1e-10).  Every member must converge and match the oracle's
    march within the metric's 1e-8 max relative error."""
    ms, refs = uneven_full
    probs = _handles(ms)
    opts = [_opts(P, precision, tol=1e-10, max_iters=2000) for P in ms]
    outs = [np.empty((P.nt + 1,) + P.space_shape()) for P in ms]
    with mk.Batch(probs, opts) as b:
        infos = b.solve([P.u0 for P in ms], outs)
    for P, u, info, ref in zip(ms, outs, infos, refs):
        assert info.rel_residual <= 1e-10 * 1.0001, (P.name, info.iterations)
        assert O.max_rel_error(u, ref) <= 1e-8, (P.name, P.nx, P.nt)
    for p in probs:
        p.close()
