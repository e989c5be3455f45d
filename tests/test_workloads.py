"""The seeded synthetic inputs follow their stated recipe (no GPU).

The discrete sine vectors s_k(i) = sin(k pi x_i), x_i = i/(n+1), are orthogonal on the n
interior points with <s_k, s_l> = (n+1)/2 delta_kl (k, l <= n), so each input's mode content
is recovered by projection and compared with the recipe: the smooth initial states
sin(pi x) + sum_{k<=8} a_k k^-2 sin(k pi x) (2D: sin(pi x) sin(pi y) +
sum_{k,l<=8} a_kl/(k^2+l^2) sin(k pi x) sin(l pi y)), a ~ N(0,1); the sources
sum_{m<=4} c_m sin(p_m pi x) sin(q_m pi t/T) with p_m <= 8, q_m <= 4; the batch ranges.
"""
import math

import numpy as np
import pytest

import workloads as W


def _sine_basis(n, kmax):
    x = np.arange(1, n + 1) / (n + 1)
    return np.stack([np.sin(k * np.pi * x) for k in range(1, kmax + 1)])


def _coeffs_1d(u):
    n = u.shape[-1]
    S = _sine_basis(n, n)
    return (u @ S.T) * (2.0 / (n + 1))


def test_initial_state_1d_recipe():
    P = W.heat1d_large()
    assert P.u0.shape == (1023,) and P.u0.dtype == np.float64 and P.u0.flags.c_contiguous
    c = _coeffs_1d(P.u0)
    a = np.random.default_rng(1).standard_normal(8)          # the workload's first draw
    want = a / np.arange(1, 9) ** 2
    want[0] += 1.0
    assert np.abs(c[:8] - want).max() <= 1e-12
    assert np.abs(c[8:]).max() <= 1e-12


def test_source_1d_recipe():
    P = W.heat1d_large()
    g = P.g
    assert g.shape == (P.nt + 1, P.nx)
    c = _coeffs_1d(g)                                         # (nt+1, n) spatial modes per step
    active = np.where(np.abs(c).max(axis=0) > 1e-9)[0] + 1
    assert len(active) <= 4 and active.max() <= 8
    t = np.arange(P.nt + 1) * (P.T / P.nt)
    for k in active:
        # each spatial mode's time profile is a combination of sin(q pi t/T), q <= 4
        Tq = np.stack([np.sin(q * np.pi * t / P.T) for q in range(1, 5)], axis=1)
        coef, *_ = np.linalg.lstsq(Tq, c[:, k - 1], rcond=None)
        assert np.abs(Tq @ coef - c[:, k - 1]).max() <= 1e-10
    assert np.abs(g[0]).max() == 0.0                          # sin(0) = 0 at t = 0


def test_initial_state_2d_recipe():
    n = 31
    u = W.smooth_modes_2d(np.random.default_rng(9), n, n)
    S = _sine_basis(n, n)
    c = (S @ u @ S.T) * (2.0 / (n + 1)) ** 2                  # c[l-1, k-1]: sin(l pi y) sin(k pi x)
    a = np.random.default_rng(9).standard_normal((8, 8))      # a[k-1, l-1]
    k = np.arange(1, 9)
    want = (a / (k[:, None] ** 2 + k[None, :] ** 2)).T
    want[0, 0] += 1.0
    assert np.abs(c[:8, :8] - want).max() <= 1e-12
    c[:8, :8] = 0.0
    assert np.abs(c).max() <= 1e-12


def test_workloads_are_seeded():
    a, b = W.heat1d_large(), W.heat1d_large()
    assert np.array_equal(a.u0, b.u0) and np.array_equal(a.g, b.g)
    assert not np.array_equal(W.heat1d_large(seed=2).u0, a.u0)


def test_named_workload_parameters():
    P = W.heat1d_small()
    assert (P.nx, P.nt, P.theta, P.T) == (63, 256, 0.5, 0.1) and P.g is None
    P = W.heat1d_large()
    assert (P.nx, P.nt, P.theta, P.T, P.tau) == (1023, 8192, 1.0, 1.0, 1.0)
    assert P.schedule.levels == 5 and P.schedule.n_cgs == 16
    P = W.heat2d_alternate(9)
    h = 1.0 / (P.nx + 1)
    assert abs(3 * P.tau * P.dt / h ** 2 - 0.16) <= 1e-12
    assert P.schedule.levels == 9


def test_batched_workload_ranges():
    probs = W.batched_problems()
    one = [p for p in probs if p.dim == 1]
    two = [p for p in probs if p.dim == 2]
    assert len(one) == 48 and len(two) == 16
    for p in one:
        assert 63 <= p.nx <= 2047 and 256 <= p.nt <= 8192 and p.nt % 64 == 0
    for p in two:
        assert 63 <= p.nx <= 255 and p.ny == p.nx and 128 <= p.nt <= 1024 and p.nt % 128 == 0
    for p in probs:
        assert 0.1 <= p.tau <= 10.0 and p.theta in (0.5, 1.0)
    # log-uniform diffusion coefficients: both decades are populated
    lt = np.log10([p.tau for p in probs])
    assert (lt < 0).any() and (lt > 0).any()


def test_batched_courant_numbers():
    """The end time of every batch member comes from a Courant number C = 2 tau dt / h^2 in the
    range of its theta (Crank-Nicolson up to 6.4, backward Euler up to 256), and the size,
    tau and theta draws do not depend on that reading."""
    probs = W.batched_problems()
    for p in probs:
        h = 1.0 / (p.nx + 1)
        C = 2.0 * p.tau * p.dt / h ** 2
        lo, hi = W.BATCH_C_RANGE[p.theta]
        assert lo * (1 - 1e-12) <= C <= hi * (1 + 1e-12), (p.name, C)
        assert abs(W.batch_end_time(C, p.nx, p.nt, p.tau) - p.T) <= 1e-12 * p.T
    cn = [2.0 * p.tau * p.dt * (p.nx + 1) ** 2 for p in probs if p.theta == 0.5]
    be = [2.0 * p.tau * p.dt * (p.nx + 1) ** 2 for p in probs if p.theta == 1.0]
    assert max(cn) > 1.0 and max(be) > 20.0   # both ranges reach well into C > 1
    small = W.batched_problems(count_1d=3, count_2d=1)
    assert [(p.nx, p.nt, p.tau, p.theta) for p in small[:3]] == \
        [(p.nx, p.nt, p.tau, p.theta) for p in probs[:3]]
