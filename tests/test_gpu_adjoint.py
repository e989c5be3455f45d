"""Adjoint gradients at the size of the adjoint workload: 2D 127 x 127, theta = 1, n_t = 512,
T = 0.05, loss J = ||u_nt - u_target||^2, 4 levels with 2 x 2 agglomeration, FP64.

* against the oracle's adjoint march (the discrete adjoint of Eq. (finesys) solved
  sequentially on the CPU): 1e-9 relative;
* through the torch.autograd.Function (forward = MK solve, backward = adjoint MK solve)
  against central finite differences of the GPU forward solve along seeded directions:
  1e-6 relative.  J is quadratic in u_0 and g, so their central differences are exact for
  any step and only the solves' rounding enters, divided by the step: a step of 1e-3 keeps
  that term near 1e-9 (with 1e-6 it reaches a few 1e-6 of a directional derivative that is
  1e-4 of J).  The tau difference has an O(step^2) truncation term; its step is 1e-6 tau.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")
torch = pytest.importorskip("torch")


def _opts(P, tol):
    s = P.schedule
    return mk.make_opts(levels=s.levels, nu=s.nu, space=s.space, m_inner=s.m_inner, n_cgs=s.n_cgs,
                        tol=tol, precision="fp64", max_iters=4000)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_adjoint_full_size_vs_oracle():
    P = W.heat2d_adjoint()
    J, gu0, gg, gtau, u_ref = O.misfit_gradients(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt,
                                                P.u0, P.g, P.u_target)
    o = _opts(P, 1e-12)
    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        u = np.empty((P.nt + 1,) + P.space_shape())
        mk.mk_solve(p.handle, P.u0, u, o)
        assert _rel(u, u_ref) <= 1e-10
        dJdu = np.zeros_like(u)
        dJdu[-1] = 2.0 * (u[-1] - P.u_target)
        g_u0 = np.empty(P.space_shape())
        g_g = np.empty_like(u)
        gt, info = mk.mk_adjoint(p.handle, u, dJdu, o, grad_u0=g_u0, grad_g=g_g, want_tau=True)
    assert info.rel_residual <= 1e-12 * 1.0001
    assert _rel(g_u0, gu0) <= 1e-9
    assert _rel(g_g, gg) <= 1e-9
    assert abs(gt - gtau) <= 1e-9 * abs(gtau)


def test_autograd_vs_central_differences():
    P = W.heat2d_adjoint()
    dev = torch.device("cuda:0")
    o = _opts(P, 1e-13)
    tgt = torch.from_numpy(P.u_target).to(dev)
    rng = np.random.default_rng(77)
    d_u0 = rng.standard_normal(P.space_shape())
    d_g = rng.standard_normal(P.g.shape)

    def loss(prob, u0, g, tau_t):
        u = mk.HeatSolve.apply(prob, u0, g, tau_t, o)
        return ((u[-1] - tgt) ** 2).sum()

    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, None, ny=P.ny) as p:
        u0 = torch.from_numpy(P.u0).to(dev).requires_grad_(True)
        g = torch.from_numpy(P.g).to(dev).requires_grad_(True)
        tau_t = torch.tensor(P.tau, dtype=torch.float64, device=dev, requires_grad=True)
        J = loss(p, u0, g, tau_t)
        J.backward()
        grads = (u0.grad.cpu().numpy(), g.grad.cpu().numpy(), float(tau_t.grad))

        def J_at(du0=0.0, dg=0.0):
            with torch.no_grad():
                x0 = torch.from_numpy(P.u0 + du0).to(dev)
                gx = torch.from_numpy(P.g + dg).to(dev)
                return float(loss(p, x0, gx, torch.tensor(P.tau, dtype=torch.float64)))

        h = 1e-3
        fd_u0 = (J_at(du0=h * d_u0) - J_at(du0=-h * d_u0)) / (2 * h)
        fd_g = (J_at(dg=h * d_g) - J_at(dg=-h * d_g)) / (2 * h)
    ad_u0 = float(np.sum(grads[0] * d_u0))
    ad_g = float(np.sum(grads[1] * d_g))
    assert abs(fd_u0 - ad_u0) <= 1e-6 * abs(ad_u0)
    assert abs(fd_g - ad_g) <= 1e-6 * abs(ad_g)

    # tau: a new problem for each perturbed diffusion coefficient
    ht = 1e-6 * P.tau
    Js = []
    for tau in (P.tau + ht, P.tau - ht):
        with mk.Problem(P.dim, P.nx, tau, P.theta, P.dt, P.nt, None, ny=P.ny) as pt:
            with torch.no_grad():
                Js.append(float(loss(pt, torch.from_numpy(P.u0).to(dev), torch.from_numpy(P.g).to(dev),
                                     torch.tensor(tau, dtype=torch.float64))))
    fd_tau = (Js[0] - Js[1]) / (2 * ht)
    assert abs(fd_tau - grads[2]) <= 1e-6 * abs(grads[2])


def test_heatsolve_leaves_the_problem_source():
    """HeatSolve solves with its own g, then restores the source the Problem holds: a plain
    solve on the same problem afterwards returns what it returned before."""
    sched = W.Schedule((2, 2), (False, False), (1,), 16)
    P = W.custom(1, 63, 256, 0.1, 1.0, 0.5, sched, seed=41, with_source=True)
    dev = torch.device("cuda:0")
    o = mk.make_opts(levels=3, nu=(2, 2), m_inner=(1,), n_cgs=16, tol=1e-12)
    u0 = torch.from_numpy(P.u0).to(dev)
    with mk.Problem(1, P.nx, P.tau, P.theta, P.dt, P.nt, torch.from_numpy(P.g).to(dev)) as p:
        before = torch.empty((P.nt + 1, P.nx), dtype=torch.float64, device=dev)
        mk.mk_solve(p.handle, u0, before, o)
        g_other = torch.from_numpy(3.0 * P.g + 1.0).to(dev)
        u = mk.HeatSolve.apply(p, u0, g_other, torch.tensor(P.tau, dtype=torch.float64), o)
        after = torch.empty_like(before)
        mk.mk_solve(p.handle, u0, after, o)
        assert torch.equal(before, after)
        assert not torch.allclose(u, before)
