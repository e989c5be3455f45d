"""The precision reading of the mixed solve with an FP32 level-1 basis, on the CPU.

The paper fixes no arithmetic precision.  The library's precision 2 keeps the FGMRES basis of
the fine level in FP32 and checks the tolerance on the FP64 true residual of the FP64 iterate,
recomputed at every restart.  The claim behind it: the preconditioned directions, and so
every correction, are FP32 in the mixed cycle anyway, and each restart refines the FP64
iterate, so rounding the basis, w = A x and the Gram-Schmidt update to FP32 changes the
iteration count only at the rounding level.  This test restates the outer cycle of Algorithm 2
(classical Gram-Schmidt, one pass, as the library runs it) with exactly those roundings
emulated around the oracle's preconditioner, and compares it with the same cycle in FP64 on
small seeded problems: both must reach the tolerance on the true residual, with iteration
counts within 15% of each other (measured differences: 0-12% on 1D C = 32-256 and 2D).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _cycle(H, f, u, restart, tol, fnorm, budget, basis32):
    """One restart cycle from u; x_j = fl32(Q_1 fl32(v_j)) in both variants (the FP32 cycle)."""
    lv = H.levels[0]
    r = f - lv.apply_A(u)
    beta = np.linalg.norm(r.ravel())
    v0 = r / beta
    V = [_f32(v0) if basis32 else v0]
    X = []
    Hm = np.zeros((restart + 1, restart))
    J = 0
    y = np.zeros(0)
    for j in range(restart):
        x = _f32(O.precondition(H, 0, _f32(V[j])))
        X.append(x)
        w = lv.apply_A(x)
        if basis32:
            w = _f32(w)
        h = np.array([np.vdot(w.ravel(), V[i].ravel()) for i in range(j + 1)])
        Hm[:j + 1, j] = h
        for i in range(j + 1):
            w = w - h[i] * V[i]
        if basis32:
            w = _f32(w)
        Hm[j + 1, j] = np.linalg.norm(w.ravel())
        J = j + 1
        e1 = np.zeros(J + 1)
        e1[0] = beta
        y = np.linalg.lstsq(Hm[:J + 1, :J], e1, rcond=None)[0]
        est = np.linalg.norm(e1 - Hm[:J + 1, :J] @ y)
        if est / fnorm < tol or J >= budget or Hm[j + 1, j] == 0.0:
            break
        vn = w / Hm[j + 1, j]
        V.append(_f32(vn) if basis32 else vn)
    d = sum(y[i] * X[i] for i in range(J))
    return u + d, J


def _solve(P, restart, tol, basis32, maxit=1500):
    s = P.schedule
    H = O.make_hierarchy(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, s.nu, s.space,
                         s.m_inner, s.n_cgs)
    f = O.assemble_rhs(P.u0, P.g, P.nt, P.theta, P.dt)
    fnorm = np.linalg.norm(f.ravel())
    u = np.zeros_like(f)
    total = 0
    while True:
        res = np.linalg.norm((f - H.levels[0].apply_A(u)).ravel()) / fnorm
        if res < tol or total >= maxit:
            return total, res, u
        u, J = _cycle(H, f, u, restart, tol, fnorm, maxit - total, basis32)
        total += J


CASES = {
    # 1D, theta = 1, C = 2 tau dt / h^2 = 2 * (1/512) * 128^2 = 64: the stiff regime
    "1d_n127_nt512_C64": lambda: W.custom(1, 127, 512, 1.0, 1.0, 1.0,
                                          W.Schedule((2, 2, 2), (False,) * 3, (2, 1), 0),
                                          seed=3, with_source=True),
    # 2D with 2 x 2 agglomeration, theta = 1/2
    "2d_31x31_nt64_TS": lambda: W.custom(2, 31, 64, 0.05, 1.0, 0.5,
                                         W.Schedule((2, 2), (True, True), (2,), 0), seed=3),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tol", [1e-8, 1e-11])
def test_fp32_basis_converges_like_fp64_basis(name, tol):
    P = CASES[name]()
    it64, res64, u64 = _solve(P, 12, tol, basis32=False)
    it32, res32, u32 = _solve(P, 12, tol, basis32=True)
    assert res64 < tol and res32 < tol, (res64, res32)
    assert abs(it32 - it64) <= max(2, 0.15 * it64), (it32, it64)
    # both iterates solve the same system: they agree to the tolerance's order
    ref = O.theta_march(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    assert O.max_rel_error(u32, ref) <= 1e3 * tol
    assert O.max_rel_error(u64, ref) <= 1e3 * tol
