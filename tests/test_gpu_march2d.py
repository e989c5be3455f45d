"""Sequential 2D theta-march on the GPU (Eq. (timemarch)) by one sine-transform solve per
step: an FFT in directions whose n + 1 is a power of two (n <= 2047), the dense sine matrix
in the others (n <= 1024); larger grids are rejected.

Against the oracle's march (sparse LU per step, FP64), max relative error within
max(1e-12, 8 eps n_t (1 + 4 max(a, b)(cx + cy))): each step rounds the explicit part
u + b L u, whose size is up to 1 + 4 b (cx + cy) times |u| for the highest modes (cx = tau /
h_x^2), and the implicit solve divides by 1 - a lambda; the theta-scheme's amplification
factors are at most 1 in modulus, so the rounding of the steps adds up at most linearly, on
both sides.  At the 255 x 255, n_t = 1024 size the first 24 steps are compared with the
oracle and the whole march must satisfy Eq. (finesys) to 1e-12 relative residual.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")

S = W.Schedule((2,), (True,), (), 4)


def _bound(P, steps=None):
    cx, cy = P.tau * (P.nx + 1) ** 2, P.tau * (P.ny + 1) ** 2
    ab = max(P.theta, 1.0 - P.theta) * P.dt
    k = P.nt if steps is None else steps
    return max(1e-12, 8 * np.finfo(float).eps * k * (1 + 4 * ab * (cx + cy)))


@pytest.mark.parametrize("nx,ny,nt,theta,src", [
    (63, 63, 64, 0.5, False),
    (127, 63, 32, 1.0, True),
    (31, 255, 16, 0.5, True),
    (7, 3, 40, 1.0, True),
    (1023, 15, 8, 0.5, False),
    (100, 60, 16, 0.5, True),
    (192, 192, 12, 0.5, False),
    (127, 50, 10, 1.0, True),
    (1, 1, 5, 0.5, True),
])
def test_march2d_sine_vs_oracle(nx, ny, nt, theta, src):
    P = W.custom(2, nx, nt, 0.05, 1.0, theta, S, seed=nx + ny, ny=ny, with_source=src)
    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        u = np.empty((P.nt + 1,) + P.space_shape())
        mk.mk_march(p.handle, P.u0, u)
    ref = O.theta_march(2, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, P.u0, P.g)
    assert O.max_rel_error(u, ref) <= _bound(P)


def test_march2d_full_size_sampled():
    P = W.heat2d_large()
    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        u = np.empty((P.nt + 1, P.ny, P.nx))
        mk.mk_march(p.handle, P.u0, u)
    ks = 24
    ref = O.theta_march(2, P.nx, P.ny, ks, P.tau, P.theta, P.dt, P.u0, None)
    assert O.max_rel_error(u[:ks + 1], ref) <= _bound(P, ks)
    lv = O.build_levels(2, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, (), (), "one")[0]
    f = O.assemble_rhs(P.u0, None, P.nt, P.theta, P.dt)
    assert np.linalg.norm(f - lv.apply_A(u)) / np.linalg.norm(f) <= 1e-12


def test_march2d_unsupported_size():
    P = W.custom(2, 1100, 4, 0.05, 1.0, 1.0, S, seed=5, ny=3)
    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        u = np.empty((P.nt + 1,) + P.space_shape())
        with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
            mk.mk_march(p.handle, P.u0, u)
