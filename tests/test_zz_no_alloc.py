"""Allocation-free residual (mk_op_residual_noalloc) against the allocating entry point
mk_op_residual, through the C ABI.

The file name sorts last, so the same tests run after every other GPU test has used the
library as well as alone in a fresh process.  Inputs are seeded device tensors; each case
makes two calls in a row with different inputs (the second call must see the reduction
counter left at zero by the first), then repeats the first call, which must reproduce its
outputs bit for bit.

Tolerance: each r entry is a sum of at most 11 products of inputs, so the two entry points,
which round in different orders, agree to a few ulps of
S = max|f| + (1 + 4 (a + b) (cx + cy)) max|u|; the test allows 16 eps S.  The norms agree to
1e-12 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")
torch = pytest.importorskip("torch")

EPS = np.finfo(np.float64).eps

# (dim, nx, ny, nt, tau, theta, dt): ragged chunk tails, one and several chunks per step,
# 1D and 2D, the 8193 x 1023 heat workload, and the largest accepted size.
CASES = {
    "1d_n63_nt256": (1, 63, 1, 256, 1.0, 0.5, 0.1 / 256),
    "1d_n2100_nt31": (1, 2100, 1, 31, 0.7, 1.0, 0.01),
    "2d_45x47_nt17": (2, 45, 47, 17, 1.0, 0.5, 0.002),
    "2d_70x61_nt9": (2, 70, 61, 9, 0.3, 0.0, 0.001),
    "1d_n1023_nt8192": (1, 1023, 1, 8192, 1.0, 1.0, 1.0 / 8192),
    "1d_n2049_nt32767_max": (1, 2049, 1, 32767, 1.0, 0.5, 1e-5),
}


def _needed(nx, ny, nt):
    chunk = mk._lib.MK_NOALLOC_CHUNK
    return (nt + 1) * ((nx * ny + chunk - 1) // chunk)


def _scale(dim, nx, ny, theta, dt, tau, f, u):
    cx = tau * (nx + 1) ** 2
    cy = tau * (ny + 1) ** 2 if dim == 2 else 0.0
    return float(f.abs().max()) + (1.0 + 4.0 * dt * (cx + cy)) * float(u.abs().max())


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_residual(name):
    dim, nx, ny, nt, tau, theta, dt = CASES[name]
    assert _needed(nx, ny, nt) <= mk._lib.MK_NOALLOC_MAX_PARTIALS
    dev = torch.device("cuda:0")
    shape = (nt + 1, nx) if dim == 1 else (nt + 1, ny, nx)
    gen = torch.Generator(device="cpu").manual_seed(1000 + len(name))
    ins = [(torch.randn(shape, generator=gen, dtype=torch.float64).to(dev),
            torch.randn(shape, generator=gen, dtype=torch.float64).to(dev)) for _ in range(2)]
    outs = [(torch.full(shape, np.nan, dtype=torch.float64, device=dev),
             torch.full((1,), np.nan, dtype=torch.float64, device=dev),
             torch.full((nt + 1,), np.nan, dtype=torch.float64, device=dev)) for _ in range(3)]
    with mk.Problem(dim, nx, tau, theta, dt, nt, None, ny=ny) as p:
        torch.cuda.synchronize()
        # first call (looks up the static scratch), second call with other inputs
        mk.mk_op_residual_noalloc(p.handle, ins[0][0], ins[0][1], *outs[0])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        n0 = mk.mk_kernel_launch_count()
        mk.mk_op_residual_noalloc(p.handle, ins[1][0], ins[1][1], *outs[1])
        mk.mk_op_residual_noalloc(p.handle, ins[0][0], ins[0][1], *outs[2])
        torch.cuda.synchronize()
        assert mk.mk_kernel_launch_count() - n0 == 2
        assert torch.cuda.mem_get_info(dev)[0] == free0   # nothing allocated
        # the allocating entry point on the same inputs
        for (f, u), (r, rn, rs) in zip(ins, outs[:2]):
            r_ref = torch.empty_like(f)
            nrm_ref = mk.mk_op_residual(p.handle, f, u, r_ref)
            S = _scale(dim, nx, ny, theta, dt, tau, f, u)
            assert float((r - r_ref).abs().max()) <= 16 * EPS * S
            assert abs(float(rn[0]) - nrm_ref) <= 1e-12 * nrm_ref
            steps_ref = torch.linalg.vector_norm(r_ref.reshape(nt + 1, -1), dim=1)
            assert float(((rs - steps_ref).abs() / steps_ref).max()) <= 1e-12
    # the repeated call reproduces the first bit for bit
    for a, b in zip(outs[0], outs[2]):
        assert torch.equal(a, b)


def test_noalloc_optional_outputs():
    dim, nx, ny, nt, tau, theta, dt = CASES["2d_45x47_nt17"]
    dev = torch.device("cuda:0")
    gen = torch.Generator(device="cpu").manual_seed(7)
    f = torch.randn((nt + 1, ny, nx), generator=gen, dtype=torch.float64).to(dev)
    u = torch.randn((nt + 1, ny, nx), generator=gen, dtype=torch.float64).to(dev)
    rn_full = torch.zeros(1, dtype=torch.float64, device=dev)
    rn_only = torch.zeros(1, dtype=torch.float64, device=dev)
    r = torch.empty_like(f)
    with mk.Problem(dim, nx, tau, theta, dt, nt, None, ny=ny) as p:
        mk.mk_op_residual_noalloc(p.handle, f, u, r, rn_full)
        mk.mk_op_residual_noalloc(p.handle, f, u, None, rn_only)
        torch.cuda.synchronize()
    assert torch.equal(rn_full, rn_only)
    assert abs(float(rn_full[0]) - float(torch.linalg.vector_norm(r))) <= 1e-12 * float(rn_full[0])


def test_noalloc_rejects():
    dev = torch.device("cuda:0")
    # one time step beyond the largest accepted size: rejected before any launch
    nx, nt = 2049, 32768
    assert _needed(nx, 1, nt) > mk._lib.MK_NOALLOC_MAX_PARTIALS
    f = torch.zeros((nt + 1, nx), dtype=torch.float64, device=dev)
    u = torch.zeros_like(f)
    rn = torch.zeros(1, dtype=torch.float64, device=dev)
    with mk.Problem(1, nx, 1.0, 0.5, 1e-5, nt, None) as p:
        n0 = mk.mk_kernel_launch_count()
        with pytest.raises(mk.MKError, match="MK_ERR_TOO_LARGE"):
            mk.mk_op_residual_noalloc(p.handle, f, u, None, rn)
        assert mk.mk_kernel_launch_count() == n0
    del f, u
    # host arrays are rejected (the call never stages)
    with mk.Problem(1, 31, 1.0, 0.5, 0.01, 8, None) as p:
        fh = np.zeros((9, 31))
        uh = np.zeros((9, 31))
        with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
            mk.mk_op_residual_noalloc(p.handle, fh, uh, None, rn)
        fd = torch.zeros((9, 31), dtype=torch.float64, device=dev)
        with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
            mk.mk_op_residual_noalloc(p.handle, fd, fd, None, np.zeros(1))
