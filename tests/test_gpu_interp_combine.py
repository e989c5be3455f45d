"""Substeps 4.4-4.5 and step 5 of Algorithm 2 with the solve's full argument set -- the scaled
basis vector sigma v and the combination vt = sum_m y_m vt_m of the coarser level's inner
FGMRES directions -- through mk_op_interp_combine, against the oracle, in the three
arithmetic paths: FP64, FP32 and the level-1 double-float path of the mixed solve.

The double-float path forms x in FP32 and w = A x in double-float arithmetic.  Its x is
checked against the oracle's x at FP32 accuracy, and its w against the oracle's A applied to
the GPU's own x at double-float accuracy: a bound 2^18 times tighter than FP32 arithmetic
could meet, so a term evaluated in plain FP32 fails it.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")

# (dim, nx, ny, nt, theta, space): 2D grids spanning several 32 x 8 blocks of 2 x 2
# aggregates with ragged edges (odd sizes: a last aggregate of one column or row), time
# chunks with a ragged tail, square (cx = cy) and non-square grids (the 2D coarse grid stays
# within the 48-point limit of the FP64 coarsest solver), theta = 1/2 (b != 0) and
# theta = 1 (b = 0); time-only coarsening in 2D, and the 1D paths
CASES = {
    "2d_95x95_TS_half": (2, 95, 95, 40, 0.5, True),
    "2d_95x95_TS_one": (2, 95, 95, 40, 1.0, True),
    "2d_95x83_TS_half": (2, 95, 83, 40, 0.5, True),
    "2d_65x71_TS_one": (2, 65, 71, 34, 1.0, True),
    "2d_66x64_TS_half": (2, 66, 64, 24, 0.5, True),
    "2d_33x31_T_half": (2, 33, 31, 24, 0.5, False),
    "1d_301_TS_half": (1, 301, 1, 64, 0.5, True),
    "1d_300_T_one": (1, 300, 1, 64, 1.0, False),
}

# combination weights by number of coarse directions (0: y = NULL, the single vector as is);
# 5 directions exceed the fused 2D kernel's specialisations and take the general path
WEIGHTS = {0: None, 1: [0.7], 2: [1.3, -0.45], 3: [0.9, -0.3, 0.15],
           4: [1.1, 0.25, -0.6, 0.05], 5: [0.8, -0.2, 0.35, 0.1, -0.05]}
SIGMA = 1.37


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    dim, nx, ny, nt, theta, space = CASES[request.param]
    sched = W.Schedule((2,), (space,), (), 1)
    P = W.custom(dim, nx, nt, 0.05, 1.0, theta, sched, seed=61, ny=ny if dim == 2 else None)
    H = O.make_hierarchy(P.dim, P.nx, P.ny, P.nt, P.tau, P.theta, P.dt, sched.nu, sched.space,
                         sched.m_inner, sched.n_cgs)
    with mk.Problem(P.dim, P.nx, P.tau, P.theta, P.dt, P.nt, P.g, ny=P.ny) as p:
        yield sched, H, p


def _opts(sched, precision):
    return mk.make_opts(levels=2, nu=sched.nu, space=sched.space, n_cgs=1, precision=precision)


def _inputs(H, nvt, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(H.levels[0].shape())
    vt = rng.standard_normal((max(nvt, 1),) + H.levels[1].shape())
    return v, vt


def _x_reference(H, v, vt, y):
    """sigma v - Z vt with vt = sum_m y_m vt_m (Eq. (constructZ) for Z)."""
    comb = vt[0] if y is None else np.tensordot(np.asarray(y), vt, axes=1)
    return SIGMA * v - O.interpolate(H.levels[0], H.nu[0], H.space[0], comb)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
@pytest.mark.parametrize("nvt", [0, 1, 3])
def test_interp_combine_fp64_fp32(case, precision, tol, nvt):
    sched, H, p = case
    y = WEIGHTS[nvt]
    v, vt = _inputs(H, nvt, 50 + nvt)
    x = np.empty_like(v)
    w = np.empty_like(v)
    mk.mk_op_interp_combine(p.handle, _opts(sched, "fp64"), 1, precision, v, SIGMA, vt,
                            max(nvt, 1), y, x, w)
    xr = _x_reference(H, v, vt, y)
    assert _rel(x, xr) <= tol
    assert _rel(w, H.levels[0].apply_A(xr)) <= tol


def _abs_rowsum(T):
    return float(np.max(np.abs(T.lo) + np.abs(T.di) + np.abs(T.up)))


@pytest.mark.parametrize("nvt", [0, 1, 2, 3, 4, 5])
def test_interp_combine_double_float_level1(case, nvt):
    sched, H, p = case
    fine = H.levels[0]
    y = WEIGHTS[nvt]
    m = max(nvt, 1)
    v, vt = _inputs(H, nvt, 70 + nvt)
    x = np.empty_like(v)
    w = np.empty_like(v)
    mk.mk_op_interp_combine(p.handle, _opts(sched, "mixed"), 1, 2, v, SIGMA, vt, m, y, x, w)
    # x = fl32(sigma v_hi - fl32(sum_m y_m fl32(vt_m))): v_hi and every vt_m are rounded to
    # FP32 (2^-24 relative each), the combination rounds once per direction and the final
    # fused multiply-add once, so |x - x_exact| <= (m + 3) 2^-24 scale_x <= 2^-21 scale_x
    ysum = 1.0 if y is None else float(np.sum(np.abs(y)))
    scale_x = abs(SIGMA) * float(np.max(np.abs(v))) + ysum * float(np.max(np.abs(vt)))
    xr = _x_reference(H, v, vt, y)
    assert float(np.max(np.abs(x - xr))) <= 2.0 ** -21 * scale_x
    # w = A x from the GPU's own (FP32) x: every w_k is (x_k - x_{k-1}) - a L x_k - b L x_{k-1},
    # whose terms are bounded by scale_w = max|x| (2 + (|a| + |b|) sum of the row sums of |L|).
    # The double-float arithmetic keeps 47-48 bits through about eight roundings (the a, b
    # coefficient pairs, the stencil sums, the products' low parts, the final low-part sums),
    # so |w - A x| <= 8 2^-47 scale_w = 2^-44 scale_w; the test allows 2^-42.  FP32 arithmetic
    # anywhere in w would leave errors of order 2^-24 scale_w.
    lsum = _abs_rowsum(fine.Lx) + (_abs_rowsum(fine.Ly) if fine.dim == 2 else 0.0)
    scale_w = float(np.max(np.abs(x))) * (2.0 + (abs(fine.a) + abs(fine.b)) * lsum)
    err = float(np.max(np.abs(w - fine.apply_A(x))))
    assert err <= 2.0 ** -42 * scale_w, (err / scale_w, 2.0 ** -42)


def test_interp_combine_rejects_bad_arguments(case):
    sched, H, p = case
    v, vt = _inputs(H, 2, 90)
    x = np.empty_like(v)
    w = np.empty_like(v)
    with pytest.raises(Exception):   # two directions without weights
        mk.mk_op_interp_combine(p.handle, _opts(sched, "mixed"), 1, 2, v, SIGMA, vt, 2, None, x, w)
    with pytest.raises(Exception):   # the double-float path needs the mixed hierarchy
        mk.mk_op_interp_combine(p.handle, _opts(sched, "fp64"), 1, 2, v, SIGMA, vt[:1], 1, None,
                                x, w)
