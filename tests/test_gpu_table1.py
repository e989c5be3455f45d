"""Table 1 (Sec. 3.3.1) on the GPU: condition numbers of A_h Q_h for the 1D heat equation,
n_x = 64, theta = 1/2, mu = 1, exact coarse matrix, C = 0.64 (n_t = 16), built from the
library's own operators: column c of A_h Q_h is mk_op_apply(mk_op_precond(e_c)), FP64; the
singular values are taken on the host.  Rows: T- and TS-coarsening with the Galerkin A_H, and
the MGRIT intergrid operators with the coarse matrix of Eq. (coarsemat); nu = 2, 4, 8.
Checked against the oracle's dense A_h Q_h (relative 1e-9) and the printed values (0.015).
"""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

mk = pytest.importorskip("paper_2401_00228_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N_X, C, N_T = 64, 0.64, 16


def _printed(name, key):
    with open(os.path.join(GOLDEN, name)) as fh:
        for l in fh:
            f = l.split()
            if f and not l.startswith("#") and f[:len(key)] == key:
                return [float(v) for v in f[len(key) + 1:len(key) + 4]]
    raise KeyError(key)


def _kappa(M):
    s = np.linalg.svd(M, compute_uv=False)
    return s[0] / s[-1]


def _kappa_gpu(p, o):
    n = (N_T + 1) * N_X
    M = np.empty((n, n))
    e = np.zeros((N_T + 1, N_X))
    x = np.empty_like(e)
    w = np.empty_like(e)
    for c in range(n):
        e.flat[c] = 1.0
        mk.mk_op_precond(p.handle, o, 1, e, x)
        mk.mk_op_apply(p.handle, o, 1, 0, x, w)
        M[:, c] = w.ravel()
        e.flat[c] = 0.0
    return _kappa(M)


def _kappa_oracle(transfer, nu, space):
    h = 1.0 / (N_X + 1)
    dt = C * h * h / 2
    lv = O.build_levels(1, N_X, 1, N_T, 1.0, 0.5, dt, (), (), "one")[0]
    A = O.dense_A(lv)
    if transfer == "mgrit":
        Y, Z = O.dense_transfers_mgrit(lv, nu)
        Q = O.dense_Q(A, Y, Z, 1.0, O.dense_coarse_theta(lv, nu, 0.5))
    else:
        Y, Z = O.dense_transfers(lv, nu, space)
        Q = O.dense_Q(A, Y, Z, 1.0)
    return _kappa(A @ Q)


@pytest.mark.parametrize("row", ["T", "TS", "MGRIT"])
def test_table1_condition_numbers_gpu(row):
    if row == "MGRIT":
        printed = _printed("table1_condition_numbers_mgrit.txt", ["0.64"])
    else:
        printed = _printed("table1_condition_numbers.txt", [row, "0.64"])
    h = 1.0 / (N_X + 1)
    dt = C * h * h / 2
    with mk.Problem(1, N_X, 1.0, 0.5, dt, N_T) as p:
        for nu, ref in zip((2, 4, 8), printed):
            o = mk.make_opts(levels=2, nu=(nu,), space=(row == "TS",), n_cgs=0, mu="one",
                             precision="fp64", transfer="mgrit" if row == "MGRIT" else "mk")
            k_gpu = _kappa_gpu(p, o)
            k_or = _kappa_oracle("mgrit" if row == "MGRIT" else "mk", nu, row == "TS")
            assert abs(k_gpu - k_or) <= 1e-9 * k_or, (row, nu, k_gpu, k_or)
            assert abs(k_gpu - ref) <= 0.015, (row, nu, k_gpu, ref)
