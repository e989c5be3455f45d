"""Host-side setup numerics of the library (csrc/setup.cpp) on the CPU, against the oracle's
dense constructions and closed forms (no GPU).  setup.cpp is compiled on its own with a small
harness (tests/host_setup_harness.cpp) that prints its results.

* agglomerated operators L' = Y^T L Z (Sec. 3.2, Eqs. (constructZ), (constructY)), repeated,
  odd sizes included, against the oracle's dense product;
* lambda_max(-L) by Sturm bisection (the shift mu of Sec. 3.1) against dense eigenvalues;
* the eigen-decomposition used by the 2D coarsest solver: L S = S diag(lam), S S^{-1} = I;
* the uniform-operator test and the sine-transform slab tables against the closed-form
  theta-scheme factor of an eigenmode (Sec. 1 recurrence);
* the padded layout's alignment rules.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2401_00228_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("setup") / "harness")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-I", CUDA_INC, "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "host_setup_harness.cpp"),
                           os.path.join(CSRC, "setup.cpp"), "-o", exe])

    def run(*args):
        out = subprocess.check_output([exe] + [str(a) for a in args], text=True)
        return np.array([float(v) for v in out.split()])
    return run


def _oracle_op(n, tau, k):
    T = O.fd_laplacian(n, tau)
    for _ in range(k):
        T = O.galerkin_space(T)
    return T.dense()


def _dense(m, lo, di, up):
    return np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)


CASES = [(7, 1.0, 1), (8, 0.5, 1), (15, 2.0, 2), (64, 1.0, 3), (63, 1.3, 3), (255, 1.0, 3)]


@pytest.mark.parametrize("n,tau,k", CASES)
def test_agglomerate_is_galerkin_product(harness, n, tau, k):
    r = harness("agg", n, tau, k)
    m = int(r[0])
    lo, di, up = r[1:1 + m], r[1 + m:1 + 2 * m], r[1 + 2 * m:1 + 3 * m]
    ref = _oracle_op(n, tau, k)
    assert ref.shape == (m, m)
    assert np.abs(_dense(m, lo, di, up) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,tau,k", CASES + [(1, 1.0, 0), (2, 1.0, 1), (5, 3.0, 0)])
def test_lambda_max_by_bisection(harness, n, tau, k):
    lam = harness("lmax", n, tau, k)[0]
    ref = np.linalg.eigvals(-_oracle_op(n, tau, k)).real.max()
    assert abs(lam - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("n,tau,k", [(7, 1.0, 1), (15, 2.0, 2), (63, 1.3, 1), (64, 1.0, 2)])
def test_eigen_decomposition(harness, n, tau, k):
    r = harness("eig", n, tau, k)
    m = int(r[0])
    lam = r[1:1 + m]
    S = r[1 + m:1 + m + m * m].reshape(m, m)
    Si = r[1 + m + m * m:].reshape(m, m)
    L = _oracle_op(n, tau, k)
    scale = np.abs(lam).max()
    assert np.abs(L @ S - S * lam[None, :]).max() <= 1e-10 * scale * np.abs(S).max()
    assert np.abs(S @ Si - np.eye(m)).max() <= 1e-10
    assert np.allclose(np.sort(lam), np.sort(np.linalg.eigvals(L).real), rtol=0,
                       atol=1e-10 * scale)


def test_uniform_operator_detection(harness):
    f, c = harness("uni", 63, 1.0, 0)
    assert f == 1 and abs(c - 64.0 ** 2) <= 1e-9
    f, c = harness("uni", 64, 1.0, 1)          # pairs of a uniform stencil: h^2 -> 2 h^2
    assert f == 1 and abs(c - 65.0 ** 2 / 2) <= 1e-9
    f, _ = harness("uni", 63, 1.0, 1)          # odd n: a singleton aggregate at the end
    assert f == 0


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_sine_transform_tables_are_eigenmode_factors(harness, theta):
    n, tau, dt = 31, 1.0, 0.003
    h = 1.0 / (n + 1)
    r = harness("dst", n, tau / h ** 2, theta * dt, (1.0 - theta) * dt)
    alpha, beta = r[:n], r[n:]
    for j in range(n):
        lam = -(4.0 * tau / h ** 2) * math.sin((j + 1) * math.pi * h / 2.0) ** 2
        assert abs(alpha[j] - O.eigenmode_factor(j + 1, n, tau, theta, dt)) <= 1e-14
        assert abs(beta[j] - 1.0 / (1.0 - theta * dt * lam)) <= 1e-14


@pytest.mark.parametrize("dim,nx,ny,nt", [(1, 1, 1, 1), (1, 1023, 1, 8192), (2, 255, 255, 1024),
                                          (2, 15, 13, 32), (1, 7, 1, 0)])
def test_padded_layout(harness, dim, nx, ny, nt):
    ldx, plane, guard, length = harness("geom", dim, nx, ny, nt).astype(np.int64)
    assert ldx % 8 == 0 and ldx >= nx + 1 and ldx < nx + 9
    assert plane == (ldx if dim == 1 else (ny + 1) * ldx)
    assert guard == ldx
    assert length % 4096 == 0 and length >= guard + (nt + 1) * plane + ldx
