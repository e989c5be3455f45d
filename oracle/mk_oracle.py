"""CPU oracle (FP64) for the parallel-in-time multilevel Krylov (MK) method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path and never calls it.

What it computes, in the paper's notation (Erlangga, "Parallel-in-time
Multilevel Krylov Methods: A Prototype"):

* Sec. 1, Eq. (thetascheme): psi_n u_k = phi_n u_{k-1} + dt gbar_k with
  psi = I - theta dt A_n, phi = I + (1-theta) dt A_n, gbar_k = (1-theta) g_{k-1}
  + theta g_k.  A_n = tau * (second-order FD Laplacian), zero Dirichlet (Sec. 3.3).
* Sec. 2, Eq. (finesys): the all-at-once system A_h u_h = f_h, block lower
  bidiagonal with I, psi on the diagonal and -phi below; f_0 = u_0,
  f_k = dt gbar_k.  Its unique solution is the sequential theta-march
  (``march.c``), the plain definition every MK solve must reproduce.
* Sec. 3.1, Eq. (Qh): Q_h = I - Z A_H^{-1} Y^T A_h + mu Z A_H^{-1} Y^T with
  A_H = Y^T A_h Z, applied through substeps 4.1-4.5 of Algorithm 2.
* Sec. 3.2, Eqs. (blockYZ), (tcoarseZ), (TS-coarsening), (constructZ),
  (constructY): block-diagonal transfers; T-coarsening sums nu consecutive
  steps (Y_k = Z_k = [I..I]^T); TS-coarsening additionally agglomerates space
  (Z 0/1 indicator, Y 1/|I_j| average).
* Sec. 3.2, Eqs. (timecoarse1)-(timecoarse3): the Galerkin coarse system is a
  theta-scheme with a larger step.  Reading (the printed formula swaps theta and
  1-theta; the literal product nu*psi - (nu-1)*phi is used):
  a' = nu a + (nu-1) b, b' = b, L' = Y^T L Z.
* Sec. 3.3.2, Eq. (Qhtilde): the perturbed, decoupled coarsest matrix; the
  coupling into the first step of each of the N_CGS slabs is dropped.
* Sec. 4.1: recursion; intermediate levels run a fixed number of FGMRES
  iterations (zero initial guess) preconditioned by the next level.
* Algorithm 2: FGMRES (Arnoldi with modified Gram-Schmidt, least squares on
  the Hessenberg matrix, u = u0 + X_J y_J).
* Sec. 3.2, Eqs. (mgritY), (mgritZ), with Eq. (coarsemat): the comparison
  two-level method with MGRIT intergrid operators.  Y^T injects the coarse
  time points (steps 0, nu, 2 nu, ...), Z is the ideal interpolation
  [-(A_ff)^{-1} A_fc; I_c], and A_H is not the Galerkin product but the
  theta-scheme with the same theta and the larger step Delta T = nu dt
  (Psi_n, Phi_n of Eq. (timemarchdT)).  Two-level only, time coarsening only.

Functions that have a plain definition (the march, the operators, the dense
builders) are written as that definition.  The MK cycle and FGMRES follow the
steps of Sec. 3.1 and Algorithm 2 in order.  ``numpy.linalg.lstsq``,
``scipy.linalg`` solvers and dense products serve as library steps.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg as sla

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    """Load the plain-C march (built by ``oracle/build.py``)."""
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "liboracle_march.so")
        if not os.path.exists(path):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_march_1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        dp, dp, dp, dp, dp]
        lib.oracle_march_1d.restype = ctypes.c_int
        lib.oracle_march_2d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.oracle_march_2d.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# -----------------------------------------------------------------------------
# Spatial operators (Sec. 3.3): one tridiagonal operator per direction.
# -----------------------------------------------------------------------------

@dataclasses.dataclass
class Tridiag:
    """(L v)_i = lo[i] v_{i-1} + di[i] v_i + up[i] v_{i+1}, v_{-1} = v_n = 0."""
    lo: np.ndarray
    di: np.ndarray
    up: np.ndarray

    @property
    def n(self) -> int:
        return self.di.shape[0]

    def dense(self) -> np.ndarray:
        n = self.n
        M = np.diag(self.di.copy())
        for i in range(1, n):
            M[i, i - 1] = self.lo[i]
            M[i - 1, i] = self.up[i - 1]
        return M

    def apply(self, v: np.ndarray, axis: int = -1) -> np.ndarray:
        """Apply along ``axis`` of v (broadcast over the other axes)."""
        v = np.moveaxis(v, axis, -1)
        out = self.di * v
        out[..., 1:] += self.lo[1:] * v[..., :-1]
        out[..., :-1] += self.up[:-1] * v[..., 1:]
        return np.moveaxis(out, -1, axis)


def fd_laplacian(n: int, tau: float) -> Tridiag:
    """tau * second-order FD d^2/dx^2 on n interior points, h = 1/(n+1), Sec. 3.3."""
    h = 1.0 / (n + 1)
    c = tau / (h * h)
    lo = np.full(n, c)
    up = np.full(n, c)
    lo[0] = 0.0
    up[-1] = 0.0
    return Tridiag(lo, np.full(n, -2.0 * c), up)


def aggregates(n: int) -> List[List[int]]:
    """Agglomeration sets I_j (Sec. 3.2, Case 2).  Reading for the missing figure:
    pairs {2j, 2j+1}; for odd n the last set is the singleton {n-1}."""
    return [list(range(2 * j, min(2 * j + 2, n))) for j in range((n + 1) // 2)]


def agglomeration_Z(n: int) -> np.ndarray:
    """Eq. (constructZ): z_ij = 1 if i in I_j else 0 (n x m)."""
    sets = aggregates(n)
    Z = np.zeros((n, len(sets)))
    for j, s in enumerate(sets):
        Z[s, j] = 1.0
    return Z


def agglomeration_Y(n: int) -> np.ndarray:
    """Eq. (constructY): y_ji = 1/|I_j| if i in I_j (returned as the n x m matrix Y)."""
    sets = aggregates(n)
    Y = np.zeros((n, len(sets)))
    for j, s in enumerate(sets):
        Y[s, j] = 1.0 / len(s)
    return Y


def galerkin_space(L: Tridiag) -> Tridiag:
    """L' = Y^T L Z (dense product, then read back as a tridiagonal operator)."""
    n = L.n
    Y = agglomeration_Y(n)
    Z = agglomeration_Z(n)
    C = Y.T @ L.dense() @ Z
    m = C.shape[0]
    band = np.zeros_like(C)
    di = np.diag(C).copy()
    lo = np.zeros(m)
    up = np.zeros(m)
    for j in range(1, m):
        lo[j] = C[j, j - 1]
        up[j - 1] = C[j - 1, j]
    band += np.diag(di)
    band += np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    if not np.allclose(band, C, rtol=0, atol=1e-12 * np.abs(C).max()):
        raise AssertionError("agglomerated operator is not tridiagonal")
    return Tridiag(lo, di, up)


# -----------------------------------------------------------------------------
# Levels of the hierarchy.
# -----------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    """One level: (A x)_0 = x_0, (A x)_k = (I - aL) x_k - (I + bL) x_{k-1}."""
    dim: int
    nt: int
    a: float
    b: float
    Lx: Tridiag
    Ly: Optional[Tridiag]
    mu: float = 1.0

    @property
    def nx(self) -> int:
        return self.Lx.n

    @property
    def ny(self) -> int:
        return 1 if self.Ly is None else self.Ly.n

    def space_shape(self) -> Tuple[int, ...]:
        return (self.nx,) if self.dim == 1 else (self.ny, self.nx)

    def shape(self) -> Tuple[int, ...]:
        return (self.nt + 1,) + self.space_shape()

    def apply_L(self, v: np.ndarray) -> np.ndarray:
        """Spatial operator on every row of v (leading axes are broadcast)."""
        if self.dim == 1:
            return self.Lx.apply(v, axis=-1)
        return self.Lx.apply(v, axis=-1) + self.Ly.apply(v, axis=-2)

    def apply_A(self, x: np.ndarray) -> np.ndarray:
        """Block lower-bidiagonal matvec, Eq. (finesys) at this level."""
        w = np.empty_like(x)
        w[0] = x[0]
        Lx = self.apply_L(x)
        w[1:] = (x[1:] - self.a * Lx[1:]) - (x[:-1] + self.b * Lx[:-1])
        return w

    def spatial_dense(self) -> np.ndarray:
        if self.dim == 1:
            return self.Lx.dense()
        return np.kron(np.eye(self.ny), self.Lx.dense()) + np.kron(self.Ly.dense(), np.eye(self.nx))

    def lambda_max(self) -> float:
        """lambda_max(A_l) = max(1, 1 + a * max(-eig(L))) since A_l is block triangular."""
        ex = np.linalg.eigvals(self.Lx.dense()).real
        lam = -ex.min()
        if self.dim == 2:
            ey = np.linalg.eigvals(self.Ly.dense()).real
            lam += -ey.min()
        return max(1.0, 1.0 + self.a * lam)


def build_levels(dim: int, nx: int, ny: int, nt: int, tau: float, theta: float, dt: float,
                 nu: Sequence[int], space: Sequence[bool], mu_mode: str = "lambda_max",
                 mu_value: Optional[float] = None) -> List[Level]:
    """Fine level from Sec. 1 (a = theta dt, b = (1-theta) dt) and each coarser level from
    the Galerkin product of Sec. 3.2: a' = nu a + (nu-1) b, b' = b, n_t' = n_t/nu,
    L' = Y^T L Z when space is agglomerated, else L' = L."""
    Lx = fd_laplacian(nx, tau)
    Ly = fd_laplacian(ny, tau) if dim == 2 else None
    levels = [Level(dim, nt, theta * dt, (1.0 - theta) * dt, Lx, Ly)]
    for f, s in zip(nu, space):
        prev = levels[-1]
        if prev.nt % f:
            raise ValueError("n_t not divisible by the coarsening factor")
        nLx = galerkin_space(prev.Lx) if s else prev.Lx
        nLy = (galerkin_space(prev.Ly) if s else prev.Ly) if dim == 2 else None
        levels.append(Level(dim, prev.nt // f, f * prev.a + (f - 1) * prev.b, prev.b, nLx, nLy))
    for lv in levels:
        if mu_mode == "lambda_max":
            lv.mu = lv.lambda_max()
        elif mu_mode == "one":
            lv.mu = 1.0
        elif mu_mode == "value":
            lv.mu = float(mu_value)
        else:
            raise ValueError(mu_mode)
    return levels


# -----------------------------------------------------------------------------
# Right-hand side and the sequential march (the plain definition of the solution).
# -----------------------------------------------------------------------------

def assemble_rhs(u0: np.ndarray, g: Optional[np.ndarray], nt: int, theta: float, dt: float) -> np.ndarray:
    """f_0 = u_0, f_k = dt ((1-theta) g_{k-1} + theta g_k), Eq. (finesys)."""
    f = np.zeros((nt + 1,) + u0.shape)
    f[0] = u0
    if g is not None:
        f[1:] = dt * ((1.0 - theta) * g[:-1] + theta * g[1:])
    return f


def march(level: Level, f: np.ndarray) -> np.ndarray:
    """Block forward substitution of A_l u = f (plain C, FP64)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.empty_like(f)
    lib = _lib()
    if level.dim == 1:
        L = level.Lx
        rc = lib.oracle_march_1d(level.nx, level.nt, level.a, level.b,
                                 _ptr(np.ascontiguousarray(L.lo)), _ptr(np.ascontiguousarray(L.di)),
                                 _ptr(np.ascontiguousarray(L.up)), _ptr(f), _ptr(u))
    else:
        X, Yd = level.Lx, level.Ly
        rc = lib.oracle_march_2d(level.nx, level.ny, level.nt, level.a, level.b,
                                 _ptr(X.lo), _ptr(X.di), _ptr(X.up),
                                 _ptr(Yd.lo), _ptr(Yd.di), _ptr(Yd.up), _ptr(f), _ptr(u))
    if rc != 0:
        raise RuntimeError(f"oracle march failed ({rc})")
    return u


def theta_march(dim: int, nx: int, ny: int, nt: int, tau: float, theta: float, dt: float,
                u0: np.ndarray, g: Optional[np.ndarray]) -> np.ndarray:
    """Sequential theta-scheme, Eq. (timemarch): the unique solution of Eq. (finesys)."""
    lv = build_levels(dim, nx, ny, nt, tau, theta, dt, (), (), mu_mode="one")[0]
    return march(lv, assemble_rhs(u0, g, nt, theta, dt))


# -----------------------------------------------------------------------------
# Intergrid transfers (Sec. 3.2).
# -----------------------------------------------------------------------------

def _space_restrict(v: np.ndarray, dim: int) -> np.ndarray:
    """Y^T on the trailing space axes (average over each aggregate)."""
    def one_axis(a, axis):
        n = a.shape[axis]
        return np.moveaxis(np.moveaxis(a, axis, -1) @ agglomeration_Y(n), -1, axis)
    out = one_axis(v, -1)
    if dim == 2:
        out = one_axis(out, -2)
    return out


def _space_interp(v: np.ndarray, dim: int, nx: int, ny: int) -> np.ndarray:
    """Z on the trailing space axes (copy each aggregate value to its members)."""
    def one_axis(a, axis, n):
        return np.moveaxis(np.moveaxis(a, axis, -1) @ agglomeration_Z(n).T, -1, axis)
    out = one_axis(v, -1, nx)
    if dim == 2:
        out = one_axis(out, -2, ny)
    return out


def restrict(fine: Level, nu: int, space: bool, v: np.ndarray) -> np.ndarray:
    """Y^T v with Y = blockdiag(Y_k): block 0 -> Y_0^T v_0; block K -> sum over its nu steps."""
    nT = fine.nt // nu
    out = np.empty((nT + 1,) + v.shape[1:])
    out[0] = v[0]
    out[1:] = v[1:].reshape((nT, nu) + v.shape[1:]).sum(axis=1)
    if space:
        out = _space_restrict(out, fine.dim)
    return out


def interpolate(fine: Level, nu: int, space: bool, vt: np.ndarray) -> np.ndarray:
    """Z vt with Z = blockdiag(Z_k): step 0 <- block 0, step k >= 1 <- block ceil(k/nu)."""
    if space:
        vt = _space_interp(vt, fine.dim, fine.nx, fine.ny)
    out = np.empty((fine.nt + 1,) + vt.shape[1:])
    out[0] = vt[0]
    out[1:] = np.repeat(vt[1:], nu, axis=0)
    return out


def restrict_inject(fine: Level, nu: int, v: np.ndarray) -> np.ndarray:
    """Y^T v for Y of Eq. (mgritY): the coarse time points, steps 0, nu, 2 nu, ..., n_t."""
    return v[::nu].copy()


def interpolate_ideal(fine: Level, nu: int, vt: np.ndarray) -> np.ndarray:
    """Z vt for the ideal interpolation of Eq. (mgritZ), Z = [-(A_ff)^{-1} A_fc; I_c].
    Coarse points take vt: x_{nu K} = vt_K.  The fine points nu K + 1 .. nu K + nu - 1 of
    interval K solve A_ff y = -A_fc vt: A_ff is lower block bidiagonal (psi on the
    diagonal, -phi below) and A_fc couples the first of them to x_{nu K} by -phi, so
    psi x_{nu K + i} = phi x_{nu K + i - 1}, i = 1 .. nu - 1 (the homogeneous march)."""
    out = np.empty((fine.nt + 1,) + vt.shape[1:])
    out[::nu] = vt
    ns = fine.space_shape()
    if nu > 1:
        psi = np.eye(int(np.prod(ns))) - fine.a * fine.spatial_dense()
        lu = sla.lu_factor(psi)
        for K in range(fine.nt // nu):
            for i in range(1, nu):
                k = nu * K + i
                prev = out[k - 1]
                rhs = prev + fine.b * fine.apply_L(prev)
                out[k] = sla.lu_solve(lu, rhs.reshape(-1)).reshape(ns)
    return out


def coarse_theta_level(fine: Level, nu: int, theta: float, mu_mode: str = "lambda_max",
                       mu_value: Optional[float] = None) -> Level:
    """The coarse time-grid matrix of Eq. (coarsemat): the theta-scheme with the same theta
    and step Delta T = nu dt, Psi_n = I - theta Delta T A_n, Phi_n = I + (1-theta) Delta T A_n
    (Eq. (timemarchdT)); not the Galerkin product Y^T A_h Z."""
    if fine.nt % nu:
        raise ValueError("n_t not divisible by the coarsening factor")
    dt = fine.a + fine.b            # a = theta dt, b = (1 - theta) dt on the fine level
    DT = nu * dt
    lv = Level(fine.dim, fine.nt // nu, theta * DT, (1.0 - theta) * DT, fine.Lx, fine.Ly)
    if mu_mode == "lambda_max":
        lv.mu = lv.lambda_max()
    elif mu_mode == "one":
        lv.mu = 1.0
    elif mu_mode == "value":
        lv.mu = float(mu_value)
    else:
        raise ValueError(mu_mode)
    return lv


# -----------------------------------------------------------------------------
# Coarsest level: perturbed, decoupled matrix (Sec. 3.3.2, Eq. (Qhtilde)).
# -----------------------------------------------------------------------------

def coarsest_solve(level: Level, r: np.ndarray, n_cgs: int) -> np.ndarray:
    """x = Atilde^{-1} r: block 0 alone (x_0 = r_0); the n_t steps split into n_cgs
    contiguous slabs whose first step has its coupling to the previous step dropped.
    n_cgs = 0 selects the exact, coupled coarse matrix A_H instead."""
    nt = level.nt
    if n_cgs == 0:          # exact (coupled) coarse solve, A_H^{-1} of Eq. (Qh)
        return march(level, r)
    if nt % n_cgs:
        raise ValueError("coarsest n_t not divisible by N_CGS")
    s = nt // n_cgs
    M = np.eye(int(np.prod(level.space_shape()))) - level.a * level.spatial_dense()
    lu = sla.lu_factor(M)
    x = np.empty_like(r)
    x[0] = r[0]
    for k in range(1, nt + 1):
        rhs = r[k].copy()
        if (k - 1) % s != 0:  # not the first step of its slab
            rhs = rhs + x[k - 1] + level.b * level.apply_L(x[k - 1])
        x[k] = sla.lu_solve(lu, rhs.reshape(-1)).reshape(level.space_shape())
    return x


# -----------------------------------------------------------------------------
# MK cycle and FGMRES (Sec. 3.1 substeps 4.1-4.5, Algorithm 2, Sec. 4.1).
# -----------------------------------------------------------------------------

@dataclasses.dataclass
class Hierarchy:
    levels: List[Level]
    nu: Tuple[int, ...]
    space: Tuple[bool, ...]
    m_inner: Tuple[int, ...]   # fixed FGMRES iterations on levels 2..L-1
    n_cgs: int
    transfer: str = "mk"       # "mk" (Sec. 3.2 block sums) or "mgrit" (Eqs. (mgritY), (mgritZ))


def make_hierarchy(dim, nx, ny, nt, tau, theta, dt, nu, space, m_inner, n_cgs,
                   mu_mode="lambda_max", mu_value=None, transfer="mk") -> Hierarchy:
    if transfer == "mgrit":
        if len(nu) != 1 or any(space):
            raise ValueError("the MGRIT comparison is two-level with time coarsening only")
        lv = build_levels(dim, nx, ny, nt, tau, theta, dt, (), (), mu_mode, mu_value)
        lv.append(coarse_theta_level(lv[0], nu[0], theta, mu_mode, mu_value))
    elif transfer == "mk":
        lv = build_levels(dim, nx, ny, nt, tau, theta, dt, nu, space, mu_mode, mu_value)
    else:
        raise ValueError(transfer)
    if len(m_inner) != max(0, len(lv) - 2):
        raise ValueError("m_inner must give one count per intermediate level")
    return Hierarchy(lv, tuple(nu), tuple(space), tuple(m_inner), n_cgs, transfer)


def coarse_solve(H: Hierarchy, l: int, vhat: np.ndarray) -> np.ndarray:
    """Step 4.3 on level l+1 (0-based l): exact decoupled solve on the coarsest level,
    else a fixed number of FGMRES iterations with zero initial guess (Sec. 4.1)."""
    if l + 1 == len(H.levels) - 1:
        return coarsest_solve(H.levels[l + 1], vhat, H.n_cgs)
    return fgmres_fixed(H, l + 1, vhat, H.m_inner[l])


def precondition(H: Hierarchy, l: int, v: np.ndarray) -> np.ndarray:
    """x = Q_l v by substeps 4.1-4.5."""
    lv = H.levels[l]
    s = lv.apply_A(v)                                    # 4.1
    if H.transfer == "mgrit":
        vhat = restrict_inject(lv, H.nu[l], s - lv.mu * v)   # 4.2, Y of Eq. (mgritY)
    else:
        vhat = restrict(lv, H.nu[l], H.space[l], s - lv.mu * v)   # 4.2
    vtil = coarse_solve(H, l, vhat)                      # 4.3
    if H.transfer == "mgrit":
        t = interpolate_ideal(lv, H.nu[l], vtil)         # 4.4, Z of Eq. (mgritZ)
    else:
        t = interpolate(lv, H.nu[l], H.space[l], vtil)   # 4.4
    return v - t                                         # 4.5


def _arnoldi_step(lv: Level, V: List[np.ndarray], w: np.ndarray, Hm: np.ndarray, j: int):
    """Modified Gram-Schmidt against v^1..v^j (Algorithm 2 with h_{l,j} = (w, v^l))."""
    for i in range(j + 1):
        Hm[i, j] = np.vdot(w.ravel(), V[i].ravel())
        w = w - Hm[i, j] * V[i]
    Hm[j + 1, j] = np.linalg.norm(w.ravel())
    return w


def fgmres_fixed(H: Hierarchy, l: int, b: np.ndarray, m: int) -> np.ndarray:
    """Algorithm 2 on level l with u^0 = 0 and exactly m iterations (no tolerance);
    stops early only on an exact (happy) breakdown."""
    lv = H.levels[l]
    beta = np.linalg.norm(b.ravel())
    if beta == 0.0:
        return np.zeros_like(b)
    V = [b / beta]
    X = []
    Hm = np.zeros((m + 1, m))
    J = m
    for j in range(m):
        x = precondition(H, l, V[j])
        X.append(x)
        w = _arnoldi_step(lv, V, lv.apply_A(x), Hm, j)
        if Hm[j + 1, j] == 0.0:
            J = j + 1
            break
        V.append(w / Hm[j + 1, j])
    rhs = np.zeros(J + 1)
    rhs[0] = beta
    y = np.linalg.lstsq(Hm[:J + 1, :J], rhs, rcond=None)[0]
    u = np.zeros_like(b)
    for i in range(J):
        u = u + y[i] * X[i]
    return u


@dataclasses.dataclass
class SolveInfo:
    iterations: int
    restarts: int
    rel_residual: float
    history: List[float]


def fgmres_cycle(H: Hierarchy, f: np.ndarray, u: np.ndarray, restart: int, extra=(),
                 tol: float = 0.0, fnorm: float = 1.0, budget: int = 1 << 30):
    """One restart cycle of the outer FGMRES from u (Algorithm 2 with u^0 = u): Arnoldi on
    r = f - A u with the directions x_j = Q_1 v_j (substeps 4.1-4.5), except that the last
    len(extra) of the `restart` slots take the given directions instead (a flexible method
    accepts any direction: the relation A X = V H stays exact).  Stops early when the
    least-squares residual estimate drops below tol * fnorm, on a happy breakdown, or after
    `budget` directions.  Returns (u + X y, X y, directions used)."""
    lv = H.levels[0]
    r = f - lv.apply_A(u)
    beta = np.linalg.norm(r.ravel())
    V = [r / beta]
    X = []
    Hm = np.zeros((restart + 1, restart))
    J = 0
    first_extra = restart - len(extra)
    y = np.zeros(0)
    for j in range(restart):
        x = extra[j - first_extra] if j >= first_extra else precondition(H, 0, V[j])
        X.append(x)
        w = _arnoldi_step(lv, V, lv.apply_A(x), Hm, j)
        J = j + 1
        e1 = np.zeros(J + 1)
        e1[0] = beta
        y = np.linalg.lstsq(Hm[:J + 1, :J], e1, rcond=None)[0]
        est = np.linalg.norm(e1 - Hm[:J + 1, :J] @ y)
        if Hm[j + 1, j] == 0.0 or est / fnorm < tol or J >= budget:
            break
        V.append(w / Hm[j + 1, j])
    d = np.zeros_like(u)
    for i in range(J):
        d = d + y[i] * X[i]
    return u + d, d, J


def fgmres(H: Hierarchy, f: np.ndarray, tol: float, restart: int = 50, maxit: int = 1000,
           u0: Optional[np.ndarray] = None, augment: int = 0) -> Tuple[np.ndarray, SolveInfo]:
    """Outer FGMRES(restart) on level 1 preconditioned by Q_1.  Convergence when
    ||f - A u|| / ||f|| < tol (Sec. 3.3.1), checked with the true residual.

    augment = k > 0: FGMRES with recycled corrections (the flexible form of augmented
    restarting, a recycling restart for the stiff regime of Sec. 3.1): the correction
    d_c = u_c - u_{c-1} of every completed cycle c is kept in ring slot (c - 1) mod k, and once
    k cycles have completed, the last k of each cycle's `restart` directions are those k
    corrections (slot order) instead of preconditioned basis vectors, so every cycle
    minimises the residual over its preconditioned Krylov directions plus the recent
    corrections."""
    lv = H.levels[0]
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fnorm = np.linalg.norm(f.ravel())
    hist = []
    total = 0
    restarts = 0
    ring = [None] * max(augment, 0)
    while True:
        r = f - lv.apply_A(u)
        beta = np.linalg.norm(r.ravel())
        hist.append(beta / fnorm)
        if beta / fnorm < tol or total >= maxit:
            return u, SolveInfo(total, restarts, beta / fnorm, hist)
        extra = tuple(ring) if augment > 0 and restarts >= augment else ()
        u, d, J = fgmres_cycle(H, f, u, restart, extra, tol, fnorm, maxit - total)
        total += J
        if augment > 0:
            ring[restarts % augment] = d
        restarts += 1


# -----------------------------------------------------------------------------
# Dense builders for small pins (Sec. 3.1-3.3).
# -----------------------------------------------------------------------------

def dense_A(level: Level) -> np.ndarray:
    """A_l as a dense (n_t+1) n x (n_t+1) n matrix."""
    n = int(np.prod(level.space_shape()))
    Ls = level.spatial_dense()
    I = np.eye(n)
    N = (level.nt + 1) * n
    A = np.zeros((N, N))
    A[:n, :n] = I
    psi = I - level.a * Ls
    phi = I + level.b * Ls
    for k in range(1, level.nt + 1):
        A[k * n:(k + 1) * n, k * n:(k + 1) * n] = psi
        A[k * n:(k + 1) * n, (k - 1) * n:k * n] = -phi
    return A


def dense_transfers(fine: Level, nu: int, space: bool) -> Tuple[np.ndarray, np.ndarray]:
    """Dense Y, Z of Eq. (blockYZ): Y_0 = Y, Z_0 = Z; Y_k, Z_k = nu stacked copies."""
    n = int(np.prod(fine.space_shape()))
    if space:
        if fine.dim == 1:
            Zs, Ys = agglomeration_Z(fine.nx), agglomeration_Y(fine.nx)
        else:
            Zs = np.kron(agglomeration_Z(fine.ny), agglomeration_Z(fine.nx))
            Ys = np.kron(agglomeration_Y(fine.ny), agglomeration_Y(fine.nx))
    else:
        Zs = Ys = np.eye(n)
    m = Zs.shape[1]
    nT = fine.nt // nu
    Z = np.zeros(((fine.nt + 1) * n, (nT + 1) * m))
    Y = np.zeros_like(Z)
    Z[:n, :m] = Zs
    Y[:n, :m] = Ys
    for K in range(1, nT + 1):
        for i in range(1, nu + 1):
            k = nu * (K - 1) + i
            Z[k * n:(k + 1) * n, K * m:(K + 1) * m] = Zs
            Y[k * n:(k + 1) * n, K * m:(K + 1) * m] = Ys
    return Y, Z


def dense_transfers_mgrit(fine: Level, nu: int) -> Tuple[np.ndarray, np.ndarray]:
    """Dense Y, Z of Eqs. (mgritY), (mgritZ) from the C/F partition of A_h: the coarse
    (C) points are the blocks of steps 0, nu, 2 nu, ...; Y = [0; I_c] and
    Z = [-(A_ff)^{-1} A_fc; I_c], both scattered back to the natural ordering."""
    n = int(np.prod(fine.space_shape()))
    A = dense_A(fine)
    N = A.shape[0]
    cblocks = list(range(0, fine.nt + 1, nu))
    c = np.concatenate([np.arange(k * n, (k + 1) * n) for k in cblocks])
    f = np.setdiff1d(np.arange(N), c)
    Y = np.zeros((N, c.size))
    Y[c, np.arange(c.size)] = 1.0
    Z = Y.copy()
    if f.size:
        Z[f, :] = -np.linalg.solve(A[np.ix_(f, f)], A[np.ix_(f, c)])
    return Y, Z


def dense_coarse_theta(fine: Level, nu: int, theta: float) -> np.ndarray:
    """A_H of Eq. (coarsemat) as a dense matrix: I, then Psi_n on the diagonal and -Phi_n
    below, Psi_n = I - theta nu dt A_n, Phi_n = I + (1-theta) nu dt A_n."""
    n = int(np.prod(fine.space_shape()))
    An = fine.spatial_dense()
    DT = nu * (fine.a + fine.b)
    I = np.eye(n)
    nT = fine.nt // nu
    AH = np.zeros(((nT + 1) * n, (nT + 1) * n))
    AH[:n, :n] = I
    for K in range(1, nT + 1):
        AH[K * n:(K + 1) * n, K * n:(K + 1) * n] = I - theta * DT * An
        AH[K * n:(K + 1) * n, (K - 1) * n:K * n] = -(I + (1.0 - theta) * DT * An)
    return AH


def dense_decoupled(level: Level, n_cgs: int) -> np.ndarray:
    """Atilde: dense A_l with the coupling into the first step of each slab removed."""
    A = dense_A(level)
    n = int(np.prod(level.space_shape()))
    s = level.nt // n_cgs
    for k in range(1, level.nt + 1):
        if (k - 1) % s == 0:
            A[k * n:(k + 1) * n, (k - 1) * n:k * n] = 0.0
    return A


def dense_Q(A: np.ndarray, Y: np.ndarray, Z: np.ndarray, mu: float,
            AH: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. (Qh) (or Eq. (Qhtilde) when a perturbed A_H is given)."""
    if AH is None:
        AH = Y.T @ A @ Z
    AHinv_Yt = np.linalg.solve(AH, Y.T)
    return np.eye(A.shape[0]) - Z @ AHinv_Yt @ A + mu * Z @ AHinv_Yt


# -----------------------------------------------------------------------------
# Adjoint (transposed system) for the terminal misfit.
# -----------------------------------------------------------------------------

def adjoint_march(level: Level, bvec: np.ndarray) -> np.ndarray:
    """Solve A^T lam = b by a backward march: psi^T lam_nt = b_nt,
    psi^T lam_k = b_k + phi^T lam_{k+1}, lam_0 = b_0 + phi^T lam_1.
    Implemented as the forward march of the time-reversed system with L^T."""
    def transpose(T: Tridiag) -> Tridiag:
        n = T.n
        lo = np.zeros(n)
        up = np.zeros(n)
        lo[1:] = T.up[:-1]
        up[:-1] = T.lo[1:]
        return Tridiag(lo, T.di.copy(), up)
    lt = Level(level.dim, level.nt, level.a, level.b, transpose(level.Lx),
               transpose(level.Ly) if level.Ly is not None else None)
    rev = np.empty_like(bvec)
    rev[0] = 0.0
    rev[1:] = bvec[:0:-1]           # rev[j] = b[nt+1-j]
    y = march(lt, rev)
    lam = np.empty_like(bvec)
    lam[1:] = y[:0:-1]              # lam[k] = y[nt+1-k]
    lam[0] = bvec[0] + lam[1] + level.b * lt.apply_L(lam[1])
    return lam


def misfit_gradients(dim, nx, ny, nt, tau, theta, dt, u0, g, u_target):
    """Loss J = ||u_nt - u_target||^2.  Returns (J, dJ/du0, dJ/dg, dJ/dtau) from the
    discrete adjoint of Eq. (finesys):
      lam = A^{-T} dJ/du,  dJ/du0 = lam_0,
      dJ/dg_k = dt (theta lam_k + (1-theta) lam_{k+1})  (lam_{nt+1} = 0, no lam_0 term),
      dJ/dtau = sum_{k>=1} dt lam_k^T Lhat (theta u_k + (1-theta) u_{k-1}),  Lhat = L/tau."""
    lv = build_levels(dim, nx, ny, nt, tau, theta, dt, (), (), mu_mode="one")[0]
    u = march(lv, assemble_rhs(u0, g, nt, theta, dt))
    diff = u[-1] - u_target
    J = float(np.sum(diff * diff))
    b = np.zeros_like(u)
    b[-1] = 2.0 * diff
    lam = adjoint_march(lv, b)
    gu0 = lam[0].copy()
    gg = np.zeros_like(u)
    gg[1:] += dt * theta * lam[1:]
    gg[:-1] += dt * (1.0 - theta) * lam[1:]
    Lu = lv.apply_L(theta * u[1:] + (1.0 - theta) * u[:-1]) / tau
    gtau = float(dt * np.sum(lam[1:] * Lu))
    return J, gu0, gg, gtau, u


def misfit_value(dim, nx, ny, nt, tau, theta, dt, u0, g, u_target) -> float:
    u = theta_march(dim, nx, ny, nt, tau, theta, dt, u0, g)
    d = u[-1] - u_target
    return float(np.sum(d * d))


# -----------------------------------------------------------------------------
# Closed form (Sec. 1 recurrence on an eigenmode).
# -----------------------------------------------------------------------------

def eigenmode_factor(k: int, n: int, tau: float, theta: float, dt: float) -> float:
    """Per-step amplification of sin(k pi x) under the theta-scheme:
    r_k = (1 + (1-theta) dt lam_k) / (1 - theta dt lam_k), lam_k = -(4 tau/h^2) sin^2(k pi h/2)."""
    h = 1.0 / (n + 1)
    lam = -(4.0 * tau / (h * h)) * math.sin(k * math.pi * h / 2.0) ** 2
    return (1.0 + (1.0 - theta) * dt * lam) / (1.0 - theta * dt * lam)


def max_rel_error(u: np.ndarray, ref: np.ndarray) -> float:
    """||u - u_ref||_inf / ||u_ref||_inf over the whole space-time array."""
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))
