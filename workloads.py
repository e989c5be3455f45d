"""Seeded synthetic heat-equation workloads.

This module only draws inputs (initial states, sources, targets, problem
parameters).  It contains none of the solver's arithmetic, so both the CPU
oracle and the CUDA path can take their inputs from here without sharing any
numerical code.

The problems follow the model of Sec. 3.3 of the paper: the heat equation
u_t = tau * Laplace(u) on the unit interval / unit square, zero Dirichlet
boundaries, second-order finite differences on n interior points per direction
(h = 1/(n+1)), theta-scheme in time with dt = T/n_t.

Every array is float64 and C-contiguous.  Space-time arrays are time-major:
shape (n_t+1, n) in 1D and (n_t+1, ny, nx) in 2D (x fastest).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Schedule:
    """Multilevel schedule: how each level is coarsened into the next one.

    nu[l]      : time-coarsening factor from level l+1 to level l+2 (1-based levels)
    space[l]   : True if the spatial grid is agglomerated (pairs / 2x2) on that coarsening
    m_inner[l] : fixed FGMRES iterations on the intermediate level l+2 (len = levels-2)
    n_cgs      : number of decoupled slabs on the coarsest level
    """
    nu: Tuple[int, ...]
    space: Tuple[bool, ...]
    m_inner: Tuple[int, ...]
    n_cgs: int

    @property
    def levels(self) -> int:
        return len(self.nu) + 1


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    nx: int
    ny: int          # 1 in 1D
    nt: int
    T: float
    tau: float
    theta: float
    u0: np.ndarray   # (n,) or (ny, nx)
    g: Optional[np.ndarray]  # (nt+1, n) / (nt+1, ny, nx) or None (g = 0)
    schedule: Schedule
    tol: float = 1e-12
    precision: str = "fp64"   # "fp64" or "mixed"
    u_target: Optional[np.ndarray] = None

    @property
    def dt(self) -> float:
        return self.T / self.nt

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def h(self) -> float:
        return 1.0 / (self.nx + 1)

    @property
    def courant(self) -> float:
        """C = 2 tau dt / h^2 (the paper's 1D definition)."""
        return 2.0 * self.tau * self.dt / self.h ** 2

    def space_shape(self) -> Tuple[int, ...]:
        return (self.nx,) if self.dim == 1 else (self.ny, self.nx)


def _grid(n: int) -> np.ndarray:
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def smooth_modes_1d(rng: np.random.Generator, n: int, kmax: int = 8) -> np.ndarray:
    """sin(pi x) + sum_{k=1..kmax} a_k k^-2 sin(k pi x), a_k ~ N(0,1)."""
    x = _grid(n)
    a = rng.standard_normal(kmax)
    u = np.sin(np.pi * x)
    for k in range(1, kmax + 1):
        u = u + a[k - 1] * k ** -2.0 * np.sin(k * np.pi * x)
    return np.ascontiguousarray(u)


def smooth_modes_2d(rng: np.random.Generator, nx: int, ny: int, kmax: int = 8) -> np.ndarray:
    """sin(pi x) sin(pi y) + sum_{k,l<=kmax} a_kl/(k^2+l^2) sin(k pi x) sin(l pi y)."""
    x = _grid(nx)
    y = _grid(ny)
    a = rng.standard_normal((kmax, kmax))
    u = np.outer(np.sin(np.pi * y), np.sin(np.pi * x))
    for k in range(1, kmax + 1):
        sx = np.sin(k * np.pi * x)
        for l in range(1, kmax + 1):
            u = u + a[k - 1, l - 1] / (k * k + l * l) * np.outer(np.sin(l * np.pi * y), sx)
    return np.ascontiguousarray(u)


def source_modes_1d(rng: np.random.Generator, n: int, nt: int, T: float, modes: int = 4) -> np.ndarray:
    """g(t,x) = sum_m c_m sin(p_m pi x) sin(q_m pi t/T) sampled at t_k = k T/nt, k=0..nt."""
    x = _grid(n)
    t = np.arange(nt + 1, dtype=np.float64) * (T / nt)
    c = rng.standard_normal(modes)
    p = rng.integers(1, 9, size=modes)
    q = rng.integers(1, 5, size=modes)
    g = np.zeros((nt + 1, n))
    for m in range(modes):
        g += c[m] * np.outer(np.sin(q[m] * np.pi * t / T), np.sin(p[m] * np.pi * x))
    return np.ascontiguousarray(g)


def source_modes_2d(rng: np.random.Generator, nx: int, ny: int, nt: int, T: float,
                    modes: int = 4) -> np.ndarray:
    x = _grid(nx)
    y = _grid(ny)
    t = np.arange(nt + 1, dtype=np.float64) * (T / nt)
    g = np.zeros((nt + 1, ny, nx))
    for _ in range(modes):
        c = rng.standard_normal()
        p, r = rng.integers(1, 9, size=2)
        q = rng.integers(1, 5)
        sp = np.outer(np.sin(r * np.pi * y), np.sin(p * np.pi * x))
        g += c * np.sin(q * np.pi * t / T)[:, None, None] * sp[None]
    return np.ascontiguousarray(g)


def random_field(rng: np.random.Generator, shape) -> np.ndarray:
    return np.ascontiguousarray(rng.standard_normal(shape))


# ----------------------------------------------------------------------------
# The named workloads.  Seeds are fixed per workload.
# ----------------------------------------------------------------------------

def heat1d_small(seed: int = 0) -> Problem:
    """1D, n=63, theta=1/2, n_t=256, T=0.1, g=0, 3 levels nu=2, 16 slabs, tol 1e-12."""
    rng = np.random.default_rng(seed)
    n, nt = 63, 256
    return Problem("heat1d_n63_nt256", 1, n, 1, nt, 0.1, 1.0, 0.5,
                   smooth_modes_1d(rng, n), None,
                   Schedule(nu=(2, 2), space=(False, False), m_inner=(1,), n_cgs=16),
                   tol=1e-12, precision="fp64")


def heat1d_large(seed: int = 1, precision: str = "mixed") -> Problem:
    """1D, n=1023, theta=1, n_t=8192, T=1, 4-mode space-time source, 5 levels nu=2."""
    rng = np.random.default_rng(seed)
    n, nt, T = 1023, 8192, 1.0
    u0 = smooth_modes_1d(rng, n)
    g = source_modes_1d(rng, n, nt, T)
    return Problem("heat1d_n1023_nt8192", 1, n, 1, nt, T, 1.0, 1.0, u0, g,
                   Schedule(nu=(2, 2, 2, 2), space=(False,) * 4, m_inner=(2, 2, 1), n_cgs=16),
                   tol=1e-12, precision=precision)


def heat2d_large(seed: int = 2) -> Problem:
    """2D 255x255, theta=1/2, n_t=1024, T=0.05, g=0, 4 levels nu=2 with 2x2 agglomeration."""
    rng = np.random.default_rng(seed)
    n, nt = 255, 1024
    return Problem("heat2d_255x255_nt1024", 2, n, n, nt, 0.05, 1.0, 0.5,
                   smooth_modes_2d(rng, n, n), None,
                   Schedule(nu=(2, 2, 2), space=(True, True, True), m_inner=(2, 1), n_cgs=16),
                   tol=1e-12, precision="mixed")


def heat2d_adjoint(seed: int = 3) -> Problem:
    """2D 127x127, theta=1, n_t=512, T=0.05, terminal misfit against a smooth target."""
    rng = np.random.default_rng(seed)
    n, nt = 127, 512
    u0 = smooth_modes_2d(rng, n, n)
    g = source_modes_2d(rng, n, n, nt, 0.05)
    target = smooth_modes_2d(rng, n, n)
    return Problem("heat2d_127x127_nt512_adjoint", 2, n, n, nt, 0.05, 1.0, 1.0, u0, g,
                   Schedule(nu=(2, 2, 2), space=(True, True, True), m_inner=(2, 1), n_cgs=16),
                   tol=1e-12, precision="fp64", u_target=target)


def heat2d_alternate(levels: int = 7, seed: int = 5, precision: str = "mixed") -> Problem:
    """The multilevel-count workload of Table 3 (Sec. 4.2): 2D 192x192, theta=1/2,
    n_t=2^11, C = 3 tau dt / h^2 = 0.16 (dt = 1.43e-6, T = 2.93e-3), g=0, alternate
    time-space coarsening (three time coarsenings, then space and time alternately), 16
    decoupled slabs, 2 inner iterations (1 on the level above the coarsest), tol 1e-6."""
    rng = np.random.default_rng(seed)
    n, nt = 192, 2048
    dt = 0.16 / (3.0 * (n + 1) ** 2)
    kinds = ("TTT" + "ST" * 4)[:levels - 1]
    sched = Schedule(nu=tuple(1 if k == "S" else 2 for k in kinds),
                     space=tuple(k == "S" for k in kinds),
                     m_inner=tuple([2] * (levels - 3) + [1]), n_cgs=16)
    return Problem(f"heat2d_192x192_nt2048_C0.16_L{levels}", 2, n, n, nt, nt * dt, 1.0, 0.5,
                   smooth_modes_2d(rng, n, n), None, sched, tol=1e-6, precision=precision)


# Courant-number ranges of the batch members by theta (the end time T is not given for the
# batch; it is read from a Courant number C = 2 tau dt / h^2 drawn per member): Crank-Nicolson
# members up to the largest theta = 1/2 single-problem workload (2D 255^2: C = 6.4), backward
# Euler members up to the largest theta = 1 one (1D n = 1023: C = 256); the lower end is the
# paper's smallest tested C (0.16).
BATCH_C_RANGE = {0.5: (0.16, 6.4), 1.0: (0.16, 256.0)}


def batch_end_time(C: float, n: int, nt: int, tau: float) -> float:
    """T with 2 tau (T / n_t) / h^2 = C, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    return C * nt * h * h / (2.0 * tau)


def batched_problems(seed: int = 4, count_1d: int = 48, count_2d: int = 16) -> List[Problem]:
    """Uneven problems: 1D n in {63..2047}, n_t in {256..8192}; 2D side in {63..255},
    n_t in {128..1024}; tau log-uniform in [0.1, 10]; theta in {1/2, 1}; the end time from a
    Courant number log-uniform in BATCH_C_RANGE[theta] (drawn from its own stream, seed + 1000,
    so the other draws do not depend on it)."""
    rng = np.random.default_rng(seed)
    rc = np.random.default_rng(seed + 1000)
    out: List[Problem] = []

    def end_time(theta, n, nt, tau):
        lo, hi = BATCH_C_RANGE[theta]
        C = float(math.exp(rc.uniform(math.log(lo), math.log(hi))))
        return batch_end_time(C, n, nt, tau)

    for i in range(count_1d):
        n = int(rng.integers(63, 2048))
        nt = int(rng.integers(256, 8193)) // 64 * 64
        nt = max(nt, 256)
        tau = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        theta = float(rng.choice([0.5, 1.0]))
        T = end_time(theta, n, nt, tau)
        u0 = smooth_modes_1d(rng, n)
        out.append(Problem(f"batch1d_{i}", 1, n, 1, nt, T, tau, theta, u0, None,
                           Schedule(nu=(2, 2), space=(False, False), m_inner=(1,), n_cgs=16),
                           tol=1e-10, precision="mixed"))
    for i in range(count_2d):
        n = int(rng.integers(63, 256))
        nt = int(rng.integers(128, 1025)) // 128 * 128
        nt = max(nt, 128)
        tau = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
        theta = float(rng.choice([0.5, 1.0]))
        T = end_time(theta, n, nt, tau)
        u0 = smooth_modes_2d(rng, n, n)
        out.append(Problem(f"batch2d_{i}", 2, n, n, nt, T, tau, theta, u0, None,
                           Schedule(nu=(2, 2, 2), space=(True, True, True), m_inner=(2, 1), n_cgs=16),
                           tol=1e-10, precision="mixed"))
    return out


def custom(dim: int, nx: int, nt: int, T: float, tau: float, theta: float, schedule: Schedule,
           seed: int = 0, ny: Optional[int] = None, with_source: bool = False,
           precision: str = "fp64", tol: float = 1e-12, name: str = "custom") -> Problem:
    """Small seeded problems for tests (any size, any schedule)."""
    rng = np.random.default_rng(seed)
    if dim == 1:
        u0 = smooth_modes_1d(rng, nx)
        g = source_modes_1d(rng, nx, nt, T) if with_source else None
        return Problem(name, 1, nx, 1, nt, T, tau, theta, u0, g, schedule, tol, precision)
    ny = nx if ny is None else ny
    u0 = smooth_modes_2d(rng, nx, ny)
    g = source_modes_2d(rng, nx, ny, nt, T) if with_source else None
    return Problem(name, 2, nx, ny, nt, T, tau, theta, u0, g, schedule, tol, precision)
