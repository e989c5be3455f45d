"""Python binding of libmk: the all-at-once space-time theta-scheme solve by FGMRES with the
multilevel Krylov (MK) preconditioner (Erlangga, parallel-in-time MK), on one GB300.

This module only marshals arguments to the C ABI (include/mk.h); every step of the solve runs
in the library's CUDA kernels.  Arrays are torch tensors (CUDA or CPU) or numpy arrays, FP64,
C-contiguous: space-time arrays (n_t+1, nx) / (n_t+1, ny, nx), spatial ones (nx) / (ny, nx).
Functions carry the ABI's names; ``Problem`` and ``HeatSolve`` are conveniences on top.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (MK_MAX_LEVELS, MKError, mk_level_desc, mk_solve_info, mk_solve_opts,
                   mk_stencil, mk_tune_info)

__all__ = ["mk_default_opts", "mk_create_problem", "mk_set_source", "mk_destroy", "mk_solve",
           "mk_solve_rhs", "mk_march", "mk_tune", "mk_trim", "mk_schedule_alternate", "mk_adjoint", "mk_level_info", "mk_op_rhs", "mk_op_apply",
           "mk_op_residual", "mk_op_residual_noalloc", "mk_problem_shape", "mk_op_restrict", "mk_op_interp_correct", "mk_op_interp_combine", "mk_op_coarsest",
           "mk_op_precond", "mk_op_orthogonalize", "mk_op_lsq", "mk_kernel_launch_count",
           "mk_create_batch", "mk_solve_batch", "mk_destroy_batch", "Batch",
           "make_opts", "Problem", "HeatSolve", "MKError", "lib", "solve"]


def lib():
    return _lib.load()


def _ptr(a) -> Optional[int]:
    """Raw pointer of a float64 C-contiguous torch tensor / numpy array (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("arrays must be float64 and C-contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _current_stream_for(*arrays):
    try:
        import torch
    except ImportError:
        return None
    for a in arrays:
        if isinstance(a, torch.Tensor) and a.is_cuda:
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def mk_default_opts() -> mk_solve_opts:
    o = mk_solve_opts()
    lib().mk_default_opts(ctypes.byref(o))
    return o


def make_opts(levels: int = 3, nu: Sequence[int] = (), space: Sequence[bool] = (),
              m_inner: Sequence[int] = (), n_cgs: int = 16, tol: float = 1e-12, restart: int = 40,
              max_iters: int = 2000, precision: str = "fp64", mu: str | float = "lambda_max",
              use_graph: bool = True, orth: int = 1, autotune: bool = False,
              transfer: str = "mk", inner: str = "auto", augment: int = 0) -> mk_solve_opts:
    """Options struct from Python values (unset per-level entries keep the defaults).
    transfer: "mk" (Sec. 3.2 block transfers, Galerkin levels) or "mgrit" (the comparison
    two-level method of Eqs. (mgritY), (mgritZ) with the coarse matrix of Eq. (coarsemat)).
    inner: "auto", "separate" (one launch per step of the inner levels) or "coop" (the inner
    recursion in one cooperative kernel).  augment: k recycled corrections per restart cycle
    (0: plain FGMRES(m)).  precision: "fp64", "mixed" (FP32 cycle, double-float level-1 basis)
    or "mixed32" (FP32 cycle and FP32 level-1 basis; FP64 true residual at every restart)."""
    o = mk_default_opts()
    o.levels = levels
    for i, v in enumerate(nu):
        o.nu[i] = int(v)
    for i, v in enumerate(space):
        o.space[i] = 1 if v else 0
    for i, v in enumerate(m_inner):
        o.m_inner[i] = int(v)
    o.n_cgs = n_cgs
    o.tol = tol
    o.restart = restart
    o.max_iters = max_iters
    o.precision = {"fp64": 0, "mixed": 1, "mixed32": 2}[precision]
    if mu == "lambda_max":
        o.mu_mode = 0
    elif mu == "one":
        o.mu_mode = 1
    else:
        o.mu_mode, o.mu_value = 2, float(mu)
    o.use_graph = 1 if use_graph else 0
    o.orth = int(orth)
    o.autotune = 1 if autotune else 0
    o.transfer = {"mk": _lib.MK_TRANSFER_MK, "mgrit": _lib.MK_TRANSFER_MGRIT}[transfer]
    o.inner_kernel = {"auto": _lib.MK_INNER_AUTO, "separate": _lib.MK_INNER_SEPARATE,
                      "coop": _lib.MK_INNER_COOP}[inner]
    o.augment = int(augment)
    return o


def mk_schedule_alternate(dim: int, nx: int, ny: int, nt: int, tau: float, dt: float, levels: int,
                          n_cgs: int = 16, c_max: float = 1.0, opts: mk_solve_opts | None = None,
                          **kw) -> mk_solve_opts:
    """Alternate time-space coarsening (Sec. 4.2): levels, nu, space, m_inner and n_cgs filled
    in by the library into `opts` (or into make_opts(**kw))."""
    o = make_opts(**kw) if opts is None else opts
    _lib.check(lib().mk_schedule_alternate(dim, nx, ny if dim == 2 else 1, nt, tau, dt, levels,
                                           n_cgs, c_max, ctypes.byref(o)), "mk_schedule_alternate")
    return o


def mk_kernel_launch_count() -> int:
    return int(lib().mk_kernel_launch_count())


def mk_create_problem(dim: int, nx: int, ny: int, tau: float, theta: float, dt: float, nt: int,
                      g=None) -> int:
    st = mk_stencil(dim, nx, ny if dim == 2 else 1, tau)
    out = ctypes.c_void_p()
    _lib.check(lib().mk_create_problem(ctypes.byref(st), theta, dt, nt, _ptr(g), ctypes.byref(out)),
               "mk_create_problem")
    return out.value


def mk_set_source(p: int, g, stream=None) -> None:
    _lib.check(lib().mk_set_source(p, _ptr(g), _stream(stream) or _current_stream_for(g)),
               "mk_set_source")


def mk_destroy(p: int) -> None:
    lib().mk_destroy(p)


def mk_solve(p: int, u0, u_out, opts: Optional[mk_solve_opts] = None, stream=None,
             allow_not_converged: bool = False) -> mk_solve_info:
    info = mk_solve_info()
    s = _stream(stream) or _current_stream_for(u0, u_out)
    code = lib().mk_solve(p, _ptr(u0), ctypes.byref(opts) if opts else None, _ptr(u_out),
                          ctypes.byref(info), s)
    _lib.check(code, "mk_solve", allow=(_lib.MK_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return info


def mk_create_batch(problems: Sequence[int], opts: Optional[Sequence[mk_solve_opts]] = None,
                    autotune: bool = True) -> int:
    """Batch handle for the given problem handles (one options struct per problem, or None)."""
    n = len(problems)
    arr = (ctypes.c_void_p * n)(*problems)
    oarr = (mk_solve_opts * n)(*opts) if opts is not None else None
    out = ctypes.c_void_p()
    _lib.check(lib().mk_create_batch(arr, n, oarr, 1 if autotune else 0, ctypes.byref(out)),
               "mk_create_batch")
    return out.value


def mk_solve_batch(b: int, u0s: Sequence, u_outs: Sequence, stream=None,
                   allow_not_converged: bool = False) -> List[mk_solve_info]:
    """Solve every member: u0s[i] -> u_outs[i]; returns the per-member infos."""
    n = len(u0s)
    if len(u_outs) != n:
        raise ValueError("u0s and u_outs differ in length")
    a0 = (ctypes.c_void_p * n)(*[_ptr(x) for x in u0s])
    a1 = (ctypes.c_void_p * n)(*[_ptr(x) for x in u_outs])
    infos = (mk_solve_info * n)()
    s = _stream(stream) or _current_stream_for(*u0s, *u_outs)
    code = lib().mk_solve_batch(b, a0, a1, infos, s)
    _lib.check(code, "mk_solve_batch",
               allow=(_lib.MK_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return list(infos)


def mk_destroy_batch(b: int) -> None:
    lib().mk_destroy_batch(b)


class Batch:
    """Owning handle of an mk_batch over Problem objects (which must outlive it)."""

    def __init__(self, problems: Sequence["Problem"], opts: Optional[Sequence[mk_solve_opts]] = None,
                 autotune: bool = True):
        self.problems = list(problems)
        self.handle = mk_create_batch([p.handle for p in self.problems], opts, autotune)

    def solve(self, u0s, u_outs, stream=None, allow_not_converged=False) -> List[mk_solve_info]:
        return mk_solve_batch(self.handle, u0s, u_outs, stream, allow_not_converged)

    def close(self):
        if self.handle:
            mk_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mk_solve_rhs(p: int, f, u_out, opts: Optional[mk_solve_opts] = None, stream=None) -> mk_solve_info:
    info = mk_solve_info()
    s = _stream(stream) or _current_stream_for(f, u_out)
    _lib.check(lib().mk_solve_rhs(p, _ptr(f), ctypes.byref(opts) if opts else None, _ptr(u_out),
                                  ctypes.byref(info), s), "mk_solve_rhs")
    return info


def mk_tune(p: int, u0, base: Optional[mk_solve_opts] = None, levels: bool = False,
            max_trials: int = 0, restart_cap: bool = False, stream=None):
    """Schedule autotuner: (best options, mk_tune_info) from timed solves of this problem
    (inner iteration counts, n_cgs, restart -- at most base.restart when `restart_cap` --, in
    up to two coordinate-descent passes; the level count too when `levels`)."""
    best = mk_solve_opts()
    info = mk_tune_info()
    s = _stream(stream) or _current_stream_for(u0)
    flags = (_lib.MK_TUNE_LEVELS if levels else 0) | (_lib.MK_TUNE_RESTART_CAP if restart_cap else 0)
    _lib.check(lib().mk_tune(p, _ptr(u0), ctypes.byref(base) if base else None, flags, max_trials,
                             ctypes.byref(best), ctypes.byref(info), s), "mk_tune")
    return best, info


def mk_trim(p: int) -> None:
    """Free the solver workspace the problem keeps for its last options."""
    _lib.check(lib().mk_trim(p), "mk_trim")


def mk_march(p: int, u0, u_out, stream=None) -> None:
    s = _stream(stream) or _current_stream_for(u0, u_out)
    _lib.check(lib().mk_march(p, _ptr(u0), _ptr(u_out), s), "mk_march")


def mk_adjoint(p: int, u, dJdu, opts: Optional[mk_solve_opts] = None, grad_u0=None, grad_g=None,
               want_tau: bool = False, lam=None, stream=None):
    """Returns (dJ/dtau or None, solve info); other gradients are written in place."""
    info = mk_solve_info()
    gt = ctypes.c_double(0.0)
    s = _stream(stream) or _current_stream_for(u, dJdu)
    _lib.check(lib().mk_adjoint(p, _ptr(u), _ptr(dJdu), ctypes.byref(opts) if opts else None,
                                _ptr(grad_u0), _ptr(grad_g),
                                ctypes.addressof(gt) if want_tau else None, _ptr(lam),
                                ctypes.byref(info), s), "mk_adjoint")
    return (gt.value if want_tau else None), info


def mk_level_info(p: int, opts: Optional[mk_solve_opts], level: int):
    d = mk_level_desc()
    # sizes first, then coefficients
    _lib.check(lib().mk_level_info(p, ctypes.byref(opts) if opts else None, level, ctypes.byref(d),
                                   None, None), "mk_level_info")
    xc = np.zeros(3 * d.nx)
    yc = np.zeros(3 * d.ny) if d.dim == 2 else None
    _lib.check(lib().mk_level_info(p, ctypes.byref(opts) if opts else None, level, None, _ptr(xc),
                                   _ptr(yc)), "mk_level_info")
    return d, xc.reshape(3, d.nx), (yc.reshape(3, d.ny) if yc is not None else None)


def mk_op_rhs(p: int, u0, f, stream=None) -> None:
    _lib.check(lib().mk_op_rhs(p, _ptr(u0), _ptr(f), _stream(stream)), "mk_op_rhs")


def mk_op_apply(p: int, opts, level: int, precision: int, x, w, stream=None) -> None:
    _lib.check(lib().mk_op_apply(p, ctypes.byref(opts) if opts else None, level, precision, _ptr(x),
                                 _ptr(w), _stream(stream)), "mk_op_apply")


def mk_op_residual(p: int, f, u, r, stream=None) -> float:
    nrm = ctypes.c_double(0.0)
    _lib.check(lib().mk_op_residual(p, _ptr(f), _ptr(u), _ptr(r), ctypes.byref(nrm), _stream(stream)),
               "mk_op_residual")
    return nrm.value


def mk_problem_shape(p: int):
    """(dim, nx, ny, nt) of a problem handle (host only)."""
    d, nx, ny, nt = (ctypes.c_int32() for _ in range(4))
    _lib.check(lib().mk_problem_shape(p, ctypes.byref(d), ctypes.byref(nx), ctypes.byref(ny),
                                      ctypes.byref(nt), None, None, None), "mk_problem_shape")
    return d.value, nx.value, ny.value, nt.value


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def mk_op_residual_noalloc(p: int, f, u, r, rnorm, rnorm_steps=None, stream=None) -> None:
    """r = f - A_h u, rnorm[0] = ||r||_2, rnorm_steps[k] = ||r_k||_2; every array on the device.

    The library allocates nothing in this call (its reduction scratch is static device
    memory); r and rnorm_steps may be None.  Results are ready in stream order.  The library
    receives bare pointers and cannot see array sizes, so they are checked here against the
    problem's shape: f, u (and r) need (n_t+1)*nx*ny elements, rnorm one, rnorm_steps n_t+1;
    a short array raises ValueError before anything is launched."""
    _, nx, ny, nt = mk_problem_shape(p)
    need = (nt + 1) * nx * ny
    for name, a, n in (("f", f, need), ("u", u, need), ("r", r, need), ("rnorm", rnorm, 1),
                       ("rnorm_steps", rnorm_steps, nt + 1)):
        if a is not None and _numel(a) < n:
            raise ValueError(f"mk_op_residual_noalloc: {name} has {_numel(a)} elements, needs {n}")
    s = _stream(stream) or _current_stream_for(f, u)
    _lib.check(lib().mk_op_residual_noalloc(p, _ptr(f), _ptr(u), _ptr(r), _ptr(rnorm),
                                            _ptr(rnorm_steps), s), "mk_op_residual_noalloc")


def mk_op_restrict(p: int, opts, level: int, precision: int, v, vhat, stream=None) -> None:
    _lib.check(lib().mk_op_restrict(p, ctypes.byref(opts) if opts else None, level, precision, _ptr(v),
                                    _ptr(vhat), _stream(stream)), "mk_op_restrict")


def mk_op_interp_correct(p: int, opts, level: int, precision: int, v, vt, x, w, stream=None) -> None:
    _lib.check(lib().mk_op_interp_correct(p, ctypes.byref(opts) if opts else None, level, precision,
                                          _ptr(v), _ptr(vt), _ptr(x), _ptr(w), _stream(stream)),
               "mk_op_interp_correct")


def mk_op_interp_combine(p: int, opts, level: int, precision: int, v, sigma: float, vt, nvt: int,
                         y, x, w, stream=None) -> None:
    """x = sigma v - Z (sum_m y_m vt_m), w = A x; vt holds nvt consecutive coarse arrays, y the
    nvt weights (a host sequence, or None with nvt = 1).  precision 2: the level-1 double-float
    path of the mixed solve."""
    yh = None if y is None else np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    if yh is not None and yh.size != nvt:
        raise ValueError("y must hold nvt weights")
    _lib.check(lib().mk_op_interp_combine(p, ctypes.byref(opts) if opts else None, level, precision,
                                          _ptr(v), float(sigma), _ptr(vt), nvt, _ptr(yh), _ptr(x),
                                          _ptr(w), _stream(stream)), "mk_op_interp_combine")


def mk_op_coarsest(p: int, opts, precision: int, r, x, stream=None) -> None:
    _lib.check(lib().mk_op_coarsest(p, ctypes.byref(opts) if opts else None, precision, _ptr(r), _ptr(x),
                                    _stream(stream)), "mk_op_coarsest")


def mk_op_precond(p: int, opts, level: int, v, x, stream=None) -> None:
    _lib.check(lib().mk_op_precond(p, ctypes.byref(opts) if opts else None, level, _ptr(v), _ptr(x),
                                   _stream(stream)), "mk_op_precond")


def mk_op_orthogonalize(p: int, j: int, V, w, h, stream=None) -> None:
    _lib.check(lib().mk_op_orthogonalize(p, j, _ptr(V), _ptr(w), _ptr(h), _stream(stream)),
               "mk_op_orthogonalize")


def mk_op_lsq(j: int, H, beta: float, y, stream=None) -> float:
    res = ctypes.c_double(0.0)
    _lib.check(lib().mk_op_lsq(j, _ptr(H), beta, _ptr(y), ctypes.byref(res), _stream(stream)),
               "mk_op_lsq")
    return res.value


def _copy(a):
    if a is None:
        return None
    return a.copy() if isinstance(a, np.ndarray) else a.detach().clone()


class Problem:
    """Owning handle of an mk_problem.  `source` is a copy of the source g the problem holds
    (given at creation or through set_source; None for g = 0)."""

    def __init__(self, dim: int, nx: int, tau: float, theta: float, dt: float, nt: int, g=None,
                 ny: int = 1):
        self.dim, self.nx, self.ny, self.nt = dim, nx, (ny if dim == 2 else 1), nt
        self.tau, self.theta, self.dt = tau, theta, dt
        self.handle = mk_create_problem(dim, nx, self.ny, tau, theta, dt, nt, g)
        self.source = _copy(g)

    def set_source(self, g, stream=None) -> None:
        """Replace the source g (None: g = 0); the object keeps a copy of it."""
        mk_set_source(self.handle, g, stream)
        self.source = _copy(g)

    @property
    def space_shape(self):
        return (self.nx,) if self.dim == 1 else (self.ny, self.nx)

    @property
    def shape(self):
        return (self.nt + 1,) + self.space_shape

    def close(self):
        if self.handle:
            mk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(u0, g=None, tau: float = 1.0, theta: float = 1.0, dt: float = 0.0, nt: int = 0,
          opts: Optional[mk_solve_opts] = None, **kw):
    """One call: the solution of Eq. (finesys) for initial state u0 ((nx,) in 1D, (ny, nx) in
    2D) and source g ((nt+1, ...) or None) by the MK solver, as an (nt+1, ...) array of the
    same kind as u0 (a torch tensor on u0's device, or a numpy array).  The problem is created
    and freed inside; options from `opts` or make_opts(**kw)."""
    if nt < 1 or not dt > 0.0:
        raise ValueError("nt >= 1 and dt > 0 are required")
    shape = tuple(u0.shape)
    if len(shape) not in (1, 2):
        raise ValueError("u0 must have shape (nx,) or (ny, nx)")
    dim = len(shape)
    nx, ny = shape[-1], (shape[0] if dim == 2 else 1)
    o = make_opts(**kw) if opts is None else opts
    out_shape = (nt + 1,) + shape
    try:
        import torch
        is_torch = isinstance(u0, torch.Tensor)
    except ImportError:
        is_torch = False
    if is_torch:
        u = torch.empty(out_shape, dtype=torch.float64, device=u0.device)
    else:
        u = np.empty(out_shape, dtype=np.float64)
    with Problem(dim, nx, tau, theta, dt, nt, g, ny=ny) as p:
        mk_solve(p.handle, u0, u, o)
    return u


class HeatSolve:
    """torch.autograd.Function factory: u = A_h^{-1} f_h(u0, g) with the MK solver forward and
    the adjoint MK solve backward (gradients w.r.t. u0, g and tau).  The forward pass solves
    with the autograd input g and then restores the problem's own source (Problem.source), so
    later solves on the same problem are unaffected."""

    @staticmethod
    def apply(problem: Problem, u0, g, tau_tensor, opts: Optional[mk_solve_opts] = None):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, u0_, g_, tau_):
                if abs(float(tau_) - problem.tau) > 0.0:
                    raise ValueError("tau differs from the problem's tau; create a new Problem")
                u = torch.empty(problem.shape, dtype=torch.float64, device=u0_.device)
                if g_ is not None:
                    mk_set_source(problem.handle, g_.contiguous())
                try:
                    mk_solve(problem.handle, u0_.contiguous(), u, opts)
                finally:
                    if g_ is not None:
                        mk_set_source(problem.handle, problem.source)
                ctx.save_for_backward(u)
                return u

            @staticmethod
            def backward(ctx, gu):
                (u,) = ctx.saved_tensors
                gu0 = torch.empty(problem.space_shape, dtype=torch.float64, device=u.device)
                gg = torch.empty(problem.shape, dtype=torch.float64, device=u.device)
                gtau, _ = mk_adjoint(problem.handle, u, gu.contiguous(), opts, grad_u0=gu0, grad_g=gg,
                                     want_tau=True)
                return gu0, gg, torch.tensor(gtau, dtype=torch.float64, device=tau_tensor.device)

        return _Fn.apply(u0, g, tau_tensor)
