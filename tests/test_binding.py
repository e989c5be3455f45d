"""Host-side logic of the Python binding (no GPU): options built from Python values land in
the right fields of the ABI struct, arrays are checked before a pointer crosses the ABI,
status codes map to exceptions, and the one-call solve rejects bad arguments before it
touches the device.  The library is loaded (it needs no GPU to load); no compute is called.
"""
import numpy as np
import pytest

import paper_2401_00228_gb300 as mk
from paper_2401_00228_gb300 import _lib


def test_make_opts_fields():
    o = mk.make_opts(levels=4, nu=(2, 4, 2), space=(False, True, True), m_inner=(3, 1),
                     n_cgs=8, tol=1e-9, restart=60, max_iters=500, precision="mixed",
                     mu="one", use_graph=False, orth=2, autotune=True, transfer="mk")
    assert o.levels == 4 and list(o.nu)[:3] == [2, 4, 2]
    assert list(o.space)[:3] == [0, 1, 1] and list(o.m_inner)[:2] == [3, 1]
    assert (o.n_cgs, o.tol, o.restart, o.max_iters) == (8, 1e-9, 60, 500)
    assert (o.precision, o.mu_mode, o.use_graph, o.orth, o.autotune, o.transfer) == \
        (1, 1, 0, 2, 1, _lib.MK_TRANSFER_MK)
    # unset per-level entries keep the library defaults
    d = mk.mk_default_opts()
    assert list(o.nu)[3:] == list(d.nu)[3:]


def test_make_opts_mu_modes():
    assert mk.make_opts(mu="lambda_max").mu_mode == 0
    assert mk.make_opts(mu="one").mu_mode == 1
    o = mk.make_opts(mu=0.25)
    assert o.mu_mode == 2 and o.mu_value == 0.25
    with pytest.raises(KeyError):
        mk.make_opts(precision="fp16")


def test_library_defaults():
    d = mk.mk_default_opts()
    assert (d.tol, d.restart, d.max_iters, d.levels, d.n_cgs) == (1e-12, 40, 2000, 3, 16)
    assert (d.mu_mode, d.precision, d.use_graph, d.orth, d.autotune, d.transfer) == \
        (0, 0, 1, 1, 0, 0)
    assert list(d.nu) == [2] * _lib.MK_MAX_LEVELS and d.m_inner[0] == 1


def test_arrays_are_checked_before_crossing_the_abi():
    from paper_2401_00228_gb300 import _ptr
    assert _ptr(None) is None
    a = np.zeros(8)
    assert _ptr(a) == a.ctypes.data
    with pytest.raises(TypeError):
        _ptr(np.zeros(8, dtype=np.float32))
    with pytest.raises(TypeError):
        _ptr(np.zeros((8, 8))[:, ::2])
    with pytest.raises(TypeError):
        _ptr([0.0, 1.0])
    torch = pytest.importorskip("torch")
    t = torch.zeros(8, dtype=torch.float64)
    assert _ptr(t) == t.data_ptr()
    with pytest.raises(TypeError):
        _ptr(torch.zeros(8, dtype=torch.float32))
    with pytest.raises(TypeError):
        _ptr(torch.zeros(8, 8, dtype=torch.float64).t())


def test_status_codes_raise():
    assert _lib.check(_lib.MK_OK, "x") == _lib.MK_OK
    assert _lib.check(_lib.MK_ERR_NOT_CONVERGED, "x", allow=(_lib.MK_ERR_NOT_CONVERGED,)) == \
        _lib.MK_ERR_NOT_CONVERGED
    for code in (_lib.MK_ERR_INVALID, _lib.MK_ERR_NOMEM, _lib.MK_ERR_TOO_LARGE):
        with pytest.raises(mk.MKError) as e:
            _lib.check(code, "where")
        assert e.value.code == code and _lib.STATUS[code] in str(e.value)


def test_one_call_solve_rejects_bad_arguments():
    u0 = np.zeros(7)
    with pytest.raises(ValueError):
        mk.solve(u0, None, 1.0, 1.0, 0.01, 0)            # nt < 1
    with pytest.raises(ValueError):
        mk.solve(u0, None, 1.0, 1.0, 0.0, 8)             # dt <= 0
    with pytest.raises(ValueError):
        mk.solve(np.zeros((2, 3, 4)), None, 1.0, 1.0, 0.01, 8)   # not 1D or 2D


def test_alternate_schedule_through_the_binding():
    """Host-only entry point: Table 3's 9-level schedule (Sec. 4.2) for the 192^2 workload."""
    n, nt = 192, 2048
    dt = 0.16 / (3.0 * (n + 1) ** 2)
    o = mk.mk_schedule_alternate(2, n, n, nt, 1.0, dt, 9, n_cgs=16)
    kinds = "".join("S" if o.space[i] else "T" for i in range(o.levels - 1))
    assert o.levels == 9 and kinds == "TTTSTSTS"
    assert [o.nu[i] for i in range(8)] == [2, 2, 2, 1, 2, 1, 2, 1]
    with pytest.raises(mk.MKError):
        mk.mk_schedule_alternate(2, n, n, nt, 1.0, dt, 1)   # fewer than 2 levels


def test_noalloc_residual_checks_sizes_before_the_abi(monkeypatch):
    """The allocation-free residual takes bare device pointers, so the binding checks every
    array against the problem's shape first: a short array raises ValueError and no compute
    entry point is reached (the stub library records any call)."""
    calls = []

    class Stub:
        def mk_problem_shape(self, p, dim, nx, ny, nt, *rest):
            dim._obj.value, nx._obj.value, ny._obj.value, nt._obj.value = 1, 63, 1, 256
            return _lib.MK_OK

        def __getattr__(self, name):
            def rec(*a):
                calls.append(name)
                return _lib.MK_OK
            return rec

    monkeypatch.setattr(mk, "lib", lambda: Stub())
    assert mk.mk_problem_shape(1) == (1, 63, 1, 256)
    full, short = np.zeros(257 * 63), np.zeros(257 * 63 - 1)
    one, steps = np.zeros(1), np.zeros(257)
    for args in ((short, full, None, one, None), (full, short, None, one, None),
                 (full, full, short, one, None), (full, full, None, np.zeros(0), None),
                 (full, full, None, one, np.zeros(256))):
        with pytest.raises(ValueError):
            mk.mk_op_residual_noalloc(1, *args)
    assert calls == []
    mk.mk_op_residual_noalloc(1, full, full, full, one, steps)
    assert calls == ["mk_op_residual_noalloc"]
