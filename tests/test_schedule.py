"""Alternate time-space coarsening schedule (Sec. 4.2), computed on the host by the library
(mk_schedule_alternate): the coarsest grids of Table 3 for 7..11 levels, the order of the
coarsenings the section describes (time coarsening until the Courant number exceeds the
limit, then space and time alternately, space first), the inner iteration counts, and the
invalid inputs.  No GPU is needed."""
import os

import pytest

mk = pytest.importorskip("paper_2401_00228_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table3():
    with open(os.path.join(GOLDEN, "table3_coarsest_grids.txt")) as fh:
        return [tuple(map(int, l.split()))[:4] for l in fh if l.strip() and not l.startswith("#")]


def _coarsest(o, n, nt):
    nx, t = n, nt
    for l in range(o.levels - 1):
        t //= o.nu[l]
        if o.space[l]:
            nx = (nx + 1) // 2
    return t, nx


@pytest.mark.parametrize("levels,nt_c,nx_c,ny_c", _table3())
def test_table3_coarsest_grids(levels, nt_c, nx_c, ny_c):
    n, nt, C = 192, 2048, 0.16
    dt = C / (3.0 * (n + 1) ** 2)
    o = mk.mk_schedule_alternate(2, n, n, nt, 1.0, dt, levels, n_cgs=16)
    assert o.levels == levels and o.n_cgs == 16
    assert _coarsest(o, n, nt) == (nt_c, nx_c)
    assert nx_c == ny_c
    kinds = "".join("S" if o.space[l] else "T" for l in range(levels - 1))
    assert kinds == ("TTT" + "ST" * 4)[:levels - 1]
    for l in range(levels - 1):
        assert o.nu[l] == (1 if o.space[l] else 2)
    assert [o.m_inner[l] for l in range(levels - 2)] == [2] * (levels - 3) + [1]


def test_switch_follows_the_courant_number():
    n, nt = 63, 1024
    h2 = 1.0 / (n + 1) ** 2
    for C, n_t_first in ((0.3, 2), (0.6, 1), (1.5, 0), (0.07, 4)):
        dt = C * h2 / 2.0
        o = mk.mk_schedule_alternate(1, n, 1, nt, 1.0, dt, 8, n_cgs=4)
        kinds = "".join("S" if o.space[l] else "T" for l in range(7))
        assert kinds.startswith("T" * n_t_first + "S"), (C, kinds)
        rest = kinds[n_t_first:]
        assert all(rest[i] == "ST"[i % 2] for i in range(len(rest))), (C, kinds)
    o = mk.mk_schedule_alternate(1, n, 1, nt, 1.0, 0.3 * h2 / 2.0, 8, n_cgs=4, c_max=0.5)
    assert o.space[1] == 1 and o.space[0] == 0


def test_other_fields_are_kept():
    o = mk.make_opts(tol=1e-7, precision="mixed", restart=17)
    o2 = mk.mk_schedule_alternate(2, 47, 47, 256, 1.0, 1e-5, 5, n_cgs=8, opts=o)
    assert o2.tol == 1e-7 and o2.precision == 1 and o2.restart == 17 and o2.n_cgs == 8


@pytest.mark.parametrize("args", [
    (3, 63, 1, 256, 1.0, 1e-4, 4, 16, 1.0),      # dim
    (1, 63, 1, 256, 1.0, 1e-4, 1, 16, 1.0),      # levels < 2
    (1, 63, 1, 256, 1.0, 1e-4, 13, 16, 1.0),     # levels > MK_MAX_LEVELS
    (1, 63, 1, 256, -1.0, 1e-4, 4, 16, 1.0),     # tau
    (1, 63, 1, 256, 1.0, 0.0, 4, 16, 1.0),       # dt
    (1, 63, 1, 256, 1.0, 1e-4, 4, 16, 0.0),      # c_max
    (1, 63, 1, 6, 1.0, 1e-9, 4, 1, 1.0),         # time coarsening of an odd n_t
    (1, 3, 1, 4096, 1.0, 1.0, 8, 1, 1.0),        # space coarsening of a single point
    (1, 63, 1, 256, 1.0, 1e-9, 4, 48, 1.0),      # coarsest n_t not divisible by n_cgs
])
def test_invalid_inputs(args):
    o = mk.make_opts()
    before = bytes(o)
    with pytest.raises(mk.MKError, match="MK_ERR_INVALID"):
        mk.mk_schedule_alternate(*args[:7], n_cgs=args[7], c_max=args[8], opts=o)
    assert bytes(o) == before
