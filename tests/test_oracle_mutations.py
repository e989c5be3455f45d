"""The oracle's pins have teeth (CPU only).

One plausible mistake at a time is planted in a scratch copy of the oracle: a swapped theta
weight, a wrong sign, an off-by-one time block, a missing average, a wrong Arnoldi index, a
dropped adjoint term, each piece of the MGRIT comparison, and in the plain-C march a wrong
elimination sign, off-by-one or mixed-up neighbour indices, a dropped source term, a band
limit off by one (the scratch copy then compiles the changed C source).  The pins aimed at
that part of the oracle (tests/test_oracle.py, selected by -k) must then fail, and pass on the
unchanged copy.
Each case runs pytest in a subprocess on the scratch copy; the repository is not modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in mk_oracle.py, planted replacement, -k selector of the pins that must catch it)
MUTATIONS = [
    ("rhs_theta_swap",
     "f[1:] = dt * ((1.0 - theta) * g[:-1] + theta * g[1:])",
     "f[1:] = dt * (theta * g[:-1] + (1.0 - theta) * g[1:])",
     "march_eigenmode_with_source"),
    ("apply_b_sign",
     "w[1:] = (x[1:] - self.a * Lx[1:]) - (x[:-1] + self.b * Lx[:-1])",
     "w[1:] = (x[1:] - self.a * Lx[1:]) - (x[:-1] - self.b * Lx[:-1])",
     "march_equals_dense_solve"),
    ("dense_phi_sign", "phi = I + level.b * Ls", "phi = I - level.b * Ls",
     "march_equals_dense_solve"),
    ("galerkin_a",
     "f * prev.a + (f - 1) * prev.b, prev.b, nLx, nLy))",
     "f * prev.a + f * prev.b, prev.b, nLx, nLy))",
     "galerkin_is_modified"),
    ("galerkin_b",
     "f * prev.a + (f - 1) * prev.b, prev.b, nLx, nLy))",
     "f * prev.a + (f - 1) * prev.b, f * prev.b, nLx, nLy))",
     "galerkin_is_modified"),
    ("Y_without_average", "Y[s, j] = 1.0 / len(s)", "Y[s, j] = 1.0", "YtZ_identity"),
    ("restrict_last_step_only",
     "out[1:] = v[1:].reshape((nT, nu) + v.shape[1:]).sum(axis=1)",
     "out[1:] = v[nu::nu]",
     "restrict_interpolate_are_dense"),
    ("interp_previous_block",
     "out[1:] = np.repeat(vt[1:], nu, axis=0)",
     "out[1:] = np.repeat(vt[:-1], nu, axis=0)",
     "restrict_interpolate_are_dense"),
    ("correction_sign",
     "    return v - t                                         # 4.5",
     "    return v + t                                         # 4.5",
     "two_level_precondition_is_dense_Q"),
    ("shift_sign",
     "vhat = restrict(lv, H.nu[l], H.space[l], s - lv.mu * v)   # 4.2",
     "vhat = restrict(lv, H.nu[l], H.space[l], s + lv.mu * v)   # 4.2",
     "two_level_precondition_is_dense_Q"),
    ("Q_without_mu",
     "return np.eye(A.shape[0]) - Z @ AHinv_Yt @ A + mu * Z @ AHinv_Yt",
     "return np.eye(A.shape[0]) - Z @ AHinv_Yt @ A + Z @ AHinv_Yt",
     "two_level_precondition_is_dense_Q"),
    ("decoupled_wrong_step",
     "if (k - 1) % s != 0:  # not the first step of its slab",
     "if k % s != 0:  # not the first step of its slab",
     "coarsest_solve_is_dense_decoupled"),
    ("coarsest_block0", "x[0] = r[0]", "x[0] = 0.5 * r[0]", "coarsest_solve_is_dense_decoupled"),
    ("lambda_max_wrong_end", "lam = -ex.min()", "lam = -ex.max()", "lambda_max_matches"),
    ("arnoldi_index",
     "Hm[i, j] = np.vdot(w.ravel(), V[i].ravel())",
     "Hm[i, j] = np.vdot(w.ravel(), V[j].ravel())",
     "inner_fgmres_minimises"),
    ("lsq_without_beta", "rhs[0] = beta", "rhs[0] = 1.0", "inner_fgmres_minimises"),
    ("adjoint_g_weight",
     "gg[1:] += dt * theta * lam[1:]",
     "gg[1:] += dt * (1.0 - theta) * lam[1:]",
     "adjoint_gradients_vs_central"),
    ("adjoint_tau_blend",
     "Lu = lv.apply_L(theta * u[1:] + (1.0 - theta) * u[:-1]) / tau",
     "Lu = lv.apply_L(theta * u[:-1] + (1.0 - theta) * u[1:]) / tau",
     "adjoint_gradients_vs_central"),
    ("adjoint_lam0_drops_phi",
     "lam[0] = bvec[0] + lam[1] + level.b * lt.apply_L(lam[1])",
     "lam[0] = bvec[0] + lam[1]",
     "adjoint_march_solves_transpose"),
    ("mgrit_inject_wrong_point",
     "return v[::nu].copy()",
     "return v[nu - 1::nu].copy() if nu > 1 else v.copy()",
     "mgrit_transfers_are_partition"),
    ("mgrit_ideal_without_psi_solve",
     "out[k] = sla.lu_solve(lu, rhs.reshape(-1)).reshape(ns)",
     "out[k] = rhs",
     "mgrit_transfers_are_partition"),
    ("mgrit_coarse_theta_swap",
     "lv = Level(fine.dim, fine.nt // nu, theta * DT, (1.0 - theta) * DT, fine.Lx, fine.Ly)",
     "lv = Level(fine.dim, fine.nt // nu, (1.0 - theta) * DT, theta * DT, fine.Lx, fine.Ly)",
     "mgrit_coarse_level_is"),
    ("mgrit_coarse_step", "DT = nu * dt\n", "DT = (nu - 1) * dt\n", "mgrit_coarse_level_is"),
]

# the same for the plain-C march (oracle/march.c)
MUTATIONS_C = [
    ("thomas_forward_sign", "if (i > 0) r -= sub * rhs[i - 1];", "if (i > 0) r += sub * rhs[i - 1];"),
    ("explicit_lo_off_by_one", "if (i > 0) lx += lo[i] * x[i - 1];",
     "if (i > 1) lx += lo[i] * x[i - 1];"),
    ("u0_not_copied", "memcpy(u, f, sizeof(double) * n); /* u_0 = f_0 */",
     "memset(u, 0, sizeof(double) * n);"),
    ("apply2d_y_index", "if (j > 0) s += ylo[j] * v[p - nx];",
     "if (j > 0) s += ylo[i % ny] * v[p - nx];"),
    ("band_x_sign", "if (i > 0) B(p, p - 1) = -a * xlo[i];", "if (i > 0) B(p, p - 1) = a * xlo[i];"),
    ("band_y_index", "if (j > 0) B(p, p - nx) = -a * ylo[j];",
     "if (j > 0) B(p, p - nx) = -a * ylo[i % ny];"),
    ("rhs2d_drops_source", "rhs[p] = prev[p] + b * lv[p] + fk[p];", "rhs[p] = prev[p] + b * lv[p];"),
    ("forward_band_limit", "int first = (p - w > 0) ? p - w : 0;",
     "int first = (p - w + 1 > 0) ? p - w + 1 : 0;"),
]
MARCH_PINS = "march_eigenmode or march_equals_dense_solve"
CASES = ([("mk_oracle.py",) + m for m in MUTATIONS] +
         [("march.c", n, o, r, MARCH_PINS) for n, o, r in MUTATIONS_C])


def _run(base, selector):
    env = dict(os.environ)
    env.pop("PYTHONPATH", None)
    # no bytecode: a planted mistake of the same length written within the same second as
    # the original would otherwise match a cached .pyc (keyed by mtime and size) and run stale
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    for d, _, _ in os.walk(base):
        if os.path.basename(d) == "__pycache__":
            shutil.rmtree(d, ignore_errors=True)
    return subprocess.run([sys.executable, "-B", "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           "tests/test_oracle.py", "-k", selector],
                          cwd=base, capture_output=True, text=True, timeout=600, env=env)


def _drop_march_library(base):
    so = os.path.join(base, "oracle", "liboracle_march.so")
    if os.path.exists(so):
        os.remove(so)


@pytest.fixture(scope="module")
def scratch(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutations"))
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(base, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(base, "tests"))
    for f in ("test_oracle.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(base, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(base, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "workloads.py"), base)
    return base


def test_unchanged_copy_passes_the_targeted_pins(scratch):
    selector = " or ".join(sorted({c[4] for c in CASES}))
    _drop_march_library(scratch)
    r = _run(scratch, selector)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("fname,name,old,new,selector", CASES, ids=[c[1] for c in CASES])
def test_planted_mistake_is_caught(scratch, fname, name, old, new, selector):
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(old) == 1, name
    path = os.path.join(scratch, "oracle", fname)
    open(path, "w").write(src.replace(old, new))
    if fname.endswith(".c"):
        _drop_march_library(scratch)
    try:
        r = _run(scratch, selector)
    finally:
        open(path, "w").write(src)
        if fname.endswith(".c"):
            _drop_march_library(scratch)
    assert r.returncode == 1, (name, r.stdout[-3000:])
