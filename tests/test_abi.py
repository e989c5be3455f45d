"""The C-ABI library builds, loads, and exports every entry point include/mk.h declares.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mk.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mk_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_00228_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2401_00228_gb300 import _lib
    for n in _declared():
        assert n in _lib.SIGNATURES, n


def test_status_strings_and_defaults(lib):
    from paper_2401_00228_gb300 import _lib, mk_default_opts
    L = _lib.load()
    for code, name in _lib.STATUS.items():
        assert L.mk_status_string(code).decode() == name
    o = mk_default_opts()
    assert o.tol == 1e-12 and o.levels == 3 and o.n_cgs == 16 and o.restart == 40
    assert list(o.nu)[:2] == [2, 2] and o.m_inner[0] == 1


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the sizes the C compiler gives them."""
    from paper_2401_00228_gb300 import _lib
    import subprocess
    import tempfile
    code = r'''
#include <stdio.h>
#include "mk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(mk_stencil), sizeof(mk_solve_opts), sizeof(mk_solve_info),
         sizeof(mk_level_desc), sizeof(mk_tune_info));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = list(map(int, subprocess.check_output([exe]).split()))
    assert sizes == [ctypes.sizeof(_lib.mk_stencil), ctypes.sizeof(_lib.mk_solve_opts),
                     ctypes.sizeof(_lib.mk_solve_info), ctypes.sizeof(_lib.mk_level_desc),
                     ctypes.sizeof(_lib.mk_tune_info)]


def test_struct_field_offsets_match_header():
    """Every field of the ctypes mirrors sits at the offset the C compiler gives it (equal sizes
    alone would not catch two fields swapped)."""
    from paper_2401_00228_gb300 import _lib
    import subprocess
    import tempfile
    structs = [_lib.mk_stencil, _lib.mk_solve_opts, _lib.mk_solve_info, _lib.mk_level_desc,
               _lib.mk_tune_info]
    lines = []
    for st in structs:
        for name, _ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({st.__name__}, {name}));')
    code = "#include <stddef.h>\n#include <stdio.h>\n#include \"mk.h\"\nint main(void) {\n" + \
        "\n".join(lines) + "\n  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        offs = list(map(int, subprocess.check_output([exe]).split()))
    want = [getattr(st, name).offset for st in structs for name, _ in st._fields_]
    assert offs == want


def test_transfer_option_values():
    from paper_2401_00228_gb300 import _lib, make_opts, mk_default_opts
    assert mk_default_opts().transfer == _lib.MK_TRANSFER_MK == 0
    assert make_opts(levels=2, transfer="mgrit").transfer == _lib.MK_TRANSFER_MGRIT == 1
    hdr = open(HEADER).read()
    assert "#define MK_TRANSFER_MK 0" in hdr and "#define MK_TRANSFER_MGRIT 1" in hdr
    with pytest.raises(KeyError):
        make_opts(transfer="parareal")


def test_product_path_does_not_import_oracle():
    """The package never references the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2401_00228_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
