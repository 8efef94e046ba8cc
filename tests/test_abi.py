"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/vmat.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vmat.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"VMAT_API\s+[\w\s\*]*?\b(vmat_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1005_4396_b300 import build
    build.build_vmat()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared()
    for n in ["vmat_create", "vmat_destroy", "vmat_dose", "vmat_price", "vmat_pricing_select",
              "vmat_add_column", "vmat_master_step", "vmat_colgen_run", "vmat_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1005_4396_b300 import vmat
    assert sorted(vmat.EXPORTS) == declared()


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the C compiler's size and field offsets."""
    import subprocess
    from paper_1005_4396_b300 import vmat
    structs = [vmat.vmat_problem, vmat.vmat_info, vmat.vmat_column, vmat.vmat_colgen_opts,
               vmat.vmat_colgen_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(){"]
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want += [getattr(st, f).offset for f, _ in st._fields_]
    assert got == want
