"""librb.so builds, loads and exports every function include/rb.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(rb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_11866_gb300 import _build, rb
    _build.build()
    return rb.library()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ["rb_create", "rb_destroy", "rb_load_operators", "rb_solve",
                     "rb_solve_theta", "rb_solve_device", "rb_serve_submit", "rb_serve_poll",
                     "rb_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    from paper_1807_11866_gb300 import rb
    assert sorted(rb.EXPORTS) == [n for n in declared_functions() if n in rb.EXPORTS]
    assert set(declared_functions()) <= set(rb.EXPORTS) | {"rb_config_default"}


def test_config_defaults(lib):
    from paper_1807_11866_gb300 import rb
    c = rb.rb_config_default()
    assert c.precision == rb.RB_PREC_FP64
    assert c.tol_update == 1e-10 and c.max_iter == 50


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the C sizes (LP64)."""
    import ctypes
    from paper_1807_11866_gb300 import rb
    assert ctypes.sizeof(rb.rb_query_info) == 32
    assert ctypes.sizeof(rb.rb_operators) == 7 * 4 + 4 + 7 * 8
    assert rb.INFO_DTYPE.itemsize == 32


def test_struct_layouts_match_c_compiler(tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's for include/rb.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_1807_11866_gb300 import rb
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"rb_config": rb.rb_config, "rb_operators": rb.rb_operators,
               "rb_query_info": rb.rb_query_info, "rb_csr": rb.rb_csr,
               "rb_trilinear_term": rb.rb_trilinear_term}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
