"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute calls: these run on a machine without a GPU.
"""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mcd_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2404_17542_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert len(declared_functions()) >= 10


def test_binding_loads_and_matches_header(libpath):
    from paper_2404_17542_gb300 import mcd
    L = mcd.lib()
    assert mcd.version().startswith("mcd-gb300")
    declared = set(declared_functions())
    for name in mcd.exported_symbols():
        assert name in declared, name
        assert hasattr(L, name)


def test_binding_struct_sizes_match_c(libpath, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's layout."""
    import ctypes as C

    from paper_2404_17542_gb300 import mcd
    src = tmp_path / "sizes.c"
    src.write_text('#include "mcd.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mcd_mesh),'
                   ' sizeof(mcd_mls_params), sizeof(mcd_solve_params), sizeof(mcd_solve_info),'
                   ' sizeof(mcd_body), sizeof(mcd_flow_params), sizeof(mcd_flow_info),'
                   ' offsetof(mcd_flow_info, skipped)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    assert sizes == [C.sizeof(mcd.c_mesh), C.sizeof(mcd.c_mls_params), C.sizeof(mcd.c_solve_params),
                     C.sizeof(mcd.c_solve_info), C.sizeof(mcd.c_body), C.sizeof(mcd.c_flow_params),
                     C.sizeof(mcd.c_flow_info), mcd.c_flow_info.skipped.offset]


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2404_17542_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), path
