"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/bspl.h declares (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2504_11498_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(bspl_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("bspl_decompose", "bspl_project_curves", "bspl_invert_curves", "bspl_project_surfaces",
              "bspl_invert_surfaces", "bspl_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(bspl_\w+)", out))
    missing = declared_functions() - exported
    assert not missing, missing


def test_library_loads_and_answers_host_queries(libpath):
    from paper_2504_11498_gb300 import bspl
    L = bspl.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    assert L.bspl_status_string(bspl.ENOSPACE).decode() == "BSPL_ENOSPACE"
    assert bspl.workspace_bytes(bspl.OP_QUERY_CURVES, 4096, 100000, 0, 2_000_000) > 8_000_000
    assert bspl.workspace_bytes(bspl.OP_DECOMPOSE_CURVES, 4096, 150000, 0, 0) > 150000 * 8
    assert bspl.workspace_bytes(99, 1, 1, 1, 1) == 0


def test_binding_struct_layout_matches_header(libpath):
    """Struct sizes and constants the binding uses equal the C compiler's."""
    import ctypes as C

    from paper_2504_11498_gb300 import bspl
    code = r'''
#include <stdio.h>
#include "bspl.h"
int main(void){printf("%zu %zu %zu %zu %d %d %d\n", sizeof(bspl_curves), sizeof(bspl_surfaces),
 sizeof(bspl_segments), sizeof(bspl_options), BSPL_OP_REFINE_CURVES, BSPL_REFINE_EVALS, BSPL_NCOUNTERS);
 return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "s.c")
        open(src, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include", src, "-o", exe],
                       check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [C.sizeof(bspl.bspl_curves), C.sizeof(bspl.bspl_surfaces), C.sizeof(bspl.bspl_segments),
                     C.sizeof(bspl.bspl_options), bspl.OP_REFINE_CURVES, bspl.REFINE_EVALS, bspl.NCOUNTERS]


def test_product_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2504_11498_gb300 import bspl
    monkeypatch.setattr(bspl, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bspl, "_lib", None)
    with pytest.raises(bspl.BsplError):
        bspl.lib()


def test_misaligned_workspace_refused_before_any_launch(libpath):
    """A workspace that does not start on a 256-byte boundary is refused
    with EINVAL by every entry point that takes one, before any use of the
    device (so this runs without a GPU)."""
    import ctypes as C

    from paper_2504_11498_gb300 import bspl
    L = bspl.lib()
    bad = C.c_void_p(0x100010)
    segs, curves, total = bspl.bspl_segments(), bspl.bspl_curves(), C.c_int64()
    one = C.c_void_p(0x100000)  # never dereferenced: the check comes first
    assert L.bspl_decompose(0, C.byref(curves), 1e-6, C.byref(segs), C.byref(total), bad, 1 << 20,
                            None) == bspl.EINVAL
    for fn in (L.bspl_project_curves, L.bspl_invert_curves, L.bspl_project_surfaces, L.bspl_invert_surfaces):
        assert fn(C.byref(segs), 1, one, one, None, one, one, one, bad, 1 << 20, None) == bspl.EINVAL
    assert L.bspl_refine_curves(C.byref(curves), None, 0, 1, one, one, 0, one, one, one, None, bad, 1 << 20,
                                None) == bspl.EINVAL
