"""The C-ABI library builds, loads and exports every symbol of include/ftq.h;
argument errors are reported without touching a GPU."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as ftq
    return ftq.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ftq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ftq_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["ftq_init_ueg", "ftq_propagate_slices", "ftq_stabilise", "ftq_green", "ftq_estimators",
              "ftq_destroy", "ftq_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_argument_errors_without_gpu(lib):
    from paper_2012_12228_gb300.binding import Opts
    h = ctypes.c_void_p()
    o = Opts(4, 5, 6, 0, 0, 0, 0, None, 0.0)
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 8, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert b"closed-shell" in lib.ftq_last_error(None)
    assert lib.ftq_init_ueg(ctypes.byref(h), 3, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 7, -1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    o.exp_order = 0
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    o.exp_order = 6
    o.overlap = 2
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert b"overlap" in lib.ftq_last_error(None)
    o.overlap = 0
    o.force_bias_cap = 0.5
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert b"force_bias_cap" in lib.ftq_last_error(None)
    o.force_bias_cap = 0.0
    o.walkers = 0
    assert lib.ftq_init_ueg(ctypes.byref(h), 2, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert lib.ftq_init_ueg(None, 2, 7, 1.0, 0.5, math.nan, 0.05, ctypes.byref(o)) == -1
    assert lib.ftq_set_wait_limit(None, 0) == -1
    assert lib.ftq_set_green_kernel(None, 1) == -1
    lib.ftq_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2012_12228_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of ftq_opts and ftq_system have the C layout: sizes
    and every field offset, from a small C program compiled against
    include/ftq.h."""
    import shutil
    import subprocess
    from paper_2012_12228_gb300.binding import Opts, System
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ftq.h"', "int main(void) {"]
    for cname, cls in (("ftq_opts", Opts), ("ftq_system", System)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, str(prog), "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, cls in (("ftq_opts", Opts), ("ftq_system", System)):
        assert got[(cname, "size")] == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
