"""The C-ABI library builds, loads and exports every function that
include/*.h declares; argument validation answers without touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ccw_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2404_00441_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["ccw_ti_prepare", "ccw_simulate", "ccw_ccf_search", "ccw_idwt_paste",
              "ccw_ti_free", "ccw_last_error"]:
        assert n in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_validation_errors_without_gpu(lib):
    lib.ccw_last_error.restype = C.c_char_p
    out = C.c_void_p()
    dims = (C.c_int32 * 3)(64, 64, 1)
    fake = C.c_void_p(1)            # never dereferenced: validation fails first
    # ndim out of range
    assert lib.ccw_ti_prepare(fake, 5, dims, 2, 1, 8, 2, None, C.byref(out)) == -1
    assert b"ndim" in lib.ccw_last_error()
    # template not a multiple of 2^level
    assert lib.ccw_ti_prepare(fake, 2, dims, 2, 2, 10, 4, None, C.byref(out)) == -1
    # template < 2 x overlap
    assert lib.ccw_ti_prepare(fake, 2, dims, 2, 1, 16, 10, None, C.byref(out)) == -1
    # too many facies
    assert lib.ccw_ti_prepare(fake, 2, dims, 9, 1, 16, 4, None, C.byref(out)) == -1
    # template larger than the TI
    small = (C.c_int32 * 3)(10, 64, 1)
    assert lib.ccw_ti_prepare(fake, 2, small, 2, 1, 16, 4, None, C.byref(out)) == -1
    assert b"template" in lib.ccw_last_error()
    # score range beyond the exact FP32 bound: F=8, J=4, T=256
    big = (C.c_int32 * 3)(4096, 4096, 1)
    assert lib.ccw_ti_prepare(fake, 2, big, 8, 4, 256, 64, None, C.byref(out)) == -1
    assert b"2^24" in lib.ccw_last_error()
    # NULL handles
    assert lib.ccw_simulate(None, None, None, None, 0, C.c_uint64(0), None, None, None) == -1
    assert lib.ccw_ti_free(None) is None or True


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    that a C compiler gives the header's structs (gcc on this host)."""
    import subprocess
    from paper_2404_00441_gb300 import ccw as binding
    pairs = [("ccw_params", binding._Params), ("ccw_group", binding._Group),
             ("ccw_ti_desc", binding._Desc)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ccw.h"', 'int main(void) {']
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                           str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
