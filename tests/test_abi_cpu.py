"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/spmm.h declares, and rejects malformed input on the
host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(spmm_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02864_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spmm_create_csr", "spmm_apply", "spmm_destroy", "spmm_last_error", "spmm_get_info"):
        assert must in names


def test_every_entry_point_cites_its_passage():
    """The comment before each declaration (the nearest one above it) names
    the paper's passage the call serves (a Section or Algorithm), or says
    that the paper has no counterpart."""
    src = open(os.path.join(ROOT, "include", "spmm.h")).read()
    comments = [(m.end(), m.group(1)) for m in re.finditer(r"/\*(.*?)\*/", src, flags=re.S)]
    uncited = []
    for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(spmm_\w+)\s*\(", src, flags=re.M):
        doc = " ".join([c for end, c in comments if end <= m.start()][-1].replace("*", " ").split())
        if not re.search(r"Section|Algorithm|paper has no counterpart", doc):
            uncited.append(m.group(1))
    assert len(comments) > 20 and not uncited, uncited


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_validation_without_gpu(lib):
    from paper_1602_02864_gb300 import spmm as sp
    h = ctypes.c_void_p(0)
    rp = np.array([0, 2, 1, 3], dtype=np.int64)       # decreasing row pointer
    ci = np.array([0, 1, 2], dtype=np.int32)
    rc = lib.spmm_create_csr(ctypes.byref(h), ctypes.c_int64(3), ctypes.c_int64(3), ctypes.c_int64(3),
                             ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data), None, 0, 0, None,
                             None)
    assert rc == sp.SPMM_ERR_FORMAT and not h.value
    assert b"decreases" in sp.lib().spmm_last_error() or "decreases" in sp.spmm_last_error()
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([0, 5, 2], dtype=np.int32)           # column out of range
    rc = lib.spmm_create_csr(ctypes.byref(h), ctypes.c_int64(3), ctypes.c_int64(3), ctypes.c_int64(3),
                             ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data), None, 0, 0, None,
                             None)
    assert rc == sp.SPMM_ERR_FORMAT
    rc = lib.spmm_create_csr(None, ctypes.c_int64(3), ctypes.c_int64(3), ctypes.c_int64(3),
                             ctypes.c_void_p(rp.ctypes.data), ctypes.c_void_p(ci.ctypes.data), None, 0, 0, None,
                             None)
    assert rc == sp.SPMM_ERR_ARG
    assert lib.spmm_destroy(None) == 0


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the header's layout: a C
    program compiled against include/spmm.h prints every field's offset and
    size and each struct's size, and the binding must agree."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1602_02864_gb300 import spmm as sp
    structs = {"spmm_opts": sp.spmm_opts, "spmm_info": sp.spmm_info, "spmm_tile_desc": sp.spmm_tile_desc}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spmm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name}*)0)->{field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            parts = line.split()
            c[tuple(parts[:-2] if parts[1] != "sizeof" else parts[:2])] = tuple(int(x) for x in parts[-2:]) \
                if parts[1] != "sizeof" else int(parts[2])
    for name, cls in structs.items():
        assert c[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            f = getattr(cls, field)
            assert c[(name, field)] == (f.offset, f.size), (name, field)
