"""The C ABI without a GPU: the library loads, exports every entry point the
headers declare, and rejects bad arguments before touching CUDA."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import paper_1710_07193_gb300 as lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(dctf_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def so():
    if not os.path.exists(lib.lib_path()):
        from paper_1710_07193_gb300 import _build
        _build.build()
    return lib.load()


def test_every_declared_symbol_is_exported(so):
    names = declared_symbols()
    assert "dctf_apply" in names and "dctf_build_operator" in names
    for n in sorted(names):
        assert hasattr(so, n), n
    assert names == set(lib.exported_symbols())


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_headers_compile_standalone(lang, tmp_path):
    """Each public header compiles on its own, first in its translation unit,
    as C and as C++ (no CUDA headers needed)."""
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
        src.write_text('#include "%s"\nint main(void) { return 0; }\n' % os.path.basename(h))
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                            str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_version(so):
    assert lib.version() >= 400      # 0.4: per-plane output tables, staged_only, admission stats


def build(mask, mh, mw, anchor, n, boundary):
    m = np.ascontiguousarray(mask, dtype=np.float64)
    a = (ctypes.c_int * 2)(*anchor)
    h = ctypes.c_void_p(0)
    st = lib.load().dctf_build_operator(m.ctypes.data, mh, mw, ctypes.addressof(a), n, boundary,
                                        None, ctypes.addressof(h))
    return st, h.value


@pytest.mark.parametrize("case", [
    dict(mh=3, mw=3, anchor=(1, 1), n=6, boundary=0),      # bad n
    dict(mh=9, mw=3, anchor=(1, 1), n=8, boundary=0),      # mask taller than block
    dict(mh=3, mw=3, anchor=(3, 1), n=8, boundary=0),      # anchor outside mask
    dict(mh=3, mw=3, anchor=(1, -1), n=8, boundary=0),
    dict(mh=3, mw=3, anchor=(1, 1), n=8, boundary=2),      # bad boundary
    dict(mh=0, mw=3, anchor=(0, 0), n=8, boundary=0),
])
def test_build_rejects_bad_arguments(so, case):
    st, h = build(np.ones(64), case["mh"], case["mw"], case["anchor"], case["n"], case["boundary"])
    assert st == 1 and h is None          # DCTF_EINVAL, nothing allocated
    assert lib.last_error() != ""


def test_build_rejects_non_finite_mask(so):
    m = np.ones(9)
    m[4] = np.nan
    st, _ = build(m, 3, 3, (1, 1), 8, 0)
    assert st == 1 and "finite" in lib.last_error()


def test_apply_rejects_null_operator(so):
    assert so.dctf_apply(None, None, 10, None, None) == 1
    assert so.dctf_apply_f64in(None, None, 10, None, None) == 1
    assert so.dctf_apply_host(None, None, 10, None) == 1
    assert so.dctf_host_buffer_direct(None, 16) == 0
    assert so.dctf_operator_set_precision(None, 0) == 1
    so.dctf_release_operator(None)        # no-op


# C struct name -> (ctypes mirror, C field name for each ctypes field)
_STRUCTS = {
    "dctf_group_item": (lib._GroupItem, {"inp": "in"}),
    "dctf_pixel_item": (lib._PixelItem, {}),
    "dctf_server_cfg": (lib._ServerCfg, {}),
    "dctf_request": (lib._Request, {"inp": "in"}),
    "dctf_stats": (lib._Stats, {}),
}


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structs have the size and field offsets the C
    header gives them (compiled and printed by the host compiler)."""
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dctf.h"', 'int main(void) {']
    for cname, (ct, rename) in _STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in ct._fields_:
            cf = rename.get(f, f)
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, cf))
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in filter(None, got):
        cname, field, value = ln.split()
        ct = _STRUCTS[cname][0]
        want = ctypes.sizeof(ct) if field == "size" else getattr(ct, field).offset
        assert int(value) == want, (cname, field, int(value), want)
