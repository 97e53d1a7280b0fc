"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/gsofa.h declares, and the ctypes structs match the C layout."""
import os
import re
import subprocess
import tempfile

import pytest

import paper_2007_00840_gb300 as gs
from paper_2007_00840_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(gsofa_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = gs.load()
    assert gs.version() >= 10000


def test_exports_every_declared_symbol():
    lib = gs.load()
    names = declared_functions()
    assert "gsofa_symbolic" in names and "gsofa_symbolic_device" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_struct_layout_matches_header():
    import ctypes
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "gsofa.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(gsofa_options), sizeof(gsofa_stats), sizeof(gsofa_result));
  printf("%zu %zu %zu %zu\n", offsetof(gsofa_options, mem_budget_bytes), offsetof(gsofa_result, L_rowptr),
         offsetof(gsofa_result, stats), offsetof(gsofa_result, _priv));
  printf("%zu %zu\n", offsetof(gsofa_stats, vertices_expanded), offsetof(gsofa_result, on_device));
  printf("%zu %zu %zu %zu\n", sizeof(gsofa_server_config), sizeof(gsofa_server_stats),
         offsetof(gsofa_server_config, opts), offsetof(gsofa_server_stats, span_s));
  printf("%zu %zu %zu %zu\n", offsetof(gsofa_options, max_ctas), offsetof(gsofa_options, team_sources),
         offsetof(gsofa_options, label_bits), offsetof(gsofa_options, schedule));
  printf("%zu\n", offsetof(gsofa_options, clean_heads));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    R, O, S = _lib.gsofa_result, _lib.gsofa_options, _lib.gsofa_stats
    assert vals[:3] == [ctypes.sizeof(O), ctypes.sizeof(S), ctypes.sizeof(R)]
    assert vals[3:7] == [O.mem_budget_bytes.offset, R.L_rowptr.offset, R.stats.offset, R._priv.offset]
    assert vals[7:9] == [S.vertices_expanded.offset, R.on_device.offset]
    C, T = _lib.gsofa_server_config, _lib.gsofa_server_stats
    assert vals[9:13] == [ctypes.sizeof(C), ctypes.sizeof(T), C.opts.offset, T.span_s.offset]
    assert vals[13:17] == [O.max_ctas.offset, O.team_sources.offset, O.label_bits.offset, O.schedule.offset]
    assert vals[17] == O.clean_heads.offset


def test_defaults_and_errors_without_gpu():
    o = gs.options()
    assert o.chunk_size == 128 and o.validate == 1 and o.fill_first == 0
    lib = gs.load()
    assert lib.gsofa_strerror(_lib.GSOFA_E_INVAL).decode().startswith("invalid")
    with pytest.raises(TypeError):
        gs.options(no_such_field=1)


def test_no_cpu_fallback_when_library_missing(tmp_path):
    # the binding refuses to run without the CUDA library instead of falling back
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
