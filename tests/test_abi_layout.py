"""The ctypes binding agrees with include/dwfmg.h: every declared function's
parameter list (count and kind: pointer, int, int64, double) and return kind,
and the byte layout of the parameter and statistics structs as the C compiler
lays them out (a host program built with gcc prints sizeof and offsetof).
Runs without a GPU and without the library."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2103_05034_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dwfmg.h")


def _header_text():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    return re.sub(r"^\s*#.*$", " ", txt, flags=re.M)


def _c_kind(decl):
    """Kind of a C parameter or return type: ptr, int, i64, double, size."""
    d = decl.strip()
    if "*" in d or "[" in d:
        return "ptr"
    d = re.sub(r"\b(const|struct)\b", " ", d).split()
    t = d[0] if d else ""
    return {"int": "int", "int64_t": "i64", "double": "double", "size_t": "size"}.get(t, "?" + t)


def _ct_kind(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int: "int", C.c_int64: "i64", C.c_double: "double", C.c_size_t: "size"}.get(t, "?" + str(t))


def _declarations():
    """{name: (return kind, [parameter kinds])} for every function in the header."""
    txt = _header_text()
    out = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(([^()]*)\)\s*;", txt):
        ret, name, params = m.group(1), m.group(2), m.group(3).strip()
        if "typedef" in ret:
            continue
        kinds = [] if params in ("", "void") else [_c_kind(p) for p in params.split(",")]
        out[name] = (_c_kind(ret), kinds)
    return out


def test_every_signature_matches_the_header():
    decls = _declarations()
    assert set(decls) == set(_lib.header_functions())
    bad = []
    for name, (ret, params) in decls.items():
        res, args = _lib._SIGS[name]
        got = (_ct_kind(res), [_ct_kind(a) for a in args])
        if got != (ret, params):
            bad.append((name, (ret, params), got))
    assert not bad, bad


STRUCTS = [("dwf_solve_stats", _lib.SolveStats), ("dwf_mg_params", _lib.MGParams),
           ("dwf_hybrid_params", _lib.HybridParams)]


def _header_fields(struct):
    txt = _header_text()
    m = re.search(r"typedef\s+struct\s+" + struct + r"\s*\{(.*?)\}\s*" + struct + r"\s*;", txt, flags=re.S)
    assert m, struct
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if decl:
            names.append(re.match(r".*?\b([A-Za-z_][A-Za-z0-9_]*)\s*(\[\s*\d+\s*\])?$", decl, flags=re.S).group(1))
    return names


@pytest.mark.parametrize("struct,cls", STRUCTS, ids=[s for s, _ in STRUCTS])
def test_struct_field_order_matches_the_header(struct, cls):
    assert _header_fields(struct) == [f for f, _ in cls._fields_]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layout_matches_the_c_compiler(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dwfmg.h"', "int main(void) {"]
    for struct, cls in STRUCTS:
        lines.append(f'  printf("{struct} size %zu\\n", sizeof({struct}));')
        for f in _header_fields(struct):
            lines.append(f'  printf("{struct} {f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for struct, cls in STRUCTS:
        assert got[(struct, "size")] == C.sizeof(cls), struct
        for f, _ in cls._fields_:
            assert got[(struct, f)] == getattr(cls, f).offset, (struct, f)
