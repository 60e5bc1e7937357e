"""The oracle and the CUDA path share no code: the package imports neither
`oracle` nor `synth`, the oracle imports only numpy, the standard library and
itself, `synth` (the seeded input generators both sides use) imports neither,
and no CUDA or C source includes anything outside the package and
include/.  Static checks on the source text; no GPU."""
import ast
import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STDLIB = set(sys.stdlib_module_names)


def _imports(path):
    """Top-level module names imported by a Python file (relative imports as '.')."""
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add("." if node.level else node.module.split(".")[0])
    return mods


def _files(d):
    return sorted(glob.glob(os.path.join(ROOT, d, "*.py")))


def test_package_imports_neither_oracle_nor_synth():
    files = _files("paper_2103_05034_gb300")
    assert files
    for f in files:
        bad = _imports(f) & {"oracle", "synth", "bench", "tests"}
        assert not bad, (f, bad)


def test_oracle_imports_only_numpy_stdlib_and_itself():
    files = _files("oracle")
    assert files
    for f in files:
        extra = {m for m in _imports(f) if m not in STDLIB and m not in (".", "numpy", "__future__")}
        assert not extra, (f, extra)


def test_synth_imports_neither_side():
    for f in _files("synth"):
        bad = _imports(f) & {"oracle", "paper_2103_05034_gb300"}
        assert not bad, (f, bad)


def test_native_sources_include_only_package_and_system_headers():
    srcs = glob.glob(os.path.join(ROOT, "paper_2103_05034_gb300", "csrc", "*.cu*"))
    assert srcs
    own = {os.path.basename(p) for p in srcs} | {"dwfmg.h"}
    for s in srcs:
        for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', open(s).read(), flags=re.M):
            assert os.path.basename(inc) in own and "oracle" not in inc, (s, inc)
