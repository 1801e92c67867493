"""The CUDA path and the oracle share no code: the package neither imports the oracle nor includes its
sources, the oracle neither imports the package nor includes the library's headers, and the benchmark
calls the oracle only in its CPU-baseline leg and its reference arm. Without the CUDA library the product
path raises instead of falling back to anything else."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1507_08549_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "_lib", "__pycache__"))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_package_does_not_reach_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s+[\"<][^\">]*oracle)", re.M)
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h")):
        assert not pat.search(open(path).read()), path


def test_oracle_does_not_reach_the_package():
    pat = re.compile(r"^\s*(import\s+paper_1507_08549_gb300|from\s+paper_1507_08549_gb300|"
                     r"#\s*include\s+[\"<][^\">]*(hydro\.h|csrc|\.cuh))", re.M)
    for path in _sources(ORACLE, (".py", ".c", ".h", ".inc")):
        assert not pat.search(open(path).read()), path


def test_benchmark_imports_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"cpu_baseline", "run_reference"}
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef):
            for sub in ast.walk(node):
                if isinstance(sub, (ast.Import, ast.ImportFrom)):
                    names = [a.name for a in sub.names] + ([sub.module] if isinstance(sub, ast.ImportFrom) else [])
                    if any(n and n.split(".")[0] == "oracle" for n in names):
                        assert node.name in allowed, node.name
    for sub in tree.body:  # nothing at module level
        if isinstance(sub, (ast.Import, ast.ImportFrom)):
            assert all(a.name.split(".")[0] != "oracle" for a in sub.names)
            assert not (isinstance(sub, ast.ImportFrom) and (sub.module or "").startswith("oracle"))


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_1507_08549_gb300 import build, hydro

    def no_build():
        raise RuntimeError("nvcc unavailable")

    monkeypatch.setattr(hydro, "_lib", None)
    monkeypatch.setattr(build, "build", no_build)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(hydro.HydroError) as e:
        hydro.load()
    assert e.value.code == hydro.ECUDA
