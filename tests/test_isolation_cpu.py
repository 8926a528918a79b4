"""The oracle and the CUDA path stay apart (static checks, CPU only).

* nothing in the package (Python, CUDA, C++ or headers) imports, includes or
  names a module of ``oracle/``;
* ``oracle/`` imports nothing from the package;
* the benchmark and the entry points import the oracle only inside the
  functions that time or check against it, never at module level;
* nothing committed refers to the ignored working folder;
* the binding fails loudly when the library is missing (no fallback).
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2409_13344_gb300")
ORACLE = os.path.join(ROOT, "oracle")
SOURCE_EXT = (".py", ".cu", ".cuh", ".cpp", ".h")


def _files(top, exts):
    for dirpath, dirnames, filenames in os.walk(top):
        dirnames[:] = [d for d in dirnames if d not in ("__pycache__", "_build")]
        for fn in filenames:
            if fn.endswith(exts):
                yield os.path.join(dirpath, fn)


def test_package_never_touches_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)",
                     re.M)
    bad = [p for p in _files(PKG, SOURCE_EXT) if pat.search(open(p, encoding="utf-8").read())]
    assert not bad, bad
    for p in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(p, encoding="utf-8").read().lower(), p


def test_oracle_imports_nothing_from_the_package():
    pat = re.compile(r"^\s*(from|import)\s+paper_2409_13344_gb300\b", re.M)
    bad = [p for p in _files(ORACLE, (".py",)) if pat.search(open(p, encoding="utf-8").read())]
    assert not bad, bad


@pytest.mark.parametrize("fn", ["bench.py", "__graft_entry__.py"])
def test_oracle_imported_only_inside_functions(fn):
    text = open(os.path.join(ROOT, fn), encoding="utf-8").read()
    for m in re.finditer(r"^(\s*)(from\s+oracle\b|import\s+oracle\b)", text, re.M):
        assert m.group(1), f"{fn}: module-level oracle import"


def test_nothing_committed_refers_to_the_working_folder():
    pat = re.compile(r"\b_work\b")
    roots = [PKG, ORACLE, os.path.join(ROOT, "include"), os.path.join(ROOT, "tests")]
    files = [p for r in roots for p in _files(r, SOURCE_EXT)]
    files += [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    bad = [p for p in files
           if os.path.abspath(p) != os.path.abspath(__file__)
           and pat.search(open(p, encoding="utf-8").read())]
    assert not bad, bad


def test_binding_raises_without_the_library(tmp_path):
    from paper_2409_13344_gb300 import appga
    saved = appga._lib
    appga._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            appga.load_library(str(tmp_path / "missing" / "libappga.so"))
    finally:
        appga._lib = saved
