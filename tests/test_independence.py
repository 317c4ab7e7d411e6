"""The product path has no CPU fallback and shares nothing with the oracle.

* The binding refuses to work without the built CUDA library (ImportError),
  rather than computing anything on the host.
* No source of the package (Python, CUDA, headers) names the oracle, and
  the oracle names nothing of the package: the two share no code, and only
  the seeded input generators (`workloads`) serve both.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1604_06667_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "__pycache__" in d or os.sep + "_build" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_binding_raises_without_library(tmp_path):
    from paper_1604_06667_gb300 import _capi
    saved = _capi._lib
    try:
        _capi._lib = None
        with pytest.raises(ImportError):
            _capi.load(str(tmp_path / "libcygrid_gb300.so"))
    finally:
        _capi._lib = saved


def test_package_does_not_touch_the_oracle():
    pat = re.compile(r"\boracle\b|cg_oracle")
    hits = []
    for p in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
        src = open(p, encoding="utf-8").read()
        for line in src.splitlines():
            if pat.search(line):
                hits.append("%s: %s" % (os.path.relpath(p, ROOT), line.strip()))
    assert not hits, hits


def test_oracle_does_not_touch_the_package():
    pat = re.compile(r"paper_1604_06667_gb300|cygrid_gb300|libcygrid")
    hits = []
    for p in _sources(ORACLE, (".py", ".c", ".h")):
        src = open(p, encoding="utf-8").read()
        for line in src.splitlines():
            if pat.search(line):
                hits.append("%s: %s" % (os.path.relpath(p, ROOT), line.strip()))
    assert not hits, hits


def test_workloads_hold_no_method_arithmetic():
    """The shared input generators import neither side."""
    p = os.path.join(ROOT, "workloads", "__init__.py")
    src = open(p, encoding="utf-8").read()
    assert not re.search(r"^\s*(from|import)\s+(oracle|paper_1604_06667_gb300)\b", src, re.M)
