"""Planted-mistake harness: build a copy of the C oracle with one textual
change and run pin checks against it; a pin that still passes on the broken
copy does not pin what it claims to."""
import os
import shutil
import subprocess
import tempfile

import oracle


def with_mutated_oracle(monkeypatch, old, new, checks):
    """True if at least one check raises AssertionError on the oracle with
    `old` replaced by `new` (which must occur in the source)."""
    src = open(oracle._build.SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %r" % old
    tmp = tempfile.mkdtemp(prefix="cgmut_")
    try:
        cpath = os.path.join(tmp, "m.c")
        with open(cpath, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "libm.so")
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", so, cpath, "-lm"])
        good = oracle.lib()
        monkeypatch.setattr(oracle, "_lib", None)
        monkeypatch.setattr(oracle._build, "build", lambda force=False: so)
        caught = False
        try:
            for chk in checks:
                try:
                    chk()
                except AssertionError:
                    caught = True
                    break
        finally:
            monkeypatch.setattr(oracle, "_lib", good)
        return caught
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
