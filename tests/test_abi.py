"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/*.h declares; the product code never reaches the oracle."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(tid_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1807_01409_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    d = _declared()
    for must in ("tid_load", "tid_match", "tid_ctx_create", "tid_set_to_host"):
        assert must in d


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tid_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_and_binds(libpath):
    from paper_1807_01409_gb300 import binding
    L = binding.lib()
    for n in _declared():
        assert hasattr(L, n)
    assert binding.last_error() == ""


def test_built_for_sm103a_only():
    """Every compile and the link name one target, sm_103a; no other GPU code is
    built (the flags are checked rather than the binary)."""
    from paper_1807_01409_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    flags = " ".join(build.NVCC_FLAGS)
    assert "-arch" not in flags and "-gencode" not in flags and "sm_" not in flags


def test_product_never_imports_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|liboracle|oracle\.c\b|or_match|or_join", re.M)
    for f in glob.glob(os.path.join(ROOT, "paper_1807_01409_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            assert not pat.search(open(f).read()), f


def test_pattern_array_matches_the_c_struct():
    import ctypes
    import numpy as np
    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300.synth import Pattern
    assert tb.PATTERN_DTYPE.itemsize == ctypes.sizeof(tb.tid_pattern) == 16
    a = tb.pattern_array(np.array([[1, 2, 3], [0, 5, 0]]))
    b = tb.pattern_array([(1, 2, 3), Pattern(0, 5, 0)])
    assert a.tobytes() == b.tobytes()
    c = tb.pattern_array([Pattern(0, 5, 0, var=(0, -1, 1))])
    t = tb.tid_pattern.from_buffer_copy(c.tobytes())
    assert (t.s, t.p, t.o, tuple(t.var)) == (0, 5, 0, (0, -1, 1))
