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
    assert isinstance(binding.last_error(), str)  # thread-local; "" until a call fails


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


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (size and every
    field offset, as gcc lays them out) and the binding's constants equal the
    header's macros: a mismatch would pass wrong arguments through the ABI."""
    import ctypes
    from paper_1807_01409_gb300 import binding as tb
    structs = {
        "tid_pattern": (tb.tid_pattern, ["s", "p", "o", "var", "reserved"]),
        "tid_pred": (tb.tid_pred, ["var", "op", "a", "b"]),
        "tid_plan_node": (tb.tid_plan_node, ["op", "n_in", ("in", "in_"), "pattern", "pred", "algo",
                                              "n_vars", "vars"]),
        "tid_rdfs_vocab": (tb.tid_rdfs_vocab, ["type", "domain", "range", "sub_property_of", "sub_class_of"]),
        "tid_entail_stats": (tb.tid_entail_stats, ["res1", "dist1", "res2", "dist2", "all"]),
        "tid_server_config": (tb.tid_server_config, ["workers", "max_wave", "batch_scans", "reserved",
                                                      "budget_bytes"]),
        "tid_server_stats": (tb.tid_server_stats, ["submitted", "completed", "failed", "waves",
                                                    "max_wave_seen", "peak_admitted_bytes", "scan_patterns",
                                                    "budget_waits"]),
    }
    consts = {
        "TID_OK": tb.TID_OK, "TID_ERR_ARG": tb.TID_ERR_ARG, "TID_ERR_ID": tb.TID_ERR_ID,
        "TID_ERR_OOM": tb.TID_ERR_OOM, "TID_ERR_CAPACITY": tb.TID_ERR_CAPACITY,
        "TID_ERR_TIMEOUT": tb.TID_ERR_TIMEOUT, "TID_ERR_CUDA": tb.TID_ERR_CUDA,
        "TID_HOST": tb.TID_HOST, "TID_DEVICE": tb.TID_DEVICE, "TID_MAX_COLS": tb.TID_MAX_COLS,
        "TID_MAX_MULTI": tb.TID_MAX_MULTI, "TID_BATCH_KEYS": tb.TID_BATCH_KEYS,
        **{f"TID_BATCH_{v.upper()}": k for k, v in tb.BATCH_SHAPES.items()},
        "TID_REQ_INDEX": tb.TID_REQ_INDEX, "TID_REQ_PLAN": tb.TID_REQ_PLAN,
        "TID_JOIN_AUTO": tb.JOIN["auto"], "TID_JOIN_SORT_MERGE": tb.JOIN["sort_merge"],
        "TID_JOIN_HASH": tb.JOIN["hash"], "TID_JOIN_LEFT": tb.TID_JOIN_LEFT,
        "TID_JOIN_RIGHT": tb.TID_JOIN_RIGHT, "TID_JOIN_FULL": tb.TID_JOIN_FULL,
        **{f"TID_CMP_{k.upper()}": v for k, v in tb.CMP.items()},
        **{f"TID_OP_{k.upper()}": v for k, v in tb.OP.items()},
        **{f"TID_RULE_R{r}": r for r in tb.RULES},
    }
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tid.h"', "int main(void) {"]
    for name, (_, fields) in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            c = f[0] if isinstance(f, tuple) else f
            lines.append(f'printf("{name} {c} %zu\\n", offsetof({name}, {c}));')
    for m in consts:
        lines.append(f'printf("#{m} %lld\\n", (long long)({m}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    layout, macro = {}, {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        f = line.split()
        if f[0].startswith("#"):
            macro[f[0][1:]] = int(f[1])
        else:
            layout[(f[0], f[1])] = int(f[2])
    for name, (cls, fields) in structs.items():
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for f in fields:
            c, py = (f if isinstance(f, tuple) else (f, f))
            assert getattr(cls, py).offset == layout[(name, c)], (name, c)
    assert macro == consts


def test_binding_checks_sizes_before_calling():
    """Sizes the library must trust are checked in the binding: a length or a
    capacity beyond an argument's own length, or a wrong integer width, raises
    before anything reaches the device (no GPU needed here)."""
    import numpy as np
    from paper_1807_01409_gb300 import binding as tb
    a = np.ones(8, np.int32)
    with pytest.raises(ValueError):
        tb.tid_load(None, a, a, a, n=9)
    with pytest.raises(TypeError):
        tb.tid_load(None, a, a.astype(np.int64), a)
    out, cnt = np.zeros(8, np.int32), np.zeros(1, np.int64)
    with pytest.raises(ValueError):
        tb.tid_match_noalloc(0, None, a, a, a, (0, 1, 0), out, cnt, n=9)
    with pytest.raises(ValueError):
        tb.tid_match_noalloc(0, None, a, a, a, (0, 1, 0), out, cnt, cap=9)
    with pytest.raises(TypeError):
        tb.tid_match_noalloc(0, None, a, a, a, (0, 1, 0), out, np.zeros(1, np.int32))
    with pytest.raises(ValueError):
        tb.tid_match_noalloc(0, None, a, a, a, (0, 1, 0), out, np.zeros(0, np.int64))
