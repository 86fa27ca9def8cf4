"""The CPU oracle against its pins (no GPU), and planted mistakes in the
oracle's C source that the pins must catch."""
import os
import subprocess

import numpy as np
import pytest

import pins

ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "oracle", "oracle.c")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


# (what the source says, a plausible mistake)
MUTATIONS = [
    ("if (kp != 0 && p != kp) return 0;", "if (kp != 0 && o != kp) return 0;"),   # transposed operand
    ("if (ko != 0 && o != ko) return 0;", ""),                                      # dropped term
    ("if (ks != 0 && s != ks) return 0;", "if (ks != 0 && s == ks) return 0;"),    # wrong sign
    ("if (out) out[h] = (int32_t)i;", "if (out) out[h] = (int32_t)(i + 1);"),       # off-by-one index
    ("else if (row[c] != term[j]) ok = 0;", ""),                                    # repeated var unchecked
    ("if (x == 0 || x != r[rkey[c]]) return 0;", "if (x != r[rkey[c]]) return 0;"),  # unbound joins
    ("for (int c = 0; c < nrest; ++c) o[kl + c] = r[rrest[c]];",
     "for (int c = 0; c < nrest; ++c) o[kl + c] = r[rrest[0]];"),                   # wrong column
    ("if (x < y) return -1;\n        if (x > y) return 1;\n    }\n    return 0;\n}\n\nstatic int sort_perm",
     "if (x > y) return -1;\n        if (x < y) return 1;\n    }\n    return 0;\n}\n\nstatic int sort_perm"),  # reversed order
    ("case 3: keep = x <= a; break;", "case 3: keep = x < a; break;"),              # LE as LT
    ("case 6: keep = a <= x && x <= b; break;", "case 6: keep = a <= x && x < b; break;"),  # open range
    ("if (m > 0 && row_cmp(tmp + (m - 1) * k, r, cols, k) == 0) continue;", ""),   # no dedupe
    ("if (outs) outs[j][counts[j]] = (int32_t)i;\n                counts[j]++;",
     "if (outs) outs[j][counts[j]] = (int32_t)i;\n                counts[j]++;\n                break;"),  # first key only
    ("keys[3 * j + 1], keys[3 * j + 2])", "keys[3 * j + 2], keys[3 * j + 1])"),     # multi: p and o keys swapped
    ("int32_t term[3] = {S[i], P[i], O[i]};", "int32_t term[3] = {S[i], O[i], P[i]};"),  # bind: p and o slots swapped
    ("int32_t x = a[cols[c]], y = b[cols[c]];",
     "uint32_t x = (uint32_t)a[cols[c]], y = (uint32_t)b[cols[c]];"),              # unsigned row order
    ("if (has_zero_key(l, nk, lkey)) { ++a; continue; }\n        if (has_zero_key(r, nk, rkey)) { ++b; continue; }",
     ""),                                                                           # sort-merge: unbound keys join
    ("while (b2 < nr && key_cmp(l, lkey, R + pr[b2] * kr, rkey, nk) == 0) ++b2;", ""),  # sort-merge: right group of one
    ("while (a2 < nl && key_cmp(L + pl[a2] * kl, lkey, r, rkey, nk) == 0) ++a2;", ""),  # sort-merge: left group of one
    ("case 1: keep = x != a; break;", "case 1: keep = x == a; break;"),            # NE as EQ
    ("case 4: keep = x > a; break;", "case 4: keep = x >= a; break;"),             # GT as GE
    ("if (x == 0) keep = 0;\n        else switch (op) {", "switch (op) {"),         # unbound rows pass filters
]


@pytest.mark.parametrize("mut", range(len(MUTATIONS)))
def test_pins_catch_planted_mistake(orc, mut, tmp_path):
    old, new = MUTATIONS[mut]
    src = open(ORACLE_C).read()
    assert old in src, "mutation site vanished from oracle.c"
    bad = tmp_path / "oracle_mut.c"
    bad.write_text(src.replace(old, new, 1))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(bad)])
    failed = []
    with orc.using_library(str(so)):
        for pin in pins.ALL_PINS:
            try:
                pin(orc)
            except Exception:  # a pin that fails or breaks on the mutant has caught it
                failed.append(pin.__name__)
    assert failed, f"no pin caught mutation {mut}: {new!r}"


def test_sortmerge_equals_nested_on_random_sets(orc):
    rng = np.random.default_rng(21)
    for _ in range(40):
        L = orc.TupleSet((0, 1, 2), orc.canonical(rng.integers(0, 6, (int(rng.integers(0, 60)), 3))))
        R = orc.TupleSet((2, 0, 3), orc.canonical(rng.integers(0, 6, (int(rng.integers(0, 60)), 3))))
        a = orc.join(L, R, method="nested")
        b = orc.join(L, R, method="sortmerge")
        assert a.vars == b.vars and np.array_equal(a.rows, b.rows)


# planted mistakes in the Python layer (oracle.py): schemas, union, project, plans,
# the rule evaluator and the left join
PY_MUTATIONS = [
    ("if v not in out:\n            out.append(v)", "out.append(v)"),                        # repeated var twice
    ("rrest = [j for j, v in enumerate(Rv) if v not in Lv]", "rrest = [j for j, v in enumerate(Rv)]"),  # shared kept twice
    ("a = np.zeros((t.n, len(uv)), np.int32)", "a = np.ones((t.n, len(uv)), np.int32)"),     # union pads with 1
    ("a[:, uv.index(v)] = t.rows[:, j]", "a[:, j] = t.rows[:, j]"),                          # union ignores schema
    ("cols = [t.vars.index(v) for v in vars_]", "cols = sorted(t.vars.index(v) for v in vars_)"),  # project order
    ('r = filter(ev(nd["input"]), nd["var"], nd["cmp"], nd["a"], nd.get("b", 0))',
     'r = ev(nd["input"])'),                                                                 # plan drops FILTER
    ('r = union([ev(j) for j in nd["inputs"]])', 'r = union([ev(nd["inputs"][0])])'),        # plan: first branch only
    ("keys = np.unique(t1.rows[:, t1.vars.index(on)])", "keys = np.unique(t1.rows[:, 0])"),  # wrong column
    ("idx2 = cand[np.isin(col[cand], keys)] if cand.shape[0] else cand", "idx2 = cand"),  # no key restriction
    ('slot = r["data"].index(r["on"])', "slot = 0"),                                         # wrong join slot
    ('for t in r["then"]:', 'for t in reversed(r["then"]):'),                                # conclusion reversed
    ("if not (all(l[i] != 0", "if (all(l[i] != 0"),                  # left join: pads the matched rows
    ("pad = [l + [0] * len(rrest)", "pad = [l + [1] * len(rrest)"),   # left join: wrong padding
    ("if all(x != 0 for x in key) and key in lkeys:",
     "if key in lkeys or not all(x != 0 for x in key):"),                      # outer: unbound right rows dropped
    ("pad.append([r[Rs.vars.index(v)] if v in Rs.vars else 0 for v in out_vars])",
     "pad.append([r[Rs.vars.index(v)] if v in Rs.vars else 1 for v in out_vars])"),  # right: wrong padding
    ("return _set(left.vars, np.concatenate([left.rows, _unmatched_right(Ls, Rs)], axis=0))",
     "return left"),                                                                   # full: right rows lost
    ('"right": right_join, "full": full_join}', '"right": left_join, "full": full_join}'),  # plan: right as left
    ("    return _set(vars_, out[:r])", "    return TupleSet(vars_, out[:r].copy())"),          # bind keeps duplicates
    ("rkey = [Rv.index(v) for v in shared]", "rkey = [Lv.index(v) for v in shared]"),         # join: key from wrong side
    ("out_vars = tuple(Lv) + tuple(Rv[j] for j in rrest)",
     "out_vars = tuple(Rv[j] for j in rrest) + tuple(Lv)"),                                  # join: schema order swapped
    ("    for t in sets:\n        for v in t.vars:", "    for t in reversed(sets):\n        for v in t.vars:"),  # union schema order
]


@pytest.mark.parametrize("mut", range(len(PY_MUTATIONS)))
def test_python_layer_pins_catch_planted_mistake(orc, mut, tmp_path):
    import importlib.util
    old, new = PY_MUTATIONS[mut]
    src = open(orc.__file__).read()
    assert old in src, "mutation site vanished from oracle.py"
    bad = tmp_path / "oracle_entail_mut.py"
    bad.write_text(src.replace(old, new, 1))
    import sys
    spec = importlib.util.spec_from_file_location("oracle_entail_mut", bad)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle_entail_mut"] = mod
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.modules.pop("oracle_entail_mut", None)
    mod._SRC, mod._BUILD, mod._SO, mod._lib = orc._SRC, orc._BUILD, orc._SO, None
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(mod)
        except Exception:
            failed.append(pin.__name__)
    assert failed, f"no pin caught Python-layer mutation {mut}: {new!r}"
