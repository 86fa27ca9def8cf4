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


def test_execute_plans_against_solution_mappings(orc):
    """Whole plans (star, chain, union, filter, project) on small graphs equal
    the solution-mapping enumeration of the same graph pattern."""
    from paper_1807_01409_gb300.synth import Pattern
    X, Y, Z = 0, 1, 2
    S, P, O = pins.tiny_graph(31, 40, ids=6)
    star = [{"op": "match", "pattern": Pattern(0, 2, 0, var=(X, -1, Y))},
            {"op": "match", "pattern": Pattern(0, 3, 0, var=(X, -1, Z))},
            {"op": "join", "inputs": [0, 1]}]
    r = orc.execute(S, P, O, star)
    want = pins.solutions(S, P, O, [((0, 2, 0), (X, -1, Y)), ((0, 3, 0), (X, -1, Z))], r.vars)
    assert r.rows.tolist() == [list(w) for w in want]
    chain = [{"op": "match", "pattern": Pattern(0, 0, 0, var=(X, -1, Y))},
             {"op": "match", "pattern": Pattern(0, 4, 0, var=(Y, -1, Z))},
             {"op": "join", "inputs": [0, 1]},
             {"op": "project", "input": 2, "vars": [X, Z]}]
    r = orc.execute(S, P, O, chain)
    want = pins.solutions(S, P, O, [((0, 0, 0), (X, -1, Y)), ((0, 4, 0), (Y, -1, Z))], (X, Z))
    assert r.rows.tolist() == [list(w) for w in want]
    # FILTER (?Y in [2, 4]) over the chain's first pattern
    flt = [{"op": "match", "pattern": Pattern(0, 0, 0, var=(X, -1, Y))},
           {"op": "filter", "input": 0, "var": Y, "cmp": "range", "a": 2, "b": 4}]
    r = orc.execute(S, P, O, flt)
    want = [w for w in pins.solutions(S, P, O, [((0, 0, 0), (X, -1, Y))], (X, Y)) if 2 <= w[1] <= 4]
    assert r.rows.tolist() == [list(w) for w in want]
    # UNION of two branches with different variables
    un = [{"op": "match", "pattern": Pattern(1, 0, 0, var=(-1, X, Y))},
          {"op": "match", "pattern": Pattern(0, 2, 0, var=(Y, -1, Z))},
          {"op": "union", "inputs": [0, 1]}]
    r = orc.execute(S, P, O, un)
    a = pins.solutions(S, P, O, [((1, 0, 0), (-1, X, Y))], (X, Y))
    b = pins.solutions(S, P, O, [((0, 2, 0), (Y, -1, Z))], (Y, Z))
    want = sorted({(x, y, 0) for x, y in a} | {(0, y, z) for y, z in b})
    assert r.vars == (X, Y, Z) and r.rows.tolist() == [list(w) for w in want]


# planted mistakes in the Python layer (oracle.py): rule evaluator and left join
ENTAIL_MUTATIONS = [
    ("keys = np.unique(t1.rows[:, t1.vars.index(on)])", "keys = np.unique(t1.rows[:, 0])"),  # wrong column
    ("idx2 = cand[np.isin(col[cand], keys)] if cand.shape[0] else cand", "idx2 = cand"),  # no key restriction
    ('slot = r["data"].index(r["on"])', "slot = 0"),                                         # wrong join slot
    ('for t in r["then"]:', 'for t in reversed(r["then"]):'),                                # conclusion reversed
    ("if not (all(l[i] != 0", "if (all(l[i] != 0"),                  # left join: pads the matched rows
    ("pad = [l + [0] * len(rrest)", "pad = [l + [1] * len(rrest)"),   # left join: wrong padding
]


@pytest.mark.parametrize("mut", range(len(ENTAIL_MUTATIONS)))
def test_entail_pins_catch_planted_mistake(orc, mut, tmp_path):
    import importlib.util
    old, new = ENTAIL_MUTATIONS[mut]
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
    for pin in (pins.pin_entail_golden, pins.pin_entail_bruteforce, pins.pin_left_join_rowwise):
        try:
            pin(mod)
        except Exception:
            failed.append(pin.__name__)
    assert failed, f"no pin caught entailment mutation {mut}: {new!r}"
