"""The plan checks that tid_exec and the request server make before anything
runs, called through the C ABI on the CPU (tid_plan_check needs no device and
no context): valid plans pass, and each malformed one is refused with the
status tid_exec would return."""
import ctypes as C

import pytest

from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300.synth import Pattern

X, Y, Z = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1807_01409_gb300 import build
    build.build()


def _m(s, p, o, var):
    return {"op": "match", "pattern": Pattern(s, p, o, var=var)}


STAR = [_m(0, 2, 0, (X, -1, Y)), _m(0, 3, 0, (X, -1, Z)), {"op": "join", "inputs": [0, 1]}]


@pytest.mark.parametrize("plan", [
    STAR,
    STAR + [{"op": "project", "input": 2, "vars": [Z, X]}],
    [_m(0, 2, 0, (X, -1, Y)), {"op": "filter", "input": 0, "var": Y, "cmp": "range", "a": 1, "b": 9}],
    [_m(1, 0, 0, (-1, X, Y)), _m(0, 2, 0, (Y, -1, Z)), _m(0, 0, 5, (X, Y, -1)), _m(0, 0, 0, (X, -1, X)),
     {"op": "union", "inputs": [0, 1, 2, 3]}],
    *[[_m(0, 2, 0, (X, -1, Y)), _m(0, 3, 0, (Y, -1, Z)), {"op": "join", "inputs": [0, 1], "algo": a}]
      for a in ("auto", "sort_merge", "hash", "left", "right", "full", tb.TID_JOIN_LEFT | tb.JOIN["sort_merge"])],
])
def test_valid_plans_pass(plan):
    assert tb.tid_plan_check(plan) == tb.TID_OK, tb.last_error()


def _nodes(n):
    return (tb.tid_plan_node * n)()


def test_malformed_plans_are_refused():
    cases = []
    cases.append(("empty", _nodes(0), tb.TID_ERR_ARG))
    fwd = tb.plan_nodes(STAR)
    fwd[2].in_[1] = 2  # reads itself
    cases.append(("input not earlier", fwd, tb.TID_ERR_ARG))
    neg = tb.plan_nodes(STAR)
    neg[2].in_[0] = -1
    cases.append(("negative input", neg, tb.TID_ERR_ARG))
    badop = tb.plan_nodes(STAR)
    badop[1].op = 9
    cases.append(("unknown op", badop, tb.TID_ERR_ARG))
    arity = tb.plan_nodes(STAR)
    arity[2].n_in = 1
    cases.append(("join with one input", arity, tb.TID_ERR_ARG))
    union5 = tb.plan_nodes([_m(0, 2, 0, (X, -1, Y))] * 2 + [{"op": "union", "inputs": [0, 1]}])
    union5[2].n_in = 5
    cases.append(("union of five", union5, tb.TID_ERR_ARG))
    for algo in (3, 0x400, tb.TID_JOIN_RIGHT | tb.JOIN["hash"], tb.TID_JOIN_LEFT | tb.JOIN["hash"]):
        j = tb.plan_nodes(STAR)
        j[2].algo = algo
        cases.append((f"join algo {algo:#x}", j, tb.TID_ERR_ARG))
    cases.append(("negative ID", tb.plan_nodes([_m(0, -2, 0, (X, -1, Y))]), tb.TID_ERR_ID))
    cases.append(("variable on a bound slot", tb.plan_nodes([_m(0, 2, 0, (X, Y, -1))]), tb.TID_ERR_ARG))
    cases.append(("no variable", tb.plan_nodes([_m(0, 2, 0, (-1, -1, -1))]), tb.TID_ERR_ARG))
    for name, nodes, want in cases:
        got = int(tb.lib().tid_plan_check(nodes if len(nodes) else None, len(nodes)))
        assert got == want, (name, got, tb.last_error())
        assert tb.last_error(), name  # the refusal says why


def test_null_plan_with_nodes_is_refused():
    assert int(tb.lib().tid_plan_check(None, 3)) == tb.TID_ERR_ARG
