"""Pins of the oracle's index-tree handling (Sec. 3, Sec. 5 ordering)."""
import os

import pytest

import workloads as W
from oracle.tree import Tree

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _set(t, v):
    nd = t.node(v)
    return "{" + ",".join(str(m + 1) for m in range(nd.lo, nd.hi)) + "}"


def test_toy_tree_levels_and_lex_order():
    p, l, idn = W.toy_tree()
    t = Tree(p, l, [3] * 6, [2] * len(p), [1] * len(p), idn)
    got = [(t.node(v).level, _set(t, v)) for v in t.lex]
    assert got == [(0, "{1,2,3,4,5,6}"), (1, "{1,2,3}"), (1, "{4}"), (1, "{5,6}"),
                   (2, "{1,2}"), (2, "{3}"), (2, "{5}"), (2, "{6}"), (3, "{1}"), (3, "{2}")]
    assert t.depth == 3


def test_sttnn_reuse_sets_match_paper_figure():
    p, l, idn = W.toy_tree()
    t = Tree(p, l, [3] * 6, [2] * len(p), [1] * len(p), idn)
    rows = [x.split(":") for x in open(os.path.join(GOLD, "sttnn_reuse_toy.txt"))
            if x.strip() and not x.startswith("#")]
    want = {a.strip(): b.split() for a, b in rows}
    for v in t.nonroot():
        S = [_set(t, s) for s in t.sttnn_reuse(v)]
        w = want[_set(t, v)]
        assert S == ([] if w == ["-"] else w)


def test_clipping_and_identity():
    p, l, idn = W.balanced_binary(3)          # root -> {0,1}, {2}; {0,1} -> {0}, {1}
    t = Tree(p, l, [4, 5, 3], [0, 7, 3, 9, 2], [0, 9, 0, 9, 1])
    by = {(t.node(v).lo, t.node(v).hi): t.node(v) for v in range(5)}
    assert (by[0, 2].r, by[0, 2].p) == (3, 9)          # r <= n_C = 3, p <= n_t - r
    assert (by[0, 1].r, by[0, 1].p, by[0, 1].identity) == (3, 0, False)  # p_t <= n_t - r_t = 1, given 0
    assert by[1, 2].identity and by[1, 2].r == 5        # leaf with r >= n: identity
    assert (by[2, 3].r, by[2, 3].p) == (2, 1)


@pytest.mark.parametrize("parent,leaf_modes,msg", [
    ([-1, 0, 0], [[], [0, 2], [1]], "contiguous"),
    ([-1, 0, 0], [[], [0], [0]], "contiguous|partition"),
    ([-1, 0], [[], [0, 1]], ">= 2 children"),
    ([-1, 0, 0], [[], [0], []], "leaf without modes"),
    ([-1, -1, 0], [[], [0], [1]], "one root"),
    ([-1, 0, 0, 0], [[], [0], [2], [1]], None),
])
def test_validation(parent, leaf_modes, msg):
    d = 3 if len(parent) == 4 else 2
    if msg is None:
        t = Tree(parent, leaf_modes, [2] * d, [1] * len(parent), [0] * len(parent))
        assert [t.node(c).lo for c in t.node(t.root).children] == [0, 1, 2]
        return
    with pytest.raises(ValueError, match=msg):
        Tree(parent, leaf_modes, [2] * 3, [1] * len(parent), [0] * len(parent))
