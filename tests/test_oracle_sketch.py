"""Pins of the oracle's sketch phase: brute-force index sums, linearity,
STTNN's two formulations, and TTN-input sketches against dense sketches."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import rounding as OR
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.quant import round_to
from oracle.tree import Tree


def _brute(T, t, drm):
    """Sketches by explicit nested sums over every tensor index (Sec. 4 sketch
    phase with the Khatri-Rao DRMs of Sec. 7 written entrywise)."""
    dims = t.dims
    idx = list(itertools.product(*[range(n) for n in dims]))
    X, Y = drm.X, drm.Y

    def yval(c, ic_flat_index, a):
        """entry of Y_c (or I) at (multi-index of c's modes, column a)."""
        nd = t.node(c)
        if nd.identity:
            return 1.0 if ic_flat_index[1] == a else 0.0
        p = 1.0
        for mu in range(nd.lo, nd.hi):
            p *= Y[mu][ic_flat_index[0][mu - nd.lo], a]
        return p

    def flat(i, lo, hi):
        f = 0
        for mu in range(lo, hi):
            f = f * dims[mu] + i[mu]
        return f

    Om, Ps = {}, {}
    for v in t.sketched():
        nd = t.node(v)
        om = np.zeros((nd.s, nd.r))
        chs = nd.children
        pshape = ([nd.n] if nd.is_leaf else [t.node(c).s for c in chs]) + [nd.r]
        ps = np.zeros(pshape)
        for i in idx:
            a_ = T[i]
            xs = np.ones(nd.r)
            for mu in range(t.d):
                if not nd.lo <= mu < nd.hi:
                    xs = xs * X[mu][i[mu], :nd.r]
            ys = np.ones(nd.s)
            for mu in range(nd.lo, nd.hi):
                ys = ys * Y[mu][i[mu], :nd.s]
            om += a_ * np.outer(ys, xs)
            if nd.is_leaf:
                ps[flat(i, nd.lo, nd.hi)] += a_ * xs
            else:
                facs = []
                for c in chs:
                    cn = t.node(c)
                    key = ([i[mu] for mu in range(cn.lo, cn.hi)], flat(i, cn.lo, cn.hi))
                    facs.append(np.array([yval(c, key, a) for a in range(cn.s)]))
                outer = facs[0]
                for f in facs[1:]:
                    outer = np.multiply.outer(outer, f)
                ps += a_ * np.multiply.outer(outer, xs)
        Om[v], Ps[v] = om, ps
    root = t.node(t.root)
    pr = np.zeros([t.node(c).s for c in root.children])
    for i in idx:
        facs = []
        for c in root.children:
            cn = t.node(c)
            key = ([i[mu] for mu in range(cn.lo, cn.hi)], flat(i, cn.lo, cn.hi))
            facs.append(np.array([yval(c, key, a) for a in range(cn.s)]))
        outer = facs[0]
        for f in facs[1:]:
            outer = np.multiply.outer(outer, f)
        pr += T[i] * outer
    return Om, Ps, pr


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    ("binary4", W.balanced_binary(4), [4, 4, 4, 4], 2, 1),
    ("toy3", W.toy_tree(), [3, 2, 3, 2, 3, 2], 2, 1),
    ("tt5", W.tensor_train(5), [3, 3, 3, 3, 3], 2, 1),
    ("tucker4", W.tucker(4), [3, 4, 3, 4], 2, 1),
]


@pytest.mark.parametrize("name,tr,dims,r,p", CASES, ids=[c[0] for c in CASES])
def test_sketch_matches_brute_force_index_sums(name, tr, dims, r, p):
    t = Tree(tr[0], tr[1], dims, [r] * len(tr[0]), [p] * len(tr[0]), tr[2])
    T = W.gaussian(dims, 3)
    drm = O.Drm(t, 99)
    Om, Ps, Pr = O.sketch_ttnn(T, t, drm)
    bOm, bPs, bPr = _brute(T, t, drm)
    for v in t.sketched():
        assert _rel(Om[v], bOm[v]) < 1e-13
        assert _rel(Ps[v], bPs[v]) < 1e-13
    assert _rel(Pr, bPr) < 1e-13


def test_sketch_linearity():
    tr = W.toy_tree()
    dims = [4, 3, 4, 3, 4, 3]
    t = Tree(tr[0], tr[1], dims, [3] * 10, [2] * 10, tr[2])
    drm = O.Drm(t, 5)
    rng = np.random.default_rng(0)
    parts = [rng.standard_normal(dims) for _ in range(4)]
    lam = [0.5, -2.0, 1.25, 3.0]
    T = sum(l * h for l, h in zip(lam, parts))
    Om, Ps, Pr = O.sketch_ttnn(T, t, drm)
    aOm, aPs, aPr = O.sketch_linear_combination(parts, lam, t, drm)
    for v in t.sketched():
        assert _rel(aOm[v], Om[v]) < 1e-13 and _rel(aPs[v], Ps[v]) < 1e-13
    assert _rel(aPr, Pr) < 1e-13
    # a dropped or duplicated update is visible
    bOm, _, _ = O.sketch_linear_combination(parts[:3], lam[:3], t, drm)
    v = t.sketched()[0]
    assert _rel(bOm[v], Om[v]) > 1e-3


def test_sttnn_contracted_tensor_equals_effective_drm():
    tr = W.toy_tree()
    dims = [4, 3, 4, 3, 4, 3]
    t = Tree(tr[0], tr[1], dims, [2] * 10, [2] * 10, tr[2])
    drm = O.Drm(t, 7, "f64", "sttnn")
    T = W.gaussian(dims, 4)
    Om, Ps, Pr = OS.sketch_sttnn(T, t, drm)
    for v in t.sketched():
        nd = t.node(v)
        G = O.unfold(T, nd.lo, nd.hi) @ OS.effective_x(t, drm, v)
        assert _rel(drm.Yt(v).T @ G, Om[v]) < 1e-13
        if nd.is_leaf:
            assert _rel(G, Ps[v]) < 1e-13
    # the first node (empty reuse set) sees exactly the TTNN sketch
    v0 = t.sketched()[0]
    assert t.sttnn_reuse(v0) == []


@pytest.mark.parametrize("tr,dims", [(W.balanced_binary(4), [5, 6, 5, 6]),
                                     (W.tensor_train(4), [5, 4, 5, 4]),
                                     (W.toy_tree(), [3, 4, 3, 4, 3, 4])])
def test_ttn_input_sketch_equals_dense_sketch(tr, dims):
    cin = W.ttn_cores(tr, dims, [3] * len(tr[0]), np.random.default_rng(8))
    Td = W.ttn_dense(tr, cin)
    t = Tree(tr[0], tr[1], dims, [2] * len(tr[0]), [2] * len(tr[0]), tr[2])
    drm = O.Drm(t, 14, "f64", "round")
    a = OR.sketch_ttn_input(cin, t, drm)
    b = O.sketch_ttnn(Td, t, drm)
    for v in t.sketched():
        assert _rel(a[0][v], b[0][v]) < 1e-12 and _rel(a[1][v], b[1][v]) < 1e-12
    assert _rel(a[2], b[2]) < 1e-12
