"""Pins of the oracle's TTN-format helpers against the dense tensor they
define (Def. "Tree tensor network format"): inner products of two networks
with different edge ranks, and entries at sampled multi-indices."""
import numpy as np
import pytest

import workloads as W
from oracle import rounding as OR
from oracle.tree import Tree

TREES = [("binary4", W.balanced_binary(4), [4, 3, 5, 3]),
         ("tt5", W.tensor_train(5), [3, 4, 3, 2, 3]),
         ("toy6", W.toy_tree(), [2, 3, 2, 3, 2, 3]),
         ("tucker4", W.tucker(4), [3, 4, 2, 3])]


@pytest.mark.parametrize("name,tr,dims", TREES, ids=[t[0] for t in TREES])
def test_ttn_inner_and_entries_match_dense(name, tr, dims):
    n = len(tr[0])
    t = Tree(tr[0], tr[1], dims, [2] * n, [1] * n, tr[2])
    A = W.ttn_cores(tr, dims, [3] * n, np.random.default_rng(1))
    B = W.ttn_cores(tr, dims, [2] * n, np.random.default_rng(2))
    Ad, Bd = W.ttn_dense(tr, A), W.ttn_dense(tr, B)
    assert abs(OR.ttn_inner(t, A, B) - np.vdot(Ad, Bd)) <= 1e-12 * np.linalg.norm(Ad) * np.linalg.norm(Bd)
    assert abs(OR.ttn_inner(t, A, A) - np.vdot(Ad, Ad)) <= 1e-12 * np.vdot(Ad, Ad)
    rng = np.random.default_rng(3)
    idx = np.stack([rng.integers(0, dm, size=50) for dm in dims], axis=1)
    want = Ad[tuple(idx.T)]
    assert np.allclose(OR.ttn_entries(t, A, idx), want, rtol=1e-12, atol=1e-12 * np.abs(Ad).max())


@pytest.mark.parametrize("name,tr,dims", TREES, ids=[t[0] for t in TREES])
def test_ttn_svd_of_a_network_equals_dense_hsvd(name, tr, dims):
    from oracle import baselines as B
    n = len(tr[0])
    A = W.ttn_cores(tr, dims, [3] * n, np.random.default_rng(5))
    Ad = W.ttn_dense(tr, A)
    t = Tree(tr[0], tr[1], dims, [2] * n, [1] * n, tr[2])
    cut, sig = OR.ttn_svd(t, A)
    want = B.hsvd(Ad, t)
    got = W.ttn_dense(tr, cut)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    # the singular values of every unfolding
    from oracle.ttnn import unfold
    for v in t.sketched():
        nd = t.node(v)
        s = np.linalg.svd(unfold(Ad, nd.lo, nd.hi), compute_uv=False)
        k = min(len(s), len(sig[v]))
        assert np.allclose(sig[v][:k], s[:k], rtol=1e-8, atol=1e-10 * s[0])


def test_orthogonal_cp_ttn_is_orthonormal_with_the_decay():
    tr = W.toy_tree()
    dims = [12] * 6
    cores = W.orthogonal_cp_ttn(tr, dims, 5, lambda i: 1.0 / i ** 2, 3)
    ch, _ = W.children_of(tr[0], tr[1])
    for v, c in cores.items():
        if not ch[v]:
            M = c.reshape(c.shape[0], -1)
            assert np.allclose(M @ M.T, np.eye(5), atol=1e-12)      # orthonormal leaf rows
    # the root's singular-value structure: a superdiagonal of 1/i^2 rotated
    root = tr[0].index(-1)
    R = cores[root]
    assert abs(np.linalg.norm(R) - np.sqrt(sum(1.0 / i ** 4 for i in range(1, 6)))) < 1e-12
