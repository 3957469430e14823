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
