"""The bench's host-side TTN evaluations, used to report the error of every
recovered network (sampled entries) and of the rounding legs (inner products
of two networks), against the dense contraction of the same cores."""
import numpy as np
import pytest

import bench
import workloads as W

TREES = {
    "toy": (W.toy_tree(), [3, 4, 3, 2, 3, 4]),
    "binary4": (W.balanced_binary(4), [4, 3, 5, 4]),
    "tt5": (W.tensor_train(5), [3, 4, 3, 3, 2]),
    "tucker4": (W.tucker(4), [3, 5, 4, 3]),
}


class _Host:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class _FakeApi:
    """ttnn_plan_node's fields that the bench reads, laid out like the
    library's core buffer (nodes in user order, each core contiguous)."""

    def __init__(self, tree, cores):
        parent, leaf_modes, _ = tree
        _, modes = W.children_of(parent, leaf_modes)
        self.nodes, off = [], 0
        for v in range(len(parent)):
            c = np.asarray(cores[v])
            self.nodes.append({"core_offset": off, "core_elems": c.size,
                               "core_shape": list(c.shape), "mode_lo": min(modes[v]),
                               "mode_hi": max(modes[v]) + 1})
            off += c.size
        self.flat = np.concatenate([np.asarray(cores[v]).ravel() for v in range(len(parent))])

    def ttnn_plan_node(self, plan, v):
        return self.nodes[v]


@pytest.mark.parametrize("name", list(TREES))
def test_sampled_entries_equal_the_dense_contraction(name):
    tree, dims = TREES[name]
    nn = len(tree[0])
    cores = W.ttn_cores(tree, dims, [3] * nn, np.random.default_rng(5))
    T = W.ttn_dense(tree, cores)
    api = _FakeApi(tree, cores)
    idx = bench._sample_idx(dims, samples=500, seed=3)
    got = bench._ttn_entries(api, None, tree, _Host(api.flat), dims, idx)
    assert np.allclose(got, T[tuple(idx.T)], rtol=1e-12, atol=1e-12 * np.abs(T).max())
    # the relative error helper: zero against the exact values, and a
    # planted 1 % perturbation of every entry reads as 1 %
    assert bench._sampled_error(api, None, tree, _Host(api.flat), dims,
                                lambda i: T[tuple(i.T)], samples=500) < 1e-13
    e = bench._sampled_error(api, None, tree, _Host(api.flat), dims,
                             lambda i: T[tuple(i.T)] * 1.01, samples=500)
    assert abs(e - 0.01 / 1.01) < 1e-12


@pytest.mark.parametrize("name", list(TREES))
def test_network_inner_product_equals_the_dense_one(name):
    tree, dims = TREES[name]
    parent, leaf_modes, _ = tree
    nn = len(parent)
    ch, _ = W.children_of(parent, leaf_modes)
    rng = np.random.default_rng(9)
    A = W.ttn_cores(tree, dims, [2] * nn, rng)
    B = W.ttn_cores(tree, dims, [3] * nn, rng)
    want = float(np.vdot(W.ttn_dense(tree, A), W.ttn_dense(tree, B)))
    got = bench._ttn_inner(parent, ch, A, B)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want)) * 10


@pytest.mark.parametrize("ws", [1, 2, 4, 8])
def test_weak_scaling_slabs(ws):
    """Under N ranks the bench's tensor has N * 64 points on mode 0 and rank k
    owns the 64 x 64^4 slab at mode-0 offset 64 k (the whole tensor at N = 1):
    every rank streams a 64^5 block, and the slabs tile the tensor."""
    n = bench.NMODE
    covered = []
    for rank in range(ws):
        dims, (off, ext) = bench._geometry(ws, rank)
        assert dims == [n * ws] + [n] * (bench.D - 1)
        if ws == 1:
            assert off is None and ext is None
            covered.append((0, n))
            continue
        assert ext == [n] * bench.D
        assert off == [n * rank] + [0] * (bench.D - 1)
        covered.append((off[0], off[0] + ext[0]))
    assert sorted(covered) == [(n * k, n * (k + 1)) for k in range(ws)]
