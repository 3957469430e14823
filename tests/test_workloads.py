"""Pins of the synthetic input recipes the benchmark and the GPU tests use:
the 1/sum(x) grid tensor and its per-rank slabs, and the rounding input's
direct sum of a dominant and a noise network with the stated norms."""
import itertools

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("d,n,world", [(3, 4, 1), (3, 4, 2), (2, 5, 3)])
def test_inv_sum_slabs_are_the_grid_tensor(d, n, world):
    # mode 0 holds n * world points of [1, 2] (endpoints included), the other
    # modes n points; rank k owns the mode-0 indices [k n, (k + 1) n)
    m = n * world
    for k in range(world):
        got = W.inv_sum_slab_torch(d, n, world, k, "cpu", torch.float64).numpy()
        for idx in itertools.product(range(n), repeat=d):
            x = [1.0 + (k * n + idx[0]) / (m - 1)] + [1.0 + i / (n - 1) for i in idx[1:]]
            # to a few units of rounding (the division by n - 1 may be taken
            # as a multiplication by its reciprocal)
            assert abs(got[idx] - 1.0 / sum(x)) <= 4e-16 / sum(x)
    if world == 1:
        whole = W.inv_sum_torch(d, n, "cpu", torch.float64).numpy()
        assert np.array_equal(W.inv_sum_slab_torch(d, n, 1, 0, "cpu", torch.float64).numpy(), whole)


def _block(tr, cores, lo, rb):
    """The [lo, lo + rb) diagonal block of every core (one part of the sum)."""
    ch, _ = W.children_of(tr[0], tr[1])
    out = {}
    for v, C in cores.items():
        if not ch[v]:
            out[v] = C[lo:lo + rb]
        else:
            out[v] = C[tuple(slice(lo, lo + rb) for _ in range(C.ndim))]
    return out


def test_rounding_input_is_a_direct_sum_with_the_stated_norms():
    tr, dims, rd, rn = W.balanced_binary(4), [3, 4, 3, 4], 2, 3
    cores = W.rounding_input(tr, dims, rd, rn, 11)
    T = W.ttn_dense(tr, cores)
    Td = W.ttn_dense(tr, _block(tr, cores, 0, rd))
    Tn = W.ttn_dense(tr, _block(tr, cores, rd, rn))
    # block-diagonal cores: the network is the sum of the two parts
    assert np.abs(T - (Td + Tn)).max() <= 1e-13 * np.abs(T).max()
    assert abs(np.linalg.norm(Tn) - 1.0) <= 1e-12
    assert abs(np.linalg.norm(Td) - 100.0) <= 1e-10
    # the dominant part has rank <= rd across every edge of the tree
    _, node_modes = W.children_of(tr[0], tr[1])
    checked = 0
    for v in range(len(tr[0])):
        if tr[0][v] < 0:
            continue
        modes = node_modes[v]
        rest = [m for m in range(len(dims)) if m not in modes]
        M = np.transpose(Td, list(modes) + rest).reshape(int(np.prod([dims[m] for m in modes])), -1)
        s = np.linalg.svd(M, compute_uv=False)
        assert np.sum(s > 1e-10 * s[0]) <= rd
        # while the whole network has the full rank rd + rn there (when the
        # unfolding allows it)
        s_all = np.linalg.svd(np.transpose(T, list(modes) + rest).reshape(M.shape), compute_uv=False)
        assert np.sum(s_all > 1e-10 * s_all[0]) == min(rd + rn, *M.shape)
        checked += 1
    assert checked == len(tr[0]) - 1


def test_streaming_updates_recipe():
    # rank-2 CP term with N(0, 1) factors + one 32^3 box of N(0, 0.01) values
    # over three distinct modes, the other modes fixed at one index
    dims = [32] * 6
    ups = W.streaming_updates(dims, 64, 5)
    vals = []
    for u in ups:
        assert np.array_equal(u["cp_weights"], np.ones(2))
        assert [f.shape for f in u["cp_factors"]] == [(32, 2)] * 6
        ext, off = u["box_extent"], u["box_offset"]
        assert sorted(ext) == [1, 1, 1, 32, 32, 32]
        assert all(0 <= o and o + e <= n for o, e, n in zip(off, ext, dims))
        assert u["box_data"].shape == tuple(ext)
        vals.append(u["box_data"].ravel())
    v = np.concatenate(vals)
    assert abs(v.std() - 0.1) < 0.002 and abs(v.mean()) < 0.002


def test_hilbert_entries():
    H = W.hilbert(3, 4)
    for idx in itertools.product(range(4), repeat=3):
        assert H[idx] == 1.0 / (1.0 + sum(idx))


def test_serving_stream_specs_stay_in_the_stated_ranges():
    rng = np.random.default_rng(9)
    kinds = set()
    for _ in range(400):
        sp = W.serving_stream_spec(rng)
        d = len(sp["dims"])
        assert 3 <= d <= 6 and set(sp["dims"]) <= {16, 32, 64, 128}
        assert np.prod(sp["dims"], dtype=float) <= 2e8
        assert 4 <= sp["r"] <= 32 and sp["p"] == sp["r"] // 2
        parent, leaf_modes, _ = sp["tree"]
        assert sorted(m for lm in leaf_modes for m in lm) == list(range(d))
        kinds.add(sp["kind"])
    assert kinds == {"binary", "tt", "tucker"}


def test_poisson_slices_rate_and_choices():
    rng = np.random.default_rng(3)
    dims_of = [[16, 32, 64], [128, 16, 16, 16]]
    ev = W.poisson_slices(rng, 2, dims_of, 2000.0, 5.0)
    t = np.array([e[0] for e in ev])
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    # 10000 arrivals expected; a Poisson count has standard deviation 100
    assert abs(len(ev) - 10000) < 500
    for _, s, mu, i in ev:
        assert 0 <= s < 2 and 0 <= mu < len(dims_of[s]) and 0 <= i < dims_of[s][mu]
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 2000.0 - 1.0) < 0.05
