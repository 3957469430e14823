"""Seeded synthetic inputs shared by the tests, ``bench.py`` and the oracle's
timing leg.  This module holds input synthesis only (trees, tensors, updates)
and none of TTNN's arithmetic; it imports neither the oracle nor the CUDA
library.

Trees are returned as (parent, leaf_modes, identity) lists in the format of
the library's ``ttnn_tree`` (0-based modes, parent -1 for the root).

Workload recipes (the paper's experiments use formula / synthetic generators,
Sec. 8; these mirror their shapes):
* exact_ttn: N(0,1) cores on a tree, contracted to a dense tensor, plus i.i.d.
  Gaussian noise at a given relative Frobenius norm (order-4, 24^4 case).
* inv_sum: f(x) = 1 / (x_1 + ... + x_d) on the uniform grid x = 1 + i/(n-1) of
  [1, 2]^d (fast-decaying multilinear spectrum; the paper's Hilbert tensor
  1/(1 + i_1 + ... + i_d) of Sec. 8 is the same family).
* cp_term / box_update: rank-2 CP terms with N(0,1) factors and dense
  sub-blocks of N(0, 0.01) noise (streamed order-6 case).
* rounding_input: TTN cores of rank R_dom + R_noise as a block-diagonal direct
  sum, N(0, 1/R) entries, the dominant part 100 times the noise part in norm
  (order-8 rounding).
* orthogonal_cp_ttn: the paper's TTN-rounding inputs (Sec. 8, second
  experiment): every transfer tensor a superdiagonal tensor of a decaying
  sequence sigma_i multiplied by Haar orthogonal matrices along each axis,
  Haar orthogonal leaf matrices.
* hilbert: the paper's Hilbert tensor 1 / (1 + i_1 + ... + i_d) (Sec. 8,
  first experiment).
"""
import numpy as np


# ---------------------------------------------------------------------------
# trees
# ---------------------------------------------------------------------------
def from_nested(spec):
    """Nested tuples of modes -> (parent, leaf_modes, identity).  An int is a
    single-mode leaf, a list a multi-mode leaf, a tuple an internal node."""
    parent, leaf_modes = [], []

    def add(s, p):
        v = len(parent)
        parent.append(p)
        if isinstance(s, int):
            leaf_modes.append([s])
        elif isinstance(s, list):
            leaf_modes.append(list(s))
        else:
            leaf_modes.append([])
            for c in s:
                add(c, v)
        return v

    add(spec, -1)
    return parent, leaf_modes, [False] * len(parent)


def balanced_binary(d):
    """Balanced binary tree: the left child takes ceil(|t|/2) contiguous modes."""
    def build(lo, hi):
        if hi - lo == 1:
            return lo
        mid = lo + (hi - lo + 1) // 2
        return (build(lo, mid), build(mid, hi))
    return from_nested(build(0, d))


def tucker(d):
    """Star tree: root -> {0}, ..., {d-1}."""
    return from_nested(tuple(range(d)))


def tensor_train(d):
    """Caterpillar {0..k} -> {0..k-1}, {k}; the single-mode leaves {k}, k >= 1,
    are identity nodes, so the sketched nodes are the prefixes {0..k-1}."""
    spec = 0
    for k in range(1, d):
        spec = (spec, k)
    parent, leaf_modes, identity = from_nested(spec)
    identity = [bool(lm) and lm[0] >= 1 for lm in leaf_modes]
    return parent, leaf_modes, identity


def toy_tree():
    """The paper's 6-mode example index tree (Sec. 3, first figure):
    {1..6} -> {1,2,3}, {4}, {5,6}; {1,2,3} -> {1,2}, {3}; {1,2} -> {1}, {2};
    {5,6} -> {5}, {6} (0-based here)."""
    return from_nested((((0, 1), 2), 3, (4, 5)))


def node_modes(parent, leaf_modes):
    """Sorted mode list of every node (union over its subtree's leaves)."""
    n = len(parent)
    modes = [list(leaf_modes[v]) for v in range(n)]
    order = sorted(range(n), key=lambda v: -depth_of(parent, v))
    for v in order:
        if parent[v] >= 0:
            modes[parent[v]].extend(modes[v])
    return [sorted(m) for m in modes]


def depth_of(parent, v):
    k = 0
    while parent[v] >= 0:
        v = parent[v]
        k += 1
    return k


def children_of(parent, leaf_modes):
    modes = node_modes(parent, leaf_modes)
    ch = [[] for _ in parent]
    for v, p in enumerate(parent):
        if p >= 0:
            ch[p].append(v)
    for c in ch:
        c.sort(key=lambda v: modes[v][0])
    return ch, modes


# ---------------------------------------------------------------------------
# dense tensors
# ---------------------------------------------------------------------------
def ttn_cores(tree, dims, ranks, rng, scale=1.0):
    """Random N(0, scale^2) TTN cores: root (r_c..), transfer (r_t, r_c..),
    leaf (r_t, n_mu..).  ranks[v] is node v's edge rank (root ignored)."""
    parent, leaf_modes, _ = tree
    ch, modes = children_of(parent, leaf_modes)
    cores = {}
    for v in range(len(parent)):
        if not ch[v]:
            shape = [ranks[v]] + [dims[m] for m in modes[v]]
        else:
            shape = ([] if parent[v] < 0 else [ranks[v]]) + [ranks[c] for c in ch[v]]
        cores[v] = rng.standard_normal(shape) * scale
    return cores


def ttn_dense(tree, cores):
    """Contract a TTN to its dense tensor (modes in increasing order)."""
    parent, leaf_modes, _ = tree
    ch, _ = children_of(parent, leaf_modes)
    root = parent.index(-1)

    def full(v):
        out = cores[v]
        for c in ch[v]:
            out = np.tensordot(out, full(c), axes=([1], [0]))
        return out

    out = cores[root]
    for c in ch[root]:
        out = np.tensordot(out, full(c), axes=([0], [0]))
    return out


def exact_ttn(tree, dims, ranks, seed, noise=0.0):
    """Dense tensor with exact TTN ranks <= ranks, plus Gaussian noise of
    relative Frobenius norm `noise`.  Returns (T, cores)."""
    rng = np.random.default_rng(seed)
    cores = ttn_cores(tree, dims, ranks, rng)
    T = ttn_dense(tree, cores)
    if noise > 0:
        E = rng.standard_normal(T.shape)
        T = T + E * (noise * np.linalg.norm(T) / np.linalg.norm(E))
    return T, cores


def inv_sum(d, n, dtype=np.float64):
    """A[i_1..i_d] = 1 / sum_mu (1 + i_mu/(n-1)) in binary64, cast to dtype."""
    x = 1.0 + np.arange(n, dtype=np.float64) / (n - 1)
    s = np.zeros([n] * d)
    for mu in range(d):
        sh = [1] * d
        sh[mu] = n
        s = s + x.reshape(sh)
    return (1.0 / s).astype(dtype)


def inv_sum_torch(d, n, device, dtype):
    """The same tensor as inv_sum, built on a torch device (same operation
    order: binary64 sum over modes in increasing order, reciprocal, cast)."""
    import torch
    x = 1.0 + torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
    s = torch.zeros([n] * d, dtype=torch.float64, device=device)
    for mu in range(d):
        sh = [1] * d
        sh[mu] = n
        s = s + x.reshape(sh)
    return (1.0 / s).to(dtype)


def inv_sum_slab_torch(d, n, world, rank, device, dtype):
    """Rank `rank`'s slab (mode-0 indices [rank*n, (rank+1)*n)) of the order-d
    tensor 1/sum(x) whose mode 0 has n*world grid points on [1, 2] and the
    other modes n; world = 1 gives inv_sum_torch(d, n)."""
    import torch
    m = n * world
    x0 = 1.0 + (rank * n + torch.arange(n, dtype=torch.float64, device=device)) / (m - 1)
    x = 1.0 + torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
    s = torch.zeros([n] * d, dtype=torch.float64, device=device)
    for mu in range(d):
        sh = [1] * d
        sh[mu] = n
        s = s + (x0 if mu == 0 else x).reshape(sh)
    return (1.0 / s).to(dtype)


def gaussian(shape, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal(shape) * scale


# ---------------------------------------------------------------------------
# streamed updates
# ---------------------------------------------------------------------------
def cp_term(dims, rank, rng):
    """Rank-`rank` CP term: weights 1, factors a_mu (n_mu x rank) ~ N(0,1)."""
    return np.ones(rank), [rng.standard_normal((n, rank)) for n in dims]


def cp_dense(weights, factors):
    d = len(factors)
    out = 0.0
    for q in range(len(weights)):
        t = np.array(weights[q])
        for mu in range(d):
            t = np.multiply.outer(t, factors[mu][:, q])
        out = out + t
    return out


def box_update(dims, varying, extent, rng, sigma=0.1):
    """Dense sub-block: `varying` modes span `extent` consecutive indices from
    a uniform offset, the other modes are fixed at a uniform index (extent 1).
    Returns (offset, extent_per_mode, data)."""
    d = len(dims)
    off = [int(rng.integers(0, n)) for n in dims]
    ext = [1] * d
    for mu in varying:
        ext[mu] = extent
        off[mu] = int(rng.integers(0, dims[mu] - extent + 1))
    data = rng.standard_normal(ext) * sigma
    return off, ext, data


def embed_box(dims, off, ext, data):
    T = np.zeros(dims)
    sl = tuple(slice(o, o + e) for o, e in zip(off, ext))
    T[sl] = data
    return T


def streaming_updates(dims, n_updates, seed, box_modes=3, box_extent=32, cp_rank=2):
    """The streamed order-6 workload: each update is one rank-2 CP term
    (N(0,1) factors) plus one dense box of N(0, 0.01) noise over `box_modes`
    distinct uniformly chosen modes."""
    rng = np.random.default_rng(seed)
    out = []
    d = len(dims)
    for _ in range(n_updates):
        w, f = cp_term(dims, cp_rank, rng)
        modes = sorted(rng.choice(d, size=box_modes, replace=False).tolist())
        off, ext, data = box_update(dims, modes, min(box_extent, min(dims)), rng)
        out.append({"cp_weights": w, "cp_factors": f, "box_offset": off,
                    "box_extent": ext, "box_data": data})
    return out


# ---------------------------------------------------------------------------
# TTN rounding input
# ---------------------------------------------------------------------------
def _block_norm2(parent, ch, modes, cores, lo, rb):
    """Squared Frobenius norm of the network formed by the [lo, lo + rb)
    diagonal block of every core (input plumbing: Gram matrices contracted
    leaves first)."""
    order = []
    stack = [parent.index(-1)]
    while stack:
        v = stack.pop()
        order.append(v)
        stack.extend(ch[v])
    G = {}
    for v in reversed(order):
        C = cores[v]
        if not ch[v]:
            B = C[lo:lo + rb].reshape(rb, -1)
            G[v] = B @ B.T
            continue
        sl = tuple(slice(lo, lo + rb) for _ in range(C.ndim))
        B = C[sl]
        head = 0 if parent[v] < 0 else 1
        # contract every child axis with that child's Gram matrix
        X = B
        for k, c in enumerate(ch[v]):
            X = np.moveaxis(np.tensordot(X, G[c], axes=([head + k], [0])), -1, head + k)
        if head:
            G[v] = np.tensordot(B, X, axes=(list(range(1, B.ndim)), list(range(1, B.ndim))))
        else:
            G[v] = np.array(np.sum(B * X))
    return float(G[order[0]])


def rounding_input(tree, dims, r_dom, r_noise, seed, dom_scale=100.0):
    """TTN with every edge of rank r_dom + r_noise: cores are block-diagonal
    direct sums of a dominant (rank r_dom) and a noise (rank r_noise) TTN,
    entries N(0, 1/R) before scaling.  Each part's root block is then scaled
    so that the noise part has unit Frobenius norm and the dominant part
    dom_scale times that (with unscaled cores the noise part, of larger
    ranks, would carry almost all of the norm)."""
    parent, leaf_modes, _ = tree
    ch, modes = children_of(parent, leaf_modes)
    rng = np.random.default_rng(seed)
    R = r_dom + r_noise
    cores = {}
    for v in range(len(parent)):
        is_root = parent[v] < 0
        blocks = []
        for b, rb in ((0, r_dom), (1, r_noise)):
            if not ch[v]:
                shape = [rb] + [dims[m] for m in modes[v]]
            else:
                shape = ([] if is_root else [rb]) + [rb] * len(ch[v])
            blocks.append(rng.standard_normal(shape) / np.sqrt(R))
        if not ch[v]:
            C = np.concatenate(blocks, axis=0)
        else:
            shape = ([] if is_root else [R]) + [R] * len(ch[v])
            C = np.zeros(shape)
            for b, (lo, rb) in enumerate(((0, r_dom), (r_dom, r_noise))):
                sl = tuple(slice(lo, lo + rb) for _ in shape)
                C[sl] = blocks[b]
        cores[v] = C
    root = parent.index(-1)
    Cr = cores[root]
    for lo, rb, target in ((0, r_dom, dom_scale), (r_dom, r_noise, 1.0)):
        nrm = np.sqrt(_block_norm2(parent, ch, modes, cores, lo, rb))
        sl = tuple(slice(lo, lo + rb) for _ in range(Cr.ndim))
        Cr[sl] *= target / nrm
    return cores


def haar_orthogonal(n, k, rng):
    """n x k with orthonormal columns, Haar distributed: Q of the QR of a
    Gaussian n x k matrix with the signs of diag(R) folded in (Mezzadri)."""
    Z = rng.standard_normal((n, k))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def orthogonal_cp_ttn(tree, dims, rank, decay, seed):
    """TTN of edge rank `rank`: each transfer tensor (and the root) is the
    superdiagonal tensor with entries sigma_i = decay(i), i = 1..rank,
    multiplied along every axis by a Haar orthogonal rank x rank matrix; each
    leaf core is the transpose of a Haar orthogonal n_leaf x rank matrix."""
    parent, leaf_modes, _ = tree
    ch, modes = children_of(parent, leaf_modes)
    rng = np.random.default_rng(seed)
    sig = np.array([decay(i) for i in range(1, rank + 1)], dtype=np.float64)
    cores = {}
    for v in range(len(parent)):
        if not ch[v]:
            n = int(np.prod([dims[m] for m in modes[v]]))
            cores[v] = haar_orthogonal(n, rank, rng).T.reshape([rank] + [dims[m] for m in modes[v]])
            continue
        k = len(ch[v]) + (0 if parent[v] < 0 else 1)
        C = np.zeros([rank] * k)
        C[tuple(np.arange(rank) for _ in range(k))] = sig
        for a in range(k):
            U = haar_orthogonal(rank, rank, rng)
            C = np.moveaxis(np.tensordot(C, U, axes=([a], [1])), -1, a)
        cores[v] = C
    return cores


def hilbert(d, n, dtype=np.float64):
    """H[i_1..i_d] = 1 / (1 + i_1 + ... + i_d), 0-based indices (Sec. 8)."""
    s = np.zeros([n] * d)
    for mu in range(d):
        sh = [1] * d
        sh[mu] = n
        s = s + np.arange(n, dtype=np.float64).reshape(sh)
    return (1.0 / (1.0 + s)).astype(dtype)


# ---------------------------------------------------------------------------
# Serving mix (many resident streams, Poisson slice updates)
# ---------------------------------------------------------------------------
def serving_stream_spec(rng, max_entries=2e8):
    """One stream of the serving mix: order d ~ U{3..6}; mode sizes drawn from
    {16, 32, 64, 128}, each redrawn while the tensor has more than
    `max_entries` entries; tree ~ U{balanced binary, tensor train, Tucker};
    rank r ~ U{4..32} on every node, oversampling p = r // 2."""
    d = int(rng.integers(3, 7))
    dims = []
    for _ in range(d):
        while True:
            n = int(rng.choice([16, 32, 64, 128]))
            if np.prod(dims + [n]) * 16 ** (d - len(dims) - 1) <= max_entries:
                break
        dims.append(n)
    kind = ["binary", "tt", "tucker"][int(rng.integers(0, 3))]
    tree = {"binary": balanced_binary, "tt": tensor_train, "tucker": tucker}[kind](d)
    r = int(rng.integers(4, 33))
    return {"kind": kind, "tree": tree, "dims": dims, "r": r, "p": r // 2}


def poisson_slices(rng, n_streams, dims_of, rate, seconds):
    """Arrival times (s) of a Poisson stream of slice updates at `rate`/s for
    `seconds`; each picks a stream uniformly, a mode uniformly and an index of
    that mode uniformly.  Returns a list of (t, stream, mode, index)."""
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= seconds:
            return out
        s = int(rng.integers(0, n_streams))
        mu = int(rng.integers(0, len(dims_of[s])))
        out.append((t, s, mu, int(rng.integers(0, dims_of[s][mu]))))
