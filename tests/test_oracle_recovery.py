"""Pins of the oracle's recovery phase: exact recovery, the two formulations
of the approximant, the special cases GN / MLN / STTA, and the eps rule."""
import numpy as np
import pytest

import workloads as W
from oracle import baselines as B
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.tree import Tree


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _tree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def test_exact_recovery_order4_24_rank5():
    """Order-4 24^4 exact TTN on ((1,2),(3,4)), ranks 5, l = 5: GN algebra
    reproduces a tensor whose unfoldings have rank <= r_t."""
    tr = W.balanced_binary(4)
    dims = [24] * 4
    T, _ = W.exact_ttn(tr, dims, [5] * 7, 1000)
    t = _tree(tr, dims, 5, 5)
    cores, _ = O.ttnn(T, t, 2000)
    assert _rel(O.reconstruct(t, cores), T) < 1e-12
    Tn, _ = W.exact_ttn(tr, dims, [5] * 7, 1000, noise=1e-8)
    cores, _ = O.ttnn(Tn, t, 2000)
    assert _rel(O.reconstruct(t, cores), Tn) < 1e-6


@pytest.mark.parametrize("variant", ["ttnn", "sttnn"])
def test_exact_recovery_rank_deficient(variant):
    """True ranks 2 below target 4: Omega_t is rank deficient and the
    eps-pseudo-inverse drops the null directions."""
    tr = W.toy_tree()
    dims = [5, 4, 5, 4, 5, 4]
    T, _ = W.exact_ttn(tr, dims, [2] * 10, 3)
    t = _tree(tr, dims, 4, 3)
    drm = O.Drm(t, 9, "f64", variant)
    sk = (O.sketch_ttnn if variant == "ttnn" else OS.sketch_sttnn)(T, t, drm)
    cores, info = O.recover(t, *sk)
    assert _rel(O.reconstruct(t, cores), T) < 1e-10
    assert min(info.values()) < 4


def test_cores_equal_projector_product():
    """Recovery-phase cores reproduce eq. (TTNN approximant projector)."""
    tr = W.toy_tree()
    dims = [4, 3, 4, 3, 4, 3]
    T = W.gaussian(dims, 11)
    t = _tree(tr, dims, 2, 2)
    cores, drm = O.ttnn(T, t, 12)
    A = O.projector_approximant(T, t, O.ttnn_projectors(T, t, drm))
    assert _rel(O.reconstruct(t, cores), A) < 1e-11
    # ... and the approximant is not trivially T
    assert _rel(A, T) > 0.1


def test_generalized_nystrom_special_case():
    """d = 2, one compressed child, one identity child: Algorithm 1."""
    tr = W.from_nested((0, 1))
    idn = [False, False, True]
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 5)) @ rng.standard_normal((5, 20)) + 1e-3 * rng.standard_normal((30, 20))
    t = Tree(tr[0], tr[1], [30, 20], [0, 4, 0], [0, 3, 0], idn)
    cores, drm = O.ttnn(A, t, 11)
    G = B.gn(A, drm.Xt(1), drm.Yt(1))
    assert _rel(O.reconstruct(t, cores), G) < 1e-12


def test_tucker_tree_is_multilinear_nystrom():
    tr = W.tucker(4)
    dims = [6, 5, 6, 5]
    T = W.gaussian(dims, 5)
    t = _tree(tr, dims, 3, 2)
    cores, drm = O.ttnn(T, t, 12)
    ch = t.node(t.root).children
    M = B.mln(T, [drm.Xt(v) for v in ch], [drm.Yt(v) for v in ch])
    assert _rel(O.reconstruct(t, cores), M) < 1e-12


def test_tt_tree_is_streaming_tt_approximation():
    tr = W.tensor_train(5)
    dims = [4, 5, 4, 5, 4]
    T = W.gaussian(dims, 6)
    t = _tree(tr, dims, 3, 2)
    cores, drm = O.ttnn(T, t, 13)
    sk = sorted(t.sketched(), key=lambda v: t.node(v).hi)
    assert [(t.node(v).lo, t.node(v).hi) for v in sk] == [(0, 1), (0, 2), (0, 3), (0, 4)]
    S = B.stta(T, [drm.Xt(v) for v in sk], [drm.Yt(v) for v in sk])
    assert _rel(O.reconstruct(t, cores), S) < 1e-12


def test_qr_sign_convention_and_uniqueness():
    A = W.gaussian((9, 4), 2)
    Q, R = O.qr_pos(A)
    assert np.all(np.diag(R) >= 0)
    assert np.allclose(Q @ R, A, atol=1e-14) and np.allclose(Q.T @ Q, np.eye(4), atol=1e-14)
    # Gram-Schmidt gives the same unique factor
    Qg = np.zeros_like(A)
    for k in range(4):
        v = A[:, k] - Qg[:, :k] @ (Qg[:, :k].T @ A[:, k])
        Qg[:, k] = v / np.linalg.norm(v)
    assert np.allclose(Qg, Q, atol=1e-12)


def test_eps_pseudo_inverse_threshold():
    """Singular values strictly larger than eps = 10 u ||R||_2 are kept and
    inverted; one at or below eps is dropped (eq. (stabilized_nystrom))."""
    U, _ = np.linalg.qr(W.gaussian((4, 4), 3))
    V, _ = np.linalg.qr(W.gaussian((4, 4), 4))
    u = 2.0 ** -52
    sv = np.array([1.0, 1e-3, 1e-9, 5 * u])
    R = U @ np.diag(sv) @ V.T
    Rp, k = O.eps_pinv(R)
    assert k == 3
    want = V[:, :3] @ np.diag(1 / sv[:3]) @ U[:, :3].T
    assert np.linalg.norm(Rp - want) <= 1e-5 * np.linalg.norm(want)
    # diagonal R: singular values exact, so the boundary is exercised exactly
    eps = 10 * u * 2.0
    assert O.eps_pinv(np.diag([2.0, eps]))[1] == 1
    assert O.eps_pinv(np.diag([2.0, eps * (1 + 2 * u)]))[1] == 2
    # a full-rank well-conditioned R: the plain inverse
    R2 = np.triu(W.gaussian((5, 5), 7)) + 5 * np.eye(5)
    Rp2, k2 = O.eps_pinv(R2)
    assert k2 == 5 and np.allclose(Rp2 @ R2, np.eye(5), atol=1e-13)


@pytest.mark.parametrize("variant", ["ttnn", "sttnn"])
def test_truncated_output_is_the_same_tensor_with_kept_ranks(variant):
    """eps-truncated cores: rank axes at the kept ranks, same reconstruction
    as the untruncated cores; exact recovery still holds."""
    tr = W.toy_tree()
    dims = [5, 4, 5, 4, 5, 4]
    T, _ = W.exact_ttn(tr, dims, [2] * 10, 3)
    t = _tree(tr, dims, 4, 3)
    drm = O.Drm(t, 9, "f64", variant)
    sk = (O.sketch_ttnn if variant == "ttnn" else OS.sketch_sttnn)(T, t, drm)
    full, info = O.recover(t, *sk)
    cut, info2 = O.recover(t, *sk, truncate=True)
    assert info == info2 and min(info.values()) < 4
    for v in t.nonroot():
        nd = t.node(v)
        if nd.identity:
            continue
        assert cut[v].shape[0] == info[v]
        if not nd.is_leaf:
            for k, c in enumerate(nd.children):
                if not t.node(c).identity:
                    assert cut[v].shape[1 + k] == info[c]
    for k, c in enumerate(t.node(t.root).children):
        if not t.node(c).identity:
            assert cut[t.root].shape[k] == info[c]
    assert _rel(O.reconstruct(t, cut), O.reconstruct(t, full)) < 1e-12
    assert _rel(O.reconstruct(t, cut), T) < 1e-10
