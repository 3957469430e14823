"""Pins of the oracle against the error analysis of Sec. 6 and against
brute-force hierarchical / TT SVD truncations."""
import numpy as np
import pytest

import workloads as W
from oracle import baselines as B
from oracle import bounds as BD
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.tree import Tree


def _tree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def test_deterministic_bound_thm_6_4():
    tr = W.balanced_binary(4)
    dims = [6] * 4
    T, _ = W.exact_ttn(tr, dims, [3] * 7, 21, noise=0.05)
    t = _tree(tr, dims, 4, 4)
    for seed in range(5):
        drm = O.Drm(t, 100 + seed)
        Om, Ps, Pr = O.sketch_ttnn(T, t, drm)
        cores, _ = O.recover(t, Om, Ps, Pr)
        err = np.linalg.norm(O.reconstruct(t, cores) - T)
        b1, b2 = BD.deterministic(T, t, drm, {v: 2 for v in t.sketched()})
        assert err <= b1 * (1 + 1e-10) and b1 <= b2 * (1 + 1e-10)


def test_deterministic_bound_thm_6_7_sttnn():
    tr = W.toy_tree()
    dims = [4, 3, 4, 3, 4, 3]
    T, _ = W.exact_ttn(tr, dims, [2] * 10, 8, noise=0.05)
    t = _tree(tr, dims, 2, 2)
    drm = O.Drm(t, 31, "f64", "sttnn")
    Om, Ps, Pr = OS.sketch_sttnn(T, t, drm)
    cores, _ = O.recover(t, Om, Ps, Pr)
    err = np.linalg.norm(O.reconstruct(t, cores) - T)
    ranges = {}
    for v in t.sketched():
        nd = t.node(v)
        ranges[v] = O.unfold(T, nd.lo, nd.hi) @ OS.effective_x(t, drm, v)
    # STTNN projectors P_t = T_S X (Y^T T_S X)^+ Y^T
    b1, _ = BD.deterministic(T, t, drm, {v: 1 for v in t.sketched()}, sttnn_ranges=ranges)
    assert err <= b1 * (1 + 1e-10)


def test_expected_bound_thm_6_6_dense_gaussian():
    tr = W.balanced_binary(3)
    dims = [8, 8, 8]
    T, _ = W.exact_ttn(tr, dims, [3] * 5, 5, noise=0.2)
    t = _tree(tr, dims, 4, 3)
    rhat = {v: 2 for v in t.sketched()}
    errs = []
    for seed in range(30):
        drm = O.DenseDrm(t, 500 + seed)
        cores, _ = O.recover(t, *O.sketch_ttnn(T, t, drm))
        errs.append(np.linalg.norm(O.reconstruct(t, cores) - T))
    assert np.mean(errs) <= BD.expected(T, t, rhat)


def test_ttnn_against_hierarchical_svd_brute_force():
    """Every TTN of ranks r_t has rank(T^(t)) <= r_t, so the TTNN error is at
    least max_t E_svd(T^(t), r_t); the HSVD error is at most
    sqrt(sum_t E_svd^2) (Grasedyck's quasi-optimality)."""
    tr = W.toy_tree()
    dims = [4, 3, 4, 3, 4, 3]
    T, _ = W.exact_ttn(tr, dims, [2] * 10, 2, noise=0.1)
    t = _tree(tr, dims, 2, 2)
    tails = [B.svd_tail(O.unfold(T, t.node(v).lo, t.node(v).hi), t.node(v).r) for v in t.sketched()]
    H = B.hsvd(T, t)
    eh = np.linalg.norm(H - T)
    assert eh <= np.sqrt(np.sum(np.square(tails))) * (1 + 1e-12)
    assert eh >= max(tails) * (1 - 1e-12)
    cores, _ = O.ttnn(T, t, 3)
    e = np.linalg.norm(O.reconstruct(t, cores) - T)
    assert e >= max(tails) * (1 - 1e-12)


def test_tt_svd_brute_force():
    dims = [4, 5, 4, 5]
    T = W.gaussian(dims, 9)
    Ts = B.tt_svd(T, [3, 4, 3])
    tails = [B.svd_tail(O.unfold(T, 0, k), r) for k, r in zip(range(1, 4), [3, 4, 3])]
    e = np.linalg.norm(Ts - T)
    assert max(tails) * (1 - 1e-12) <= e <= np.sqrt(np.sum(np.square(tails))) * (1 + 1e-12)
    assert np.allclose(B.tt_svd(T, [4, 20, 5]), T, atol=1e-12)


def test_hosvd_on_tucker_tree():
    dims = [5, 6, 5]
    tr = W.tucker(3)
    T = W.gaussian(dims, 10)
    t = _tree(tr, dims, 3, 1)
    H = B.hsvd(T, t)
    tails = [B.svd_tail(O.unfold(T, m, m + 1), 3) for m in range(3)]
    e = np.linalg.norm(H - T)
    assert max(tails) * (1 - 1e-12) <= e <= np.sqrt(np.sum(np.square(tails))) * (1 + 1e-12)


@pytest.mark.parametrize("tr,dims", [(W.toy_tree(), [3, 4, 3, 4, 3, 4]),
                                     (W.balanced_binary(4), [5, 4, 6, 3]),
                                     (W.tensor_train(4), [4, 5, 4, 3])])
def test_ttn_hmt_equals_its_projector_form_and_recovers_exact_ranks(tr, dims):
    """TTN-HMT cores reproduce (prod_levels kron P_t) T with the orthogonal
    projectors P_t = Q_t Q_t^T, Q_t = orth(T^(t) X_t); exact for a tensor
    whose TTN ranks are at most the targets."""
    n = len(tr[0])
    t = _tree(tr, dims, 2, 2)
    T = W.gaussian(dims, 21)
    drm = O.DenseDrm(t, 8)
    cores = B.ttn_hmt(T, t, drm)
    proj = {}
    for v in t.sketched():
        nd = t.node(v)
        Qv, _ = np.linalg.qr(O.unfold(T, nd.lo, nd.hi) @ drm.Xt(v), mode="reduced")
        proj[v] = Qv @ Qv.T
    A = O.projector_approximant(T, t, proj)
    assert np.linalg.norm(O.reconstruct(t, cores) - A) <= 1e-12 * np.linalg.norm(T)
    Te, _ = W.exact_ttn(tr, dims, [2] * n, 4)
    ce = B.ttn_hmt(Te, t, O.DenseDrm(t, 9))
    assert np.linalg.norm(O.reconstruct(t, ce) - Te) <= 1e-12 * np.linalg.norm(Te)
