"""STTNN: the sequential variant (Sec. 5).  ORACLE: test infrastructure only.

For each non-root node t, in lexicographic order, the projection of
eq. (general_seq_projection) uses T_{S_t} = T x_{s in S_t} Y_s^T, the tensor
contracted on the already-sketched groups disjoint from t
(``Tree.sttnn_reuse``), and a right DRM X_t whose rows follow the axes of
T_{S_t} outside t: a contracted group s contributes XT_s (s_s x r, Philox kind
XT keyed by s), an untouched mode mu contributes X_mu (Khatri-Rao, Sec. 7).
Omega_t = Y_t^T T_{S_t}^(t) X_t and Psi_t = (kron_c Y_c)^T T_{S_t}^(t) X_t;
the root's Psi uses the full T (eq. (STTNN approximant projector) keeps the
TTNN hierarchy).  Recovery is the TTNN recovery phase unchanged.

The pass-side rounding rule of ``ttnn.Drm`` applies with the STTNN split
(L = first root child, whose Y is applied to A in the pass): the R modes of an
L-subtree node's X_t form the rounded block B_R, and Y of the first root child
is the rounded block.
"""
import numpy as np

from .ttnn import kr, contract_axis, psi_root, _psi_internal


def contracted_tensor(T, tree, drm, S):
    """T_S with each group s in S replaced by one axis of size s_s.
    Returns (tensor, axes) where axes lists ('m', mu) or ('g', s) in order."""
    axes = [("m", mu) for mu in range(tree.d)]
    out = np.asarray(T, dtype=np.float64)
    for s in sorted(S, key=lambda s: tree.node(s).lo):
        nd = tree.node(s)
        pos = axes.index(("m", nd.lo))
        k = nd.hi - nd.lo
        sh = out.shape
        out = out.reshape(sh[:pos] + (int(np.prod(sh[pos:pos + k])),) + sh[pos + k:])
        out = contract_axis(out, pos, drm.Yt(s))
        axes = axes[:pos] + [("g", s)] + axes[pos + k:]
    return out, axes


def sttnn_xt(tree, drm, v, axes):
    """Right DRM of node v over the non-t axes of T_{S_t}."""
    nd = tree.node(v)
    t = set(range(nd.lo, nd.hi))
    rest = [ax for ax in axes if not (ax[0] == "m" and ax[1] in t)]
    if drm.in_left(v):
        # R modes are never contracted for L-subtree nodes: one rounded block
        left = [ax for ax in rest if not (ax[0] == "m" and ax[1] in drm.Rmodes)]
        mats = [drm.XT[ax[1]] if ax[0] == "g" else drm.X[ax[1]] for ax in left] + [drm.BRX]
    else:
        mats = [drm.XT[ax[1]] if ax[0] == "g" else drm.X[ax[1]] for ax in rest]
    return kr(mats)[:, :nd.r]


def sketch_sttnn(T, tree, drm):
    """All STTNN sketches of T; same return convention as sketch_ttnn."""
    T = np.asarray(T, dtype=np.float64)
    Om, Ps = {}, {}
    for v in tree.sketched():
        nd = tree.node(v)
        TS, axes = contracted_tensor(T, tree, drm, tree.sttnn_reuse(v))
        pos = axes.index(("m", nd.lo))
        k = nd.hi - nd.lo
        perm = list(range(pos, pos + k)) + [i for i in range(TS.ndim) if not pos <= i < pos + k]
        U = np.transpose(TS, perm).reshape(nd.n, -1)
        G = U @ sttnn_xt(tree, drm, v, axes)
        Om[v] = drm.Yt(v).T @ G
        Ps[v] = G if nd.is_leaf else _psi_internal(tree, drm, v, G)
    return Om, Ps, psi_root(T, tree, drm)


def effective_x(tree, drm, v):
    """X_t^eff over the original complement modes with T_{S_t}^(t) X_t =
    T^(t) X_t^eff: a contracted group s contributes Y_s XT_s (Sec. 6.3, the
    term T^(l,k)(I x Y x ... x I) X_{l,k})."""
    nd = tree.node(v)
    t = set(range(nd.lo, nd.hi))
    S = sorted(tree.sttnn_reuse(v), key=lambda s: tree.node(s).lo)
    blocks, mu = [], 0
    while mu < tree.d:
        grp = [s for s in S if tree.node(s).lo == mu]
        if mu in t:
            mu += 1
            continue
        if grp:
            s = grp[0]
            blocks.append(drm.Yt(s) @ drm.XT[s][:, :nd.r])
            mu = tree.node(s).hi
        else:
            blocks.append(drm.X[mu][:, :nd.r])
            mu += 1
    if drm.in_left(v):
        # the R modes enter as the rounded block B_R
        nR = len(drm.Rmodes)
        blocks = blocks[:len(blocks) - nR] + [drm.BRX[:, :nd.r]]
    return kr(blocks)
