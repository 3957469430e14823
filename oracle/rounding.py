"""Sketches of a tensor already in TTN format (Sec. 7, "Structured sketchings
for TTNN and STTNN").  ORACLE: test infrastructure only.

With Khatri-Rao DRMs every sketch entry is a contraction of the input network
with rank-one vectors (the entrywise formulas for Omega_{1,1}, Psi_{1,1} of
Sec. 7), so the sketches are formed by two sweeps over the input cores C_t
(axis order: root (R_c1..R_cm), transfer (R_t, R_c1..R_cm), leaf (R_t, n..)):

up   UX_t[a, j] = sum C_t[a, b_1..b_m] prod_k UX_{c_k}[b_k, j]
     (leaf: sum_i C_t[a, i] kr(X_mu : mu in t)[i, j]); UK_t likewise with the
     Y_mu (the Khatri-Rao Y_t of t itself, columns shared).
down E_{c_k}[b_k, j] = sum C_t[a, b..] E_t[a, j] prod_{k' != k} UX_{c_k'}[b_k', j]
     (root: no E_t factor).
Omega_t = UK_t[:, :s_t]^T E_t[:, :r_t];   Psi_leaf = C_t^T E_t;
Psi_t[a_1..a_m, j] = sum C_t[a, b..] E_t[a, j] prod_k UY_{c_k}[b_k, a_k];
Psi_root[a_1..a_m] = sum C_root[b..] prod_k UY_{c_k}[b_k, a_k],
with UY_c = UK_c[:, :s_c], or the raw leaf core C_c for an identity node c.

The DRMs are those of ``ttnn.Drm(..., variant="round")`` (no second rounding
of KR blocks: nothing here multiplies a dense tensor on tensor cores).
"""
import numpy as np

from .ttnn import kr

_B = "bcdefghi"      # child rank letters
_O = "pqstuvwx"      # child output (sketch) letters


def _up(C, mats):
    """sum_b C[a, b_1..b_m] prod_k mats[k][b_k, j]  ->  (a, j)."""
    m = len(mats)
    spec = "a" + _B[:m] + "," + ",".join(_B[k] + "j" for k in range(m)) + "->aj"
    return np.einsum(spec, C, *mats, optimize=True)


def _down(C, k, ux, Et):
    """E_{c_k}[b_k, j] from the parent's core, E_t (None at the root) and the
    siblings' UX."""
    m = len(ux)
    ins, ops = [], []
    if Et is None:
        ins.append(_B[:m])
        ops.append(C)
    else:
        ins += ["a" + _B[:m], "aj"]
        ops += [C, Et]
    for i in range(m):
        if i != k:
            ins.append(_B[i] + "j")
            ops.append(ux[i])
    return np.einsum(",".join(ins) + "->" + _B[k] + "j", *ops, optimize=True)


def _psi(C, Et, uy):
    """sum_{a,b} C[a, b..] E_t[a, j] prod_k uy[k][b_k, o_k] -> (o_1..o_m, j);
    at the root (Et None) -> (o_1..o_m)."""
    m = len(uy)
    ins, ops = [], []
    if Et is None:
        ins.append(_B[:m])
        ops.append(C)
        out = _O[:m]
    else:
        ins += ["a" + _B[:m], "aj"]
        ops += [C, Et]
        out = _O[:m] + "j"
    for k in range(m):
        ins.append(_B[k] + _O[k])
        ops.append(uy[k])
    return np.einsum(",".join(ins) + "->" + out, *ops, optimize=True)


def sketch_ttn_input(cores_in, tree, drm):
    """All sketches of the TTN-format tensor given by cores_in (user-indexed),
    for the target ranks of `tree` and the DRMs of `drm` (same tree shape).
    Same return convention as ttnn.sketch_ttnn."""
    C = {v: np.asarray(c, dtype=np.float64) for v, c in cores_in.items()}
    UX, UK = {}, {}
    for v in reversed(tree.lex):               # children before parents
        if v == tree.root:
            continue
        nd = tree.node(v)
        if nd.is_leaf:
            C2 = C[v].reshape(C[v].shape[0], -1)
            UX[v] = C2 @ kr([drm.X[mu] for mu in range(nd.lo, nd.hi)])
            UK[v] = C2 @ kr([drm.Y[mu] for mu in range(nd.lo, nd.hi)])
        else:
            UX[v] = _up(C[v], [UX[c] for c in nd.children])
            UK[v] = _up(C[v], [UK[c] for c in nd.children])

    def uy(c):
        nc = tree.node(c)
        if nc.identity:
            return C[c].reshape(C[c].shape[0], -1)
        return UK[c][:, :nc.s]

    E = {}
    for v in tree.lex:                          # parents before children
        nd = tree.node(v)
        if nd.is_leaf:
            continue
        ux = [UX[c] for c in nd.children]
        for k, c in enumerate(nd.children):
            E[c] = _down(C[v], k, ux, None if v == tree.root else E[v])
    Om, Ps = {}, {}
    for v in tree.sketched():
        nd = tree.node(v)
        Et = E[v][:, :nd.r]
        Om[v] = UK[v][:, :nd.s].T @ Et
        if nd.is_leaf:
            Ps[v] = C[v].reshape(C[v].shape[0], -1).T @ Et
        else:
            Ps[v] = _psi(C[v], Et, [uy(c) for c in nd.children])
    root = tree.node(tree.root)
    Pr = _psi(C[tree.root], None, [uy(c) for c in root.children])
    return Om, Ps, Pr


# ---------------------------------------------------------------------------
# TTN-format inner products and entries (tensors too large to form densely)
# ---------------------------------------------------------------------------
def ttn_inner(tree, A, B):
    """<T_A, T_B> of two TTNs on the same tree (cores in the axis order
    above; edge ranks may differ between A and B), by contracting leaves
    upward: M_t[a, a'] = sum A_t[a, ..] B_t[a', ..] prod_c M_c[b_c, b'_c]
    (leaf: A_t B_t^T over its modes), and at the root the scalar with no
    parent axis.  Definition: the Frobenius inner product of the two dense
    tensors (Def. "Tree tensor network format")."""
    M = {}
    for v in reversed(tree.lex):
        nd = tree.node(v)
        a = np.asarray(A[v], dtype=np.float64)
        b = np.asarray(B[v], dtype=np.float64)
        if nd.is_leaf:
            M[v] = a.reshape(a.shape[0], -1) @ b.reshape(b.shape[0], -1).T
            continue
        m = len(nd.children)
        head = "" if v == tree.root else "a"
        headb = "" if v == tree.root else "z"
        bl, br = _B[:m], _O[:m]
        ins = [head + bl, headb + br] + [bl[k] + br[k] for k in range(m)]
        ops = [a, b] + [M[c] for c in nd.children]
        out = head + headb
        M[v] = np.einsum(",".join(ins) + "->" + out, *ops, optimize=True)
    return float(M[tree.root])


def ttn_entries(tree, cores, idx):
    """Entries of the TTN at the multi-indices idx (k x d integer array):
    each leaf core read at the leaf's modes, then each transfer tensor
    contracted with its children's vectors, per sample."""
    idx = np.asarray(idx)
    dims = tree.dims

    def val(v):
        nd = tree.node(v)
        C = np.asarray(cores[v], dtype=np.float64)
        if nd.is_leaf:
            flat = np.ravel_multi_index(tuple(idx[:, nd.lo:nd.hi].T), dims[nd.lo:nd.hi])
            return C.reshape(C.shape[0], -1)[:, flat].T            # (k, R_v)
        vecs = [val(c) for c in nd.children]
        m = len(vecs)
        head = "" if v == tree.root else "a"
        spec = head + _B[:m] + "," + ",".join("s" + _B[k] for k in range(m)) + "->s" + head
        return np.einsum(spec, C, *vecs, optimize=True)

    return val(tree.root)


# ---------------------------------------------------------------------------
# TTN-SVD of a network (the hierarchical SVD of Sec. 8's comparisons, on a
# tensor given in TTN format)
# ---------------------------------------------------------------------------
def _axes_except(nd_ndim, a):
    return [i for i in range(nd_ndim) if i != a]


def ttn_svd(tree, cores):
    """The TTN-SVD approximant (every non-root node t projected onto the r_t
    dominant left singular vectors of the unfolding T^(t), as
    ``baselines.hsvd`` does on a dense tensor), computed without forming T:
    1. orthogonalise the network leaves first (QR of each core against its
       parent axis, the R factor absorbed by the parent), so that the subtree
       of t spans T^(t)'s columns with an orthonormal basis U_t;
    2. top-down Gram matrices G_t = M_t M_t^T of the rest of the network
       (T^(t) = U_t M_t), so that the left singular vectors of T^(t) are
       U_t W_t with W_t the dominant eigenvectors of G_t;
    3. W_t W_t^T inserted on every edge (the orthogonal projector P_t acts on
       that edge only), written as cores of ranks r_t.
    Returns (cores, sigma) with sigma[t] the singular values of T^(t)."""
    C = {v: np.array(c, dtype=np.float64) for v, c in cores.items()}
    root = tree.root
    # 1. orthogonalise: children before parents
    for v in reversed(tree.lex):
        if v == root:
            continue
        nd = tree.node(v)
        X = C[v]
        M = np.moveaxis(X, 0, -1).reshape(-1, X.shape[0])       # (rest, R_v)
        Q, R = np.linalg.qr(M)
        k = Q.shape[1]
        C[v] = np.moveaxis(Q.reshape(list(np.moveaxis(X, 0, -1).shape[:-1]) + [k]), -1, 0)
        par = tree.node(nd.parent)
        a = par.children.index(v) + (0 if nd.parent == root else 1)
        C[nd.parent] = np.moveaxis(np.tensordot(C[nd.parent], R, axes=([a], [1])), -1, a)
    # 2. Gram matrices of the rest of the network, parents before children
    G = {}
    for v in tree.lex:
        nd = tree.node(v)
        if nd.is_leaf:
            continue
        X = C[v]
        head = 0 if v == root else 1
        Xg = X if v == root else np.tensordot(G[v], X, axes=([1], [0]))
        for k, c in enumerate(nd.children):
            a = head + k
            G[c] = np.tensordot(X, Xg, axes=(_axes_except(X.ndim, a), _axes_except(X.ndim, a)))
    # 3. projectors on the edges
    W, sig = {}, {}
    for v in tree.nonroot():
        nd = tree.node(v)
        ev, V = np.linalg.eigh((G[v] + G[v].T) / 2)
        order = np.argsort(ev)[::-1]
        sig[v] = np.sqrt(np.maximum(ev[order], 0.0))
        W[v] = V[:, order[:min(nd.r, V.shape[1])]]
    out = {}
    for v in tree.lex:
        nd = tree.node(v)
        X = C[v]
        head = 0 if v == root else 1
        if v != root:
            X = np.tensordot(W[v].T, X, axes=([1], [0]))
        if not nd.is_leaf:
            for k, c in enumerate(nd.children):
                X = np.moveaxis(np.tensordot(X, W[c], axes=([head + k], [0])), -1, head + k)
        out[v] = X
    return out, sig
