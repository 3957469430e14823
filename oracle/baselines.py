"""Textbook methods the paper compares with or specialises to.  ORACLE: test
infrastructure only.  Each is written from its own defining formula, not
through the TTNN code path, so that the special-case pins are independent.

* gn(A, X, Y)            generalized Nystrom, Algorithm 1 (Sec. 2):
                         (A X R^-1)(Q^T Y^T A) with QR = Y^T A X.
* mln(T, X, Y)           multilinear Nystrom, eq. (MLN): T x_mu P_{mu}.
* stta(T, X, Y)          streaming TT approximation, eq. (STTA):
                         (P_1 x I)...(P_{1:d-2} x I) P_{1:d-1} T^{1..d-1}.
* hsvd(T, tree)          TTN-SVD (Sec. 8): the hierarchical SVD of Grasedyck
                         (ref. [grasedyck2010hierarchical]) with each node's
                         orthogonal projector U_t U_t^T onto the r_t dominant
                         left singular vectors of T^(t), level 1 first.
* tt_svd(T, ranks)       TT-SVD of Oseledets (sequential truncated SVDs).
* svd_tail(M, r)         sqrt(sum_{i > r} sigma_i(M)^2), the Eckart-Young error.
"""
import numpy as np

from .ttnn import unfold, apply_on_modes


def svd_tail(M, r):
    s = np.linalg.svd(M, compute_uv=False)
    return float(np.sqrt(np.sum(s[r:] ** 2)))


def gn(A, X, Y):
    """Algorithm 1: economy QR of Y^T A X, return (A X R^-1)(Q^T Y^T A)."""
    AX = A @ X
    YtA = Y.T @ A
    Q, R = np.linalg.qr(Y.T @ AX, mode="reduced")
    return np.linalg.solve(R.T, AX.T).T @ (Q.T @ YtA)


def _proj(U, X, Y):
    UX = U @ X
    return UX @ np.linalg.pinv(Y.T @ UX) @ Y.T


def mln(T, X, Y):
    """eq. (MLN): T x_{mu=1}^d P_{mu}, P_mu = T^mu X_mu (Y_mu^T T^mu X_mu)^+ Y_mu^T,
    with X[mu] (n_{D\\mu} x r_mu) and Y[mu] (n_mu x s_mu)."""
    out = np.asarray(T, dtype=np.float64)
    for mu in range(T.ndim):
        P = _proj(unfold(T, mu, mu + 1), X[mu], Y[mu])
        out = apply_on_modes(out, mu, mu + 1, P)
    return out


def stta(T, X, Y):
    """eq. (STTA): P_{1:k} = T^{1..k} X_k (Y_k^T T^{1..k} X_k)^+ Y_k^T for
    k = 1..d-1 (X[k-1]: n_{k+1..d} x r, Y[k-1]: n_{1..k} x s), applied to the
    unfolding T^{1..d-1}: the largest k first, each smaller one with (P x I)."""
    T = np.asarray(T, dtype=np.float64)
    d = T.ndim
    out = T
    for k in range(d - 1, 0, -1):
        P = _proj(unfold(T, 0, k), X[k - 1], Y[k - 1])
        out = apply_on_modes(out, 0, k, P)
    return out


def hsvd(T, tree):
    """TTN-SVD: orthogonal HSVD projectors of every non-root, non-identity node."""
    T = np.asarray(T, dtype=np.float64)
    proj = {}
    for v in tree.sketched():
        nd = tree.node(v)
        U, _, _ = np.linalg.svd(unfold(T, nd.lo, nd.hi), full_matrices=False)
        Ur = U[:, :nd.r]
        proj[v] = Ur @ Ur.T
    out = T
    for lvl in range(1, tree.depth + 1):
        for v in tree.lex:
            if v in proj and tree.node(v).level == lvl:
                nd = tree.node(v)
                out = apply_on_modes(out, nd.lo, nd.hi, proj[v])
    return out


def tt_svd(T, ranks):
    """TT-SVD (Oseledets 2011): left-to-right truncated SVDs of the remainder.
    ranks[k] is the TT rank between modes k and k+1 (length d-1)."""
    T = np.asarray(T, dtype=np.float64)
    dims = T.shape
    d = len(dims)
    cores, C, rprev = [], T.reshape(dims[0], -1), 1
    for k in range(d - 1):
        C = C.reshape(rprev * dims[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        r = min(ranks[k], s.size)
        cores.append(U[:, :r].reshape(rprev, dims[k], r))
        C = s[:r, None] * Vt[:r]
        rprev = r
    cores.append(C.reshape(rprev, dims[-1], 1))
    out = cores[0]
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([-1], [0]))
    return out.reshape(dims)


def ttn_hmt(T, tree, drm):
    """TTN-HMT (Sec. 8): the TTN-SVD with each SVD replaced by the HMT range
    finder on the same right sketches X_t as TTNN: Q_t = orth(T^(t) X_t)
    (n_t x r_t), P_t = Q_t Q_t^T, and the approximant (prod over levels of
    kron_t P_t) T in TTN format -- leaf core Q_t^T, transfer core
    (kron_c Q_c)^T Q_t as (r_t, r_c1, .., r_cm), root core (kron_c Q_c)^T T^D.
    Two passes over T: the sketches, then the root core.  Identity nodes keep
    Q = I.  Returns cores keyed by user index (the library's axis order)."""
    from .ttnn import contract_axis
    T = np.asarray(T, dtype=np.float64)
    Q = {}
    for v in tree.sketched():
        nd = tree.node(v)
        Q[v], _ = np.linalg.qr(unfold(T, nd.lo, nd.hi) @ drm.Xt(v), mode="reduced")

    def Qc(c):
        nd = tree.node(c)
        return np.eye(nd.n) if nd.identity else Q[c]

    cores = {}
    for v in tree.nonroot():
        nd = tree.node(v)
        if nd.identity:
            cores[v] = np.eye(nd.n).reshape([nd.n] + tree.dims[nd.lo:nd.hi])
            continue
        if nd.is_leaf:
            cores[v] = Q[v].T.reshape([Q[v].shape[1]] + tree.dims[nd.lo:nd.hi])
            continue
        P = Q[v].reshape([tree.node(c).n for c in nd.children] + [Q[v].shape[1]])
        for k, c in enumerate(nd.children):
            P = contract_axis(P, k, Qc(c))
        cores[v] = np.moveaxis(P, -1, 0)
    root = tree.node(tree.root)
    P = T.reshape([tree.node(c).n for c in root.children])
    for k, c in enumerate(root.children):
        P = contract_axis(P, k, Qc(c))
    cores[tree.root] = P
    return cores
