"""Error bounds of Sec. 6.  ORACLE: test infrastructure only.

Per non-root node t (Thm 6.4), with Q_t = orth(T^(t) X_t) and V_t the r^_t
dominant right singular vectors of T^(t):
  eta_t = 1 + ||(Y_t^T Q_t)^+ Y_t^T Q_t,perp||_2
  tau_t = sqrt(1 + ||(Y_t^T Q_t)^+ Y_t^T Q_t,perp||_2^2)
  rho_t = sqrt(1 + ||V_t,perp^T X_t (V_t^T X_t)^+||_2^2)
  e_t   = ||(I - P_t) T^(t)||_F   (the GN error of node t)
Lemmas 6.2-6.3:  ||T - T^|| <= sum_t [prod_{u > t} eta_u] e_t, the product over
the nodes after t in the lexicographic order; Thm 6.4 then bounds
e_t <= rho_t tau_t sqrt(sum_{i > r^_t} sigma_i(T^(t))^2).
Thm 6.6 (independent standard Gaussian DRMs, p_t >= 2, r^_t < r_t - 1):
  E||T - T^|| <= sum_t [prod_{u > t} c_u] c'_t sqrt(sum_{i > r^_t} sigma_i^2),
  c = 1 + sqrt(r/(p-1)),  c' = sqrt(1 + r/(p-1)) sqrt(1 + r^/(r - r^ - 1)).
Thm 6.7 (STTNN) is Thm 6.4 with Q_t = orth(T_{S_t}^(t) X_t) and P_t the STTNN
projection.
"""
import numpy as np

from .ttnn import unfold
from .baselines import svd_tail


def _complement(Q):
    """Orthonormal basis of range(Q)^perp."""
    n, r = Q.shape
    U, _, _ = np.linalg.svd(Q, full_matrices=True)
    return U[:, r:]


def node_factors(U, X, Y, rhat, UXS=None):
    """(eta, tau, rho, e) of one node; U = T^(t), UXS = the sketched range
    T_{S}^(t) X (STTNN) or None for U X (TTNN)."""
    UX = U @ X if UXS is None else UXS
    Q, _ = np.linalg.qr(UX, mode="reduced")
    Qp = _complement(Q)
    M = np.linalg.pinv(Y.T @ Q) @ (Y.T @ Qp)
    g = np.linalg.norm(M, 2) if M.size else 0.0
    eta, tau = 1.0 + g, np.sqrt(1.0 + g * g)
    _, _, Vt = np.linalg.svd(U, full_matrices=True)
    V, Vp = Vt[:rhat].T, Vt[rhat:].T
    W = (Vp.T @ X) @ np.linalg.pinv(V.T @ X)
    h = np.linalg.norm(W, 2) if W.size else 0.0
    rho = np.sqrt(1.0 + h * h)
    P = UX @ np.linalg.pinv(Y.T @ UX) @ Y.T
    e = np.linalg.norm(U - P @ U)
    return eta, tau, rho, e


def deterministic(T, tree, drm, rhat, sttnn_ranges=None):
    """(sum_t [prod eta] e_t, sum_t [prod eta] rho tau E_svd(t)) of Thm 6.4
    (or 6.7 when sttnn_ranges maps node -> T_{S_t}^(t) X_t)."""
    nodes = tree.sketched()
    fac = {}
    for v in nodes:
        nd = tree.node(v)
        U = unfold(T, nd.lo, nd.hi)
        UXS = None if sttnn_ranges is None else sttnn_ranges[v]
        fac[v] = node_factors(U, drm.Xt(v), drm.Yt(v), rhat[v], UXS) + (svd_tail(U, rhat[v]),)
    b1 = b2 = 0.0
    for i, v in enumerate(nodes):
        later = np.prod([fac[u][0] for u in nodes[i + 1:]]) if i + 1 < len(nodes) else 1.0
        eta, tau, rho, e, esvd = fac[v]
        b1 += later * e
        b2 += later * rho * tau * esvd
    return b1, b2


def expected(T, tree, rhat):
    """Right-hand side of Thm 6.6 (first inequality)."""
    nodes = tree.sketched()
    c = {v: 1.0 + np.sqrt(tree.node(v).r / (tree.node(v).p - 1.0)) for v in nodes}
    tot = 0.0
    for i, v in enumerate(nodes):
        nd = tree.node(v)
        r, p, rh = nd.r, nd.p, rhat[v]
        cp = np.sqrt(1.0 + r / (p - 1.0)) * np.sqrt(1.0 + rh / (r - rh - 1.0))
        later = np.prod([c[u] for u in nodes[i + 1:]]) if i + 1 < len(nodes) else 1.0
        tot += later * cp * svd_tail(unfold(T, nd.lo, nd.hi), rh)
    return tot
