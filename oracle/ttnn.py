"""TTNN: DRMs, sketch phase, recovery phase, reconstruction, projector form.
ORACLE: test infrastructure only.

Layout convention of this library (the paper's matricization, Sec. 3, is
column-major; every sketch below is defined by index sums, so the convention
only fixes how indices are flattened): tensors are row-major (last mode
fastest); the unfolding T^(t) has rows indexed by t's modes and columns by the
remaining modes, each flattened row-major in increasing mode order; the
Khatri-Rao product kr(F_1, ..., F_k)[(i_1..i_k), j] = prod_m F_m[i_m, j] and
the Kronecker product are flattened the same way.

DRMs (Sec. 7, Khatri-Rao sketchings, with per-node ranks): per-mode factors
X_mu (n_mu x r_max), Y_mu (n_mu x s_max) drawn by ``philox.gaussian_matrix``
and rounded to the run's number format q (the rounded matrix *is* the DRM);
X_t = kr of the complement modes' X_mu, first r_t columns;
Y_t = kr of t's Y_mu, first s_t columns.
The tensor-core side of the first-level pass multiplies A by KR blocks that
must themselves be stored in q, so those blocks are rounded once more after
the exact binary64 product (left-to-right over increasing modes):
  B_R = q(kr(X_mu : mu in R)),  B_L = q(kr(X_mu : mu in L)),
  and Y_c of the root child on the pass's Y side = q(kr(Y_mu : mu in c)),
where L / R are the root-children groups of ``Tree.root_split``.  For q = f64
the extra rounding is the identity.  Each node's X_t and Y_t are single
matrices used consistently by Omega_t, Psi_t and the parent's Psi.
"""
import numpy as np

from . import philox, quant


# ---------------------------------------------------------------------------
# small tensor helpers
# ---------------------------------------------------------------------------
def kr(mats):
    """Column-wise Khatri-Rao product, first factor's row index slowest."""
    out = np.asarray(mats[0], dtype=np.float64)
    for m in mats[1:]:
        m = np.asarray(m, dtype=np.float64)
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, out.shape[1])
    return out


def unfold(T, lo, hi):
    """T^(t) for the contiguous mode range [lo, hi): (n_t, n_{D\\t})."""
    d = T.ndim
    perm = list(range(lo, hi)) + list(range(0, lo)) + list(range(hi, d))
    nt = int(np.prod(T.shape[lo:hi], dtype=np.int64))
    return np.transpose(T, perm).reshape(nt, -1)


def contract_axis(A, axis, M):
    """A with axis `axis` contracted against the rows of M; M's column index
    takes the axis' place: out[..., b, ...] = sum_i A[..., i, ...] M[i, b]."""
    out = np.tensordot(A, M, axes=([axis], [0]))
    return np.moveaxis(out, -1, axis)


# ---------------------------------------------------------------------------
# DRMs
# ---------------------------------------------------------------------------
def pass_block(factors, fmt):
    """A Khatri-Rao block that multiplies the dense tensor on the tensor cores
    (Sec. 7 Khatri-Rao DRMs, stored in the plan's format): the exact binary64
    product of the (already rounded) per-mode factors, rounded once to fmt.
    Each entry is within fmt's unit roundoff (relative, normal range) of the
    exact product; for fmt = "f64" it is the exact product."""
    return quant.round_to(kr(factors), fmt)


class Drm:
    """Per-mode factors and the per-node DRMs of one plan (Sec. 7)."""

    def __init__(self, tree, seed, fmt="f64", variant="ttnn"):
        self.tree, self.seed, self.fmt, self.variant = tree, int(seed), fmt, variant
        sk = tree.sketched()
        self.rmax = max([tree.node(v).r for v in sk] + [1])
        self.smax = max([tree.node(v).s for v in sk] + [1])
        q = lambda a: quant.round_to(a, fmt)
        self.X = [q(philox.gaussian_matrix(seed, philox.KIND_X, mu, n, self.rmax))
                  for mu, n in enumerate(tree.dims)]
        self.Y = [q(philox.gaussian_matrix(seed, philox.KIND_Y, mu, n, self.smax))
                  for mu, n in enumerate(tree.dims)]
        # STTNN right factors on contracted groups, keyed by node (lex index)
        self.XT = {}
        for v in sk:
            nd = tree.node(v)
            self.XT[v] = q(philox.gaussian_matrix(seed, philox.KIND_XT, nd.lex, nd.s, self.rmax))
        root = tree.node(tree.root)
        a, yside = tree.root_split("sttnn" if variant == "sttnn" else "ttnn")
        self.split, self.yside = a, yside
        ch = root.children
        self.Lch, self.Rch = ch[:a], ch[a:]
        self.Lmodes = list(range(tree.node(ch[0]).lo, tree.node(ch[a - 1]).hi))
        self.Rmodes = list(range(tree.node(ch[a]).lo, tree.node(ch[-1]).hi))
        ygrp = self.Rch if yside == "R" else self.Lch
        self.ychild = ygrp[0] if len(ygrp) == 1 else None
        self._blocks = {}

    def _block(self, key, factors):
        # "round": sketches of a TTN input (Sec. 7) never multiply a dense A
        # on the tensor cores, so no KR block is rounded a second time.  The
        # blocks are formed on first use (a TTN input never needs them).
        if key not in self._blocks:
            self._blocks[key] = (kr(factors) if self.variant == "round"
                                 else pass_block(factors, self.fmt))
        return self._blocks[key]

    @property
    def BRX(self):
        return self._block("BRX", [self.X[mu] for mu in self.Rmodes])

    @property
    def BLX(self):
        return self._block("BLX", [self.X[mu] for mu in self.Lmodes])

    @property
    def Yside(self):
        if self.ychild is None or self.tree.node(self.ychild).identity:
            return None
        c = self.tree.node(self.ychild)
        return self._block("Yside", [self.Y[mu] for mu in range(c.lo, c.hi)])

    def in_left(self, v):
        return self.tree.node(v).lo < self.Rmodes[0]

    def Yt(self, v):
        """Y_t (n_t x s_t); the identity for identity nodes."""
        nd = self.tree.node(v)
        if nd.identity:
            return np.eye(nd.n)
        if v == self.ychild:
            return self.Yside[:, :nd.s]
        return kr([self.Y[mu] for mu in range(nd.lo, nd.hi)])[:, :nd.s]

    def Xt(self, v):
        """X_t (n_{D\\t} x r_t) of TTNN."""
        nd = self.tree.node(v)
        t = set(range(nd.lo, nd.hi))
        if self.in_left(v):
            mats = [self.X[mu] for mu in self.Lmodes if mu not in t] + [self.BRX]
        else:
            mats = [self.BLX] + [self.X[mu] for mu in self.Rmodes if mu not in t]
        return kr(mats)[:, :nd.r]


# ---------------------------------------------------------------------------
# sketch phase (Sec. 4)
# ---------------------------------------------------------------------------
def _psi_internal(tree, drm, v, G):
    """(kron_c Y_c)^T applied to G = T^(t) X_t, returned as (s'_c1..s'_cm, r_t)."""
    nd = tree.node(v)
    shape = [tree.node(c).n for c in nd.children] + [G.shape[1]]
    P = G.reshape(shape)
    for k, c in enumerate(nd.children):
        P = contract_axis(P, k, drm.Yt(c))
    return P


def psi_root(T, tree, drm):
    """Psi_root = (Y_{1,1}^T x ... x Y_{1,m}^T) T^D (Sec. 4), as (s'_c1..s'_cm)."""
    root = tree.node(tree.root)
    P = T.reshape([tree.node(c).n for c in root.children])
    for k, c in enumerate(root.children):
        P = contract_axis(P, k, drm.Yt(c))
    return P


def sketch_ttnn(T, tree, drm):
    """All TTNN sketches of T (Sec. 4, sketch phase).

    Returns (Omega, Psi, Psi_root): dicts keyed by user node index.
    Omega_t = Y_t^T T^(t) X_t  (s_t x r_t);
    Psi_t   = (kron of the children's Y)^T T^(t) X_t  (internal t),
              T^(t) X_t (leaf t);
    Psi_root = (kron of the root children's Y)^T T^D.
    """
    T = np.asarray(T, dtype=np.float64)
    Om, Ps = {}, {}
    for v in tree.sketched():
        nd = tree.node(v)
        G = unfold(T, nd.lo, nd.hi) @ drm.Xt(v)
        Om[v] = drm.Yt(v).T @ G
        Ps[v] = G if nd.is_leaf else _psi_internal(tree, drm, v, G)
    return Om, Ps, psi_root(T, tree, drm)


def sketch_linear_combination(parts, lambdas, tree, drm, sketch=sketch_ttnn):
    """Sum_i lambda_i sketch(H_i) (Sec. 4, streaming by linearity)."""
    acc = None
    for H, lam in zip(parts, lambdas):
        Om, Ps, Pr = sketch(H, tree, drm)
        if acc is None:
            acc = ({k: lam * x for k, x in Om.items()}, {k: lam * x for k, x in Ps.items()}, lam * Pr)
        else:
            for k in Om:
                acc[0][k] = acc[0][k] + lam * Om[k]
                acc[1][k] = acc[1][k] + lam * Ps[k]
            acc = (acc[0], acc[1], acc[2] + lam * Pr)
    return acc


# ---------------------------------------------------------------------------
# recovery phase (Sec. 4; stabilised least squares with eps = 10 u ||R||_2)
# ---------------------------------------------------------------------------
U_DEFAULT = 2.0 ** -52      # "machine precision" read as MATLAB eps


def qr_pos(A):
    """Economy Householder QR with diag(R) >= 0 (the unique factorisation of a
    full-column-rank A)."""
    Q, R = np.linalg.qr(A, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn[None, :], R * sgn[:, None]


def eps_pinv(R, eps_factor=10.0, u=U_DEFAULT):
    """R_eps^+ = V_1 Sigma_1^-1 U_1^T keeping singular values > eps,
    eps = eps_factor * u * ||R||_2 (eqs. (stabilized_nystrom) and Sec. 4)."""
    Uu, sv, Vt = np.linalg.svd(R)
    if sv.size == 0:
        return np.zeros(R.T.shape), 0
    eps = eps_factor * u * sv[0]
    keep = sv > eps
    Rp = (Vt[keep].T / sv[keep][None, :]) @ Uu[:, keep].T
    return Rp, int(keep.sum())


def eps_pinv_factors(R, eps_factor=10.0, u=U_DEFAULT):
    """R_eps^+ = A U_1^T split into A = V_1 Sigma_1^-1 (r x k) and U_1 (r x k),
    the k singular values > eps kept in decreasing order."""
    Uu, sv, Vt = np.linalg.svd(R)
    eps = eps_factor * u * (sv[0] if sv.size else 0.0)
    keep = sv > eps
    return Vt[keep].T / sv[keep][None, :], Uu[:, keep]


def recover(tree, Om, Ps, Pr, eps_factor=10.0, u=U_DEFAULT, truncate=False):
    """Cores B_t from the sketches (Sec. 4 recovery phase, Algorithm 2).

    [Q_t, R_t] = qr(Omega_t);  leaf: B_t = Psi_t R_t,eps^+;
    internal: B_t = (kron_c Q_c)^T Psi_t R_t,eps^+ (the *children's* Q, which
    is what the dimensions and Algorithm 2's W_{l,k} require);
    root: B = (kron_c Q_c)^T Psi_root.  Identity nodes: Q = I, core = I.
    Cores use the axis order root (r_c1..r_cm), transfer (r_t, r_c1..r_cm),
    leaf (r_t, n_mu1..n_mus).  Returns (cores, info) keyed by user index;
    info[v] = (numerical rank kept by the eps-pseudo-inverse).  truncate:
    the rank axes carry the kept ranks (the same tensor, eq.
    (stabilized_nystrom) with the dropped directions cut).
    """
    Q, Rp, info = {}, {}, {}
    for v in tree.sketched():
        Q[v], R = qr_pos(Om[v])
        Rp[v], info[v] = eps_pinv(R, eps_factor, u)
        if truncate:
            # eps-truncated output: R_eps^+ = (V_1 Sigma_1^-1) U_1^T with U_1
            # moved into Q_v, so node v's rank axis carries the kept rank only
            A, U1 = eps_pinv_factors(R, eps_factor, u)
            Q[v], Rp[v] = Q[v] @ U1, A

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
            B = Ps[v] @ Rp[v]                              # (n_t, r_t)
            cores[v] = B.T.reshape([B.shape[1]] + tree.dims[nd.lo:nd.hi])
        else:
            P = Ps[v]
            for k, c in enumerate(nd.children):
                P = contract_axis(P, k, Qc(c))             # Q_c^T on axis k
            P = contract_axis(P, P.ndim - 1, Rp[v])        # ... R_eps^+ on the right
            cores[v] = np.moveaxis(P, -1, 0)
    root = tree.node(tree.root)
    P = Pr
    for k, c in enumerate(root.children):
        P = contract_axis(P, k, Qc(c))
    cores[tree.root] = P
    return cores, info


def reconstruct(tree, cores):
    """Dense tensor of a TTN (Def. "Tree tensor network format", eq.
    (tree_tensor_def)): contract each transfer tensor with its children."""
    def full(v):
        nd = tree.node(v)
        if nd.is_leaf:
            return cores[v]
        out = cores[v]
        for c in nd.children:
            out = np.tensordot(out, full(c), axes=([1], [0]))
        return out
    root = tree.node(tree.root)
    out = cores[tree.root]
    for c in root.children:
        out = np.tensordot(out, full(c), axes=([0], [0]))
    return out


def ttnn(T, tree, seed, fmt="f64", eps_factor=10.0, u=U_DEFAULT):
    """Algorithm 2 end to end: DRMs, sketches, recovery.  Returns (cores, drm)."""
    drm = Drm(tree, seed, fmt, "ttnn")
    Om, Ps, Pr = sketch_ttnn(T, tree, drm)
    cores, _ = recover(tree, Om, Ps, Pr, eps_factor, u)
    return cores, drm


# ---------------------------------------------------------------------------
# projector form (eq. (TTNN approximant projector)) -- tiny tensors only
# ---------------------------------------------------------------------------
def projector(U, X, Y):
    """P = U X (Y^T U X)^+ Y^T (eq. (projectors)), Moore-Penrose pseudo-inverse."""
    UX = U @ X
    return UX @ np.linalg.pinv(Y.T @ UX) @ Y.T


def apply_on_modes(T, lo, hi, P):
    """T with P (n_t x n_t) applied on the left of its unfolding T^(t)."""
    d = T.ndim
    perm = list(range(lo, hi)) + list(range(0, lo)) + list(range(hi, d))
    Tp = np.transpose(T, perm)
    sh = Tp.shape
    out = (P @ Tp.reshape(P.shape[1], -1)).reshape(sh)
    return np.transpose(out, np.argsort(perm))


def projector_approximant(T, tree, projectors):
    """(prod_{l=L..1} kron_k P_{l,k}) T^D: level-1 projectors act first."""
    out = np.asarray(T, dtype=np.float64)
    for lvl in range(1, tree.depth + 1):
        for v in tree.lex:
            nd = tree.node(v)
            if nd.level == lvl and v in projectors:
                out = apply_on_modes(out, nd.lo, nd.hi, projectors[v])
    return out


def ttnn_projectors(T, tree, drm):
    """P_t of every sketched node (eq. (projectors)) with the plan's DRMs."""
    return {v: projector(unfold(T, tree.node(v).lo, tree.node(v).hi), drm.Xt(v), drm.Yt(v))
            for v in tree.sketched()}


class DenseDrm:
    """Independent unstructured Gaussian DRMs X_{l,k} (n_{D\\t} x r_t) and
    Y_{l,k} (n_t x s_t) of eq. (sketch), as Thm 6.6 assumes (Philox kinds
    DX / DY keyed by the node's lexicographic index), rounded to the run's
    number format (the rounded matrix is the DRM)."""

    def __init__(self, tree, seed, fmt="f64"):
        self.tree, self.seed, self.fmt = tree, int(seed), fmt

    def Yt(self, v):
        nd = self.tree.node(v)
        if nd.identity:
            return np.eye(nd.n)
        return quant.round_to(philox.gaussian_matrix(self.seed, philox.KIND_DY, nd.lex, nd.n, nd.s),
                              self.fmt)

    def Xt(self, v):
        nd = self.tree.node(v)
        return quant.round_to(philox.gaussian_matrix(self.seed, philox.KIND_DX, nd.lex,
                                                     self.tree.N // nd.n, nd.r), self.fmt)
