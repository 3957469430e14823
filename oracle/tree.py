"""Index trees (Sec. 3, Def. "index tree", "extended index tree") and the
per-node parameters of TTNN / STTNN.  ORACLE: test infrastructure only.

Input format (the same *interface* as the C library's ``ttnn_tree``; this is an
independent implementation): ``parent[v]`` is the parent of node v (-1 for the
root); ``leaf_modes[v]`` lists the 0-based tensor modes of a leaf v (empty for
an internal node); ``identity[v]`` forces P_v = I on a leaf.

Readings of the paper (each stated once, here):
* Children partition their parent (Def. "index tree" allows a superset; a
  transfer tensor has no physical mode, so a node's modes are the union of its
  children's).  Internal nodes have at least two children.
* Every node's modes form a contiguous range and children are ordered by their
  first mode, so the row-major unfolding of a node is a plain reshape.
* Nodes are numbered lexicographically by (level l, position k) (Sec. 5 uses
  this order for STTNN); "position" is left-to-right, i.e. by first mode.
* Dummy nodes of the extended tree (identity DRMs/projectors, Sec. 4) are not
  materialised.  A leaf with r >= n_t, or flagged identity, is such a node:
  P_t = I, its core is the n_t x n_t identity, and its parent sees raw indices.
* r_t is clipped to min(n_t, n_{D\\t}) and p_t to n_t - r_t (a Gaussian sketch
  with more rows or columns than the unfolding adds nothing).
* STTNN reuse set S_t (Sec. 5 and its figure of circled/boxed nodes): the
  non-identity preceding siblings of t and of every non-root ancestor of t.
"""
import numpy as np


class Node:
    __slots__ = ("idx", "parent", "children", "lo", "hi", "level", "pos", "lex",
                 "is_leaf", "identity", "r", "p", "s", "n")

    def __repr__(self):
        return (f"Node(idx={self.idx}, modes=[{self.lo},{self.hi}), level={self.level}, "
                f"lex={self.lex}, r={self.r}, s={self.s}, identity={self.identity})")


class Tree:
    """A validated, normalised index tree with ranks and oversamples."""

    def __init__(self, parent, leaf_modes, dims, ranks, oversample, identity=None):
        parent = [int(v) for v in parent]
        n = len(parent)
        dims = [int(x) for x in dims]
        d = len(dims)
        if n == 0 or d == 0:
            raise ValueError("empty tree or tensor")
        if any(x < 1 for x in dims):
            raise ValueError("mode sizes must be >= 1")
        roots = [v for v in range(n) if parent[v] == -1]
        if len(roots) != 1:
            raise ValueError("exactly one root required")
        if any(not (-1 <= parent[v] < n) or parent[v] == v for v in range(n)):
            raise ValueError("bad parent index")
        nodes = []
        for v in range(n):
            nd = Node()
            nd.idx, nd.parent, nd.children = v, parent[v], []
            nodes.append(nd)
        for v in range(n):
            if parent[v] >= 0:
                nodes[parent[v]].children.append(v)
        self.root = roots[0]
        # acyclicity / reachability
        seen, stack = set(), [self.root]
        while stack:
            v = stack.pop()
            if v in seen:
                raise ValueError("cycle")
            seen.add(v)
            stack.extend(nodes[v].children)
        if len(seen) != n:
            raise ValueError("tree not connected")
        identity = [False] * n if identity is None else [bool(x) for x in identity]
        # mode ranges
        modes_seen = []

        def visit(v):
            nd = nodes[v]
            lm = [int(m) for m in leaf_modes[v]] if leaf_modes[v] is not None else []
            if not nd.children:
                if not lm:
                    raise ValueError("leaf without modes")
                lm = sorted(lm)
                if lm != list(range(lm[0], lm[0] + len(lm))):
                    raise ValueError("leaf modes must be contiguous")
                nd.lo, nd.hi = lm[0], lm[-1] + 1
                nd.is_leaf = True
                modes_seen.extend(lm)
                return
            if lm:
                raise ValueError("internal node with own modes")
            if len(nd.children) < 2:
                raise ValueError("internal node needs >= 2 children")
            if identity[v]:
                raise ValueError("identity flag only on leaves")
            for c in nd.children:
                visit(c)
            nd.children.sort(key=lambda c: nodes[c].lo)
            for a, b in zip(nd.children, nd.children[1:]):
                if nodes[a].hi != nodes[b].lo:
                    raise ValueError("node modes must be contiguous")
            nd.lo, nd.hi = nodes[nd.children[0]].lo, nodes[nd.children[-1]].hi
            nd.is_leaf = False

        visit(self.root)
        if sorted(modes_seen) != list(range(d)):
            raise ValueError("leaf modes must partition 0..d-1")
        self.nodes = nodes
        self.dims = dims
        self.d = d
        self.N = int(np.prod(dims, dtype=np.int64))
        # levels and lexicographic order
        order, level = [], [self.root]
        lvl = 0
        while level:
            for k, v in enumerate(level):
                nodes[v].level, nodes[v].pos = lvl, k
                order.append(v)
            level = [c for v in level for c in nodes[v].children]
            lvl += 1
        self.depth = lvl - 1
        self.lex = order                      # lex position -> user index
        for i, v in enumerate(order):
            nodes[v].lex = i
        # ranks
        for v in range(n):
            nd = nodes[v]
            nd.n = int(np.prod(dims[nd.lo:nd.hi], dtype=np.int64))
            nd.identity = False
            nd.r = nd.p = nd.s = 0
            if v == self.root:
                continue
            r, p = int(ranks[v]), int(oversample[v])
            if nd.is_leaf and identity[v]:
                nd.identity, nd.r, nd.p, nd.s = True, nd.n, 0, nd.n
                continue
            if r < 1 or p < 0:
                raise ValueError("ranks must be >= 1 and oversample >= 0")
            nc = self.N // nd.n
            if nd.is_leaf and r >= nd.n:
                nd.identity, nd.r, nd.p, nd.s = True, nd.n, 0, nd.n
                continue
            r = min(r, nd.n, nc)
            p = min(p, nd.n - r)
            nd.r, nd.p, nd.s = r, p, r + p

    # -- helpers ---------------------------------------------------------
    def node(self, v):
        return self.nodes[v]

    def modes(self, v):
        nd = self.nodes[v]
        return list(range(nd.lo, nd.hi))

    def nonroot(self):
        """Non-root user indices in lexicographic order."""
        return [v for v in self.lex if v != self.root]

    def sketched(self):
        """Non-root, non-identity nodes in lexicographic order."""
        return [v for v in self.nonroot() if not self.nodes[v].identity]

    def ancestors(self, v):
        out = []
        while self.nodes[v].parent >= 0:
            v = self.nodes[v].parent
            out.append(v)
        return out

    def subtree(self, v):
        out, stack = [], [v]
        while stack:
            u = stack.pop()
            out.append(u)
            stack.extend(self.nodes[u].children)
        return out

    def sidesize(self, v):
        """s'_v: the index range node v shows its parent's Psi (s_v, or n_v
        for an identity node)."""
        return self.nodes[v].s

    def sttnn_reuse(self, v):
        """S_t: non-identity preceding siblings of t and of its non-root
        ancestors (Sec. 5, lexicographic ordering)."""
        out = []
        chain = [v] + [a for a in self.ancestors(v) if a != self.root]
        for u in chain:
            par = self.nodes[self.nodes[u].parent]
            for c in par.children:
                if c == u:
                    break
                if not self.nodes[c].identity:
                    out.append(c)
        return sorted(out, key=lambda c: self.nodes[c].lo)

    def root_split(self, variant):
        """Which root children form the pass's left group L (a prefix) and on
        which side the root's Y contraction happens.  Returns (a, y_side):
        L = children[:a], R = children[a:].

        TTNN, two children: a = 1 and the Y side is the one with the smaller
        s' (ties: R).  TTNN, m >= 3 children: a = m - 1 (R is the last child),
        Y on R.  STTNN: a = 1, Y on L (the first child is contracted first).
        """
        ch = self.nodes[self.root].children
        m = len(ch)
        if variant == "sttnn":
            return 1, "L"
        if m == 2:
            sl, sr = self.sidesize(ch[0]), self.sidesize(ch[1])
            return 1, ("R" if sr <= sl else "L")
        return m - 1, "R"
