// Host plan (tree normalisation, first-level split, layouts) and the update /
// recovery programs: the first-level pass over the dense block, the tree walk
// that turns its two products into every node's Omega_v and Psi_v, and the
// binary64 core assembly.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <functional>
#include <numeric>

#include "plan.cuh"
#include "program.cuh"

namespace ttnn {

// tensor-core pass (pass_tc.cu)
ttnn_status tc_pass_supported(const ttnn_plan_s& P, int64_t nL, int64_t nR);
ttnn_status launch_tc_pass(const ttnn_plan_s& P, const void* A, int64_t nL, int64_t nR,
                           const void* sR, int64_t ldR, const void* sL, int64_t ldL, void* D1,
                           void* D2, const float* tile_scale, void* ws, int64_t ws_bytes,
                           cudaStream_t st, bool dry, int64_t* ws_need);
// BF16X2 / E4M3 tensor-core pass (pass_cvt.cu)
ttnn_status cvt_pass_supported(const ttnn_plan_s& P, int64_t nL, int64_t nR);
ttnn_status launch_cvt_pass(const ttnn_plan_s& P, const void* A, int64_t nL, int64_t nR,
                            const void* sR, int64_t ldR, const void* sL, int64_t ldL, void* D1,
                            void* D2, const float* tile_scale, void* ws, int64_t ws_bytes,
                            cudaStream_t st, bool dry, int64_t* ws_need);

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------
ttnn_status build_plan(ttnn_plan_s& P, const ttnn_tree* tree, int32_t d, const int64_t* dims,
                       const int32_t* ranks, const int32_t* oversample, uint64_t seed,
                       const ttnn_opts* opts) {
  TTNN_CHECK_ARG(tree && dims && ranks && oversample, "null argument");
  TTNN_CHECK_ARG(d >= 1 && d <= 16, "order d must be in 1..16");
  const int n = tree->n_nodes;
  TTNN_CHECK_ARG(n >= 1 && tree->parent && tree->leaf_mode_ptr, "empty tree");
  P.d = d;
  P.dims.assign(dims, dims + d);
  P.N = 1;
  for (int m = 0; m < d; ++m) {
    TTNN_CHECK_ARG(dims[m] >= 1, "mode size %d must be >= 1", m);
    TTNN_CHECK_ARG(P.N <= (int64_t(1) << 62) / dims[m], "tensor too large");
    P.N *= dims[m];
  }
  if (opts) {
    P.variant = opts->variant;
    P.dtype = opts->sketch_dtype;
    P.eps_factor = opts->eps_factor;
    P.u = opts->unit_roundoff;
    P.flags = opts->flags;
  }
  // dense tensors are indexed with 64-bit products of their size; a plan
  // for structured (CP / TTN-format) inputs never forms the tensor
  TTNN_CHECK_ARG((P.flags & TTNN_FLAG_STRUCTURED_ONLY) || P.N <= (int64_t(1) << 46),
                 "tensor too large for dense updates (more than 2^46 entries): use "
                 "TTNN_FLAG_STRUCTURED_ONLY");
  TTNN_CHECK_ARG(P.variant == 0 || P.variant == 1, "bad variant");
  TTNN_CHECK_ARG(P.dtype >= 0 && P.dtype <= 4, "bad sketch dtype");
  TTNN_CHECK_ARG(P.eps_factor >= 0 && P.u >= 0, "eps_factor and unit_roundoff must be >= 0");
  P.seed = seed;
  P.nodes.assign(n, TNode());
  int root = -1;
  for (int v = 0; v < n; ++v) {
    const int p = tree->parent[v];
    TTNN_CHECK_ARG(p >= -1 && p < n && p != v, "bad parent index of node %d", v);
    if (p == -1) {
      TTNN_CHECK_ARG(root < 0, "more than one root");
      root = v;
    }
    P.nodes[v].user = v;
    P.nodes[v].parent = p;
  }
  TTNN_CHECK_ARG(root >= 0, "no root");
  P.root = root;
  for (int v = 0; v < n; ++v)
    if (P.nodes[v].parent >= 0) P.nodes[P.nodes[v].parent].ch.push_back(v);
  // reachability / acyclicity
  {
    std::vector<char> seen(n, 0);
    std::vector<int> stack{root};
    int cnt = 0;
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      TTNN_CHECK_ARG(!seen[v], "cycle in tree");
      seen[v] = 1;
      ++cnt;
      for (int c : P.nodes[v].ch) stack.push_back(c);
    }
    TTNN_CHECK_ARG(cnt == n, "tree is not connected");
  }
  // mode ranges, bottom-up
  std::vector<int> mode_owner(d, -1);
  std::function<ttnn_status(int)> visit = [&](int v) -> ttnn_status {
    TNode& nd = P.nodes[v];
    const int b = tree->leaf_mode_ptr[v], e = tree->leaf_mode_ptr[v + 1];
    TTNN_CHECK_ARG(e >= b, "bad leaf_mode_ptr");
    const bool ident = tree->identity && tree->identity[v];
    if (nd.ch.empty()) {
      TTNN_CHECK_ARG(e > b && tree->leaf_modes, "leaf %d without modes", v);
      std::vector<int> lm(tree->leaf_modes + b, tree->leaf_modes + e);
      std::sort(lm.begin(), lm.end());
      for (size_t k = 0; k < lm.size(); ++k) {
        TTNN_CHECK_ARG(lm[k] >= 0 && lm[k] < d, "leaf mode out of range");
        TTNN_CHECK_ARG(lm[k] == lm[0] + (int)k, "leaf modes must be contiguous");
        TTNN_CHECK_ARG(mode_owner[lm[k]] < 0, "leaf modes must partition 0..d-1");
        mode_owner[lm[k]] = v;
      }
      nd.lo = lm.front();
      nd.hi = lm.back() + 1;
      nd.leaf = true;
      return TTNN_OK;
    }
    TTNN_CHECK_ARG(e == b, "internal node %d with own modes", v);
    TTNN_CHECK_ARG(nd.ch.size() >= 2, "internal node %d needs >= 2 children", v);
    TTNN_CHECK_ARG(!ident, "identity flag only on leaves");
    for (int c : nd.ch) TTNN_TRY(visit(c));
    std::sort(nd.ch.begin(), nd.ch.end(), [&](int x, int y) { return P.nodes[x].lo < P.nodes[y].lo; });
    for (size_t k = 0; k + 1 < nd.ch.size(); ++k)
      TTNN_CHECK_ARG(P.nodes[nd.ch[k]].hi == P.nodes[nd.ch[k + 1]].lo, "node modes must be contiguous");
    nd.lo = P.nodes[nd.ch.front()].lo;
    nd.hi = P.nodes[nd.ch.back()].hi;
    nd.leaf = false;
    return TTNN_OK;
  };
  TTNN_TRY(visit(root));
  for (int m = 0; m < d; ++m) TTNN_CHECK_ARG(mode_owner[m] >= 0, "leaf modes must partition 0..d-1");
  // lexicographic order
  {
    std::vector<int> level{root};
    int lvl = 0;
    while (!level.empty()) {
      for (size_t k = 0; k < level.size(); ++k) {
        P.nodes[level[k]].level = lvl;
        P.nodes[level[k]].pos = (int)k;
        P.nodes[level[k]].lex = (int)P.lex.size();
        P.lex.push_back(level[k]);
      }
      std::vector<int> next;
      for (int v : level)
        for (int c : P.nodes[v].ch) next.push_back(c);
      level.swap(next);
      ++lvl;
    }
  }
  // ranks
  for (int v = 0; v < n; ++v) {
    TNode& nd = P.nodes[v];
    nd.n = 1;
    for (int m = nd.lo; m < nd.hi; ++m) nd.n *= P.dims[m];
    if (v == root) continue;
    const bool ident = tree->identity && tree->identity[v];
    if (nd.leaf && ident) {
      nd.identity = true;
      nd.r = (int)std::min<int64_t>(nd.n, 1 << 30);
      nd.p = 0;
      nd.s = nd.r;
      continue;
    }
    int r = ranks[v], p = oversample[v];
    TTNN_CHECK_ARG(r >= 1 && p >= 0, "ranks must be >= 1 and oversample >= 0 (node %d)", v);
    const int64_t nc = P.N / nd.n;
    if (nd.leaf && r >= nd.n) {
      nd.identity = true;
      nd.r = nd.s = (int)nd.n;
      nd.p = 0;
      continue;
    }
    r = (int)std::min<int64_t>(std::min<int64_t>(r, nd.n), nc);
    p = (int)std::min<int64_t>(p, nd.n - r);
    nd.r = r;
    nd.p = p;
    nd.s = r + p;
  }
  // rsub (post-order) and r_max / s_max
  P.rmax = P.smax = 1;
  std::function<int(int)> rs = [&](int v) -> int {
    TNode& nd = P.nodes[v];
    int m = nd.sketched() ? nd.r : 0;
    for (int c : nd.ch) m = std::max(m, rs(c));
    nd.rsub = m;
    return m;
  };
  rs(root);
  P.n_sketched = 0;
  for (auto& nd : P.nodes)
    if (nd.sketched()) {
      P.rmax = std::max(P.rmax, nd.r);
      P.smax = std::max(P.smax, nd.s);
      TTNN_CHECK_ARG(nd.r <= kMaxRecoverR && nd.s <= kMaxRecoverS,
                     "rank %d / sketch size %d above the recovery limits (%d, %d)", nd.r, nd.s,
                     kMaxRecoverR, kMaxRecoverS);
      ++P.n_sketched;
    }
  // STTNN reuse sets
  for (int v = 0; v < n; ++v) {
    if (v == root) continue;
    std::vector<int> S;
    int u = v;
    while (P.nodes[u].parent >= 0) {
      const TNode& par = P.nodes[P.nodes[u].parent];
      for (int c : par.ch) {
        if (c == u) break;
        if (!P.nodes[c].identity) S.push_back(c);
      }
      u = P.nodes[u].parent;
      if (u == root) break;
    }
    std::sort(S.begin(), S.end(), [&](int x, int y) { return P.nodes[x].lo < P.nodes[y].lo; });
    P.nodes[v].reuse = S;
  }
  // number formats
  P.walk_f64 = (P.dtype == TTNN_F64);
  P.tc_ok = (P.dtype == TTNN_BF16 || P.dtype == TTNN_BF16X2 || P.dtype == TTNN_E4M3);
  // BF16X2: binary32 tensor, bfloat16 DRM blocks.  E4M3: E4M3 tensor, DRM
  // blocks rounded to E4M3 values and stored as bfloat16 (exact) for the
  // bfloat16 tensor cores that multiply the dequantised tiles.
  switch (P.dtype) {
    case TTNN_F64: P.pass_store = 0; P.side_store = 0; P.round_fmt = RF_F64; break;
    case TTNN_F32: P.pass_store = 1; P.side_store = 1; P.round_fmt = RF_F32; break;
    case TTNN_BF16: P.pass_store = 2; P.side_store = 2; P.round_fmt = RF_BF16; break;
    case TTNN_E4M3: P.pass_store = 3; P.side_store = 2; P.round_fmt = RF_E4M3; break;
    default: P.pass_store = 1; P.side_store = 2; P.round_fmt = RF_BF16; break;   // BF16X2
  }
  // first-level split
  const TNode& R0 = P.nodes[root];
  const int m = (int)R0.ch.size();
  if (R0.ch.empty()) {
    set_error("the root must have children (d >= 2)");
    return TTNN_EINVAL;
  }
  auto sprime = [&](int c) { return P.nodes[c].identity ? (int64_t)P.nodes[c].n : (int64_t)P.nodes[c].s; };
  if (P.variant == TTNN_VARIANT_STTNN) {
    P.a = 1;
    P.yside = 1;
    if (P.nodes[R0.ch[0]].identity) {
      set_error("STTNN with an identity first root child is not supported");
      return TTNN_EUNSUPPORTED;
    }
  } else if (m == 2) {
    P.a = 1;
    P.yside = (sprime(R0.ch[1]) <= sprime(R0.ch[0])) ? 0 : 1;
  } else {
    P.a = m - 1;
    P.yside = 0;
  }
  P.Lch.assign(R0.ch.begin(), R0.ch.begin() + P.a);
  P.Rch.assign(R0.ch.begin() + P.a, R0.ch.end());
  P.Llo = P.nodes[P.Lch.front()].lo;
  P.Lhi = P.nodes[P.Lch.back()].hi;
  P.Rlo = P.nodes[P.Rch.front()].lo;
  P.Rhi = P.nodes[P.Rch.back()].hi;
  P.ychild = (P.yside == 0) ? P.Rch[0] : P.Lch[0];
  if (P.yside == 0 && P.Rch.size() != 1) P.ychild = -1;
  if (P.yside == 1 && P.Lch.size() != 1) P.ychild = -1;
  if (P.ychild < 0) {
    set_error("internal: pass Y side must be a single root child");
    return TTNN_EUNSUPPORTED;
  }
  P.rXL = 0;
  for (int c : P.Lch) P.rXL = std::max(P.rXL, P.nodes[c].rsub);
  P.rXR = 0;
  if (P.variant == TTNN_VARIANT_TTNN)
    for (int c : P.Rch) P.rXR = std::max(P.rXR, P.nodes[c].rsub);
  const int64_t wy = sprime(P.ychild);
  TTNN_CHECK_ARG(wy <= 4096, "pass Y block too wide (%lld columns)", (long long)wy);
  P.wYR = P.yside == 0 ? (int)wy : 0;
  P.wYL = P.yside == 1 ? (int)wy : 0;
  P.yR_ident = P.yside == 0 && P.nodes[P.ychild].identity;
  P.yL_ident = P.yside == 1 && P.nodes[P.ychild].identity;
  P.wR = P.rXL + P.wYR;
  P.wL = P.rXR + P.wYL;
  P.wRpad = (int)round_up(P.wR, 16);
  P.wLpad = (int)round_up(P.wL, 16);
  // state layout (lex order): Omega_v then Psi_v; root: Psi_root
  int64_t off = 0;
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    nd.ps_shape.clear();
    if (v == root) {
      nd.ps_el = 1;
      for (int c : nd.ch) {
        nd.ps_shape.push_back(sprime(c));
        nd.ps_el *= sprime(c);
      }
      TTNN_CHECK_ARG(nd.ps_el <= (int64_t(1) << 33), "root sketch too large");
      nd.ps_off = off;
      off += nd.ps_el;
      continue;
    }
    if (!nd.sketched()) continue;
    nd.om_off = off;
    nd.om_el = (int64_t)nd.s * nd.r;
    off += nd.om_el;
    if (nd.leaf) {
      nd.ps_shape = {nd.n, (int64_t)nd.r};
      nd.ps_el = nd.n * nd.r;
    } else {
      nd.ps_el = nd.r;
      for (int c : nd.ch) {
        nd.ps_shape.push_back(sprime(c));
        nd.ps_el *= sprime(c);
      }
      nd.ps_shape.push_back(nd.r);
    }
    nd.ps_off = off;
    off += nd.ps_el;
  }
  P.state_elems = off;
  // core layout (lex order)
  off = 0;
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    nd.core_shape.clear();
    if (v == root) {
      for (int c : nd.ch) nd.core_shape.push_back(P.nodes[c].r);
    } else if (nd.identity) {
      nd.core_shape = {nd.n};
      for (int mm = nd.lo; mm < nd.hi; ++mm) nd.core_shape.push_back(P.dims[mm]);
    } else if (nd.leaf) {
      nd.core_shape = {(int64_t)nd.r};
      for (int mm = nd.lo; mm < nd.hi; ++mm) nd.core_shape.push_back(P.dims[mm]);
    } else {
      nd.core_shape = {(int64_t)nd.r};
      for (int c : nd.ch) nd.core_shape.push_back(P.nodes[c].r);
    }
    nd.core_el = 1;
    for (int64_t x : nd.core_shape) nd.core_el *= x;
    nd.core_off = off;
    off += nd.core_el;
  }
  P.core_elems = off;
  // factor layout: X_mu, Y_mu, then XT_v of sketched nodes
  off = 0;
  P.x_off.assign(d, 0);
  P.y_off.assign(d, 0);
  for (int mm = 0; mm < d; ++mm) {
    P.x_off[mm] = off;
    off += P.dims[mm] * P.rmax;
    P.y_off[mm] = off;
    off += P.dims[mm] * P.smax;
  }
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    nd.xt_off = off;
    off += (int64_t)nd.s * P.rmax;
  }
  P.fac_elems = off;
  return TTNN_OK;
}

// ---------------------------------------------------------------------------
// workspace stack and tensor views
// ---------------------------------------------------------------------------
// Workspace of one update or recovery: a bump allocator.  Nothing is reused
// inside a program, so the executor may reorder independent ops freely.
struct Ws {
  char* base;
  int64_t cap, top = 0, peak = 0;
  bool dry;
  Program* prog = nullptr;
  Ws(char* b, int64_t c, bool d) : base(b), cap(c), dry(d) {}
  char* alloc(int64_t bytes) {
    const int64_t o = round_up(top, 256);
    top = o + std::max<int64_t>(bytes, 0);
    peak = std::max(peak, top);
    // dry runs hand out offsets from a fake base so that buffer identities
    // (and therefore the recorded program's levels) match a real run
    char* p = (dry ? (char*)(uintptr_t)0x100000000ull : base) + o;
    if (prog) prog->buffer(p, std::max<int64_t>(bytes, 1));
    return p;
  }
  bool ok() const { return dry || top <= cap; }
};

enum AxKind { AX_MODE = 0, AX_SK = 1, AX_J = 2 };
struct Ax {
  int kind;
  int id;          // mode (AX_MODE) or child node (AX_SK)
  int64_t size;
  int64_t off;     // box offset (AX_MODE)
  // > 0: a broadcast of this logical size (the data holds one entry along
  // the axis, size == 1): the outer products with one row of a DRM block
  // that a box fixing modes produces, left to the scatter
  int64_t bc = 0;
};
struct View {
  char* ptr;
  std::vector<Ax> ax;
  int64_t ld;      // stride of the next-to-last axis
  // scales not yet applied: the view's values times prod_k sc_k[index on the
  // axis (kind, id)].  They are rows of the DRM factors of box-fixed modes
  // (X_mu[c, :] on the column axis, Y_mu[c, :] on a sketch axis), commute
  // with every contraction over the other axes and are applied by the
  // scatter into the state (or by a scaled copy before their own axis is
  // contracted).
  struct Scale {
    int kind, id;
    const char* ptr;
  };
  std::vector<Scale> sc;
};

static int64_t vstride(const View& v, int k) {
  const int L = (int)v.ax.size() - 1;
  if (k == L) return 1;
  if (k == L - 1) return v.ld;
  return vstride(v, k + 1) * v.ax[k + 1].size;
}
static int64_t vsize(const View& v) {
  int64_t s = 1;
  for (auto& a : v.ax) s *= a.size;
  return s;
}

struct Ctx {
  ttnn_plan_s& P;
  Ws& ws;
  cudaStream_t st;
  bool dry;
  int eb;               // walk element bytes
  ElemType et;
  const Box& box;
  const char* facw;     // walk-type factors
  const char* yw;       // walk-type copy of the pass Y block (rows of the Y child, box)
  int64_t yw_ld;
  Program* prog;
  // rank-one box with the Y child on the matrix-vector side: Y^T m, the Y
  // child's Omega before its broadcast column factor (walk type, s entries)
  const char* yom = nullptr;
  // Y child over the L modes, whole 2-D box: Omega_y = Y^T (M X) = (M^T Y)^T X
  // as a reduction over the R index: d2y = M^T Y (the Y columns of D2, row
  // stride d2y_ld, nRo rows) and xo = the stored X block of the L side over
  // the R modes (walk type, [rXL][nRo])
  const char* d2y = nullptr;
  int64_t d2y_ld = 0;
  const char* xo = nullptr;
  int64_t nRo = 0;
};

static int find_ax(const View& v, int kind, int id) {
  for (int k = 0; k < (int)v.ax.size(); ++k)
    if (v.ax[k].kind == kind && v.ax[k].id == id) return k;
  return -1;
}

// Contract axis k of `in` against W.  shared < 0: mode product creating a new
// axis `nax` at position k, W(i, b) = W[i*wsI + b*wsX].  shared == last or
// shared == k + 1: the reduction shares that axis' index x with W,
// W(i, x) = W[i*wsI + x*wsX]; the axis stays.  The output is contiguous.
static ttnn_status apply_scales(Ctx& C, const View& in, View* out);

// A Khatri-Rao weight of up to four per-mode factors (walk type): W(i, b) =
// prod_f f[f][d_f * wsI + b * wsX], d_f the digits of i over `rows` (first
// factor slowest).  Only binary32 walks, sketch sizes <= 32.
struct KrSpec {
  int n = 0;
  const char* f[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t rows[4] = {0, 0, 0, 0};
};

static ttnn_status contract_view(Ctx& C, const View& in, int k, const void* W, int64_t wsI,
                                 int64_t wsX, int shared, const Ax* nax, View* out,
                                 const KrSpec* kr = nullptr) {
  const int L = (int)in.ax.size() - 1;
  // a broadcast axis that is contracted or shared (other than the column axis
  // in the shared == L form, which makes it real) is expanded first
  bool expand = in.ax[k].bc > 0 || (shared >= 0 && shared != L && in.ax[shared].bc > 0);
  for (const View::Scale& x : in.sc)
    if (x.kind == in.ax[k].kind && x.id == in.ax[k].id) expand = true;
  if (expand) {
    // the contracted axis carries pending scales or a broadcast: apply them
    View m;
    TTNN_TRY(apply_scales(C, in, &m));
    return contract_view(C, m, k, W, wsI, wsX, shared, nax, out, kr);
  }
  Contract c;
  if (kr) {
    if (shared >= 0 || C.et != ET_F32 || nax->size > 32 || kr->n < 1 || kr->n > 4) {
      set_error("internal: Khatri-Rao weight outside its form");
      return TTNN_EUNSUPPORTED;
    }
    c.nkr = kr->n;
    for (int f = 0; f < kr->n; ++f) {
      c.kr[f] = kr->f[f];
      c.krn[f] = kr->rows[f];
    }
    W = nullptr;
  }
  c.P = 1;
  for (int a = 0; a < k; ++a) c.P *= in.ax[a].size;
  c.isP = k > 0 ? vstride(in, k - 1) : 0;
  c.NI = in.ax[k].size;
  c.isI = vstride(in, k);
  c.w = W;
  c.wsI = wsI;
  std::vector<Ax> oax;
  if (shared < 0) {
    c.NB = nax->size;
    c.wsB = wsX;
    if (k < L) {
      c.Q = 1;
      for (int a = k + 1; a < L; ++a) c.Q *= in.ax[a].size;
      c.isQ = (k < L - 1) ? vstride(in, L - 1) : 0;
      c.J = in.ax[L].size;
      c.isJ = 1;
    }
    oax.assign(in.ax.begin(), in.ax.begin() + k);
    oax.push_back(*nax);
    oax.insert(oax.end(), in.ax.begin() + k + 1, in.ax.end());
  } else if (shared == L) {
    if (k >= L) { set_error("internal: bad shared-column contraction"); return TTNN_EUNSUPPORTED; }
    c.Q = 1;
    for (int a = k + 1; a < L; ++a) c.Q *= in.ax[a].size;
    c.isQ = (k < L - 1) ? vstride(in, L - 1) : 0;
    // a broadcast column axis becomes real here (W's columns differ)
    c.J = in.ax[L].bc > 0 ? in.ax[L].bc : in.ax[L].size;
    c.isJ = in.ax[L].bc > 0 ? 0 : 1;
    c.wsJ = wsX;
    oax = in.ax;
    oax.erase(oax.begin() + k);
    oax.back().size = c.J;
    oax.back().bc = 0;
  } else if (shared == k + 1) {
    c.Q = in.ax[k + 1].size;
    c.isQ = vstride(in, k + 1);
    c.J = 1;
    for (int a = k + 2; a <= L; ++a) c.J *= in.ax[a].size;
    c.isJ = 1;
    if (k + 2 <= L - 1 && in.ld != in.ax[L].size) {
      set_error("internal: non-contiguous column group");
      return TTNN_EUNSUPPORTED;
    }
    c.wsQ = wsX;
    oax = in.ax;
    oax.erase(oax.begin() + k);
  } else if (shared == 0 && k == 1) {
    // the shared axis is the whole prefix: W(i, x) indexed by p
    c.P = in.ax[0].size;
    c.isP = vstride(in, 0);
    c.wsP = wsX;
    if (k < L) {
      c.Q = 1;
      for (int a = k + 1; a < L; ++a) c.Q *= in.ax[a].size;
      c.isQ = (k < L - 1) ? vstride(in, L - 1) : 0;
      c.J = in.ax[L].size;
      c.isJ = 1;
      if (k + 1 <= L - 1 && in.ld != in.ax[L].size) {
        set_error("internal: non-contiguous column group");
        return TTNN_EUNSUPPORTED;
      }
    }
    oax = in.ax;
    oax.erase(oax.begin() + k);
  } else {
    set_error("internal: unsupported shared axis");
    return TTNN_EUNSUPPORTED;
  }
  View o;
  o.ax = oax;
  o.ld = o.ax.back().size;
  o.sc = in.sc;
  const int64_t total = vsize(o);
  o.ptr = C.ws.alloc(total * C.eb);
  c.out = o.ptr;
  c.osJ = 1;
  c.osQ = c.J;
  c.osB = c.Q * c.J;
  c.osP = c.NB * c.Q * c.J;
  c.in = in.ptr;
  Op op;
  op.tin = op.tw = op.tout = C.et;
  op.c = c;
  const int64_t pe = plan_contract(op);
  op.partial = pe ? C.ws.alloc(pe * C.eb) : nullptr;
  C.prog->add(op, in.ptr, W);
  *out = o;
  return TTNN_OK;
}

static const char* facX(Ctx& C, int mode) { return C.facw + (C.P.x_off[mode] + C.box.off[mode] * C.P.rmax) * C.eb; }
static const char* facY(Ctx& C, int mode) { return C.facw + (C.P.y_off[mode] + C.box.off[mode] * C.P.smax) * C.eb; }

// Mode of `modes` (ascending, adjacent axes of `in`) at which a Khatri-Rao Y
// chain creates its sketch axis: the mode with the largest extent when it is
// the view's first axis (every later mode is then contracted against the
// sketch axis as the whole prefix), else the last mode.
static int chain_first(const View& in, const std::vector<int>& modes) {
  const int lo = modes.front(), last = modes.back();
  int best = last;
  const int k0 = find_ax(in, AX_MODE, lo);
  if (k0 == 0) {
    int64_t big = -1;
    for (int m : modes) {
      const int k = find_ax(in, AX_MODE, m);
      if (k >= 0 && in.ax[k].size > big) {
        big = in.ax[k].size;
        best = m;
      }
    }
    if (best != lo) best = last;
    // keep the last mode when it is as large as the first
    const int kl = find_ax(in, AX_MODE, last);
    if (kl >= 0 && in.ax[kl].size >= in.ax[k0].size) best = last;
  }
  return best;
}

// Whether a Y chain over the modes [lo, hi) of `in` creates its sketch axis
// at mode hi - 1 (extent > 1; box-fixed modes become scales, not steps).
static bool chain_starts_last(const View& in, int lo, int hi) {
  View v = in;
  std::vector<int> modes;
  for (int m = lo; m < hi; ++m) {
    const int k = find_ax(v, AX_MODE, m);
    if (k < 0) return false;
    if (v.ax[k].size == 1) {
      if (m == hi - 1) return false;
      v.ax.erase(v.ax.begin() + k);
      continue;
    }
    modes.push_back(m);
  }
  return chain_first(v, modes) == hi - 1;
}

// Khatri-Rao contraction of the modes [lo, hi) of `in` with the Y factors,
// producing one sketch axis (kind AX_SK, id = node) of size s at the place of
// the modes (Sec. 7: Y_t = kr of its modes' Y_mu, columns shared).
// With first_done the sketch axis already replaces mode hi - 1 (a shared
// first mode product) and only the Khatri-Rao steps remain.  Box-fixed modes
// become deferred scales of the sketch axis (their axes are dropped: no data
// moves).
static ttnn_status y_chain(Ctx& C, const View& in, int node, int lo, int hi, int s, View* out,
                           bool first_done = false) {
  View cur = in;
  const int top = first_done ? hi - 1 : hi;
  // with first_done the sketch axis exists already; else one mode must create it
  bool any_free = first_done;
  for (int m = lo; m < top; ++m) {
    const int k = find_ax(cur, AX_MODE, m);
    if (k < 0) { set_error("internal: mode axis missing"); return TTNN_EUNSUPPORTED; }
    if (cur.ax[k].size > 1) any_free = true;
  }
  std::vector<int> modes;
  for (int m = lo; m < top; ++m) {
    const int k = find_ax(cur, AX_MODE, m);
    const bool creates = !any_free && m == top - 1;
    if (cur.ax[k].size == 1 && k < (int)cur.ax.size() - 1 && cur.sc.size() < (size_t)kMaxScales) {
      if (creates) {
        // every mode fixed: the sketch axis is the outer product with the
        // row, a broadcast in place of the mode (no data moves)
        cur.ax[k] = Ax{AX_SK, node, 1, 0, s};
      } else {
        cur.ax.erase(cur.ax.begin() + k);
      }
      cur.sc.push_back(View::Scale{AX_SK, node, facY(C, m)});
      continue;
    }
    modes.push_back(m);
  }
  if (modes.empty()) {
    *out = cur;
    return TTNN_OK;
  }
  View nx;
  const int first = first_done ? -1 : chain_first(cur, modes);
  if (!first_done && first == modes.front() && first != modes.back()) {
    // sketch axis at the first (largest) mode, then the others against it
    const int k0 = find_ax(cur, AX_MODE, first);
    Ax nax{AX_SK, node, s, 0};
    TTNN_TRY(contract_view(C, cur, k0, facY(C, first), C.P.smax, 1, -1, &nax, &nx));
    cur = nx;
    for (size_t i = 1; i < modes.size(); ++i) {
      const int k = find_ax(cur, AX_MODE, modes[i]);
      if (k != 1) { set_error("internal: Khatri-Rao chain layout"); return TTNN_EUNSUPPORTED; }
      TTNN_TRY(contract_view(C, cur, k, facY(C, modes[i]), C.P.smax, 1, 0, nullptr, &nx));
      cur = nx;
    }
    *out = cur;
    return TTNN_OK;
  }
  for (int i = (int)modes.size() - 1; i >= 0; --i) {
    const int mode = modes[i];
    const int k = find_ax(cur, AX_MODE, mode);
    if (k < 0) { set_error("internal: mode axis missing"); return TTNN_EUNSUPPORTED; }
    if (!first_done && i == (int)modes.size() - 1) {
      Ax nax{AX_SK, node, s, 0};
      TTNN_TRY(contract_view(C, cur, k, facY(C, mode), C.P.smax, 1, -1, &nax, &nx));
    } else {
      if (k + 1 >= (int)cur.ax.size() || cur.ax[k + 1].kind != AX_SK || cur.ax[k + 1].id != node) {
        set_error("internal: Khatri-Rao chain layout");
        return TTNN_EUNSUPPORTED;
      }
      TTNN_TRY(contract_view(C, cur, k, facY(C, mode), C.P.smax, 1, k + 1, nullptr, &nx));
    }
    cur = nx;
  }
  *out = cur;
  return TTNN_OK;
}

// Contraction of one mode with X_mu sharing the column axis (last axis).
static ttnn_status x_mode(Ctx& C, const View& in, int mode, View* out) {
  const int k = find_ax(in, AX_MODE, mode);
  if (k < 0) { set_error("internal: mode axis missing"); return TTNN_EUNSUPPORTED; }
  const int L = (int)in.ax.size() - 1;
  if (in.ax[k].size == 1 && k < L && in.sc.size() < (size_t)kMaxScales &&
      in.ax[L].kind == AX_J) {
    // a mode the box fixes: the contraction is a column scale by the row
    // X_mu[c, :]; drop the axis (no data moves) and defer the scale
    View o = in;
    o.ax.erase(o.ax.begin() + k);
    o.sc.push_back(View::Scale{AX_J, -1, facX(C, mode)});
    *out = o;
    return TTNN_OK;
  }
  return contract_view(C, in, k, facX(C, mode), C.P.rmax, 1, L, nullptr, out);
}

// The Y chain of `node` over the modes [lo, hi) of `in` whose sketch axis is
// already the view's first axis (a Khatri-Rao prefix contracted before, with
// the same columns): each remaining mode, in turn the view's second axis, is
// contracted against it.  The sketch axis is relabelled to `node`.
static ttnn_status y_chain_rest(Ctx& C, const View& in, int node, int lo, int hi, View* out) {
  View cur = in;
  if (cur.ax.empty() || cur.ax[0].kind != AX_SK) {
    set_error("internal: Khatri-Rao prefix layout");
    return TTNN_EUNSUPPORTED;
  }
  const int old = cur.ax[0].id;
  cur.ax[0].id = node;
  for (auto& x : cur.sc)
    if (x.kind == AX_SK && x.id == old) x.id = node;
  for (int m = lo; m < hi; ++m) {
    if (find_ax(cur, AX_MODE, m) != 1) {
      set_error("internal: Khatri-Rao prefix layout");
      return TTNN_EUNSUPPORTED;
    }
    View nx;
    TTNN_TRY(contract_view(C, cur, 1, facY(C, m), C.P.smax, 1, 0, nullptr, &nx));
    cur = nx;
  }
  *out = cur;
  return TTNN_OK;
}

// Contraction of the leading modes [lo, hi) of `in` (its first axes, no
// broadcasts or pending scales on them) with kr(Y_mu, mu in [lo, hi))[:, :s]
// as one long reduction over their merged index; the new sketch axis (kind
// AX_SK, id `node`, size s) replaces them.
static ttnn_status kr_prefix(Ctx& C, const View& in, int node, int lo, int hi, int s, View* out) {
  const int m = hi - lo;
  View v = in;
  int64_t n = 1;
  KrSpec kr;
  kr.n = m;
  for (int k = 0; k < m; ++k) {
    const Ax& a = in.ax[k];
    if (a.kind != AX_MODE || a.id != lo + k || a.bc > 0) {
      set_error("internal: Khatri-Rao prefix layout");
      return TTNN_EUNSUPPORTED;
    }
    n *= a.size;
    kr.f[k] = facY(C, lo + k);
    kr.rows[k] = (int32_t)a.size;
  }
  for (const View::Scale& x : in.sc)
    for (int k = 0; k < m; ++k)
      if (x.kind == in.ax[k].kind && x.id == in.ax[k].id) {
        set_error("internal: Khatri-Rao prefix with a pending scale");
        return TTNN_EUNSUPPORTED;
      }
  // the prefix axes are contiguous (row-major): one merged axis
  v.ax.erase(v.ax.begin(), v.ax.begin() + m);
  v.ax.insert(v.ax.begin(), Ax{AX_MODE, lo, n, 0});
  if (v.ax.size() < 2) {
    set_error("internal: Khatri-Rao prefix without columns");
    return TTNN_EUNSUPPORTED;
  }
  Ax nax{AX_SK, node, s, 0};
  return contract_view(C, v, 0, nullptr, C.P.smax, 1, -1, &nax, out, &kr);
}

// STTNN: contraction of group s with E_s = Y_s XT_s (Y chain, then XT_s on
// the new sketch axis sharing the column axis).
static ttnn_status e_group(Ctx& C, const View& in, int s, View* out) {
  const TNode& ns = C.P.nodes[s];
  View y;
  TTNN_TRY(y_chain(C, in, s, ns.lo, ns.hi, ns.s, &y));
  const int k = find_ax(y, AX_SK, s);
  const char* xt = C.facw + ns.xt_off * C.eb;
  return contract_view(C, y, k, xt, C.P.rmax, 1, (int)y.ax.size() - 1, nullptr, out);
}

static ttnn_status scatter_op(Ctx& C, const View& v, char* base, const std::vector<int64_t>& os,
                              double alpha, bool assign, bool box_off) {
  const int nd = (int)v.ax.size();
  // per axis: logical size, strides, scale (box offsets fold into the base)
  struct A {
    int64_t size, is, os;
    int scaled;   // carries scales (never merged)
    int orig;     // the view axis (scaled axes)
  };
  std::vector<A> ax(nd);
  int64_t boff = 0;
  for (int a = 0; a < nd; ++a) {
    const bool bcast = v.ax[a].bc > 0;
    ax[a] = A{bcast ? v.ax[a].bc : v.ax[a].size, bcast ? 0 : vstride(v, a), os[a], 0, a};
    if (ax[a].size < 1) return TTNN_OK;   // nothing to add
    if (box_off && v.ax[a].kind == AX_MODE) boff += v.ax[a].off * os[a];
  }
  if (v.sc.size() > (size_t)kMaxScales) { set_error("internal: too many scales"); return TTNN_EUNSUPPORTED; }
  for (size_t k = 0; k < v.sc.size(); ++k) {
    const int a = find_ax(v, v.sc[k].kind, v.sc[k].id);
    if (a < 0) { set_error("internal: scale without its axis"); return TTNN_EUNSUPPORTED; }
    ax[a].scaled = 1;
  }
  // merge neighbouring unscaled axes whose strides chain (fewer index
  // divisions per element); extent-1 axes without a scale drop out
  std::vector<A> m;
  for (int a = nd - 1; a >= 0; --a) {
    const A& x = ax[a];
    if (x.size == 1 && !x.scaled) continue;
    if (!m.empty()) {
      A& in = m.back();
      if (!x.scaled && !in.scaled && x.is == in.is * in.size && x.os == in.os * in.size) {
        in.size *= x.size;
        continue;
      }
    }
    m.push_back(x);
  }
  if (m.empty()) m.push_back(A{1, 0, 0, 0, -1});
  std::reverse(m.begin(), m.end());
  Scatter s;
  s.nd = (int)m.size();
  if (s.nd > 12) { set_error("internal: too many axes"); return TTNN_EUNSUPPORTED; }
  for (int a = 0; a < s.nd; ++a) {
    if (m[a].size >= (int64_t(1) << 31)) { set_error("internal: axis too long"); return TTNN_EUNSUPPORTED; }
    s.size[a] = (int32_t)m[a].size;
    s.is[a] = m[a].is;
    s.os[a] = m[a].os;
    div_magic((uint32_t)s.size[a], &s.mag[a], &s.shf[a]);
    if (!m[a].scaled) continue;
    for (const View::Scale& x : v.sc)
      if (find_ax(v, x.kind, x.id) == m[a].orig) {
        s.sc[s.nsc] = x.ptr;
        s.scax[s.nsc] = (int8_t)a;
        ++s.nsc;
      }
  }
  s.in = v.ptr;
  s.out = base + boff * C.eb;
  s.alpha = alpha;
  s.assign = assign ? 1 : 0;
  Op op;
  op.kind = OP_SCATTER;
  op.tin = op.tw = op.tout = C.et;
  op.s = s;
  plan_simple(op);
  C.prog->add(op, v.ptr);
  return TTNN_OK;
}

// Adds alpha * view (its pending scales applied) into the state at `base`
// with per-axis output strides (mode axes offset by the box).
static ttnn_status scatter_into(Ctx& C, const View& v, char* base, const std::vector<int64_t>& os,
                                double alpha) {
  return scatter_op(C, v, base, os, alpha, false, true);
}

// A contiguous copy of `in` with its pending scales applied.
static ttnn_status apply_scales(Ctx& C, const View& in, View* out) {
  View o;
  o.ax = in.ax;
  for (Ax& a : o.ax)
    if (a.bc > 0) {
      a.size = a.bc;
      a.bc = 0;
    }
  o.ld = o.ax.back().size;
  o.ptr = C.ws.alloc(vsize(o) * C.eb);
  std::vector<int64_t> os(o.ax.size());
  for (int a = 0; a < (int)o.ax.size(); ++a) os[a] = vstride(o, a);
  TTNN_TRY(scatter_op(C, in, o.ptr, os, 1.0, true, false));
  *out = o;
  return TTNN_OK;
}

// Output strides of a Psi-shaped target: children axes (sketch or raw modes of
// identity children) then optionally the column axis.
static std::vector<int64_t> psi_strides(Ctx& C, const View& v, const TNode& nd, bool with_j) {
  const int m = (int)nd.ch.size();
  std::vector<int64_t> cs(m);
  int64_t acc = with_j ? nd.r : 1;
  for (int k = m - 1; k >= 0; --k) {
    cs[k] = acc;
    const TNode& c = C.P.nodes[nd.ch[k]];
    acc *= c.identity ? c.n : c.s;
  }
  std::vector<int64_t> os(v.ax.size(), 0);
  for (size_t a = 0; a < v.ax.size(); ++a) {
    const Ax& x = v.ax[a];
    if (x.kind == AX_J) { os[a] = 1; continue; }
    for (int k = 0; k < m; ++k) {
      const TNode& c = C.P.nodes[nd.ch[k]];
      if (x.kind == AX_SK && x.id == nd.ch[k]) os[a] = cs[k];
      if (x.kind == AX_MODE && x.id >= c.lo && x.id < c.hi) {
        int64_t sub = 1;
        for (int mm = x.id + 1; mm < c.hi; ++mm) sub *= C.P.dims[mm];
        os[a] = cs[k] * sub;
      }
    }
  }
  return os;
}

static View truncate_j(const View& v, int64_t j) {
  View o = v;
  if (o.ax.back().bc > 0) o.ax.back().bc = std::min<int64_t>(o.ax.back().bc, j);
  else o.ax.back().size = std::min<int64_t>(o.ax.back().size, j);
  return o;
}

static char* state_at(Ctx& C, void* acc, int64_t elem_off) { return (char*)acc + elem_off * C.eb; }

// Node v with G_v = T^(v) X_v over the box (axes: v's modes, then columns).
// pre (optional): G_v with the modes of v's first child already contracted
// with that child's Khatri-Rao Y (sketch axis first, same columns as Y_v's
// leading factors): Omega_v and Psi_v start from it.
static ttnn_status walk(Ctx& C, void* acc, int v, const View& G, double lambda,
                        const View* pre = nullptr) {
  ttnn_plan_s& P = C.P;
  const TNode& nd = P.nodes[v];
  if (nd.rsub == 0) return TTNN_OK;
  if (nd.sketched() && pre) {
    const TNode& c1 = P.nodes[nd.ch.front()];
    const View pt = truncate_j(*pre, nd.r);
    View om;
    TTNN_TRY(y_chain_rest(C, pt, v, c1.hi, nd.hi, &om));
    TTNN_TRY(scatter_into(C, om, state_at(C, acc, nd.om_off), {(int64_t)nd.r, 1}, lambda));
    View cur = pt;
    for (int k = (int)nd.ch.size() - 1; k >= 1; --k) {
      const TNode& c = P.nodes[nd.ch[k]];
      if (c.identity) continue;
      View nx;
      TTNN_TRY(y_chain(C, cur, c.user, c.lo, c.hi, c.s, &nx));
      cur = nx;
    }
    TTNN_TRY(scatter_into(C, cur, state_at(C, acc, nd.ps_off), psi_strides(C, cur, nd, true), lambda));
  } else if (nd.sketched()) {
    const View Gt = truncate_j(G, nd.r);
    View om;
    // Omega_t and Psi_t both start by contracting t's last mode with the same
    // Y columns when the last child's sketch size equals s_t: do it once.
    const TNode* lastc = nd.leaf ? nullptr : &P.nodes[nd.ch.back()];
    const bool share = v != P.ychild && lastc && !lastc->identity && lastc->s == nd.s &&
                       chain_starts_last(Gt, nd.lo, nd.hi);
    View z;
    if (share) {
      const int k = find_ax(Gt, AX_MODE, nd.hi - 1);
      Ax nax{AX_SK, v, nd.s, 0};
      TTNN_TRY(contract_view(C, Gt, k, facY(C, nd.hi - 1), P.smax, 1, -1, &nax, &z));
    }
    std::vector<int64_t> om_os = {(int64_t)nd.r, 1};   // Omega [s][r] in the state
    if (v == P.ychild && C.yom && Gt.ax.back().bc > 0) {
      // rank-one box: G = m (x) x, so Omega = (Y^T m) (x) x, and Y^T m is
      // the Y part of the pass's matrix-vector product
      om.ptr = (char*)C.yom;
      om.ax = {Ax{AX_SK, v, nd.s, 0}, Gt.ax.back()};
      om.ld = 1;
      om.sc = Gt.sc;
    } else if (v == P.ychild && C.d2y) {
      // reduction over the (shorter) R index: Omega[b][j] = sum_i D2[i][b] X[j][i]
      // (axes j, b: written transposed); whole 2-D boxes carry no scales
      if (!Gt.sc.empty()) {
        set_error("internal: scaled Y-child Omega through D2");
        return TTNN_EUNSUPPORTED;
      }
      View h;
      h.ptr = (char*)C.d2y;
      h.ax = {Ax{AX_MODE, P.Rlo, C.nRo, 0}, Ax{AX_SK, v, nd.s, 0}};
      h.ld = C.d2y_ld;
      Ax nax{AX_J, -1, nd.r, 0};
      TTNN_TRY(contract_view(C, h, 0, C.xo, 1, C.nRo, -1, &nax, &om));
      om_os = {1, (int64_t)nd.r};
    } else if (v == P.ychild) {
      // Y of the pass-side root child is the stored (rounded) block
      View mg = Gt;
      int64_t nb = 1;
      for (int a = 0; a + 1 < (int)Gt.ax.size(); ++a) nb *= Gt.ax[a].size;
      mg.ax = {Ax{AX_MODE, nd.lo, nb, 0}, Gt.ax.back()};
      Ax nax{AX_SK, v, nd.s, 0};
      TTNN_TRY(contract_view(C, mg, 0, C.yw, 1, C.yw_ld, -1, &nax, &om));
    } else if (share) {
      TTNN_TRY(y_chain(C, z, v, nd.lo, nd.hi, nd.s, &om, true));
    } else {
      TTNN_TRY(y_chain(C, Gt, v, nd.lo, nd.hi, nd.s, &om));
    }
    TTNN_TRY(scatter_into(C, om, state_at(C, acc, nd.om_off), om_os, lambda));
    if (nd.leaf) {
      std::vector<int64_t> os(Gt.ax.size(), 1);
      for (int a = 0; a + 1 < (int)Gt.ax.size(); ++a) {
        int64_t sub = nd.r;
        for (int mm = Gt.ax[a].id + 1; mm < nd.hi; ++mm) sub *= P.dims[mm];
        os[a] = sub;
      }
      TTNN_TRY(scatter_into(C, Gt, state_at(C, acc, nd.ps_off), os, lambda));
    } else {
      View cur = Gt;
      for (int k = (int)nd.ch.size() - 1; k >= 0; --k) {
        const TNode& c = P.nodes[nd.ch[k]];
        if (c.identity) continue;
        View nx;
        if (share && k == (int)nd.ch.size() - 1) {
          View zc = z;
          for (auto& a : zc.ax)
            if (a.kind == AX_SK && a.id == v) a.id = c.user;
          for (auto& x : zc.sc)
            if (x.kind == AX_SK && x.id == v) x.id = c.user;
          TTNN_TRY(y_chain(C, zc, c.user, c.lo, c.hi, c.s, &nx, true));
        } else {
          TTNN_TRY(y_chain(C, cur, c.user, c.lo, c.hi, c.s, &nx));
        }
        cur = nx;
      }
      TTNN_TRY(scatter_into(C, cur, state_at(C, acc, nd.ps_off), psi_strides(C, cur, nd, true), lambda));
    }
  }
  // children
  for (size_t k = 0; k < nd.ch.size(); ++k) {
    const TNode& c = P.nodes[nd.ch[k]];
    if (c.rsub == 0) continue;
    View cur = truncate_j(G, c.rsub);
    for (size_t k2 = 0; k2 < nd.ch.size(); ++k2) {
      if (k2 == k) continue;
      const TNode& sib = P.nodes[nd.ch[k2]];
      View nx;
      if (P.variant == TTNN_VARIANT_STTNN && k2 < k && !sib.identity) {
        TTNN_TRY(e_group(C, cur, sib.user, &nx));
        cur = nx;
      } else {
        for (int mm = sib.hi - 1; mm >= sib.lo; --mm) {
          TTNN_TRY(x_mode(C, cur, mm, &nx));
          cur = nx;
        }
      }
    }
    TTNN_TRY(walk(C, acc, c.user, cur, lambda));
  }
  return TTNN_OK;
}

static void side_spec_common(ttnn_plan_s& P, const Box& box, int lo, int hi, SideSpec& s) {
  s.nmodes = hi - lo;
  for (int k = 0; k < s.nmodes; ++k) {
    s.ext[k] = box.ext[lo + k];
    s.off[k] = box.off[lo + k];
    s.full[k] = P.dims[lo + k];
    s.xf[k] = P.fac64 + P.x_off[lo + k];
    s.yf[k] = P.fac64 + P.y_off[lo + k];
  }
  s.rmax = P.rmax;
  s.smax = P.smax;
  s.round_fmt = P.round_fmt;
  s.store = P.side_store;
}

static int store_bytes(int store) { return store == 0 ? 8 : store == 1 ? 4 : store == 2 ? 2 : 1; }

ttnn_status make_side(ttnn_plan_s& P, const Box& box, int which, void* out, int64_t ld,
                      cudaStream_t st, std::vector<GatherJob>* defer) {
  SideSpec s;
  if (which == 0) {   // B_R: rows over R modes
    side_spec_common(P, box, P.Rlo, P.Rhi, s);
    s.x_cols = P.rXL;
    s.y_cols = P.wYR;
    s.y_kind = P.yR_ident;
    s.total_cols = P.wRpad;
    if (P.yside == 0 && P.wYR && !P.yR_ident) {
      // Y block of the single R child = Khatri-Rao over its modes (all R modes)
    }
  } else {
    side_spec_common(P, box, P.Llo, P.Lhi, s);
    s.x_cols = P.rXR;
    s.y_cols = P.wYL;
    s.y_kind = P.yL_ident;
    s.total_cols = P.wLpad;
  }
  s.ld = ld;
  // a box of a plan with cached whole-tensor blocks: cut its rows from them
  const void* cache = which == 0 ? P.sideR : P.sideL;
  if (!box.full && cache) {
    int64_t nfull = 1;
    for (int k = 0; k < s.nmodes; ++k) nfull *= s.full[k];
    if (defer) {
      defer->push_back(GatherJob{s, cache, nfull, out});
      return TTNN_OK;
    }
    return launch_side_gather(s, cache, nfull, out, st);
  }
  return launch_side(s, out, st);
}

// Walk-type copy of the pass Y block (rows over the Y child's box modes).
ttnn_status make_side_yw(ttnn_plan_s& P, const Box& box, void* out, int64_t ld, cudaStream_t st,
                         std::vector<GatherJob>* defer) {
  SideSpec s;
  const TNode& c = P.nodes[P.ychild];
  side_spec_common(P, box, c.lo, c.hi, s);
  s.x_cols = 0;
  s.y_cols = c.s;
  s.y_kind = 0;
  s.total_cols = c.s;
  s.store = P.walk_f64 ? 0 : 1;
  s.ld = ld;
  if (!box.full && P.yW) {
    if (defer) {
      defer->push_back(GatherJob{s, P.yW, c.n, out});
      return TTNN_OK;
    }
    return launch_side_gather(s, P.yW, c.n, out, st);
  }
  return launch_side(s, out, st);
}

// Walk-type copy of the pass X block of the L side (rows over the R modes of
// the box, the rXL columns of B_R): the X factor of Omega for an L-side Y
// child taken through D2.
ttnn_status make_side_xo(ttnn_plan_s& P, const Box& box, void* out, int64_t ld, cudaStream_t st) {
  SideSpec s;
  side_spec_common(P, box, P.Rlo, P.Rhi, s);
  s.x_cols = P.rXL;
  s.y_cols = 0;
  s.y_kind = 0;
  s.total_cols = P.rXL;
  s.store = P.walk_f64 ? 0 : 1;
  s.ld = ld;
  return launch_side(s, out, st);
}

bool omega_via_d2(const ttnn_plan_s& P, int64_t nL, int64_t nR) {
  const TNode& yc = P.nodes[P.ychild];
  return P.yside == 1 && !P.walk_f64 && !yc.identity && P.wYL > 0 && P.rXL > 0 &&
         yc.r <= P.rXL && nR * 2 <= nL && !(P.flags & TTNN_FLAG_DENSE_DRM);
}

ttnn_status UpdateBatch::launch(cudaStream_t st) {
  if (!gathers.empty()) TTNN_TRY(launch_side_gather_batch(gathers.data(), (int)gathers.size(), st));
  for (auto& p : passes) TTNN_TRY(p(st));
  return walks.run(st);
}

ttnn_status dense_update_need(ttnn_plan_s& P, const Box& box, int64_t* need) {
  std::vector<int64_t> key = box.ext;
  key.push_back(box.full ? 1 : 0);
  auto it = P.ws_need_cache.find(key);
  if (it != P.ws_need_cache.end()) {
    *need = it->second;
    return TTNN_OK;
  }
  int64_t n = 0;
  TTNN_TRY(run_dense_update(P, nullptr, nullptr, box, nullptr, 1.0, nullptr, true, &n));
  P.ws_need_cache[key] = n;
  *need = n;
  return TTNN_OK;
}

ttnn_status run_dense_update(ttnn_plan_s& P, void* acc, const void* data, const Box& box,
                             const float* tile_scale, double lambda, cudaStream_t st, bool dry,
                             int64_t* peak, UpdateBatch* batch) {
  if (P.flags & TTNN_FLAG_DENSE_DRM) {
    if (batch) {
      set_error("unstructured Gaussian DRMs: no batched (served) updates");
      return TTNN_EUNSUPPORTED;
    }
    if (!dry) {
      int64_t need = 0;
      TTNN_TRY(dense_update_need(P, box, &need));
      if (need > P.ws_bytes) {
        set_error("dense update needs %lld workspace bytes, the plan holds %lld", (long long)need,
                  (long long)P.ws_bytes);
        return TTNN_ENOMEM;
      }
    }
    return run_dense_drm_update(P, acc, data, box, lambda, st, dry, peak);
  }
  if (!dry && P.dtype == TTNN_E4M3 && (!tile_scale || ((uintptr_t)tile_scale & 3))) {
    set_error("E4M3 updates need their tile scales (4-byte aligned)");
    return TTNN_EINVAL;
  }
  if (!dry) {
    int64_t need = 0;
    TTNN_TRY(dense_update_need(P, box, &need));
    if (need > P.ws_bytes) {
      set_error("dense update needs %lld workspace bytes, the plan holds %lld", (long long)need,
                (long long)P.ws_bytes);
      return TTNN_ENOMEM;
    }
  }
  Ws ws(P.ws, P.ws_bytes, dry);
  Program prog;
  ws.prog = &prog;
  const int eb = P.walk_f64 ? 8 : 4;
  Ctx C{P, ws, st, dry, eb, P.walk_f64 ? ET_F64 : ET_F32, box, (const char*)P.facw, nullptr, 0,
        &prog};
  int64_t nL = 1, nR = 1;
  for (int m = P.Llo; m < P.Lhi; ++m) nL *= box.ext[m];
  for (int m = P.Rlo; m < P.Rhi; ++m) nR *= box.ext[m];
  const int sb = store_bytes(P.side_store);
  // A box whose right (r1 = 1) or left (r1 = 2) pass side is a single index:
  // the product against that side is rank one, M times one row of its side
  // block, and is left to the walk as a broadcast with that row as a pending
  // scale; the product against the other side is a matrix-vector product
  // with its side block, read straight from the cached whole-tensor block
  // when there is one (no box block is formed).
  const bool r1_fmt = P.dtype == TTNN_F64 || P.dtype == TTNN_F32 || P.dtype == TTNN_BF16 ||
                      P.dtype == TTNN_BF16X2 || P.dtype == TTNN_E4M3;
  const int r1 = !r1_fmt || (P.flags & TTNN_FLAG_SIMT_PASS) ? 0
                 : (nR == 1 && nL > 1)                       ? 1
                 : (nL == 1 && nR > 1)                       ? 2
                                                             : 0;
  // side blocks of the box
  const void* sR = nullptr;
  const void* sL = nullptr;
  if (box.full && P.sideR) sR = P.sideR;
  if (box.full && P.sideL) sL = P.sideL;
  // the matrix-vector side of a rank-one box: source block, its leading
  // dimension, and whether rows are cut from the whole-tensor block
  const void* gsrc = nullptr;
  int64_t gld = 0;
  bool gcut = false;
  if (r1) {
    const bool right = r1 == 2;                 // the matrix-vector side is R
    const void* cache = right ? P.sideR : P.sideL;
    const int64_t rows = right ? nR : nL;
    if (box.full && cache) {
      gsrc = cache;
      gld = rows;
    } else if (cache) {
      int64_t nfull = 1;
      for (int m = right ? P.Rlo : P.Llo; m < (right ? P.Rhi : P.Lhi); ++m) nfull *= P.dims[m];
      gsrc = cache;
      gld = nfull;
      gcut = true;
    }
    if (right) sR = gsrc;
    else sL = gsrc;
  }
  if (P.wR > 0 && !sR) {
    char* b = ws.alloc((int64_t)P.wRpad * nR * sb);
    if (!dry) TTNN_TRY(make_side(P, box, 0, b, nR, st, batch ? &batch->gathers : nullptr));
    sR = b;
    if (r1 == 2) {
      gsrc = b;
      gld = nR;
    }
  }
  if (P.wL > 0 && !sL) {
    char* b = ws.alloc((int64_t)P.wLpad * nL * sb);
    if (!dry) TTNN_TRY(make_side(P, box, 1, b, nL, st, batch ? &batch->gathers : nullptr));
    sL = b;
    if (r1 == 1) {
      gsrc = b;
      gld = nL;
    }
  }
  // rank-one box whose Y child lies on the matrix-vector side: the walk takes
  // the Y child's Omega from that product and needs no Y block
  const bool y_from_gemv = (r1 == 1 && P.yside == 1) || (r1 == 2 && P.yside == 0);
  // whole 2-D boxes with an L-side Y child take its Omega through D2 and
  // need no Y block copy
  const bool y_via_d2 = r1 == 0 && omega_via_d2(P, nL, nR);
  if (!P.nodes[P.ychild].identity && !y_from_gemv && !y_via_d2) {
    const TNode& yc = P.nodes[P.ychild];
    int64_t ny = 1;
    for (int m = yc.lo; m < yc.hi; ++m) ny *= box.ext[m];
    C.yw_ld = ny;
    if (box.full && P.yW) {
      C.yw = (const char*)P.yW;
    } else {
      char* b = ws.alloc((int64_t)yc.s * ny * eb);
      if (!dry) TTNN_TRY(make_side_yw(P, box, b, ny, st, batch ? &batch->gathers : nullptr));
      C.yw = b;
    }
  }
  // first-level pass: D1 = M B_R^T (nL x wRpad), D2 = M^T B_L^T (nR x wLpad);
  // for a rank-one box only the matrix-vector product (one row), plus walk
  // copies of M and of the broadcast side row when the formats differ
  char* D1 = r1 == 1 ? nullptr : ws.alloc(nL * P.wRpad * eb);
  char* D2 = r1 == 2 ? nullptr : ws.alloc(nR * P.wLpad * eb);
  const int64_t r1_rows = r1 == 1 ? nL : nR;
  const int r1_bpad = r1 == 1 ? P.wRpad : P.wLpad;
  const void* r1_brow = r1 == 1 ? sR : sL;
  // the rows' format for the rank-one kernels (BF16x2 rows are split, E4M3
  // rows dequantised with their tile scales)
  const int r1_store = P.dtype == TTNN_BF16X2 ? kStoreSplit
                       : P.dtype == TTNN_E4M3 ? kStoreFp8
                                              : P.pass_store;
  const bool r1_copy = r1_store == 2 || r1_store == kStoreSplit || r1_store == kStoreFp8;
  const char* Mw = r1 && r1_copy ? ws.alloc(r1_rows * eb) : (const char*)data;
  const char* bw = r1 && P.side_store == 2 ? ws.alloc((int64_t)r1_bpad * eb) : (const char*)r1_brow;
  if (y_from_gemv) C.yom = r1 == 1 ? D2 + (int64_t)P.rXR * eb : D1 + (int64_t)P.rXL * eb;
  if (y_via_d2) {
    C.d2y = D2 + (int64_t)P.rXR * eb;
    C.d2y_ld = P.wLpad;
    C.nRo = nR;
    if (box.full && P.xWo) {
      C.xo = (const char*)P.xWo;
    } else {
      char* b = ws.alloc((int64_t)P.rXL * nR * eb);
      if (!dry) TTNN_TRY(make_side_xo(P, box, b, nR, st));
      C.xo = b;
    }
  }
  cudaEvent_t ev0 = dry ? nullptr : prof_event(P, st);
  // the pass's own temporaries are released right after it and are not
  // program buffers: keep them out of the dependency registry
  ws.prog = nullptr;
  // binary32 plans: whole-tensor updates on the tensor cores with the split
  // (bf16 hi + lo) data and DRM blocks
  const bool f32s = P.dtype == TTNN_F32 && box.full && P.sideRs && P.sideLs &&
                    !(P.flags & TTNN_FLAG_SIMT_PASS);
  const bool cvt = P.dtype == TTNN_BF16X2 || P.dtype == TTNN_E4M3 || f32s;
  const bool use_tc = (P.tc_ok || f32s) && !(P.flags & TTNN_FLAG_SIMT_PASS) &&
                      (cvt ? cvt_pass_supported(P, nL, nR) : tc_pass_supported(P, nL, nR)) ==
                          TTNN_OK;
  if (r1) {
    const int64_t mark = ws.top;
    SideSpec gs;
    if (r1 == 1) side_spec_common(P, box, P.Llo, P.Lhi, gs);
    else side_spec_common(P, box, P.Rlo, P.Rhi, gs);
    const int gcols = r1 == 1 ? P.wL : P.wR, gpad = r1 == 1 ? P.wLpad : P.wRpad;
    void* Dout = r1 == 1 ? (void*)D2 : (void*)D1;
    int64_t need = 0;
    TTNN_TRY(launch_side_gemv(gs, nullptr, 0, false, nullptr, r1_store, nullptr, r1_rows, gcols,
                              gpad, nullptr, P.walk_f64, nullptr, 0, st, true, &need));
    char* part = ws.alloc(need);
    if (!dry) {
      ++P.n_simt_pass;
      const int pstore = r1_store, sstore = P.side_store, wf64 = P.walk_f64 ? 1 : 0;
      auto go = [=](cudaStream_t s) -> ttnn_status {
        if (Mw != (const char*)data)
          TTNN_TRY(launch_to_walk(data, pstore, tile_scale, (void*)Mw, wf64, r1_rows, s));
        if (bw != (const char*)r1_brow)
          TTNN_TRY(launch_to_walk(r1_brow, sstore, nullptr, (void*)bw, wf64, r1_bpad, s));
        return launch_side_gemv(gs, gsrc, gld, gcut, data, pstore, tile_scale, r1_rows, gcols,
                                gpad, Dout, wf64, part, need, s, false, nullptr);
      };
      if (batch) batch->passes.push_back(go);
      else TTNN_TRY(go(st));
    }
    ws.top = mark;
  } else if (use_tc) {
    auto launch = cvt ? launch_cvt_pass : launch_tc_pass;
    const int64_t mark = ws.top;
    int64_t need = 0;
    TTNN_TRY(launch(P, data, nL, nR, sR, nR, sL, nL, D1, D2, tile_scale, nullptr, 0, st, true,
                    &need));
    char* tw = ws.alloc(need);
    if (!dry) {
      ++P.n_tc_pass;
      auto go = [&P, launch, data, nL, nR, sR, sL, D1, D2, tile_scale, tw, need](cudaStream_t s) {
        return launch(P, data, nL, nR, sR, nR, sL, nL, D1, D2, tile_scale, tw, need, s, false,
                      nullptr);
      };
      if (batch) {
        batch->passes.push_back(go);
      } else {
        // profiling: the pass kernel alone, from just before its launch to
        // the event the launch records right after it
        cudaEvent_t k0 = prof_event(P, st), k1 = nullptr;
        if (k0 && cudaEventCreate(&k1) != cudaSuccess) k1 = nullptr;
        P.prof_kernel_end = k1;
        const ttnn_status ls = go(st);
        P.prof_kernel_end = nullptr;
        prof_push(P, 3, k0, k1);
        TTNN_TRY(ls);
      }
    }
    // released: in stream order the walk (which reuses the bytes) runs after
    // the pass, deferred or not
    ws.top = mark;
  } else {
    if (P.pass_store == 3 || P.dtype == TTNN_BF16X2) {
      set_error("this number format needs the tensor-core pass (unsupported shape)");
      return TTNN_EUNSUPPORTED;
    }
    const int in_type = P.pass_store == 0 ? 0 : P.pass_store == 1 ? 1 : 2;
    if (!dry) ++P.n_simt_pass;
    if (P.wR > 0) {
      Gemm g;
      g.I = nL; g.Jn = P.wR; g.K = nR;
      g.A = data; g.asi = nR; g.ask = 1;
      g.B = sR; g.bsj = nR; g.bsk = 1;
      g.C = D1; g.ldc = P.wRpad; g.in_type = in_type;
      const int ns = gemm_choose_split(g);
      const int64_t mark = ws.top;
      char* part = ns > 1 ? ws.alloc((int64_t)ns * nL * P.wRpad * eb) : nullptr;
      if (!dry) {
        if (batch) batch->passes.push_back([g, ns, part](cudaStream_t s) { return launch_gemm(g, ns, part, s); });
        else TTNN_TRY(launch_gemm(g, ns, part, st));
      }
      ws.top = mark;
    }
    if (P.wL > 0) {
      Gemm g;
      g.I = nR; g.Jn = P.wL; g.K = nL;
      g.A = data; g.asi = 1; g.ask = nR;
      g.B = sL; g.bsj = nL; g.bsk = 1;
      g.C = D2; g.ldc = P.wLpad; g.in_type = in_type;
      const int ns = gemm_choose_split(g);
      const int64_t mark = ws.top;
      char* part = ns > 1 ? ws.alloc((int64_t)ns * nR * P.wLpad * eb) : nullptr;
      if (!dry) {
        if (batch) batch->passes.push_back([g, ns, part](cudaStream_t s) { return launch_gemm(g, ns, part, s); });
        else TTNN_TRY(launch_gemm(g, ns, part, st));
      }
      ws.top = mark;
    }
  }
  ws.prog = &prog;
  // each interval owns its two events (an event is destroyed with its interval)
  prof_push(P, 0, ev0, dry ? nullptr : prof_event(P, st));
  cudaEvent_t ev1 = dry ? nullptr : prof_event(P, st);
  // views of the pass products
  auto mode_axes = [&](int lo, int hi) {
    std::vector<Ax> ax;
    for (int m = lo; m < hi; ++m) ax.push_back(Ax{AX_MODE, m, box.ext[m], box.off[m]});
    return ax;
  };
  // a rank-one product: M (walk copy) with a broadcast last axis scaled by
  // the row `scale` of the single-index side's block
  auto bview = [&](int lo, int hi, Ax last, int64_t logical, const char* scale) {
    View v{(char*)Mw, mode_axes(lo, hi), 1};
    last.bc = logical;
    v.ax.push_back(last);
    v.sc.push_back(View::Scale{last.kind, last.id, scale});
    return v;
  };
  const TNode& root = P.nodes[P.root];
  // Khatri-Rao prefix (TTNN, binary32 walk, whole first-level products): with
  // one left root child Lc whose first child c1 spans Lc's leading modes with
  // s_c1 = s_Lc, the Y chains of Omega_Lc, of Psi_Lc's c1 axis and of the
  // root's Psi (its L axis, when the root's Y is on the R side) all start by
  // contracting c1's modes with the same columns of kr(Y_mu, mu in c1).  That
  // contraction runs as one long reduction over c1's merged index on each of
  // D1's two column groups (G_Lc and the root's H), instead of mode by mode
  // through large intermediates.
  const TNode* krL = nullptr;
  if (P.variant == TTNN_VARIANT_TTNN && r1 == 0 && !P.walk_f64 && P.Lch.size() == 1) {
    const TNode& Lc = P.nodes[P.Lch[0]];
    if (Lc.sketched() && !Lc.leaf && Lc.user != P.ychild && Lc.r <= P.rXL && Lc.s <= 32) {
      const TNode& c1 = P.nodes[Lc.ch.front()];
      int64_t n1 = 1;
      for (int m = c1.lo; m < c1.hi; ++m) n1 *= box.ext[m];
      if (!c1.identity && c1.s == Lc.s && c1.lo == P.Llo && c1.hi - c1.lo <= 4 && n1 >= 512 &&
          n1 < (int64_t(1) << 31))
        krL = &Lc;
    }
  }
  // L side (both variants): G over L modes from D1's X part
  if (P.rXL > 0) {
    View GL{D1, mode_axes(P.Llo, P.Lhi), P.wRpad};
    GL.ax.push_back(Ax{AX_J, -1, P.rXL, 0});
    if (r1 == 1) GL = bview(P.Llo, P.Lhi, Ax{AX_J, -1, 1, 0}, P.rXL, bw);
    if (krL) {
      const TNode& c1 = P.nodes[krL->ch.front()];
      View pre;
      TTNN_TRY(kr_prefix(C, truncate_j(GL, krL->r), c1.user, c1.lo, c1.hi, c1.s, &pre));
      TTNN_TRY(walk(C, acc, krL->user, truncate_j(GL, krL->rsub), lambda, &pre));
    }
    for (size_t k = 0; k < P.Lch.size() && !krL; ++k) {
      const TNode& c = P.nodes[P.Lch[k]];
      if (c.rsub == 0) continue;
      View cur = truncate_j(GL, c.rsub);
      for (size_t k2 = 0; k2 < P.Lch.size(); ++k2) {
        if (k2 == k) continue;
        const TNode& sib = P.nodes[P.Lch[k2]];
        for (int mm = sib.hi - 1; mm >= sib.lo; --mm) {
          View nx;
          TTNN_TRY(x_mode(C, cur, mm, &nx));
          cur = nx;
        }
      }
      TTNN_TRY(walk(C, acc, c.user, cur, lambda));
    }
  }
  if (P.variant == TTNN_VARIANT_TTNN) {
    if (P.rXR > 0) {
      View GR{D2, mode_axes(P.Rlo, P.Rhi), P.wLpad};
      GR.ax.push_back(Ax{AX_J, -1, P.rXR, 0});
      if (r1 == 2) GR = bview(P.Rlo, P.Rhi, Ax{AX_J, -1, 1, 0}, P.rXR, bw);
      for (size_t k = 0; k < P.Rch.size(); ++k) {
        const TNode& c = P.nodes[P.Rch[k]];
        if (c.rsub == 0) continue;
        View cur = truncate_j(GR, c.rsub);
        for (size_t k2 = 0; k2 < P.Rch.size(); ++k2) {
          if (k2 == k) continue;
          const TNode& sib = P.nodes[P.Rch[k2]];
          for (int mm = sib.hi - 1; mm >= sib.lo; --mm) {
            View nx;
            TTNN_TRY(x_mode(C, cur, mm, &nx));
            cur = nx;
          }
        }
        TTNN_TRY(walk(C, acc, c.user, cur, lambda));
      }
    }
    // root Psi
    if (P.yside == 0) {
      View H{D1 + (int64_t)P.rXL * eb, mode_axes(P.Llo, P.Lhi), P.wRpad};
      H.ax.push_back(Ax{AX_SK, P.ychild, P.wYR, 0});
      if (r1 == 1 && P.yR_ident && P.Rhi - P.Rlo == 1) {
        // identity Y child: its row is one-hot, so only the fixed index of
        // the state is touched (a raw mode axis at the box offset)
        H = View{(char*)Mw, mode_axes(P.Llo, P.Lhi), 1};
        H.ax.push_back(Ax{AX_MODE, P.Rlo, 1, box.off[P.Rlo]});
      } else if (r1 == 1) {
        H = bview(P.Llo, P.Lhi, Ax{AX_SK, P.ychild, 1, 0}, P.wYR, bw + (int64_t)P.rXL * eb);
      }
      View cur = H;
      if (krL) {
        const TNode& c1 = P.nodes[krL->ch.front()];
        View e;
        TTNN_TRY(kr_prefix(C, H, krL->user, c1.lo, c1.hi, krL->s, &e));
        TTNN_TRY(y_chain_rest(C, e, krL->user, c1.hi, krL->hi, &cur));
      }
      for (int k = (int)P.Lch.size() - 1; k >= 0 && !krL; --k) {
        const TNode& c = P.nodes[P.Lch[k]];
        if (c.identity) continue;
        View nx;
        TTNN_TRY(y_chain(C, cur, c.user, c.lo, c.hi, c.s, &nx));
        cur = nx;
      }
      std::vector<int64_t> os = psi_strides(C, cur, root, false);
      // the last axis is the R child's pass-side sketch (or its full raw index)
      os.back() = 1;
      TTNN_TRY(scatter_into(C, cur, state_at(C, acc, root.ps_off), os, lambda));
    } else {
      View H{D2 + (int64_t)P.rXR * eb, mode_axes(P.Rlo, P.Rhi), P.wLpad};
      H.ax.push_back(Ax{AX_SK, P.ychild, P.wYL, 0});
      if (r1 == 2 && P.yL_ident && P.Lhi - P.Llo == 1) {
        H = View{(char*)Mw, mode_axes(P.Rlo, P.Rhi), 1};
        H.ax.push_back(Ax{AX_MODE, P.Llo, 1, box.off[P.Llo]});
      } else if (r1 == 2) {
        H = bview(P.Rlo, P.Rhi, Ax{AX_SK, P.ychild, 1, 0}, P.wYL, bw + (int64_t)P.rXR * eb);
      }
      View cur = H;
      for (int k = (int)P.Rch.size() - 1; k >= 0; --k) {
        const TNode& c = P.nodes[P.Rch[k]];
        if (c.identity) continue;
        View nx;
        TTNN_TRY(y_chain(C, cur, c.user, c.lo, c.hi, c.s, &nx));
        cur = nx;
      }
      std::vector<int64_t> os = psi_strides(C, cur, root, false);
      int64_t rest = 1;
      for (size_t k = 1; k < root.ch.size(); ++k) {
        const TNode& c = P.nodes[root.ch[k]];
        rest *= c.identity ? c.n : c.s;
      }
      os.back() = rest;
      TTNN_TRY(scatter_into(C, cur, state_at(C, acc, root.ps_off), os, lambda));
    }
  } else {
    // STTNN: D2 = M^T Y_c1 (nR x s'_c1): R children and the root
    View H{D2, mode_axes(P.Rlo, P.Rhi), P.wLpad};
    H.ax.push_back(Ax{AX_SK, P.ychild, P.wYL, 0});
    if (r1 == 2) H = bview(P.Rlo, P.Rhi, Ax{AX_SK, P.ychild, 1, 0}, P.wYL, bw);
    const TNode& c1 = P.nodes[P.ychild];
    for (size_t k = 0; k < P.Rch.size(); ++k) {
      const TNode& c = P.nodes[P.Rch[k]];
      if (c.rsub == 0) continue;
      // contract the c1 sketch axis with XT_c1: creates the column axis
      View cur;
      Ax jax{AX_J, -1, c.rsub, 0};
      TTNN_TRY(contract_view(C, H, (int)H.ax.size() - 1, C.facw + c1.xt_off * eb, P.rmax, 1, -1,
                             &jax, &cur));
      for (size_t k2 = 0; k2 < P.Rch.size(); ++k2) {
        if (k2 == k) continue;
        const TNode& sib = P.nodes[P.Rch[k2]];
        View nx;
        if (k2 < k && !sib.identity) {
          TTNN_TRY(e_group(C, cur, sib.user, &nx));
          cur = nx;
        } else {
          for (int mm = sib.hi - 1; mm >= sib.lo; --mm) {
            TTNN_TRY(x_mode(C, cur, mm, &nx));
            cur = nx;
          }
        }
      }
      TTNN_TRY(walk(C, acc, c.user, cur, lambda));
    }
    View cur = H;
    for (int k = (int)P.Rch.size() - 1; k >= 0; --k) {
      const TNode& c = P.nodes[P.Rch[k]];
      if (c.identity) continue;
      View nx;
      TTNN_TRY(y_chain(C, cur, c.user, c.lo, c.hi, c.s, &nx));
      cur = nx;
    }
    std::vector<int64_t> os = psi_strides(C, cur, root, false);
    int64_t rest = 1;
    for (size_t k = 1; k < root.ch.size(); ++k) {
      const TNode& c = P.nodes[root.ch[k]];
      rest *= c.identity ? c.n : c.s;
    }
    os.back() = rest;
    TTNN_TRY(scatter_into(C, cur, state_at(C, acc, root.ps_off), os, lambda));
  }
  if (!dry) {
    if (batch) batch->walks.absorb(prog);
    else TTNN_TRY(prog.run(st, P.flags & TTNN_FLAG_DUMP_PROGRAM));
  }
  P.last_walk_ops = (int)prog.size();
  P.last_walk_levels = prog.levels();
  cudaEvent_t ev2 = dry ? nullptr : prof_event(P, st);
  prof_push(P, 1, ev1, ev2);
  if (peak) *peak = ws.peak;
  if (!ws.ok()) {
    set_error("internal: workspace overflow (%lld > %lld)", (long long)ws.peak, (long long)ws.cap);
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}

// ---------------------------------------------------------------------------
// TTN-format input (Sec. 7, structured sketchings; TTN rounding)
// ---------------------------------------------------------------------------
// With Khatri-Rao DRMs every sketch entry of a TTN input is a contraction of
// its cores with rank-one vectors, formed by two sweeps:
//   up    UX_t[a, j] = sum_b C_t[a, b_1..b_m] prod_k UX_ck[b_k, j]
//         (leaf: sum_i C_t[a, i] kr(X_mu, mu in t)[i, j]); UY_t likewise with Y_mu
//   down  E_ck[b_k, j] = sum C_t[a, b..] E_t[a, j] prod_{k' != k} UX_ck'[b_k', j]
//         (root: without E_t)
//   Omega_t = UY_t[:, :s_t]^T E_t[:, :r_t];  Psi_leaf = C_t^T E_t;
//   Psi_t = C_t x_a E_t x_bk V_ck (V_c = UY_c[:, :s_c], or the raw core C_c of
//   an identity child);  Psi_root = C_root x_bk V_ck.
// The DRM factors are the stored (rounded) values; products are taken in
// the walk type, never rounded to the pass format.
namespace {

constexpr int kRankAxis = -1000;   // id offset of input-rank axes (AX_SK)

// Weight strides (wsI, wsX) of a two-axis view used as W(i, x), i on axis ki.
void view_w(const View& w, int ki, int64_t* wsI, int64_t* wsX) {
  *wsI = vstride(w, ki);
  *wsX = vstride(w, 1 - ki);
}

// Position of the column axis (AX_J) in a view, -1 if none.
int j_axis(const View& v) { return find_ax(v, AX_J, -1); }

}  // namespace

ttnn_status run_ttn_update(ttnn_plan_s& P, void* acc, const double* const* cores_in,
                           const int32_t* ranks_in, double lambda, cudaStream_t st, bool dry,
                           int64_t* peak) {
  if (P.flags & TTNN_FLAG_DENSE_DRM) {
    set_error("TTN-format updates need the Khatri-Rao DRMs");
    return TTNN_EUNSUPPORTED;
  }
  if (P.variant != TTNN_VARIANT_TTNN) {
    set_error("TTN-format updates take TTNN plans");
    return TTNN_EUNSUPPORTED;
  }
  Box box;
  box.off.assign(P.d, 0);
  box.ext = P.dims;
  box.full = true;
  Ws ws(P.ws, P.ws_bytes, dry);
  Program prog;
  ws.prog = &prog;
  const int eb = P.walk_f64 ? 8 : 4;
  Ctx C{P, ws, st, dry, eb, P.walk_f64 ? ET_F64 : ET_F32, box, (const char*)P.facw, nullptr, 0,
        &prog};
  const int nn = (int)P.nodes.size();
  auto R = [&](int v) { return (int64_t)ranks_in[v]; };
  // input cores in the walk type (binary32 plans: converted copies)
  std::vector<const char*> core(nn, nullptr);
  ConvertBatch conv;
  for (int v = 0; v < nn; ++v) {
    const TNode& nd = P.nodes[v];
    int64_t el = 1;
    if (v != P.root) el *= R(v);
    if (nd.leaf) el *= nd.n;
    else
      for (int c : nd.ch) el *= R(c);
    if (P.walk_f64) {
      core[v] = (const char*)cores_in[v];
      prog.buffer(core[v], el * 8);
    } else {
      char* b = ws.alloc(el * 4);
      if (conv.count == kConvertSegs) {
        if (!dry) TTNN_TRY(launch_convert_batch(conv, st));
        conv.count = 0;
      }
      conv.src[conv.count] = cores_in[v];
      conv.dst[conv.count] = (float*)b;
      conv.n[conv.count] = el;
      ++conv.count;
      core[v] = b;
    }
  }
  if (!dry && conv.count > 0) TTNN_TRY(launch_convert_batch(conv, st));
  auto core_view = [&](int v) {
    const TNode& nd = P.nodes[v];
    View w;
    w.ptr = (char*)core[v];
    if (v != P.root) w.ax.push_back(Ax{AX_SK, kRankAxis - v, R(v), 0});
    if (nd.leaf) {
      w.ax.push_back(Ax{AX_SK, v, nd.n, 0});
    } else {
      for (int c : nd.ch) w.ax.push_back(Ax{AX_SK, kRankAxis - c, R(c), 0});
    }
    w.ld = w.ax.back().size;
    return w;
  };
  // up sweep: UX_v (R_v x rmax), UY_v (R_v x smax), children before parents
  std::vector<View> UX(nn), UY(nn);
  for (int li = (int)P.lex.size() - 1; li >= 0; --li) {
    const int v = P.lex[li];
    if (v == P.root) continue;
    const TNode& nd = P.nodes[v];
    for (int which = 0; which < 2; ++which) {
      const int64_t w = which == 0 ? P.rmax : P.smax;
      View cur = core_view(v);
      if (nd.leaf) {
        // the leaf's raw axis as its modes (row-major), then Khatri-Rao
        View m;
        m.ptr = cur.ptr;
        m.ax = {cur.ax[0]};
        for (int mu = nd.lo; mu < nd.hi; ++mu) m.ax.push_back(Ax{AX_MODE, mu, P.dims[mu], 0});
        m.ld = m.ax.back().size;
        cur = m;
        for (int mu = nd.hi - 1; mu >= nd.lo; --mu) {
          const int k = find_ax(cur, AX_MODE, mu);
          const char* F = which == 0 ? facX(C, mu) : facY(C, mu);
          View nx;
          if (mu == nd.hi - 1) {
            Ax nax{AX_J, -1, w, 0};
            TTNN_TRY(contract_view(C, cur, k, F, w, 1, -1, &nax, &nx));
          } else {
            TTNN_TRY(contract_view(C, cur, k, F, w, 1, (int)cur.ax.size() - 1, nullptr, &nx));
          }
          cur = nx;
        }
      } else {
        for (int k = (int)nd.ch.size() - 1; k >= 0; --k) {
          const int c = nd.ch[k];
          const View& uc = which == 0 ? UX[c] : UY[c];
          const int ka = find_ax(cur, AX_SK, kRankAxis - c);
          int64_t wsI, wsX;
          view_w(uc, 0, &wsI, &wsX);
          View nx;
          if (k == (int)nd.ch.size() - 1) {
            Ax nax{AX_J, -1, w, 0};
            TTNN_TRY(contract_view(C, cur, ka, uc.ptr, wsI, wsX, -1, &nax, &nx));
          } else {
            TTNN_TRY(contract_view(C, cur, ka, uc.ptr, wsI, wsX, (int)cur.ax.size() - 1, nullptr,
                                   &nx));
          }
          cur = nx;
        }
      }
      (which == 0 ? UX[v] : UY[v]) = cur;
    }
  }
  // down sweep: E_c has two axes, the rank axis of c and the column axis.
  // Every other axis of C_v is contracted; the column axis is created by
  // the first contraction and each later one shares it (it is either the
  // last axis, or sits right before c's axis).
  std::vector<View> E(nn);
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (nd.leaf || (v != P.root && nd.rsub == 0)) continue;
    for (int c : nd.ch) {
      if (P.nodes[c].rsub == 0) continue;
      const int bc = kRankAxis - c;
      auto is_c = [&](const Ax& a) { return a.kind == AX_SK && a.id == bc; };
      View cur = core_view(v);
      bool have_j = false;
      while (!have_j || cur.ax.size() > 2) {
        const int L = (int)cur.ax.size() - 1;
        int pick, shared = -1;
        if (!have_j) {
          pick = is_c(cur.ax[L]) ? L - 1 : L;
        } else if (j_axis(cur) == L) {
          pick = is_c(cur.ax[0]) ? 1 : 0;
          shared = L;
        } else {
          shared = j_axis(cur);   // layout [..., x, j, c]
          pick = shared - 1;
        }
        const int id = cur.ax[pick].id;
        const View& Wv = id == kRankAxis - v ? E[v] : UX[kRankAxis - id];
        const int ki = id == kRankAxis - v ? find_ax(E[v], AX_SK, id) : 0;
        int64_t wsI, wsX;
        view_w(Wv, ki, &wsI, &wsX);
        View nx;
        if (!have_j) {
          Ax nax{AX_J, -1, P.nodes[c].rsub, 0};
          TTNN_TRY(contract_view(C, cur, pick, Wv.ptr, wsI, wsX, -1, &nax, &nx));
          have_j = true;
        } else {
          TTNN_TRY(contract_view(C, cur, pick, Wv.ptr, wsI, wsX, shared, nullptr, &nx));
        }
        cur = nx;
      }
      E[c] = cur;
    }
  }
  // sketches.  V_c: UY_c (first s_c columns) or the raw core of an identity c
  auto children_y = [&](View cur, const TNode& nd, View* out) -> ttnn_status {
    for (int k = (int)nd.ch.size() - 1; k >= 0; --k) {
      const int c = nd.ch[k];
      const TNode& cn = P.nodes[c];
      const View Wc = cn.identity ? core_view(c) : UY[c];
      const int ka = find_ax(cur, AX_SK, kRankAxis - c);
      int64_t wsI, wsX;
      view_w(Wc, 0, &wsI, &wsX);
      Ax nax{AX_SK, c, cn.identity ? cn.n : (int64_t)cn.s, 0};
      View nx;
      TTNN_TRY(contract_view(C, cur, ka, Wc.ptr, wsI, wsX, -1, &nax, &nx));
      cur = nx;
    }
    *out = cur;
    return TTNN_OK;
  };
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (v == P.root) {
      View cur;
      TTNN_TRY(children_y(core_view(v), nd, &cur));
      TTNN_TRY(scatter_into(C, cur, state_at(C, acc, nd.ps_off), psi_strides(C, cur, nd, false),
                            lambda));
      continue;
    }
    if (!nd.sketched()) continue;
    const View& Et = E[v];
    const int ka = find_ax(Et, AX_SK, kRankAxis - v);
    {  // Omega_t = UY_t[:, :s_t]^T E_t[:, :r_t]
      View e = Et;
      e.ax[j_axis(e)].size = nd.r;   // the first or the last axis: strides unchanged
      int64_t wsI, wsX;
      view_w(UY[v], 0, &wsI, &wsX);
      Ax nax{AX_SK, v, nd.s, 0};
      View om;
      TTNN_TRY(contract_view(C, e, ka, UY[v].ptr, wsI, wsX, -1, &nax, &om));
      std::vector<int64_t> os(2);
      for (int a = 0; a < 2; ++a) os[a] = om.ax[a].kind == AX_J ? 1 : nd.r;
      TTNN_TRY(scatter_into(C, om, state_at(C, acc, nd.om_off), os, lambda));
    }
    {  // Psi_t: C_t's parent rank axis against E_t (new column axis first)
      int64_t wsI, wsX;
      view_w(Et, ka, &wsI, &wsX);
      Ax nax{AX_J, -1, nd.r, 0};
      View cur;
      TTNN_TRY(contract_view(C, core_view(v), 0, Et.ptr, wsI, wsX, -1, &nax, &cur));
      if (nd.leaf) {
        TTNN_TRY(scatter_into(C, cur, state_at(C, acc, nd.ps_off), {1, (int64_t)nd.r}, lambda));
      } else {
        View y;
        TTNN_TRY(children_y(cur, nd, &y));
        TTNN_TRY(scatter_into(C, y, state_at(C, acc, nd.ps_off), psi_strides(C, y, nd, true),
                              lambda));
      }
    }
  }
  if (!dry) TTNN_TRY(prog.run(st, P.flags & TTNN_FLAG_DUMP_PROGRAM));
  if (peak) *peak = ws.peak;
  if (!ws.ok()) {
    set_error("internal: workspace overflow (%lld > %lld)", (long long)ws.peak, (long long)ws.cap);
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}

cudaEvent_t prof_event(ttnn_plan_s& P, cudaStream_t st) {
  if (!P.profile) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, st);
  return e;
}

void prof_push(ttnn_plan_s& P, int phase, cudaEvent_t a, cudaEvent_t b) {
  if (!a || !b) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return;
  }
  auto& v = P.prof[phase];
  if (v.size() >= 4096) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return;
  }
  v.emplace_back(a, b);
}

// ---------------------------------------------------------------------------
// recovery: QR / eps-pseudo-inverse, then core assembly in binary64
// ---------------------------------------------------------------------------
ttnn_status plan_sync(ttnn_plan_s& P) {
  if (!P.kept_pending) return TTNN_OK;
  P.kept_pending = false;
  TTNN_TRY_CUDA(cudaEventSynchronize(P.kept_ev));
  const size_t nj = P.kept_nodes.size();
  for (size_t k = 0; k < nj; ++k) {
    P.nodes[P.kept_nodes[k]].kept = P.host_kept[k];
    P.nodes[P.kept_nodes[k]].sweeps = P.host_kept[nj + k];
  }
  const int err = P.host_kept[2 * nj];
  if (err) {
    TTNN_TRY_CUDA(cudaMemset(P.err_dev, 0, sizeof(int)));
    set_error("a bounded device wait ran out in an earlier update or recovery (code %d)", err);
    return TTNN_ETIMEOUT;
  }
  return TTNN_OK;
}

ttnn_status run_recover(ttnn_plan_s& P, const void* acc, double* cores, cudaStream_t st, bool dry,
                        int64_t* peak, bool async) {
  Ws ws(P.ws_rec, P.ws_rec_bytes, dry);
  // eps-truncated output: the cores are assembled rank-padded in the
  // workspace, then copied into their kept shapes
  const bool trunc = (P.flags & TTNN_FLAG_TRUNCATE) != 0;
  double* padded = trunc ? (double*)ws.alloc(P.core_elems * 8) : nullptr;
  double* const out_cores = cores;
  if (trunc) cores = padded;
  Program prog;
  cudaEvent_t ev0 = dry ? nullptr : prof_event(P, st);
  const int seb = P.walk_f64 ? 8 : 4;
  const ElemType set = P.walk_f64 ? ET_F64 : ET_F32;
  std::vector<QrJob> jobs;
  std::vector<int> job_node;
  std::vector<double*> Qp(P.nodes.size(), nullptr), Rp(P.nodes.size(), nullptr);
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    double* q = (double*)ws.alloc((int64_t)nd.s * nd.r * 8);
    double* rp = (double*)ws.alloc((int64_t)nd.r * nd.r * 8);
    Qp[v] = q;
    Rp[v] = rp;
    jobs.push_back(QrJob{(const char*)acc + nd.om_off * seb, q, rp, nd.s, nd.r});
    job_node.push_back(v);
  }
  if (!dry && !jobs.empty()) {
    if (jobs.size() != P.jobs_host.size() ||
        memcmp(jobs.data(), P.jobs_host.data(), jobs.size() * sizeof(QrJob)) != 0) {
      TTNN_TRY_CUDA(cudaMemcpyAsync(P.jobs_dev, jobs.data(), jobs.size() * sizeof(QrJob),
                                    cudaMemcpyHostToDevice, st));
      P.jobs_host = jobs;
    }
    TTNN_TRY(launch_qr_pinv(P.jobs_dev, (int)jobs.size(), P.rmax, P.walk_f64, P.eps_factor, P.u,
                            P.kept_dev, trunc ? 1 : 0, st));
  }
  ws.prog = &prog;   // Q and R_eps^+ above are produced before the program (level 0)
  // contraction of axis k of a contiguous tensor `dims` with W(i, b) =
  // W[i*wsI + b*wsB] into a new axis of nb, written with strides (osP, osB, osQ)
  auto mp = [&](const void* in, bool in_state, const std::vector<int64_t>& dims, int k,
                const double* W, int64_t wsI, int64_t wsB, int64_t nb, double* out, int64_t osP,
                int64_t osB, int64_t osQ) -> ttnn_status {
    Op op;
    Contract& c = op.c;
    c.P = 1;
    for (int a = 0; a < k; ++a) c.P *= dims[a];
    c.NI = dims[k];
    c.Q = 1;
    for (size_t a = k + 1; a < dims.size(); ++a) c.Q *= dims[a];
    c.isP = c.NI * c.Q;
    c.isI = c.Q;
    c.isQ = 1;
    c.NB = nb;
    c.w = W;
    c.wsI = wsI;
    c.wsB = wsB;
    c.in = in;
    c.out = out;
    c.osP = osP;
    c.osB = osB;
    c.osQ = osQ;
    op.tin = in_state ? set : ET_F64;
    op.tw = ET_F64;
    op.tout = ET_F64;
    const int64_t pe = plan_contract(op);
    op.partial = pe ? ws.alloc(pe * 8) : nullptr;
    if (!dry) prog.add(op, in, W);
    return TTNN_OK;
  };
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    double* core = cores + nd.core_off;
    if (v != P.root && nd.identity) {
      Op op;
      op.kind = OP_EYE;
      op.tout = ET_F64;
      op.eye_n = nd.n;
      op.c.out = core;
      plan_simple(op);
      if (!dry) prog.add(op, nullptr);
      continue;
    }
    if (v != P.root && nd.leaf) {
      // core[j][i] = sum_k Psi[i][k] Rp[k][j]
      TTNN_TRY(mp((const char*)acc + nd.ps_off * seb, true, {nd.n, (int64_t)nd.r}, 1, Rp[v], nd.r,
                  1, nd.r, core, 1, nd.n, 0));
      continue;
    }
    // transfer tensor or root: Q_c^T on each non-identity child axis, then
    // R_eps^+ on the column axis and the permutation (r_v, r_c1, ...)
    std::vector<int64_t> dims = nd.ps_shape;
    const void* cur = (const char*)acc + nd.ps_off * seb;
    bool in_state = true;
    const int m = (int)nd.ch.size();
    for (int k = 0; k < m; ++k) {
      const TNode& c = P.nodes[nd.ch[k]];
      if (c.identity) continue;
      std::vector<int64_t> od = dims;
      od[k] = c.r;
      int64_t tot = 1;
      for (auto x : od) tot *= x;
      double* o = (double*)ws.alloc(tot * 8);
      int64_t Q = 1;
      for (size_t a = k + 1; a < od.size(); ++a) Q *= od[a];
      TTNN_TRY(mp(cur, in_state, dims, k, Qp[c.user], c.r, 1, c.r, o, (int64_t)c.r * Q, Q, 1));
      cur = o;
      in_state = false;
      dims = od;
    }
    if (v == P.root) {
      int64_t tot = 1;
      for (auto x : dims) tot *= x;
      Op op;
      op.c.P = tot;
      op.c.NI = 1;
      op.c.isP = 1;
      op.c.in = cur;
      op.c.out = core;
      op.c.osP = 1;
      op.tin = in_state ? set : ET_F64;
      op.tw = ET_F64;
      op.tout = ET_F64;
      plan_contract(op);
      if (!dry) prog.add(op, cur);
    } else {
      int64_t rest = 1;
      for (int k = 0; k < m; ++k) rest *= dims[k];
      // out[b][p] = sum_k cur[p][k] Rp[k][b]
      TTNN_TRY(mp(cur, in_state, {rest, (int64_t)nd.r}, 1, Rp[v], nd.r, 1, nd.r, core, 1, rest, 0));
    }
  }
  if (peak) *peak = ws.peak;
  if (!ws.ok()) {
    set_error("internal: workspace overflow in recovery");
    return TTNN_ENOMEM;
  }
  if (!dry) TTNN_TRY(prog.run(st, P.flags & TTNN_FLAG_DUMP_PROGRAM));
  if (!dry && trunc) {
    // every core into its kept shape (device-side kept ranks)
    std::vector<int> job_of(P.nodes.size(), -1);
    for (size_t j = 0; j < job_node.size(); ++j) job_of[job_node[j]] = (int)j;
    CompactBatch b;
    b.src = padded;
    b.dst = out_cores;
    b.kept = P.kept_dev;
    int64_t maxel = 0;
    for (int v : P.lex) {
      const TNode& nd = P.nodes[v];
      if (nd.core_shape.size() > 10) {
        set_error("eps-truncated output: cores of at most 10 axes");
        return TTNN_EUNSUPPORTED;
      }
      CompactNode& c = b.nd[b.n];
      c.off = nd.core_off;
      c.ndim = (int)nd.core_shape.size();
      for (int a = 0; a < c.ndim; ++a) {
        c.full[a] = (int32_t)nd.core_shape[a];
        c.job[a] = -1;
      }
      int a0 = 0;
      if (v != P.root) {
        if (!nd.identity) c.job[0] = job_of[v];
        a0 = 1;
      }
      if (!nd.leaf)
        for (size_t k = 0; k < nd.ch.size(); ++k) {
          const TNode& ch = P.nodes[nd.ch[k]];
          if (!ch.identity) c.job[a0 + k] = job_of[ch.user];
        }
      maxel = std::max(maxel, nd.core_el);
      if (++b.n == kCompactNodes) {
        TTNN_TRY(launch_compact_cores(b, maxel, st));
        b.n = 0;
        maxel = 0;
      }
    }
    TTNN_TRY(launch_compact_cores(b, maxel, st));
  }
  if (!dry) prof_push(P, 2, ev0, prof_event(P, st));
  if (dry) return TTNN_OK;
  // read-back of kept ranks, sweeps and the device error word into pinned
  // host memory, completed by an event (plan_sync waits for it)
  if (P.kept_pending) {
    // an earlier read-back nobody waited for: its data is superseded
    TTNN_TRY_CUDA(cudaEventSynchronize(P.kept_ev));
    P.kept_pending = false;
    if (P.host_kept[2 * P.kept_nodes.size()]) P.timeout_seen = true;
  }
  const size_t nj = jobs.size();
  P.kept_nodes = job_node;
  if (nj)
    TTNN_TRY_CUDA(cudaMemcpyAsync(P.host_kept, P.kept_dev, 2 * nj * sizeof(int),
                                  cudaMemcpyDeviceToHost, st));
  TTNN_TRY_CUDA(cudaMemcpyAsync(P.host_kept + 2 * nj, P.err_dev, sizeof(int),
                                cudaMemcpyDeviceToHost, st));
  TTNN_TRY_CUDA(cudaEventRecord(P.kept_ev, st));
  P.kept_pending = true;
  if (!async) TTNN_TRY(plan_sync(P));
  return TTNN_OK;
}

}  // namespace ttnn
