// Unstructured Gaussian DRMs (TTNN_FLAG_DENSE_DRM): every sketched node t
// has its own independent X_t (n_{D\t} x r_t) and Y_t (n_t x s_t), drawn by
// the Philox generator (kinds 4 and 5, keyed by t's lexicographic index) and
// rounded once to the plan's format -- the sketch of Sec. 4 eq. (sketch) with
// the Gaussian DRMs that the expected error bound of Thm 6.6 assumes, instead
// of the Khatri-Rao DRMs of Sec. 7.  Their size is the product of the other
// modes' sizes, so the form is for small trees (binary64 / binary32 plans,
// TTNN, whole-tensor dense updates).
//
// One update of the dense tensor A, per sketched node t with modes [lo, hi):
//   B = A permuted to [t's modes][modes before lo][modes from hi]  (skipped
//       when lo = 0: A is then already the unfolding A^(t));
//   G_t = B X_t                                     (n_t x r_t)
//   Omega_t += lambda Y_t^T G_t
//   Psi_t   += lambda G_t                           (leaf)
//   Psi_t   += lambda G_t x_{c} Y_c^T for every non-identity child c (internal)
// and Psi_root += lambda A x_{c} Y_c^T over the root's children.  Every step is
// a strided contraction (launch_contract) in the walk type.
#include <algorithm>

#include "plan.cuh"

namespace ttnn {

namespace {

struct Bump {
  char* base;
  int64_t cap;
  bool dry;
  int64_t top = 0;
  Bump(char* b, int64_t c, bool d) : base(b), cap(c), dry(d) {}
  char* alloc(int64_t bytes) {
    const int64_t o = round_up(top, 256);
    top = o + std::max<int64_t>(bytes, 0);
    return dry ? nullptr : base + o;
  }
};

// out[p, b, q, j] (+)= alpha * sum_i in[p, i, q, j] W[i, b] on a contiguous
// [P][NI][Q][J] input, W (NI x NB) row-major, output [P][NB][Q][J].
ttnn_status mode_product(const void* in, int64_t P, int64_t NI, int64_t Q, int64_t J,
                         const void* W, int64_t NB, void* out, double alpha, int accumulate,
                         ElemType et, Bump& ws, cudaStream_t st) {
  Contract c;
  c.P = P;
  c.NI = NI;
  c.NB = NB;
  c.Q = Q;
  c.J = J;
  c.isP = NI * Q * J;
  c.isI = Q * J;
  c.isQ = J;
  c.isJ = 1;
  c.w = W;
  c.wsI = NB;
  c.wsB = 1;
  c.osP = NB * Q * J;
  c.osB = Q * J;
  c.osQ = J;
  c.osJ = 1;
  c.in = in;
  c.out = out;
  c.alpha = alpha;
  c.accumulate = accumulate;
  const int64_t pe = contract_partial_elems(c);
  char* part = ws.alloc(pe * (et == ET_F64 ? 8 : 4));
  if (ws.dry) return TTNN_OK;
  return launch_contract(c, et, et, et, part, pe, st);
}

}  // namespace

ttnn_status dense_drm_check(const ttnn_plan_s& P) {
  if (P.variant != TTNN_VARIANT_TTNN || (P.dtype != TTNN_F64 && P.dtype != TTNN_F32)) {
    set_error("unstructured Gaussian DRMs: TTNN plans in binary64 or binary32 only");
    return TTNN_EUNSUPPORTED;
  }
  if (P.N >= (int64_t(1) << 31)) {
    set_error("unstructured Gaussian DRMs: tensors below 2^31 entries only");
    return TTNN_EUNSUPPORTED;
  }
  int64_t el = 0;
  for (const TNode& nd : P.nodes)
    if (nd.sketched()) el += (P.N / nd.n) * nd.r + nd.n * nd.s;
  if (el * 8 > (int64_t(1) << 30)) {
    set_error("unstructured Gaussian DRMs need %lld bytes (> 1 GiB): use the Khatri-Rao DRMs",
              (long long)(el * 8));
    return TTNN_EUNSUPPORTED;
  }
  return TTNN_OK;
}

int64_t dense_drm_elems(ttnn_plan_s& P) {
  int64_t el = 0;
  for (int v : P.lex) {
    TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    nd.dx_off = el;
    el += (P.N / nd.n) * nd.r;
    nd.dy_off = el;
    el += nd.n * nd.s;
  }
  return el;
}

ttnn_status dense_drm_generate(ttnn_plan_s& P, double* tmp64, cudaStream_t st) {
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    TTNN_TRY(launch_philox(P.seed, 4, nd.lex, P.N / nd.n, nd.r, P.round_fmt, tmp64 + nd.dx_off, st));
    TTNN_TRY(launch_philox(P.seed, 5, nd.lex, nd.n, nd.s, P.round_fmt, tmp64 + nd.dy_off, st));
  }
  return TTNN_OK;
}

ttnn_status run_dense_drm_update(ttnn_plan_s& P, void* acc, const void* data, const Box& box,
                                 double lambda, cudaStream_t st, bool dry, int64_t* peak) {
  if (!box.full) {
    set_error("unstructured Gaussian DRMs: whole-tensor updates only");
    return TTNN_EUNSUPPORTED;
  }
  const ElemType et = P.walk_f64 ? ET_F64 : ET_F32;
  const int eb = P.walk_f64 ? 8 : 4;
  Bump ws(P.ws, P.ws_bytes, dry);
  auto fac = [&](int64_t off) { return (const char*)P.dxy + off * eb; };
  auto at = [&](int64_t off) { return (char*)acc + off * eb; };
  const int64_t mark0 = ws.top;
  int64_t pk = 0;
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    pk = std::max(pk, ws.top);
    ws.top = mark0;
    int64_t npre = 1, npost = 1;
    for (int m = 0; m < nd.lo; ++m) npre *= P.dims[m];
    for (int m = nd.hi; m < P.d; ++m) npost *= P.dims[m];
    const int64_t nt = nd.n, K = npre * npost;
    // B = A permuted so that t's modes come first: out[i, p, q] = A[p, i, q]
    const void* B = data;
    if (npre > 1) {
      char* b = ws.alloc(P.N * eb);
      Contract c;
      c.P = nt;
      c.NI = 1;
      c.Q = npre;
      c.J = npost;
      c.isP = npost;
      c.isQ = nt * npost;
      c.isJ = 1;
      c.osP = npre * npost;
      c.osQ = npost;
      c.osJ = 1;
      c.in = data;
      c.out = b;
      if (!dry) TTNN_TRY(launch_contract(c, et, et, et, nullptr, 0, st));
      B = b;
    }
    // G_t = B X_t (nt x r)
    char* G = ws.alloc(nt * nd.r * eb);
    TTNN_TRY(mode_product(B, nt, K, 1, 1, fac(nd.dx_off), nd.r, G, 1.0, 0, et, ws, st));
    // (mode_product's output [P][NB][Q][J] = [nt][r] here)
    // Omega_t += lambda Y_t^T G_t: contract G's row axis with Y_t
    TTNN_TRY(mode_product(G, 1, nt, 1, nd.r, fac(nd.dy_off), nd.s, at(nd.om_off), lambda, 1, et,
                          ws, st));
    if (nd.leaf) {
      Contract c;
      c.P = nt * nd.r;
      c.isP = 1;
      c.osP = 1;
      c.in = G;
      c.out = at(nd.ps_off);
      c.alpha = lambda;
      c.accumulate = 1;
      if (!dry) TTNN_TRY(launch_contract(c, et, et, et, nullptr, 0, st));
      continue;
    }
    // Psi_t: each non-identity child axis of [n_c1 .. n_cm, r] against Y_c
    std::vector<int64_t> dims;
    for (int c : nd.ch) dims.push_back(P.nodes[c].n);
    const int m = (int)dims.size();
    int last = -1;
    for (int k = 0; k < m; ++k)
      if (!P.nodes[nd.ch[k]].identity) last = k;
    const void* cur = G;
    if (last < 0) {
      Contract c;
      c.P = nt * nd.r;
      c.isP = 1;
      c.osP = 1;
      c.in = G;
      c.out = at(nd.ps_off);
      c.alpha = lambda;
      c.accumulate = 1;
      if (!dry) TTNN_TRY(launch_contract(c, et, et, et, nullptr, 0, st));
      continue;
    }
    for (int k = 0; k < m; ++k) {
      const TNode& c = P.nodes[nd.ch[k]];
      if (c.identity) continue;
      int64_t pre = 1, post = 1;
      for (int a = 0; a < k; ++a) pre *= dims[a];
      for (int a = k + 1; a < m; ++a) post *= dims[a];
      const bool fin = k == last;
      char* o = fin ? at(nd.ps_off) : ws.alloc(pre * c.s * post * nd.r * eb);
      TTNN_TRY(mode_product(cur, pre, dims[k], post, nd.r, fac(c.dy_off), c.s, o,
                            fin ? lambda : 1.0, fin ? 1 : 0, et, ws, st));
      dims[k] = c.s;
      cur = o;
    }
  }
  // Psi_root: A against Y_c on each non-identity root child
  {
    pk = std::max(pk, ws.top);
    ws.top = mark0;
    const TNode& rt = P.nodes[P.root];
    std::vector<int64_t> dims;
    for (int c : rt.ch) dims.push_back(P.nodes[c].n);
    const int m = (int)dims.size();
    int last = -1;
    for (int k = 0; k < m; ++k)
      if (!P.nodes[rt.ch[k]].identity) last = k;
    const void* cur = data;
    for (int k = 0; k < m && last >= 0; ++k) {
      const TNode& c = P.nodes[rt.ch[k]];
      if (c.identity) continue;
      int64_t pre = 1, post = 1;
      for (int a = 0; a < k; ++a) pre *= dims[a];
      for (int a = k + 1; a < m; ++a) post *= dims[a];
      const bool fin = k == last;
      char* o = fin ? at(rt.ps_off) : ws.alloc(pre * c.s * post * eb);
      TTNN_TRY(mode_product(cur, pre, dims[k], post, 1, fac(c.dy_off), c.s, o, fin ? lambda : 1.0,
                            fin ? 1 : 0, et, ws, st));
      dims[k] = c.s;
      cur = o;
    }
    if (last < 0) {
      Contract c;
      c.P = P.N;
      c.isP = 1;
      c.osP = 1;
      c.in = data;
      c.out = at(rt.ps_off);
      c.alpha = lambda;
      c.accumulate = 1;
      if (!dry) TTNN_TRY(launch_contract(c, et, et, et, nullptr, 0, st));
    }
  }
  pk = std::max(pk, ws.top);
  if (peak) *peak = std::max<int64_t>(pk, 1);
  if (!dry && pk > ws.cap) {
    set_error("internal: workspace overflow (unstructured DRMs)");
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}

}  // namespace ttnn
