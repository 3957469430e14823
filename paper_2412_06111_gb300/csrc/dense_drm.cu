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
  if (Q * J == 1 && alpha == 1.0 && !accumulate && P >= 512) {
    // out[p][b] = sum_i in[p][i] W[i][b] with many rows: a plain GEMM
    // (128-row tiles, split-K; fewer rows leave most of a tile idle)
    Gemm g;
    g.I = P;
    g.Jn = NB;
    g.K = NI;
    g.A = in;
    g.asi = NI;
    g.ask = 1;
    g.B = W;
    g.bsj = 1;
    g.bsk = NB;
    g.C = out;
    g.ldc = NB;
    g.in_type = et == ET_F64 ? 0 : 1;
    const int ns = gemm_choose_split(g);
    char* part = ns > 1 ? ws.alloc((int64_t)ns * P * NB * (et == ET_F64 ? 8 : 4)) : nullptr;
    if (ws.dry) return TTNN_OK;
    return launch_gemm(g, ns, part, st);
  }
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
  if (el * 8 > (int64_t(8) << 30)) {
    set_error("unstructured Gaussian DRMs need %lld bytes (> 8 GiB): use the Khatri-Rao DRMs",
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

// G_t = A^(t) X_t (n_t x r_t, walk type, row-major) into ws: A permuted so
// that t's modes come first (when t does not start at mode 0), then one
// contraction over the other modes' merged index.
static ttnn_status dense_g(ttnn_plan_s& P, const TNode& nd, const void* data, Bump& ws,
                           cudaStream_t st, char** G) {
  const ElemType et = P.walk_f64 ? ET_F64 : ET_F32;
  const int eb = P.walk_f64 ? 8 : 4;
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
    if (!ws.dry) TTNN_TRY(launch_contract(c, et, et, et, nullptr, 0, st));
    B = b;
  }
  *G = ws.alloc(nt * nd.r * eb);
  return mode_product(B, nt, K, 1, 1, (const char*)P.dxy + nd.dx_off * eb, nd.r, *G, 1.0, 0, et,
                      ws, st);
}

// Psi_root-shaped contraction of the dense tensor: every non-identity root
// child's axis of A against W_c (n_c x w_c, walk type, row-major) -- Y_c for
// the sketch, Q_c for TTN-HMT's root core -- into out (alpha, accumulate).
static ttnn_status root_contract(ttnn_plan_s& P, const void* data, const char* const* W,
                                 const int* wcols, void* out, double alpha, int accumulate,
                                 Bump& ws, cudaStream_t st) {
  const ElemType et = P.walk_f64 ? ET_F64 : ET_F32;
  const int eb = P.walk_f64 ? 8 : 4;
  const TNode& rt = P.nodes[P.root];
  std::vector<int64_t> dims;
  for (int c : rt.ch) dims.push_back(P.nodes[c].n);
  const int m = (int)dims.size();
  int last = -1;
  for (int k = 0; k < m; ++k)
    if (!P.nodes[rt.ch[k]].identity) last = k;
  if (last < 0) {
    Contract c;
    c.P = P.N;
    c.isP = 1;
    c.osP = 1;
    c.in = data;
    c.out = out;
    c.alpha = alpha;
    c.accumulate = accumulate;
    return ws.dry ? TTNN_OK : launch_contract(c, et, et, et, nullptr, 0, st);
  }
  const void* cur = data;
  for (int k = 0; k < m; ++k) {
    if (P.nodes[rt.ch[k]].identity) continue;
    int64_t pre = 1, post = 1;
    for (int a = 0; a < k; ++a) pre *= dims[a];
    for (int a = k + 1; a < m; ++a) post *= dims[a];
    const bool fin = k == last;
    char* o = fin ? (char*)out : ws.alloc(pre * wcols[k] * post * eb);
    TTNN_TRY(mode_product(cur, pre, dims[k], post, 1, W[k], wcols[k], o, fin ? alpha : 1.0,
                          fin ? accumulate : 0, et, ws, st));
    dims[k] = wcols[k];
    cur = o;
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
    const int64_t nt = nd.n;
    char* G = nullptr;
    TTNN_TRY(dense_g(P, nd, data, ws, st, &G));
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
    std::vector<const char*> W;
    std::vector<int> wc;
    for (int c : rt.ch) {
      const TNode& cn = P.nodes[c];
      W.push_back(cn.identity ? nullptr : fac(cn.dy_off));
      wc.push_back(cn.identity ? (int)cn.n : cn.s);
    }
    TTNN_TRY(root_contract(P, data, W.data(), wc.data(), at(rt.ps_off), lambda, 1, ws, st));
  }
  pk = std::max(pk, ws.top);
  if (peak) *peak = std::max<int64_t>(pk, 1);
  if (!dry && pk > ws.cap) {
    set_error("internal: workspace overflow (unstructured DRMs)");
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}



// ---------------------------------------------------------------------------
// TTN-HMT (Sec. 8's randomised comparator): the TTN-SVD with every SVD
// replaced by the HMT range finder on the same right sketches X_t.
// ---------------------------------------------------------------------------
namespace {

constexpr int kTsqrThreads = 1024;
constexpr int kTsqrChunk = 16;   // columns reduced together

struct TsqrJob {
  double* A;     // n x r, row-major: overwritten by the Householder vectors
  double* Q;     // n x r, row-major: the orthonormal factor
  int64_t n;
  int r;
};

// Sum over the CTA of up to kTsqrChunk per-thread values (returned to every
// thread through shared memory).
__device__ void block_sum(double* v, int m, double (*red)[kTsqrChunk], double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < m; ++c) {
    double x = v[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][c] = x;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
    for (int w = 0; w < kTsqrThreads / 32; ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Householder QR of one tall n x r block per CTA (binary64, in global
// memory): reflector k zeroes column k below the diagonal, then Q = H_0 ..
// H_{r-1} [I; 0].  A zero column keeps its reflector empty (Q's column is
// then the unit vector e_k, orthogonal to the others).
__global__ void __launch_bounds__(kTsqrThreads) tsqr_kernel(const TsqrJob job) {
  __shared__ double red[kTsqrThreads / 32][kTsqrChunk];
  __shared__ double w[kTsqrChunk];
  __shared__ double tau[kMaxRecoverR];
  double* A = job.A;
  double* Qm = job.Q;
  const int64_t n = job.n;
  const int r = job.r;
  for (int k = 0; k < r; ++k) {
    double part[kTsqrChunk];
    part[0] = 0.0;
    for (int64_t i = k + threadIdx.x; i < n; i += kTsqrThreads) part[0] += A[i * r + k] * A[i * r + k];
    block_sum(part, 1, red, w);
    if (threadIdx.x == 0) {
      const double nrm2 = w[0], alpha = A[(int64_t)k * r + k], nrm = sqrt(nrm2);
      double t = 0.0;
      if (nrm > 0.0) {
        const double beta = alpha > 0.0 ? -nrm : nrm;
        const double v0 = alpha - beta;
        const double vn2 = nrm2 - alpha * alpha + v0 * v0;
        A[(int64_t)k * r + k] = v0;
        t = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
      }
      tau[k] = t;
    }
    __syncthreads();
    if (tau[k] == 0.0) continue;
    for (int j0 = k + 1; j0 < r; j0 += kTsqrChunk) {
      const int m = min(kTsqrChunk, r - j0);
      for (int c = 0; c < m; ++c) part[c] = 0.0;
      for (int64_t i = k + threadIdx.x; i < n; i += kTsqrThreads) {
        const double vi = A[i * r + k];
        for (int c = 0; c < m; ++c) part[c] += vi * A[i * r + j0 + c];
      }
      block_sum(part, m, red, w);
      for (int64_t i = k + threadIdx.x; i < n; i += kTsqrThreads) {
        const double vi = tau[k] * A[i * r + k];
        for (int c = 0; c < m; ++c) A[i * r + j0 + c] -= vi * w[c];
      }
      __syncthreads();
    }
  }
  for (int64_t e = threadIdx.x; e < n * r; e += kTsqrThreads)
    Qm[e] = (e / r == e % r) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    for (int j0 = k; j0 < r; j0 += kTsqrChunk) {
      const int m = min(kTsqrChunk, r - j0);
      double part[kTsqrChunk];
      for (int c = 0; c < m; ++c) part[c] = 0.0;
      for (int64_t i = k + threadIdx.x; i < n; i += kTsqrThreads) {
        const double vi = A[i * r + k];
        for (int c = 0; c < m; ++c) part[c] += vi * Qm[i * r + j0 + c];
      }
      block_sum(part, m, red, w);
      for (int64_t i = k + threadIdx.x; i < n; i += kTsqrThreads) {
        const double vi = tau[k] * A[i * r + k];
        for (int c = 0; c < m; ++c) Qm[i * r + j0 + c] -= vi * w[c];
      }
      __syncthreads();
    }
  }
}

// out[b][a] = in[a][b] for an (m x k) row-major binary64 matrix.
ttnn_status transpose_f64(const double* in, int64_t m, int64_t k, double* out, bool dry,
                          cudaStream_t st) {
  if (dry) return TTNN_OK;
  Contract c;
  c.P = m;
  c.J = k;
  c.isP = k;
  c.isJ = 1;
  c.osP = 1;
  c.osJ = m;
  c.in = in;
  c.out = out;
  return launch_contract(c, ET_F64, ET_F64, ET_F64, nullptr, 0, st);
}

}  // namespace

ttnn_status run_hmt(ttnn_plan_s& P, const void* data, double* cores, cudaStream_t st, bool dry,
                    int64_t* peak) {
  if (!(P.flags & TTNN_FLAG_DENSE_DRM) || !P.walk_f64 || P.variant != TTNN_VARIANT_TTNN) {
    set_error("TTN-HMT: binary64 TTNN plans with TTNN_FLAG_DENSE_DRM only");
    return TTNN_EUNSUPPORTED;
  }
  Bump ws(P.ws, P.ws_bytes, dry);
  int64_t pk = 0;
  std::vector<double*> Q(P.nodes.size(), nullptr);
  // pass 1: Q_t = orth(A^(t) X_t) for every sketched node
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    Q[v] = (double*)ws.alloc(nd.n * nd.r * 8);
    const int64_t mark = ws.top;
    char* G = nullptr;
    TTNN_TRY(dense_g(P, nd, data, ws, st, &G));
    if (!dry) {
      tsqr_kernel<<<1, kTsqrThreads, 0, st>>>(TsqrJob{(double*)G, Q[v], nd.n, nd.r});
      TTNN_TRY(check_launch("tsqr_kernel"));
    }
    pk = std::max(pk, ws.top);
    ws.top = mark;
  }
  // cores: leaf Q_t^T, transfer (kron_c Q_c)^T Q_t as (r_t, r_c..), identity I
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (v == P.root) continue;
    double* core = dry ? nullptr : cores + nd.core_off;
    if (nd.identity) {
      if (!dry) TTNN_TRY(launch_eye(core, nd.n, st));
      continue;
    }
    if (nd.leaf) {
      TTNN_TRY(transpose_f64(Q[v], nd.n, nd.r, core, dry, st));
      continue;
    }
    const int64_t mark = ws.top;
    std::vector<int64_t> dims;
    for (int c : nd.ch) dims.push_back(P.nodes[c].n);
    const int m = (int)dims.size();
    const void* cur = Q[v];
    for (int k = 0; k < m; ++k) {
      const TNode& c = P.nodes[nd.ch[k]];
      if (c.identity) continue;
      int64_t pre = 1, post = 1;
      for (int a = 0; a < k; ++a) pre *= dims[a];
      for (int a = k + 1; a < m; ++a) post *= dims[a];
      char* o = ws.alloc(pre * c.r * post * nd.r * 8);
      TTNN_TRY(mode_product(cur, pre, dims[k], post, nd.r, Q[c.user], c.r, o, 1.0, 0, ET_F64, ws,
                            st));
      dims[k] = c.r;
      cur = o;
    }
    int64_t rest = 1;
    for (auto x : dims) rest *= x;
    TTNN_TRY(transpose_f64((const double*)cur, rest, nd.r, core, dry, st));
    pk = std::max(pk, ws.top);
    ws.top = mark;
  }
  // pass 2: the root core (kron_c Q_c)^T A
  {
    const TNode& rt = P.nodes[P.root];
    std::vector<const char*> W;
    std::vector<int> wc;
    for (int c : rt.ch) {
      const TNode& cn = P.nodes[c];
      W.push_back(cn.identity ? nullptr : (const char*)Q[c]);
      wc.push_back(cn.identity ? (int)cn.n : cn.r);
    }
    TTNN_TRY(root_contract(P, data, W.data(), wc.data(), dry ? nullptr : cores + rt.core_off, 1.0,
                           0, ws, st));
    pk = std::max(pk, ws.top);
  }
  if (peak) *peak = std::max<int64_t>(pk, 1);
  if (!dry && pk > ws.cap) {
    set_error("internal: workspace overflow (TTN-HMT)");
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}

}  // namespace ttnn
