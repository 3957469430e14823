// C ABI entry points (declared in include/ttnn.h).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>

#include "plan.cuh"

namespace ttnn {

long long launches_so_far();
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

// Allocation-failure injection for tests (ttnn_debug_fail_alloc): the
// device allocation that brings this counter from 1 to 0 fails.
static std::atomic<int> g_fail_alloc{0};

static ttnn_status dev_alloc(void** p, int64_t bytes) {
  *p = nullptr;
  if (bytes <= 0) return TTNN_OK;
  if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
    set_error("cudaMalloc(%lld) failed: injected allocation failure", (long long)bytes);
    return TTNN_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, (size_t)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%lld) failed: %s", (long long)bytes, cudaGetErrorString(e));
    *p = nullptr;
    return TTNN_ENOMEM;
  }
  return TTNN_OK;
}

static void free_plan(ttnn_plan_s* P) {
  if (!P) return;
  for (auto& v : P->prof)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : P->prof_pool) cudaEventDestroy(e);
  cudaFree(P->fac64);
  if (P->facw != (void*)P->fac64) cudaFree(P->facw);
  cudaFree(P->sideR);
  cudaFree(P->sideL);
  cudaFree(P->yW);
  cudaFree(P->xWo);
  cudaFree(P->sideRs);
  cudaFree(P->sideLs);
  cudaFree(P->dxy);
  cudaFree(P->ws);
  cudaFree(P->ws_rec);
  cudaFree(P->jobs_dev);
  cudaFree(P->kept_dev);
  cudaFree(P->err_dev);
  if (P->host_kept) cudaFreeHost(P->host_kept);
  if (P->kept_ev) cudaEventDestroy(P->kept_ev);
  delete P;
}

// Replaces the plan workspace by a larger one.  The new block is allocated
// first, so a failed allocation leaves the plan as it was (TTNN_ENOMEM, no
// work launched); cudaFree synchronises the device, so no earlier work still
// uses the old block when it is released.
static ttnn_status grow_workspace(ttnn_plan_s& P, int64_t bytes) {
  char* fresh = nullptr;
  TTNN_TRY(dev_alloc((void**)&fresh, bytes));
  cudaFree(P.ws);
  P.dev_bytes += bytes - P.ws_bytes;
  P.ws = fresh;
  P.ws_bytes = bytes;
  return TTNN_OK;
}

// A device timeout seen while ttnn_plan_node waited for a read-back is
// reported by the next recovery / sync call.
static ttnn_status take_timeout(ttnn_plan_s& P) {
  if (!P.timeout_seen) return TTNN_OK;
  P.timeout_seen = false;
  set_error("a bounded device wait ran out in an earlier update or recovery");
  return TTNN_ETIMEOUT;
}

static int store_bytes(int store) { return store == 0 ? 8 : store == 1 ? 4 : store == 2 ? 2 : 1; }

static Box full_box(const ttnn_plan_s& P) {
  Box b;
  b.off.assign(P.d, 0);
  b.ext = P.dims;
  b.full = true;
  return b;
}

}  // namespace ttnn

using namespace ttnn;

extern "C" {

const char* ttnn_status_string(ttnn_status s) {
  switch (s) {
    case TTNN_OK: return "ok";
    case TTNN_EINVAL: return "invalid argument";
    case TTNN_ENOMEM: return "out of memory";
    case TTNN_ECUDA: return "CUDA error";
    case TTNN_ENUMERIC: return "non-finite values";
    case TTNN_ETIMEOUT: return "device wait timed out";
    case TTNN_EBUSY: return "busy";
    case TTNN_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

ttnn_status ttnn_debug_fail_alloc(int32_t nth) {
  TTNN_CHECK_ARG(nth >= 0, "nth must be >= 0");
  g_fail_alloc.store(nth);
  return TTNN_OK;
}

ttnn_status ttnn_last_error(char* buf, size_t n) {
  if (buf && n) {
    strncpy(buf, last_error(), n - 1);
    buf[n - 1] = 0;
  }
  return TTNN_OK;
}

ttnn_status ttnn_philox_gaussian(uint64_t seed, int32_t kind, int32_t ident, int64_t rows,
                                 int64_t cols, int32_t round_dtype, double* dst, void* stream) {
  TTNN_CHECK_ARG(rows >= 0 && cols >= 0, "negative size");
  TTNN_CHECK_ARG(kind >= 1 && kind <= 5, "kind must be in 1..5");
  TTNN_CHECK_ARG(ident >= 0 && ident < (1 << 24), "ident must be in [0, 2^24)");
  TTNN_CHECK_ARG(round_dtype >= 0 && round_dtype <= 3, "round_dtype must be F64/F32/BF16/E4M3");
  TTNN_CHECK_ARG(dst || rows * cols == 0, "null dst");
  return launch_philox(seed, kind, ident, rows, cols, round_dtype, dst, (cudaStream_t)stream);
}

ttnn_status ttnn_plan_create(const ttnn_tree* tree, int32_t d, const int64_t* dims,
                             const int32_t* ranks, const int32_t* oversample, uint64_t seed,
                             const ttnn_opts* opts, void* stream, ttnn_plan_t* out) {
  TTNN_CHECK_ARG(out, "null output");
  *out = nullptr;
  std::unique_ptr<ttnn_plan_s> hold(new (std::nothrow) ttnn_plan_s());
  if (!hold) {
    set_error("host allocation failed");
    return TTNN_ENOMEM;
  }
  ttnn_plan_s& P = *hold;
  auto palloc = [&P](void** ptr, int64_t bytes) {
    const ttnn_status r = dev_alloc(ptr, bytes);
    if (r == TTNN_OK && bytes > 0) P.dev_bytes += bytes;
    return r;
  };
  ttnn_opts def{TTNN_VARIANT_TTNN, TTNN_F32, 10.0, 2.220446049250313e-16, 0};
  TTNN_TRY(build_plan(P, tree, d, dims, ranks, oversample, seed, opts ? opts : &def));
  cudaStream_t st = (cudaStream_t)stream;
  ttnn_status s = TTNN_OK;
  auto fail = [&](ttnn_status e) {
    ttnn_plan_s* raw = hold.release();
    free_plan(raw);
    return e;
  };
  // DRM factors (binary64 master, walk-type copy)
  if ((s = palloc((void**)&P.fac64, P.fac_elems * 8)) != TTNN_OK) return fail(s);
  for (int m = 0; m < P.d; ++m) {
    if ((s = launch_philox(seed, 1, m, P.dims[m], P.rmax, P.round_fmt, P.fac64 + P.x_off[m], st))) return fail(s);
    if ((s = launch_philox(seed, 2, m, P.dims[m], P.smax, P.round_fmt, P.fac64 + P.y_off[m], st))) return fail(s);
  }
  for (int v : P.lex) {
    const TNode& nd = P.nodes[v];
    if (!nd.sketched()) continue;
    if ((s = launch_philox(seed, 3, nd.lex, nd.s, P.rmax, P.round_fmt, P.fac64 + nd.xt_off, st))) return fail(s);
  }
  if (P.walk_f64) {
    P.facw = P.fac64;
  } else {
    if ((s = palloc(&P.facw, P.fac_elems * 4)) != TTNN_OK) return fail(s);
    if ((s = launch_convert_f64_to_f32(P.fac64, (float*)P.facw, P.fac_elems, st))) return fail(s);
  }
  // cached full-size pass blocks
  Box fb = full_box(P);
  int64_t nL = 1, nR = 1;
  for (int m = P.Llo; m < P.Lhi; ++m) nL *= P.dims[m];
  for (int m = P.Rlo; m < P.Rhi; ++m) nR *= P.dims[m];
  const int sb = store_bytes(P.side_store);
  const bool dense = !(P.flags & TTNN_FLAG_STRUCTURED_ONLY);
  if (P.flags & TTNN_FLAG_DENSE_DRM) {
    // unstructured Gaussian X_t, Y_t per node (binary64 draws rounded to the
    // plan's format, stored in the walk type)
    if ((s = dense_drm_check(P)) != TTNN_OK) return fail(s);
    const int64_t el = dense_drm_elems(P);
    if ((s = palloc(&P.dxy, el * (P.walk_f64 ? 8 : 4))) != TTNN_OK) return fail(s);
    double* tmp = (double*)P.dxy;
    if (!P.walk_f64 && (s = dev_alloc((void**)&tmp, el * 8)) != TTNN_OK) return fail(s);
    s = dense_drm_generate(P, tmp, st);
    if (s == TTNN_OK && !P.walk_f64) s = launch_convert_f64_to_f32(tmp, (float*)P.dxy, el, st);
    if (!P.walk_f64) {
      cudaStreamSynchronize(st);
      cudaFree(tmp);
    }
    if (s != TTNN_OK) return fail(s);
  }
  if (dense && !(P.flags & (TTNN_FLAG_NO_SIDE_CACHE | TTNN_FLAG_DENSE_DRM))) {
    if (P.wR > 0) {
      if ((s = palloc(&P.sideR, (int64_t)P.wRpad * nR * sb)) != TTNN_OK) return fail(s);
      if ((s = make_side(P, fb, 0, P.sideR, nR, st))) return fail(s);
    }
    if (P.wL > 0) {
      if ((s = palloc(&P.sideL, (int64_t)P.wLpad * nL * sb)) != TTNN_OK) return fail(s);
      if ((s = make_side(P, fb, 1, P.sideL, nL, st))) return fail(s);
    }
    const TNode& yc = P.nodes[P.ychild];
    // (a Y child whose Omega goes through D2 needs its block only for
    // rank-one boxes: generated then)
    if (!yc.identity && !omega_via_d2(P, nL, nR)) {
      if ((s = palloc(&P.yW, (int64_t)yc.s * yc.n * (P.walk_f64 ? 8 : 4))) != TTNN_OK) return fail(s);
      if ((s = make_side_yw(P, fb, P.yW, yc.n, st))) return fail(s);
    }
    // binary32 plans whose whole-tensor pass fits the tensor cores: the side
    // blocks split into bf16 hi + lo
    if (P.dtype == TTNN_F32 && P.sideR && P.sideL && nL % 8 == 0 && nR % 8 == 0 &&
        !(P.flags & TTNN_FLAG_SIMT_PASS)) {
      const int64_t eR = (int64_t)P.wRpad * nR, eL = (int64_t)P.wLpad * nL;
      if ((s = palloc(&P.sideRs, eR * 4)) != TTNN_OK) return fail(s);
      if ((s = palloc(&P.sideLs, eL * 4)) != TTNN_OK) return fail(s);
      if ((s = launch_split_bf16((const float*)P.sideR, eR, P.sideRs, (char*)P.sideRs + eR * 2,
                                 st)) != TTNN_OK)
        return fail(s);
      if ((s = launch_split_bf16((const float*)P.sideL, eL, P.sideLs, (char*)P.sideLs + eL * 2,
                                 st)) != TTNN_OK)
        return fail(s);
    }
    if (omega_via_d2(P, nL, nR)) {
      if ((s = palloc(&P.xWo, (int64_t)P.rXL * nR * (P.walk_f64 ? 8 : 4))) != TTNN_OK) return fail(s);
      if ((s = make_side_xo(P, fb, P.xWo, nR, st))) return fail(s);
    }
  }
  // workspaces: updates -- the larger of a whole-tensor update (cached DRM
  // blocks), an update of a box as large as the tensor (blocks generated into
  // the workspace: bounds every box update) and a CP update; TTN-format
  // updates grow it on demand -- and, apart, the recovery's
  int64_t need_u = 0, need_r = 0;
  if (dense) {
    if ((s = dense_update_need(P, fb, &need_u))) return fail(s);
    if (!(P.flags & TTNN_FLAG_DENSE_DRM)) {   // that form takes whole tensors only
      Box bb = fb;
      bb.full = false;
      int64_t need_b = 0;
      if ((s = dense_update_need(P, bb, &need_b))) return fail(s);
      need_u = std::max(need_u, need_b);
    }
  }
  if (P.variant == TTNN_VARIANT_TTNN && !(P.flags & TTNN_FLAG_DENSE_DRM))
    need_u = std::max(need_u, cp_update_need(P));
  if ((s = run_recover(P, nullptr, nullptr, st, true, &need_r))) return fail(s);
  P.ws_bytes = need_u + 4096;
  if ((s = palloc((void**)&P.ws, P.ws_bytes)) != TTNN_OK) return fail(s);
  P.ws_rec_bytes = need_r + 4096;
  if ((s = palloc((void**)&P.ws_rec, P.ws_rec_bytes)) != TTNN_OK) return fail(s);
  if ((s = palloc((void**)&P.jobs_dev, std::max(1, P.n_sketched) * (int64_t)sizeof(QrJob))) != TTNN_OK) return fail(s);
  if ((s = palloc((void**)&P.kept_dev, 2 * std::max(1, P.n_sketched) * (int64_t)sizeof(int))) != TTNN_OK) return fail(s);
  if ((s = palloc((void**)&P.err_dev, sizeof(int))) != TTNN_OK) return fail(s);
  if (cudaHostAlloc((void**)&P.host_kept, (2 * std::max(1, P.n_sketched) + 1) * sizeof(int),
                    cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&P.kept_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan creation: pinned read-back buffer or event");
    return fail(TTNN_ENOMEM);
  }
  if ((s = launch_fill_zero(P.err_dev, sizeof(int), st)) != TTNN_OK) return fail(s);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("plan creation: %s", cudaGetErrorString(e));
    return fail(TTNN_ECUDA);
  }
  *out = hold.release();
  return TTNN_OK;
}

void ttnn_plan_destroy(ttnn_plan_t plan) { free_plan(plan); }

ttnn_status ttnn_plan_device_bytes(ttnn_plan_t P, int64_t* total, int64_t* workspace) {
  TTNN_CHECK_ARG(P, "null plan");
  if (total) *total = P->dev_bytes;
  if (workspace) *workspace = P->ws_bytes;
  return TTNN_OK;
}

ttnn_status ttnn_plan_sizes(ttnn_plan_t P, int64_t* state_elems, int32_t* state_elem_bytes,
                            int64_t* core_elems, int32_t* n_nodes) {
  TTNN_CHECK_ARG(P, "null plan");
  if (state_elems) *state_elems = P->state_elems;
  if (state_elem_bytes) *state_elem_bytes = P->walk_f64 ? 8 : 4;
  if (core_elems) *core_elems = P->core_elems;
  if (n_nodes) *n_nodes = (int32_t)P->nodes.size();
  return TTNN_OK;
}

ttnn_status ttnn_plan_node(ttnn_plan_t P, int32_t v, ttnn_node_info* o) {
  TTNN_CHECK_ARG(P && o, "null argument");
  TTNN_CHECK_ARG(v >= 0 && v < (int)P->nodes.size(), "node index out of range");
  // kept ranks of a recovery still in flight: wait for its read-back (a
  // device timeout it carries is reported by ttnn_plan_sync / ttnn_recover)
  if (P->kept_pending) {
    const ttnn_status ss = plan_sync(*P);
    if (ss != TTNN_OK && ss != TTNN_ETIMEOUT) return ss;
    if (ss == TTNN_ETIMEOUT) P->timeout_seen = true;
  }
  const TNode& nd = P->nodes[v];
  memset(o, 0, sizeof(*o));
  o->user_index = v;
  o->lex_index = nd.lex;
  o->level = nd.level;
  o->parent = nd.parent;
  o->n_children = (int32_t)nd.ch.size();
  o->mode_lo = nd.lo;
  o->mode_hi = nd.hi;
  o->is_leaf = nd.leaf;
  o->identity = nd.identity;
  o->r = nd.r;
  o->p = nd.p;
  o->s = nd.s;
  o->n = nd.n;
  o->omega_offset = nd.om_off;
  o->omega_elems = nd.om_el;
  o->psi_offset = nd.ps_off;
  o->psi_elems = nd.ps_el;
  o->psi_ndim = (int32_t)std::min<size_t>(nd.ps_shape.size(), 10);
  for (int k = 0; k < o->psi_ndim; ++k) o->psi_shape[k] = nd.ps_shape[k];
  o->core_offset = nd.core_off;
  o->core_elems = nd.core_el;
  o->core_ndim = (int32_t)std::min<size_t>(nd.core_shape.size(), 10);
  for (int k = 0; k < o->core_ndim; ++k) o->core_shape[k] = nd.core_shape[k];
  if (P->flags & TTNN_FLAG_TRUNCATE) {
    // eps-truncated output: the shape of the last recovery's core (its rank
    // axes at the kept ranks), once every kept rank it involves is known
    auto kept = [&](int u) { return P->nodes[u].identity ? P->nodes[u].n : (int64_t)P->nodes[u].kept; };
    std::vector<int64_t> sh(nd.core_shape.begin(), nd.core_shape.end());
    bool known = true;
    int a0 = 0;
    if (v != P->root) {
      if (!nd.identity) sh[0] = kept(v);
      known = known && sh[0] >= 0;
      a0 = 1;
    }
    if (!nd.leaf)
      for (size_t k = 0; k < nd.ch.size(); ++k) {
        sh[a0 + k] = kept(nd.ch[k]);
        known = known && sh[a0 + k] >= 0;
      }
    if (known) {
      int64_t el = 1;
      for (int k = 0; k < o->core_ndim; ++k) {
        o->core_shape[k] = sh[k];
        el *= sh[k];
      }
      o->core_elems = el;
    }
  }
  o->kept_rank = nd.kept;
  o->jacobi_sweeps = nd.sweeps;
  return TTNN_OK;
}

ttnn_status ttnn_plan_factor(ttnn_plan_t P, int32_t which, int32_t mode, double* dst, int64_t* rows,
                             int64_t* cols, void* stream) {
  TTNN_CHECK_ARG(P, "null plan");
  int64_t r = 0, c = 0, off = 0;
  if (which == 1 || which == 2) {
    TTNN_CHECK_ARG(mode >= 0 && mode < P->d, "mode out of range");
    r = P->dims[mode];
    c = which == 1 ? P->rmax : P->smax;
    off = which == 1 ? P->x_off[mode] : P->y_off[mode];
  } else if (which == 3) {
    TTNN_CHECK_ARG(mode >= 0 && mode < (int)P->lex.size(), "lex index out of range");
    const TNode& nd = P->nodes[P->lex[mode]];
    TTNN_CHECK_ARG(nd.sketched(), "node has no XT factor");
    r = nd.s;
    c = P->rmax;
    off = nd.xt_off;
  } else {
    set_error("which must be 1, 2 or 3");
    return TTNN_EINVAL;
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (dst)
    TTNN_TRY_CUDA(cudaMemcpyAsync(dst, P->fac64 + off, r * c * 8, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
  return TTNN_OK;
}

ttnn_status ttnn_state_create(ttnn_plan_t P, void* stream, ttnn_state_t* out) {
  TTNN_CHECK_ARG(P && out, "null argument");
  *out = nullptr;
  ttnn_state_s* S = new (std::nothrow) ttnn_state_s();
  if (!S) {
    set_error("host allocation failed");
    return TTNN_ENOMEM;
  }
  S->plan = P;
  S->elems = P->state_elems;
  ttnn_status s = dev_alloc(&S->acc, S->elems * (P->walk_f64 ? 8 : 4));
  if (s != TTNN_OK) {
    delete S;
    return s;
  }
  s = launch_fill_zero(S->acc, S->elems * (P->walk_f64 ? 8 : 4), (cudaStream_t)stream);
  if (s != TTNN_OK) {
    cudaFree(S->acc);
    delete S;
    return s;
  }
  *out = S;
  return TTNN_OK;
}

void ttnn_state_destroy(ttnn_state_t S) {
  if (!S) return;
  cudaFree(S->acc);
  delete S;
}

ttnn_status ttnn_state_zero(ttnn_state_t S, void* stream) {
  TTNN_CHECK_ARG(S, "null state");
  return launch_fill_zero(S->acc, S->elems * (S->plan->walk_f64 ? 8 : 4), (cudaStream_t)stream);
}

ttnn_status ttnn_state_buffer(ttnn_state_t S, void** p, int64_t* elems) {
  TTNN_CHECK_ARG(S, "null state");
  if (p) *p = S->acc;
  if (elems) *elems = S->elems;
  return TTNN_OK;
}

ttnn_status ttnn_state_axpy(ttnn_state_t dst, ttnn_state_t src, double alpha, void* stream) {
  TTNN_CHECK_ARG(dst && src, "null state");
  TTNN_CHECK_ARG(dst->plan == src->plan || dst->elems == src->elems, "states of different plans");
  return launch_axpy(dst->acc, src->acc, alpha, dst->elems, dst->plan->walk_f64, (cudaStream_t)stream);
}

ttnn_status ttnn_state_save(ttnn_state_t S, void* host, size_t bytes, void* stream) {
  TTNN_CHECK_ARG(S && host, "null argument");
  const size_t need = (size_t)S->elems * (S->plan->walk_f64 ? 8 : 4);
  TTNN_CHECK_ARG(bytes == need, "buffer must be %zu bytes", need);
  TTNN_TRY_CUDA(cudaMemcpyAsync(host, S->acc, need, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  TTNN_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return TTNN_OK;
}

ttnn_status ttnn_state_load(ttnn_state_t S, const void* host, size_t bytes, void* stream) {
  TTNN_CHECK_ARG(S && host, "null argument");
  const size_t need = (size_t)S->elems * (S->plan->walk_f64 ? 8 : 4);
  TTNN_CHECK_ARG(bytes == need, "buffer must be %zu bytes", need);
  TTNN_TRY_CUDA(cudaMemcpyAsync(S->acc, host, need, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  TTNN_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return TTNN_OK;
}

ttnn_status ttnn_update_dense(ttnn_state_t S, const void* data, const int64_t* offset,
                              const int64_t* extent, const float* tile_scale, double lambda,
                              void* stream) {
  TTNN_CHECK_ARG(S && data, "null argument");
  ttnn_plan_s& P = *S->plan;
  Box b;
  b.off.assign(P.d, 0);
  b.ext = P.dims;
  b.full = true;
  for (int m = 0; m < P.d; ++m) {
    if (offset) b.off[m] = offset[m];
    if (extent) b.ext[m] = extent[m];
    TTNN_CHECK_ARG(b.ext[m] >= 1 && b.off[m] >= 0 && b.off[m] + b.ext[m] <= P.dims[m],
                   "box outside the tensor on mode %d", m);
    if (b.off[m] != 0 || b.ext[m] != P.dims[m]) b.full = false;
  }
  TTNN_CHECK_ARG(P.pass_store != 3 || tile_scale, "E4M3 updates need tile scales");
  if (P.flags & TTNN_FLAG_STRUCTURED_ONLY) {
    set_error("the plan was made with TTNN_FLAG_STRUCTURED_ONLY: no dense updates");
    return TTNN_EUNSUPPORTED;
  }
  int64_t need = 0;
  TTNN_TRY(dense_update_need(P, b, &need));
  if (need > P.ws_bytes) TTNN_TRY(grow_workspace(P, need + 4096));
  return run_dense_update(P, S->acc, data, b, tile_scale, lambda, (cudaStream_t)stream, false,
                          nullptr);
}

ttnn_status ttnn_update_cp(ttnn_state_t S, int32_t cp_rank, const double* weights,
                           const double* const* factors, double lambda, void* stream) {
  TTNN_CHECK_ARG(S && weights && factors, "null argument");
  TTNN_CHECK_ARG(cp_rank >= 1, "cp_rank must be >= 1");
  ttnn_plan_s& P = *S->plan;
  for (int mu = 0; mu < P.d; ++mu) TTNN_CHECK_ARG(factors[mu], "null factor %d", mu);
  for (int q = 0; q < cp_rank; ++q)
    TTNN_CHECK_ARG(std::isfinite(weights[q]), "non-finite weight %d", q);
  TTNN_CHECK_ARG(std::isfinite(lambda), "non-finite lambda");
  return run_cp_update(P, S->acc, cp_rank, weights, factors, lambda, (cudaStream_t)stream);
}

ttnn_status ttnn_update_ttn(ttnn_state_t S, const double* const* cores_in, const int32_t* ranks_in,
                            double lambda, void* stream) {
  TTNN_CHECK_ARG(S && cores_in && ranks_in, "null argument");
  ttnn_plan_s& P = *S->plan;
  for (int v = 0; v < (int)P.nodes.size(); ++v) {
    TTNN_CHECK_ARG(cores_in[v], "null core %d", v);
    TTNN_CHECK_ARG(v == P.root || ranks_in[v] >= 1, "input rank of node %d must be >= 1", v);
  }
  TTNN_CHECK_ARG(std::isfinite(lambda), "non-finite lambda");
  const cudaStream_t st = (cudaStream_t)stream;
  int64_t need = 0;
  TTNN_TRY(run_ttn_update(P, nullptr, cores_in, ranks_in, lambda, st, true, &need));
  if (need > P.ws_bytes) TTNN_TRY(grow_workspace(P, need + 4096));
  return run_ttn_update(P, S->acc, cores_in, ranks_in, lambda, st, false, nullptr);
}

ttnn_status ttnn_recover(ttnn_state_t S, double* cores, void* stream) {
  TTNN_CHECK_ARG(S && cores, "null argument");
  TTNN_TRY(take_timeout(*S->plan));
  return run_recover(*S->plan, S->acc, cores, (cudaStream_t)stream, false, nullptr);
}

ttnn_status ttnn_recover_async(ttnn_state_t S, double* cores, void* stream) {
  TTNN_CHECK_ARG(S && cores, "null argument");
  TTNN_TRY(take_timeout(*S->plan));
  return run_recover(*S->plan, S->acc, cores, (cudaStream_t)stream, false, nullptr, true);
}

ttnn_status ttnn_plan_sync(ttnn_plan_t P) {
  TTNN_CHECK_ARG(P, "null plan");
  TTNN_TRY(take_timeout(*P));
  return plan_sync(*P);
}

ttnn_status sttnn_run(ttnn_plan_t P, const void* dense, const float* tile_scale, double* cores,
                      void* stream) {
  TTNN_CHECK_ARG(P && dense && cores, "null argument");
  TTNN_CHECK_ARG(P->variant == TTNN_VARIANT_STTNN, "sttnn_run needs an STTNN plan");
  ttnn_state_t S = nullptr;
  TTNN_TRY(ttnn_state_create(P, stream, &S));
  ttnn_status s = ttnn_update_dense(S, dense, nullptr, nullptr, tile_scale, 1.0, stream);
  if (s == TTNN_OK) s = ttnn_recover(S, cores, stream);
  ttnn_state_destroy(S);
  return s;
}

ttnn_status ttnn_hmt(ttnn_plan_t P, const void* dense, double* cores, void* stream) {
  TTNN_CHECK_ARG(P && dense && cores, "null argument");
  const cudaStream_t st = (cudaStream_t)stream;
  int64_t need = 0;
  TTNN_TRY(run_hmt(*P, dense, nullptr, st, true, &need));
  if (need > P->ws_bytes) TTNN_TRY(grow_workspace(*P, need + 4096));
  return run_hmt(*P, dense, cores, st, false, nullptr);
}

ttnn_status ttnn_round(ttnn_plan_t P, const double* const* cores_in, const int32_t* ranks_in,
                       double* cores, void* stream) {
  TTNN_CHECK_ARG(P && cores_in && ranks_in && cores, "null argument");
  ttnn_state_t S = nullptr;
  TTNN_TRY(ttnn_state_create(P, stream, &S));
  ttnn_status s = ttnn_update_ttn(S, cores_in, ranks_in, 1.0, stream);
  if (s == TTNN_OK) s = ttnn_recover(S, cores, stream);
  ttnn_state_destroy(S);
  return s;
}

ttnn_status ttnn_fp8_quantize(ttnn_plan_t P, const float* src, const int64_t* extent, uint8_t* dst,
                              float* scales, void* stream) {
  TTNN_CHECK_ARG(P && src && dst && scales, "null argument");
  int64_t rows = 1, cols = 1;
  for (int m = 0; m < P->d; ++m) {
    const int64_t e = extent ? extent[m] : P->dims[m];
    TTNN_CHECK_ARG(e >= 1 && e <= P->dims[m], "extent of mode %d outside 1..n", m);
    if (m >= P->Llo && m < P->Lhi) rows *= e;
    else cols *= e;
  }
  return launch_quantize_fp8(src, rows, cols, dst, scales, (cudaStream_t)stream);
}

ttnn_status ttnn_profile(ttnn_plan_t P, int32_t enable) {
  TTNN_CHECK_ARG(P, "null plan");
  P->profile = enable != 0;
  return TTNN_OK;
}

ttnn_status ttnn_profile_read(ttnn_plan_t P, int32_t phase, double* total_ms, int32_t* count) {
  TTNN_CHECK_ARG(P && phase >= 0 && phase < 4, "bad argument");
  double tot = 0.0;
  int cnt = 0;
  ttnn_status s = TTNN_OK;
  for (auto& pr : P->prof[phase]) {
    float ms = 0.f;
    if (s == TTNN_OK) {
      cudaError_t e = cudaEventSynchronize(pr.second);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
      if (e != cudaSuccess) {
        set_error("profile read: %s", cudaGetErrorString(e));
        s = TTNN_ECUDA;
      }
    }
    tot += ms;
    ++cnt;
    P->prof_pool.push_back(pr.first);
    P->prof_pool.push_back(pr.second);
  }
  P->prof[phase].clear();
  if (total_ms) *total_ms = tot;
  if (count) *count = cnt;
  return s;
}

ttnn_status ttnn_plan_pass_counts(ttnn_plan_t P, int64_t* tensor_core, int64_t* simt) {
  TTNN_CHECK_ARG(P, "null plan");
  if (tensor_core) *tensor_core = P->n_tc_pass;
  if (simt) *simt = P->n_simt_pass;
  return TTNN_OK;
}

ttnn_status ttnn_kernel_launches(int64_t* count) {
  TTNN_CHECK_ARG(count, "null argument");
  *count = launches_so_far();
  return TTNN_OK;
}

}  // extern "C"
