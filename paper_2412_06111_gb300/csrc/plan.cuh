// Host-side plan and state structures.
#pragma once

#include <array>
#include <functional>
#include <map>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "program.cuh"

struct TNode {
  int user = -1, lex = -1, level = 0, parent = -1, pos = 0;
  int lo = 0, hi = 0;
  bool leaf = false, identity = false;
  int r = 0, p = 0, s = 0;
  int64_t n = 1;
  int rsub = 0;                 // max r over sketched nodes of the subtree
  std::vector<int> ch;          // children (user indices), ordered by first mode
  std::vector<int> reuse;       // STTNN reuse set S_v (user indices), by first mode
  int64_t om_off = -1, om_el = 0, ps_off = -1, ps_el = 0;
  std::vector<int64_t> ps_shape;
  int64_t core_off = 0, core_el = 0;
  std::vector<int64_t> core_shape;
  int64_t xt_off = -1;          // STTNN XT_v factor offset (elements) in the factor arrays
  int kept = -1;
  int sweeps = 0;
  int64_t dx_off = -1, dy_off = -1;   // unstructured DRMs X_t, Y_t (TTNN_FLAG_DENSE_DRM)
  bool sketched() const { return parent >= 0 && !identity; }
};

struct ttnn_plan_s {
  int d = 0;
  std::vector<int64_t> dims;
  int64_t N = 1;
  std::vector<TNode> nodes;
  int root = -1;
  std::vector<int> lex;         // lex position -> user index
  int variant = 0, dtype = 1;
  double eps_factor = 10.0, u = 2.220446049250313e-16;
  uint64_t seed = 0;
  uint32_t flags = 0;
  int rmax = 1, smax = 1;
  // first-level split: L = root children [0, a), R = [a, m)
  int a = 1;
  int yside = 0;                // 0: root's Y applied on the R side (in D1), 1: on the L side (D2)
  int ychild = -1;              // the single root child whose Y is a pass-side block
  std::vector<int> Lch, Rch;
  int Llo = 0, Lhi = 0, Rlo = 0, Rhi = 0;
  int rXL = 0, rXR = 0;         // X-part widths of the side blocks B_R / B_L
  int wYR = 0, wYL = 0;         // Y-part widths
  int yR_ident = 0, yL_ident = 0;
  int wR = 0, wL = 0, wRpad = 0, wLpad = 0;
  // number formats
  int walk_f64 = 0;             // tree walk / accumulators in binary64
  int pass_store = 1;           // storage of the tensor: 0 f64 1 f32 2 bf16 3 e4m3
  int side_store = 1;           // storage of the pass DRM side blocks (same codes)
  int round_fmt = 1;            // DRM rounding (RoundFmt)
  // device memory
  double* fac64 = nullptr;      // X_mu, Y_mu, XT_v (binary64)
  void* facw = nullptr;         // the same in the walk type
  std::vector<int64_t> x_off, y_off;
  int64_t fac_elems = 0;
  void* sideR = nullptr;        // cached full-size side blocks (pass storage)
  void* sideL = nullptr;
  void* yW = nullptr;           // walk-type copy of the pass Y block (full box)
  void* xWo = nullptr;          // walk-type copy of the L side's X block over the R modes (full box)
  // binary32 plans: the cached side blocks as bf16 hi then lo halves (the
  // tensor-core pass of whole-tensor updates)
  void* sideRs = nullptr;
  void* sideLs = nullptr;
  void* dxy = nullptr;          // unstructured DRMs of every node, walk type (TTNN_FLAG_DENSE_DRM)
  char* ws = nullptr;
  int64_t ws_bytes = 0;
  // the recovery's own scratch: a recovery may run on another stream while
  // the next update of another state of the plan uses `ws`
  char* ws_rec = nullptr;
  int64_t ws_rec_bytes = 0;
  int64_t dev_bytes = 0;        // device memory the plan holds (all its allocations)
  // workspace bytes a dense update needs, by box extents (+ whole-tensor flag)
  std::map<std::vector<int64_t>, int64_t> ws_need_cache;
  ttnn::QrJob* jobs_dev = nullptr;
  std::vector<ttnn::QrJob> jobs_host;   // what jobs_dev holds (upload skipped when unchanged)
  int* kept_dev = nullptr;
  int* err_dev = nullptr;       // device error word of bounded waits (tensor-core pass)
  // read-back of the last recovery: kept ranks, Jacobi sweeps, error word
  int* host_kept = nullptr;     // pinned, 2 * n_sketched + 1 ints
  cudaEvent_t kept_ev = nullptr;
  bool kept_pending = false;
  bool timeout_seen = false;    // a read-back waited for by ttnn_plan_node carried a timeout
  std::vector<int> kept_nodes;  // node of each job of the pending read-back
  int n_sketched = 0;
  int64_t state_elems = 0;
  int64_t core_elems = 0;
  int tc_ok = 0;                // tensor-core pass usable for this plan
  int64_t n_tc_pass = 0, n_simt_pass = 0;
  int last_walk_ops = 0, last_walk_levels = 0;   // shape of the last update's walk program
  // profiling: event pairs per phase (0 pass, 1 walk, 2 recovery)
  int profile = 0;
  // profiled intervals: 0 pass phase, 1 walk, 2 recovery, 3 the first-level
  // pass kernel alone (to its end, before any partial-sum reduction)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof[4];
  cudaEvent_t prof_kernel_end = nullptr;   // recorded by a pass launch right after its kernel
  std::vector<cudaEvent_t> prof_pool;   // events of read intervals, reused
};

struct ttnn_state_s {
  ttnn_plan_s* plan = nullptr;
  void* acc = nullptr;
  int64_t elems = 0;
};

namespace ttnn {

struct Box {
  std::vector<int64_t> off, ext;
  bool full = true;
};

ttnn_status build_plan(ttnn_plan_s& P, const ttnn_tree* tree, int32_t d, const int64_t* dims,
                       const int32_t* ranks, const int32_t* oversample, uint64_t seed,
                       const ttnn_opts* opts);

// Runs (or, with dry = true, sizes) one dense update.  Returns the peak
// workspace bytes through *peak when dry.
// Workspace bytes a dense update of `box` needs (dry run, cached per shape).
ttnn_status dense_update_need(ttnn_plan_s& P, const Box& box, int64_t* need);
// Workspace bytes of a CP update (any rank: ranks are taken kProjQ at a time).
int64_t cp_update_need(const ttnn_plan_s& P);
// Unstructured Gaussian DRMs (dense_drm.cu): the plan's restrictions, the
// factor layout (sets dx_off / dy_off, returns the element count), their
// generation in binary64 (rounded to the plan's format) and one update.
ttnn_status dense_drm_check(const ttnn_plan_s& P);
int64_t dense_drm_elems(ttnn_plan_s& P);
ttnn_status dense_drm_generate(ttnn_plan_s& P, double* tmp64, cudaStream_t st);
ttnn_status run_dense_drm_update(ttnn_plan_s& P, void* acc, const void* data, const Box& box,
                                 double lambda, cudaStream_t st, bool dry, int64_t* peak);
// TTN-HMT of a dense tensor with the plan's unstructured X_t (binary64):
// cores in the plan's core layout; dry: only the workspace peak.
ttnn_status run_hmt(ttnn_plan_s& P, const void* data, double* cores, cudaStream_t st, bool dry,
                    int64_t* peak);
// Bytes of the library's static scratch block (ttnn_update_dense_static),
// resident on a device once the library's module is loaded there.
int64_t static_scratch_resident_bytes();
// A real (non-dry) update first checks its workspace need against the plan's
// workspace and returns TTNN_ENOMEM, launching nothing, when it does not fit.
// Work of several dense updates recorded for joint launches: the box side
// blocks cut from cached blocks (one batched gather), the first-level
// passes (launched in order after the gathers), and the tree walks (one
// merged program after the passes).
struct UpdateBatch {
  std::vector<GatherJob> gathers;
  std::vector<std::function<ttnn_status(cudaStream_t)>> passes;
  Program walks;
  ttnn_status launch(cudaStream_t st);
};
// batch != NULL: nothing is launched; the update's work is appended to *batch.
ttnn_status run_dense_update(ttnn_plan_s& P, void* acc, const void* data, const Box& box,
                             const float* tile_scale, double lambda, cudaStream_t st, bool dry,
                             int64_t* peak, UpdateBatch* batch = nullptr);
// CP term update (structured.cu): factors are d device pointers, n_mu x Q
// row-major binary64; weights host [Q].
ttnn_status run_cp_update(ttnn_plan_s& P, void* acc, int Q, const double* weights,
                          const double* const* factors, double lambda, cudaStream_t st);
// TTN-format input update (plan.cu): cores_in host array of device binary64
// cores, ranks_in host [n_nodes].  dry: records only, *peak = workspace bytes.
ttnn_status run_ttn_update(ttnn_plan_s& P, void* acc, const double* const* cores_in,
                           const int32_t* ranks_in, double lambda, cudaStream_t st, bool dry,
                           int64_t* peak);
// Per-128x128-tile E4M3 quantisation of a binary32 rows x cols matrix (pass_cvt.cu).
ttnn_status launch_quantize_fp8(const float* src, int64_t rows, int64_t cols, uint8_t* dst,
                                float* scales, cudaStream_t st);
// defer != NULL: a block that is a gather from the cached blocks is appended
// to *defer instead of launched (blocks that need computing are launched).
ttnn_status make_side(ttnn_plan_s& P, const Box& box, int which, void* out, int64_t ld,
                      cudaStream_t st, std::vector<GatherJob>* defer = nullptr);
ttnn_status launch_split_bf16(const float* src, int64_t n, void* hi, void* lo, cudaStream_t st);
ttnn_status make_side_xo(ttnn_plan_s& P, const Box& box, void* out, int64_t ld, cudaStream_t st);
// Omega of an L-side Y child is taken through D2 (a reduction over the R
// index) for whole 2-D boxes of nL x nR
bool omega_via_d2(const ttnn_plan_s& P, int64_t nL, int64_t nR);
ttnn_status make_side_yw(ttnn_plan_s& P, const Box& box, void* out, int64_t ld, cudaStream_t st,
                         std::vector<GatherJob>* defer = nullptr);
// records an event on `st` if profiling is on (returns nullptr otherwise)
cudaEvent_t prof_event(ttnn_plan_s& P, cudaStream_t st);
void prof_push(ttnn_plan_s& P, int phase, cudaEvent_t a, cudaEvent_t b);
// Waits for a pending recovery read-back and stores kept ranks / sweeps in
// the nodes; TTNN_ETIMEOUT (and clears the device word) if a bounded device
// wait of an earlier update or recovery ran out.
ttnn_status plan_sync(ttnn_plan_s& P);
// async: returns once everything is enqueued (read-back completes later,
// see plan_sync); otherwise waits and checks like plan_sync.
ttnn_status run_recover(ttnn_plan_s& P, const void* acc, double* cores, cudaStream_t st, bool dry,
                        int64_t* peak, bool async = false);

}  // namespace ttnn
