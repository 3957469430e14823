/*
 * ttnn.h -- C ABI of the GB300 (sm_103a) implementation of tree tensor network
 * Nystrom (TTNN) and its sequential variant STTNN, after Bucci & Verzella,
 * "Randomized algorithms for streaming low-rank approximation in tree tensor
 * network format", arXiv:2412.06111.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers are plain host or device pointers as stated per argument; no
 *   argument is a C++ or framework type.  A "stream" is a cudaStream_t passed
 *   as void* (NULL = the legacy default stream).
 * - The caller owns every buffer it passes in; the library never frees one.
 *   A plan owns its DRM factors and workspace; a state owns its sketch
 *   accumulators.  Both are freed by their destroy call.
 * - Dense tensors are row-major over their modes (last mode fastest).
 * - Errors are returned as ttnn_status; nothing is thrown across the ABI.  A
 *   call that fails validation leaves plan and state unchanged.  After
 *   TTNN_ECUDA the state content is unspecified.  ttnn_last_error() returns a
 *   one-line message for the calling thread's last failure.
 * - Calls on one plan (and the states made from it) are serialised by the
 *   caller, with one exception: the plan keeps one workspace for updates and
 *   another for recoveries, so a recovery (ttnn_recover / _async) of one state
 *   may run on another stream while an update of another state of the same
 *   plan runs (the caller orders the two with events; updates among
 *   themselves, and recoveries among themselves, stay on one stream or are
 *   otherwise serialised).  Different plans may run concurrently on
 *   different streams.
 * - Work is enqueued on the given stream; a call returns once its work is
 *   enqueued unless stated otherwise.
 *
 * Layout of the tree and of the results (paper notation in brackets)
 * ------------------------------------------------------------------
 * - Index tree [Sec. 3, Def. "index tree"]: node v has parent parent[v]
 *   (-1 = root); leaves list their modes (0-based) in the CSR arrays
 *   leaf_mode_ptr / leaf_modes.  Every node's modes (the union over its
 *   leaves) must form one contiguous range and children partition their
 *   parent; children are ordered by first mode.  Internal nodes need >= 2
 *   children.
 * - identity[v] != 0 (or r_v >= n_v on a leaf) makes v a dummy-like node
 *   [Sec. 4: X = Y = P = I on dummy nodes]: its core is the identity.
 * - Ranks r_v and oversampling p_v are per node (root entries ignored); r_v
 *   is clipped to min(n_v, n_{D\v}) and p_v to n_v - r_v.  s_v = r_v + p_v.
 * - Sketches [Sec. 4, sketch phase]: Omega_v is s_v x r_v; Psi of an
 *   internal node is (s'_c1, ..., s'_cm, r_v) with s'_c = s_c (n_c for an
 *   identity child); Psi of a leaf is (n_v, r_v); Psi_root is
 *   (s'_c1, ..., s'_cm).  All row-major.
 * - Cores [Def. "Tree tensor network format"]: root (r_c1..r_cm); transfer
 *   (r_v, r_c1..r_cm); leaf (r_v, n_mu1..n_muk); identity leaf (n_v, n_v).
 *   Binary64, row-major, at the per-node offsets of ttnn_node_info.
 *
 * DRMs [Sec. 7, Khatri-Rao sketchings]: per-mode Gaussian factors X_mu
 * (n_mu x r_max), Y_mu (n_mu x s_max) drawn by Philox4x32-10 + Box-Muller
 * (bit-identical on host and device, see ttnn_philox_gaussian), rounded to the
 * plan's sketch number format; X_v / Y_v are their Khatri-Rao products over
 * the complement / own modes, first r_v / s_v columns.  The Khatri-Rao blocks
 * that multiply the dense tensor on the first-level pass are stored in the
 * sketch format and are therefore rounded once more (exact for binary64).
 */
#ifndef TTNN_H
#define TTNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TTNN_OK = 0,
  TTNN_EINVAL = 1,       /* invalid argument, tree, size or pointer */
  TTNN_ENOMEM = 2,       /* device or host allocation failed */
  TTNN_ECUDA = 3,        /* a CUDA call or kernel launch failed */
  TTNN_ENUMERIC = 4,     /* non-finite values; reserved: non-finite scalar arguments
                            (CP weights, lambda) are refused with TTNN_EINVAL, and tensor
                            data are not scanned (a NaN or Inf in an update reaches the
                            sketches and the recovered cores) */
  TTNN_ETIMEOUT = 5,     /* a bounded device wait ran out */
  TTNN_EBUSY = 6,        /* resource in use (serving: no free slot) */
  TTNN_EUNSUPPORTED = 7  /* valid request this library does not implement */
} ttnn_status;

/* Number formats of the tensor and of the pass-side DRM blocks. */
typedef enum {
  TTNN_F64 = 0,   /* binary64 everywhere (accumulators binary64) */
  TTNN_F32 = 1,   /* binary32 tensor, FP32 FMA pass, FP32 accumulators */
  TTNN_BF16 = 2,  /* bfloat16 tensor + DRM blocks on tensor cores, FP32 accumulation */
  TTNN_E4M3 = 3,  /* FP8 E4M3 tensor with one FP32 scale per 128x128 tile, FP32 accumulation */
  TTNN_BF16X2 = 4 /* FP32 tensor split hi+lo into two bf16 MMAs, FP32 accumulation */
} ttnn_dtype;

typedef enum { TTNN_VARIANT_TTNN = 0, TTNN_VARIANT_STTNN = 1 } ttnn_variant;

typedef struct {
  int32_t n_nodes;
  const int32_t* parent;        /* host [n_nodes]; -1 marks the root */
  const int32_t* leaf_mode_ptr; /* host [n_nodes + 1]; CSR offsets into leaf_modes */
  const int32_t* leaf_modes;    /* host; 0-based modes of each leaf */
  const uint8_t* identity;      /* host [n_nodes] or NULL; nonzero forces P = I on a leaf */
} ttnn_tree;

typedef struct {
  int32_t variant;       /* ttnn_variant */
  int32_t sketch_dtype;  /* ttnn_dtype */
  double eps_factor;     /* eps = eps_factor * unit_roundoff * ||R_v||_2; paper: 10 */
  double unit_roundoff;  /* paper's "machine precision" u; default 2^-52 */
  uint32_t flags;        /* TTNN_FLAG_* */
} ttnn_opts;

#define TTNN_FLAG_NO_SIDE_CACHE 1u  /* do not cache full-size pass DRM blocks */
#define TTNN_FLAG_SIMT_PASS 2u      /* use the SIMT pass even for BF16 (testing) */
#define TTNN_FLAG_STRUCTURED_ONLY 8u /* the plan takes CP / TTN-format updates only: no
                                         cached pass blocks, no dense-pass workspace
                                         (ttnn_update_dense returns TTNN_EUNSUPPORTED) */
#define TTNN_FLAG_CLUSTER_REDUCE 4u /* tensor-core pass: sum the column-chunk partials of D1
                                       across a thread-block cluster (distributed shared
                                       memory) instead of by the last CTA of each row block */
#define TTNN_FLAG_DUMP_PROGRAM 16u  /* debugging: run every tree-walk / assembly op as its own
                                       launch, synchronise, and print its time, level, kind,
                                       shape and blocks to stderr */
#define TTNN_FLAG_RESERVE_SMS 64u   /* the tensor-core first-level passes leave max(8, sketched
                                       nodes) SMs (at most a quarter) free, so that a recovery
                                       of another state issued on another stream runs beside
                                       the next update's pass instead of after it */
#define TTNN_FLAG_DENSE_DRM 128u    /* unstructured Gaussian DRMs [Sec. 4 eq. (sketch), the DRMs
                                       of Thm 6.6]: node v draws its own X_v (n_{D\v} x r_v,
                                       Philox kind 4) and Y_v (n_v x s_v, kind 5) keyed by its
                                       lexicographic index, rounded to the plan's format,
                                       instead of Khatri-Rao products of per-mode factors.
                                       TTNN, binary64 / binary32 plans, at most 8 GiB of DRMs,
                                       whole-tensor dense updates only (boxes, CP and
                                       TTN-format updates: TTNN_EUNSUPPORTED) */
#define TTNN_FLAG_TRUNCATE 256u    /* eps-truncated output [Sec. 4 recovery, eq.
                                       (stabilized_nystrom)]: the directions the eps-pseudo-
                                       inverse drops are cut from the cores, R_v,eps^+ being
                                       applied as (V_1 Sigma_1^-1) U_1^T with U_1 moved into the
                                       parent's Q_v: every core has its rank axes at the kept
                                       ranks, written compactly (row-major) from its offset;
                                       ttnn_plan_node reports those shapes after the recovery */
#define TTNN_FLAG_WAIT_TEST 32u     /* testing the bounded-wait error path: the pipeline waits
                                       of the tensor-core passes give up at once, so a dense
                                       update on this plan is abandoned on the device and the
                                       next ttnn_recover / ttnn_plan_sync returns TTNN_ETIMEOUT
                                       (the plan and its CUDA context stay usable) */

typedef struct ttnn_plan_s* ttnn_plan_t;
typedef struct ttnn_state_s* ttnn_state_t;

typedef struct {
  int32_t user_index;   /* index in the caller's parent[] */
  int32_t lex_index;    /* position in the (level, position) order */
  int32_t level, parent, n_children, mode_lo, mode_hi;
  int32_t is_leaf, identity, r, p, s;
  int64_t n;            /* n_v = prod of the node's mode sizes */
  int64_t omega_offset, omega_elems;  /* in the state buffer (elements) */
  int64_t psi_offset, psi_elems;
  int32_t psi_ndim;
  int64_t psi_shape[10];
  int64_t core_offset, core_elems;    /* in the caller's core buffer (binary64 elements) */
  int32_t core_ndim;
  int64_t core_shape[10];
  int32_t kept_rank;    /* after ttnn_recover: rank kept by the eps-pseudo-inverse (-1 before) */
  int32_t jacobi_sweeps; /* after ttnn_recover: sweeps of the one-sided Jacobi SVD of R_v */
} ttnn_node_info;

/* ---------------------------------------------------------------------- */
/* Status text.  Never NULL.                                               */
const char* ttnn_status_string(ttnn_status s);
/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to n bytes) into buf (host).  Returns TTNN_OK. */
ttnn_status ttnn_last_error(char* buf, size_t n);

/* ttnn_debug_fail_alloc -- allocation-failure injection for tests (the paper
 * has no counterpart).  nth >= 1: the nth device allocation the library makes
 * from now on (in any thread) fails as if cudaMalloc had run out of memory;
 * nth = 0 disarms.  The failing call returns TTNN_ENOMEM and leaves every
 * existing plan and state as it was (a plan creation frees what it had
 * allocated; a workspace that would have grown keeps its old block).
 * EINVAL: nth < 0. */
ttnn_status ttnn_debug_fail_alloc(int32_t nth);

/* ttnn_philox_gaussian -- the DRM generator [Sec. 7 per-mode factors; the
 * paper draws N(0,1) entries].  Writes rows x cols binary64 N(0,1) values to
 * dst (device, row-major): element (i, j) is Box-Muller output (j & 1) of
 * Philox4x32-10 with counter (i, j >> 1, (kind << 24) | ident, 0) and key
 * (seed mod 2^32, seed >> 32); kind 1 = X_mu, 2 = Y_mu, 3 = STTNN XT_s.  If
 * round_dtype is TTNN_F32/BF16/E4M3 the values are rounded (nearest-even)
 * into that format's value set and still stored as binary64.
 * EINVAL: rows/cols < 0, kind outside 1..5, ident >= 2^24, dst NULL. */
ttnn_status ttnn_philox_gaussian(uint64_t seed, int32_t kind, int32_t ident, int64_t rows,
                                 int64_t cols, int32_t round_dtype, double* dst, void* stream);

/* ttnn_plan_create -- A1/A2 of the method [Sec. 4 Algorithm 2, first loop;
 * Sec. 5 ordering]: validates and normalises the tree, fixes the
 * lexicographic order, the STTNN reuse sets and the first-level split,
 * draws the DRM factors on the device and sizes the workspace.
 * tree, dims (host [d]), ranks and oversample (host [n_nodes]) are read during
 * the call only.  opts may be NULL (TTNN, F32, eps_factor 10, u = 2^-52).
 * EINVAL: invalid tree/sizes (see conventions), a tensor of more than 2^46
 * entries without TTNN_FLAG_STRUCTURED_ONLY (up to 2^62 with it: CP and
 * TTN-format inputs never form the tensor); EUNSUPPORTED: STTNN whose
 * first root child is an identity leaf, or a TTNN_BF16X2 / TTNN_E4M3 plan
 * whose whole-tensor pass matrix (n_L x n_R) the tensor-core pass does not
 * take (n_L a multiple of 8; n_R a multiple of 8, or of 16 for E4M3; side
 * widths of at most 256 columns); ENOMEM/ECUDA. */
ttnn_status ttnn_plan_create(const ttnn_tree* tree, int32_t d, const int64_t* dims,
                             const int32_t* ranks, const int32_t* oversample, uint64_t seed,
                             const ttnn_opts* opts, void* stream, ttnn_plan_t* out);
void ttnn_plan_destroy(ttnn_plan_t plan);

/* ttnn_plan_device_bytes -- the plan's device footprint (no counterpart in
 * the paper): *total = bytes of device memory the plan holds (DRM factors,
 * cached pass blocks, workspace, recovery buffers; states are separate),
 * *workspace = its workspace block, which dense / TTN-format updates grow on
 * demand.  Either pointer may be NULL.  EINVAL: null plan. */
ttnn_status ttnn_plan_device_bytes(ttnn_plan_t P, int64_t* total, int64_t* workspace);

/* Sizes: state elements (binary64 for TTNN_F64 plans, binary32 otherwise),
 * bytes per state element, total binary64 elements of all cores, number of
 * tree nodes.  Any output pointer may be NULL. */
ttnn_status ttnn_plan_sizes(ttnn_plan_t plan, int64_t* state_elems, int32_t* state_elem_bytes,
                            int64_t* core_elems, int32_t* n_nodes);
/* Per-node layout, by the caller's node index. */
ttnn_status ttnn_plan_node(ttnn_plan_t plan, int32_t user_index, ttnn_node_info* out);
/* Copies one per-mode DRM factor as stored by the plan (binary64, device dst,
 * row-major n_mu x cols): which = 1 for X_mu (cols = r_max), 2 for Y_mu
 * (cols = s_max), 3 for XT of the node with lexicographic index `mode`. */
ttnn_status ttnn_plan_factor(ttnn_plan_t plan, int32_t which, int32_t mode, double* dst,
                             int64_t* rows, int64_t* cols, void* stream);

/* States: zeroed device accumulators for all Omega_v, Psi_v, Psi_root. */
ttnn_status ttnn_state_create(ttnn_plan_t plan, void* stream, ttnn_state_t* out);
void ttnn_state_destroy(ttnn_state_t state);
ttnn_status ttnn_state_zero(ttnn_state_t state, void* stream);
/* Raw accumulator buffer (device) and its element count. */
ttnn_status ttnn_state_buffer(ttnn_state_t state, void** device_ptr, int64_t* elems);
/* dst += alpha * src (same plan): sums partial sketches of disjoint parts of
 * a tensor, e.g. from several GPUs or processes (Sec. 4: the sketch phase is
 * linear in T). */
ttnn_status ttnn_state_axpy(ttnn_state_t dst, ttnn_state_t src, double alpha, void* stream);
/* Checkpoint: copies the accumulators to / from host memory (bytes must be
 * state_elems * state_elem_bytes); synchronous on the stream. */
ttnn_status ttnn_state_save(ttnn_state_t state, void* host_buf, size_t bytes, void* stream);
ttnn_status ttnn_state_load(ttnn_state_t state, const void* host_buf, size_t bytes, void* stream);

/* ttnn_update_dense -- A3-A6 [Sec. 4 sketch phase + "streaming by
 * linearity"]: adds lambda * sketch(H) to the state, where H is zero outside
 * the box offset[mu] <= i_mu < offset[mu] + extent[mu] and equals `data` on
 * it.  data: device, row-major over the extents, in the plan's format
 * (TTNN_BF16X2 plans take binary32 and sketch hi + lo with hi = bf16(x),
 * lo = bf16(x - hi); TTNN_E4M3 plans take the E4M3 bytes with `tile_scale`
 * (device, one binary32 per 128x128 tile of the box's pass matrix, see
 * ttnn_fp8_quantize) ).  offset/extent: host [d], NULL = whole tensor.
 * EINVAL: box outside the tensor, empty box, NULL data. */
ttnn_status ttnn_update_dense(ttnn_state_t state, const void* data, const int64_t* offset,
                              const int64_t* extent, const float* tile_scale, double lambda,
                              void* stream);

/* ttnn_update_dense_static -- ttnn_update_dense (same arguments, same
 * result) for callers that must not allocate device memory while they stream
 * updates, e.g. callers whose memory comes from their own pool, or who must
 * not let cudaMalloc / cudaFree synchronise the device mid-stream.  The paper
 * has no counterpart: this is an interface of this library only.
 * Its scratch is one fixed block of static device memory of 32 MiB per device
 * (not the plan's workspace); the call allocates no device memory.  The
 * block is part of the library's device module: once that module is loaded on
 * a device (at the first call here, or at context creation under
 * CUDA_MODULE_LOADING=EAGER) the 32 MiB stay resident there until the process
 * exits, whether or not this entry point is ever called.
 * EINVAL (before any work is enqueued) if the update needs more scratch than
 * that; otherwise as ttnn_update_dense.  The block's address is looked up on
 * the first call made with a device current, and again when that device's
 * current context has changed (e.g. after cudaDeviceReset): make the first
 * call before any stream capture begins.  Calls that overlap in time (any
 * plan, any stream, any host thread of the process) share the block and race:
 * serialise them.  No profiling intervals are recorded. */
ttnn_status ttnn_update_dense_static(ttnn_state_t state, const void* data, const int64_t* offset,
                                     const int64_t* extent, const float* tile_scale,
                                     double lambda, void* stream);

/* ttnn_update_cp -- A5 [Sec. 4 streaming by linearity; Sec. 7 Khatri-Rao
 * sketchings]: adds lambda * sum_q w_q a_1q o ... o a_dq (a CP term) to the
 * sketches without forming it: with x_mu = X_mu^T a_mu, y_mu = Y_mu^T a_mu,
 * Omega_t[i,j] = sum_q w_q prod_{mu in t} y_muq[i] prod_{mu not in t} x_muq[j],
 * and Psi likewise (identity children and leaves use the raw factors).
 * weights: host [cp_rank], finite; factors: host array of d device pointers,
 * factor mu is n_mu x cp_rank row-major binary64.  Products are binary64 on
 * the stored DRM factors (no second rounding), added into the state.
 * Two launches per 16 ranks.  EINVAL: null pointers, cp_rank < 1, non-finite
 * weights or lambda; EUNSUPPORTED: STTNN plans, order > 16, nodes with more
 * than 9 children. */
ttnn_status ttnn_update_cp(ttnn_state_t state, int32_t cp_rank, const double* weights,
                           const double* const* factors, double lambda, void* stream);

/* ttnn_update_ttn -- A8 [Sec. 7 structured sketchings, TTN rounding]: adds
 * lambda * sketch(T_in) for a tensor given in TTN format on the same tree,
 * by an up sweep (cores against the Khatri-Rao X and Y factors) and a down
 * sweep (environments E_t), never forming T_in.
 * cores_in: host array (n_nodes) of device pointers to binary64 cores in the
 * core layout above with input ranks ranks_in (host [n_nodes] >= 1, root
 * ignored); identity leaves of the plan still take an (R_v, n_v) input core.
 * Computed in the plan's walk type (binary64 for TTNN_F64 plans, binary32
 * otherwise, cores converted once); the DRM factors are the stored values
 * and their Khatri-Rao products are not rounded again.  The plan workspace
 * grows (cudaFree + cudaMalloc, which synchronise the device) when an input
 * needs more than it holds.  EUNSUPPORTED for STTNN plans. */
ttnn_status ttnn_update_ttn(ttnn_state_t state, const double* const* cores_in,
                            const int32_t* ranks_in, double lambda, void* stream);

/* ttnn_recover -- A9 [Sec. 4 recovery phase, Algorithm 2, stabilised least
 * squares with eps = eps_factor * u * ||R_v||_2]: QR of every Omega_v
 * (diag R >= 0; CholeskyQR2 when both Gram matrices are safely positive
 * definite, else Householder), eps-pseudo-inverse of R_v (R_v^-1 when
 * sigma_min(R_v) > eps is certified, else by one-sided Jacobi SVD), then
 * B_v = (kron_c Q_c)^T Psi_v R_v,eps^+ (children's Q), leaf B_v = Psi_v
 * R_v,eps^+, root B = (kron_c Q_c)^T Psi_root; all in binary64.
 * cores: device, core_elems binary64 values at the per-node offsets.
 * Synchronises the stream before returning (kept ranks are read back).
 * ETIMEOUT: a bounded device wait of an earlier update or recovery on this
 * plan ran out (the cores are then unspecified). */
ttnn_status ttnn_recover(ttnn_state_t state, double* cores, void* stream);
/* ttnn_recover without the wait: returns once the recovery is enqueued; the
 * kept ranks and the device error word are copied back asynchronously and
 * taken in by the next ttnn_plan_sync, ttnn_plan_node or recovery call on
 * the plan.  For pipelines that read the cores on the device. */
ttnn_status ttnn_recover_async(ttnn_state_t state, double* cores, void* stream);
/* Waits for the read-back of the last asynchronous recovery; ETIMEOUT if a
 * bounded device wait of an earlier call on the plan ran out. */
ttnn_status ttnn_plan_sync(ttnn_plan_t plan);

/* sttnn_run -- STTNN end to end on a whole dense tensor [Sec. 5]: a plan made
 * with variant TTNN_VARIANT_STTNN, one pass over `dense` (plan format), then
 * recovery into `cores`.  EINVAL if the plan is not an STTNN plan. */
ttnn_status sttnn_run(ttnn_plan_t plan, const void* dense, const float* tile_scale,
                      double* cores, void* stream);

/* ttnn_hmt -- TTN-HMT, the randomised comparator of Sec. 8 (the TTN-SVD with
 * every SVD replaced by the HMT range finder, on the same right sketches X_t
 * as TTNN): two passes over the dense tensor (device, binary64, row-major);
 * pass 1 forms Q_t = orth(T^(t) X_t) for every node (Householder QR in
 * binary64), pass 2 the root core (kron_c Q_c)^T T; leaf cores Q_t^T,
 * transfer cores (kron_c Q_c)^T Q_t.  cores: device, the plan's core layout
 * (ttnn_plan_node).  Needs a TTNN_F64 plan with TTNN_FLAG_DENSE_DRM (the X_t
 * are the plan's unstructured DRMs); grows the plan's workspace if needed.
 * Synchronous with the stream's order only (no host wait).
 * EINVAL: NULL arguments; EUNSUPPORTED: other plans; ENOMEM / ECUDA. */
ttnn_status ttnn_hmt(ttnn_plan_t plan, const void* dense, double* cores, void* stream);

/* ttnn_round -- TTN rounding end to end [Sec. 7]: sketches of a TTN-format
 * input (see ttnn_update_ttn) followed by recovery into `cores`. */
ttnn_status ttnn_round(ttnn_plan_t plan, const double* const* cores_in, const int32_t* ranks_in,
                       double* cores, void* stream);

/* ttnn_fp8_quantize -- helper for TTNN_E4M3 plans: quantises a binary32
 * dense tensor (device, whole tensor or box extents; extent host [d] or NULL)
 * to E4M3 bytes (device dst, same element order) with one binary32 scale per
 * 128 x 128 tile of the pass matrix (rows = the plan's first-level left modes,
 * columns = the rest): s = max|tile| / 448 (binary32 division; 1 for an
 * all-zero tile), q = e4m3(x / s) (binary32 division, nearest-even,
 * saturating at +-448).  scales (device) is row-major [ceil(rows/128)]
 * [ceil(cols/128)].  The E4M3 pass sketches the dequantised tiles
 * bf16(f32(q * s)).  Inputs must be finite.  EINVAL: null pointers, extents
 * outside 1..n_mu. */
ttnn_status ttnn_fp8_quantize(ttnn_plan_t plan, const float* src, const int64_t* extent,
                              uint8_t* dst, float* scales, void* stream);

/* Profiling (no counterpart in the paper; this library's instrumentation):
 * with enable != 0 every later update / recovery on this plan records CUDA
 * events around its phases on the stream it runs on.  ttnn_profile_read
 * synchronises those events and returns the summed milliseconds and the
 * number of recorded intervals of one phase since the last read, then clears
 * them.  phase 0 = first-level pass kernel(s) with their partial-sum
 * reductions, 1 = tree walk and accumulation, 2 = recovery, 3 = the
 * tensor-core pass kernel alone (whole dense updates not batched by a
 * server).  At most 4096 intervals are kept per phase. */
ttnn_status ttnn_profile(ttnn_plan_t plan, int32_t enable);
ttnn_status ttnn_profile_read(ttnn_plan_t plan, int32_t phase, double* total_ms, int32_t* count);
/* Counts of first-level passes this plan has run on the tensor cores
 * (tcgen05) and on the SIMT path (FP64 / FP32 plans, or shapes the
 * tensor-core pass does not take). */
ttnn_status ttnn_plan_pass_counts(ttnn_plan_t plan, int64_t* tensor_core, int64_t* simt);
/* Number of device kernels this library has launched in this process. */
ttnn_status ttnn_kernel_launches(int64_t* count);

/* ---------------------------------------------------------------------- */
/* Serving (A11): many resident sketch streams on one GPU.                 */
/* The paper streams updates into one sketch (Sec. 4, linearity); a server */
/* keeps many such streams resident and folds a continuous flow of update  */
/* requests into them.  Worker threads, each with its own CUDA stream and  */
/* queue (stream k is served by worker k % workers), take batches (at most  */
/* one request per stream per batch, so each stream applies its requests   */
/* in submission order), launch every update's first-level pass and then   */
/* the tree walks of the whole batch as one merged program; completion is  */
/* tracked with CUDA events.  A stream's sketch is the same, bit for bit,  */
/* as applying its updates alone with ttnn_update_dense.  All server calls */
/* are thread-safe.                                                        */
/* ---------------------------------------------------------------------- */
typedef struct ttnn_server_s* ttnn_server_t;

typedef struct {
  int64_t hbm_budget_bytes;  /* device memory all open streams may hold (plans + states);
                                the library's 32 MiB static scratch block (resident once
                                its module is loaded) is counted against it: must exceed it */
  int32_t max_batch;         /* requests per batch; <= 0: 64 */
  int32_t queue_capacity;    /* requests outstanding (queued or on the device) before
                                submits are refused with EBUSY; <= 0: 65536 */
  int32_t workers;           /* worker threads, each with its own CUDA stream; <= 0: 4 */
  int32_t stream_queue_capacity; /* requests outstanding per stream before its submits are
                                    refused with EBUSY (keeps one busy stream from filling
                                    the queue); <= 0: unbounded */
} ttnn_server_opts;

typedef struct {
  int64_t completed_updates, completed_recoveries, failed, batches;
  int64_t update_bytes;      /* tensor bytes of the completed updates */
  double p50_us, p99_us, max_us;  /* request latency: submit -> completion seen by the worker */
  double seconds;            /* since the last reset */
  int64_t device_bytes;      /* held by the open streams */
  int32_t open_streams;
  int64_t queued;
  double worker_host_s;      /* worker time spent recording and launching batches */
} ttnn_server_report;

/* Creates a server on the current device (its own CUDA streams and worker
 * thread).  EINVAL: budget <= 0; ECUDA / ENOMEM. */
ttnn_status ttnn_server_create(const ttnn_server_opts* opts, ttnn_server_t* out);
/* Finishes every queued request, stops the worker and frees all streams. */
void ttnn_server_destroy(ttnn_server_t server);
/* Opens a stream: a plan + zeroed state as ttnn_plan_create /
 * ttnn_state_create (same arguments).  Admission: EBUSY (nothing kept) when
 * the stream's device memory would take the open streams over the budget. */
ttnn_status ttnn_server_open(ttnn_server_t server, const ttnn_tree* tree, int32_t d,
                             const int64_t* dims, const int32_t* ranks,
                             const int32_t* oversample, uint64_t seed, const ttnn_opts* opts,
                             int32_t* stream_id);
/* Closes a stream once its requests are done (waits at most timeout_us:
 * ETIMEOUT, stream kept) and frees its memory. */
ttnn_status ttnn_server_close(ttnn_server_t server, int32_t stream_id, int64_t timeout_us);
/* Queues ttnn_update_dense(stream, data, offset, extent, tile_scale, lambda).
 * data / tile_scale (device) must stay valid until the ticket is done.
 * Argument errors as ttnn_update_dense (checked here); EBUSY: queue_capacity
 * requests outstanding, or stream_queue_capacity of this stream (back-pressure:
 * wait for one of the stream's tickets, then submit again). */
ttnn_status ttnn_server_submit(ttnn_server_t server, int32_t stream_id, const void* data,
                               const int64_t* offset, const int64_t* extent,
                               const float* tile_scale, double lambda, uint64_t* ticket);
/* Queues ttnn_recover of the stream into `cores` (device, core_elems). */
ttnn_status ttnn_server_recover(ttnn_server_t server, int32_t stream_id, double* cores,
                                uint64_t* ticket);
/* Waits at most timeout_us for a ticket: TTNN_OK with *result = the
 * request's status (a failed request's message via ttnn_last_error), or
 * ETIMEOUT (ticket still pending; wait again).  A finished ticket is
 * reported once.  EINVAL: unknown ticket. */
ttnn_status ttnn_server_wait(ttnn_server_t server, uint64_t ticket, int64_t timeout_us,
                             ttnn_status* result);
/* The stream's state (read it only when its tickets are done). */
ttnn_status ttnn_server_stream_state(ttnn_server_t server, int32_t stream_id,
                                     ttnn_state_t* state);
/* Statistics since the last reset (reset != 0 restarts them). */
ttnn_status ttnn_server_stats(ttnn_server_t server, int32_t reset, ttnn_server_report* out);

#ifdef __cplusplus
}
#endif

#endif /* TTNN_H */
