// ttnn_update_dense_static: the dense update of ttnn_update_dense with its
// scratch (pass products, box DRM blocks, walk temporaries) in a fixed block
// of static device memory instead of the plan's workspace.
//
// Why: a caller that must not allocate device memory while it streams
// updates -- one whose memory is handed out by its own pool and must not
// grow behind its back, or one that must not let cudaMalloc / cudaFree
// synchronise the device in the middle of its stream work -- can still
// feed tensors in.  The call itself allocates no device memory: no
// cudaMalloc, no cudaFree, no allocating library routine.
//
// Limits and rules:
//  - One update may use at most kStaticScratchBytes (32 MiB) of scratch;
//    a larger request is rejected with TTNN_EINVAL before any work is
//    enqueued.
//  - The scratch is one block per device and per process: calls that
//    overlap in time (other host threads, or work still running on another
//    stream) race on it and give wrong results.  Serialise them.
//  - The block's address is looked up on the first call made with a device
//    current, and again whenever that device's current CUDA context has
//    changed since (e.g. after cudaDeviceReset); make the first call before
//    any stream capture begins.
//  - The block is device memory of the library's module: once the module is
//    loaded on a device (at the first call here, or at context creation under
//    CUDA_MODULE_LOADING=EAGER) the 32 MiB stay resident there until the
//    process exits, whether or not this entry point is ever called.
//  - Nothing in the scratch has to start at zero: every buffer an update
//    uses is written in full before it is read.
//  - Profiling intervals are not recorded by this call.
#include <mutex>

#include "plan.cuh"

namespace ttnn {

static constexpr int64_t kStaticScratchBytes = 32ll << 20;
static constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[kMaxDevices] = {nullptr};
static void* g_static_ctx[kMaxDevices] = {nullptr};

typedef int (*CtxGetCurrentFn)(void**);

// The current CUDA context (driver API cuCtxGetCurrent, reached through the
// runtime's entry-point query so that no driver library is linked).
static ttnn_status current_context(void** ctx) {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !ptr) {
      cudaGetLastError();
      set_error("static scratch: cuCtxGetCurrent unavailable");
      return TTNN_ECUDA;
    }
    fn = (CtxGetCurrentFn)ptr;
  }
  *ctx = nullptr;
  if (fn(ctx) != 0) {
    set_error("static scratch: cuCtxGetCurrent failed");
    return TTNN_ECUDA;
  }
  return TTNN_OK;
}

// Device address of g_static_scratch in the current device's context, looked
// up again when the context is not the one the cached address belongs to.
static ttnn_status static_scratch(void** out) {
  int dev = 0;
  TTNN_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("static scratch: device %d outside the %d supported", dev, kMaxDevices);
    return TTNN_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  void* ctx = nullptr;
  if (g_static_addr[dev]) TTNN_TRY(current_context(&ctx));
  if (!g_static_addr[dev] || ctx != g_static_ctx[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
                cudaGetErrorString(e));
      return TTNN_ECUDA;
    }
    // the symbol lookup made the primary context current if none was
    TTNN_TRY(current_context(&ctx));
    g_static_addr[dev] = p;
    g_static_ctx[dev] = ctx;
  }
  *out = g_static_addr[dev];
  return TTNN_OK;
}

int64_t static_scratch_resident_bytes() { return kStaticScratchBytes; }

}  // namespace ttnn

using namespace ttnn;

extern "C" {

ttnn_status ttnn_update_dense_static(ttnn_state_t S, const void* data, const int64_t* offset,
                                     const int64_t* extent, const float* tile_scale,
                                     double lambda, void* stream) {
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
  const cudaStream_t st = (cudaStream_t)stream;
  // the scratch this update needs (recorded once per box shape, then cached)
  int64_t need = 0;
  TTNN_TRY(dense_update_need(P, b, &need));
  TTNN_CHECK_ARG(need <= kStaticScratchBytes,
                 "this update needs %lld bytes of scratch; ttnn_update_dense_static has %lld "
                 "(use ttnn_update_dense or a smaller box)",
                 (long long)need, (long long)kStaticScratchBytes);
  void* scratch = nullptr;
  TTNN_TRY(static_scratch(&scratch));
  char* const ws0 = P.ws;
  const int64_t wb0 = P.ws_bytes;
  const int prof0 = P.profile;
  P.ws = (char*)scratch;
  P.ws_bytes = kStaticScratchBytes;
  P.profile = 0;
  const ttnn_status s = run_dense_update(P, S->acc, data, b, tile_scale, lambda, st, false, nullptr);
  P.ws = ws0;
  P.ws_bytes = wb0;
  P.profile = prof0;
  return s;
}

}  // extern "C"
