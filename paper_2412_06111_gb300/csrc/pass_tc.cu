// Tensor-core (tcgen05) first-level pass: placeholder until the kernel lands.
#include "plan.cuh"

namespace ttnn {

ttnn_status tc_pass_supported(const ttnn_plan_s& P, int64_t nL, int64_t nR) {
  (void)P; (void)nL; (void)nR;
  return TTNN_EUNSUPPORTED;
}

ttnn_status launch_tc_pass(const ttnn_plan_s& P, const void* A, int64_t nL, int64_t nR,
                           const void* sR, int64_t ldR, const void* sL, int64_t ldL, void* D1,
                           void* D2, const float* tile_scale, void* ws, int64_t ws_bytes,
                           cudaStream_t st, bool dry, int64_t* ws_need) {
  (void)P; (void)A; (void)nL; (void)nR; (void)sR; (void)ldR; (void)sL; (void)ldL; (void)D1;
  (void)D2; (void)tile_scale; (void)ws; (void)ws_bytes; (void)st; (void)dry;
  if (ws_need) *ws_need = 0;
  set_error("tensor-core pass not available");
  return TTNN_EUNSUPPORTED;
}

}  // namespace ttnn
