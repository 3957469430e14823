// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ttnn.h"

namespace ttnn {

// --- error reporting ------------------------------------------------------
void set_error(const char* fmt, ...);
const char* last_error();

#define TTNN_TRY_CUDA(call)                                                   \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::ttnn::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                  \
      return TTNN_ECUDA;                                                      \
    }                                                                         \
  } while (0)

#define TTNN_TRY(expr)                 \
  do {                                 \
    ttnn_status s_ = (expr);           \
    if (s_ != TTNN_OK) return s_;      \
  } while (0)

#define TTNN_CHECK_ARG(cond, ...)                 \
  do {                                            \
    if (!(cond)) {                                \
      ::ttnn::set_error(__VA_ARGS__);             \
      return TTNN_EINVAL;                         \
    }                                             \
  } while (0)

ttnn_status check_launch(const char* what);   // also counts the launch
void count_launch();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// number formats of the DRM rounding (index = ttnn_dtype for F64..E4M3)
enum RoundFmt { RF_F64 = 0, RF_F32 = 1, RF_BF16 = 2, RF_E4M3 = 3 };

}  // namespace ttnn
