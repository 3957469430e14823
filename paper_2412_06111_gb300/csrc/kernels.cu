// Generic device kernels: DRM generation, pass-side Khatri-Rao blocks, the
// strided contraction used by the tree walk and the core assembly, the SIMT
// GEMM of the binary64 / binary32 first-level pass, and small helpers.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "kernels.cuh"
#include "philox.cuh"

namespace ttnn {

static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }

ttnn_status check_launch(const char* what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return TTNN_ECUDA;
  }
  return TTNN_OK;
}

// ---------------------------------------------------------------------------
// DRM generation
// ---------------------------------------------------------------------------
__global__ void philox_kernel(uint64_t seed, uint32_t kind, uint32_t ident, int64_t rows,
                              int64_t cols, int fmt, double* dst) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    dst[e] = round_fmt(philox_gaussian(seed, kind, ident, (uint64_t)i, (uint64_t)j), fmt);
  }
}

ttnn_status launch_philox(uint64_t seed, int kind, int ident, int64_t rows, int64_t cols,
                          int fmt, double* dst, cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n == 0) return TTNN_OK;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, threads), 65535);
  philox_kernel<<<(unsigned)blocks, threads, 0, st>>>(seed, (uint32_t)kind, (uint32_t)ident, rows,
                                                      cols, fmt, dst);
  return check_launch("philox_kernel");
}

__global__ void convert_kernel(const double* src, float* dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

ttnn_status launch_convert_f64_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), 65535);
  convert_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n);
  return check_launch("convert_kernel");
}

// Several binary64 -> binary32 copies in one launch: block b converts
// kConvBlock consecutive elements of the segment whose block range holds b,
// two per load (16-byte loads, 8-byte stores) when the segment's ends allow.
constexpr int kConvBlock = 2048;

__global__ void convert_batch_kernel(const __grid_constant__ ConvertBatch b) {
  int lo = 0, hi = b.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (b.start[mid] <= (int64_t)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const double* src = b.src[lo];
  float* dst = b.dst[lo];
  const int64_t n = b.n[lo];
  const int64_t e0 = ((int64_t)blockIdx.x - b.start[lo]) * kConvBlock;
  const int64_t e1 = e0 + kConvBlock < n ? e0 + kConvBlock : n;
  if (b.pairs[lo]) {
    // e0 is even and both pointers are aligned for pairs
    for (int64_t e = e0 + 2 * threadIdx.x; e < e1; e += 2 * blockDim.x) {
      if (e + 1 < e1) {
        const double2 v = *reinterpret_cast<const double2*>(src + e);
        *reinterpret_cast<float2*>(dst + e) = make_float2((float)v.x, (float)v.y);
      } else {
        dst[e] = (float)src[e];
      }
    }
  } else {
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) dst[e] = (float)src[e];
  }
}

ttnn_status launch_convert_batch(const ConvertBatch& batch, cudaStream_t st) {
  if (batch.count <= 0 || batch.count > kConvertSegs) {
    set_error("internal: conversion batch of %d segments", batch.count);
    return TTNN_EUNSUPPORTED;
  }
  ConvertBatch b = batch;
  int64_t blocks = 0;
  for (int k = 0; k < b.count; ++k) {
    b.start[k] = blocks;
    b.pairs[k] = ((uintptr_t)b.src[k] % 16 == 0) && ((uintptr_t)b.dst[k] % 8 == 0);
    blocks += ceil_div(b.n[k], (int64_t)kConvBlock);
  }
  if (blocks == 0) return TTNN_OK;
  if (blocks >= (int64_t(1) << 31)) {
    set_error("conversion batch too large");
    return TTNN_EUNSUPPORTED;
  }
  convert_batch_kernel<<<(unsigned)blocks, 256, 0, st>>>(b);
  return check_launch("convert_batch_kernel");
}

// ---------------------------------------------------------------------------
// pass-side Khatri-Rao blocks
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_fmt(void* out, int64_t idx, double v, int store) {
  switch (store) {
    case 0: ((double*)out)[idx] = v; break;
    case 1: ((float*)out)[idx] = (float)v; break;
    case 2: {
      // v is already a bfloat16 value: its binary32 image has 16 zero low bits
      const uint32_t b = __float_as_uint((float)v);
      ((uint16_t*)out)[idx] = (uint16_t)(b >> 16);
      break;
    }
    default: {
      __nv_fp8_e4m3 q((float)v);  // exact: v is an E4M3 value
      ((uint8_t*)out)[idx] = q.__x;
      break;
    }
  }
}

__global__ void side_kernel(SideSpec s, void* out) {
  int64_t rows = 1;
  for (int m = 0; m < s.nmodes; ++m) rows *= s.ext[m];
  const int64_t n = rows * s.total_cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, row = e - c * rows;
    double v = 0.0;
    if (c < s.x_cols + s.y_cols) {
      // decompose the row index (row-major over the side's modes)
      int64_t idx[8];
      int64_t rem = row;
      for (int m = s.nmodes - 1; m >= 0; --m) {
        idx[m] = rem % s.ext[m];
        rem /= s.ext[m];
      }
      if (c < s.x_cols) {
        v = s.xf[0][(s.off[0] + idx[0]) * s.rmax + c];
        for (int m = 1; m < s.nmodes; ++m) v = __dmul_rn(v, s.xf[m][(s.off[m] + idx[m]) * s.rmax + c]);
      } else if (s.y_kind == 0) {
        const int64_t cc = c - s.x_cols;
        v = s.yf[0][(s.off[0] + idx[0]) * s.smax + cc];
        for (int m = 1; m < s.nmodes; ++m) v = __dmul_rn(v, s.yf[m][(s.off[m] + idx[m]) * s.smax + cc]);
      } else {
        int64_t flat = 0;
        for (int m = 0; m < s.nmodes; ++m) flat = flat * s.full[m] + (s.off[m] + idx[m]);
        v = (flat == c - s.x_cols) ? 1.0 : 0.0;
      }
      v = round_fmt(v, s.round_fmt);
    }
    store_fmt(out, c * s.ld + row, v, s.store);
  }
}

template <typename T>
__global__ void side_gather_kernel(SideSpec s, const T* src, int64_t src_ld, T* out) {
  int64_t rows = 1;
  for (int m = 0; m < s.nmodes; ++m) rows *= s.ext[m];
  const int64_t n = rows * s.total_cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, row = e - c * rows;
    int64_t rem = row, full = 0, stride = 1;
    for (int m = s.nmodes - 1; m >= 0; --m) {
      const int64_t i = rem % s.ext[m];
      rem /= s.ext[m];
      full += (s.off[m] + i) * stride;
      stride *= s.full[m];
    }
    out[c * s.ld + row] = src[c * src_ld + full];
  }
}

ttnn_status launch_side_gather(const SideSpec& s, const void* src, int64_t src_ld, void* out,
                               cudaStream_t st) {
  int64_t rows = 1;
  for (int m = 0; m < s.nmodes; ++m) rows *= s.ext[m];
  const int64_t n = rows * s.total_cols;
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), 65535);
  switch (s.store) {
    case 0:
      side_gather_kernel<uint64_t><<<(unsigned)blocks, 256, 0, st>>>(s, (const uint64_t*)src, src_ld,
                                                                     (uint64_t*)out);
      break;
    case 1:
      side_gather_kernel<uint32_t><<<(unsigned)blocks, 256, 0, st>>>(s, (const uint32_t*)src, src_ld,
                                                                     (uint32_t*)out);
      break;
    case 2:
      side_gather_kernel<uint16_t><<<(unsigned)blocks, 256, 0, st>>>(s, (const uint16_t*)src, src_ld,
                                                                     (uint16_t*)out);
      break;
    default:
      side_gather_kernel<uint8_t><<<(unsigned)blocks, 256, 0, st>>>(s, (const uint8_t*)src, src_ld,
                                                                    (uint8_t*)out);
      break;
  }
  return check_launch("side_gather_kernel");
}

constexpr int kGatherJobs = 32;
struct GatherBatch {
  int n;
  int64_t start[kGatherJobs + 1];   // prefix sums of blocks
  GatherJob jobs[kGatherJobs];
};

template <typename T>
__device__ void gather_rows(const GatherJob& g, int64_t e) {
  const SideSpec& s = g.s;
  int64_t rows = 1;
  for (int m = 0; m < s.nmodes; ++m) rows *= s.ext[m];
  if (e >= rows * s.total_cols) return;
  const int64_t c = e / rows, row = e - c * rows;
  int64_t rem = row, full = 0, stride = 1;
  for (int m = s.nmodes - 1; m >= 0; --m) {
    const int64_t i = rem % s.ext[m];
    rem /= s.ext[m];
    full += (s.off[m] + i) * stride;
    stride *= s.full[m];
  }
  ((T*)g.out)[c * s.ld + row] = ((const T*)g.src)[c * g.src_ld + full];
}

__global__ void side_gather_batch_kernel(const __grid_constant__ GatherBatch b) {
  const int64_t blk = blockIdx.x;
  int lo = 0, hi = b.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (b.start[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const GatherJob& g = b.jobs[lo];
  const int64_t e = (blk - b.start[lo]) * blockDim.x + threadIdx.x;
  switch (g.s.store) {
    case 0: gather_rows<uint64_t>(g, e); break;
    case 1: gather_rows<uint32_t>(g, e); break;
    case 2: gather_rows<uint16_t>(g, e); break;
    default: gather_rows<uint8_t>(g, e); break;
  }
}

ttnn_status launch_side_gather_batch(const GatherJob* jobs, int n, cudaStream_t st) {
  for (int j0 = 0; j0 < n; j0 += kGatherJobs) {
    GatherBatch b;
    b.n = 0;
    b.start[0] = 0;
    for (int j = j0; j < n && b.n < kGatherJobs; ++j) {
      int64_t rows = 1;
      for (int m = 0; m < jobs[j].s.nmodes; ++m) rows *= jobs[j].s.ext[m];
      const int64_t blocks = ceil_div(rows * jobs[j].s.total_cols, 256);
      if (blocks == 0) continue;
      b.jobs[b.n] = jobs[j];
      b.start[b.n + 1] = b.start[b.n] + blocks;
      ++b.n;
    }
    if (b.n == 0) continue;
    if (b.start[b.n] >= (int64_t(1) << 31)) {
      set_error("side gather batch too large");
      return TTNN_EUNSUPPORTED;
    }
    side_gather_batch_kernel<<<(unsigned)b.start[b.n], 256, 0, st>>>(b);
    TTNN_TRY(check_launch("side_gather_batch_kernel"));
  }
  return TTNN_OK;
}

// ---------------------------------------------------------------------------
// rank-one pass: a box whose other side is a single index
// ---------------------------------------------------------------------------
__device__ __forceinline__ float load_acc(const uint16_t* p, int64_t i, float) {
  return __uint_as_float((uint32_t)p[i] << 16);   // bfloat16 -> binary32, exact
}
__device__ __forceinline__ float load_acc(const float* p, int64_t i, float) { return p[i]; }
__device__ __forceinline__ double load_acc(const double* p, int64_t i, double) { return p[i]; }

constexpr int kGemvCols = 8;

// The value the passes sketch for element `i` of the box's rows, per format:
// plain (f64 / f32 / bf16), BF16x2 (hi + lo with hi = bf16(x), lo = bf16(x -
// hi)) or E4M3 (bf16(f32(q) * s), s the binary32 scale of the element's 128-
// element tile of these rows).
enum { RV_PLAIN = 0, RV_SPLIT = 1, RV_FP8 = 2 };
template <int MODE, typename Tm, typename Tacc>
__device__ __forceinline__ Tacc row_value(const Tm* m, int64_t i, const float* scale) {
  if constexpr (MODE == RV_SPLIT) {
    const float x = ((const float*)m)[i];
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    const float l = __bfloat162float(__float2bfloat16_rn(x - h));
    return (Tacc)(h + l);
  } else if constexpr (MODE == RV_FP8) {
    __nv_fp8_e4m3 q;
    q.__x = ((const uint8_t*)m)[i];
    const float v = __fmul_rn(static_cast<float>(q), scale[i >> 7]);
    return (Tacc)__bfloat162float(__float2bfloat16_rn(v));
  } else {
    return load_acc(m, i, Tacc(0));
  }
}

template <typename Tm, typename Ts, typename Tacc, int MODE = RV_PLAIN>
__global__ void __launch_bounds__(256) side_gemv_kernel(SideSpec s, const Ts* src, int64_t src_ld,
                                                        int cut, const Tm* m, int64_t rows,
                                                        int cols, int64_t rpb, Tacc* part,
                                                        const float* scale) {
  __shared__ Tacc red[8][kGemvCols];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = r0 + rpb < rows ? r0 + rpb : rows;
  for (int c0 = 0; c0 < cols; c0 += kGemvCols) {
    Tacc acc[kGemvCols];
#pragma unroll
    for (int k = 0; k < kGemvCols; ++k) acc[k] = 0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
      int64_t f = row;
      if (cut) {
        int64_t rem = row, stride = 1;
        f = 0;
        for (int mm = s.nmodes - 1; mm >= 0; --mm) {
          const int64_t i = rem % s.ext[mm];
          rem /= s.ext[mm];
          f += (s.off[mm] + i) * stride;
          stride *= s.full[mm];
        }
      }
      const Tacc mv = row_value<MODE, Tm, Tacc>(m, row, scale);
#pragma unroll
      for (int k = 0; k < kGemvCols; ++k)
        if (c0 + k < cols) acc[k] += mv * load_acc(src, (int64_t)(c0 + k) * src_ld + f, Tacc(0));
    }
#pragma unroll
    for (int k = 0; k < kGemvCols; ++k) {
      Tacc v = acc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kGemvCols && c0 + (int)threadIdx.x < cols) {
      Tacc t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
      part[(int64_t)blockIdx.x * cols + c0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

template <typename Tacc>
__global__ void gemv_reduce_kernel(const Tacc* part, int nblk, int cols, int cols_pad, Tacc* D) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols_pad; c += gridDim.x * blockDim.x) {
    Tacc t = 0;
    if (c < cols)
      for (int b = 0; b < nblk; ++b) t += part[(int64_t)b * cols + c];
    D[c] = t;
  }
}

ttnn_status launch_side_gemv(const SideSpec& s, const void* src, int64_t src_ld, bool cut,
                             const void* m, int m_store, const float* scale, int64_t rows,
                             int cols, int cols_pad, void* D, int d_f64, void* part,
                             int64_t part_bytes, cudaStream_t st, bool dry, int64_t* need) {
  const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 1024), (int64_t)num_sms() * 4));
  const int64_t rpb = ceil_div(rows, nblk);
  const int64_t bytes = nblk * std::max(cols, 1) * (d_f64 ? 8 : 4);
  if (dry) {
    if (need) *need = bytes;
    return TTNN_OK;
  }
  if (part_bytes < bytes) {
    set_error("rank-one pass: scratch too small");
    return TTNN_ENOMEM;
  }
  if (cols_pad == 0) return TTNN_OK;
  if (d_f64) {
    if (m_store != 0 || s.store != 0) {
      set_error("rank-one pass: unsupported formats");
      return TTNN_EUNSUPPORTED;
    }
    if (cols > 0)
      side_gemv_kernel<double, double, double><<<(unsigned)nblk, 256, 0, st>>>(
          s, (const double*)src, src_ld, cut ? 1 : 0, (const double*)m, rows, cols, rpb,
          (double*)part, scale);
  } else if (m_store == 1 && s.store == 1) {
    if (cols > 0)
      side_gemv_kernel<float, float, float><<<(unsigned)nblk, 256, 0, st>>>(
          s, (const float*)src, src_ld, cut ? 1 : 0, (const float*)m, rows, cols, rpb,
          (float*)part, scale);
  } else if (m_store == 2 && s.store == 2) {
    if (cols > 0)
      side_gemv_kernel<uint16_t, uint16_t, float><<<(unsigned)nblk, 256, 0, st>>>(
          s, (const uint16_t*)src, src_ld, cut ? 1 : 0, (const uint16_t*)m, rows, cols, rpb,
          (float*)part, scale);
  } else if (m_store == kStoreSplit && s.store == 2) {
    if (cols > 0)
      side_gemv_kernel<float, uint16_t, float, RV_SPLIT><<<(unsigned)nblk, 256, 0, st>>>(
          s, (const uint16_t*)src, src_ld, cut ? 1 : 0, (const float*)m, rows, cols, rpb,
          (float*)part, scale);
  } else if (m_store == kStoreFp8 && s.store == 2 && scale) {
    if (cols > 0)
      side_gemv_kernel<uint8_t, uint16_t, float, RV_FP8><<<(unsigned)nblk, 256, 0, st>>>(
          s, (const uint16_t*)src, src_ld, cut ? 1 : 0, (const uint8_t*)m, rows, cols, rpb,
          (float*)part, scale);
  } else {
    set_error("rank-one pass: unsupported formats");
    return TTNN_EUNSUPPORTED;
  }
  if (cols > 0) TTNN_TRY(check_launch("side_gemv_kernel"));
  const unsigned rb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cols_pad, 256), 64));
  if (d_f64) gemv_reduce_kernel<double><<<rb, 256, 0, st>>>((const double*)part, (int)nblk, cols, cols_pad, (double*)D);
  else gemv_reduce_kernel<float><<<rb, 256, 0, st>>>((const float*)part, (int)nblk, cols, cols_pad, (float*)D);
  return check_launch("gemv_reduce_kernel");
}

template <typename Ts, typename Td, int MODE = RV_PLAIN>
__global__ void to_walk_kernel(const Ts* src, Td* dst, int64_t n, const float* scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = row_value<MODE, Ts, Td>(src, e, scale);
}

ttnn_status launch_to_walk(const void* src, int src_store, const float* scale, void* dst,
                           int d_f64, int64_t n, cudaStream_t st) {
  if (n == 0) return TTNN_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8);
  if (!d_f64 && src_store == 2)
    to_walk_kernel<uint16_t, float><<<blocks, 256, 0, st>>>((const uint16_t*)src, (float*)dst, n, scale);
  else if (!d_f64 && src_store == 1)
    to_walk_kernel<float, float><<<blocks, 256, 0, st>>>((const float*)src, (float*)dst, n, scale);
  else if (d_f64 && src_store == 0)
    to_walk_kernel<double, double><<<blocks, 256, 0, st>>>((const double*)src, (double*)dst, n, scale);
  else if (!d_f64 && src_store == kStoreSplit)
    to_walk_kernel<float, float, RV_SPLIT><<<blocks, 256, 0, st>>>((const float*)src, (float*)dst, n, scale);
  else if (!d_f64 && src_store == kStoreFp8 && scale)
    to_walk_kernel<uint8_t, float, RV_FP8><<<blocks, 256, 0, st>>>((const uint8_t*)src, (float*)dst, n, scale);
  else {
    set_error("walk copy: unsupported formats");
    return TTNN_EUNSUPPORTED;
  }
  return check_launch("to_walk_kernel");
}

ttnn_status launch_side(const SideSpec& s, void* out, cudaStream_t st) {
  int64_t rows = 1;
  for (int m = 0; m < s.nmodes; ++m) rows *= s.ext[m];
  const int64_t n = rows * s.total_cols;
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), 65535);
  side_kernel<<<(unsigned)blocks, 256, 0, st>>>(s, out);
  return check_launch("side_kernel");
}

// ---------------------------------------------------------------------------
// strided contraction
// ---------------------------------------------------------------------------
template <typename Tin, typename Tw, typename Tout, typename Tacc>
__global__ void contract_kernel(Contract c, int nsplit, int64_t chunk, Tout* partial) {
  const int64_t total = c.P * c.NB * c.Q * c.J;
  const Tin* in = (const Tin*)c.in;
  const Tw* w = (const Tw*)c.w;
  Tout* out = (Tout*)c.out;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total * nsplit;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t split = e / total, o = e - split * total;
    int64_t t = o;
    const int64_t j = t % c.J;
    t /= c.J;
    const int64_t q = t % c.Q;
    t /= c.Q;
    const int64_t b = t % c.NB;
    const int64_t p = t / c.NB;
    const int64_t i0 = split * chunk;
    const int64_t i1 = min(c.NI, i0 + chunk);
    const Tin* ip = in + p * c.isP + q * c.isQ + j * c.isJ;
    Tacc acc = 0;
    if (w) {
      const Tw* wp = w + b * c.wsB + q * c.wsQ + j * c.wsJ;
      for (int64_t i = i0; i < i1; ++i) acc += (Tacc)ip[i * c.isI] * (Tacc)wp[i * c.wsI];
    } else {
      for (int64_t i = i0; i < i1; ++i) acc += (Tacc)ip[i * c.isI];
    }
    if (nsplit > 1) {
      partial[split * total + o] = (Tout)acc;
    } else {
      const int64_t oi = p * c.osP + b * c.osB + q * c.osQ + j * c.osJ;
      const Tout v = (Tout)((Tacc)c.alpha * acc);
      out[oi] = c.accumulate ? (Tout)(out[oi] + v) : v;
    }
  }
}

template <typename Tout>
__global__ void contract_reduce_kernel(Contract c, int nsplit, const Tout* partial) {
  const int64_t total = c.P * c.NB * c.Q * c.J;
  Tout* out = (Tout*)c.out;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    Tout acc = 0;
    for (int s = 0; s < nsplit; ++s) acc += partial[s * total + o];
    int64_t t = o;
    const int64_t j = t % c.J;
    t /= c.J;
    const int64_t q = t % c.Q;
    t /= c.Q;
    const int64_t b = t % c.NB;
    const int64_t p = t / c.NB;
    const int64_t oi = p * c.osP + b * c.osB + q * c.osQ + j * c.osJ;
    const Tout v = (Tout)(c.alpha * acc);
    out[oi] = c.accumulate ? (Tout)(out[oi] + v) : v;
  }
}

static void contract_split(const Contract& c, int* nsplit, int64_t* chunk) {
  const int64_t total = c.P * c.NB * c.Q * c.J;
  const int64_t target = (int64_t)num_sms() * 2048;
  int ns = 1;
  if (c.NI >= 256 && total < target) {
    ns = (int)std::min<int64_t>(std::min<int64_t>(ceil_div(target, std::max<int64_t>(total, 1)),
                                                  c.NI / 64),
                                256);
    ns = std::max(ns, 1);
  }
  *chunk = ceil_div(c.NI, ns);
  *nsplit = (int)ceil_div(c.NI, *chunk);
  if (*nsplit < 1) *nsplit = 1;
}

int64_t contract_partial_elems(const Contract& c) {
  int ns;
  int64_t chunk;
  contract_split(c, &ns, &chunk);
  return ns > 1 ? ns * c.P * c.NB * c.Q * c.J : 0;
}

// Mode product as a batched small GEMM: for every batch item (p, q),
// out[p,b,q,j] (+)= alpha * sum_i W[i*wsI + b*wsB] * in[p,i,q,j].  W is staged
// in shared memory once per K chunk; each thread owns a 4 x 4 tile of
// (b, column) outputs, where the columns are the (item, j) pairs of CH items.
constexpr int kMpKC = 32;

template <typename T>
__global__ void __launch_bounds__(256) mp_kernel(Contract c, int BG, int CG, int CH) {
  extern __shared__ __align__(16) unsigned char mp_smem[];
  T* Ws = (T*)mp_smem;                 // [kMpKC][4*BG]
  T* Is = Ws + kMpKC * 4 * BG;         // [kMpKC][4*CG]
  const T* in = (const T*)c.in;
  const T* w = (const T*)c.w;
  T* out = (T*)c.out;
  const int tid = threadIdx.x;
  const int bg = tid / CG, cg = tid % CG;
  const int ncol = CH * (int)c.J;
  const int64_t items = c.P * c.Q;
  const int WB = 4 * BG, WC = 4 * CG;
  for (int64_t it0 = (int64_t)blockIdx.x * CH; it0 < items; it0 += (int64_t)gridDim.x * CH) {
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0;
    for (int64_t i0 = 0; i0 < c.NI; i0 += kMpKC) {
      const int kc = (int)min((int64_t)kMpKC, c.NI - i0);
      __syncthreads();
      for (int e = tid; e < kc * WB; e += 256) {
        const int ii = e / WB, b = e % WB;
        Ws[ii * WB + b] = (b < c.NB) ? w[(i0 + ii) * c.wsI + b * c.wsB] : (T)0;
      }
      for (int e = tid; e < kc * WC; e += 256) {
        const int ii = e / WC, col = e % WC;
        T v = 0;
        if (col < ncol) {
          const int64_t item = it0 + col / c.J;
          if (item < items) {
            const int64_t j = col % c.J;
            const int64_t p = item / c.Q, q = item % c.Q;
            v = in[p * c.isP + (i0 + ii) * c.isI + q * c.isQ + j * c.isJ];
          }
        }
        Is[ii * WC + col] = v;
      }
      __syncthreads();
      if (bg < BG) {
        for (int ii = 0; ii < kc; ++ii) {
          T a[4], b[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            a[x] = Ws[ii * WB + 4 * bg + x];
            b[x] = Is[ii * WC + 4 * cg + x];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
        }
      }
    }
    if (bg < BG) {
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int col = 4 * cg + y;
        if (col >= ncol) continue;
        const int64_t item = it0 + col / c.J;
        if (item >= items) continue;
        const int64_t j = col % c.J;
        const int64_t p = item / c.Q, q = item % c.Q;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int b = 4 * bg + x;
          if (b >= c.NB) continue;
          const int64_t oi = p * c.osP + b * c.osB + q * c.osQ + j * c.osJ;
          const T v = (T)c.alpha * acc[x][y];
          out[oi] = c.accumulate ? out[oi] + v : v;
        }
      }
    }
  }
}

// Shapes the batched kernel takes: W independent of q and j, enough work.
static bool mp_shape(const Contract& c, int elem_bytes, int* BG, int* CG, int* CH) {
  if (!c.w || c.wsQ != 0 || c.wsJ != 0 || c.NI < 8 || c.NB > 64) return false;
  int bg = (int)((c.NB + 3) / 4);
  int p2 = 1;
  while (p2 < bg) p2 <<= 1;
  // shared memory kMpKC * 4 * (BG + CG) elements stays within 48 KB
  const int cg = std::min(256 / p2, elem_bytes == 8 ? 32 : 64);
  if (c.J > 4 * cg) return false;
  const int ch = (int)(4 * cg / c.J);
  if (c.P * c.Q * c.NB * c.J < 4096) return false;
  *BG = p2;
  *CG = cg;
  *CH = ch;
  return true;
}

template <typename Tin, typename Tw, typename Tout, typename Tacc>
static ttnn_status run_contract(const Contract& c, void* partial, int64_t partial_elems,
                                cudaStream_t st) {
  const int64_t total = c.P * c.NB * c.Q * c.J;
  if (total == 0) return TTNN_OK;
  int BG, CG, CH;
  if (std::is_same<Tin, Tw>::value && std::is_same<Tin, Tout>::value && mp_shape(c, (int)sizeof(Tin), &BG, &CG, &CH)) {
    const size_t smem = (size_t)kMpKC * 4 * (BG + CG) * sizeof(Tin);
    const int64_t items = c.P * c.Q;
    const int64_t blocks = std::min<int64_t>(ceil_div(items, CH), (int64_t)num_sms() * 8);
    mp_kernel<Tin><<<(unsigned)blocks, 256, smem, st>>>(c, BG, CG, CH);
    return check_launch("mp_kernel");
  }
  int ns;
  int64_t chunk;
  contract_split(c, &ns, &chunk);
  if (ns > 1 && (partial == nullptr || partial_elems < ns * total)) {
    ns = 1;
    chunk = c.NI;
  }
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>(ceil_div(total * ns, threads), (int64_t)num_sms() * 32);
  contract_kernel<Tin, Tw, Tout, Tacc><<<(unsigned)blocks, threads, 0, st>>>(c, ns, chunk, (Tout*)partial);
  TTNN_TRY(check_launch("contract_kernel"));
  if (ns > 1) {
    const int64_t b2 = std::min<int64_t>(ceil_div(total, threads), (int64_t)num_sms() * 32);
    contract_reduce_kernel<Tout><<<(unsigned)b2, threads, 0, st>>>(c, ns, (const Tout*)partial);
    TTNN_TRY(check_launch("contract_reduce_kernel"));
  }
  return TTNN_OK;
}

ttnn_status launch_contract(const Contract& c, ElemType tin, ElemType tw, ElemType tout,
                            void* partial, int64_t partial_elems, cudaStream_t st) {
  if (tin == ET_F32 && tw == ET_F32 && tout == ET_F32)
    return run_contract<float, float, float, float>(c, partial, partial_elems, st);
  if (tin == ET_F64 && tw == ET_F64 && tout == ET_F64)
    return run_contract<double, double, double, double>(c, partial, partial_elems, st);
  if (tin == ET_F32 && tw == ET_F64 && tout == ET_F64)
    return run_contract<float, double, double, double>(c, partial, partial_elems, st);
  set_error("unsupported contraction type combination");
  return TTNN_EUNSUPPORTED;
}

// ---------------------------------------------------------------------------
// SIMT GEMM (binary64 / binary32 pass, and the BF16 fallback)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f32(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename Tin, typename Tacc>
__device__ __forceinline__ Tacc load_as(const Tin* p) { return (Tacc)to_f32(*p); }
template <>
__device__ __forceinline__ double load_as<double, double>(const double* p) { return *p; }

constexpr int GB_M = 128, GB_N = 64, GB_K = 16;
constexpr int GB_PAD = 4;   // keeps 16-byte rows for the vector reads

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float* v) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double* p, double* v) {
    const double2 x = reinterpret_cast<const double2*>(p)[0];
    const double2 y = reinterpret_cast<const double2*>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
};

// 256 threads; the output tile is 128 x BN (BN = 64, 32 or 16: the narrowest
// that holds the output columns, so narrow products compute no padding), each
// thread a (BN / 8) x 4 block of it.  The next k-tile's elements are fetched
// into registers while the current one is multiplied out of shared memory.
template <typename Tin, typename Tacc, int BN>
__global__ void __launch_bounds__(256) gemm_kernel(Gemm g, int nsplit, int64_t kchunk, Tacc* partial) {
  constexpr int TX = BN / 4;            // threads along the columns
  constexpr int TM = GB_M * TX / 256;   // rows per thread
  constexpr int BPT = BN * GB_K / 256;  // B-tile elements per thread
  __shared__ __align__(16) Tacc As[GB_K][GB_M + GB_PAD];
  __shared__ __align__(16) Tacc Bs[GB_K][BN + GB_PAD];
  const Tin* A = (const Tin*)g.A;
  const Tin* B = (const Tin*)g.B;
  const int tid = threadIdx.x;
  const int64_t i0 = blockIdx.x * (int64_t)GB_M;
  const int64_t j0 = blockIdx.y * (int64_t)BN;
  const int split = blockIdx.z;
  const int64_t kb = split * kchunk;
  const int64_t ke = min(g.K, kb + kchunk);
  const int ty = tid / TX, tx = tid % TX;   // output rows ty*TM.., cols tx*4..
  Tacc acc[TM][4];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  const bool a_k_contig = (g.ask == 1);
  const bool b_k_contig = (g.bsk == 1);
  // this thread's elements of a tile: A 128 x 16 (8 each), B BN x 16
  int aii[8], akk[8], bjj[BPT], bkk[BPT];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    const int e = tid + l * 256;
    if (a_k_contig) { aii[l] = e / GB_K; akk[l] = e % GB_K; }
    else { akk[l] = e / GB_M; aii[l] = e % GB_M; }
  }
#pragma unroll
  for (int l = 0; l < BPT; ++l) {
    const int e = tid + l * 256;
    if (b_k_contig) { bjj[l] = e / GB_K; bkk[l] = e % GB_K; }
    else { bkk[l] = e / BN; bjj[l] = e % BN; }
  }
  Tacc ra[8], rb[BPT];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int64_t gi = i0 + aii[l], gk = k0 + akk[l];
      ra[l] = (gi < g.I && gk < ke) ? load_as<Tin, Tacc>(A + gi * g.asi + gk * g.ask) : (Tacc)0;
    }
#pragma unroll
    for (int l = 0; l < BPT; ++l) {
      const int64_t gj = j0 + bjj[l], gk = k0 + bkk[l];
      rb[l] = (gj < g.Jn && gk < ke) ? load_as<Tin, Tacc>(B + gj * g.bsj + gk * g.bsk) : (Tacc)0;
    }
  };
  if (kb < ke) fetch(kb);
  for (int64_t k0 = kb; k0 < ke; k0 += GB_K) {
#pragma unroll
    for (int l = 0; l < 8; ++l) As[akk[l]][aii[l]] = ra[l];
#pragma unroll
    for (int l = 0; l < BPT; ++l) Bs[bkk[l]][bjj[l]] = rb[l];
    __syncthreads();
    if (k0 + GB_K < ke) fetch(k0 + GB_K);
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      Tacc a[TM], b[4];
      if (TM % 4 == 0) {
#pragma unroll
        for (int q = 0; q < TM / 4; ++q) Vec4<Tacc>::load(&As[kk][ty * TM + 4 * q], a + 4 * q);
      } else {
#pragma unroll
        for (int q = 0; q < TM; ++q) a[q] = As[kk][ty * TM + q];
      }
      Vec4<Tacc>::load(&Bs[kk][tx * 4], b);
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
  Tacc* C = nsplit > 1 ? partial + (int64_t)split * g.I * g.ldc : (Tacc*)g.C;
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int64_t gi = i0 + ty * TM + x;
    if (gi >= g.I) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gj = j0 + tx * 4 + y;
      if (gj < g.Jn) C[gi * g.ldc + gj] = acc[x][y];
    }
  }
}

// Column tile of a GEMM: the narrowest of 64 / 32 / 16 that holds Jn.
static int gemm_bn(const Gemm& g) { return g.Jn <= 16 ? 16 : g.Jn <= 32 ? 32 : GB_N; }

template <typename Tacc>
__global__ void gemm_reduce_kernel(Gemm g, int nsplit, const Tacc* partial) {
  const int64_t n = g.I * g.ldc;
  Tacc* C = (Tacc*)g.C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e % g.ldc >= g.Jn) continue;
    Tacc acc = 0;
    for (int s = 0; s < nsplit; ++s) acc += partial[(int64_t)s * n + e];
    C[e] = acc;
  }
}

int gemm_choose_split(const Gemm& g) {
  const int64_t tiles = ceil_div(g.I, GB_M) * ceil_div(g.Jn, (int64_t)gemm_bn(g));
  const int64_t want = (int64_t)num_sms() * 4;
  if (tiles >= want) return 1;
  int64_t ns = ceil_div(want, tiles);
  // reductions as short as 64 per split: small products spread over the
  // GPU (binary64 runs at a few DFMA per clock per SM)
  ns = std::min<int64_t>(ns, ceil_div(g.K, 64));
  return (int)std::max<int64_t>(1, std::min<int64_t>(ns, 512));
}

template <typename Tin, typename Tacc>
static ttnn_status run_gemm(const Gemm& g, int nsplit, void* partial, cudaStream_t st) {
  if (g.I == 0 || g.Jn == 0) return TTNN_OK;
  int64_t kchunk = round_up(ceil_div(g.K, nsplit), GB_K);
  nsplit = (int)ceil_div(g.K, kchunk);
  if (nsplit < 1) nsplit = 1;
  const int bn = gemm_bn(g);
  dim3 grid((unsigned)ceil_div(g.I, GB_M), (unsigned)ceil_div(g.Jn, (int64_t)bn), (unsigned)nsplit);
  if (grid.y > 65535 || grid.z > 65535) {
    set_error("gemm grid too large");
    return TTNN_EUNSUPPORTED;
  }
  if (bn == 16) gemm_kernel<Tin, Tacc, 16><<<grid, 256, 0, st>>>(g, nsplit, kchunk, (Tacc*)partial);
  else if (bn == 32) gemm_kernel<Tin, Tacc, 32><<<grid, 256, 0, st>>>(g, nsplit, kchunk, (Tacc*)partial);
  else gemm_kernel<Tin, Tacc, GB_N><<<grid, 256, 0, st>>>(g, nsplit, kchunk, (Tacc*)partial);
  TTNN_TRY(check_launch("gemm_kernel"));
  if (nsplit > 1) {
    const int64_t n = g.I * g.ldc;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 32);
    gemm_reduce_kernel<Tacc><<<(unsigned)blocks, 256, 0, st>>>(g, nsplit, (const Tacc*)partial);
    TTNN_TRY(check_launch("gemm_reduce_kernel"));
  }
  return TTNN_OK;
}

ttnn_status launch_gemm(const Gemm& g, int nsplit, void* partial, cudaStream_t st) {
  switch (g.in_type) {
    case 0: return run_gemm<double, double>(g, nsplit, partial, st);
    case 1: return run_gemm<float, float>(g, nsplit, partial, st);
    case 2: return run_gemm<__nv_bfloat16, float>(g, nsplit, partial, st);
    default: set_error("gemm: bad input type"); return TTNN_EINVAL;
  }
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
ttnn_status launch_fill_zero(void* p, int64_t bytes, cudaStream_t st) {
  if (bytes == 0) return TTNN_OK;
  TTNN_TRY_CUDA(cudaMemsetAsync(p, 0, (size_t)bytes, st));
  return TTNN_OK;
}

template <typename T>
__global__ void axpy_kernel(T* y, const T* x, double alpha, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (T)(y[e] + (T)alpha * x[e]);
}

ttnn_status launch_axpy(void* y, const void* x, double alpha, int64_t n, int is_f64, cudaStream_t st) {
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), 65535);
  if (is_f64) axpy_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((double*)y, (const double*)x, alpha, n);
  else axpy_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((float*)y, (const float*)x, alpha, n);
  return check_launch("axpy_kernel");
}

// block (node k, chunk): the padded core's entries whose indices all lie
// below the axes' kept extents, to their compact row-major positions.
__global__ void compact_cores_kernel(const __grid_constant__ CompactBatch b) {
  const CompactNode& nd = b.nd[blockIdx.y];
  int32_t keep[10];
  int64_t tot = 1;
  for (int a = 0; a < nd.ndim; ++a) {
    keep[a] = nd.job[a] >= 0 ? min(b.kept[nd.job[a]], nd.full[a]) : nd.full[a];
    tot *= nd.full[a];
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e, dst = 0, stride = 1;
    bool in = true;
    for (int a = nd.ndim - 1; a >= 0; --a) {
      const int64_t i = rem % nd.full[a];
      rem /= nd.full[a];
      if (i >= keep[a]) in = false;
      dst += i * stride;
      stride *= keep[a];
    }
    if (in) b.dst[nd.off + dst] = b.src[nd.off + e];
  }
}

ttnn_status launch_compact_cores(const CompactBatch& b, int64_t max_elems, cudaStream_t st) {
  if (b.n == 0) return TTNN_OK;
  const int64_t bx = std::min<int64_t>(std::max<int64_t>(ceil_div(max_elems, 256), 1), 1024);
  compact_cores_kernel<<<dim3((unsigned)bx, (unsigned)b.n, 1), 256, 0, st>>>(b);
  return check_launch("compact_cores_kernel");
}

__global__ void eye_kernel(double* dst, int64_t n) {
  const int64_t m = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (e / n == e % n) ? 1.0 : 0.0;
}

ttnn_status launch_eye(double* dst, int64_t n, cudaStream_t st) {
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>(ceil_div(n * n, 256), 65535);
  eye_kernel<<<(unsigned)blocks, 256, 0, st>>>(dst, n);
  return check_launch("eye_kernel");
}

}  // namespace ttnn
