// First-level pass for the narrow and split storage formats, on the bfloat16
// tcgen05 tensor cores (sm_103a).  Same products as the BF16 pass:
//   D1 = M B_R^T (nL x wR),  D2 = M^T B_L^T (nR x wL),
// but the tile of M arrives in its storage format and converter warps turn
// it into bfloat16 operand tiles in shared memory before the MMAs:
//
//  SPLIT (binary32 M): hi = bf16(M), lo = bf16(M - hi); both tiles are
//    multiplied by the same bfloat16 DRM tile and summed in the TMEM
//    accumulators (four MMA streams per tile).  The conversion is in place:
//    each 64-column half of the binary32 tile (32 KB) becomes its hi and lo
//    swizzled boxes (16 KB each) in the same bytes.
//  FP8 (E4M3 M with one binary32 scale per 128 x 128 tile): the tile is
//    dequantised to bf16(f32(q * s)) into a separate bfloat16 operand tile.
//
// Pipeline per stage: TMA (raw tile + DRM tile) -> converters (4 warps) ->
// MMA issuer -> stage free.  Warp roles (448 threads): warp 0 TMA producer,
// warp 1 TMEM owner + MMA issuer, warps 2-5 epilogue, warps 6-13 converters.
// Every wait is bounded (globaltimer); on expiry the kernel records an error
// bit, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "tc_ptx.cuh"

namespace ttnn {
namespace tc {

constexpr int kConvThreads = 256;   // converter warps 6..13
constexpr int kCvtThreads = 192 + kConvThreads;
constexpr int MODE_SPLIT = 1;
constexpr int MODE_FP8 = 2;
constexpr int MODE_SPLIT3 = 3;   // binary32 M and binary32 DRM blocks, both split
template <int MODE>
__host__ __device__ constexpr bool is_split() { return MODE == MODE_SPLIT || MODE == MODE_SPLIT3; }

struct CvtParams {
  int64_t nL, nR;
  int C, G, nb, tiles, stages;
  int wRpad, wLpad;
  int ncolt;             // column tiles of M (row stride of the scale array)
  const float* scale;    // FP8: [ceil(nL/128)][ncolt]
  float* D1;             // [nL][wRpad] (C == 1)
  float* D1p;            // [C][nb*128][wRpad] chunk partials (C > 1)
  int* cnt;              // [nb][4] chunk arrivals per row block and epilogue warp, zero at launch
  int discard;           // partial rows are whole 128-byte lines
  float* D2p;            // [G][C*tiles*128][wLpad]
  int* err;
};

template <int MODE>
struct Layout {
  // operand bytes (bf16 tiles the MMAs read), raw bytes kept apart from them
  static constexpr uint32_t op = is_split<MODE>() ? 65536u : 32768u;
  static constexpr uint32_t raw = is_split<MODE>() ? 0u : 16384u;
  // distance between the two 64-column boxes of one operand tile
  static constexpr uint32_t box = is_split<MODE>() ? 32768u : 16384u;
  // DRM blocks per stage / row block: bf16 (hi) or, SPLIT3, hi and lo
  static constexpr uint32_t bparts = MODE == MODE_SPLIT3 ? 2u : 1u;
};

__device__ __forceinline__ void named_sync_conv() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConvThreads) : "memory");
}
// AND of `ok` over the 128 converter threads (named barrier 1 with a
// reduction): every converter takes the same branch, so the named barriers
// of the in-place conversion are always reached by all of them.
__device__ __forceinline__ bool conv_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)ok), "n"(kConvThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // .x = a (low half)
  return *reinterpret_cast<const uint32_t*>(&v);
}

// SPLIT: one 64-column half (h) of the binary32 tile at `tile`, in place.
// Raw layout: [128 rows][64 floats] (256-byte rows).  Output: hi box at
// tile + h*32K, lo box at tile + h*32K + 16K, each [128 rows][64 bf16] with
// the 128-byte swizzle (16-byte chunk c of row y at chunk c ^ (y & 7)).
// Thread task: 4 consecutive floats of a row (16 lanes cover a row, so every
// shared-memory phase touches 128 contiguous bytes), giving 8 bytes of hi
// and 8 bytes of lo.
__device__ __forceinline__ void convert_split_half(uint8_t* tile, int h, int ct) {
  uint8_t* half = tile + h * 32768;
  constexpr int kTasks = 2048 / kConvThreads;
  float4 v[kTasks];
#pragma unroll
  for (int i = 0; i < kTasks; ++i) {
    const int id = i * kConvThreads + ct;
    v[i] = *reinterpret_cast<const float4*>(half + (id >> 4) * 256 + (id & 15) * 16);
  }
  named_sync_conv();   // every read of this half precedes every write into it
#pragma unroll
  for (int i = 0; i < kTasks; ++i) {
    const int id = i * kConvThreads + ct;
    const int y = id >> 4, q = id & 15;   // floats 4q..4q+3 of row y
    const float h0 = __bfloat162float(__float2bfloat16_rn(v[i].x));
    const float h1 = __bfloat162float(__float2bfloat16_rn(v[i].y));
    const float h2 = __bfloat162float(__float2bfloat16_rn(v[i].z));
    const float h3 = __bfloat162float(__float2bfloat16_rn(v[i].w));
    const uint2 hi = make_uint2(pack_bf16(h0, h1), pack_bf16(h2, h3));
    // the differences are exact in binary32
    const uint2 lo = make_uint2(pack_bf16(v[i].x - h0, v[i].y - h1),
                                pack_bf16(v[i].z - h2, v[i].w - h3));
    const uint32_t off = (uint32_t)(y * 128 + (((q >> 1) ^ (y & 7)) << 4) + (q & 1) * 8);
    *reinterpret_cast<uint2*>(half + off) = hi;
    *reinterpret_cast<uint2*>(half + 16384 + off) = lo;
  }
}

__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two) {
  __nv_fp8x2_e4m3 p;
  p.__x = (__nv_fp8x2_storage_t)two;
  return static_cast<float2>(p);   // exact: E4M3 values are binary32 values
}

// FP8: the [128][128] E4M3 tile at `raw` -> two bf16 boxes at `op`, op + 16K.
__device__ __forceinline__ void convert_fp8(const uint8_t* raw, uint8_t* op, float s, int ct) {
  constexpr int kTasks = 2048 / kConvThreads;
#pragma unroll
  for (int i = 0; i < kTasks; ++i) {
    const int id = i * kConvThreads + ct;
    const int y = id >> 4, c = id & 15;
    const uint2 q = *reinterpret_cast<const uint2*>(raw + y * 128 + c * 8);
    const float2 f0 = e4m3x2_to_float2(q.x & 0xFFFFu), f1 = e4m3x2_to_float2(q.x >> 16);
    const float2 f2 = e4m3x2_to_float2(q.y & 0xFFFFu), f3 = e4m3x2_to_float2(q.y >> 16);
    const uint4 out = make_uint4(pack_bf16(__fmul_rn(f0.x, s), __fmul_rn(f0.y, s)),
                                 pack_bf16(__fmul_rn(f1.x, s), __fmul_rn(f1.y, s)),
                                 pack_bf16(__fmul_rn(f2.x, s), __fmul_rn(f2.y, s)),
                                 pack_bf16(__fmul_rn(f3.x, s), __fmul_rn(f3.y, s)));
    const int bx = c >> 3, cc = c & 7;
    const uint32_t off = (uint32_t)(bx * 16384 + y * 128 + ((cc ^ (y & 7)) << 4));
    *reinterpret_cast<uint4*>(op + off) = out;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kCvtThreads, 1)
    pass_cvt_kernel(const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapBR,
                    const __grid_constant__ CUtensorMap mapBL,
                    const __grid_constant__ CUtensorMap mapBRlo,
                    const __grid_constant__ CUtensorMap mapBLlo, const CvtParams p) {
  using Lay = Layout<MODE>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[4], bar_conv[4], bar_empty[4];
  __shared__ __align__(8) uint64_t bar_blfull[2], bar_blempty[2], bar_d1full[2], bar_d1empty[2];
  __shared__ __align__(8) uint64_t bar_d2full;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const uint32_t br_bytes = (uint32_t)p.wRpad * 128 * 2;
  const uint32_t bl_bytes = (uint32_t)p.wLpad * 128 * 2;
  const uint32_t stage_bytes = Lay::op + Lay::raw + Lay::bparts * br_bytes;
  const uint32_t raw_tx = is_split<MODE>() ? 65536u : 16384u;
  const uint32_t base = smem_u32(smem);
  const uint32_t bl_base = base + S * stage_bytes;

  const int c = blockIdx.x % p.C, g = blockIdx.x / p.C;
  const int b0 = (int)((int64_t)g * p.nb / p.G), b1 = (int)((int64_t)(g + 1) * p.nb / p.G);
  const int nu = b1 - b0;
  const int64_t cw = (int64_t)p.tiles * kTileN;
  const int64_t col0 = c * cw;
  const int64_t left_tiles = (p.nR - col0 + kTileN - 1) / kTileN;
  const int nt = left_tiles < p.tiles ? (int)left_tiles : p.tiles;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_conv[s]), kConvThreads / 32);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_u32(&bar_blfull[k]), 1);
      mbar_init(smem_u32(&bar_blempty[k]), 1);
      mbar_init(smem_u32(&bar_d1full[k]), 1);
      mbar_init(smem_u32(&bar_d1empty[k]), 4);
    }
    mbar_init(smem_u32(&bar_d2full), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t d1_col = 0, d2_col = 2 * p.wRpad;

  if (warp == 0) {
    if (lane == 0 && nu > 0) {
      // ---------------- TMA producer ----------------
      uint64_t pol_stream, pol_keep;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_stream));
      asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
      int stage = 0;
      uint32_t ph = 0;
      uint32_t used = 0, last_ph = 0;   // per stage: issued at all / phase of the last fill
      uint32_t bl_used = 0, bl_ph = 0;
      bool ok = true;
      for (int u = 0; u < nu && ok; ++u) {
        const int b = b0 + u, ub = u & 1;
        const int row = b * kTileM;
        ok = mbar_wait(smem_u32(&bar_blempty[ub]), ((u >> 1) & 1) ^ 1, &abort_flag);
        if (!ok) break;
        const uint32_t blb = bl_base + ub * Lay::bparts * bl_bytes;
        mbar_expect_tx(smem_u32(&bar_blfull[ub]), Lay::bparts * bl_bytes);
        tma_2d(blb, &mapBL, row, 0, smem_u32(&bar_blfull[ub]), pol_keep);
        tma_2d(blb + bl_bytes / 2, &mapBL, row + 64, 0, smem_u32(&bar_blfull[ub]), pol_keep);
        if (MODE == MODE_SPLIT3) {
          tma_2d(blb + bl_bytes, &mapBLlo, row, 0, smem_u32(&bar_blfull[ub]), pol_keep);
          tma_2d(blb + bl_bytes + bl_bytes / 2, &mapBLlo, row + 64, 0, smem_u32(&bar_blfull[ub]),
                 pol_keep);
        }
        bl_used |= 1u << ub;
        bl_ph = (bl_ph & ~(1u << ub)) | ((uint32_t)((u >> 1) & 1) << ub);
        for (int t = 0; t < nt; ++t) {
          ok = mbar_wait(smem_u32(&bar_empty[stage]), ph ^ 1, &abort_flag);
          if (!ok) break;
          const uint32_t sb = base + stage * stage_bytes;
          const uint32_t bar = smem_u32(&bar_full[stage]);
          const int col = (int)(col0 + t * kTileN);
          mbar_expect_tx(bar, raw_tx + Lay::bparts * br_bytes);
          if (is_split<MODE>()) {
            tma_2d(sb, &mapA, col, row, bar, pol_stream);
            tma_2d(sb + 32768, &mapA, col + 64, row, bar, pol_stream);
          } else {
            tma_2d(sb + Lay::op, &mapA, col, row, bar, pol_stream);
          }
          const uint32_t sbr = sb + Lay::op + Lay::raw;
          tma_2d(sbr, &mapBR, col, 0, bar, pol_keep);
          tma_2d(sbr + br_bytes / 2, &mapBR, col + 64, 0, bar, pol_keep);
          if (MODE == MODE_SPLIT3) {
            tma_2d(sbr + br_bytes, &mapBRlo, col, 0, bar, pol_keep);
            tma_2d(sbr + br_bytes + br_bytes / 2, &mapBRlo, col + 64, 0, bar, pol_keep);
          }
          used |= 1u << stage;
          last_ph = (last_ph & ~(1u << stage)) | (ph << stage);
          if (++stage == S) {
            stage = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(p.err, 1);
      }
      for (int s = 0; s < S; ++s)
        if (((used >> s) & 1u) && !mbar_drain(smem_u32(&bar_full[s]), (last_ph >> s) & 1u))
          atomicOr(p.err, 2);
      for (int k = 0; k < 2; ++k)
        if (((bl_used >> k) & 1u) && !mbar_drain(smem_u32(&bar_blfull[k]), (bl_ph >> k) & 1u))
          atomicOr(p.err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0 && nu > 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id1 = idesc_bf16(kTileM, p.wRpad, false);
      const uint32_t id2 = idesc_bf16(kTileN, p.wLpad, true);
      constexpr int nparts = is_split<MODE>() ? 2 : 1;   // hi (+ lo)
      int stage = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int u = 0; u < nu && ok; ++u) {
        const int buf = u & 1;
        if (u >= 2) ok = mbar_wait(smem_u32(&bar_d1empty[buf]), ((u >> 1) - 1) & 1, &abort_flag);
        if (ok) ok = mbar_wait(smem_u32(&bar_blfull[buf]), (u >> 1) & 1, &abort_flag);
        if (!ok) break;
        fence_after();
        const uint32_t blb = bl_base + buf * Lay::bparts * bl_bytes;
        const uint32_t d1 = tmem + d1_col + buf * p.wRpad;
        for (int t = 0; t < nt; ++t) {
          ok = mbar_wait(smem_u32(&bar_conv[stage]), ph, &abort_flag);
          if (!ok) break;
          fence_after();
          const uint32_t sa = base + stage * stage_bytes;
          const uint32_t sbr = sa + Lay::op + Lay::raw;
#pragma unroll
          for (int part = 0; part < nparts; ++part) {
            const uint32_t pa = sa + part * 16384;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t da = sdesc(pa + (kk >> 2) * Lay::box + (kk & 3) * 32, 16, 1024);
              const uint64_t db = sdesc(sbr + (kk >> 2) * (br_bytes / 2) + (kk & 3) * 32, 16, 1024);
              mma_bf16(d1, da, db, id1, (part | t | kk) != 0);
            }
          }
          if (MODE == MODE_SPLIT3) {
            // hi part of M against the lo part of the DRM block
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t da = sdesc(sa + (kk >> 2) * Lay::box + (kk & 3) * 32, 16, 1024);
              const uint64_t db =
                  sdesc(sbr + br_bytes + (kk >> 2) * (br_bytes / 2) + (kk & 3) * 32, 16, 1024);
              mma_bf16(d1, da, db, id1, true);
            }
          }
          const uint32_t d2 = tmem + d2_col + t * p.wLpad;
#pragma unroll
          for (int part = 0; part < nparts; ++part) {
            const uint32_t pa = sa + part * 16384;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t da = sdesc(pa + kk * 2048, Lay::box, 1024);
              const uint64_t db = sdesc(blb + (kk >> 2) * (bl_bytes / 2) + (kk & 3) * 32, 16, 1024);
              mma_bf16(d2, da, db, id2, (part | u | kk) != 0);
            }
          }
          if (MODE == MODE_SPLIT3) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t da = sdesc(sa + kk * 2048, Lay::box, 1024);
              const uint64_t db =
                  sdesc(blb + bl_bytes + (kk >> 2) * (bl_bytes / 2) + (kk & 3) * 32, 16, 1024);
              mma_bf16(d2, da, db, id2, true);
            }
          }
          mma_commit(smem_u32(&bar_empty[stage]));
          if (++stage == S) {
            stage = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_blempty[buf]));
        mma_commit(smem_u32(&bar_d1full[buf]));
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(p.err, 4);
      }
      mma_commit(smem_u32(&bar_d2full));
    }
  } else if (warp >= 6) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 192;
    int stage = 0;
    uint32_t ph = 0;
    bool ok = true;
    // FP8: the scale of the next tile is loaded while the current one converts
    auto scale_of = [&](int u, int t) -> float {
      if (MODE != MODE_FP8 || u >= nu) return 1.f;
      return __ldg(p.scale + (int64_t)(b0 + u) * p.ncolt + (int)(col0 / kTileN) + t);
    };
    float s_next = scale_of(0, 0);
    for (int u = 0; u < nu && ok; ++u) {
      for (int t = 0; t < nt; ++t) {
        const float s_cur = s_next;
        s_next = t + 1 < nt ? scale_of(u, t + 1) : scale_of(u + 1, 0);
        // all converters agree before any of them enters a named barrier
        ok = conv_all(mbar_wait(smem_u32(&bar_full[stage]), ph, &abort_flag));
        if (!ok) break;
        uint8_t* st = smem + stage * stage_bytes;
        if (is_split<MODE>()) {
          convert_split_half(st, 0, ct);
          convert_split_half(st, 1, ct);
        } else {
          convert_fp8(st + Lay::op, st, s_cur, ct);
        }
        fence_proxy_async();   // generic-proxy writes -> visible to the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_conv[stage]));
        if (++stage == S) {
          stage = 0;
          ph ^= 1;
        }
      }
    }
    if (!ok) {
      abort_flag = 1;
      atomicOr(p.err, 64);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;
    const int r_in = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int u = 0; u < nu && ok; ++u) {
      const int buf = u & 1;
      ok = mbar_wait(smem_u32(&bar_d1full[buf]), (u >> 1) & 1, &abort_flag);
      if (!ok) break;
      fence_after();
      const int64_t row = (int64_t)(b0 + u) * kTileM + r_in;
      float* dst = p.C == 1 ? p.D1 + row * p.wRpad
                            : p.D1p + ((int64_t)c * p.nb * kTileM + row) * p.wRpad;
      for (int cg = 0; cg < p.wRpad; cg += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + lane_off + d1_col + buf * p.wRpad + cg, v);
        tmem_wait_ld();
        if (row < p.nL) {
          float4* d4 = reinterpret_cast<float4*>(dst + cg);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            d4[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_d1empty[buf]));
      if (p.C > 1)
        fold_d1_rows(&p.cnt[(int64_t)(b0 + u) * 4 + q], p.C, p.D1p, p.D1, p.nb, p.wRpad,
                     (int64_t)(b0 + u) * kTileM + 32 * q, p.nL, p.discard, lane);
    }
    if (!ok) {
      abort_flag = 1;
      atomicOr(p.err, 8);
    }
    if (nu == 0) {
      for (int t = 0; t < p.tiles; ++t) {
        const int64_t col = col0 + t * kTileN + r_in;
        if (col >= p.nR) continue;
        float* dst = p.D2p + ((int64_t)g * p.C * cw + col) * p.wLpad;
        for (int k = 0; k < p.wLpad; ++k) dst[k] = 0.f;
      }
    } else if (ok && mbar_wait(smem_u32(&bar_d2full), 0, &abort_flag)) {
      fence_after();
      for (int t = 0; t < nt; ++t) {
        const int64_t col = col0 + t * kTileN + r_in;
        float* dst = p.D2p + ((int64_t)g * p.C * cw + col) * p.wLpad;
        for (int cg = 0; cg < p.wLpad; cg += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + lane_off + d2_col + t * p.wLpad + cg, v);
          tmem_wait_ld();
          if (col < p.nR) {
            float4* d4 = reinterpret_cast<float4*>(dst + cg);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              d4[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                  __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
          }
        }
      }
    } else {
      atomicOr(p.err, 16);
    }
  }
  if (warp == 1 && lane == 0 && nu > 0) {
    if (!mbar_drain(smem_u32(&bar_d2full), 0)) atomicOr(p.err, 32);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

struct CvtGeometry {
  int C, G, nb, tiles, stages, grid;
  int64_t d1p_elems, d2p_elems;
  size_t smem;
};

static bool cvt_geometry(int mode, const ttnn_plan_s& P, int64_t nL, int64_t nR, CvtGeometry* g) {
  if (P.wRpad < 16 || P.wLpad < 16 || P.wRpad > 256 || P.wLpad > 256) return false;
  int tiles = (512 - 2 * P.wRpad) / P.wLpad;
  tiles = std::min(tiles, kMaxTiles);
  const int64_t ntile = (nR + kTileN - 1) / kTileN;
  tiles = (int)std::min<int64_t>(tiles, ntile);
  if (tiles < 1) return false;
  // as few chunks as TMEM allows, tiles spread evenly over them
  tiles = (int)((ntile + (ntile + tiles - 1) / tiles - 1) / ((ntile + tiles - 1) / tiles));
  const bool split = mode == MODE_SPLIT || mode == MODE_SPLIT3;
  const int64_t bparts = mode == MODE_SPLIT3 ? 2 : 1;
  const int64_t op = split ? 65536 : 32768, raw = split ? 0 : 16384;
  const int64_t stage_bytes = op + raw + bparts * (int64_t)P.wRpad * 256;
  const int64_t bl = 2 * bparts * (int64_t)P.wLpad * 256;
  const int stages = (int)std::min<int64_t>(split ? 3 : 4,
                                            (kSmemBudget - 1024 - bl) / stage_bytes);
  if (stages < 2) return false;
  g->tiles = tiles;
  g->stages = stages;
  g->smem = (size_t)(1024 + stages * stage_bytes + bl);
  g->C = (int)((nR + tiles * kTileN - 1) / (tiles * kTileN));
  g->nb = (int)((nL + kTileM - 1) / kTileM);
  const int sms = pass_sms(P);
  g->G = std::max(1, std::min(sms / g->C, g->nb));
  if (sms < g->C) g->G = 1;
  g->grid = g->C * g->G;
  g->d1p_elems = g->C == 1 ? 0 : (int64_t)g->C * g->nb * kTileM * P.wRpad;
  g->d2p_elems = (int64_t)g->G * g->C * tiles * kTileN * P.wLpad;
  return true;
}

// Per-tile E4M3 quantisation of a binary32 matrix (rows x cols, row-major):
// one block per 128 x 128 tile; s = max|tile| / 448 (s = 1 for a zero tile),
// q = e4m3(x / s) with nearest-even rounding, saturating at +-448.
// One 128 x 128 tile per block, read from global memory once: warp w holds
// rows 16 w .. 16 w + 15, lane l columns 4 l .. 4 l + 3 of each (coalesced
// 512-byte rows), the tile max over the registers, then E4M3 codes of
// x / s (binary32 division, nearest-even, saturating), four bytes per lane
// and row.  Ragged edge tiles take the same path with bounds checks.
__global__ void __launch_bounds__(256) quantize_fp8_kernel(const float* src, int64_t rows,
                                                           int64_t cols, uint8_t* dst,
                                                           float* scales, int ncolt) {
  __shared__ float red[8];
  const int64_t r0 = (int64_t)blockIdx.y * kTileM, c0 = (int64_t)blockIdx.x * kTileN;
  const int nr = (int)min((int64_t)kTileM, rows - r0), nc = (int)min((int64_t)kTileN, cols - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = 4 * lane;
  const bool full = nc == kTileN && (cols & 3) == 0 && (((uintptr_t)src) & 15) == 0;
  float4 v[16];
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int r = 16 * warp + k;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nr) {
      const float* row = src + (r0 + r) * cols + c0;
      if (full) {
        x = *reinterpret_cast<const float4*>(row + cl);
      } else {
        if (cl < nc) x.x = row[cl];
        if (cl + 1 < nc) x.y = row[cl + 1];
        if (cl + 2 < nc) x.z = row[cl + 2];
        if (cl + 3 < nc) x.w = row[cl + 3];
      }
    }
    v[k] = x;
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  mx = red[0];
  for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
  const float s = mx == 0.f ? 1.f : __fdiv_rn(mx, 448.f);
  if (threadIdx.x == 0) scales[(int64_t)blockIdx.y * ncolt + blockIdx.x] = s;
  const bool wfull = nc == kTileN && (cols & 3) == 0 && (((uintptr_t)dst) & 3) == 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int r = 16 * warp + k;
    if (r >= nr) continue;
    const float4 x = v[k];
    const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(
        make_float2(__fdiv_rn(x.x, s), __fdiv_rn(x.y, s)), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t b = __nv_cvt_float2_to_fp8x2(
        make_float2(__fdiv_rn(x.z, s), __fdiv_rn(x.w, s)), __NV_SATFINITE, __NV_E4M3);
    uint8_t* out = dst + (r0 + r) * cols + c0;
    if (wfull) {
      *reinterpret_cast<uint32_t*>(out + cl) = (uint32_t)a | ((uint32_t)b << 16);
    } else {
      if (cl < nc) out[cl] = (uint8_t)(a & 0xFF);
      if (cl + 1 < nc) out[cl + 1] = (uint8_t)(a >> 8);
      if (cl + 2 < nc) out[cl + 2] = (uint8_t)(b & 0xFF);
      if (cl + 3 < nc) out[cl + 3] = (uint8_t)(b >> 8);
    }
  }
}

}  // namespace tc

ttnn_status launch_quantize_fp8(const float* src, int64_t rows, int64_t cols, uint8_t* dst,
                                float* scales, cudaStream_t st) {
  if (rows == 0 || cols == 0) return TTNN_OK;
  const int64_t nrt = (rows + tc::kTileM - 1) / tc::kTileM, ncolt = (cols + tc::kTileN - 1) / tc::kTileN;
  if (nrt >= 65536 || ncolt >= (int64_t(1) << 31)) {
    set_error("fp8 quantisation: too many row tiles");
    return TTNN_EUNSUPPORTED;
  }
  tc::quantize_fp8_kernel<<<dim3((unsigned)ncolt, (unsigned)nrt), 256, 0, st>>>(src, rows, cols, dst,
                                                                               scales, (int)ncolt);
  return check_launch("quantize_fp8_kernel");
}

static int cvt_mode(const ttnn_plan_s& P) {
  if (P.dtype == TTNN_F32) return P.sideRs && P.sideLs ? tc::MODE_SPLIT3 : 0;
  return P.dtype == TTNN_BF16X2 ? tc::MODE_SPLIT : P.dtype == TTNN_E4M3 ? tc::MODE_FP8 : 0;
}

// hi = bf16(x), lo = bf16(x - hi) (both rounded to nearest; x - hi is exact
// in binary32): the two bfloat16 blocks a binary32 DRM block is carried as
// on the tensor cores.
__global__ void split_bf16_kernel(const float* src, int64_t n, __nv_bfloat16* hi,
                                  __nv_bfloat16* lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float x = src[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

ttnn_status launch_split_bf16(const float* src, int64_t n, void* hi, void* lo, cudaStream_t st) {
  if (n == 0) return TTNN_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)tc::sm_count() * 16);
  split_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, n, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
  return check_launch("split_bf16_kernel");
}

ttnn_status cvt_pass_supported(const ttnn_plan_s& P, int64_t nL, int64_t nR) {
  const int mode = cvt_mode(P);
  if (!mode) return TTNN_EUNSUPPORTED;
  if (P.wR <= 0 || P.wL <= 0) return TTNN_EUNSUPPORTED;
  // 16-byte TMA row strides of the tensor (and of the bf16 side blocks)
  if (nL % 8 != 0 || nR % (mode == tc::MODE_FP8 ? 16 : 8) != 0) return TTNN_EUNSUPPORTED;
  if (nL >= (int64_t(1) << 31) || nR >= (int64_t(1) << 31)) return TTNN_EUNSUPPORTED;
  tc::CvtGeometry g;
  if (!tc::cvt_geometry(mode, P, nL, nR, &g)) return TTNN_EUNSUPPORTED;
  return TTNN_OK;
}

ttnn_status launch_cvt_pass(const ttnn_plan_s& P, const void* A, int64_t nL, int64_t nR,
                            const void* sR, int64_t ldR, const void* sL, int64_t ldL, void* D1,
                            void* D2, const float* tile_scale, void* ws, int64_t ws_bytes,
                            cudaStream_t st, bool dry, int64_t* ws_need) {
  const int mode = cvt_mode(P);
  tc::CvtGeometry g;
  if (!mode || !tc::cvt_geometry(mode, P, nL, nR, &g)) {
    set_error("tensor-core pass (converted formats): unsupported geometry");
    return TTNN_EUNSUPPORTED;
  }
  const int64_t cnt_bytes = g.C > 1 ? ((int64_t)g.nb * 16 + 255) / 256 * 256 : 0;
  const int64_t need = (g.d1p_elems + g.d2p_elems) * 4 + cnt_bytes + 512;
  if (dry) {
    if (ws_need) *ws_need = need;
    return TTNN_OK;
  }
  if (ws_bytes < need) {
    set_error("tensor-core pass: workspace too small");
    return TTNN_ENOMEM;
  }
  if (((uintptr_t)A & 15) || ldR != nR || ldL != nL) {
    set_error("tensor-core pass: operands must be 16-byte aligned and dense");
    return TTNN_EUNSUPPORTED;
  }
  if (mode == tc::MODE_FP8 && (!tile_scale || ((uintptr_t)tile_scale & 3))) {
    set_error("E4M3 pass: tile scales missing or misaligned");
    return TTNN_EINVAL;
  }
  CUtensorMap mA, mBR, mBL, mBRlo, mBLlo;
  if (mode == tc::MODE_SPLIT || mode == tc::MODE_SPLIT3)
    TTNN_TRY(tc::encode_map(&mA, A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nR, nL, 64u, 128u,
                            CU_TENSOR_MAP_SWIZZLE_NONE));
  else
    TTNN_TRY(tc::encode_map(&mA, A, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, nR, nL, 128u, 128u,
                            CU_TENSOR_MAP_SWIZZLE_NONE));
  // SPLIT3: the plan's whole-tensor blocks as bf16 hi and lo halves
  const void* bR = sR;
  const void* bL = sL;
  if (mode == tc::MODE_SPLIT3) {
    bR = P.sideRs;
    bL = P.sideLs;
  }
  TTNN_TRY(tc::encode_map(&mBR, bR, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, nR, P.wRpad, 64u,
                          (uint32_t)P.wRpad, CU_TENSOR_MAP_SWIZZLE_128B));
  TTNN_TRY(tc::encode_map(&mBL, bL, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, nL, P.wLpad, 64u,
                          (uint32_t)P.wLpad, CU_TENSOR_MAP_SWIZZLE_128B));
  mBRlo = mBR;
  mBLlo = mBL;
  if (mode == tc::MODE_SPLIT3) {
    TTNN_TRY(tc::encode_map(&mBRlo, (const char*)bR + (int64_t)P.wRpad * nR * 2,
                            CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, nR, P.wRpad, 64u,
                            (uint32_t)P.wRpad, CU_TENSOR_MAP_SWIZZLE_128B));
    TTNN_TRY(tc::encode_map(&mBLlo, (const char*)bL + (int64_t)P.wLpad * nL * 2,
                            CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, nL, P.wLpad, 64u,
                            (uint32_t)P.wLpad, CU_TENSOR_MAP_SWIZZLE_128B));
  }
  tc::CvtParams prm;
  prm.nL = nL;
  prm.nR = nR;
  prm.C = g.C;
  prm.G = g.G;
  prm.nb = g.nb;
  prm.tiles = g.tiles;
  prm.stages = g.stages;
  prm.wRpad = P.wRpad;
  prm.wLpad = P.wLpad;
  prm.ncolt = (int)((nR + tc::kTileN - 1) / tc::kTileN);
  prm.scale = tile_scale;
  prm.D1 = (float*)D1;
  prm.D1p = (float*)ws;
  prm.D2p = (float*)ws + g.d1p_elems;
  prm.err = P.err_dev;
  prm.cnt = g.C > 1 ? (int*)((char*)ws + (g.d1p_elems + g.d2p_elems) * 4 + 256 -
                            (((uintptr_t)ws + (g.d1p_elems + g.d2p_elems) * 4) & 255))
                    : nullptr;
  prm.discard = (P.wRpad * 4) % 128 == 0 && ((uintptr_t)prm.D1p & 127) == 0;
  if (g.C > 1) TTNN_TRY_CUDA(cudaMemsetAsync(prm.cnt, 0, (size_t)g.nb * 16, st));
  if (mode == tc::MODE_SPLIT) {
    TTNN_TRY(tc::smem_limit_once((const void*)tc::pass_cvt_kernel<tc::MODE_SPLIT>, 1));
    tc::pass_cvt_kernel<tc::MODE_SPLIT><<<g.grid, tc::kCvtThreads, g.smem, st>>>(
        mA, mBR, mBL, mBRlo, mBLlo, prm);
  } else if (mode == tc::MODE_SPLIT3) {
    TTNN_TRY(tc::smem_limit_once((const void*)tc::pass_cvt_kernel<tc::MODE_SPLIT3>, 3));
    tc::pass_cvt_kernel<tc::MODE_SPLIT3><<<g.grid, tc::kCvtThreads, g.smem, st>>>(
        mA, mBR, mBL, mBRlo, mBLlo, prm);
  } else {
    TTNN_TRY(tc::smem_limit_once((const void*)tc::pass_cvt_kernel<tc::MODE_FP8>, 2));
    tc::pass_cvt_kernel<tc::MODE_FP8><<<g.grid, tc::kCvtThreads, g.smem, st>>>(
        mA, mBR, mBL, mBRlo, mBLlo, prm);
  }
  TTNN_TRY(check_launch("tc pass_cvt_kernel"));
  if (P.prof_kernel_end) cudaEventRecord(P.prof_kernel_end, st);
  const int sms = tc::sm_count();
  tc::reduce_partials<<<sms * 4, 256, 0, st>>>(prm.D2p, g.G, (int64_t)g.C * g.tiles * tc::kTileN * P.wLpad,
                                               nR, P.wLpad, (float*)D2);
  TTNN_TRY(check_launch("reduce_partials(D2)"));
  return TTNN_OK;
}

}  // namespace ttnn
