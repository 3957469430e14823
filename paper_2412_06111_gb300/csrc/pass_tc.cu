// First-level pass on the 5th-generation tensor cores (sm_103a, tcgen05).
//
// The dense block is viewed as M (nL x nR, row-major: rows = the root's
// left-group modes, columns = the right-group modes).  One pass over M forms
// both products of the sketch phase (Sec. 4) that touch the tensor:
//   D1 = M  B_R^T   (nL x wR)  contraction over the right modes
//   D2 = M^T B_L^T  (nR x wL)  contraction over the left modes
// with B_R / B_L the Khatri-Rao DRM blocks stored [w][n] in bf16.
//
// Each 128 x 128 tile of M is staged into shared memory once by TMA (128-byte
// swizzle) and read by two tcgen05.mma streams: as a K-major A operand for D1
// (M = 128 rows) and as an MN-major A operand for D2 (M = 128 columns).  D1
// of the current row block and D2 of the CTA's column chunk accumulate in
// TMEM in FP32.  Persistent CTAs, one per SM: CTA (chunk c, group g) owns the
// columns [c*CW, (c+1)*CW) and a contiguous range of row blocks; D1 partials
// per chunk and D2 partials per group are summed by two small reductions.
//
// Warp roles (192 threads): warp 0 TMA producer, warp 1 TMEM owner + MMA
// issuer, warps 2-5 epilogue (TMEM lane quarter = warp % 4).  Every mbarrier
// wait is bounded by a %globaltimer deadline; on expiry the kernel records
// an error flag, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tc_ptx.cuh"

namespace ttnn {

namespace tc {

constexpr int kThreads = 192;

struct Params {
  int64_t nL, nR;
  int C, G, nb, tiles, stages;
  int wRpad, wLpad;
  int cluster;     // 1: the C chunk CTAs of a row range form a cluster and sum D1 on chip
  float* D1;       // [nL][wRpad] output
  float* D1p;      // [C][nb*128][wRpad] chunk partials (C > 1, no cluster)
  float* D2p;      // [G][C*tiles*128][wLpad]
  int* err;
  int* cnt;        // [nb][4] chunk arrivals per row block and epilogue warp (C > 1, no cluster), zero at launch
  int discard;     // partial rows are whole 128-byte lines: drop them from L2 once summed
  uint64_t wait_ns;  // limit of each pipeline wait (drains of own copies keep the 2 s limit)
};

// --- thread-block cluster (distributed shared memory) helpers
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
  return out;
}
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity,
                                                  volatile int* abort) {
  if (mbar_try_cluster(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try_cluster(bar, parity)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > kTimeoutNs) return false;
  }
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    pass_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBR,
                const __grid_constant__ CUtensorMap mapBL, const Params p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[8], bar_empty[8];
  __shared__ __align__(8) uint64_t bar_blfull[2], bar_blempty[2], bar_d1full[2], bar_d1empty[2];
  __shared__ __align__(8) uint64_t bar_d2full;
  __shared__ __align__(8) uint64_t bar_ready[2], bar_freed[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const uint32_t a_bytes = kTileM * 128 * 2;                   // two 64-column boxes
  const uint32_t br_bytes = (uint32_t)p.wRpad * 128 * 2;
  const uint32_t bl_bytes = (uint32_t)p.wLpad * 128 * 2;
  const uint32_t stage_bytes = a_bytes + br_bytes;
  const uint32_t base = smem_u32(smem);
  const uint32_t bl_base = base + S * stage_bytes;
  const uint32_t part_bytes = (uint32_t)kTileM * p.wRpad * 4;
  const uint32_t part_base = bl_base + 2 * bl_bytes;          // 2 D1 partial tiles (cluster)
  float* part_ptr = (float*)(smem + (part_base - base));
  const uint32_t crank = p.cluster ? cluster_rank() : 0;

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
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_u32(&bar_blfull[k]), 1);
      mbar_init(smem_u32(&bar_blempty[k]), 1);
      mbar_init(smem_u32(&bar_d1full[k]), 1);
      mbar_init(smem_u32(&bar_d1empty[k]), 4);
    }
    mbar_init(smem_u32(&bar_d2full), 1);
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_u32(&bar_ready[k]), 4 * p.C);
      mbar_init(smem_u32(&bar_freed[k]), 4 * p.C);
    }
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
  if (p.cluster) cluster_sync_all();   // peers' barriers are initialised before any remote arrive
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
      int last_ph[8];
      for (int s = 0; s < 8; ++s) last_ph[s] = -1;
      int bl_last[2] = {-1, -1};
      bool ok = true;
      for (int u = 0; u < nu && ok; ++u) {
        const int b = b0 + u, ub = u & 1;
        const int row = b * kTileM;
        if (p.wLpad > 0) {
          ok = mbar_wait(smem_u32(&bar_blempty[ub]), ((u >> 1) & 1) ^ 1, &abort_flag, p.wait_ns);
          if (!ok) break;
          const uint32_t blb = bl_base + ub * bl_bytes;
          mbar_expect_tx(smem_u32(&bar_blfull[ub]), bl_bytes);
          tma_2d(blb, &mapBL, row, 0, smem_u32(&bar_blfull[ub]), pol_keep);
          tma_2d(blb + bl_bytes / 2, &mapBL, row + 64, 0, smem_u32(&bar_blfull[ub]), pol_keep);
          bl_last[ub] = (u >> 1) & 1;
        }
        for (int t = 0; t < nt; ++t) {
          ok = mbar_wait(smem_u32(&bar_empty[stage]), ph ^ 1, &abort_flag, p.wait_ns);
          if (!ok) break;
          const uint32_t sb = base + stage * stage_bytes;
          const int col = (int)(col0 + t * kTileN);
          mbar_expect_tx(smem_u32(&bar_full[stage]), stage_bytes);
          tma_2d(sb, &mapA, col, row, smem_u32(&bar_full[stage]), pol_stream);
          tma_2d(sb + a_bytes / 2, &mapA, col + 64, row, smem_u32(&bar_full[stage]), pol_stream);
          tma_2d(sb + a_bytes, &mapBR, col, 0, smem_u32(&bar_full[stage]), pol_keep);
          tma_2d(sb + a_bytes + br_bytes / 2, &mapBR, col + 64, 0, smem_u32(&bar_full[stage]),
                 pol_keep);
          last_ph[stage] = (int)ph;
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
      // the copies this thread issued must land before the CTA may exit
      for (int s = 0; s < S; ++s)
        if (last_ph[s] >= 0 && !mbar_drain(smem_u32(&bar_full[s]), (uint32_t)last_ph[s]))
          atomicOr(p.err, 2);
      for (int k = 0; k < 2; ++k)
        if (bl_last[k] >= 0 && !mbar_drain(smem_u32(&bar_blfull[k]), (uint32_t)bl_last[k]))
          atomicOr(p.err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0 && nu > 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id1 = idesc_bf16(kTileM, p.wRpad, false);
      const uint32_t id2 = idesc_bf16(kTileN, p.wLpad, true);
      int stage = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int u = 0; u < nu && ok; ++u) {
        const int buf = u & 1;
        if (u >= 2) ok = mbar_wait(smem_u32(&bar_d1empty[buf]), ((u >> 1) - 1) & 1, &abort_flag, p.wait_ns);
        if (ok && p.wLpad > 0) ok = mbar_wait(smem_u32(&bar_blfull[buf]), (u >> 1) & 1, &abort_flag, p.wait_ns);
        if (!ok) break;
        fence_after();
        const uint32_t blb = bl_base + buf * bl_bytes;
        const uint32_t d1 = tmem + d1_col + buf * p.wRpad;
        for (int t = 0; t < nt; ++t) {
          ok = mbar_wait(smem_u32(&bar_full[stage]), ph, &abort_flag, p.wait_ns);
          if (!ok) break;
          fence_after();
          const uint32_t sa = base + stage * stage_bytes;
          const uint32_t sbr = sa + a_bytes;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint64_t da = sdesc(sa + (kk >> 2) * (a_bytes / 2) + (kk & 3) * 32, 16, 1024);
            const uint64_t db = sdesc(sbr + (kk >> 2) * (br_bytes / 2) + (kk & 3) * 32, 16, 1024);
            mma_bf16(d1, da, db, id1, (t | kk) != 0);
          }
          if (p.wLpad > 0) {
            const uint32_t d2 = tmem + d2_col + t * p.wLpad;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t da = sdesc(sa + kk * 2048, a_bytes / 2, 1024);
              const uint64_t db = sdesc(blb + (kk >> 2) * (bl_bytes / 2) + (kk & 3) * 32, 16, 1024);
              mma_bf16(d2, da, db, id2, (u | kk) != 0);
            }
          }
          mma_commit(smem_u32(&bar_empty[stage]));
          if (++stage == S) {
            stage = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        if (p.wLpad > 0) mma_commit(smem_u32(&bar_blempty[buf]));
        mma_commit(smem_u32(&bar_d1full[buf]));
      }
      if (!ok) {
        abort_flag = 1;
        atomicOr(p.err, 4);
      }
      // completion of every MMA issued here (also on the abort path)
      mma_commit(smem_u32(&bar_d2full));
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;
    const int r_in = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int u = 0; u < nu && ok; ++u) {
      const int buf = u & 1;
      ok = mbar_wait(smem_u32(&bar_d1full[buf]), (u >> 1) & 1, &abort_flag, p.wait_ns);
      if (!ok) break;
      fence_after();
      const int64_t row = (int64_t)(b0 + u) * kTileM + r_in;
      if (!p.cluster) {
        // C == 1: D1 directly; C > 1: this chunk's partial.  The chunk CTA
        // that finishes a row block last sums its C partials in chunk order
        // into D1 (deterministic: the order does not depend on who is last)
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
        continue;
      }
      // cluster: partial tile -> own shared memory, then every CTA sums its
      // share of the rows over the C partials (fixed order) into D1.
      if (u >= 2) {
        ok = mbar_wait_cluster(smem_u32(&bar_freed[buf]), ((u >> 1) - 1) & 1, &abort_flag);
        if (!ok) break;
      }
      float* prow = part_ptr + (buf * kTileM + r_in) * p.wRpad;
      for (int cg = 0; cg < p.wRpad; cg += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + lane_off + d1_col + buf * p.wRpad + cg, v);
        tmem_wait_ld();
        float4* d4 = reinterpret_cast<float4*>(prow + cg);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          d4[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                              __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bar_d1empty[buf]));
        for (int cc = 0; cc < p.C; ++cc) remote_arrive(mapa(smem_u32(&bar_ready[buf]), cc));
      }
      ok = mbar_wait_cluster(smem_u32(&bar_ready[buf]), (u >> 1) & 1, &abort_flag);
      if (!ok) break;
      {
        const int rows_per = kTileM / p.C;
        const int q4 = p.wRpad / 4;
        const int et = threadIdx.x - 64;            // 0..127 over the epilogue warps
        const uint32_t pb = part_base + buf * part_bytes;
        // up to 4 row-chunks x C sources of remote loads in flight before any add
        for (int idx0 = et; idx0 < rows_per * q4; idx0 += 4 * 128) {
          float4 acc[4];
          uint32_t offs[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int idx = idx0 + k * 128;
            const int rr = (int)crank * rows_per + idx / q4, c4 = idx % q4;
            offs[k] = (uint32_t)(rr * p.wRpad + c4 * 4) * 4;
            acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            if (cc >= p.C) break;
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
              v[k] = (idx0 + k * 128 < rows_per * q4) ? ld_cluster_f4(mapa(pb + offs[k], cc))
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              acc[k].x += v[k].x;
              acc[k].y += v[k].y;
              acc[k].z += v[k].z;
              acc[k].w += v[k].w;
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int idx = idx0 + k * 128;
            if (idx >= rows_per * q4) continue;
            const int rr = (int)crank * rows_per + idx / q4, c4 = idx % q4;
            const int64_t grow = (int64_t)(b0 + u) * kTileM + rr;
            if (grow < p.nL) reinterpret_cast<float4*>(p.D1p + grow * p.wRpad)[c4] = acc[k];
          }
        }
      }
      __syncwarp();
      if (lane == 0)
        for (int cc = 0; cc < p.C; ++cc) remote_arrive(mapa(smem_u32(&bar_freed[buf]), cc));
    }
    if (!ok) {
      abort_flag = 1;
      atomicOr(p.err, 8);
    }
    // D2 of the column chunk (none when the plan has no left-side block)
    if (p.wLpad == 0) {
      // no D2 product to write
    } else if (nu == 0) {
      for (int t = 0; t < p.tiles; ++t) {
        const int64_t col = col0 + t * kTileN + r_in;
        if (col >= p.nR) continue;
        float* dst = p.D2p + ((int64_t)g * p.C * cw + col) * p.wLpad;
        for (int k = 0; k < p.wLpad; ++k) dst[k] = 0.f;
      }
    } else if (ok && mbar_wait(smem_u32(&bar_d2full), 0, &abort_flag, p.wait_ns)) {
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
  // all MMAs must be complete before TMEM is released
  if (warp == 1 && lane == 0 && nu > 0) {
    if (!mbar_drain(smem_u32(&bar_d2full), 0)) atomicOr(p.err, 32);
  }
  fence_before();
  __syncthreads();
  if (p.cluster) cluster_sync_all();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

__global__ void reduce_partials(const float* P, int K, int64_t stride_k, int64_t rows, int wpad,
                                float* D) {
  const int64_t n4 = rows * wpad / 4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4;
       e += (int64_t)gridDim.x * blockDim.x) {
    float4 acc = reinterpret_cast<const float4*>(P)[e];
    for (int k = 1; k < K; ++k) {
      const float4 v = reinterpret_cast<const float4*>(P + k * stride_k)[e];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    reinterpret_cast<float4*>(D)[e] = acc;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
  }
  return fn;
}

// 2-D map over a row-major (outer x inner) array of esize-byte elements.
ttnn_status encode_map(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize,
                       int64_t inner, int64_t outer, uint32_t box_inner, uint32_t box_outer,
                       CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return TTNN_ECUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)inner * esize};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = enc(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TTNN_ECUDA;
  }
  return TTNN_OK;
}

// bf16 map with 64 x box_outer boxes, 128-byte swizzle.
static ttnn_status make_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer,
                            int box_outer) {
  return encode_map(m, ptr, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, inner, outer, 64u,
                    (uint32_t)box_outer, CU_TENSOR_MAP_SWIZZLE_128B);
}

struct Geometry {
  int C, G, nb, tiles, stages, grid, cluster;
  int64_t d1p_elems, d2p_elems;
  size_t smem;
};

ttnn_status smem_limit_once(const void* func, int slot) {
  static std::mutex mu;
  static bool done[4][64] = {};
  int dev = 0;
  TTNN_TRY_CUDA(cudaGetDevice(&dev));
  if (slot < 0 || slot >= 4 || dev < 0 || dev >= 64) {
    set_error("internal: shared-memory limit slot");
    return TTNN_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!done[slot][dev]) {
    TTNN_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBudget));
    done[slot][dev] = true;
  }
  return TTNN_OK;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

int pass_sms(const ttnn_plan_s& P) {
  const int sms = sm_count();
  if (!(P.flags & TTNN_FLAG_RESERVE_SMS)) return sms;
  const int keep = std::min(std::max(8, P.n_sketched), sms / 4);
  return sms - keep;
}

static int max_clusters(int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 64, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (smem_limit_once((const void*)pass_kernel, 0) != TTNN_OK ||
      cudaOccupancyMaxActiveClusters(&n, pass_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

static bool geometry(const ttnn_plan_s& P, int64_t nL, int64_t nR, Geometry* g) {
  if (P.wRpad < 16 || (P.wLpad != 0 && P.wLpad < 16) || P.wRpad > 256 || P.wLpad > 256)
    return false;
  // without a D2 product (w_L = 0) TMEM holds only the double-buffered D1
  int tiles = P.wLpad > 0 ? (512 - 2 * P.wRpad) / P.wLpad : kMaxTiles;
  tiles = std::min(tiles, kMaxTiles);
  const int64_t ntile = (nR + kTileN - 1) / kTileN;
  tiles = (int)std::min<int64_t>(tiles, ntile);
  if (tiles < 1) return false;
  // as few chunks as TMEM allows, then tiles spread evenly over them (the
  // CTAs of a short last chunk would idle while the others finish)
  tiles = (int)((ntile + (ntile + tiles - 1) / tiles - 1) / ((ntile + tiles - 1) / tiles));
  const int64_t stage_bytes = kTileM * 128 * 2 + (int64_t)P.wRpad * 256;
  const int64_t bl = 2 * (int64_t)P.wLpad * 256;
  g->tiles = tiles;
  g->C = (int)((nR + tiles * kTileN - 1) / (tiles * kTileN));
  g->nb = (int)((nL + kTileM - 1) / kTileM);
  const int sms = pass_sms(P);
  // cluster path: C in {2, 4, 8}, D1 partial tiles fit beside >= 3 stages
  g->cluster = 0;
  const int64_t parts = 2 * (int64_t)kTileM * P.wRpad * 4;
  if ((g->C == 2 || g->C == 4 || g->C == 8) && P.wRpad <= 64 && (P.flags & TTNN_FLAG_CLUSTER_REDUCE)) {
    const int stages = (int)std::min<int64_t>(8, (kSmemBudget - 1024 - bl - parts) / stage_bytes);
    if (stages >= 3) {
      const size_t smem = (size_t)(1024 + stages * stage_bytes + bl + parts);
      const int mc = max_clusters(g->C, smem);
      if (mc >= 1) {
        g->cluster = 1;
        g->stages = stages;
        g->smem = smem;
        g->G = std::max(1, std::min(mc, g->nb));
      }
    }
  }
  if (!g->cluster) {
    const int stages = (int)std::min<int64_t>(8, (kSmemBudget - 1024 - bl) / stage_bytes);
    if (stages < 2) return false;
    g->stages = stages;
    g->smem = (size_t)(1024 + stages * stage_bytes + bl);
    g->G = std::max(1, std::min(sms / g->C, g->nb));
    if (sms < g->C) g->G = 1;
  }
  g->grid = g->C * g->G;
  g->d1p_elems = (g->cluster || g->C == 1) ? 0 : (int64_t)g->C * g->nb * kTileM * P.wRpad;
  g->d2p_elems = (int64_t)g->G * g->C * tiles * kTileN * P.wLpad;
  return true;
}

}  // namespace tc

ttnn_status tc_pass_supported(const ttnn_plan_s& P, int64_t nL, int64_t nR) {
  if (P.dtype != TTNN_BF16 || P.pass_store != 2) return TTNN_EUNSUPPORTED;
  if (P.wR <= 0 || P.wL < 0) return TTNN_EUNSUPPORTED;
  if (nL % 8 != 0 || nR % 8 != 0) return TTNN_EUNSUPPORTED;   // 16-byte TMA row strides
  if (nL >= (int64_t(1) << 31) || nR >= (int64_t(1) << 31)) return TTNN_EUNSUPPORTED;
  tc::Geometry g;
  if (!tc::geometry(P, nL, nR, &g)) return TTNN_EUNSUPPORTED;
  return TTNN_OK;
}

ttnn_status launch_tc_pass(const ttnn_plan_s& P, const void* A, int64_t nL, int64_t nR,
                           const void* sR, int64_t ldR, const void* sL, int64_t ldL, void* D1,
                           void* D2, const float* tile_scale, void* ws, int64_t ws_bytes,
                           cudaStream_t st, bool dry, int64_t* ws_need) {
  (void)tile_scale;
  tc::Geometry g;
  if (!tc::geometry(P, nL, nR, &g)) {
    set_error("tensor-core pass: unsupported geometry");
    return TTNN_EUNSUPPORTED;
  }
  const bool fold = !g.cluster && g.C > 1;   // D1 partials summed inside the kernel
  const int64_t cnt_bytes = fold ? ((int64_t)g.nb * 16 + 255) / 256 * 256 : 0;
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
  CUtensorMap mA, mBR, mBL;
  TTNN_TRY(tc::make_map(&mA, A, nR, nL, tc::kTileM));
  TTNN_TRY(tc::make_map(&mBR, sR, nR, P.wRpad, P.wRpad));
  if (P.wLpad > 0) TTNN_TRY(tc::make_map(&mBL, sL, nL, P.wLpad, P.wLpad));
  else mBL = mBR;   // never read: the kernel forms no D2 product
  tc::Params prm;
  prm.nL = nL;
  prm.nR = nR;
  prm.C = g.C;
  prm.G = g.G;
  prm.nb = g.nb;
  prm.tiles = g.tiles;
  prm.stages = g.stages;
  prm.wRpad = P.wRpad;
  prm.wLpad = P.wLpad;
  prm.cluster = g.cluster;
  prm.D1 = (float*)D1;
  prm.D1p = g.cluster ? (float*)D1 : (float*)ws;
  prm.D2p = (float*)ws + g.d1p_elems;

  prm.err = P.err_dev;
  prm.wait_ns = (P.flags & TTNN_FLAG_WAIT_TEST) ? 0 : tc::kTimeoutNs;
  prm.cnt = fold ? (int*)((char*)ws + (g.d1p_elems + g.d2p_elems) * 4 + 256 -
                          (((uintptr_t)ws + (g.d1p_elems + g.d2p_elems) * 4) & 255))
                 : nullptr;
  prm.discard = (P.wRpad * 4) % 128 == 0 && ((uintptr_t)prm.D1p & 127) == 0;
  if (fold) TTNN_TRY_CUDA(cudaMemsetAsync(prm.cnt, 0, (size_t)g.nb * 16, st));
  TTNN_TRY(tc::smem_limit_once((const void*)tc::pass_kernel, 0));
  if (g.cluster) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.grid, 1, 1);
    cfg.blockDim = dim3(tc::kThreads, 1, 1);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TTNN_TRY_CUDA(cudaLaunchKernelEx(&cfg, tc::pass_kernel, mA, mBR, mBL, prm));
    count_launch();
  } else {
    tc::pass_kernel<<<g.grid, tc::kThreads, g.smem, st>>>(mA, mBR, mBL, prm);
    TTNN_TRY(check_launch("tc pass_kernel"));
  }
  if (P.prof_kernel_end) cudaEventRecord(P.prof_kernel_end, st);
  const int sms = tc::sm_count();
  if (P.wLpad > 0) {
    tc::reduce_partials<<<sms * 4, 256, 0, st>>>(prm.D2p, g.G, (int64_t)g.C * g.tiles * tc::kTileN * P.wLpad,
                                                 nR, P.wLpad, (float*)D2);
    TTNN_TRY(check_launch("reduce_partials(D2)"));
  }
  return TTNN_OK;
}

}  // namespace ttnn
