// Inline-PTX building blocks of the tcgen05 first-level passes (sm_103a):
// mbarriers with bounded waits, TMA tile loads, shared-memory and instruction
// descriptors of kind::f16 MMAs, TMEM loads, and the host helpers the pass
// launchers share.
#pragma once

#include <cuda.h>

#include "plan.cuh"

namespace ttnn {
namespace tc {

constexpr int kTileM = 128;           // rows of M per tile (MMA M for D1)
constexpr int kTileN = 128;           // columns of M per tile (MMA M for D2)
constexpr int kMaxTiles = 16;         // column tiles per chunk (TMEM bounds it first)
constexpr int kSmemBudget = 232448 - 2048;   // 227 KB opt-in minus static shared memory
constexpr uint64_t kTimeoutNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after limit_ns or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = kTimeoutNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > limit_ns) return false;
  }
}
// Bounded wait that ignores the abort flag (used to drain own work).
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > kTimeoutNs) return false;
  return true;
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                       uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

// tcgen05 shared-memory descriptor: start, leading / stride byte offsets,
// fixed version bits 46-48 = 0b001, 128-byte swizzle (mode 2, bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: D f32, A/B bf16, A K- or MN-major,
// B K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Host helpers (pass_tc.cu).
// Raises a kernel's dynamic shared memory limit to kSmemBudget, once per
// device.  Setting it per launch to the launch's own size would race between
// host threads launching the same kernel with different sizes.
ttnn_status smem_limit_once(const void* func, int slot);
ttnn_status encode_map(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize,
                       int64_t inner, int64_t outer, uint32_t box_inner, uint32_t box_outer,
                       CUtensorMapSwizzle sw);
int sm_count();
// SMs a first-level pass spreads its persistent CTAs over: all of them, or,
// with TTNN_FLAG_RESERVE_SMS, all but max(8, sketched nodes) (at most a
// quarter), which stay free for a recovery running on another stream.
int pass_sms(const ttnn_plan_s& P);
// D[i][w] = sum_k P[k][i][w] for w < wpad (rows i < rows).
__global__ void reduce_partials(const float* P, int K, int64_t stride_k, int64_t rows, int wpad,
                                float* D);

// D1 of a pass split into C column chunks: every chunk CTA writes its partial
// rows of a row block (D1p = [C][nb*128][wRpad]) and then, per epilogue warp
// (its 32 rows row0..row0+31), counts its arrival in *slot.  The warp that
// arrives last sums the C partials in chunk order (the same order as
// reduce_partials, whoever is last) into D1, with coalesced loads of the 32
// contiguous rows, and drops the dead partial lines from L2 (`discard`: rows
// are whole 128-byte lines).  Called by all 32 lanes after their own stores;
// no thread waits on another.
__device__ __forceinline__ void fold_d1_rows(int* slot, int C, const float* D1p, float* D1,
                                             int64_t nb, int wRpad, int64_t row0, int64_t nL,
                                             int discard, int lane) {
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atomicAdd(slot, 1) == C - 1;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  const int per = wRpad / 4;                       // float4 per row
  const int64_t cs4 = nb * kTileM * per;           // chunk stride
  const int64_t lim = (nL - row0) * per;           // valid float4 of the 32 rows
  const float4* src = reinterpret_cast<const float4*>(D1p) + row0 * per;
  float4* out = reinterpret_cast<float4*>(D1) + row0 * per;
  const int n4 = 32 * per;
  if (C <= 4) {
    // every partial's loads of a batch in flight at once (one L2 round trip
    // per batch instead of one per partial), then the sums in chunk order
    for (int e0 = lane; e0 < n4; e0 += 128) {
      float4 v[4][4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = e0 + 32 * j;
          v[cc][j] = (cc < C && e < n4) ? __ldcg(src + cc * cs4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float4 acc = v[0][j];
#pragma unroll
        for (int cc = 1; cc < 4; ++cc) {
          if (cc >= C) break;
          acc.x += v[cc][j].x;
          acc.y += v[cc][j].y;
          acc.z += v[cc][j].z;
          acc.w += v[cc][j].w;
        }
        const int e = e0 + 32 * j;
        if (e < n4 && e < lim) out[e] = acc;
      }
    }
  }
  for (int e0 = lane; C > 4 && e0 < n4; e0 += 128) {
    float4 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = e0 + 32 * j;
      acc[j] = e < n4 ? __ldcg(src + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int cc = 1; cc < C; ++cc) {
      float4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = e0 + 32 * j;
        v[j] = e < n4 ? __ldcg(src + cc * cs4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[j].x += v[j].x;
        acc[j].y += v[j].y;
        acc[j].z += v[j].z;
        acc[j].w += v[j].w;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = e0 + 32 * j;
      if (e < n4 && e < lim) out[e] = acc[j];
    }
  }
  if (discard) {
    const int lines = 32 * wRpad * 4 / 128;
    for (int cc = 0; cc < C; ++cc)
      for (int l = lane; l < lines; l += 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"((const char*)(src + cc * cs4) +
                                                            (int64_t)l * 128)
                     : "memory");
  }
}

}  // namespace tc
}  // namespace ttnn
