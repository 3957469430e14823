// Batched executor of small-contraction programs (see program.cuh).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cstdio>

#include "program.cuh"

namespace ttnn {

constexpr int kExecThreads = 256;
static_assert(sizeof(LevelBatch) <= 32000, "level batch must fit the kernel parameter space");
constexpr int kMpKC2 = 32;
constexpr size_t kExecSmem = 48 * 1024;

static int exec_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// ---------------------------------------------------------------------------
// device parts
// ---------------------------------------------------------------------------
template <typename Tin, typename Tw, typename Tout, typename Tacc, typename I>
__device__ void dev_contract(const DevOp& op, int64_t blk) {
  const Contract& c = op.c;
  const int g = op.g;
  const I J = (I)c.J, Q = (I)c.Q, NB = (I)c.NB;
  const I total = (I)(c.P * c.NB * c.Q * c.J);
  const I vo = (I)(blk * (kExecThreads / g)) + (I)(threadIdx.x / g);
  const int lg = threadIdx.x % g;
  const bool valid = vo < total * (I)op.nsplit;
  Tacc acc = 0;
  I split = 0, o = 0, p = 0, b = 0, q = 0, j = 0;
  if (valid) {
    split = vo / total;
    o = vo - split * total;
    I t = o;
    j = t % J;
    t /= J;
    q = t % Q;
    t /= Q;
    b = t % NB;
    p = t / NB;
    const int64_t i0 = (int64_t)split * op.chunk;
    const int64_t i1 = min(c.NI, i0 + op.chunk);
    const Tin* ip = (const Tin*)c.in + (int64_t)p * c.isP + (int64_t)q * c.isQ + (int64_t)j * c.isJ;
    // four independent partial sums: loads and multiply-adds of different
    // terms overlap instead of waiting on one accumulator
    Tacc a1 = 0, a2 = 0, a3 = 0;
    int64_t i = i0 + lg;
    if (c.w) {
      const Tw* wp = (const Tw*)c.w + (int64_t)p * c.wsP + (int64_t)b * c.wsB + (int64_t)q * c.wsQ +
                     (int64_t)j * c.wsJ;
      for (; i + 3 * g < i1; i += 4 * g) {
        acc += (Tacc)ip[i * c.isI] * (Tacc)wp[i * c.wsI];
        a1 += (Tacc)ip[(i + g) * c.isI] * (Tacc)wp[(i + g) * c.wsI];
        a2 += (Tacc)ip[(i + 2 * g) * c.isI] * (Tacc)wp[(i + 2 * g) * c.wsI];
        a3 += (Tacc)ip[(i + 3 * g) * c.isI] * (Tacc)wp[(i + 3 * g) * c.wsI];
      }
      for (; i < i1; i += g) acc += (Tacc)ip[i * c.isI] * (Tacc)wp[i * c.wsI];
    } else {
      for (; i + 3 * g < i1; i += 4 * g) {
        acc += (Tacc)ip[i * c.isI];
        a1 += (Tacc)ip[(i + g) * c.isI];
        a2 += (Tacc)ip[(i + 2 * g) * c.isI];
        a3 += (Tacc)ip[(i + 3 * g) * c.isI];
      }
      for (; i < i1; i += g) acc += (Tacc)ip[i * c.isI];
    }
    acc = (acc + a1) + (a2 + a3);
  }
  for (int off = g >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (valid && lg == 0) {
    if (op.nsplit > 1) {
      ((Tout*)op.partial)[(int64_t)split * total + o] = (Tout)acc;
    } else {
      Tout* out = (Tout*)c.out;
      const int64_t oi = (int64_t)p * c.osP + (int64_t)b * c.osB + (int64_t)q * c.osQ + (int64_t)j * c.osJ;
      const Tout v = (Tout)((Tacc)c.alpha * acc);
      out[oi] = c.accumulate ? (Tout)(out[oi] + v) : v;
    }
  }
}

template <typename T, typename I>
__device__ void dev_reduce(const DevOp& op, int64_t blk) {
  const Contract& c = op.c;
  const I total = (I)(c.P * c.NB * c.Q * c.J);
  const I o = (I)(blk * kExecThreads) + (I)threadIdx.x;
  if (o >= total) return;
  const T* part = (const T*)op.partial;
  T acc = 0;
  for (int s = 0; s < op.nsplit; ++s) acc += part[(int64_t)s * total + o];
  I t = o;
  const I j = t % (I)c.J;
  t /= (I)c.J;
  const I q = t % (I)c.Q;
  t /= (I)c.Q;
  const I b = t % (I)c.NB;
  const I p = t / (I)c.NB;
  T* out = (T*)c.out;
  const int64_t oi = (int64_t)p * c.osP + (int64_t)b * c.osB + (int64_t)q * c.osQ + (int64_t)j * c.osJ;
  const T v = (T)c.alpha * acc;
  out[oi] = c.accumulate ? out[oi] + v : v;
}

// Mode product as a batched small GEMM over one chunk of CH batch items:
// out[p,b,q,j] (+)= alpha * sum_i W[i*wsI + b*wsB] * in[p,i,q,j].
template <typename T, typename I>
__device__ void dev_mp(const DevOp& op, int64_t blk, unsigned char* smem) {
  const Contract& c = op.c;
  const int BG = op.BG, CG = op.CG, CH = op.CH;
  const int WB = 4 * BG, WC = 4 * CG;
  T* Ws = (T*)smem;                   // [kMpKC2][WB]
  T* Is = Ws + kMpKC2 * WB;           // [kMpKC2][WC]
  const int tid = threadIdx.x;
  const int bg = tid / CG, cg = tid % CG;
  const int J = (int)c.J;
  const int ncol = CH * J;
  const I items = (I)(c.P * c.Q);
  const I Qi = (I)c.Q;
  const I it0 = (I)(blk * CH);
  // fixed load column of this thread (WC divides the block size)
  const int lcol = tid % WC, lrow0 = tid / WC, lstep = kExecThreads / WC;
  bool lvalid = false;
  int64_t lbase = 0;
  if (lcol < ncol) {
    const I item = it0 + (I)(lcol / J);
    if (item < items) {
      const I p = item / Qi, q = item - p * Qi;
      lbase = (int64_t)p * c.isP + (int64_t)q * c.isQ + (int64_t)(lcol % J) * c.isJ;
      lvalid = true;
    }
  }
  const int wcol = tid % WB, wrow0 = tid / WB, wstep = kExecThreads / WB;
  const T* in = (const T*)c.in;
  const T* w = (const T*)c.w;
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0;
  for (int64_t i0 = 0; i0 < c.NI; i0 += kMpKC2) {
    const int kc = (int)min((int64_t)kMpKC2, c.NI - i0);
    __syncthreads();
    for (int ii = wrow0; ii < kc; ii += wstep)
      Ws[ii * WB + wcol] = (wcol < c.NB) ? w[(i0 + ii) * c.wsI + wcol * c.wsB] : (T)0;
    for (int ii = lrow0; ii < kc; ii += lstep)
      Is[ii * WC + lcol] = lvalid ? in[lbase + (i0 + ii) * c.isI] : (T)0;
    __syncthreads();
    if (bg < BG) {
      for (int ii = 0; ii < kc; ++ii) {
        // 4 consecutive elements per thread: one vector load each (the column
        // tile is read conflict-free, the weight tile is a broadcast)
        T a[4], bb[4];
        if (sizeof(T) == 4) {
          const float4 av = *reinterpret_cast<const float4*>(&Ws[ii * WB + 4 * bg]);
          const float4 bv = *reinterpret_cast<const float4*>(&Is[ii * WC + 4 * cg]);
          a[0] = (T)av.x; a[1] = (T)av.y; a[2] = (T)av.z; a[3] = (T)av.w;
          bb[0] = (T)bv.x; bb[1] = (T)bv.y; bb[2] = (T)bv.z; bb[3] = (T)bv.w;
        } else {
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            a[x] = Ws[ii * WB + 4 * bg + x];
            bb[x] = Is[ii * WC + 4 * cg + x];
          }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * bb[y];
      }
    }
  }
  if (bg >= BG) return;
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int col = 4 * cg + y;
    if (col >= ncol) continue;
    const I item = it0 + (I)(col / J);
    if (item >= items) continue;
    const int j = col % J;
    const I p = item / Qi, q = item - p * Qi;
    T* out = (T*)c.out;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int b = 4 * bg + x;
      if (b >= c.NB) continue;
      const int64_t oi = (int64_t)p * c.osP + (int64_t)b * c.osB + (int64_t)q * c.osQ + (int64_t)j * c.osJ;
      const T v = (T)c.alpha * acc[x][y];
      out[oi] = c.accumulate ? out[oi] + v : v;
    }
  }
}

// Mode product, weight-stationary: W (NI x NB, NI <= 128, NB <= NBT) sits
// in shared memory; each thread owns one output column (an (item, j) pair)
// and all NB outputs of it in registers, streaming its NI inputs.
// out[p,b,q,j] (+)= alpha * sum_i W[i*wsI + b*wsB] * in[p,i,q,j].
constexpr int kWsMaxNI = 128;

template <int NBT, typename I>
__device__ void dev_mpw(const DevOp& op, int64_t blk, unsigned char* smem) {
  const Contract& c = op.c;
  float* Ws = (float*)smem;                 // [NI][NBT]
  const int NI = (int)c.NI, NB = (int)c.NB;
  const float* w = (const float*)c.w;
  for (int e = threadIdx.x; e < NI * NBT; e += kExecThreads) {
    const int i = e / NBT, b = e % NBT;
    Ws[e] = b < NB ? w[(int64_t)i * c.wsI + (int64_t)b * c.wsB] : 0.f;
  }
  __syncthreads();
  const I J = (I)c.J, Q = (I)c.Q;
  const I ncols = (I)(c.P * c.Q * c.J);
  const I col = (I)(blk * kExecThreads) + (I)threadIdx.x;
  if (col >= ncols) return;
  const I item = col / J, j = col - item * J;
  const I p = item / Q, q = item - p * Q;
  const float* in = (const float*)c.in + (int64_t)p * c.isP + (int64_t)q * c.isQ + (int64_t)j * c.isJ;
  float acc[NBT];
#pragma unroll
  for (int b = 0; b < NBT; ++b) acc[b] = 0.f;
  int i = 0;
  for (; i + 4 <= NI; i += 4) {
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = in[(int64_t)(i + u) * c.isI];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4* wr = reinterpret_cast<const float4*>(Ws + (i + u) * NBT);
#pragma unroll
      for (int b4 = 0; b4 < NBT / 4; ++b4) {
        const float4 wv = wr[b4];
        acc[4 * b4] += wv.x * x[u];
        acc[4 * b4 + 1] += wv.y * x[u];
        acc[4 * b4 + 2] += wv.z * x[u];
        acc[4 * b4 + 3] += wv.w * x[u];
      }
    }
  }
  for (; i < NI; ++i) {
    const float x = in[(int64_t)i * c.isI];
    const float4* wr = reinterpret_cast<const float4*>(Ws + i * NBT);
#pragma unroll
    for (int b4 = 0; b4 < NBT / 4; ++b4) {
      const float4 wv = wr[b4];
      acc[4 * b4] += wv.x * x;
      acc[4 * b4 + 1] += wv.y * x;
      acc[4 * b4 + 2] += wv.z * x;
      acc[4 * b4 + 3] += wv.w * x;
    }
  }
  float* out = (float*)c.out + (int64_t)p * c.osP + (int64_t)q * c.osQ + (int64_t)j * c.osJ;
  const float alpha = (float)c.alpha;
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    if (b < NB) {
      float* o = out + (int64_t)b * c.osB;
      *o = c.accumulate ? *o + alpha * acc[b] : alpha * acc[b];
    }
  }
}

// Long reduction of a mode product with few batch items (e.g. Y_t^T G_t over
// all rows of a node): block (item, split) sums its K slice of
// out[p,b,q,j] = sum_i W[i*wsI + b*wsB] in[p,i,q,j] through shared-memory
// tiles (coalesced loads) into partial[split][p][b][q][j].
constexpr int kKredTile = 64;

__device__ void dev_kred(const DevOp& op, int64_t blk, unsigned char* smem) {
  const Contract& c = op.c;
  const int NB = (int)c.NB, J = (int)c.J;
  const int64_t items = c.P * c.Q;
  const int64_t item = blk % items;
  const int64_t split = blk / items;
  const int64_t p = item / c.Q, q = item % c.Q;
  const int64_t i0 = split * op.chunk;
  const int64_t i1 = min(c.NI, i0 + op.chunk);
  float* Wt = (float*)smem;                    // [kKredTile][NB]
  float* It = Wt + kKredTile * 64;             // [kKredTile][J]
  const float* in = (const float*)c.in + p * c.isP + q * c.isQ;
  const float* w = (const float*)c.w;
  const int nout = NB * J;
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  for (int64_t t0 = i0; t0 < i1; t0 += kKredTile) {
    const int kc = (int)min((int64_t)kKredTile, i1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < kKredTile * NB; e += kExecThreads) {
      const int b = e / kKredTile, ii = e % kKredTile;   // consecutive threads: consecutive i
      Wt[ii * 64 + b] = ii < kc ? w[(t0 + ii) * c.wsI + (int64_t)b * c.wsB] : 0.f;
    }
    for (int e = threadIdx.x; e < kKredTile * J; e += kExecThreads) {
      const int ii = e / J, jj = e % J;                 // consecutive threads: consecutive j
      It[ii * J + jj] = ii < kc ? in[(t0 + ii) * c.isI + (int64_t)jj * c.isJ] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int o = threadIdx.x + k * kExecThreads;
      if (o < nout) {
        const int b = o / J, jj = o % J;
        float a = acc[k];
        for (int ii = 0; ii < kc; ++ii) a += Wt[ii * 64 + b] * It[ii * J + jj];
        acc[k] = a;
      }
    }
  }
  float* part = (float*)op.partial;
  const int64_t total = c.P * c.NB * c.Q * c.J;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o = threadIdx.x + k * kExecThreads;
    if (o < nout) {
      const int b = o / J, jj = o % J;
      part[split * total + ((p * c.NB + b) * c.Q + q) * c.J + jj] = acc[k];
    }
  }
}

// Split-K register-tiled contraction for long reductions (e.g. the
// Khatri-Rao contraction of all leading modes of a first-level product at
// once, or a TTN core against a sketch block):
//   out[p,b,q,j] (+)= alpha * sum_i W(i, b) in[p,i,q,j],
// with W(i, b) = w[i*wsI + b*wsB] or the Khatri-Rao product of the factors
// c.kr (nkr > 0).  Columns n = (p, q, j) are tiled kKgNT per block, the
// outputs b in groups of kKgMB (op.BG groups) and the reduction index in
// chunks of op.chunk: block = (tile, b group, split).  Each thread
// accumulates 8 (b) x 4 (n) outputs from shared-memory tiles of kKgKT rows,
// the next rows prefetched into registers.  Tiles are read column-wise
// (consecutive threads, consecutive columns: contiguous j) or, with op.CG = 1
// (J = Q = 1 and a contiguous reduction index), row-wise (16 consecutive i of
// a column per 16 threads).  With nsplit > 1 the block writes its partial
// sums [split][p][b][q][j], reduced in a fixed order (OP_REDUCE), else the
// outputs.
constexpr int kKgKT = 16, kKgNT = 256, kKgMB = 32;
constexpr int kKgLd = kKgNT + 4;               // padded tile row (row-wise stores: 2-way banks)
constexpr int kKgWPT = kKgKT * kKgMB / 256;   // weight-tile entries per thread
static_assert(kKgKT * kKgMB % 256 == 0 && kKgWPT >= 1, "weight tile must split over 256 threads");
static_assert(kKgKT == 16 && kKgNT == 256, "row-wise tile loads assume 16 x 256 tiles");

// W(i, b) of a split-K contraction; i < 2^31 (the recorder checks).
__device__ __forceinline__ float kg_weight(const Contract& c, int64_t i, int b) {
  if (c.nkr == 0) return ((const float*)c.w)[i * c.wsI + (int64_t)b * c.wsB];
  float v = 1.f;
  uint32_t rem = (uint32_t)i;
#pragma unroll
  for (int f = 3; f >= 0; --f) {
    if (f >= c.nkr) continue;
    const uint32_t n = (uint32_t)c.krn[f];
    const uint32_t q = rem / n;
    const uint32_t d = rem - q * n;
    rem = q;
    v *= ((const float*)c.kr[f])[(int64_t)d * c.wsI + (int64_t)b * c.wsB];
  }
  return v;
}

template <typename I>
__device__ void dev_kgemm(const DevOp& op, int64_t blk, unsigned char* smem) {
  const Contract& c = op.c;
  float* Ws = (float*)smem;                       // [kKgKT][kKgMB]
  float* Is = Ws + kKgKT * kKgMB;                 // [kKgKT][kKgLd]
  const int t = threadIdx.x;
  const int64_t ncols = c.P * c.Q * c.J;
  const int64_t ntile = (ncols + kKgNT - 1) / kKgNT;
  const int nbg = op.BG > 0 ? op.BG : 1;
  const int64_t tile = blk % ntile, rest = blk / ntile;
  const int b0 = (int)(rest % nbg) * kKgMB;
  const int64_t split = rest / nbg;
  const int64_t i0 = split * op.chunk;
  const int64_t i1 = min(c.NI, i0 + op.chunk);
  const int NB = (int)c.NB;
  const int NBg = min(kKgMB, NB - b0);
  const bool rows = op.CG == 1;
  // load role, column-wise: column t of the tile, all kKgKT rows of a step;
  // row-wise: row t % 16 of columns t / 16 + 16 u
  const int lc = rows ? t / kKgKT : t, lr = rows ? t % kKgKT : 0;
  const float* in = (const float*)c.in;
  int64_t lbase = 0;
  bool lval = false;
  if (rows) {
    lbase = (tile * kKgNT + lc) * c.isP;
  } else {
    const I ln = (I)(tile * kKgNT + lc);
    lval = (int64_t)ln < ncols;
    if (lval) {
      const I j = ln % (I)c.J, pq = ln / (I)c.J;
      const I q = pq % (I)c.Q, p = pq / (I)c.Q;
      lbase = (int64_t)p * c.isP + (int64_t)q * c.isQ + (int64_t)j * c.isJ;
    }
  }
  const int64_t rstep = (int64_t)(kKgNT / kKgKT) * c.isP;   // row-wise: 16 columns on
  const int64_t rcols = ncols - tile * kKgNT;                // row-wise: valid columns
  // compute role: outputs b in [8 bg, 8 bg + 8), columns [4 cg, 4 cg + 4)
  const int cg = t % 64, bg = t / 64;
  float acc[8][4];
#pragma unroll
  for (int x = 0; x < 8; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
  // the next step's rows are read into registers while this step computes
  constexpr int kRows = kKgKT * kKgNT / 256;      // tile entries each thread loads per step
  float ri[kRows], rw[kKgWPT];
#define KG_FETCH(k0_)                                                              \
  {                                                                                \
    const int nk_ = (int)min((int64_t)kKgKT, i1 - (k0_));                          \
    if (rows) {                                                                    \
      _Pragma("unroll") for (int u = 0; u < kRows; ++u)                            \
        ri[u] = (lr < nk_ && lc + u * (kKgNT / kKgKT) < rcols)                     \
                    ? in[lbase + u * rstep + (k0_) + lr] : 0.f;                    \
    } else {                                                                       \
      _Pragma("unroll") for (int u = 0; u < kRows; ++u)                            \
        ri[u] = (lval && u < nk_) ? in[lbase + ((k0_) + u) * c.isI] : 0.f;         \
    }                                                                              \
    _Pragma("unroll") for (int h = 0; h < kKgWPT; ++h) {                          \
      const int e_ = t + h * 256, kk_ = e_ / kKgMB, b_ = e_ % kKgMB;               \
      rw[h] = (b_ < NBg && kk_ < nk_) ? kg_weight(c, (k0_) + kk_, b0 + b_) : 0.f;  \
    }                                                                              \
  }
  if (i0 < i1) KG_FETCH(i0);
  for (int64_t k0 = i0; k0 < i1; k0 += kKgKT) {
    if (rows) {
#pragma unroll
      for (int u = 0; u < kRows; ++u) Is[lr * kKgLd + lc + u * (kKgNT / kKgKT)] = ri[u];
    } else {
#pragma unroll
      for (int u = 0; u < kRows; ++u) Is[u * kKgLd + lc] = ri[u];
    }
#pragma unroll
    for (int h = 0; h < kKgWPT; ++h) Ws[t + h * 256] = rw[h];
    __syncthreads();
    if (k0 + kKgKT < i1) KG_FETCH(k0 + kKgKT);
#pragma unroll
    for (int kk = 0; kk < kKgKT; ++kk) {
      const float4 w0 = *reinterpret_cast<const float4*>(&Ws[kk * kKgMB + 8 * bg]);
      const float4 w1 = *reinterpret_cast<const float4*>(&Ws[kk * kKgMB + 8 * bg + 4]);
      const float4 xv = *reinterpret_cast<const float4*>(&Is[kk * kKgLd + 4 * cg]);
#define KG_ROW(row_, w_)          \
  acc[row_][0] += (w_) * xv.x;    \
  acc[row_][1] += (w_) * xv.y;    \
  acc[row_][2] += (w_) * xv.z;    \
  acc[row_][3] += (w_) * xv.w;
      KG_ROW(0, w0.x) KG_ROW(1, w0.y) KG_ROW(2, w0.z) KG_ROW(3, w0.w)
      KG_ROW(4, w1.x) KG_ROW(5, w1.y) KG_ROW(6, w1.z) KG_ROW(7, w1.w)
#undef KG_ROW
    }
    __syncthreads();
  }
#undef KG_FETCH
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const I n = (I)(tile * kKgNT) + (I)(4 * cg + y);
    if ((int64_t)n >= ncols) continue;
    const I j = n % (I)c.J, pq = n / (I)c.J;
    const I q = pq % (I)c.Q, p = pq / (I)c.Q;
    // partial [split][p][b][q][j] or the output, at b = b0 + 8 bg
    const int64_t pbase = ((int64_t)split * c.P + p) * c.NB * c.Q * c.J + (int64_t)q * c.J + j;
    const int64_t pstep = c.Q * c.J;
    float* o = (float*)c.out + (int64_t)p * c.osP + (int64_t)q * c.osQ + (int64_t)j * c.osJ;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int b = b0 + 8 * bg + x;
      if (8 * bg + x >= NBg) continue;
      if (op.nsplit > 1) {
        ((float*)op.partial)[pbase + (int64_t)b * pstep] = acc[x][y];
      } else {
        float* ob = o + (int64_t)b * c.osB;
        const float v = (float)c.alpha * acc[x][y];
        *ob = c.accumulate ? *ob + v : v;
      }
    }
  }
}

template <typename I>
__device__ __forceinline__ I scatter_div(const Scatter& s, int a, I n) {
  if (sizeof(I) == 4) {
    const uint32_t r = (uint32_t)n;
    return (I)(uint32_t)(((uint64_t)__umulhi(r, s.mag[a]) + r) >> s.shf[a]);
  }
  return n / (I)s.size[a];
}

// Element e's offsets in `in` and `out` and its index on every scaled axis.
template <typename I>
__device__ __forceinline__ void scatter_decode(const Scatter& s, I e, int64_t* io, int64_t* oo,
                                               I* si) {
  int64_t ii = 0, o = 0;
  I rem = e;
  for (int a = s.nd - 1; a >= 0; --a) {
    const I q = scatter_div(s, a, rem);
    const I i = rem - q * (I)s.size[a];
    rem = q;
    ii += i * s.is[a];
    o += i * s.os[a];
#pragma unroll
    for (int k = 0; k < kMaxScales; ++k)
      if (k < s.nsc && s.scax[k] == a) si[k] = i;
  }
  *io = ii;
  *oo = o;
}

template <typename T, typename I>
__device__ void dev_scatter(const DevOp& op, int64_t blk) {
  const Scatter& s = op.s;
  I total = 1;
  for (int a = 0; a < s.nd; ++a) total *= (I)s.size[a];
  // op.chunk elements per thread, kExecThreads apart: after the first, a
  // step stays on the last axis' row while it can (no full decode)
  const int L = s.nd - 1;
  const I nl = (I)s.size[L];
  const int64_t isl = s.is[L], osl = s.os[L];
  int lk = -1;   // the scale on the last axis, if any
  for (int k = 0; k < s.nsc; ++k)
    if (s.scax[k] == L) lk = k;
  I e = (I)(blk * op.chunk * kExecThreads) + (I)threadIdx.x;
  if (e >= total) return;
  int64_t io, oo;
  I si[kMaxScales];
#pragma unroll
  for (int k = 0; k < kMaxScales; ++k) si[k] = 0;
  scatter_decode(s, e, &io, &oo, si);
  I il = e - scatter_div(s, L, e) * nl;
  const T* in = (const T*)s.in;
  T* out = (T*)s.out;
  for (int it = 0;;) {
    T v = in[io];
#pragma unroll
    for (int k = 0; k < kMaxScales; ++k)
      if (k < s.nsc) v *= ((const T*)s.sc[k])[si[k]];
    if (s.assign) out[oo] = (T)s.alpha * v;
    else out[oo] = out[oo] + (T)s.alpha * v;
    if (++it == op.chunk) return;
    e += (I)kExecThreads;
    if (e >= total) return;
    il += (I)kExecThreads;
    if (il < nl) {
      io += (int64_t)kExecThreads * isl;
      oo += (int64_t)kExecThreads * osl;
      if (lk >= 0) {
#pragma unroll
        for (int k = 0; k < kMaxScales; ++k)
          if (k == lk) si[k] = il;
      }
    } else {
      scatter_decode(s, e, &io, &oo, si);
      il = e - scatter_div(s, L, e) * nl;
    }
  }
}

__device__ void dev_proj(const DevOp& op, int64_t blk) {
  const Proj& m = op.pj;
  const int64_t e = blk * kExecThreads + threadIdx.x;
  if (e >= (int64_t)m.nq * m.ncols) return;
  const int q = (int)(e / m.ncols), j = (int)(e % m.ncols);
  const double* a = m.a + (int64_t)(m.q0 + q) * m.saq;
  double acc = 0.0;
  if (!m.F) {
    acc = a[(int64_t)j * m.sak];
  } else {
    const double* F = m.F + j;
    for (int64_t k = 0; k < m.n; ++k) acc += F[k * m.ldF] * a[k * m.sak];
  }
  if (m.has_w) acc *= m.w[q];
  m.out[(int64_t)q * m.ldo + j] = acc;
}

__device__ void dev_outer(const DevOp& op, int64_t blk) {
  const Outer& m = op.ou;
  int64_t total = 1;
  for (int a = 0; a < m.A; ++a) total *= m.n[a];
  const int64_t e = blk * kExecThreads + threadIdx.x;
  if (e >= total) return;
  int64_t idx[kOuterAxes];
  int64_t rem = e, oo = 0;
  for (int a = m.A - 1; a >= 0; --a) {
    idx[a] = rem % m.n[a];
    rem /= m.n[a];
    oo += idx[a] * m.os[a];
  }
  int64_t xo[kOuterVecs];
  for (int k = 0; k < m.K; ++k) xo[k] = ((idx[m.ax[k]] / m.dv[k]) % m.md[k]) * m.si[k];
  double acc = 0.0;
  for (int q = 0; q < m.Q; ++q) {
    double t = 1.0;
    for (int k = 0; k < m.K; ++k) t *= m.v[k][(int64_t)q * m.sq[k] + xo[k]];
    acc += t;
  }
  if (m.out_f64) ((double*)m.out)[oo] += m.alpha * acc;
  else ((float*)m.out)[oo] += (float)(m.alpha * acc);
}

__device__ void dev_eye(const DevOp& op, int64_t blk) {
  const int64_t n = op.eye_n;
  const int64_t e = blk * kExecThreads + threadIdx.x;
  if (e < n * n) ((double*)op.c.out)[e] = (e / n == e % n) ? 1.0 : 0.0;
}

template <typename I>
__device__ __forceinline__ void dispatch(const DevOp& op, int64_t blk, unsigned char* dsm) {
  switch (op.kind) {
    case OP_CONTRACT:
      if (op.tin == ET_F32 && op.tw == ET_F32 && op.tout == ET_F32)
        dev_contract<float, float, float, float, I>(op, blk);
      else if (op.tin == ET_F64 && op.tout == ET_F64 && op.tw == ET_F64)
        dev_contract<double, double, double, double, I>(op, blk);
      else
        dev_contract<float, double, double, double, I>(op, blk);
      break;
    case OP_MP:
      if (op.CG == 0) {   // weight-stationary variant, NBT = op.BG
        switch (op.BG) {
          case 8: dev_mpw<8, I>(op, blk, dsm); break;
          case 16: dev_mpw<16, I>(op, blk, dsm); break;
          default: dev_mpw<32, I>(op, blk, dsm); break;
        }
      } else if (op.tout == ET_F64) {
        dev_mp<double, I>(op, blk, dsm);
      } else {
        dev_mp<float, I>(op, blk, dsm);
      }
      break;
    case OP_SCATTER:
      if (op.tout == ET_F64) dev_scatter<double, I>(op, blk);
      else dev_scatter<float, I>(op, blk);
      break;
    case OP_REDUCE:
      if (op.tout == ET_F64) dev_reduce<double, I>(op, blk);
      else dev_reduce<float, I>(op, blk);
      break;
    case OP_EYE:
      dev_eye(op, blk);
      break;
    case OP_KRED:
      dev_kred(op, blk, dsm);
      break;
    case OP_PROJ:
      dev_proj(op, blk);
      break;
    case OP_OUTER:
      dev_outer(op, blk);
      break;
    default:
      break;
  }
}

__global__ void __launch_bounds__(kExecThreads, 3) level_kernel(const __grid_constant__ LevelBatch lb) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int64_t b = blockIdx.x;
  int lo = 0, hi = lb.nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (lb.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const DevOp& op = lb.ops[lo];
  const int64_t blk = b - lb.start[lo];
  if (op.idx32) dispatch<uint32_t>(op, blk, dsm);
  else dispatch<int64_t>(op, blk, dsm);
}

// The split-K GEMM ops of a level in a kernel of their own: its code stays
// small enough for the instruction caches (the generic level kernel's many op
// kinds do not, and its ops stall on instruction fetch).
// MINB resident blocks per SM: 2 (128 registers) for levels of a few waves,
// 3 (80 registers) for levels of many waves, where the extra warps hide more
// shared-memory latency and the coarser last wave costs little.
template <int MINB>
__global__ void __launch_bounds__(kExecThreads, MINB) kgemm_level_kernel(const __grid_constant__ LevelBatch lb) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int64_t b = blockIdx.x;
  int lo = 0, hi = lb.nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (lb.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const DevOp& op = lb.ops[lo];
  const int64_t blk = b - lb.start[lo];
  // one instantiation (64-bit column decoding: a few divisions per thread)
  dev_kgemm<int64_t>(op, blk, dsm);
}

// ---------------------------------------------------------------------------
// host parts
// ---------------------------------------------------------------------------
static bool mp_tiling(Op& op) {
  const Contract& c = op.c;
  if (!c.w || c.wsQ != 0 || c.wsJ != 0 || c.wsP != 0 || c.NI < 8 || c.NB > 64) return false;
  if (!(op.tin == op.tw && op.tw == op.tout)) return false;
  if (op.tout == ET_F64) return false;    // few FP64 units per SM: spread FP64 work thin instead
  if (c.P * c.Q * c.NB * c.J < 8192) return false;
  if (c.NI <= kWsMaxNI && c.NB <= 32) {
    // at most 32 outputs per thread (3 resident blocks per SM; wider weights
    // take the tiled form below)
    const int nbt = c.NB <= 8 ? 8 : c.NB <= 16 ? 16 : 32;
    op.kind = OP_MP;
    op.BG = nbt;
    op.CG = 0;
    op.CH = 0;
    op.blocks = ceil_div(c.P * c.Q * c.J, kExecThreads);
    return true;
  }
  int bg = (int)((c.NB + 3) / 4), p2 = 1;
  while (p2 < bg) p2 <<= 1;
  const int cg = std::min(kExecThreads / p2, 64);   // smem kMpKC2*4*(BG+CG)*4 <= 48 KB
  if (c.J > 4 * cg) return false;
  op.BG = p2;
  op.CG = cg;
  op.CH = (int)(4 * cg / c.J);
  const int64_t items = c.P * c.Q;
  op.blocks = ceil_div(items, op.CH);
  op.kind = OP_MP;
  return true;
}

int64_t plan_contract(Op& op) {
  op.kind = OP_CONTRACT;
  const Contract& c = op.c;
  const int64_t total = c.P * c.NB * c.Q * c.J;
  if (total == 0) {
    op.blocks = 0;
    return 0;
  }
  // split-K tiled form: b groups of kKgMB, long reductions split until the
  // blocks fill the GPU twice over (at least 64 reduction rows each)
  auto kgemm = [&]() -> int64_t {
    const int64_t ntile = ceil_div(c.P * c.Q * c.J, (int64_t)kKgNT);
    const int64_t nbg = ceil_div(c.NB, (int64_t)kKgMB);
    const int64_t want = (int64_t)exec_sms() * 2;
    // short reductions stay whole (the partial sums and their reduction
    // would cost more than the extra blocks gain)
    int64_t ns = c.NI < 1024 ? 1
                 : std::max<int64_t>(1, std::min<int64_t>(ceil_div(want, ntile * nbg), c.NI / 64));
    op.chunk = round_up(ceil_div(c.NI, ns), (int64_t)kKgKT);
    op.nsplit = (int)ceil_div(c.NI, op.chunk);
    op.kind = OP_KGEMM;
    op.BG = (int)nbg;
    // row-wise tile loads: one column per (p), contiguous reduction index
    op.CG = (c.J == 1 && c.Q == 1 && c.isI == 1 && c.P > 1) ? 1 : 0;
    op.blocks = ntile * nbg * op.nsplit;
    return op.nsplit > 1 ? total * op.nsplit : 0;
  };
  if (c.nkr > 0) {
    // Khatri-Rao weights exist only in the split-K tiled form (binary32,
    // NB <= kKgMB, weights independent of p, q, j: the recorder checks)
    return kgemm();
  }
  // long reductions with few outputs: split-K through shared-memory tiles
  if (c.w && c.wsQ == 0 && c.wsJ == 0 && c.wsP == 0 && op.tin == ET_F32 && op.tw == ET_F32 &&
      op.tout == ET_F32 && c.NI >= 2048 && c.NB <= 64 && c.J <= 64 &&
      c.NB * c.J <= 16 * kExecThreads && c.P * c.Q <= 64) {
    const int64_t items = c.P * c.Q;
    const int64_t want = (int64_t)exec_sms() * 4;
    int64_t ns = std::max<int64_t>(1, std::min<int64_t>(ceil_div(want, items), c.NI / kKredTile));
    op.chunk = round_up(ceil_div(c.NI, ns), kKredTile);
    op.nsplit = (int)ceil_div(c.NI, op.chunk);
    op.kind = OP_KRED;
    op.blocks = items * op.nsplit;
    return total * op.nsplit;
  }
  // the tiled and weight-stationary mode products give each thread many
  // outputs: for small ops that leaves most SMs idle while a few blocks run
  // long; there one lane group per output spreads the work instead
  const int64_t want = (int64_t)exec_sms() * 1024;   // threads that keep the GPU busy
  // binary32 mode products with reductions longer than the weight-stationary
  // form holds (e.g. a rank-200 TTN core against a sketch block) take the
  // split-K tiled form
  if (total >= want / 4 && c.w && c.wsQ == 0 && c.wsJ == 0 && c.wsP == 0 && c.NI > kWsMaxNI &&
      c.NI < (int64_t(1) << 31) && op.tin == ET_F32 && op.tw == ET_F32 && op.tout == ET_F32)
    return kgemm();
  if (total >= want / 4 && mp_tiling(op)) return 0;
  int g = 1;
  while (g < 32 && total * g < want && c.NI >= 8 * g) g <<= 1;
  op.g = g;
  op.nsplit = 1;
  op.chunk = c.NI;
  if (c.NI >= 2048 && total * g < want) {
    int64_t ns = std::min<int64_t>(ceil_div(want, total * g), c.NI / 512);
    ns = std::max<int64_t>(1, std::min<int64_t>(ns, 256));
    op.chunk = ceil_div(c.NI, ns);
    op.nsplit = (int)ceil_div(c.NI, op.chunk);
  }
  op.blocks = ceil_div(total * op.nsplit, kExecThreads / g);
  return op.nsplit > 1 ? total * op.nsplit : 0;
}

void plan_simple(Op& op) {
  int64_t total = 0;
  if (op.kind == OP_SCATTER) {
    total = 1;
    for (int a = 0; a < op.s.nd; ++a) total *= op.s.size[a];
    // large scatters: several elements per thread (fewer, fuller blocks)
    op.chunk = total >= (int64_t)exec_sms() * kExecThreads * 32 ? 8 : 1;
    op.blocks = ceil_div(total, (int64_t)kExecThreads * op.chunk);
    return;
  } else if (op.kind == OP_EYE) {
    total = op.eye_n * op.eye_n;
  } else if (op.kind == OP_REDUCE) {
    total = op.c.P * op.c.NB * op.c.Q * op.c.J;
  } else if (op.kind == OP_PROJ) {
    total = (int64_t)op.pj.nq * op.pj.ncols;
  } else if (op.kind == OP_OUTER) {
    total = 1;
    for (int a = 0; a < op.ou.A; ++a) total *= op.ou.n[a];
  }
  op.blocks = ceil_div(total, kExecThreads);
}

void Program::buffer(const void* p, int64_t bytes, int level) {
  if (!p || bytes <= 0) return;
  bufs_.push_back(Buf{(const char*)p, (const char*)p + bytes, level});
}

int Program::level_of(const void* p) const {
  if (!p) return 0;
  const char* c = (const char*)p;
  int lvl = 0;
  for (const Buf& b : bufs_)
    if (c >= b.lo && c < b.hi) lvl = std::max(lvl, b.level);
  return lvl;
}

void Program::add(Op op, const void* in1, const void* in2) {
  const int lvl = 1 + std::max(level_of(in1), level_of(in2));
  const void* out = op.kind == OP_SCATTER ? op.s.out
                    : op.kind == OP_PROJ  ? (const void*)op.pj.out
                    : op.kind == OP_OUTER ? op.ou.out
                                          : op.c.out;
  if (((op.kind == OP_CONTRACT || op.kind == OP_KGEMM) && op.nsplit > 1) || op.kind == OP_KRED) {
    Op part = op;
    part.level = lvl;
    ops_.push_back(part);
    Op red = op;
    red.kind = OP_REDUCE;
    red.level = lvl + 1;
    plan_simple(red);
    ops_.push_back(red);
    for (Buf& b : bufs_)
      if ((const char*)out >= b.lo && (const char*)out < b.hi) b.level = std::max(b.level, lvl + 1);
    return;
  }
  op.level = lvl;
  ops_.push_back(op);
  for (Buf& b : bufs_)
    if ((const char*)out >= b.lo && (const char*)out < b.hi) b.level = std::max(b.level, lvl);
}

int Program::levels() const {
  int m = 0;
  for (const Op& o : ops_) m = std::max(m, o.level);
  return m;
}

static DevOp to_dev(const Op& o) {
  DevOp d;
  memset(&d, 0, sizeof(d));
  d.kind = o.kind;
  d.tin = o.tin;
  d.tw = o.tw;
  d.tout = o.tout;
  d.c = o.c;
  if (o.kind == OP_PROJ) d.pj = o.pj;
  else if (o.kind == OP_OUTER) d.ou = o.ou;
  else d.s = o.s;
  d.g = o.g;
  d.nsplit = o.nsplit;
  d.chunk = o.chunk;
  d.partial = o.partial;
  d.BG = o.BG;
  d.CG = o.CG;
  d.CH = o.CH;
  d.eye_n = o.eye_n;
  // 32-bit decoding when every extent and count stays below 2^31
  const int64_t lim = (int64_t(1) << 31) - 1;
  int64_t m = o.c.P * o.c.NB * o.c.Q * o.c.J * std::max(o.nsplit, 1);
  if (o.kind == OP_SCATTER) {
    int64_t st = 1;
    for (int a = 0; a < o.s.nd; ++a) st *= std::max<int64_t>(o.s.size[a], 1);
    m = std::max(m, st + (int64_t)kExecThreads * std::max<int64_t>(o.chunk, 1));
  }
  m = std::max(m, o.eye_n * o.eye_n);
  m = std::max(m, o.blocks * kExecThreads);
  d.idx32 = m < lim;
  return d;
}

// A second stream per host thread and device for the split-K GEMM launches
// of a level, forked from and joined back into the caller's stream (so the
// two kernels of a level overlap; each thread keeps its own, so concurrent
// callers never wait on one another's work).
struct ForkStream {
  int device = -1;
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

static ttnn_status fork_stream(ForkStream** out) {
  thread_local ForkStream fs[8];
  int dev = 0;
  TTNN_TRY_CUDA(cudaGetDevice(&dev));
  ForkStream* f = nullptr;
  for (auto& x : fs)
    if (x.device == dev) f = &x;
  if (!f) {
    for (auto& x : fs)
      if (x.device < 0) {
        f = &x;
        break;
      }
    if (!f) {
      *out = nullptr;   // more devices than slots: run the level's kernels in order
      return TTNN_OK;
    }
    TTNN_TRY_CUDA(cudaStreamCreateWithFlags(&f->st, cudaStreamNonBlocking));
    TTNN_TRY_CUDA(cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming));
    TTNN_TRY_CUDA(cudaEventCreateWithFlags(&f->join, cudaEventDisableTiming));
    f->device = dev;
  }
  *out = f;
  return TTNN_OK;
}

ttnn_status Program::run(cudaStream_t st, bool dump) {
  const int L = levels();
  // per level: the split-K GEMM ops in one launch of their kernel, every
  // other op in one level_kernel launch; when a level has both, the GEMM
  // launch goes on the fork stream and runs beside the other
  ForkStream* fs = nullptr;
  LevelBatch lb[2];
  cudaStream_t gst = st;   // stream of the GEMM launches
  auto flush = [&](int k) -> ttnn_status {
    LevelBatch& b = lb[k];
    if (b.nops == 0) return TTNN_OK;
    const int64_t blocks = b.start[b.nops];
    if (blocks > 0) {
      if (blocks >= (int64_t(1) << 31)) {
        set_error("program level too large");
        return TTNN_EUNSUPPORTED;
      }
      if (k == 0) {
        // at least three full waves at three blocks per SM: the 80-register form
        if (blocks >= 9 * (int64_t)exec_sms())
          kgemm_level_kernel<3><<<(unsigned)blocks, kExecThreads, kExecSmem, gst>>>(b);
        else
          kgemm_level_kernel<2><<<(unsigned)blocks, kExecThreads, kExecSmem, gst>>>(b);
        TTNN_TRY(check_launch("kgemm_level_kernel"));
      } else {
        level_kernel<<<(unsigned)blocks, kExecThreads, kExecSmem, st>>>(b);
        TTNN_TRY(check_launch("level_kernel"));
      }
    }
    b.nops = 0;
    return TTNN_OK;
  };
  for (int lvl = 1; lvl <= L; ++lvl) {
    for (int k = 0; k < 2; ++k) {
      lb[k].nops = 0;
      lb[k].start[0] = 0;
    }
    bool has[2] = {false, false};
    for (const Op& o : ops_)
      if (o.level == lvl && o.blocks > 0) has[o.kind == OP_KGEMM ? 0 : 1] = true;
    gst = st;
    if (has[0] && has[1] && !dump) {
      if (!fs) TTNN_TRY(fork_stream(&fs));
      if (fs) {
        TTNN_TRY_CUDA(cudaEventRecord(fs->fork, st));
        TTNN_TRY_CUDA(cudaStreamWaitEvent(fs->st, fs->fork, 0));
        gst = fs->st;
      }
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (const Op& o : ops_) {
        if (o.level != lvl || o.blocks == 0) continue;
        const int k = o.kind == OP_KGEMM ? 0 : 1;
        if (k != pass) continue;
        LevelBatch& b = lb[k];
        if (dump) {
          // debugging: each op alone, timed (the stream is synchronised)
          cudaEvent_t a = nullptr, e = nullptr;
          TTNN_TRY_CUDA(cudaEventCreate(&a));
          TTNN_TRY_CUDA(cudaEventCreate(&e));
          b.ops[0] = to_dev(o);
          b.start[0] = 0;
          b.start[1] = o.blocks;
          b.nops = 1;
          TTNN_TRY_CUDA(cudaEventRecord(a, st));
          TTNN_TRY(flush(k));
          TTNN_TRY_CUDA(cudaEventRecord(e, st));
          TTNN_TRY_CUDA(cudaEventSynchronize(e));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, a, e);
          cudaEventDestroy(a);
          cudaEventDestroy(e);
          fprintf(stderr, "[ttnn] %8.1f us  ", ms * 1e3f);
          if (o.kind == OP_SCATTER)
            fprintf(stderr, "[ttnn] L%d scatter nd %d nsc %d blocks %lld\n", lvl, o.s.nd, o.s.nsc,
                    (long long)o.blocks);
          else
            fprintf(stderr,
                    "[ttnn] L%d kind %d P %lld NI %lld NB %lld Q %lld J %lld isJ %lld wsJ %lld "
                    "wsQ %lld wsP %lld g %d nsplit %d blocks %lld\n",
                    lvl, (int)o.kind, (long long)o.c.P, (long long)o.c.NI, (long long)o.c.NB,
                    (long long)o.c.Q, (long long)o.c.J, (long long)o.c.isJ, (long long)o.c.wsJ,
                    (long long)o.c.wsQ, (long long)o.c.wsP, o.g, o.nsplit, (long long)o.blocks);
          continue;
        }
        if (b.nops == kMaxLevelOps) TTNN_TRY(flush(k));
        b.ops[b.nops] = to_dev(o);
        b.start[b.nops + 1] = b.start[b.nops] + o.blocks;
        ++b.nops;
      }
      TTNN_TRY(flush(pass));
    }
    if (gst != st) {
      TTNN_TRY_CUDA(cudaEventRecord(fs->join, gst));
      TTNN_TRY_CUDA(cudaStreamWaitEvent(st, fs->join, 0));
    }
  }
  return TTNN_OK;
}

}  // namespace ttnn
