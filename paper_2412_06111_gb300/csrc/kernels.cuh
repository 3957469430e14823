// Launch wrappers of the library's device kernels (defined in *.cu).
#pragma once

#include "common.cuh"

namespace ttnn {

// Generic strided contraction ("walk" op), one output element per thread:
//   out[p,b,q,j] (+)= alpha * sum_{i<NI} in[p*isP+i*isI+q*isQ+j*isJ]
//                                  * W[i*wsI+b*wsB+q*wsQ+j*wsJ]
// with out at p*osP+b*osB+q*osQ+j*osJ.  W == nullptr means W = 1.  When
// `partial` is given the sum over i is split into nsplit chunks that are
// reduced in a fixed order (deterministic).
struct Contract {
  int64_t P = 1, NI = 1, NB = 1, Q = 1, J = 1;
  int64_t isP = 0, isI = 0, isQ = 0, isJ = 0;
  int64_t wsI = 0, wsB = 0, wsQ = 0, wsJ = 0;
  int64_t wsP = 0;   // weight stride over the prefix index (a sketch axis shared from before)
  int64_t osP = 0, osB = 0, osQ = 0, osJ = 0;
  const void* in = nullptr;
  const void* w = nullptr;
  void* out = nullptr;
  double alpha = 1.0;
  int accumulate = 0;
  // Khatri-Rao weight (nkr > 0, w == nullptr; binary32 walk ops only):
  // W(i, b) = prod_f kr[f][d_f * wsI + b * wsB] where (d_0, .., d_{nkr-1})
  // are the digits of i in the mixed radix krn (d_0 slowest): the columns of
  // several per-mode factors multiplied entrywise, never materialised.
  int nkr = 0;
  int32_t krn[4] = {0, 0, 0, 0};
  const void* kr[4] = {nullptr, nullptr, nullptr, nullptr};
};

// element type codes for the contraction
enum ElemType { ET_F32 = 0, ET_F64 = 1 };

// Launches the contraction: (in, w, out, accumulation) types
// (f32,f32,f32,f32), (f64,f64,f64,f64), (f32,f64,f64,f64).
ttnn_status launch_contract(const Contract& c, ElemType tin, ElemType tw, ElemType tout,
                            void* partial, int64_t partial_elems, cudaStream_t st);
// Workspace elements (of the output type) the contraction needs for split-K.
int64_t contract_partial_elems(const Contract& c);

// SIMT GEMM C[i][j] (+)= alpha * sum_k A(i,k) B(j,k), A(i,k) = A[i*asi+k*ask],
// B(j,k) = B[j*bsj+k*bsk]; C row-major with leading dimension ldc.
// Input types: 0 = f64, 1 = f32, 2 = bf16; accumulation f64 for f64 inputs,
// f32 otherwise; C has the accumulation type.  Split-K over `nsplit` chunks
// writes partials [nsplit][I][ldc] to `partial` and reduces in order.
struct Gemm {
  int64_t I = 0, Jn = 0, K = 0;
  int64_t asi = 0, ask = 0, bsj = 0, bsk = 0, ldc = 0;
  const void* A = nullptr;
  const void* B = nullptr;
  void* C = nullptr;
  int in_type = 1;
};
ttnn_status launch_gemm(const Gemm& g, int nsplit, void* partial, cudaStream_t st);
int gemm_choose_split(const Gemm& g);

// DRM kernels
ttnn_status launch_philox(uint64_t seed, int kind, int ident, int64_t rows, int64_t cols,
                          int round_fmt, double* dst, cudaStream_t st);
ttnn_status launch_convert_f64_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st);
// Up to kConvertSegs binary64 -> binary32 copies (dst[k][e] = (float)src[k][e],
// e < n[k]) in one launch; start / pairs are filled by the launcher.
constexpr int kConvertSegs = 64;
struct ConvertBatch {
  int count = 0;
  const double* src[kConvertSegs];
  float* dst[kConvertSegs];
  int64_t n[kConvertSegs];
  int64_t start[kConvertSegs];
  int pairs[kConvertSegs];
};
ttnn_status launch_convert_batch(const ConvertBatch& batch, cudaStream_t st);

// Side (pass DRM) block: out[col][row] for col < w, row < nrows (leading dim
// ld_out >= nrows), in the pass storage format (0 f64, 1 f32, 2 bf16, 3 e4m3).
// Column c of the block is described by a SideCol: a Khatri-Rao product of
// per-mode factor columns (kr), a Kronecker/identity column (ident), or zero.
struct SideSpec {
  int nmodes = 0;                 // modes of the side (row index = row-major over them)
  int64_t ext[8] = {0};           // extents of the box on these modes
  int64_t off[8] = {0};           // box offsets on these modes
  int64_t full[8] = {0};          // full mode sizes (identity blocks)
  const double* xf[8] = {nullptr};   // X factor of each mode (n_mu x rmax, f64)
  const double* yf[8] = {nullptr};   // Y factor of each mode (n_mu x smax, f64)
  int rmax = 0, smax = 0;
  int x_cols = 0;                 // columns [0, x_cols): kr of X
  int y_cols = 0;                 // next y_cols: kr of Y (y_kind 0) or identity (y_kind 1)
  int y_kind = 0;
  int total_cols = 0;             // padded width (zero columns after)
  int round_fmt = 0;              // rounding of the exact f64 product
  int store = 1;                  // 0 f64, 1 f32, 2 bf16, 3 e4m3
  int64_t ld = 0;                 // leading dim (>= rows)
};
ttnn_status launch_side(const SideSpec& s, void* out, cudaStream_t st);
// The side block of a box cut from the whole-tensor block `src` (the same
// values: a gather of the box's rows); src is [total_cols][prod full] with
// leading dimension src_ld, in the storage format s.store.
ttnn_status launch_side_gather(const SideSpec& s, const void* src, int64_t src_ld, void* out,
                               cudaStream_t st);
// Many such gathers (possibly of different plans and formats) in few launches.
struct GatherJob {
  SideSpec s;
  const void* src = nullptr;
  int64_t src_ld = 0;
  void* out = nullptr;
};
ttnn_status launch_side_gather_batch(const GatherJob* jobs, int n, cudaStream_t st);

// Pass products of a box whose other side is a single index (every mode of
// that side fixed): the product against the fixed side is rank one and is
// left to the walk as a broadcast, and the product against this side is a
// matrix-vector product with the side block.
//   D[c] = sum_row m[row] * B[c][map(row)]   (c < cols; zero up to cols_pad)
// m: the box's rows (format m_store: 0 f64, 1 f32, 2 bf16, kStoreSplit,
// kStoreFp8 with `scale`); B: a side
// block [cols][...] with leading dimension src_ld in format s.store; map(row)
// is the row's place in a whole-tensor block (s.ext/off/full) when `cut`,
// else the row itself.  Accumulates in the walk type (f64 when d_f64) per
// block of rows, then sums the block partials in a fixed order
// (deterministic).  With dry, only reports the scratch bytes (`need`).
// Row formats of launch_side_gemv / launch_to_walk beyond the storage codes
// 0 f64, 1 f32, 2 bf16: binary32 rows sketched as bf16 hi + lo (BF16x2
// plans), and E4M3 rows with one binary32 scale per 128 consecutive rows,
// sketched as bf16(f32(q) * s) (E4M3 plans; `scale` required).
constexpr int kStoreFp8 = 3, kStoreSplit = 4;
ttnn_status launch_side_gemv(const SideSpec& s, const void* src, int64_t src_ld, bool cut,
                             const void* m, int m_store, const float* scale, int64_t rows,
                             int cols, int cols_pad, void* D, int d_f64, void* part,
                             int64_t part_bytes, cudaStream_t st, bool dry, int64_t* need);
// dst[e] = the value sketched for src[e] (format src_store as above) in the
// walk type (f32, or f64 when d_f64) for e < n.
ttnn_status launch_to_walk(const void* src, int src_store, const float* scale, void* dst,
                           int d_f64, int64_t n, cudaStream_t st);

// misc
ttnn_status launch_fill_zero(void* p, int64_t bytes, cudaStream_t st);
ttnn_status launch_axpy(void* y, const void* x, double alpha, int64_t n, int is_f64, cudaStream_t st);
ttnn_status launch_eye(double* dst, int64_t n, cudaStream_t st);

// Recovery (binary64): for each job, QR of Omega (s x r, state type) into
// Q (s x r) with diag R >= 0, one-sided Jacobi SVD of R and the
// eps-pseudo-inverse Rp (r x r); kept rank to kept[job].
struct QrJob {
  const void* omega;
  double* q;
  double* rp;
  int s, r;
};
ttnn_status launch_qr_pinv(const QrJob* jobs_dev, int njobs, int rmax, int state_f64,
                           double eps_factor, double u, int* kept_dev, int trunc,
                           cudaStream_t st);
// Copies the assembled (rank-padded) cores into their eps-truncated shapes:
// per node, the entries whose every index lies below its axis' kept rank,
// row-major and compact, from src + off to dst + off.  Axis a of a node keeps
// kept[job[a]] entries (job[a] >= 0) or all of full[a] (job[a] < 0).
struct CompactNode {
  int64_t off = 0;
  int ndim = 0;
  int32_t full[10] = {0};
  int32_t job[10] = {0};
};
constexpr int kCompactNodes = 32;
struct CompactBatch {
  int n = 0;
  const double* src = nullptr;
  double* dst = nullptr;
  const int* kept = nullptr;
  CompactNode nd[kCompactNodes];
};
ttnn_status launch_compact_cores(const CompactBatch& b, int64_t max_elems, cudaStream_t st);
constexpr int kMaxRecoverS = 128;
constexpr int kMaxRecoverR = 64;

}  // namespace ttnn

namespace ttnn {
constexpr int kMaxScales = 8;
// out[sum_a i_a * os_a] += alpha * v (or = alpha * v with `assign`) over
// the box of sizes `size` (up to 12 axes, last fastest), where
// v = in[sum_a i_a * is_a] * prod_k sc_k[i_{scax_k}]: scale k is a vector
// along axis scax_k.  in / out / scales share one type (f32 / f64).  The scales are
// rows of the DRM factors of modes a box fixes (X_mu[c, :] on the column
// axis, Y_mu[c, :] on a sketch axis), applied here instead of contracting
// an extent-1 mode over a whole intermediate.
struct Scatter {
  int nd = 0, nsc = 0, assign = 0;
  int32_t size[12] = {0};
  int64_t is[12] = {0}, os[12] = {0};
  // division by size[a] as a multiply-high and shift (32-bit indices)
  uint32_t mag[12] = {0};
  uint8_t shf[12] = {0};
  int8_t scax[kMaxScales] = {0};   // axis of each scale
  const void* sc[kMaxScales] = {nullptr};
  const void* in = nullptr;
  void* out = nullptr;
  double alpha = 1.0;
};

// Multiplier and shift that divide any 32-bit unsigned n by d (1 <= d < 2^31)
// as q = (umulhi(n, mag) + n) >> shf, the sum taken in 64 bits (division by
// invariant integers, Granlund and Montgomery 1994: l = ceil(log2 d),
// mag = floor(2^32 (2^l - d) / d) + 1).
inline void div_magic(uint32_t d, uint32_t* mag, uint8_t* shf) {
  int l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  *mag = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  *shf = (uint8_t)l;
}
}  // namespace ttnn
