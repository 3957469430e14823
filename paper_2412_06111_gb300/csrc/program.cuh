// Small-contraction programs: the tree walk of an update and the core
// assembly of a recovery are recorded as lists of ops with buffer
// dependencies, grouped by dependency level, and each level runs as one
// batched launch of a kernel that dispatches per block on the op kind.
#pragma once

#include <vector>

#include "kernels.cuh"

namespace ttnn {

enum OpKind {
  OP_CONTRACT = 0, OP_MP = 1, OP_SCATTER = 2, OP_REDUCE = 3, OP_EYE = 4, OP_KRED = 5,
  OP_PROJ = 6,    // projections of CP factors onto DRM factors (binary64)
  OP_OUTER = 7,   // sums of outer products of vector products into a sketch
  OP_KGEMM = 8    // split-K register-tiled contraction (long reduction, <= 32 outputs per column)
};

// OP_PROJ:  out[q * ldo + j] = w_q * sum_{k < n} F[k * ldF + j] * a[k * sak + (q0 + q) * saq]
// for q < nq, j < ncols (w_q = 1 when has_w == 0); with F == NULL it copies
// out[q * ldo + j] = w_q * a[j * sak + (q0 + q) * saq].
constexpr int kProjQ = 16;
struct Proj {
  const double* F;
  const double* a;
  double* out;
  int64_t n;
  int ldF, ncols, sak, saq, q0, nq, ldo, has_w;
  double w[kProjQ];
};

// OP_OUTER:  out[sum_a i_a * os_a] += alpha * sum_{q < Q} prod_k v_k[q * sq_k + x_k * si_k]
// with x_k = (i_{ax_k} / dv_k) % md_k: vector k is indexed by a digit of
// output axis ax_k (a Kronecker factor of that axis).
constexpr int kOuterVecs = 16;
constexpr int kOuterAxes = 10;
struct Outer {
  const double* v[kOuterVecs];
  int sq[kOuterVecs], si[kOuterVecs], dv[kOuterVecs], md[kOuterVecs];
  int8_t ax[kOuterVecs];
  int K, A, Q, out_f64;
  int64_t n[kOuterAxes], os[kOuterAxes];
  void* out;
  double alpha;
};

// One recorded op.  Types: tin / tw / tout are ElemType (f32 or f64).
struct Op {
  int kind = OP_CONTRACT;
  int tin = ET_F32, tw = ET_F32, tout = ET_F32;
  Contract c;
  Scatter s;
  Proj pj;
  Outer ou;
  // contraction details
  int g = 1;            // lanes cooperating on one output (power of two <= 32)
  int nsplit = 1;       // split of the reduction index (partials + OP_REDUCE)
  int64_t chunk = 0;
  void* partial = nullptr;
  int BG = 0, CG = 0, CH = 0;   // OP_MP tiling
  int64_t eye_n = 0;            // OP_EYE: n x n identity at c.out (f64)
  int64_t blocks = 0;
  int level = 0;
};

// Device-side copy of an op (plain data, fits the kernel parameter space).
struct DevOp {
  int kind, tin, tw, tout;
  Contract c;
  union {
    Scatter s;
    Proj pj;
    Outer ou;
  };
  DevOp() {}   // filled field by field (after a memset) on the host
  int g, nsplit;
  int64_t chunk;
  void* partial;
  int BG, CG, CH;
  int64_t eye_n;
  int idx32;   // every index of the op fits 31 bits: decode with 32-bit math
};

constexpr int kMaxLevelOps = 34;   // ops per batched launch (parameter space)

struct LevelBatch {
  LevelBatch() {}
  int nops;
  int64_t start[kMaxLevelOps + 1];   // prefix sums of blocks
  DevOp ops[kMaxLevelOps];
};

class Program {
 public:
  // Registers a buffer written by the program (or produced before it, level 0).
  void buffer(const void* p, int64_t bytes, int level = 0);
  // Records an op; its level follows the buffers it reads.
  void add(Op op, const void* in1, const void* in2 = nullptr);
  // Launches every level in order on `st`; dump: print each op (level, kind,
  // shape, blocks) to stderr first (a plan's TTNN_FLAG_DUMP_PROGRAM).
  ttnn_status run(cudaStream_t st, bool dump = false);
  void clear() {
    ops_.clear();
    bufs_.clear();
  }
  // Appends another program's ops (levels kept): programs over disjoint
  // buffers then share their level launches.
  void absorb(const Program& o) { ops_.insert(ops_.end(), o.ops_.begin(), o.ops_.end()); }
  size_t size() const { return ops_.size(); }
  int levels() const;

 private:
  struct Buf {
    const char* lo;
    const char* hi;
    int level;
  };
  int level_of(const void* p) const;
  std::vector<Op> ops_;
  std::vector<Buf> bufs_;
};

// Fills op.g / nsplit / chunk / blocks and the MP tiling for a contraction;
// returns the number of partial elements (of the output type) it needs.
int64_t plan_contract(Op& op);
// blocks of a scatter / eye op
void plan_simple(Op& op);

}  // namespace ttnn
