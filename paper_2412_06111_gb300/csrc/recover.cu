// Recovery phase kernels (binary64): for each non-root node, the Householder
// QR of Omega_v (s x r) with diag(R) >= 0, the singular values of R by
// one-sided Jacobi (Hestenes) with round-robin pair ordering, and the
// eps-pseudo-inverse R_eps^+ = V_1 Sigma_1^-1 U_1^T keeping sigma > eps,
// eps = eps_factor * u * sigma_max (Sec. 4 recovery phase and stabilised
// least squares; eq. (stabilized_nystrom)).  One CTA per node; every step
// works on all trailing columns at once (one warp per column).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace ttnn {

// one warp per Jacobi pair (r / 2 warps, at least 8): every rotation round is
// one pass; the CTA size is chosen at launch
constexpr int kQrMaxThreads = 1024;
constexpr int kQrMaxWarps = kQrMaxThreads / 32;
constexpr int kMaxSweeps = 60;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Upper Cholesky factor of the symmetric r x r matrix in W (upper triangle,
// column-major W[j * r + i] = G[i][j], i <= j) in place: G = R^T R with
// diag(R) > 0.  Returns false (all threads) when a pivot falls to `tol` times
// the largest diagonal entry of G or below: the Gram matrix is then too close
// to singular for Cholesky-based QR.
__device__ bool chol_upper(double* W, int r, double* rd, int* bad) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    double gmax = 0.0;
    for (int k = 0; k < r; ++k) gmax = fmax(gmax, W[k * r + k]);
    rd[r] = gmax;
    *bad = 0;
  }
  __syncthreads();
  const double tol = 1e-10 * rd[r];
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      const double d = W[k * r + k];
      if (!(d > tol)) *bad = 1;
      const double rkk = d > 0.0 ? sqrt(d) : 1.0;
      W[k * r + k] = rkk;
      rd[k] = 1.0 / rkk;
    }
    __syncthreads();
    if (*bad) return false;
    const double inv = rd[k];
    // trailing G[i][j] -= G[k][i] G[k][j] / G[k][k] (row k still unscaled)
    const int m = r - k - 1;
    for (int e = tid; e < m * m; e += (int)blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (i <= j) W[j * r + i] -= (W[i * r + k] * inv) * (W[j * r + k] * inv);
    }
    __syncthreads();
    for (int j = k + 1 + tid; j < r; j += (int)blockDim.x) W[j * r + k] *= inv;   // row k of R
    __syncthreads();
  }
  return true;
}

// X = R^-1 for the upper triangular R in W (both column-major), one thread
// per column (back substitution); rd holds 1 / diag(R).
__device__ void tri_inv_upper(const double* W, double* X, int r, const double* rd) {
  for (int j = threadIdx.x; j < r; j += (int)blockDim.x) {
    for (int i = j + 1; i < r; ++i) X[j * r + i] = 0.0;
    X[j * r + j] = rd[j];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int k = i + 1; k <= j; ++k) acc += W[k * r + i] * X[j * r + k];
      X[j * r + i] = -acc * rd[i];
    }
  }
  __syncthreads();
}

// dynamic shared memory (column-major, leading dimension s for A and Q,
// r for W, V and X): A (s x r), Q (s x r), W, V, X (r x r), small arrays.
// trunc != 0 (eps-truncated output): when singular values of R are dropped,
// q receives Q U_1 and rp receives V_1 Sigma_1^-1 (kept columns first, in
// index order, zero columns after), so that the cores assembled from them
// carry the kept ranks; R_eps^+ = (V_1 Sigma_1^-1) U_1^T is the same map.
__global__ void __launch_bounds__(kQrMaxThreads) qr_pinv_kernel(const QrJob* jobs, int state_f64,
                                                             double eps_factor, double u,
                                                             int* kept, int trunc) {
  extern __shared__ double sm[];
  const QrJob job = jobs[blockIdx.x];
  const int s = job.s, r = job.r;
  double* A = sm;                         // A[j * s + i]
  double* Q = A + kMaxRecoverS * kMaxRecoverR;
  double* W = Q + kMaxRecoverS * kMaxRecoverR;   // W[k * r + i]: column k of R V
  double* V = W + kMaxRecoverR * kMaxRecoverR;   // V[k * r + i]
  double* X2 = V + kMaxRecoverR * kMaxRecoverR;  // second triangular inverse
  double* vn = X2 + kMaxRecoverR * kMaxRecoverR; // reflector norms (r + 1)
  double* rd = vn + kMaxRecoverR + 1;            // diag of R / signs / sigmas (r + 1)
  __shared__ int flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = (int)(blockDim.x >> 5);

  for (int e = tid; e < s * r; e += (int)blockDim.x) {
    const int i = e / r, j = e % r;      // Omega is row-major (s x r)
    A[j * s + i] = state_f64 ? ((const double*)job.omega)[e] : (double)((const float*)job.omega)[e];
  }
  __syncthreads();

  // ---- fast path: Cholesky QR twice (CholeskyQR2).  Omega = Q1 R1 from
  // the Gram matrix, then Q1 = Q R2 again; R = R2 R1 with diag(R) > 0, the
  // same factors as the Householder path below (QR with a positive diagonal
  // is unique).  Taken when both Gram matrices are safely positive definite
  // (kappa(Omega) below ~1e5, where CholeskyQR2 is as accurate as Householder)
  // and R^-1 is certified as for the Householder path; otherwise the
  // Householder path runs from the untouched A.
  __shared__ int cbad;
  {
    for (int e = tid; e < r * r; e += (int)blockDim.x) {
      const int i = e / r, j = e % r;
      if (i > j) continue;
      double acc = 0.0;
      for (int k = 0; k < s; ++k) acc += A[i * s + k] * A[j * s + k];
      W[j * r + i] = acc;
    }
    __syncthreads();
    bool ok = chol_upper(W, r, rd, &cbad);
    if (ok) {
      tri_inv_upper(W, V, r, rd);                      // V = R1^-1
      for (int e = tid; e < s * r; e += (int)blockDim.x) {  // Q1 = A R1^-1 (into Q)
        const int j = e / s, i = e % s;
        double acc = 0.0;
        for (int k = 0; k <= j; ++k) acc += A[k * s + i] * V[j * r + k];
        Q[j * s + i] = acc;
      }
      __syncthreads();
      for (int e = tid; e < r * r; e += (int)blockDim.x) {  // G2 = Q1^T Q1
        const int i = e / r, j = e % r;
        if (i > j) continue;
        double acc = 0.0;
        for (int k = 0; k < s; ++k) acc += Q[i * s + k] * Q[j * s + k];
        W[j * r + i] = acc;
      }
      __syncthreads();
      ok = chol_upper(W, r, rd, &cbad);
    }
    if (ok) {
      tri_inv_upper(W, X2, r, rd);                     // X2 = R2^-1
      // R^-1 = R1^-1 R2^-1 into W (upper triangular, column-major)
      for (int e = tid; e < r * r; e += (int)blockDim.x) {
        const int j = e / r, i = e % r;
        double acc = 0.0;
        for (int k = i; k <= j; ++k) acc += V[k * r + i] * X2[j * r + k];
        W[j * r + i] = i <= j ? acc : 0.0;
      }
      __syncthreads();
      // certification: ||R||_F = ||Omega||_F (Q orthonormal)
      __shared__ double cred[2 * kQrMaxWarps];
      double pa = 0.0, px = 0.0;
      for (int e = tid; e < s * r; e += (int)blockDim.x) pa += A[e] * A[e];
      for (int e = tid; e < r * r; e += (int)blockDim.x) px += W[e] * W[e];
      pa = warp_sum(pa);
      px = warp_sum(px);
      if (lane == 0) {
        cred[warp] = pa;
        cred[nwarps + warp] = px;
      }
      __syncthreads();
      double rf2 = 0.0, xf2 = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        rf2 += cred[w];
        xf2 += cred[nwarps + w];
      }
      const double margin = 4.0 * eps_factor * u;
      if (margin * margin * rf2 * xf2 < 1.0 && xf2 > 0.0) {
        // Q = Q1 R2^-1 (row-major output), R^-1 row-major
        for (int e = tid; e < s * r; e += (int)blockDim.x) {
          const int i = e / r, j = e % r;
          double acc = 0.0;
          for (int k = 0; k <= j; ++k) acc += Q[k * s + i] * X2[j * r + k];
          job.q[e] = acc;
        }
        for (int e = tid; e < r * r; e += (int)blockDim.x) {
          const int i = e / r, j = e % r;
          job.rp[e] = W[j * r + i];
        }
        if (tid == 0) {
          kept[blockIdx.x] = r;
          kept[gridDim.x + blockIdx.x] = 0;
        }
        return;
      }
    }
    __syncthreads();
  }

  // ---- Householder QR; reflector k is v = A[k:s, k] with v[0] stored in place
  for (int k = 0; k < r; ++k) {
    if (warp == 0) {
      double part = 0.0;
      for (int i = k + lane; i < s; i += 32) part += A[k * s + i] * A[k * s + i];
      const double nrm2 = warp_sum(part);
      if (lane == 0) {
        const double alpha = A[k * s + k];
        const double nrm = sqrt(nrm2);
        double beta = 0.0, vn2 = 0.0;
        if (nrm > 0.0) {
          beta = alpha > 0.0 ? -nrm : nrm;
          const double v0 = alpha - beta;
          vn2 = nrm2 - alpha * alpha + v0 * v0;
          A[k * s + k] = v0;
        }
        vn[k] = vn2 > 0.0 ? 2.0 / vn2 : 0.0;   // scale of the reflector, one division
        rd[k] = beta;
      }
    }
    __syncthreads();
    const double sc = vn[k];
    if (sc > 0.0) {
      for (int j = k + 1 + warp; j < r; j += nwarps) {
        double part = 0.0;
        for (int i = k + lane; i < s; i += 32) part += A[k * s + i] * A[j * s + i];
        const double f = warp_sum(part) * sc;
        for (int i = k + lane; i < s; i += 32) A[j * s + i] -= f * A[k * s + i];
      }
    }
    __syncthreads();
  }
  // ---- Q = H_0 ... H_{r-1} [I; 0]
  for (int e = tid; e < s * r; e += (int)blockDim.x) {
    const int j = e / s, i = e % s;
    Q[j * s + i] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    const double sc = vn[k];
    if (sc > 0.0) {
      for (int j = k + warp; j < r; j += nwarps) {   // columns j < k are untouched by H_k
        double part = 0.0;
        for (int i = k + lane; i < s; i += 32) part += A[k * s + i] * Q[j * s + i];
        const double f = warp_sum(part) * sc;
        for (int i = k + lane; i < s; i += 32) Q[j * s + i] -= f * A[k * s + i];
      }
    }
    __syncthreads();
  }
  // ---- R (upper triangle) into W, signs so that diag(R) >= 0
  for (int e = tid; e < r * r; e += (int)blockDim.x) {
    const int j = e / r, i = e % r;      // W column-major: W[j * r + i] = R[i][j]
    double v = 0.0;
    if (i == j) v = rd[i];
    else if (i < j) v = A[j * s + i];
    W[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += (int)blockDim.x) {
    const int j = e / r, i = e % r;
    if (rd[i] < 0.0) W[e] = -W[e];               // row i of R
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  for (int e = tid; e < s * r; e += (int)blockDim.x) {
    const int j = e / s, i = e % s;
    const double q = rd[j] < 0.0 ? -Q[j * s + i] : Q[j * s + i];   // column j of Q
    job.q[i * r + j] = q;                          // row-major s x r output
  }
  __syncthreads();

  // ---- fast path: R_eps^+ = R^-1 when no singular value can fall below eps.
  // sigma_min(R) >= 1/||R^-1||_F and ||R||_2 <= ||R||_F, so
  // 1/||R^-1||_F > 4 * eps_factor * u * ||R||_F certifies sigma_min > eps.
  // R^-1 (upper triangular) by back substitution, one thread per column.
  double* X = Q;   // Q was written out above; reuse its storage (r x r, column-major)
  __shared__ double red2[2 * kQrMaxWarps];
  __shared__ int singular;
  if (tid == 0) singular = 0;
  __syncthreads();
  for (int i = tid; i < r; i += (int)blockDim.x) {
    const double dgi = W[i * r + i];
    if (dgi == 0.0) singular = 1;
    rd[i] = dgi != 0.0 ? 1.0 / dgi : 0.0;   // reciprocal diagonal (rd: diag no longer needed)
  }
  __syncthreads();
  if (!singular) {
    for (int j = tid; j < r; j += (int)blockDim.x) {
      for (int i = 0; i < r; ++i) X[j * r + i] = 0.0;
      X[j * r + j] = rd[j];
      for (int i = j - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int k = i + 1; k <= j; ++k) acc += W[k * r + i] * X[j * r + k];
        X[j * r + i] = -acc * rd[i];
      }
    }
    __syncthreads();
    double pr = 0.0, px = 0.0;
    for (int e = tid; e < r * r; e += (int)blockDim.x) {
      pr += W[e] * W[e];
      px += X[e] * X[e];
    }
    pr = warp_sum(pr);
    px = warp_sum(px);
    if (lane == 0) {
      red2[warp] = pr;
      red2[nwarps + warp] = px;
    }
    __syncthreads();
    double rf2 = 0.0, xf2 = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      rf2 += red2[w];
      xf2 += red2[nwarps + w];
    }
    const double margin = 4.0 * eps_factor * u;
    if (margin * margin * rf2 * xf2 < 1.0 && xf2 > 0.0) {
      for (int e = tid; e < r * r; e += (int)blockDim.x) {
        const int i = e / r, j = e % r;
        job.rp[e] = X[j * r + i];    // row-major R^-1
      }
      if (tid == 0) {
        kept[blockIdx.x] = r;
        kept[gridDim.x + blockIdx.x] = 0;   // no Jacobi sweep needed
      }
      return;
    }
  }
  __syncthreads();

  // ---- one-sided Jacobi on the columns of W = R: W V = U Sigma
  const int n2 = r + (r & 1);   // even number of players (a dummy column if r is odd)
  // a rotation is skipped once |gamma| <= sqrt(r) * eps * sqrt(alpha beta):
  // below this the computed gamma is rounding noise (the one-sided Jacobi
  // stopping test of Demmel & Veselic with m = r rows)
  const double tol = sqrt((double)r) * 2.220446049250313e-16;
  int sweeps = 0;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    sweeps = sweep + 1;
    if (tid == 0) flag = 0;
    __syncthreads();
    for (int round = 0; round < n2 - 1; ++round) {
      for (int pr = warp; pr < n2 / 2; pr += nwarps) {
        int a, b;
        if (pr == 0) { a = round % (n2 - 1); b = n2 - 1; }
        else { a = (round + pr) % (n2 - 1); b = (round - pr + n2 - 1) % (n2 - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= r) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < r; i += 32) {
          const double x = W[a * r + i], y = W[b * r + i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        // the rotation's scalars are evaluated by one lane: FP64 division and
        // square root are long instruction sequences on this part
        double c = 1.0, sn = 0.0;
        int rot = 0;
        if (lane == 0 && ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          rot = 1;
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = c * t;
          flag = 1;
        }
        rot = __shfl_sync(0xffffffffu, rot, 0);
        if (!rot) continue;
        c = __shfl_sync(0xffffffffu, c, 0);
        sn = __shfl_sync(0xffffffffu, sn, 0);
        for (int i = lane; i < r; i += 32) {
          const double x = W[a * r + i], y = W[b * r + i];
          W[a * r + i] = c * x - sn * y;
          W[b * r + i] = sn * x + c * y;
          const double vx = V[a * r + i], vy = V[b * r + i];
          V[a * r + i] = c * vx - sn * vy;
          V[b * r + i] = sn * vx + c * vy;
        }
      }
      __syncthreads();
    }
    if (flag == 0) break;
    __syncthreads();
  }
  // singular values sigma_k = ||W[:, k]||
  for (int k = warp; k < r; k += nwarps) {
    double p = 0.0;
    for (int i = lane; i < r; i += 32) p += W[k * r + i] * W[k * r + i];
    p = warp_sum(p);
    if (lane == 0) rd[k] = sqrt(p);
  }
  __syncthreads();
  double smax = 0.0;
  for (int k = 0; k < r; ++k) smax = fmax(smax, rd[k]);
  const double eps = eps_factor * u * smax;
  // 1 / sigma_k^2 of the kept singular values (0 for the dropped ones)
  double* inv2 = vn;
  for (int k = tid; k < r; k += (int)blockDim.x) inv2[k] = rd[k] > eps ? 1.0 / (rd[k] * rd[k]) : 0.0;
  __syncthreads();
  if (trunc) {
    // kept columns in index order: slot[k] = position among the kept, -1 dropped
    __shared__ int slot[kMaxRecoverR];
    if (tid == 0) {
      int c = 0;
      for (int k = 0; k < r; ++k) slot[k] = rd[k] > eps ? c++ : -1;
    }
    __syncthreads();
    // rp = V_1 Sigma_1^-1 (r x r, row-major, kept columns first)
    for (int e = tid; e < r * r; e += (int)blockDim.x) {
      const int i = e / r, c = e % r;
      double v = 0.0;
      for (int k = 0; k < r; ++k)
        if (slot[k] == c) v = V[k * r + i] / rd[k];
      job.rp[e] = v;
    }
    // q <- Q U_1 with U_1[:, c] = W[:, k] / sigma_k; A (no longer needed)
    // holds the product until every thread has read Q
    double* QU = A;
    for (int e = tid; e < s * r; e += (int)blockDim.x) {
      const int i = e / r, c = e % r;
      double acc = 0.0;
      for (int k = 0; k < r; ++k)
        if (slot[k] == c)
          for (int l = 0; l < r; ++l) acc += job.q[i * r + l] * (W[k * r + l] / rd[k]);
      QU[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < s * r; e += (int)blockDim.x) job.q[e] = QU[e];
  } else {
    // Rp[i][j] = sum_{kept k} V[i][k] W[j][k] / sigma_k^2  (row-major output)
    for (int e = tid; e < r * r; e += (int)blockDim.x) {
      const int i = e / r, j = e % r;
      double acc = 0.0;
      for (int k = 0; k < r; ++k) acc += V[k * r + i] * W[k * r + j] * inv2[k];
      job.rp[e] = acc;
    }
  }
  if (tid == 0) {
    int cnt = 0;
    for (int k = 0; k < r; ++k) cnt += rd[k] > eps;
    kept[blockIdx.x] = cnt;
    kept[gridDim.x + blockIdx.x] = sweeps;   // diagnostic: Jacobi sweeps used
  }
}

ttnn_status launch_qr_pinv(const QrJob* jobs_dev, int njobs, int rmax, int state_f64,
                           double eps_factor, double u, int* kept_dev, int trunc,
                           cudaStream_t st) {
  if (njobs == 0) return TTNN_OK;
  const size_t smem = (size_t)(2 * kMaxRecoverS * kMaxRecoverR + 3 * kMaxRecoverR * kMaxRecoverR +
                               2 * (kMaxRecoverR + 1)) * sizeof(double);
  TTNN_TRY_CUDA(cudaFuncSetAttribute(qr_pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const int warps = std::min(kQrMaxWarps, std::max(8, (rmax + 1) / 2));
  qr_pinv_kernel<<<njobs, warps * 32, smem, st>>>(jobs_dev, state_f64, eps_factor, u, kept_dev,
                                                  trunc);
  return check_launch("qr_pinv_kernel");
}

}  // namespace ttnn
