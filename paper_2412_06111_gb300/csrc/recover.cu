// Recovery phase kernels (binary64): for each non-root node, the Householder
// QR of Omega_v (s x r) with diag(R) >= 0, the singular values of R by
// one-sided Jacobi (Hestenes) with round-robin pair ordering, and the
// eps-pseudo-inverse R_eps^+ = V_1 Sigma_1^-1 U_1^T keeping sigma > eps,
// eps = eps_factor * u * sigma_max (Sec. 4 recovery phase and stabilised
// least squares; eq. (stabilized_nystrom)).  One CTA per node.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace ttnn {

constexpr int kQrThreads = 256;
constexpr int kMaxSweeps = 60;

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kQrThreads / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// dynamic shared memory: A (s x r), W (r x r), V (r x r), v0/vn2 (r), red
__global__ void __launch_bounds__(kQrThreads) qr_pinv_kernel(const QrJob* jobs, int state_f64,
                                                             double eps_factor, double u,
                                                             int* kept) {
  extern __shared__ double sm[];
  const QrJob job = jobs[blockIdx.x];
  const int s = job.s, r = job.r;
  double* A = sm;                       // s x r row-major
  double* W = A + s * r;                // r x r  (R, then R V)
  double* V = W + r * r;                // r x r
  double* vnorm = V + r * r;            // r
  double* red = vnorm + r;              // 8
  __shared__ int flag;
  const int tid = threadIdx.x;

  for (int e = tid; e < s * r; e += kQrThreads)
    A[e] = state_f64 ? ((const double*)job.omega)[e] : (double)((const float*)job.omega)[e];
  __syncthreads();

  // --- Householder QR: reflector k stored as v = A[k:s, k] (v[0] in place)
  for (int k = 0; k < r; ++k) {
    double part = 0.0;
    for (int i = k + tid; i < s; i += kQrThreads) part += A[i * r + k] * A[i * r + k];
    const double nrm2 = block_sum(part, red);
    const double alpha = A[k * r + k];
    const double nrm = sqrt(nrm2);
    double beta = 0.0, vn2 = 0.0;
    if (nrm > 0.0) {
      beta = alpha > 0.0 ? -nrm : nrm;
      const double v0 = alpha - beta;
      vn2 = nrm2 - alpha * alpha + v0 * v0;
    }
    __syncthreads();
    if (tid == 0) {
      vnorm[k] = vn2;
      A[k * r + k] = alpha - beta;   // v[0]; R[k][k] = beta kept in W below
      W[k * r + k] = beta;
    }
    __syncthreads();
    if (vn2 > 0.0) {
      // apply H = I - 2 v v^T / vn2 to columns j > k
      for (int j = k + 1; j < r; ++j) {
        double p = 0.0;
        for (int i = k + tid; i < s; i += kQrThreads) p += A[i * r + k] * A[i * r + j];
        const double dot = block_sum(p, red);
        const double f = 2.0 * dot / vn2;
        for (int i = k + tid; i < s; i += kQrThreads) A[i * r + j] -= f * A[i * r + k];
        __syncthreads();
      }
    }
    __syncthreads();
  }
  // R (upper triangle) into W, with R[k][k] already there
  for (int e = tid; e < r * r; e += kQrThreads) {
    const int i = e / r, j = e % r;
    if (j > i) W[e] = A[i * r + j];
    else if (j < i) W[e] = 0.0;
  }
  __syncthreads();
  // sign convention diag(R) >= 0: flip rows of R (and columns of Q below)
  // Q = H_0 ... H_{r-1} [I; 0] formed in global memory (job.q, s x r)
  for (int e = tid; e < s * r; e += kQrThreads) {
    const int i = e / r, j = e % r;
    job.q[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    const double vn2 = vnorm[k];
    if (vn2 > 0.0) {
      for (int j = 0; j < r; ++j) {
        double p = 0.0;
        for (int i = k + tid; i < s; i += kQrThreads) p += A[i * r + k] * job.q[i * r + j];
        const double dot = block_sum(p, red);
        const double f = 2.0 * dot / vn2;
        for (int i = k + tid; i < s; i += kQrThreads) job.q[i * r + j] -= f * A[i * r + k];
        __syncthreads();
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < r; k += kQrThreads) vnorm[k] = (W[k * r + k] < 0.0) ? -1.0 : 1.0;
  __syncthreads();
  for (int e = tid; e < r * r; e += kQrThreads) W[e] *= vnorm[e / r];
  for (int e = tid; e < s * r; e += kQrThreads) job.q[e] *= vnorm[e % r];
  for (int e = tid; e < r * r; e += kQrThreads) V[e] = (e / r == e % r) ? 1.0 : 0.0;
  __syncthreads();

  // --- one-sided Jacobi on the columns of W = R: W V = U Sigma
  const int n2 = r + (r & 1);   // even number of "players" (a dummy column if odd)
  const int warp = tid >> 5, lane = tid & 31, nwarps = kQrThreads / 32;
  const double tol = 4.0 * 1.1102230246251565e-16;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) flag = 0;
    __syncthreads();
    for (int round = 0; round < n2 - 1; ++round) {
      for (int pr = warp; pr < n2 / 2; pr += nwarps) {
        int a, b;
        if (pr == 0) { a = round % (n2 - 1); b = n2 - 1; }
        else { a = (round + pr) % (n2 - 1); b = (round - pr + n2 - 1) % (n2 - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= r) continue;      // dummy column
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < r; i += 32) {
          const double x = W[i * r + a], y = W[i * r + b];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
        if (lane == 0) flag = 1;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int i = lane; i < r; i += 32) {
          const double x = W[i * r + a], y = W[i * r + b];
          W[i * r + a] = c * x - sn * y;
          W[i * r + b] = sn * x + c * y;
          const double vx = V[i * r + a], vy = V[i * r + b];
          V[i * r + a] = c * vx - sn * vy;
          V[i * r + b] = sn * vx + c * vy;
        }
      }
      __syncthreads();
    }
    if (flag == 0) break;
    __syncthreads();
  }
  __syncthreads();
  // singular values sigma_k = ||W[:, k]||
  double* sig = vnorm;
  for (int k = warp; k < r; k += nwarps) {
    double p = 0.0;
    for (int i = lane; i < r; i += 32) p += W[i * r + k] * W[i * r + k];
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) sig[k] = sqrt(p);
  }
  __syncthreads();
  double smax = 0.0;
  for (int k = 0; k < r; ++k) smax = fmax(smax, sig[k]);
  const double eps = eps_factor * u * smax;
  // Rp[i][j] = sum_{kept k} V[i][k] W[j][k] / sigma_k^2
  for (int e = tid; e < r * r; e += kQrThreads) {
    const int i = e / r, j = e % r;
    double acc = 0.0;
    for (int k = 0; k < r; ++k)
      if (sig[k] > eps) acc += V[i * r + k] * W[j * r + k] / (sig[k] * sig[k]);
    job.rp[e] = acc;
  }
  if (tid == 0) {
    int cnt = 0;
    for (int k = 0; k < r; ++k) cnt += sig[k] > eps;
    kept[blockIdx.x] = cnt;
  }
}

ttnn_status launch_qr_pinv(const QrJob* jobs_dev, int njobs, int state_f64, double eps_factor,
                           double u, int* kept_dev, cudaStream_t st) {
  if (njobs == 0) return TTNN_OK;
  const size_t smem = (size_t)(kMaxRecoverS * kMaxRecoverR + 2 * kMaxRecoverR * kMaxRecoverR +
                               kMaxRecoverR + 8) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    TTNN_TRY_CUDA(cudaFuncSetAttribute(qr_pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    attr_set = true;
  }
  qr_pinv_kernel<<<njobs, kQrThreads, smem, st>>>(jobs_dev, state_f64, eps_factor, u, kept_dev);
  return check_launch("qr_pinv_kernel");
}

}  // namespace ttnn
