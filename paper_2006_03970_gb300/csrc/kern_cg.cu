// Conjugate-gradient solve of the Newton system (I_m + kappa A_J A_J^T) d = -g
// (eq. AJ_system), which Algorithm 1 step (1) allows in place of the direct solve and
// Sec. 3.2 proposes when m and r are both large.  Matrix-free: the product
// V p = p + kappa A_J (A_J^T p) is the panel GEMV pair of kern_vec.cu (k_gemv_t, then
// k_gemv_cl / k_gemv_n); the scalars of the iteration stay on the device:
//   * k_cg_init:  d = 0, res = -g, p = res, rr = ||res||^2, the stopping threshold;
//   * k_cg_step:  alpha = rr / p^T V p, d += alpha p, res -= alpha V p,
//                 beta = ||res||^2 / rr, p = res + beta p, and the stopping test
//                 ||res|| <= rtol ||g|| (DevState::cg_done).
// Both run on one CTA (m <= 4096 entries, a few per thread, fixed-order reductions), so
// the iteration is deterministic.  After cg_done every later step returns at once, which
// lets the host launch iterations in batches and read the state once per batch.
#include "common.cuh"

namespace ssnal {

constexpr int kCgThreads = 1024;

__global__ void __launch_bounds__(kCgThreads) k_cg_init(const double* __restrict__ g, double* __restrict__ d,
                                                        double* __restrict__ res, double* __restrict__ p, int m,
                                                        double rtol, DevState* st) {
  pdl_entry();
  __shared__ double red[kCgThreads];
  double q[1] = {0.0};
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double gi = g[i];
    d[i] = 0.0;
    res[i] = -gi;
    p[i] = -gi;
    q[0] = fma(gi, gi, q[0]);
  }
  const double rr = block_sum_k<1>(q, red, kCgThreads / 32);
  if (threadIdx.x == 0) {
    st->cg_rr = rr;
    st->cg_stop2 = rtol * rtol * rr;
    st->cg_iters = 0;
    st->cg_done = (rr == 0.0) ? 1 : 0;
  }
}

// One CG iteration given Vp = V p (computed by the GEMV pair since the last step).
__global__ void __launch_bounds__(kCgThreads) k_cg_step(double* __restrict__ d, double* __restrict__ res,
                                                        double* __restrict__ p, const double* __restrict__ Vp, int m,
                                                        DevState* st) {
  pdl_entry();
  if (st->cg_done) return;
  __shared__ double red[kCgThreads];
  __shared__ double bc[2];
  double q[1] = {0.0};
  for (int i = threadIdx.x; i < m; i += blockDim.x) q[0] = fma(p[i], Vp[i], q[0]);
  double t = block_sum_k<1>(q, red, kCgThreads / 32);
  if (threadIdx.x == 0) bc[0] = t;
  __syncthreads();
  const double pvp = bc[0];
  const double rr = st->cg_rr;
  if (!(pvp > 0.0) || !isfinite(pvp)) {  // V is SPD: only an exact zero p (or overflow) gets here
    if (threadIdx.x == 0) st->cg_done = 1;
    return;
  }
  const double alpha = rr / pvp;
  q[0] = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double pi = p[i];
    d[i] = fma(alpha, pi, d[i]);
    const double ri = fma(-alpha, Vp[i], res[i]);
    res[i] = ri;
    q[0] = fma(ri, ri, q[0]);
  }
  t = block_sum_k<1>(q, red, kCgThreads / 32);
  if (threadIdx.x == 0) bc[1] = t;
  __syncthreads();
  const double rr_next = bc[1];
  const double beta = rr_next / rr;
  for (int i = threadIdx.x; i < m; i += blockDim.x) p[i] = fma(beta, p[i], res[i]);
  if (threadIdx.x == 0) {
    st->cg_rr = rr_next;
    st->cg_iters += 1;
    if (!(rr_next > st->cg_stop2)) st->cg_done = 1;
  }
}

void launch_cg_init(const double* g, double* d, double* res, double* p, int m, double rtol, DevState* st,
                    cudaStream_t s) {
  count_launch();
  launch_k(k_cg_init, dim3(1), dim3(kCgThreads), (size_t)0, s, g, d, res, p, m, rtol, st);
}

void launch_cg_step(double* d, double* res, double* p, const double* Vp, int m, DevState* st, cudaStream_t s) {
  count_launch();
  launch_k(k_cg_step, dim3(1), dim3(kCgThreads), (size_t)0, s, d, res, p, Vp, m, st);
}

}  // namespace ssnal
