// The dual-to-primal stream over all n columns of A:
//   kModeU    u = A^T y                                 (Prop. 2, eq. Q_def)
//   kModeGmax u = A^T b and ||A^T b||_inf               (Sec. 3.3 / 4.1 lambda_max)
//   kModeT    t = A^T d fused with the line search of eq. line_search:
//             for trial steps s_k = beta^k it accumulates
//               sum_j soft(v_j - s_k sigma t_j)^2 - soft(v_j)^2,   v = x - sigma u,
//             so psi(y + s_k d) - psi(y) (Prop. 2 (1)) is known for every trial
//             after one pass over A; the last block picks the first trial that
//             satisfies the Armijo condition.
// One warp per column, grid-stride over columns, y/d staged in shared memory.
#include "common.cuh"

namespace ssnal {

constexpr int kStreamThreads = 256;

int stream_grid(int sms) { return 4 * sms; }

struct LsParams {
  ProxParams pp;
  double mu, beta;
  int max_ls, fused;
};

// Contribution of column j to the trial sums of trial k: soft(a)^2 - soft(v)^2
// written as (fa - fv)(fa + fv), a = v - s_k sigma t_j.
__device__ __forceinline__ double trial_term(double v, double tj, double sk, const ProxParams& pp) {
  const double a = __dsub_rn(v, __dmul_rn(sk * pp.sigma, tj));
  const double fa = shrink_mag(a, pp.thr), fv = shrink_mag(v, pp.thr);
  return (fa - fv) * (fa + fv);
}

// True when no trial step can move column j across the threshold: for s in
// (0, 1] the argument lies between v and v - sigma t.
__device__ __forceinline__ bool trial_skip(double v, double tj, const ProxParams& pp) {
  return fabs(v) <= pp.thr && fabs(__dsub_rn(v, __dmul_rn(pp.sigma, tj))) <= pp.thr;
}

// Armijo selection over trials [k0, k1) given the trial sums; returns the
// accepted index or -1.
__device__ int armijo_select(const DevState* st, const LsParams& lp, int k0, int k1, double& s_out) {
  const double coef = 1.0 / (2.0 * lp.pp.sigma * lp.pp.onep);
  double s = 1.0;
  for (int k = 0; k < k0; k++) s *= lp.beta;
  for (int k = k0; k < k1; k++) {
    const double dpsi = s * (st->yd + st->bd) + 0.5 * s * s * st->dd + coef * st->lsdiff[k];
    if (dpsi <= lp.mu * s * st->gd) {
      s_out = s;
      return k;
    }
    if (k < lp.max_ls - 1) s *= lp.beta;
  }
  s_out = s;
  return -1;
}

template <int MODE>
__global__ void __launch_bounds__(kStreamThreads) k_stream_f64(const double* __restrict__ A, long long lda, int m,
                                                               long long n, const double* __restrict__ vec,
                                                               double* __restrict__ out,
                                                               const double* __restrict__ x,
                                                               const double* __restrict__ u, LsParams lp,
                                                               DevState* st, double* __restrict__ partials) {
  extern __shared__ double sv[];
  __shared__ double wred[kStreamThreads / 32][32];
  __shared__ double red[32];
  const int mpad = (m + 63) & ~63;
  for (int i = threadIdx.x; i < mpad; i += blockDim.x) sv[i] = i < m ? vec[i] : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = kStreamThreads / 32;
  const long long gw = (long long)blockIdx.x * nw + warp, tw = (long long)gridDim.x * nw;
  // trial step of this lane (kModeT): s_lane = beta^lane
  double s_lane = 1.0;
  if (MODE == kModeT)
    for (int k = 0; k < lane; k++) s_lane *= lp.beta;
  double cand = 0.0;   // trial sum of trial `lane`
  double amax = 0.0;   // kModeGmax
  for (long long j = gw; j < n; j += tw) {
    const double* col = A + j * lda;
    double acc = 0.0;
    for (int i = 2 * lane; i < m; i += 64) {
      const double2 a = *reinterpret_cast<const double2*>(col + i);
      acc = fma(a.x, sv[i], acc);
      const double a1 = (i + 1 < m) ? a.y : 0.0;
      acc = fma(a1, sv[i + 1], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[j] = acc;
    if (MODE == kModeGmax) amax = fmax(amax, fabs(acc));
    if (MODE == kModeT) {
      const double v = v_of(x[j], u[j], lp.pp.sigma);
      if (!trial_skip(v, acc, lp.pp) && lane < lp.fused) cand += trial_term(v, acc, s_lane, lp.pp);
    }
  }
  if (MODE == kModeU) return;
  if (MODE == kModeGmax) {
    const double bm = block_max(amax, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = bm;
    if (!last_block(&st->counters[kCtrGmax])) return;
    double mx = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) mx = fmax(mx, ld_cg(&partials[b]));
    mx = block_max(mx, red);
    if (threadIdx.x == 0) st->gmax = mx;
    reset_counter(&st->counters[kCtrGmax]);
    return;
  }
  // kModeT: per-block trial sums, fixed order over warps
  wred[warp][lane] = cand;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += wred[w][lane];
    partials[(long long)blockIdx.x * 32 + lane] = s;
  }
  if (!last_block(&st->counters[kCtrStream])) return;
  if (warp == 0) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) s += ld_cg(&partials[(long long)b * 32 + lane]);
    if (lane < lp.fused) st->lsdiff[lane] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_block();
    double s;
    int k = armijo_select(st, lp, 0, lp.fused, s);
    if (k >= 0) {
      st->s = s;
      st->ls_k = k;
      st->ls_state = 0;
    } else if (lp.fused < lp.max_ls) {
      st->ls_state = 1;  // more trials in the fallback pass
    } else {
      st->s = s;  // every trial failed: the last trial step is taken
      st->ls_k = lp.max_ls - 1;
      st->ls_state = 0;
    }
  }
  reset_counter(&st->counters[kCtrStream]);
}

// Trials [fused, max_ls) over the stored vectors x, u, t (no pass over A).
// Runs only when the fused trials all failed; otherwise every block exits.
constexpr int kFbChunk = 16;
__global__ void __launch_bounds__(256) k_ls_fallback(const double* __restrict__ x, const double* __restrict__ u,
                                                     const double* __restrict__ t, long long n, LsParams lp,
                                                     DevState* st, double* __restrict__ partials) {
  __shared__ double red[32];
  if (st->ls_state != 1) return;
  const int extra = lp.max_ls - lp.fused;
  double s0 = 1.0;
  for (int k = 0; k < lp.fused; k++) s0 *= lp.beta;
  for (int c0 = 0; c0 < extra; c0 += kFbChunk) {
    double acc[kFbChunk];
#pragma unroll
    for (int q = 0; q < kFbChunk; q++) acc[q] = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
      const double v = v_of(x[j], u[j], lp.pp.sigma);
      const double tj = t[j];
      if (trial_skip(v, tj, lp.pp)) continue;
      double s = s0;
      for (int q = 0; q < c0; q++) s *= lp.beta;
#pragma unroll
      for (int q = 0; q < kFbChunk; q++) {
        if (c0 + q < extra) acc[q] += trial_term(v, tj, s, lp.pp);
        s *= lp.beta;
      }
    }
#pragma unroll
    for (int q = 0; q < kFbChunk; q++) {
      double b = block_sum(acc[q], red);
      if (threadIdx.x == 0) partials[(long long)blockIdx.x * kMaxLS + c0 + q] = b;
    }
  }
  if (!last_block(&st->counters[kCtrFallback])) return;
  for (int q = threadIdx.x; q < extra; q += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) s += ld_cg(&partials[(long long)b * kMaxLS + q]);
    st->lsdiff[lp.fused + q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_block();
    double s;
    int k = armijo_select(st, lp, lp.fused, lp.max_ls, s);
    if (k < 0) k = lp.max_ls - 1;
    st->s = s;
    st->ls_k = k;
    st->ls_state = 0;
  }
  reset_counter(&st->counters[kCtrFallback]);
}

void launch_stream(int mode, int dtype, const void* A, long long lda, int m, long long n, const double* vec,
                   double* out, const double* x, const double* u, ProxParams pp, double mu, double beta, int max_ls,
                   int fused, DevState* st, double* partials, int grid, cudaStream_t s) {
  LsParams lp{pp, mu, beta, max_ls, fused};
  const size_t smem = (size_t)((m + 63) & ~63) * sizeof(double);
  (void)dtype;
  const double* Ad = (const double*)A;
  count_launch();
  if (mode == kModeU)
    k_stream_f64<kModeU><<<grid, kStreamThreads, smem, s>>>(Ad, lda, m, n, vec, out, x, u, lp, st, partials);
  else if (mode == kModeT)
    k_stream_f64<kModeT><<<grid, kStreamThreads, smem, s>>>(Ad, lda, m, n, vec, out, x, u, lp, st, partials);
  else
    k_stream_f64<kModeGmax><<<grid, kStreamThreads, smem, s>>>(Ad, lda, m, n, vec, out, x, u, lp, st, partials);
}

void launch_ls_fallback(const double* x, const double* u, const double* t, long long n, ProxParams pp, double mu,
                        double beta, int max_ls, int fused, DevState* st, double* partials, int grid, cudaStream_t s) {
  if (fused >= max_ls) return;
  LsParams lp{pp, mu, beta, max_ls, fused};
  count_launch();
  k_ls_fallback<<<grid, 256, 0, s>>>(x, u, t, n, lp, st, partials);
}

}  // namespace ssnal
