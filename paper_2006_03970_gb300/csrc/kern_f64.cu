// The Newton system of eqs. AJ_system / smw_formula formed, factored and solved in
// FP64 on the device:
//   * k_syrk64: G = diag I + scale A_J^T A_J (r x r) or diag I + scale A_J A_J^T (m x m)
//     from the FP64 panel, lower triangle, 64 x 64 tiles, FP64 FMAs;
//   * a right-looking blocked Cholesky with 32-column panels: k_potrf64_diag factors the
//     diagonal block in shared memory, k_trsm64_panel solves the rows below it,
//     k_syrk64_update applies the panel to the trailing matrix;
//   * k_trsv64: forward and backward substitution on one CTA, blocked by 32 rows;
//   * k_refine_update: an iterative-refinement correction of the FP32 solve, with the
//     contraction test that decides whether the FP64 system is needed.
// The FP32 factor with FP64 refinement (kern_linalg.cu) is the fast path.  These kernels
// take over when the FP32 factor meets a non-positive pivot or its refinement does not
// contract (the Newton matrix is too ill-conditioned for the FP32 factor of a matrix
// formed with FP32 accumulation: its condition number is up to 1 + kappa ||A_J||^2 and
// kappa grows with sigma when lambda2 is small), and on request for every Newton step.
// GB300 runs FP64 FMAs at about two per clock per SM, so these kernels are far slower
// than the FP32 ones; they spread the O(N^3) and O(m N^2) work over many CTAs and keep
// everything else simple.  A non-positive FP64 pivot sets
// DevState::f64_fail and every later kernel of the factor and solve returns at once.
#include "common.cuh"

namespace ssnal {

namespace {

constexpr int kT64 = 64;   // output tile of the SYRK kernels
constexpr int kK64 = 16;   // K chunk staged in shared memory by k_syrk64
constexpr int kNB64 = 32;  // panel width of the blocked Cholesky

// (ti, tj), ti >= tj, of lower-triangular tile number `t` (row-major over the triangle).
__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  int i = 0;
  while ((i + 1) * (i + 2) / 2 <= t) i++;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

}  // namespace

// G[i, j] = diag [i == j] + scale sum_k X[k, i] X[k, j] for the lower tiles, where
// TRANS = 0: X = P (m x r, K = m, N = r), X[k, i] = P[k + i ldp];
// TRANS = 1: X = P^T (K = r, N = m),      X[k, i] = P[i + k ldp].
// 256 threads, each a 4 x 4 block of the 64 x 64 tile (rows ty + 16 a, columns tx + 16 b).
template <int TRANS>
__global__ void __launch_bounds__(256) k_syrk64(const double* __restrict__ P, long long ldp, int m, int r,
                                                double diag, double scale, double* __restrict__ G, long long ldg,
                                                const DevState* st) {
  pdl_entry();
  __shared__ double As[kK64][kT64 + 1];
  __shared__ double Bs[kK64][kT64 + 1];
  const int N = TRANS ? m : r;
  const int K = TRANS ? r : m;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = ti * kT64, j0 = tj * kT64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += kK64) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int e = tid + 256 * q;
      int kk, ii;
      if (TRANS == 0) {  // consecutive k contiguous in a column of P
        kk = e & (kK64 - 1);
        ii = e >> 4;
      } else {  // consecutive rows contiguous
        ii = e & (kT64 - 1);
        kk = e >> 6;
      }
      const int k = k0 + kk, ia = i0 + ii, jb = j0 + ii;
      double va = 0.0, vb = 0.0;
      if (k < K) {
        if (TRANS == 0) {
          if (ia < N) va = P[k + (long long)ia * ldp];
          if (jb < N) vb = P[k + (long long)jb * ldp];
        } else {
          if (ia < N) va = P[ia + (long long)k * ldp];
          if (jb < N) vb = P[jb + (long long)k * ldp];
        }
      }
      As[kk][ii] = va;
      Bs[kk][ii] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK64; kk++) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; b++) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      if (i < N && j < N && i >= j) G[i + (long long)j * ldg] = (i == j ? diag : 0.0) + scale * acc[a][b];
    }
  }
}

// Factor of the nb x nb diagonal block at (kb, kb), column by column, one thread per
// entry of a 32 x 32 shared tile.  A pivot that is not positive (or NaN) sets f64_fail.
__global__ void __launch_bounds__(1024) k_potrf64_diag(double* __restrict__ G, long long ld, int kb, int nb,
                                                       DevState* st) {
  pdl_entry();
  if (st->f64_fail) return;
  __shared__ double a[kNB64][kNB64 + 1];
  const int j = threadIdx.x & 31, i = threadIdx.x >> 5;
  a[i][j] = (i < nb && j < nb && i >= j) ? G[(kb + i) + (long long)(kb + j) * ld] : 0.0;
  for (int p = 0; p < nb; p++) {
    __syncthreads();
    const double d = a[p][p];
    if (!(d > 0.0)) {  // uniform: every thread read the same value
      if (threadIdx.x == 0) st->f64_fail = 1;
      return;
    }
    const double lpp = sqrt(d);
    __syncthreads();
    if (j == p && i >= p) a[i][p] = (i == p) ? lpp : a[i][p] / lpp;
    __syncthreads();
    if (j > p && i >= j) a[i][j] = fma(-a[i][p], a[j][p], a[i][j]);
  }
  __syncthreads();
  if (i < nb && j < nb && i >= j) G[(kb + i) + (long long)(kb + j) * ld] = a[i][j];
}

// Rows kb + nb .. N - 1 of panel kb: row_i <- row_i L_kk^{-T} (one thread per row, the
// factored diagonal block in shared memory).
__global__ void __launch_bounds__(128) k_trsm64_panel(double* __restrict__ G, long long ld, int kb, int nb, int N,
                                                      const DevState* st) {
  pdl_entry();
  if (st->f64_fail) return;
  __shared__ double L[kNB64][kNB64 + 1];
  for (int e = threadIdx.x; e < kNB64 * kNB64; e += blockDim.x) {
    const int r = e & 31, c = e >> 5;
    L[r][c] = (r < nb && c < nb) ? G[(kb + r) + (long long)(kb + c) * ld] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  const int i = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[kNB64];
#pragma unroll
  for (int c = 0; c < kNB64; c++) x[c] = c < nb ? G[i + (long long)(kb + c) * ld] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB64; c++) {
    double v = x[c];
#pragma unroll
    for (int l = 0; l < c; l++) v = fma(-x[l], L[c][l], v);
    x[c] = v / L[c][c];
  }
#pragma unroll
  for (int c = 0; c < kNB64; c++)
    if (c < nb) G[i + (long long)(kb + c) * ld] = x[c];
}

// Trailing update of the lower triangle: G[i, j] -= sum_{l < nb} G[i, kb + l] G[j, kb + l]
// for i >= j >= c0 = kb + nb, 64 x 64 tiles of the trailing matrix.
__global__ void __launch_bounds__(256) k_syrk64_update(double* __restrict__ G, long long ld, int kb, int nb, int N,
                                                       const DevState* st) {
  pdl_entry();
  if (st->f64_fail) return;
  __shared__ double Ls[kNB64][kT64 + 1];
  __shared__ double Rs[kNB64][kT64 + 1];
  const int c0 = kb + nb;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = c0 + ti * kT64, j0 = c0 + tj * kT64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < kNB64 * kT64; e += 256) {
    const int ii = e & (kT64 - 1), l = e >> 6;
    const int ia = i0 + ii, jb = j0 + ii;
    Ls[l][ii] = (l < nb && ia < N) ? G[ia + (long long)(kb + l) * ld] : 0.0;
    Rs[l][ii] = (l < nb && jb < N) ? G[jb + (long long)(kb + l) * ld] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
#pragma unroll 8
  for (int l = 0; l < kNB64; l++) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; a++) av[a] = Ls[l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; b++) bv[b] = Rs[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      if (i < N && j < N && i >= j) {
        double* g = G + i + (long long)j * ld;
        *g = *g - acc[a][b];
      }
    }
  }
}

// L L^T x = rhs on one CTA of 1024 threads, x kept in shared memory (N doubles):
// forward substitution by 32-row blocks (warp 0 solves the diagonal block with shuffles,
// then every thread updates its rows below), backward substitution with L^T the same way
// (warp w forms the contribution of the rows below to column w of the block).
// acc = alpha x (first) or acc += alpha x.
__global__ void __launch_bounds__(1024) k_trsv64(const double* __restrict__ L, long long ld, int N,
                                                 const double* __restrict__ rhs, double* __restrict__ acc, int first,
                                                 double alpha, const DevState* st) {
  pdl_entry();
  if (st->f64_fail) return;
  extern __shared__ double xs[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += blockDim.x) xs[i] = rhs[i];
  __syncthreads();
  // forward: L y = rhs
  for (int b0 = 0; b0 < N; b0 += 32) {
    const int nb = N - b0 < 32 ? N - b0 : 32;
    if (warp == 0) {
      double v = lane < nb ? xs[b0 + lane] : 0.0;
      for (int p = 0; p < nb; p++) {
        double xp = __shfl_sync(0xffffffffu, v, p);
        xp = xp / L[(b0 + p) + (long long)(b0 + p) * ld];
        if (lane == p) v = xp;
        if (lane > p && lane < nb) v = fma(-L[(b0 + lane) + (long long)(b0 + p) * ld], xp, v);
      }
      if (lane < nb) xs[b0 + lane] = v;
    }
    __syncthreads();
    for (int i = b0 + nb + tid; i < N; i += blockDim.x) {
      double s = xs[i];
      for (int p = 0; p < nb; p++) s = fma(-L[i + (long long)(b0 + p) * ld], xs[b0 + p], s);
      xs[i] = s;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  const int nblk = (N + 31) / 32;
  for (int bb = nblk - 1; bb >= 0; bb--) {
    const int b0 = bb * 32;
    const int nb = N - b0 < 32 ? N - b0 : 32;
    if (warp < nb) {  // column b0 + warp: sum over the rows below the block
      double s = 0.0;
      for (int i = b0 + nb + lane; i < N; i += 32) s = fma(L[i + (long long)(b0 + warp) * ld], xs[i], s);
      s = warp_sum(s);
      if (lane == 0) xs[b0 + warp] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      double v = lane < nb ? xs[b0 + lane] : 0.0;
      for (int p = nb - 1; p >= 0; p--) {
        double xp = __shfl_sync(0xffffffffu, v, p);
        xp = xp / L[(b0 + p) + (long long)(b0 + p) * ld];
        if (lane == p) v = xp;
        if (lane < p) v = fma(-L[(b0 + p) + (long long)(b0 + lane) * ld], xp, v);
      }
      if (lane < nb) xs[b0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < N; i += blockDim.x) acc[i] = first ? alpha * xs[i] : fma(alpha, xs[i], acc[i]);
}

// acc += c, with ||c||^2 and ||acc||^2 (after the update) summed in a fixed order; the
// ratio ||c|| / ||acc|| goes to DevState::refine_ratio, and when it exceeds tau (or is
// not finite) the FP32 solve is declared unreliable.
__global__ void __launch_bounds__(1024) k_refine_update(double* __restrict__ acc, const double* __restrict__ c,
                                                        int len, double tau2, DevState* st) {
  pdl_entry();
  __shared__ double red[2 * 1024];
  double q[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double ci = c[i];
    const double ai = acc[i] + ci;
    acc[i] = ai;
    q[0] = fma(ci, ci, q[0]);
    q[1] = fma(ai, ai, q[1]);
  }
  const double tot = block_sum_k<2>(q, red, blockDim.x / 32);
  __shared__ double tots[2];
  if (threadIdx.x < 2) tots[threadIdx.x] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->refine_ratio = tots[1] > 0.0 ? sqrt(tots[0] / tots[1]) : (tots[0] > 0.0 ? INFINITY : 0.0);
    if (!(tots[0] <= tau2 * tots[1])) st->newton_bad = 1;
  }
}

void launch_syrk64(const double* P, long long ldp, int m, int r, int trans, double diag, double scale, double* G64,
                   long long ldg64, const DevState* st, cudaStream_t s) {
  const int N = trans ? m : r;
  if (N <= 0) return;
  const int T = (N + kT64 - 1) / kT64;
  count_launch();
  if (trans)
    launch_k(k_syrk64<1>, dim3(T * (T + 1) / 2), dim3(256), (size_t)0, s, P, ldp, m, r, diag, scale, G64, ldg64, st);
  else
    launch_k(k_syrk64<0>, dim3(T * (T + 1) / 2), dim3(256), (size_t)0, s, P, ldp, m, r, diag, scale, G64, ldg64, st);
}

void chol64(double* G64, long long ldg64, int N, DevState* st, cudaStream_t s) {
  for (int kb = 0; kb < N; kb += kNB64) {
    const int nb = N - kb < kNB64 ? N - kb : kNB64;
    count_launch();
    launch_k(k_potrf64_diag, dim3(1), dim3(1024), (size_t)0, s, G64, ldg64, kb, nb, st);
    const int rem = N - kb - nb;
    if (rem > 0) {
      const int T = (rem + kT64 - 1) / kT64;
      count_launch(2);
      launch_k(k_trsm64_panel, dim3((rem + 127) / 128), dim3(128), (size_t)0, s, G64, ldg64, kb, nb, N,
               (const DevState*)st);
      launch_k(k_syrk64_update, dim3(T * (T + 1) / 2), dim3(256), (size_t)0, s, G64, ldg64, kb, nb, N,
               (const DevState*)st);
    }
  }
}

void launch_trsv64(const double* L, long long ldl, int N, const double* rhs, double* acc, int first, double alpha,
                   const DevState* st, cudaStream_t s) {
  if (N <= 0) return;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !done[dev]) {
    cudaFuncSetAttribute(k_trsv64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * kMaxM));
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  count_launch();
  launch_k(k_trsv64, dim3(1), dim3(1024), sizeof(double) * (size_t)N, s, L, ldl, N, rhs, acc, first, alpha, st);
}

void launch_refine_update(double* acc, const double* c, int len, double tau, DevState* st, cudaStream_t s) {
  if (len <= 0) return;
  count_launch();
  launch_k(k_refine_update, dim3(1), dim3(1024), (size_t)0, s, acc, c, len, tau * tau, st);
}

}  // namespace ssnal
