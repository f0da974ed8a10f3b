// Newton-system kernels (eqs. AJ_system, smw_formula):
//   * SYRK of the packed panel: G = kappa^{-1} I + A_J^T A_J (r x r) or
//     M = I + kappa A_J A_J^T (m x m), lower triangle, FP32 accumulation;
//   * blocked right-looking Cholesky factorisation (textbook algorithm, FP32);
//   * forward/backward substitution with the factor, accumulating the
//     correction into an FP64 vector (the solve of an iterative refinement).
#include <math.h>

#include "common.cuh"

namespace ssnal {

constexpr int kT = 32;  // tile edge

// Maps a linear block id onto a lower-triangular tile (ti >= tj).
__device__ __forceinline__ void tri_tile(int id, int& ti, int& tj) {
  int t = (int)((sqrtf(8.0f * (float)id + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= id) t++;
  while (t * (t + 1) / 2 > id) t--;
  ti = t;
  tj = id - t * (t + 1) / 2;
}

// G[a, b] = diag*[a == b] + sum_i P[i, a] P[i, b] for a >= b (a, b < r).
__global__ void __launch_bounds__(256) k_syrk_tn(const float* __restrict__ P, long long ldp, int m, int r,
                                                 float diag, float* __restrict__ G, long long ldg) {
  __shared__ float As[kT][kT + 1];
  __shared__ float Bs[kT][kT + 1];
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float acc[4] = {0, 0, 0, 0};
  const int a0 = ti * kT, b0 = tj * kT;
  for (int i0 = 0; i0 < m; i0 += kT) {
    const int i = i0 + tx;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int c = ty + 8 * e;
      As[tx][c] = (i < m && a0 + c < r) ? P[i + (long long)(a0 + c) * ldp] : 0.0f;
      Bs[tx][c] = (i < m && b0 + c < r) ? P[i + (long long)(b0 + c) * ldp] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < kT; ii++) {
      const float bv = Bs[ii][tx];
#pragma unroll
      for (int e = 0; e < 4; e++) acc[e] = fmaf(As[ii][ty + 8 * e], bv, acc[e]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int a = a0 + ty + 8 * e, b = b0 + tx;
    if (a < r && b < r && a >= b) G[a + (long long)b * ldg] = acc[e] + (a == b ? diag : 0.0f);
  }
}

// M[i, j] = [i == j] + kappa * sum_k P[i, k] P[j, k] for i >= j (i, j < m), K = r.
__global__ void __launch_bounds__(256) k_syrk_nt(const float* __restrict__ P, long long ldp, int m, long long r,
                                                 float kappa, float* __restrict__ G, long long ldg) {
  __shared__ float As[kT][kT + 1];
  __shared__ float Bs[kT][kT + 1];
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0, 0, 0, 0};
  const int i0 = ti * kT, j0 = tj * kT;
  for (long long k0 = 0; k0 < r; k0 += kT) {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const long long k = k0 + ty + 8 * e;
      As[ty + 8 * e][tx] = (k < r && i0 + tx < m) ? P[(i0 + tx) + k * ldp] : 0.0f;
      Bs[ty + 8 * e][tx] = (k < r && j0 + tx < m) ? P[(j0 + tx) + k * ldp] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kT; kk++) {
      const float bv = Bs[kk][tx];
#pragma unroll
      for (int e = 0; e < 4; e++) acc[e] = fmaf(As[kk][ty + 8 * e], bv, acc[e]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int i = i0 + ty + 8 * e, j = j0 + tx;
    if (i < m && j < m && i >= j) G[i + (long long)j * ldg] = kappa * acc[e] + (i == j ? 1.0f : 0.0f);
  }
}

// Unblocked Cholesky of the nb x nb diagonal block at (kb, kb).
__global__ void k_potrf_diag(float* __restrict__ G, long long ld, int kb, int nb, DevState* st) {
  __shared__ float a[kT][kT + 1];
  const int i = threadIdx.x, j = threadIdx.y;  // 32 x 32
  if (i < nb && j < nb && j <= i) a[i][j] = G[(kb + i) + (long long)(kb + j) * ld];
  __syncthreads();
  for (int k = 0; k < nb; k++) {
    if (i == k && j == k) {
      float piv = a[k][k];
      if (!(piv > 0.0f)) {
        st->chol_fail = 1;
        piv = 1.0f;
      }
      a[k][k] = sqrtf(piv);
    }
    __syncthreads();
    if (j == k && i > k && i < nb) a[i][k] = a[i][k] / a[k][k];
    __syncthreads();
    if (j > k && i >= j && i < nb) a[i][j] = fmaf(-a[i][k], a[j][k], a[i][j]);
    __syncthreads();
  }
  if (i < nb && j < nb && j <= i) G[(kb + i) + (long long)(kb + j) * ld] = a[i][j];
}

// Panel below the diagonal block: L21 = A21 L11^{-T}, one row per thread.
__global__ void k_trsm_panel(float* __restrict__ G, long long ld, int kb, int nb, int N) {
  __shared__ float L[kT][kT + 1];
  for (int e = threadIdx.x; e < kT * kT; e += blockDim.x) {
    const int i = e % kT, j = e / kT;
    L[i][j] = (i < nb && j < nb && j <= i) ? G[(kb + i) + (long long)(kb + j) * ld] : 0.0f;
  }
  __syncthreads();
  const int row = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= N) return;
  float xv[kT];
#pragma unroll
  for (int j = 0; j < kT; j++) {
    if (j < nb) {
      float s = G[row + (long long)(kb + j) * ld];
      for (int k = 0; k < j; k++) s = fmaf(-xv[k], L[j][k], s);
      xv[j] = s / L[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < kT; j++)
    if (j < nb) G[row + (long long)(kb + j) * ld] = xv[j];
}

// Trailing update A22 -= L21 L21^T on lower tiles of [k1, N).
__global__ void __launch_bounds__(256) k_syrk_update(float* __restrict__ G, long long ld, int kb, int nb, int N) {
  __shared__ float As[kT][kT + 1];
  __shared__ float Bs[kT][kT + 1];
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int k1 = kb + nb;
  const int i0 = k1 + ti * kT, j0 = k1 + tj * kT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int k = ty + 8 * e;
    As[k][tx] = (k < nb && i0 + tx < N) ? G[(i0 + tx) + (long long)(kb + k) * ld] : 0.0f;
    Bs[k][tx] = (k < nb && j0 + tx < N) ? G[(j0 + tx) + (long long)(kb + k) * ld] : 0.0f;
  }
  __syncthreads();
  float acc[4] = {0, 0, 0, 0};
#pragma unroll 8
  for (int k = 0; k < kT; k++) {
    const float bv = Bs[k][tx];
#pragma unroll
    for (int e = 0; e < 4; e++) acc[e] = fmaf(As[k][ty + 8 * e], bv, acc[e]);
  }
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int i = i0 + ty + 8 * e, j = j0 + tx;
    if (i < N && j < N && i >= j) {
      float* p = G + i + (long long)j * ld;
      *p = *p - acc[e];
    }
  }
}

// (L L^T) c = rhs by forward then backward substitution in one block;
// acc = c (first) or acc + c, in FP64.
constexpr int kTrsvThreads = 1024;
__global__ void __launch_bounds__(kTrsvThreads) k_trsv_llt(const float* __restrict__ L, long long ld, int N,
                                                           const double* __restrict__ rhs, double* __restrict__ acc,
                                                           int first) {
  extern __shared__ float z[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += blockDim.x) z[i] = (float)rhs[i];
  __syncthreads();
  // forward: L z' = z
  for (int jb = 0; jb < N; jb += kT) {
    const int nb = min(kT, N - jb);
    if (warp == 0) {
      for (int j = 0; j < nb; j++) {
        if (lane == j) z[jb + j] = z[jb + j] / L[(jb + j) + (long long)(jb + j) * ld];
        __syncwarp();
        const float zj = z[jb + j];
        if (lane > j && lane < nb) z[jb + lane] = fmaf(-L[(jb + lane) + (long long)(jb + j) * ld], zj, z[jb + lane]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = jb + nb + tid; i < N; i += blockDim.x) {
      float s = z[i];
      for (int j = 0; j < nb; j++) s = fmaf(-L[i + (long long)(jb + j) * ld], z[jb + j], s);
      z[i] = s;
    }
    __syncthreads();
  }
  // backward: L^T c = z'
  const int last = ((N - 1) / kT) * kT;
  for (int jb = last; jb >= 0; jb -= kT) {
    const int nb = min(kT, N - jb);
    if (warp == 0) {
      for (int j = nb - 1; j >= 0; j--) {
        if (lane == j) z[jb + j] = z[jb + j] / L[(jb + j) + (long long)(jb + j) * ld];
        __syncwarp();
        const float zj = z[jb + j];
        if (lane < j) z[jb + lane] = fmaf(-L[(jb + j) + (long long)(jb + lane) * ld], zj, z[jb + lane]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < jb; i += blockDim.x) {
      float s = z[i];
      const float* col = L + (long long)i * ld + jb;
      for (int j = 0; j < nb; j++) s = fmaf(-col[j], z[jb + j], s);
      z[i] = s;
    }
    __syncthreads();
  }
  for (int i = tid; i < N; i += blockDim.x) acc[i] = first ? (double)z[i] : acc[i] + (double)z[i];
}

// ---------------------------------------------------------------- launchers
void launch_syrk_tn(const float* P32, long long ldp32, int m, long long r, double diag, float* G, long long ldg,
                    cudaStream_t s) {
  int T = (int)((r + kT - 1) / kT);
  int blocks = T * (T + 1) / 2;
  if (blocks > 0) count_launch();
  if (blocks > 0) k_syrk_tn<<<blocks, 256, 0, s>>>(P32, ldp32, m, (int)r, (float)diag, G, ldg);
}

void launch_syrk_nt(const float* P32, long long ldp32, int m, long long r, double kappa, float* G, long long ldg,
                    cudaStream_t s) {
  int T = (m + kT - 1) / kT;
  int blocks = T * (T + 1) / 2;
  if (blocks > 0) count_launch();
  if (blocks > 0) k_syrk_nt<<<blocks, 256, 0, s>>>(P32, ldp32, m, r, (float)kappa, G, ldg);
}

void chol_factor(float* G, long long ldg, int N, DevState* st, cudaStream_t s) {
  for (int kb = 0; kb < N; kb += kCholNB) {
    const int nb = N - kb < kCholNB ? N - kb : kCholNB;
    count_launch();
    k_potrf_diag<<<1, dim3(32, 32), 0, s>>>(G, ldg, kb, nb, st);
    const int rem = N - kb - nb;
    if (rem > 0) {
      count_launch(2);
      k_trsm_panel<<<(rem + 255) / 256, 256, 0, s>>>(G, ldg, kb, nb, N);
      const int T = (rem + kT - 1) / kT;
      k_syrk_update<<<T * (T + 1) / 2, 256, 0, s>>>(G, ldg, kb, nb, N);
    }
  }
}

void launch_trsv_llt(const float* L, long long ldl, int N, const double* rhs, double* acc, int first,
                     cudaStream_t s) {
  if (N <= 0) return;
  count_launch();
  k_trsv_llt<<<1, kTrsvThreads, (size_t)N * sizeof(float), s>>>(L, ldl, N, rhs, acc, first);
}

}  // namespace ssnal
