// Newton-system kernels (eqs. AJ_system, smw_formula):
//   * SYRK of the packed panel: G = kappa^{-1} I + A_J^T A_J (r x r) or
//     M = I + kappa A_J A_J^T (m x m), lower triangle, FP32 accumulation;
//   * blocked right-looking Cholesky factorisation (textbook algorithm, FP32);
//   * forward/backward substitution with the factor, accumulating the
//     correction into an FP64 vector (the solve of an iterative refinement).
#include <cooperative_groups.h>
#include <cuda.h>
#include <math.h>

#include <mutex>

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
  pdl_entry();
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
  pdl_entry();
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
  pdl_entry();
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
  pdl_entry();
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
  pdl_entry();
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
                                                           int first, double alpha) {
  pdl_entry();
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
  for (int i = tid; i < N; i += blockDim.x)
    acc[i] = first ? alpha * (double)z[i] : acc[i] + alpha * (double)z[i];
}

// ---------------------------------------------------------------------------
// Small systems without inverse diagonal blocks (32 < N <= kSmallN: a factor
// whose caller wants no W_II, and the solves after a factor that left none): one
// CTA factors the matrix (column by column) or stages L in shared memory and
// solves.  One tile (N <= 32) goes to k_tile1_solve instead.
constexpr int kSmallN = 128;
constexpr int kSmallThreads = 1024;

__device__ void smem_forward_backward(const float* __restrict__ Ls, int ldl, int N, float* z) {
  // L z' = z then L^T c = z' with L in shared memory (lower, column-major, ld ldl).
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int jb = 0; jb < N; jb += kT) {
    const int nb = min(kT, N - jb);
    if (warp == 0) {
      float zl = lane < nb ? z[jb + lane] : 0.0f;
      for (int j = 0; j < nb; j++) {
        const float zj = __shfl_sync(0xffffffffu, zl / Ls[(jb + j) + (jb + j) * ldl], j);
        if (lane == j) zl = zj;
        if (lane > j && lane < nb) zl = fmaf(-Ls[(jb + lane) + (jb + j) * ldl], zj, zl);
      }
      if (lane < nb) z[jb + lane] = zl;
    }
    __syncthreads();
    for (int i = jb + nb + tid; i < N; i += blockDim.x) {
      float acc = z[i];
      for (int j = 0; j < nb; j++) acc = fmaf(-Ls[i + (jb + j) * ldl], z[jb + j], acc);
      z[i] = acc;
    }
    __syncthreads();
  }
  const int last = ((N - 1) / kT) * kT;
  for (int jb = last; jb >= 0; jb -= kT) {
    const int nb = min(kT, N - jb);
    if (warp == 0) {
      float zl = lane < nb ? z[jb + lane] : 0.0f;
      for (int j = nb - 1; j >= 0; j--) {
        const float zj = __shfl_sync(0xffffffffu, zl / Ls[(jb + j) + (jb + j) * ldl], j);
        if (lane == j) zl = zj;
        if (lane < j) zl = fmaf(-Ls[(jb + j) + (jb + lane) * ldl], zj, zl);
      }
      if (lane < nb) z[jb + lane] = zl;
    }
    __syncthreads();
    for (int i = tid; i < jb; i += blockDim.x) {
      float acc = z[i];
      for (int j = 0; j < nb; j++) acc = fmaf(-Ls[(jb + j) + i * ldl], z[jb + j], acc);
      z[i] = acc;
    }
    __syncthreads();
  }
}

constexpr size_t kSmallSmem = (size_t)(kSmallN * (kSmallN + 1) + kSmallN) * sizeof(float);

// Factor G (N <= kSmallN) with the matrix held in registers: thread t owns the
// elements (lane + 32a, warp + 32b), a, b < 4.  Column k: the owner of (k, k)
// takes the square root, the owners of column k scale it into a shared column
// buffer, and every thread applies the rank-one update to its own elements
// (two block barriers per column).  L is written back to G.
__global__ void __launch_bounds__(kSmallThreads) k_chol_small(float* __restrict__ G, long long ld, int N,
                                                              DevState* st) {
  pdl_entry();
  __shared__ float col[kSmallN];
  __shared__ float rdiag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float a[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = lane + 32 * p, j = warp + 32 * q;
      a[p][q] = (i < N && j < N && i >= j) ? G[i + (long long)j * ld] : 0.0f;
    }
  for (int k = 0; k < N; k++) {
    const int kl = k & 31, kb = k >> 5;
    if (lane == kl && warp == kl) {
      float piv = 0.0f;
#pragma unroll
      for (int p = 0; p < 4; p++)
        if (p == kb) piv = a[p][p];
      if (!(piv > 0.0f)) {
        st->chol_fail = 1;
        piv = 1.0f;
      }
      const float d = sqrtf(piv);
#pragma unroll
      for (int p = 0; p < 4; p++)
        if (p == kb) a[p][p] = d;
      rdiag = 1.0f / d;
    }
    __syncthreads();
    if (warp == kl) {
      const float rd = rdiag;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const int i = lane + 32 * p;
        if (i > k && i < N) {
#pragma unroll
          for (int q = 0; q < 4; q++)
            if (q == kb) {
              a[p][q] *= rd;
              col[i] = a[p][q];
            }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int j = warp + 32 * q;
      if (j > k && j < N) {
        const float cj = col[j];
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const int i = lane + 32 * p;
          if (i >= j && i < N) a[p][q] = fmaf(-col[i], cj, a[p][q]);
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = lane + 32 * p, j = warp + 32 * q;
      if (i < N && j < N && i >= j) G[i + (long long)j * ld] = a[p][q];
    }
}

// (L L^T) c = rhs with L (N <= kSmallN) staged into shared memory; acc = c or acc + c.
__global__ void __launch_bounds__(kSmallThreads) k_trsv_small(const float* __restrict__ L, long long ld, int N,
                                                              const double* __restrict__ rhs,
                                                              double* __restrict__ acc, int first, double alpha) {
  pdl_entry();
  extern __shared__ float sm_small[];
  float* Ls = sm_small;
  float* z = sm_small + kSmallN * (kSmallN + 1);
  const int ldl = kSmallN + 1;
  const int tid = threadIdx.x;
  for (int e = tid; e < N * N; e += blockDim.x) {
    const int i = e % N, j = e / N;
    Ls[i + j * ldl] = (i >= j) ? L[i + (long long)j * ld] : 0.0f;
  }
  for (int i = tid; i < N; i += blockDim.x) z[i] = (float)rhs[i];
  __syncthreads();
  smem_forward_backward(Ls, ldl, N, z);
  for (int i = tid; i < N; i += blockDim.x)
    acc[i] = first ? alpha * (double)z[i] : acc[i] + alpha * (double)z[i];
}

// ---------------------------------------------------------------------------
// Medium systems (kSmallN < N <= kMidN): forward and backward substitution in
// one CTA, block by block (32 rows/columns), with the next block of L copied
// into a second shared-memory buffer (cp.async) while the current block is
// solved, so that L2 latency stays off the critical path.
constexpr int kMidN = 768;
constexpr int kMidThreads = 1024;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Row block I of L (rows [32I, 32I+32) x columns [0, 32I + 32)) -> buf, column j at buf + 32 j.
__device__ __forceinline__ void prefetch_rows(const float* L, long long ld, int N, int I, float* buf) {
  const int r0 = 32 * I;
  const int ncols = min(r0 + 32, N);
  for (int e = threadIdx.x; e < ncols * 8; e += blockDim.x) {
    const int j = e >> 3, ch = e & 7;
    const int row = r0 + 4 * ch;
    const int valid = row < N ? min(4, N - row) : 0;
    const float* src = L + (long long)j * ld + (valid > 0 ? row : 0);
    cp_async16(buf + 32 * j + 4 * ch, src, valid * 4);
  }
}

// Column block I of L (columns [32I, 32I+32) x rows [32I, N)) -> buf, column c at buf + c ldb.
__device__ __forceinline__ void prefetch_cols(const float* L, long long ld, int N, int I, float* buf, int ldb) {
  const int r0 = 32 * I;
  const int nc = min(32, N - r0);
  const int chunks = ldb / 4;
  for (int e = threadIdx.x; e < nc * chunks; e += blockDim.x) {
    const int c = e / chunks, ch = e % chunks;
    const int row = r0 + 4 * ch;
    const int valid = row < N ? min(4, N - row) : 0;
    const float* src = L + (long long)(r0 + c) * ld + (valid > 0 ? row : r0);
    cp_async16(buf + c * ldb + 4 * ch, src, valid * 4);
  }
}

__global__ void __launch_bounds__(kMidThreads) k_trsv_mid(const float* __restrict__ L, long long ld, int N,
                                                          const double* __restrict__ rhs, double* __restrict__ acc,
                                                          int first, double alpha,
                                                          const float* __restrict__ Wdiag) {
  pdl_entry();
  extern __shared__ __align__(16) float sm_mid[];
  const int ldb = (N + 3) & ~3;
  float* buf[2] = {sm_mid, sm_mid + 32 * ldb};
  float* z = sm_mid + 64 * ldb;
  float* red = z + ldb;  // 32 x 33
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = (N + 31) / 32;
  for (int i = tid; i < N; i += blockDim.x) z[i] = (float)rhs[i];
  // ---- forward: z_I = L_II^{-1} (z_I - L[I, 0:I] z[0:I])
  prefetch_rows(L, ld, N, 0, buf[0]);
  cp_async_commit();
  for (int I = 0; I < T; I++) {
    if (I + 1 < T) prefetch_rows(L, ld, N, I + 1, buf[(I + 1) & 1]);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const float* B = buf[I & 1];
    const int r0 = 32 * I, nb = min(32, N - r0);
    float a = 0.0f;
    for (int j = warp; j < r0; j += 32) a = fmaf(B[32 * j + lane], z[j], a);
    red[warp * 33 + lane] = a;
    __syncthreads();
    if (warp == 0) {
      float sum = 0.0f;
      for (int w = 0; w < 32; w++) sum += red[w * 33 + lane];
      float zl = lane < nb ? z[r0 + lane] - sum : 0.0f;
      if (Wdiag) {
        // z_I = W_II (b_I - ...): a 32 x 32 product with the stored inverse block
        const float* W = Wdiag + (long long)I * 1024;
        float out = 0.0f;
        for (int t = 0; t < 32; t++) out = fmaf(W[lane * 32 + t], __shfl_sync(0xffffffffu, zl, t), out);
        zl = out;
      } else {
        const float rinv = lane < nb ? 1.0f / B[32 * (r0 + lane) + lane] : 0.0f;
        for (int j = 0; j < nb; j++) {
          const float zj = __shfl_sync(0xffffffffu, zl * rinv, j);
          if (lane == j) zl = zj;
          if (lane > j && lane < nb) zl = fmaf(-B[32 * (r0 + j) + lane], zj, zl);
        }
      }
      if (lane < nb) z[r0 + lane] = zl;
    }
    __syncthreads();
  }
  cp_async_wait0();
  __syncthreads();
  // ---- backward: c_I = L_II^{-T} (z_I - L[>I, I]^T c[>I])
  prefetch_cols(L, ld, N, T - 1, buf[(T - 1) & 1], ldb);
  cp_async_commit();
  for (int I = T - 1; I >= 0; I--) {
    if (I > 0) prefetch_cols(L, ld, N, I - 1, buf[(I - 1) & 1], ldb);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const float* B = buf[I & 1];
    const int r0 = 32 * I, nb = min(32, N - r0);
    // column c of the block sits at B + c*ldb, row i at offset i - r0
    float a = 0.0f;
    if (lane < nb)
      for (int i = r0 + 32 + warp; i < N; i += 32) a = fmaf(B[lane * ldb + (i - r0)], z[i], a);
    red[warp * 33 + lane] = a;
    __syncthreads();
    if (warp == 0) {
      float sum = 0.0f;
      for (int w = 0; w < 32; w++) sum += red[w * 33 + lane];
      float zl = lane < nb ? z[r0 + lane] - sum : 0.0f;
      if (Wdiag) {
        // c_I = W_II^T (z_I - ...)
        const float* W = Wdiag + (long long)I * 1024;
        float out = 0.0f;
        for (int t = 0; t < 32; t++) out = fmaf(W[t * 32 + lane], __shfl_sync(0xffffffffu, zl, t), out);
        zl = out;
      } else {
        const float rinv = lane < nb ? 1.0f / B[lane * ldb + lane] : 0.0f;
        for (int j = nb - 1; j >= 0; j--) {
          const float zj = __shfl_sync(0xffffffffu, zl * rinv, j);
          if (lane == j) zl = zj;
          if (lane < j) zl = fmaf(-B[lane * ldb + j], zj, zl);
        }
      }
      if (lane < nb) z[r0 + lane] = zl;
    }
    __syncthreads();
  }
  cp_async_wait0();
  for (int i = tid; i < N; i += blockDim.x)
    acc[i] = first ? alpha * (double)z[i] : acc[i] + alpha * (double)z[i];
}

// ---------------------------------------------------------------------------
// Cluster tile Cholesky (32 < N <= kClusterN on 8 CTAs, up to kCluster16N on 16).
// The lower triangle is cut into 32x32 tiles; tile (i, j), i >= j, with linear
// index i(i+1)/2 + j lives in the shared memory of CTA (index mod C) of one
// thread-block cluster of C CTAs.  Right-looking blocked Cholesky with a
// lookahead of one column.  In step k the four diagonal warps of the owner of
// (k+1, k+1) update that tile with panel tile (k+1, k) as soon as it has
// arrived, warp 0 factors it and pushes L^T of it to the owners of the panel
// tiles (i, k+1); each of those tiles belongs to one trailing warp for good,
// which updates it with panel k, solves L_i,k+1 L_k+1,k+1^T = A_i,k+1 once the
// diagonal factor has arrived and pushes the solved tile (stored transposed) into
// the panel buffer of every CTA, the consumer on the critical chain first; then it
// applies panel k to its other tiles.  The diagonal warps apply panel k to the
// other owned diagonal tiles.  Pushes are bulk shared-to-shared copies that
// complete on the receivers' per-tile mbarriers.  Where two panel buffers fit in
// shared memory the cluster barrier that frees a buffer is split (each warp
// waits for the previous phase only where it pushes); otherwise a full cluster
// barrier precedes each push.  At the end each CTA inverts its diagonal tiles for
// the triangular solves.  Rows and columns beyond N are padded with the
// identity, so the factor of the padded matrix is L plus an identity block.
// Layout in shared memory: owned tiles (row stride 33; off-diagonal tiles are
// stored transposed with row stride 32 once solved), the panel buffer(s) of
// transposed tiles (32 x 32), L^T of the current diagonal tile with its
// reciprocal diagonal, and a staging copy of it; the mbarriers are static.
// With hrow (N not a multiple of 32) the forward substitution z = L^{-1} h runs inside
// the factor: h^T is appended as row N of the matrix (a padding row of the last tile
// row) with the diagonal entry kAugDiag, so the right-looking factor of the augmented
// matrix forms row N of its factor as z^T (the panel solves of the last tile row apply
// the same substitution to it), at no extra tile.  z goes to zout; that row is then reset
// to a unit row, so the factor and its inverse diagonal blocks of the first N rows are
// those of G alone.
namespace cgx = cooperative_groups;
constexpr int kClusterCTAs = 8;
// Threads per CTA of k_chol_cluster: warps 0-3 keep the diagonal tiles (warp 0
// factors), warps 4 and 8 share warp 0's scheduler and only take part in the
// barriers, warps 5-7 and 9-11 do the trailing updates.
constexpr int kCholThreads = 384;
constexpr int kCholTrail = 6;  // trailing warps
constexpr int kClusterN = 640;
constexpr int kClusterT = kClusterN / 32;                 // 20 tiles per side
constexpr int kCluster16CTAs = 16;                        // the wide variant: one 16-CTA cluster (where allowed)
constexpr int kCluster16N = 864;                          // its limit: 27 tiles per side
constexpr int kClusterTMax = kCluster16N / 32;
constexpr size_t kClusterSmemLimit = 232448 - 2048;       // dynamic shared memory per CTA (static part aside)
constexpr int kTileF = 32 * 33;                           // floats per padded tile
constexpr unsigned kTileBytes = kTileF * sizeof(float);   // 4224, a multiple of 16
constexpr unsigned kPanelBytes = 1024 * sizeof(float);    // a transposed panel tile
// diagonal entry of the appended row h^T: its pivot kAugDiag - ||z||^2 stays positive
// and finite (L_NN about 1e15, 1 / L_NN about 1e-15)
constexpr float kAugDiag = 1e30f;

__host__ __device__ constexpr int cluster_slots(int T, int C = kClusterCTAs) { return (T * (T + 1) / 2 + C - 1) / C; }
// bytes of shared memory with nb panel buffers
__host__ __device__ constexpr size_t cluster_bytes(int T, int C, int nb) {
  return ((size_t)(cluster_slots(T, C) + 2) * kTileF + (size_t)nb * T * 1024) * sizeof(float) + 32;
}
// the panel is double-buffered wherever two buffers fit (T <= 16 with 8 CTAs, T <= 19 with 16)
__host__ __device__ constexpr int cluster_nbuf(int T, int C = kClusterCTAs) {
  return cluster_bytes(T, C, 2) <= kClusterSmemLimit ? 2 : 1;
}
__host__ __device__ constexpr size_t cluster_smem(int T, int C = kClusterCTAs) {
  return cluster_bytes(T, C, cluster_nbuf(T, C));
}
constexpr size_t cluster_smem_max(int C = kClusterCTAs, int Tmax = kClusterT) {
  size_t m = 0;
  for (int T = 5; T <= Tmax; T++) m = cluster_smem(T, C) > m ? cluster_smem(T, C) : m;
  return m;
}
static_assert(cluster_slots(kClusterT) <= 32, "one lane per owned slot");
static_assert(cluster_slots(kClusterTMax, kCluster16CTAs) <= 32, "one lane per owned slot");
static_assert(cluster_smem_max() <= kClusterSmemLimit, "shared memory per CTA");
static_assert(cluster_smem_max(kCluster16CTAs, kClusterTMax) <= kClusterSmemLimit, "shared memory per CTA");
static_assert(cluster_nbuf(16) == 2 && cluster_nbuf(17) == 1, "8 CTAs: two panel buffers up to 16 tile rows");
static_assert(cluster_nbuf(19, kCluster16CTAs) == 2, "16 CTAs: two panel buffers up to 19 tile rows");

// bulk copy of `bytes` from this CTA's shared memory to (possibly) another
// CTA's, completing `bytes` on that CTA's mbarrier
__device__ __forceinline__ void bulk_s2c(unsigned dst, unsigned src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ int tri_index(int i, int j) { return i * (i + 1) / 2 + j; }

// C -= Li Lj^T for 32x32 tiles by one warp; C has row stride 33, Pi = Li^T and
// Pj = Lj^T have row stride 32 (one 128-bit load brings 4 rows of Li at one k).
// Lane (tr, tc) owns rows 4tr..4tr+3 and columns 8tc..8tc+7 of C.
__device__ __forceinline__ void tile_update_warp(float* C, const float* Pi, const float* Pj, int lane) {
  const int tr = lane >> 2, tc = lane & 3;
  float acc[4][8] = {};
#pragma unroll 4
  for (int q = 0; q < 32; q++) {
    const float4 a = reinterpret_cast<const float4*>(Pi + q * 32)[tr];
    const float4 b0 = reinterpret_cast<const float4*>(Pj + q * 32)[2 * tc];
    const float4 b1 = reinterpret_cast<const float4*>(Pj + q * 32)[2 * tc + 1];
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 8; v++) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 8; v++) C[(4 * tr + u) * 33 + 8 * tc + v] -= acc[u][v];
}

// Factor the 32x32 tile D (row stride 33) in place, D = L L^T, by one warp,
// two pivots per round: lane l holds row l; in round q (pivots q, q+1) every
// lane publishes its entries of columns q and q+1 in cb (2 x 32 floats,
// double-buffered), factors the 2x2 pivot block from broadcast loads, forms
// L_lq, L_l,q+1 and applies the rank-2 update as a Schur complement on the
// unscaled columns, A_lc -= alpha_l A_cq + beta_l A_c,q+1, so that one broadcast
// serves both pivots.  Entries above the diagonal collect products that are
// never read.  Also writes U = L^T (row stride 32) and the reciprocal diagonal
// to U[1024..].  Returns false if a pivot was not positive (it is replaced by 1).
__device__ __forceinline__ bool factor_tile_warp(float* D, float* U, float* cb, int lane) {
  float row[32];
#pragma unroll
  for (int c = 0; c < 32; c++) row[c] = (c <= lane) ? D[lane * 33 + c] : 0.0f;
  bool bad = false;
  float rl = 1.0f;
#pragma unroll
  for (int q = 0; q < 32; q += 2) {
    float* col = cb + ((q >> 1) & 1) * 64;  // [0..31]: column q, [32..63]: column q+1
    const float u0 = row[q], u1 = row[q + 1];  // A_lq, A_l,q+1 after the earlier rounds
    col[lane] = u0;
    col[32 + lane] = u1;
    __syncwarp();
    float a00 = col[q], a10 = col[q + 1], a11 = col[32 + q + 1];
    if (!(a00 > 0.0f)) {
      bad = true;
      a00 = 1.0f;
    }
    const float r0 = rsqrtf(a00);
    const float l10 = a10 * r0;
    float d1 = fmaf(-l10, l10, a11);
    if (!(d1 > 0.0f)) {
      bad = true;
      d1 = 1.0f;
    }
    const float r1 = rsqrtf(d1);
    const float x0 = u0 * r0;                  // L_lq
    const float x1 = fmaf(-x0, l10, u1) * r1;  // L_l,q+1
    row[q] = x0;
    row[q + 1] = x1;
    if (lane == q) rl = r0;
    if (lane == q + 1) rl = r1;
    const float beta = x1 * r1;
    const float alpha = r0 * fmaf(-beta, l10, x0);
#pragma unroll
    for (int g = 0; g < 8; g++) {
      if (4 * g + 3 > q + 1) {
        const float4 v0 = reinterpret_cast<const float4*>(col)[g];
        const float4 v1 = reinterpret_cast<const float4*>(col + 32)[g];
        const float c0[4] = {v0.x, v0.y, v0.z, v0.w}, c1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int e = 0; e < 4; e++)
          if (4 * g + e > q + 1) row[4 * g + e] = fmaf(-alpha, c0[e], fmaf(-beta, c1[e], row[4 * g + e]));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 32; c++) {
    const float v = (c <= lane) ? row[c] : 0.0f;
    D[lane * 33 + c] = v;
    U[c * 32 + lane] = v;
  }
  U[1024 + lane] = rl;
  return !bad;
}

// D -= P P^T on rows 8g .. 8g+7 of the lower triangle of the 32x32 tile D (row
// stride 33) by one warp; P = L^T of one panel tile (row stride 32).  Same
// operands and summation order per entry as tile_update_warp.
__device__ __forceinline__ void diag_update_rows(float* D, const float* P, int g, int lane) {
  const int r = 8 * g + (lane >> 2), c0 = 8 * (lane & 3);
  float acc[8] = {};
#pragma unroll 8
  for (int q = 0; q < 32; q++) {
    const float a = P[q * 32 + r];
    const float4 b0 = reinterpret_cast<const float4*>(P + q * 32 + c0)[0];
    const float4 b1 = reinterpret_cast<const float4*>(P + q * 32 + c0)[1];
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int e = 0; e < 8; e++) acc[e] = fmaf(a, bv[e], acc[e]);
  }
#pragma unroll
  for (int e = 0; e < 8; e++)
    if (c0 + e <= r) D[r * 33 + c0 + e] -= acc[e];
}

// Solve X L^T = A for one 32x32 panel tile A (row stride 33) by one warp, lane
// r owning row r; U = L^T (row stride 32) with 1/L_jj at U[1024 + j].  X is
// written back transposed (row stride 32) over A.
__device__ __forceinline__ void panel_solve_warp(float* A, const float* U, int lane) {
  float x[32];
#pragma unroll
  for (int c = 0; c < 32; c++) x[c] = A[lane * 33 + c];
#pragma unroll
  for (int j = 0; j < 32; j++) {
    x[j] *= U[1024 + j];
    const float4* u4 = reinterpret_cast<const float4*>(U + j * 32);
#pragma unroll
    for (int g = 0; g < 8; g++) {
      if (4 * g + 3 > j) {
        const float4 v = u4[g];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; e++)
          if (4 * g + e > j) x[4 * g + e] = fmaf(-x[j], vv[e], x[4 * g + e]);
      }
    }
  }
  __syncwarp();  // every lane has read its row before the transposed write
#pragma unroll
  for (int c = 0; c < 32; c++) A[c * 32 + lane] = x[c];
}

// A warp pushes `bytes` from src (this CTA) to dst in the CTAs of `mask`,
// completing on their mbarrier `bar`: the copy to CTA `first` (the next
// consumer on the critical chain) is issued on its own, then lanes 0..7 issue
// the others.  The data must have been fenced for the async proxy and
// synchronised within the warp.
template <int C>
__device__ __forceinline__ void push_tile(unsigned src, unsigned dst, unsigned bytes, unsigned bar, unsigned mask,
                                          int first, int lane) {
  if (lane == 0 && (mask >> first & 1u)) bulk_s2c(cluster_addr(dst, first), src, bytes, cluster_addr(bar, first));
  __syncwarp();
  if (lane < C && lane != first && (mask >> lane & 1u))
    bulk_s2c(cluster_addr(dst, lane), src, bytes, cluster_addr(bar, lane));
}

// W = L^{-1} for the factored 32 x 32 diagonal tile D (lower, row stride 33) by one warp:
// lane j forms column j by forward substitution; W is stored row-major at Wout.
// (Four partial sums per entry keep the dependent chain of each step short.)
__device__ __forceinline__ void inverse_diag_warp(const float* D, float* __restrict__ Wout, int lane) {
  float w[32];
  const float rd = __frcp_rn(D[lane * 33 + lane]);  // 1 / L_ll, formed off the chain
#pragma unroll
  for (int i = 0; i < 32; i++) {
    float s[4] = {(i == lane) ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < i; q++) s[q & 3] = fmaf(-D[i * 33 + q], w[q], s[q & 3]);
    w[i] = ((s[0] + s[1]) + (s[2] + s[3])) * __shfl_sync(0xffffffffu, rd, i);
  }
#pragma unroll
  for (int i = 0; i < 32; i++) Wout[i * 32 + lane] = w[i];
}

// Named barrier of the four diagonal warps (0-3) of a CTA.
__device__ __forceinline__ void diag_quad_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kCholThreads)
    k_chol_cluster(float* __restrict__ G, long long ld, int N, DevState* st, float* __restrict__ Wdiag,
                   const double* __restrict__ hrow, float* __restrict__ zout) {
  pdl_entry();
  __shared__ __align__(16) float fcol[128];                  // column exchange of the diagonal factor
  __shared__ __align__(8) unsigned long long tbar_s[2 * kClusterTMax];  // panel tile arrivals per (buffer, tile row)
  __shared__ __align__(8) unsigned long long dbar_s;               // diagonal factor arrivals
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) float csm[];
  const int T = (N + 31) / 32;
  const int nbuf = cluster_nbuf(T, C);
  float* own = csm;                                        // owned tiles
  float* panel = own + cluster_slots(T, C) * kTileF;          // nbuf x T transposed panel tiles
  float* dbuf = panel + nbuf * T * 1024;                   // L^T of the next diagonal tile, 1/diag at [1024..]
  float* ustage = dbuf + kTileF;                           // the owner of a diagonal tile builds that buffer here
  const unsigned dbar = smem_u32(&dbar_s);
  __shared__ int slot_ij[32];                    // (i << 8) | j of the tile in each owned slot
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned all = (1u << C) - 1u;
  const int nslots = (T * (T + 1) / 2 - rank + C - 1) / C;
  for (int sl = tid; sl < nslots; sl += blockDim.x) {
    int ti, tj;
    tri_tile(rank + sl * C, ti, tj);
    slot_ij[sl] = (ti << 8) | tj;
  }
  __syncthreads();
  // lane l of every warp keeps (i, j) of slot l: the per-step work lists are
  // ballots over these
  const int my_i = lane < nslots ? slot_ij[lane] >> 8 : -1;
  const int my_j = lane < nslots ? slot_ij[lane] & 255 : -1;
  auto panel_tile = [&](int k, int i) { return panel + ((k % nbuf) * T + i) * 1024; };
  // tile i of panel k arrives on tbar(k, i); its phase parity is tpar(k)
  auto tbar = [&](int k, int i) { return smem_u32(&tbar_s[(k % nbuf) * kClusterTMax + i]); };
  auto tpar = [&](int k) { return (unsigned)((k / nbuf) & 1); };
  auto owner = [&](int i, int j) { return tri_index(i, j) % C; };
  // the first consumer of panel tile (i, k) on the critical chain: the owner of
  // (k+1, k+1) for the first tile, else the owner of (i, k+1), which solves it next
  auto first_of = [&](int i, int k) { return i == k + 1 ? owner(k + 1, k + 1) : owner(i, k + 1); };

  // ---- load the owned tiles, zero outside N x N; then the identity on the padded
  //      diagonal.  Item e is rows 4q .. 4q+3 of column c of slot e / 256 (q = e mod 8,
  //      c = (e / 8) mod 32): one 16-byte load where G and ld allow it, eight loads in
  //      flight per thread before their shared-memory stores (bank 4q + c + row within
  //      the four: conflict-free).  The strict upper triangle of a diagonal tile is
  //      loaded too and never read.
  {
    const bool v4 = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
    const int items = nslots * 256;
    for (int b0 = 0; b0 < items; b0 += 8 * (int)blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int e = b0 + k * (int)blockDim.x + tid;
        v[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e >= items) continue;
        const int sl = e >> 8, q = e & 7, c = (e >> 3) & 31;
        const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
        const int gi = ti * 32 + 4 * q, gj = tj * 32 + c;
        if (gj >= N) continue;
        const float* src = G + gi + (long long)gj * ld;
        if (v4 && gi + 3 < N) {
          v[k] = *reinterpret_cast<const float4*>(src);
        } else {
          if (gi < N) v[k].x = src[0];
          if (gi + 1 < N) v[k].y = src[1];
          if (gi + 2 < N) v[k].z = src[2];
          if (gi + 3 < N) v[k].w = src[3];
        }
      }
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int e = b0 + k * (int)blockDim.x + tid;
        if (e >= items) continue;
        const int sl = e >> 8, q = e & 7, c = (e >> 3) & 31;
        float* dst = own + sl * kTileF + (4 * q) * 33 + c;
        dst[0] = v[k].x;
        dst[33] = v[k].y;
        dst[66] = v[k].z;
        dst[99] = v[k].w;
      }
    }
  }
  __syncthreads();
  const bool aug = hrow != nullptr;  // the host passes h only when N % 32 != 0
  const int rN = N - 32 * (T - 1);   // row N within the last tile row (with aug)
  for (int sl = 0; sl < nslots; sl++) {
    const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
    if (ti == tj && tid < 32 && ti * 32 + tid >= N)
      own[sl * kTileF + tid * 33 + tid] = (aug && ti * 32 + tid == N) ? kAugDiag : 1.0f;
    if (aug && ti == T - 1 && tid < 32 && tj * 32 + tid < N) own[sl * kTileF + rN * 33 + tid] = (float)hrow[tj * 32 + tid];
  }
  // panel-column ownership of column j: the CTAs owning a tile (i, j), i > j
  auto receivers_of = [&](int j) {
    unsigned m = 0;
    for (int i = j + 1; i < T; i++) m |= 1u << (tri_index(i, j) % C);
    return m;
  };
  // one barrier per thread.  Armed for the first diagonal push and the first panel(s)
  // (tile i of panel b, i > b): panel k + nbuf is armed at the end of step k, once every
  // tile of panel k has arrived
  if (tid < nbuf * T) {
    const int b = tid / T, i = tid % T;
    const unsigned bar = smem_u32(&tbar_s[b * kClusterTMax + i]);
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (i > b) mbar_expect_tx(bar, kPanelBytes);
  }
  if (tid == kCholThreads - 1) {
    mbar_init(dbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (receivers_of(0) >> rank & 1u) mbar_expect_tx(dbar, kTileBytes);
  }
  __syncthreads();
  cluster.sync();
  if (nbuf == 2) cluster_arrive();  // the split barrier runs one phase ahead
  bool ok = true, bad = false;
  unsigned dphase = 0;  // completed phases of dbar

  // ---- prologue: factor (0, 0), solve and push panel column 0
  if (rank == 0 && warp == 0) {
    bad |= !factor_tile_warp(own, ustage, fcol, lane);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    push_tile<C>(smem_u32(ustage), smem_u32(dbuf), kTileBytes, dbar, receivers_of(0), owner(1, 0), lane);
  }
  if (receivers_of(0) >> rank & 1u) {
    if (ok && !mbar_wait(dbar, dphase & 1u)) ok = false;
    dphase++;
    unsigned m = __ballot_sync(0xffffffffu, my_j == 0 && my_i > 0);
    for (int e = 0; m; e++, m &= m - 1) {
      if ((e & 7) != warp) continue;
      const int sl = __ffs(m) - 1, i = __shfl_sync(0xffffffffu, my_i, sl);
      float* Ai = own + sl * kTileF;
      panel_solve_warp(Ai, dbuf, lane);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      push_tile<C>(smem_u32(Ai), smem_u32(panel_tile(0, i)), kPanelBytes, tbar(0, i), all, first_of(i, 0), lane);
    }
  }

  for (int k = 0; k + 1 < T; k++) {
    const int next = tri_index(k + 1, k + 1);
    const bool diag_here = next % C == rank;
    const unsigned recv_next = receivers_of(k + 1);
    const bool solve_here = (recv_next >> rank & 1u) != 0;
    // arm for the push of the next diagonal tile (the previous one was consumed)
    if (tid == 0 && solve_here) mbar_expect_tx(dbar, kTileBytes);
    // ---- diagonal warps 0-3 (one per scheduler) keep the owned diagonal tiles and
    //      synchronise only with each other.  In the owner of (k+1, k+1) they update
    //      it with panel tile (k+1, k), eight rows each, as soon as that tile has
    //      arrived; warp 0 factors and publishes it while warps 1-3 apply panel k
    //      to the other owned diagonal tiles (elsewhere all four share those).
    if (warp < 4) {
      diag_quad_sync();  // the four are done with step k-1
      if (diag_here) {
        float* D = own + (next / C) * kTileF;
        if (ok && !mbar_wait(tbar(k, k + 1), tpar(k))) ok = false;
        if (ok) diag_update_rows(D, panel_tile(k, k + 1), warp, lane);
        diag_quad_sync();
        if (warp == 0) {
          bad |= !factor_tile_warp(D, ustage, fcol, lane);
          if (recv_next) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            push_tile<C>(smem_u32(ustage), smem_u32(dbuf), kTileBytes, dbar, recv_next,
                      k + 2 < T ? owner(k + 2, k + 1) : rank, lane);
          }
        }
      }
      if (ok && !(diag_here && warp == 0)) {
        const int nd = diag_here ? 3 : 4, me = diag_here ? warp - 1 : warp;
        int e = 0;
        for (unsigned m = __ballot_sync(0xffffffffu, my_i == my_j && my_i > k + 1); m; m &= m - 1, e++) {
          if (e % nd != me) continue;
          const int sl = __ffs(m) - 1, ti = __shfl_sync(0xffffffffu, my_i, sl);
          if (ok && !mbar_wait(tbar(k, ti), tpar(k))) ok = false;
          tile_update_warp(own + sl * kTileF, panel_tile(k, ti), panel_tile(k, ti), lane);
        }
      }
    }
    // ---- trailing warps 5-7, 9-11 (schedulers 1-3): owned off-diagonal slot s
    //      belongs to trailing warp s % 6 for good, so all updates of a tile, its
    //      solve and its push run in one warp's program order.  The tiles of panel column k+1 come first, each
    //      solved once the diagonal factor has arrived and pushed at once.
    unsigned mine = 0;    // slots of panel column k+1 this warp updated and solved
    bool pushed = false;  // this warp has waited on the cluster barrier and pushed them
    const int trail = warp >= 5 && warp != 8 ? (warp < 8 ? warp - 5 : warp - 6) : -1;
    if (trail >= 0 && ok) {
      const bool lane_mine = lane % kCholTrail == trail;
      for (unsigned m = __ballot_sync(0xffffffffu, lane_mine && my_j == k + 1 && my_i > k + 1); m; m &= m - 1) {
        const int sl = __ffs(m) - 1;
        const int ti = __shfl_sync(0xffffffffu, my_i, sl);
        if (ok && !mbar_wait(tbar(k, ti), tpar(k))) ok = false;
        if (ok && !mbar_wait(tbar(k, k + 1), tpar(k))) ok = false;
        tile_update_warp(own + sl * kTileF, panel_tile(k, ti), panel_tile(k, k + 1), lane);
        mine |= 1u << sl;
      }
      if (mine) {
        if (ok && !mbar_wait(dbar, dphase & 1u)) ok = false;
        for (unsigned m = mine; m; m &= m - 1) panel_solve_warp(own + (__ffs(m) - 1) * kTileF, dbuf, lane);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (nbuf == 2) {
          // the buffer of panel k+1 held panel k-1, free once every thread has
          // arrived after step k-1: wait for that phase here and push at once,
          // ahead of this warp's share of the rest of the trailing update
          cluster_wait();
          pushed = true;
          for (unsigned m = mine; m; m &= m - 1) {
            const int sl = __ffs(m) - 1, i = __shfl_sync(0xffffffffu, my_i, sl);
            push_tile<C>(smem_u32(own + sl * kTileF), smem_u32(panel_tile(k + 1, i)), kPanelBytes, tbar(k + 1, i), all,
                      first_of(i, k + 1), lane);
          }
        }
      }
      for (unsigned m = __ballot_sync(0xffffffffu, lane_mine && my_j > k + 1 && my_i != my_j); m; m &= m - 1) {
        const int sl = __ffs(m) - 1;
        const int ti = __shfl_sync(0xffffffffu, my_i, sl), tj = __shfl_sync(0xffffffffu, my_j, sl);
        if (ok && !mbar_wait(tbar(k, ti), tpar(k))) ok = false;
        if (ok && !mbar_wait(tbar(k, tj), tpar(k))) ok = false;
        tile_update_warp(own + sl * kTileF, panel_tile(k, ti), panel_tile(k, tj), lane);
      }
    }
    // warp 5: every tile of panel k has arrived; arm panel k + nbuf, which reuses
    // the same barriers (before this warp's cluster arrive, hence before any push)
    if (warp == 5) {
      bool got = ok;
      for (int i = k + 1 + lane; i < T; i += 32)
        if (got && !mbar_wait(tbar(k, i), tpar(k))) got = false;
      got = __all_sync(0xffffffffu, got);
      if (!got) ok = false;
      if (got && lane == 0)
        for (int i = k + nbuf + 1; i < T; i++) mbar_expect_tx(tbar(k + nbuf, i), kPanelBytes);
      __syncwarp();
    }
    if (solve_here) {
      // warp 0 (tid 0 arms the next phase) makes sure this phase has completed
      if (warp == 0 && ok && !mbar_wait(dbar, dphase & 1u)) ok = false;
      dphase++;
    }
    // the buffer that panel k+1 goes to must be free: with two buffers it was
    // read in step k-1 (the wait matches the arrive issued then; warps that
    // pushed have waited already); with one it is panel k itself, so every CTA
    // must be done with this step
    if (nbuf == 2) {
      if (!pushed) cluster_wait();
      cluster_arrive();  // this warp is done reading panel k
    } else {
      cluster.sync();
    }
    if (!pushed)  // each warp pushes the tiles it solved (after its own proxy fence)
      for (unsigned m = mine; m; m &= m - 1) {
        const int sl = __ffs(m) - 1, i = __shfl_sync(0xffffffffu, my_i, sl);
        push_tile<C>(smem_u32(own + sl * kTileF), smem_u32(panel_tile(k + 1, i)), kPanelBytes, tbar(k + 1, i), all,
                  first_of(i, k + 1), lane);
      }
  }
  if (nbuf == 2) cluster_wait();
  if (bad) st->chol_fail = 1;
  if (!ok) st->timeout = 1;
  __syncthreads();
  if (aug) {
    // z = row N of the factor (solved off-diagonal tiles are stored transposed); then
    // row N of the last diagonal tile becomes a unit row again
    for (int sl = 0; sl < nslots; sl++) {
      const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
      if (ti != T - 1 || tid >= 32 || tj * 32 + tid >= N) continue;
      const float* src = own + sl * kTileF;
      zout[tj * 32 + tid] = (ti == tj) ? src[rN * 33 + tid] : src[tid * 32 + rN];
    }
    __syncthreads();
    for (int sl = 0; sl < nslots; sl++) {
      const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
      if (ti == T - 1 && tj == T - 1 && tid < 32) own[sl * kTileF + rN * 33 + tid] = tid == rN ? 1.0f : 0.0f;
    }
    __syncthreads();
  }
  // ---- inverse diagonal blocks for the triangular solves, W_kk = L_kk^{-1}:
  //      one warp per owned diagonal tile, lane j forms column j of W by forward
  //      substitution; W is stored row-major
  if (Wdiag) {
    unsigned m = __ballot_sync(0xffffffffu, my_i >= 0 && my_i == my_j);
    for (int e = 0; m; e++, m &= m - 1) {
      if ((e & 7) != warp) continue;
      const int sl = __ffs(m) - 1, k = __shfl_sync(0xffffffffu, my_i, sl);
      inverse_diag_warp(own + sl * kTileF, Wdiag + (long long)k * 1024, lane);
    }
  }
  // ---- write the factor back (lower part, inside N).  Off-diagonal tiles are stored
  //      transposed (column c of the tile is contiguous): rows 4q .. 4q+3 of a column
  //      go out as one 16-byte store where G and ld allow it; diagonal tiles (row stride
  //      33) entry by entry, consecutive threads on consecutive rows of a column.
  {
    const bool v4 = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
    for (int e = tid; e < nslots * 256; e += blockDim.x) {
      const int sl = e >> 8, q = e & 7, c = (e >> 3) & 31;
      const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
      const int gi = ti * 32 + 4 * q, gj = tj * 32 + c;
      if (ti == tj || gj >= N || gi >= N) continue;
      const float4 val = *reinterpret_cast<const float4*>(own + sl * kTileF + c * 32 + 4 * q);
      float* dst = G + gi + (long long)gj * ld;
      if (v4 && gi + 3 < N) {
        *reinterpret_cast<float4*>(dst) = val;
      } else {
        dst[0] = val.x;
        if (gi + 1 < N) dst[1] = val.y;
        if (gi + 2 < N) dst[2] = val.z;
        if (gi + 3 < N) dst[3] = val.w;
      }
    }
    for (int sl = 0; sl < nslots; sl++) {
      const int ti = slot_ij[sl] >> 8, tj = slot_ij[sl] & 255;
      if (ti != tj) continue;
      const float* src = own + sl * kTileF;
      for (int e = tid; e < 1024; e += blockDim.x) {
        const int r = e & 31, c = e >> 5;
        const int gi = ti * 32 + r, gj = tj * 32 + c;
        if (gi < N && gj < N && gi >= gj) G[gi + (long long)gj * ld] = src[r * 33 + c];
      }
    }
  }
}
template __global__ void k_chol_cluster<kClusterCTAs>(float*, long long, int, DevState*, float*, const double*, float*);
template __global__ void k_chol_cluster<kCluster16CTAs>(float*, long long, int, DevState*, float*, const double*,
                                                         float*);

// ---------------------------------------------------------------------------
// One-tile Newton systems (N <= 32) by one warp.  The lower triangle of G is
// staged into a 32x32 shared tile padded with the identity beyond N.  With
// `factor` the tile is factored by factor_tile_warp, L is written back to the
// lower triangle of G and a non-positive pivot sets st->chol_fail; otherwise G
// already holds L.  If rhs != nullptr, (L L^T) c = rhs is then solved by two
// 32-step chains with lane l holding entry l: each row of L (forward) or column
// (backward) is scaled once by 1/L_ll, so step q broadcasts lane q's final
// value and the lanes still open subtract one product.  acc = alpha c, or
// acc + alpha c when !first (FP64 output).
__global__ void __launch_bounds__(32) k_tile1_solve(float* __restrict__ G, long long ld, int N, int factor,
                                                    DevState* st, const double* __restrict__ rhs,
                                                    double* __restrict__ acc, int first, double alpha) {
  pdl_entry();
  __shared__ float D[32 * 33];
  __shared__ __align__(16) float U[1024 + 32];
  __shared__ __align__(16) float cb[128];
  const int lane = threadIdx.x;
#pragma unroll 8
  for (int j = 0; j < 32; j++) {
    float v = (lane == j) ? 1.0f : 0.0f;
    if (lane < N && j < N && lane >= j) v = G[lane + (long long)j * ld];
    D[lane * 33 + j] = v;
  }
  __syncwarp();
  if (factor) {
    const bool ok = factor_tile_warp(D, U, cb, lane);
    __syncwarp();
    for (int j = 0; j < N; j++)
      if (lane >= j && lane < N) G[lane + (long long)j * ld] = D[lane * 33 + j];
    if (!__all_sync(0xffffffffu, ok) && lane == 0) st->chol_fail = 1;
  }
  if (!rhs) return;
  const float rl = __frcp_rn(D[lane * 33 + lane]);
  float a[32], b[32];
#pragma unroll
  for (int q = 0; q < 32; q++) {
    a[q] = D[lane * 33 + q] * rl;  // L_lq / L_ll, read for q < l
    b[q] = D[q * 33 + lane] * rl;  // L_ql / L_ll, read for q > l
  }
  float r = lane < N ? (float)rhs[lane] * rl : 0.0f;
#pragma unroll
  for (int q = 0; q < 32; q++) {
    if (q < N) {
      const float zq = __shfl_sync(0xffffffffu, r, q);
      if (lane > q) r = fmaf(-a[q], zq, r);
    }
  }
  r *= rl;  // z_l / L_ll
#pragma unroll
  for (int q = 31; q >= 0; q--) {
    if (q < N) {
      const float cq = __shfl_sync(0xffffffffu, r, q);
      if (lane < q) r = fmaf(-b[q], cq, r);
    }
  }
  if (lane < N) acc[lane] = first ? alpha * (double)r : acc[lane] + alpha * (double)r;
}

// ---------------------------------------------------------------------------
// Triangular solves with the factor of the cluster Cholesky (N <= kClusterN)
// and its inverse diagonal blocks W_II = L_II^{-1}: right-looking block
// substitution in one CTA (the fallback of k_trsv_pair and k_trsv_cluster when a
// cluster launch is refused).  Thread t owns row t of the right-hand side.
// Step I of the forward pass: warp I forms z_I = W_II r_I; every row below
// block I then subtracts L[t, I] z_I.  The backward pass runs the same way
// with L^T.  The block column (forward) or block row (backward) that the next
// step reads is staged into shared memory with cp.async while the current
// step runs; rows at or beyond N are zero-filled.
constexpr int kBlkThreads = 1024;
constexpr int kBlkRowStride = 36;  // floats per staged column of a block row (16-byte rows, 4-way bank spread)

__host__ __device__ constexpr int blk_stage_floats(int N) {
  // forward: 32 columns x ldb rows; backward: up to 32 (T - 1) columns x 36
  return (32 * ((N + 3) & ~3)) > (kBlkRowStride * 32 * ((N + 31) / 32 - 1))
             ? (32 * ((N + 3) & ~3))
             : (kBlkRowStride * 32 * ((N + 31) / 32 - 1));
}

__device__ __forceinline__ void blk_stage_forward(const float* __restrict__ L, long long ld, int N, int I,
                                                  const float* __restrict__ Wd, float* dst, float* wdst) {
  const int r0 = 32 * (I + 1), ldb = (N + 3) & ~3;
  const int nch = (N - r0 + 3) / 4;  // 4-row chunks per column below the diagonal block
  for (int e = threadIdx.x; e < 32 * nch; e += blockDim.x) {
    const int q = e / nch, c = e - q * nch, row = r0 + 4 * c;
    cp_async16(dst + q * ldb + 4 * c, L + row + (long long)(32 * I + q) * ld, 4 * min(4, N - row));
  }
  for (int e = threadIdx.x; e < 256; e += blockDim.x) cp_async16(wdst + 4 * e, Wd + (long long)I * 1024 + 4 * e, 16);
}

__device__ __forceinline__ void blk_stage_backward(const float* __restrict__ L, long long ld, int N, int I,
                                                   const float* __restrict__ Wd, float* dst, float* wdst) {
  for (int e = threadIdx.x; e < 32 * I * 8; e += blockDim.x) {
    const int j = e >> 3, g = e & 7, row = 32 * I + 4 * g;
    const int valid = max(0, min(4, N - row));
    cp_async16(dst + j * kBlkRowStride + 4 * g, valid ? L + row + (long long)j * ld : L, 4 * valid);
  }
  for (int e = threadIdx.x; e < 256; e += blockDim.x) cp_async16(wdst + 4 * e, Wd + (long long)I * 1024 + 4 * e, 16);
}

__global__ void __launch_bounds__(kBlkThreads) k_trsv_blk(const float* __restrict__ L, long long ld, int N,
                                                          const double* __restrict__ rhs, double* __restrict__ acc,
                                                          int first, double alpha, const float* __restrict__ Wd) {
  pdl_entry();
  extern __shared__ __align__(16) float sm_blk[];
  const int T = (N + 31) / 32, ldb = (N + 3) & ~3, stage = blk_stage_floats(N);
  // staging buffer b: L part at sm_blk + b * stage, W_II at sm_blk + 2 * stage + b * 1024
  auto Lb = [&](int b) { return sm_blk + b * stage; };
  auto Wb = [&](int b) { return sm_blk + 2 * stage + b * 1024; };
  float* vec = sm_blk + 2 * stage + 2048;  // z_I (forward) or c_I (backward) of the current step
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float r = (t < N) ? (float)rhs[t] : 0.0f;
  // ---- forward: z = L^{-1} rhs
  blk_stage_forward(L, ld, N, 0, Wd, Lb(0), Wb(0));
  cp_async_commit();
  for (int I = 0; I < T; I++) {
    cp_async_wait0();
    __syncthreads();  // step I staged for everyone; step I-1 finished reading the other buffer
    if (I + 1 < T) blk_stage_forward(L, ld, N, I + 1, Wd, Lb((I + 1) & 1), Wb((I + 1) & 1));
    cp_async_commit();
    if (warp == I) {
      // z_l = sum_p W[l][p] r_p, the column index rotated by the lane (no bank conflicts)
      const float* W = Wb(I & 1);
      float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 32; q++) {
        const int p = (q + lane) & 31;
        a[q & 3] = fmaf(W[lane * 32 + p], __shfl_sync(0xffffffffu, r, p), a[q & 3]);
      }
      r = (a[0] + a[1]) + (a[2] + a[3]);  // this row is final: r holds z from here on
      vec[lane] = r;
    }
    __syncthreads();
    if (t >= 32 * (I + 1) && t < N) {
      const float* B = Lb(I & 1) + (t - 32 * (I + 1));
      float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 32; q++) a[q & 3] = fmaf(B[q * ldb], vec[q], a[q & 3]);
      r -= (a[0] + a[1]) + (a[2] + a[3]);
    }
  }
  // ---- backward: c = L^{-T} z
  cp_async_wait0();
  __syncthreads();
  blk_stage_backward(L, ld, N, T - 1, Wd, Lb(0), Wb(0));
  cp_async_commit();
  for (int I = T - 1, sidx = 0; I >= 0; I--, sidx ^= 1) {
    cp_async_wait0();
    __syncthreads();
    if (I > 0) blk_stage_backward(L, ld, N, I - 1, Wd, Lb(sidx ^ 1), Wb(sidx ^ 1));
    cp_async_commit();
    if (warp == I) {
      // c_l = sum_q W[q][l] r_q
      const float* W = Wb(sidx);
      float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 32; q++) a[q & 3] = fmaf(W[q * 32 + lane], __shfl_sync(0xffffffffu, r, q), a[q & 3]);
      r = (a[0] + a[1]) + (a[2] + a[3]);
      vec[lane] = r;
      if (t < N) acc[t] = first ? alpha * (double)r : acc[t] + alpha * (double)r;
    }
    __syncthreads();
    if (t < 32 * I) {
      const float4* B = reinterpret_cast<const float4*>(Lb(sidx) + t * kBlkRowStride);
      const float4* v4 = reinterpret_cast<const float4*>(vec);
      float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int g = 0; g < 8; g++) {
        const float4 l = B[g], v = v4[g];
        a[0] = fmaf(l.x, v.x, a[0]);
        a[1] = fmaf(l.y, v.y, a[1]);
        a[2] = fmaf(l.z, v.z, a[2]);
        a[3] = fmaf(l.w, v.w, a[3]);
      }
      r -= (a[0] + a[1]) + (a[2] + a[3]);
    }
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------------------
// Triangular solves with the inverse diagonal blocks W_II = L_II^{-1} for any N
// up to kMaxM, spread over an 8-CTA cluster.  Row block I (32 rows) belongs to
// warp I / 8 of CTA I mod 8; lane l of that warp owns row 32I + l.  Forward
// pass: the owner of block J subtracts L[J, I] z_I for every I < J as soon as
// z_I has arrived (its tile of L is loaded one step ahead into registers), then
// forms z_J = W_JJ r_J and stores it into every CTA's shared memory with st.async,
// completing on that CTA's mbarrier for block J.  The backward pass runs the
// same way with L^T.  Only 32 values per block cross the cluster; each CTA reads
// just its own rows of L (from L2).  Every wait is bounded (DevState::timeout).
constexpr int kTrsvCL = 8;        // CTAs per cluster
constexpr int kTrsvCLMaxT = 128;  // 4096 / 32 row blocks

__device__ __forceinline__ void st_async_f32(unsigned addr, float v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
               "r"(__float_as_uint(v)), "r"(bar)
               : "memory");
}

__global__ void __cluster_dims__(kTrsvCL, 1, 1) __launch_bounds__(512)
    k_trsv_cluster(const float* __restrict__ L, long long ld, int N, const double* __restrict__ rhs,
                   double* __restrict__ acc, int first, double alpha, const float* __restrict__ Wd, DevState* st) {
  pdl_entry();
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) float tcl[];
  const int T = (N + 31) / 32;
  float* zbuf = tcl;                 // T x 32: z_I (forward)
  float* cbuf = tcl + T * 32;        // T x 32: c_I (backward)
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(tcl + 2 * T * 32);  // 2T: forward, backward
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < 2 * T; k += blockDim.x) {
    mbar_init(smem_u32(bars + k), 1);
    mbar_expect_tx(smem_u32(bars + k), 128);  // the single arrival; the 128 bytes come from the owner
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  cluster.sync();
  const int J = rank + kTrsvCL * warp;  // this warp's row block
  bool ok = true;
  if (J < T) {
    const int row = 32 * J + lane;
    const bool live = row < N;
    float r = live ? (float)rhs[row] : 0.0f;
    const float* Wb = Wd + (long long)J * 1024;
    // ---- forward: z = L^{-1} rhs
    float a[32], an[32];
    auto load_row_tile = [&](float* dst, int I) {  // L[row, 32I .. 32I+31]
#pragma unroll
      for (int q = 0; q < 32; q++) dst[q] = live ? L[row + (long long)(32 * I + q) * ld] : 0.0f;
    };
    if (J > 0) load_row_tile(a, 0);
    for (int I = 0; I < J; I++) {
      if (I + 1 < J) load_row_tile(an, I + 1);
      if (ok && !mbar_wait(smem_u32(bars + I), 0u)) ok = false;
      const float4* z4 = reinterpret_cast<const float4*>(zbuf + I * 32);
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
      for (int g = 0; g < 8; g++) {
        const float4 z = z4[g];
        s0 = fmaf(a[4 * g], z.x, s0);
        s1 = fmaf(a[4 * g + 1], z.y, s1);
        s0 = fmaf(a[4 * g + 2], z.z, s0);
        s1 = fmaf(a[4 * g + 3], z.w, s1);
      }
      r -= s0 + s1;
#pragma unroll
      for (int q = 0; q < 32; q++) a[q] = an[q];
    }
    {
      // z_J = W_JJ r_J: lane l takes row l of W, the entries of r from the other lanes
      float w[32];
#pragma unroll
      for (int g = 0; g < 8; g++) {
        const float4 v = reinterpret_cast<const float4*>(Wb + lane * 32)[g];
        w[4 * g] = v.x; w[4 * g + 1] = v.y; w[4 * g + 2] = v.z; w[4 * g + 3] = v.w;
      }
      float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        z0 = fmaf(w[q], __shfl_sync(0xffffffffu, r, q), z0);
        z1 = fmaf(w[q + 1], __shfl_sync(0xffffffffu, r, q + 1), z1);
      }
      r = z0 + z1;
    }
    {
      const unsigned dst = smem_u32(zbuf + J * 32 + lane), bar = smem_u32(bars + J);
#pragma unroll 1
      for (int c = 0; c < kTrsvCL; c++) st_async_f32(cluster_addr(dst, c), r, cluster_addr(bar, c));
    }
    // ---- backward: c = L^{-T} z
    auto load_col_tile = [&](float* dst, int I) {  // L[32I .. 32I+31, row] (column `row` of L)
      const int nrow = min(32, N - 32 * I);
      if (live && nrow == 32) {
#pragma unroll
        for (int g = 0; g < 8; g++) {
          const float4 v = *reinterpret_cast<const float4*>(L + 32 * I + 4 * g + (long long)row * ld);
          dst[4 * g] = v.x; dst[4 * g + 1] = v.y; dst[4 * g + 2] = v.z; dst[4 * g + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; q++) dst[q] = (live && q < nrow) ? L[32 * I + q + (long long)row * ld] : 0.0f;
      }
    };
    if (J < T - 1) load_col_tile(a, T - 1);
    for (int I = T - 1; I > J; I--) {
      if (I - 1 > J) load_col_tile(an, I - 1);
      if (ok && !mbar_wait(smem_u32(bars + T + I), 0u)) ok = false;
      const float4* c4 = reinterpret_cast<const float4*>(cbuf + I * 32);
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
      for (int g = 0; g < 8; g++) {
        const float4 cv = c4[g];
        s0 = fmaf(a[4 * g], cv.x, s0);
        s1 = fmaf(a[4 * g + 1], cv.y, s1);
        s0 = fmaf(a[4 * g + 2], cv.z, s0);
        s1 = fmaf(a[4 * g + 3], cv.w, s1);
      }
      r -= s0 + s1;
#pragma unroll
      for (int q = 0; q < 32; q++) a[q] = an[q];
    }
    {
      // c_J = W_JJ^T r_J: lane l takes column l of W
      float w[32];
#pragma unroll
      for (int q = 0; q < 32; q++) w[q] = Wb[q * 32 + lane];
      float c0 = 0.0f, c1 = 0.0f;
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        c0 = fmaf(w[q], __shfl_sync(0xffffffffu, r, q), c0);
        c1 = fmaf(w[q + 1], __shfl_sync(0xffffffffu, r, q + 1), c1);
      }
      r = c0 + c1;
    }
    {  // the next link of the chain first; the FP64 accumulation (a global load) after it
      const unsigned dst = smem_u32(cbuf + J * 32 + lane), bar = smem_u32(bars + T + J);
#pragma unroll 1
      for (int c = 0; c < kTrsvCL; c++) st_async_f32(cluster_addr(dst, c), r, cluster_addr(bar, c));
    }
    if (live) acc[row] = first ? alpha * (double)r : acc[row] + alpha * (double)r;
  }
  // every value sent to this CTA has landed before it exits
  for (int k = tid; k < 2 * T; k += blockDim.x)
    if (ok && !mbar_wait(smem_u32(bars + k), 0u)) ok = false;
  if (!ok) st->timeout = 1;
  __syncthreads();
  cluster.sync();
}

// ---------------------------------------------------------------------------
// The same solves for N <= 32 kTrsvPairMaxT on a cluster of kTrsvQ CTAs with
// the row blocks split into contiguous parts of T0 = ceil(T / kTrsvQ) blocks, so
// that all but kTrsvQ - 1 links of each pass stay inside a CTA; every tile of L
// passes from L2 to one SM per pass, so the parts also spread that traffic (about
// 64 GB/s per SM), which bounds a link inside a CTA.  Warp w of CTA c owns
// block J = c T0 + w, lane l row (forward) or column (backward) 32J + l.  Each warp streams the T-1 tiles of L it needs (forward: L[J, I],
// I < J; backward: L[I, J], I > J, in the order they are consumed) through its
// own ring of kTrsvRing shared-memory tiles, one 2-D TMA copy per tile (128-byte
// swizzle: the 16-byte chunk index is XORed with the tile column mod 8, so both
// the row reads of the forward pass and the column reads of the backward pass
// are free of bank conflicts).  z_J and c_J reach the owner's warps through
// shared memory and a local mbarrier arrival, the other CTAs through st.async
// completing on their per-block mbarriers.  Every wait is bounded
// (DevState::timeout).  With zin the forward pass is already done (z = L^{-1} h from the
// factor): each warp starts from z_J and streams only the backward tiles.
constexpr int kTrsvPairMaxT = 32;  // 32 tile rows: N <= 1024 (the m x m systems of m = 1000 included)
static_assert(kTrsvPairMaxT <= 32, "the contraction test reduces one row block per lane");
constexpr int kTrsvQ = 4;     // CTAs per cluster
constexpr int kTrsvRing = 6;  // tiles in flight per warp
constexpr int kTrsvMaxT0 = (kTrsvPairMaxT + kTrsvQ - 1) / kTrsvQ;

__global__ void __cluster_dims__(kTrsvQ, 1, 1) __launch_bounds__(32 * kTrsvMaxT0)
    k_trsv_pair(const __grid_constant__ CUtensorMap tmL, int N, const double* __restrict__ rhs,
                double* __restrict__ acc, int first, double alpha, const float* __restrict__ Wd, DevState* st,
                double* __restrict__ rpart, double tau2, const float* __restrict__ zin) {
  pdl_entry();
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(1024) float tpr[];
  const int T = (N + 31) / 32, T0 = (T + kTrsvQ - 1) / kTrsvQ;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  // 1 KB alignment for the swizzled tiles
  float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tpr) + 1023) & ~(uintptr_t)1023);
  float* ring = base + warp * kTrsvRing * 1024;    // this warp's tile ring
  float* zbuf = base + nwarp * kTrsvRing * 1024;   // T x 32: z_I
  float* cbuf = zbuf + T * 32;                     // T x 32: c_I
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(cbuf + T * 32);  // 2T: forward, backward
  unsigned long long* rbars = bars + 2 * T + warp * kTrsvRing;                      // this warp's ring slots
  float* rscr = reinterpret_cast<float*>(bars + 2 * T + nwarp * kTrsvRing);            // nwarp x 32 scratch
  // block J belongs to CTA J / T0; its values reach the owner's own barrier by
  // one local arrival after plain stores, the other CTAs' by 128 bytes of st.async
  for (int k = tid; k < 2 * T; k += blockDim.x) {
    mbar_init(smem_u32(bars + k), 1);
    if ((k % T) / T0 != rank) mbar_expect_tx(smem_u32(bars + k), 128);
  }
  if (lane < kTrsvRing) mbar_init(smem_u32(rbars + lane), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  cluster.sync();
  const int J = rank * T0 + warp;  // this warp's row block
  bool ok = true;
  if (J < T) {
    const int row = 32 * J + lane;
    const bool live = row < N;
    float r = live ? (zin ? zin[row] : (float)rhs[row]) : 0.0f;
    const float* Wb = Wd + (long long)J * 1024;
    // tile t of this warp: forward L[J, t] for t < J, then backward L[I, J], I = T-1 .. J+1
    // (with zin only the backward ones: t from t0 = J); ring slots count from t0
    const int t0 = zin ? J : 0;
    auto issue = [&](int t) {
      if (lane == 0) {
        const int slot = (t - t0) % kTrsvRing;
        const unsigned bar = smem_u32(rbars + slot);
        mbar_expect_tx(bar, 4096);
        if (t < J)
          tma_load_2d(smem_u32(ring + slot * 1024), &tmL, 32 * J, 32 * t, bar);
        else
          tma_load_2d(smem_u32(ring + slot * 1024), &tmL, 32 * (T - 1 - (t - J)), 32 * J, bar);
      }
    };
    const int ntile = T - 1;
    for (int t = t0; t < t0 + kTrsvRing && t < ntile; t++) issue(t);
    // W_JJ row l (forward) in registers
    float w[32];
#pragma unroll
    for (int g = 0; g < 8; g++) {
      const float4 v = reinterpret_cast<const float4*>(Wb + lane * 32)[g];
      w[4 * g] = v.x; w[4 * g + 1] = v.y; w[4 * g + 2] = v.z; w[4 * g + 3] = v.w;
    }
    if (zin) {
      // z_J is given: publish it (the forward barriers complete as in a forward pass) and
      // take column l of W for the backward pass
#pragma unroll
      for (int q = 0; q < 32; q++) w[q] = Wb[q * 32 + lane];
    }
    auto publish = [&](float* buf, unsigned long long* bar) {
      const unsigned dst = smem_u32(buf + J * 32 + lane), b = smem_u32(bar);
      buf[J * 32 + lane] = r;  // this CTA first: its consumers are the next link
      __syncwarp();
      if (lane == 0) mbar_arrive(b);  // release: the warp's stores before the arrival
#pragma unroll
      for (int c = 1; c < kTrsvQ; c++) {
        const int d = (rank + c) % kTrsvQ;  // the next CTA first: the chain continues there
        st_async_f32(cluster_addr(dst, d), r, cluster_addr(b, d));
      }
    };
    // r through shared memory (one 128-bit broadcast load per four entries)
    float* rb = rscr + warp * 32;
    auto wr_product = [&]() {  // sum_q w[q] r_q, even q then odd q
      rb[lane] = r;
      __syncwarp();
      const float4* r4 = reinterpret_cast<const float4*>(rb);
      float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
      for (int g = 0; g < 8; g++) {
        const float4 v = r4[g];
        z0 = fmaf(w[4 * g], v.x, z0);
        z1 = fmaf(w[4 * g + 1], v.y, z1);
        z0 = fmaf(w[4 * g + 2], v.z, z0);
        z1 = fmaf(w[4 * g + 3], v.w, z1);
      }
      __syncwarp();  // every lane has read rb before it is written again
      return z0 + z1;
    };
    auto form_z = [&]() {  // z_J = W_JJ r_J: lane l takes row l of W
      r = wr_product();
      publish(zbuf, bars + J);
#pragma unroll
      for (int q = 0; q < 32; q++) w[q] = Wb[q * 32 + lane];  // column l of W for the backward pass
    };
    if (zin)
      publish(zbuf, bars + J);
    else if (J == 0)
      form_z();
    const int sw = lane >> 2, se = lane & 3;  // forward: chunk and element of row `lane` in a tile column
    for (int t = t0; t < ntile; t++) {
      const int slot = (t - t0) % kTrsvRing;
      // always waited (bounded), so that no copy is in flight when the CTA leaves
      if (!mbar_wait(smem_u32(rbars + slot), (unsigned)(((t - t0) / kTrsvRing) & 1))) ok = false;
      const float* tile = ring + slot * 1024;
      float s0 = 0.0f, s1 = 0.0f;
      if (t < J) {
        if (ok && !mbar_wait(smem_u32(bars + t), 0u)) ok = false;
        const float4* z4 = reinterpret_cast<const float4*>(zbuf + t * 32);
#pragma unroll
        for (int g = 0; g < 8; g++) {
          const float4 z = z4[g];
          // element (row lane, column q) of the tile: column q is the q-th 128-byte row
          s0 = fmaf(tile[(4 * g) * 32 + ((sw ^ ((4 * g) & 7)) << 2) + se], z.x, s0);
          s1 = fmaf(tile[(4 * g + 1) * 32 + ((sw ^ ((4 * g + 1) & 7)) << 2) + se], z.y, s1);
          s0 = fmaf(tile[(4 * g + 2) * 32 + ((sw ^ ((4 * g + 2) & 7)) << 2) + se], z.z, s0);
          s1 = fmaf(tile[(4 * g + 3) * 32 + ((sw ^ ((4 * g + 3) & 7)) << 2) + se], z.w, s1);
        }
        r -= s0 + s1;
        if (t == J - 1) form_z();
      } else {
        const int I = T - 1 - (t - J);
        if (ok && !mbar_wait(smem_u32(bars + T + I), 0u)) ok = false;
        const float4* c4 = reinterpret_cast<const float4*>(cbuf + I * 32);
#pragma unroll
        for (int g = 0; g < 8; g++) {
          // column `lane` of the tile is its lane-th 128-byte row; rows 4g .. 4g+3 are chunk g
          const float4 v = *reinterpret_cast<const float4*>(tile + lane * 32 + ((g ^ (lane & 7)) << 2));
          const float4 cv = c4[g];
          s0 = fmaf(v.x, cv.x, s0);
          s1 = fmaf(v.y, cv.y, s1);
          s0 = fmaf(v.z, cv.z, s0);
          s1 = fmaf(v.w, cv.w, s1);
        }
        r -= s0 + s1;
      }
      __syncwarp();  // every lane has read the slot (the reads fed r) before it is refilled
      if (t + kTrsvRing < ntile) issue(t + kTrsvRing);
    }
    r = wr_product();  // c_J = W_JJ^T r_J: lane l takes column l of W
    // the next link of the chain first; the FP64 accumulation (a global load) after it
    publish(cbuf, bars + T + J);
    if (rpart) {
      // refinement step: acc += c, and this row block's ||c||^2, ||acc + c||^2 (fixed order)
      double ci = 0.0, ai = 0.0;
      if (live) {
        ci = (double)r;
        ai = acc[row] + ci;
        acc[row] = ai;
      }
      const double q0 = warp_sum(ci * ci), q1 = warp_sum(ai * ai);
      if (lane == 0) {
        rpart[2 * J] = q0;
        rpart[2 * J + 1] = q1;
      }
    } else if (live) {
      acc[row] = first ? alpha * (double)r : acc[row] + alpha * (double)r;
    }
  }
  // every value sent to this CTA has landed before it exits (the ring copies of a
  // warp were all waited for: each issued tile is consumed)
  for (int k = tid; k < 2 * T; k += blockDim.x)
    if (ok && !mbar_wait(smem_u32(bars + k), 0u)) ok = false;
  if (!ok) st->timeout = 1;
  if (rpart && last_block(&st->counters[kCtrRefine])) {
    // the contraction test of the refinement: the row blocks' partial norms, one per
    // lane of warp 0 (T <= 32: all loads in flight at once), summed in a fixed order
    if (tid < 32) {
      const double c2 = warp_sum(tid < T ? ld_cg(rpart + 2 * tid) : 0.0);
      const double a2 = warp_sum(tid < T ? ld_cg(rpart + 2 * tid + 1) : 0.0);
      if (tid == 0) {
        st->refine_ratio = a2 > 0.0 ? sqrt(c2 / a2) : (c2 > 0.0 ? INFINITY : 0.0);
        if (!(c2 <= tau2 * a2)) st->newton_bad = 1;
      }
    }
    reset_counter(&st->counters[kCtrRefine]);
  }
  __syncthreads();
  cluster.sync();
}

// ---------------------------------------------------------------------------
// Newton systems above kClusterN: right-looking Cholesky over super-blocks of at
// most kClusterN rows.  Each diagonal super-block is factored by k_chol_cluster
// (which also leaves its inverse 32x32 diagonal blocks), the rows below it are
// solved against it by k_trsm_blocks, and the trailing matrix is updated by
// k_syrk_sub.  The 32x32 inverse diagonal blocks then cover the whole factor,
// so the solves run in k_trsv_cluster.

// X L^T = A for the R x nk block A = G[r0 .., k0 ..] (in place), L = the factored
// super-block G[k0 .., k0 ..] (nk a multiple of 32) with inverse diagonal blocks Wd:
// blocked forward substitution, X_J = (A_J - sum_{I<J} X_I L_JI^T) W_JJ^T.  One CTA per
// RB rows of A, which stay in shared memory (k-major: the RB rows of one column are
// contiguous).  The block rows of L stream through a ring of kTrsmStages slots filled by
// 16-byte cp.async, kTrsmChunk columns of one block row per slot, W_JJ in the slot after
// the chunks of block row J; the copies run kTrsmStages - 1 slots ahead of the arithmetic.
// The 256 threads form 64 / RB k-groups; thread (tr, tc) of a group holds the 2 x 4
// register tile of rows 2tr, 2tr+1 and columns 4tc..4tc+3 of the block column and takes
// every (64 / RB)-th column of each chunk; at the end of block row J the groups' partial
// sums are added in a fixed order.
constexpr int kTrsmThreads = 256;
constexpr int kTrsmRows = 8;    // RB
constexpr int kTrsmChunk = 128;
constexpr int kTrsmStages = 8;
constexpr int kTrsmSlot = kTrsmChunk * 32;  // floats per slot (a W tile takes 32 x 33)
__host__ __device__ constexpr size_t trsm_smem(int nk, int RB = kTrsmRows) {
  return ((size_t)nk * RB + (size_t)kTrsmStages * kTrsmSlot + (size_t)(64 / RB) * 32 * (RB + 1) + (size_t)RB * 33) *
         sizeof(float);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int RB>
__global__ void __launch_bounds__(kTrsmThreads) k_trsm_blocks(float* __restrict__ G, long long ld, int k0, int nk,
                                                              int r0, int R, const float* __restrict__ Wd) {
  pdl_entry();
  constexpr int KG = 64 / RB;  // k-groups of 4 RB threads
  extern __shared__ __align__(16) float tsm[];
  float* Xs = tsm;                                // nk x RB, k-major
  float* ring = Xs + nk * RB;                     // kTrsmStages slots
  float* red = ring + kTrsmStages * kTrsmSlot;    // KG x 32 x (RB + 1): partial sums, column-major
  float* Ys = red + KG * 32 * (RB + 1);           // RB x 33
  const int tid = threadIdx.x;
  const int rb = RB * blockIdx.x;                 // first row of this CTA within the R rows
  const int Tk = nk / 32;
  // ---- the CTA's rows of A (rows past R read as zeros)
  for (int e = tid; e < (RB / 4) * nk; e += kTrsmThreads) {
    const int q = e % (RB / 4), k = e / (RB / 4);
    const int row = rb + 4 * q;
    const int valid = R - row >= 4 ? 4 : (R - row > 0 ? R - row : 0);
    cp_async16(Xs + k * RB + 4 * q, valid ? G + (r0 + row) + (long long)(k0 + k) * ld : G, 4 * valid);
  }
  // ---- the ring: item (J, c), c < nch(J): columns [kTrsmChunk c, ..) of block row J of L;
  //      c == nch(J): W_JJ (row stride 33)
  auto nch = [](int J) { return (32 * J + kTrsmChunk - 1) / kTrsmChunk; };
  auto issue = [&](int J, int c, int slot) {
    float* dst = ring + slot * kTrsmSlot;
    if (c == nch(J)) {
      for (int e = tid; e < 1024; e += kTrsmThreads) cp_async4(dst + (e >> 5) * 33 + (e & 31), Wd + (long long)J * 1024 + e);
    } else {
      const int kb = c * kTrsmChunk, kn = min(kTrsmChunk, 32 * J - kb);
      for (int e = tid; e < 8 * kn; e += kTrsmThreads) {
        const int q = e & 7, kk = e >> 3;
        cp_async16(dst + kk * 32 + 4 * q, G + (k0 + 32 * J + 4 * q) + (long long)(k0 + kb + kk) * ld, 16);
      }
    }
  };
  int pJ = 0, pc = 0, pslot = 0;  // next item to issue
  auto advance = [&](int& J, int& c) {
    if (c < nch(J)) {
      c++;
    } else {
      J++;
      c = 0;
    }
  };
  for (int s = 0; s < kTrsmStages - 1; s++) {
    if (pJ < Tk) {
      issue(pJ, pc, pslot);
      advance(pJ, pc);
      pslot = pslot + 1 == kTrsmStages ? 0 : pslot + 1;
    }
    cp_async_commit();
  }
  const int kg = tid / (4 * RB), t = tid % (4 * RB), tr = t >> 3, tc = t & 7;
  float acc[2][4] = {};
  int cslot = 0;
  for (int J = 0, c = 0; J < Tk; advance(J, c), cslot = cslot + 1 == kTrsmStages ? 0 : cslot + 1) {
    cp_async_wait_n<kTrsmStages - 2>();  // item (J, c) has landed (this thread's copies)
    __syncthreads();                     // everyone's copies; everyone is done with the previous slot
    if (pJ < Tk) {
      issue(pJ, pc, pslot);
      advance(pJ, pc);
      pslot = pslot + 1 == kTrsmStages ? 0 : pslot + 1;
    }
    cp_async_commit();
    const float* sl = ring + cslot * kTrsmSlot;
    if (c < nch(J)) {
      const int kb = c * kTrsmChunk, kn = min(kTrsmChunk, 32 * J - kb);
#pragma unroll 4
      for (int kk = kg; kk < kn; kk += KG) {
        const float2 x = *reinterpret_cast<const float2*>(Xs + (kb + kk) * RB + 2 * tr);
        const float4 l = *reinterpret_cast<const float4*>(sl + kk * 32 + 4 * tc);
        acc[0][0] = fmaf(x.x, l.x, acc[0][0]);
        acc[0][1] = fmaf(x.x, l.y, acc[0][1]);
        acc[0][2] = fmaf(x.x, l.z, acc[0][2]);
        acc[0][3] = fmaf(x.x, l.w, acc[0][3]);
        acc[1][0] = fmaf(x.y, l.x, acc[1][0]);
        acc[1][1] = fmaf(x.y, l.y, acc[1][1]);
        acc[1][2] = fmaf(x.y, l.z, acc[1][2]);
        acc[1][3] = fmaf(x.y, l.w, acc[1][3]);
      }
      continue;
    }
    // ---- end of block row J: Y = A_J - (sum over the k-groups, in order), X_J = Y W_JJ^T
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) {
        red[(kg * 32 + 4 * tc + v) * (RB + 1) + 2 * tr + u] = acc[u][v];
        acc[u][v] = 0.0f;
      }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < RB / 8; p++) {
      const int o = tid + kTrsmThreads * p, r = o % RB, cc = o / RB;
      float s = 0.0f;
#pragma unroll
      for (int g = 0; g < KG; g++) s += red[(g * 32 + cc) * (RB + 1) + r];
      Ys[r * 33 + cc] = Xs[(32 * J + cc) * RB + r] - s;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < RB / 8; p++) {
      const int o = tid + kTrsmThreads * p, r = o % RB, cc = o / RB;
      float x = 0.0f;
#pragma unroll 8
      for (int q = 0; q < 32; q++) x = fmaf(Ys[r * 33 + q], sl[cc * 33 + q], x);
      Xs[(32 * J + cc) * RB + r] = x;
    }
  }
  cp_async_wait_n<0>();
  __syncthreads();
  for (int e = tid; e < RB * nk; e += kTrsmThreads) {
    const int r = e % RB, k = e / RB;
    if (rb + r < R) G[(r0 + rb + r) + (long long)(k0 + k) * ld] = Xs[k * RB + r];
  }
}

// C -= X X^T on the lower triangle of the R x R block C = G[r0 .., r0 ..], with
// X = G[r0 .., k0 .. k0 + nk): one CTA per 32 x 32 lower tile.  Both row blocks of X
// are staged whole (k-major: the 32 rows of one column are one 128-byte line; 16-byte
// cp.async, all in flight at once, rows past R as zeros); four k-groups of 64 threads
// take every fourth k with a 4 x 4 register tile each, and the groups' partial sums are
// added in a fixed order.
constexpr int kSubThreads = 256;
__host__ __device__ constexpr size_t syrk_sub_smem(int nk) {
  return ((size_t)2 * 32 * nk + (size_t)3 * 32 * 33) * sizeof(float);
}

__global__ void __launch_bounds__(kSubThreads) k_syrk_sub(float* __restrict__ G, long long ld, int r0, int R, int k0,
                                                          int nk) {
  pdl_entry();
  extern __shared__ __align__(16) float ssm[];
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = 32 * ti, j0 = 32 * tj;
  float* As = ssm;
  float* Bs = ti == tj ? As : As + 32 * nk;
  float* red = ssm + 64 * nk;  // 3 x 32 x 33
  const int tid = threadIdx.x;
  auto stage = [&](float* dst, int b0) {
    for (int e = tid; e < 8 * nk; e += kSubThreads) {
      const int q = e & 7, k = e >> 3, row = b0 + 4 * q;
      const int valid = R - row >= 4 ? 4 : (R - row > 0 ? R - row : 0);
      cp_async16(dst + k * 32 + 4 * q, valid ? G + (r0 + row) + (long long)(k0 + k) * ld : G, 4 * valid);
    }
  };
  stage(As, i0);
  if (ti != tj) stage(Bs, j0);
  cp_async_commit();
  cp_async_wait0();
  __syncthreads();
  const int kg = tid >> 6, t = tid & 63, tr = t >> 3, tc = t & 7;
  float acc[4][4] = {};
#pragma unroll 4
  for (int k = kg; k < nk; k += 4) {
    const float4 a4 = reinterpret_cast<const float4*>(As + k * 32)[tr];
    const float4 b4 = reinterpret_cast<const float4*>(Bs + k * 32)[tc];
    const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
  }
  if (kg > 0)
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) red[((kg - 1) * 32 + 4 * tr + u) * 33 + 4 * tc + v] = acc[u][v];
  __syncthreads();
  if (kg == 0)
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) {
        const int gi = i0 + 4 * tr + u, gj = j0 + 4 * tc + v;
        float s = acc[u][v];
#pragma unroll
        for (int g = 0; g < 3; g++) s += red[(g * 32 + 4 * tr + u) * 33 + 4 * tc + v];
        if (gi < R && gj < R && gi >= gj) G[(r0 + gi) + (long long)(r0 + gj) * ld] -= s;
      }
}

static_assert(trsm_smem(kClusterN) <= kClusterSmemLimit, "k_trsm_blocks: shared memory at the largest super-block");
static_assert(syrk_sub_smem(kClusterN) <= kClusterSmemLimit, "k_syrk_sub: shared memory at the largest super-block");

// Shared-memory limits of the super-block kernels (k_chol_cluster<8>, k_trsm_blocks,
// k_syrk_sub), set once per device.
static void super_block_attrs() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && done[dev]) return;
  cudaFuncSetAttribute(k_chol_cluster<kClusterCTAs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)cluster_smem_max());
  cudaFuncSetAttribute(k_trsm_blocks<kTrsmRows>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)trsm_smem(kClusterN));
  cudaFuncSetAttribute(k_syrk_sub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)syrk_sub_smem(kClusterN));
  if (dev >= 0 && dev < 64) done[dev] = true;
}

// X L^T = A on the R x nk block at (r0, k0) (nk a multiple of 32, at most kClusterN).
static void launch_trsm_blocks(float* G, long long ld, int k0, int nk, int r0, int R, const float* Wd,
                               cudaStream_t s) {
  launch_k(k_trsm_blocks<kTrsmRows>, dim3((R + kTrsmRows - 1) / kTrsmRows), dim3(kTrsmThreads), trsm_smem(nk), s, G,
           ld, k0, nk, r0, R, Wd);
}

// ---------------------------------------------------------------------------
// Larger Newton systems: blocked right-looking Cholesky in ONE cooperative
// launch.  Phases (diagonal block, panel, trailing update) are separated by a
// grid barrier with a bounded wait; all CTAs are co-resident (cooperative
// launch), so the barrier cannot deadlock, and a timeout raises
// DevState::timeout instead of hanging.
constexpr int kCoopThreads = 256;

__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, DevState* st) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      *bar = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > 4000000000LL) {
          ok = 0;
          st->timeout = 1;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__global__ void __launch_bounds__(kCoopThreads) k_chol_coop(float* __restrict__ G, long long ld, int N,
                                                            DevState* st, unsigned* bar) {
  pdl_entry();
  __shared__ float Ld[kT][kT + 1];
  __shared__ float As[kT][kT + 1];
  __shared__ float Bs[kT][kT + 1];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const unsigned nblk = gridDim.x;
  for (int kb = 0; kb < N; kb += kT) {
    const int nb = min(kT, N - kb);
    // (1) diagonal block, CTA 0
    if (blockIdx.x == 0) {
      for (int e = tid; e < kT * kT; e += blockDim.x) {
        const int i = e % kT, j = e / kT;
        Ld[i][j] = (i < nb && j < nb && j <= i) ? G[(kb + i) + (long long)(kb + j) * ld] : 0.0f;
      }
      __syncthreads();
      for (int k = 0; k < nb; k++) {
        if (tid == 0) {
          float piv = Ld[k][k];
          if (!(piv > 0.0f)) {
            st->chol_fail = 1;
            piv = 1.0f;
          }
          Ld[k][k] = sqrtf(piv);
        }
        __syncthreads();
        if (tid > k && tid < nb) Ld[tid][k] /= Ld[k][k];
        __syncthreads();
        for (int e = tid; e < kT * kT; e += blockDim.x) {
          const int i = e % kT, j = e / kT;
          if (j > k && i >= j && i < nb) Ld[i][j] = fmaf(-Ld[i][k], Ld[j][k], Ld[i][j]);
        }
        __syncthreads();
      }
      for (int e = tid; e < kT * kT; e += blockDim.x) {
        const int i = e % kT, j = e / kT;
        if (i < nb && j < nb && j <= i) G[(kb + i) + (long long)(kb + j) * ld] = Ld[i][j];
      }
    }
    if (!grid_barrier(bar, nblk, st)) return;
    const int k1 = kb + nb;
    const int rem = N - k1;
    if (rem <= 0) break;
    // (2) panel L21 = A21 L11^{-T}, one row per thread across the grid
    for (int e = tid; e < kT * kT; e += blockDim.x) {
      const int i = e % kT, j = e / kT;
      Ld[i][j] = (i < nb && j < nb && j <= i) ? G[(kb + i) + (long long)(kb + j) * ld] : 0.0f;
    }
    __syncthreads();
    for (int row = k1 + blockIdx.x * blockDim.x + tid; row < N; row += gridDim.x * blockDim.x) {
      float xv[kT];
#pragma unroll
      for (int j = 0; j < kT; j++) {
        if (j < nb) {
          float sacc = G[row + (long long)(kb + j) * ld];
#pragma unroll
          for (int k = 0; k < kT; k++)
            if (k < j) sacc = fmaf(-xv[k], Ld[j][k], sacc);
          xv[j] = sacc / Ld[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < kT; j++)
        if (j < nb) G[row + (long long)(kb + j) * ld] = xv[j];
    }
    if (!grid_barrier(bar, nblk, st)) return;
    // (3) trailing update on lower tiles of [k1, N)
    const int T = (rem + kT - 1) / kT;
    const int ntiles = T * (T + 1) / 2;
    for (int id = blockIdx.x; id < ntiles; id += gridDim.x) {
      int ti, tj;
      tri_tile(id, ti, tj);
      const int i0 = k1 + ti * kT, j0 = k1 + tj * kT;
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = ty + 8 * e;
        As[k][tx] = (k < nb && i0 + tx < N) ? G[(i0 + tx) + (long long)(kb + k) * ld] : 0.0f;
        Bs[k][tx] = (k < nb && j0 + tx < N) ? G[(j0 + tx) + (long long)(kb + k) * ld] : 0.0f;
      }
      __syncthreads();
      float a4[4] = {0, 0, 0, 0};
#pragma unroll 8
      for (int k = 0; k < kT; k++) {
        const float bv = Bs[k][tx];
#pragma unroll
        for (int e = 0; e < 4; e++) a4[e] = fmaf(As[k][ty + 8 * e], bv, a4[e]);
      }
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int i = i0 + ty + 8 * e, j = j0 + tx;
        if (i < N && j < N && i >= j) {
          float* p = G + i + (long long)j * ld;
          *p = *p - a4[e];
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, nblk, st)) return;
  }
}

// ---------------------------------------------------------------- launchers
void launch_syrk_tn(const float* P32, long long ldp32, int m, long long r, double diag, float* G, long long ldg,
                    cudaStream_t s) {
  int T = (int)((r + kT - 1) / kT);
  int blocks = T * (T + 1) / 2;
  if (blocks > 0) count_launch();
  if (blocks > 0) launch_k(k_syrk_tn, dim3(blocks), dim3(256), (size_t)(0), s, P32, ldp32, m, (int)r, (float)diag, G, ldg);
}

void launch_syrk_nt(const float* P32, long long ldp32, int m, long long r, double kappa, float* G, long long ldg,
                    cudaStream_t s) {
  int T = (m + kT - 1) / kT;
  int blocks = T * (T + 1) / 2;
  if (blocks > 0) count_launch();
  if (blocks > 0) launch_k(k_syrk_nt, dim3(blocks), dim3(256), (size_t)(0), s, P32, ldp32, m, r, (float)kappa, G, ldg);
}

static void small_smem_attr() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && done[dev]) return;
  cudaFuncSetAttribute(k_trsv_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem);
  if (dev >= 0 && dev < 64) done[dev] = true;
}

// ---------------------------------------------------------------------------
// Trace of the inverse of an SPD matrix for the degrees of freedom of the tuning
// criteria (Sec. 3.3): with G = L L^T, tr(G^{-1}) = ||L^{-1}||_F^2.  The factor
// and the identity are laid out in one buffer S (row stride ldS >= 2 Np, Np =
// N rounded up to 32): S[0:Np, 0:Np] = L padded with the identity, S[Np:2Np,
// 0:Np] = I; k_trsm_blocks then turns the bottom block into I L^{-T}, and
// ||L^{-T}||_F^2 = ||L^{-1}||_F^2 + (Np - N) (the padded part contributes ones).

// Identity padding of the factor (rows / columns N..Np-1) and the identity below it.
__global__ void k_inv_trace_setup(float* __restrict__ S, long long ldS, int N, int Np) {
  pdl_entry();
  const long long total = (long long)Np * Np;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % Np), j = (int)(e / Np);  // row, column
    const float id = (i == j) ? 1.0f : 0.0f;
    S[Np + i + (long long)j * ldS] = id;             // bottom block: I
    if (i >= N || j >= N) S[i + (long long)j * ldS] = id;
  }
}

// Fixed-order sum of squares of the Np x Np block B (column-major, ld), one
// partial per column block of 32; the last block adds the partials in order.
__global__ void __launch_bounds__(256) k_frob2(const float* __restrict__ B, long long ld, int Np,
                                               double* __restrict__ partial, double* __restrict__ out,
                                               DevState* st) {
  pdl_entry();
  __shared__ double red[32];
  double a = 0.0;
  for (int e = threadIdx.x; e < 32 * Np; e += blockDim.x) {
    const int i = e % Np, j = 32 * blockIdx.x + e / Np;
    const double v = (double)B[i + (long long)j * ld];
    a = fma(v, v, a);
  }
  a = block_sum(a, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  if (!last_block(&st->counters[kCtrMisc])) return;
  if (threadIdx.x == 0) *out = ordered_sum_cg(partial, 1, (int)gridDim.x);
  reset_counter(&st->counters[kCtrMisc]);
}

bool inv_trace(float* S, long long ldS, int N, DevState* st, float* Wdiag, double* partial, double* out,
               cudaStream_t s) {
  const int Np = (N + 31) / 32 * 32;
  if (N <= 0 || Np > kClusterN) return false;
  super_block_attrs();
  count_launch(4);
  launch_k(k_chol_cluster<kClusterCTAs>, dim3(kClusterCTAs), dim3(kCholThreads), (size_t)(cluster_smem((N + 31) / 32)), s, S, ldS, N, st, Wdiag,
           (const double*)nullptr, (float*)nullptr);
  launch_k(k_inv_trace_setup, dim3(64), dim3(256), (size_t)(0), s, S, ldS, N, Np);
  launch_trsm_blocks(S, ldS, 0, Np, Np, Np, Wdiag, s);
  launch_k(k_frob2, dim3(Np / 32), dim3(256), (size_t)(0), s, S + Np, ldS, Np, partial, out, st);
  return cudaGetLastError() == cudaSuccess;
}

// ||L^{-1}||_F^2 for a factor of any size up to kMaxM (the super-block factor of
// chol_factor, with the inverses W_II of all its 32 x 32 diagonal blocks): column block
// J of Y = L^{-1} by blocked forward substitution,
//   Y_IJ = W_II (delta_IJ I - sum_{K=J}^{I-1} L_IK Y_KJ),   I = J .. T-1,
// one CTA per column block (the blocks are independent).  Y lives in global scratch
// (column-major, ldy >= 32 T; the CTA reads back only what it wrote before a block
// barrier); the K sums run in chunks of 64 staged in shared memory, the next chunk
// fetched into registers while the current one is used.  Entries of L outside N x N
// are read as zero; the padded part of the last diagonal block is the identity (as
// the factor kernels pad it), so Y is exact there and only entries inside N x N are
// summed.  Per CTA the FP64 sum of squares goes to partial[J]; the last CTA adds the
// partials in order into *out.
constexpr int kInvKC = 64;
constexpr int kInvKP = kInvKC + 1;
__global__ void __launch_bounds__(256) k_inv_frob(const float* __restrict__ L, long long ld, int N,
                                                  const float* __restrict__ Wd, float* __restrict__ Yall,
                                                  long long ldy, double* __restrict__ partial,
                                                  double* __restrict__ out, DevState* st) {
  pdl_entry();
  __shared__ __align__(16) float Ls[2][kInvKC * 32];  // L[32 I + row, kc + k] at [32 k + row]
  __shared__ float Ys[2][32 * kInvKP];                // Y[kc + k, 32 J + col] at [col * kInvKP + k]
  __shared__ float Ws[32 * 33];                        // W_II transposed: W[i][q] at [q * 33 + i]
  __shared__ float Bs[32 * 33];                        // delta - sum, row-major
  __shared__ double red[32];
  const int J = blockIdx.x, T = (N + 31) / 32;
  const int tid = threadIdx.x, rg = tid & 7, c = tid >> 3;  // rows 4 rg .. 4 rg + 3, column c
  float* Y = Yall + (long long)J * 32 * ldy;
  double ss = 0.0;
  float pl[8], py[8];
  auto fetch = [&](int I, int kc, int nk) {
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int e = tid + 256 * t, row = e & 31, k = e >> 5;
      const int gi = 32 * I + row, gk = kc + k;
      pl[t] = (k < nk && gi < N && gk < N) ? L[gi + (long long)gk * ld] : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int e = tid + 256 * t, k = e % kInvKC, col = e / kInvKC;
      py[t] = k < nk ? Y[(kc + k) + (long long)col * ldy] : 0.0f;
    }
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int e = tid + 256 * t;
      Ls[buf][32 * (e >> 5) + (e & 31)] = pl[t];
      Ys[buf][(e / kInvKC) * kInvKP + e % kInvKC] = py[t];
    }
  };
  for (int I = J; I < T; I++) {
    for (int e = tid; e < 1024; e += 256) Ws[(e & 31) * 33 + (e >> 5)] = Wd[(long long)I * 1024 + e];
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int kbeg = 32 * J, kend = 32 * I;
    const int nch = (kend - kbeg + kInvKC - 1) / kInvKC;
    if (nch > 0) {
      fetch(I, kbeg, min(kInvKC, kend - kbeg));
      put(0);
    }
    __syncthreads();
    for (int ch = 0; ch < nch; ch++) {
      const int buf = ch & 1, kc = kbeg + ch * kInvKC, nk = min(kInvKC, kend - kc);
      if (ch + 1 < nch) fetch(I, kc + kInvKC, min(kInvKC, kend - kc - kInvKC));
      const float* Lb = Ls[buf];
      const float* Yb = Ys[buf] + c * kInvKP;
#pragma unroll 4
      for (int k = 0; k < nk; k++) {
        const float y = Yb[k];
        const float4 l = reinterpret_cast<const float4*>(Lb + 32 * k)[rg];
        acc[0] = fmaf(l.x, y, acc[0]);
        acc[1] = fmaf(l.y, y, acc[1]);
        acc[2] = fmaf(l.z, y, acc[2]);
        acc[3] = fmaf(l.w, y, acc[3]);
      }
      if (ch + 1 < nch) put(buf ^ 1);  // read in the previous chunk, before the last barrier
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int row = 4 * rg + e;
      Bs[row * 33 + c] = ((I == J && row == c) ? 1.0f : 0.0f) - acc[e];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int row = 4 * rg + e;
      float a = 0.0f;
#pragma unroll 8
      for (int q = 0; q < 32; q++) a = fmaf(Ws[q * 33 + row], Bs[q * 33 + c], a);
      const int gi = 32 * I + row;
      Y[gi + (long long)c * ldy] = a;
      if (gi < N && 32 * J + c < N) ss = fma((double)a, (double)a, ss);
    }
    __syncthreads();  // block I of Y is written before a later block stages it; Ws, Bs free
  }
  ss = block_sum(ss, red);
  if (tid == 0) partial[J] = ss;
  if (!last_block(&st->counters[kCtrMisc])) return;
  if (tid == 0) *out = ordered_sum_cg(partial, 1, (int)gridDim.x);
  reset_counter(&st->counters[kCtrMisc]);
}

bool inv_trace_large(float* G, long long ldg, int N, DevState* st, float* Wdiag, float* Y, long long ldy,
                     double* partial, double* out, cudaStream_t s) {
  const int T = (N + 31) / 32;
  if (N <= 0 || N > kMaxM || ldy < 32LL * T || !Wdiag) return false;
  if (!chol_factor(G, ldg, N, st, Wdiag, s)) return false;  // no inverse diagonal blocks
  count_launch();
  launch_k(k_inv_frob, dim3(T), dim3(256), (size_t)0, s, (const float*)G, ldg, N, (const float*)Wdiag, Y, ldy,
           partial, out, st);
  return cudaGetLastError() == cudaSuccess;
}

// Whether a 16-CTA cluster of k_chol_cluster can be resident on this device
// (a non-portable cluster size); decided once per process.
static bool chol16_ok() {
  static int ok = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    ok = 0;
    const size_t smem = cluster_smem_max(kCluster16CTAs, kClusterTMax);
    if (cudaFuncSetAttribute(k_chol_cluster<kCluster16CTAs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_chol_cluster<kCluster16CTAs>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCluster16CTAs);
    cfg.blockDim = dim3(kCholThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCluster16CTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_chol_cluster<kCluster16CTAs>, &cfg) == cudaSuccess && nclusters > 0)
      ok = 1;
    else
      cudaGetLastError();
  });
  return ok == 1;
}

bool chol_factor(float* G, long long ldg, int N, DevState* st, float* Wdiag, cudaStream_t s, const double* hrow,
                 float* zout, bool* fused) {
  // one tile: one CTA; up to kSmallN also without inverse diagonal blocks.  From two
  // tiles on, the cluster factor and the 4-CTA solves are faster (N = 64: 20 us
  // against 61 us for the single-CTA factor and solves; N = 128: 37 against 131)
  if (N <= kSmallNewton) {
    count_launch();
    launch_k(k_tile1_solve, dim3(1), dim3(32), 0, s, G, ldg, N, 1, st, (const double*)nullptr, (double*)nullptr, 1,
             1.0);
    return false;
  }
  if (N <= kSmallN && !Wdiag) {
    count_launch();
    launch_k(k_chol_small, dim3(1), dim3(kSmallThreads), (size_t)0, s, G, ldg, N, st);
    return false;
  }
  // above 16 tile rows the 8-CTA kernel holds one panel buffer (a full cluster barrier per step);
  // the 16-CTA kernel keeps two up to 19 tile rows and covers N <= kCluster16N
  const bool wide = Wdiag && N > 512 && N <= kCluster16N && chol16_ok();
  // the forward substitution inside the factor (an appended row h^T): one cluster launch,
  // N not a multiple of 32, inverse diagonal blocks for the backward solve
  const bool aug = hrow && zout && Wdiag && N % 32 != 0;
  const double* h = aug ? hrow : nullptr;
  if (fused) *fused = false;
  if (wide) {
    count_launch();
    launch_k(k_chol_cluster<kCluster16CTAs>, dim3(kCluster16CTAs), dim3(kCholThreads),
             (size_t)(cluster_smem((N + 31) / 32, kCluster16CTAs)), s, G, ldg, N, st, Wdiag, h, zout);
    if (cudaGetLastError() == cudaSuccess) {
      if (fused) *fused = aug;
      return true;
    }
  }
  if (N <= kClusterN) {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(k_chol_cluster<kClusterCTAs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem_max());
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
    count_launch();
    launch_k(k_chol_cluster<kClusterCTAs>, dim3(kClusterCTAs), dim3(kCholThreads), (size_t)(cluster_smem((N + 31) / 32)), s, G, ldg, N, st, Wdiag,
             h, zout);
    if (cudaGetLastError() == cudaSuccess) {
      if (fused) *fused = aug;
      return Wdiag != nullptr;
    }
  }
  if (Wdiag && N <= kMaxM) {
    // super-blocks of equal size (a multiple of 32, at most kClusterN)
    super_block_attrs();
    const int nb = (N + kClusterN - 1) / kClusterN;
    const int B = ((N + nb - 1) / nb + 31) / 32 * 32;
    bool launched = true;
    for (int k0 = 0; k0 < N && launched; k0 += B) {
      const int nk = N - k0 < B ? N - k0 : B;
      float* Gkk = G + k0 + (long long)k0 * ldg;
      count_launch();
      launch_k(k_chol_cluster<kClusterCTAs>, dim3(kClusterCTAs), dim3(kCholThreads), (size_t)(cluster_smem((nk + 31) / 32)), s, Gkk, ldg, nk, st,
               Wdiag + (long long)(k0 / 32) * 1024, (const double*)nullptr, (float*)nullptr);
      const int r0 = k0 + nk, R = N - r0;
      if (R > 0) {
        count_launch(2);
        launch_trsm_blocks(G, ldg, k0, nk, r0, R, Wdiag + (long long)(k0 / 32) * 1024, s);
        const int nt = (R + 31) / 32;
        launch_k(k_syrk_sub, dim3(nt * (nt + 1) / 2), dim3(kSubThreads), syrk_sub_smem(nk), s, G, ldg, r0, R, k0, nk);
      }
      launched = cudaGetLastError() == cudaSuccess;
    }
    if (launched) return true;
  }
  {
    // one cooperative launch; the grid barrier counters live in DevState
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_coop, kCoopThreads, 0);
    int grid = sms * (per_sm > 0 ? 1 : 0);
    const int T = (N + kT - 1) / kT;
    if (grid > T * (T + 1) / 2) grid = T * (T + 1) / 2;
    if (grid > 64) grid = 64;
    if (grid >= 1) {
      unsigned* bar = &st->counters[kCtrBarrier];
      void* args[] = {&G, &ldg, &N, &st, &bar};
      count_launch();
      if (cudaLaunchCooperativeKernel((void*)k_chol_coop, grid, kCoopThreads, args, 0, s) == cudaSuccess) return false;
      cudaGetLastError();
    }
  }
  for (int kb = 0; kb < N; kb += kCholNB) {
    const int nb = N - kb < kCholNB ? N - kb : kCholNB;
    count_launch();
    launch_k(k_potrf_diag, dim3(1), dim3(dim3(32, 32)), (size_t)(0), s, G, ldg, kb, nb, st);
    const int rem = N - kb - nb;
    if (rem > 0) {
      count_launch(2);
      launch_k(k_trsm_panel, dim3((rem + 255) / 256), dim3(256), (size_t)(0), s, G, ldg, kb, nb, N);
      const int T = (rem + kT - 1) / kT;
      launch_k(k_syrk_update, dim3(T * (T + 1) / 2), dim3(256), (size_t)(0), s, G, ldg, kb, nb, N);
    }
  }
  return false;
}

void launch_chol_solve_small(float* G, long long ldg, int N, DevState* st, const double* rhs, double* acc,
                             double alpha, cudaStream_t s) {
  if (N <= 0) return;
  count_launch();
  launch_k(k_tile1_solve, dim3(1), dim3(32), 0, s, G, ldg, N, 1, st, rhs, acc, 1, alpha);
}

// The pair solve (k_trsv_pair) when N <= 32 kTrsvPairMaxT and a tensor map over L can be made;
// false when it does not apply or the launch failed.  rpart != nullptr: the refinement mode
// (acc += c with the contraction test, see k_trsv_pair).
static bool launch_trsv_pair(const float* L, long long ldl, int N, const double* rhs, double* acc, int first,
                             double alpha, const float* Wdiag, DevState* st, double* rpart, double tau2,
                             cudaStream_t s, const float* zin = nullptr) {
  CUtensorMap tmL;
  if (N <= kSmallNewton || N > 32 * kTrsvPairMaxT || !make_factor_tensor_map(&tmL, L, ldl, N)) return false;
  const int T = (N + 31) / 32, T0 = (T + kTrsvQ - 1) / kTrsvQ;
  const size_t smem = 1024 + (size_t)T0 * kTrsvRing * 4096 + (size_t)2 * T * 32 * sizeof(float) +
                      (size_t)(2 * T + T0 * kTrsvRing) * 8 + (size_t)T0 * 32 * sizeof(float);
  static bool done_pr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !done_pr[dev]) {
    const int T0m = kTrsvMaxT0;
    cudaFuncSetAttribute(k_trsv_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(1024 + (size_t)T0m * kTrsvRing * 4096 + (size_t)2 * kTrsvPairMaxT * 32 * sizeof(float) +
                               (size_t)(2 * kTrsvPairMaxT + T0m * kTrsvRing) * 8 + (size_t)T0m * 32 * sizeof(float)));
    if (dev >= 0 && dev < 64) done_pr[dev] = true;
  }
  count_launch();
  launch_k(k_trsv_pair, dim3(kTrsvQ), dim3(32 * T0), smem, s, tmL, N, rhs, acc, first, alpha, Wdiag, st, rpart,
           tau2, zin);
  return cudaGetLastError() == cudaSuccess;
}

bool launch_trsv_back(const float* L, long long ldl, int N, const float* z, double* acc, int first, double alpha,
                      const float* Wdiag, DevState* st, cudaStream_t s) {
  if (N <= 0 || !Wdiag || !z) return false;
  return launch_trsv_pair(L, ldl, N, nullptr, acc, first, alpha, Wdiag, st, nullptr, 0.0, s, z);
}

void launch_trsv_refine(const float* L, long long ldl, int N, const double* rhs, double* acc, double* corr,
                        const float* Wdiag, double* rpart, double tau, DevState* st, cudaStream_t s) {
  if (N <= 0) return;
  if (Wdiag && rpart && launch_trsv_pair(L, ldl, N, rhs, acc, 0, 1.0, Wdiag, st, rpart, tau * tau, s)) return;
  launch_trsv_llt(L, ldl, N, rhs, corr, 1, 1.0, Wdiag, st, s);
  launch_refine_update(acc, corr, N, tau, st, s);
}

void launch_trsv_llt(const float* L, long long ldl, int N, const double* rhs, double* acc, int first,
                     double alpha, const float* Wdiag, DevState* st, cudaStream_t s) {
  if (N <= 0) return;
  if (N <= kSmallNewton) {
    count_launch();
    launch_k(k_tile1_solve, dim3(1), dim3(32), 0, s, const_cast<float*>(L), ldl, N, 0, st, rhs, acc, first, alpha);
    return;
  }
  if (N <= kSmallN && !Wdiag) {
    small_smem_attr();
    count_launch();
    launch_k(k_trsv_small, dim3(1), dim3(kSmallThreads), (size_t)(kSmallSmem), s, L, ldl, N, rhs, acc, first, alpha);
    return;
  }
  if (Wdiag && launch_trsv_pair(L, ldl, N, rhs, acc, first, alpha, Wdiag, st, nullptr, 0.0, s)) return;
  if (Wdiag && N <= 32 * kTrsvCLMaxT) {
    const int T = (N + 31) / 32;
    const int warps = (T + kTrsvCL - 1) / kTrsvCL;
    const size_t smem = (size_t)2 * T * 32 * sizeof(float) + (size_t)2 * T * 8;
    static bool done_cl[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done_cl[dev]) {
      cudaFuncSetAttribute(k_trsv_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((size_t)2 * kTrsvCLMaxT * 32 * sizeof(float) + (size_t)2 * kTrsvCLMaxT * 8));
      if (dev >= 0 && dev < 64) done_cl[dev] = true;
    }
    count_launch();
    launch_k(k_trsv_cluster, dim3(kTrsvCL), dim3(32 * warps), (size_t)(smem), s, L, ldl, N, rhs, acc, first, alpha, Wdiag, st);
    if (cudaGetLastError() == cudaSuccess) return;
  }
  if (Wdiag && N <= kClusterN) {
    static bool done_blk[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done_blk[dev]) {
      cudaFuncSetAttribute(k_trsv_blk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((2 * blk_stage_floats(kClusterN) + 2048 + 32) * sizeof(float)));
      if (dev >= 0 && dev < 64) done_blk[dev] = true;
    }
    count_launch();
    launch_k(k_trsv_blk, dim3(1), dim3(kBlkThreads), (size_t)((size_t)(2 * blk_stage_floats(N) + 2048 + 32) * sizeof(float)), s, 
        L, ldl, N, rhs, acc, first, alpha, Wdiag);
    return;
  }
  if (N <= kMidN) {
    const int ldb = (N + 3) & ~3;
    const size_t smem = (size_t)(64 * ldb + ldb + 32 * 33) * sizeof(float);
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      const int lb = (kMidN + 3) & ~3;
      cudaFuncSetAttribute(k_trsv_mid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((64 * lb + lb + 32 * 33) * sizeof(float)));
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
    count_launch();
    launch_k(k_trsv_mid, dim3(1), dim3(kMidThreads), (size_t)(smem), s, L, ldl, N, rhs, acc, first, alpha, Wdiag);
    return;
  }
  count_launch();
  launch_k(k_trsv_llt, dim3(1), dim3(kTrsvThreads), (size_t)((size_t)N * sizeof(float)), s, L, ldl, N, rhs, acc, first, alpha);
}

}  // namespace ssnal
