// Device-resident batched solver: many independent fits (Algorithm 1 each) in one
// launch.  A persistent kernel of one CTA per SM; each CTA takes the next instance from a
// device work queue (an atomic counter over an order the host sorts by size, largest
// first) and runs that instance's whole AL / SsN loop on-chip, then takes the next.  No
// host round trip and no launch per Newton step: the Newton loop itself runs on the
// device.  Every step of a fit is a block-level routine here:
//   * u = A^T y and t = A^T d (eq. Q_def / line_search): warp per column, float-float
//     products of the stored FP32 values with the hi/lo split of the vector;
//   * prox, the active set J (eq. Q_def) compacted in ascending order, the norms;
//   * g = y + b - A_J w_J (eq. grad_phy) and the panel products A_J v, A_J^T v, read from
//     A's columns through J (no gathered panel: r can be two orders above m);
//   * the Newton matrix kappa^{-1} I + A_J^T A_J (eq. smw_formula, r < m) or I + kappa A_J
//     A_J^T (eq. AJ_system, r >= m) in FP32 (32 x 32 tiles staged in shared memory), its
//     blocked Cholesky factor, triangular solves and one FP64 refinement step through A;
//   * the Armijo line search (eq. line_search) over the stored n-vectors, trials in
//     chunks of eight, and the multiplier update / KKT test of Algorithm 1.
// An instance whose FP32 Newton solve fails (non-positive pivot) or does not contract
// (refinement correction above half the solution) stops with kBatchNeedsHost; the host
// re-solves it on the regular path (FP64 Newton system).  All reductions are fixed-order
// block reductions, so results are repeatable.
#include "common.cuh"

namespace ssnal {

namespace {

struct BatchInst {
  const float* A;
  long long lda, n;
  int m, pad;
  const double* b;
  double lam1, lam2;
  double* x;  // in: warm start, out: solution
};

struct BatchOut {
  int status;  // 0 converged, 3 iteration caps, kBatchNeedsHost
  int al_iters, newton_iters, ls_trials;
  long long active;
  double kkt1, kkt3, primal_obj, dual_gap, sigma;
};

struct BatchOpts {
  double sigma0, sigma_growth, sigma_max, mu, beta, tol;
  int max_al, max_newton, max_ls, refine;
};

// Byte offsets of the per-CTA scratch (sized for the largest n and m of the batch).
struct BatchLayout {
  size_t slot_bytes;
  size_t u, t, w, rv, xw, J, y, d, g, tm, q, h, rs, cr, G, cs;
  int m_max;
};

constexpr int kBatchNeedsHost = 7;
constexpr int kTile = 32;
// Threads per CTA.  Fixed: the block reductions' order depends on it, and results must not
// depend on what the tuner picks.
constexpr int kBatchThreads = 512;

template <int BT>
struct Blk {
  static constexpr int NW = BT / 32;
};

// K values summed over the block in a fixed order; every thread returns the totals.
// red: 32 * K doubles of shared memory (K <= BT / 32).
template <int BT, int K>
__device__ __forceinline__ void bsum(double (&v)[K], double* red) {
  constexpr int NW = BT / 32;
  static_assert(K <= NW, "one warp per value in the second stage");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; k++) red[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp < K) {
    double s = lane < NW ? red[warp * 32 + lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[warp * 32] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; k++) v[k] = red[k * 32];
  __syncthreads();
}

// (S, L) += a * (dh + dl) with the product error kept (a exact in FP32).
__device__ __forceinline__ void ffmadd(float& S, float& L, float a, float dh, float dl) {
  const float p = __fmul_rn(a, dh);
  float e = __fmaf_rn(a, dh, -p);
  e = __fmaf_rn(a, dl, e);
  const float s = __fadd_rn(S, p);
  const float z = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(p, z));
  S = s;
  L = __fadd_rn(L, __fadd_rn(t, e));
}

__device__ __forceinline__ void ffadd(float& S, float& L, float S2, float L2) {
  const float s = __fadd_rn(S, S2);
  const float z = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(S2, z));
  S = s;
  L = __fadd_rn(__fadd_rn(L, L2), t);
}

// Columns of a 16-byte-aligned A, CW = VD / PS at a time per warp: lane l owns rows
// 4 l .. 4 l + 3 of each 128-row stripe (PS stripes per column, compile time, at least
// the S stripes of a column), so the VD 16-byte loads of a batch are all in flight
// before the first product.  Every lane accumulates its rows of a column in increasing
// order whatever VD and PS are.
template <int NW, int VD, int PS, typename Finish>
__device__ __forceinline__ void bstream_cols(const float* __restrict__ A, long long lda, int m, long long n, int S,
                                             const float* dh, const float* dl, int warp, int lane, Finish finish) {
  constexpr int CW = VD / PS;
  static_assert(CW >= 1 && CW * PS == VD, "whole columns per batch");
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (long long j0 = (long long)warp * CW; j0 < n; j0 += (long long)NW * CW) {
    float4 a[VD];
#pragma unroll
    for (int e = 0; e < VD; e++) {
      const int c = e / PS, st = e % PS;
      const long long j = j0 + c;
      const int i4 = lane + 32 * st;
      a[e] = (j < n && st < S && 4 * i4 < m) ? reinterpret_cast<const float4*>(A + j * lda)[i4] : zero4;
    }
    float FS[CW], FL[CW];
#pragma unroll
    for (int c = 0; c < CW; c++) FS[c] = FL[c] = 0.0f;
#pragma unroll
    for (int e = 0; e < VD; e++) {
      const int c = e / PS, st = e % PS;
      if (st >= S) continue;
      const int i0 = 4 * (lane + 32 * st);
      if (i0 >= m) continue;
      const float av[4] = {a[e].x, a[e].y, a[e].z, a[e].w};
      // 16-byte reads of the split vector (rows up to a multiple of 4 past m are in the buffer)
      const float4 h4 = *reinterpret_cast<const float4*>(dh + i0), l4 = *reinterpret_cast<const float4*>(dl + i0);
      const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (i0 + q < m) ffmadd(FS[c], FL[c], av[q], hv[q], lv[q]);
    }
#pragma unroll
    for (int c = 0; c < CW; c++)
      if (j0 + c < n) finish(j0 + c, FS[c], FL[c]);
  }
}

// out_j = sum_i A[i, j] vec_i for j < n, float-float (products of the FP32 entries with
// the hi / lo split of the vector scaled by a power of two), one warp per column.
// Columns 16-byte aligned (A and lda): lane l owns rows 4 l .. 4 l + 3 of every stripe of
// 128 rows and reads them with one 16-byte load; DEPTH / 2 such loads are in flight per
// lane, over several short columns at once (bstream_cols) or over stripes of one long
// column.  Otherwise: lane l owns rows l, l + 32, ..., DEPTH 4-byte loads in flight.
// Either way every lane accumulates its rows in increasing order and the lanes are merged
// by the same butterfly, so the result does not depend on DEPTH.
template <int BT, int DEPTH>
__device__ void bstream(const float* __restrict__ A, long long lda, int m, long long n, const double* vec,
                        double* out, float* dh, float* dl, unsigned long long* bits) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = BT / 32;
  if (tid == 0) *bits = 0ull;
  __syncthreads();
  unsigned long long mb = 0ull;
  for (int i = tid; i < m; i += BT) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(vec[i]) & 0x7FFFFFFFFFFFFFFFull;
    mb = b > mb ? b : mb;
  }
  atomicMax(bits, mb);
  __syncthreads();
  int ex = (int)((*bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) ex = 1023;
  const double scale = __longlong_as_double((long long)(2046 - ex) << 52);
  const double unscale = __longlong_as_double((long long)ex << 52);
  for (int i = tid; i < m; i += BT) {
    const double v = vec[i] * scale;
    const float h = __double2float_rn(v);
    dh[i] = h;
    dl[i] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  auto finish = [&](long long j, float S, float L) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S, o), L2 = __shfl_xor_sync(0xffffffffu, L, o);
      ffadd(S, L, S2, L2);
    }
    if (lane == 0) out[j] = ((double)S + (double)L) * unscale;
  };
  const bool vec4 = ((reinterpret_cast<unsigned long long>(A) & 15ull) == 0) && ((lda & 3) == 0);
  constexpr int VD = DEPTH / 2;
  const int S = (m + 127) / 128;
  if (vec4 && S <= VD) {
    // lda >= m and lda % 4 == 0: a 16-byte load that starts inside a column ends inside it
    if (S <= 1)
      bstream_cols<NW, VD, 1>(A, lda, m, n, S, dh, dl, warp, lane, finish);
    else if (S <= 2)
      bstream_cols<NW, VD, (VD >= 2 ? 2 : VD)>(A, lda, m, n, S, dh, dl, warp, lane, finish);
    else if (S <= 4)
      bstream_cols<NW, VD, (VD >= 4 ? 4 : VD)>(A, lda, m, n, S, dh, dl, warp, lane, finish);
    else
      bstream_cols<NW, VD, VD>(A, lda, m, n, S, dh, dl, warp, lane, finish);
  } else if (vec4) {
    // long columns: stripes in chunks of VD loads
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (long long j = warp; j < n; j += NW) {
      const float4* c0 = reinterpret_cast<const float4*>(A + j * lda);
      float S0 = 0.0f, L0 = 0.0f;
      for (int s0 = 0; s0 < S; s0 += VD) {
        float4 a[VD];
#pragma unroll
        for (int e = 0; e < VD; e++) {
          const int i4 = lane + 32 * (s0 + e);
          a[e] = (s0 + e < S && 4 * i4 < m) ? c0[i4] : zero4;
        }
#pragma unroll
        for (int e = 0; e < VD; e++) {
          if (s0 + e >= S) continue;
          const int i0 = 4 * (lane + 32 * (s0 + e));
          if (i0 >= m) continue;
          const float av[4] = {a[e].x, a[e].y, a[e].z, a[e].w};
          const float4 h4 = *reinterpret_cast<const float4*>(dh + i0), l4 = *reinterpret_cast<const float4*>(dl + i0);
          const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
          for (int q = 0; q < 4; q++)
            if (i0 + q < m) ffmadd(S0, L0, av[q], hv[q], lv[q]);
        }
      }
      finish(j, S0, L0);
    }
  } else {
    for (long long j = warp; j < n; j += NW) {
      const float* col = A + j * lda;
      float S = 0.0f, L = 0.0f;
      int i = lane;
      for (; i + 32 * (DEPTH - 1) < m; i += 32 * DEPTH) {
        float a[DEPTH];
#pragma unroll
        for (int e = 0; e < DEPTH; e++) a[e] = col[i + 32 * e];
#pragma unroll
        for (int e = 0; e < DEPTH; e++) ffmadd(S, L, a[e], dh[i + 32 * e], dl[i + 32 * e]);
      }
      for (; i < m; i += 32) ffmadd(S, L, col[i], dh[i], dl[i]);
      finish(j, S, L);
    }
  }
  __syncthreads();
}

// Power-of-two scale of a vector for the float-float products: every thread returns the
// scale that brings max |v_k| (k < len) into [1, 2) and its inverse (bits: one shared
// 64-bit word).  Ends with a block barrier.
template <int BT>
__device__ __forceinline__ void bscale(const double* v, long long len, unsigned long long* bits, double& scale,
                                       double& unscale) {
  if (threadIdx.x == 0) *bits = 0ull;
  __syncthreads();
  unsigned long long mb = 0ull;
  for (long long k = threadIdx.x; k < len; k += BT) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[k]) & 0x7FFFFFFFFFFFFFFFull;
    mb = b > mb ? b : mb;
  }
  atomicMax(bits, mb);
  __syncthreads();
  int ex = (int)((*bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) ex = 1023;
  scale = __longlong_as_double((long long)(2046 - ex) << 52);
  unscale = __longlong_as_double((long long)ex << 52);
}

// out_i = ca a_i + cb b_i + cs sum_k A[i, J_k] coef_k for i < m (a, b may be null).  The
// sum runs in float-float on the FP32 pipe (one SM's FP64 pipe retires about two FMAs
// per clock): coef is scaled by a power of two and split into FP32 hi / lo parts (csplit,
// r entries of scratch), every product of an FP32 entry with the split coefficient keeps
// its error (about 2^-46 relative per product), and the FP64 combination follows.
// With which != 0 also the dots used by the SsN step: which = 1 (gradient): ||out||^2,
// ||y||^2, ||y - out||^2, b^T y; which = 2 (direction): g^T out, y^T out, ||out||^2,
// b^T out, returned in dots[4] (every thread).
template <int BT>
__device__ void bgemv_n(const float* __restrict__ A, long long lda, int m, const int* __restrict__ J, long long r,
                        const double* coef, double* out, const double* a, double ca, const double* b, double cb,
                        double cs, int which, const double* yv, const double* bv, const double* gv, double* dots,
                        double* red, float2* csplit, unsigned long long* bits) {
  double scale, unscale;
  bscale<BT>(coef, r, bits, scale, unscale);
  for (long long k = threadIdx.x; k < r; k += BT) {
    const double v = coef[k] * scale;
    const float hi = __double2float_rn(v);
    csplit[k] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
  __syncthreads();
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < m; i += BT) {
    float S = 0.0f, Lo = 0.0f;
    long long k = 0;
    for (; k + 4 <= r; k += 4) {
      const float p0 = A[(long long)J[k] * lda + i], p1 = A[(long long)J[k + 1] * lda + i];
      const float p2 = A[(long long)J[k + 2] * lda + i], p3 = A[(long long)J[k + 3] * lda + i];
      const float2 c0 = csplit[k], c1 = csplit[k + 1], c2 = csplit[k + 2], c3 = csplit[k + 3];
      ffmadd(S, Lo, p0, c0.x, c0.y);
      ffmadd(S, Lo, p1, c1.x, c1.y);
      ffmadd(S, Lo, p2, c2.x, c2.y);
      ffmadd(S, Lo, p3, c3.x, c3.y);
    }
    for (; k < r; k++) {
      const float2 c = csplit[k];
      ffmadd(S, Lo, A[(long long)J[k] * lda + i], c.x, c.y);
    }
    const double acc = ((double)S + (double)Lo) * unscale;
    double lin = 0.0;
    if (a) lin = ca * a[i];
    if (b) lin = a ? lin + cb * b[i] : cb * b[i];
    const double o = (a || b) ? lin + cs * acc : cs * acc;
    out[i] = o;
    if (which == 1) {
      const double yi = yv[i];
      q[0] += o * o;
      q[1] += yi * yi;
      q[2] += (yi - o) * (yi - o);
      q[3] += bv[i] * yi;
    } else if (which == 2) {
      q[0] += gv[i] * o;
      q[1] += yv[i] * o;
      q[2] += o * o;
      q[3] += bv[i] * o;
    }
  }
  if (which) {
    bsum<BT, 4>(q, red);
    if (dots)
      for (int k = 0; k < 4; k++) dots[k] = q[k];
  } else {
    __syncthreads();
  }
}

// out_k = ch h_k + cq q_k + cd sum_i A[i, J_k] v_i for k < r, one warp per k, the sum in
// float-float as in bstream (v scaled by a power of two and split into vh, vl: m floats of
// shared memory each).
template <int BT>
__device__ void bgemv_t(const float* __restrict__ A, long long lda, int m, const int* __restrict__ J, long long r,
                        const double* v, double* out, const double* h, double ch, const double* q, double cq,
                        double cd, float* vh, float* vl, unsigned long long* bits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BT / 32;
  double scale, unscale;
  bscale<BT>(v, m, bits, scale, unscale);
  for (int i = threadIdx.x; i < m; i += BT) {
    const double z = v[i] * scale;
    const float hi = __double2float_rn(z);
    vh[i] = hi;
    vl[i] = __double2float_rn(z - (double)hi);
  }
  __syncthreads();
  for (long long k = warp; k < r; k += NW) {
    const float* col = A + (long long)J[k] * lda;
    float S = 0.0f, Lo = 0.0f;
    for (int i = lane; i < m; i += 32) ffmadd(S, Lo, col[i], vh[i], vl[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float S2 = __shfl_xor_sync(0xffffffffu, S, o), L2 = __shfl_xor_sync(0xffffffffu, Lo, o);
      ffadd(S, Lo, S2, L2);
    }
    if (lane == 0) {
      double o = cd * (((double)S + (double)Lo) * unscale);
      if (h) o = ch * h[k] + o;
      if (q) o = cq * q[k] + o;
      out[k] = o;
    }
  }
  __syncthreads();
}

// FP32 Newton matrix, lower triangle, ld = N:
//   trans = 0 (N = r): G[k1, k2] = diag [k1 == k2] + scale sum_i A[i, J_k1] A[i, J_k2]
//   trans = 1 (N = m): G[i1, i2] = diag [i1 == i2] + scale sum_k A[i1, J_k] A[i2, J_k]
// Output tiles of 32 x 32 (lower tile pairs), the K dimension in chunks of 32 staged in
// shared memory (As, Bs: 32 x 33 floats each).
template <int BT>
__device__ void bsyrk(const float* __restrict__ A, long long lda, int m, const int* __restrict__ J, long long r,
                      int trans, float diag, float scale, float* G, float* As, float* Bs) {
  const int N = trans ? m : (int)r;
  const long long K = trans ? r : (long long)m;
  const int T = (N + kTile - 1) / kTile;
  const int tid = threadIdx.x;
  for (int ti = 0; ti < T; ti++) {
    for (int tj = 0; tj <= ti; tj++) {
      const int i0 = ti * kTile, j0 = tj * kTile;
      float acc[1024 / BT > 0 ? 1024 / BT : 1];
      constexpr int PER = 1024 / BT;
#pragma unroll
      for (int e = 0; e < PER; e++) acc[e] = 0.0f;
      for (long long k0 = 0; k0 < K; k0 += kTile) {
        // stage As[kk][a] = X[k0 + kk, i0 + a] and Bs[kk][b] = X[k0 + kk, j0 + b]
        for (int e = tid; e < kTile * kTile; e += BT) {
          int kk, aa;
          float va = 0.0f, vb = 0.0f;
          if (trans == 0) {  // X[k, c] = A[k, J_c]: consecutive k contiguous
            kk = e & 31;
            aa = e >> 5;
            const long long k = k0 + kk;
            if (k < K) {
              if (i0 + aa < N) va = A[(long long)J[i0 + aa] * lda + k];
              if (j0 + aa < N) vb = A[(long long)J[j0 + aa] * lda + k];
            }
          } else {  // X[k, c] = A[c, J_k]: consecutive c contiguous
            aa = e & 31;
            kk = e >> 5;
            const long long k = k0 + kk;
            if (k < K) {
              const float* col = A + (long long)J[k] * lda;
              if (i0 + aa < N) va = col[i0 + aa];
              if (j0 + aa < N) vb = col[j0 + aa];
            }
          }
          As[kk * 33 + aa] = va;
          Bs[kk * 33 + aa] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PER; e++) {
          const int o = tid + e * BT, a = o >> 5, bq = o & 31;
          float s = acc[e];
#pragma unroll 8
          for (int kk = 0; kk < kTile; kk++) s = fmaf(As[kk * 33 + a], Bs[kk * 33 + bq], s);
          acc[e] = s;
        }
        __syncthreads();
      }
#pragma unroll
      for (int e = 0; e < PER; e++) {
        const int o = tid + e * BT, a = o >> 5, bq = o & 31;
        const int i = i0 + a, j = j0 + bq;
        if (i < N && j < N && i >= j) G[(long long)i * N + j] = (i == j ? diag : 0.0f) + scale * acc[e];
      }
    }
  }
  __syncthreads();
}

// Blocked right-looking Cholesky of the N x N lower triangle (row-major, ld = N), in
// place.  tile: 32 x 33 floats; panel: N x 33 floats (the current 32-column panel);
// flag: shared int set on a non-positive pivot.  Returns false on failure.
template <int BT>
__device__ bool bchol(float* G, int N, float* tile, float* panel, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = BT / 32;
  if (tid == 0) *flag = 0;
  __syncthreads();
  for (int kb = 0; kb < N; kb += kTile) {
    const int nb = N - kb < kTile ? N - kb : kTile;
    for (int e = tid; e < kTile * kTile; e += BT) {
      const int i = e >> 5, j = e & 31;
      tile[i * 33 + j] = (i < nb && j <= i) ? G[(long long)(kb + i) * N + kb + j] : 0.0f;
    }
    __syncthreads();
    // the diagonal block, column by column (warp 0; lane i owns row i)
    if (warp == 0) {
      for (int p = 0; p < nb; p++) {
        const float d = tile[p * 33 + p];
        if (!(d > 0.0f)) {
          if (lane == 0) *flag = 1;
          break;
        }
        const float l = sqrtf(d);
        __syncwarp();
        if (lane == p) tile[p * 33 + p] = l;
        if (lane > p && lane < nb) tile[lane * 33 + p] = tile[lane * 33 + p] / l;
        __syncwarp();
        if (lane > p && lane < nb) {
          const float lp = tile[lane * 33 + p];
          for (int j = p + 1; j <= lane; j++) tile[lane * 33 + j] = fmaf(-lp, tile[j * 33 + p], tile[lane * 33 + j]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (*flag) return false;
    for (int e = tid; e < kTile * kTile; e += BT) {
      const int i = e >> 5, j = e & 31;
      if (i < nb && j <= i) G[(long long)(kb + i) * N + kb + j] = tile[i * 33 + j];
    }
    // the rows below: row <- row L_kk^{-T}, kept in the panel buffer
    const int r0 = kb + nb;
    for (int i = r0 + tid; i < N; i += BT) {
      float x[kTile];
#pragma unroll
      for (int c = 0; c < kTile; c++) x[c] = c < nb ? G[(long long)i * N + kb + c] : 0.0f;
#pragma unroll
      for (int c = 0; c < kTile; c++) {
        if (c < nb) {
          float v = x[c];
          for (int l = 0; l < c; l++) v = fmaf(-x[l], tile[c * 33 + l], v);
          x[c] = v / tile[c * 33 + c];
        }
      }
#pragma unroll
      for (int c = 0; c < kTile; c++) {
        if (c < nb) G[(long long)i * N + kb + c] = x[c];
        panel[(i - r0) * 33 + c] = c < nb ? x[c] : 0.0f;
      }
    }
    __syncthreads();
    // trailing update of the lower triangle: a warp per row, lanes across columns
    for (int i = r0 + warp; i < N; i += NW) {
      const float* pi = panel + (i - r0) * 33;
      for (int j = r0 + lane; j <= i; j += 32) {
        const float* pj = panel + (j - r0) * 33;
        float s = 0.0f;
#pragma unroll 8
        for (int l = 0; l < kTile; l++) s = fmaf(pi[l], pj[l], s);
        G[(long long)i * N + j] -= s;
      }
    }
    __syncthreads();
  }
  return true;
}

// acc = alpha x (first) or acc += alpha x with L L^T x = rhs (L row-major lower, ld = N):
// FP32 arithmetic throughout (the FP32 factor bounds the solve's accuracy; the caller's
// refinement through A recovers the rest), with rhs scaled by a power of two into FP32's
// range.  xs: N doubles of scratch (global, used as N floats).
template <int BT>
__device__ void btrsv(const float* __restrict__ L, int N, const double* rhs, double* acc, int first, double alpha,
                      double* xs_scratch, unsigned long long* bits) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = BT / 32;
  float* xs = reinterpret_cast<float*>(xs_scratch);
  double scale, unscale;
  bscale<BT>(rhs, N, bits, scale, unscale);
  for (int i = tid; i < N; i += BT) xs[i] = __double2float_rn(rhs[i] * scale);
  __syncthreads();
  for (int b0 = 0; b0 < N; b0 += 32) {  // forward: L y = rhs
    const int nb = N - b0 < 32 ? N - b0 : 32;
    if (warp == 0) {
      float v = lane < nb ? xs[b0 + lane] : 0.0f;
      for (int p = 0; p < nb; p++) {
        float xp = __shfl_sync(0xffffffffu, v, p);
        xp = __fdiv_rn(xp, L[(long long)(b0 + p) * N + b0 + p]);
        if (lane == p) v = xp;
        if (lane > p && lane < nb) v = fmaf(-L[(long long)(b0 + lane) * N + b0 + p], xp, v);
      }
      if (lane < nb) xs[b0 + lane] = v;
    }
    __syncthreads();
    for (int i = b0 + nb + tid; i < N; i += BT) {
      float sacc = xs[i];
      const float* row = L + (long long)i * N + b0;
      for (int p = 0; p < nb; p++) sacc = fmaf(-row[p], xs[b0 + p], sacc);
      xs[i] = sacc;
    }
    __syncthreads();
  }
  for (int bb = (N + 31) / 32 - 1; bb >= 0; bb--) {  // backward: L^T x = y
    const int b0 = bb * 32;
    const int nb = N - b0 < 32 ? N - b0 : 32;
    for (int c = warp; c < nb; c += NW) {  // column b0 + c: the rows below the block
      float sacc = 0.0f;
      for (int i = b0 + nb + lane; i < N; i += 32) sacc = fmaf(L[(long long)i * N + b0 + c], xs[i], sacc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) xs[b0 + c] -= sacc;
    }
    __syncthreads();
    if (warp == 0) {
      float v = lane < nb ? xs[b0 + lane] : 0.0f;
      for (int p = nb - 1; p >= 0; p--) {
        float xp = __shfl_sync(0xffffffffu, v, p);
        xp = __fdiv_rn(xp, L[(long long)(b0 + p) * N + b0 + p]);
        if (lane == p) v = xp;
        if (lane < p) v = fmaf(-L[(long long)(b0 + p) * N + b0 + lane], xp, v);
      }
      if (lane < nb) xs[b0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < N; i += BT) {
    const double xi = (double)xs[i] * unscale;
    acc[i] = first ? alpha * xi : fma(alpha, xi, acc[i]);
  }
  __syncthreads();
}

struct PassNorms {
  long long r;
  double w2, w1, xw2, vw2, pen;
};

// Prox pass (eqs. prox_elastic, Q_def) over the n coordinates, optionally applying the
// accepted step first (u += s t, y += s d).  support != 0: J = support of x, w_J = x_J.
// J is compacted in ascending order (per chunk of BT entries: warp ballots and a block
// scan of the warp counts).
template <int BT>
__device__ PassNorms bprox(const double* x, double* u, const double* t, double* y, const double* d, long long n, int m,
                           ProxParams pp, int apply, double s, int support, int* J, double* w, int* wcnt,
                           double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = BT / 32;
  if (apply)
    for (int i = tid; i < m; i += BT) y[i] = __dadd_rn(y[i], __dmul_rn(s, d[i]));
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  long long pos = 0;
  for (long long base = 0; base < n; base += BT) {
    const long long j = base + tid;
    bool act = false, rare = false;
    double wv = 0.0, xj = 0.0, uj = 0.0, v = 0.0;
    if (j < n) {
      xj = x[j];
      if (support) {
        act = !is_zero_bits(xj);
        wv = xj;
      } else {
        uj = u[j];
        if (apply) {
          uj = fma(s, t[j], uj);
          u[j] = uj;
        }
        v = v_of(xj, uj, pp.sigma);
        act = abs_gt(v, pp.thr);
        rare = act || !is_zero_bits(xj) || abs_gt(uj, pp.lam1);
      }
    }
    // the rare terms (active entries, nonzero x, |u| > lam1) behind a warp-uniform
    // branch: as predicated instructions they would occupy the FP64 pipe for every entry
    if (!support) {
      if (!__any_sync(0xffffffffu, rare)) {
        if (j < n) q[3] += v * v;
      } else if (j < n) {
        if (act) {
          const double mag = __dsub_rn(fabs(v), pp.thr) * pp.inv_onep;
          const double wn = v < 0.0 ? -mag : mag;
          q[0] += wn * wn;
          q[1] += mag;
          q[2] += (xj - wn) * (xj - wn);
          q[3] += (v - wn) * (v - wn);
          wv = prox_value(v, pp);
        } else {
          q[3] += v * v;
          if (!is_zero_bits(xj)) q[2] += xj * xj;
        }
        if (abs_gt(uj, pp.lam1)) {
          const double e = fabs(uj) - pp.lam1;
          q[4] += e * e;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    long long off = pos;
    for (int w2 = 0; w2 < warp; w2++) off += wcnt[w2];
    long long total = 0;
    for (int w2 = 0; w2 < NW; w2++) total += wcnt[w2];
    if (act) {
      const long long p = off + __popc(bal & ((1u << lane) - 1u));
      J[p] = (int)j;
      w[p] = wv;
    }
    pos += total;
    __syncthreads();
  }
  PassNorms out;
  out.r = pos;
  if (!support) {
    bsum<BT, 5>(q, red);
    out.w2 = q[0];
    out.w1 = q[1];
    out.xw2 = q[2];
    out.vw2 = q[3];
    out.pen = q[4];
  } else {
    out.w2 = out.w1 = out.xw2 = out.vw2 = out.pen = 0.0;
  }
  return out;
}

// Trial sums of eq. line_search for trials [k0, k0 + 8) over the stored vectors.
template <int BT>
__device__ void btrials(const double* x, const double* u, const double* t, long long n, ProxParams pp, double s0,
                        double beta, int count, double (&acc)[8], double* red) {
#pragma unroll
  for (int q = 0; q < 8; q++) acc[q] = 0.0;
  for (long long j = threadIdx.x; j < n; j += BT) {
    const double v = v_of(x[j], u[j], pp.sigma);
    const double tj = t[j];
    if (fabs(v) <= pp.thr && fabs(__dsub_rn(v, __dmul_rn(pp.sigma, tj))) <= pp.thr) continue;
    double s = s0;
    const double fv = fmax(fabs(v) - pp.thr, 0.0);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (q < count) {
        const double a = __dsub_rn(v, __dmul_rn(s * pp.sigma, tj));
        const double fa = fmax(fabs(a) - pp.thr, 0.0);
        acc[q] += (fa - fv) * (fa + fv);
      }
      s *= beta;
    }
  }
  bsum<BT, 8>(acc, red);
}

struct BatchShared {
  int cur;
  int flag;
  int wcnt[32];
  unsigned long long bits;
};

template <int BT, int DEPTH>
__device__ void solve_one(const BatchInst& P, BatchOut& O, const BatchOpts& o, const BatchLayout& L, unsigned char* my,
                          BatchShared& sh, float* dh, float* dl, double* red, float* As, float* Bs, float* panel) {
  const float* A = P.A;
  const long long lda = P.lda, n = P.n;
  const int m = P.m;
  double* u = reinterpret_cast<double*>(my + L.u);
  double* t = reinterpret_cast<double*>(my + L.t);
  double* w = reinterpret_cast<double*>(my + L.w);
  double* rv = reinterpret_cast<double*>(my + L.rv);
  int* J = reinterpret_cast<int*>(my + L.J);
  double* y = reinterpret_cast<double*>(my + L.y);
  double* d = reinterpret_cast<double*>(my + L.d);
  double* g = reinterpret_cast<double*>(my + L.g);
  double* tm = reinterpret_cast<double*>(my + L.tm);
  double* q = reinterpret_cast<double*>(my + L.q);
  double* h = reinterpret_cast<double*>(my + L.h);
  double* rs = reinterpret_cast<double*>(my + L.rs);
  double* cr = reinterpret_cast<double*>(my + L.cr);
  float* G = reinterpret_cast<float*>(my + L.G);
  float2* csp = reinterpret_cast<float2*>(my + L.cs);
  const double* b = P.b;
  // the fit works on a copy of x: an instance handed back to the host keeps its warm start
  double* x = reinterpret_cast<double*>(my + L.xw);
  const int tid = threadIdx.x;
  for (long long j = tid; j < n; j += BT) x[j] = P.x[j];
  __syncthreads();
  double dots[4];
  // 1 + ||b||
  {
    double v[1] = {0.0};
    for (int i = tid; i < m; i += BT) v[0] += b[i] * b[i];
    bsum<BT, 1>(v, red);
    dots[0] = v[0];
  }
  const double nb1 = 1.0 + sqrt(dots[0]);
  // y0 = A x0 - b over the support of the warm start; u = A^T y0
  ProxParams pp;
  pp.sigma = o.sigma0;
  pp.lam1 = P.lam1;
  pp.lam2 = P.lam2;
  pp.thr = pp.sigma * pp.lam1;
  pp.onep = 1.0 + pp.sigma * pp.lam2;
  pp.inv_onep = 1.0 / pp.onep;
  PassNorms pn = bprox<BT>(x, u, t, y, d, n, m, pp, 0, 0.0, 1, J, w, sh.wcnt, red);
  bgemv_n<BT>(A, lda, m, J, pn.r, w, y, nullptr, 0.0, b, -1.0, 1.0, 0, nullptr, nullptr, nullptr, nullptr, red, csp, &sh.bits);
  bstream<BT, DEPTH>(A, lda, m, n, y, u, dh, dl, &sh.bits);
  double sigma = o.sigma0;
  int al = 0, newton = 0, trials = 0, converged = 0, host = 0;
  double kkt1 = INFINITY, kkt3 = INFINITY, s = 0.0;
  double pobj = 0.0, gap = NAN;
  long long active = 0;
  for (al = 1; al <= o.max_al; al++) {
    pp.sigma = sigma;
    pp.thr = sigma * pp.lam1;
    pp.onep = 1.0 + sigma * pp.lam2;
    pp.inv_onep = 1.0 / pp.onep;
    const double kappa = sigma / (1.0 + sigma * pp.lam2);
    int apply = 0, here = 0;
    double gdots[4];
    for (;;) {
      pn = bprox<BT>(x, u, t, y, d, n, m, pp, apply, s, 0, J, w, sh.wcnt, red);
      apply = 0;
      const long long r = pn.r;
      // g = y + b - A_J w_J with ||g||^2, ||y||^2, ||y - g||^2, b^T y
      bgemv_n<BT>(A, lda, m, J, r, w, g, y, 1.0, b, 1.0, -1.0, 1, y, b, nullptr, gdots, red, csp, &sh.bits);
      const double gn = sqrt(gdots[0]) / nb1;
      if (!(gn > o.tol) || here >= o.max_newton) break;
      // ---- Newton direction: (I + kappa A_J A_J^T) d = -g
      if (r == 0) {
        bgemv_n<BT>(A, lda, m, J, 0, w, d, nullptr, 0.0, g, -1.0, 0.0, 2, y, b, g, dots, red, csp, &sh.bits);
      } else if (r < m) {
        const int N = (int)r;
        bsyrk<BT>(A, lda, m, J, r, 0, (float)(1.0 / kappa), 1.0f, G, As, Bs);
        bgemv_t<BT>(A, lda, m, J, r, g, h, nullptr, 0.0, nullptr, 0.0, 1.0, dh, dl, &sh.bits);
        if (!bchol<BT>(G, N, As, panel, &sh.flag)) {
          host = 1;
          break;
        }
        btrsv<BT>(G, N, h, q, 1, 1.0, cr, &sh.bits);
        double rho = 0.0;
        for (int it = 0; it < o.refine; it++) {
          // rs = h - kappa^{-1} q - A_J^T (A_J q); correction cr2 = G^{-1} rs
          bgemv_n<BT>(A, lda, m, J, r, q, tm, nullptr, 0.0, nullptr, 0.0, 1.0, 0, nullptr, nullptr, nullptr, nullptr,
                      red, csp, &sh.bits);
          bgemv_t<BT>(A, lda, m, J, r, tm, rs, h, 1.0, q, -1.0 / kappa, -1.0, dh, dl, &sh.bits);
          btrsv<BT>(G, N, rs, rv, 1, 1.0, cr, &sh.bits);
          double v2[2] = {0.0, 0.0};
          for (int k = tid; k < N; k += BT) {
            const double c = rv[k], nq = q[k] + c;
            q[k] = nq;
            v2[0] += c * c;
            v2[1] += nq * nq;
          }
          bsum<BT, 2>(v2, red);
          if (it == 0) rho = v2[1] > 0.0 ? sqrt(v2[0] / v2[1]) : (v2[0] > 0.0 ? INFINITY : 0.0);
        }
        if (!(rho <= 0.5)) {
          host = 1;
          break;
        }
        bgemv_n<BT>(A, lda, m, J, r, q, d, nullptr, 0.0, g, -1.0, 1.0, 2, y, b, g, dots, red, csp, &sh.bits);
      } else {
        bsyrk<BT>(A, lda, m, J, r, 1, 1.0f, (float)kappa, G, As, Bs);
        if (!bchol<BT>(G, m, As, panel, &sh.flag)) {
          host = 1;
          break;
        }
        btrsv<BT>(G, m, g, d, 1, -1.0, cr, &sh.bits);
        double rho = 0.0;
        for (int it = 0; it < o.refine; it++) {
          // tm = -g - d - kappa A_J (A_J^T d); d += M^{-1} tm
          bgemv_t<BT>(A, lda, m, J, r, d, rv, nullptr, 0.0, nullptr, 0.0, 1.0, dh, dl, &sh.bits);
          bgemv_n<BT>(A, lda, m, J, r, rv, tm, g, -1.0, d, -1.0, -kappa, 0, nullptr, nullptr, nullptr, nullptr, red, csp, &sh.bits);
          btrsv<BT>(G, m, tm, rs, 1, 1.0, cr, &sh.bits);
          double v2[2] = {0.0, 0.0};
          for (int i = tid; i < m; i += BT) {
            const double c = rs[i], nd = d[i] + c;
            d[i] = nd;
            v2[0] += c * c;
            v2[1] += nd * nd;
          }
          bsum<BT, 2>(v2, red);
          if (it == 0) rho = v2[1] > 0.0 ? sqrt(v2[0] / v2[1]) : (v2[0] > 0.0 ? INFINITY : 0.0);
        }
        if (!(rho <= 0.5)) {
          host = 1;
          break;
        }
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = tid; i < m; i += BT) {
          const double di = d[i];
          v4[0] += g[i] * di;
          v4[1] += y[i] * di;
          v4[2] += di * di;
          v4[3] += b[i] * di;
        }
        bsum<BT, 4>(v4, red);
        for (int k = 0; k < 4; k++) dots[k] = v4[k];
      }
      // ---- t = A^T d and the line search (eq. line_search): the first trial s = beta^k
      // with psi(y + s d) - psi(y) <= mu s g^T d, at most max_ls trials (the last if none)
      bstream<BT, DEPTH>(A, lda, m, n, d, t, dh, dl, &sh.bits);
      const double coef = 1.0 / (2.0 * sigma * pp.onep);
      double sk = 1.0;
      int acc_k = -1;
      for (int k0 = 0; k0 < o.max_ls && acc_k < 0; k0 += 8) {
        const int cnt = o.max_ls - k0 < 8 ? o.max_ls - k0 : 8;
        double sums[8];
        btrials<BT>(x, u, t, n, pp, sk, o.beta, cnt, sums, red);
        for (int qk = 0; qk < cnt; qk++) {
          const double dpsi = sk * (dots[1] + dots[3]) + 0.5 * sk * sk * dots[2] + coef * sums[qk];
          if (dpsi <= o.mu * sk * dots[0]) {
            acc_k = k0 + qk;
            break;
          }
          if (k0 + qk < o.max_ls - 1) sk *= o.beta;
        }
      }
      trials += (acc_k >= 0 ? acc_k : o.max_ls - 1) + 1;
      s = sk;
      apply = 1;
      here++;
      newton++;
    }
    if (host) break;
    // ---- AL update (eq. update_x through the Moreau decomposition) and eq. kkt_res
    kkt1 = sqrt(gdots[0]) / nb1;
    const double aty_z = sqrt(pn.xw2) / sigma, znorm = sqrt(pn.vw2) / sigma;
    kkt3 = aty_z / (1.0 + sqrt(gdots[1]) + znorm);
    active = pn.r;
    pobj = 0.5 * gdots[2] + pp.lam1 * pn.w1 + 0.5 * pp.lam2 * pn.w2;
    const double dual = -(0.5 * gdots[1] + gdots[3]) - (pp.lam2 > 0 ? pn.pen / (2.0 * pp.lam2) : 0.0);
    gap = pp.lam2 > 0 ? pobj - dual : NAN;
    for (long long base = 0; base < n; base += BT) {  // the division behind a warp-uniform branch
      const long long j = base + tid;
      const bool in = j < n;
      const double v = in ? v_of(x[j], u[j], pp.sigma) : 0.0;
      const bool act = in && abs_gt(v, pp.thr);
      double w = 0.0;
      if (__any_sync(0xffffffffu, act) && act) w = prox_value(v, pp);  // zero exactly when inactive
      if (in) x[j] = w;
    }
    __syncthreads();
    if (kkt1 <= o.tol && kkt3 <= o.tol) {
      converged = 1;
      break;
    }
    sigma = fmin(sigma * o.sigma_growth, o.sigma_max);
  }
  if (!host)
    for (long long j = tid; j < n; j += BT) P.x[j] = x[j];
  if (tid == 0) {
    O.status = host ? kBatchNeedsHost : (converged ? 0 : 3);
    O.al_iters = al > o.max_al ? o.max_al : al;
    O.newton_iters = newton;
    O.ls_trials = trials;
    O.active = active;
    O.kkt1 = kkt1;
    O.kkt3 = kkt3;
    O.primal_obj = pobj;
    O.dual_gap = gap;
    O.sigma = sigma;
  }
  __syncthreads();
}

template <int BT, int DEPTH>
__global__ void __launch_bounds__(BT, 1) k_batch_solve(const BatchInst* __restrict__ insts,
                                                       const int* __restrict__ order, int count, int* next,
                                                       BatchOut* out, BatchOpts o, BatchLayout L,
                                                       unsigned char* scratch) {
  extern __shared__ __align__(16) unsigned char smb[];
  __shared__ BatchShared sh;
  __shared__ double red[8 * 32];
  float* As = reinterpret_cast<float*>(smb);
  float* Bs = As + kTile * 33;
  float* dh = Bs + kTile * 33;
  float* dl = dh + L.m_max;
  float* panel = dl + L.m_max;
  unsigned char* my = scratch + (size_t)blockIdx.x * L.slot_bytes;
  for (;;) {
    if (threadIdx.x == 0) sh.cur = atomicAdd(next, 1);
    __syncthreads();
    const int cur = sh.cur;
    __syncthreads();
    if (cur >= count) return;
    const int idx = order[cur];
    solve_one<BT, DEPTH>(insts[idx], out[idx], o, L, my, sh, dh, dl, red, As, Bs, panel);
  }
}

}  // namespace

// Host side: sizes the scratch, builds the descriptors, launches the persistent kernel.
// m_max rounded up to a multiple of 4: the split vector (dh, dl) is read 16 bytes at a time
static int m_max4(int m_max) { return (m_max + 3) & ~3; }

size_t batch_smem_bytes(int m_max) {
  m_max = m_max4(m_max);
  return sizeof(float) * ((size_t)2 * kTile * 33 + (size_t)2 * m_max + (size_t)m_max * 33);
}

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

size_t batch_slot_bytes(long long n_max, int m_max) {
  m_max = m_max4(m_max);
  size_t off = 0;
  off += 5 * align256(sizeof(double) * (size_t)n_max);  // u, t, w, rv, xw
  off += align256(sizeof(int) * (size_t)n_max);          // J
  off += 9 * align256(sizeof(double) * (size_t)m_max);   // y, d, g, tm, q, h, rs, cr, spare
  off += align256(sizeof(float) * (size_t)m_max * (size_t)m_max);
  off += align256(sizeof(float2) * (size_t)n_max);      // cs: split coefficients of the panel products
  return off;
}

// Launches one persistent solve of `count` instances (device descriptors inst_dev, visited
// in the order order_dev[0..count)) on `blocks` CTAs of kBatchThreads threads; depth: loads
// in flight per lane in the passes over A (4, 8 or 16).  Returns false on a launch error.
bool launch_batch_solve(const void* inst_dev, const int* order_dev, int count, int* next_dev, void* out_dev,
                        const double* opt6, const int* opt4, long long n_max, int m_max, unsigned char* scratch,
                        int blocks, int depth, cudaStream_t s) {
  m_max = m_max4(m_max);
  BatchOpts o;
  o.sigma0 = opt6[0];
  o.sigma_growth = opt6[1];
  o.sigma_max = opt6[2];
  o.mu = opt6[3];
  o.beta = opt6[4];
  o.tol = opt6[5];
  o.max_al = opt4[0];
  o.max_newton = opt4[1];
  o.max_ls = opt4[2];
  o.refine = opt4[3];
  BatchLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += align256(bytes);
    return at;
  };
  L.u = take(sizeof(double) * (size_t)n_max);
  L.t = take(sizeof(double) * (size_t)n_max);
  L.w = take(sizeof(double) * (size_t)n_max);
  L.rv = take(sizeof(double) * (size_t)n_max);
  L.xw = take(sizeof(double) * (size_t)n_max);
  L.J = take(sizeof(int) * (size_t)n_max);
  L.y = take(sizeof(double) * (size_t)m_max);
  L.d = take(sizeof(double) * (size_t)m_max);
  L.g = take(sizeof(double) * (size_t)m_max);
  L.tm = take(sizeof(double) * (size_t)m_max);
  L.q = take(sizeof(double) * (size_t)m_max);
  L.h = take(sizeof(double) * (size_t)m_max);
  L.rs = take(sizeof(double) * (size_t)m_max);
  L.cr = take(sizeof(double) * (size_t)m_max);
  take(sizeof(double) * (size_t)m_max);
  L.G = take(sizeof(float) * (size_t)m_max * (size_t)m_max);
  L.cs = take(sizeof(float2) * (size_t)n_max);
  L.slot_bytes = off;
  L.m_max = m_max;
  const size_t smem = batch_smem_bytes(m_max);
  const BatchInst* in = static_cast<const BatchInst*>(inst_dev);
  BatchOut* out = static_cast<BatchOut*>(out_dev);
  count_launch();
  cudaError_t e = cudaErrorInvalidValue;
#define SSNAL_BATCH(D)                                                                                      \
  do {                                                                                                    \
    cudaFuncSetAttribute(k_batch_solve<kBatchThreads, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         (int)smem);                                                                      \
    k_batch_solve<kBatchThreads, D><<<blocks, kBatchThreads, smem, s>>>(in, order_dev, count, next_dev, out, o, \
                                                                        L, scratch);                      \
    e = cudaGetLastError();                                                                               \
  } while (0)
  if (depth <= 4) SSNAL_BATCH(4);
  else if (depth <= 8) SSNAL_BATCH(8);
  else SSNAL_BATCH(16);
#undef SSNAL_BATCH
  return e == cudaSuccess;
}

size_t batch_inst_bytes() { return sizeof(BatchInst); }
size_t batch_out_bytes() { return sizeof(BatchOut); }

// Fills the device-layout descriptor of one instance into dst (batch_inst_bytes() bytes).
void batch_fill_inst(void* dst, const float* A, long long lda, long long n, int m, const double* b, double lam1,
                     double lam2, double* x) {
  BatchInst bi{};
  bi.A = A;
  bi.lda = lda;
  bi.n = n;
  bi.m = m;
  bi.b = b;
  bi.lam1 = lam1;
  bi.lam2 = lam2;
  bi.x = x;
  memcpy(dst, &bi, sizeof(bi));
}

// Reads one result (batch_out_bytes() bytes at src) into the public result struct.
void batch_read_out(const void* src, ssnal_en_result* r, int* needs_host) {
  BatchOut bo;
  memcpy(&bo, src, sizeof(bo));
  *needs_host = bo.status == kBatchNeedsHost;
  r->status = bo.status == 0 ? SSNAL_EN_OK : SSNAL_EN_ENOCONV;
  r->al_iters = bo.al_iters;
  r->newton_iters = bo.newton_iters;
  r->ls_trials = bo.ls_trials;
  r->active = bo.active;
  r->kkt1 = bo.kkt1;
  r->kkt3 = bo.kkt3;
  r->primal_obj = bo.primal_obj;
  r->dual_gap = bo.dual_gap;
  r->sigma = bo.sigma;
}

}  // namespace ssnal
