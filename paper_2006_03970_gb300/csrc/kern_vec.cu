// O(n) and O(m r) kernels of the SsN step:
//   * prox + active set + ordered compaction of J (eqs. prox_elastic, Q_def),
//   * gather of A_J into a packed panel,
//   * the panel GEMVs A_J w (eq. grad_phy) and A_J^T v (eq. smw_formula),
//   * m-vector combines with the scalar products the line search needs,
//   * the start of a solve (state zeroed, b copied), vector copies, and the copy
//     of the solver state into the host mirror that the host polls.
// Every reduction runs in a fixed order, so results are bitwise repeatable.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"

namespace ssnal {

std::atomic<long long> g_launches{0};

constexpr int kVecThreads = 256;
constexpr int kVecMaxBlocks = 1024;  // every block of pass 2 reads all per-block counts

// Blocks for the O(n) passes: at most four per SM (and kVecMaxBlocks) and at least
// 256 entries per block, so that the FP64 work (a few FP64 operations per entry,
// at the GPU's low FP64 rate) is spread evenly over the SMs.  At n = 1e5 four
// blocks per SM (one entry per thread) made the whole solve path about 1 % faster
// than two per SM (401.9 against 398.7 fits/s on the m = 500, n = 1e5 path).
int vec_grid(long long n, int sms) {
  long long g = (n + 255) / 256;
  long long cap = 4LL * sms;
  if (cap > kVecMaxBlocks) cap = kVecMaxBlocks;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Inclusive scan over the block of one long long per thread (blockDim == 256).
__device__ long long block_incl_scan(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    long long w = (lane < (kVecThreads / 32)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < (kVecThreads / 32)) sh[lane] = w;
  }
  __syncthreads();
  long long add = warp > 0 ? sh[warp - 1] : 0;
  __syncthreads();
  return v + add;
}

__device__ __forceinline__ void block_range(long long n, long long& start, long long& stop) {
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  start = (long long)blockIdx.x * chunk;
  stop = start + chunk;
  if (stop > n) stop = n;
  if (start > n) start = n;
}

// Pass 1 of the prox / active-set step.  Optionally applies the accepted
// line-search step first (u += s t, y += s d).  Per block: number of active
// entries (integer reduction) and five partial norms (one FP64 reduction),
// written to counts[b] and partials[6 b ..].  No tail: the next kernel (pass 2)
// reads them once this grid has completed.
template <int MODE>
__global__ void __launch_bounds__(kVecThreads) k_prox_count(const double* __restrict__ x, double* __restrict__ u,
                                                            const double* __restrict__ t, double* __restrict__ y,
                                                            const double* __restrict__ d, long long n, int m,
                                                            ProxParams pp, int apply_update, DevState* st,
                                                            long long* counts, double* partials) {
  pdl_entry();
  __shared__ double red[5 * kVecThreads];
  __shared__ unsigned cred[kVecThreads / 32];
  long long start, stop;
  block_range(n, start, stop);
  // a Newton direction flagged as unreliable (failed FP32 factor or a refinement that
  // does not contract) is not applied: y and u stay, and the host recomputes the
  // direction in FP64.  The flags are read from memory written by earlier kernels, so
  // every block takes the same decision.
  if (apply_update && (st->chol_fail | st->newton_bad | st->f64_fail)) apply_update = 0;
  const double s = apply_update ? st->s : 0.0;
  // y += s d in the last block, whose range of entries is the shortest
  if (apply_update && blockIdx.x == gridDim.x - 1) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = __dadd_rn(y[i], __dmul_rn(s, d[i]));
  }
  unsigned cnt = 0;
  double w2 = 0, w1 = 0, xw2 = 0, vw2 = 0, pen = 0;
  // every lane of a warp runs the same iterations (entries past `stop` masked), so that
  // the rare terms sit behind warp-uniform branches: as predicated instructions they
  // would occupy the FP64 pipe, the slow one here, for every entry
  const int lane = threadIdx.x & 31;
  for (long long base = start + (threadIdx.x & ~31); base < stop; base += blockDim.x) {
    const long long j = base + lane;
    const bool in = j < stop;
    const double xj = in ? x[j] : 0.0;
    if (MODE == kProxSupport) {
      if (!is_zero_bits(xj)) cnt++;
      continue;
    }
    double uj = in ? u[j] : 0.0;
    if (apply_update && in) {
      uj = fma(s, t[j], uj);
      u[j] = uj;
    }
    const double v = v_of(xj, uj, pp.sigma);
    // the count uses the active test itself (eq. Q_def); w only feeds the norms,
    // so the reciprocal of 1 + sigma*lam2 replaces the division here.  Terms that
    // are exactly zero (w = 0, x = 0, |u| <= lam1) are skipped: FP64 is slow here
    const bool act = in && is_active(v, pp), xnz = !is_zero_bits(xj), pu = in && abs_gt(uj, pp.lam1);
    if (__any_sync(0xffffffffu, act || xnz || pu)) {
      if (act) {
        cnt++;
        const double mag = __dsub_rn(fabs(v), pp.thr) * pp.inv_onep;  // > 0
        const double w = v < 0.0 ? -mag : mag;
        w2 += w * w;
        w1 += mag;
        xw2 += (xj - w) * (xj - w);
        vw2 += (v - w) * (v - w);
      } else if (in) {  // w = 0
        vw2 += v * v;
        if (xnz) xw2 += xj * xj;
      }
      if (pu) {
        const double e = fabs(uj) - pp.lam1;
        pen += e * e;
      }
    } else if (in) {  // w = 0, x = 0, |u| <= lam1
      vw2 += v * v;
    }
  }
  const unsigned wc = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0) cred[threadIdx.x >> 5] = wc;
  if (MODE == kProxThreshold) {
    const double q[5] = {w2, w1, xw2, vw2, pen};
    const double tot = block_sum_k<5>(q, red, kVecThreads / 32);  // its barriers also publish cred
    if (threadIdx.x < 5) partials[blockIdx.x * 6 + threadIdx.x] = tot;
  } else {
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    long long c = 0;
    for (int w = 0; w < kVecThreads / 32; w++) c += cred[w];
    counts[blockIdx.x] = c;
  }
}

// Sum of a long long over the block (blockDim == kVecThreads); every thread
// gets the total.
__device__ __forceinline__ long long block_sum_ll(long long v, long long* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  long long tot = 0;
#pragma unroll
  for (int w = 0; w < kVecThreads / 32; w++) tot += sh[w];
  return tot;
}

// Pass 2: ordered compaction.  Block b first forms its offset, the sum of the
// counts of blocks 0..b-1 written by pass 1 (block 0 also writes r and reduces
// the norms into the state, in a fixed order); then it writes its active
// indices, ascending, from that offset; w_J holds the prox values (eq.
// prox_elastic).
template <int MODE>
__global__ void __launch_bounds__(kVecThreads) k_prox_scatter(const double* __restrict__ x,
                                                              const double* __restrict__ u, long long n,
                                                              ProxParams pp, const long long* __restrict__ counts,
                                                              const double* __restrict__ partials, DevState* st,
                                                              int32_t* __restrict__ J, double* __restrict__ wJ) {
  pdl_entry();
  __shared__ long long shl[32];
  __shared__ long long tile_total;
  __shared__ double red[5 * kVecThreads];
  const int G = gridDim.x, b = blockIdx.x;
  long long start, stop;
  block_range(n, start, stop);
  // the entries of the first tile are loaded and classified before the counts of
  // the blocks ahead are read, so that the two latencies overlap
  // called by every thread of the block alike: the prox value (a division) is formed
  // behind a warp-uniform branch, so inactive warps issue no FP64 division
  auto classify = [&](long long j, double& w, bool& act) {
    w = 0.0;
    act = false;
    double v = 0.0;
    if (j < stop) {
      const double xj = x[j];
      if (MODE == kProxSupport) {
        w = xj;
        act = !is_zero_bits(xj);
      } else {
        v = v_of(xj, u[j], pp.sigma);
        act = is_active(v, pp);
      }
    }
    if (MODE != kProxSupport && __any_sync(0xffffffffu, act) && act) w = prox_value(v, pp);  // zero exactly when inactive
  };
  double w0;
  bool act0;
  classify(start + threadIdx.x, w0, act0);
  long long before = 0, all_cnt = 0;
  for (int c = threadIdx.x; c < G; c += kVecThreads) {
    const long long v = __ldcg(&counts[c]);
    all_cnt += v;
    if (c < b) before += v;
  }
  before = block_sum_ll(before, shl);
  all_cnt = block_sum_ll(all_cnt, shl);
  if (b == 0) {
    if (threadIdx.x == 0) st->r = all_cnt;
    if (MODE == kProxThreshold) {
      double q[5] = {0, 0, 0, 0, 0};
      for (int c = threadIdx.x; c < G; c += kVecThreads)
#pragma unroll
        for (int k = 0; k < 5; k++) q[k] += ld_cg(&partials[c * 6 + k]);
      const double tot = block_sum_k<5>(q, red, kVecThreads / 32);
      if (threadIdx.x == 0) st->w2 = tot;
      if (threadIdx.x == 1) st->w1 = tot;
      if (threadIdx.x == 2) st->xw2 = tot;
      if (threadIdx.x == 3) st->vw2 = tot;
      if (threadIdx.x == 4) st->dualpen = tot;
    }
  }
  long long pos = before;
  for (long long base = start; base < stop; base += blockDim.x) {
    const long long j = base + threadIdx.x;
    double w = w0;
    bool act = act0;
    if (base != start) classify(j, w, act);
    long long incl = block_incl_scan(act ? 1 : 0, shl);
    if (act) {
      long long p = pos + incl - 1;
      J[p] = (int32_t)j;
      wJ[p] = w;
    }
    if (threadIdx.x == kVecThreads - 1) tile_total = incl;
    __syncthreads();
    pos += tile_total;
    __syncthreads();
  }
}

// x <- prox_{sigma p}(x - sigma u): the multiplier update of eq. update_x
// written through the Moreau decomposition.
// The lanes of a warp run the same iterations, and the prox value (a division) is formed
// behind a warp-uniform branch: warps without an active entry issue no FP64 division.
__global__ void k_set_x(double* __restrict__ x, const double* __restrict__ u, long long n, ProxParams pp) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < n;
       base += (long long)gridDim.x * blockDim.x) {
    const long long j = base + lane;
    const bool in = j < n;
    const double v = in ? v_of(x[j], u[j], pp.sigma) : 0.0;
    const bool act = in && is_active(v, pp);
    double w = 0.0;
    if (__any_sync(0xffffffffu, act) && act) w = prox_value(v, pp);  // zero exactly when inactive
    if (in) x[j] = w;
  }
}

// Element loaders for the gather: value of A(i, col) as double.
struct LoadF64 {
  const double* __restrict__ A;
  __device__ double operator()(long long, long long off) const { return __ldg(A + off); }
};
struct LoadF32 {
  const float* A;
  __device__ double operator()(long long, long long off) const { return (double)A[off]; }
};
struct LoadBF16 {
  const __nv_bfloat16* A;
  __device__ double operator()(long long, long long off) const { return (double)__bfloat162float(A[off]); }
};
// genotype codes: entry (code - mean_j) * scale_j, evaluated in FP64
struct LoadI8 {
  const int8_t* A;
  const float* mean;
  const float* scale;
  __device__ double operator()(long long col, long long off) const {
    return ((double)A[off] - (double)mean[col]) * (double)scale[col];
  }
};

// 2-bit genotype codes, four per byte (element offset off counts codes: byte off / 4,
// bits 2 (off mod 4) ..): entry (code - mean_j) * scale_j, evaluated in FP64.  The
// column stride is a multiple of 64 codes, so off mod 4 is the row mod 4.
struct LoadI2 {
  const uint8_t* A;
  const float* mean;
  const float* scale;
  __device__ double operator()(long long col, long long off) const {
    const unsigned code = (A[off >> 2] >> (2 * (unsigned)(off & 3))) & 3u;
    return ((double)code - (double)mean[col]) * (double)scale[col];
  }
};

// Gather of A_J: P[:, k] = A[:, J[k]] (FP64) and P32[:, k] = float(P[:, k]).
// One warp per column, grid-stride, 16 loads per lane in flight.  If r exceeds the panel capacity nothing is
// written and the overflow flag is raised for the host.
template <class Load>
__global__ void __launch_bounds__(256) k_gather(Load ld, long long lda, int m, const int32_t* __restrict__ J, const DevState* st,
                         long long r_host, long long rcap, double* __restrict__ P, long long ldp,
                         float* __restrict__ P32, long long ldp32, int* overflow) {
  pdl_entry();
  const long long r = r_host >= 0 ? r_host : st->r;
  if (r > rcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *overflow = 1;
    return;
  }
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long tw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = gw; k < r; k += tw) {
    const long long col = J[k], src = col * lda;
    double* dst = P + k * ldp;
    float* dst32 = P32 + k * ldp32;
    // 16 loads per lane in flight before any store: one column of up to 512 rows
    // costs one memory round trip
    for (int i0 = 0; i0 < m; i0 += 32 * 16) {
      double v[16];
#pragma unroll
      for (int e = 0; e < 16; e++) {
        const int i = i0 + lane + 32 * e;
        v[e] = i < m ? ld(col, src + i) : 0.0;
      }
#pragma unroll
      for (int e = 0; e < 16; e++) {
        const int i = i0 + lane + 32 * e;
        if (i < m) {
          dst[i] = v[e];
          dst32[i] = (float)v[e];
        }
      }
    }
  }
}

// part[g*m + i] = sum_{k in group g} P[i, k] * coef[k]; groups are contiguous
// ranges of ceil(r / kGemvGroups) columns.  Grid (ceil(m/256), kGemvGroups).
__global__ void __launch_bounds__(kVecThreads) k_gemv_n_partial(const double* __restrict__ P, long long ldp, int m,
                                                                const double* __restrict__ coef,
                                                                const DevState* st, long long r_host,
                                                                long long rcap, double* __restrict__ part) {
  pdl_entry();
  const long long r = r_host >= 0 ? r_host : st->r;
  if (r > rcap) return;  // the gather raised the overflow flag; the host redoes this step
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  const long long gs = (r + kGemvGroups - 1) / kGemvGroups;
  long long k0 = g * gs, k1 = k0 + gs;
  if (k1 > r) k1 = r;
  if (i >= m) return;
  double acc = 0.0;
  for (long long k = k0; k < k1; k++) acc = fma(P[i + k * ldp], coef[k], acc);
  part[(long long)g * m + i] = acc;
}

// out_i = ca*a_i + cb*b_i + cs*sum_g part[g][i], then optional scalar products.
// which = 1: gradient (g2, y2, yg2, by); which = 2: direction (gd, yd, dd, bd).
__global__ void __launch_bounds__(kVecThreads) k_combine(double* __restrict__ out, const double* __restrict__ a,
                                                         double ca, const double* __restrict__ b, double cb,
                                                         const double* __restrict__ part, double cs, int m,
                                                         int which, const double* __restrict__ yv,
                                                         const double* __restrict__ bv,
                                                         const double* __restrict__ gv, DevState* st,
                                                         double* scratch) {
  pdl_entry();
  __shared__ double red4[4 * kVecThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double o = 0.0;
  if (i < m) {
    double sum = 0.0;
    if (part) {
      sum = ordered_sum_cg(part + i, m, kGemvGroups);
    }
    double lin = 0.0;
    if (a) lin = ca * a[i];
    if (b) lin = a ? lin + cb * b[i] : cb * b[i];
    o = (a || b) ? (part ? lin + cs * sum : lin) : cs * sum;
    out[i] = o;
  }
  if (which == 0) return;
  double q[4] = {0, 0, 0, 0};
  if (i < m) {
    const double yi = yv[i], bi = bv[i];
    if (which == 1) {
      q[0] = o * o;
      q[1] = yi * yi;
      q[2] = (yi - o) * (yi - o);
      q[3] = bi * yi;
    } else {
      const double gi = gv[i];
      q[0] = gi * o;
      q[1] = yi * o;
      q[2] = o * o;
      q[3] = bi * o;
    }
  }
  {
    const double tot = block_sum_k<4>(q, red4, kVecThreads / 32);
    if (threadIdx.x < 4) scratch[blockIdx.x * 4 + threadIdx.x] = tot;
  }
  if (!last_block(&st->counters[kCtrCombine])) return;
  if (threadIdx.x < 4) {
    const int k = threadIdx.x;
    const double tot = ordered_sum_cg(scratch + k, 4, (int)gridDim.x);
    double* dst = which == 1 ? (k == 0 ? &st->g2 : k == 1 ? &st->y2 : k == 2 ? &st->yg2 : &st->by)
                             : (k == 0 ? &st->gd : k == 1 ? &st->yd : k == 2 ? &st->dd : &st->bd);
    *dst = tot;
  }
  reset_counter(&st->counters[kCtrCombine]);
}

// out_i = ca*a_i + cb*b_i + cs*sum_k P[i, k] coef[k]: 32 rows x 8 column groups per
// block (coalesced column reads), the groups summed in a fixed order; optional
// scalar products as in k_combine, reduced by the last block.
constexpr int kGemvChunk = 64;     // columns per block of the panel GEMV
constexpr int kGemvMaxSplit = 32;  // column chunks per row tile (more columns loop inside a chunk)

__global__ void __launch_bounds__(256) k_gemv_n(const double* __restrict__ P, long long ldp, int m,
                                                const double* __restrict__ coef, const DevState* st,
                                                long long r_host, long long rcap, double* __restrict__ out,
                                                const double* __restrict__ a, double ca, const double* __restrict__ b,
                                                double cb, double cs, int which, const double* __restrict__ yv,
                                                const double* __restrict__ bv, const double* __restrict__ gv,
                                                DevState* stw, double* scratch, double* __restrict__ cpart,
                                                unsigned* tile_ctr) {
  pdl_entry();
  __shared__ double part[8][33];
  __shared__ double red4[4 * 32];
  __shared__ bool tile_last;
  const long long r = r_host >= 0 ? r_host : st->r;
  if (r > rcap) return;  // the gather raised the overflow flag; the host redoes this step
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  // column chunks depend on r only (never on the launch shape), so the
  // summation order -- and the result -- is the same for every launch
  long long nsplit = (r + kGemvChunk - 1) / kGemvChunk;
  if (nsplit > (long long)gridDim.y) nsplit = gridDim.y;
  if (nsplit < 1) nsplit = 1;
  const long long per = (r + nsplit - 1) / nsplit;
  const long long k0 = blockIdx.y < nsplit ? (long long)blockIdx.y * per : r;
  const long long k1 = (k0 + per) < r ? (k0 + per) : r;
  double acc = 0.0;
  if (i < m) {
#pragma unroll 4
    for (long long k = k0 + grp; k < k1; k += 8) acc = fma(P[i + k * ldp], coef[k], acc);
  }
  part[grp][lane] = acc;
  __syncthreads();
  if (gridDim.y > 1) {
    if (grp == 0) {
      double sum = 0.0;
      for (int g = 0; g < 8; g++) sum += part[g][lane];
      if (i < m) cpart[(long long)blockIdx.y * m + i] = sum;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&tile_ctr[blockIdx.x], 1u);
      tile_last = (prev == gridDim.y - 1);
      if (tile_last) tile_ctr[blockIdx.x] = 0u;
    }
    __syncthreads();
    if (!tile_last) return;
    __threadfence();
  }
  double o = 0.0;
  if (grp == 0 && i < m) {
    double sum = 0.0;
    if (gridDim.y > 1)
      sum = ordered_sum_cg(cpart + i, m, (int)nsplit);
    else
      for (int g = 0; g < 8; g++) sum += part[g][lane];
    double lin = 0.0;
    if (a) lin = ca * a[i];
    if (b) lin = a ? lin + cb * b[i] : cb * b[i];
    o = (a || b) ? lin + cs * sum : cs * sum;
    out[i] = o;
  }
  if (which == 0) return;
  double q[4] = {0, 0, 0, 0};
  if (grp == 0 && i < m) {
    const double yi = yv[i], bi = bv[i];
    if (which == 1) {
      q[0] = o * o;
      q[1] = yi * yi;
      q[2] = (yi - o) * (yi - o);
      q[3] = bi * yi;
    } else {
      const double gi = gv[i];
      q[0] = gi * o;
      q[1] = yi * o;
      q[2] = o * o;
      q[3] = bi * o;
    }
  }
  {
    const double tot = block_sum_k<4>(q, red4, 1);  // warp 0 holds the rows
    if (threadIdx.x < 4) scratch[blockIdx.x * 4 + threadIdx.x] = tot;
  }
  // only the row tiles' last blocks get here: count them against gridDim.x
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&stw->counters[kCtrGemv], 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (threadIdx.x < 4) {
    const int k = threadIdx.x;
    const double tot = ordered_sum_cg(scratch + k, 4, (int)gridDim.x);
    double* dst = which == 1 ? (k == 0 ? &stw->g2 : k == 1 ? &stw->y2 : k == 2 ? &stw->yg2 : &stw->by)
                             : (k == 0 ? &stw->gd : k == 1 ? &stw->yd : k == 2 ? &stw->dd : &stw->bd);
    *dst = tot;
  }
  reset_counter(&stw->counters[kCtrGemv]);
}

// The same GEMV, combine and scalar products on one thread-block cluster, for
// panels that sit in L2 (m times the panel capacity <= 2^22).  The C CTAs split the r
// columns into C equal contiguous chunks; CTA c sums P[i, k] coef[k] over its
// chunk for every row (one row per thread per pass, kGemvClUnroll columns of
// loads in flight) into its shared memory.  After a cluster barrier CTA c owns
// rows [c*mr, (c+1)*mr): it adds the C partial sums of each row in CTA order
// (distributed shared memory), applies the combine and reduces its rows' scalar
// products, which CTA 0 sums in CTA order after a second barrier.  One launch,
// no global atomics; the order depends on r and C only.
constexpr int kGemvClThreads = 512;
constexpr int kGemvClUnroll = 16;
constexpr int kGemvClMax = 16;                  // largest cluster the kernel is launched with
constexpr int kGemvClMaxRows = 16384;           // rows of the partial-sum vector in shared memory
constexpr long long kGemvClMaxEntries = 1 << 22;  // m * rcap up to which the cluster kernel is used

__global__ void __launch_bounds__(kGemvClThreads) k_gemv_cl(const double* __restrict__ P, long long ldp, int m,
                                                            const double* __restrict__ coef, const DevState* st,
                                                            long long r_host, long long rcap,
                                                            double* __restrict__ out, const double* __restrict__ a,
                                                            double ca, const double* __restrict__ b, double cb,
                                                            double cs, int which, const double* __restrict__ yv,
                                                            const double* __restrict__ bv,
                                                            const double* __restrict__ gv, DevState* stw) {
  pdl_entry();
  extern __shared__ double cl_part[];  // m partial row sums of this CTA's columns
  __shared__ double red[4 * kGemvClThreads];
  __shared__ double scal[kGemvClMax][4];
  const int C = (int)cluster_size(), c = (int)cluster_rank();
  const int tid = threadIdx.x;
  // this CTA's rows of the combine; the operands of each thread's first row are
  // loaded now, so that their latency is spent during the products
  const int mr = (m + C - 1) / C;
  const int r0 = min(m, c * mr), r1 = min(m, r0 + mr);
  double fa = 0.0, fb = 0.0, fy = 0.0, fbv = 0.0, fg = 0.0;
  if (r0 + tid < r1) {
    const int i = r0 + tid;
    if (a) fa = a[i];
    if (b) fb = b[i];
    if (which != 0) {
      fy = yv[i];
      fbv = bv[i];
    }
    if (which == 2) fg = gv[i];
  }
  const long long r = r_host >= 0 ? r_host : st->r;
  if (r > rcap) return;  // the same r in every CTA: none reaches a barrier
  const long long per = (r + C - 1) / C;
  const long long k0 = min(r, (long long)c * per), k1 = min(r, k0 + per);
  for (int i0 = 0; i0 < m; i0 += kGemvClThreads) {
    const int i = i0 + tid;
    if (i >= m) break;
    const double* p = P + i;
    double acc = 0.0;
    long long k = k0;
    for (; k + kGemvClUnroll <= k1; k += kGemvClUnroll) {
      double pv[kGemvClUnroll], cv[kGemvClUnroll];
#pragma unroll
      for (int e = 0; e < kGemvClUnroll; e++) {
        pv[e] = p[(k + e) * ldp];
        cv[e] = coef[k + e];
      }
#pragma unroll
      for (int e = 0; e < kGemvClUnroll; e++) acc = fma(pv[e], cv[e], acc);
    }
    // the last partial group: all its loads in flight, but only the products that
    // exist (the FP64 pipe, not the loads, bounds this phase)
    const int rem = (int)(k1 - k);
    if (rem > 0) {
      double pv[kGemvClUnroll], cv[kGemvClUnroll];
#pragma unroll
      for (int e = 0; e < kGemvClUnroll; e++) {
        const bool ok = e < rem;
        pv[e] = ok ? p[(k + e) * ldp] : 0.0;
        cv[e] = ok ? coef[k + e] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < kGemvClUnroll; e++) {
        if (e >= rem) break;
        acc = fma(pv[e], cv[e], acc);
      }
    }
    cl_part[i] = acc;
  }
  cluster_arrive();
  cluster_wait();
  double q[4] = {0, 0, 0, 0};
  for (int i = r0 + tid; i < r1; i += kGemvClThreads) {
    const unsigned loc = smem_u32(cl_part + i);
    double pv[kGemvClMax];
#pragma unroll
    for (int e = 0; e < kGemvClMax; e++) pv[e] = e < C ? ld_dsmem(cluster_addr(loc, e)) : 0.0;
    double sum = 0.0;
#pragma unroll
    for (int e = 0; e < kGemvClMax; e++)
      if (e < C) sum += pv[e];
    const bool first = i == r0 + tid;
    double ai = 0.0, bi_ = 0.0;
    if (a) ai = first ? fa : a[i];
    if (b) bi_ = first ? fb : b[i];
    double lin = 0.0;
    if (a) lin = ca * ai;
    if (b) lin = a ? lin + cb * bi_ : cb * bi_;
    const double o = (a || b) ? lin + cs * sum : cs * sum;
    out[i] = o;
    if (which == 1) {
      const double yi = first ? fy : yv[i], bi = first ? fbv : bv[i];
      q[0] += o * o;
      q[1] += yi * yi;
      q[2] += (yi - o) * (yi - o);
      q[3] += bi * yi;
    } else if (which == 2) {
      const double yi = first ? fy : yv[i], bi = first ? fbv : bv[i], gi = first ? fg : gv[i];
      q[0] += gi * o;
      q[1] += yi * o;
      q[2] += o * o;
      q[3] += bi * o;
    }
  }
  if (which != 0) {
    // only the warps that hold rows of this CTA contribute
    const int rows = r1 - r0;
    int nw = (min(rows, kGemvClThreads) + 31) / 32;
    if (nw < 1) nw = 1;
    const double tot = block_sum_k<4>(q, red, nw);
    if (tid < 4) st_dsmem(cluster_addr(smem_u32(&scal[c][tid]), 0), tot);
  }
  // every CTA is done with the others' shared memory: none may leave before
  cluster_arrive();
  cluster_wait();
  if (which != 0 && c == 0 && tid < 4) {
    double tot = 0.0;
    for (int e = 0; e < C; e++) tot += scal[e][tid];
    const int k = tid;
    double* dst = which == 1 ? (k == 0 ? &stw->g2 : k == 1 ? &stw->y2 : k == 2 ? &stw->yg2 : &stw->by)
                             : (k == 0 ? &stw->gd : k == 1 ? &stw->yd : k == 2 ? &stw->dd : &stw->bd);
    *dst = tot;
  }
}

// out_k = ch*h_k + cq*q_k + cd*dot(P[:, k], v), one warp per column.
__global__ void k_gemv_t(const double* __restrict__ P, long long ldp, int m, long long r, const double* __restrict__ v,
                         double* __restrict__ out, const double* __restrict__ h, double ch,
                         const double* __restrict__ q, double cq, double cd) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long tw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = gw; k < r; k += tw) {
    const double* col = P + k * ldp;
    double acc = 0.0;
    // 16 rows per lane in flight; the padding terms add 0 * 0
    for (int i0 = 0; i0 < m; i0 += 32 * 16) {
      double pv[16], vv[16];
#pragma unroll
      for (int e = 0; e < 16; e++) {
        const int i = i0 + lane + 32 * e;
        pv[e] = i < m ? col[i] : 0.0;
        vv[e] = i < m ? v[i] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < 16; e++) acc = fma(pv[e], vv[e], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      double o = cd * acc;
      if (h) o = ch * h[k] + o;
      if (q) o = cq * q[k] + o;
      out[k] = o;
    }
  }
}

// Copies the solver state to its pinned host mirror (device-mapped) and then,
// after a system-scope fence, writes `seq` to the host flag, which the host polls.
// It waits (programmatic dependent launch) for every kernel before it.
__global__ void k_state_out(const unsigned long long* __restrict__ st, unsigned long long* host, int words,
                            unsigned* flag, unsigned seq) {
  pdl_entry();
  for (int i = threadIdx.x; i < words; i += blockDim.x) host[i] = st[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile unsigned*>(flag) = seq;
  }
}

// Start of a solve: zeroes the solver state and copies b into the context's
// copy (one launch instead of a memset and a copy-engine transfer).
__global__ void k_solve_begin(unsigned long long* __restrict__ st, int st_words, double* __restrict__ bdev,
                              const double* __restrict__ b, int m) {
  pdl_entry();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < st_words; i += nt) st[i] = 0ull;
  for (int i = tid; i < m; i += nt) bdev[i] = b[i];
}

// dst[0..n) = src[0..n) (FP64, grid-stride).
__global__ void k_copy_f64(double* __restrict__ dst, const double* __restrict__ src, long long n) {
  pdl_entry();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < n; i += nt) dst[i] = src[i];
}

// dst[0..n) = -src[0..n) (FP64, grid-stride; negation is exact).
__global__ void k_neg_f64(double* __restrict__ dst, const double* __restrict__ src, long long n) {
  pdl_entry();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < n; i += nt) dst[i] = -src[i];
}

// ---------------------------------------------------------------- launchers
void launch_solve_begin(DevState* st, double* bdev, const double* b, int m, cudaStream_t s) {
  count_launch();
  launch_k(k_solve_begin, dim3(4), dim3(256), (size_t)0, s, reinterpret_cast<unsigned long long*>(st),
           (int)(sizeof(DevState) / 8), bdev, b, m);
}

void launch_copy_f64(double* dst, const double* src, long long n, int sms, cudaStream_t s) {
  long long g = (n + 255) / 256;
  if (g > 4LL * sms) g = 4LL * sms;
  if (g < 1) g = 1;
  count_launch();
  launch_k(k_copy_f64, dim3((int)g), dim3(256), (size_t)0, s, dst, src, n);
}

void launch_neg_f64(double* dst, const double* src, long long n, int sms, cudaStream_t s) {
  long long g = (n + 255) / 256;
  if (g > 4LL * sms) g = 4LL * sms;
  if (g < 1) g = 1;
  count_launch();
  launch_k(k_neg_f64, dim3((int)g), dim3(256), (size_t)0, s, dst, src, n);
}

void launch_state_out(const DevState* st, DevState* host, unsigned* flag, unsigned seq, cudaStream_t s) {
  static_assert(sizeof(DevState) % 8 == 0, "DevState is copied in 8-byte words");
  count_launch();
  launch_k(k_state_out, dim3(1), dim3(64), (size_t)0, s, reinterpret_cast<const unsigned long long*>(st),
           reinterpret_cast<unsigned long long*>(host), (int)(sizeof(DevState) / 8), flag, seq);
}

void launch_prox_count(int mode, const double* x, double* u, const double* t, double* y, const double* d,
                       long long n, int m, ProxParams pp, int apply_update, DevState* st, long long* counts,
                       double* partials, int grid, cudaStream_t s) {
  count_launch();
  if (mode == kProxSupport)
    launch_k(k_prox_count<kProxSupport>, dim3(grid), dim3(kVecThreads), (size_t)(0), s, x, u, t, y, d, n, m, pp, 0, st, counts, partials);
  else
    launch_k(k_prox_count<kProxThreshold>, dim3(grid), dim3(kVecThreads), (size_t)(0), s, x, u, t, y, d, n, m, pp, apply_update, st, counts,
                                                               partials);
}

void launch_prox_scatter(int mode, const double* x, const double* u, long long n, ProxParams pp,
                         const long long* counts, const double* partials, DevState* st, int32_t* J, double* wJ,
                         int grid, cudaStream_t s) {
  count_launch();
  if (mode == kProxSupport)
    launch_k(k_prox_scatter<kProxSupport>, dim3(grid), dim3(kVecThreads), (size_t)(0), s, x, u, n, pp, counts,
             partials, st, J, wJ);
  else
    launch_k(k_prox_scatter<kProxThreshold>, dim3(grid), dim3(kVecThreads), (size_t)(0), s, x, u, n, pp, counts,
             partials, st, J, wJ);
}

void launch_set_x(double* x, const double* u, long long n, ProxParams pp, int sms, cudaStream_t s) {
  long long g = (n + kVecThreads - 1) / kVecThreads;
  if (g > 8LL * sms) g = 8LL * sms;
  if (g < 1) g = 1;
  count_launch();
  launch_k(k_set_x, dim3((int)g), dim3(kVecThreads), (size_t)(0), s, x, u, n, pp);
}

void launch_gather(const void* A, int dtype, long long lda, int m, const int32_t* J, const DevState* st,
                   long long r_host, long long rcap, double* P, long long ldp, float* P32, long long ldp32, int sms,
                   cudaStream_t s, const float* cmean, const float* cscale) {
  int grid = 2 * sms;
  count_launch();
  int* ovf = const_cast<int*>(&st->overflow);
  if (dtype == 0)
    launch_k(k_gather<LoadF64>, dim3(grid), dim3(256), (size_t)0, s, LoadF64{(const double*)A}, lda, m, J, st, r_host,
             rcap, P, ldp, P32, ldp32, ovf);
  else if (dtype == 1)
    launch_k(k_gather<LoadF32>, dim3(grid), dim3(256), (size_t)0, s, LoadF32{(const float*)A}, lda, m, J, st, r_host,
             rcap, P, ldp, P32, ldp32, ovf);
  else if (dtype == 2)
    launch_k(k_gather<LoadBF16>, dim3(grid), dim3(256), (size_t)0, s, LoadBF16{(const __nv_bfloat16*)A}, lda, m, J, st,
             r_host, rcap, P, ldp, P32, ldp32, ovf);
  else if (dtype == 3)
    launch_k(k_gather<LoadI8>, dim3(grid), dim3(256), (size_t)0, s, LoadI8{(const int8_t*)A, cmean, cscale}, lda, m, J,
             st, r_host, rcap, P, ldp, P32, ldp32, ovf);
  else
    launch_k(k_gather<LoadI2>, dim3(grid), dim3(256), (size_t)0, s, LoadI2{(const uint8_t*)A, cmean, cscale}, lda, m, J,
             st, r_host, rcap, P, ldp, P32, ldp32, ovf);
}

void launch_gemv_n_partial(const double* P, long long ldp, int m, const double* coef, const DevState* st,
                           long long r_host, long long rcap, double* part, cudaStream_t s) {
  dim3 grid((m + kVecThreads - 1) / kVecThreads, kGemvGroups);
  count_launch();
  launch_k(k_gemv_n_partial, dim3(grid), dim3(kVecThreads), (size_t)(0), s, P, ldp, m, coef, st, r_host, rcap, part);
}

void launch_combine(double* out, const double* a, double ca, const double* b, double cb, const double* part,
                    double cs, int m, int which, const double* y, const double* bb, const double* g, DevState* st,
                    double* scratch, cudaStream_t s) {
  int grid = (m + kVecThreads - 1) / kVecThreads;
  count_launch();
  launch_k(k_combine, dim3(grid), dim3(kVecThreads), (size_t)(0), s, out, a, ca, b, cb, part, cs, m, which, y, bb, g, st, scratch);
}

// The cluster GEMV serves panels of at most kGemvClMaxEntries entries (the
// panel capacity decides, so one context always takes the same kernel).
static bool gemv_cluster_ok(int m, long long rcap) {
  return m <= kGemvClMaxRows && (long long)m * rcap <= kGemvClMaxEntries;
}

// Cluster size for k_gemv_cl: 16 CTAs where the device allows a cluster that
// large, else 8; 0 if neither can be resident.  Decided once per process.
static int gemv_cluster_size() {
  static int C = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    C = 0;
    if (cudaFuncSetAttribute(k_gemv_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * kGemvClMaxRows)) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    if (cudaFuncSetAttribute(k_gemv_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      cudaGetLastError();
    for (int cand : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cand);
      cfg.blockDim = dim3(kGemvClThreads);
      cfg.dynamicSmemBytes = sizeof(double) * kGemvClMaxRows;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cand;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_gemv_cl, &cfg) == cudaSuccess && nclusters > 0) {
        C = cand;
        return;
      }
      cudaGetLastError();
    }
  });
  return C;
}

void launch_gemv_n(const double* P, long long ldp, int m, const double* coef, const DevState* st, long long r_host,
                   long long rcap, double* out, const double* a, double ca, const double* b, double cb, double cs,
                   int which, const double* yv, const double* bv, const double* gv, DevState* stw, double* scratch,
                   double* cpart, unsigned* tile_ctr, cudaStream_t s) {
  count_launch();
  if (gemv_cluster_ok(m, rcap)) {
    const int C = gemv_cluster_size();
    if (C > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(kGemvClThreads);
      cfg.dynamicSmemBytes = sizeof(double) * (size_t)m;
      cfg.stream = s;
      cudaLaunchAttribute at[2];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 2;
      if (cudaLaunchKernelEx(&cfg, k_gemv_cl, P, ldp, m, coef, st, r_host, rcap, out, a, ca, b, cb, cs, which, yv, bv,
                             gv, stw) == cudaSuccess)
        return;
      cudaGetLastError();
    }
  }
  // a fixed launch shape; the kernel derives its column chunks from r alone
  const long long split = kGemvMaxSplit;
  dim3 grid((m + 31) / 32, (unsigned)split);
  launch_k(k_gemv_n, dim3(grid), dim3(256), (size_t)(0), s, P, ldp, m, coef, st, r_host, rcap, out, a, ca, b, cb, cs, which, yv, bv, gv, stw,
                                scratch, cpart, tile_ctr);
}

void launch_gemv_t(const double* P, long long ldp, int m, long long r, const double* v, double* out, const double* h,
                   double ch, const double* q, double cq, double cd, int sms, cudaStream_t s) {
  if (r <= 0) return;
  long long warps = r;
  long long blocks = (warps * 32 + 255) / 256;
  if (blocks > 4LL * sms) blocks = 4LL * sms;
  count_launch();
  launch_k(k_gemv_t, dim3((int)blocks), dim3(256), (size_t)(0), s, P, ldp, m, r, v, out, h, ch, q, cq, cd);
}

}  // namespace ssnal
