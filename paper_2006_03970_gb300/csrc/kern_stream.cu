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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/ssnal_en.h"
#include "lane_common.cuh"

namespace ssnal {

constexpr int kStreamThreads = 256;

int stream_grid(int sms) { return 4 * sms; }


template <int MODE>
__global__ void __launch_bounds__(kStreamThreads) k_stream_f64(const double* __restrict__ A, long long lda, int m,
                                                               long long n, const double* __restrict__ vec,
                                                               double* __restrict__ out,
                                                               const double* __restrict__ x,
                                                               const double* __restrict__ u, LsParams lp,
                                                               DevState* st, double* __restrict__ partials) {
  pdl_entry();
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
  {
    const double s = rows_sum32(partials, (int)gridDim.x, &wred[0][0]);
    if (warp == 0 && lane < lp.fused) st->lsdiff[lane] = s;
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
  pdl_entry();
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
    st->lsdiff[lp.fused + q] = ordered_sum_cg(partials + q, kMaxLS, (int)gridDim.x);
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


// ---------------------------------------------------------------------------
// Float-float stream: FP64-stored A, dot products evaluated on the FP32 pipe.
//
// GB300 retires about 2 FP64 FMAs per clock per SM, too few for one FMA per
// 8-byte element at HBM speed.  Each FP64 entry a is split exactly into
// a_hi + a_lo (24 + 23 significant bits, integer bit operations only), the
// vector entry d into a float-float pair, and each product a*d is formed as a
// float-float (error-free product via FMA plus the cross terms) and added into
// a float-float accumulator with Knuth's TwoSum.  The result is accurate to
// about 2^-47 relative per product, the same order as FP64 accumulation.
//
// Staging: a persistent CTA per SM; one producer warp moves tiles of whole
// columns (row chunks for tall columns) into a 4-stage shared-memory ring with
// cp.async.bulk, completing on mbarriers; 8 consumer warps each own whole
// columns of a tile.  Per-column epilogues are batched 32 columns at a time so
// that the FP64 work (v = x - sigma u, trial sums) runs with full warps.
// Every mbarrier wait is bounded; a timeout raises DevState::timeout.
// ---------------------------------------------------------------------------
constexpr int kFFConsumers = 8;
constexpr int kFFThreads = (kFFConsumers + 1) * 32;
constexpr int kFFStages = 4;
constexpr int kFFStageBytes = 40 * 1024;

struct FFCfg {
  int cpw;          // columns per consumer warp in a tile
  int tc;           // columns per tile (kFFConsumers * cpw)
  int rows;         // rows per chunk (even)
  int nchunks;      // chunks per tile
  int mm;           // m rounded up to even: rows actually streamed
  long long ntiles;
};

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Exact split of an FP64 value (0 or |a| in [2^-100, 2^100]) into float hi + lo
// with 24 + 23 significant bits, using integer operations only.
__device__ __forceinline__ void split_f64(unsigned long long bits, float& hi, float& lo) {
  const unsigned H = (unsigned)(bits >> 32), L = (unsigned)bits;
  const unsigned sign = H & 0x80000000u;
  const unsigned habs = H & 0x7FFFFFFFu;
  const unsigned e = habs - (896u << 20);                 // exponent bias 1023 -> 127
  const unsigned hib = __funnelshift_l(L, e, 3) | sign;  // sign | exp | top 23 mantissa bits
  const unsigned ebits = (hib & 0x7F800000u) - (23u << 23);
  const unsigned fbits = ebits | ((L >> 6) & 0x7FFFFFu) | sign;
  const unsigned mbits = ebits | sign;
  const bool zero = habs < (1u << 20);
  hi = zero ? 0.0f : __uint_as_float(hib);
  lo = zero ? 0.0f : __fsub_rn(__uint_as_float(fbits), __uint_as_float(mbits));
}

// (S, L) += (ah + al) * (dh + dl) in float-float.
__device__ __forceinline__ void ff_madd(float& S, float& L, float ah, float al, float dh, float dl) {
  const float p = __fmul_rn(ah, dh);
  float e = __fmaf_rn(ah, dh, -p);
  e = __fmaf_rn(ah, dl, e);
  e = __fmaf_rn(al, dh, e);
  const float s = __fadd_rn(S, p);
  const float z = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(p, z));
  S = s;
  L = __fadd_rn(L, __fadd_rn(t, e));
}



template <int MODE, bool PRESPLIT>
__global__ void __launch_bounds__(kFFThreads, 1) k_stream_ff(const double* __restrict__ A, long long lda, int m,
                                                             long long n, const double* __restrict__ vec,
                                                             double* __restrict__ out, const double* __restrict__ x,
                                                             const double* __restrict__ u, LsParams lp, DevState* st,
                                                             double* __restrict__ partials, FFCfg cfg) {
  pdl_entry();
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem;
  float2* d2 = reinterpret_cast<float2*>(smem + (size_t)kFFStages * kFFStageBytes);
  const int mpad = (m + 63) & ~63;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(smem + (size_t)kFFStages * kFFStageBytes + (size_t)mpad * 12);
  __shared__ double wred[kFFConsumers + 1][32];
  __shared__ double red[32];
  __shared__ unsigned long long dmax_bits;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + kFFStages);

  // ---- prologue: barriers, and the vector scaled by a power of two and split
  if (tid == 0) {
    for (int s = 0; s < kFFStages; s++) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, kFFConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dmax_bits = 0ull;
  }
  __syncthreads();
  unsigned long long mb = 0ull;
  for (int i = tid; i < m; i += blockDim.x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(vec[i]) & 0x7FFFFFFFFFFFFFFFull;
    mb = b > mb ? b : mb;
  }
  atomicMax(&dmax_bits, mb);
  __syncthreads();
  int ex = (int)((dmax_bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) ex = 1023;  // zero vector (or non-finite): no scaling
  const double scale = __longlong_as_double((long long)(2046 - ex) << 52);    // 2^(1023-ex)
  const double unscale = __longlong_as_double((long long)ex << 52);           // 2^(ex-1023)
  // PRESPLIT layout per row pair k: D4[k] = (dh0, dh1, -dh0, -dh1), DL[k] = (-dl0, -dl1)
  float4* D4 = reinterpret_cast<float4*>(d2);
  float2* DL = reinterpret_cast<float2*>(D4 + mpad / 2);
  if (PRESPLIT) {
    for (int k = tid; k < mpad / 2; k += blockDim.x) {
      float h[2] = {0.0f, 0.0f}, l[2] = {0.0f, 0.0f};
      for (int q = 0; q < 2; q++) {
        const int i = 2 * k + q;
        if (i < m) {
          const double v = vec[i] * scale;
          h[q] = __double2float_rn(v);
          l[q] = __double2float_rn(v - (double)h[q]);
        }
      }
      D4[k] = make_float4(h[0], h[1], -h[0], -h[1]);
      DL[k] = make_float2(-l[0], -l[1]);
    }
  } else {
    for (int i = tid; i < mpad; i += blockDim.x) {
      float hi = 0.0f, lo = 0.0f;
      if (i < m) {
        const double v = vec[i] * scale;
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
      }
      d2[i] = make_float2(hi, lo);
    }
  }
  __syncthreads();

  bool timed_out = false;
  if (warp == kFFConsumers) {
    // ---- producer: one elected lane issues the bulk copies
    if (lane == 0) {
      unsigned it = 0;
      for (long long tile = blockIdx.x; tile < cfg.ntiles && !timed_out; tile += gridDim.x) {
        const long long c0 = tile * cfg.tc;
        const int ncol = (int)((n - c0) < cfg.tc ? (n - c0) : cfg.tc);
        for (int ch = 0; ch < cfg.nchunks; ch++, it++) {
          const int r0 = ch * cfg.rows;
          const int nr = (cfg.mm - r0) < cfg.rows ? (cfg.mm - r0) : cfg.rows;
          const int s = it % kFFStages;
          const unsigned ph = (it / kFFStages) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
            timed_out = true;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, (unsigned)(ncol * nr * 8));
          const unsigned dst = smem_u32(stages + (size_t)s * kFFStageBytes);
          for (int c = 0; c < ncol; c++)
            bulk_g2s(dst + (unsigned)(c * nr * 8), A + (c0 + c) * lda + r0, (unsigned)(nr * 8), full0 + 8 * s);
        }
      }
      if (timed_out) {
        st->timeout = 1;
        // let the copies already issued land before the block can exit
        const unsigned issued = it;
        for (unsigned k = issued > (unsigned)kFFStages ? issued - kFFStages : 0; k < issued; k++)
          mbar_wait(full0 + 8 * (k % kFFStages), (k / kFFStages) & 1u);
      }
    }
  } else {
    // ---- consumers
    float S[8], Lr[8];
    double cand = 0.0, amax = 0.0;
    double s_lane = 1.0;
    if (MODE == kModeT)
      for (int k = 0; k < lane; k++) s_lane *= lp.beta;
    long long ej = -1;
    float es = 0.0f, el = 0.0f;
    int nb = 0;
    auto flush = [&](int cnt) {
      const bool mine = lane < cnt;
      const double et = ((double)es + (double)el) * unscale;
      if (mine) out[ej] = et;
      if (MODE == kModeGmax && mine) amax = fmax(amax, fabs(et));
      if (MODE == kModeT) {
        double v = 0.0;
        bool live = false;
        if (mine) {
          v = v_of(x[ej], u[ej], lp.pp.sigma);
          live = !trial_skip(v, et, lp.pp);
        }
        unsigned mask = __ballot_sync(0xffffffffu, live);
        while (mask) {
          const int q = __ffs(mask) - 1;
          mask &= mask - 1;
          const double bv = __shfl_sync(0xffffffffu, v, q);
          const double bt = __shfl_sync(0xffffffffu, et, q);
          if (lane < lp.fused) cand += trial_term(bv, bt, s_lane, lp.pp);
        }
      }
    };
    unsigned it = 0;
    for (long long tile = blockIdx.x; tile < cfg.ntiles && !timed_out; tile += gridDim.x) {
      const long long c0 = tile * cfg.tc;
      const int ncol = (int)((n - c0) < cfg.tc ? (n - c0) : cfg.tc);
#pragma unroll
      for (int q = 0; q < 8; q++) S[q] = Lr[q] = 0.0f;
      for (int ch = 0; ch < cfg.nchunks; ch++, it++) {
        const int r0 = ch * cfg.rows;
        const int nr = (cfg.mm - r0) < cfg.rows ? (cfg.mm - r0) : cfg.rows;
        const int s = it % kFFStages;
        if (!mbar_wait(full0 + 8 * s, (it / kFFStages) & 1u)) {
          timed_out = true;
          break;
        }
        const unsigned char* stg = stages + (size_t)s * kFFStageBytes;
        const float4* dq = reinterpret_cast<const float4*>(d2 + r0);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int c = warp * cfg.cpw + q;
          if (q < cfg.cpw && c < ncol) {
            const ulonglong2* col = reinterpret_cast<const ulonglong2*>(stg + (size_t)c * nr * 8);
            float s0 = 0.0f, l0 = 0.0f, s1 = 0.0f, l1 = 0.0f;
            if (PRESPLIT) {
              // pairs of rows: col[k] = (ah0, ah1 | al0, al1)
              const ulonglong2* D4p = reinterpret_cast<const ulonglong2*>(D4 + r0 / 2);
              const unsigned long long* DLp = reinterpret_cast<const unsigned long long*>(DL + r0 / 2);
              unsigned long long Sa = 0ull, La = 0ull, Sb = 0ull, Lb = 0ull;
              int k = lane;
              for (; k + 32 < nr / 2; k += 64) {
                const ulonglong2 a0 = col[k], a1 = col[k + 32];
                const ulonglong2 d0 = D4p[k], d1 = D4p[k + 32];
                const unsigned long long n0 = DLp[k], n1 = DLp[k + 32];
                ff2_madd(Sa, La, a0.x, a0.y, d0.x, d0.y, n0);
                ff2_madd(Sb, Lb, a1.x, a1.y, d1.x, d1.y, n1);
              }
              if (k < nr / 2) {
                const ulonglong2 a0 = col[k];
                const ulonglong2 d0 = D4p[k];
                ff2_madd(Sa, La, a0.x, a0.y, d0.x, d0.y, DLp[k]);
              }
              s0 = lo32f(Sa);
              l0 = lo32f(La);
              ff_merge(s0, l0, hi32f(Sa), hi32f(La));
              s1 = lo32f(Sb);
              l1 = lo32f(Lb);
              ff_merge(s1, l1, hi32f(Sb), hi32f(Lb));
            } else {
#pragma unroll 2
              for (int i = lane; 2 * i < nr; i += 32) {
                ulonglong2 a = col[i];
                const float4 dd = dq[i];
                if (r0 + 2 * i + 1 >= m) a.y = 0ull;
                float ah, al, bh, bl;
                split_f64(a.x, ah, al);
                split_f64(a.y, bh, bl);
                ff_madd(s0, l0, ah, al, dd.x, dd.y);
                ff_madd(s1, l1, bh, bl, dd.z, dd.w);
              }
            }
            ff_merge(s0, l0, s1, l1);
            ff_merge(S[q], Lr[q], s0, l0);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * s);
      }
      if (timed_out) break;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int c = warp * cfg.cpw + q;
        if (q < cfg.cpw && c < ncol) {
          float Sq = S[q], Lq = Lr[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float So = __shfl_xor_sync(0xffffffffu, Sq, o);
            const float Lo = __shfl_xor_sync(0xffffffffu, Lq, o);
            ff_merge(Sq, Lq, So, Lo);
          }
          if (lane == (nb & 31)) {
            ej = c0 + c;
            es = Sq;
            el = Lq;
          }
          nb++;
          if ((nb & 31) == 0) flush(32);
        }
      }
    }
    if (!timed_out && (nb & 31)) flush(nb & 31);
    if (timed_out) st->timeout = 1;
    if (MODE == kModeT) wred[warp][lane] = cand;
    if (MODE == kModeGmax) wred[warp][lane] = amax;
  }
  if (warp == kFFConsumers) wred[warp][lane] = 0.0;
  __syncthreads();
  if (MODE == kModeU) return;
  if (MODE == kModeGmax) {
    double mx = 0.0;
    if (warp == 0)
      for (int w = 0; w < kFFConsumers; w++) mx = fmax(mx, wred[w][lane]);
    mx = block_max(warp == 0 ? mx : 0.0, red);
    if (tid == 0) partials[blockIdx.x] = mx;
    if (!last_block(&st->counters[kCtrGmax])) return;
    double g = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += blockDim.x) g = fmax(g, ld_cg(&partials[b]));
    g = block_max(g, red);
    if (tid == 0) st->gmax = g;
    reset_counter(&st->counters[kCtrGmax]);
    return;
  }
  // kModeT: per-block trial sums in a fixed order, then the selection
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < kFFConsumers; w++) s += wred[w][lane];
    partials[(long long)blockIdx.x * 32 + lane] = s;
  }
  if (!last_block(&st->counters[kCtrStream])) return;
  {
    const double s = rows_sum32(partials, (int)gridDim.x, &wred[0][0]);
    if (warp == 0 && lane < lp.fused) st->lsdiff[lane] = s;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence_block();
    double s;
    int k = armijo_select(st, lp, 0, lp.fused, s);
    if (k >= 0) {
      st->s = s;
      st->ls_k = k;
      st->ls_state = 0;
    } else if (lp.fused < lp.max_ls) {
      st->ls_state = 1;
    } else {
      st->s = s;
      st->ls_k = lp.max_ls - 1;
      st->ls_state = 0;
    }
  }
  reset_counter(&st->counters[kCtrStream]);
}

static FFCfg ff_config(int m, long long n) {
  FFCfg c;
  c.mm = (m + 1) & ~1;
  const long long colb = (long long)c.mm * 8;
  if ((long long)kFFConsumers * colb <= kFFStageBytes) {
    c.rows = c.mm;
    c.nchunks = 1;
    long long cpw = kFFStageBytes / (kFFConsumers * colb);
    c.cpw = (int)(cpw > 8 ? 8 : (cpw < 1 ? 1 : cpw));
  } else {
    c.cpw = 1;
    c.rows = (kFFStageBytes / (kFFConsumers * 8)) / 64 * 64;
    c.nchunks = (c.mm + c.rows - 1) / c.rows;
  }
  c.tc = kFFConsumers * c.cpw;
  c.ntiles = (n + c.tc - 1) / c.tc;
  return c;
}

static size_t ff_smem(int m) {
  return (size_t)kFFStages * kFFStageBytes + (size_t)((m + 63) & ~63) * 12 + 2 * kFFStages * 8;
}

template <int MODE, bool PRESPLIT>
static void launch_ff(const double* A, long long lda, int m, long long n, const double* vec, double* out,
                      const double* x, const double* u, LsParams lp, DevState* st, double* partials, int sms,
                      cudaStream_t s) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_stream_ff<MODE, PRESPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ff_smem(kMaxM));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  FFCfg cfg = ff_config(m, n);
  long long grid = cfg.ntiles < sms ? cfg.ntiles : sms;
  if (grid < 1) grid = 1;
  launch_k(k_stream_ff<MODE, PRESPLIT>, dim3((int)grid), dim3(kFFThreads), (size_t)(ff_smem(m)), s, A, lda, m, n, vec,
           out, x, u, lp, st, partials, cfg);
}

// One-time conversion of FP64 A into the float-float pair layout read by the
// PRESPLIT stream: per column, row pair k is (hi(2k), hi(2k+1), lo(2k), lo(2k+1))
// as four floats; rows >= m are zero.  Column stride: mm = m rounded up to even.
__global__ void k_presplit(const double* __restrict__ A, long long lda, int m, long long n, float4* __restrict__ S) {
  pdl_entry();
  const int pairs = (m + 1) / 2;
  const long long total = (long long)pairs * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / pairs;
    const int k = (int)(e % pairs);
    const double* col = A + j * lda;
    float h0, l0, h1 = 0.0f, l1 = 0.0f;
    split_f64((unsigned long long)__double_as_longlong(col[2 * k]), h0, l0);
    if (2 * k + 1 < m) split_f64((unsigned long long)__double_as_longlong(col[2 * k + 1]), h1, l1);
    S[e] = make_float4(h0, h1, l0, l1);
  }
}

void launch_presplit(const double* A, long long lda, int m, long long n, void* S, int sms, cudaStream_t s) {
  count_launch();
  launch_k(k_presplit, dim3(8 * sms), dim3(256), (size_t)(0), s, A, lda, m, n, reinterpret_cast<float4*>(S));
}

// ---------------------------------------------------------------------------
// Lane-per-column stream over the pre-split float-pair copy of A.
//
// Each warp owns groups of 32 consecutive columns; lane l accumulates column
// (32 g + l) over all rows, so no cross-lane reduction is needed and the
// per-column epilogue runs on full warps.  Each warp streams its groups through
// its own ring of shared-memory stages filled by 2-D TMA tensor copies
// (cp.async.bulk.tensor.2d, box = 16 rows x 32 columns = 4 KB, zero fill past
// the last row and column).  Lanes read the 8 row pairs of a stage in a
// staggered order, which keeps the 16-byte shared loads conflict-free.
// ---------------------------------------------------------------------------


template <int MODE, int ELT>
__global__ void __launch_bounds__(kLThreads, 1) k_stream_lane(const __grid_constant__ CUtensorMap tmap, int m, long long n,
                                                              const double* __restrict__ vec, double* __restrict__ out,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ u, LsParams lp, DevState* st,
                                                              double* __restrict__ partials, LaneCfg cfg,
                                                              const float* __restrict__ cmean,
                                                              const float* __restrict__ cscale) {
  // A is never written while a solve runs: the first copies of every warp's ring
  // are issued before waiting for the preceding kernel (programmatic dependent
  // launch); the vectors are read only after the wait.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(1024) unsigned char smem_lane[];
  constexpr int R = elt_rows(ELT);   // rows per box
  constexpr int P = R / 16;          // row pairs per 16-byte chunk of a column
  const int mpad = lane_mpad(m, ELT);
  unsigned char* ring = smem_lane;  // [kLWarps][stages][kLBoxBytes]
  float4* D4 = reinterpret_cast<float4*>(smem_lane + (size_t)kLWarps * cfg.stages * kLBoxBytes);
  float2* DL = reinterpret_cast<float2*>(D4 + mpad / 2);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(DL + mpad / 2);
  __shared__ double wred[kLWarps][32];
  __shared__ double red[32];
  __shared__ unsigned long long dmax_bits;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int b = 0; b < kLWarps * cfg.stages; b++) mbar_init(smem_u32(bars + b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    dmax_bits = 0ull;
  }
  __syncthreads();
  // ---- work split: the CTA owns column groups g = blockIdx.x + q * gridDim.x;
  // warp w streams row chunks w, w + 8, ... of each group through its own ring.
  // Per group, the warps' per-column partials are merged in shared memory.
  __shared__ float2 part[2][kLWarps][kLCols];
  const long long ngrp = (long long)blockIdx.x < cfg.groups ? (cfg.groups - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int nw = warp < cfg.chunks ? (cfg.chunks - warp + kLWarps - 1) / kLWarps : 0;  // chunks per group
  const long long total = ngrp * nw;
  unsigned char* wring = ring + (size_t)warp * cfg.stages * kLBoxBytes;
  unsigned long long* wbars = bars + warp * cfg.stages;
  // item i = q nw + k of this warp: chunk warp + 8 k of group blockIdx.x + q gridDim.x, ring
  // slot i mod stages.  Lane 0 issues the items in order.  The float-float passes
  // (bound by the FP32 pipe) keep the issue position and the consumer's slot and phase
  // by increments, no 64-bit division per box: 433 against 480 us per u = A^T y pass at
  // m = 1000, n = 1e6 (BF16).  The FP32-accumulation passes (memory-bound, a few
  // instructions per box) derive them from the item index: measured 322 against 332 us
  // per t = A^T d pass on the same matrix with the increments (the cause is not
  // established; both forms give the same slots).
  auto issue_item = [&](long long item) {
    const long long q = item / nw;
    const int ch = warp + kLWarps * (int)(item % nw);
    const int sx = (int)(item % cfg.stages);
    const unsigned bar = smem_u32(wbars + sx);
    mbar_expect_tx(bar, kLBoxBytes);
    tma_load_2d(smem_u32(wring + (size_t)sx * kLBoxBytes), &tmap, ch * elt_box_inner(ELT),
                (int)(((long long)blockIdx.x + q * gridDim.x) * kLCols), bar);
  };
  long long iq = 0;
  int ik = 0, islot = 0;
  auto issue_next = [&]() {
    const int ch = warp + kLWarps * ik;
    const unsigned bar = smem_u32(wbars + islot);
    mbar_expect_tx(bar, kLBoxBytes);
    tma_load_2d(smem_u32(wring + (size_t)islot * kLBoxBytes), &tmap, ch * elt_box_inner(ELT),
                (int)(((long long)blockIdx.x + iq * gridDim.x) * kLCols), bar);
    if (++ik == nw) {
      ik = 0;
      iq++;
    }
    if (++islot == cfg.stages) islot = 0;
  };
  if (lane == 0)
    for (long long it = 0; it < total && it < cfg.stages; it++) issue_next();
  __syncwarp();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the vector, scaled by a power of two and split: row pair k goes to slot pair_slot<P>(k),
  // D4 = (dh0, dh1, -dh0, -dh1), DL = (-dl0, -dl1)
  unsigned long long mb = 0ull;
  for (int i = tid; i < m; i += blockDim.x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(vec[i]) & 0x7FFFFFFFFFFFFFFFull;
    mb = b > mb ? b : mb;
  }
  atomicMax(&dmax_bits, mb);
  __syncthreads();
  int ex = (int)((dmax_bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) ex = 1023;
  const double scale = __longlong_as_double((long long)(2046 - ex) << 52);
  const double unscale = __longlong_as_double((long long)ex << 52);
  for (int k = tid; k < mpad / 2; k += blockDim.x) {
    float h[2] = {0.0f, 0.0f}, l[2] = {0.0f, 0.0f};
    for (int q = 0; q < 2; q++) {
      const int i = 2 * k + q;
      if (i < m) {
        const double v = vec[i] * scale;
        h[q] = __double2float_rn(v);
        l[q] = __double2float_rn(v - (double)h[q]);
      }
    }
    const int slot = pair_slot<P>(k);
    D4[slot] = make_float4(h[0], h[1], -h[0], -h[1]);
    DL[slot] = make_float2(-l[0], -l[1]);
  }
  __syncthreads();

  double ysum = 0.0;  // sum_i vec_i (genotype mean correction)
  if constexpr (elt_geno(ELT)) {
    double a = 0.0;
    for (int i = tid; i < m; i += blockDim.x) a += vec[i];
    ysum = block_sum(a, red);
  }


  double s_lane = 1.0;
  if (MODE == kModeT)
    for (int k = 0; k < lane; k++) s_lane *= lp.beta;
  double cand = 0.0, amax = 0.0;
  bool timed_out = false;
  long long it = 0;
  int sidx = 0;         // ring slot of item it
  unsigned rphase = 0;  // phase parity of that slot's barrier for item it
  for (long long q = 0; q < ngrp; q++) {
    // float-float: four accumulator pairs per column (row pair index mod 4) for four
    // independent dependency chains; FP32: one FMA chain per column
    unsigned long long S2 = 0ull, S2b = 0ull;
    unsigned long long FS[4] = {0ull, 0ull, 0ull, 0ull}, FL[4] = {0ull, 0ull, 0ull, 0ull};
    unsigned long long FSb[4] = {0ull, 0ull, 0ull, 0ull}, FLb[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k = 0; k < nw && !timed_out; k++, it++) {
      if constexpr (!elt_ff(ELT)) {
        sidx = (int)(it % cfg.stages);
        rphase = (unsigned)((it / cfg.stages) & 1);
      }
      if (!mbar_wait(smem_u32(wbars + sidx), rphase)) {
        timed_out = true;
        break;
      }
      const int ch = warp + kLWarps * k;
      const unsigned char* colbase = wring + (size_t)sidx * kLBoxBytes + lane * 128;
      const ulonglong2* D4p = reinterpret_cast<const ulonglong2*>(D4 + ch * (R / 2));
      const unsigned long long* D4h = reinterpret_cast<const unsigned long long*>(D4 + ch * (R / 2));  // (dh0, dh1)
      const unsigned long long* DLp = reinterpret_cast<const unsigned long long*>(DL + ch * (R / 2));
#pragma unroll
      for (int p = 0; p < 8; p++) {
        const int pp = (p + lane) & 7;
        if constexpr (P == 32) {
          // 2-bit codes: 64 rows per 16-byte chunk, byte b of a word holds rows 4b .. 4b + 3
          // (bits 2q, 2q + 1 for row 4b + q).  Each word is spread into four words of one
          // code per byte (masks), each code becomes 2^23 + code in FP32 by a byte permute
          // (exact), and the bias goes with one packed subtract per row pair.
          const uint4 a = *reinterpret_cast<const uint4*>(colbase + pp * 16);
          const uint4 b = *reinterpret_cast<const uint4*>(colbase + 32 * 128 + pp * 16);
          const unsigned aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
          const unsigned long long bias = 0x4B0000004B000000ull;  // (2^23, 2^23)
#pragma unroll
          for (int q = 0; q < 4; q++) {
            unsigned ea[4], eb[4];
#pragma unroll
            for (int f = 0; f < 4; f++) {
              ea[f] = (aw[q] >> (2 * f)) & 0x03030303u;
              eb[f] = (bw[q] >> (2 * f)) & 0x03030303u;
            }
#pragma unroll
            for (int e = 0; e < 8; e++) {  // row pair 8 q + e: rows 16 q + 2 e, + 1 = 4 (e/2) + 2 (e%2) + {0, 1}
              const int byte = e >> 1, f0 = 2 * (e & 1);
              const unsigned long long av =
                  f2sub((unsigned long long)code_biased(ea[f0], byte) |
                            ((unsigned long long)code_biased(ea[f0 + 1], byte) << 32),
                        bias);
              const unsigned long long bv =
                  f2sub((unsigned long long)code_biased(eb[f0], byte) |
                            ((unsigned long long)code_biased(eb[f0 + 1], byte) << 32),
                        bias);
              const int slot = 8 * (8 * q + e) + pp;
              if constexpr (elt_ff(ELT)) {
                const ulonglong2 d = D4p[slot];
                const unsigned long long dl = DLp[slot];
                ff2_madd_exact(FS[e & 3], FL[e & 3], av, d.x, d.y, dl);
                ff2_madd_exact(FSb[e & 3], FLb[e & 3], bv, d.x, d.y, dl);
              } else {
                const unsigned long long dh = D4h[2 * slot];
                S2 = f2fma(av, dh, S2);
                S2b = f2fma(bv, dh, S2b);
              }
            }
          }
        } else if constexpr (ELT == kEltSplit) {
          const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(colbase + pp * 16);
          const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(colbase + 32 * 128 + pp * 16);
          const ulonglong2 d = D4p[pp];
          const unsigned long long dl = DLp[pp];
          ff2_madd(FS[p & 3], FL[p & 3], a.x, a.y, d.x, d.y, dl);
          ff2_madd(FSb[p & 3], FLb[p & 3], b.x, b.y, d.x, d.y, dl);
        } else {
          const uint4 a = *reinterpret_cast<const uint4*>(colbase + pp * 16);
          const uint4 b = *reinterpret_cast<const uint4*>(colbase + 32 * 128 + pp * 16);
          unsigned long long ap[P], bp[P];
          if constexpr (P == 4) {  // 8 BF16 rows
            ap[0] = bf16x2_to_f32x2(a.x); ap[1] = bf16x2_to_f32x2(a.y);
            ap[2] = bf16x2_to_f32x2(a.z); ap[3] = bf16x2_to_f32x2(a.w);
            bp[0] = bf16x2_to_f32x2(b.x); bp[1] = bf16x2_to_f32x2(b.y);
            bp[2] = bf16x2_to_f32x2(b.z); bp[3] = bf16x2_to_f32x2(b.w);
          } else if constexpr (P == 8) {  // 16 int8 codes: exact (code + 128 + 2^23) - (2^23 + 128)
            const unsigned long long bias = 0x4B0000804B000080ull;  // (8388736.0f, 8388736.0f)
            const unsigned aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
              ap[2 * q] = f2sub(i8x2_biased(aw[q], 0), bias);
              ap[2 * q + 1] = f2sub(i8x2_biased(aw[q], 2), bias);
              bp[2 * q] = f2sub(i8x2_biased(bw[q], 0), bias);
              bp[2 * q + 1] = f2sub(i8x2_biased(bw[q], 2), bias);
            }
          } else {  // 4 FP32 rows
            ap[0] = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
            ap[1] = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
            bp[0] = (unsigned long long)b.x | ((unsigned long long)b.y << 32);
            bp[1] = (unsigned long long)b.z | ((unsigned long long)b.w << 32);
          }
#pragma unroll
          for (int e = 0; e < P; e++) {
            const int slot = 8 * e + pp;
            if constexpr (elt_ff(ELT)) {
              const ulonglong2 d = D4p[slot];
              const unsigned long long dl = DLp[slot];
              const int ch4 = (p * P + e) & 3;
              ff2_madd_exact(FS[ch4], FL[ch4], ap[e], d.x, d.y, dl);
              ff2_madd_exact(FSb[ch4], FLb[ch4], bp[e], d.x, d.y, dl);
            } else {
              const unsigned long long dh = D4h[2 * slot];
              S2 = f2fma(ap[e], dh, S2);
              S2b = f2fma(bp[e], dh, S2b);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0 && it + cfg.stages < total) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (elt_ff(ELT))
          issue_next();  // item it + stages
        else
          issue_item(it + cfg.stages);
      }
      if (++sidx == cfg.stages) {  // ring slot and phase of item it + 1
        sidx = 0;
        rphase ^= 1u;
      }
    }
    {
      float Sq, Lq, Sb, Lb;
      if constexpr (elt_ff(ELT)) {
        Sq = lo32f(FS[0]), Lq = lo32f(FL[0]);
        ff_merge(Sq, Lq, hi32f(FS[0]), hi32f(FL[0]));
        Sb = lo32f(FSb[0]), Lb = lo32f(FLb[0]);
        ff_merge(Sb, Lb, hi32f(FSb[0]), hi32f(FLb[0]));
#pragma unroll
        for (int c4 = 1; c4 < 4; c4++) {
          ff_merge(Sq, Lq, lo32f(FS[c4]), lo32f(FL[c4]));
          ff_merge(Sq, Lq, hi32f(FS[c4]), hi32f(FL[c4]));
          ff_merge(Sb, Lb, lo32f(FSb[c4]), lo32f(FLb[c4]));
          ff_merge(Sb, Lb, hi32f(FSb[c4]), hi32f(FLb[c4]));
        }
      } else {
        Sq = lo32f(S2), Lq = 0.0f;
        ff_merge(Sq, Lq, hi32f(S2), 0.0f);
        Sb = lo32f(S2b), Lb = 0.0f;
        ff_merge(Sb, Lb, hi32f(S2b), 0.0f);
      }
      part[q & 1][warp][lane] = make_float2(Sq, Lq);
      part[q & 1][warp][lane + 32] = make_float2(Sb, Lb);
    }
    __syncthreads();
    if (warp < 2) {
      // warps 0 and 1 merge the partials of columns lane and lane + 32 in a fixed
      // order, then run the column epilogue
      const int cc = lane + 32 * warp;
      float Sm = part[q & 1][0][cc].x, Lm = part[q & 1][0][cc].y;
      for (int w = 1; w < kLWarps; w++) ff_merge(Sm, Lm, part[q & 1][w][cc].x, part[q & 1][w][cc].y);
      const long long j = ((long long)blockIdx.x + q * gridDim.x) * kLCols + cc;
      const bool mine = j < n;
      double t = ((double)Sm + (double)Lm) * unscale;
      if constexpr (elt_geno(ELT)) {
        if (mine) t = (double)cscale[j] * (t - (double)cmean[j] * ysum);
      }
      if (mine) out[j] = t;
      if (MODE == kModeGmax && mine) amax = fmax(amax, fabs(t));
      if (MODE == kModeT) {
        double v = 0.0;
        bool live = false;
        if (mine) {
          v = v_of(x[j], u[j], lp.pp.sigma);
          live = !trial_skip(v, t, lp.pp);
        }
        unsigned mask = __ballot_sync(0xffffffffu, live);
        while (mask) {
          const int qq = __ffs(mask) - 1;
          mask &= mask - 1;
          const double bv = __shfl_sync(0xffffffffu, v, qq);
          const double bt = __shfl_sync(0xffffffffu, t, qq);
          if (lane < lp.fused) cand += trial_term(bv, bt, s_lane, lp.pp);
        }
      }
    }
  }
  if (timed_out) {
    st->timeout = 1;
    if (lane == 0)  // let this warp's copies in flight land before the block exits
      for (long long k = it; k < total && k < it + cfg.stages; k++)
        mbar_wait(smem_u32(wbars + (int)(k % cfg.stages)), (unsigned)((k / cfg.stages) & 1));
    __syncwarp();
  }
  wred[warp][lane] = (MODE == kModeGmax) ? amax : cand;
  __syncthreads();
  if (MODE == kModeU) return;
  if (MODE == kModeGmax) {
    double mx = 0.0;
    if (warp == 0)
      for (int w = 0; w < kLWarps; w++) mx = fmax(mx, wred[w][lane]);
    mx = block_max(warp == 0 ? mx : 0.0, red);
    if (tid == 0) partials[blockIdx.x] = mx;
    if (!last_block(&st->counters[kCtrGmax])) return;
    double g = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += blockDim.x) g = fmax(g, ld_cg(&partials[b]));
    g = block_max(g, red);
    if (tid == 0) st->gmax = g;
    reset_counter(&st->counters[kCtrGmax]);
    return;
  }
  if (warp == 0) {
    double sum = 0.0;
    for (int w = 0; w < kLWarps; w++) sum += wred[w][lane];
    partials[(long long)blockIdx.x * 32 + lane] = sum;
  }
  if (!last_block(&st->counters[kCtrStream])) return;
  {
    const double sum = rows_sum32(partials, (int)gridDim.x, &wred[0][0]);
    if (warp == 0 && lane < lp.fused) st->lsdiff[lane] = sum;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence_block();
    double sel;
    int k = armijo_select(st, lp, 0, lp.fused, sel);
    if (k >= 0) {
      st->s = sel;
      st->ls_k = k;
      st->ls_state = 0;
    } else if (lp.fused < lp.max_ls) {
      st->ls_state = 1;
    } else {
      st->s = sel;
      st->ls_k = lp.max_ls - 1;
      st->ls_state = 0;
    }
  }
  reset_counter(&st->counters[kCtrStream]);
}

constexpr size_t kLDynMax = 232448 - 12288;  // per-block limit minus the kernel's static shared memory

static size_t lane_smem(int m, int stages, int elt) {
  const int mpad = lane_mpad(m, elt);
  return (size_t)kLWarps * stages * kLBoxBytes + (size_t)mpad * 12 + (size_t)kLWarps * stages * 8 + 1024;
}

static int lane_stages(int m, int elt, size_t budget = kLDynMax) {  // budget: dynamic bytes beside the static part
  const int mpad = lane_mpad(m, elt);
  int st = (int)((budget - (size_t)mpad * 12 - 1024) / ((size_t)kLWarps * kLBoxBytes + kLWarps * 8));
  if (st > 8) st = 8;
  return st;
}

// Tensor map over the pre-split copy: 2-D, inner dimension = the 2 mm floats of
// one column, outer = the n columns; boxes of 32 floats x 32 columns.
bool make_split_tensor_map(void* map_out, const void* split, int m, long long n) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const long long mm = (m + 1) & ~1;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * mm), (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)(2 * mm * sizeof(float))};
  cuuint32_t box[2] = {32, (cuuint32_t)kLCols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(split), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor map over A stored as BF16, FP32, int8 codes or 2-bit codes (column-major,
// lda elements per column, the column stride a multiple of 16 bytes): boxes of 128
// bytes of a column x 64 columns, zero fill past row m (2-bit codes: bytes, four rows
// each, zero fill past byte ceil(m / 4); the zero codes past row m meet zero entries
// of the vector).
bool make_elt_tensor_map(void* map_out, const void* A, int dtype, long long lda, int m, long long n) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const bool bf16 = dtype == SSNAL_EN_BF16, i2 = dtype == SSNAL_EN_I2_GENO;
  const bool i8 = dtype == SSNAL_EN_I8_GENO || i2;
  const size_t es = i8 ? 1 : bf16 ? 2 : 4;
  const long long ld_bytes = i2 ? lda / 4 : lda * (long long)es;  // column stride in bytes
  if ((i2 && lda % 4 != 0) || ld_bytes % 16 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(i2 ? (m + 3) / 4 : m), (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ld_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)kLCols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out),
                      i8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                         : bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(A), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor map over a Cholesky factor L (FP32, column-major, ld floats per
// column, ld * 4 a multiple of 16 bytes): N x N, 32 x 32 boxes with the 128-byte
// swizzle (16-byte chunk index XOR row index mod 8 within each 1 KB), zero fill
// past N.
bool make_factor_tensor_map(void* map_out, const float* L, long long ld, int N) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  if ((ld * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(L) & 15) != 0 || N <= 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)N};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<float*>(L), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

template <int MODE, int ELT>
static void launch_lane(const void* map, int m, long long n, const double* vec, double* out, const double* x,
                        const double* u, LsParams lp, DevState* st, double* partials, int sms, cudaStream_t s,
                        const float* cmean, const float* cscale) {
  static bool configured[64] = {};
  static size_t dyn_max = kLDynMax;  // per-block shared memory minus this instantiation's static part
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_stream_lane<MODE, ELT>) == cudaSuccess && fa.sharedSizeBytes < 232448)
      dyn_max = 232448 - fa.sharedSizeBytes;
    cudaGetLastError();
    cudaFuncSetAttribute(k_stream_lane<MODE, ELT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const int stages = lane_stages(m, ELT, dyn_max);
  LaneCfg cfg;
  cfg.stages = stages;
  cfg.chunks = ELT == kEltSplit ? (((m + 1) & ~1) + 15) / 16 : (m + elt_rows(ELT) - 1) / elt_rows(ELT);
  cfg.groups = (n + kLCols - 1) / kLCols;
  long long grid = cfg.groups;
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(map);
  launch_k(k_stream_lane<MODE, ELT>, dim3((int)grid), dim3(kLThreads), (size_t)(lane_smem(m, stages, ELT)), s, *tm, m, n, vec, out, x, u, lp, st,
                                                                              partials, cfg, cmean, cscale);
}

template <int ELT>
static void launch_lane_modes(int mode, const void* map, int m, long long n, const double* vec, double* out,
                              const double* x, const double* u, LsParams lp, DevState* st, double* partials, int sms,
                              cudaStream_t s, const float* cmean, const float* cscale) {
  if (mode == kModeU)
    launch_lane<kModeU, ELT>(map, m, n, vec, out, x, u, lp, st, partials, sms, s, cmean, cscale);
  else if (mode == kModeT)
    launch_lane<kModeT, ELT>(map, m, n, vec, out, x, u, lp, st, partials, sms, s, cmean, cscale);
  else
    launch_lane<kModeGmax, ELT>(map, m, n, vec, out, x, u, lp, st, partials, sms, s, cmean, cscale);
}

void launch_stream_lane(int mode, int elt, const void* map, int m, long long n, const double* vec, double* out,
                        const double* x, const double* u, ProxParams pp, double mu, double beta, int max_ls, int fused,
                        DevState* st, double* partials, int sms, cudaStream_t s, const float* cmean,
                        const float* cscale) {
  LsParams lp{pp, mu, beta, max_ls, fused};
  count_launch();
#define SSNAL_LANE(E) launch_lane_modes<E>(mode, map, m, n, vec, out, x, u, lp, st, partials, sms, s, cmean, cscale)
  switch (elt) {
    case kEltBf16FF: SSNAL_LANE(kEltBf16FF); break;
    case kEltBf16: SSNAL_LANE(kEltBf16); break;
    case kEltF32FF: SSNAL_LANE(kEltF32FF); break;
    case kEltF32: SSNAL_LANE(kEltF32); break;
    case kEltI8FF: SSNAL_LANE(kEltI8FF); break;
    case kEltI8: SSNAL_LANE(kEltI8); break;
    case kEltI2FF: SSNAL_LANE(kEltI2FF); break;
    case kEltI2: SSNAL_LANE(kEltI2); break;
    default: SSNAL_LANE(kEltSplit); break;
  }
#undef SSNAL_LANE
}

void launch_stream(int mode, int dtype, const void* A, long long lda, int m, long long n, const double* vec,
                   double* out, const double* x, const double* u, ProxParams pp, double mu, double beta, int max_ls,
                   int fused, DevState* st, double* partials, int grid, cudaStream_t s) {
  LsParams lp{pp, mu, beta, max_ls, fused};
  const size_t smem = (size_t)((m + 63) & ~63) * sizeof(double);
  const double* Ad = (const double*)A;
  count_launch();
  if (dtype == kStreamFloatFloat) {
    const int sms = grid / 4;
    if (mode == kModeU)
      launch_ff<kModeU, false>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    else if (mode == kModeT)
      launch_ff<kModeT, false>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    else
      launch_ff<kModeGmax, false>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    return;
  }
  if (dtype == kStreamSplit) {
    const int sms = grid / 4;
    if (mode == kModeU)
      launch_ff<kModeU, true>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    else if (mode == kModeT)
      launch_ff<kModeT, true>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    else
      launch_ff<kModeGmax, true>(Ad, lda, m, n, vec, out, x, u, lp, st, partials, sms, s);
    return;
  }
  if (mode == kModeU)
    launch_k(k_stream_f64<kModeU>, dim3(grid), dim3(kStreamThreads), (size_t)(smem), s, Ad, lda, m, n, vec, out, x, u, lp, st, partials);
  else if (mode == kModeT)
    launch_k(k_stream_f64<kModeT>, dim3(grid), dim3(kStreamThreads), (size_t)(smem), s, Ad, lda, m, n, vec, out, x, u, lp, st, partials);
  else
    launch_k(k_stream_f64<kModeGmax>, dim3(grid), dim3(kStreamThreads), (size_t)(smem), s, Ad, lda, m, n, vec, out, x, u, lp, st, partials);
}

// Flags entries of A (rows < m) that the float-float split cannot represent:
// non-zero values outside [2^-100, 2^100], subnormals, infinities and NaN.
__global__ void k_check_range(const double* __restrict__ A, long long lda, int m, long long n, int* bad) {
  pdl_entry();
  const long long total = lda * n;
  int local = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    if (k % lda >= m) continue;
    const unsigned long long b = (unsigned long long)__double_as_longlong(A[k]);
    const int e = (int)((b >> 52) & 0x7FF);
    const bool zero = (b & 0x7FFFFFFFFFFFFFFFull) == 0ull;
    if (!zero && (e < 1023 - 100 || e > 1023 + 100)) local = 1;
  }
  if (__syncthreads_or(local) && threadIdx.x == 0) atomicOr(bad, 1);
}

void launch_check_range(const double* A, long long lda, int m, long long n, int* bad, int sms, cudaStream_t s) {
  count_launch();
  launch_k(k_check_range, dim3(4 * sms), dim3(256), (size_t)(0), s, A, lda, m, n, bad);
}

void launch_ls_fallback(const double* x, const double* u, const double* t, long long n, ProxParams pp, double mu,
                        double beta, int max_ls, int fused, DevState* st, double* partials, int grid, cudaStream_t s) {
  if (fused >= max_ls) return;
  LsParams lp{pp, mu, beta, max_ls, fused};
  count_launch();
  launch_k(k_ls_fallback, dim3(grid), dim3(256), (size_t)(0), s, x, u, t, n, lp, st, partials);
}

}  // namespace ssnal
