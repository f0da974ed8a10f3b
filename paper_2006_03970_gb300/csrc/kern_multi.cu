// One pass over A for several fits on the same matrix: t_f = A^T d_f for up to
// kMultiMax direction vectors d_f (the Newton-step pass of eq. line_search for each fit),
// each with its own fused line search.  This is the multi right-hand-side form
// A^T [d_1 ... d_k] of the serving loop: A is read once for k fits.
//
// The pass follows the single-vector lane stream (kern_stream.cu, k_stream_lane with
// FP32 accumulation) step for step for every vector: the same power-of-two scaling of
// the vector, the same TMA boxes, chunk-to-warp assignment and product order per
// column, the same merges and epilogue, the same trial sums and Armijo selection in
// the fit's own DevState.  Each fit's t, trial sums and accepted step are therefore
// bitwise those of the single-vector pass, whatever the other fits of the pass are.
//
// Layout per CTA: the warps' TMA rings as in the lane stream, the vectors' FP32 parts
// (one packed pair per row pair and vector), and the per-warp column partials of every
// vector (double buffered).  Warps 2f and 2f + 1 run the column epilogue of vector f.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/ssnal_en.h"
#include "lane_common.cuh"

namespace ssnal {

constexpr int kMultiMax = 4;  // vectors per pass (two epilogue warps each)

struct MultiFit {
  const double* d;    // direction, m
  double* t;          // A^T d, n
  const double* x;    // n
  const double* u;    // n
  DevState* st;       // the fit's state: trial sums, step, counters
  double* partials;   // gridDim x 32 doubles
  LsParams lp;
};
struct MultiArgs {
  int nv;
  MultiFit f[kMultiMax];
};

static size_t multi_smem(int m, int elt, int nv, int stages) {
  return (size_t)kLWarps * stages * kLBoxBytes + (size_t)nv * lane_mpad(m, elt) * 4 +
         (size_t)2 * nv * kLWarps * kLCols * sizeof(float2) + (size_t)kLWarps * stages * 8 + 1024;
}
constexpr size_t kMultiDynMax = 232448 - 8192;  // per-block limit minus the static shared memory

template <int ELT>
__global__ void __launch_bounds__(kLThreads, 1) k_stream_multi(const __grid_constant__ CUtensorMap tmap, int m,
                                                               long long n, const __grid_constant__ MultiArgs args,
                                                               LaneCfg cfg, const float* __restrict__ cmean,
                                                               const float* __restrict__ cscale) {
  static_assert(!elt_ff(ELT), "the multi-vector pass accumulates in FP32");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(1024) unsigned char smem_multi[];
  constexpr int R = elt_rows(ELT);
  constexpr int P = R / 16;
  const int nv = args.nv;
  const int mpad = lane_mpad(m, ELT);
  unsigned char* ring = smem_multi;
  unsigned long long* DV = reinterpret_cast<unsigned long long*>(smem_multi + (size_t)kLWarps * cfg.stages * kLBoxBytes);
  float2* part = reinterpret_cast<float2*>(DV + (size_t)nv * (mpad / 2));  // [2][nv][kLWarps][kLCols]
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(part + (size_t)2 * nv * kLWarps * kLCols);
  __shared__ double wred[kLWarps][32];
  __shared__ double red[32];
  __shared__ unsigned long long dmax_bits[kMultiMax];
  __shared__ double ysum_s[kMultiMax];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int b = 0; b < kLWarps * cfg.stages; b++) mbar_init(smem_u32(bars + b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int f = 0; f < kMultiMax; f++) dmax_bits[f] = 0ull;
  }
  __syncthreads();
  const long long ngrp = (long long)blockIdx.x < cfg.groups ? (cfg.groups - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int nw = warp < cfg.chunks ? (cfg.chunks - warp + kLWarps - 1) / kLWarps : 0;
  const long long total = ngrp * nw;
  unsigned char* wring = ring + (size_t)warp * cfg.stages * kLBoxBytes;
  unsigned long long* wbars = bars + warp * cfg.stages;
  auto issue = [&](long long item) {
    const long long q = item / nw;
    const int ch = warp + kLWarps * (int)(item % nw);
    const int sidx = (int)(item % cfg.stages);
    const unsigned bar = smem_u32(wbars + sidx);
    mbar_expect_tx(bar, kLBoxBytes);
    tma_load_2d(smem_u32(wring + (size_t)sidx * kLBoxBytes), &tmap, ch * elt_box_inner(ELT),
                (int)(((long long)blockIdx.x + q * gridDim.x) * kLCols), bar);
  };
  if (lane == 0)
    for (long long it = 0; it < total && it < cfg.stages; it++) issue(it);
  __syncwarp();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // every vector scaled by its own power of two; DV[f][pair_slot(k)] = (dh0, dh1) of rows
  // 2k, 2k + 1 (the slot order of the single-vector pass)
  for (int f = 0; f < nv; f++) {
    const double* vec = args.f[f].d;
    unsigned long long mb = 0ull;
    for (int i = tid; i < m; i += blockDim.x) {
      unsigned long long b = (unsigned long long)__double_as_longlong(vec[i]) & 0x7FFFFFFFFFFFFFFFull;
      mb = b > mb ? b : mb;
    }
    atomicMax(&dmax_bits[f], mb);
  }
  __syncthreads();
  for (int f = 0; f < nv; f++) {
    int ex = (int)((dmax_bits[f] >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) ex = 1023;
    {
      const double scale = __longlong_as_double((long long)(2046 - ex) << 52);
      const double* vec = args.f[f].d;
      for (int k = tid; k < mpad / 2; k += blockDim.x) {
        float h[2] = {0.0f, 0.0f};
        for (int q = 0; q < 2; q++) {
          const int i = 2 * k + q;
          if (i < m) h[q] = __double2float_rn(vec[i] * scale);
        }
        DV[(size_t)f * (mpad / 2) + pair_slot<P>(k)] =
            (unsigned long long)__float_as_uint(h[0]) | ((unsigned long long)__float_as_uint(h[1]) << 32);
      }
    }
  }
  if constexpr (elt_geno(ELT)) {
    for (int f = 0; f < nv; f++) {
      const double* vec = args.f[f].d;
      double a = 0.0;
      for (int i = tid; i < m; i += blockDim.x) a += vec[i];
      const double ys = block_sum(a, red);
      if (tid == 0) ysum_s[f] = ys;
    }
  }
  __syncthreads();

  // epilogue role: warps 2f, 2f + 1 serve vector f (columns lane and lane + 32 of a group)
  const int ef = warp >> 1;
  const bool epi = ef < nv;
  double unscale = 1.0;
  if (epi) {
    int ex = (int)((dmax_bits[ef] >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) ex = 1023;
    unscale = __longlong_as_double((long long)ex << 52);
  }
  const LsParams lp = args.f[epi ? ef : 0].lp;
  double s_lane = 1.0;
  for (int k = 0; k < lane; k++) s_lane *= lp.beta;
  double cand = 0.0;
  bool timed_out = false;
  long long it = 0;
  for (long long q = 0; q < ngrp; q++) {
    unsigned long long S2[kMultiMax], S2b[kMultiMax];
#pragma unroll
    for (int f = 0; f < kMultiMax; f++) S2[f] = S2b[f] = 0ull;
    for (int k = 0; k < nw && !timed_out; k++, it++) {
      const int sidx = (int)(it % cfg.stages);
      if (!mbar_wait(smem_u32(wbars + sidx), (unsigned)((it / cfg.stages) & 1))) {
        timed_out = true;
        break;
      }
      const int ch = warp + kLWarps * k;
      const unsigned char* colbase = wring + (size_t)sidx * kLBoxBytes + lane * 128;
      const unsigned long long* DVc = DV + ch * (R / 2);
      // the products of one row pair with every vector, in the single-vector order
      auto fma_pair = [&](int slot, unsigned long long av, unsigned long long bv) {
#pragma unroll
        for (int f = 0; f < kMultiMax; f++) {
          if (f < nv) {
            const unsigned long long d = DVc[(size_t)f * (mpad / 2) + slot];
            S2[f] = f2fma(av, d, S2[f]);
            S2b[f] = f2fma(bv, d, S2b[f]);
          }
        }
      };
#pragma unroll
      for (int p = 0; p < 8; p++) {
        const int pp = (p + lane) & 7;
        const uint4 a = *reinterpret_cast<const uint4*>(colbase + pp * 16);
        const uint4 b = *reinterpret_cast<const uint4*>(colbase + 32 * 128 + pp * 16);
        if constexpr (P == 32) {  // 2-bit codes
          const unsigned aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
          const unsigned long long bias = 0x4B0000004B000000ull;
#pragma unroll
          for (int qq = 0; qq < 4; qq++) {
            unsigned ea[4], eb[4];
#pragma unroll
            for (int g = 0; g < 4; g++) {
              ea[g] = (aw[qq] >> (2 * g)) & 0x03030303u;
              eb[g] = (bw[qq] >> (2 * g)) & 0x03030303u;
            }
#pragma unroll
            for (int e = 0; e < 8; e++) {
              const int byte = e >> 1, f0 = 2 * (e & 1);
              const unsigned long long av =
                  f2sub((unsigned long long)code_biased(ea[f0], byte) |
                            ((unsigned long long)code_biased(ea[f0 + 1], byte) << 32),
                        bias);
              const unsigned long long bv =
                  f2sub((unsigned long long)code_biased(eb[f0], byte) |
                            ((unsigned long long)code_biased(eb[f0 + 1], byte) << 32),
                        bias);
              fma_pair(8 * (8 * qq + e) + pp, av, bv);
            }
          }
        } else {
          unsigned long long ap[P], bp[P];
          if constexpr (P == 4) {  // 8 BF16 rows
            ap[0] = bf16x2_to_f32x2(a.x); ap[1] = bf16x2_to_f32x2(a.y);
            ap[2] = bf16x2_to_f32x2(a.z); ap[3] = bf16x2_to_f32x2(a.w);
            bp[0] = bf16x2_to_f32x2(b.x); bp[1] = bf16x2_to_f32x2(b.y);
            bp[2] = bf16x2_to_f32x2(b.z); bp[3] = bf16x2_to_f32x2(b.w);
          } else if constexpr (P == 8) {  // 16 int8 codes
            const unsigned long long bias = 0x4B0000804B000080ull;
            const unsigned aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int qq = 0; qq < 4; qq++) {
              ap[2 * qq] = f2sub(i8x2_biased(aw[qq], 0), bias);
              ap[2 * qq + 1] = f2sub(i8x2_biased(aw[qq], 2), bias);
              bp[2 * qq] = f2sub(i8x2_biased(bw[qq], 0), bias);
              bp[2 * qq + 1] = f2sub(i8x2_biased(bw[qq], 2), bias);
            }
          } else {  // 4 FP32 rows
            ap[0] = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
            ap[1] = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
            bp[0] = (unsigned long long)b.x | ((unsigned long long)b.y << 32);
            bp[1] = (unsigned long long)b.z | ((unsigned long long)b.w << 32);
          }
#pragma unroll
          for (int e = 0; e < P; e++) fma_pair(8 * e + pp, ap[e], bp[e]);
        }
      }
      __syncwarp();
      if (lane == 0 && it + cfg.stages < total) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(it + cfg.stages);
      }
    }
    float2* pq = part + (size_t)(q & 1) * nv * kLWarps * kLCols;
#pragma unroll
    for (int f = 0; f < kMultiMax; f++) {
      if (f < nv) {
        float Sq = lo32f(S2[f]), Lq = 0.0f;
        ff_merge(Sq, Lq, hi32f(S2[f]), 0.0f);
        pq[((size_t)f * kLWarps + warp) * kLCols + lane] = make_float2(Sq, Lq);
        float Sb = lo32f(S2b[f]), Lb = 0.0f;
        ff_merge(Sb, Lb, hi32f(S2b[f]), 0.0f);
        pq[((size_t)f * kLWarps + warp) * kLCols + lane + 32] = make_float2(Sb, Lb);
      }
    }
    __syncthreads();
    if (epi) {
      const MultiFit& F = args.f[ef];
      const int cc = lane + 32 * (warp & 1);
      const float2* pf = pq + (size_t)ef * kLWarps * kLCols;
      float Sm = pf[cc].x, Lm = pf[cc].y;
      for (int w = 1; w < kLWarps; w++) ff_merge(Sm, Lm, pf[w * kLCols + cc].x, pf[w * kLCols + cc].y);
      const long long j = ((long long)blockIdx.x + q * gridDim.x) * kLCols + cc;
      const bool mine = j < n;
      double t = ((double)Sm + (double)Lm) * unscale;
      if constexpr (elt_geno(ELT)) {
        if (mine) t = (double)cscale[j] * (t - (double)cmean[j] * ysum_s[ef]);
      }
      if (mine) F.t[j] = t;
      double v = 0.0;
      bool live = false;
      if (mine) {
        v = v_of(F.x[j], F.u[j], lp.pp.sigma);
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
  if (timed_out) {
    for (int f = 0; f < nv; f++) args.f[f].st->timeout = 1;
    if (lane == 0)
      for (long long k = it; k < total && k < it + cfg.stages; k++)
        mbar_wait(smem_u32(wbars + (int)(k % cfg.stages)), (unsigned)((k / cfg.stages) & 1));
    __syncwarp();
  }
  wred[warp][lane] = cand;
  __syncthreads();
  // per fit: the block's trial sums (warps 2f, 2f + 1, in the single-vector order:
  // zero plus the first epilogue warp plus the second), then the last block of this
  // fit's counter reduces them and selects the step
  if (warp == 0) {
    for (int f = 0; f < nv; f++) {
      double sum = 0.0;
      sum += wred[2 * f][lane];
      sum += wred[2 * f + 1][lane];
      args.f[f].partials[(long long)blockIdx.x * 32 + lane] = sum;
    }
  }
  for (int f = 0; f < nv; f++) {
    const MultiFit& F = args.f[f];
    if (!last_block(&F.st->counters[kCtrStream])) continue;
    {
      const double sum = rows_sum32(F.partials, (int)gridDim.x, &wred[0][0]);
      if (warp == 0 && lane < F.lp.fused) F.st->lsdiff[lane] = sum;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence_block();
      double sel;
      int k = armijo_select(F.st, F.lp, 0, F.lp.fused, sel);
      if (k >= 0) {
        F.st->s = sel;
        F.st->ls_k = k;
        F.st->ls_state = 0;
      } else if (F.lp.fused < F.lp.max_ls) {
        F.st->ls_state = 1;
      } else {
        F.st->s = sel;
        F.st->ls_k = F.lp.max_ls - 1;
        F.st->ls_state = 0;
      }
    }
    reset_counter(&F.st->counters[kCtrStream]);
    __syncthreads();
  }
}

template <int ELT>
static bool launch_multi_elt(const void* map, int m, long long n, const MultiArgs& args, int sms, cudaStream_t s,
                             const float* cmean, const float* cscale) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_stream_multi<ELT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiDynMax);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  int stages = 8;
  while (stages > 1 && multi_smem(m, ELT, args.nv, stages) > kMultiDynMax) stages--;
  if (multi_smem(m, ELT, args.nv, stages) > kMultiDynMax) return false;
  LaneCfg cfg;
  cfg.stages = stages;
  cfg.chunks = (m + elt_rows(ELT) - 1) / elt_rows(ELT);
  cfg.groups = (n + kLCols - 1) / kLCols;
  long long grid = cfg.groups;
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(map);
  count_launch();
  launch_k(k_stream_multi<ELT>, dim3((int)grid), dim3(kLThreads), multi_smem(m, ELT, args.nv, stages), s, *tm, m, n,
           args, cfg, cmean, cscale);
  return cudaGetLastError() == cudaSuccess;
}

bool launch_stream_multi(int elt, const void* map, int m, long long n, int nv, const double* const* d, double* const* t,
                         const double* const* x, const double* const* u, DevState* const* st,
                         double* const* partials, const ProxParams* pp, double mu, double beta, int max_ls, int fused,
                         int sms, cudaStream_t s, const float* cmean, const float* cscale) {
  if (nv < 1 || nv > kMultiMax) return false;
  MultiArgs args{};
  args.nv = nv;
  for (int f = 0; f < nv; f++) {
    args.f[f].d = d[f];
    args.f[f].t = t[f];
    args.f[f].x = x[f];
    args.f[f].u = u[f];
    args.f[f].st = st[f];
    args.f[f].partials = partials[f];
    args.f[f].lp = LsParams{pp[f], mu, beta, max_ls, fused};
  }
  switch (elt) {
    case kEltBf16: return launch_multi_elt<kEltBf16>(map, m, n, args, sms, s, cmean, cscale);
    case kEltF32: return launch_multi_elt<kEltF32>(map, m, n, args, sms, s, cmean, cscale);
    case kEltI8: return launch_multi_elt<kEltI8>(map, m, n, args, sms, s, cmean, cscale);
    case kEltI2: return launch_multi_elt<kEltI2>(map, m, n, args, sms, s, cmean, cscale);
    default: return false;
  }
}

}  // namespace ssnal
