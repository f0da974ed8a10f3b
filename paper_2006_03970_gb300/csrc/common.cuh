// Device helpers shared by the kernels: deterministic reductions, the
// last-block-done pattern and the Elastic Net prox (eq. prox_elastic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace ssnal {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block in a fixed order (warp tree, then warp 0 over warp sums).
// `red` must hold at least 32 doubles.  Result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double out = red[0];
  __syncthreads();
  return out;
}

// Deterministic multi-value block reduction.  FP64 arithmetic is slow on this
// GPU (about two lanes per clock per SM: one warp-wide add holds the pipe for 16
// cycles), so the adds are kept to a minimum.  Threads of the first nw warps store
// their K values to shared memory; warp 0 adds them per lane (lane l takes
// threads l, l + 32, ... in order) and reduces the 32 lane sums by transposition:
// at each step the lanes of a pair exchange half of their values, about K +
// log2(32 / K) adds per lane instead of 5 K for K separate warp sums.
// Thread k < K of warp 0 returns total k.  red: K * 32 * nw doubles.
template <int K>
__device__ __forceinline__ double block_sum_k(const double (&v)[K], double* red, int nw) {
  static_assert(K >= 1 && K <= 32, "1..32 values");
  constexpr int KP = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nt = 32 * nw;
  __syncthreads();  // red may still be read by an earlier call
  if (tid < nt)
#pragma unroll
    for (int k = 0; k < K; k++) red[k * nt + tid] = v[k];
  __syncthreads();
  double out = 0.0;
  if (tid < 32) {
    double s[KP];
#pragma unroll
    for (int k = 0; k < KP; k++) {
      double a = 0.0;
      if (k < K)
        for (int w = 0; w < nw; w++) a += red[k * nt + lane + 32 * w];
      s[k] = a;
    }
#pragma unroll
    for (int h = KP / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; i++) {
        const double send = up ? s[i] : s[i + h];
        const double keep = up ? s[i + h] : s[i];
        s[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    // lane l now holds a partial of value l / (32 / KP); finish over the low bits
#pragma unroll
    for (int o = 16 / KP; o >= 1; o >>= 1) s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
    out = __shfl_sync(0xffffffffu, s[0], (lane < K ? lane : 0) * (32 / KP));
  }
  return out;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double out = red[0];
  __syncthreads();
  return out;
}

// Last-block-done: after every block has written its partial results, exactly
// one block (the last to arrive) sees `true` and may reduce the partials in a
// fixed order.  That block resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

__device__ __forceinline__ void reset_counter(unsigned int* counter) {
  if (threadIdx.x == 0) *counter = 0u;
}

// Loads that bypass L1 so that values written by other blocks of the same
// kernel (before the fence of last_block) are observed.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ long long ld_cg(const long long* p) { return __ldcg(p); }

// soft(t, thr) magnitude part: max(|t| - thr, 0)
__device__ __forceinline__ double shrink_mag(double t, double thr) { return fmax(fabs(t) - thr, 0.0); }

// prox_{sigma p}(v) of eq. prox_elastic: sign(v) max(|v| - sigma*lam1, 0) / (1 + sigma*lam2).
// The active test |v| > thr (eq. Q_def) and this value must agree: the value is
// nonzero exactly when the test holds.
__device__ __forceinline__ double prox_value(double v, const ProxParams& pp) {
  double mag = __dsub_rn(fabs(v), pp.thr);
  if (!(mag > 0.0)) return 0.0;
  double w = __ddiv_rn(mag, pp.onep);
  return v < 0.0 ? -w : w;
}

// |v| > thr, compared on the bit patterns (thr >= 0; for finite values the
// integer order of non-negative doubles is their numeric order), which keeps the
// test off the FP64 pipe.
__device__ __forceinline__ bool abs_gt(double v, double thr) {
  return (unsigned long long)(__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL) >
         (unsigned long long)__double_as_longlong(thr);
}
__device__ __forceinline__ bool is_active(double v, const ProxParams& pp) { return abs_gt(v, pp.thr); }

// v = x - sigma*u with two roundings (no contraction into an FMA), the same
// rounding sequence as the plain elementwise evaluation of the definition.
__device__ __forceinline__ double v_of(double x, double u, double sigma) { return __dsub_rn(x, __dmul_rn(sigma, u)); }

// x == +0 or -0, tested on the bit pattern (integer pipe, not the FP64 pipe)
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }


// Sum p[0], p[stride], ..., p[(count-1) stride] in index order (the same
// association as a plain loop), with B loads in flight at a time: partial
// results written by other blocks are read at L2 latency, so a serial chain of
// dependent round trips would dominate a reduction tail.
template <int B = 8>
__device__ __forceinline__ double ordered_sum_cg(const double* p, long long stride, int count) {
  double s = 0.0;
  int b = 0;
  for (; b + B <= count; b += B) {
    double v[B];
#pragma unroll
    for (int e = 0; e < B; e++) v[e] = ld_cg(p + (long long)(b + e) * stride);
#pragma unroll
    for (int e = 0; e < B; e++) s += v[e];
  }
  for (; b < count; b++) s += ld_cg(p + (long long)b * stride);
  return s;
}

// Lane-wise sum of the 32-wide rows 0..nb-1 of P (row b at P + 32 b) with every
// warp of the block: warp w adds its contiguous share of rows in order, then
// warp 0 adds the warps' results in order (a fixed order for a given block
// size).  Every thread must call it; the result is valid in warp 0.
// scratch: (blockDim.x / 32) x 32 doubles of shared memory.
__device__ __forceinline__ double rows_sum32(const double* P, int nb, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (nb + nw - 1) / nw;
  const int b0 = min(nb, warp * per), b1 = min(nb, b0 + per);
  const double s = ordered_sum_cg(P + (long long)b0 * 32 + lane, 32, b1 - b0);
  __syncthreads();
  scratch[warp * 32 + lane] = s;
  __syncthreads();
  double t = 0.0;
  if (warp == 0)
    for (int w = 0; w < nw; w++) t += scratch[w * 32 + lane];
  return t;
}

// ---- programmatic dependent launch: every kernel lets the next one in its stream
// be launched at once, then waits until its own prerequisites have completed
// (and their memory is visible) before touching any data.  This hides the
// launch latency between consecutive kernels; kernels launched without the
// attribute treat both instructions as no-ops.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- mbarrier helpers.  Every wait is bounded: it gives up after about two
// seconds of SM clock (or kSpinLimit rounds), so a protocol error cannot hang
// the GPU; the caller raises DevState::timeout and leaves.
constexpr unsigned kSpinLimit = 1u << 28;          // try_wait rounds
constexpr long long kWaitCycles = 4000000000LL;    // about 2 s of SM clock

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait for the phase with the given parity; false on a timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  for (unsigned it = 0; it < kSpinLimit; it++) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitCycles) break;
  }
  return false;
}
// 2-D tensor copy (TMA) of one box at (x, y) into shared memory, completing on
// the mbarrier `bar` of this CTA.
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 3-D tensor copy (TMA) of one box at (x, y, z) into shared memory, completing on the
// mbarrier `bar` of this CTA.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// ---- thread-block clusters: rank, size, distributed shared memory, barrier
__device__ __forceinline__ unsigned cluster_addr(unsigned a, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ double ld_dsmem(unsigned addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_dsmem(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Launches kernel k on stream s with programmatic stream serialization (see
// pdl_entry); if the launch with the attribute is refused, launches plainly.
template <typename... ExpT, typename... ActT>
inline void launch_k(void (*k)(ExpT...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, ActT&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k, args...) != cudaSuccess) {
    cudaGetLastError();
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, k, args...);
  }
}

}  // namespace ssnal
