// Newton-matrix SYRK on the 5th-generation tensor cores (tcgen05), the dense
// contraction of eqs. AJ_system / smw_formula:
//     C = sum_{(p, q) in pairs} X_p^T X_q ,   out = alpha C + beta I  (lower triangle)
// X_p are BF16 "row panels" (R rows, K-major, row stride ldk): the packed A_J
// (SMW form, R = r, K = m) or its transpose (m x m form, R = m, K = r).  For
// FP64 panels X_0 + X_1 + X_2 is a three-way BF16 split of each entry and the
// six products with p + q <= 2 (p, q in {0, 1, 2}) give an FP32-accurate
// result; BF16-stored A needs the single product (0, 0), which is exact before
// the FP32 accumulation.
//
// One CTA (4 warps) computes a 128 x 128 output tile over a range of K chunks
// (split-K): cp.async fills a ring of shared-memory stages in the canonical
// K-major core-matrix layout, one elected thread issues tcgen05.mma
// (M = 128, N = 128, K = 16, FP32 accumulator in TMEM) and commits to the
// stage's mbarrier; the epilogue reads TMEM with tcgen05.ld.  Partial tiles
// of a split are summed in a fixed order by a second kernel (deterministic).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace ssnal {

constexpr int kTcThreads = 128;
constexpr int kTcChunk = 64;                        // K elements per stage
constexpr int kTcTileBytes = 128 * kTcChunk * 2;    // one operand tile per stage (16 KB)
constexpr int kTcStages = 4;

struct TcPairs {
  int n;           // number of products
  int p[6], q[6];  // X index of the A and B operands of each product
};

__device__ __forceinline__ uint64_t smem_desc(unsigned saddr) {
  // canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes;
  // K-adjacent core matrices 128 B apart (LBO), 8-row groups 1024 B apart (SBO)
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}

// BF16 x BF16 -> FP32, both operands K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void cp16(unsigned dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tri_tile_tc(int id, int& ti, int& tj) {
  int t = (int)((sqrtf(8.0f * (float)id + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= id) t++;
  while (t * (t + 1) / 2 > id) t--;
  ti = t;
  tj = id - t * (t + 1) / 2;
}

// grid = (tiles, splits).  X: 3 panels of R x ldk BF16 at X + p*R*ldk.
// out: FP32 ldo-strided lower triangle (when splits == 1) or the partial
// workspace part[(tile * splits + split) * 128 * 128] (row-major tile).
__global__ void __launch_bounds__(kTcThreads, 1) k_syrk_tc(const __nv_bfloat16* __restrict__ X, int R, int ldk,
                                                           TcPairs pairs, float alpha, float beta, float* out,
                                                           long long ldo, float* part, DevState* st) {
  pdl_entry();
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) unsigned long long bars[kTcStages];
  __shared__ unsigned tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ti, tj;
  tri_tile_tc(blockIdx.x, ti, tj);
  const int a0 = ti * 128, b0 = tj * 128;
  const int chunks_per_pair = ldk / kTcChunk;
  const int total = pairs.n * chunks_per_pair;
  const int per = (total + gridDim.y - 1) / gridDim.y;
  const int c_begin = blockIdx.y * per;
  const int c_end = min(total, c_begin + per);
  const int nloc = c_end > c_begin ? c_end - c_begin : 0;
  const size_t panel = (size_t)R * ldk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; s++) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;

  // stage s holds the A tile at tsm + s*2*kTcTileBytes and the B tile right after it
  auto load = [&](int lc, int s) {
    const int c = c_begin + lc;
    const int pi = c / chunks_per_pair;
    const int k0 = (c % chunks_per_pair) * kTcChunk;
    const __nv_bfloat16* XA = X + (size_t)pairs.p[pi] * panel;
    const __nv_bfloat16* XB = X + (size_t)pairs.q[pi] * panel;
    unsigned char* sa = tsm + (size_t)s * 2 * kTcTileBytes;
    for (int e = tid; e < 128 * 8; e += kTcThreads) {
      const int row = e >> 3, kg = e & 7;
      const int off = (row >> 3) * 1024 + kg * 128 + (row & 7) * 16;
      const int ra = a0 + row, rb = b0 + row;
      cp16(smem_u32(sa + off), XA + (size_t)(ra < R ? ra : 0) * ldk + k0 + 8 * kg, ra < R ? 16 : 0);
      cp16(smem_u32(sa + kTcTileBytes + off), XB + (size_t)(rb < R ? rb : 0) * ldk + k0 + 8 * kg, rb < R ? 16 : 0);
    }
  };

  bool ok = true;
  const int pre = nloc < kTcStages ? nloc : kTcStages;
  for (int lc = 0; lc < pre; lc++) {
    load(lc, lc);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int lc = 0; lc < nloc; lc++) {
    const int s = lc % kTcStages;
    // data of chunk lc has landed (younger groups may still be in flight)
    const int younger = (nloc - 1 - lc) < (kTcStages - 1) ? (nloc - 1 - lc) : (kTcStages - 1);
    if (younger >= 3)
      asm volatile("cp.async.wait_group 3;" ::: "memory");
    else if (younger == 2)
      asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (younger == 1)
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned sa = smem_u32(tsm + (size_t)s * 2 * kTcTileBytes);
      for (int k = 0; k < kTcChunk / 16; k++) {
        const uint64_t ad = smem_desc(sa + k * 256);
        const uint64_t bd = smem_desc(sa + kTcTileBytes + k * 256);
        const unsigned acc = (lc > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bars[s]))
                   : "memory");
    }
    // refill this stage with chunk lc + kTcStages once its MMAs have read it
    if (lc + kTcStages < nloc) {
      if (!mbar_wait(smem_u32(&bars[s]), (unsigned)((lc / kTcStages) & 1))) ok = false;
      __syncthreads();
      if (ok) load(lc + kTcStages, s);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  // all MMAs done: wait for the last commit of every stage still pending
  if (nloc > 0) {
    const int last = nloc - 1;
    if (!mbar_wait(smem_u32(&bars[last % kTcStages]), (unsigned)((last / kTcStages) & 1))) ok = false;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && tid == 0) st->timeout = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---- epilogue: warp w holds tile rows 32w..32w+31 (TMEM lanes), 32 columns per load
  const int row = 32 * warp + lane;
  for (int cb = 0; cb < 128; cb += 32) {
    unsigned v[32];
    const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)cb;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (nloc == 0)
      for (int c = 0; c < 32; c++) v[c] = 0u;
    if (gridDim.y == 1) {
      const int a = a0 + row;
      for (int c = 0; c < 32; c++) {
        const int b = b0 + cb + c;
        if (a < R && b < R && a >= b) out[a + (long long)b * ldo] = alpha * __uint_as_float(v[c]) + (a == b ? beta : 0.0f);
      }
    } else {
      // column-major partial tile: for each column the lanes store consecutive rows
      float* pt = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 128 * 128;
      for (int c = 0; c < 32; c++) pt[(size_t)(cb + c) * 128 + row] = __uint_as_float(v[c]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
}

// ---- TMA-fed variant with the split-K reduction inside a cluster --------------
// Same products, chunk partition and summation order as k_syrk_tc + k_syrk_tc_reduce
// (so the same result bit for bit), but:
//   * operand tiles arrive by 3-D TMA (tensor map over the panels: dims {ldk, R, panels},
//     box {8, 128, 1}: one 16-byte column of 128 rows per copy, eight copies per operand
//     and stage) into a K-major layout whose K-adjacent core matrices are 2048 B apart
//     and 8-row groups 128 B apart; zero fill past row R;
//   * warp 1 produces (waits for a stage to be free, arms and issues its copies), warp 0
//     issues the MMAs (waits for the stage's copies, commits to the stage's free barrier);
//   * the S splits of one tile form a cluster: each CTA parks its FP32 partial tile in its
//     own shared memory (column-major), and after a cluster barrier CTA q adds, for the
//     columns [q 128 / S, (q + 1) 128 / S), the partials of ranks 0 .. S - 1 in order
//     through distributed shared memory and writes alpha C + beta I (no partial tiles in
//     global memory and no second kernel).
__device__ __forceinline__ uint64_t smem_desc_lbo_sbo(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(lbo >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// A read of another CTA's shared memory, ordered after the cluster barrier that precedes
// it (volatile: not moved across that barrier; no memory clobber, so a batch of such
// loads is issued back to back and their latencies overlap).
__device__ __forceinline__ float ld_dsmem_f32(unsigned addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

template <int S>
__global__ void __cluster_dims__(S, 1, 1) __launch_bounds__(kTcThreads, 1)
    k_syrk_tc_tma(const __grid_constant__ CUtensorMap tm, int R, int ldk, TcPairs pairs, float alpha, float beta,
                  float* out, long long ldo, DevState* st) {
  pdl_entry();
  extern __shared__ __align__(1024) unsigned char tsm2[];
  __shared__ __align__(8) unsigned long long full[kTcStages], empty[kTcStages], done;
  __shared__ unsigned tmem_base;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = (int)blockIdx.x;  // = rank in the cluster
  int ti, tj;
  tri_tile_tc(blockIdx.y, ti, tj);
  const int a0 = ti * 128, b0 = tj * 128;
  const int chunks_per_pair = ldk / kTcChunk;
  const int total = pairs.n * chunks_per_pair;
  const int per = (total + S - 1) / S;
  const int c_begin = split * per;
  const int c_end = min(total, c_begin + per);
  const int nloc = c_end > c_begin ? c_end - c_begin : 0;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)tsm2 + 1023) & ~(uintptr_t)1023);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < kTcStages; q++) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  bool ok = true;

  if (warp == 1 && lane == 0) {
    // producer: chunk lc goes to stage lc % kTcStages once the MMAs of chunk lc - kTcStages are done
    int issued = 0;
    for (int lc = 0; lc < nloc; lc++) {
      const int q = lc % kTcStages;
      if (lc >= kTcStages && !mbar_wait(smem_u32(&empty[q]), (unsigned)((lc / kTcStages - 1) & 1))) {
        ok = false;
        break;
      }
      if (*(volatile int*)&abort_s) break;
      const int c = c_begin + lc;
      const int pi = c / chunks_per_pair;
      const int k0 = (c % chunks_per_pair) * kTcChunk;
      unsigned char* sa = ring + (size_t)q * 2 * kTcTileBytes;
      const unsigned bar = smem_u32(&full[q]);
      mbar_expect_tx(bar, 2 * kTcTileBytes);
#pragma unroll
      for (int kg = 0; kg < 8; kg++) {
        tma_load_3d(smem_u32(sa + kg * 2048), &tm, k0 + 8 * kg, a0, pairs.p[pi], bar);
        tma_load_3d(smem_u32(sa + kTcTileBytes + kg * 2048), &tm, k0 + 8 * kg, b0, pairs.q[pi], bar);
      }
      issued = lc + 1;
    }
    // every copy issued has landed before the CTA leaves: the last phase of each stage
    // (earlier phases completed before the stage was refilled); immediate when the MMA
    // issuer consumed them, bounded otherwise
    for (int lc = issued > kTcStages ? issued - kTcStages : 0; lc < issued; lc++)
      if (!mbar_wait(smem_u32(&full[lc % kTcStages]), (unsigned)((lc / kTcStages) & 1))) ok = false;
  } else if (warp == 0 && lane == 0) {
    // MMA issuer
    int lc = 0;
    for (; lc < nloc; lc++) {
      const int q = lc % kTcStages;
      if (!mbar_wait(smem_u32(&full[q]), (unsigned)((lc / kTcStages) & 1))) {
        ok = false;
        *(volatile int*)&abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned sa = smem_u32(ring + (size_t)q * 2 * kTcTileBytes);
#pragma unroll
      for (int k = 0; k < kTcChunk / 16; k++) {
        const uint64_t ad = smem_desc_lbo_sbo(sa + k * 4096, 2048, 128);
        const uint64_t bd = smem_desc_lbo_sbo(sa + kTcTileBytes + k * 4096, 2048, 128);
        const unsigned acc = (lc > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[q]))
                   : "memory");
    }
    if (lc > 0)  // arrives once every MMA issued above has completed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done))
                   : "memory");
    else
      mbar_arrive(smem_u32(&done));
  }
  __syncwarp();
  if (!mbar_wait(smem_u32(&done), 0u)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---- epilogue: warp w holds tile rows 32w..32w+31 (TMEM lanes), 32 columns per load
  const int row = 32 * warp + lane;
  float* C = reinterpret_cast<float*>(ring);  // column-major 128 x 128 partial (the ring is free now)
  __syncthreads();                             // the producer's final waits are over: no copy lands in the ring
  for (int cb = 0; cb < 128; cb += 32) {
    unsigned v[32];
    const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)cb;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (nloc == 0 || !ok)
      for (int c = 0; c < 32; c++) v[c] = 0u;
    if (S == 1) {
      const int a = a0 + row;
      for (int c = 0; c < 32; c++) {
        const int b = b0 + cb + c;
        if (a < R && b < R && a >= b) out[a + (long long)b * ldo] = alpha * __uint_as_float(v[c]) + (a == b ? beta : 0.0f);
      }
    } else {
      for (int c = 0; c < 32; c++) C[(cb + c) * 128 + row] = __uint_as_float(v[c]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  if (!ok && tid == 0) st->timeout = 1;
  if (S > 1) {
    cluster_arrive();  // this CTA's partial is in place
    cluster_wait();
    constexpr int W = 128 / S;       // columns reduced by this CTA
    constexpr int CB = 32 / S < W ? 32 / S : W;  // columns per batch: 32 remote loads in flight per thread
    static_assert(W % CB == 0, "whole batches");
    const unsigned base = smem_u32(C);
    unsigned rbase[S];
#pragma unroll
    for (int q = 0; q < S; q++) rbase[q] = cluster_addr(base, q);
    for (int c0 = 0; c0 < W; c0 += CB) {
      float vals[CB][S];
#pragma unroll
      for (int cc = 0; cc < CB; cc++)
#pragma unroll
        for (int q = 0; q < S; q++)
          vals[cc][q] = ld_dsmem_f32(rbase[q] + (unsigned)(((split * W + c0 + cc) * 128 + row) * 4));
#pragma unroll
      for (int cc = 0; cc < CB; cc++) {
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < S; q++) sum += vals[cc][q];  // ranks in order, as the reduce kernel adds splits
        const int col = split * W + c0 + cc;
        const int a = a0 + row, b = b0 + col;
        if (a < R && b < R && a >= b) out[a + (long long)b * ldo] = alpha * sum + (a == b ? beta : 0.0f);
      }
    }
    cluster_arrive();  // no CTA leaves while another reads its shared memory
    cluster_wait();
  }
}

// Sum of the split-K partial tiles in a fixed order, then alpha C + beta I.
// grid = (tiles, 64): block y handles columns 2y, 2y+1 of the tile.
__global__ void k_syrk_tc_reduce(const float* __restrict__ part, int splits, int R, float alpha, float beta,
                                 float* __restrict__ out, long long ldo) {
  pdl_entry();
  int ti, tj;
  tri_tile_tc(blockIdx.x, ti, tj);
  const int a0 = ti * 128, b0 = tj * 128;
  const int e = blockIdx.y * 256 + threadIdx.x;
  const int row = e & 127, col = e >> 7;  // consecutive threads: consecutive rows of one column
  const int a = a0 + row, b = b0 + col;
  if (a >= R || b >= R || a < b) return;
  float sum = 0.0f;
  for (int y = 0; y < splits; y++)
    sum += part[((size_t)blockIdx.x * splits + y) * 128 * 128 + (size_t)col * 128 + row];
  out[a + (long long)b * ldo] = alpha * sum + (a == b ? beta : 0.0f);
}

// BF16 row panels of the FP64 packed A_J.  trans = 0 (SMW form): row a = column a
// of P (R = r, K = m); trans = 1 (m x m form): row i = row i of P (R = m, K = r).
// nsplit = 3: X_0 + X_1 + X_2 is the three-way BF16 split of each entry; 1: X_0 only.
// Entries with k >= K are zero up to ldk.
__global__ void k_panel_bf16(const double* __restrict__ P, long long ldp, int m, int r, int trans, int nsplit,
                             __nv_bfloat16* __restrict__ X, int ldk) {
  pdl_entry();
  __shared__ double tile[32][33];
  const int R = trans ? m : r, K = trans ? r : m;
  const size_t panel = (size_t)R * ldk;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  // block covers rows [row0, row0+32) and k in [k0, k0+32)
  const int row0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  for (int yy = ty; yy < 32; yy += 8) {
    double v = 0.0;
    if (!trans) {
      // X row a = row0 + yy, k = k0 + tx  <-  P[k + a ldp]  (coalesced along k)
      const int a = row0 + yy, k = k0 + tx;
      if (a < R && k < K) v = P[k + (long long)a * ldp];
      tile[yy][tx] = v;
    } else {
      // X row i, k  <-  P[i + k ldp]: read coalesced along i, transpose through shared memory
      const int i = row0 + tx, k = k0 + yy;
      if (i < R && k < K) v = P[i + (long long)k * ldp];
      tile[tx][yy] = v;
    }
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int rr = row0 + yy, k = k0 + tx;
    if (rr >= R || k >= ldk) continue;
    const double v = tile[yy][tx];
    const __nv_bfloat16 h0 = __double2bfloat16(v);
    X[(size_t)rr * ldk + k] = h0;
    if (nsplit == 3) {
      const double r1 = v - (double)__bfloat162float(h0);
      const __nv_bfloat16 h1 = __double2bfloat16(r1);
      const double r2 = r1 - (double)__bfloat162float(h1);
      X[panel + (size_t)rr * ldk + k] = h1;
      X[2 * panel + (size_t)rr * ldk + k] = __double2bfloat16(r2);
    }
  }
}

// ---------------------------------------------------------------- launchers
size_t syrk_tc_panel_elems(int R, int K, int nsplit) {
  const int ldk = (K + kTcChunk - 1) / kTcChunk * kTcChunk;
  return (size_t)nsplit * R * ldk;
}

// split-K partials: splits * tiles <= sms whenever splits > 1
size_t syrk_tc_part_floats(int sms) { return (size_t)sms * 128 * 128; }

// Tensor map over the BF16 panels X (panels x R rows x ldk, K contiguous): dims {ldk, R,
// panels}, boxes of 8 K values (16 bytes) x 128 rows x 1 panel, zero fill past row R.
static bool make_panel_tensor_map(CUtensorMap* map, const void* X, int R, int ldk, int panels) {
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
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0 || R <= 0 || ldk % kTcChunk != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)ldk, (cuuint64_t)R, (cuuint64_t)panels};
  cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)R * (cuuint64_t)ldk * 2};
  cuuint32_t box[3] = {8, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(X), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S>
static bool launch_tc_tma(const CUtensorMap& tm, int tiles, int R, int ldk, const TcPairs& pr, float alpha,
                          float beta, float* out, long long ldo, DevState* st, cudaStream_t s) {
  static int state[64] = {};  // per device: 0 not yet set up, 1 usable, -1 not usable
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = (size_t)kTcStages * 2 * kTcTileBytes + 1024;
  if (dev >= 0 && dev < 64 && state[dev] < 0) return false;
  if (dev < 0 || dev >= 64 || state[dev] == 0) {
    if (dev >= 0 && dev < 64) state[dev] = -1;  // until the set-up below succeeds
    if (cudaFuncSetAttribute(k_syrk_tc_tma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        (S > 8 && cudaFuncSetAttribute(k_syrk_tc_tma<S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)) {
      cudaGetLastError();
      return false;
    }
    if (S > 8) {
      // a 16-CTA cluster must fit on this device with this shared memory
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(S, 1);
      cfg.blockDim = dim3(kTcThreads);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = S;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_syrk_tc_tma<S>, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return false;
      }
    }
    if (dev >= 0 && dev < 64) state[dev] = 1;
  }
  count_launch();
  launch_k(k_syrk_tc_tma<S>, dim3(S, tiles), dim3(kTcThreads), smem, s, tm, R, ldk, pr, alpha, beta, out, ldo, st);
  return cudaGetLastError() == cudaSuccess;
}

// out = alpha * (sum of products of the split panels) + beta * I, lower triangle.
void launch_syrk_tc(const double* P, long long ldp, int m, int r, int trans, int nsplit, void* Xbuf, float* part,
                    float alpha, float beta, float* out, long long ldo, DevState* st, int sms, cudaStream_t s) {
  const int R = trans ? m : r, K = trans ? r : m;
  const int ldk = (K + kTcChunk - 1) / kTcChunk * kTcChunk;
  __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(Xbuf);
  {
    dim3 grid((ldk + 31) / 32, (R + 31) / 32);
    count_launch();
    launch_k(k_panel_bf16, dim3(grid), dim3(256), (size_t)(0), s, P, ldp, m, r, trans, nsplit, X, ldk);
  }
  TcPairs pr;
  if (nsplit == 3) {
    const int pp[6] = {0, 0, 1, 0, 2, 1}, qq[6] = {0, 1, 0, 2, 0, 1};
    pr.n = 6;
    for (int i = 0; i < 6; i++) {
      pr.p[i] = pp[i];
      pr.q[i] = qq[i];
    }
  } else {
    pr.n = 1;
    pr.p[0] = pr.q[0] = 0;
    for (int i = 1; i < 6; i++) pr.p[i] = pr.q[i] = 0;
  }
  const int T = (R + 127) / 128;
  const int tiles = T * (T + 1) / 2;
  const int total = pr.n * (ldk / kTcChunk);
  {
    // TMA-fed kernel, split-K over a cluster of S (a power of two, at most 8) CTAs
    CUtensorMap tm;
    if (make_panel_tensor_map(&tm, X, R, ldk, nsplit)) {
      // S: a power of two, at most 16 (a non-portable cluster size) and at most sms / tiles,
      // with at least two K chunks per CTA
      int S = 1;
      while (2 * S <= 16 && 2 * S * tiles <= sms && 2 * S <= total / 2) S *= 2;
      bool launched = false;
      switch (S) {
        case 1: launched = launch_tc_tma<1>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s); break;
        case 2: launched = launch_tc_tma<2>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s); break;
        case 4: launched = launch_tc_tma<4>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s); break;
        case 8: launched = launch_tc_tma<8>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s); break;
        default:
          launched = launch_tc_tma<16>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s) ||
                     launch_tc_tma<8>(tm, tiles, R, ldk, pr, alpha, beta, out, ldo, st, s);
          break;
      }
      if (launched) return;
    }
  }
  int splits = sms / tiles;
  if (splits > total / 2) splits = total / 2;
  if (splits > 16) splits = 16;
  if (splits < 1) splits = 1;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = (size_t)kTcStages * 2 * kTcTileBytes + 1024;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  count_launch();
  launch_k(k_syrk_tc, dim3(dim3(tiles, splits)), dim3(kTcThreads), (size_t)(smem), s, X, R, ldk, pr, alpha, beta, out, ldo, part, st);
  if (splits > 1) {
    count_launch();
    launch_k(k_syrk_tc_reduce, dim3(dim3(tiles, 64)), dim3(256), (size_t)(0), s, part, splits, R, alpha, beta, out, ldo);
  }
}

}  // namespace ssnal
