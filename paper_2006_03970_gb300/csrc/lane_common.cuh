// Device helpers shared by the passes over A (kern_stream.cu: the single-vector
// streams; kern_multi.cu: the pass that serves several fits on one matrix): the
// line-search trial terms and the Armijo selection of eq. line_search, packed
// FP32 (f32x2) and float-float arithmetic, and the element types and box layout of
// the lane-per-column stream.
#pragma once

#include "common.cuh"

namespace ssnal {

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
// (The comparisons run on the bit patterns, off the FP64 pipe.)
__device__ __forceinline__ bool trial_skip(double v, double tj, const ProxParams& pp) {
  return !abs_gt(v, pp.thr) && !abs_gt(__dsub_rn(v, __dmul_rn(pp.sigma, tj)), pp.thr);
}

// Armijo selection over trials [k0, k1) given the trial sums; returns the
// accepted index or -1.
__device__ __forceinline__ int armijo_select(const DevState* st, const LsParams& lp, int k0, int k1, double& s_out) {
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

// (S, L) += (S2, L2)
__device__ __forceinline__ void ff_merge(float& S, float& L, float S2, float L2) {
  const float s = __fadd_rn(S, S2);
  const float z = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(S2, z));
  S = s;
  L = __fadd_rn(__fadd_rn(L, L2), t);
}

// Packed (f32x2) float-float step on an element pair: (S, L) += a * d for both
// lanes, with a = ah + al, d = dh + dl and the negated parts ndh = -dh,
// ndl = -dl supplied (there is no packed negation).
__device__ __forceinline__ unsigned long long f2add(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long x, unsigned long long y,
                                                    unsigned long long z) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(y), "l"(z));
  return r;
}
__device__ __forceinline__ void ff2_madd(unsigned long long& S, unsigned long long& L, unsigned long long ah,
                                         unsigned long long al, unsigned long long dh, unsigned long long ndh,
                                         unsigned long long ndl) {
  const unsigned long long p = f2mul(ah, dh);
  unsigned long long ne = f2fma(ah, ndh, p);  // -(exact product error)
  ne = f2fma(ah, ndl, ne);
  ne = f2fma(al, ndh, ne);                     // -(error + cross terms)
  const unsigned long long s = f2add(S, p);
  const unsigned long long z = f2sub(s, S);
  const unsigned long long t = f2add(f2sub(S, f2sub(s, z)), f2sub(p, z));
  S = s;
  L = f2add(L, f2sub(t, ne));
}
__device__ __forceinline__ float lo32f(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi32f(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }

constexpr int kLWarps = 8;
constexpr int kLThreads = kLWarps * 32;
constexpr int kLCols = 64;                   // columns per group: lane l owns columns l and l + 32
constexpr int kLBoxBytes = kLCols * 128;     // 64 columns x 16 rows x 8 bytes

// Stored element types the lane stream reads.  Every 2-D TMA box is 128 bytes
// of one column (the inner dimension) by 64 columns; kEltRows rows per box.
constexpr int kEltSplit = 0;    // pre-split FP64 copy: (hi, hi, lo, lo) per row pair, float-float
constexpr int kEltBf16FF = 1;   // BF16, float-float accumulation (products of the exact values)
constexpr int kEltBf16 = 2;     // BF16, FP32 accumulation
constexpr int kEltF32FF = 3;    // FP32, float-float accumulation
constexpr int kEltF32 = 4;      // FP32, FP32 accumulation
constexpr int kEltI8FF = 5;     // int8 genotype codes, float-float accumulation
constexpr int kEltI8 = 6;       // int8 genotype codes, FP32 accumulation
constexpr int kEltI2FF = 7;     // 2-bit genotype codes (four per byte), float-float accumulation
constexpr int kEltI2 = 8;       // 2-bit genotype codes, FP32 accumulation
// The genotype entries are (code - mean_j) * scale_j: the stream sums code * y
// and applies mean and scale per column, sum_i a_ij y_i = scale_j (sum_i c_ij y_i
// - mean_j sum_i y_i).
__host__ __device__ constexpr int elt_rows(int elt) {
  return elt == kEltSplit                            ? 16
         : (elt == kEltBf16FF || elt == kEltBf16)     ? 64
         : (elt == kEltI8FF || elt == kEltI8)         ? 128
         : (elt == kEltI2FF || elt == kEltI2)         ? 512
                                                      : 32;
}
// Shared-memory slot of row pair k of the vector.  A box holds 8P row pairs, P per
// 16-byte chunk of a column (P = elt_rows / 16); pair e of chunk c sits at slot
// 8 e + c.  The lanes of a quarter warp read eight different chunks at once (the
// chunk order is rotated by the lane), so they hit eight consecutive slots: no bank
// conflicts for 16-byte or 8-byte entries.
template <int P>
__device__ __forceinline__ int pair_slot(int k) {
  const int w = k & (8 * P - 1);
  return (k - w) + (w & (P - 1)) * 8 + w / P;
}
// genotype codes (int8 or 2-bit): the column epilogue applies mean and scale
__host__ __device__ constexpr bool elt_geno(int elt) {
  return elt == kEltI8FF || elt == kEltI8 || elt == kEltI2FF || elt == kEltI2;
}
// elements (of the tensor map's data type) of the inner box dimension (128 bytes)
__host__ __device__ constexpr int elt_box_inner(int elt) {
  return elt_rows(elt) == 16 ? 32 : (elt == kEltI2FF || elt == kEltI2) ? 128 : elt_rows(elt);
}
// rows the vector d is padded to in shared memory (whole boxes)
__host__ __device__ constexpr int lane_mpad(int m, int elt) {
  return elt_rows(elt) > 128 ? (m + elt_rows(elt) - 1) / elt_rows(elt) * elt_rows(elt) : (m + 127) & ~127;
}
__host__ __device__ constexpr bool elt_ff(int elt) {
  return elt == kEltSplit || elt == kEltBf16FF || elt == kEltF32FF || elt == kEltI8FF || elt == kEltI2FF;
}

// (S, L) += a * d on an element pair, a exact in FP32 (no low part)
__device__ __forceinline__ void ff2_madd_exact(unsigned long long& S, unsigned long long& L, unsigned long long a,
                                               unsigned long long dh, unsigned long long ndh, unsigned long long ndl) {
  const unsigned long long p = f2mul(a, dh);
  unsigned long long ne = f2fma(a, ndh, p);  // -(exact product error)
  ne = f2fma(a, ndl, ne);
  const unsigned long long s = f2add(S, p);
  const unsigned long long z = f2sub(s, S);
  const unsigned long long t = f2add(f2sub(S, f2sub(s, z)), f2sub(p, z));
  S = s;
  L = f2add(L, f2sub(t, ne));
}
// bytes k and k + 1 of w (int8 codes, memory order) as a packed FP32 pair of
// (code + 128) + 2^23; the caller subtracts 2^23 + 128 (exact)
__device__ __forceinline__ unsigned long long i8x2_biased(unsigned w, int k) {
  const unsigned x = w ^ 0x80808080u;  // code + 128 in 0..255
  const unsigned lo = __byte_perm(x, 0x4B000000u, 0x7540u + (unsigned)k);
  const unsigned hi = __byte_perm(x, 0x4B000000u, 0x7540u + (unsigned)k + 1u);
  return (unsigned long long)lo | ((unsigned long long)hi << 32);
}
// the code of byte k of w (a value 0..3 in each byte) as FP32 2^23 + code (exact)
__device__ __forceinline__ unsigned code_biased(unsigned w, int k) {
  return __byte_perm(w, 0x4B000000u, 0x7540u + (unsigned)k);
}
// two BF16 values of one 32-bit word (memory order) as a packed FP32 pair
__device__ __forceinline__ unsigned long long bf16x2_to_f32x2(unsigned w) {
  return (unsigned long long)(w << 16) | ((unsigned long long)(w & 0xFFFF0000u) << 32);
}

struct LaneCfg {
  int stages;        // ring depth per warp
  int chunks;        // boxes per column group (16 rows each)
  long long groups;  // column groups of 32
};

}  // namespace ssnal
