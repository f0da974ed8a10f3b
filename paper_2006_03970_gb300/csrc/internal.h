// Internal declarations shared by the CUDA translation units of libssnal_en.
// Nothing here is part of the public C ABI (include/ssnal_en.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/ssnal_en.h"

namespace ssnal {

// Number of kernels this library has launched (all contexts).
extern std::atomic<long long> g_launches;
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr int kMaxM = 4096;       // largest supported number of observations m
constexpr int kMaxLS = 64;        // largest supported number of line-search trials
constexpr int kFusedLS = 16;      // trial steps evaluated inside the A^T d stream
constexpr int kGemvGroups = 32;   // column groups of the panel GEMV partial sums
constexpr int kCholNB = 32;       // block size of the blocked Cholesky
constexpr int kNumCounters = 16;  // last-block-done counters

// Counter slots (one per kernel that uses the last-block pattern).
enum CounterSlot {
  kCtrProx = 0, kCtrCombine = 1, kCtrStream = 2, kCtrFallback = 3, kCtrGmax = 4, kCtrMisc = 5,
  kCtrBarrier = 6,  // two words: arrival count and generation of the cooperative grid barrier
  kCtrGemv = 8,
  kCtrRefine = 9  // the refinement step fused into the pair triangular solve
};
constexpr int kSmallNewton = 32;  // Newton systems up to this size (one tile) are factored by one CTA

// Values computed on the device and read by the host once per Newton step.
// The host never writes these except through cudaMemsetAsync of the whole struct.
struct DevState {
  // prox / active-set pass (eqs. prox_elastic, Q_def) at the current y
  long long r;        // |J|
  double w2;          // ||w||^2, w = prox_{sigma p}(v)
  double w1;          // ||w||_1
  double xw2;         // ||x - w||^2       (sigma^2 ||A^T y + z||^2)
  double vw2;         // ||v - w||^2       (sigma^2 ||z||^2)
  double dualpen;     // sum_j (|u_j| - lambda1)_+^2   (p*(-A^T y) * 2 lambda2)
  // gradient pass (eq. grad_phy)
  double g2;          // ||g||^2
  double y2;          // ||y||^2
  double yg2;         // ||y - g||^2 = ||A x - b||^2
  double by;          // b^T y
  // Newton direction dots used by the line search
  double gd, yd, dd, bd;
  // line search (eq. line_search)
  double s;           // accepted step
  int32_t ls_k;       // index of the accepted trial (trials = ls_k + 1)
  int32_t ls_state;   // 0 accepted, 1 fallback pending
  double lsdiff[kMaxLS];  // sum_j soft(v_j - s_k sigma t_j)^2 - soft(v_j)^2 per trial k
  // flags
  int32_t overflow;   // panel capacity exceeded by r
  // chol_fail, newton_bad and f64_fail are contiguous: the host clears the three at once.
  // While any of them is set the next prox pass does not apply the pending step.
  int32_t chol_fail;  // non-positive pivot in the FP32 Cholesky factorisation
  int32_t newton_bad; // the first refinement correction of the FP32 solve exceeded the contraction bound
  int32_t f64_fail;   // non-positive pivot in the FP64 Cholesky factorisation
  int32_t timeout;    // a bounded device-side wait gave up
  double gmax;        // ||A^T b||_inf (path)
  double refine_ratio;  // ||first refinement correction|| / ||refined solution|| of the last FP32 solve
  // conjugate-gradient Newton solve (kern_cg.cu)
  double cg_rr;       // ||res||^2 of the current iterate
  double cg_stop2;    // (rtol ||g||)^2
  int32_t cg_iters;   // iterations of the current solve
  int32_t cg_done;    // stopping test met (or breakdown)
  unsigned int counters[kNumCounters];
};

// Element access for the supported storage types.
enum StreamMode { kModeU = 0, kModeT = 1, kModeGmax = 2 };
// Stream arithmetic selector passed as `dtype` to launch_stream for FP64 storage.
constexpr int kStreamDfma = 0;         // FP64 FMA per element
constexpr int kStreamFloatFloat = 16;  // float-float on the FP32 pipe (entries 0 or in [2^-100, 2^100])
constexpr int kStreamSplit = 17;       // same arithmetic on a pre-split float-pair copy of A (packed f32x2)
constexpr int kStreamLane = 18;        // pre-split copy, lane per column, 2-D TMA tiles (tensor map)
// element types of the lane stream (see kern_stream.cu)
constexpr int kLaneSplit = 0, kLaneBf16FF = 1, kLaneBf16 = 2, kLaneF32FF = 3, kLaneF32 = 4, kLaneI8FF = 5,
              kLaneI8 = 6, kLaneI2FF = 7, kLaneI2 = 8;
enum ProxMode { kProxThreshold = 0, kProxSupport = 1 };

struct ProxParams {
  double sigma, lam1, lam2, thr, onep;  // thr = sigma*lam1, onep = 1 + sigma*lam2
  double inv_onep;                      // 1 / onep, for values that only feed norms
};

// ---- launch wrappers (kern_vec.cu)
int vec_grid(long long n, int sms);
// Zeroes *st and copies b (m values) to bdev, in one launch.
void launch_solve_begin(DevState* st, double* bdev, const double* b, int m, cudaStream_t s);
// dst[0..n) = src[0..n) on the stream.
void launch_copy_f64(double* dst, const double* src, long long n, int sms, cudaStream_t s);
// dst[0..n) = -src[0..n) on the stream.
void launch_neg_f64(double* dst, const double* src, long long n, int sms, cudaStream_t s);
// Copies *st to the pinned, device-mapped host mirror and then writes seq to flag
// (host memory), after a system-scope fence.
void launch_state_out(const DevState* st, DevState* host, unsigned* flag, unsigned seq, cudaStream_t s);
void launch_prox_count(int mode, const double* x, double* u, const double* t, double* y, const double* d,
                       long long n, int m, ProxParams pp, int apply_update, DevState* st,
                       long long* counts, double* partials, int grid, cudaStream_t s);
void launch_prox_scatter(int mode, const double* x, const double* u, long long n, ProxParams pp,
                         const long long* counts, const double* partials, DevState* st, int32_t* J, double* wJ,
                         int grid, cudaStream_t s);
void launch_set_x(double* x, const double* u, long long n, ProxParams pp, int sms, cudaStream_t s);
void launch_gather(const void* A, int dtype, long long lda, int m, const int32_t* J, const DevState* st,
                   long long r_host, long long rcap, double* P, long long ldp, float* P32, long long ldp32,
                   int sms, cudaStream_t s, const float* cmean = nullptr,
                   const float* cscale = nullptr);
void launch_gemv_n_partial(const double* P, long long ldp, int m, const double* coef, const DevState* st,
                           long long r_host, long long rcap, double* part, cudaStream_t s);
// out = ca*a + cb*b + cs*sum_groups(part); norms selected by `which` (see kern_vec.cu)
void launch_combine(double* out, const double* a, double ca, const double* b, double cb, const double* part,
                    double cs, int m, int which, const double* y, const double* bb, const double* g,
                    DevState* st, double* scratch, cudaStream_t s);
// out_i = ca*a_i + cb*b_i + cs*sum_k P[i,k] coef[k] in one launch, with the scalar products
// of k_combine (which = 1: gradient, 2: direction); r read from st when r_host < 0.
// cpart: kGemvSplitMax x m doubles; tile_ctr: ceil(m / 32) zeroed counters.
constexpr int kGemvSplitMax = 32;
void launch_gemv_n(const double* P, long long ldp, int m, const double* coef, const DevState* st, long long r_host,
                   long long rcap, double* out, const double* a, double ca, const double* b, double cb, double cs,
                   int which, const double* yv, const double* bv, const double* gv, DevState* stw, double* scratch,
                   double* cpart, unsigned* tile_ctr, cudaStream_t s);
// out_k = ch*h_k + cq*q_k + cd*dot(P[:,k], v)
void launch_gemv_t(const double* P, long long ldp, int m, long long r, const double* v, double* out,
                   const double* h, double ch, const double* q, double cq, double cd, int sms, cudaStream_t s);
void launch_absmax_finish(DevState* st, cudaStream_t s);

// ---- linear algebra (kern_linalg.cu)
void launch_syrk_tn(const float* P32, long long ldp32, int m, long long r, double diag, float* G, long long ldg,
                    cudaStream_t s);
void launch_syrk_nt(const float* P32, long long ldp32, int m, long long r, double kappa, float* G, long long ldg,
                    cudaStream_t s);
// Wdiag (may be null): receives the inverses of the 32 x 32 diagonal blocks of L
// when the factorisation produces them (the cluster kernel).  Returns whether
// they were written.  hrow, zout (may be null): the right-hand side h (N doubles) of
// the first solve; where the factor can run the forward substitution itself (one
// cluster launch, N % 32 != 0, Wdiag given) it writes z = L^{-1} h (FP32) to zout and
// sets *fused, so that launch_trsv_back finishes the solve.
bool chol_factor(float* G, long long ldg, int N, DevState* st, float* Wdiag, cudaStream_t s,
                 const double* hrow = nullptr, float* zout = nullptr, bool* fused = nullptr);
// *out = tr(G^{-1}) - (Np - N) + ... see kern_linalg.cu: factors the N x N SPD matrix in S (row
// stride ldS >= 2 * round_up(N, 32)) and writes ||L^{-1}||_F^2 + (Np - N) to *out (device).
// N <= 640; returns false otherwise or on a launch error.
bool inv_trace(float* S, long long ldS, int N, DevState* st, float* Wdiag, double* partial, double* out,
               cudaStream_t s);
// Any N <= kMaxM: factors the N x N SPD matrix G in place (chol_factor) and writes
// ||L^{-1}||_F^2 = tr(G^{-1}) to *out (device), Y scratch of ldy x 32 ceil(N / 32)
// floats (ldy >= 32 ceil(N / 32)), partial of ceil(N / 32) doubles.  Returns false when
// the factorisation gives no inverse diagonal blocks or on a launch error.
bool inv_trace_large(float* G, long long ldg, int N, DevState* st, float* Wdiag, float* Y, long long ldy,
                     double* partial, double* out, cudaStream_t s);
// N <= kSmallNewton: factor and solve one right-hand side in one launch by one warp (acc = alpha c)
void launch_chol_solve_small(float* G, long long ldg, int N, DevState* st, const double* rhs, double* acc,
                             double alpha, cudaStream_t s);
// acc = (first ? alpha c : acc + alpha c) with (L L^T) c = rhs
// Tensor map over an FP32 factor for the 2-CTA triangular solves (kern_stream.cu).
bool make_factor_tensor_map(void* map_out, const float* L, long long ld, int N);
void launch_trsv_llt(const float* L, long long ldl, int N, const double* rhs, double* acc, int first,
                     double alpha, const float* Wdiag, DevState* st, cudaStream_t s);
// The backward half of that solve, L^T c = z (z = L^{-1} h from chol_factor, FP32):
// acc = (first ? alpha c : acc + alpha c).  Returns false when the pair solve does not
// apply or its launch failed (the caller then solves with launch_trsv_llt from h).
bool launch_trsv_back(const float* L, long long ldl, int N, const float* z, double* acc, int first, double alpha,
                      const float* Wdiag, DevState* st, cudaStream_t s);
// One refinement step of an FP32 solve with its contraction test: acc += c with
// (L L^T) c = rhs, st->refine_ratio = ||c|| / ||acc + c|| and st->newton_bad when it exceeds
// tau.  One launch of the pair solve where it applies (rpart: 2 ceil(N / 32) doubles of
// scratch for its per-row-block partial norms); otherwise the solve into corr (N doubles)
// followed by launch_refine_update.
void launch_trsv_refine(const float* L, long long ldl, int N, const double* rhs, double* acc, double* corr,
                        const float* Wdiag, double* rpart, double tau, DevState* st, cudaStream_t s);

// ---- FP64 Newton system (kern_f64.cu): the Newton matrix formed, factored and solved in FP64,
// used when the FP32 factor fails or its refinement does not contract, or always on request.
// G64: N x N column-major (lower triangle used), ldg64 >= N.
// trans = 0: G64 = diag I + scale A_J^T A_J (N = r); trans = 1: G64 = diag I + scale A_J A_J^T (N = m).
void launch_syrk64(const double* P, long long ldp, int m, int r, int trans, double diag, double scale, double* G64,
                   long long ldg64, const DevState* st, cudaStream_t s);
// Blocked Cholesky G64 = L L^T in place (lower); a non-positive pivot sets st->f64_fail.
void chol64(double* G64, long long ldg64, int N, DevState* st, cudaStream_t s);
// acc = alpha x (first) or acc += alpha x, with L L^T x = rhs (one CTA; skipped after f64_fail).
void launch_trsv64(const double* L, long long ldl, int N, const double* rhs, double* acc, int first, double alpha,
                   const DevState* st, cudaStream_t s);
// acc += c over len entries; writes ||c|| / ||acc + c|| to st->refine_ratio and sets
// st->newton_bad when it exceeds tau (a refinement correction measures the relative
// error of the solution it corrects; above 1/2 the refinement does not contract).
void launch_refine_update(double* acc, const double* c, int len, double tau, DevState* st, cudaStream_t s);

// ---- one pass over A for several fits on the same matrix (kern_multi.cu): t_f = A^T d_f
// with each fit's fused line search, nv <= 4 vectors, element types with FP32
// accumulation (kLaneBf16, kLaneF32, kLaneI8, kLaneI2).  Returns false (nothing
// launched) for an unsupported element type or size.
constexpr int kMultiVectors = 4;
bool launch_stream_multi(int elt, const void* map, int m, long long n, int nv, const double* const* d, double* const* t,
                         const double* const* x, const double* const* u, DevState* const* st,
                         double* const* partials, const ProxParams* pp, double mu, double beta, int max_ls, int fused,
                         int sms, cudaStream_t s, const float* cmean, const float* cscale);

// ---- device-resident batched solver (kern_batch.cu): one persistent kernel, one CTA per
// instance at a time, the whole AL / SsN loop on the device (FP32 storage)
constexpr int kBatchMaxM = 1024;  // rows per instance (the Cholesky panel lives in shared memory)
size_t batch_smem_bytes(int m_max);
size_t batch_slot_bytes(long long n_max, int m_max);
size_t batch_inst_bytes();
size_t batch_out_bytes();
void batch_fill_inst(void* dst, const float* A, long long lda, long long n, int m, const double* b, double lam1,
                     double lam2, double* x);
void batch_read_out(const void* src, ssnal_en_result* r, int* needs_host);
// opt6: sigma0, sigma_growth, sigma_max, mu, beta, tol; opt4: max_al, max_newton, max_ls, refine
bool launch_batch_solve(const void* inst_dev, const int* order_dev, int count, int* next_dev, void* out_dev,
                        const double* opt6, const int* opt4, long long n_max, int m_max, unsigned char* scratch,
                        int blocks, int threads, cudaStream_t s);

// ---- conjugate-gradient Newton solve (kern_cg.cu), m <= 4096
// d = 0, res = p = -g, rr = ||g||^2, stop when ||res|| <= rtol ||g||
void launch_cg_init(const double* g, double* d, double* res, double* p, int m, double rtol, DevState* st,
                    cudaStream_t s);
// one iteration from Vp = (I + kappa A_J A_J^T) p; no-op once DevState::cg_done is set
void launch_cg_step(double* d, double* res, double* p, const double* Vp, int m, DevState* st, cudaStream_t s);

// ---- tensor-core SYRK (kern_tc.cu)
size_t syrk_tc_panel_elems(int R, int K, int nsplit);
size_t syrk_tc_part_floats(int sms);
void launch_syrk_tc(const double* P, long long ldp, int m, int r, int trans, int nsplit, void* Xbuf, float* part,
                    float alpha, float beta, float* out, long long ldo, DevState* st, int sms, cudaStream_t s);

// ---- streams over A (kern_stream.cu)
void launch_stream(int mode, int dtype, const void* A, long long lda, int m, long long n, const double* vec,
                   double* out, const double* x, const double* u, ProxParams pp, double mu, double beta,
                   int max_ls, int fused, DevState* st, double* partials, int grid, cudaStream_t s);
void launch_ls_fallback(const double* x, const double* u, const double* t, long long n, ProxParams pp, double mu,
                        double beta, int max_ls, int fused, DevState* st, double* partials, int grid,
                        cudaStream_t s);
int stream_grid(int sms);
// Tensor map (opaque bytes, tensor_map_bytes() of them) over the pre-split copy.
bool make_split_tensor_map(void* map_out, const void* split, int m, long long n);
size_t tensor_map_bytes();
bool make_elt_tensor_map(void* map_out, const void* A, int dtype, long long lda, int m, long long n);
void launch_stream_lane(int mode, int elt, const void* map, int m, long long n, const double* vec, double* out,
                        const double* x, const double* u, ProxParams pp, double mu, double beta, int max_ls, int fused,
                        DevState* st, double* partials, int sms, cudaStream_t s, const float* cmean = nullptr,
                        const float* cscale = nullptr);
void launch_presplit(const double* A, long long lda, int m, long long n, void* S, int sms, cudaStream_t s);
void launch_check_range(const double* A, long long lda, int m, long long n, int* bad, int sms, cudaStream_t s);

// api.cu: switch the stream of a context (returns the previous one)
cudaStream_t ctx_set_stream(ssnal_en_ctx* c, cudaStream_t s);
double ctx_mn(const ssnal_en_ctx* c);  // m * n of the context's matrix
int64_t ctx_m(const ssnal_en_ctx* c);  // m of the context's matrix
// frees a panel wider than keep_cols columns (regrown on demand)
void ctx_trim(ssnal_en_ctx* c, int64_t keep_cols);

// ---- fits advanced together, one Newton step at a time (api.cu); the passes over A of
// the fits that need one are merged where their contexts share the matrix
struct Fit;
enum { kFitPhaseRunning = 0, kFitPhaseNeedPass = 1, kFitPhaseDone = 2 };
Fit* fit_new();
void fit_delete(Fit* f);
int fit_phase(const Fit* f);
// scaled = 0: penalties (p1, p2); scaled = 1: (alpha, c) = (p1, p2) relative to ||A^T b||_inf
ssnal_en_status fit_start(Fit* f, ssnal_en_ctx* c, const double* b, int scaled, double p1, double p2, double* x,
                          double* lambdas_out);
ssnal_en_status fit_step(Fit* f);                               // until a pass is needed or the fit is done
ssnal_en_status fit_passes(Fit* const* f, int k, int* passes);  // the passes of k fits that need one
ssnal_en_status fit_end(Fit* f, ssnal_en_result* out);          // synchronises the fit's stream

}  // namespace ssnal
