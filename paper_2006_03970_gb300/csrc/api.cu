// Host side of libssnal_en: the C ABI of include/ssnal_en.h, the context and
// its device workspaces, and the AL / SsN control flow of Algorithm 1.  All
// arithmetic on vectors and matrices runs in the kernels of kern_*.cu; the
// host only sequences launches and reads a small status block once per
// Newton step (r, norms, flags) to take the control-flow decisions.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <new>
#include <utility>
#include <vector>

#include "../../include/ssnal_en.h"
#include "internal.h"

using namespace ssnal;

// Phases timed by ssnal_en_profile_phases.
enum { kPhaseGrad = 0, kPhaseNewton = 1, kPhaseStream = 2, kPhaseUpdate = 3, kPhaseRefresh = 4, kPhases = 5 };
static_assert(kPhases == SSNAL_EN_PROFILE_PHASES, "phase count in the header");

struct ssnal_en_ctx {
  int64_t m = 0, n = 0, lda = 0;
  int dtype = 0;
  const void* A = nullptr;
  const float* col_mean = nullptr;
  const float* col_scale = nullptr;
  ssnal_en_options opt;
  cudaStream_t stream = nullptr;
  int sms = 0;
  int grid_stream = 0, grid_vec = 0;
  int ff_ok = 0;       // A's entries allow the float-float stream
  void* Asplit = nullptr;  // float-pair copy of A for the stream (FP64 storage), or null
  int64_t lda_split = 0;
  const void* A_stream = nullptr;  // what the stream reads (A or Asplit) and its leading dimension
  int64_t lda_stream = 0;
  alignas(64) unsigned char tmap[128];  // 2-D TMA tensor map over Asplit
  int tmap_ok = 0;
  int stream_kind = 0;  // kStreamFloatFloat or kStreamDfma (FP64 storage)
  // device workspaces
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned mirror (device-mapped)
  unsigned* st_flag = nullptr;  // pinned: sequence number written after the mirror
  unsigned st_seq = 0;
  double *u = nullptr, *t = nullptr, *xpath = nullptr;
  double *y = nullptr, *d = nullptr, *g = nullptr, *bdev = nullptr, *res = nullptr, *tmpm = nullptr;
  double* bstage = nullptr;  // b of ssnal_en_path_host
  double *h = nullptr, *q = nullptr, *resr = nullptr;  // r-space vectors (capacity rcap)
  int32_t* J = nullptr;
  double* wJ = nullptr;
  long long* counts = nullptr;
  double* partials = nullptr;
  double* vpartials = nullptr;
  double* gemv_part = nullptr;
  double* comb_scratch = nullptr;
  double* cpart = nullptr;      // column-chunk partials of the panel GEMV
  unsigned* tile_ctr = nullptr;  // per-row-tile counters of the panel GEMV
  double* P = nullptr;
  float* P32 = nullptr;
  int64_t ldp = 0, ldp32 = 0, rcap = 0;
  double last_nb1 = 0.0;  // 1 + ||b|| of the last solve's b
  float* G = nullptr;
  int64_t ldg = 0;
  float* Wdiag = nullptr;  // inverses of the factor's 32 x 32 diagonal blocks
  float* zf = nullptr;     // z = L^{-1} h from a factor that ran the forward substitution (m floats)
  double* rpart = nullptr; // per-row-block norms of the refinement step fused into the pair solve
  int last_wdiag = 0;      // the last FP32 factor wrote Wdiag
  double* corr = nullptr;  // first refinement correction (capacity max(m, rcap))
  double* cgp = nullptr;   // search direction of the CG Newton solve (m)
  double* G64 = nullptr;   // FP64 Newton matrix / factor, allocated on first use (m x m)
  int64_t ldg64 = 0;
  float* tuneS = nullptr;  // tuning: factor and identity for tr(G^{-1}) (2 Np x Np), allocated on first use
  double* tune_dev = nullptr;  // tuning: per-column-block partial sums and the result
  float* tuneY = nullptr;      // tuning above N = 640: Y = L^{-1} (Np x Np), allocated on first use
  int64_t tuneY_np = 0;        // its Np
  void* Xtc = nullptr;     // BF16 split panels of the tensor-core SYRK (capacity rcap)
  float* tc_part = nullptr;
  double* Xdev = nullptr;  // path_host output staging
  int64_t Xcap = 0;
  // event timing of the A^T d stream kernel (ssnal_en_profile)
  int prof = 0;
  int64_t prof_seq = 0;  // launches of the A^T d stream since profiling was enabled
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool, ev_pending;
  std::vector<int> ev_phase;  // phase of each pending pair
  double prof_ms = 0.0, prof_bytes = 0.0;
  int64_t prof_launches = 0;
  double phase_ms[kPhases] = {};
  int64_t phase_n[kPhases] = {};
};

namespace {

int64_t round_up(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

// Bytes per stored entry of A (a quarter for 2-bit codes), 0 for an unknown type.
double elem_bytes(int dtype) {
  switch (dtype) {
    case SSNAL_EN_F64: return 8;
    case SSNAL_EN_F32: return 4;
    case SSNAL_EN_BF16: return 2;
    case SSNAL_EN_I8_GENO: return 1;
    case SSNAL_EN_I2_GENO: return 0.25;
    default: return 0;
  }
}
bool is_geno(int dtype) { return dtype == SSNAL_EN_I8_GENO || dtype == SSNAL_EN_I2_GENO; }

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return SSNAL_EN_ECUDA; \
  } while (0)

template <class T>
ssnal_en_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return SSNAL_EN_ENOMEM;
  }
  return SSNAL_EN_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

// Panel capacity: r columns of m rows (FP64 and FP32 copies) plus r-space vectors.
// Capacity grows by doubling while the panel is small next to the m x m system; beyond
// 4 m columns (A_J then holds many times the bytes of the Newton matrix) it grows to the
// need plus an eighth, so that a panel of 1e5 columns does not reserve twice that.
ssnal_en_status grow_panel(ssnal_en_ctx* c, int64_t need) {
  if (need <= c->rcap) return SSNAL_EN_OK;
  int64_t cap = c->rcap > 0 ? c->rcap : 256;
  while (cap < need) cap *= 2;
  if (need > 4 * c->m) cap = (need + need / 8 + 63) / 64 * 64;
  if (cap > c->n) cap = c->n;
  if (cap < need) cap = need;
  cudaStreamSynchronize(c->stream);
  dev_free(c->P);
  dev_free(c->P32);
  dev_free(c->h);
  dev_free(c->q);
  dev_free(c->resr);
  dev_free(c->Xtc);
  dev_free(c->corr);
  c->corr = nullptr;
  c->P = nullptr;
  c->P32 = nullptr;
  c->Xtc = nullptr;
  c->h = c->q = c->resr = nullptr;
  c->rcap = 0;
  ssnal_en_status s;
  if ((s = dev_alloc(&c->P, (size_t)(c->ldp * cap))) != SSNAL_EN_OK) return s;
  if ((s = dev_alloc(&c->P32, (size_t)(c->ldp32 * cap))) != SSNAL_EN_OK) return s;
  if ((s = dev_alloc(&c->h, (size_t)cap)) != SSNAL_EN_OK) return s;
  if ((s = dev_alloc(&c->q, (size_t)cap)) != SSNAL_EN_OK) return s;
  if ((s = dev_alloc(&c->resr, (size_t)cap)) != SSNAL_EN_OK) return s;
  if ((s = dev_alloc(&c->corr, (size_t)(cap > c->m ? cap : c->m))) != SSNAL_EN_OK) return s;
  {
    // both orientations fit in 3 x m x round_up(max(m, cap), 64) BF16 entries
    const int64_t big = c->m > cap ? c->m : cap;
    const size_t elems = 3 * (size_t)c->m * (size_t)((big + 63) / 64 * 64);
    unsigned short* xt = nullptr;
    if ((s = dev_alloc(&xt, elems)) != SSNAL_EN_OK) return s;
    c->Xtc = xt;
  }
  c->rcap = cap;
  return SSNAL_EN_OK;
}

void free_all(ssnal_en_ctx* c) {
  for (auto& pr : c->ev_pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto& pr : c->ev_pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  c->ev_pool.clear();
  c->ev_pending.clear();
  dev_free(c->st);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->st_flag) cudaFreeHost(c->st_flag);
  dev_free(c->u);
  dev_free(c->t);
  dev_free(c->xpath);
  dev_free(c->y);
  dev_free(c->d);
  dev_free(c->g);
  dev_free(c->bdev);
  dev_free(c->res);
  dev_free(c->tmpm);
  dev_free(c->bstage);
  dev_free(c->h);
  dev_free(c->q);
  dev_free(c->resr);
  dev_free(c->J);
  dev_free(c->wJ);
  dev_free(c->counts);
  dev_free(c->partials);
  dev_free(c->vpartials);
  dev_free(c->gemv_part);
  dev_free(c->comb_scratch);
  dev_free(c->cpart);
  dev_free(c->tile_ctr);
  dev_free(c->P);
  dev_free(c->P32);
  dev_free(c->G);
  dev_free(c->Wdiag);
  dev_free(c->zf);
  dev_free(c->rpart);
  dev_free(c->corr);
  dev_free(c->cgp);
  dev_free(c->G64);
  dev_free(c->tuneS);
  dev_free(c->tune_dev);
  dev_free(c->tuneY);
  dev_free(c->Xtc);
  dev_free(c->tc_part);
  dev_free(c->Xdev);
  dev_free(c->Asplit);
}

// Arithmetic of the pass over A: float-float on the pre-split copy when it
// exists, float-float with on-the-fly splitting, or FP64 FMAs (precision = 2 or
// entries outside the range of the split).
void set_stream_kind(ssnal_en_ctx* c) {
  if (c->dtype != SSNAL_EN_F64) {
    // BF16 / FP32 / genotype storage: the lane stream over A itself (tensor map built at create)
    c->stream_kind = kStreamLane;
    c->A_stream = c->A;
    c->lda_stream = c->lda;
    return;
  }
  if (!c->ff_ok || c->opt.precision == 2) {
    c->stream_kind = kStreamDfma;
    c->A_stream = c->A;
    c->lda_stream = c->lda;
  } else if (c->Asplit && c->tmap_ok && c->opt.precision == 0) {
    c->stream_kind = kStreamLane;
    c->A_stream = c->Asplit;
    c->lda_stream = c->lda_split;
  } else if (c->Asplit && c->opt.precision != 3) {
    c->stream_kind = kStreamSplit;
    c->A_stream = c->Asplit;
    c->lda_stream = c->lda_split;
  } else {
    c->stream_kind = kStreamFloatFloat;
    c->A_stream = c->A;
    c->lda_stream = c->lda;
  }
}

bool is_finite_d(double v) { return std::isfinite(v); }

ProxParams make_pp(double sigma, double lam1, double lam2) {
  ProxParams pp;
  pp.sigma = sigma;
  pp.lam1 = lam1;
  pp.lam2 = lam2;
  pp.thr = sigma * lam1;
  pp.onep = 1.0 + sigma * lam2;
  pp.inv_onep = 1.0 / pp.onep;
  return pp;
}

// Profiling level 1 brackets every kProfEvery-th launch of the A^T d stream:
// the events cut the launch off from the programmatic overlap with its
// neighbours, so the fewer launches carry them, the closer the timed loop stays
// to the loop without profiling.
constexpr int64_t kProfEvery = 8;

// Times of the launches recorded since the last synchronisation.
void prof_harvest(ssnal_en_ctx* c) {
  for (size_t k = 0; k < c->ev_pending.size(); k++) {
    auto& pr = c->ev_pending[k];
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      const int ph = c->ev_phase[k];
      if (ph == kPhaseStream) c->prof_ms += ms;
      c->phase_ms[ph] += ms;
      c->phase_n[ph]++;
    }
    c->ev_pool.push_back(pr);
  }
  c->ev_pending.clear();
  c->ev_phase.clear();
}

// The same for the recorded pairs that have completed (in recording order), without
// waiting: called while the device still runs the work queued behind them.
void prof_harvest_ready(ssnal_en_ctx* c) {
  size_t k = 0;
  for (; k < c->ev_pending.size(); k++) {
    auto& pr = c->ev_pending[k];
    if (cudaEventQuery(pr.second) != cudaSuccess) break;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      const int ph = c->ev_phase[k];
      if (ph == kPhaseStream) c->prof_ms += ms;
      c->phase_ms[ph] += ms;
      c->phase_n[ph]++;
    }
    c->ev_pool.push_back(pr);
  }
  cudaGetLastError();  // a pair not yet reached leaves cudaErrorNotReady behind
  c->ev_pending.erase(c->ev_pending.begin(), c->ev_pending.begin() + (long)k);
  c->ev_phase.erase(c->ev_phase.begin(), c->ev_phase.begin() + (long)k);
}

// Event pair around one phase (no-op unless profiling).
struct PhaseTimer {
  ssnal_en_ctx* c;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  int phase;
  PhaseTimer(ssnal_en_ctx* c_, int ph, bool on = true) : c(c_), phase(ph) {
    // level 1 times the passes over A only: one A^T d pass in kProfEvery and every
    // u = A^T y pass (a few per fit)
    if (!on || !c->prof || (ph != kPhaseStream && ph != kPhaseRefresh && c->prof < 2)) {
      c = nullptr;
      return;
    }
    if (c->ev_pool.empty()) {
      if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
        c = nullptr;
        return;
      }
    } else {
      ev = c->ev_pool.back();
      c->ev_pool.pop_back();
    }
    cudaEventRecord(ev.first, c->stream);
  }
  ~PhaseTimer() {
    if (!c || !c->prof) return;
    cudaEventRecord(ev.second, c->stream);
    c->ev_pending.push_back(ev);
    c->ev_phase.push_back(phase);
  }
};

// The state after the work queued so far.  A kernel behind that work writes the
// state into the host mirror and then a sequence number, which this thread
// polls: no copy-engine transfer and no blocking wake-up on the common path (the
// work between two reads is a few microseconds to a few milliseconds: one Newton
// step's prox / gather / gradient kernels, or a Newton step and a pass over A).
// The poll checks the stream for errors now and then and, after kPollMax, falls
// back to a blocking synchronisation.  Recorded profiling events are waited for
// before they are read.
constexpr std::chrono::microseconds kPollMax(20000);
ssnal_en_status read_state(ssnal_en_ctx* c) {
  if (!c->st_flag) {
    CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!c->ev_pending.empty()) prof_harvest(c);
    return SSNAL_EN_OK;
  }
  const unsigned want = ++c->st_seq;
  launch_state_out(c->st, c->st_host, c->st_flag, want, c->stream);
  CK(cudaGetLastError());
  if (!c->ev_pending.empty()) prof_harvest_ready(c);
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned it = 1;; it++) {
    if (__atomic_load_n(c->st_flag, __ATOMIC_ACQUIRE) == want) break;
    if ((it & 1023) == 0) {
      const cudaError_t e = cudaStreamQuery(c->stream);
      if (e == cudaSuccess) {  // the stream has drained: the flag must be there
        if (__atomic_load_n(c->st_flag, __ATOMIC_ACQUIRE) != want) return SSNAL_EN_ECUDA;
        break;
      }
      if (e != cudaErrorNotReady) return SSNAL_EN_ECUDA;
      if (std::chrono::steady_clock::now() - t0 > kPollMax) {
        CK(cudaStreamSynchronize(c->stream));
        if (__atomic_load_n(c->st_flag, __ATOMIC_ACQUIRE) != want) return SSNAL_EN_ECUDA;
        break;
      }
    }
  }
  return SSNAL_EN_OK;
}

// One pass over A with the arithmetic and layout chosen at create time.
// Element type and accumulation of a lane-stream pass.  FP64 storage: the
// pre-split copy in float-float.  BF16 / FP32 storage: float-float for u = A^T y
// and max|A^T b| (the values the KKT test and the x update use); the Newton
// passes t = A^T d accumulate in FP32 in the mixed precision mode.
int lane_elt(const ssnal_en_ctx* c, int mode) {
  const bool plain = c->opt.precision == 1 && mode == kModeT;
  if (c->dtype == SSNAL_EN_BF16) return plain ? kLaneBf16 : kLaneBf16FF;
  if (c->dtype == SSNAL_EN_F32) return plain ? kLaneF32 : kLaneF32FF;
  if (c->dtype == SSNAL_EN_I8_GENO) return plain ? kLaneI8 : kLaneI8FF;
  if (c->dtype == SSNAL_EN_I2_GENO) return plain ? kLaneI2 : kLaneI2FF;
  return kLaneSplit;
}

// True when the Newton passes are accumulated in FP32: u then drifts from A^T y
// by FP32 rounding and is recomputed before the KKT test.
bool mixed_stream(const ssnal_en_ctx* c) {
  return c->opt.precision == 1 && c->dtype != SSNAL_EN_F64;
}

// BF16 parts per panel entry in the tensor-core SYRK: a BF16-stored A_J is
// exact in one part (one product per pair of entries); FP64 / FP32 need three.
int syrk_splits(const ssnal_en_ctx* c) { return c->dtype == SSNAL_EN_BF16 ? 1 : 3; }

void run_stream(ssnal_en_ctx* c, int mode, const double* vec, double* out, const double* x, const double* u,
                ProxParams pp) {
  const ssnal_en_options& o = c->opt;
  if (c->stream_kind == kStreamLane)
    launch_stream_lane(mode, lane_elt(c, mode), c->tmap, (int)c->m, c->n, vec, out, x, u, pp, o.mu, o.beta, o.max_ls,
                       o.ls_fused, c->st, c->partials, c->sms, c->stream, c->col_mean, c->col_scale);
  else
    launch_stream(mode, c->stream_kind, c->A_stream, c->lda_stream, (int)c->m, c->n, vec, out, x, u, pp, o.mu,
                  o.beta, o.max_ls, o.ls_fused, c->st, c->partials, c->grid_stream, c->stream);
}

// The A^T d stream of one Newton step, bracketed by CUDA events when profiling
// (at level 1 every kProfEvery-th launch, at level 2 every launch).
ssnal_en_status stream_t(ssnal_en_ctx* c, const double* x, ProxParams pp) {
  const bool timed = c->prof >= 2 || (c->prof == 1 && c->prof_seq++ % kProfEvery == 0);
  {
    PhaseTimer timer(c, kPhaseStream, timed);
    run_stream(c, kModeT, c->d, c->t, x, c->u, pp);
  }
  if (timed) {
    c->prof_launches++;
    const double es = elem_bytes(c->dtype);
    c->prof_bytes += (double)c->m * (double)c->n * es + 3.0 * 8.0 * (double)c->n + 8.0 * (double)c->m;
  }
  return SSNAL_EN_OK;
}

// ---- pieces of the SsN step ------------------------------------------------

// J, w_J at the current (x, u) (or the support of x in support mode), gather
// of A_J, and g = y + b - A_J w_J (or y = A_J x_J - b in support mode).
void launch_grad(ssnal_en_ctx* c, int mode, const double* b, long long r_host) {
  const int m = (int)c->m;
  if (mode == kProxSupport)
    launch_gemv_n(c->P, c->ldp, m, c->wJ, c->st, r_host, c->rcap, c->y, nullptr, 0.0, b, -1.0, 1.0, 0, nullptr,
                  nullptr, nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, c->stream);
  else
    launch_gemv_n(c->P, c->ldp, m, c->wJ, c->st, r_host, c->rcap, c->g, c->y, 1.0, b, 1.0, -1.0, 1, c->y, b,
                  nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, c->stream);
}

ssnal_en_status prox_gather_grad(ssnal_en_ctx* c, int mode, const double* x, const double* b, ProxParams pp,
                                 int apply_update) {
  cudaStream_t s = c->stream;
  {
  PhaseTimer timer(c, kPhaseGrad);
  launch_prox_count(mode, x, c->u, c->t, c->y, c->d, c->n, (int)c->m, pp, apply_update, c->st, c->counts,
                    c->vpartials, c->grid_vec, s);
  launch_prox_scatter(mode, x, c->u, c->n, pp, c->counts, c->vpartials, c->st, c->J, c->wJ, c->grid_vec, s);
  launch_gather(c->A, c->dtype, c->lda, (int)c->m, c->J, c->st, -1, c->rcap, c->P, c->ldp, c->P32, c->ldp32, c->sms,
                s, c->col_mean, c->col_scale);
  launch_grad(c, mode, b, -1);
  }
  CK(cudaGetLastError());
  ssnal_en_status st = read_state(c);
  if (st != SSNAL_EN_OK) return st;
  if (c->st_host->timeout) return SSNAL_EN_ETIMEOUT;
  if (c->st_host->overflow) {
    // the panel was too small for r: grow it and redo the gather and the GEMV
    int64_t r = c->st_host->r;
    if ((st = grow_panel(c, r)) != SSNAL_EN_OK) return st;
    CK(cudaMemsetAsync(&c->st->overflow, 0, sizeof(int32_t), s));
    launch_gather(c->A, c->dtype, c->lda, (int)c->m, c->J, c->st, r, c->rcap, c->P, c->ldp, c->P32, c->ldp32,
                  c->sms, s, c->col_mean, c->col_scale);
    launch_grad(c, mode, b, r);
    CK(cudaGetLastError());
    if ((st = read_state(c)) != SSNAL_EN_OK) return st;
  }
  return SSNAL_EN_OK;
}

// Contraction test of the FP32 solve.  The first refinement correction relative to the
// refined solution, rho, estimates the relative error of the FP32 solve and the factor by
// which each refinement step shrinks it (the error of the FP32 factor of a matrix formed
// with FP32 accumulation is of the order of cond(G) 2^-24, times a growth with the
// accumulation length).  rho > kRefineTau: the refinement does not contract and the
// Newton step is redone with the FP64 system.  rho > kRefineMore: the direction is still
// usable (its error after one step is about rho^2) but later steps of the fit take one
// more refinement step (at most kRefineExtraMax more).
constexpr double kRefineTau = 0.5;
constexpr double kRefineMore = 1e-2;
constexpr int kRefineExtraMax = 2;

// Newton direction d for (I + kappa A_J A_J^T) d = -g on the gathered panel:
// FP32 SYRK and Cholesky factor of the Newton matrix, FP64 residuals through
// the panel (iterative refinement), and the dot products the line search needs.
ssnal_en_status newton_direction(ssnal_en_ctx* c, int64_t r, double kappa, const double* g, double* d,
                                 const double* yv, const double* bv, int dots, int extra_refine = 0) {
  cudaStream_t s = c->stream;
  PhaseTimer timer(c, kPhaseNewton);
  const int m = (int)c->m;
  const int refine = (c->opt.refine_steps > 0 ? c->opt.refine_steps : 0) + extra_refine;
  const int which = dots ? 2 : 0;
  const float* wd = nullptr;  // inverse diagonal blocks of the factor, when available
  if (r == 0) {
    launch_gemv_n(c->P, c->ldp, m, c->wJ, c->st, 0, c->rcap, d, nullptr, 0.0, g, -1.0, 0.0, which, yv, bv, g, c->st,
                  c->comb_scratch, c->cpart, c->tile_ctr, s);
  } else if (r < m) {
    // SMW (eq. smw_formula): G = kappa^{-1} I + A_J^T A_J, h = A_J^T g, q = G^{-1} h, d = A_J q - g
    const int N = (int)r;
    if (c->opt.syrk_tc)
      launch_syrk_tc(c->P, c->ldp, m, (int)r, 0, syrk_splits(c), c->Xtc, c->tc_part, 1.0f, (float)(1.0 / kappa), c->G,
                     c->ldg, c->st, c->sms, s);
    else
      launch_syrk_tn(c->P32, c->ldp32, m, r, 1.0 / kappa, c->G, c->ldg, s);
    launch_gemv_t(c->P, c->ldp, m, r, g, c->h, nullptr, 0.0, nullptr, 0.0, 1.0, c->sms, s);
    if (N <= kSmallNewton) {
      launch_chol_solve_small(c->G, c->ldg, N, c->st, c->h, c->q, 1.0, s);
      c->last_wdiag = 0;
    } else {
      // the factor runs the forward substitution of h where it can (z in zf)
      bool fused = false;
      wd = chol_factor(c->G, c->ldg, N, c->st, c->Wdiag, s, c->h, c->zf, &fused) ? c->Wdiag : nullptr;
      c->last_wdiag = wd != nullptr;
      if (!(fused && wd && launch_trsv_back(c->G, c->ldg, N, c->zf, c->q, 1, 1.0, wd, c->st, s)))
        launch_trsv_llt(c->G, c->ldg, N, c->h, c->q, 1, 1.0, wd, c->st, s);
    }
    for (int it = 0; it < refine; it++) {
      // resr = h - kappa^{-1} q - A_J^T (A_J q)
      launch_gemv_n(c->P, c->ldp, m, c->q, c->st, r, c->rcap, c->tmpm, nullptr, 0.0, nullptr, 0.0, 1.0, 0, nullptr,
                    nullptr, nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
      launch_gemv_t(c->P, c->ldp, m, r, c->tmpm, c->resr, c->h, 1.0, c->q, -1.0 / kappa, -1.0, c->sms, s);
      if (it == 0) {  // the first correction is the FP32 solve's error: test the contraction
        launch_trsv_refine(c->G, c->ldg, N, c->resr, c->q, c->corr, wd, c->rpart, kRefineTau, c->st, s);
      } else {
        launch_trsv_llt(c->G, c->ldg, N, c->resr, c->q, 0, 1.0, wd, c->st, s);
      }
    }
    launch_gemv_n(c->P, c->ldp, m, c->q, c->st, r, c->rcap, d, nullptr, 0.0, g, -1.0, 1.0, which, yv, bv, g, c->st,
                  c->comb_scratch, c->cpart, c->tile_ctr, s);
  } else {
    // m x m form (eq. AJ_system): M = I + kappa A_J A_J^T, d = -M^{-1} g
    if (c->opt.syrk_tc)
      launch_syrk_tc(c->P, c->ldp, m, (int)r, 1, syrk_splits(c), c->Xtc, c->tc_part, (float)kappa, 1.0f, c->G, c->ldg,
                     c->st,
                     c->sms, s);
    else
      launch_syrk_nt(c->P32, c->ldp32, m, r, kappa, c->G, c->ldg, s);
    if (m <= kSmallNewton) {
      launch_chol_solve_small(c->G, c->ldg, m, c->st, g, d, -1.0, s);
      c->last_wdiag = 0;
    } else {
      bool fused = false;
      wd = chol_factor(c->G, c->ldg, m, c->st, c->Wdiag, s, g, c->zf, &fused) ? c->Wdiag : nullptr;
      c->last_wdiag = wd != nullptr;
      if (!(fused && wd && launch_trsv_back(c->G, c->ldg, m, c->zf, d, 1, -1.0, wd, c->st, s)))
        launch_trsv_llt(c->G, c->ldg, m, g, d, 1, -1.0, wd, c->st, s);
    }
    for (int it = 0; it < refine; it++) {
      // tmpm = -g - d - kappa A_J (A_J^T d)
      launch_gemv_t(c->P, c->ldp, m, r, d, c->h, nullptr, 0.0, nullptr, 0.0, 1.0, c->sms, s);
      launch_gemv_n(c->P, c->ldp, m, c->h, c->st, r, c->rcap, c->tmpm, g, -1.0, d, -1.0, -kappa, 0, nullptr, nullptr,
                    nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
      if (it == 0) {
        launch_trsv_refine(c->G, c->ldg, m, c->tmpm, d, c->corr, wd, c->rpart, kRefineTau, c->st, s);
      } else {
        launch_trsv_llt(c->G, c->ldg, m, c->tmpm, d, 0, 1.0, wd, c->st, s);
      }
    }
    if (dots)
      launch_combine(d, nullptr, 0.0, d, 1.0, nullptr, 0.0, m, 2, yv, bv, g, c->st, c->comb_scratch, s);
  }
  CK(cudaGetLastError());
  return SSNAL_EN_OK;
}

// One more refinement step of the last FP32 solve (same panel, factor and g): the FP64
// residual through the panel, an FP32 correction and the contraction test.  The
// solution is q (r-space, SMW form) or d (m x m form).
ssnal_en_status refine_once(ssnal_en_ctx* c, int64_t r, double kappa, const double* g, double* d) {
  cudaStream_t s = c->stream;
  const int m = (int)c->m;
  const float* wd = c->last_wdiag ? c->Wdiag : nullptr;
  if (r == 0) return SSNAL_EN_OK;
  if (r < m) {
    const int N = (int)r;
    launch_gemv_n(c->P, c->ldp, m, c->q, c->st, r, c->rcap, c->tmpm, nullptr, 0.0, nullptr, 0.0, 1.0, 0, nullptr,
                  nullptr, nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
    launch_gemv_t(c->P, c->ldp, m, r, c->tmpm, c->resr, c->h, 1.0, c->q, -1.0 / kappa, -1.0, c->sms, s);
    launch_trsv_refine(c->G, c->ldg, N, c->resr, c->q, c->corr, wd, c->rpart, kRefineTau, c->st, s);
    launch_gemv_n(c->P, c->ldp, m, c->q, c->st, r, c->rcap, d, nullptr, 0.0, g, -1.0, 1.0, 0, nullptr, nullptr,
                  nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
  } else {
    launch_gemv_t(c->P, c->ldp, m, r, d, c->h, nullptr, 0.0, nullptr, 0.0, 1.0, c->sms, s);
    launch_gemv_n(c->P, c->ldp, m, c->h, c->st, r, c->rcap, c->tmpm, g, -1.0, d, -1.0, -kappa, 0, nullptr, nullptr,
                  nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
    launch_trsv_refine(c->G, c->ldg, m, c->tmpm, d, c->corr, wd, c->rpart, kRefineTau, c->st, s);
  }
  CK(cudaGetLastError());
  return SSNAL_EN_OK;
}

// The FP64 Newton matrix (m x m doubles), allocated the first time a context needs it.
ssnal_en_status ensure_g64(ssnal_en_ctx* c) {
  if (c->G64) return SSNAL_EN_OK;
  c->ldg64 = round_up(c->m, 2);
  return dev_alloc(&c->G64, (size_t)c->ldg64 * (size_t)c->m);
}

// Newton direction with the FP64 system: the Newton matrix of eq. smw_formula (r < m) or
// eq. AJ_system (r >= m) formed from the FP64 panel with FP64 FMAs, its FP64 Cholesky
// factor and FP64 triangular solves (kern_f64.cu); then the same final GEMV and scalar
// products as the FP32 path.  A non-positive FP64 pivot sets DevState::f64_fail.
ssnal_en_status newton_direction_f64(ssnal_en_ctx* c, int64_t r, double kappa, const double* g, double* d,
                                     const double* yv, const double* bv, int dots) {
  cudaStream_t s = c->stream;
  ssnal_en_status e = ensure_g64(c);
  if (e != SSNAL_EN_OK) return e;
  PhaseTimer timer(c, kPhaseNewton);
  const int m = (int)c->m;
  const int which = dots ? 2 : 0;
  if (r == 0) {
    launch_gemv_n(c->P, c->ldp, m, c->wJ, c->st, 0, c->rcap, d, nullptr, 0.0, g, -1.0, 0.0, which, yv, bv, g, c->st,
                  c->comb_scratch, c->cpart, c->tile_ctr, s);
  } else if (r < m) {
    // G = kappa^{-1} I + A_J^T A_J, h = A_J^T g, q = G^{-1} h, d = A_J q - g
    const int N = (int)r;
    launch_syrk64(c->P, c->ldp, m, N, 0, 1.0 / kappa, 1.0, c->G64, c->ldg64, c->st, s);
    launch_gemv_t(c->P, c->ldp, m, r, g, c->h, nullptr, 0.0, nullptr, 0.0, 1.0, c->sms, s);
    chol64(c->G64, c->ldg64, N, c->st, s);
    launch_trsv64(c->G64, c->ldg64, N, c->h, c->q, 1, 1.0, c->st, s);
    launch_gemv_n(c->P, c->ldp, m, c->q, c->st, r, c->rcap, d, nullptr, 0.0, g, -1.0, 1.0, which, yv, bv, g, c->st,
                  c->comb_scratch, c->cpart, c->tile_ctr, s);
  } else {
    // M = I + kappa A_J A_J^T, d = -M^{-1} g
    launch_syrk64(c->P, c->ldp, m, (int)r, 1, 1.0, kappa, c->G64, c->ldg64, c->st, s);
    chol64(c->G64, c->ldg64, m, c->st, s);
    launch_trsv64(c->G64, c->ldg64, m, g, d, 1, -1.0, c->st, s);
    if (dots)
      launch_combine(d, nullptr, 0.0, d, 1.0, nullptr, 0.0, m, 2, yv, bv, g, c->st, c->comb_scratch, s);
  }
  CK(cudaGetLastError());
  return SSNAL_EN_OK;
}

// True when the Newton system of this step is solved by conjugate gradients: m and r both
// above options.cg_above (Algorithm 1 step (1); Sec. 3.2 proposes CG when both exceed 1e4).
bool use_cg(const ssnal_en_ctx* c, int64_t r) { return c->m > c->opt.cg_above && r > c->opt.cg_above; }

constexpr int kCgBatch = 8;  // CG iterations launched between two reads of the state

// Newton direction by conjugate gradients on (I + kappa A_J A_J^T) d = -g, matrix-free
// (V p = p + kappa A_J (A_J^T p) by the panel GEMV pair), FP64 throughout.  The scalars
// stay on the device; the host reads the state once per kCgBatch iterations and stops
// at the stopping test or after cg_maxit (default 10 m) iterations.  *iters receives
// the iteration count.
ssnal_en_status newton_direction_cg(ssnal_en_ctx* c, int64_t r, double kappa, const double* g, double* d,
                                    const double* yv, const double* bv, int dots, int* iters) {
  cudaStream_t s = c->stream;
  const int m = (int)c->m;
  const int64_t maxit = c->opt.cg_maxit > 0 ? c->opt.cg_maxit : 10 * c->m;
  {
    PhaseTimer timer(c, kPhaseNewton);
    launch_cg_init(g, d, c->res, c->cgp, m, c->opt.cg_rtol, c->st, s);
  }
  CK(cudaGetLastError());
  int64_t launched = 0;
  for (;;) {
    const int64_t batch = maxit - launched < kCgBatch ? maxit - launched : kCgBatch;
    {
      PhaseTimer timer(c, kPhaseNewton);
      for (int64_t k = 0; k < batch; k++) {
        // tmpm = p + kappa A_J (A_J^T p)
        launch_gemv_t(c->P, c->ldp, m, r, c->cgp, c->h, nullptr, 0.0, nullptr, 0.0, 1.0, c->sms, s);
        launch_gemv_n(c->P, c->ldp, m, c->h, c->st, r, c->rcap, c->tmpm, c->cgp, 1.0, nullptr, 0.0, kappa, 0,
                      nullptr, nullptr, nullptr, c->st, c->comb_scratch, c->cpart, c->tile_ctr, s);
        launch_cg_step(d, c->res, c->cgp, c->tmpm, m, c->st, s);
      }
    }
    CK(cudaGetLastError());
    launched += batch;
    ssnal_en_status e = read_state(c);
    if (e != SSNAL_EN_OK) return e;
    if (c->st_host->cg_done || launched >= maxit) break;
  }
  *iters = c->st_host->cg_iters;
  if (dots) {
    PhaseTimer timer(c, kPhaseNewton);
    launch_combine(d, nullptr, 0.0, d, 1.0, nullptr, 0.0, m, 2, yv, bv, g, c->st, c->comb_scratch, s);
  }
  CK(cudaGetLastError());
  return SSNAL_EN_OK;
}

// Clears DevState::chol_fail, newton_bad and f64_fail (contiguous).
ssnal_en_status clear_newton_flags(ssnal_en_ctx* c) {
  CK(cudaMemsetAsync(&c->st->chol_fail, 0, 3 * sizeof(int32_t), c->stream));
  return SSNAL_EN_OK;
}

// One fit (Algorithm 1) as a resumable state machine.  fit_begin starts the fit (the
// initial dual iterate and u = A^T y); fit_advance runs the host side of the SsN / AL
// loop -- prox / active set / gradient with the state read, the stopping tests, the AL
// update and the Newton direction -- until the fit needs its pass over A (t = A^T d with
// the fused line search: NeedPass) or has finished (Done); fit_after_pass queues the
// line-search trials the pass did not evaluate.  A single fit alternates fit_advance
// and stream_t (solve_impl); several fits on one matrix share their passes
// (solve_group).  The kernels each fit launches, and their order, are the same either
// way, so a fit's iterates do not depend on how its passes are taken.
enum FitPhase { kFitRunning = 0, kFitNeedPass = 1, kFitDone = 2 };

struct FitState {
  ssnal_en_ctx* c = nullptr;
  const double* b = nullptr;
  double lam1 = 0.0, lam2 = 0.0;
  double* x = nullptr;
  double* y_io = nullptr;
  ssnal_en_result R{};
  std::chrono::steady_clock::time_point t0;
  double nb1 = 0.0;
  ProxParams pp{};
  double sigma = 0.0, kappa = 0.0;
  int al = 0, apply = 0, newton_here = 0;
  bool fresh = true;
  // Newton systems in FP64: always on request; otherwise from the first step whose FP32
  // factor failed or whose refinement did not contract to the end of this fit (sigma
  // only grows within a fit, so the FP32 system would not recover).
  bool use_f64 = false;
  int extra_refine = 0;  // refinement steps added after a slowly contracting FP32 solve
  double kkt1 = INFINITY, kkt3 = INFINITY;
  int converged = 0, failed = 0;
  int phase = kFitRunning;
};

void fit_al_begin(FitState& F) {
  F.pp = make_pp(F.sigma, F.lam1, F.lam2);
  F.kappa = F.sigma / (1.0 + F.sigma * F.lam2);
  F.apply = 0;
  F.newton_here = 0;
  F.fresh = true;  // u = A^T y to the stream's full accuracy (false after FP32-accumulated steps)
}

// nb1_known > 0: 1 + ||b|| of this b, already known (points of one path); else it is
// computed here (one host round trip).  atb (may be null): A^T b of this b, just formed by
// the ||A^T b||_inf pass with the arithmetic of the u = A^T y pass; when the fit starts at
// x = 0 (y0 = -b) the initial u is then -atb, bitwise what the pass over A would give (the
// pass is odd in its vector: the split, the products and every sum change sign exactly).
ssnal_en_status fit_begin(FitState& F, ssnal_en_ctx* c, const double* b, double lam1, double lam2, double* x,
                          double* y_io, double nb1_known, const double* atb = nullptr) {
  F = FitState();
  F.c = c;
  F.b = b;
  F.lam1 = lam1;
  F.lam2 = lam2;
  F.x = x;
  F.y_io = y_io;
  F.t0 = std::chrono::steady_clock::now();
  F.R.lambda1 = lam1;
  F.R.lambda2 = lam2;
  const ssnal_en_options& o = c->opt;
  cudaStream_t s = c->stream;
  const int m = (int)c->m;
  launch_solve_begin(c->st, c->bdev, b, m, s);  // state := 0, bdev := b
  ssnal_en_status e = SSNAL_EN_OK;
  double nb1 = nb1_known;
  if (!(nb1 > 0.0)) {
    // ||b|| via the combine kernel's scalar products (y := b temporarily)
    launch_combine(c->tmpm, c->bdev, 1.0, nullptr, 0.0, nullptr, 0.0, m, 1, c->bdev, c->bdev, nullptr, c->st,
                   c->comb_scratch, s);
    if ((e = read_state(c)) != SSNAL_EN_OK) return e;
    nb1 = 1.0 + sqrt(c->st_host->g2);
  }
  c->last_nb1 = nb1;
  F.nb1 = nb1;
  // ---- initial dual iterate and u = A^T y (reading: y0 = A x0 - b)
  ProxParams pp = make_pp(o.sigma0, lam1, lam2);
  bool cold = false;  // x0 = 0, so y0 = -b
  if (o.use_y0 && y_io) {
    CK(cudaMemcpyAsync(c->y, y_io, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  } else {
    if ((e = prox_gather_grad(c, kProxSupport, x, c->bdev, pp, 0)) != SSNAL_EN_OK) return e;
    cold = c->st_host->r == 0;
  }
  if (cold && atb) {
    launch_neg_f64(c->u, atb, c->n, c->sms, s);
  } else {
    PhaseTimer timer(c, kPhaseRefresh);
    run_stream(c, kModeU, c->y, c->u, nullptr, nullptr, pp);
  }
  CK(cudaGetLastError());
  F.sigma = o.sigma0;
  F.use_f64 = o.newton_fp64 == 1;
  F.al = 1;
  fit_al_begin(F);
  return SSNAL_EN_OK;
}

ssnal_en_status fit_advance(FitState& F) {
  ssnal_en_ctx* c = F.c;
  const ssnal_en_options& o = c->opt;
  cudaStream_t s = c->stream;
  ssnal_en_status e = SSNAL_EN_OK;
  F.phase = kFitRunning;
  while (F.al <= o.max_al) {
    // ---- SsN loop of AL iteration F.al (Algorithm 1, lower half)
    bool stop_ssn = false;
    for (;;) {
      if ((e = prox_gather_grad(c, kProxThreshold, F.x, c->bdev, F.pp, F.apply)) != SSNAL_EN_OK) return e;
      const DevState& h = *c->st_host;
      if (F.apply) F.R.ls_trials += h.ls_k + 1;
      F.apply = 0;
      if (h.chol_fail | h.newton_bad | h.f64_fail) {
        // The last direction came from an unreliable FP32 solve (non-positive pivot, or a
        // refinement that does not contract) or a failed FP64 factor; the prox pass above
        // did not apply it, so y and u are those of the step before.
        if (h.f64_fail) {  // the Newton matrix is not positive definite even in FP64
          F.failed = 1;
          stop_ssn = true;
          break;
        }
        if ((e = clear_newton_flags(c)) != SSNAL_EN_OK) return e;
        F.use_f64 = true;  // recompute this direction, and the rest of the fit, in FP64
      } else if (h.refine_ratio > kRefineMore && F.extra_refine < kRefineExtraMax && o.refine_steps > 0) {
        F.extra_refine++;  // the FP32 solve contracts slowly: one more refinement step from now on
      }
      const double gn = sqrt(h.g2) / F.nb1;
      if (!(gn > o.tol) || F.newton_here >= o.max_newton) {
        if (!F.fresh) {
          // mixed precision: recompute u = A^T y in float-float before the SsN
          // stopping test is trusted (the KKT residuals and the x update read u)
          {
            PhaseTimer timer(c, kPhaseRefresh);
            run_stream(c, kModeU, c->y, c->u, nullptr, nullptr, F.pp);
          }
          CK(cudaGetLastError());
          F.fresh = true;
          continue;
        }
        stop_ssn = true;
        break;
      }
      F.fresh = !mixed_stream(c);
      const int64_t r = h.r;
      if (use_cg(c, r)) {
        int it = 0;
        if ((e = newton_direction_cg(c, r, F.kappa, c->g, c->d, c->y, c->bdev, 1, &it)) != SSNAL_EN_OK) return e;
        F.R.cg_iters += it;
      } else if (F.use_f64) {
        if ((e = newton_direction_f64(c, r, F.kappa, c->g, c->d, c->y, c->bdev, 1)) != SSNAL_EN_OK) return e;
        F.R.newton_fp64++;
      } else if ((e = newton_direction(c, r, F.kappa, c->g, c->d, c->y, c->bdev, 1, F.extra_refine)) !=
                 SSNAL_EN_OK) {
        return e;
      }
      F.phase = kFitNeedPass;  // the caller runs t = A^T d with the fused line search
      return SSNAL_EN_OK;
    }
    (void)stop_ssn;
    const DevState& h = *c->st_host;
    // AL step (2) via the Moreau decomposition; residuals of eq. kkt_res.
    F.kkt1 = sqrt(h.g2) / F.nb1;
    const double aty_z = sqrt(h.xw2) / F.sigma;
    const double znorm = sqrt(h.vw2) / F.sigma;
    F.kkt3 = aty_z / (1.0 + sqrt(h.y2) + znorm);
    F.R.active = h.r;
    F.R.primal_obj = 0.5 * h.yg2 + F.lam1 * h.w1 + 0.5 * F.lam2 * h.w2;
    const double dual = -(0.5 * h.y2 + h.by) - (F.lam2 > 0 ? h.dualpen / (2.0 * F.lam2) : 0.0);
    F.R.dual_gap = F.lam2 > 0 ? F.R.primal_obj - dual : NAN;
    F.R.sigma = F.sigma;
    {
      PhaseTimer timer(c, kPhaseUpdate);
      launch_set_x(F.x, c->u, c->n, F.pp, c->sms, s);
    }
    CK(cudaGetLastError());
    if (F.failed) break;
    if (F.kkt1 <= o.tol && F.kkt3 <= o.tol) {
      F.converged = 1;
      break;
    }
    F.sigma = fmin(F.sigma * o.sigma_growth, o.sigma_max);
    F.al++;
    if (F.al <= o.max_al) fit_al_begin(F);
  }
  F.phase = kFitDone;
  return SSNAL_EN_OK;
}

// After the pass over A of a Newton step: the trials the pass did not evaluate.
ssnal_en_status fit_after_pass(FitState& F) {
  ssnal_en_ctx* c = F.c;
  const ssnal_en_options& o = c->opt;
  launch_ls_fallback(F.x, c->u, c->t, c->n, F.pp, o.mu, o.beta, o.max_ls, o.ls_fused, c->st, c->partials,
                     c->grid_stream, c->stream);
  CK(cudaGetLastError());
  F.apply = 1;
  F.newton_here++;
  F.R.newton_iters++;
  return SSNAL_EN_OK;
}

ssnal_en_status fit_finish(FitState& F, ssnal_en_result* out) {
  ssnal_en_ctx* c = F.c;
  const ssnal_en_options& o = c->opt;
  cudaStream_t s = c->stream;
  if (F.y_io) CK(cudaMemcpyAsync(F.y_io, c->y, sizeof(double) * c->m, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  F.R.al_iters = F.al > o.max_al ? o.max_al : F.al;
  F.R.kkt1 = F.kkt1;
  F.R.kkt3 = F.kkt3;
  F.R.status = F.converged ? SSNAL_EN_OK : SSNAL_EN_ENOCONV;
  F.R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - F.t0).count();
  if (out) *out = F.R;
  return F.converged ? SSNAL_EN_OK : SSNAL_EN_ENOCONV;
}

// nb1_known > 0: 1 + ||b|| of this b, already known (points of one path); else it is
// computed here (one host round trip).
ssnal_en_status solve_impl(ssnal_en_ctx* c, const double* b, double lam1, double lam2, double* x, double* y_io,
                           ssnal_en_result* out, double nb1_known = 0.0, const double* atb = nullptr) {
  FitState F;
  ssnal_en_status e = fit_begin(F, c, b, lam1, lam2, x, y_io, nb1_known, atb);
  if (e != SSNAL_EN_OK) return e;
  for (;;) {
    if ((e = fit_advance(F)) != SSNAL_EN_OK) return e;
    if (F.phase == kFitDone) break;
    if ((e = stream_t(c, F.x, F.pp)) != SSNAL_EN_OK) return e;
    if ((e = fit_after_pass(F)) != SSNAL_EN_OK) return e;
  }
  return fit_finish(F, out);
}

// True when the contexts of fits[0..k) stream the same matrix with the same element
// type and line-search options, so that their Newton-step passes can be merged.
bool can_merge(FitState* const* fits, int k) {
  const ssnal_en_ctx* a = fits[0]->c;
  if (a->stream_kind != kStreamLane || !a->tmap_ok) return false;
  const int elt = lane_elt(a, kModeT);
  if (elt != kLaneBf16 && elt != kLaneF32 && elt != kLaneI8 && elt != kLaneI2) return false;
  for (int i = 1; i < k; i++) {
    const ssnal_en_ctx* b = fits[i]->c;
    if (b->A != a->A || b->m != a->m || b->n != a->n || b->lda != a->lda || b->dtype != a->dtype ||
        b->col_mean != a->col_mean || b->col_scale != a->col_scale || lane_elt(b, kModeT) != elt ||
        b->stream_kind != kStreamLane || !b->tmap_ok || b->opt.mu != a->opt.mu || b->opt.beta != a->opt.beta ||
        b->opt.max_ls != a->opt.max_ls || b->opt.ls_fused != a->opt.ls_fused || b->stream != a->stream)
      return false;
  }
  return true;
}

// The Newton-step passes of the fits that need one: merged into passes of up to
// kMultiVectors fits where the contexts allow (same matrix, FP32-accumulated pass,
// same stream), else one pass per fit; then each fit's remaining trials.  *passes
// receives the number of passes over A.
ssnal_en_status run_passes(FitState* const* fits, int k, int* passes) {
  ssnal_en_status e = SSNAL_EN_OK;
  int np = 0;
  const bool merge = k > 1 && can_merge(fits, k);
  for (int i0 = 0; i0 < k;) {
    const int nv = merge ? (k - i0 < kMultiVectors ? k - i0 : kMultiVectors) : 1;
    bool done = false;
    if (nv > 1) {
      ssnal_en_ctx* a = fits[i0]->c;
      const ssnal_en_options& o = a->opt;
      const double* d[kMultiVectors];
      double* t[kMultiVectors];
      const double* x[kMultiVectors];
      const double* u[kMultiVectors];
      DevState* st[kMultiVectors];
      double* part[kMultiVectors];
      ProxParams pp[kMultiVectors];
      for (int f = 0; f < nv; f++) {
        ssnal_en_ctx* c = fits[i0 + f]->c;
        d[f] = c->d;
        t[f] = c->t;
        x[f] = fits[i0 + f]->x;
        u[f] = c->u;
        st[f] = c->st;
        part[f] = c->partials;
        pp[f] = fits[i0 + f]->pp;
      }
      done = launch_stream_multi(lane_elt(a, kModeT), a->tmap, (int)a->m, a->n, nv, d, t, x, u, st, part, pp, o.mu,
                                 o.beta, o.max_ls, o.ls_fused, a->sms, a->stream, a->col_mean, a->col_scale);
    }
    if (!done) {
      for (int f = 0; f < nv; f++)
        if ((e = stream_t(fits[i0 + f]->c, fits[i0 + f]->x, fits[i0 + f]->pp)) != SSNAL_EN_OK) return e;
      np += nv;
    } else {
      np += 1;
    }
    for (int f = 0; f < nv; f++)
      if ((e = fit_after_pass(*fits[i0 + f])) != SSNAL_EN_OK) return e;
    i0 += nv;
  }
  if (passes) *passes += np;
  return SSNAL_EN_OK;
}

ssnal_en_status check_options(const ssnal_en_options* o) {
  if (!(o->sigma0 > 0) || !(o->sigma_growth >= 1) || !(o->sigma_max >= o->sigma0)) return SSNAL_EN_EINVAL;
  if (!(o->mu > 0 && o->mu < 0.5) || !(o->beta > 0 && o->beta < 1) || !(o->tol > 0)) return SSNAL_EN_EINVAL;
  if (o->max_al < 1 || o->max_newton < 0 || o->max_ls < 1 || o->max_ls > kMaxLS) return SSNAL_EN_EINVAL;
  if (o->ls_fused < 1 || o->ls_fused > kFusedLS) return SSNAL_EN_EINVAL;
  if (o->refine_steps < 0 || o->refine_steps > 8 || o->max_active < 0) return SSNAL_EN_EINVAL;
  if (o->precision < 0 || o->precision > 3) return SSNAL_EN_EINVAL;
  if (o->syrk_tc < 0 || o->syrk_tc > 1) return SSNAL_EN_EINVAL;
  if (o->newton_fp64 < 0 || o->newton_fp64 > 1 || o->cg_maxit < 0 || o->cg_above < 0) return SSNAL_EN_EINVAL;
  if (!(o->cg_rtol > 0.0) || !(o->cg_rtol < 1.0)) return SSNAL_EN_EINVAL;
  return SSNAL_EN_OK;
}

}  // namespace

namespace ssnal {
// Releases a panel larger than `keep_cols` columns (it is grown again on demand), so that
// a context kept between requests does not hold the panel of its largest active set.
void ctx_trim(ssnal_en_ctx* c, int64_t keep_cols) {
  if (!c || c->rcap <= keep_cols) return;
  cudaStreamSynchronize(c->stream);
  dev_free(c->P);
  dev_free(c->P32);
  dev_free(c->h);
  dev_free(c->q);
  dev_free(c->resr);
  dev_free(c->Xtc);
  dev_free(c->corr);
  c->P = nullptr;
  c->P32 = nullptr;
  c->Xtc = nullptr;
  c->h = c->q = c->resr = c->corr = nullptr;
  c->rcap = 0;
  if (grow_panel(c, c->m < c->n ? c->m : c->n) != SSNAL_EN_OK) cudaGetLastError();
}
int64_t ctx_m(const ssnal_en_ctx* c) { return c->m; }

// The stream a context enqueues on; the batch and serving drivers give each
// worker thread its own stream for the duration of one solve.
cudaStream_t ctx_set_stream(ssnal_en_ctx* c, cudaStream_t s) {
  cudaStream_t old = c->stream;
  c->stream = s;
  return old;
}
double ctx_mn(const ssnal_en_ctx* c) { return (double)c->m * (double)c->n; }

// ---- fits advanced together (the serving loop's groups); see FitState
struct Fit {
  FitState F;
};
Fit* fit_new() { return new (std::nothrow) Fit(); }
void fit_delete(Fit* f) { delete f; }
int fit_phase(const Fit* f) { return f->F.phase; }

// Starts a fit on c: penalties (lambda1, lambda2) = (p1, p2), or with scaled != 0 the
// parameterisation of Sec. 4.1: lambda1 = c ||A^T b||_inf, lambda2 = (1 - alpha)/alpha c
// ||A^T b||_inf with (alpha, c) = (p1, p2), ||A^T b||_inf from one pass over A.
ssnal_en_status fit_start(Fit* f, ssnal_en_ctx* c, const double* b, int scaled, double p1, double p2, double* x,
                          double* lambdas_out) {
  double lam1 = p1, lam2 = p2;
  if (scaled) {
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
    ProxParams pp0 = make_pp(c->opt.sigma0, 0.0, 0.0);
    run_stream(c, kModeGmax, b, c->t, nullptr, nullptr, pp0);
    CK(cudaGetLastError());
    ssnal_en_status e = read_state(c);
    if (e != SSNAL_EN_OK) return e;
    const double gmax = c->st_host->gmax;
    lam1 = p2 * gmax;
    lam2 = (1.0 - p1) / p1 * p2 * gmax;
  }
  if (lambdas_out) {
    lambdas_out[0] = lam1;
    lambdas_out[1] = lam2;
  }
  const int use_y0 = c->opt.use_y0;
  c->opt.use_y0 = 0;
  // after the ||A^T b||_inf pass, t holds A^T b (the initial u of a cold start is -t)
  ssnal_en_status e = fit_begin(f->F, c, b, lam1, lam2, x, nullptr, 0.0, scaled ? c->t : nullptr);
  c->opt.use_y0 = use_y0;
  return e;
}
ssnal_en_status fit_step(Fit* f) { return fit_advance(f->F); }
ssnal_en_status fit_passes(Fit* const* f, int k, int* passes) {
  std::vector<FitState*> v((size_t)k);
  for (int i = 0; i < k; i++) v[(size_t)i] = &f[i]->F;
  return run_passes(v.data(), k, passes);
}
ssnal_en_status fit_end(Fit* f, ssnal_en_result* out) { return fit_finish(f->F, out); }
}  // namespace ssnal

extern "C" {

void ssnal_en_default_options(ssnal_en_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->sigma0 = 5e-3;
  o->sigma_growth = 5.0;
  o->sigma_max = 1e8;
  o->mu = 0.2;
  o->beta = 0.5;
  o->tol = 1e-6;
  o->max_al = 100;
  o->max_newton = 50;
  o->max_ls = 40;
  o->precision = 0;
  o->refine_steps = 1;
  o->use_y0 = 0;
  o->ls_fused = kFusedLS;
  o->syrk_tc = 1;
  o->max_active = 0;
  o->newton_fp64 = 0;
  o->cg_maxit = 0;
  o->cg_above = 10000;
  o->cg_rtol = 1e-10;
}

const char* ssnal_en_status_string(int32_t s) {
  switch (s) {
    case SSNAL_EN_OK: return "ok";
    case SSNAL_EN_EINVAL: return "invalid argument";
    case SSNAL_EN_ENOMEM: return "out of device memory";
    case SSNAL_EN_ENOCONV: return "iteration limit reached before the KKT tolerance";
    case SSNAL_EN_ECUDA: return "CUDA runtime error";
    case SSNAL_EN_ETIMEOUT: return "device wait timed out";
    case SSNAL_EN_ENOTSUP: return "unsupported size or type";
    default: return "unknown status";
  }
}

ssnal_en_status ssnal_en_create(ssnal_en_ctx** out, const ssnal_en_matrix* A, const ssnal_en_options* opts,
                                void* stream) {
  if (!out || !A) return SSNAL_EN_EINVAL;
  *out = nullptr;
  const double es = elem_bytes(A->dtype);
  if (es == 0 || !A->data || A->m <= 0 || A->n <= 0 || A->lda < A->m) return SSNAL_EN_EINVAL;
  // the column stride must be whole 16-byte units (2-bit codes: lda a multiple of 64 codes)
  if (A->dtype == SSNAL_EN_I2_GENO ? (A->lda % 64 != 0) : ((int64_t)(A->lda * es) % 16 != 0)) return SSNAL_EN_EINVAL;
  if (((uintptr_t)A->data) % 16 != 0) return SSNAL_EN_EINVAL;
  if (A->n >= (int64_t)0x7fffffff) return SSNAL_EN_ENOTSUP;
  if (A->m > kMaxM) return SSNAL_EN_ENOTSUP;
  if (is_geno(A->dtype) && (!A->col_mean || !A->col_scale)) return SSNAL_EN_EINVAL;
  ssnal_en_options o;
  if (opts)
    o = *opts;
  else
    ssnal_en_default_options(&o);
  if (check_options(&o) != SSNAL_EN_OK) return SSNAL_EN_EINVAL;
  ssnal_en_ctx* c = new (std::nothrow) ssnal_en_ctx();
  if (!c) return SSNAL_EN_ENOMEM;
  c->m = A->m;
  c->n = A->n;
  c->lda = A->lda;
  c->dtype = A->dtype;
  c->A = A->data;
  c->col_mean = A->col_mean;
  c->col_scale = A->col_scale;
  c->opt = o;
  c->stream = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    delete c;
    return SSNAL_EN_ECUDA;
  }
  c->grid_stream = stream_grid(c->sms);
  c->grid_vec = vec_grid(c->n, c->sms);
  const int64_t m = c->m, n = c->n;
  c->ldp = round_up(m, 2);
  c->ldp32 = round_up(m, 4);
  c->ldg = round_up(m, 4);
  ssnal_en_status s = SSNAL_EN_OK;
#define AL(ptr, cnt)                                         \
  do {                                                       \
    if (s == SSNAL_EN_OK) s = dev_alloc(&(ptr), (size_t)(cnt)); \
  } while (0)
  AL(c->st, 1);
  AL(c->u, n);
  AL(c->t, n);
  AL(c->xpath, n);
  AL(c->y, m);
  AL(c->d, m);
  AL(c->g, m);
  AL(c->bdev, m);
  AL(c->res, m);
  AL(c->tmpm, m);
  AL(c->cgp, m);
  AL(c->bstage, m);
  AL(c->J, n);
  AL(c->wJ, n);
  AL(c->counts, 2 * c->grid_vec + 2);
  AL(c->partials, (size_t)c->grid_stream * kMaxLS);
  AL(c->vpartials, (size_t)c->grid_vec * 6);
  AL(c->gemv_part, (size_t)kGemvGroups * m);
  AL(c->comb_scratch, 4 * ((m + 31) / 32) + 4);
  AL(c->cpart, (size_t)kGemvSplitMax * m);
  AL(c->tile_ctr, (m + 31) / 32);
  AL(c->rpart, 2 * ((m + 31) / 32) + 2);
  AL(c->G, c->ldg * m);
  AL(c->Wdiag, (size_t)((m + 31) / 32) * 1024);
  AL(c->zf, m);
  AL(c->tc_part, syrk_tc_part_floats(c->sms));
#undef AL
  if (s == SSNAL_EN_OK && cudaMallocHost((void**)&c->st_host, sizeof(DevState)) != cudaSuccess) s = SSNAL_EN_ENOMEM;
  if (s == SSNAL_EN_OK && cudaMallocHost((void**)&c->st_flag, 64) != cudaSuccess) s = SSNAL_EN_ENOMEM;
  if (s == SSNAL_EN_OK) *c->st_flag = 0;
  if (s == SSNAL_EN_OK) s = grow_panel(c, m < n ? m : n);
  if (s == SSNAL_EN_OK && cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream) != cudaSuccess) s = SSNAL_EN_ECUDA;
  if (s == SSNAL_EN_OK &&
      cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned) * ((c->m + 31) / 32), c->stream) != cudaSuccess)
    s = SSNAL_EN_ECUDA;
  if (s == SSNAL_EN_OK && c->dtype == SSNAL_EN_F64) {
    // one pass over A: may the stream use the float-float split?
    launch_check_range((const double*)c->A, c->lda, (int)c->m, c->n, &c->st->overflow, c->sms, c->stream);
    if (read_state(c) != SSNAL_EN_OK) s = SSNAL_EN_ECUDA;
    else c->ff_ok = c->st_host->overflow ? 0 : 1;
  }
  if (s == SSNAL_EN_OK && cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream) != cudaSuccess) s = SSNAL_EN_ECUDA;
  if (s == SSNAL_EN_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) s = SSNAL_EN_ECUDA;
  if (s == SSNAL_EN_OK && c->dtype != SSNAL_EN_F64) {
    // BF16 / FP32 storage: the lane stream reads A directly through a tensor map
    c->tmap_ok = (tensor_map_bytes() <= sizeof(c->tmap) &&
                  make_elt_tensor_map(c->tmap, c->A, c->dtype, c->lda, (int)c->m, c->n)) ? 1 : 0;
    if (!c->tmap_ok) s = SSNAL_EN_ENOTSUP;
  }
  if (s == SSNAL_EN_OK && c->dtype == SSNAL_EN_F64 && c->ff_ok && c->opt.precision != 3) {
    // float-pair copy of A read by the stream (same bytes as A); without it the
    // stream splits each FP64 entry on the fly
    const int64_t mm = (c->m + 1) & ~1LL;
    if (cudaMalloc(&c->Asplit, (size_t)mm * (size_t)c->n * sizeof(double)) == cudaSuccess) {
      c->lda_split = mm;
      launch_presplit((const double*)c->A, c->lda, (int)c->m, c->n, c->Asplit, c->sms, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) s = SSNAL_EN_ECUDA;
      c->tmap_ok = (tensor_map_bytes() <= sizeof(c->tmap) &&
                    make_split_tensor_map(c->tmap, c->Asplit, (int)c->m, c->n)) ? 1 : 0;
    } else {
      cudaGetLastError();
      c->Asplit = nullptr;
    }
  }
  set_stream_kind(c);
  if (s != SSNAL_EN_OK) {
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return SSNAL_EN_OK;
}

void ssnal_en_destroy(ssnal_en_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

ssnal_en_status ssnal_en_set_options(ssnal_en_ctx* c, const ssnal_en_options* opts) {
  if (!c) return SSNAL_EN_EINVAL;
  ssnal_en_options o;
  if (opts)
    o = *opts;
  else
    ssnal_en_default_options(&o);
  if (check_options(&o) != SSNAL_EN_OK) return SSNAL_EN_EINVAL;
  c->opt = o;
  set_stream_kind(c);
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_solve(ssnal_en_ctx* c, const double* b, double lambda1, double lambda2, double* x, double* y,
                               ssnal_en_result* out) {
  if (!c || !b || !x) return SSNAL_EN_EINVAL;
  if (!is_finite_d(lambda1) || !is_finite_d(lambda2) || lambda1 < 0 || lambda2 < 0) return SSNAL_EN_EINVAL;
  if (c->opt.use_y0 && !y) return SSNAL_EN_EINVAL;
  return solve_impl(c, b, lambda1, lambda2, x, y, out);
}

ssnal_en_status ssnal_en_solve_shared(ssnal_en_instance* inst, int32_t count, ssnal_en_result* out, int32_t* passes) {
  if (passes) *passes = 0;
  if (!inst || count < 1) return SSNAL_EN_EINVAL;
  for (int32_t i = 0; i < count; i++) {
    const ssnal_en_instance& q = inst[i];
    if (!q.ctx || !q.b || !q.x || !is_finite_d(q.lambda1) || !is_finite_d(q.lambda2) || q.lambda1 < 0 ||
        q.lambda2 < 0)
      return SSNAL_EN_EINVAL;
    if (q.ctx->opt.use_y0 && !q.y) return SSNAL_EN_EINVAL;
    for (int32_t j = 0; j < i; j++)
      if (inst[j].ctx == q.ctx) return SSNAL_EN_EINVAL;  // every fit needs its own workspaces
  }
  // all fits run on the first context's stream (their kernels and the merged passes are
  // ordered on it); the contexts' own streams are restored at the end
  cudaStream_t s0 = inst[0].ctx->stream;
  std::vector<cudaStream_t> saved((size_t)count);
  for (int32_t i = 0; i < count; i++) {
    saved[(size_t)i] = inst[i].ctx->stream;
    if (i > 0) {
      CK(cudaStreamSynchronize(inst[i].ctx->stream));
      inst[i].ctx->stream = s0;
    }
  }
  std::vector<FitState> F((size_t)count);
  std::vector<ssnal_en_status> st((size_t)count, SSNAL_EN_OK);
  for (int32_t i = 0; i < count; i++) {
    st[(size_t)i] = fit_begin(F[(size_t)i], inst[i].ctx, inst[i].b, inst[i].lambda1, inst[i].lambda2, inst[i].x,
                              inst[i].y, 0.0);
    if (st[(size_t)i] != SSNAL_EN_OK) F[(size_t)i].phase = kFitDone;
  }
  int np = 0;
  for (;;) {
    std::vector<FitState*> need;
    for (int32_t i = 0; i < count; i++) {
      FitState& f = F[(size_t)i];
      if (f.phase == kFitDone || st[(size_t)i] != SSNAL_EN_OK) continue;
      if ((st[(size_t)i] = fit_advance(f)) != SSNAL_EN_OK) {
        f.phase = kFitDone;
        continue;
      }
      if (f.phase == kFitNeedPass) need.push_back(&f);
    }
    if (need.empty()) break;
    ssnal_en_status e = run_passes(need.data(), (int)need.size(), &np);
    if (e != SSNAL_EN_OK) {
      for (FitState* f : need) st[(size_t)(f - F.data())] = e;
      for (FitState* f : need) f->phase = kFitDone;
    }
  }
  ssnal_en_status worst = SSNAL_EN_OK;
  for (int32_t i = 0; i < count; i++) {
    ssnal_en_result r{};
    if (st[(size_t)i] == SSNAL_EN_OK) {
      st[(size_t)i] = fit_finish(F[(size_t)i], &r);
    } else {
      r = F[(size_t)i].R;
      r.status = st[(size_t)i];
    }
    if (out) out[i] = r;
    if (st[(size_t)i] != SSNAL_EN_OK && worst == SSNAL_EN_OK) worst = st[(size_t)i];
  }
  CK(cudaStreamSynchronize(s0));
  for (int32_t i = 0; i < count; i++) inst[i].ctx->stream = saved[(size_t)i];
  if (passes) *passes = np;
  return worst;
}

ssnal_en_status ssnal_en_path(ssnal_en_ctx* c, const double* b, double alpha, const double* c_grid, int32_t K,
                              double* X, ssnal_en_result* out, int32_t* n_done) {
  if (n_done) *n_done = 0;
  if (!c || !b || !c_grid || K < 0) return SSNAL_EN_EINVAL;
  if (!(alpha > 0.0 && alpha <= 1.0)) return SSNAL_EN_EINVAL;
  for (int k = 0; k < K; k++)
    if (!is_finite_d(c_grid[k]) || c_grid[k] < 0) return SSNAL_EN_EINVAL;
  if (out) memset(out, 0, sizeof(ssnal_en_result) * (size_t)K);
  cudaStream_t s = c->stream;
  // ||A^T b||_inf from the same stream kernel that later forms u = A^T y
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  ProxParams pp0 = make_pp(c->opt.sigma0, 0.0, 0.0);
  run_stream(c, kModeGmax, b, c->t, nullptr, nullptr, pp0);
  CK(cudaGetLastError());
  ssnal_en_status e = read_state(c);
  if (e != SSNAL_EN_OK) return e;
  const double gmax = c->st_host->gmax;
  CK(cudaMemsetAsync(c->xpath, 0, sizeof(double) * c->n, s));
  ssnal_en_status worst = SSNAL_EN_OK;
  const ssnal_en_options saved = c->opt;
  c->opt.use_y0 = 0;
  double nb1 = 0.0;  // 1 + ||b||, the same at every point of the path
  for (int k = 0; k < K; k++) {
    const double lam1 = c_grid[k] * gmax;
    const double lam2 = (1.0 - alpha) / alpha * c_grid[k] * gmax;
    ssnal_en_result r;
    // the first point starts at x = 0: its initial u is -A^T b from the pass above
    e = solve_impl(c, b, lam1, lam2, c->xpath, nullptr, &r, nb1, k == 0 ? c->t : nullptr);
    nb1 = c->last_nb1;
    if (e != SSNAL_EN_OK && e != SSNAL_EN_ENOCONV) {
      c->opt = saved;
      return e;
    }
    if (e == SSNAL_EN_ENOCONV) worst = SSNAL_EN_ENOCONV;
    if (out) out[k] = r;
    if (X) {
      launch_copy_f64(X + (size_t)k * c->n, c->xpath, c->n, c->sms, s);
      if (cudaGetLastError() != cudaSuccess) {
        c->opt = saved;
        return SSNAL_EN_ECUDA;
      }
    }
    if (n_done) *n_done = k + 1;
    if (saved.max_active > 0 && r.active >= saved.max_active) break;
  }
  c->opt = saved;
  CK(cudaStreamSynchronize(s));
  return worst;
}

// Model-selection criteria along a path (Sec. 3.3, eq. gcv_bic).
ssnal_en_status ssnal_en_tune(ssnal_en_ctx* c, const double* b, double alpha, const double* c_grid, int32_t K,
                              double* X, ssnal_en_result* out, ssnal_en_tune_point* crit, int32_t* best_gcv,
                              int32_t* best_ebic, int32_t* n_done) {
  if (best_gcv) *best_gcv = -1;
  if (best_ebic) *best_ebic = -1;
  if (n_done) *n_done = 0;
  if (!c || !b || !c_grid || !X || !out || !crit || K < 0) return SSNAL_EN_EINVAL;
  int32_t done = 0;
  ssnal_en_status e = ssnal_en_path(c, b, alpha, c_grid, K, X, out, &done);
  if (e != SSNAL_EN_OK && e != SSNAL_EN_ENOCONV) return e;
  if (n_done) *n_done = done;
  cudaStream_t s = c->stream;
  const int64_t m = c->m, n = c->n;
  // ||b||^2 for the empty model
  launch_combine(c->tmpm, c->bdev, 1.0, nullptr, 0.0, nullptr, 0.0, (int)m, 1, c->bdev, c->bdev, nullptr, c->st,
                 c->comb_scratch, s);
  if ((e = read_state(c)) != SSNAL_EN_OK) return e;
  const double bb = c->st_host->g2;
  double best_g = INFINITY, best_e = INFINITY;
  for (int k = 0; k < done; k++) {
    ssnal_en_tune_point& P = crit[k];
    memset(&P, 0, sizeof(P));
    const double* xk = X + (int64_t)k * n;
    const double lam2 = out[k].lambda2;
    ProxParams pp = make_pp(c->opt.sigma0, out[k].lambda1, lam2);
    // J = support of x_k and the panel A_J (y := A_J x_J - b as a by-product)
    if ((e = prox_gather_grad(c, kProxSupport, xk, c->bdev, pp, 0)) != SSNAL_EN_OK) return e;
    const int64_t r = c->st_host->r;
    P.active = r;
    const int64_t N = r < m ? r : m;
    // degrees of freedom: nu = N - lam2 tr(G^{-1}), G = A_J^T A_J + lam2 I (r <= m) or A_J A_J^T + lam2 I
    double nu = NAN;
    if (r == 0) {
      nu = 0.0;
    } else if (!(lam2 > 0.0)) {
      nu = (double)N;  // full column (or row) rank assumed: the trace of a projection
    } else {
      const int64_t Np = (N + 31) / 32 * 32;
      constexpr int kOut = kMaxM / 32;  // tune_dev: partials [0, kOut), result at kOut
      if (c->tune_dev == nullptr && dev_alloc(&c->tune_dev, kOut + 1) != SSNAL_EN_OK) return SSNAL_EN_ENOMEM;
      if (Np <= 640) {
        if (c->tuneS == nullptr && dev_alloc(&c->tuneS, (size_t)2 * 640 * 640) != SSNAL_EN_OK) return SSNAL_EN_ENOMEM;
        const long long ldS = 2 * Np;
        if (r <= m)
          launch_syrk_tc(c->P, c->ldp, (int)m, (int)r, 0, syrk_splits(c), c->Xtc, c->tc_part, 1.0f, (float)lam2,
                         c->tuneS, ldS, c->st, c->sms, s);
        else
          launch_syrk_tc(c->P, c->ldp, (int)m, (int)r, 1, syrk_splits(c), c->Xtc, c->tc_part, 1.0f, (float)lam2,
                         c->tuneS, ldS, c->st, c->sms, s);
        if (inv_trace(c->tuneS, ldS, (int)N, c->st, c->Wdiag, c->tune_dev, c->tune_dev + kOut, s)) {
          double tr = 0.0;
          CK(cudaMemcpyAsync(&tr, c->tune_dev + kOut, sizeof(double), cudaMemcpyDeviceToHost, s));
          if ((e = read_state(c)) != SSNAL_EN_OK) return e;
          tr -= (double)(Np - N);
          if (!c->st_host->chol_fail) nu = (double)N - lam2 * tr;
        }
      } else {
        // larger systems: the Newton-matrix buffer, the super-block factor and the
        // blocked inverse of k_inv_frob (Y = L^{-1} in scratch)
        if (c->tuneY_np < Np) {
          dev_free(c->tuneY);
          c->tuneY = nullptr;
          c->tuneY_np = 0;
          if (dev_alloc(&c->tuneY, (size_t)Np * (size_t)Np) != SSNAL_EN_OK) return SSNAL_EN_ENOMEM;
          c->tuneY_np = Np;
        }
        if (r <= m)
          launch_syrk_tc(c->P, c->ldp, (int)m, (int)r, 0, syrk_splits(c), c->Xtc, c->tc_part, 1.0f, (float)lam2,
                         c->G, c->ldg, c->st, c->sms, s);
        else
          launch_syrk_tc(c->P, c->ldp, (int)m, (int)r, 1, syrk_splits(c), c->Xtc, c->tc_part, 1.0f, (float)lam2,
                         c->G, c->ldg, c->st, c->sms, s);
        if (inv_trace_large(c->G, c->ldg, (int)N, c->st, c->Wdiag, c->tuneY, Np, c->tune_dev, c->tune_dev + kOut,
                            s)) {
          double tr = 0.0;
          CK(cudaMemcpyAsync(&tr, c->tune_dev + kOut, sizeof(double), cudaMemcpyDeviceToHost, s));
          if ((e = read_state(c)) != SSNAL_EN_OK) return e;
          if (!c->st_host->chol_fail) nu = (double)N - lam2 * tr;
        }
      }
    }
    // de-biased fit: ordinary least squares on J, rss = ||b - A_J x_ols||^2 (the SMW Newton
    // solve with kappa = infinity gives d = A_J G0^{-1} A_J^T b - b with G0 = A_J^T A_J)
    double rss = NAN;
    if (r == 0) {
      rss = bb;
    } else if (r >= m) {
      rss = 0.0;
    } else {
      if ((e = newton_direction(c, r, INFINITY, c->bdev, c->d, c->bdev, c->bdev, 1)) != SSNAL_EN_OK) return e;
      if ((e = read_state(c)) != SSNAL_EN_OK) return e;
      if (c->st_host->chol_fail | c->st_host->newton_bad) {  // redo the least-squares solve in FP64
        if ((e = clear_newton_flags(c)) != SSNAL_EN_OK) return e;
        if ((e = newton_direction_f64(c, r, INFINITY, c->bdev, c->d, c->bdev, c->bdev, 1)) != SSNAL_EN_OK) return e;
        if ((e = read_state(c)) != SSNAL_EN_OK) return e;
      }
      if (!(c->st_host->chol_fail | c->st_host->f64_fail)) rss = c->st_host->dd;
    }
    P.nu = nu;
    P.rss = rss;
    const double md = (double)m;
    P.gcv = (rss / md) / ((1.0 - nu / md) * (1.0 - nu / md));
    P.ebic = log(rss / md) + (nu / md) * (log(md) + log((double)n));
    if (std::isfinite(P.gcv) && P.gcv < best_g) {
      best_g = P.gcv;
      if (best_gcv) *best_gcv = k;
    }
    if (std::isfinite(P.ebic) && P.ebic < best_e) {
      best_e = P.ebic;
      if (best_ebic) *best_ebic = k;
    }
  }
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  CK(cudaStreamSynchronize(s));
  return e;
}

ssnal_en_status ssnal_en_path_host(ssnal_en_ctx* c, const double* b_host, double alpha, const double* c_grid,
                                   int32_t K, double* X_host, ssnal_en_result* out, int32_t* n_done) {
  if (!c || !b_host || K < 0) return SSNAL_EN_EINVAL;
  cudaStream_t s = c->stream;
  double* X = nullptr;
  if (X_host && K > 0) {
    if (c->Xcap < (int64_t)K * c->n) {
      dev_free(c->Xdev);
      c->Xdev = nullptr;
      c->Xcap = 0;
      ssnal_en_status e = dev_alloc(&c->Xdev, (size_t)K * (size_t)c->n);
      if (e != SSNAL_EN_OK) return e;
      c->Xcap = (int64_t)K * c->n;
    }
    X = c->Xdev;
  }
  CK(cudaMemcpyAsync(c->bstage, b_host, sizeof(double) * c->m, cudaMemcpyHostToDevice, s));
  int32_t done = 0;
  ssnal_en_status e = ssnal_en_path(c, c->bstage, alpha, c_grid, K, X, out, &done);
  if (n_done) *n_done = done;
  if (e != SSNAL_EN_OK && e != SSNAL_EN_ENOCONV) return e;
  if (X && done > 0)
    CK(cudaMemcpyAsync(X_host, X, sizeof(double) * (size_t)done * c->n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return e;
}

ssnal_en_status ssnal_en_profile(ssnal_en_ctx* c, int32_t enable, int32_t reset, double* stream_ms,
                                 int64_t* stream_launches, double* stream_bytes, int64_t* kernel_launches) {
  if (!c) return SSNAL_EN_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  prof_harvest(c);
  if (reset) {
    c->prof_ms = 0.0;
    c->prof_bytes = 0.0;
    c->prof_launches = 0;
    for (int k = 0; k < kPhases; k++) {
      c->phase_ms[k] = 0.0;
      c->phase_n[k] = 0;
    }
  }
  c->prof = enable < 0 ? 0 : enable > 2 ? 2 : enable;
  c->prof_seq = 0;
  if (stream_ms) *stream_ms = c->prof_ms;
  if (stream_launches) *stream_launches = c->prof_launches;
  if (stream_bytes) *stream_bytes = c->prof_bytes;
  if (kernel_launches) *kernel_launches = g_launches.load();
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_profile_phases(ssnal_en_ctx* c, double* phase_ms, int64_t* phase_count) {
  if (!c) return SSNAL_EN_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  prof_harvest(c);
  for (int k = 0; k < kPhases; k++) {
    if (phase_ms) phase_ms[k] = c->phase_ms[k];
    if (phase_count) phase_count[k] = c->phase_n[k];
  }
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_op_at_y(ssnal_en_ctx* c, const double* y, double* u) {
  if (!c || !y || !u) return SSNAL_EN_EINVAL;
  ProxParams pp = make_pp(1.0, 0.0, 0.0);
  run_stream(c, kModeU, y, u, nullptr, nullptr, pp);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_op_at_d(ssnal_en_ctx* c, const double* d, double* t) {
  if (!c || !d || !t) return SSNAL_EN_EINVAL;
  const ssnal_en_options& o = c->opt;
  ProxParams pp = make_pp(1.0, 0.0, 0.0);
  if (c->stream_kind == kStreamLane)  // the Newton pass's element type, without the trial sums
    launch_stream_lane(kModeU, lane_elt(c, kModeT), c->tmap, (int)c->m, c->n, d, t, nullptr, nullptr, pp, o.mu,
                       o.beta, o.max_ls, o.ls_fused, c->st, c->partials, c->sms, c->stream, c->col_mean, c->col_scale);
  else
    run_stream(c, kModeU, d, t, nullptr, nullptr, pp);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_op_prox_active(ssnal_en_ctx* c, const double* x, const double* u, double sigma,
                                        double lambda1, double lambda2, int32_t* J, double* wJ, int64_t* r) {
  if (!c || !x || !u || !J || !wJ || !r) return SSNAL_EN_EINVAL;
  if (!(sigma > 0) || !is_finite_d(lambda1) || !is_finite_d(lambda2) || lambda1 < 0 || lambda2 < 0) return SSNAL_EN_EINVAL;
  ProxParams pp = make_pp(sigma, lambda1, lambda2);
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  launch_prox_count(kProxThreshold, x, const_cast<double*>(u), nullptr, nullptr, nullptr, c->n, (int)c->m, pp, 0,
                    c->st, c->counts, c->vpartials, c->grid_vec, s);
  launch_prox_scatter(kProxThreshold, x, u, c->n, pp, c->counts, c->vpartials, c->st, J, wJ, c->grid_vec, s);
  CK(cudaGetLastError());
  ssnal_en_status e = read_state(c);
  if (e != SSNAL_EN_OK) return e;
  *r = c->st_host->r;
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_op_grad(ssnal_en_ctx* c, const int32_t* J, const double* wJ, int64_t r, const double* y,
                                 const double* b, double* g) {
  if (!c || (r > 0 && (!J || !wJ)) || !y || !b || !g || r < 0 || r > c->n) return SSNAL_EN_EINVAL;
  ssnal_en_status e = grow_panel(c, r);
  if (e != SSNAL_EN_OK) return e;
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  const int m = (int)c->m;
  launch_gather(c->A, c->dtype, c->lda, m, J, c->st, r, c->rcap, c->P, c->ldp, c->P32, c->ldp32, c->sms, s, c->col_mean,
                c->col_scale);
  launch_gemv_n(c->P, c->ldp, m, wJ, c->st, r, c->rcap, g, y, 1.0, b, 1.0, -1.0, 0, nullptr, nullptr, nullptr, c->st,
                c->comb_scratch, c->cpart, c->tile_ctr, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_op_newton(ssnal_en_ctx* c, int64_t r, double kappa, const double* g, double* d) {
  if (!c || !g || !d || r < 0 || r > c->rcap || !(kappa > 0) || !is_finite_d(kappa)) return SSNAL_EN_EINVAL;
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  ssnal_en_status e = SSNAL_EN_OK;
  if (use_cg(c, r)) {
    int it = 0;
    if ((e = newton_direction_cg(c, r, kappa, g, d, nullptr, nullptr, 0, &it)) != SSNAL_EN_OK) return e;
    return c->st_host->cg_done ? SSNAL_EN_OK : SSNAL_EN_ENOCONV;
  }
  if (c->opt.newton_fp64 == 0) {
    if ((e = newton_direction(c, r, kappa, g, d, nullptr, nullptr, 0)) != SSNAL_EN_OK) return e;
    if ((e = read_state(c)) != SSNAL_EN_OK) return e;
    // more refinement steps while the corrections keep shrinking (by at least half each) and
    // are above 1e-12 of the solution; a solve that stops contracting goes to FP64
    double last = c->st_host->refine_ratio;
    for (int extra = 0; extra < 16 && !(c->st_host->chol_fail | c->st_host->newton_bad) &&
                        c->opt.refine_steps > 0 && last > 1e-12; extra++) {
      if ((e = refine_once(c, r, kappa, g, d)) != SSNAL_EN_OK) return e;
      if ((e = read_state(c)) != SSNAL_EN_OK) return e;
      const double now = c->st_host->refine_ratio;
      if (!(now < 0.5 * last)) break;  // stagnation at the accuracy of the FP64 residual
      last = now;
    }
    if (!(c->st_host->chol_fail | c->st_host->newton_bad)) return SSNAL_EN_OK;
    if ((e = clear_newton_flags(c)) != SSNAL_EN_OK) return e;  // the FP32 solve is unreliable: FP64
  }
  if ((e = newton_direction_f64(c, r, kappa, g, d, nullptr, nullptr, 0)) != SSNAL_EN_OK) return e;
  if ((e = read_state(c)) != SSNAL_EN_OK) return e;
  return c->st_host->f64_fail ? SSNAL_EN_ENOCONV : SSNAL_EN_OK;
}

}  // extern "C"
