// Serving loop: design matrices stay resident on the device, requests (a new
// right-hand side and penalties on one of them) arrive at any time and are
// admitted while others run (continuous batching).  Worker threads, each with
// its own CUDA stream, take admitted requests in arrival order: a free worker takes
// the oldest request and the queued requests on the same matrix (up to max_group),
// advances their fits together one Newton step at a time with the passes over A
// merged (one pass forms A^T [d_1 ... d_k] for up to four fits), finishes fits as
// they converge and admits newly arrived requests on that matrix into the freed
// places between steps.  A worker keeps contexts per matrix (workspaces, x, y,
// sigma and the Cholesky factor live on the device for the whole solve) and reuses
// them for later requests.  Admission also bounds the device bytes of the contexts
// that requests in flight occupy.  A request's b is copied from host memory at the
// start of its solve and its x back at the end, so a request's latency covers its
// transfers.  Each request runs the same kernels in the same order as ssnal_en_solve
// on its own (a merged pass gives each fit bitwise the result of its own pass), so its
// result does not depend on the mix.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ssnal_en.h"
#include "internal.h"

namespace {

struct Request {
  int64_t ticket = 0;
  int32_t mat = 0;
  std::vector<double> b;
  double lambda1 = 0.0, lambda2 = 0.0;
  bool scaled = false;     // penalties given as (alpha, c) relative to ||A^T b||_inf
  double alpha = 1.0, c = 0.0;
  std::vector<double> x;
  ssnal_en_result res{};
  bool done = false;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;  // seconds since server start
};

// The device workspaces a worker keeps for one matrix.
struct Slot {
  ssnal_en_ctx* ctx = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct ssnal_en_server {
  std::vector<ssnal_en_matrix> mats;
  ssnal_en_options opts{};
  int device = 0;
  int64_t max_bytes = 0;  // bound on the bytes of contexts in use by requests in flight (0 = none)
  int max_group = 8;      // requests on one matrix a worker advances together
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<int64_t, std::shared_ptr<Request>> tickets;
  int64_t next_ticket = 1;
  int64_t bytes_in_flight = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// Device bytes of a context for matrix a (the vectors and panels it allocates;
// an estimate used for admission only).
int64_t context_bytes(const ssnal_en_matrix& a) {
  const int64_t m = a.m, n = a.n;
  const int64_t r = m < n ? m : n;
  return 8 * (6 * n + 12 * m) + 12 * m * r + 4 * m * m + 6 * m * r + 4 * n;
}

// A request of a worker's group: its context slot and its fit.
struct Member {
  std::shared_ptr<Request> q;
  Slot* slot = nullptr;
  ssnal::Fit* fit = nullptr;
  int64_t need = 0;
  bool retried = false;
  ssnal_en_status st = SSNAL_EN_OK;
};

// Takes queued requests on matrix `mat` (the caller holds S->mu) while the group has room
// and the footprint bound allows; the first request of a group is always admitted.
void admit_same_matrix(ssnal_en_server* S, int mat, std::vector<Member>& group, bool first) {
  for (auto it = S->queue.begin(); it != S->queue.end() && (int)group.size() < S->max_group;) {
    if ((*it)->mat != mat) {
      ++it;
      continue;
    }
    const int64_t need = context_bytes(S->mats[mat]);
    const bool fits = S->max_bytes <= 0 || S->bytes_in_flight == 0 || S->bytes_in_flight + need <= S->max_bytes;
    if (!fits && !(first && group.empty())) break;
    Member mb;
    mb.q = *it;
    mb.need = need;
    mb.q->t_start = S->now();
    S->bytes_in_flight += need;
    group.push_back(std::move(mb));
    it = S->queue.erase(it);
  }
}

// A slot of pool[mat] not used by the group (created on first use).
Slot* free_slot(ssnal_en_server* S, std::vector<std::vector<Slot>>& pool, const std::vector<Member>& group, int mat,
                cudaStream_t s, ssnal_en_status* st) {
  *st = SSNAL_EN_OK;
  for (Slot& sl : pool[(size_t)mat]) {
    bool used = false;
    for (const Member& mb : group) used = used || mb.slot == &sl;
    if (!used) return &sl;
  }
  if (pool[(size_t)mat].size() >= (size_t)S->max_group) {  // never happens: one slot per member
    *st = SSNAL_EN_EINVAL;
    return nullptr;
  }
  const ssnal_en_matrix& A = S->mats[(size_t)mat];
  Slot sl;
  *st = ssnal_en_create(&sl.ctx, &A, &S->opts, s);
  if (*st == SSNAL_EN_OK && (cudaMalloc(&sl.b, sizeof(double) * A.m) != cudaSuccess ||
                             cudaMalloc(&sl.x, sizeof(double) * A.n) != cudaSuccess))
    *st = SSNAL_EN_ENOMEM;
  if (*st != SSNAL_EN_OK) {
    cudaGetLastError();
    if (sl.ctx) ssnal_en_destroy(sl.ctx);
    if (sl.b) cudaFree(sl.b);
    return nullptr;
  }
  pool[(size_t)mat].push_back(sl);
  return &pool[(size_t)mat].back();
}

void release_slot(Slot& sl) {
  if (sl.ctx) ssnal_en_destroy(sl.ctx);
  if (sl.b) cudaFree(sl.b);
  if (sl.x) cudaFree(sl.x);
  sl = Slot();
}

// Copies b in, zeroes x and starts the member's fit.
ssnal_en_status start_member(ssnal_en_server* S, Member& mb, cudaStream_t s) {
  const ssnal_en_matrix& A = S->mats[(size_t)mb.q->mat];
  Slot& sl = *mb.slot;
  if (cudaMemcpyAsync(sl.b, mb.q->b.data(), sizeof(double) * A.m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(sl.x, 0, sizeof(double) * A.n, s) != cudaSuccess)
    return SSNAL_EN_ECUDA;
  if (!mb.fit && !(mb.fit = ssnal::fit_new())) return SSNAL_EN_ENOMEM;
  const Request& q = *mb.q;
  return q.scaled ? ssnal::fit_start(mb.fit, sl.ctx, sl.b, 1, q.alpha, q.c, sl.x, nullptr)
                  : ssnal::fit_start(mb.fit, sl.ctx, sl.b, 0, q.lambda1, q.lambda2, sl.x, nullptr);
}

// Worker: forms a group of requests on one matrix (the oldest queued request's, plus
// queued requests on the same matrix up to max_group), advances every fit of the group
// one Newton step at a time with the passes over A merged (A^T [d_1 ... d_k]), finishes
// fits as they converge and admits newly queued requests on the same matrix into the
// freed places between steps.  Contexts are kept per matrix (as many as the largest
// group needed) and reused by later requests.
void worker_main(ssnal_en_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  std::vector<std::vector<Slot>> pool(S->mats.size());
  for (auto& p : pool) p.reserve(64);  // slots are referenced by address: no reallocation
  for (;;) {
    std::vector<Member> group;
    int mat = -1;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        if (!S->queue.empty()) {
          const int64_t need = context_bytes(S->mats[(size_t)S->queue.front()->mat]);
          if (S->max_bytes <= 0 || S->bytes_in_flight == 0 || S->bytes_in_flight + need <= S->max_bytes) break;
        }
        S->cv_work.wait(lk);
      }
      if (S->stop) break;
      mat = S->queue.front()->mat;
      admit_same_matrix(S, mat, group, true);
    }
    size_t started = 0;  // members [0, started) have slots and fits
    int passes = 0;
    for (;;) {
      // start the members admitted since the last step
      for (; started < group.size(); started++) {
        Member& mb = group[started];
        ssnal_en_status st = SSNAL_EN_OK;
        mb.slot = free_slot(S, pool, group, mat, s, &st);
        if (st == SSNAL_EN_OK) st = start_member(S, mb, s);
        mb.st = st;
      }
      // one Newton step of every running fit; the passes of those that need one merged
      std::vector<ssnal::Fit*> need;
      for (Member& mb : group) {
        if (mb.st != SSNAL_EN_OK || ssnal::fit_phase(mb.fit) == ssnal::kFitPhaseDone) continue;
        if ((mb.st = ssnal::fit_step(mb.fit)) != SSNAL_EN_OK) continue;
        if (ssnal::fit_phase(mb.fit) == ssnal::kFitPhaseNeedPass) need.push_back(mb.fit);
      }
      if (!need.empty()) {
        const ssnal_en_status st = ssnal::fit_passes(need.data(), (int)need.size(), &passes);
        if (st != SSNAL_EN_OK)
          for (Member& mb : group)
            for (ssnal::Fit* f : need)
              if (mb.fit == f) mb.st = st;
      }
      // finished or failed members: results out, places freed
      std::vector<Member> keep;
      bool retry_room = false;
      for (Member& mb : group) {
        const bool done = mb.st != SSNAL_EN_OK || ssnal::fit_phase(mb.fit) == ssnal::kFitPhaseDone;
        if (!done) {
          keep.push_back(std::move(mb));
          continue;
        }
        Request& q = *mb.q;
        ssnal_en_status st = mb.st;
        if (st == SSNAL_EN_ENOMEM && !mb.retried) {
          // a large active set ran out of device memory: free this worker's contexts of
          // other matrices and this one's panel, and run the request again
          cudaGetLastError();
          retry_room = true;
          mb.retried = true;
          ssnal::ctx_trim(mb.slot->ctx, 0);
          if ((mb.st = start_member(S, mb, s)) == SSNAL_EN_OK) {
            keep.push_back(std::move(mb));
            continue;
          }
          st = mb.st;
        }
        if (st == SSNAL_EN_OK) {
          st = ssnal::fit_end(mb.fit, &q.res);
        } else {
          q.res = ssnal_en_result{};
        }
        q.x.resize((size_t)S->mats[(size_t)q.mat].n);
        if ((st == SSNAL_EN_OK || st == SSNAL_EN_ENOCONV) && mb.slot &&
            (cudaMemcpyAsync(q.x.data(), mb.slot->x, sizeof(double) * q.x.size(), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
          st = SSNAL_EN_ECUDA;
        q.res.status = st;
        // a context kept for later requests does not keep the panel of a large active set
        if (mb.slot && mb.slot->ctx) ssnal::ctx_trim(mb.slot->ctx, 4 * ssnal::ctx_m(mb.slot->ctx));
        ssnal::fit_delete(mb.fit);
        {
          std::lock_guard<std::mutex> lk(S->mu);
          q.done = true;
          q.t_done = S->now();
          S->bytes_in_flight -= mb.need;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
      }
      if (retry_room)
        for (size_t k = 0; k < pool.size(); k++)
          if ((int)k != mat) {
            for (Slot& sl : pool[k]) release_slot(sl);
            pool[k].clear();
          }
      group = std::move(keep);
      started = group.size();
      // continuous batching: queued requests on this matrix join the group
      {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->stop) admit_same_matrix(S, mat, group, false);
      }
      if (group.empty()) break;
    }
  }
  for (auto& p : pool)
    for (Slot& sl : p) release_slot(sl);
  if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

ssnal_en_status ssnal_en_server_create(ssnal_en_server** out, const ssnal_en_matrix* mats, int32_t nmat,
                                       const ssnal_en_options* opts, int32_t workers, int64_t max_bytes) {
  if (!out || !mats || nmat <= 0 || workers <= 0 || workers > 256) return SSNAL_EN_EINVAL;
  *out = nullptr;
  for (int32_t i = 0; i < nmat; i++)
    if (!mats[i].data || mats[i].m <= 0 || mats[i].n <= 0) return SSNAL_EN_EINVAL;
  ssnal_en_server* S = new (std::nothrow) ssnal_en_server();
  if (!S) return SSNAL_EN_ENOMEM;
  S->mats.assign(mats, mats + nmat);
  if (opts)
    S->opts = *opts;
  else
    ssnal_en_default_options(&S->opts);
  S->max_bytes = max_bytes;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return SSNAL_EN_ECUDA;
  }
  for (int32_t w = 0; w < workers; w++) S->workers.emplace_back(worker_main, S);
  *out = S;
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_server_set_group(ssnal_en_server* S, int32_t max_group) {
  if (!S || max_group < 1 || max_group > 64) return SSNAL_EN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_group = max_group;
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_server_submit(ssnal_en_server* S, int32_t mat, const double* b_host, double lambda1,
                                       double lambda2, int64_t* ticket) {
  if (!S || !b_host || !ticket || mat < 0 || mat >= (int32_t)S->mats.size()) return SSNAL_EN_EINVAL;
  if (!std::isfinite(lambda1) || !std::isfinite(lambda2) || lambda1 < 0 || lambda2 < 0) return SSNAL_EN_EINVAL;
  auto q = std::make_shared<Request>();
  q->mat = mat;
  q->b.assign(b_host, b_host + S->mats[mat].m);
  q->lambda1 = lambda1;
  q->lambda2 = lambda2;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->ticket = S->next_ticket++;
    q->t_submit = S->now();
    S->tickets[q->ticket] = q;
    S->queue.push_back(q);
  }
  S->cv_work.notify_one();
  *ticket = q->ticket;
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_server_submit_scaled(ssnal_en_server* S, int32_t mat, const double* b_host, double alpha,
                                              double c, int64_t* ticket) {
  if (!S || !b_host || !ticket || mat < 0 || mat >= (int32_t)S->mats.size()) return SSNAL_EN_EINVAL;
  if (!(alpha > 0.0 && alpha <= 1.0) || !std::isfinite(c) || c < 0) return SSNAL_EN_EINVAL;
  auto q = std::make_shared<Request>();
  q->mat = mat;
  q->b.assign(b_host, b_host + S->mats[mat].m);
  q->scaled = true;
  q->alpha = alpha;
  q->c = c;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->ticket = S->next_ticket++;
    q->t_submit = S->now();
    S->tickets[q->ticket] = q;
    S->queue.push_back(q);
  }
  S->cv_work.notify_one();
  *ticket = q->ticket;
  return SSNAL_EN_OK;
}

ssnal_en_status ssnal_en_server_poll(ssnal_en_server* S, int64_t ticket, int32_t wait, double* x_host,
                                     ssnal_en_result* out, double* times, int32_t* done) {
  if (!S || !done) return SSNAL_EN_EINVAL;
  *done = 0;
  std::shared_ptr<Request> q;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return SSNAL_EN_EINVAL;
    q = it->second;
    if (wait)
      S->cv_done.wait(lk, [&] { return q->done; });
    if (!q->done) return SSNAL_EN_OK;
    S->tickets.erase(it);
  }
  if (x_host) memcpy(x_host, q->x.data(), sizeof(double) * q->x.size());
  if (out) *out = q->res;
  if (times) {
    times[0] = q->t_submit;
    times[1] = q->t_start;
    times[2] = q->t_done;
  }
  *done = 1;
  return SSNAL_EN_OK;
}

void ssnal_en_server_destroy(ssnal_en_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
