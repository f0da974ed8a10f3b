// Serving loop: design matrices stay resident on the device, requests (a new
// right-hand side and penalties on one of them) arrive at any time and are
// admitted while others run (continuous batching).  Worker threads, each with
// its own CUDA stream, take admitted requests in arrival order; a worker keeps
// one context per matrix it has served (workspaces, x, y, sigma and the
// Cholesky factor live on the device for the whole solve) and reuses it for the
// next request on that matrix.  Admission also bounds the device bytes of the
// contexts that requests in flight occupy.  A request's b is copied from host
// memory at the start of its solve and its x back at the end, so a request's
// latency covers its transfers.  Each request runs the same kernels in the same
// order as ssnal_en_solve on its own, so its result does not depend on the mix.
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

void worker_main(ssnal_en_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  std::vector<Slot> slots(S->mats.size());
  for (;;) {
    std::shared_ptr<Request> q;
    int64_t need = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        if (!S->queue.empty()) {
          need = context_bytes(S->mats[S->queue.front()->mat]);
          // admit by footprint: always when nothing is in flight, else within the bound
          if (S->max_bytes <= 0 || S->bytes_in_flight == 0 || S->bytes_in_flight + need <= S->max_bytes) break;
        }
        S->cv_work.wait(lk);
      }
      if (S->stop) break;
      q = S->queue.front();
      S->queue.pop_front();
      S->bytes_in_flight += need;
      q->t_start = S->now();
    }
    Slot& sl = slots[q->mat];
    ssnal_en_status st = SSNAL_EN_OK;
    const ssnal_en_matrix& A = S->mats[q->mat];
    if (!sl.ctx) {
      st = ssnal_en_create(&sl.ctx, &A, &S->opts, s);
      if (st == SSNAL_EN_OK && (cudaMalloc(&sl.b, sizeof(double) * A.m) != cudaSuccess ||
                                cudaMalloc(&sl.x, sizeof(double) * A.n) != cudaSuccess))
        st = SSNAL_EN_ENOMEM;
      if (st != SSNAL_EN_OK) {
        if (sl.ctx) ssnal_en_destroy(sl.ctx);
        if (sl.b) cudaFree(sl.b);
        sl = Slot();
      }
    }
    // a solve that runs out of device memory (a large active set grows the panel) is
    // retried once after this worker releases the contexts of its other matrices
    for (int attempt = 0; attempt < 2 && st == SSNAL_EN_OK; attempt++) {
      if (cudaMemcpyAsync(sl.b, q->b.data(), sizeof(double) * A.m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemsetAsync(sl.x, 0, sizeof(double) * A.n, s) != cudaSuccess) {
        st = SSNAL_EN_ECUDA;
        break;
      }
      if (q->scaled) {
        int32_t ndone = 0;
        st = ssnal_en_path(sl.ctx, sl.b, q->alpha, &q->c, 1, sl.x, &q->res, &ndone);
      } else {
        st = ssnal_en_solve(sl.ctx, sl.b, q->lambda1, q->lambda2, sl.x, nullptr, &q->res);
      }
      if (st != SSNAL_EN_ENOMEM || attempt > 0) break;
      cudaGetLastError();
      for (size_t k = 0; k < slots.size(); k++) {
        if ((int)k == q->mat || !slots[k].ctx) continue;
        ssnal_en_destroy(slots[k].ctx);
        cudaFree(slots[k].b);
        cudaFree(slots[k].x);
        slots[k] = Slot();
      }
      ssnal::ctx_trim(sl.ctx, 0);
      st = SSNAL_EN_OK;
    }
    if (st == SSNAL_EN_OK || st == SSNAL_EN_ENOCONV) {
      q->x.resize((size_t)A.n);
      if (cudaMemcpyAsync(q->x.data(), sl.x, sizeof(double) * A.n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        st = SSNAL_EN_ECUDA;
    }
    // a context kept for later requests does not keep the panel of a large active set
    if (sl.ctx) ssnal::ctx_trim(sl.ctx, 4 * ssnal::ctx_m(sl.ctx));
    q->res.status = st;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      q->done = true;
      q->t_done = S->now();
      S->bytes_in_flight -= need;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  for (Slot& sl : slots) {
    if (sl.ctx) ssnal_en_destroy(sl.ctx);
    if (sl.b) cudaFree(sl.b);
    if (sl.x) cudaFree(sl.x);
  }
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
