// Many independent fits at once (uneven sizes): worker threads, each with its
// own non-blocking CUDA stream, take instances from a shared queue in index
// order and drive one SsNAL-EN solve at a time on their stream, so the small
// kernels and host round trips of different fits overlap on the device.  The
// number of workers is tuned on the batch itself when the caller passes 0:
// successive chunks of instances run with 4, 8, 16 and 32 workers and the rest
// of the batch uses the count that processed the most m*n per second (the
// entries of A summed over the chunk's instances, per second of wall time).  Every
// instance is solved exactly once, by the same kernels as ssnal_en_solve, so
// its result does not depend on the batch or the worker count.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/ssnal_en.h"
#include "internal.h"

namespace {

// Runs instances [begin, end) with `workers` threads; returns the wall time in seconds.
double run_range(ssnal_en_instance* inst, int64_t begin, int64_t end, int workers, ssnal_en_result* out, int dev) {
  std::atomic<int64_t> next{begin};
  auto t0 = std::chrono::steady_clock::now();
  std::vector<std::thread> pool;
  for (int w = 0; w < workers; w++) {
    pool.emplace_back([&, w]() {
      (void)w;
      cudaSetDevice(dev);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
      for (;;) {
        const int64_t i = next.fetch_add(1);
        if (i >= end) break;
        ssnal_en_instance& q = inst[i];
        cudaStream_t old = ssnal::ctx_set_stream(q.ctx, s);
        const ssnal_en_status st = ssnal_en_solve(q.ctx, q.b, q.lambda1, q.lambda2, q.x, q.y, &out[i]);
        out[i].status = st;
        ssnal::ctx_set_stream(q.ctx, old);
      }
      if (s) cudaStreamDestroy(s);
    });
  }
  for (auto& t : pool) t.join();
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" ssnal_en_status ssnal_en_solve_batch(ssnal_en_instance* inst, int64_t count, int32_t workers,
                                                ssnal_en_result* out, int32_t* workers_used) {
  if (workers_used) *workers_used = 0;
  if (!inst || !out || count < 0 || workers < 0) return SSNAL_EN_EINVAL;
  if (count == 0) return SSNAL_EN_OK;
  std::vector<ssnal_en_ctx*> seen;
  seen.reserve((size_t)count);
  for (int64_t i = 0; i < count; i++) {
    const ssnal_en_instance& q = inst[i];
    if (!q.ctx || !q.b || !q.x || !std::isfinite(q.lambda1) || !std::isfinite(q.lambda2) || q.lambda1 < 0 ||
        q.lambda2 < 0)
      return SSNAL_EN_EINVAL;
    seen.push_back(q.ctx);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return SSNAL_EN_EINVAL;  // one context per instance
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SSNAL_EN_ECUDA;
  int used = workers;
  int64_t done = 0;
  if (workers == 0) {
    // tune on the batch: chunks of about count / 16 instances per candidate
    static const int cand[4] = {4, 8, 16, 32};
    const int64_t chunk = std::max<int64_t>(8, count / 16);
    double best = -1.0;
    used = 8;
    for (int c = 0; c < 4 && done < count; c++) {
      const int64_t end = std::min<int64_t>(count, done + chunk);
      double work = 0.0;  // entries of A streamed per pass, summed over the chunk
      for (int64_t i = done; i < end; i++) work += ssnal::ctx_mn(inst[i].ctx);
      const double sec = run_range(inst, done, end, std::min<int64_t>(cand[c], end - done), out, dev);
      const double rate = sec > 0 ? work / sec : 0.0;
      if (rate > best) {
        best = rate;
        used = cand[c];
      }
      done = end;
    }
  }
  if (done < count) run_range(inst, done, count, (int)std::min<int64_t>(used, count - done), out, dev);
  if (workers_used) *workers_used = used;
  for (int64_t i = 0; i < count; i++)
    if (out[i].status != SSNAL_EN_OK) return (ssnal_en_status)out[i].status;
  return SSNAL_EN_OK;
}
