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

// ---------------------------------------------------------------------------
// Device-resident batch (kern_batch.cu): one persistent kernel for all instances.
// The host sorts the instances by m * n, largest first (the kernel's CTAs take them in
// that order from a device counter, so the long fits start first and the short ones fill
// the tail), copies the descriptors, and picks the loads in flight per lane of the
// passes over A on the batch itself: the first three slices of the order (one instance
// per CTA each) run with 4, 8 and 16 loads in flight and the rest of the batch with the
// depth that processed the most m * n per second.  The depth does not change any sum's
// order, so the results do not depend on the choice.  Instances the kernel hands back
// (their FP32 Newton solve failed or did not contract) are solved again on the regular
// path (FP64 Newton system) from their warm start.
extern "C" ssnal_en_status ssnal_en_solve_batch_resident(const ssnal_en_batch_fit* fits, int64_t count,
                                                         const ssnal_en_options* opts, ssnal_en_result* out,
                                                         int32_t* info, void* stream) {
  if (info) info[0] = info[1] = 0;
  if (!fits || !out || count < 1 || count > 0x7fffffff) return SSNAL_EN_EINVAL;
  ssnal_en_options o;
  if (opts)
    o = *opts;
  else
    ssnal_en_default_options(&o);
  if (!(o.sigma0 > 0) || !(o.tol > 0) || o.max_al < 1 || o.max_ls < 1 || o.max_ls > 64 || o.refine_steps < 0)
    return SSNAL_EN_EINVAL;
  long long n_max = 0;
  int m_max = 0;
  for (int64_t i = 0; i < count; i++) {
    const ssnal_en_batch_fit& f = fits[i];
    if (!f.A || !f.b || !f.x || f.m <= 0 || f.n <= 0 || f.lda < f.m) return SSNAL_EN_EINVAL;
    if (!std::isfinite(f.lambda1) || !std::isfinite(f.lambda2) || f.lambda1 < 0 || f.lambda2 < 0)
      return SSNAL_EN_EINVAL;
    if (f.m > ssnal::kBatchMaxM || f.n >= 0x7fffffffLL) return SSNAL_EN_ENOTSUP;
    n_max = std::max<long long>(n_max, f.n);
    m_max = std::max<int>(m_max, (int)f.m);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SSNAL_EN_ECUDA;
  const int blocks = sms;
  std::vector<int> order((size_t)count);
  for (int64_t i = 0; i < count; i++) order[(size_t)i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)fits[a].m * (double)fits[a].n > (double)fits[b].m * (double)fits[b].n;
  });
  const size_t ib = ssnal::batch_inst_bytes(), ob = ssnal::batch_out_bytes();
  std::vector<unsigned char> hin(ib * (size_t)count), hout(ob * (size_t)count);
  for (int64_t i = 0; i < count; i++) {
    const ssnal_en_batch_fit& f = fits[i];
    ssnal::batch_fill_inst(hin.data() + ib * (size_t)i, f.A, f.lda, f.n, (int)f.m, f.b, f.lambda1, f.lambda2, f.x);
  }
  unsigned char *din = nullptr, *dout = nullptr, *scratch = nullptr;
  int *dorder = nullptr, *dnext = nullptr;
  const size_t slot = ssnal::batch_slot_bytes(n_max, m_max);
  ssnal_en_status st = SSNAL_EN_OK;
  if (cudaMalloc(&din, ib * (size_t)count) != cudaSuccess || cudaMalloc(&dout, ob * (size_t)count) != cudaSuccess ||
      cudaMalloc(&dorder, sizeof(int) * (size_t)count) != cudaSuccess || cudaMalloc(&dnext, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&scratch, slot * (size_t)blocks) != cudaSuccess)
    st = SSNAL_EN_ENOMEM;
  if (st == SSNAL_EN_OK &&
      (cudaMemcpyAsync(din, hin.data(), ib * (size_t)count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(dorder, order.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemsetAsync(dnext, 0, sizeof(int) * 4, s) != cudaSuccess))
    st = SSNAL_EN_ECUDA;
  const double opt6[6] = {o.sigma0, o.sigma_growth, o.sigma_max, o.mu, o.beta, o.tol};
  const int opt4[4] = {o.max_al, o.max_newton, o.max_ls, o.refine_steps};
  int depth = 8;
  int64_t done = 0;
  if (st == SSNAL_EN_OK && count >= 4 * (int64_t)blocks) {
    // tune the loads in flight on three slices of the (largest-first) order
    static const int cand[3] = {4, 8, 16};
    double best = -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < 3 && st == SSNAL_EN_OK; c++) {
      const int64_t end = std::min<int64_t>(count, done + blocks);
      double work = 0.0;
      for (int64_t i = done; i < end; i++) work += (double)fits[order[(size_t)i]].m * (double)fits[order[(size_t)i]].n;
      cudaEventRecord(e0, s);
      if (!ssnal::launch_batch_solve(din, dorder + done, (int)(end - done), dnext + c, dout, opt6, opt4, n_max, m_max,
                                     scratch, blocks, cand[c], s))
        st = SSNAL_EN_ECUDA;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = SSNAL_EN_ECUDA;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = ms > 0 ? work / ms : 0.0;
      if (rate > best) {
        best = rate;
        depth = cand[c];
      }
      done = end;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (st == SSNAL_EN_OK && done < count &&
      !ssnal::launch_batch_solve(din, dorder + done, (int)(count - done), dnext + 3, dout, opt6, opt4, n_max, m_max,
                                 scratch, blocks, depth, s))
    st = SSNAL_EN_ECUDA;
  if (st == SSNAL_EN_OK &&
      (cudaMemcpyAsync(hout.data(), dout, ob * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    st = SSNAL_EN_ECUDA;
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dorder);
  cudaFree(dnext);
  cudaFree(scratch);
  if (st != SSNAL_EN_OK) return st;
  // read the results; instances handed back are solved on the regular path
  int rehost = 0;
  ssnal_en_status worst = SSNAL_EN_OK;
  for (int64_t i = 0; i < count; i++) {
    int needs = 0;
    ssnal_en_result r{};
    ssnal::batch_read_out(hout.data() + ob * (size_t)i, &r, &needs);
    const ssnal_en_batch_fit& f = fits[i];
    r.lambda1 = f.lambda1;
    r.lambda2 = f.lambda2;
    if (needs) {
      rehost++;
      ssnal_en_matrix A{f.m, f.n, f.lda, SSNAL_EN_F32, 0, f.A, nullptr, nullptr};
      ssnal_en_ctx* ctx = nullptr;
      ssnal_en_status e = ssnal_en_create(&ctx, &A, &o, stream);
      if (e == SSNAL_EN_OK) {
        e = ssnal_en_solve(ctx, f.b, f.lambda1, f.lambda2, f.x, nullptr, &r);
        ssnal_en_destroy(ctx);
      }
      if (e != SSNAL_EN_OK && e != SSNAL_EN_ENOCONV) r.status = e;
    }
    out[i] = r;
    if (r.status != SSNAL_EN_OK && worst == SSNAL_EN_OK) worst = (ssnal_en_status)r.status;
  }
  if (info) {
    info[0] = depth;
    info[1] = rehost;
  }
  return worst;
}
