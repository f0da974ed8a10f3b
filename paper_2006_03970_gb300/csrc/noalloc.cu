// Allocation-free entry point: the prox / active-set step (the kernels of
// kern_vec.cu) with its scratch memory in a file-scope device array instead of
// a context's cudaMalloc'ed workspaces.
//
// Why: some callers must not allocate device memory -- for example code that
// runs while another component owns the whole device memory budget through its
// own pool, latency-critical loops where cudaMalloc/cudaFree (which may
// synchronise the device) are not acceptable, or plug-in code that is only
// allowed to use the buffers it is handed.  This entry point needs nothing but
// the caller's inputs and outputs.
//
// The scratch array is sized for at most kStaticMaxBlocks blocks of
// kStaticChunk elements, i.e. n <= SSNAL_EN_STATIC_MAX_N; it is held by every
// GPU that loads the library until the process exits.  All calls share it.
#include <math.h>

#include <mutex>

#include "../../include/ssnal_en.h"
#include "internal.h"

using namespace ssnal;

namespace {

constexpr long long kStaticChunk = 2048;   // elements per block
constexpr int kStaticMaxBlocks = 1024;     // blocks covered by the scratch array
static_assert(kStaticChunk * kStaticMaxBlocks == SSNAL_EN_STATIC_MAX_N, "limit in the header");

struct StaticScratch {
  DevState st;                                // r and the norms
  long long counts[2 * kStaticMaxBlocks + 2];  // per-block counts
  double partials[6 * kStaticMaxBlocks];      // per-block partial norms
};

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // device address of the array, per device
std::mutex g_scratch_mu;

}  // namespace

// The scratch itself (about 66 KB), zero at module load.
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

// Device address of the scratch array on the current device.  The array's name
// is only a host-side stand-in in host code, so the address is looked up once
// per device, with that device current, and cached.
static ssnal_en_status scratch_on_current_device(StaticScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SSNAL_EN_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SSNAL_EN_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SSNAL_EN_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<StaticScratch*>(g_scratch_addr[dev]);
  return SSNAL_EN_OK;
}

extern "C" ssnal_en_status ssnal_en_prox_active_static(const double* x, const double* u, int64_t n, double sigma,
                                                       double lambda1, double lambda2, int32_t* J, double* wJ,
                                                       int64_t* r, void* stream) {
  if (!x || !u || !J || !wJ || !r || n <= 0) return SSNAL_EN_EINVAL;
  if (n > SSNAL_EN_STATIC_MAX_N) return SSNAL_EN_ENOTSUP;  // beyond what the scratch array covers
  if (!(sigma > 0) || !std::isfinite(sigma) || !std::isfinite(lambda1) || !std::isfinite(lambda2) || lambda1 < 0 ||
      lambda2 < 0)
    return SSNAL_EN_EINVAL;
  StaticScratch* sc = nullptr;
  ssnal_en_status e = scratch_on_current_device(&sc);
  if (e != SSNAL_EN_OK) return e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the state starts at zero; counts and partials are written before they are read.
  if (cudaMemsetAsync(&sc->st, 0, sizeof(DevState), s) != cudaSuccess) return SSNAL_EN_ECUDA;
  const int grid = (int)((n + kStaticChunk - 1) / kStaticChunk);
  ProxParams pp;
  pp.sigma = sigma;
  pp.lam1 = lambda1;
  pp.lam2 = lambda2;
  pp.thr = sigma * lambda1;
  pp.onep = 1.0 + sigma * lambda2;
  pp.inv_onep = 1.0 / pp.onep;
  launch_prox_count(kProxThreshold, x, const_cast<double*>(u), nullptr, nullptr, nullptr, n, 0, pp, 0, &sc->st,
                    sc->counts, sc->partials, grid, s);
  launch_prox_scatter(kProxThreshold, x, u, n, pp, sc->counts, sc->partials, &sc->st, J, wJ, grid, s);
  if (cudaGetLastError() != cudaSuccess) return SSNAL_EN_ECUDA;
  long long rv = 0;
  if (cudaMemcpyAsync(&rv, &sc->st.r, sizeof(rv), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SSNAL_EN_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SSNAL_EN_ECUDA;
  *r = rv;
  return SSNAL_EN_OK;
}
