// Allocation-free VEGAS iteration (mc_vegas_iterate_noalloc in
// include/mcint.h) for callers that must not allocate device memory while
// they run.  The only scratch of the fused launch, the per-block partial
// sums, lives in the file-scope device array below; the histograms and the
// sums go to buffers the caller passes in.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "handles.h"

namespace {

__device__ __align__(256) mc::BlockPartial g_noalloc_partials[MC_NOALLOC_MAX_BLOCKS];

static_assert(sizeof(mc_device_sums) == sizeof(mc::BlockPartial), "mc_device_sums must mirror BlockPartial");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
cudaError_t scratch_for(int dev, mc::BlockPartial** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = static_cast<mc::BlockPartial*>(g_scratch[dev]);
  return cudaSuccess;
}

int reject(int code, const char* msg) {
  mc::set_last_error((std::string("mc_vegas_iterate_noalloc: ") + msg).c_str());
  return code;
}

}  // namespace

extern "C" int mc_vegas_iterate_noalloc(const mc_integrand* itg, mc_pdf pdf, int ndim, int nbins,
                                        const double* edges64, const float* edges32, int prec, uint64_t seed,
                                        uint32_t iteration, uint32_t gid, int64_t nevents, int blocks,
                                        double* hist_w2, uint32_t* hist_n, mc_device_sums* sums, void* stream) {
  if (!itg || !edges64 || !hist_w2 || !hist_n || !sums) return reject(MC_EINVAL, "NULL argument");
  if (prec != MC_FP64 && prec != MC_FP32_KAHAN) return reject(MC_EINVAL, "bad precision");
  if (prec == MC_FP32_KAHAN && !edges32) return reject(MC_EINVAL, "FP32 mode needs edges32");
  if (ndim < 1 || ndim > MC_MAX_DIM || nbins < 2 || nbins > MC_MAX_BINS) return reject(MC_EINVAL, "bad grid shape");
  // the three-channel process keeps its channel probabilities and their
  // update sums in a VEGAS handle, which this entry point does not take
  if (itg->proc == MC_GG_TTBARG_MC)
    return reject(MC_EINVAL, "MC_GG_TTBARG_MC is not supported (it needs a VEGAS handle; use mc_vegas_iterate)");
  const int nd = mc::process_dim(itg);
  if (nd < 1) return reject(MC_EINVAL, "unknown process or gauss_dim outside 1..16");
  if (nd != ndim) return reject(MC_EINVAL, "grid dimension does not match the process");
  if (nevents < 0) return reject(MC_EINVAL, "negative event count");
  if (blocks < 0 || blocks > MC_NOALLOC_MAX_BLOCKS)
    return reject(MC_EINVAL, "blocks exceeds MC_NOALLOC_MAX_BLOCKS (the size of the static scratch)");
  if (gid > 255) return reject(MC_EINVAL, "gid outside 0..255");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return reject(MC_ECUDA, "no device");
  mc::BlockPartial* scratch = nullptr;
  if (scratch_for(dev, &scratch) != cudaSuccess) return reject(MC_ECUDA, "cudaGetSymbolAddress failed");

  // the same validation and process arguments as mc_vegas_iterate (host
  // work only: it allocates nothing on the device)
  mc::KernelArgs a;
  if (int rc = mc::fill_process_args(itg, pdf, &a)) {
    const std::string msg = mc_last_error();
    return reject(rc, msg.c_str());
  }
  a.ndim = ndim;
  a.nbins = nbins;
  a.edges64 = edges64;
  a.edges32 = edges32;
  a.seed = seed;
  a.iteration = iteration;
  a.gid = gid;
  a.hist_w2 = hist_w2;
  a.hist_n = hist_n;
  a.partials = scratch;
  a.first = 0;
  a.n = nevents;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool fp64 = prec == MC_FP64;
  const size_t smem = mc::integrand_smem(itg->proc, fp64, ndim, nbins, pdf ? pdf->nx : 0);
  int grid = blocks;
  if (grid == 0) {
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (long long)sms * mc::integrand_max_blocks_per_sm(itg->proc, fp64, smem);
    const int per_block = mc::integrand_block_events(itg->proc, fp64);
    const long long need = (nevents + per_block - 1) / per_block;
    if (g > need) g = need;
    if (g > MC_NOALLOC_MAX_BLOCKS) g = MC_NOALLOC_MAX_BLOCKS;
    grid = int(g < 1 ? 1 : g);
  }
  if (nevents == 0) {
    if (cudaMemsetAsync(sums, 0, sizeof(*sums), st) != cudaSuccess) return reject(MC_ECUDA, "cudaMemsetAsync failed");
    return MC_OK;
  }
  if (mc::launch_integrand(itg->proc, fp64, a, grid, smem, st) != cudaSuccess)
    return reject(MC_ECUDA, "integrand launch failed");
  if (mc::launch_finalize(scratch, grid, reinterpret_cast<mc::BlockPartial*>(sums), st) != cudaSuccess)
    return reject(MC_ECUDA, "finalize launch failed");
  return MC_OK;
}
