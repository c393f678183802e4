// FMA throughput of the CUDA cores (C ABI: mc_fma_peak in include/mcint.h):
// the denominators of the roofline of the integrand kernels, measured on the
// device instead of derived from unit counts.  Every thread of a full-occupancy
// grid runs kChains independent chains of dependent fused multiply-adds
// x <- x a + b, so the FMA pipe of every sub-partition always has independent
// work; the chains' results are stored so nothing is folded away.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/mcint.h"

namespace mc {
void set_last_error(const char* msg);  // api.cu

namespace {
constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float sum_pair(unsigned long long v) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(v));
  return l + h;
}
__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// kind 0: fma.rn.f32 (2 FLOP per lane), 1: fma.rn.f32x2 (4 FLOP per lane),
// 2: fma.rn.f64 (2 FLOP per lane)
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, float a, float b, float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (KIND == 0) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = float(t + j) * 1e-9f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[t] = s;
  } else if constexpr (KIND == 1) {
    unsigned long long x[kChains];
    const unsigned long long a2 = pk(a, a), b2 = pk(b, b);
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = pk(float(t + j) * 1e-9f, float(t - j) * 1e-9f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma_x2(x[j], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += sum_pair(x[j]);
    out[t] = s;
  } else {
    double x[kChains];
    const double ad = a, bd = b;
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = double(t + j) * 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], ad, bd);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[t] = float(s);
  }
}

int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}
}  // namespace
}  // namespace mc

extern "C" int mc_fma_peak(int kind, int iters, float* out, int64_t out_len, double* flop, void* stream) {
  if (kind < 0 || kind > 2 || iters < 1 || !out || !flop) return mc::fail(MC_EINVAL, "mc_fma_peak: bad argument");
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
    return mc::fail(MC_ECUDA, "mc_fma_peak: no device");
  const int blocks = sms * (per_sm / mc::kPeakThreads);
  const int64_t threads = int64_t(blocks) * mc::kPeakThreads;
  if (out_len < threads) return mc::fail(MC_EINVAL, "mc_fma_peak: out must hold one float per thread");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a and b keep every chain bounded: x -> x a + b with |a| < 1 converges
  const float a = 0.999f, b = 1e-3f;
  if (kind == 0) mc::fma_peak_kernel<0><<<blocks, mc::kPeakThreads, 0, st>>>(iters, a, b, out);
  if (kind == 1) mc::fma_peak_kernel<1><<<blocks, mc::kPeakThreads, 0, st>>>(iters, a, b, out);
  if (kind == 2) mc::fma_peak_kernel<2><<<blocks, mc::kPeakThreads, 0, st>>>(iters, a, b, out);
  if (cudaGetLastError() != cudaSuccess) return mc::fail(MC_ECUDA, "mc_fma_peak: launch failed");
  *flop = double(threads) * iters * mc::kChains * (kind == 1 ? 4.0 : 2.0);
  return MC_OK;
}
