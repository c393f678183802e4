// CUDA kernels of the hot path and their launchers.
//
//  * integrand_kernel: one fused pass over a range of events: Philox
//    uniforms -> VEGAS map -> phase space -> PDFs -> |M|^2 -> weight ->
//    Kahan FP64 sums and shared-memory histograms -> per-block partials and
//    global histogram atomics.  Nothing per event touches global memory.
//  * ws_integrand_kernel (ws_integrand.cuh): the same pass for gg -> t tbar g
//    in FP32 mode with producer (kinematics) and consumer (|M|^2) warps.
//  * finalize_kernel: fixed-order reduction of the per-block partials
//    (deterministic sums for a given launch shape).
//  * refine_kernel: VEGAS rebinning, one thread per dimension, FP64.
//  * pdf_xfxq2_kernel: batched log-bicubic PDF interpolation (all flavours).
#include <cstdio>
#include <type_traits>

#include "../../include/mcint.h"
#include "event.cuh"
#include "integrand.cuh"
#include "launch.h"
#include "refine.cuh"
#include "ws_integrand.cuh"

namespace mc {

template <class R> MC_D const R* edges_of(const KernelArgs& a);
template <> MC_D const double* edges_of<double>(const KernelArgs& a) { return a.edges64; }
template <> MC_D const float* edges_of<float>(const KernelArgs& a) { return a.edges32; }

template <int PROC, bool FP64, bool RECORD>
__global__ void __launch_bounds__(kBlock) integrand_kernel(KernelArgs a) {
  using R = typename std::conditional<FP64, double, float>::type;
  // per-bin sums of w^2: FP64 in FP64 mode, FP32 in FP32 mode (a block's
  // partial histogram only steers the refinement; the global sum is FP64)
  using H = typename std::conditional<FP64, double, float>::type;
  constexpr int NFL = ProcTraits<PROC>::NFL;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ndim = a.ndim, nb = a.nbins;
  const int nedge = ndim * (nb + 1), nhist = ndim * nb;
  H* sh_w2 = reinterpret_cast<H*>(smem);
  unsigned int* sh_n = reinterpret_cast<unsigned int*>(smem + size_t(nhist) * 8);
  R* sh_edges = reinterpret_cast<R*>(smem + ((size_t(nhist) * 12 + 15) / 16) * 16);
  R* sh_pdf = sh_edges + nedge;

  const R* g_edges = edges_of<R>(a);
  for (int i = threadIdx.x; i < nedge; i += blockDim.x) sh_edges[i] = g_edges[i];
  if (!RECORD)
    for (int i = threadIdx.x; i < nhist; i += blockDim.x) {
      sh_w2[i] = H(0);
      sh_n[i] = 0u;
    }
  SmPdf<R> pdf;
  if constexpr (NFL > 0) {
    const int nx = a.pdf.nx;
    R* t = sh_pdf;
    R* f = t + nx;
    R* d = f + NFL * nx;
    build_pdf_tables<R>(a.pdf, a.logq2_f, a.fl, NFL, t, f, d);  // ends with __syncthreads
#pragma unroll
    for (int k = 0; k < NFL; ++k) pdf.tab[k] = {t, f + k * nx, d + k * nx, nx};
  } else {
    __syncthreads();
  }

  Acc acc;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double* rec = RECORD ? a.record + size_t(i) * MC_REC_STRIDE : nullptr;
    const double w = process_event<PROC, FP64, RECORD, R, H>(a, pdf, sh_edges, sh_w2, sh_n, a.first + uint64_t(i),
                                                             rec, acc);
    if (!RECORD && a.wout) a.wout[i] = w;
  }
  if (RECORD) return;
  if constexpr (PROC == P_GG_TTBARG_MC) channel_sums_add(acc, a.wch);
  __shared__ BlockPartial warp_part[kBlock / 32];
  block_reduce(acc, warp_part, &a.partials[blockIdx.x]);
  for (int i = threadIdx.x; i < nhist; i += blockDim.x) {
    if (sh_n[i]) {
      atomicAdd(&a.hist_n[i], sh_n[i]);
      atomicAdd(&a.hist_w2[i], double(sh_w2[i]));
    }
  }
}

// Fixed-order reduction of nblocks partials into out (one block of 256).
__global__ void finalize_kernel(const BlockPartial* parts, int nblocks, BlockPartial* out) {
  __shared__ BlockPartial sh[256];
  BlockPartial b = {0.0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) partial_add(b, parts[i]);
  sh[threadIdx.x] = b;
  __syncthreads();
  for (int width = blockDim.x / 2; width > 0; width >>= 1) {
    if (int(threadIdx.x) < width) partial_add(sh[threadIdx.x], sh[threadIdx.x + width]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Refinement kernel of one grid: one warp per dimension (refine_dimension in
// refine.cuh); dynamic shared memory ndim * (3 nbins + 2) doubles.
__global__ void refine_kernel(double* edges, float* edges32, double* hist_w2, unsigned int* hist_n, int ndim,
                              int nbins, double alpha) {
  extern __shared__ double refine_smem[];
  const int d = threadIdx.x >> 5;
  if (d >= ndim) return;
  refine_dimension(edges + size_t(d) * (nbins + 1), edges32 + size_t(d) * (nbins + 1), hist_w2 + size_t(d) * nbins,
                   hist_n + size_t(d) * nbins, nbins, alpha, refine_smem + size_t(d) * (3 * nbins + 2));
}

// Batched xf(x, Q^2) for all flavours: one thread per (point, flavour).
template <class R>
__global__ void pdf_xfxq2_kernel(PdfDev pdf, long long n, const double* x, const double* q2, double* out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * pdf.nflav) return;
  const long long i = idx / pdf.nflav;
  const int fl = int(idx % pdf.nflav);
  const double xv = x[i], qv = q2[i];
  const int nx = pdf.nx, nq = pdf.nq;
  const double lx = log(xv), lq = log(qv);
  if (!(lx >= pdf.logx[0] && lx <= pdf.logx[nx - 1] && lq >= pdf.logq2[0] && lq <= pdf.logq2[nq - 1])) {
    out[idx] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  int j0;
  double w[4];
  q_weights(pdf.logq2, nq, lq, &j0, w);
  const int ix = knot_cell(pdf.logx, nx, lx);
  const R h = R(pdf.logx[ix + 1] - pdf.logx[ix]);
  const R tau = R((lx - pdf.logx[ix]) / double(h));
  // slope stencil in x: knots ix-1 .. ix+2
  R tk[4];
  for (int t = 0; t < 4; ++t) {
    const int ii = min(max(ix - 1 + t, 0), nx - 1);
    tk[t] = R(pdf.logx[ii]);
  }
  double acc = 0.0;
  for (int t = 0; t < 4; ++t) {
    const int j = j0 + t;
    if (j < 0 || j >= nq || w[t] == 0.0) continue;
    const size_t base = (size_t(fl) * nq + j) * nx;
    R f[4];
    for (int u = 0; u < 4; ++u) {
      const int ii = min(max(ix - 1 + u, 0), nx - 1);
      f[u] = sizeof(R) == 8 ? R(pdf.xf64[base + ii]) : R(pdf.xf32[base + ii]);
    }
    R d0, d1;
    if (ix == 0)
      d0 = (f[2] - f[1]) / (tk[2] - tk[1]);
    else
      d0 = R(0.5) * ((f[2] - f[1]) / (tk[2] - tk[1]) + (f[1] - f[0]) / (tk[1] - tk[0]));
    if (ix + 1 == nx - 1)
      d1 = (f[2] - f[1]) / (tk[2] - tk[1]);
    else
      d1 = R(0.5) * ((f[3] - f[2]) / (tk[3] - tk[2]) + (f[2] - f[1]) / (tk[2] - tk[1]));
    acc += w[t] * double(hermite<R>(tau, h, f[1], f[2], d0, d1));
  }
  out[idx] = acc;
}

// ------------------------------------------------------------------ launchers
template <int PROC, bool FP64, bool RECORD>
static cudaError_t launch_one(const KernelArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto k = integrand_kernel<PROC, FP64, RECORD>;
  (void)cudaGetLastError();  // report only this launch's error below
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k<<<grid, kBlock, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PROC>
static cudaError_t launch_ws(const KernelArgs& a, int grid, cudaStream_t st) {
  const bool rows = ws_rows_in_smem(PROC, a.ndim, a.nbins, a.pdf.nx);
  auto k = a.wout ? (rows ? ws_integrand_kernel<PROC, true, true> : ws_integrand_kernel<PROC, true, false>)
                  : (rows ? ws_integrand_kernel<PROC, false, true> : ws_integrand_kernel<PROC, false, false>);
  const size_t smem = ws_smem_bytes(PROC, a.ndim, a.nbins, a.pdf.nx, rows);
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, kWsThreads, smem, st>>>(a);
  return cudaGetLastError();
}

bool integrand_ws(int proc, bool fp64) {
  return !fp64 && (proc == P_GG_TTBARG || proc == P_GG_TTBARG_7D || proc == P_GG_TTBARG_MC);
}
int integrand_threads(int proc, bool fp64) { return integrand_ws(proc, fp64) ? kWsThreads : kBlock; }
// events one block takes per round of its grid-stride loop
int integrand_block_events(int proc, bool fp64) { return integrand_ws(proc, fp64) ? 32 * kWsProducerWarps : kBlock; }

template <bool RECORD>
static cudaError_t dispatch(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (!RECORD && integrand_ws(proc, fp64))
    return proc == P_GG_TTBARG      ? launch_ws<P_GG_TTBARG>(a, grid, st)
           : proc == P_GG_TTBARG_7D ? launch_ws<P_GG_TTBARG_7D>(a, grid, st)
                                    : launch_ws<P_GG_TTBARG_MC>(a, grid, st);
  switch (proc) {
    case P_EE_MUMU:
      return fp64 ? launch_one<P_EE_MUMU, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_EE_MUMU, false, RECORD>(a, grid, smem, st);
    case P_PP_TTBAR:
      return fp64 ? launch_one<P_PP_TTBAR, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_PP_TTBAR, false, RECORD>(a, grid, smem, st);
    case P_GG_TTBARG:
      return fp64 ? launch_one<P_GG_TTBARG, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_GG_TTBARG, false, RECORD>(a, grid, smem, st);
    case P_GAUSS:
      return fp64 ? launch_one<P_GAUSS, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_GAUSS, false, RECORD>(a, grid, smem, st);
    case P_GG_TTBARG_7D:
      return fp64 ? launch_one<P_GG_TTBARG_7D, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_GG_TTBARG_7D, false, RECORD>(a, grid, smem, st);
    case P_GG_TTBARG_MC:
      return fp64 ? launch_one<P_GG_TTBARG_MC, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_GG_TTBARG_MC, false, RECORD>(a, grid, smem, st);
    case P_PP_TTBARJ:
      return fp64 ? launch_one<P_PP_TTBARJ, true, RECORD>(a, grid, smem, st)
                  : launch_one<P_PP_TTBARJ, false, RECORD>(a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

size_t integrand_smem(int proc, bool fp64, int ndim, int nbins, int nx) {
  if (integrand_ws(proc, fp64)) return ws_smem_bytes(proc, ndim, nbins, nx);
  const size_t r = fp64 ? 8 : 4;
  const int nfl = (proc == P_PP_TTBAR || proc == P_PP_TTBARJ)
                      ? 11
                      : ((proc == P_GG_TTBARG || proc == P_GG_TTBARG_7D || proc == P_GG_TTBARG_MC) ? 1 : 0);
  const size_t hist = ((size_t(ndim) * nbins * 12 + 15) / 16) * 16;
  return hist + r * (size_t(ndim) * (nbins + 1) + (nfl > 0 ? size_t(nx) * (1 + 2 * nfl) : 0));
}

int integrand_max_blocks_per_sm(int proc, bool fp64, size_t smem) {
  if (integrand_ws(proc, fp64)) return 1;
  int nb = 0;
  cudaError_t e = cudaSuccess;
#define MC_OCC(P)                                                                                        \
  e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, integrand_kernel<P, true, false>, kBlock, smem) \
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, integrand_kernel<P, false, false>, kBlock, smem)
  switch (proc) {
    case P_EE_MUMU: MC_OCC(P_EE_MUMU); break;
    case P_PP_TTBAR: MC_OCC(P_PP_TTBAR); break;
    case P_GG_TTBARG: MC_OCC(P_GG_TTBARG); break;
    case P_GG_TTBARG_7D: MC_OCC(P_GG_TTBARG_7D); break;
    case P_GG_TTBARG_MC: MC_OCC(P_GG_TTBARG_MC); break;
    case P_PP_TTBARJ: MC_OCC(P_PP_TTBARJ); break;
    default: MC_OCC(P_GAUSS); break;
  }
#undef MC_OCC
  if (e != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_integrand(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem, cudaStream_t st) {
  return dispatch<false>(proc, fp64, a, grid, smem, st);
}
cudaError_t launch_integrand_record(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem,
                                    cudaStream_t st) {
  return dispatch<true>(proc, fp64, a, grid, smem, st);
}
cudaError_t launch_finalize(const BlockPartial* parts, int nblocks, BlockPartial* out, cudaStream_t st) {
  (void)cudaGetLastError();
  finalize_kernel<<<1, 256, 0, st>>>(parts, nblocks, out);
  return cudaGetLastError();
}
cudaError_t launch_refine(double* edges, float* edges32, double* hist_w2, unsigned int* hist_n, int ndim, int nbins,
                          double alpha, cudaStream_t st) {
  const size_t smem = sizeof(double) * size_t(ndim) * (3 * nbins + 2);
  (void)cudaGetLastError();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  refine_kernel<<<1, 32 * ndim, smem, st>>>(edges, edges32, hist_w2, hist_n, ndim, nbins, alpha);
  return cudaGetLastError();
}
cudaError_t launch_pdf_xfxq2(const PdfDev& pdf, bool fp64, long long n, const double* x, const double* q2,
                             double* out, cudaStream_t st) {
  const long long total = n * pdf.nflav;
  if (total == 0) return cudaSuccess;
  (void)cudaGetLastError();
  const int block = 256;
  const long long grid = (total + block - 1) / block;
  if (fp64)
    pdf_xfxq2_kernel<double><<<unsigned(grid), block, 0, st>>>(pdf, n, x, q2, out);
  else
    pdf_xfxq2_kernel<float><<<unsigned(grid), block, 0, st>>>(pdf, n, x, q2, out);
  return cudaGetLastError();
}

}  // namespace mc
