// Internal: launchers of the CUDA kernels (kernels.cu) used by the C ABI
// (api.cu).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/mcint.h"
#include "integrand.cuh"

namespace mc {

constexpr int kBlock = 128;  // threads per block of the fused integrand kernel

// The fused integrand launch: gg -> t tbar g in FP32 mode runs the
// warp-specialised kernel (integrand_threads() threads, one block per SM,
// integrand_block_events() events per block and round); everything else the
// per-thread kernel of kBlock threads.
bool integrand_ws(int proc, bool fp64);
int integrand_threads(int proc, bool fp64);
int integrand_block_events(int proc, bool fp64);
size_t integrand_smem(int proc, bool fp64, int ndim, int nbins, int nx);
int integrand_max_blocks_per_sm(int proc, bool fp64, size_t smem);
cudaError_t launch_integrand(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_integrand_record(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem,
                                    cudaStream_t st);
// The warp-specialised FP32 kernel at given points (KernelArgs::pts, nbins
// 0, no wout): g g -> t tbar g (14 or 7 dims) and p p -> t tbar + parton;
// the block sums of the weights f exp(-log q) into a.partials[grid] (one
// block per SM).
bool points_ws(int proc);
cudaError_t launch_points_ws(int proc, const KernelArgs& a, int grid, cudaStream_t st);
cudaError_t launch_finalize(const BlockPartial* parts, int nblocks, BlockPartial* out, cudaStream_t st);
cudaError_t launch_refine(double* edges, float* edges32, double* hist_w2, unsigned int* hist_n, int ndim, int nbins,
                          double alpha, cudaStream_t st);
// Unweighting of the events of a weights pass (unweight.cu): decision,
// scan, ordered compaction and export of the accepted events.  Scratch of
// unweight_scratch_bytes(n, cap) bytes, starting with counts
// [kUwMaxChunks + 1] whose last entry receives the number accepted.
constexpr int kUwMaxChunks = 1024;
cudaError_t unweight_launch(int proc, bool fp64, const KernelArgs& a, const double* w, double wmax, void* scratch,
                            mc_event* out, long long cap, int nsm, cudaStream_t st);
size_t unweight_scratch_bytes(long long n, long long cap);
cudaError_t launch_pdf_xfxq2(const PdfDev& pdf, bool fp64, long long n, const double* x, const double* q2,
                             double* out, cudaStream_t st);

}  // namespace mc
