// Internal: tcgen05 BF16 GEMM C[M x N] (+)= A[M x K] . B[N x K]^T (tc_gemm.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mc {

enum TcEpilogue : int {
  kEpiBiasReluBf16 = 0,  // c_bf16 = bf16(relu(acc + bias))
  kEpiBiasF32 = 1,       // c_f32 = acc + bias (bias may be null)
  kEpiReluMaskBf16 = 2,  // c_bf16 = bf16(acc * [mask > 0]) (gradient through ReLU)
  kEpiAtomicF32 = 3,     // c_f32 += acc (split-K)
  kEpiPartialF32 = 4,    // c_f32[split] = acc: per-split partial tiles, summed by tc_reduce_splits
};

struct TcGemmArgs {
  int M, N, K;  // M % 128 == 0, K % 64 == 0, N % bn == 0
  int bn;       // N tile: multiple of 16, <= 256
  int epilogue;
  const float* bias;           // [N] or null
  float* c_f32;                // row-major, leading dimension ldc
  __nv_bfloat16* c_bf16;       // row-major, leading dimension ldc
  int ldc;
  const __nv_bfloat16* mask;   // kEpiReluMaskBf16: activation of the layer, leading dimension ld_mask
  int ld_mask;                 // (or, in tc_gemm_rs, mask == null and mask_t: the activation transposed,
  const __nv_bfloat16* mask_t; //  mask_t[col * ld_mask_t + row])
  int ld_mask_t;
  int* error;                  // device flag: set non-zero when a bounded wait timed out
  // optional transposed copies written by the persistent kernel (tc_gemm_rs):
  // c_t_bf16[col * ldt + row] (epilogues 0 and 2), c_t_f32[col * ldt + row] (epilogue 1)
  __nv_bfloat16* c_t_bf16;
  float* c_t_f32;
  int ldt;
  // optional with kEpiPartialF32 and a K-major B (tc_gemm, tc_gemm_xn): per
  // split the row sums of B over the split's K range, rowsum_b[split][N]
  // (the bias gradient of a dense layer beside its weight gradient), summed
  // by tc_reduce_splits like the partial tiles
  float* rowsum_b;
};

size_t tc_gemm_smem(int bn);
// 2D BF16 tensor map (128-byte swizzle) of a row-major [rows x k] matrix
// with leading dimension ld elements, box [box_rows x 64]; false on failure.
bool tc_make_map(CUtensorMap* m, const void* base, int rows, int k, int ld, int box_rows);
// a: [M x K] row-major (leading dimension lda), b: [N x K] row-major (ldb);
// 16-byte aligned, lda and ldb multiples of 8.  splits > 1 divides K across
// gridDim.z (use kEpiAtomicF32).  Returns cudaErrorInvalidValue on bad shapes.
cudaError_t tc_gemm(const TcGemmArgs& g, const __nv_bfloat16* a, int lda, const __nv_bfloat16* b, int ldb,
                    int splits, cudaStream_t st);

// Both operands MN-major: C[M x N] (+)= X^T Y with X [K x M] (leading
// dimension ldx >= M) and Y [K x N] (ldy >= N) row-major, split-K over
// `splits`; bn a multiple of 64, epilogues 1, 3 or 4.  The weight gradient
// of a dense layer straight from row-major activations and gradients.
cudaError_t tc_gemm_tn(const TcGemmArgs& g, const __nv_bfloat16* x, int ldx, const __nv_bfloat16* y, int ldy,
                       int splits, cudaStream_t st);

// A MN-major, B K-major: C[M x N] (+)= X^T B^T with X [K x M] row-major
// (ldx >= M) and B [N x K] row-major (ldb >= K), split-K over `splits`; bn a
// multiple of 16, epilogues 1, 3 or 4.  The weight gradient of a dense layer
// from row-major activations and transposed gradients.
cudaError_t tc_gemm_xn(const TcGemmArgs& g, const __nv_bfloat16* x, int ldx, const __nv_bfloat16* b, int ldb,
                       int splits, cudaStream_t st);

// Persistent variant for a long A and a short B (the dense layers applied to
// a batch): B [N x K] stays resident in shared memory (bn * K * 2 bytes <=
// 160 KiB, K <= 320), A tiles stream through a TMA ring, two TMEM
// accumulators let the epilogue of one tile overlap the MMAs of the next.
// Epilogues 0-2; row-major output optional when a transposed copy is asked
// for (c_bf16 / c_f32 may be null).  Same alignment rules as tc_gemm.
cudaError_t tc_gemm_rs(const TcGemmArgs& g, const __nv_bfloat16* a, int lda, const __nv_bfloat16* b, int ldb,
                       cudaStream_t st);

// out[i] += sum over s < splits of part[s * n + i] (fixed order), n floats.
cudaError_t tc_reduce_splits(const float* part, int splits, size_t n, float* out, cudaStream_t st);

// Up to kMaxRedSegs such sums in one launch, each segment summed exactly as
// tc_reduce_splits sums it alone (the segments' outputs must not overlap).
struct TcRedSeg {
  const float* part;
  int splits;
  size_t n;
  float* out;
};
constexpr int kMaxRedSegs = 8;
cudaError_t tc_reduce_splits_multi(const TcRedSeg* segs, int nseg, cudaStream_t st);

}  // namespace mc
