// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the dense layers
// of the normalizing-flow sampler:
//     C[M x N] (+)= A[M x K] . B[N x K]^T,   A, B in BF16, K-major (row-major);
// FP32 accumulation in tensor memory, with fused epilogues.
//
// One CTA (4 warps) computes one 128 x BN tile (BN <= 256, a multiple of 16)
// over its K range (split-K over gridDim.z).  One thread of warp 0 streams the
// K blocks (64 BF16 = 128 B per row, 128-byte swizzle) into a ring of shared-
// memory stages with TMA (cp.async.bulk.tensor, completion on an mbarrier);
// one thread of warp 1 issues tcgen05.mma (M = 128, N = BN, K = 16 per
// instruction) into a TMEM accumulator, and tcgen05.commit on a per-stage
// mbarrier returns the stage to the loader.  After the last MMA all four
// warps read the accumulator with tcgen05.ld (warp w owns rows 32w..32w+31,
// one row per thread) and apply the epilogue.  Every mbarrier wait is bounded: on timeout the kernel records an
// error code, waits (bounded) for its TMA copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace mc {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;          // K elements per stage (one 128-byte swizzle atom)
constexpr int kStages = 4;

// A_MN / B_MN: that operand is MN-major, i.e. it comes from a row-major
// [K x M] (or [K x N]) array (C = X^T Y from row-major activations and
// gradients: the weight gradient of a dense layer): its stage holds 64-wide
// MN blocks of 64 k rows (8 KiB each) side by side and its descriptor steps
// 2 KiB (16 k rows) per MMA; a K-major operand's stage is one box of 64 k
// columns and its descriptor steps 32 bytes inside the swizzle atom.
template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stages
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int bn = g.bn;
  const uint32_t a_bytes = kBM * kBK * 2, b_bytes = uint32_t(bn) * kBK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_m = blockIdx.x, tile_n = blockIdx.y;
  const int kblocks_total = g.K / kBK;
  const int kb_per_split = (kblocks_total + gridDim.z - 1) / gridDim.z;
  const int kb0 = blockIdx.z * kb_per_split;
  const int nkb = max(0, min(kblocks_total, kb0 + kb_per_split) - kb0);
  uint32_t ncols = 32;
  while (ncols < uint32_t(bn)) ncols <<= 1;
  // warps 2 and 3 of the CTAs of m-tile 0 sum the rows of every B stage
  // (kEpiPartialF32 with rowsum_b, B K-major): a stage returns to the
  // producer after the MMA's commit and their 64 arrivals
  const bool sum_b = !B_MN && g.rowsum_b != nullptr && g.epilogue == kEpiPartialF32 && tile_m == 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], sum_b ? 1 + 64 : 1);
    }
    mbar_init(&done_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  // lanes 1-31 of warps 0 and 1 wait at __syncwarp while lane 0 runs its
  // role (spinning on the accumulator barrier there would compete with it)
  if (warp == 0 && lane == 0 && nkb > 0) {
    // producer: the K blocks of this split through the ring of stages
    int issued = 0;
    for (int i = 0; i < nkb && !failed; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !mbar_wait(&empty_bar[s], uint32_t(i / kStages - 1) & 1u)) {
        failed = 1;
        atomicExch(g.error, 1);
        break;
      }
      unsigned char* st = smem + size_t(s) * stage_bytes;
      mbar_expect_tx(&full_bar[s], stage_bytes);
      if (A_MN) {
        for (int q = 0; q < kBM / 64; ++q)
          tma_load_2d(st + q * 8192, &map_a, tile_m * kBM + q * 64, (kb0 + i) * kBK, &full_bar[s]);
      } else {
        tma_load_2d(st, &map_a, (kb0 + i) * kBK, tile_m * kBM, &full_bar[s]);
      }
      if (B_MN) {
        for (int q = 0; q < bn / 64; ++q)
          tma_load_2d(st + a_bytes + q * 8192, &map_b, tile_n * bn + q * 64, (kb0 + i) * kBK, &full_bar[s]);
      } else {
        tma_load_2d(st + a_bytes, &map_b, (kb0 + i) * kBK, tile_n * bn, &full_bar[s]);
      }
      ++issued;
    }
    // every copy issued lands before the CTA may exit
    for (int s = 0; s < kStages && s < issued; ++s)
      mbar_wait(&full_bar[s], uint32_t((issued - 1 - s) / kStages) & 1u);
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // MMA issuer: D = F32, A = B = BF16, each K-major or MN-major, N = bn, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (A_MN ? (1u << 15) : 0u) | (B_MN ? (1u << 16) : 0u) |
                           (uint32_t(bn >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(&full_bar[s], uint32_t(i / kStages) & 1u)) {
        failed = 1;
        atomicExch(g.error, 2);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_addr = smem_u32(smem + size_t(s) * stage_bytes);
      const uint64_t ad = A_MN ? smem_desc_mn(a_addr, 8192) : smem_desc(a_addr);
      const uint64_t bd = B_MN ? smem_desc_mn(a_addr + a_bytes, 8192) : smem_desc(a_addr + a_bytes);
      // per 16 k: an MN-major operand advances 16 k rows = 2 KiB, a K-major one
      // 16 BF16 = 32 bytes along K inside the swizzle atom (descriptor units of 16 bytes)
      constexpr uint64_t kStepA = A_MN ? 128 : 2, kStepB = B_MN ? 128 : 2;
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)
        mma_bf16(tmem, ad + uint64_t(k) * kStepA, bd + uint64_t(k) * kStepB, idesc, (i > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);  // completes once every MMA issued above has
  }
  else if (sum_b && warp >= 2 && nkb > 0) {
    // row r = t + 64 j of this n-tile's B: its 64 k values of a stage are
    // eight 16-byte units in the 128-byte swizzled row (unit u at
    // (u ^ (r % 8)) x 16); each unit's eight values are added as a tree
    // into the unit's own accumulator, stage after stage, and the eight
    // accumulators of a row in unit order at the end (a fixed order with
    // short dependency chains)
    const int t = threadIdx.x - 64;
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[j][u] = 0.0f;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(&full_bar[s], uint32_t(i / kStages) & 1u)) {
        failed = 1;
        atomicExch(g.error, 5);
        break;
      }
      const unsigned char* bst = smem + size_t(s) * stage_bytes + a_bytes;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = t + 64 * j;
        if (r < bn) {
          const unsigned char* row = bst + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const uint4 v = *reinterpret_cast<const uint4*>(row + ((u ^ (r & 7)) << 4));
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
            const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
            const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
            acc[j][u] += ((f0.x + f0.y) + (f1.x + f1.y)) + ((f2.x + f2.y) + (f3.x + f3.y));
          }
        }
      }
      mbar_arrive(&empty_bar[s]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = t + 64 * j;
      if (r < bn)
        g.rowsum_b[size_t(blockIdx.z) * g.N + size_t(tile_n) * bn + r] =
            ((acc[j][0] + acc[j][1]) + (acc[j][2] + acc[j][3])) + ((acc[j][4] + acc[j][5]) + (acc[j][6] + acc[j][7]));
    }
  }
  if (warp < 2) __syncwarp();
  if (nkb > 0) {
    // every thread waits for the accumulator (or the failure release)
    if (!mbar_wait(&done_bar, 0)) {
      if (lane == 0) atomicExch(g.error, 3);
      failed = 1;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (!failed && nkb > 0) {
    const int row = tile_m * kBM + warp * 32 + lane;
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    for (int c0 = 0; c0 < bn; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + uint32_t(c0), v);
      const int col0 = tile_n * bn + c0;
      if (row >= g.M) continue;
      switch (g.epilogue) {
        case kEpiBiasReluBf16: {
          __nv_bfloat16* out = g.c_bf16 + size_t(row) * g.ldc + col0;
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float a = fmaxf(v[j] + (g.bias ? g.bias[col0 + j] : 0.0f), 0.0f);
            const float b = fmaxf(v[j + 1] + (g.bias ? g.bias[col0 + j + 1] : 0.0f), 0.0f);
            *reinterpret_cast<__nv_bfloat162*>(out + j) = __floats2bfloat162_rn(a, b);
          }
          break;
        }
        case kEpiBiasF32: {
          float* out = g.c_f32 + size_t(row) * g.ldc + col0;
#pragma unroll
          for (int j = 0; j < 16; ++j) out[j] = v[j] + (g.bias ? g.bias[col0 + j] : 0.0f);
          break;
        }
        case kEpiReluMaskBf16: {
          // gradient through ReLU: keep where the layer's activation is positive
          __nv_bfloat16* out = g.c_bf16 + size_t(row) * g.ldc + col0;
          const __nv_bfloat16* act = g.mask + size_t(row) * g.ld_mask + col0;
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float a = __bfloat162float(act[j]) > 0.0f ? v[j] : 0.0f;
            const float b = __bfloat162float(act[j + 1]) > 0.0f ? v[j + 1] : 0.0f;
            *reinterpret_cast<__nv_bfloat162*>(out + j) = __floats2bfloat162_rn(a, b);
          }
          break;
        }
        case kEpiPartialF32: {  // this split's partial tile, summed later in a fixed order
          float4* out = reinterpret_cast<float4*>(g.c_f32 + size_t(blockIdx.z) * g.M * g.ldc + size_t(row) * g.ldc + col0);
#pragma unroll
          for (int j = 0; j < 4; ++j) out[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          break;
        }
        default: {  // kEpiAtomicF32: split-K accumulation
          float* out = g.c_f32 + size_t(row) * g.ldc + col0;
#pragma unroll
          for (int j = 0; j < 16; ++j) atomicAdd(out + j, v[j]);
        }
      }
    }
  }
  if (!failed && nkb == 0 && g.epilogue == kEpiPartialF32) {  // an empty split contributes zeros
    const int row = tile_m * kBM + warp * 32 + lane;
    float4* out = reinterpret_cast<float4*>(g.c_f32 + size_t(blockIdx.z) * g.M * g.ldc + size_t(row) * g.ldc +
                                            tile_n * bn);
    for (int j = 0; j < bn / 4; ++j) out[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (sum_b)
      for (int r = threadIdx.x; r < bn; r += blockDim.x)
        g.rowsum_b[size_t(blockIdx.z) * g.N + size_t(tile_n) * bn + r] = 0.0f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}


// ---------------------------------------------------------------------------
// Persistent B-resident GEMM (tc_gemm_rs).  Warp roles: warp 0 loads B once
// and then streams the A tiles of this CTA's M tiles through the ring; warp 1
// owns the TMEM allocation and issues the MMAs (tile i into accumulator
// i % 2); warps 2-9 read accumulator i % 2 back and run the epilogue (warp w
// may only access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, i.e. one quarter
// of the tile's rows; the two warps of a quarter take alternate 16-column
// chunks), then hand the accumulator back.
constexpr int kRsThreads = 320;
constexpr int kRsEpiThreads = 256;
constexpr int kRsMaxStages = 6;
constexpr uint32_t kAStage = kBM * kBK * 2;  // 16 KiB

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16* dst, const float* o) {
  uint4 w[2];
  uint32_t* u = reinterpret_cast<uint32_t*>(w);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(o[2 * j], o[2 * j + 1]);
    u[j] = *reinterpret_cast<const uint32_t*>(&h);
  }
  reinterpret_cast<uint4*>(dst)[0] = w[0];
  reinterpret_cast<uint4*>(dst)[1] = w[1];
}

__device__ __forceinline__ void rs_epilogue16(const TcGemmArgs& g, int row, int col0, const float* v) {
  float o[16];
  if (g.epilogue == kEpiReluMaskBf16) {
    if (g.mask) {
      uint4 mw[2];
      const uint4* mp = reinterpret_cast<const uint4*>(g.mask + size_t(row) * g.ld_mask + col0);
      mw[0] = mp[0];
      mw[1] = mp[1];
      const __nv_bfloat16* m = reinterpret_cast<const __nv_bfloat16*>(mw);
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = __bfloat162float(m[j]) > 0.0f ? v[j] : 0.0f;
    } else {  // transposed activation: coalesced over the warp's rows
#pragma unroll
      for (int j = 0; j < 16; ++j)
        o[j] = __bfloat162float(g.mask_t[size_t(col0 + j) * g.ld_mask_t + row]) > 0.0f ? v[j] : 0.0f;
    }
  } else {
    if (g.bias) {
      const float4* bp = reinterpret_cast<const float4*>(g.bias + col0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 b4 = __ldg(bp + j);
        o[4 * j] = v[4 * j] + b4.x;
        o[4 * j + 1] = v[4 * j + 1] + b4.y;
        o[4 * j + 2] = v[4 * j + 2] + b4.z;
        o[4 * j + 3] = v[4 * j + 3] + b4.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = v[j];
    }
    if (g.epilogue == kEpiBiasReluBf16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = fmaxf(o[j], 0.0f);
    }
  }
  if (g.epilogue == kEpiBiasF32) {
    if (g.c_f32) {
      float4* out = reinterpret_cast<float4*>(g.c_f32 + size_t(row) * g.ldc + col0);
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
    }
    if (g.c_t_f32) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g.c_t_f32[size_t(col0 + j) * g.ldt + row] = o[j];
    }
  } else {
    if (g.c_bf16) store_bf16x16(g.c_bf16 + size_t(row) * g.ldc + col0, o);
    if (g.c_t_bf16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g.c_t_bf16[size_t(col0 + j) * g.ldt + row] = __float2bfloat16_rn(o[j]);
    }
  }
}

__global__ void __launch_bounds__(kRsThreads, 1)
    tc_gemm_rs_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      TcGemmArgs g, int stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t b_full;
  __shared__ __align__(8) uint64_t a_full[kRsMaxStages];
  __shared__ __align__(8) uint64_t a_empty[kRsMaxStages];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bn = g.bn, nkb = g.K / kBK;
  const uint32_t b_chunk = uint32_t(bn) * kBK * 2;  // one 64-wide K chunk of B (bn rows x 128 bytes)
  unsigned char* smem_b = smem;
  unsigned char* smem_a = smem + size_t(nkb) * b_chunk;
  const int n_tile = blockIdx.y;
  const int m_tiles = g.M / kBM;
  const int my_tiles = int(blockIdx.x) < m_tiles ? (m_tiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  uint32_t acc_cols = 32;
  while (acc_cols < uint32_t(bn)) acc_cols <<= 1;

  if (threadIdx.x == 0) {
    mbar_init(&b_full, 1);
    for (int s = 0; s < stages; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kRsEpiThreads);
    }
    mbar_init(&fin_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * acc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0 && my_tiles > 0) {
      mbar_expect_tx(&b_full, uint32_t(nkb) * b_chunk);
      for (int kb = 0; kb < nkb; ++kb) tma_load_2d(smem_b + size_t(kb) * b_chunk, &map_b, kb * kBK, n_tile * bn, &b_full);
      int it = 0;
      for (int i = 0; i < my_tiles && !failed; ++i) {
        const int m = int(blockIdx.x) + i * int(gridDim.x);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % stages;
          const uint32_t use = uint32_t(it / stages);
          if (use > 0 && !mbar_wait(&a_empty[s], (use - 1) & 1u)) {
            failed = 1;
            atomicExch(g.error, 11);
            break;
          }
          mbar_expect_tx(&a_full[s], kAStage);
          tma_load_2d(smem_a + size_t(s) * kAStage, &map_a, kb * kBK, m * kBM, &a_full[s]);
          ++it;
        }
      }
      // every copy issued must land before the CTA may exit
      mbar_wait(&b_full, 0);
      for (int s = 0; s < stages && s < it; ++s) {
        const int uses = (it - 1 - s) / stages + 1;  // loads issued into stage s
        mbar_wait(&a_full[s], uint32_t(uses - 1) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      // idesc: D = F32, A = B = BF16, both K-major, N = bn, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(bn >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
      bool ok = mbar_wait(&b_full, 0);
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 12);
      }
      int it = 0;
      for (int i = 0; i < my_tiles && ok && !failed; ++i) {
        const int acc = i & 1;
        const uint32_t use = uint32_t(i >> 1);
        if (use > 0 && !mbar_wait(&acc_empty[acc], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d = tmem + uint32_t(acc) * acc_cols;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % stages;
          if (!mbar_wait(&a_full[s], uint32_t(it / stages) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t ad = smem_desc(smem_u32(smem_a + size_t(s) * kAStage));
          const uint64_t bd = smem_desc(smem_u32(smem_b + size_t(kb) * b_chunk));
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            mma_bf16(d, ad + uint64_t(k * 2), bd + uint64_t(k * 2), idesc, (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(&a_empty[s]);
        }
        if (!ok) break;
        mma_commit(&acc_full[acc]);
      }
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 13);
      }
      // all MMAs issued by this thread complete before the accumulators are released
      mma_commit(&fin_bar);
      mbar_wait(&fin_bar, 0);
    }
  } else {
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // which alternate 16-column chunks
    const int rl = q * 32 + lane;
    const int nchunks = bn / 16;
    for (int i = 0; i < my_tiles; ++i) {
      const int acc = i & 1;
      // warp-uniform decisions: the tcgen05.ld below needs the whole warp
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[acc], uint32_t(i >> 1) & 1u))) {
        failed = 1;
        if (lane == 0) atomicExch(g.error, 14);
        break;
      }
      if (__any_sync(0xffffffffu, failed != 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row = (int(blockIdx.x) + i * int(gridDim.x)) * kBM + rl;
      const uint32_t base = tmem + (uint32_t(q * 32) << 16) + uint32_t(acc) * acc_cols;
      // four chunks in flight per wait
      for (int c = half; c < nchunks; c += 8) {
        uint32_t r[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (c + 2 * u < nchunks) tmem_ld16_nw(base + uint32_t((c + 2 * u) * 16), r[u]);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (c + 2 * u < nchunks) {
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[u][j]);
            rs_epilogue16(g, row, n_tile * bn + (c + 2 * u) * 16, v);
          }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&acc_empty[acc]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols));
}

// out[i] += sum over s of part[s][i], in a fixed order: the splits are cut
// into kRedGroups contiguous ranges, each summed in order by its own thread
// (so a thread has a short chain of independent loads in flight), and the
// range sums are added in range order.  Blocks of kRedGroups x 32 threads
// cover 32 groups of four consecutive elements (n % 4 == 0, 16-byte
// aligned arrays); a thread that holds no full group reads nothing.  `blk`
// is the block's index within its array.
constexpr int kRedGroups = 8;
__device__ __forceinline__ void reduce_splits_block(const float* part, int splits, size_t n, float* out,
                                                    unsigned blk) {
  __shared__ float4 red[kRedGroups][32];
  const int c = threadIdx.x & 31, gr = threadIdx.x >> 5;
  const size_t q = size_t(blk) * 32 + c;  // float4 index
  const bool live = 4 * q + 4 <= n;
  const int per = (splits + kRedGroups - 1) / kRedGroups;
  const int s0 = gr * per, s1 = min(splits, s0 + per);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (live) {
    const float4* p = reinterpret_cast<const float4*>(part) + q;
    const size_t stride = n / 4;
    int s = s0;
#pragma unroll 1
    for (; s + 4 <= s1; s += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = p[size_t(s + u) * stride];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.x += v[u].x;
        acc.y += v[u].y;
        acc.z += v[u].z;
        acc.w += v[u].w;
      }
    }
    for (; s < s1; ++s) {
      const float4 v = p[size_t(s) * stride];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  red[gr][c] = acc;
  __syncthreads();
  if (gr == 0 && live) {
    float4 o = reinterpret_cast<float4*>(out)[q];
#pragma unroll
    for (int g = 0; g < kRedGroups; ++g) {
      o.x += red[g][c].x;
      o.y += red[g][c].y;
      o.z += red[g][c].z;
      o.w += red[g][c].w;
    }
    reinterpret_cast<float4*>(out)[q] = o;
  }
}

__global__ void __launch_bounds__(kRedGroups * 32) reduce_splits_kernel(const float* part, int splits, size_t n,
                                                                      float* out) {
  reduce_splits_block(part, splits, n, out, blockIdx.x);
}

// Several reductions in one launch: segment k owns blocks [first[k],
// first[k + 1]) and sums exactly as reduce_splits_kernel would alone.
struct RedSegs {
  TcRedSeg seg[kMaxRedSegs];
  unsigned first[kMaxRedSegs + 1];
  int nseg;
};
__global__ void __launch_bounds__(kRedGroups * 32) reduce_splits_multi_kernel(const RedSegs r) {
  int k = 0;
  while (k + 1 < r.nseg && blockIdx.x >= r.first[k + 1]) ++k;
  const TcRedSeg& sg = r.seg[k];
  reduce_splits_block(sg.part, sg.splits, sg.n, sg.out, blockIdx.x - r.first[k]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

// 2D BF16 tensor map of a row-major [rows x K] matrix, box [box_rows x 64].
bool tc_make_map(CUtensorMap* m, const void* base, int rows, int k, int ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cuuint64_t(k), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
  const cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
bool make_map(CUtensorMap* m, const void* base, int rows, int k, int ld, int box_rows) {
  return tc_make_map(m, base, rows, k, ld, box_rows);
}

int num_sms_cached() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = v;
    if (n <= 0) n = 1;
  }
  return n;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

size_t tc_gemm_smem(int bn) { return size_t(kStages) * (kBM * kBK * 2 + size_t(bn) * kBK * 2) + 1024; }

cudaError_t tc_gemm(const TcGemmArgs& g_in, const __nv_bfloat16* a, int lda, const __nv_bfloat16* b, int ldb,
                    int splits, cudaStream_t st) {
  TcGemmArgs g = g_in;
  if (g.rowsum_b && (g.epilogue != kEpiPartialF32 || (reinterpret_cast<uintptr_t>(g.rowsum_b) & 15)))
    return cudaErrorInvalidValue;
  if (g.M % kBM || g.K % kBK || g.bn % 16 || g.bn < 16 || g.bn > 256 || g.N % g.bn || splits < 1 || !g.error ||
      (reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15) || (lda % 8) || (ldb % 8))
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, g.M, g.K, lda, kBM) || !make_map(&mb, b, g.N, g.K, ldb, g.bn)) return cudaErrorInvalidValue;
  const size_t smem = tc_gemm_smem(g.bn);
  (void)cudaGetLastError();
  cudaError_t e =
      cudaFuncSetAttribute(tc_gemm_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(g.M / kBM, g.N / g.bn, splits);
  tc_gemm_kernel<false, false><<<grid, 128, smem, st>>>(ma, mb, g);
  return cudaGetLastError();
}

cudaError_t tc_gemm_tn(const TcGemmArgs& g_in, const __nv_bfloat16* x, int ldx, const __nv_bfloat16* y, int ldy,
                       int splits, cudaStream_t st) {
  TcGemmArgs g = g_in;
  if (g.rowsum_b) return cudaErrorInvalidValue;  // row sums of B need a K-major B
  if (g.M % kBM || g.K % kBK || g.bn % 64 || g.bn < 64 || g.bn > 256 || g.N % g.bn || splits < 1 || !g.error ||
      !aligned16(x) || !aligned16(y) || (ldx % 8) || (ldy % 8) || ldx < g.M || ldy < g.N ||
      (g.epilogue != kEpiBiasF32 && g.epilogue != kEpiAtomicF32 && g.epilogue != kEpiPartialF32) || !g.c_f32)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;  // [K rows x M] and [K rows x N], boxes of 64 x 64
  if (!tc_make_map(&ma, x, g.K, g.M, ldx, 64) || !tc_make_map(&mb, y, g.K, g.N, ldy, 64)) return cudaErrorInvalidValue;
  const size_t smem = tc_gemm_smem(g.bn);
  (void)cudaGetLastError();
  cudaError_t e =
      cudaFuncSetAttribute(tc_gemm_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(g.M / kBM, g.N / g.bn, splits);
  tc_gemm_kernel<true, true><<<grid, 128, smem, st>>>(ma, mb, g);
  return cudaGetLastError();
}

cudaError_t tc_gemm_xn(const TcGemmArgs& g_in, const __nv_bfloat16* x, int ldx, const __nv_bfloat16* b, int ldb,
                       int splits, cudaStream_t st) {
  TcGemmArgs g = g_in;
  if (g.rowsum_b && (g.epilogue != kEpiPartialF32 || (reinterpret_cast<uintptr_t>(g.rowsum_b) & 15)))
    return cudaErrorInvalidValue;
  if (g.M % kBM || g.K % kBK || g.bn % 16 || g.bn < 16 || g.bn > 256 || g.N % g.bn || splits < 1 || !g.error ||
      !aligned16(x) || !aligned16(b) || (ldx % 8) || (ldb % 8) || ldx < g.M || ldb < g.K ||
      (g.epilogue != kEpiBiasF32 && g.epilogue != kEpiAtomicF32 && g.epilogue != kEpiPartialF32) || !g.c_f32)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;  // x: [K rows x M], boxes of 64 x 64; b: [N rows x K], boxes of bn x 64
  if (!tc_make_map(&ma, x, g.K, g.M, ldx, 64) || !make_map(&mb, b, g.N, g.K, ldb, g.bn)) return cudaErrorInvalidValue;
  const size_t smem = tc_gemm_smem(g.bn);
  (void)cudaGetLastError();
  cudaError_t e =
      cudaFuncSetAttribute(tc_gemm_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(g.M / kBM, g.N / g.bn, splits);
  tc_gemm_kernel<true, false><<<grid, 128, smem, st>>>(ma, mb, g);
  return cudaGetLastError();
}

cudaError_t tc_gemm_rs(const TcGemmArgs& g, const __nv_bfloat16* a, int lda, const __nv_bfloat16* b, int ldb,
                       cudaStream_t st) {
  constexpr size_t kMaxSmem = 232448 - 1024;  // 227 KiB opt-in limit per block, less the static barriers
  if (g.M % kBM || g.K % kBK || g.K > 5 * kBK || g.bn % 16 || g.bn < 16 || g.bn > 256 || g.N % g.bn || !g.error ||
      g.epilogue < kEpiBiasReluBf16 || g.epilogue > kEpiReluMaskBf16 || !aligned16(a) || !aligned16(b) || (lda % 8) ||
      (ldb % 8))
    return cudaErrorInvalidValue;
  if (g.epilogue == kEpiBiasF32 ? (!g.c_f32 && !g.c_t_f32) : (!g.c_bf16 && !g.c_t_bf16)) return cudaErrorInvalidValue;
  if ((g.c_f32 && !aligned16(g.c_f32)) || (g.c_bf16 && !aligned16(g.c_bf16)) || (g.ldc % 8) ||
      ((g.c_t_bf16 || g.c_t_f32) && g.ldt < g.M))
    return cudaErrorInvalidValue;
  if (g.epilogue == kEpiReluMaskBf16 &&
      (g.mask ? (!aligned16(g.mask) || (g.ld_mask % 8)) : (!g.mask_t || g.ld_mask_t < g.M)))
    return cudaErrorInvalidValue;
  if (g.bias && !aligned16(g.bias)) return cudaErrorInvalidValue;
  const size_t b_bytes = size_t(g.bn) * g.K * 2;
  const size_t room = kMaxSmem - 1024 - b_bytes;
  const int stages = int(std::min<size_t>(kRsMaxStages, room / kAStage));
  if (b_bytes + 1024 > kMaxSmem || stages < 2) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, g.M, g.K, lda, kBM) || !make_map(&mb, b, g.N, g.K, ldb, g.bn)) return cudaErrorInvalidValue;
  const size_t smem = b_bytes + size_t(stages) * kAStage + 1024;
  (void)cudaGetLastError();
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_rs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int n_tiles = g.N / g.bn, m_tiles = g.M / kBM;
  const int per_n = std::max(1, std::min(m_tiles, num_sms_cached() / n_tiles));
  tc_gemm_rs_kernel<<<dim3(per_n, n_tiles), kRsThreads, smem, st>>>(ma, mb, g, stages);
  return cudaGetLastError();
}

cudaError_t tc_reduce_splits(const float* part, int splits, size_t n, float* out, cudaStream_t st) {
  if (splits < 1 || !part || !out) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  if (n % 4 != 0 || (reinterpret_cast<uintptr_t>(part) | reinterpret_cast<uintptr_t>(out)) % 16 != 0)
    return cudaErrorInvalidValue;
  const unsigned grid = unsigned((n / 4 + 31) / 32);
  reduce_splits_kernel<<<grid, kRedGroups * 32, 0, st>>>(part, splits, n, out);
  return cudaGetLastError();
}

cudaError_t tc_reduce_splits_multi(const TcRedSeg* segs, int nseg, cudaStream_t st) {
  if (nseg < 1 || nseg > kMaxRedSegs || !segs) return cudaErrorInvalidValue;
  RedSegs r;
  std::memset(&r, 0, sizeof(r));
  r.nseg = nseg;
  unsigned blocks = 0;
  for (int k = 0; k < nseg; ++k) {
    const TcRedSeg& sg = segs[k];
    if (sg.splits < 1 || !sg.part || !sg.out || sg.n % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(sg.part) | reinterpret_cast<uintptr_t>(sg.out)) % 16 != 0)
      return cudaErrorInvalidValue;
    r.seg[k] = sg;
    r.first[k] = blocks;
    blocks += unsigned((sg.n / 4 + 31) / 32);
  }
  r.first[nseg] = blocks;
  if (blocks == 0) return cudaSuccess;
  reduce_splits_multi_kernel<<<blocks, kRedGroups * 32, 0, st>>>(r);
  return cudaGetLastError();
}

}  // namespace mc
