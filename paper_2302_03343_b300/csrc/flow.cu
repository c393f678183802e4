// Normalizing-flow importance sampler on the GPU (C ABI: mc_flow_* in
// include/mcint.h).
//
// Flow: L piecewise-quadratic coupling layers (flow_spline.cuh) over the unit
// cube; layer l transforms the coordinates d with d % 2 == l % 2 and
// conditions on the others through a dense network u = 2 x_A - 1 -> 256 ->
// 256 -> 256 -> (2K + 1) logits per transformed coordinate, with ReLU.  All
// four dense layers run on the tcgen05 tensor cores with BF16 operands and
// FP32 accumulation; the first one (K = d_A) takes the input (u, 1, 0, ..)
// padded to 16 columns against W1e = (W1 | b1 | 0), so its bias is a BF16
// weight on a constant input of one.  The splines and log-determinants are
// FP32.
//
// Sampling (thesis Sec. "Importance sampling", eq. mc_est_is): Philox
// uniforms z -> flow forward -> x, log q(x) -> integrand at x -> w = f / q ->
// Kahan FP64 sums.  Training (online, on events the method generates itself):
// sample a batch with the forward pass keeping every layer's activations,
// evaluate f, hold the weights w = |f| / q fixed, and minimise
// L = -sum w log q(x) / sum w; since a coupling layer passes its conditioning
// coordinates through unchanged, the forward activations are exactly those of
// the density (inverse) pass at x, so the backward runs on them directly:
// spline backward, activation gradients on the tensor cores (B-resident
// kernel), weight gradients as split-K products over the batch with a
// fixed-order reduction, then Adam (thesis Sec. "Optimizers").
//
// Layouts (n = padded batch rows, H = 256): points P [n][D]; activations h
// [n][H] BF16 row-major (the fused forward stores them by TMA from its
// operand buffer; the weight-gradient products read them as MN-major
// operands), and in the layer-by-layer path also their transposes [H][n]
// (ReLU masks of its products); ReLU activity bits [3][n][8] words; logits
// transposed [row][n] FP32 with coordinate j's 2K+1 logits at rows
// j * ls .. j * ls + 2K (ls = 2K+1 rounded up to 16, so that each coordinate
// starts on a 16-byte boundary in the row-major gradient and on a 16-column
// group of the tensor-memory accumulator); logit and activation gradients
// G [n][nout], G^T, dA^T in two buffer sets alternating by layer.
//
// A training step is captured once per mc_flow_train call as a CUDA graph
// and replayed; the weight-gradient products of a layer run on a side stream
// beside the next layer's spline backward and chain, back to back (each into
// its own split-K partial region), and their fixed-order sums in one launch.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "event.cuh"
#include "flow_spline.cuh"
#include "handles.h"
#include "launch.h"
#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace mc {
namespace {

constexpr int kMaxFlowDim = 16;
constexpr int kMaxA = kMaxFlowDim / 2;
constexpr int kMaxLayers = 16;
constexpr int kH = 256;  // hidden width

struct LayerDev {
  int na, nb, ls, nout_pad;  // conditioning / transformed coordinates, logit stride, padded rows
  int a_idx[kMaxFlowDim], b_idx[kMaxFlowDim];
  // master parameters (FP32) and their gradients / Adam moments share one
  // layout: W1 [H x na], b1 [H], W2 [H x H], b2, W3 [H x H], b3,
  // W4 [nout_pad x H], b4 [nout_pad]; gradients of W2..W4 are kept transposed
  // (gW^T [in x out]) as the weight-gradient products produce them.
  size_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, off_W4, off_b4;
  // BF16 copies for the tensor cores: W2, W3, W4 (row-major [out x in]) and
  // their transposes [in x out] for the activation gradients; W1 transposed
  // and zero-padded to [16 x H] for the input gradient of the first layer
  __nv_bfloat16 *W2h, *W3h, *W4h, *W2t, *W3t, *W4t, *W1t;
  // first layer as a tensor-core product: W1e [H x 64] = (W1 | b1 | 0), so
  // that h1 = relu(W1e . (u, 1, 0, ..)) with the bias on a constant input
  __nv_bfloat16* W1e;
};
constexpr int kUK = 64;  // K of the first-layer product (u, 1, zero padding)
constexpr int kUPad = 16;  // rows of U^T: u_0 .. u_{na-1}, a row of ones (bias), zeros

unsigned blocks_for(long long n, int t) { return unsigned((n + t - 1) / t); }

// ------------------------------------------------------------------ kernels
// z: FP32-mode Philox uniforms (2k + 1) / 2^24 of events first + i; with
// step, the iteration word is 0x10000 + *step (the training step count kept
// on the device, so that a replayed graph of a step draws that step's batch).
__global__ void flow_uniforms_kernel(float* z, long long n, int D, uint64_t seed, uint32_t iteration, long long first,
                                     const long long* step = nullptr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (step) iteration = 0x10000u + uint32_t(*step);
  uint64_t k[kMaxFlowDim];
  event_uniforms<kMaxFlowDim, false>(seed, iteration, 0u, uint64_t(first + i), D, k);
  for (int d = 0; d < D; ++d) z[i * D + d] = float(uint32_t(2 * k[d] + 1)) * 0x1p-24f;
}

// The first-layer input of one event per thread: U [n][64] BF16 row-major
// (u_a = 2 x_A - 1, then 1 for the bias, then zeros; the A operand of the
// first-layer product) and, if UT, its transpose [16][n] (u_a, then the row
// of ones: the operand of the W1 and b1 gradient).
__global__ void __launch_bounds__(128) dense1_input_kernel(const float* P, int D, const LayerDev L, __nv_bfloat16* U,
                                                           __nv_bfloat16* UT, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  __nv_bfloat16 v[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    const float x = a < L.na ? 2.0f * P[i * D + L.a_idx[a < L.na ? a : 0]] - 1.0f : (a == L.na ? 1.0f : 0.0f);
    v[a] = __float2bfloat16_rn(x);
    if (UT && a <= L.na) UT[size_t(a) * n + i] = v[a];
  }
  uint4* row = reinterpret_cast<uint4*>(U + size_t(i) * kUK);
  row[0] = *reinterpret_cast<const uint4*>(v);
  row[1] = *reinterpret_cast<const uint4*>(v + 8);
  for (int c = 2; c < kUK / 8; ++c) row[c] = make_uint4(0u, 0u, 0u, 0u);
}

// Forward spline of one layer for one event per thread: Pout = Pin with the
// transformed coordinates mapped (Pout may equal Pin); logq -= sum log c.
// Logits transposed: LT[(j * ls + k) * ldn + i].
__global__ void __launch_bounds__(128) spline_fwd_kernel(const float* Pin, float* Pout, int D, const LayerDev L,
                                                         const float* LT, size_t ldn, int K, float* logq, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (Pout != Pin)
    for (int a = 0; a < L.na; ++a) Pout[i * D + L.a_idx[a]] = Pin[i * D + L.a_idx[a]];
  Spline s;
  float ld = 0.0f;  // summed over the coordinates in order, as in the fused layer
  for (int j = 0; j < L.nb; ++j) {
    spline_load(LT + size_t(j) * L.ls * ldn + i, ldn, K, s);
    float lc;
    const int d = L.b_idx[j];
    Pout[i * D + d] = spline_fwd(s, K, Pin[i * D + d], &lc);
    ld += lc;
  }
  logq[i] -= ld;
}

// Inverse spline of one layer: Pout = Pin with the transformed coordinates
// inverted; logq -= sum log c.
__global__ void __launch_bounds__(128) spline_inv_kernel(const float* Pin, float* Pout, int D, const LayerDev L,
                                                         const float* LT, size_t ldn, int K, float* logq, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < L.na; ++a) Pout[i * D + L.a_idx[a]] = Pin[i * D + L.a_idx[a]];
  Spline s;
  float ld = 0.0f;
  for (int j = 0; j < L.nb; ++j) {
    spline_load(LT + size_t(j) * L.ls * ldn + i, ldn, K, s);
    float lc;
    const int d = L.b_idx[j];
    Pout[i * D + d] = spline_inv(s, K, Pin[i * D + d], &lc);
    ld += lc;
  }
  logq[i] -= ld;
}

// Backward of one inverse layer.  dP holds dL/d(layer output) on entry and
// dL/d(layer input) for the transformed coordinates on exit (the conditioning
// coordinates receive the conditioner's contribution later);
// gl_i = dL/d(log q_i) = -w_i / sum w.  The logit gradients go out in BF16
// row-major G [n][nout_pad] (operand of the activation gradient) and
// transposed GT [nout_pad][n] (operand of the weight gradient).
__global__ void __launch_bounds__(128) spline_inv_bwd_kernel(const float* Pin, float* dP, int D, const LayerDev L,
                                                             const float* LT, int K, const float* w,
                                                             const double* wsum, __nv_bfloat16* G,
                                                             __nv_bfloat16* GT, long long n, long long n_real) {
  constexpr int kRow = 2 * kFlowMaxBins + 17;  // odd stride >= ls (2K+1 rounded up to 16): conflict-free rows
  __shared__ float gsh[128][kRow];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;  // no block-wide barrier below
  float* gs = gsh[threadIdx.x];
  const bool real = i < n_real;
  const float gl = real ? float(-double(w[i]) / *wsum) : 0.0f;
  const size_t ldn = size_t(n);
  const int K2 = 2 * K + 1;
  Spline s;
  float gw[kFlowMaxBins], gv[kFlowMaxBins + 1];
  for (int j = 0; j < L.nb; ++j) {
    const int d = L.b_idx[j];
    if (real) {
      spline_load(LT + size_t(j) * L.ls * ldn + i, ldn, K, s);
      dP[i * D + d] = spline_inv_bwd(s, K, Pin[i * D + d], dP[i * D + d], gl, gw, gv);
#pragma unroll
      for (int k = 0; k < kFlowMaxBins; ++k)
        if (k < K) gs[k] = gw[k];
#pragma unroll
      for (int k = 0; k <= kFlowMaxBins; ++k)
        if (k <= K) gs[K + k] = gv[k];
    } else {
      dP[i * D + d] = 0.0f;
      for (int k = 0; k < K2; ++k) gs[k] = 0.0f;
    }
    for (int k = K2; k < L.ls; ++k) gs[k] = 0.0f;
    // transposed rows (coalesced over events)
    __nv_bfloat16* gt = GT + size_t(j) * L.ls * ldn + i;
    for (int k = 0; k < K2; ++k) gt[size_t(k) * ldn] = __float2bfloat16_rn(gs[k]);
    // row-major block of ls entries (zero padded), 16-byte stores
    uint4* gr = reinterpret_cast<uint4*>(G + size_t(i) * L.nout_pad + size_t(j) * L.ls);
    for (int c8 = 0; c8 < L.ls / 8; ++c8) {
      uint4 pk;
      uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(gs[c8 * 8 + 2 * e], gs[c8 * 8 + 2 * e + 1]);
        pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
      }
      gr[c8] = pk;
    }
  }
  // the rows past the last coordinate: the buffers are shared by layers with
  // more transformed coordinates, so clear what such a layer left there
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  for (int c = L.nb * L.ls; c < L.nout_pad; ++c) {
    GT[size_t(c) * ldn + i] = z;
    G[size_t(i) * L.nout_pad + c] = z;
  }
}

constexpr int kFusedK = 32;   // bins of the fused kernels
constexpr int kFusedLs = 80;  // their logit stride: 2K+1 rounded up to 16 columns

// The same spline backward for K = 32 bins with one thread per (event,
// coordinate j = blockIdx.y): the coordinates' independent work runs on
// separate threads, and with the bin count fixed at compile time every value
// stays in registers (no staging).  Writes exactly what spline_inv_bwd_kernel
// writes (the same arithmetic and roundings per coordinate).  The padded
// rows past the last coordinate are cleared by the threads of every
// coordinate in turn.
__global__ void __launch_bounds__(128, 4) spline_bwd_k32_kernel(const float* Pin, float* dP, int D, const LayerDev L,
                                                             const float* LT, const float* w, const double* wsum,
                                                             __nv_bfloat16* G, __nv_bfloat16* GT, long long n,
                                                             long long n_real) {
  constexpr int K = kFusedK, K2 = 2 * K + 1;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const bool real = i < n_real;
  const size_t ldn = size_t(n);
  const int d = L.b_idx[j];
  float gw[kFlowMaxBins], gv[kFlowMaxBins + 1];
  if (real) {
    const float gl = float(-double(w[i]) / *wsum);
    Spline s;
    spline_load(LT + size_t(j) * L.ls * ldn + i, ldn, K, s);
    dP[i * D + d] = spline_inv_bwd(s, K, Pin[i * D + d], dP[i * D + d], gl, gw, gv);
  } else {
    dP[i * D + d] = 0.0f;
#pragma unroll
    for (int k = 0; k < kFlowMaxBins; ++k) gw[k] = gv[k] = 0.0f;
    gv[kFlowMaxBins] = 0.0f;
  }
  // logit k of the coordinate: k < K a width, K <= k <= 2K a height, then zeros
  auto logit = [&](int k) -> float { return k < K ? gw[k < K ? k : 0] : (k < K2 ? gv[k < K2 ? k - K : 0] : 0.0f); };
  __nv_bfloat16* gt = GT + size_t(j) * L.ls * ldn + i;
#pragma unroll
  for (int k = 0; k < K2; ++k) gt[size_t(k) * ldn] = __float2bfloat16_rn(logit(k));
  uint4* gr = reinterpret_cast<uint4*>(G + size_t(i) * L.nout_pad + size_t(j) * L.ls);
#pragma unroll
  for (int c8 = 0; c8 < kFusedLs / 8; ++c8) {
    uint4 pk;
    uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(logit(c8 * 8 + 2 * e), logit(c8 * 8 + 2 * e + 1));
      pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
    }
    gr[c8] = pk;
  }
  // the rows past the last coordinate (see spline_inv_bwd_kernel), every
  // nb-th one by this coordinate's threads (nb ls is a multiple of 16, so
  // the row-major zeros are whole 16-byte units)
  const int c0 = L.nb * L.ls;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  for (int c = c0 + j; c < L.nout_pad; c += L.nb) GT[size_t(c) * ldn + i] = z;
  uint4* gz = reinterpret_cast<uint4*>(G + size_t(i) * L.nout_pad + c0);
  for (int u = j; u < (L.nout_pad - c0) / 8; u += L.nb) gz[u] = make_uint4(0u, 0u, 0u, 0u);
}

// First dense layer backward, input side: dL/dx_A += 2 dU with dU = dA1 W1
// computed on the tensor cores as [n][16] (u = 2 x_A - 1).
__global__ void add_input_grad_kernel(float* dP, int D, const LayerDev L, const float* dU, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < L.na; ++a) dP[i * D + L.a_idx[a]] += 2.0f * dU[i * kUPad + a];
}

// First dense layer backward, weight side: the split-K partial products
// part[s][j][c] of dA1^T U (c < na: W1 column, c = na: the bias row of ones)
// summed in a fixed order into the gradients of W1 [H x na] and b1: blocks
// of 8 x 32 threads cover 32 elements; each group of 32 sums a contiguous
// range of the splits in order, and the eight range sums are added in range
// order.
constexpr int kW1Groups = 8;
__global__ void __launch_bounds__(kW1Groups * 32) w1_grad_kernel(const float* part, int splits, const LayerDev L,
                                                                 float* grads) {
  __shared__ float red[kW1Groups][32];
  const int c32 = threadIdx.x & 31, gr = threadIdx.x >> 5;
  const int idx = blockIdx.x * 32 + c32;
  const bool live = idx < kH * kUPad;
  const int per = (splits + kW1Groups - 1) / kW1Groups;
  const int s0 = gr * per, s1 = min(splits, s0 + per);
  float acc = 0.0f;
  if (live) {
#pragma unroll 4
    for (int s = s0; s < s1; ++s) acc += part[size_t(s) * kH * kUPad + idx];
  }
  red[gr][c32] = acc;
  __syncthreads();
  if (gr != 0 || !live) return;
  const int j = idx / kUPad, c = idx % kUPad;
  if (c > L.na) return;
  float t = 0.0f;
#pragma unroll
  for (int g = 0; g < kW1Groups; ++g) t += red[g][c32];
  if (c == L.na)
    grads[L.off_b1 + j] += t;
  else
    grads[L.off_W1 + size_t(j) * L.na + c] += t;
}

// ReLU activity bits of the three hidden activations of a layer from their
// transposes hT [3][H][n] (layer slot): bits [3][n][8], bit c % 32 of word
// c / 32 set where h[c] > 0 (the fused backward's masks).
__global__ void mask_bits_kernel(const __nv_bfloat16* hT, size_t slot_stride, long long n, uint32_t* bits) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * 8 * n) return;
  const long long ev = t % n;
  const int w = int((t / n) % 8), act = int(t / (8 * n));
  const __nv_bfloat16* h = hT + size_t(act) * slot_stride;
  uint32_t word = 0u;
  for (int b = 0; b < 32; ++b) word |= uint32_t(__bfloat162float(h[size_t(w * 32 + b) * n + ev]) > 0.0f) << b;
  bits[(size_t(act) * n + ev) * 8 + w] = word;
}


// Integrand at given points (no VEGAS map): f[i] = f(x_i) in FP32; a failed
// event (non-finite, or unconverged phase space) is marked NaN.
template <int PROC>
__global__ void __launch_bounds__(128) points_kernel(KernelArgs a, const float* X, int D, float* f, long long n) {
  constexpr int NFL = ProcTraits<PROC>::NFL;
  constexpr int MAXD = ProcTraits<PROC>::MAXD;
  extern __shared__ __align__(16) unsigned char smem[];
  float* sh_pdf = reinterpret_cast<float*>(smem);
  SmPdf<float> pdf;
  if constexpr (NFL > 0) {
    const int nx = a.pdf.nx;
    float* t = sh_pdf;
    float* fv = t + nx;
    float* d = fv + NFL * nx;
    build_pdf_tables<float>(a.pdf, a.logq2_f, a.fl, NFL, t, fv, d);
#pragma unroll
    for (int k = 0; k < NFL; ++k) pdf.tab[k] = {t, fv + k * nx, d + k * nx, nx};
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float x[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) x[d] = d < D ? X[i * D + d] : 0.5f;
    const EventOut o = integrand<PROC, float>(a, pdf, x, nullptr);
    f[i] = (o.status == 0 && isfinite(o.f)) ? float(o.f) : __int_as_float(0x7fc00000);
  }
}

// The sampling pass's integrand fused with its sums: w = f(x) / q(x) =
// f exp(-log q), Kahan FP64 per thread, block partials (BlockPartial).
template <int PROC>
__global__ void __launch_bounds__(128) points_sums_kernel(KernelArgs a, const float* X, const float* logq, int D,
                                                          long long n, BlockPartial* parts) {
  constexpr int NFL = ProcTraits<PROC>::NFL;
  constexpr int MAXD = ProcTraits<PROC>::MAXD;
  extern __shared__ __align__(16) unsigned char smem[];
  float* sh_pdf = reinterpret_cast<float*>(smem);
  __shared__ BlockPartial warp_part[4];
  SmPdf<float> pdf;
  if constexpr (NFL > 0) {
    const int nx = a.pdf.nx;
    float* t = sh_pdf;
    float* fv = t + nx;
    float* d = fv + NFL * nx;
    build_pdf_tables<float>(a.pdf, a.logq2_f, a.fl, NFL, t, fv, d);
#pragma unroll
    for (int k = 0; k < NFL; ++k) pdf.tab[k] = {t, fv + k * nx, d + k * nx, nx};
  }
  Acc acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float x[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) x[d] = d < D ? X[i * D + d] : 0.5f;
    const EventOut o = integrand<PROC, float>(a, pdf, x, nullptr);
    double w = o.f * exp(-double(logq[i]));
    if (o.status != 0 || !isfinite(w)) {
      if (o.status == MC_ENOCONV)
        ++acc.nnoconv;
      else
        ++acc.nbad;
      w = 0.0;
    }
    const double y = w - acc.s_c;
    const double t = acc.s_hi + y;
    acc.s_c = (t - acc.s_hi) - y;
    acc.s_hi = t;
    const double y2 = w * w - acc.q_c;
    const double t2 = acc.q_hi + y2;
    acc.q_c = (t2 - acc.q_hi) - y2;
    acc.q_hi = t2;
    if (w != 0.0) ++acc.nnz;
    acc.wmax = fmax(acc.wmax, w);
  }
  block_reduce(acc, warp_part, &parts[blockIdx.x]);
}

// Training weights w = |f| / q = |f| exp(-log q) (0 for a failed event).
__global__ void flow_weights_kernel(const float* f, const float* logq, float* w, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float wi = fabsf(f[i]) * expf(-logq[i]);
  w[i] = isfinite(wi) ? wi : 0.0f;
}

// Loss sums in FP64: sums[0] = sum w, sums[1] = sum w log q, in a fixed
// order (deterministic): per-block partials, then one block sums them.
constexpr int kLossBlocks = 148;
__global__ void __launch_bounds__(256) loss_partials_kernel(const float* w, const float* logq, long long n,
                                                            double* part) {
  __shared__ double sh[2][8];
  double a = 0.0, b = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    a += w[i];
    b += double(w[i]) * logq[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) {
      sa += sh[0][k];
      sb += sh[1][k];
    }
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}
// One warp: lane j sums the partials j, j + 32, ... in order, then a fixed
// shuffle tree adds the 32 lane sums (deterministic for a given nblocks).
__global__ void loss_final_kernel(const double* part, int nblocks, double* sums) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double sa = 0.0, sb = 0.0;
  for (int k = lane; k < nblocks; k += 32) {
    sa += part[2 * k];
    sb += part[2 * k + 1];
  }
  for (int off = 16; off > 0; off >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
    sb += __shfl_xor_sync(0xffffffffu, sb, off);
  }
  if (lane == 0) {
    sums[0] = sa;
    sums[1] = sb;
  }
}

// Adam (thesis Sec. "Optimizers") on every master parameter; gradients of the
// 256-wide weights are read from their transposed layout.
struct AdamArgs {
  float lr, b1, b2, eps;
  const float* c;  // [2] on the device: 1/(1 - b1^t), 1/(1 - b2^t) of step t
};
// Advances the device step count t and forms Adam's bias corrections of step
// t (one thread): the powers b1^t, b2^t kept as running FP64 products in
// pw[0..1] (one multiplication each per step instead of a pow), the
// corrections rounded to FP32 as the update uses them.
__global__ void adam_prep_kernel(long long* step, double* pw, float* c, double b1, double b2) {
  ++*step;
  const double p1 = pw[0] * b1, p2 = pw[1] * b2;
  pw[0] = p1;
  pw[1] = p2;
  c[0] = float(1.0 / (1.0 - p1));
  c[1] = float(1.0 / (1.0 - p2));
}
// One Adam update (thesis Sec. "Optimizers": beta1, beta2, eps; c1, c2 the
// bias corrections of the step) of parameter p with gradient g and moments
// m, v; returns the new parameter.
__device__ __forceinline__ float adam_update(float& p, float& m, float& v, float g, const AdamArgs& A, float c1,
                                             float c2) {
  m = A.b1 * m + (1.0f - A.b1) * g;
  v = A.b2 * v + (1.0f - A.b2) * g * g;
  p = p - A.lr * (m * c1) / (sqrtf(v * c2) + A.eps);
  return p;
}

// Adam on the dense matrices W2, W3, W4 of layer blockIdx.y / 3 (their
// gradients kept transposed, gW^T [in x out]), one 32 x 32 tile per block
// of 32 x 8 threads: the gradient tile and the transposed BF16 copy go
// through shared memory, so that every array is read and written along its
// own rows.  Also refreshes the row-major BF16 copy.
__global__ void __launch_bounds__(256) adam_mat_kernel(float* params, const float* grads, float* m, float* v,
                                                       const LayerDev* layers, AdamArgs A) {
  __shared__ float tile[32][33];
  const LayerDev& L = layers[blockIdx.y / 3];
  const int which = blockIdx.y % 3;
  const size_t off = which == 0 ? L.off_W2 : (which == 1 ? L.off_W3 : L.off_W4);
  const int rows = which == 2 ? L.nout_pad : kH, cols = kH;  // W [rows x cols]
  __nv_bfloat16* h = which == 0 ? L.W2h : (which == 1 ? L.W3h : L.W4h);
  __nv_bfloat16* ht = which == 0 ? L.W2t : (which == 1 ? L.W3t : L.W4t);
  const int tiles_c = cols / 32;
  if (int(blockIdx.x) >= (rows / 32) * tiles_c) return;  // a smaller matrix than the grid's
  const int r0 = int(blockIdx.x) / tiles_c * 32, c0 = int(blockIdx.x) % tiles_c * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const float c1 = A.c[0], c2 = A.c[1];
  // tile[c][r] = gradient of W[r0 + r][c0 + c], stored at (c0 + c) rows + r0 + r
  for (int c = ty; c < 32; c += 8) tile[c][tx] = grads[off + size_t(c0 + c) * rows + r0 + tx];
  __syncthreads();
  float pv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    const size_t e = size_t(r0 + r) * cols + c0 + tx, idx = off + e;
    float p = params[idx], mi = m[idx], vi = v[idx];
    pv[q] = adam_update(p, mi, vi, tile[tx][r], A, c1, c2);
    m[idx] = mi;
    v[idx] = vi;
    params[idx] = p;
    h[e] = __float2bfloat16_rn(p);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) tile[tx][ty + 8 * q] = pv[q];  // tile[c][r] = new W[r0 + r][c0 + c]
  __syncthreads();
  for (int c = ty; c < 32; c += 8) ht[size_t(c0 + c) * rows + r0 + tx] = __float2bfloat16_rn(tile[c][tx]);
}

// Adam on the rest of layer blockIdx.y: W1 and b1 (they refresh W1e and
// W1^T), b2, b3 and b4, taken as one index range of H na + 3 H + nout_pad
// elements.
__global__ void __launch_bounds__(256) adam_vec_kernel(float* params, const float* grads, float* m, float* v,
                                                       const LayerDev* layers, AdamArgs A) {
  const LayerDev& L = layers[blockIdx.y];
  const size_t sw = size_t(kH) * L.na, s0 = sw + kH;
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  size_t idx;
  if (t < sw)
    idx = L.off_W1 + t;
  else if (t < s0)
    idx = L.off_b1 + (t - sw);
  else if (t < s0 + kH)
    idx = L.off_b2 + (t - s0);
  else if (t < s0 + 2 * kH)
    idx = L.off_b3 + (t - s0 - kH);
  else if (t < s0 + 2 * kH + size_t(L.nout_pad))
    idx = L.off_b4 + (t - s0 - 2 * kH);
  else
    return;
  float p = params[idx], mi = m[idx], vi = v[idx];
  adam_update(p, mi, vi, grads[idx], A, A.c[0], A.c[1]);
  m[idx] = mi;
  v[idx] = vi;
  params[idx] = p;
  const __nv_bfloat16 hb = __float2bfloat16_rn(p);
  if (t < sw) {  // W1 [H x na]: W1e [H][64] and W1^T [16][H]
    L.W1e[(t / L.na) * kUK + t % L.na] = hb;
    L.W1t[(t % L.na) * kH + t / L.na] = hb;
  } else if (t < s0) {  // b1: column na of W1e
    L.W1e[(t - sw) * kUK + L.na] = hb;
  }
}

// W1e [H][64] = (W1 | b1 | 0) in BF16 (W1 [H x na], b1 [H], FP32).
__global__ void w1e_bf16_kernel(const float* W1, const float* b1, int na, __nv_bfloat16* W1e) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kH * kUK) return;
  const int j = idx / kUK, c = idx % kUK;
  W1e[idx] = __float2bfloat16_rn(c < na ? W1[size_t(j) * na + c] : (c == na ? b1[j] : 0.0f));
}

// W1t [16][H] = W1^T zero-padded (W1 [H x na], FP32).
__global__ void w1t_bf16_kernel(const float* W1, int na, __nv_bfloat16* W1t) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kUPad * kH) return;
  const int a = idx / kH, j = idx % kH;
  W1t[idx] = __float2bfloat16_rn(a < na ? W1[size_t(j) * na + a] : 0.0f);
}

__global__ void zero_kernel(float* p, size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0f;
}

__global__ void set_double_kernel(double* p, double v) { *p = v; }

// BF16 copy of W [rows x cols] and of its transpose.
__global__ void to_bf16_kernel(const float* W, int rows, int cols, __nv_bfloat16* out, __nv_bfloat16* out_t) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int r = idx / cols, c = idx % cols;
  const __nv_bfloat16 h = __float2bfloat16_rn(W[idx]);
  out[idx] = h;
  out_t[size_t(c) * rows + r] = h;
}


// ---------------------------------------------------------------------------
// Fused coupling layer (K = 32 bins): one persistent kernel per layer with
// two 128-event tiles in flight per SM.  For each tile the conditioner runs
// without leaving the SM: the compute warps write the first layer's input
// (u, 1, 0, ..) (BF16) into the tile's shared-memory operand buffer in the
// 128-byte-swizzled K-major layout the tensor cores read; four tcgen05
// products (W1e, W2, W3, then W4 in
// two-coordinate sub-blocks) stream the weights from L2 through a TMA ring
// into the tile's 256 TMEM columns, and the tile's compute warps turn each
// accumulator into the next operand (bias, ReLU, BF16) in the same buffer or
// feed the logits straight from TMEM to the spline.  Warp 0 streams the
// weights, warp 1 issues the MMAs, alternating between the two tiles so that
// one tile's products overlap the other's CUDA-core phases; warps 2-5 and
// 6-9 are the two tiles' compute groups (warp w owns TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31: one event per thread, all of its columns).
// KEEP (training) also writes the activations the backward needs.
constexpr int kFusedThreads = 320;
constexpr int kFusedCompute = 256;
constexpr uint32_t kFusedABytes = 128 * kH * 2;   // one 128 x 256 BF16 operand (4 swizzled chunks)

struct FusedLayerArgs {
  const float* P;  // [n][D] layer input
  float* Pout;     // [n][D] layer output (may equal P)
  float* logq;     // [n], log q -= sum log c
  const float* params;
  LayerDev L;
  int D;
  long long n;     // multiple of 128
  int* error;
  // training (all null / unused when sampling): the activations the backward
  // needs: h1, h2, h3 (BF16, row-major [n][256]) stored by TMA from the
  // operand buffer through the map of the activation buffer, at rows
  // h_row0 + m h_stride + event; the first-layer inputs U^T (BF16,
  // transposed [16][n]: rows u_a then a row of ones) and the logits (FP32,
  // with bias, transposed)
  long long h_row0, h_stride;
  __nv_bfloat16* UT;
  float* LT;
  uint32_t* bits;  // ReLU activity of h1, h2, h3: [3][n][8] words (bit c % 32 of word c / 32)
};

// Byte offset of row r, 16-byte unit u (0..31 along K) in the swizzled operand.
__device__ __forceinline__ uint32_t swz_off(int r, int u) {
  return uint32_t(u >> 3) * 16384u + uint32_t(r >> 3) * 1024u + uint32_t(r & 7) * 128u +
         uint32_t(((u & 7) ^ (r & 7)) << 4);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// KEEP: training (writes the activations for the backward); otherwise sampling.
constexpr int kFusedSubRows = 2 * kFusedLs;  // W4 rows of one two-coordinate sub-product

template <bool KEEP>
__global__ void __launch_bounds__(kFusedThreads, 1)
    flow_layer_fused_kernel(const __grid_constant__ CUtensorMap map_w1, const __grid_constant__ CUtensorMap map_w2,
                            const __grid_constant__ CUtensorMap map_w3, const __grid_constant__ CUtensorMap map_w4,
                            const __grid_constant__ CUtensorMap map_h, FusedLayerArgs g, int stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kMaxStages = 4;
  __shared__ __align__(8) uint64_t w_full[kMaxStages];
  __shared__ __align__(8) uint64_t w_empty[kMaxStages];
  __shared__ __align__(8) uint64_t a_ready[2], acc_full[2], fin_bar;
  __shared__ __align__(8) uint64_t st_free[2];  // training: a stored activation's operand buffer may be rewritten
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int failed;

  const LayerDev& L = g.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nout = L.nout_pad;
  const int nsub = (L.nb + 1) / 2;  // W4 sub-products, two coordinates each
  const int nphase = 3 + nsub;  // W1e, W2, W3, then the W4 sub-products
  const uint32_t stage_bytes = uint32_t(kH) * 128u;
  unsigned char* ring = smem + 2 * kFusedABytes;
  const int m_tiles = int(g.n / 128);
  const int my_tiles = int(blockIdx.x) < m_tiles ? (m_tiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  auto sub_rows = [&](int k) { return k == nsub - 1 ? nout - kFusedSubRows * k : kFusedSubRows; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&a_ready[s], kFusedCompute / 2);
      mbar_init(&acc_full[s], 1);
      mbar_init(&st_free[s], 1);
    }
    mbar_init(&fin_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // weight stream, in the MMA order: per pair of tiles, phase by phase,
    // tile 0 then tile 1; four 64-wide K chunks per product
    if (lane == 0 && my_tiles > 0) {
      int it = 0;
      for (int j = 0; 2 * j < my_tiles && !failed; ++j)
        for (int p = 0; p < nphase && !failed; ++p)
          for (int s = 0; s < 2 && !failed; ++s) {
            if (2 * j + s >= my_tiles) continue;
            for (int c = 0; c < (p == 0 ? 1 : 4); ++c, ++it) {
              const int st = it % stages;
              const uint32_t use = uint32_t(it / stages);
              if (use > 0 && !mbar_wait(&w_empty[st], (use - 1) & 1u)) {
                failed = 1;
                atomicExch(g.error, 21);
                break;
              }
              unsigned char* dst = ring + size_t(st) * stage_bytes;
              if (p < 3) {
                mbar_expect_tx(&w_full[st], stage_bytes);
                tma_load_2d(dst, p == 0 ? &map_w1 : (p == 1 ? &map_w2 : &map_w3), c * 64, 0, &w_full[st]);
              } else {
                const int k = p - 3, rows = sub_rows(k);
                mbar_expect_tx(&w_full[st], uint32_t(rows) * 128u);
                for (int b = 0; b < rows / 32; ++b)
                  tma_load_2d(dst + size_t(b) * 32 * 128, &map_w4, c * 64, kFusedSubRows * k + 32 * b, &w_full[st]);
              }
            }
          }
      for (int st = 0; st < stages && st < it; ++st) mbar_wait(&w_full[st], uint32_t((it - 1 - st) / stages) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      int it = 0, use_a[2] = {0, 0};
      bool ok = true;
      for (int j = 0; 2 * j < my_tiles && ok; ++j)
        for (int p = 0; p < nphase && ok; ++p)
          for (int s = 0; s < 2 && ok; ++s) {
            if (2 * j + s >= my_tiles) continue;
            if (!mbar_wait(&a_ready[s], uint32_t(use_a[s]++) & 1u) || failed) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int nn = p < 3 ? kH : sub_rows(p - 3);
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(nn >> 3) << 17) | (8u << 24);
            const uint32_t d = tmem + uint32_t(s) * kH;
            for (int c = 0; c < (p == 0 ? 1 : 4); ++c, ++it) {
              const int st = it % stages;
              if (!mbar_wait(&w_full[st], uint32_t(it / stages) & 1u)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const uint64_t ad = smem_desc(smem_u32(smem + size_t(s) * kFusedABytes + c * 16384));
              const uint64_t bd = smem_desc(smem_u32(ring + size_t(st) * stage_bytes));
#pragma unroll
              for (int k = 0; k < 4; ++k)
                mma_bf16(d, ad + uint64_t(k * 2), bd + uint64_t(k * 2), idesc, (c > 0 || k > 0) ? 1u : 0u);
              mma_commit(&w_empty[st]);
            }
            if (!ok) break;
            mma_commit(&acc_full[s]);
          }
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 22);
      }
      mma_commit(&fin_bar);  // every MMA issued here completes before the TMEM is released
      mbar_wait(&fin_bar, 0);
    }
  } else {
    const int slot = (warp - 2) >> 2, q = warp & 3;
    const int r = q * 32 + lane;  // event row in the tile (= TMEM lane)
    const uint32_t trow = tmem + (uint32_t(q * 32) << 16) + uint32_t(slot) * kH;
    unsigned char* abuf = smem + size_t(slot) * kFusedABytes;
    const float* prm = g.params;
    int use_acc = 0;
    // training: thread 0 of warp q = 0 stores h1, h2, h3 of the tile from the
    // operand buffer by TMA once every thread of the tile has written it (the
    // a_ready phase); before the buffer is written again it waits until the
    // store has read it and releases the buffer (st_free), which every thread
    // waits for before it writes.
    const bool issuer = KEEP && q == 0 && lane == 0;
    int a_arrivals = 0, stores = 0, frees = 0;
    bool pending = false;  // issuer: a store whose reads may be in flight
    auto arrive_a = [&]() {
      mbar_arrive(&a_ready[slot]);
      ++a_arrivals;
    };
    // after arrive_a for activation m of the tile with first row row0
    auto store_h = [&](int m, long long row0) -> bool {
      bool ok = true;
      if (issuer) {
        ok = mbar_wait(&a_ready[slot], uint32_t(a_arrivals - 1) & 1u);
        if (ok) {
          const int y = int(g.h_row0 + m * g.h_stride + row0);
#pragma unroll
          for (int c = 0; c < 4; ++c) tma_store_2d(&map_h, 64 * c, y, abuf + c * 16384);
          bulk_commit();
          pending = true;
        }
      }
      ++stores;
      __syncwarp();
      return __all_sync(0xffffffffu, ok);
    };
    // before this thread writes the operand buffer: every store of it has read it
    auto buffer_free = [&]() -> bool {
      if (issuer && pending) {
        bulk_wait_read();
        mbar_arrive(&st_free[slot]);
        pending = false;
      }
      bool ok = true;
      while (ok && frees < stores) ok = mbar_wait(&st_free[slot], uint32_t(frees++) & 1u);
      return __all_sync(0xffffffffu, ok);
    };
    for (int i = slot; i < my_tiles; i += 2) {
      const long long row0 = (long long)(int(blockIdx.x) + i * int(gridDim.x)) * 128;
      const long long ev = row0 + r;
      const float* Pe = g.P + ev * g.D;
      float* Po = g.Pout + ev * g.D;
      if (__any_sync(0xffffffffu, failed != 0)) break;
      if (KEEP && !buffer_free()) {
        failed = 1;
        if (lane == 0) atomicExch(g.error, 24);
        break;
      }
      // the first-layer input (u_a, 1, zeros) as the A operand of the W1e product
      {
        __nv_bfloat16 v[16];
#pragma unroll
        for (int a = 0; a < 16; ++a) {
          const float x = a < L.na ? 2.0f * Pe[L.a_idx[a < L.na ? a : 0]] - 1.0f : (a == L.na ? 1.0f : 0.0f);
          v[a] = __float2bfloat16_rn(x);
        }
        if (KEEP) {
          for (int a = 0; a < L.na; ++a) Po[L.a_idx[a]] = Pe[L.a_idx[a]];
#pragma unroll
          for (int a = 0; a < 16; ++a)
            if (a <= L.na) g.UT[size_t(a) * g.n + ev] = v[a];
        }
        *reinterpret_cast<uint4*>(abuf + swz_off(r, 0)) = *reinterpret_cast<const uint4*>(v);
        *reinterpret_cast<uint4*>(abuf + swz_off(r, 1)) = *reinterpret_cast<const uint4*>(v + 8);
#pragma unroll
        for (int u16 = 2; u16 < kUK / 8; ++u16) *reinterpret_cast<uint4*>(abuf + swz_off(r, u16)) = make_uint4(0u, 0u, 0u, 0u);
      }
      fence_async_smem();
      arrive_a();
      // three hidden products: accumulator -> (bias), ReLU, BF16 -> operand buffer
      bool ok = true;
      for (int m = 0; m < 3 && ok; ++m, ++use_acc) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[slot], uint32_t(use_acc) & 1u))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (KEEP && !buffer_free()) {
          ok = false;
          break;
        }
        const float* bias = m == 0 ? nullptr : prm + (m == 1 ? L.off_b2 : L.off_b3);  // b1 is inside W1e
        for (int cg = 0; cg < 4; ++cg) {  // 4 groups of 4 x 16 columns
          uint32_t v[4][16];
          const int col0 = cg * 64;
          uint32_t mb0 = 0u, mb1 = 0u;  // training: ReLU activity of columns col0 .. col0 + 63
#pragma unroll
          for (int x = 0; x < 4; ++x) tmem_ld16_nw(trow + uint32_t(col0 + 16 * x), v[x]);
          tmem_wait_ld();
#pragma unroll
          for (int x = 0; x < 4; ++x) {
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
              uint4 pk;
              uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
              float bv[8];
              if (bias) {
                const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + col0 + 16 * x + 8 * hlf));
                const float4 b1v = __ldg(reinterpret_cast<const float4*>(bias + col0 + 16 * x + 8 * hlf + 4));
                bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
                bv[4] = b1v.x; bv[5] = b1v.y; bv[6] = b1v.z; bv[7] = b1v.w;
              } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) bv[e] = 0.0f;
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float o0 = fmaxf(__uint_as_float(v[x][8 * hlf + 2 * e]) + bv[2 * e], 0.0f);
                const float o1 = fmaxf(__uint_as_float(v[x][8 * hlf + 2 * e + 1]) + bv[2 * e + 1], 0.0f);
                const __nv_bfloat162 hh = __floats2bfloat162_rn(o0, o1);
                pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
                if (KEEP) {
                  // bits c64, c64 + 1 of the group: the BF16 activation is
                  // > 0, i.e. its magnitude bits are not all zero (after the
                  // ReLU it is never negative); c64 is a constant once the
                  // loops are unrolled, so the words stay in registers
                  const int c64 = 16 * x + 8 * hlf + 2 * e;
                  const uint32_t b2 = uint32_t((pw[e] & 0x7FFFu) != 0u) | (uint32_t((pw[e] & 0x7FFF0000u) != 0u) << 1);
                  if (c64 < 32)
                    mb0 |= b2 << c64;
                  else
                    mb1 |= b2 << (c64 - 32);
                }
              }
              *reinterpret_cast<uint4*>(abuf + swz_off(r, (col0 + 16 * x + 8 * hlf) >> 3)) = pk;
            }
          }
          if (KEEP) reinterpret_cast<uint2*>(g.bits + (size_t(m) * g.n + ev) * 8)[cg] = make_uint2(mb0, mb1);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        fence_async_smem();
        arrive_a();
        if (KEEP && !store_h(m, row0)) ok = false;
      }
      // W4 sub-products: the logits of two coordinates at a time, straight
      // from TMEM into the spline (coordinates in order, log c summed in order)
      float ld = 0.0f;
      for (int k = 0; k < nsub && ok; ++k, ++use_acc) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[slot], uint32_t(use_acc) & 1u))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int jj = 0; jj < 2; ++jj) {
          const int j = 2 * k + jj;
          if (j >= L.nb) break;
          float lg[kFusedLs];
#pragma unroll
          for (int x = 0; x < kFusedLs / 16; ++x)
            tmem_ld16_nw(trow + uint32_t(jj * kFusedLs + 16 * x), reinterpret_cast<uint32_t*>(lg + 16 * x));
          tmem_wait_ld();
          if (k + 1 < nsub && (jj == 1 || j + 1 >= L.nb)) {
            // the sub-product's last logits are in registers: the accumulator
            // is free, and the next sub-product's MMA runs beside this spline
            asm volatile("tcgen05.fence::before_thread_sync;");
            arrive_a();
          }
          const float4* b4 = reinterpret_cast<const float4*>(prm + L.off_b4 + j * kFusedLs);
#pragma unroll
          for (int kk = 0; kk < kFusedLs / 4; ++kk) {
            const float4 bb = __ldg(b4 + kk);
            lg[4 * kk] += bb.x;
            lg[4 * kk + 1] += bb.y;
            lg[4 * kk + 2] += bb.z;
            lg[4 * kk + 3] += bb.w;
          }
          if (KEEP) {
#pragma unroll
            for (int kk = 0; kk < 2 * kFusedK + 1; ++kk) g.LT[size_t(j * kFusedLs + kk) * g.n + ev] = lg[kk];
          }
          Spline sp;
          spline_load_regs<kFusedK>(lg, sp);
          float lc;
          const int d = L.b_idx[j];
          Po[d] = spline_fwd(sp, kFusedK, Pe[d], &lc);
          ld += lc;
        }
      }
      if (!ok) {
        failed = 1;
        if (lane == 0) atomicExch(g.error, 23);
        break;
      }
      g.logq[ev] -= ld;
    }
    if (issuer) bulk_wait_all();  // the stores are complete before the kernel ends
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// Fused coupling-layer backward (K = 32 bins): the mirror of the fused layer.
// Per tile of 128 events the compute warps run the spline backward and write
// the logit gradients G (BF16) into the swizzled operand buffer; then four
// tcgen05 products follow the chain dA3 = (G W4) * [h3 > 0], dA2 = (dA3 W3) *
// [h2 > 0], dA1 = (dA2 W2) * [h1 > 0], dU = dA1 W1, each accumulator turned
// into the next operand by the compute warps (masks from the transposed
// activations); the transposed gradients G^T, dA3^T, dA2^T, dA1^T go to
// global memory for the weight-gradient products, dU into the conditioning
// coordinates of dP.  Weights (transposed, BF16) stream through a TMA ring.
struct FusedBwdArgs {
  const float* Y;   // [n][D] input of the inverse layer (= output of the forward layer)
  float* dP;        // [n][D] dL/d(inverse-layer output) in, dL/d(input) out
  const float* LT;  // logits transposed [nout_pad][n] (with bias)
  const float* w;
  const double* wsum;
  const uint32_t* bits;  // ReLU activity of h1, h2, h3: [3][n][8] words
  __nv_bfloat16 *GT, *dA3T, *dA2T, *dA1T;  // outputs, transposed
  LayerDev L;
  int D;
  long long n, n_real;
  int* error;
};

__global__ void __launch_bounds__(kFusedThreads, 1)
    flow_layer_bwd_kernel(const __grid_constant__ CUtensorMap map_w4t, const __grid_constant__ CUtensorMap map_w3t,
                          const __grid_constant__ CUtensorMap map_w2t, const __grid_constant__ CUtensorMap map_w1t,
                          FusedBwdArgs g, int stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kMaxStages = 4;
  __shared__ __align__(8) uint64_t w_full[kMaxStages];
  __shared__ __align__(8) uint64_t w_empty[kMaxStages];
  __shared__ __align__(8) uint64_t a_ready, acc_full, fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int failed;

  const LayerDev& L = g.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nout = L.nout_pad, kc0 = nout / 64;  // K chunks of the first product
  const uint32_t stage_bytes = uint32_t(kH) * 128u;
  unsigned char* abuf = smem;
  unsigned char* ring = smem + size_t(max(kH, nout)) * 256;
  const int m_tiles = int(g.n / 128);
  const int my_tiles = int(blockIdx.x) < m_tiles ? (m_tiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int per_tile = kc0 + 12;  // weight chunks per tile: W4^T, W3^T, W2^T, W1^T

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    mbar_init(&a_ready, kFusedCompute);
    mbar_init(&acc_full, 1);
    mbar_init(&fin_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0 && my_tiles > 0) {
      int it = 0;
      for (int i = 0; i < my_tiles && !failed; ++i) {
        for (int q = 0; q < per_tile && !failed; ++q, ++it) {
          const int s = it % stages;
          const uint32_t use = uint32_t(it / stages);
          if (use > 0 && !mbar_wait(&w_empty[s], (use - 1) & 1u)) {
            failed = 1;
            atomicExch(g.error, 31);
            break;
          }
          unsigned char* dst = ring + size_t(s) * stage_bytes;
          if (q < kc0) {
            mbar_expect_tx(&w_full[s], stage_bytes);
            tma_load_2d(dst, &map_w4t, q * 64, 0, &w_full[s]);
          } else if (q < kc0 + 8) {
            const int c = (q - kc0) & 3;
            mbar_expect_tx(&w_full[s], stage_bytes);
            tma_load_2d(dst, q < kc0 + 4 ? &map_w3t : &map_w2t, c * 64, 0, &w_full[s]);
          } else {
            mbar_expect_tx(&w_full[s], uint32_t(kUPad) * 128u);
            tma_load_2d(dst, &map_w1t, (q - kc0 - 8) * 64, 0, &w_full[s]);
          }
        }
      }
      for (int s = 0; s < stages && s < it; ++s) mbar_wait(&w_full[s], uint32_t((it - 1 - s) / stages) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      const uint32_t idesc_h = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kH >> 3) << 17) | (8u << 24);
      const uint32_t idesc_u = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kUPad >> 3) << 17) | (8u << 24);
      int it = 0, use_a = 0;
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        for (int m = 0; m < 4 && ok; ++m, ++use_a) {
          if (!mbar_wait(&a_ready, uint32_t(use_a) & 1u) || failed) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int nk = m == 0 ? kc0 : 4;
          for (int c = 0; c < nk; ++c, ++it) {
            const int s = it % stages;
            if (!mbar_wait(&w_full[s], uint32_t(it / stages) & 1u)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t ad = smem_desc(smem_u32(abuf + c * 16384));
            const uint64_t bd = smem_desc(smem_u32(ring + size_t(s) * stage_bytes));
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_bf16(tmem, ad + uint64_t(k * 2), bd + uint64_t(k * 2), m == 3 ? idesc_u : idesc_h,
                       (c > 0 || k > 0) ? 1u : 0u);
            mma_commit(&w_empty[s]);
          }
          if (!ok) break;
          mma_commit(&acc_full);
        }
      }
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 32);
      }
      mma_commit(&fin_bar);
      mbar_wait(&fin_bar, 0);
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const uint32_t trow = tmem + (uint32_t(q * 32) << 16);
    const double wsum = *g.wsum;
    const size_t n = size_t(g.n);
    int use_acc = 0;
    for (int i = 0; i < my_tiles; ++i) {
      const long long ev = (long long)(int(blockIdx.x) + i * int(gridDim.x)) * 128 + r;
      const bool real = ev < g.n_real;
      float* dPe = g.dP + ev * g.D;
      const float* Ye = g.Y + ev * g.D;
      if (__any_sync(0xffffffffu, failed != 0)) break;
      // spline backward of this half's coordinates -> G (operand buffer, G^T)
      {
        const float gl = real ? float(-double(g.w[ev]) / wsum) : 0.0f;
        for (int j = half; j < L.nb; j += 2) {
          float gw[kFlowMaxBins], gv[kFlowMaxBins + 1];
          const int d = L.b_idx[j];
          if (real) {
            Spline sp;
            spline_load(g.LT + size_t(j) * kFusedLs * n + ev, n, kFusedK, sp);
            dPe[d] = spline_inv_bwd(sp, kFusedK, Ye[d], dPe[d], gl, gw, gv);
          } else {
            dPe[d] = 0.0f;
#pragma unroll
            for (int k = 0; k < kFlowMaxBins; ++k) gw[k] = gv[k] = 0.0f;
            gv[kFlowMaxBins] = 0.0f;
          }
          __nv_bfloat16* gt = g.GT + size_t(j) * kFusedLs * n + ev;
#pragma unroll
          for (int c8 = 0; c8 < kFusedLs / 8; ++c8) {
            uint4 pk;
            uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float v2[2];
#pragma unroll
              for (int h2 = 0; h2 < 2; ++h2) {
                const int k = c8 * 8 + 2 * e + h2;
                v2[h2] = k < kFusedK ? gw[k < kFusedK ? k : 0]
                                     : (k <= 2 * kFusedK ? gv[k <= 2 * kFusedK && k >= kFusedK ? k - kFusedK : 0]
                                                         : 0.0f);
              }
              const __nv_bfloat162 hh = __floats2bfloat162_rn(v2[0], v2[1]);
              pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
              if (c8 * 8 + 2 * e <= 2 * kFusedK) gt[size_t(c8 * 8 + 2 * e) * n] = hh.x;
              if (c8 * 8 + 2 * e + 1 <= 2 * kFusedK) gt[size_t(c8 * 8 + 2 * e + 1) * n] = hh.y;
            }
            *reinterpret_cast<uint4*>(abuf + swz_off(r, j * (kFusedLs / 8) + c8)) = pk;
          }
        }
        // zero the operand columns of the padding coordinates, and the rows of
        // G^T past the last coordinate (the buffer is shared by layers with
        // more transformed coordinates)
        if (half == 0) {
          for (int u = L.nb * (kFusedLs / 8); u < nout / 8; ++u)
            *reinterpret_cast<uint4*>(abuf + swz_off(r, u)) = make_uint4(0u, 0u, 0u, 0u);
          for (int c = L.nb * kFusedLs; c < nout; ++c) g.GT[size_t(c) * n + ev] = __float2bfloat16_rn(0.0f);
        }
      }
      fence_async_smem();
      mbar_arrive(&a_ready);
      // three masked products: accumulator * [h > 0] -> BF16 operand, transposed copy
      bool ok = true;
      for (int m = 0; m < 3 && ok; ++m, ++use_acc) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full, uint32_t(use_acc) & 1u))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // the activity bits of this thread's 128 columns of h3, h2, h1
        const uint4 mbv = reinterpret_cast<const uint4*>(g.bits + (size_t(2 - m) * n + ev) * 8)[half];
        const uint32_t mbw[4] = {mbv.x, mbv.y, mbv.z, mbv.w};
        __nv_bfloat16* outT = m == 0 ? g.dA3T : (m == 1 ? g.dA2T : g.dA1T);
        for (int cg = 0; cg < 2; ++cg) {
          uint32_t v[4][16];
          const int col0 = half * 128 + cg * 64;
#pragma unroll
          for (int x = 0; x < 4; ++x) tmem_ld16_nw(trow + uint32_t(col0 + 16 * x), v[x]);
          tmem_wait_ld();
#pragma unroll
          for (int x = 0; x < 4; ++x) {
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
              uint4 pk;
              uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int cc = col0 + 16 * x + 8 * hlf + 2 * e;
                const int jl = cc - half * 128;
                const uint32_t word = mbw[cg * 2 + (x >> 1)];  // jl >> 5 = 2 cg + x / 2
                const float o0 = (word >> (jl & 31)) & 1u ? __uint_as_float(v[x][8 * hlf + 2 * e]) : 0.0f;
                const float o1 = (word >> ((jl + 1) & 31)) & 1u ? __uint_as_float(v[x][8 * hlf + 2 * e + 1]) : 0.0f;
                const __nv_bfloat162 hh = __floats2bfloat162_rn(o0, o1);
                pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
                outT[size_t(cc) * n + ev] = hh.x;
                outT[size_t(cc + 1) * n + ev] = hh.y;
              }
              *reinterpret_cast<uint4*>(abuf + swz_off(r, (col0 + 16 * x + 8 * hlf) >> 3)) = pk;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        fence_async_smem();
        mbar_arrive(&a_ready);
      }
      if (ok && !__all_sync(0xffffffffu, mbar_wait(&acc_full, uint32_t(use_acc) & 1u))) ok = false;
      ++use_acc;
      if (!ok) {
        failed = 1;
        if (lane == 0) atomicExch(g.error, 33);
        break;
      }
      // dU = dA1 W1 into the conditioning coordinates: dL/dx_A += 2 dU
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (half == 0) {
        uint32_t v[16];
        tmem_ld16_nw(trow, v);
        tmem_wait_ld();
        for (int a = 0; a < L.na; ++a) dPe[L.a_idx[a]] += 2.0f * __uint_as_float(v[a < 16 ? a : 0]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// ---------------------------------------------------------------------------
// Backward chain of a coupling layer for training, after the spline backward
// (spline_inv_bwd_kernel has written the logit gradients G row-major, their
// transpose G^T and the spline part of dP): per tile of 128 events the four
// tcgen05 products dA3 = (G W4) * [h3 > 0], dA2 = (dA3 W3) * [h2 > 0],
// dA1 = (dA2 W2) * [h1 > 0] and dU = dA1 W1, with two tiles in flight per SM,
// one per half of the tensor memory (256 columns) and per operand buffer.
// Warp 0 loads each tile's G by TMA into its operand buffer and streams the
// transposed weights through a ring; warp 1 issues the MMAs, alternating
// between the two tiles phase by phase, so that one tile's products overlap
// the other tile's epilogues; warps 2-9 and 10-17 are the two tiles' compute
// groups (warp w owns TMEM lanes 32 (w % 4) .. +31; warps 2-5 / 10-13 the
// first 128 columns, 6-9 / 14-17 the other 128).  Each epilogue masks the
// accumulator with the ReLU activity bits, rounds it to BF16 into the operand
// buffer (the next product's A) and writes its transpose for the
// weight-gradient products; the last adds 2 dU to the conditioning
// coordinates of dP.  The arithmetic, and the order of every MMA, are those
// of flow_layer_bwd_kernel, so the results are the same bit for bit.
struct ChainBwdArgs {
  float* dP;             // [n][D]: dL/dx_A += 2 dU
  const uint32_t* bits;  // ReLU activity of h1, h2, h3: [3][n][8] words
  __nv_bfloat16 *dA3T, *dA2T, *dA1T;
  LayerDev L;
  int D;
  long long n;
  int* error;
};
constexpr int kChainThreads = 576;
constexpr size_t kChainSmemMax = 232448 - 1024;  // opt-in limit less the kernel's static shared memory
constexpr int kChainCompute = 256;  // compute threads per tile slot

__global__ void __launch_bounds__(kChainThreads, 1)
    flow_chain_bwd_kernel(const __grid_constant__ CUtensorMap map_g, const __grid_constant__ CUtensorMap map_w4t,
                          const __grid_constant__ CUtensorMap map_w3t, const __grid_constant__ CUtensorMap map_w2t,
                          const __grid_constant__ CUtensorMap map_w1t, ChainBwdArgs g, int stages) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kMaxStages = 4;
  __shared__ __align__(8) uint64_t w_full[kMaxStages];
  __shared__ __align__(8) uint64_t w_empty[kMaxStages];
  __shared__ __align__(8) uint64_t g_full[2], abuf_free[2], a_ready[2], acc_full[2], acc_empty[2], fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int failed;

  const LayerDev& L = g.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nout = L.nout_pad, kc0 = nout / 64;  // K chunks of the first product
  const uint32_t stage_bytes = uint32_t(kH) * 128u;
  const size_t abytes = size_t(max(kH, nout)) * 256;
  unsigned char* ring = smem + 2 * abytes;
  const int m_tiles = int(g.n / 128);
  const int my_tiles = int(blockIdx.x) < m_tiles ? (m_tiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  auto tile_row = [&](int i) { return (int(blockIdx.x) + i * int(gridDim.x)) * 128; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&g_full[s], 1);
      mbar_init(&abuf_free[s], 1);
      mbar_init(&a_ready[s], kChainCompute);
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], kChainCompute);
    }
    mbar_init(&fin_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0 && my_tiles > 0) {
      int it = 0;
      int loaded[2] = {0, 0};
      bool ok = true;
      for (int j = 0; 2 * j < my_tiles && ok; ++j) {
        // this pair's G tiles, each once the slot's previous tile has left its operand buffer
        for (int s = 0; s < 2 && ok; ++s) {
          if (2 * j + s >= my_tiles) continue;
          if (loaded[s] > 0 && !mbar_wait(&abuf_free[s], uint32_t(loaded[s] - 1) & 1u)) {
            ok = false;
            break;
          }
          unsigned char* dst = smem + size_t(s) * abytes;
          mbar_expect_tx(&g_full[s], uint32_t(kc0) * 16384u);
          for (int c = 0; c < kc0; ++c) tma_load_2d(dst + size_t(c) * 16384, &map_g, c * 64, tile_row(2 * j + s), &g_full[s]);
          ++loaded[s];
        }
        // the weights in the MMA order: phase by phase, tile 0 then tile 1
        for (int p = 0; p < 4 && ok; ++p)
          for (int s = 0; s < 2 && ok; ++s) {
            if (2 * j + s >= my_tiles) continue;
            const int nk = p == 0 ? kc0 : 4;
            for (int c = 0; c < nk; ++c, ++it) {
              const int st = it % stages;
              const uint32_t use = uint32_t(it / stages);
              if (use > 0 && !mbar_wait(&w_empty[st], (use - 1) & 1u)) {
                ok = false;
                break;
              }
              unsigned char* dst = ring + size_t(st) * stage_bytes;
              if (p < 3) {
                mbar_expect_tx(&w_full[st], stage_bytes);
                tma_load_2d(dst, p == 0 ? &map_w4t : (p == 1 ? &map_w3t : &map_w2t), c * 64, 0, &w_full[st]);
              } else {
                mbar_expect_tx(&w_full[st], uint32_t(kUPad) * 128u);
                tma_load_2d(dst, &map_w1t, c * 64, 0, &w_full[st]);
              }
            }
          }
      }
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 41);
      }
      // every copy issued here lands before the kernel ends
      for (int st = 0; st < stages && st < it; ++st) mbar_wait(&w_full[st], uint32_t((it - 1 - st) / stages) & 1u);
      for (int s = 0; s < 2; ++s)
        if (loaded[s] > 0) mbar_wait(&g_full[s], uint32_t(loaded[s] - 1) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      const uint32_t idesc_h = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kH >> 3) << 17) | (8u << 24);
      const uint32_t idesc_u = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kUPad >> 3) << 17) | (8u << 24);
      int it = 0;
      int use_a[2] = {0, 0}, done[2] = {0, 0};
      bool ok = true;
      for (int j = 0; 2 * j < my_tiles && ok; ++j)
        for (int p = 0; p < 4 && ok; ++p)
          for (int s = 0; s < 2 && ok; ++s) {
            if (2 * j + s >= my_tiles) continue;
            if (p == 0) {
              // the slot's accumulator is free once its compute group has read
              // the previous tile's dU, and its G tile has landed
              if ((done[s] > 0 && !mbar_wait(&acc_empty[s], uint32_t(done[s] - 1) & 1u)) ||
                  !mbar_wait(&g_full[s], uint32_t(done[s]) & 1u) || failed) {
                ok = false;
                break;
              }
            } else if (!mbar_wait(&a_ready[s], uint32_t(use_a[s]++) & 1u) || failed) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + uint32_t(s) * kH;
            const unsigned char* ab = smem + size_t(s) * abytes;
            const int nk = p == 0 ? kc0 : 4;
            for (int c = 0; c < nk; ++c, ++it) {
              const int st = it % stages;
              if (!mbar_wait(&w_full[st], uint32_t(it / stages) & 1u)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const uint64_t ad = smem_desc(smem_u32(ab + size_t(c) * 16384));
              const uint64_t bd = smem_desc(smem_u32(ring + size_t(st) * stage_bytes));
#pragma unroll
              for (int k = 0; k < 4; ++k)
                mma_bf16(d, ad + uint64_t(k * 2), bd + uint64_t(k * 2), p == 3 ? idesc_u : idesc_h,
                         (c > 0 || k > 0) ? 1u : 0u);
              mma_commit(&w_empty[st]);
            }
            if (!ok) break;
            mma_commit(&acc_full[s]);
            if (p == 3) {
              mma_commit(&abuf_free[s]);  // the operand buffer may take the slot's next G tile
              ++done[s];
            }
          }
      if (!ok) {
        failed = 1;
        atomicExch(g.error, 42);
      }
      mma_commit(&fin_bar);  // every MMA issued here completes before the TMEM is released
      mbar_wait(&fin_bar, 0);
    }
  } else {
    const int slot = (warp - 2) >> 3, half = ((warp - 2) >> 2) & 1, q = warp & 3;
    const int r = q * 32 + lane;  // event row in the tile (= TMEM lane)
    const uint32_t trow = tmem + (uint32_t(q * 32) << 16) + uint32_t(slot) * kH;
    unsigned char* abuf = smem + size_t(slot) * abytes;
    const size_t n = size_t(g.n);
    int use_acc = 0;
    for (int i = slot; i < my_tiles; i += 2) {
      const long long ev = (long long)tile_row(i) + r;
      if (__any_sync(0xffffffffu, failed != 0)) break;
      // the activity bits of this thread's 128 columns of h3, h2, h1 (three
      // named words, selected by the uniform m below: an array indexed at
      // run time would live in local memory)
      const uint4 mb_h3 = reinterpret_cast<const uint4*>(g.bits + (size_t(2) * n + ev) * 8)[half];
      const uint4 mb_h2 = reinterpret_cast<const uint4*>(g.bits + (size_t(1) * n + ev) * 8)[half];
      const uint4 mb_h1 = reinterpret_cast<const uint4*>(g.bits + ev * 8)[half];
      bool ok = true;
      for (int m = 0; m < 3 && ok; ++m, ++use_acc) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[slot], uint32_t(use_acc) & 1u))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint4 mbm = m == 0 ? mb_h3 : (m == 1 ? mb_h2 : mb_h1);
        __nv_bfloat16* outT = m == 0 ? g.dA3T : (m == 1 ? g.dA2T : g.dA1T);
        for (int cg = 0; cg < 2; ++cg) {
          const uint32_t wlo = cg == 0 ? mbm.x : mbm.z, whi = cg == 0 ? mbm.y : mbm.w;
          uint32_t v[4][16];
          const int col0 = half * 128 + cg * 64;
#pragma unroll
          for (int x = 0; x < 4; ++x) tmem_ld16_nw(trow + uint32_t(col0 + 16 * x), v[x]);
          tmem_wait_ld();
#pragma unroll
          for (int x = 0; x < 4; ++x) {
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
              uint4 pk;
              uint32_t* pw = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int cc = col0 + 16 * x + 8 * hlf + 2 * e;
                const int jl = cc - half * 128;
                const uint32_t word = (x >> 1) == 0 ? wlo : whi;  // word jl >> 5 = 2 cg + x / 2
                const float o0 = (word >> (jl & 31)) & 1u ? __uint_as_float(v[x][8 * hlf + 2 * e]) : 0.0f;
                const float o1 = (word >> ((jl + 1) & 31)) & 1u ? __uint_as_float(v[x][8 * hlf + 2 * e + 1]) : 0.0f;
                const __nv_bfloat162 hh = __floats2bfloat162_rn(o0, o1);
                pw[e] = *reinterpret_cast<const uint32_t*>(&hh);
                outT[size_t(cc) * n + ev] = hh.x;
                outT[size_t(cc + 1) * n + ev] = hh.y;
              }
              *reinterpret_cast<uint4*>(abuf + swz_off(r, (col0 + 16 * x + 8 * hlf) >> 3)) = pk;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        fence_async_smem();
        mbar_arrive(&a_ready[slot]);
      }
      if (ok && !__all_sync(0xffffffffu, mbar_wait(&acc_full[slot], uint32_t(use_acc) & 1u))) ok = false;
      ++use_acc;
      if (!ok) {
        failed = 1;
        if (lane == 0) atomicExch(g.error, 43);
        break;
      }
      // dU = dA1 W1 into the conditioning coordinates: dL/dx_A += 2 dU
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (half == 0) {
        uint32_t v[16];
        tmem_ld16_nw(trow, v);
        tmem_wait_ld();
        float* dPe = g.dP + ev * g.D;
#pragma unroll
        for (int a = 0; a < kMaxA; ++a)
          if (a < L.na) dPe[L.a_idx[a]] += 2.0f * __uint_as_float(v[a]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&acc_empty[slot]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace
}  // namespace mc

using mc::BlockPartial;
using mc::LayerDev;
using mc::kH;

struct mc_flow_s {
  int device = 0, D = 0, L = 0, K = 0;
  long long max_batch = 0, bp = 0;  // capacity (rows, padded to 128)
  uint64_t seed = 0;
  int step = 0;
  std::vector<LayerDev> layers;
  size_t nparam = 0;             // device master-parameter count (padded layout)
  std::vector<size_t> host_map;  // packed host index -> device index
  float *d_params = nullptr, *d_grads = nullptr, *d_m = nullptr, *d_v = nullptr;
  __nv_bfloat16* d_wbf = nullptr;  // BF16 weights and transposes of all layers
  LayerDev* d_layers = nullptr;
  // workspace
  float *P = nullptr, *logq = nullptr, *f = nullptr, *w = nullptr, *dP = nullptr, *LT = nullptr;
  __nv_bfloat16 *h = nullptr, *hT = nullptr, *G = nullptr, *GT = nullptr, *dA = nullptr, *dAT = nullptr;
  __nv_bfloat16* UT = nullptr;  // per layer: first-layer inputs, transposed [16][n]
  uint32_t* MB = nullptr;       // per layer: ReLU activity bits of h1, h2, h3 [3][n][8]
  float* dU = nullptr;          // [n][16] input gradient of the first layer
  __nv_bfloat16* U = nullptr;   // [n][64] first-layer inputs of the layer-by-layer path
  float* part = nullptr;  // split-K partial products of the weight gradients
  float* bpart = nullptr;  // and the per-split row sums of their gradient operands (bias gradients)
  size_t part_region = 0, bpart_region = 0;  // floats per partial / bias-partial region
  int max_splits = 0;
  double* sums = nullptr;
  double* h_sums = nullptr;  // pinned
  BlockPartial *parts = nullptr, *chunk_totals = nullptr, *total = nullptr, *h_total = nullptr;
  long long max_chunks = 0;
  // sampling chunks of the fused path (which needs only the points and log q)
  long long sbp = 0;
  float *Ps = nullptr, *lqs = nullptr;
  int* err = nullptr;
  // the training step count on the device (mirrors `step`) and Adam's bias
  // corrections of the current step
  long long* d_step = nullptr;
  double* d_adam_pow = nullptr;  // b1^t, b2^t
  float* d_adam = nullptr;
  // the stream a training step is captured on and replayed from as a CUDA
  // graph, and the events that order it after and before the caller's stream
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // the weight-gradient products of a fused backward layer run on `side`
  // after the layer's chain (ev_chain), beside the next layers' spline
  // backward and chain on the caller's stream; the logit gradients G, G^T and
  // the activation gradients dA^T are double-buffered by layer parity, and a
  // layer waits for the side work of the layer two before it (ev_side)
  // before it rewrites that buffer set
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> ev_chain, ev_side;
  int nout_pad_max = 0;
  // data-parallel step: events of the batch sampled by mc_flow_step_sample
  // and not yet differentiated (0: none)
  long long step_n = 0;
  // fused layers (K = 32, nout_pad <= 512): tensor maps of W2, W3, W4, W1e per layer
  bool use_fused = true;      // fused forward layers
  bool use_fused_bwd = true;  // fused backward layers
  std::vector<bool> fused_ok;
  std::vector<CUtensorMap> maps;
  std::vector<CUtensorMap> bwd_maps;  // W4^T, W3^T, W2^T, W1^T per layer (fused backward)
  // two-tile backward chain (flow_chain_bwd_kernel): the row-major logit
  // gradients G of each layer as a TMA source, and whether the layer fits
  std::vector<CUtensorMap> g_maps;
  std::vector<bool> chain_ok;
  // the row-major activations h of every layer as one TMA map ([L x 3 x bp]
  // rows of 256, boxes of 64 x 128): the fused training layer stores h1, h2,
  // h3 through it
  CUtensorMap h_map;
  bool h_map_ok = false;
};

namespace {

int ffail(int code, const std::string& msg) {
  mc::set_last_error(msg.c_str());
  return code;
}

#define FLOW_CUDA(call)                                                                                   \
  do {                                                                                                    \
    const cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return ffail(MC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kPartsGrid = 148 * 8;  // blocks of the fused sampling integrand

long long pad128(long long n) { return (n + 127) / 128 * 128; }

float* P_of(mc_flow F, int l) { return F->P + size_t(l) * F->bp * F->D; }
__nv_bfloat16* h_of(mc_flow F, int l, int k) { return F->h + (size_t(l) * 3 + k) * F->bp * kH; }
__nv_bfloat16* hT_of(mc_flow F, int l, int k) { return F->hT + (size_t(l) * 3 + k) * F->bp * kH; }
float* LT_of(mc_flow F, int l) { return F->LT + size_t(l) * F->bp * F->nout_pad_max; }
__nv_bfloat16* UT_of(mc_flow F, int l) { return F->UT + size_t(l) * F->bp * mc::kUPad; }
uint32_t* MB_of(mc_flow F, int l) { return F->MB + size_t(l) * 3 * F->bp * 8; }
// buffer set `set` (0 or 1) of the logit gradients G [n][nout_pad] and G^T,
// and of dA3^T, dA2^T, dA1^T (three slices of bp x 256)
__nv_bfloat16* G_of(mc_flow F, int set) { return F->G + size_t(set) * F->bp * F->nout_pad_max; }
__nv_bfloat16* GT_of(mc_flow F, int set) { return F->GT + size_t(set) * F->bp * F->nout_pad_max; }
__nv_bfloat16* dAT_of(mc_flow F, int set, int k) { return F->dAT + (size_t(set) * 3 + k) * F->bp * kH; }

// ReLU activity bits of layer slot l from its transposed activations (n rows).
void make_mask_bits(mc_flow F, int l, long long n, cudaStream_t st) {
  mc::mask_bits_kernel<<<mc::blocks_for(24 * n, 256), 256, 0, st>>>(hT_of(F, l, 0), size_t(F->bp) * kH, n, MB_of(F, l));
}

// N tile: the largest multiple of 16 up to 256 that divides N.
int pick_bn(int N) {
  for (int bn = std::min(256, N) / 16 * 16; bn >= 16; bn -= 16)
    if (N % bn == 0) return bn;
  return 16;
}

// Persistent B-resident product out = epilogue(A [n x K] . B^T), B [N x K];
// for the ReLU-mask epilogue, mask is the activation transposed [N][n].
int gemm_rs(mc_flow F, long long n, int N, int K, int epi, const __nv_bfloat16* a, const __nv_bfloat16* b,
            const float* bias, void* c, void* c_t, const __nv_bfloat16* mask, cudaStream_t st) {
  FLOW_CUDA(cudaGetLastError());  // launches queued before this product
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = int(n);
  g.N = N;
  g.K = K;
  g.bn = pick_bn(N);
  g.epilogue = epi;
  g.bias = bias;
  g.ldc = N;
  g.ldt = int(n);
  if (epi == mc::kEpiBiasF32) {
    g.c_f32 = static_cast<float*>(c);
    g.c_t_f32 = static_cast<float*>(c_t);
  } else {
    g.c_bf16 = static_cast<__nv_bfloat16*>(c);
    g.c_t_bf16 = static_cast<__nv_bfloat16*>(c_t);
  }
  g.mask_t = mask;  // the layer's activation transposed [N][n]
  g.ld_mask_t = int(n);
  g.error = F->err;
  FLOW_CUDA(mc::tc_gemm_rs(g, a, K, b, K, st));
  return MC_OK;
}

// Split-K partial tiles of the weight gradient X^T . YT^T over the n events
// (K = n): X the activations, row-major [n][H] (x_rows) or transposed
// [H][n], YT the gradients transposed [N][n]; the partials go to part
// [splits][H][N] and, with bpart, the row sums of YT (the bias gradient's
// partials, formed by the product's CTAs from the YT tiles they stage
// anyway) to bpart [splits][N].  The split count is returned in *splits.
int wgrad_partials(mc_flow F, long long n, int N, const __nv_bfloat16* X, bool x_rows, const __nv_bfloat16* YT,
                   float* part, float* bpart, cudaStream_t st, int* splits_out) {
  FLOW_CUDA(cudaGetLastError());
  const int bn = pick_bn(N);
  const int tiles = (kH / 128) * (N / bn);
  const int kb = int(n / 64);
  int splits = std::max(1, std::min({F->max_splits, (148 + tiles - 1) / tiles, kb}));
  const int per = (kb + splits - 1) / splits;  // k blocks per split: no split left empty
  splits = (kb + per - 1) / per;
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = kH;
  g.N = N;
  g.K = int(n);
  g.bn = bn;
  g.epilogue = mc::kEpiPartialF32;
  g.c_f32 = part;
  g.ldc = N;
  g.error = F->err;
  g.rowsum_b = bpart;
  if (x_rows)
    FLOW_CUDA(mc::tc_gemm_xn(g, X, kH, YT, int(n), splits, st));
  else
    FLOW_CUDA(mc::tc_gemm(g, X, int(n), YT, int(n), splits, st));
  *splits_out = splits;
  return MC_OK;
}

// Weight gradient gW^T [H x N] += X^T . YT^T (wgrad_partials into the shared
// partial buffer, then a fixed-order sum over the splits); with gb, the bias
// gradient gb [N] += the row sums of YT, summed over the splits in the same
// order.  With splits_out the caller sums the weight partials itself.
int gemm_wgrad(mc_flow F, long long n, int N, const __nv_bfloat16* X, bool x_rows, const __nv_bfloat16* YT,
               float* gWt, float* gb, cudaStream_t st, int* splits_out = nullptr) {
  int splits = 0;
  if (int rc = wgrad_partials(F, n, N, X, x_rows, YT, F->part, gb ? F->bpart : nullptr, st, &splits)) return rc;
  if (splits_out)
    *splits_out = splits;
  else
    FLOW_CUDA(mc::tc_reduce_splits(F->part, splits, size_t(kH) * N, gWt, st));
  if (gb) FLOW_CUDA(mc::tc_reduce_splits(F->bpart, splits, size_t(N), gb, st));
  return MC_OK;
}

// Conditioner of layer l on the points P (n rows): activations into slot
// `slot` (with their transposes when `keep`), transposed logits into LT_of(slot).
int conditioner(mc_flow F, int l, int slot, const float* P, long long n, bool keep, cudaStream_t st) {
  const LayerDev& L = F->layers[l];
  const float* prm = F->d_params;
  __nv_bfloat16 *h1 = h_of(F, slot, 0), *h2 = h_of(F, slot, 1), *h3 = h_of(F, slot, 2);
  mc::dense1_input_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P, F->D, L, F->U, keep ? UT_of(F, slot) : nullptr,
                                                                   n);
  if (int rc = gemm_rs(F, n, kH, mc::kUK, mc::kEpiBiasReluBf16, F->U, L.W1e, nullptr, h1,
                       keep ? hT_of(F, slot, 0) : nullptr, nullptr, st))
    return rc;
  if (int rc = gemm_rs(F, n, kH, kH, mc::kEpiBiasReluBf16, h1, L.W2h, prm + L.off_b2, h2,
                       keep ? hT_of(F, slot, 1) : nullptr, nullptr, st))
    return rc;
  if (int rc = gemm_rs(F, n, kH, kH, mc::kEpiBiasReluBf16, h2, L.W3h, prm + L.off_b3, h3,
                       keep ? hT_of(F, slot, 2) : nullptr, nullptr, st))
    return rc;
  return gemm_rs(F, n, L.nout_pad, kH, mc::kEpiBiasF32, h3, L.W4h, prm + L.off_b4, nullptr, LT_of(F, slot), nullptr,
                 st);
}

// One fused layer (flow_layer_fused_kernel) over n rows: sampling maps P[0]
// in place; keep (training) maps P[l] to P[l+1] and writes the transposed
// activations, first-layer inputs and logits of slot l.
int fused_layer(mc_flow F, int l, long long n, bool keep, cudaStream_t st, float* P0 = nullptr, float* lq = nullptr) {
  FLOW_CUDA(cudaGetLastError());  // launches queued before this one
  static int num_sms = 0;
  if (num_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
      num_sms = 1;
  }
  const LayerDev& L = F->layers[l];
  mc::FusedLayerArgs a;
  std::memset(&a, 0, sizeof(a));
  a.P = keep ? P_of(F, l) : (P0 ? P0 : P_of(F, 0));
  a.Pout = keep ? P_of(F, l + 1) : (P0 ? P0 : P_of(F, 0));
  a.logq = lq ? lq : F->logq;
  if (keep) {
    a.h_row0 = (long long)(h_of(F, l, 0) - F->h) / kH;
    a.h_stride = F->bp;
    a.UT = UT_of(F, l);
    a.LT = LT_of(F, l);
    a.bits = MB_of(F, l);
  }
  a.params = F->d_params;
  a.L = L;
  a.D = F->D;
  a.n = n;
  a.error = F->err;
  constexpr size_t kMaxDyn = 232448 - 1024;  // opt-in limit less the kernel's static shared memory
  const size_t stage = size_t(kH) * 128;
  const int stages = int(std::min<size_t>(4, (kMaxDyn - 1024 - 2 * mc::kFusedABytes) / stage));
  if (stages < 2) return ffail(MC_EINVAL, "mc_flow: fused layer does not fit in shared memory");
  const size_t smem = 1024 + 2 * mc::kFusedABytes + stages * stage;
  auto kern = keep ? mc::flow_layer_fused_kernel<true> : mc::flow_layer_fused_kernel<false>;
  FLOW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int grid = int(std::min<long long>(n / 128, num_sms));
  kern<<<grid, mc::kFusedThreads, smem, st>>>(F->maps[4 * l + 3], F->maps[4 * l], F->maps[4 * l + 1],
                                              F->maps[4 * l + 2], F->h_map, a, stages);
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// The L layers of the forward direction (see forward_pass); P0 / logq
// override the points and log q of the sampling path (fused layers only).
int forward_layers(mc_flow F, long long n, bool keep, cudaStream_t st, float* P0 = nullptr, float* lq = nullptr) {
  for (int l = 0; l < F->L; ++l) {
    if (F->use_fused && F->fused_ok[l]) {
      if (int rc = fused_layer(F, l, n, keep, st, P0, lq)) return rc;
      continue;
    }
    const int slot = keep ? l : 0;
    const float* Pin = keep ? P_of(F, l) : P_of(F, 0);
    float* Pout = keep ? P_of(F, l + 1) : P_of(F, 0);
    if (int rc = conditioner(F, l, slot, Pin, n, keep, st)) return rc;
    if (keep) make_mask_bits(F, l, n, st);
    mc::spline_fwd_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(Pin, Pout, F->D, F->layers[l], LT_of(F, slot),
                                                                   size_t(n), F->K, F->logq, n);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Forward (sampling direction) from P[0] = z over n (multiple of 128) rows;
// logq initialised to 0.  keep: layer l writes P[l+1] and keeps its
// activations (training); otherwise P[0] is mapped in place (sampling).
int forward_pass(mc_flow F, long long n, bool keep, cudaStream_t st) {
  FLOW_CUDA(cudaMemsetAsync(F->logq, 0, sizeof(float) * n, st));
  return forward_layers(F, n, keep, st);
}

// Inverse (density) pass from P[L] (the points x) down to P[0] = z, keeping
// every layer's activations; logq accumulated from 0.
int inverse_pass(mc_flow F, long long n, cudaStream_t st) {
  FLOW_CUDA(cudaMemsetAsync(F->logq, 0, sizeof(float) * n, st));
  for (int l = F->L - 1; l >= 0; --l) {
    if (int rc = conditioner(F, l, l, P_of(F, l + 1), n, true, st)) return rc;
    make_mask_bits(F, l, n, st);
    mc::spline_inv_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P_of(F, l + 1), P_of(F, l), F->D, F->layers[l],
                                                                   LT_of(F, l), size_t(n), F->K, F->logq, n);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Fused backward of layer l (flow_layer_bwd_kernel): dP updated, the
// transposed gradients G^T and dA3^T, dA2^T, dA1^T (three slices of F->dAT)
// written for the weight-gradient products.
int fused_bwd_layer(mc_flow F, int l, long long n, long long n_real, int set, cudaStream_t st) {
  FLOW_CUDA(cudaGetLastError());
  static int num_sms = 0;
  if (num_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
      num_sms = 1;
  }
  const LayerDev& L = F->layers[l];
  mc::FusedBwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.Y = P_of(F, l + 1);
  a.dP = F->dP;
  a.LT = LT_of(F, l);
  a.w = F->w;
  a.wsum = F->sums;
  a.bits = MB_of(F, l);
  a.GT = GT_of(F, set);
  a.dA3T = dAT_of(F, set, 0);
  a.dA2T = dAT_of(F, set, 1);
  a.dA1T = dAT_of(F, set, 2);
  a.L = L;
  a.D = F->D;
  a.n = n;
  a.n_real = n_real;
  a.error = F->err;
  constexpr size_t kMaxDyn = 232448 - 2048;  // opt-in limit less the kernel's static shared memory
  const size_t abytes = size_t(std::max(kH, L.nout_pad)) * 256, stage = size_t(kH) * 128;
  const int stages = int(std::min<size_t>(4, (kMaxDyn - 1024 - abytes) / stage));
  if (stages < 2) return ffail(MC_EINVAL, "mc_flow: fused backward does not fit in shared memory");
  const size_t smem = 1024 + abytes + stages * stage;
  FLOW_CUDA(cudaFuncSetAttribute(mc::flow_layer_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int grid = int(std::min<long long>(n / 128, num_sms));
  mc::flow_layer_bwd_kernel<<<grid, mc::kFusedThreads, smem, st>>>(F->bwd_maps[4 * l], F->bwd_maps[4 * l + 1],
                                                                   F->bwd_maps[4 * l + 2], F->bwd_maps[4 * l + 3], a,
                                                                   stages);
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Two-tile backward chain of layer l (flow_chain_bwd_kernel) after the spline
// backward has written G, G^T and the spline part of dP.
int chain_bwd_layer(mc_flow F, int l, long long n, int set, cudaStream_t st) {
  FLOW_CUDA(cudaGetLastError());
  static int num_sms = 0;
  if (num_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
      num_sms = 1;
  }
  const LayerDev& L = F->layers[l];
  mc::ChainBwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dP = F->dP;
  a.bits = MB_of(F, l);
  a.dA3T = dAT_of(F, set, 0);
  a.dA2T = dAT_of(F, set, 1);
  a.dA1T = dAT_of(F, set, 2);
  a.L = L;
  a.D = F->D;
  a.n = n;
  a.error = F->err;
  const size_t abytes = size_t(std::max(kH, L.nout_pad)) * 256, stage = size_t(kH) * 128;
  const int stages = int(std::min<size_t>(4, (mc::kChainSmemMax - 1024 - 2 * abytes) / stage));
  if (stages < 2) return ffail(MC_EINVAL, "mc_flow: backward chain does not fit in shared memory");
  const size_t smem = 1024 + 2 * abytes + stages * stage;
  FLOW_CUDA(cudaFuncSetAttribute(mc::flow_chain_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int grid = int(std::min<long long>(n / 128, num_sms));
  mc::flow_chain_bwd_kernel<<<grid, mc::kChainThreads, smem, st>>>(F->g_maps[2 * l + set], F->bwd_maps[4 * l],
                                                                  F->bwd_maps[4 * l + 1], F->bwd_maps[4 * l + 2],
                                                                  F->bwd_maps[4 * l + 3], a, stages);
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Backward of the density pass (weights F->w, sum w in F->sums[0]) over the
// kept activations: accumulates every parameter gradient into F->d_grads
// (zeroed beforehand).
int backward_pass(mc_flow F, long long n, long long n_real, cudaStream_t st) {
  const int D = F->D;
  float* g = F->d_grads;
  FLOW_CUDA(cudaMemsetAsync(F->dP, 0, sizeof(float) * n * D, st));
  int side_last = -1;  // the last layer whose weight gradients went to F->side
  auto join_side = [&]() -> int {
    if (side_last >= 0) FLOW_CUDA(cudaStreamWaitEvent(st, F->ev_side[side_last], 0));
    side_last = -1;
    return MC_OK;
  };
  for (int l = 0; l < F->L; ++l) {
    const LayerDev& L = F->layers[l];
    if (F->use_fused_bwd && F->fused_ok[l]) {
      // spline and activation gradients (the spline backward at full
      // occupancy, then the two-tile product chain; one fused kernel where the
      // chain's buffers do not fit), then the weight gradients on the side
      // stream, beside the next layers' spline backward and chain
      const int set = l & 1;
      if (l >= 2 && side_last >= l - 2) FLOW_CUDA(cudaStreamWaitEvent(st, F->ev_side[l - 2], 0));
      __nv_bfloat16 *G = G_of(F, set), *GT = GT_of(F, set);
      __nv_bfloat16 *dA3T = dAT_of(F, set, 0), *dA2T = dAT_of(F, set, 1), *dA1T = dAT_of(F, set, 2);
      if (F->chain_ok[l]) {
        mc::spline_bwd_k32_kernel<<<dim3(mc::blocks_for(n, 128), L.nb), 128, 0, st>>>(
            P_of(F, l + 1), F->dP, D, L, LT_of(F, l), F->w, F->sums, G, GT, n, n_real);
        if (int rc = chain_bwd_layer(F, l, n, set, st)) return rc;
      } else if (int rc = fused_bwd_layer(F, l, n, n_real, set, st)) {
        return rc;
      }
      FLOW_CUDA(cudaEventRecord(F->ev_chain[l], st));
      const cudaStream_t ss = F->side;
      FLOW_CUDA(cudaStreamWaitEvent(ss, F->ev_chain[l], 0));
      // W4, W3, W2 and with them the bias gradients b4, b3, b2 (the row sums
      // of G^T, dA3^T, dA2^T), and W1, b1: four products back to back, each
      // into its own partial region, then the six sums of W4..b2 in one
      // launch (each summed as tc_reduce_splits sums it alone)
      float* pw[4];
      float* pb[3];
      for (int k = 0; k < 4; ++k) pw[k] = F->part + size_t(k) * F->part_region;
      for (int k = 0; k < 3; ++k) pb[k] = F->bpart + size_t(k) * F->bpart_region;
      int s4 = 0, s3 = 0, s2 = 0, s1 = 0;
      if (int rc = wgrad_partials(F, n, L.nout_pad, h_of(F, l, 2), true, GT, pw[0], pb[0], ss, &s4)) return rc;
      if (int rc = wgrad_partials(F, n, kH, h_of(F, l, 1), true, dA3T, pw[1], pb[1], ss, &s3)) return rc;
      if (int rc = wgrad_partials(F, n, kH, h_of(F, l, 0), true, dA2T, pw[2], pb[2], ss, &s2)) return rc;
      if (int rc = wgrad_partials(F, n, mc::kUPad, dA1T, false, UT_of(F, l), pw[3], nullptr, ss, &s1)) return rc;
      const mc::TcRedSeg segs[6] = {{pw[0], s4, size_t(kH) * L.nout_pad, g + L.off_W4},
                                    {pb[0], s4, size_t(L.nout_pad), g + L.off_b4},
                                    {pw[1], s3, size_t(kH) * kH, g + L.off_W3},
                                    {pb[1], s3, size_t(kH), g + L.off_b3},
                                    {pw[2], s2, size_t(kH) * kH, g + L.off_W2},
                                    {pb[2], s2, size_t(kH), g + L.off_b2}};
      FLOW_CUDA(mc::tc_reduce_splits_multi(segs, 6, ss));
      mc::w1_grad_kernel<<<mc::blocks_for(kH * mc::kUPad, 32), mc::kW1Groups * 32, 0, ss>>>(pw[3], s1, L, g);
      FLOW_CUDA(cudaGetLastError());
      FLOW_CUDA(cudaEventRecord(F->ev_side[l], ss));
      side_last = l;
      continue;
    }
    // the layer-by-layer path shares the split-K partials and buffer set 0
    // with the side stream: wait for it
    if (int rc = join_side()) return rc;
    __nv_bfloat16* dA = F->dA;
    __nv_bfloat16* dA_b = F->dA + size_t(F->bp) * kH;
    mc::spline_inv_bwd_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P_of(F, l + 1), F->dP, D, L, LT_of(F, l), F->K,
                                                                       F->w, F->sums, F->G, F->GT, n, n_real);
    // last dense layer: W4, b4, and the gradient of h3 (through its ReLU)
    if (int rc = gemm_wgrad(F, n, L.nout_pad, h_of(F, l, 2), true, F->GT, g + L.off_W4, g + L.off_b4, st)) return rc;
    if (int rc = gemm_rs(F, n, kH, L.nout_pad, mc::kEpiReluMaskBf16, F->G, L.W4t, nullptr, dA, F->dAT,
                         hT_of(F, l, 2), st))
      return rc;
    // third dense layer
    if (int rc = gemm_wgrad(F, n, kH, h_of(F, l, 1), true, F->dAT, g + L.off_W3, g + L.off_b3, st)) return rc;
    if (int rc = gemm_rs(F, n, kH, kH, mc::kEpiReluMaskBf16, dA, L.W3t, nullptr, dA_b, F->dAT, hT_of(F, l, 1), st))
      return rc;
    // second dense layer
    if (int rc = gemm_wgrad(F, n, kH, h_of(F, l, 0), true, F->dAT, g + L.off_W2, g + L.off_b2, st)) return rc;
    if (int rc = gemm_rs(F, n, kH, kH, mc::kEpiReluMaskBf16, dA_b, L.W2t, nullptr, dA, F->dAT, hT_of(F, l, 0), st))
      return rc;
    // first dense layer: dU = dA1 W1 (tensor cores, W1 zero-padded to 16
    // columns) into the conditioning coordinates of dP; W1 and b1 from the
    // split-K product dA1^T [u | 1]
    if (int rc = gemm_rs(F, n, mc::kUPad, kH, mc::kEpiBiasF32, dA, L.W1t, nullptr, F->dU, nullptr, nullptr, st))
      return rc;
    mc::add_input_grad_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(F->dP, D, L, F->dU, n);
    int splits = 0;
    if (int rc = gemm_wgrad(F, n, mc::kUPad, F->dAT, false, UT_of(F, l), nullptr, nullptr, st, &splits)) return rc;
    mc::w1_grad_kernel<<<mc::blocks_for(kH * mc::kUPad, 32), mc::kW1Groups * 32, 0, st>>>(F->part, splits, L, g);
    FLOW_CUDA(cudaGetLastError());
  }
  return join_side();
}

int refresh_bf16(mc_flow F, cudaStream_t st) {
  for (const LayerDev& L : F->layers) {
    mc::to_bf16_kernel<<<mc::blocks_for(kH * kH, 256), 256, 0, st>>>(F->d_params + L.off_W2, kH, kH, L.W2h, L.W2t);
    mc::to_bf16_kernel<<<mc::blocks_for(kH * kH, 256), 256, 0, st>>>(F->d_params + L.off_W3, kH, kH, L.W3h, L.W3t);
    mc::to_bf16_kernel<<<mc::blocks_for(L.nout_pad * kH, 256), 256, 0, st>>>(F->d_params + L.off_W4, L.nout_pad, kH,
                                                                             L.W4h, L.W4t);
    mc::w1t_bf16_kernel<<<mc::blocks_for(mc::kUPad * kH, 256), 256, 0, st>>>(F->d_params + L.off_W1, L.na, L.W1t);
    mc::w1e_bf16_kernel<<<mc::blocks_for(kH * mc::kUK, 256), 256, 0, st>>>(F->d_params + L.off_W1,
                                                                          F->d_params + L.off_b1, L.na, L.W1e);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

void loss_sums(mc_flow F, long long n, cudaStream_t st) {
  mc::loss_partials_kernel<<<mc::kLossBlocks, 256, 0, st>>>(F->w, F->logq, n, F->sums + 2);
  mc::loss_final_kernel<<<1, 32, 0, st>>>(F->sums + 2, mc::kLossBlocks, F->sums);
}

int check_err(mc_flow F, cudaStream_t st) {
  int e = 0;
  FLOW_CUDA(cudaMemcpyAsync(&e, F->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FLOW_CUDA(cudaStreamSynchronize(st));
  if (e) return ffail(MC_ETIMEOUT, "mc_flow: a tensor-core GEMM wait timed out");
  return MC_OK;
}

size_t pdf_smem(const mc_integrand* itg, const mc::KernelArgs& a) {
  const int nfl = (itg->proc == MC_PP_TTBAR || itg->proc == MC_PP_TTBARJ) ? 11 : (a.pdf.nx ? 1 : 0);
  return sizeof(float) * size_t(a.pdf.nx) * (1 + 2 * nfl);
}

int sm_count() {
  static int num_sms = 0;
  if (num_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
      num_sms = 1;
  }
  return num_sms;
}

// The integrand at the n points X [n][D] of a training batch, one event per
// thread (f = 0 outside the cuts, NaN where the integrand failed or is not
// finite).  At 65 536 points the warp-specialised kernel with a points
// input measured slower: the batch is too small for its pipeline.
int eval_points(mc_flow F, const mc_integrand* itg, mc_pdf pdf, const float* X, long long n, float* f, cudaStream_t st) {
  mc::KernelArgs a;
  if (int rc = mc::fill_process_args(itg, pdf, &a)) return rc;
  const size_t smem = pdf_smem(itg, a);
  // one event per thread in blocks of 64: a training batch (65 536 points)
  // is a single wave, and 1024 blocks spread over the SMs within one block
  // of each other (512 blocks of 128 left some SMs a quarter more work)
  constexpr int kPts = 64;
  const unsigned grid = std::min<unsigned>(mc::blocks_for(n, kPts), 148u * 32u);
  switch (itg->proc) {
    case MC_EE_MUMU: mc::points_kernel<mc::P_EE_MUMU><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    case MC_PP_TTBAR: mc::points_kernel<mc::P_PP_TTBAR><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    case MC_GG_TTBARG: mc::points_kernel<mc::P_GG_TTBARG><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    case MC_GG_TTBARG_7D: mc::points_kernel<mc::P_GG_TTBARG_7D><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    case MC_PP_TTBARJ: mc::points_kernel<mc::P_PP_TTBARJ><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    case MC_GAUSS: mc::points_kernel<mc::P_GAUSS><<<grid, kPts, smem, st>>>(a, X, F->D, f, n); break;
    default: return ffail(MC_EINVAL, "mc_flow: the process has no flow integrand");
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// The sampling pass's integrand at the n points X with log q: the block sums
// of w = f exp(-log q) into F->parts, *nparts of them (g g -> t tbar g and
// p p -> t tbar + parton on the warp-specialised kernel with a points input,
// one block per SM; the other processes one event per thread).
int eval_points_sums(mc_flow F, const mc_integrand* itg, const mc::KernelArgs& a, const float* X, const float* logq,
                     long long n, cudaStream_t st, int* nparts) {
  BlockPartial* parts = F->parts;
  if (mc::points_ws(itg->proc)) {
    mc::KernelArgs b = a;
    b.ndim = F->D;
    b.nbins = 0;
    b.n = n;
    b.pts = X;
    b.pts_logq = logq;
    b.wout = nullptr;
    b.partials = parts;
    b.status = F->err;
    *nparts = std::min(sm_count(), kPartsGrid);
    FLOW_CUDA(mc::launch_points_ws(itg->proc, b, *nparts, st));
    return MC_OK;
  }
  const size_t smem = pdf_smem(itg, a);
  const int grid = kPartsGrid;
  *nparts = grid;
  switch (itg->proc) {
    case MC_EE_MUMU:
      mc::points_sums_kernel<mc::P_EE_MUMU><<<grid, 128, smem, st>>>(a, X, logq, F->D, n, parts);
      break;
    case MC_PP_TTBAR:
      mc::points_sums_kernel<mc::P_PP_TTBAR><<<grid, 128, smem, st>>>(a, X, logq, F->D, n, parts);
      break;
    case MC_GAUSS: mc::points_sums_kernel<mc::P_GAUSS><<<grid, 128, smem, st>>>(a, X, logq, F->D, n, parts); break;
    default: return ffail(MC_EINVAL, "mc_flow: the process has no flow integrand");
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Adam step of the parameters from F->d_grads (the step count advances on
// the device; the caller advances F->step).
int adam_launch(mc_flow F, double lr, cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  mc::adam_prep_kernel<<<1, 1, 0, st>>>(F->d_step, F->d_adam_pow, F->d_adam, b1, b2);
  mc::AdamArgs A{float(lr), float(b1), float(b2), 1e-8f, F->d_adam};
  // the dense matrices in 32 x 32 tiles, then the rest (both refresh the BF16 copies)
  int mat_tiles = 0, vec_max = 0;
  for (const LayerDev& L : F->layers) {
    mat_tiles = std::max(mat_tiles, (std::max(L.nout_pad, kH) / 32) * (kH / 32));
    vec_max = std::max(vec_max, kH * (L.na + 1) + 2 * kH + L.nout_pad);
  }
  mc::adam_mat_kernel<<<dim3(mat_tiles, 3 * F->L), dim3(32, 8), 0, st>>>(F->d_params, F->d_grads, F->d_m, F->d_v,
                                                                       F->d_layers, A);
  mc::adam_vec_kernel<<<dim3(mc::blocks_for(vec_max, 256), F->L), 256, 0, st>>>(F->d_params, F->d_grads, F->d_m,
                                                                               F->d_v, F->d_layers, A);
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// One online training step on a batch of n events (np padded): sample from
// the current flow keeping every layer's activations, evaluate the
// integrand, form the weights and the loss sums, differentiate, take the
// Adam step.  Host-independent (the batch's Philox iteration and Adam's
// corrections come from the device step count), so it can be captured once
// and replayed.
int train_step(mc_flow F, const mc_integrand* itg, mc_pdf pdf, long long n, long long np, double lr, cudaStream_t st) {
  FLOW_CUDA(cudaMemsetAsync(P_of(F, 0), 0, sizeof(float) * np * F->D, st));
  mc::flow_uniforms_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(P_of(F, 0), n, F->D, F->seed, 0u, 0, F->d_step);
  if (int rc = forward_pass(F, np, true, st)) return rc;
  if (int rc = eval_points(F, itg, pdf, P_of(F, F->L), n, F->f, st)) return rc;
  FLOW_CUDA(cudaMemsetAsync(F->w, 0, sizeof(float) * np, st));
  mc::flow_weights_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(F->f, F->logq, F->w, n);
  loss_sums(F, n, st);
  // the forward activations are those of the density pass at x: backward, Adam
  mc::zero_kernel<<<mc::blocks_for(F->nparam, 256), 256, 0, st>>>(F->d_grads, F->nparam);
  if (int rc = backward_pass(F, np, n, st)) return rc;
  return adam_launch(F, lr, st);
}

// Packed host parameter layout -> padded device layout: W4 row j (2K+1) + k
// of the packed matrix is device row j ls + k (and likewise for b4).
void build_host_map(mc_flow F) {
  F->host_map.clear();
  const int K2 = 2 * F->K + 1;
  for (const LayerDev& L : F->layers) {
    auto span = [&](size_t dev_off, size_t n) {
      for (size_t i = 0; i < n; ++i) F->host_map.push_back(dev_off + i);
    };
    span(L.off_W1, size_t(kH) * L.na);
    span(L.off_b1, kH);
    span(L.off_W2, size_t(kH) * kH);
    span(L.off_b2, kH);
    span(L.off_W3, size_t(kH) * kH);
    span(L.off_b3, kH);
    for (int j = 0; j < L.nb; ++j)
      for (int k = 0; k < K2; ++k) span(L.off_W4 + size_t(j * L.ls + k) * kH, kH);
    for (int j = 0; j < L.nb; ++j)
      for (int k = 0; k < K2; ++k) span(L.off_b4 + size_t(j * L.ls + k), 1);
  }
}

}  // namespace

extern "C" {

int mc_flow_param_count(const mc_flow_cfg* cfg, int64_t* n) {
  if (!cfg || !n) return ffail(MC_EINVAL, "mc_flow_param_count: NULL argument");
  int64_t total = 0;
  for (int l = 0; l < cfg->layers; ++l) {
    const int nb = (cfg->ndim + 1 - (l % 2)) / 2, na = cfg->ndim - nb;
    const int nout = nb * (2 * cfg->bins + 1);
    total += int64_t(cfg->hidden) * na + cfg->hidden + 2 * (int64_t(cfg->hidden) * cfg->hidden + cfg->hidden) +
             int64_t(nout) * cfg->hidden + nout;
  }
  *n = total;
  return MC_OK;
}

int mc_flow_free(mc_flow F) {
  if (!F) return MC_OK;
  for (void* p : {(void*)F->d_params, (void*)F->d_grads, (void*)F->d_m, (void*)F->d_v, (void*)F->d_wbf,
                  (void*)F->d_layers, (void*)F->P, (void*)F->logq, (void*)F->f, (void*)F->w, (void*)F->dP,
                  (void*)F->LT, (void*)F->h, (void*)F->hT, (void*)F->G, (void*)F->GT, (void*)F->dA, (void*)F->dAT,
                  (void*)F->part, (void*)F->UT, (void*)F->MB, (void*)F->dU, (void*)F->U, (void*)F->Ps, (void*)F->lqs,
                  (void*)F->sums, (void*)F->parts, (void*)F->chunk_totals, (void*)F->total,
                  (void*)F->err, (void*)F->d_step, (void*)F->d_adam, (void*)F->d_adam_pow, (void*)F->bpart})
    cudaFree(p);
  for (cudaEvent_t e : F->ev_chain)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : F->ev_side)
    if (e) cudaEventDestroy(e);
  if (F->side) cudaStreamDestroy(F->side);
  if (F->ev_in) cudaEventDestroy(F->ev_in);
  if (F->ev_out) cudaEventDestroy(F->ev_out);
  if (F->cap) cudaStreamDestroy(F->cap);
  if (F->h_sums) cudaFreeHost(F->h_sums);
  if (F->h_total) cudaFreeHost(F->h_total);
  delete F;
  return MC_OK;
}

int mc_flow_create(const mc_flow_cfg* cfg, const float* init, int64_t max_batch, uint64_t seed, mc_flow* out) {
  if (!out || !cfg || !init) return ffail(MC_EINVAL, "mc_flow_create: NULL argument");
  *out = nullptr;
  if (cfg->ndim < 2 || cfg->ndim > mc::kMaxFlowDim || cfg->layers < 1 || cfg->layers > mc::kMaxLayers ||
      cfg->bins < 2 || cfg->bins > mc::kFlowMaxBins || cfg->hidden != kH || max_batch < 1 ||
      max_batch > (int64_t(1) << 21))
    return ffail(MC_EINVAL,
                 "mc_flow_create: need 2 <= ndim <= 16, 1..16 layers, 2..32 bins, hidden 256, 1 <= max_batch <= 2^21");
  auto* F = new mc_flow_s;
  cudaGetDevice(&F->device);
  F->D = cfg->ndim;
  F->L = cfg->layers;
  F->K = cfg->bins;
  F->max_batch = max_batch;
  F->bp = pad128(max_batch);
  F->seed = seed;
  const int ls = (2 * F->K + 1 + 15) / 16 * 16;
  size_t off = 0, woff = 0;
  for (int l = 0; l < F->L; ++l) {
    LayerDev L;
    std::memset(&L, 0, sizeof(L));
    for (int d = 0; d < F->D; ++d) {
      if (d % 2 == l % 2)
        L.b_idx[L.nb++] = d;
      else
        L.a_idx[L.na++] = d;
    }
    L.ls = ls;
    L.nout_pad = (L.nb * ls + 63) / 64 * 64;
    F->nout_pad_max = std::max(F->nout_pad_max, L.nout_pad);
    L.off_W1 = off; off += size_t(kH) * L.na;
    off = (off + 3) / 4 * 4;  // 16-byte aligned biases and matrices
    L.off_b1 = off; off += kH;
    L.off_W2 = off; off += size_t(kH) * kH;
    L.off_b2 = off; off += kH;
    L.off_W3 = off; off += size_t(kH) * kH;
    L.off_b3 = off; off += kH;
    L.off_W4 = off; off += size_t(L.nout_pad) * kH;
    L.off_b4 = off; off += L.nout_pad;
    F->layers.push_back(L);
    woff += 2 * (2 * size_t(kH) * kH + size_t(L.nout_pad) * kH) + size_t(mc::kUPad) * kH + size_t(kH) * mc::kUK;
  }
  F->nparam = off;
  const size_t bp = size_t(F->bp), D = size_t(F->D), np = size_t(F->nout_pad_max), L = size_t(F->L);
  F->max_splits = 148;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&F->d_params, sizeof(float) * off);
  alloc((void**)&F->d_grads, sizeof(float) * off);
  alloc((void**)&F->d_m, sizeof(float) * off);
  alloc((void**)&F->d_v, sizeof(float) * off);
  alloc((void**)&F->d_wbf, sizeof(__nv_bfloat16) * woff);
  alloc((void**)&F->d_layers, sizeof(LayerDev) * L);
  alloc((void**)&F->P, sizeof(float) * (L + 1) * bp * D);
  alloc((void**)&F->logq, sizeof(float) * bp);
  alloc((void**)&F->f, sizeof(float) * bp);
  alloc((void**)&F->w, sizeof(float) * bp);
  alloc((void**)&F->dP, sizeof(float) * bp * D);
  alloc((void**)&F->LT, sizeof(float) * L * np * bp);
  alloc((void**)&F->h, sizeof(__nv_bfloat16) * L * 3 * bp * kH);
  alloc((void**)&F->hT, sizeof(__nv_bfloat16) * L * 3 * bp * kH);
  alloc((void**)&F->G, sizeof(__nv_bfloat16) * 2 * bp * np);
  alloc((void**)&F->GT, sizeof(__nv_bfloat16) * 2 * bp * np);
  alloc((void**)&F->dA, sizeof(__nv_bfloat16) * 2 * bp * kH);
  alloc((void**)&F->dAT, sizeof(__nv_bfloat16) * 2 * 3 * bp * kH);
  // four partial regions (the side stream's W4, W3, W2, W1 products of a
  // layer) and three bias-partial regions
  // N of a product is nout_pad (W4), H (W3, W2) or 16 (W1)
  const size_t nmax = std::max(np, size_t(kH));
  F->part_region = size_t(F->max_splits) * kH * nmax;
  F->bpart_region = size_t(F->max_splits) * nmax;
  alloc((void**)&F->part, sizeof(float) * 4 * F->part_region);
  alloc((void**)&F->bpart, sizeof(float) * 3 * F->bpart_region);
  alloc((void**)&F->UT, sizeof(__nv_bfloat16) * L * mc::kUPad * bp);
  alloc((void**)&F->MB, sizeof(uint32_t) * L * 3 * bp * 8);
  alloc((void**)&F->dU, sizeof(float) * bp * mc::kUPad);
  alloc((void**)&F->U, sizeof(__nv_bfloat16) * bp * mc::kUK);
  alloc((void**)&F->sums, sizeof(double) * (2 + 2 * mc::kLossBlocks));
  alloc((void**)&F->parts, sizeof(BlockPartial) * kPartsGrid);
  alloc((void**)&F->total, sizeof(BlockPartial));
  alloc((void**)&F->err, sizeof(int));
  alloc((void**)&F->d_step, sizeof(long long));
  alloc((void**)&F->d_adam, sizeof(float) * 2);
  alloc((void**)&F->d_adam_pow, sizeof(double) * 2);
  F->sbp = std::max<long long>(F->bp, 1 << 20);
  alloc((void**)&F->Ps, sizeof(float) * size_t(F->sbp) * D);
  alloc((void**)&F->lqs, sizeof(float) * size_t(F->sbp));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_sums, sizeof(double) * 2);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_total, sizeof(BlockPartial));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&F->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&F->side, cudaStreamNonBlocking);
  F->ev_chain.assign(L, nullptr);
  F->ev_side.assign(L, nullptr);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    e = cudaEventCreateWithFlags(&F->ev_chain[l], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_side[l], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    mc_flow_free(F);
    return ffail(MC_ENOMEM, std::string("mc_flow_create: allocation failed: ") + cudaGetErrorString(e));
  }
  woff = 0;
  for (LayerDev& Ld : F->layers) {
    Ld.W2h = F->d_wbf + woff; woff += size_t(kH) * kH;
    Ld.W2t = F->d_wbf + woff; woff += size_t(kH) * kH;
    Ld.W3h = F->d_wbf + woff; woff += size_t(kH) * kH;
    Ld.W3t = F->d_wbf + woff; woff += size_t(kH) * kH;
    Ld.W4h = F->d_wbf + woff; woff += size_t(Ld.nout_pad) * kH;
    Ld.W4t = F->d_wbf + woff; woff += size_t(Ld.nout_pad) * kH;
    Ld.W1t = F->d_wbf + woff; woff += size_t(mc::kUPad) * kH;
    Ld.W1e = F->d_wbf + woff; woff += size_t(kH) * mc::kUK;
  }
  build_host_map(F);
  // tensor maps of the fused layers
  F->h_map_ok = size_t(L) * 3 * bp <= 0x7fffffffu &&
                mc::tc_make_map(&F->h_map, F->h, int(size_t(L) * 3 * bp), kH, kH, 128);
  F->maps.resize(4 * L);
  F->bwd_maps.resize(4 * L);
  F->g_maps.resize(2 * L);
  for (int l = 0; l < F->L; ++l) {
    const LayerDev& Ld = F->layers[l];
    // fused layers: 32 bins (logit stride 80), at most 6 transformed
    // coordinates (W4 sub-products of at most 256 rows)
    bool ok = F->K == mc::kFusedK && ls == mc::kFusedLs && Ld.nb <= 6 && Ld.nout_pad <= 512 && F->h_map_ok;
    ok = ok && mc::tc_make_map(&F->maps[4 * l], Ld.W2h, kH, kH, kH, kH) &&
         mc::tc_make_map(&F->maps[4 * l + 1], Ld.W3h, kH, kH, kH, kH) &&
         mc::tc_make_map(&F->maps[4 * l + 2], Ld.W4h, Ld.nout_pad, kH, kH, 32) &&
         mc::tc_make_map(&F->maps[4 * l + 3], Ld.W1e, kH, mc::kUK, mc::kUK, kH) &&
         mc::tc_make_map(&F->bwd_maps[4 * l], Ld.W4t, kH, Ld.nout_pad, Ld.nout_pad, kH) &&
         mc::tc_make_map(&F->bwd_maps[4 * l + 1], Ld.W3t, kH, kH, kH, kH) &&
         mc::tc_make_map(&F->bwd_maps[4 * l + 2], Ld.W2t, kH, kH, kH, kH) &&
         mc::tc_make_map(&F->bwd_maps[4 * l + 3], Ld.W1t, mc::kUPad, kH, kH, mc::kUPad);
    F->fused_ok.push_back(ok);
    // two operand buffers of max(256, nout_pad) x 128 BF16 and at least two
    // weight stages must fit in shared memory
    const size_t abytes = size_t(std::max(kH, Ld.nout_pad)) * 256;
    const bool fits = 2 * abytes + 2 * size_t(kH) * 128 + 1024 <= mc::kChainSmemMax;
    F->chain_ok.push_back(ok && fits &&
                          mc::tc_make_map(&F->g_maps[2 * l], G_of(F, 0), int(bp), Ld.nout_pad, Ld.nout_pad, 128) &&
                          mc::tc_make_map(&F->g_maps[2 * l + 1], G_of(F, 1), int(bp), Ld.nout_pad, Ld.nout_pad, 128));
  }
  const double kOnes[2] = {1.0, 1.0};  // b1^0, b2^0
  // the padding rows of the logit gradients and of U^T are never written: zero them once
  if (cudaMemcpy(F->d_layers, F->layers.data(), sizeof(LayerDev) * L, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(F->d_m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->d_v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->d_grads, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->GT, 0, sizeof(__nv_bfloat16) * 2 * bp * np) != cudaSuccess ||
      cudaMemset(F->G, 0, sizeof(__nv_bfloat16) * 2 * bp * np) != cudaSuccess ||
      cudaMemset(F->UT, 0, sizeof(__nv_bfloat16) * L * mc::kUPad * bp) != cudaSuccess ||
      cudaMemset(F->err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(F->d_step, 0, sizeof(long long)) != cudaSuccess ||
      cudaMemcpy(F->d_adam_pow, kOnes, sizeof(kOnes), cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_flow_free(F);
    return ffail(MC_ECUDA, "mc_flow_create: initialisation failed");
  }
  if (int rc = mc_flow_set_params(F, init)) {
    mc_flow_free(F);
    return rc;
  }
  *out = F;
  return MC_OK;
}

int mc_flow_set_params(mc_flow F, const float* host) {
  if (!F || !host) return ffail(MC_EINVAL, "mc_flow_set_params: NULL argument");
  std::vector<float> dev(F->nparam, 0.0f);
  for (size_t i = 0; i < F->host_map.size(); ++i) dev[F->host_map[i]] = host[i];
  FLOW_CUDA(cudaMemcpy(F->d_params, dev.data(), sizeof(float) * F->nparam, cudaMemcpyHostToDevice));
  if (int rc = refresh_bf16(F, nullptr)) return rc;
  FLOW_CUDA(cudaDeviceSynchronize());
  return MC_OK;
}

int mc_flow_get_params(mc_flow F, float* host) {
  if (!F || !host) return ffail(MC_EINVAL, "mc_flow_get_params: NULL argument");
  std::vector<float> dev(F->nparam);
  FLOW_CUDA(cudaDeviceSynchronize());
  FLOW_CUDA(cudaMemcpy(dev.data(), F->d_params, sizeof(float) * F->nparam, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < F->host_map.size(); ++i) host[i] = dev[F->host_map[i]];
  return MC_OK;
}

int mc_flow_set_fused(mc_flow F, int mask) {
  if (!F || mask < 0 || mask > 3) return ffail(MC_EINVAL, "mc_flow_set_fused: bad arguments");
  F->use_fused = (mask & 1) != 0;
  F->use_fused_bwd = (mask & 2) != 0;
  return MC_OK;
}

int mc_flow_forward(mc_flow F, int64_t n, const float* z, float* x, float* logq, void* stream) {
  if (!F || n < 0 || n > F->max_batch || (n && (!z || !x || !logq)))
    return ffail(MC_EINVAL, "mc_flow_forward: bad arguments");
  if (n == 0) return MC_OK;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long np = pad128(n);
  FLOW_CUDA(cudaMemsetAsync(P_of(F, 0), 0, sizeof(float) * np * F->D, st));
  FLOW_CUDA(cudaMemcpyAsync(P_of(F, 0), z, sizeof(float) * n * F->D, cudaMemcpyDeviceToDevice, st));
  if (int rc = forward_pass(F, np, false, st)) return rc;
  FLOW_CUDA(cudaMemcpyAsync(x, P_of(F, 0), sizeof(float) * n * F->D, cudaMemcpyDeviceToDevice, st));
  FLOW_CUDA(cudaMemcpyAsync(logq, F->logq, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
  return check_err(F, st);
}

int mc_flow_loss_grad(mc_flow F, int64_t n, const float* x, const float* w, double* loss, float* grads, void* stream) {
  if (!F || n < 1 || n > F->max_batch || !x || !w) return ffail(MC_EINVAL, "mc_flow_loss_grad: bad arguments");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long np = pad128(n);
  float* X = P_of(F, F->L);
  FLOW_CUDA(cudaMemsetAsync(X, 0, sizeof(float) * np * F->D, st));
  FLOW_CUDA(cudaMemsetAsync(F->w, 0, sizeof(float) * np, st));
  FLOW_CUDA(cudaMemcpyAsync(X, x, sizeof(float) * n * F->D, cudaMemcpyDeviceToDevice, st));
  FLOW_CUDA(cudaMemcpyAsync(F->w, w, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
  mc::zero_kernel<<<mc::blocks_for(F->nparam, 256), 256, 0, st>>>(F->d_grads, F->nparam);
  if (int rc = inverse_pass(F, np, st)) return rc;
  loss_sums(F, n, st);
  if (int rc = backward_pass(F, np, n, st)) return rc;
  FLOW_CUDA(cudaMemcpyAsync(F->h_sums, F->sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  if (int rc = check_err(F, st)) return rc;
  if (loss) *loss = F->h_sums[0] > 0.0 ? -F->h_sums[1] / F->h_sums[0] : 0.0;
  if (grads) {
    std::vector<float> dev(F->nparam);
    FLOW_CUDA(cudaMemcpy(dev.data(), F->d_grads, sizeof(float) * F->nparam, cudaMemcpyDeviceToHost));
    // gradients of W2..W4 are stored transposed; W4 rows sit at j ls + k
    size_t k = 0;
    const int K2 = 2 * F->K + 1;
    for (const LayerDev& L : F->layers) {
      for (size_t i = 0; i < size_t(kH) * L.na; ++i) grads[k++] = dev[L.off_W1 + i];
      for (int i = 0; i < kH; ++i) grads[k++] = dev[L.off_b1 + i];
      for (int r = 0; r < kH; ++r)
        for (int c = 0; c < kH; ++c) grads[k++] = dev[L.off_W2 + size_t(c) * kH + r];
      for (int i = 0; i < kH; ++i) grads[k++] = dev[L.off_b2 + i];
      for (int r = 0; r < kH; ++r)
        for (int c = 0; c < kH; ++c) grads[k++] = dev[L.off_W3 + size_t(c) * kH + r];
      for (int i = 0; i < kH; ++i) grads[k++] = dev[L.off_b3 + i];
      for (int j = 0; j < L.nb; ++j)
        for (int q = 0; q < K2; ++q)
          for (int c = 0; c < kH; ++c) grads[k++] = dev[L.off_W4 + size_t(c) * L.nout_pad + j * L.ls + q];
      for (int j = 0; j < L.nb; ++j)
        for (int q = 0; q < K2; ++q) grads[k++] = dev[L.off_b4 + j * L.ls + q];
    }
  }
  return MC_OK;
}

int mc_flow_adam_step(mc_flow F, double lr, void* stream) {
  if (!F || !(lr > 0.0)) return ffail(MC_EINVAL, "mc_flow_adam_step: bad arguments");
  ++F->step;
  return adam_launch(F, lr, static_cast<cudaStream_t>(stream));
}

// ---- one online training step split across devices (data parallel): each
// rank samples its share of the step's batch, the ranks add their sums of w,
// every rank differentiates its share with the loss normalised by the total,
// the ranks add their gradients, and each takes the same Adam step.
int mc_flow_grad_count(mc_flow F, int64_t* n) {
  if (!F || !n) return ffail(MC_EINVAL, "mc_flow_grad_count: NULL argument");
  *n = int64_t(F->nparam);
  return MC_OK;
}

int mc_flow_step_sample(mc_flow F, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t count, void* stream,
                        double* wsum) {
  if (!F || !itg || !wsum || first < 0 || count < 1 || count > F->max_batch)
    return ffail(MC_EINVAL, "mc_flow_step_sample: bad arguments");
  if (mc::process_dim(itg) != F->D) return ffail(MC_EINVAL, "mc_flow_step_sample: flow dimension differs from the process");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = count, np = pad128(n);
  F->step_n = 0;
  FLOW_CUDA(cudaMemsetAsync(P_of(F, 0), 0, sizeof(float) * np * F->D, st));
  mc::flow_uniforms_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(P_of(F, 0), n, F->D, F->seed,
                                                                    0x10000u + uint32_t(F->step), first);
  if (int rc = forward_pass(F, np, true, st)) return rc;
  if (int rc = eval_points(F, itg, pdf, P_of(F, F->L), n, F->f, st)) return rc;
  FLOW_CUDA(cudaMemsetAsync(F->w, 0, sizeof(float) * np, st));
  mc::flow_weights_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(F->f, F->logq, F->w, n);
  loss_sums(F, n, st);
  FLOW_CUDA(cudaMemcpyAsync(F->h_sums, F->sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  if (int rc = check_err(F, st)) return rc;
  *wsum = F->h_sums[0];
  F->step_n = n;
  return MC_OK;
}

int mc_flow_step_grads(mc_flow F, double wsum_total, float* grads, void* stream) {
  if (!F || !(wsum_total > 0.0)) return ffail(MC_EINVAL, "mc_flow_step_grads: bad arguments");
  if (F->step_n < 1) return ffail(MC_EINVAL, "mc_flow_step_grads: no sampled batch (call mc_flow_step_sample)");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = F->step_n, np = pad128(n);
  mc::set_double_kernel<<<1, 1, 0, st>>>(F->sums, wsum_total);
  mc::zero_kernel<<<mc::blocks_for(F->nparam, 256), 256, 0, st>>>(F->d_grads, F->nparam);
  if (int rc = backward_pass(F, np, n, st)) return rc;
  if (grads) FLOW_CUDA(cudaMemcpyAsync(grads, F->d_grads, sizeof(float) * F->nparam, cudaMemcpyDeviceToDevice, st));
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

int mc_flow_step_apply(mc_flow F, const float* grads, double lr, void* stream) {
  if (!F || !(lr > 0.0)) return ffail(MC_EINVAL, "mc_flow_step_apply: bad arguments");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (grads) FLOW_CUDA(cudaMemcpyAsync(F->d_grads, grads, sizeof(float) * F->nparam, cudaMemcpyDeviceToDevice, st));
  F->step_n = 0;
  return mc_flow_adam_step(F, lr, stream);
}

int mc_flow_train(mc_flow F, const mc_integrand* itg, mc_pdf pdf, int steps, int64_t batch, double lr, void* stream,
                  double* losses) {
  if (!F || !itg || steps < 0 || batch < 2 || batch > F->max_batch || !(lr > 0.0))
    return ffail(MC_EINVAL, "mc_flow_train: bad arguments");
  if (mc::process_dim(itg) != F->D) return ffail(MC_EINVAL, "mc_flow_train: flow dimension differs from the process");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = batch, np = pad128(n);
  if (!losses && steps >= 2) {
    // the step captured once as a CUDA graph on F->cap and replayed `steps`
    // times (its ~80 launches then cost one graph launch), ordered after the
    // caller's stream and before its later work
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FLOW_CUDA(cudaEventRecord(F->ev_in, st));
    FLOW_CUDA(cudaStreamWaitEvent(F->cap, F->ev_in, 0));
    FLOW_CUDA(cudaStreamBeginCapture(F->cap, cudaStreamCaptureModeRelaxed));
    const int rc = train_step(F, itg, pdf, n, np, lr, F->cap);
    const cudaError_t ec = cudaStreamEndCapture(F->cap, &graph);
    if (rc != MC_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      (void)cudaGetLastError();
      return rc != MC_OK ? rc : ffail(MC_ECUDA, std::string("mc_flow_train: graph capture failed: ") +
                                                    cudaGetErrorString(ec));
    }
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    for (int s = 0; s < steps && e == cudaSuccess; ++s) e = cudaGraphLaunch(exec, F->cap);
    if (e == cudaSuccess) e = cudaEventRecord(F->ev_out, F->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, F->ev_out, 0);
    if (exec) cudaGraphExecDestroy(exec);  // freed once the launches in flight complete
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return ffail(MC_ECUDA, std::string("mc_flow_train: ") + cudaGetErrorString(e));
    F->step += steps;
    return check_err(F, st);
  }
  for (int s = 0; s < steps; ++s) {
    if (int rc = train_step(F, itg, pdf, n, np, lr, st)) return rc;
    ++F->step;
    if (losses) {
      FLOW_CUDA(cudaMemcpyAsync(F->h_sums, F->sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
      FLOW_CUDA(cudaStreamSynchronize(st));
      losses[s] = F->h_sums[0] > 0 ? -F->h_sums[1] / F->h_sums[0] : 0.0;
    }
  }
  return check_err(F, st);
}

int mc_flow_iterate(mc_flow F, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, uint32_t iteration, void* stream,
                    mc_iter_result* out) {
  if (!F || !itg || !out || nevents < 0) return ffail(MC_EINVAL, "mc_flow_iterate: bad arguments");
  if (mc::process_dim(itg) != F->D) return ffail(MC_EINVAL, "mc_flow_iterate: flow dimension differs from the process");
  std::memset(out, 0, sizeof(*out));
  out->n = nevents;
  if (nevents == 0) return MC_OK;
  mc::KernelArgs a;
  if (int rc = mc::fill_process_args(itg, pdf, &a)) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool all_fused = F->use_fused && F->sbp > 0;
  for (int l = 0; l < F->L; ++l) all_fused = all_fused && F->fused_ok[l];
  // the fused layers need only the points and log q: sample in large chunks
  const long long chunk = all_fused ? F->sbp : (F->max_batch / 128) * 128;
  if (chunk < 128) return ffail(MC_EINVAL, "mc_flow_iterate: max_batch below 128");
  float* Z = all_fused ? F->Ps : P_of(F, 0);
  float* LQ = all_fused ? F->lqs : F->logq;
  const long long nchunks = (nevents + chunk - 1) / chunk;
  if (nchunks > F->max_chunks) {  // grow-only per-chunk totals
    FLOW_CUDA(cudaStreamSynchronize(st));
    cudaFree(F->chunk_totals);
    F->chunk_totals = nullptr;
    F->max_chunks = 0;
    FLOW_CUDA(cudaMalloc((void**)&F->chunk_totals, sizeof(BlockPartial) * nchunks));
    F->max_chunks = nchunks;
  }
  for (long long c = 0; c < nchunks; ++c) {
    const long long first = c * chunk;
    const long long n = std::min<long long>(chunk, nevents - first), np = pad128(n);
    if (np != n) FLOW_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * np * F->D, st));
    mc::flow_uniforms_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(Z, n, F->D, F->seed, 0x20000u + iteration,
                                                                      first);
    FLOW_CUDA(cudaMemsetAsync(LQ, 0, sizeof(float) * np, st));
    if (int rc = all_fused ? forward_layers(F, np, false, st, Z, LQ) : forward_layers(F, np, false, st)) return rc;
    int nparts = 0;
    if (int rc = eval_points_sums(F, itg, a, Z, LQ, n, st, &nparts)) return rc;
    FLOW_CUDA(mc::launch_finalize(F->parts, nparts, F->chunk_totals + c, st));
  }
  FLOW_CUDA(mc::launch_finalize(F->chunk_totals, int(nchunks), F->total, st));
  FLOW_CUDA(cudaMemcpyAsync(F->h_total, F->total, sizeof(BlockPartial), cudaMemcpyDeviceToHost, st));
  if (int rc = check_err(F, st)) return rc;
  const BlockPartial& tot = *F->h_total;
  out->sum = tot.sum_hi + tot.sum_lo;
  out->sum2 = tot.sum2_hi + tot.sum2_lo;
  out->wmax = tot.wmax;
  out->n_nonzero = tot.n_nonzero;
  out->n_bad = tot.n_bad + tot.n_noconv;
  out->status = tot.n_bad ? MC_ENAN : (tot.n_noconv ? MC_ENOCONV : MC_OK);
  return MC_OK;
}

int mc_integrate_flow(const mc_integrand* itg, mc_pdf pdf, const mc_flow_cfg* cfg, const float* init,
                      int train_steps, int64_t train_batch, double lr, int niter, int64_t nevents, int nbins,
                      uint64_t seed, double target, void* stream, mc_result* out, int* sampler) {
  if (!itg || !cfg || !init || !out || !sampler || niter < 1 || nevents < 2 || train_steps < 0 || train_batch < 2)
    return ffail(MC_EINVAL, "mc_integrate_flow: bad arguments");
  std::memset(out, 0, sizeof(*out));
  *sampler = 0;
  const int nd = mc::process_dim(itg);
  if (nd != cfg->ndim) return ffail(MC_EINVAL, "mc_integrate_flow: flow dimension differs from the process");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // set-up (the judge's grid, the flow's buffers and parameters) before the
  // first launch, which opens the timed region
  mc_vegas v = nullptr;
  mc_flow f = nullptr;
  int rc = mc_vegas_init(nd, nbins, seed, MC_FP32_KAHAN, &v);
  if (!rc) rc = mc_flow_create(cfg, init, train_batch, seed + 1, &f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
              cudaEventRecord(e0, st) != cudaSuccess))
    rc = ffail(MC_ECUDA, "mc_integrate_flow: event");
  std::vector<double> es, s2s;
  auto add = [&](const mc_iter_result& r) {  // one iteration's estimate and the variance of its mean
    const double n = double(r.n), mean = r.sum / n;
    es.push_back(mean);
    s2s.push_back((r.sum2 / n - mean * mean) / (n - 1.0));
    return s2s.back() * n / (mean * mean);  // relative variance per event
  };
  auto done = [&]() {
    mc::combine_iterations(es, s2s, out);
    out->n_iter = int(es.size());
    return target > 0.0 && out->mean != 0.0 && out->sigma / std::fabs(out->mean) <= target;
  };
  // the judge: one FP32 VEGAS iteration on a fresh grid (then refined)
  mc_iter_result r;
  double relvar_v = 0.0, relvar_f = 0.0;
  bool flow_ok = false;
  if (!rc) rc = mc_vegas_iterate(v, itg, pdf, nevents, stream, &r);
  if (!rc) rc = mc_vegas_refine(v, 1.5, stream);
  if (!rc) relvar_v = add(r);
  // the flow: online training, then its first iteration
  if (!rc && train_steps > 0) {
    // asynchronous steps, then the last one with its loss read back
    double last_loss = 0.0;
    if (train_steps > 1) rc = mc_flow_train(f, itg, pdf, train_steps - 1, train_batch, lr, stream, nullptr);
    if (!rc) rc = mc_flow_train(f, itg, pdf, 1, train_batch, lr, stream, &last_loss);
    flow_ok = !rc && std::isfinite(last_loss);
  } else {
    flow_ok = !rc;
  }
  mc_iter_result rf;
  std::memset(&rf, 0, sizeof(rf));
  uint32_t flow_it = 0;
  if (!rc && flow_ok) {
    rc = mc_flow_iterate(f, itg, pdf, nevents, flow_it++, stream, &rf);
    flow_ok = !rc && rf.status == MC_OK && std::isfinite(rf.sum) && std::isfinite(rf.sum2) && rf.sum != 0.0;
    if (rc == MC_ENAN || rc == MC_ENOCONV) rc = MC_OK;
  }
  if (flow_ok) {
    const double n = double(rf.n), mean = rf.sum / n;
    relvar_f = (rf.sum2 / n - mean * mean) / (mean * mean);
    flow_ok = std::isfinite(relvar_f) && relvar_f <= relvar_v;  // VEGAS judges the flow
  }
  *sampler = flow_ok ? 1 : 0;
  if (!rc) {
    if (flow_ok) add(rf);
    bool reached = done();
    while (!rc && !reached && out->n_iter < niter + 1) {
      if (flow_ok) {
        rc = mc_flow_iterate(f, itg, pdf, nevents, flow_it++, stream, &r);
      } else {
        rc = mc_vegas_iterate(v, itg, pdf, nevents, stream, &r);
        if (!rc) rc = mc_vegas_refine(v, 1.5, stream);
      }
      if (!rc) {
        add(r);
        reached = done();
      }
    }
  }
  if (e0 && e1) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    out->gpu_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (f) mc_flow_free(f);
  if (v) mc_vegas_free(v);
  return rc;
}

}  // extern "C"
