// Normalizing-flow importance sampler on the GPU (C ABI: mc_flow_* in
// include/mcint.h).
//
// Flow: L piecewise-quadratic coupling layers (flow_spline.cuh) over the unit
// cube; layer l transforms the coordinates d with d % 2 == l % 2 and
// conditions on the others through a dense network u = 2 x_A - 1 -> 256 ->
// 256 -> 256 -> d_B (2K + 1) with ReLU.  The first dense layer (K = d_A) runs
// on the CUDA cores in FP32; the three 256-wide layers run on the tcgen05
// tensor cores (tc_gemm.cu) with BF16 operands and FP32 accumulation.
//
// Sampling: Philox uniforms z -> flow forward -> x, log q(x) -> integrand at
// x -> weight w = f(x) / q(x) -> Kahan FP64 sums (thesis Sec. "Importance
// sampling", eq. mc_est_is).  Training (online, on events the method itself
// generates): sample a batch, evaluate f, weights w = |f| / q held fixed, then
// L = -sum w log q(x) / sum w through the inverse pass (x -> z) with its
// activations kept, backward through the splines and the dense layers (BF16
// tensor-core GEMMs for the activation gradients and, split-K over the batch,
// for the weight gradients), and one Adam step (thesis Sec. "Optimizers").
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "event.cuh"
#include "flow_spline.cuh"
#include "handles.h"
#include "tc_gemm.h"

namespace mc {
namespace {

constexpr int kMaxFlowDim = 16;
constexpr int kMaxLayers = 16;

struct LayerDev {
  int na, nb, nout, nout_pad;
  int a_idx[kMaxFlowDim], b_idx[kMaxFlowDim];
  // master parameters (FP32) and their gradients / Adam moments share one
  // layout: W1 [H x na], b1 [H], W2 [H x H], b2, W3 [H x H], b3,
  // W4 [nout_pad x H], b4 [nout_pad]; gradients of W2..W4 are kept transposed
  // (gW^T [in x out]) as the split-K GEMMs produce them.
  size_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, off_W4, off_b4;
  // BF16 copies for the GEMMs: W2, W3, W4 (row-major [out x in]) and their
  // transposes [in x out] for the backward activation products
  __nv_bfloat16 *W2h, *W3h, *W4h, *W2t, *W3t, *W4t;
};

// ------------------------------------------------------------------ kernels
__global__ void flow_uniforms_kernel(float* z, long long n, int D, uint64_t seed, uint32_t iteration, uint32_t gid,
                                     long long first) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k[kMaxFlowDim];
  event_uniforms<kMaxFlowDim, false>(seed, iteration, gid, uint64_t(first + i), D, k);
  for (int d = 0; d < D; ++d) z[i * D + d] = float(uint32_t(2 * k[d] + 1)) * 0x1p-24f;
}

// h1 = bf16(relu(W1 (2 x_A - 1) + b1)), one thread per (event, hidden unit).
__global__ void dense1_kernel(const float* P, int D, const LayerDev L, const float* params, __nv_bfloat16* h1, int H,
                              long long n) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * H) return;
  const long long i = idx / H;
  const int j = int(idx % H);
  const float* W1 = params + L.off_W1 + size_t(j) * L.na;
  float acc = params[L.off_b1 + j];
  for (int a = 0; a < L.na; ++a) acc += W1[a] * (2.0f * P[i * D + L.a_idx[a]] - 1.0f);
  h1[idx] = __float2bfloat16_rn(fmaxf(acc, 0.0f));
}

// Forward spline of one layer, in place on P; logq -= sum log c.
__global__ void spline_fwd_kernel(float* P, int D, const LayerDev L, const float* logits, int K, float* logq,
                                  long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  SplineCoef s;
  float ld = 0.0f;
  for (int j = 0; j < L.nb; ++j) {
    spline_coef(logits + i * L.nout_pad + j * (2 * K + 1), K, s);
    float lc;
    const int d = L.b_idx[j];
    P[i * D + d] = spline_fwd(s, K, P[i * D + d], &lc);
    ld += lc;
  }
  logq[i] -= ld;
}

// Inverse spline of one layer: Pout = Pin with the B coordinates inverted;
// logq -= sum log c.
__global__ void spline_inv_kernel(const float* Pin, float* Pout, int D, const LayerDev L, const float* logits, int K,
                                  float* logq, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < D; ++d) Pout[i * D + d] = Pin[i * D + d];
  SplineCoef s;
  float ld = 0.0f;
  for (int j = 0; j < L.nb; ++j) {
    spline_coef(logits + i * L.nout_pad + j * (2 * K + 1), K, s);
    float lc;
    const int d = L.b_idx[j];
    Pout[i * D + d] = spline_inv(s, K, Pin[i * D + d], &lc);
    ld += lc;
  }
  logq[i] -= ld;
}

// Backward of one inverse layer.  dP holds dL/d(layer output) on entry and
// dL/d(layer input) for the B coordinates on exit (the A coordinates receive
// the conditioner's contribution later); gl_i = dL/d(log q_i) = -w_i / sum w.
__global__ void spline_inv_bwd_kernel(const float* Pin, float* dP, int D, const LayerDev L, const float* logits, int K,
                                      const float* w, const double* wsum, float* glog32, __nv_bfloat16* glog16,
                                      long long n, long long n_real) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gl = i < n_real ? float(-double(w[i]) / *wsum) : 0.0f;
  SplineCoef s;
  float g[2 * kFlowMaxBins + 1];
  for (int j = 0; j < L.nb; ++j) {
    const int d = L.b_idx[j];
    const size_t row = size_t(i) * L.nout_pad + j * (2 * K + 1);
    if (i < n_real) {
      spline_coef(logits + row, K, s);
      dP[i * D + d] = spline_inv_bwd(s, K, Pin[i * D + d], dP[i * D + d], gl, g);
    } else {
      dP[i * D + d] = 0.0f;
      for (int k = 0; k < 2 * K + 1; ++k) g[k] = 0.0f;
    }
    for (int k = 0; k < 2 * K + 1; ++k) {
      glog32[row + k] = g[k];
      glog16[row + k] = __float2bfloat16_rn(g[k]);
    }
  }
  for (int c = L.nb * (2 * K + 1); c < L.nout_pad; ++c) {  // padding columns
    glog32[size_t(i) * L.nout_pad + c] = 0.0f;
    glog16[size_t(i) * L.nout_pad + c] = __float2bfloat16_rn(0.0f);
  }
}

// First dense layer backward, input side: dL/dx_A += 2 W1^T dA1 (u = 2 x_A - 1);
// one thread per event, W1 [H x na] staged in shared memory.
constexpr int kMaxA = kMaxFlowDim / 2;
__global__ void dense1_bwd_input_kernel(float* dP, int D, const LayerDev L, const float* params,
                                        const __nv_bfloat16* dA1, int H, long long n) {
  extern __shared__ float w1[];  // [H * na]
  const int na = L.na;
  for (int t = threadIdx.x; t < H * na; t += blockDim.x) w1[t] = params[L.off_W1 + t];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gu[kMaxA];
#pragma unroll
  for (int a = 0; a < kMaxA; ++a) gu[a] = 0.0f;
  const uint4* row = reinterpret_cast<const uint4*>(dA1 + size_t(i) * H);
  for (int j8 = 0; j8 < H / 8; ++j8) {
    const uint4 v = row[j8];
    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 g = __bfloat1622float2(h2[q]);
      const float* wa = w1 + (j8 * 8 + 2 * q) * na;
#pragma unroll
      for (int a = 0; a < kMaxA; ++a)
        if (a < na) gu[a] += g.x * wa[a] + g.y * wa[na + a];
    }
  }
#pragma unroll
  for (int a = 0; a < kMaxA; ++a)
    if (a < na) dP[i * D + L.a_idx[a]] += 2.0f * gu[a];
}

// First dense layer backward, weight side: dL/dW1[j][a] = sum_i dA1[i][j] u[i][a]
// and dL/db1[j] = sum_i dA1[i][j]; a block of H threads (one per hidden unit)
// over `rows` events staged in shared memory, then one atomic per entry.
__global__ void dense1_bwd_weight_kernel(const float* Pin, int D, const LayerDev L, const __nv_bfloat16* dA1, int H,
                                         long long n, int rows, float* grads) {
  extern __shared__ float u[];  // [rows * na]
  const int na = L.na;
  const long long r0 = (long long)blockIdx.x * rows;
  const int nr = int(min((long long)rows, n - r0));
  for (int t = threadIdx.x; t < nr * na; t += blockDim.x) {
    const int r = t / na, a = t % na;
    u[t] = 2.0f * Pin[(r0 + r) * D + L.a_idx[a]] - 1.0f;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float acc[kMaxA], accb = 0.0f;
#pragma unroll
    for (int a = 0; a < kMaxA; ++a) acc[a] = 0.0f;
    for (int r = 0; r < nr; ++r) {
      const float g = __bfloat162float(dA1[size_t(r0 + r) * H + j]);
      accb += g;
#pragma unroll
      for (int a = 0; a < kMaxA; ++a)
        if (a < na) acc[a] += g * u[r * na + a];
    }
#pragma unroll
    for (int a = 0; a < kMaxA; ++a)
      if (a < na) atomicAdd(&grads[L.off_W1 + size_t(j) * na + a], acc[a]);
    atomicAdd(&grads[L.off_b1 + j], accb);
  }
}

// out[c] += sum over rows of m[r][c] (bias gradients); one thread per column
// and block-row chunk.
template <class T>
__global__ void colsum_kernel(const T* m, long long rows, int cols, int ld, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const long long r0 = (long long)blockIdx.y * 1024, r1 = min(rows, r0 + 1024);
  float acc = 0.0f;
  for (long long r = r0; r < r1; ++r) acc += float(m[r * ld + c]);
  atomicAdd(&out[c], acc);
}

// dst[c][r] = src[r][c] for a BF16 [rows x cols] matrix (32 x 32 tiles).
__global__ void transpose_bf16_kernel(const __nv_bfloat16* src, long long rows, int cols, __nv_bfloat16* dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const long long r0 = (long long)blockIdx.y * 32;
  const int c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const long long r = r0 + k;
    const int c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = src[r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k;
    const long long r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[size_t(c) * rows + r] = tile[threadIdx.x][k];
  }
}

// Integrand at given points (no VEGAS map): f[i] = f(x_i), FP32 path.
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
    // a failed event (non-finite or unconverged phase space) is marked NaN
    f[i] = (o.status == 0 && isfinite(o.f)) ? float(o.f) : __int_as_float(0x7fc00000);
  }
}

// Training weights w = |f| / q = |f| exp(-log q) (0 for a failed event).
__global__ void flow_weights_kernel(const float* f, const float* logq, float* w, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float wi = fabsf(f[i]) * expf(-logq[i]);
  w[i] = isfinite(wi) ? wi : 0.0f;
}

// Loss sums in FP64: sums[0] += sum w, sums[1] += sum w log q.
__global__ void loss_sums_kernel(const float* w, const float* logq, long long n, double* sums) {
  __shared__ double sh[2][32];
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
    atomicAdd(&sums[0], sa);
    atomicAdd(&sums[1], sb);
  }
}

// Sampling sums over a chunk: w = f exp(-log q) accumulated with Kahan FP64
// per thread into per-block partials (BlockPartial, fixed-order reduced).
__global__ void flow_sums_kernel(const float* f, const float* logq, long long n, BlockPartial* parts) {
  Acc acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double w = double(f[i]) * exp(-double(logq[i]));
    if (!isfinite(w)) {
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
  __shared__ BlockPartial warp_part[8];
  block_reduce(acc, warp_part, &parts[blockIdx.x]);
}

// Adam (thesis Sec. "Optimizers") on every master parameter; gradients of the
// 256-wide weights are read from their transposed layout.  Then the BF16
// copies (and transposes) are refreshed and the gradients cleared.
struct AdamArgs {
  float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t)
};
__global__ void adam_kernel(float* params, float* grads, float* m, float* v, size_t n, const LayerDev* layers, int nl,
                            int H, AdamArgs A) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  // locate the tensor: transposed-gradient mapping for W2, W3, W4
  size_t gidx = idx;
  for (int l = 0; l < nl; ++l) {
    const LayerDev& L = layers[l];
    auto tr = [&](size_t off, int rows, int cols) {  // W [rows x cols], gradient stored [cols x rows]
      if (idx >= off && idx < off + size_t(rows) * cols) {
        const size_t e = idx - off;
        const size_t r = e / cols, c = e % cols;
        gidx = off + c * rows + r;
      }
    };
    tr(L.off_W2, H, H);
    tr(L.off_W3, H, H);
    tr(L.off_W4, L.nout_pad, H);
  }
  const float g = grads[gidx];
  const float mi = A.b1 * m[idx] + (1.0f - A.b1) * g;
  const float vi = A.b2 * v[idx] + (1.0f - A.b2) * g * g;
  m[idx] = mi;
  v[idx] = vi;
  params[idx] -= A.lr * (mi * A.c1) / (sqrtf(vi * A.c2) + A.eps);
}

__global__ void zero_kernel(float* p, size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0f;
}

// BF16 copy of W [rows x cols] and of its transpose.
__global__ void to_bf16_kernel(const float* W, int rows, int cols, __nv_bfloat16* out, __nv_bfloat16* out_t) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int r = idx / cols, c = idx % cols;
  const __nv_bfloat16 h = __float2bfloat16_rn(W[idx]);
  out[idx] = h;
  out_t[size_t(c) * rows + r] = h;
}

unsigned blocks_for(long long n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace
}  // namespace mc

using mc::BlockPartial;
using mc::LayerDev;

struct mc_flow_s {
  int device = 0, D = 0, L = 0, K = 0, H = 256;
  long long max_batch = 0, bp = 0;  // capacity (rows, padded to 128)
  uint64_t seed = 0;
  int step = 0;
  std::vector<LayerDev> layers;
  size_t nparam = 0;                // device master-parameter count (padded layout)
  std::vector<size_t> host_map;     // packed host index -> device index
  float *d_params = nullptr, *d_grads = nullptr, *d_m = nullptr, *d_v = nullptr;
  __nv_bfloat16* d_wbf = nullptr;   // BF16 weights and transposes of all layers
  LayerDev* d_layers = nullptr;
  // workspace
  float *P = nullptr, *logq = nullptr, *f = nullptr, *w = nullptr, *dP = nullptr;
  float *logits = nullptr, *glog32 = nullptr;
  __nv_bfloat16 *h = nullptr, *glog16 = nullptr, *dA = nullptr, *tA = nullptr, *tB = nullptr;
  double* sums = nullptr;
  double* h_sums = nullptr;  // pinned
  BlockPartial *parts = nullptr, *total = nullptr, *h_total = nullptr;
  int* err = nullptr;
  int nout_pad_max = 0;
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

long long pad128(long long n) { return (n + 127) / 128 * 128; }

float* P_of(mc_flow F, int l) { return F->P + size_t(l) * F->bp * F->D; }
__nv_bfloat16* h_of(mc_flow F, int l, int k) { return F->h + (size_t(l) * 3 + k) * F->bp * F->H; }
float* logits_of(mc_flow F, int l) { return F->logits + size_t(l) * F->bp * F->nout_pad_max; }

// N tile: the largest multiple of 16 up to 256 that divides N (N % 64 == 0).
int pick_bn(int N) {
  for (int bn = std::min(256, N) / 16 * 16; bn >= 16; bn -= 16)
    if (N % bn == 0) return bn;
  return 16;
}

// split-K factor for a weight-gradient product (K = batch): about two CTAs
// per SM, at least four 64-deep k-blocks per split.
int pick_splits(int M, int N, long long K) {
  const int tiles = (M / 128) * (N / pick_bn(N));
  const long long kb = K / 64;
  return int(std::max<long long>(1, std::min<long long>(kb / 4, (2 * 148 + tiles - 1) / tiles)));
}

int gemm(mc_flow F, int M, int N, int K, int epi, const __nv_bfloat16* a, int lda, const __nv_bfloat16* b, int ldb,
         const float* bias, void* c, int ldc, const __nv_bfloat16* mask, int splits, cudaStream_t st) {
  FLOW_CUDA(cudaGetLastError());  // launches queued before this product
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.bn = pick_bn(N);
  g.epilogue = epi;
  g.bias = bias;
  g.ldc = ldc;
  if (epi == mc::kEpiBiasF32 || epi == mc::kEpiAtomicF32)
    g.c_f32 = static_cast<float*>(c);
  else
    g.c_bf16 = static_cast<__nv_bfloat16*>(c);
  g.mask = mask;
  g.ld_mask = ldc;
  g.error = F->err;
  FLOW_CUDA(mc::tc_gemm(g, a, lda, b, ldb, splits, st));
  return MC_OK;
}

// Conditioner of layer l on the points P (rows n padded to F->bp granularity):
// h1..h3 into the layer's activation slots, logits into logits_of(l).
int conditioner(mc_flow F, int l, const float* P, long long n, bool keep, cudaStream_t st) {
  const LayerDev& L = F->layers[l];
  const int H = F->H;
  const int slot = keep ? l : 0;
  __nv_bfloat16 *h1 = h_of(F, slot, 0), *h2 = h_of(F, slot, 1), *h3 = h_of(F, slot, 2);
  mc::dense1_kernel<<<mc::blocks_for(n * H, 256), 256, 0, st>>>(P, F->D, L, F->d_params, h1, H, n);
  if (int rc = gemm(F, int(n), H, H, mc::kEpiBiasReluBf16, h1, H, L.W2h, H, F->d_params + L.off_b2, h2, H, nullptr, 1,
                    st))
    return rc;
  if (int rc = gemm(F, int(n), H, H, mc::kEpiBiasReluBf16, h2, H, L.W3h, H, F->d_params + L.off_b3, h3, H, nullptr, 1,
                    st))
    return rc;
  return gemm(F, int(n), L.nout_pad, H, mc::kEpiBiasF32, h3, H, L.W4h, H, F->d_params + L.off_b4,
              logits_of(F, keep ? l : 0), L.nout_pad, nullptr, 1, st);
}

// Forward (sampling) pass over n (multiple of 128) rows of P[0] -> P[0] in
// place; logq initialised to 0 and accumulated.
int forward_pass(mc_flow F, long long n, cudaStream_t st) {
  float* P = P_of(F, 0);
  FLOW_CUDA(cudaMemsetAsync(F->logq, 0, sizeof(float) * n, st));
  for (int l = 0; l < F->L; ++l) {
    if (int rc = conditioner(F, l, P, n, false, st)) return rc;
    mc::spline_fwd_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P, F->D, F->layers[l], logits_of(F, 0), F->K,
                                                                   F->logq, n);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

// Inverse (density) pass from P[L] (the points x) down to P[0] = z, keeping
// every layer's activations and logits; logq accumulated.
int inverse_pass(mc_flow F, long long n, cudaStream_t st) {
  FLOW_CUDA(cudaMemsetAsync(F->logq, 0, sizeof(float) * n, st));
  for (int l = F->L - 1; l >= 0; --l) {
    if (int rc = conditioner(F, l, P_of(F, l + 1), n, true, st)) return rc;
    mc::spline_inv_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P_of(F, l + 1), P_of(F, l), F->D, F->layers[l],
                                                                   logits_of(F, l), F->K, F->logq, n);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

void transpose(const __nv_bfloat16* src, long long rows, int cols, __nv_bfloat16* dst, cudaStream_t st) {
  const dim3 grid(unsigned((cols + 31) / 32), unsigned((rows + 31) / 32));
  mc::transpose_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, dst);
}

// Backward of the inverse pass (weights F->w and sums F->sums[0] = sum w):
// accumulates all parameter gradients into F->d_grads (zeroed beforehand).
int backward_pass(mc_flow F, long long n, long long n_real, cudaStream_t st) {
  const int H = F->H, D = F->D;
  FLOW_CUDA(cudaMemsetAsync(F->dP, 0, sizeof(float) * n * D, st));
  for (int l = 0; l < F->L; ++l) {
    const LayerDev& L = F->layers[l];
    float* g = F->d_grads;
    mc::spline_inv_bwd_kernel<<<mc::blocks_for(n, 128), 128, 0, st>>>(P_of(F, l + 1), F->dP, D, L, logits_of(F, l),
                                                                       F->K, F->w, F->sums, F->glog32, F->glog16, n,
                                                                       n_real);
    // last dense layer: dW4^T = H3^T . dY (split-K over the batch), db4, dH3
    const __nv_bfloat16 *h1 = h_of(F, l, 0), *h2 = h_of(F, l, 1), *h3 = h_of(F, l, 2);
    __nv_bfloat16* dA = F->dA;
    __nv_bfloat16* dA_b = F->dA + size_t(F->bp) * H;
    transpose(h3, n, H, F->tA, st);
    transpose(F->glog16, n, L.nout_pad, F->tB, st);
    if (int rc = gemm(F, H, L.nout_pad, int(n), mc::kEpiAtomicF32, F->tA, int(n), F->tB, int(n), nullptr,
                      g + L.off_W4, L.nout_pad, nullptr, pick_splits(H, L.nout_pad, n), st))
      return rc;
    mc::colsum_kernel<float><<<dim3(mc::blocks_for(L.nout_pad, 128), unsigned((n + 1023) / 1024)), 128, 0, st>>>(
        F->glog32, n, L.nout_pad, L.nout_pad, g + L.off_b4);
    if (int rc = gemm(F, int(n), H, L.nout_pad, mc::kEpiReluMaskBf16, F->glog16, L.nout_pad, L.W4t, L.nout_pad,
                      nullptr, dA, H, h3, 1, st))
      return rc;
    // third dense layer
    transpose(h2, n, H, F->tA, st);
    transpose(dA, n, H, F->tB, st);
    if (int rc = gemm(F, H, H, int(n), mc::kEpiAtomicF32, F->tA, int(n), F->tB, int(n), nullptr, g + L.off_W3, H,
                      nullptr, pick_splits(H, H, n), st))
      return rc;
    mc::colsum_kernel<__nv_bfloat16><<<dim3(mc::blocks_for(H, 128), unsigned((n + 1023) / 1024)), 128, 0, st>>>(
        dA, n, H, H, g + L.off_b3);
    if (int rc = gemm(F, int(n), H, H, mc::kEpiReluMaskBf16, dA, H, L.W3t, H, nullptr, dA_b, H, h2, 1, st)) return rc;
    // second dense layer
    transpose(h1, n, H, F->tA, st);
    transpose(dA_b, n, H, F->tB, st);
    if (int rc = gemm(F, H, H, int(n), mc::kEpiAtomicF32, F->tA, int(n), F->tB, int(n), nullptr, g + L.off_W2, H,
                      nullptr, pick_splits(H, H, n), st))
      return rc;
    mc::colsum_kernel<__nv_bfloat16><<<dim3(mc::blocks_for(H, 128), unsigned((n + 1023) / 1024)), 128, 0, st>>>(
        dA_b, n, H, H, g + L.off_b2);
    if (int rc = gemm(F, int(n), H, H, mc::kEpiReluMaskBf16, dA_b, H, L.W2t, H, nullptr, dA, H, h1, 1, st)) return rc;
    // first dense layer (CUDA cores): adds 2 W1^T dA1 to the A coordinates of dP; W1, b1 gradients
    mc::dense1_bwd_input_kernel<<<mc::blocks_for(n, 128), 128, sizeof(float) * H * L.na, st>>>(
        F->dP, D, L, F->d_params, dA, H, n);
    constexpr int kRows = 256;
    mc::dense1_bwd_weight_kernel<<<mc::blocks_for(n, kRows), H, sizeof(float) * kRows * L.na, st>>>(
        P_of(F, l + 1), D, L, dA, H, n, kRows, g);
    FLOW_CUDA(cudaGetLastError());
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

int refresh_bf16(mc_flow F, cudaStream_t st) {
  const int H = F->H;
  for (const LayerDev& L : F->layers) {
    mc::to_bf16_kernel<<<mc::blocks_for(H * H, 256), 256, 0, st>>>(F->d_params + L.off_W2, H, H, L.W2h, L.W2t);
    mc::to_bf16_kernel<<<mc::blocks_for(H * H, 256), 256, 0, st>>>(F->d_params + L.off_W3, H, H, L.W3h, L.W3t);
    mc::to_bf16_kernel<<<mc::blocks_for(L.nout_pad * H, 256), 256, 0, st>>>(F->d_params + L.off_W4, L.nout_pad, H,
                                                                             L.W4h, L.W4t);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
}

int check_err(mc_flow F, cudaStream_t st) {
  int e = 0;
  FLOW_CUDA(cudaMemcpyAsync(&e, F->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FLOW_CUDA(cudaStreamSynchronize(st));
  if (e) return ffail(MC_ETIMEOUT, "mc_flow: a tensor-core GEMM wait timed out");
  return MC_OK;
}

int eval_points(mc_flow F, const mc_integrand* itg, mc_pdf pdf, const float* X, long long n, float* f, cudaStream_t st) {
  mc::KernelArgs a;
  if (int rc = mc::fill_process_args(itg, pdf, &a)) return rc;
  const int nfl = itg->proc == MC_PP_TTBAR ? 11 : (a.pdf.nx ? 1 : 0);
  const size_t smem = sizeof(float) * size_t(a.pdf.nx) * (1 + 2 * nfl);
  const unsigned grid = std::min<unsigned>(mc::blocks_for(n, 128), 148u * 16u);
  switch (itg->proc) {
    case MC_EE_MUMU: mc::points_kernel<mc::P_EE_MUMU><<<grid, 128, smem, st>>>(a, X, F->D, f, n); break;
    case MC_PP_TTBAR: mc::points_kernel<mc::P_PP_TTBAR><<<grid, 128, smem, st>>>(a, X, F->D, f, n); break;
    case MC_GG_TTBARG: mc::points_kernel<mc::P_GG_TTBARG><<<grid, 128, smem, st>>>(a, X, F->D, f, n); break;
    case MC_GG_TTBARG_7D: mc::points_kernel<mc::P_GG_TTBARG_7D><<<grid, 128, smem, st>>>(a, X, F->D, f, n); break;
    default: mc::points_kernel<mc::P_GAUSS><<<grid, 128, smem, st>>>(a, X, F->D, f, n);
  }
  FLOW_CUDA(cudaGetLastError());
  return MC_OK;
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
                  (void*)F->logits, (void*)F->glog32, (void*)F->h, (void*)F->glog16, (void*)F->dA, (void*)F->tA,
                  (void*)F->tB, (void*)F->sums, (void*)F->parts, (void*)F->total, (void*)F->err})
    cudaFree(p);
  if (F->h_sums) cudaFreeHost(F->h_sums);
  if (F->h_total) cudaFreeHost(F->h_total);
  delete F;
  return MC_OK;
}

int mc_flow_create(const mc_flow_cfg* cfg, const float* init, int64_t max_batch, uint64_t seed, mc_flow* out) {
  if (!out || !cfg || !init) return ffail(MC_EINVAL, "mc_flow_create: NULL argument");
  *out = nullptr;
  if (cfg->ndim < 2 || cfg->ndim > mc::kMaxFlowDim || cfg->layers < 1 || cfg->layers > mc::kMaxLayers ||
      cfg->bins < 2 || cfg->bins > mc::kFlowMaxBins || cfg->hidden != 256 || max_batch < 1 || max_batch > (int64_t(1) << 21))
    return ffail(MC_EINVAL,
                 "mc_flow_create: need 2 <= ndim <= 16, 1..16 layers, 2..32 bins, hidden 256, 1 <= max_batch <= 2^21");
  auto* F = new mc_flow_s;
  cudaGetDevice(&F->device);
  F->D = cfg->ndim;
  F->L = cfg->layers;
  F->K = cfg->bins;
  F->H = cfg->hidden;
  F->max_batch = max_batch;
  F->bp = pad128(max_batch);
  F->seed = seed;
  const int H = F->H;
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
    L.nout = L.nb * (2 * F->K + 1);
    L.nout_pad = (L.nout + 63) / 64 * 64;
    F->nout_pad_max = std::max(F->nout_pad_max, L.nout_pad);
    L.off_W1 = off; off += size_t(H) * L.na;
    L.off_b1 = off; off += H;
    L.off_W2 = off; off += size_t(H) * H;
    L.off_b2 = off; off += H;
    L.off_W3 = off; off += size_t(H) * H;
    L.off_b3 = off; off += H;
    L.off_W4 = off; off += size_t(L.nout_pad) * H;
    L.off_b4 = off; off += L.nout_pad;
    F->layers.push_back(L);
    woff += 2 * (2 * size_t(H) * H + size_t(L.nout_pad) * H);
  }
  F->nparam = off;
  const size_t bp = size_t(F->bp), D = size_t(F->D), np = size_t(F->nout_pad_max);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&F->d_params, sizeof(float) * off);
  alloc((void**)&F->d_grads, sizeof(float) * off);
  alloc((void**)&F->d_m, sizeof(float) * off);
  alloc((void**)&F->d_v, sizeof(float) * off);
  alloc((void**)&F->d_wbf, sizeof(__nv_bfloat16) * woff);
  alloc((void**)&F->d_layers, sizeof(LayerDev) * F->L);
  alloc((void**)&F->P, sizeof(float) * (F->L + 1) * bp * D);
  alloc((void**)&F->logq, sizeof(float) * bp);
  alloc((void**)&F->f, sizeof(float) * bp);
  alloc((void**)&F->w, sizeof(float) * bp);
  alloc((void**)&F->dP, sizeof(float) * bp * D);
  alloc((void**)&F->logits, sizeof(float) * F->L * bp * np);
  alloc((void**)&F->glog32, sizeof(float) * bp * np);
  alloc((void**)&F->h, sizeof(__nv_bfloat16) * F->L * 3 * bp * H);
  alloc((void**)&F->glog16, sizeof(__nv_bfloat16) * bp * np);
  alloc((void**)&F->dA, sizeof(__nv_bfloat16) * 2 * bp * H);
  alloc((void**)&F->tA, sizeof(__nv_bfloat16) * bp * std::max<size_t>(H, np));
  alloc((void**)&F->tB, sizeof(__nv_bfloat16) * bp * std::max<size_t>(H, np));
  alloc((void**)&F->sums, sizeof(double) * 2);
  alloc((void**)&F->parts, sizeof(BlockPartial) * 148 * 32);
  alloc((void**)&F->total, sizeof(BlockPartial));
  alloc((void**)&F->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_sums, sizeof(double) * 2);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&F->h_total, sizeof(BlockPartial));
  if (e != cudaSuccess) {
    mc_flow_free(F);
    return ffail(MC_ENOMEM, std::string("mc_flow_create: allocation failed: ") + cudaGetErrorString(e));
  }
  woff = 0;
  for (LayerDev& L : F->layers) {
    L.W2h = F->d_wbf + woff; woff += size_t(H) * H;
    L.W2t = F->d_wbf + woff; woff += size_t(H) * H;
    L.W3h = F->d_wbf + woff; woff += size_t(H) * H;
    L.W3t = F->d_wbf + woff; woff += size_t(H) * H;
    L.W4h = F->d_wbf + woff; woff += size_t(L.nout_pad) * H;
    L.W4t = F->d_wbf + woff; woff += size_t(L.nout_pad) * H;
  }
  // packed host layout -> padded device layout
  for (const LayerDev& L : F->layers) {
    auto span = [&](size_t dev_off, size_t n) {
      for (size_t i = 0; i < n; ++i) F->host_map.push_back(dev_off + i);
    };
    span(L.off_W1, size_t(H) * L.na);
    span(L.off_b1, H);
    span(L.off_W2, size_t(H) * H);
    span(L.off_b2, H);
    span(L.off_W3, size_t(H) * H);
    span(L.off_b3, H);
    span(L.off_W4, size_t(L.nout) * H);
    span(L.off_b4, L.nout);
  }
  if (cudaMemcpy(F->d_layers, F->layers.data(), sizeof(LayerDev) * F->L, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(F->d_m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->d_v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->d_grads, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(F->err, 0, sizeof(int)) != cudaSuccess) {
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

int mc_flow_forward(mc_flow F, int64_t n, const float* z, float* x, float* logq, void* stream) {
  if (!F || n < 0 || n > F->max_batch || (n && (!z || !x || !logq))) return ffail(MC_EINVAL, "mc_flow_forward: bad arguments");
  if (n == 0) return MC_OK;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long np = pad128(n);
  FLOW_CUDA(cudaMemsetAsync(P_of(F, 0), 0, sizeof(float) * np * F->D, st));
  FLOW_CUDA(cudaMemcpyAsync(P_of(F, 0), z, sizeof(float) * n * F->D, cudaMemcpyDeviceToDevice, st));
  if (int rc = forward_pass(F, np, st)) return rc;
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
  FLOW_CUDA(cudaMemsetAsync(F->sums, 0, sizeof(double) * 2, st));
  mc::loss_sums_kernel<<<std::min<unsigned>(mc::blocks_for(n, 256), 1184u), 256, 0, st>>>(F->w, F->logq, n, F->sums);
  if (int rc = backward_pass(F, np, n, st)) return rc;
  FLOW_CUDA(cudaMemcpyAsync(F->h_sums, F->sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  if (int rc = check_err(F, st)) return rc;
  if (loss) *loss = F->h_sums[0] > 0.0 ? -F->h_sums[1] / F->h_sums[0] : 0.0;
  if (grads) {
    std::vector<float> dev(F->nparam);
    FLOW_CUDA(cudaMemcpy(dev.data(), F->d_grads, sizeof(float) * F->nparam, cudaMemcpyDeviceToHost));
    // gradients of W2..W4 are stored transposed
    size_t k = 0;
    const int H = F->H;
    for (const LayerDev& L : F->layers) {
      for (size_t i = 0; i < size_t(H) * L.na; ++i) grads[k++] = dev[L.off_W1 + i];
      for (int i = 0; i < H; ++i) grads[k++] = dev[L.off_b1 + i];
      for (int r = 0; r < H; ++r)
        for (int c = 0; c < H; ++c) grads[k++] = dev[L.off_W2 + size_t(c) * H + r];
      for (int i = 0; i < H; ++i) grads[k++] = dev[L.off_b2 + i];
      for (int r = 0; r < H; ++r)
        for (int c = 0; c < H; ++c) grads[k++] = dev[L.off_W3 + size_t(c) * H + r];
      for (int i = 0; i < H; ++i) grads[k++] = dev[L.off_b3 + i];
      for (int r = 0; r < L.nout; ++r)
        for (int c = 0; c < H; ++c) grads[k++] = dev[L.off_W4 + size_t(c) * L.nout_pad + r];
      for (int i = 0; i < L.nout; ++i) grads[k++] = dev[L.off_b4 + i];
    }
  }
  return MC_OK;
}

int mc_flow_adam_step(mc_flow F, double lr, void* stream) {
  if (!F || !(lr > 0.0)) return ffail(MC_EINVAL, "mc_flow_adam_step: bad arguments");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  ++F->step;
  const double b1 = 0.9, b2 = 0.999;
  mc::AdamArgs A{float(lr), float(b1), float(b2), 1e-8f, float(1.0 / (1.0 - std::pow(b1, F->step))),
                 float(1.0 / (1.0 - std::pow(b2, F->step)))};
  mc::adam_kernel<<<mc::blocks_for(F->nparam, 256), 256, 0, st>>>(F->d_params, F->d_grads, F->d_m, F->d_v, F->nparam,
                                                                   F->d_layers, F->L, F->H, A);
  FLOW_CUDA(cudaGetLastError());
  return refresh_bf16(F, st);
}

int mc_flow_train(mc_flow F, const mc_integrand* itg, mc_pdf pdf, int steps, int64_t batch, double lr, void* stream,
                  double* losses) {
  if (!F || !itg || steps < 0 || batch < 2 || batch > F->max_batch || !(lr > 0.0))
    return ffail(MC_EINVAL, "mc_flow_train: bad arguments");
  if (mc::process_dim(itg) != F->D) return ffail(MC_EINVAL, "mc_flow_train: flow dimension differs from the process");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = batch, np = pad128(n);
  for (int s = 0; s < steps; ++s) {
    // sample a batch from the current flow: z -> x (into P[L]), log q
    float* Z = P_of(F, 0);
    FLOW_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * np * F->D, st));
    mc::flow_uniforms_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(Z, n, F->D, F->seed, 0x10000u + uint32_t(F->step),
                                                                      0u, 0);
    if (int rc = forward_pass(F, np, st)) return rc;
    FLOW_CUDA(cudaMemcpyAsync(P_of(F, F->L), Z, sizeof(float) * np * F->D, cudaMemcpyDeviceToDevice, st));
    if (int rc = eval_points(F, itg, pdf, P_of(F, F->L), n, F->f, st)) return rc;
    FLOW_CUDA(cudaMemsetAsync(F->w, 0, sizeof(float) * np, st));
    mc::flow_weights_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(F->f, F->logq, F->w, n);
    // density pass with activations, loss sums, backward, Adam
    mc::zero_kernel<<<mc::blocks_for(F->nparam, 256), 256, 0, st>>>(F->d_grads, F->nparam);
    if (int rc = inverse_pass(F, np, st)) return rc;
    FLOW_CUDA(cudaMemsetAsync(F->sums, 0, sizeof(double) * 2, st));
    mc::loss_sums_kernel<<<std::min<unsigned>(mc::blocks_for(n, 256), 1184u), 256, 0, st>>>(F->w, F->logq, n,
                                                                                            F->sums);
    if (int rc = backward_pass(F, np, n, st)) return rc;
    if (int rc = mc_flow_adam_step(F, lr, stream)) return rc;
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
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long chunk = (F->max_batch / 128) * 128;
  if (chunk < 128) return ffail(MC_EINVAL, "mc_flow_iterate: max_batch below 128");
  BlockPartial tot = {0.0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0};
  for (long long first = 0; first < nevents; first += chunk) {
    const long long n = std::min<long long>(chunk, nevents - first), np = pad128(n);
    float* Z = P_of(F, 0);
    FLOW_CUDA(cudaMemsetAsync(Z, 0, sizeof(float) * np * F->D, st));
    mc::flow_uniforms_kernel<<<mc::blocks_for(n, 256), 256, 0, st>>>(Z, n, F->D, F->seed, 0x20000u + iteration, 0u,
                                                                      first);
    if (int rc = forward_pass(F, np, st)) return rc;
    if (int rc = eval_points(F, itg, pdf, Z, n, F->f, st)) return rc;
    const int grid = 148 * 8;
    mc::flow_sums_kernel<<<grid, 256, 0, st>>>(F->f, F->logq, n, F->parts);
    FLOW_CUDA(mc::launch_finalize(F->parts, grid, F->total, st));
    FLOW_CUDA(cudaMemcpyAsync(F->h_total, F->total, sizeof(BlockPartial), cudaMemcpyDeviceToHost, st));
    FLOW_CUDA(cudaStreamSynchronize(st));
    mc::partial_add(tot, *F->h_total);
  }
  out->sum = tot.sum_hi + tot.sum_lo;
  out->sum2 = tot.sum2_hi + tot.sum2_lo;
  out->wmax = tot.wmax;
  out->n_nonzero = tot.n_nonzero;
  out->n_bad = tot.n_bad;
  out->status = tot.n_bad ? MC_ENAN : MC_OK;
  return check_err(F, st);
}

}  // extern "C"
