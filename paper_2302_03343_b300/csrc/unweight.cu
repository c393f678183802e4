// Unweighting on the device (thesis Sec. "Unweighted event exporter", with the
// acceptance-rejection rule of Sec. "Monte Carlo integration"): event i of the
// weighted sample survives when w_i > r_i w_max, so that it is kept with
// probability w_i / w_max and the survivors follow the integrand's
// distribution with unit weight.
//
// The weights come from the weights pass of the fused integrand kernel
// (KernelArgs::wout, 8 bytes per event); r_i is Philox call 255 of the
// event's own counter, a call the integrand never makes, so every decision
// can be re-derived from (seed, iteration, integrand id, event index).
// Four passes:
//  * uw_count_kernel: block b takes the contiguous chunk b of the events,
//    decides every event (one read of its weight, one Philox call for the
//    events of positive weight), stores the decisions as a bit mask (one
//    word per 32 events, a warp ballot) and counts them;
//  * uw_scan_kernel: exclusive scan of the per-chunk counts (one block);
//  * uw_compact_kernel: reads the mask chunk by chunk and writes the indices
//    of the accepted events in event order (block prefix over the warps'
//    population counts), so the output order does not depend on scheduling;
//  * uw_export_kernel: one thread per accepted event regenerates the event
//    from its Philox counter (uniforms, VEGAS map, phase space) through the
//    recording path of the fused integrand and writes its mc_event record in
//    the laboratory frame.  Only the accepted fraction (a few per cent) is
//    regenerated, densely packed, so no warp runs a mostly idle |M|^2.
#include <cstring>

#include "../../include/mcint.h"
#include "event.cuh"
#include "handles.h"
#include "launch.h"

static_assert(sizeof(mc_event) == 200, "mc_event layout");

namespace mc {

constexpr int kUwBlock = 256;  // kUwMaxChunks (launch.h): chunks of the count / compact passes, one scan block

// Acceptance uniform of event ev: counter (ev lo, ev hi, iteration,
// gid | 255 << 8), r = (2k + 1) 2^-53 with k the top 52 bits of words 0:1,
// so r lies strictly inside (0, 1).  Returned as the odd integer 2k + 1.
MC_D uint64_t acceptance_odd(uint64_t seed, uint32_t iteration, uint32_t gid, uint64_t ev) {
  const uint4 w = philox4x32_10(make_uint4(uint32_t(ev), uint32_t(ev >> 32), iteration, (gid & 0xffu) | (255u << 8)),
                                make_uint2(uint32_t(seed), uint32_t(seed >> 32)));
  return ((((uint64_t(w.x) << 32) | w.y) >> 12) << 1) | 1u;
}

// The FP64 bits of RN(r w_max), r = odd 2^-53, for a w_max whose biased
// exponent e_b is at least 54 (so the product is a normal number): the
// integer product P = odd * M (M the 53-bit significand of w_max, P below
// 2^106) rounded to 53 significant bits, to nearest with ties to even, and
// the exponent e_b - 53 + (bits dropped).  This is the IEEE product done
// with integer multiply-adds; B300 issues FP64 arithmetic at 1/64 of the
// FP32 rate, and three FP64 operations per event made the decision pass
// FP64-bound.
MC_D uint64_t product_bits(uint64_t odd, uint64_t m_w, int e_b) {
  const uint64_t lo = odd * m_w, hi = __umul64hi(odd, m_w);
  const int lead = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // >= 52
  const int s = lead - 52;                                                               // 0 .. 53
  uint64_t m = lo;
  if (s > 0) {
    m = (lo >> s) | (hi << (64 - s));
    const uint64_t rem = lo & ((1ull << s) - 1), half = 1ull << (s - 1);
    m += (rem > half || (rem == half && (m & 1u))) ? 1u : 0u;
  }
  int e = e_b - 53 + s;
  if (m == (1ull << 53)) {
    m >>= 1;
    ++e;
  }
  return (uint64_t(e) << 52) | (m - (1ull << 52));
}

struct UwArgs {
  const double* w;  // [n] weights of the sample
  long long n, chunk;
  double wmax;
  uint64_t m_w;     // significand of wmax with its hidden bit (integer path)
  int e_w;          // biased exponent of wmax; 0: take the FP64 path
  uint64_t seed, first;
  uint32_t iteration, gid;
};

// The decision w > r w_max, identical to the FP64 comparison: positive
// doubles order like their bit patterns, so the integer path compares the
// weight's bits with those of RN(r w_max); zero, negative and NaN weights are
// never accepted, and cut events (w = 0) never draw their uniform.
MC_D bool uw_accept(const UwArgs& u, long long i) {
  const double wi = u.w[i];
  const uint64_t wb = uint64_t(__double_as_longlong(wi));
  if (wb == 0u || wb > 0x7FF0000000000000ull) return false;  // +0, negative (sign bit), NaN
  const uint64_t odd = acceptance_odd(u.seed, u.iteration, u.gid, u.first + uint64_t(i));
  if (u.e_w) return wb > product_bits(odd, u.m_w, u.e_w);
  return wi > double(odd) * 0x1p-53 * u.wmax;
}

// Chunks are multiples of kUwBlock events, so the 32 events of a warp in one
// round share one mask word: word (r0 + 32 warp) / 32.
__global__ void __launch_bounds__(kUwBlock) uw_count_kernel(UwArgs u, unsigned long long* counts, uint32_t* mask) {
  const long long lo = (long long)blockIdx.x * u.chunk;
  const long long hi = min(u.n, lo + u.chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned int c = 0;
  for (long long r0 = lo; r0 < hi; r0 += kUwBlock) {
    const long long i = r0 + threadIdx.x;
    const bool acc = i < hi && uw_accept(u, i);
    const unsigned m = __ballot_sync(0xffffffffu, acc);
    if (lane == 0 && r0 + 32 * wid < hi) mask[(r0 >> 5) + wid] = m;
    c += acc;
  }
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  __shared__ unsigned int part[kUwBlock / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < kUwBlock / 32; ++k) t += part[k];
    counts[blockIdx.x] = t;
  }
}

// Exclusive scan of counts[0 .. nchunks) (nchunks <= 1024) in place; total to
// *total.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) uw_scan_kernel(unsigned long long* counts, int nchunks,
                                                        unsigned long long* total) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const unsigned long long v = t < nchunks ? counts[t] : 0ull;
  unsigned long long incl = v;
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  __shared__ unsigned long long warp_sum[32];
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned long long s = warp_sum[lane], si = s;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, si, off);
      if (lane >= off) si += o;
    }
    warp_sum[lane] = si - s;  // exclusive prefix of the warps
    if (lane == 31) *total = si;
  }
  __syncthreads();
  if (t < nchunks) counts[t] = warp_sum[wid] + incl - v;
}

// Indices (within the launch) of the accepted events, in event order, to
// idx[offset ..], the first `cap` of them, from the decision mask.
__global__ void __launch_bounds__(kUwBlock) uw_compact_kernel(UwArgs u, const unsigned long long* offsets,
                                                               const uint32_t* mask, uint32_t* idx, long long cap) {
  const long long lo = (long long)blockIdx.x * u.chunk;
  const long long hi = min(u.n, lo + u.chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ unsigned int wcount[kUwBlock / 32];
  unsigned long long base = offsets[blockIdx.x];
  for (long long r0 = lo; r0 < hi; r0 += kUwBlock) {
    const long long i = r0 + threadIdx.x;
    const unsigned m = r0 + 32 * wid < hi ? mask[(r0 >> 5) + wid] : 0u;
    const bool acc = (m >> lane) & 1u;
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    unsigned int before = 0, round = 0;
#pragma unroll
    for (int k = 0; k < kUwBlock / 32; ++k) {
      before += k < wid ? wcount[k] : 0u;
      round += wcount[k];
    }
    if (acc) {
      const unsigned long long pos = base + before + __popc(m & ((1u << lane) - 1u));
      if ((long long)pos < cap) idx[pos] = uint32_t(i);
    }
    base += round;
    __syncthreads();
  }
}

template <class R> MC_D const R* uw_edges(const KernelArgs& a);
template <> MC_D const double* uw_edges<double>(const KernelArgs& a) { return a.edges64; }
template <> MC_D const float* uw_edges<float>(const KernelArgs& a) { return a.edges32; }

// Regenerates the accepted events idx[0 .. min(*total, cap)) and writes their
// records.  Shared memory as in the fused kernel: grid edges and PDF tables.
template <int PROC, bool FP64>
__global__ void __launch_bounds__(kBlock) uw_export_kernel(KernelArgs a, const uint32_t* idx,
                                                           const unsigned long long* total, long long cap,
                                                           const double* wts, mc_event* out) {
  using R = typename std::conditional<FP64, double, float>::type;
  constexpr int NFL = ProcTraits<PROC>::NFL;
  constexpr int NOUT = PROC == P_EE_MUMU ? 2 : 3;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nedge = a.ndim * (a.nbins + 1);
  R* sh_edges = reinterpret_cast<R*>(smem);
  const R* g_edges = uw_edges<R>(a);
  for (int i = threadIdx.x; i < nedge; i += blockDim.x) sh_edges[i] = g_edges[i];
  SmPdf<R> pdf;
  if constexpr (NFL > 0) {
    const int nx = a.pdf.nx;
    R* t = sh_edges + nedge;
    R* f = t + nx;
    R* d = f + NFL * nx;
    build_pdf_tables<R>(a.pdf, a.logq2_f, a.fl, NFL, t, f, d);  // ends with __syncthreads
#pragma unroll
    for (int k = 0; k < NFL; ++k) pdf.tab[k] = {t, f + k * nx, d + k * nx, nx};
  } else {
    __syncthreads();
  }
  const long long m = min((long long)*total, cap);
  Acc unused;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
    const uint32_t i = idx[j];
    double rec[MC_REC_STRIDE];
    process_event<PROC, FP64, true, R, R>(a, pdf, sh_edges, nullptr, nullptr, a.first + i, rec, unused);
    mc_event e;
    e.event = (int64_t)(a.first + i);
    e.weight = wts[i];
    const double x1 = rec[MC_REC_X1], x2 = rec[MC_REC_X2], half = 0.5 * a.prm.sqrt_s;
    e.x1 = x1;
    e.x2 = x2;
    e.proc = PROC == P_EE_MUMU ? MC_EE_MUMU
                               : (PROC == P_GG_TTBARG ? MC_GG_TTBARG : (PROC == P_GG_TTBARG_7D ? MC_GG_TTBARG_7D : MC_GG_TTBARG_MC));
    e.nout = NOUT;
    // incoming partons along the beams; outgoing momenta boosted along z from
    // the partonic frame: gamma = (x1 + x2) / (2 sqrt(x1 x2)),
    // gamma beta = (x1 - x2) / (2 sqrt(x1 x2))
    const double pa[4] = {x1 * half, 0.0, 0.0, x1 * half}, pb[4] = {x2 * half, 0.0, 0.0, -x2 * half};
    const double r2 = 2.0 * sqrt(x1 * x2);
    const double g = (x1 + x2) / r2, gb = (x1 - x2) / r2;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      e.p[0][c] = pa[c];
      e.p[1][c] = pb[c];
    }
#pragma unroll
    for (int k = 0; k < 5 - 2; ++k) {
      const double* q = rec + MC_REC_P + 4 * (2 + k);
      if (k < NOUT) {
        e.p[2 + k][0] = g * q[0] + gb * q[3];
        e.p[2 + k][1] = q[1];
        e.p[2 + k][2] = q[2];
        e.p[2 + k][3] = gb * q[0] + g * q[3];
      } else {
        e.p[2 + k][0] = e.p[2 + k][1] = e.p[2 + k][2] = e.p[2 + k][3] = 0.0;
      }
    }
    out[j] = e;
  }
}

template <int PROC, bool FP64>
static cudaError_t launch_export(const KernelArgs& a, const uint32_t* idx, const unsigned long long* total,
                                 long long cap, const double* wts, mc_event* out, int grid, cudaStream_t st) {
  using R = typename std::conditional<FP64, double, float>::type;
  constexpr int NFL = ProcTraits<PROC>::NFL;
  const size_t smem = sizeof(R) * (size_t(a.ndim) * (a.nbins + 1) + (NFL > 0 ? size_t(a.pdf.nx) * (1 + 2 * NFL) : 0));
  auto k = uw_export_kernel<PROC, FP64>;
  (void)cudaGetLastError();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k<<<grid, kBlock, smem, st>>>(a, idx, total, cap, wts, out);
  return cudaGetLastError();
}

// The four passes on `st`.  a: the arguments of the weights pass (grid,
// seed, iteration, gid, first, n); scratch (unweight_scratch_bytes): counts
// [kUwMaxChunks + 1] (the last entry receives the total), the decision mask
// [ceil(n / 32)], idx [min(n, cap)].
cudaError_t unweight_launch(int proc, bool fp64, const KernelArgs& a, const double* w, double wmax, void* scratch,
                            mc_event* out, long long cap, int nsm, cudaStream_t st) {
  const long long n = a.n;
  auto* counts = static_cast<unsigned long long*>(scratch);
  unsigned long long* total = counts + kUwMaxChunks;
  auto* mask = reinterpret_cast<uint32_t*>(counts + kUwMaxChunks + 1);
  uint32_t* idx = mask + (n + 31) / 32;
  int nchunks = int(min((long long)kUwMaxChunks, (n + 4 * kUwBlock - 1) / (4 * kUwBlock)));
  if (nchunks < 1) nchunks = 1;
  const long long chunk = ((n + nchunks - 1) / nchunks + kUwBlock - 1) / kUwBlock * kUwBlock;
  uint64_t wbits;
  std::memcpy(&wbits, &wmax, sizeof(wbits));
  const int e_b = int(wbits >> 52) & 0x7ff;
  // integer path for normal w_max >= 2^-969 (products stay normal)
  const int e_w = (wbits >> 63) == 0 && e_b >= 54 && e_b < 0x7ff ? e_b : 0;
  UwArgs u = {w, n, chunk, wmax, (wbits & ((1ull << 52) - 1)) | (1ull << 52), e_w, a.seed, a.first, a.iteration,
              a.gid};
  (void)cudaGetLastError();
  uw_count_kernel<<<nchunks, kUwBlock, 0, st>>>(u, counts, mask);
  uw_scan_kernel<<<1, 1024, 0, st>>>(counts, nchunks, total);
  uw_compact_kernel<<<nchunks, kUwBlock, 0, st>>>(u, counts, mask, idx, cap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || cap == 0) return e;
  const long long maxg = (min(n, cap) + kBlock - 1) / kBlock;
  const int grid = int(max(1ll, min(maxg, (long long)nsm * 16)));
  switch (proc) {
    case P_EE_MUMU:
      return fp64 ? launch_export<P_EE_MUMU, true>(a, idx, total, cap, w, out, grid, st)
                  : launch_export<P_EE_MUMU, false>(a, idx, total, cap, w, out, grid, st);
    case P_GG_TTBARG:
      return fp64 ? launch_export<P_GG_TTBARG, true>(a, idx, total, cap, w, out, grid, st)
                  : launch_export<P_GG_TTBARG, false>(a, idx, total, cap, w, out, grid, st);
    case P_GG_TTBARG_7D:
      return fp64 ? launch_export<P_GG_TTBARG_7D, true>(a, idx, total, cap, w, out, grid, st)
                  : launch_export<P_GG_TTBARG_7D, false>(a, idx, total, cap, w, out, grid, st);
    case P_GG_TTBARG_MC:
      return fp64 ? launch_export<P_GG_TTBARG_MC, true>(a, idx, total, cap, w, out, grid, st)
                  : launch_export<P_GG_TTBARG_MC, false>(a, idx, total, cap, w, out, grid, st);
  }
  return cudaErrorInvalidValue;
}

size_t unweight_scratch_bytes(long long n, long long cap) {
  return sizeof(unsigned long long) * (kUwMaxChunks + 1) + sizeof(uint32_t) * size_t((n + 31) / 32) +
         sizeof(uint32_t) * size_t(max(0ll, min(n, cap)));
}

}  // namespace mc
