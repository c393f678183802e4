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
//  * refine_kernel: VEGAS rebinning, one warp (block) per dimension, FP64.
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

// Refinement kernel of one grid: one block of one warp per dimension
// (refine_dimension in refine.cuh), so that the FP64 logarithms and powers of
// the damping (B300's FP64 pipe runs at 1/64 of FP32) spread over ndim SMs;
// dynamic shared memory 3 nbins + 2 doubles.
__global__ void refine_kernel(double* edges, float* edges32, double* hist_w2, unsigned int* hist_n, int ndim,
                              int nbins, double alpha) {
  extern __shared__ double refine_smem[];
  const int d = blockIdx.x;
  if (d >= ndim) return;
  refine_dimension(edges + size_t(d) * (nbins + 1), edges32 + size_t(d) * (nbins + 1), hist_w2 + size_t(d) * nbins,
                   hist_n + size_t(d) * nbins, nbins, alpha, refine_smem);
}

// Batched xf(x, Q^2) for all flavours, one thread per point: the range
// check, the logarithms, both cell searches, the Q weights and the x stencil
// are formed once per point, in the working precision R (FP32 mode: FP32
// logarithms, whose rounding at the grid's edges is clamped back into the
// grid), and every flavour is interpolated from them.  The block's outputs
// are staged in shared memory and written as one contiguous range.
constexpr int kPdfBlock = 128;
template <class R>
__global__ void __launch_bounds__(kPdfBlock) pdf_xfxq2_kernel(PdfDev pdf, long long n, const double* x,
                                                               const double* q2, double* out) {
  extern __shared__ double sh_xf[];  // [kPdfBlock][nflav]
  const int nfl = pdf.nflav, nx = pdf.nx, nq = pdf.nq;
  const long long i0 = (long long)blockIdx.x * kPdfBlock;
  const long long i = i0 + threadIdx.x;
  double* mine = sh_xf + threadIdx.x * nfl;
  if (i < n) {
    const double xv = x[i], qv = q2[i];
    if (!(xv >= pdf.x_lo && xv <= pdf.x_hi && qv >= pdf.q2_lo && qv <= pdf.q2_hi)) {
      for (int fl = 0; fl < nfl; ++fl) mine[fl] = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      R lx, lq;
      if constexpr (sizeof(R) == 8) {
        lx = log(xv);
        lq = log(qv);
      } else {
        lx = fminf(fmaxf(logf(float(xv)), float(pdf.logx[0])), float(pdf.logx[nx - 1]));
        lq = fminf(fmaxf(logf(float(qv)), float(pdf.logq2[0])), float(pdf.logq2[nq - 1]));
      }
      int j0;
      R w[4];
      q_weights_r<R>(pdf.logq2, nq, lq, &j0, w);
      const int ix = knot_cell(pdf.logx, nx, double(lx));
      const R h = R(pdf.logx[ix + 1] - pdf.logx[ix]);
      const R tau = (lx - R(pdf.logx[ix])) / h;
      // the x stencil ix-1 .. ix+2 (clamped at the ends, where the one-sided
      // slopes do not use the clamped knot) and its reciprocal spacings
      int ii[4];
      R r[3];
#pragma unroll
      for (int t = 0; t < 4; ++t) ii[t] = min(max(ix - 1 + t, 0), nx - 1);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const double d = pdf.logx[ii[t + 1]] - pdf.logx[ii[t]];
        r[t] = d != 0.0 ? R(1.0 / d) : R(0);
      }
      const bool first = ix == 0, last = ix + 1 == nx - 1;
      const R t2 = tau * tau, t3 = t2 * tau;
      const R c0 = R(2) * t3 - R(3) * t2 + R(1), c1 = (t3 - R(2) * t2 + tau) * h, c2 = R(-2) * t3 + R(3) * t2,
              c3 = (t3 - t2) * h;
      // the Hermite step as weights of the four x knots: slopes
      // d0 = al s12 + be s01, d1 = ga s12 + de s23 (one-sided at the ends),
      // s01 = r0 (f1 - f0), s12 = r1 (f2 - f1), s23 = r2 (f3 - f2)
      const R al = first ? R(1) : R(0.5), be = first ? R(0) : R(0.5), ga = last ? R(1) : R(0.5),
              de = last ? R(0) : R(0.5);
      const R m12 = (c1 * al + c3 * ga) * r[1];
      const R ax[4] = {-c1 * be * r[0], c0 + c1 * be * r[0] - m12, c2 + m12 - c3 * de * r[2], c3 * de * r[2]};
      R cc[16];
      size_t off[16];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = j0 + t;
        const bool in = j >= 0 && j < nq;
        const int jr = min(max(j, 0), nq - 1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cc[4 * t + u] = in ? w[t] * ax[u] : R(0);
          off[4 * t + u] = size_t(jr) * nx + ii[u];
        }
      }
      const size_t fstride = size_t(nq) * nx;
      for (int fl = 0; fl < nfl; ++fl) {
        const size_t base = size_t(fl) * fstride;
        R acc = R(0);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          acc += cc[e] * (sizeof(R) == 8 ? R(pdf.xf64[base + off[e]]) : R(pdf.xf32[base + off[e]]));
        mine[fl] = double(acc);
      }
    }
  }
  __syncthreads();
  const long long npts = n - i0 < kPdfBlock ? n - i0 : kPdfBlock;
  double* dst = out + i0 * nfl;
  for (int k = threadIdx.x; k < npts * nfl; k += kPdfBlock) dst[k] = sh_xf[k];
}

// Helpers of the FP32 path that keep it off the FP64 pipe (on B300 about
// 1/64 of the FP32 rate, f32 <-> f64 conversions included):
// positive doubles order like their bit patterns read as integers
MC_D bool pos_f64_le(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
// log v in FP32 for a positive normal double, from its binary exponent and
// its significand cut to 23 bits: e ln 2 + log m, m in [1, 2)
MC_D float log_f64_to_f32(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = int((b >> 52) & 0x7ff) - 1023;
  const float m = __uint_as_float(0x3f800000u | uint32_t((b >> 29) & 0x7fffffu));
  // e as a float without a conversion instruction: 1.5 2^23 + e has e in its
  // low significand bits (|e| < 2^22)
  const float ef = __int_as_float(0x4b400000 + e) - 12582912.0f;
  return ef * 0.693147180559945309f + logf(m);
}
// float -> double from the IEEE-754 fields (exactly, every class of value):
// normal numbers re-bias the exponent (127 -> 1023) and widen the
// significand; subnormals m 2^-149 are normalised at their leading bit p
// (exponent field p + 874); zeros keep their sign; infinities and NaN keep
// their significand bits
MC_D double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long bits;
  if (e == 0xffu) {
    bits = sign | 0x7ff0000000000000ull | (unsigned long long)m << 29;
  } else if (e != 0u) {
    bits = sign | (unsigned long long)(e + 896u) << 52 | (unsigned long long)m << 29;
  } else if (m == 0u) {
    bits = sign;
  } else {
    const int p = 31 - __clz(m);
    bits = sign | (unsigned long long)(p + 874) << 52 | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double((long long)bits);
}
// largest i in [0, n-2] with t[i] <= v
MC_D int knot_cell_f(const float* t, int n, float v) {
  int lo = 0, hi = n - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// FP32 batch interpolation with the whole grid in shared memory (when it
// fits, 188 KB for 100 x 40 knots and 11 flavours padded to 12): flavours
// innermost, so one 16-byte load brings four flavours of a knot.  Per point
// the sixteen (Q, x) stencil knots combine with coefficients formed once: the
// Q weights times the x Hermite weights of the four x knots (the knot slopes
// written out as differences, one-sided at the grid's ends), so each flavour
// costs sixteen multiply-adds.  The knots and their reciprocal spacings are
// kept in FP32 in shared memory too, and nothing in the loop runs on the FP64
// pipe.  One block of kPdfThreads per SM; every warp walks its own chunks of
// 32 points (chunk c = points 32 c .. 32 c + 31, warp w of the grid takes
// chunks w, w + W, ...) with no block-wide barrier, loading the next chunk's
// queries while it evaluates the current one; outputs are staged in FP32 per
// warp and widened to FP64 as the warp writes its chunk out as one contiguous
// range.
constexpr int kPdfThreads = 512;
constexpr int kPdfWarps = kPdfThreads / 32;
constexpr int kPdfLut = 256;  // entries of each knot lookup table
constexpr size_t kPdfSmemMax = 224 * 1024;
// shared memory: the grid, per warp its FP32 output staging (32 x nflav,
// which holds the chunk's gather order before the outputs), the knots and
// their reciprocal spacings, the two lookup tables
inline size_t pdf_smem_bytes(const PdfDev& p) {
  return size_t(p.nq) * p.nx * p.nfp * 4 + size_t(kPdfWarps) * 32 * p.nflav * 4 + 8 * size_t(p.nx + p.nq) +
         2 * size_t(kPdfLut) * 4;
}

// The same cell as knot_cell_f (t strictly increasing, t[0] <= v <= t[n-1]):
// lut[b] is the cell of t[0] + b (t[n-1] - t[0]) / kPdfLut, and from the
// entry of v's step a walk (at most n steps, one or none on grids whose
// spacing varies less than the steps) reaches the largest i in [0, n-2] with
// t[i] <= v.
MC_D int knot_cell_lut(const float* t, const int* lut, int n, float v, float inv_step) {
  const int b = min(max(int((v - t[0]) * inv_step), 0), kPdfLut - 1);
  int i = lut[b];
  while (i < n - 2 && t[i + 1] <= v) ++i;
  while (i > 0 && t[i] > v) --i;
  return i;
}

// Points of a chunk are gathered in an order that spreads the 16-byte bank
// groups: the stencil of a point starts at float4 index base = (row of its
// first Q knot x nx + its first x knot) x nfp / 4 and its sixteen loads sit at
// offsets common to all interior points, so when the 8 lanes of a
// quarter-warp hold points with distinct base mod 8 every load of the
// quarter-warp is one wavefront.  Each lane finds its point's cells and key
// (base mod 8) and its rank within its key (warp ballots); the gather order
// interleaves the keys rank by rank (position = sum over keys of
// min(count, rank) + the keys below its own that still have a point of that
// rank).  The lane at a position evaluates that point and writes its outputs
// to the point's own staging row, so results and output order do not depend
// on the order.  (A quarter-warp pays the largest multiplicity of a key among
// its 8 lanes; the most frequent of the 8 keys among 32 random points occurs
// about 7.5 times, so a stencil load costs about 8 wavefronts per warp
// instead of 4 whatever the order.  Chunks of 64 points on 12 warps, which
// the shared memory allows, measured slower.)
__global__ void __launch_bounds__(kPdfThreads, 1) pdf_xfxq2_smem_kernel(PdfDev pdf, long long n, const double* x,
                                                                        const double* q2, double* out) {
  extern __shared__ __align__(16) unsigned char pdf_smem[];
  float4* tab = reinterpret_cast<float4*>(pdf_smem);
  const int nx = pdf.nx, nq = pdf.nq, nfl = pdf.nflav, nf4 = pdf.nfp / 4;
  float* stage_all = reinterpret_cast<float*>(pdf_smem + size_t(nq) * nx * pdf.nfp * 4);  // [warps][32][nfl]
  float* lxf = stage_all + size_t(kPdfWarps) * 32 * nfl;  // [nx] knots, [nx] 1/spacing
  float* rxf = lxf + nx;
  float* lqf = rxf + nx;  // [nq], [nq]
  float* rqf = lqf + nq;
  int* lutx = reinterpret_cast<int*>(rqf + nq);  // [kPdfLut], [kPdfLut]
  int* lutq = lutx + kPdfLut;
  {
    const float4* g = reinterpret_cast<const float4*>(pdf.xf32t);
    const int n4 = nq * nx * nf4;
    for (int k = threadIdx.x; k < n4; k += kPdfThreads) tab[k] = g[k];
    for (int k = threadIdx.x; k < nx; k += kPdfThreads) {
      lxf[k] = float(pdf.logx[k]);
      rxf[k] = k + 1 < nx ? float(1.0 / (pdf.logx[k + 1] - pdf.logx[k])) : 0.0f;
    }
    for (int k = threadIdx.x; k < nq; k += kPdfThreads) {
      lqf[k] = float(pdf.logq2[k]);
      rqf[k] = k + 1 < nq ? float(1.0 / (pdf.logq2[k + 1] - pdf.logq2[k])) : 0.0f;
    }
  }
  __syncthreads();
  const float stx = (lxf[nx - 1] - lxf[0]) / float(kPdfLut), stq = (lqf[nq - 1] - lqf[0]) / float(kPdfLut);
  for (int b = threadIdx.x; b < kPdfLut; b += kPdfThreads) {
    lutx[b] = knot_cell_f(lxf, nx, lxf[0] + float(b) * stx);
    lutq[b] = knot_cell_f(lqf, nq, lqf[0] + float(b) * stq);
  }
  __syncthreads();
  const float inv_stx = 1.0f / stx, inv_stq = 1.0f / stq;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + size_t(warp) * 32 * nfl;
  int* perm = reinterpret_cast<int*>(stage);  // [32], read before the outputs are staged
  const long long nchunks = (n + 31) / 32;
  const long long nw = (long long)gridDim.x * kPdfWarps;
  long long c = (long long)blockIdx.x * kPdfWarps + warp;
  double xv = 0.0, qv = 0.0;  // this lane's query of chunk c
  if (c < nchunks && c * 32 + lane < n) {
    xv = x[c * 32 + lane];
    qv = q2[c * 32 + lane];
  }
  for (; c < nchunks; c += nw) {
    const long long i0 = c * 32;
    const int npts = int(n - i0 < 32 ? n - i0 : 32);
    const bool act = lane < npts;
    const double xc = xv, qc = qv;
    if (c + nw < nchunks && (c + nw) * 32 + lane < n) {  // the next chunk's query, in flight meanwhile
      xv = x[(c + nw) * 32 + lane];
      qv = q2[(c + nw) * 32 + lane];
    }
    // cells and key of this lane's point (ix = -1: outside the grid)
    float lx = 0.0f, lq = 0.0f;
    int ix = -1, iq = -1, key = 0;
    // x_lo, q2_lo > 0, so a NaN or a negative query fails one of the tests
    if (act && pos_f64_le(pdf.x_lo, xc) && pos_f64_le(xc, pdf.x_hi) && pos_f64_le(pdf.q2_lo, qc) &&
        pos_f64_le(qc, pdf.q2_hi)) {
      lx = fminf(fmaxf(log_f64_to_f32(xc), lxf[0]), lxf[nx - 1]);
      lq = fminf(fmaxf(log_f64_to_f32(qc), lqf[0]), lqf[nq - 1]);
      iq = knot_cell_lut(lqf, lutq, nq, lq, inv_stq);
      ix = knot_cell_lut(lxf, lutx, nx, lx, inv_stx);
      key = ((max(iq - 1, 0) * nx + max(ix - 1, 0)) * nf4) & 7;
    }
    // gather order
    int cnt[8];
    unsigned mine_keys = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, act && key == k);
      cnt[k] = __popc(m);
      if (key == k) mine_keys = m;
    }
    if (act) {
      const int rank = __popc(mine_keys & ((1u << lane) - 1u));
      int pos = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) pos += min(cnt[k], rank) + (k < key && cnt[k] > rank ? 1 : 0);
      perm[pos] = lane;
    }
    __syncwarp();
    // the point at this lane's position in the gather order
    const int pt = act ? perm[lane] : lane;
    __syncwarp();  // the gather order is read: the staging rows may be written
    const float plx = __shfl_sync(0xffffffffu, lx, pt), plq = __shfl_sync(0xffffffffu, lq, pt);
    const int pix = __shfl_sync(0xffffffffu, ix, pt), piq = __shfl_sync(0xffffffffu, iq, pt);
    if (act) {
      float* mine = stage + pt * nfl;
      if (pix < 0) {
        for (int fl = 0; fl < nfl; ++fl) mine[fl] = __int_as_float(0x7fc00000);
      } else {
        // Q weights of the knots j0 .. j0+3 (as q_weights)
        const int j0 = piq - 1;
        float w[4];
        {
          const float hq = lqf[piq + 1] - lqf[piq];
          const float tq = (plq - lqf[piq]) * rqf[piq];
          const float q2_ = tq * tq, q3 = q2_ * tq;
          w[0] = 0.0f;
          w[1] = 2.0f * q3 - 3.0f * q2_ + 1.0f;
          w[2] = -2.0f * q3 + 3.0f * q2_;
          w[3] = 0.0f;
          auto add_slope = [&](int k, float coef) {
            const int b = k - j0;
            if (k == 0) {
              w[b] -= coef * rqf[0];
              w[b + 1] += coef * rqf[0];
            } else if (k == nq - 1) {
              w[b] += coef * rqf[k - 1];
              w[b - 1] -= coef * rqf[k - 1];
            } else {
              w[b + 1] += 0.5f * coef * rqf[k];
              w[b] += 0.5f * coef * (rqf[k - 1] - rqf[k]);
              w[b - 1] -= 0.5f * coef * rqf[k - 1];
            }
          };
          add_slope(piq, (q3 - 2.0f * q2_ + tq) * hq);
          add_slope(piq + 1, (q3 - q2_) * hq);
        }
        const float h = lxf[pix + 1] - lxf[pix];
        const float tau = (plx - lxf[pix]) * rxf[pix];
        int ii[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) ii[t] = min(max(pix - 1 + t, 0), nx - 1);
        const float r[3] = {pix >= 1 ? rxf[pix - 1] : 0.0f, rxf[pix], pix + 2 <= nx - 1 ? rxf[pix + 1] : 0.0f};
        const bool first = pix == 0, last = pix + 1 == nx - 1;
        const float t2 = tau * tau, t3 = t2 * tau;
        const float c0 = 2.0f * t3 - 3.0f * t2 + 1.0f, c1 = (t3 - 2.0f * t2 + tau) * h, c2 = -2.0f * t3 + 3.0f * t2,
                    c3 = (t3 - t2) * h;
        // slopes d0 = al s12 + be s01, d1 = ga s12 + de s23 (one-sided at the ends),
        // s01 = r0 (f1 - f0), s12 = r1 (f2 - f1), s23 = r2 (f3 - f2)
        const float al = first ? 1.0f : 0.5f, be = first ? 0.0f : 0.5f, ga = last ? 1.0f : 0.5f,
                    de = last ? 0.0f : 0.5f;
        const float m12 = (c1 * al + c3 * ga) * r[1];
        const float a[4] = {-c1 * be * r[0], c0 + c1 * be * r[0] - m12, c2 + m12 - c3 * de * r[2], c3 * de * r[2]};
        float cc[16];
        int off[16];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = j0 + t;
          const bool in = j >= 0 && j < nq;
          const int jr = min(max(j, 0), nq - 1);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            cc[4 * t + u] = in ? w[t] * a[u] : 0.0f;
            off[4 * t + u] = (jr * nx + ii[u]) * nf4;
          }
        }
        for (int k = 0; k < nf4; ++k) {
          float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float4 f = tab[off[e] + k];
            acc.x = fmaf(cc[e], f.x, acc.x);
            acc.y = fmaf(cc[e], f.y, acc.y);
            acc.z = fmaf(cc[e], f.z, acc.z);
            acc.w = fmaf(cc[e], f.w, acc.w);
          }
          const float v4_[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (4 * k + q < nfl) mine[4 * k + q] = v4_[q];
        }
      }
    }
    __syncwarp();
    double* dst = out + i0 * nfl;
    for (int k = lane; k < npts * nfl; k += 32) dst[k] = f32_to_f64(stage[k]);
    __syncwarp();
  }
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
  k<<<grid, ws_threads(PROC), smem, st>>>(a);
  return cudaGetLastError();
}

// the points-input instance (no weights pass, no row store)
template <int PROC>
static cudaError_t launch_points(const KernelArgs& a, int grid, cudaStream_t st) {
  auto k = ws_integrand_kernel<PROC, false, false, true>;
  const size_t smem = ws_smem_bytes(PROC, a.ndim, 0, a.pdf.nx, false);
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, ws_threads(PROC), smem, st>>>(a);
  return cudaGetLastError();
}

bool points_ws(int proc) { return proc == P_GG_TTBARG || proc == P_GG_TTBARG_7D || proc == P_PP_TTBARJ; }
cudaError_t launch_points_ws(int proc, const KernelArgs& a, int grid, cudaStream_t st) {
  if (!points_ws(proc) || !a.pts || a.nbins != 0 || !a.partials || a.wout || grid < 1 || a.n < 0)
    return cudaErrorInvalidValue;
  return proc == P_GG_TTBARG      ? launch_points<P_GG_TTBARG>(a, grid, st)
         : proc == P_GG_TTBARG_7D ? launch_points<P_GG_TTBARG_7D>(a, grid, st)
                                  : launch_points<P_PP_TTBARJ>(a, grid, st);
}

bool integrand_ws(int proc, bool fp64) {
  return !fp64 && (proc == P_GG_TTBARG || proc == P_GG_TTBARG_7D || proc == P_GG_TTBARG_MC || proc == P_PP_TTBARJ);
}
int integrand_threads(int proc, bool fp64) { return integrand_ws(proc, fp64) ? ws_threads(proc) : kBlock; }
// events one block takes per round of its grid-stride loop
int integrand_block_events(int proc, bool fp64) {
  return integrand_ws(proc, fp64) ? 32 * ws_producer_warps(proc) : kBlock;
}

template <bool RECORD>
static cudaError_t dispatch(int proc, bool fp64, const KernelArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (!RECORD && integrand_ws(proc, fp64))
    return proc == P_GG_TTBARG      ? launch_ws<P_GG_TTBARG>(a, grid, st)
           : proc == P_GG_TTBARG_7D ? launch_ws<P_GG_TTBARG_7D>(a, grid, st)
           : proc == P_PP_TTBARJ    ? launch_ws<P_PP_TTBARJ>(a, grid, st)
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
  const size_t smem = sizeof(double) * size_t(3 * nbins + 2);
  (void)cudaGetLastError();
  refine_kernel<<<ndim, 32, smem, st>>>(edges, edges32, hist_w2, hist_n, ndim, nbins, alpha);
  return cudaGetLastError();
}
cudaError_t launch_pdf_xfxq2(const PdfDev& pdf, bool fp64, long long n, const double* x, const double* q2,
                             double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  (void)cudaGetLastError();
  if (!fp64 && pdf.xf32t && pdf_smem_bytes(pdf) <= kPdfSmemMax) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = ((n + 31) / 32 + kPdfWarps - 1) / kPdfWarps;
    const int grid = int(blocks < sms ? blocks : sms);
    const size_t smem = pdf_smem_bytes(pdf);
    const cudaError_t e =
        cudaFuncSetAttribute(pdf_xfxq2_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    pdf_xfxq2_smem_kernel<<<grid, kPdfThreads, smem, st>>>(pdf, n, x, q2, out);
    return cudaGetLastError();
  }
  const long long grid = (n + kPdfBlock - 1) / kPdfBlock;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t smem = size_t(kPdfBlock) * pdf.nflav * sizeof(double);  // nflav <= 64: at most 64 KB
  auto k = fp64 ? pdf_xfxq2_kernel<double> : pdf_xfxq2_kernel<float>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k<<<unsigned(grid), kPdfBlock, smem, st>>>(pdf, n, x, q2, out);
  return cudaGetLastError();
}

}  // namespace mc
