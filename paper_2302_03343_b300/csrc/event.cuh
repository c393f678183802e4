// One event of the fused path and the block-level reduction of the per-thread
// accumulators; shared by the single-integrand kernel and the persistent
// multi-integrand kernel.
#pragma once
#include <type_traits>

#include "../../include/mcint.h"
#include "integrand.cuh"

namespace mc {

// Per-thread accumulators: Kahan-compensated FP64 sums of w and w^2.
struct Acc {
  double s_hi = 0.0, s_c = 0.0, q_hi = 0.0, q_c = 0.0, wmax = 0.0;
  unsigned int nnz = 0, nbad = 0, nnoconv = 0;  // per thread: below 2^32 events
};

// value = hi + lo pairs: compensated addition of two such pairs
MC_HD void pair_add(double& hi, double& lo, double h2, double l2) {
  const double s = hi + h2;
  const double bp = s - hi;
  const double e = (hi - (s - bp)) + (h2 - bp);
  hi = s;
  lo = lo + l2 + e;
}

MC_HD void partial_add(BlockPartial& b, const BlockPartial& o) {
  pair_add(b.sum_hi, b.sum_lo, o.sum_hi, o.sum_lo);
  pair_add(b.sum2_hi, b.sum2_lo, o.sum2_hi, o.sum2_lo);
  b.wmax = fmax(b.wmax, o.wmax);
  b.n_nonzero += o.n_nonzero;
  b.n_bad += o.n_bad;
  b.n_noconv += o.n_noconv;
}

// Uniforms -> VEGAS map (grid in shared memory) -> integrand -> weight, then
// the Kahan sums and the shared-memory histograms (or, with RECORD, the
// per-event record `rec`).  H is the histogram accumulation type.  Returns
// the event's weight (0 when it is cut or its weight is not finite).
template <int PROC, bool FP64, bool RECORD, class R, class H>
MC_D double process_event(const KernelArgs& a, const SmPdf<R>& pdf, const R* sh_edges, H* sh_w2, unsigned int* sh_n,
                          uint64_t ev, double* rec, Acc& acc) {
  constexpr int MAXD = ProcTraits<PROC>::MAXD;
  const int ndim = a.ndim, nb = a.nbins;
  uint64_t k[MAXD];
  event_uniforms<MAXD, FP64>(a.seed, a.iteration, a.gid, ev, ndim, k);
  R x[MAXD];
  int bin[MAXD];
  // bin indices (< 256) packed four to a word while the integrand runs
  uint32_t binw[(MAXD + 3) / 4];
#pragma unroll
  for (int j = 0; j < (MAXD + 3) / 4; ++j) binw[j] = 0u;
  R jac = R(1);
#pragma unroll
  for (int dd = 0; dd < MAXD; ++dd) {
    if (dd < ndim) {
      R jd;
      x[dd] = vegas_map_1d<R, FP64>(sh_edges + dd * (nb + 1), nb, k[dd], &bin[dd], &jd);
      binw[dd / 4] |= uint32_t(bin[dd]) << (8 * (dd % 4));
      jac *= jd;
    }
  }
  const EventOut o = integrand<PROC, R>(a, pdf, x, rec);
  double w = o.f * double(jac);
  int status = o.status;
  if (!isfinite(w)) {
    status = MC_ENAN;
    w = 0.0;
  }
  if (RECORD) {
#pragma unroll
    for (int dd = 0; dd < MAXD; ++dd) {
      if (dd < ndim) {
        rec[MC_REC_K + dd] = double(k[dd]);
        rec[MC_REC_X + dd] = double(x[dd]);
        rec[MC_REC_BIN + dd] = double(bin[dd]);
      }
    }
    rec[MC_REC_JAC] = double(jac);
    rec[MC_REC_F] = o.f;
    rec[MC_REC_W] = w;
    rec[MC_REC_PASS] = double(o.pass);
    rec[MC_REC_STATUS] = double(status);
    return w;
  }
  if (status != 0) {
    if (status == -5)
      ++acc.nnoconv;
    else
      ++acc.nbad;
  }
  const double y = w - acc.s_c;
  const double t = acc.s_hi + y;
  acc.s_c = (t - acc.s_hi) - y;
  acc.s_hi = t;
  const double w2 = w * w;
  const double y2 = w2 - acc.q_c;
  const double t2 = acc.q_hi + y2;
  acc.q_c = (t2 - acc.q_hi) - y2;
  acc.q_hi = t2;
  if (w != 0.0) ++acc.nnz;
  acc.wmax = fmax(acc.wmax, w);
#pragma unroll
  for (int dd = 0; dd < MAXD; ++dd) {
    if (dd < ndim) {
      const int b = int((binw[dd / 4] >> (8 * (dd % 4))) & 0xffu);
      atomicAdd(&sh_w2[dd * nb + b], H(w2));
      atomicAdd(&sh_n[dd * nb + b], 1u);
    }
  }
  return w;
}

// Block reduction of the accumulators (warp shuffles, then thread 0 over the
// warps in order); the result is written by thread 0 to *out.  warp_part holds
// blockDim.x / 32 entries.  Contains __syncthreads.
MC_D void block_reduce(Acc acc, BlockPartial* warp_part, BlockPartial* out) {
  double s_hi = acc.s_hi, lo = -acc.s_c, q_hi = acc.q_hi, lo2 = -acc.q_c, wmax = acc.wmax;
  long long nnz = acc.nnz, nbad = acc.nbad, nnoconv = acc.nnoconv;
  for (int off = 16; off > 0; off >>= 1) {
    const double h2 = __shfl_xor_sync(0xffffffffu, s_hi, off), l2 = __shfl_xor_sync(0xffffffffu, lo, off);
    pair_add(s_hi, lo, h2, l2);
    const double g2 = __shfl_xor_sync(0xffffffffu, q_hi, off), m2 = __shfl_xor_sync(0xffffffffu, lo2, off);
    pair_add(q_hi, lo2, g2, m2);
    wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, off));
    nnz += __shfl_xor_sync(0xffffffffu, nnz, off);
    nbad += __shfl_xor_sync(0xffffffffu, nbad, off);
    nnoconv += __shfl_xor_sync(0xffffffffu, nnoconv, off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_part[wid] = {s_hi, lo, q_hi, lo2, wmax, nnz, nbad, nnoconv};
  __syncthreads();
  if (threadIdx.x == 0) {
    BlockPartial b = warp_part[0];
    for (int w = 1; w < int(blockDim.x / 32); ++w) partial_add(b, warp_part[w]);
    *out = b;
  }
  __syncthreads();
}

}  // namespace mc
