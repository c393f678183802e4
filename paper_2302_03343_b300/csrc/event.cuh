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
  double wch[kChannels] = {0.0, 0.0, 0.0};      // three-channel process: sums of w^2 p_i / p
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

// Kahan sums, count and maximum of one event's weight.
MC_D void acc_add(Acc& acc, double w) {
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
}

// The kinematic part of one three-channel gg -> t tbar g event (thesis Sec.
// "Multi-channel Monte Carlo"): the channel from Philox call 254, the 7
// uniforms through the (x1, x2) grid and that channel's grid, the channel's
// map, the densities of all three channels at the point (the others by
// their inverse maps and grid densities), the lab-frame gluon cuts and the
// gluon luminosity.  kin.psw = 1 / sum_j alpha_j p_j, so that the weight is
// gg_weight(kin, |M|^2) * jx.
template <class R>
struct McEvent {
  int ch, pass;
  uint64_t k[7];
  R x[7];
  int bin[7];
  R jx, jrest;
  double dens[kChannels], pden;
  GgKin<R> kin;
};

template <bool FP64, class R>
MC_D void mc_prepare(const KernelArgs& a, const SmPdf<R>& pdf, const R* sh_edges, uint64_t ev, McEvent<R>& e) {
  constexpr int ND = 7;
  const int nb = a.nbins;
  const uint4 cw = philox4x32_10(make_uint4(uint32_t(ev), uint32_t(ev >> 32), a.iteration,
                                            (a.gid & 0xffu) | (254u << 8)),
                                 make_uint2(uint32_t(a.seed), uint32_t(a.seed >> 32)));
  const double uc = (double(cw.x >> 8) + 0.5) * 0x1p-24;
  const int ch = uc < a.alpha_cum[0] ? 0 : (uc < a.alpha_cum[1] ? 1 : 2);
  e.ch = ch;
  e.pass = 0;
  event_uniforms<ND, FP64>(a.seed, a.iteration, a.gid, ev, ND, e.k);
  e.jx = R(1);
  e.jrest = R(1);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    R jd;
    e.x[d] = vegas_map_1d<R, FP64>(sh_edges + ch_grid_dim(d, ch) * (nb + 1), nb, e.k[d], &e.bin[d], &jd);
    if (d < 2) e.jx *= jd; else e.jrest *= jd;
  }
  const Params& p = a.prm;
  const R m = R(p.m_top);
  const R x1 = e.x[0], x2 = e.x[1];
  const R shat = sizeof(R) == 4 ? R(x1 * x2 * R(p.sqrt_s * p.sqrt_s)) : R(double(x1) * double(x2) * p.sqrt_s * p.sqrt_s);
  e.dens[0] = e.dens[1] = e.dens[2] = 0.0;
  e.pden = 0.0;
  e.kin.shat = shat;
  e.kin.k[0] = e.kin.k[1] = e.kin.k[2] = v4<R>{R(0), R(0), R(0), R(0)};
  if (!(shat > R(4) * m * m)) return;
  const R rs = m_sqrt(shat);
  e.kin.rs = rs;
  const ChCtx<R> c = ch_ctx<R>(m, rs, R(p.ptcut_g), R(p.etacut_g), R(0.5) * m_log(x1 / x2));
  v4<R>& t = e.kin.k[0];
  v4<R>& tb = e.kin.k[1];
  v4<R>& g = e.kin.k[2];
  R wi;
  if (!ch_forward<R>(ch, c, e.x + 2, &t, &tb, &g, &wi) || !(wi > R(0))) return;
  e.dens[ch] = 1.0 / (double(e.jrest) * double(wi));
#pragma unroll
  for (int j = 0; j < kChannels; ++j) {
    if (j == ch) continue;
    R uj[5], wj;
    if (ch_inverse<R>(j, c, t, tb, g, uj, &wj) && wj > R(0)) {
      R rho = R(1);
#pragma unroll
      for (int d = 0; d < 5; ++d) rho *= grid_density<R>(sh_edges + ch_grid_dim(d + 2, j) * (nb + 1), nb, uj[d]);
      e.dens[j] = double(rho) / double(wj);
    }
  }
  e.pden = a.alpha[0] * e.dens[0] + a.alpha[1] * e.dens[1] + a.alpha[2] * e.dens[2];
  // the gluon cuts in the lab frame (pT, and |eta_cm + y_b| < cut without logarithms)
  const R pt2 = g.x * g.x + g.y * g.y, ptc = R(p.ptcut_g);
  const R pabs = m_sqrt(pt2 + g.z * g.z);
  const R fwd = (pabs + g.z) * x1, bwd = (pabs - g.z) * x2, e2 = R(a.e2eta);
  if (!(pt2 > ptc * ptc && fwd < e2 * bwd && bwd < e2 * fwd)) return;
  e.pass = 1;
  e.kin.lgg = xf_over_x(pdf.tab[0], x1) * xf_over_x(pdf.tab[0], x2);
  e.kin.flux = sizeof(R) == 4 ? R(p.gev2pb) / (R(2) * shat) : R(0);
  e.kin.psw = 1.0 / e.pden;
}

// One three-channel event: mc_prepare, |M|^2 and w = f J_x / sum_j alpha_j
// p_j, then the sums, the alpha-update sums and the histograms of the grid
// dimensions used (or, with RECORD, the per-event record).
template <bool FP64, bool RECORD, class R, class H>
MC_D double process_event_mc(const KernelArgs& a, const SmPdf<R>& pdf, const R* sh_edges, H* sh_w2,
                             unsigned int* sh_n, uint64_t ev, double* rec, Acc& acc) {
  constexpr int ND = 7;
  const int nb = a.nbins;
  McEvent<R> e;
  mc_prepare<FP64, R>(a, pdf, sh_edges, ev, e);
  double w = 0.0;
  R me2 = R(0);
  if (e.pass) {
    me2 = gg_me2<R>(a, e.kin);
    w = gg_weight<R>(a, e.kin, me2) * double(e.jx);
  }
  int status = 0;
  if (!isfinite(w)) {
    status = MC_ENAN;
    w = 0.0;
  }
  if (RECORD) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      rec[MC_REC_K + d] = double(e.k[d]);
      rec[MC_REC_X + d] = double(e.x[d]);
      rec[MC_REC_BIN + d] = double(e.bin[d]);
    }
    const R h = m_sqrt(m_max(e.kin.shat, R(0))) * R(0.5);
    rec_p4(rec, 0, v4<R>{h, R(0), R(0), h});
    rec_p4(rec, 1, v4<R>{h, R(0), R(0), -h});
    rec_p4(rec, 2, e.kin.k[0]);
    rec_p4(rec, 3, e.kin.k[1]);
    rec_p4(rec, 4, e.kin.k[2]);
    rec[MC_REC_X1] = double(e.x[0]);
    rec[MC_REC_X2] = double(e.x[1]);
    rec[MC_REC_SHAT] = double(e.kin.shat);
    rec[MC_REC_LUMI] = e.pass ? double(e.kin.lgg) : 0.0;
    rec[MC_REC_ME2] = double(me2);
    rec[MC_REC_PSW] = e.pden > 0.0 ? 1.0 / e.pden : 0.0;
    rec[MC_REC_JAC] = double(e.jx) * double(e.jrest);
    rec[MC_REC_F] = w / double(e.jx);
    rec[MC_REC_W] = w;
    rec[MC_REC_PASS] = double(e.pass);
    rec[MC_REC_STATUS] = double(status);
    rec[MC_REC_CHANNEL] = double(e.ch);
#pragma unroll
    for (int j = 0; j < kChannels; ++j) rec[MC_REC_DENS + j] = e.dens[j];
    return w;
  }
  if (status != 0) ++acc.nbad;
  acc_add(acc, w);
  if (w != 0.0) {
    const double w2p = w * w / e.pden;
#pragma unroll
    for (int j = 0; j < kChannels; ++j) acc.wch[j] += w2p * e.dens[j];
  }
  const H w2h = H(w * w);
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int gd = ch_grid_dim(d, e.ch);
    atomicAdd(&sh_w2[gd * nb + e.bin[d]], w2h);
    atomicAdd(&sh_n[gd * nb + e.bin[d]], 1u);
  }
  return w;
}

// Uniforms -> VEGAS map (grid in shared memory) -> integrand -> weight, then
// the Kahan sums and the shared-memory histograms (or, with RECORD, the
// per-event record `rec`).  H is the histogram accumulation type.  Returns
// the event's weight (0 when it is cut or its weight is not finite).
template <int PROC, bool FP64, bool RECORD, class R, class H>
MC_D double process_event_one(const KernelArgs& a, const SmPdf<R>& pdf, const R* sh_edges, H* sh_w2,
                              unsigned int* sh_n, uint64_t ev, double* rec, Acc& acc) {
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

template <int PROC, bool FP64, bool RECORD, class R, class H>
MC_D double process_event(const KernelArgs& a, const SmPdf<R>& pdf, const R* sh_edges, H* sh_w2, unsigned int* sh_n,
                          uint64_t ev, double* rec, Acc& acc) {
  if constexpr (PROC == P_GG_TTBARG_MC)
    return process_event_mc<FP64, RECORD, R, H>(a, pdf, sh_edges, sh_w2, sh_n, ev, rec, acc);
  else
    return process_event_one<PROC, FP64, RECORD, R, H>(a, pdf, sh_edges, sh_w2, sh_n, ev, rec, acc);
}

// Adds the block's alpha-update sums (three-channel process) to out[3]:
// warp shuffles, then one FP64 atomic per warp and channel.
MC_D void channel_sums_add(const Acc& acc, double* out) {
#pragma unroll
  for (int j = 0; j < kChannels; ++j) {
    double v = acc.wch[j];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&out[j], v);
  }
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
