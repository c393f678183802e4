// The per-event integrand (thesis Sec. "The MadFlow event generator",
// eq. mc_master_formula) with the flux factor and the unit conversion made
// explicit:
//   f = sum_ab f_a(x1) f_b(x2) <|M_ab|^2> / (2 shat) * w_PS * gev2pb,
// f_a = (x f_a)(x, mu_F^2) / x.  The VEGAS event weight is f * J.
#pragma once
#include "matrix_elements.cuh"
#include "pdf.cuh"
#include "phasespace.cuh"
#include "channels.cuh"
#include "sampling.cuh"

namespace mc {

enum : int {
  P_EE_MUMU = 0, P_PP_TTBAR = 1, P_GG_TTBARG = 2, P_GAUSS = 3, P_GG_TTBARG_7D = 4, P_GG_TTBARG_MC = 5, P_PP_TTBARJ = 6
};

template <int PROC> struct ProcTraits;
template <> struct ProcTraits<P_EE_MUMU> { static constexpr int MAXD = 2, NFL = 0; };
template <> struct ProcTraits<P_PP_TTBAR> { static constexpr int MAXD = 4, NFL = 11; };
template <> struct ProcTraits<P_GG_TTBARG> { static constexpr int MAXD = 14, NFL = 1; };
template <> struct ProcTraits<P_GAUSS> { static constexpr int MAXD = 16, NFL = 0; };
template <> struct ProcTraits<P_GG_TTBARG_7D> { static constexpr int MAXD = 7, NFL = 1; };
// three-channel gg -> t tbar g: 7 uniforms per event, 17 grid dimensions
template <> struct ProcTraits<P_GG_TTBARG_MC> { static constexpr int MAXD = 7, NFL = 1; };
// p p -> t tbar + parton: 7 dims, gluon and the five quark and antiquark flavours
template <> struct ProcTraits<P_PP_TTBARJ> { static constexpr int MAXD = 7, NFL = 11; };

// Arguments of one launch of the fused kernel (passed by value).
struct BlockPartial {
  double sum_hi, sum_lo, sum2_hi, sum2_lo, wmax;
  long long n_nonzero, n_bad, n_noconv;
};

struct KernelArgs {
  Params prm;
  int ndim, nbins;
  const double* edges64;  // [ndim][nbins+1]
  const float* edges32;
  PdfDev pdf;
  int fl[11];             // flavour indices used by the process (see ProcTraits::NFL)
  double logq2_f;         // log(mu_F^2)
  double w0_coef3;        // RAMBO flat-weight coefficient for three particles
  double e2eta;           // exp(2 * etacut_g)
  uint64_t seed;
  uint32_t iteration, gid;
  uint64_t first;
  long long n;
  BlockPartial* partials;  // [gridDim.x]
  double* hist_w2;         // [ndim][nbins]
  unsigned int* hist_n;    // [ndim][nbins]
  double* record;          // [n][MC_REC_STRIDE] (debug launches only)
  int* status;             // optional: MC_ETIMEOUT when a bounded wait of the launch gave up
  double* wout;            // optional, [n]: weight of every event (0 outside the cuts), weights pass
  // points input of the warp-specialised kernel (launch_points_ws): the
  // points pts [n][ndim] in the unit cube replace Philox and the VEGAS map
  // (nbins 0), and the weight is f exp(-pts_logq[i]) (pts_logq optional: f)
  const float* pts;
  const float* pts_logq;
  // three-channel process: cumulative channel probabilities (the channel of
  // an event is the first i with u < alpha_cum[i], u from Philox call 254),
  // the probabilities, and the alpha-update sums W_i (device, [3], added to)
  double alpha_cum[3], alpha[3];
  double* wch;
  // p p -> t tbar + parton: colour matrix of the light-line amplitudes
  // (me2_qline_ttbarg), re/im pairs, in FP64 and FP32
  double cqq[50];
  float cqqf[50];
};

// Shared-memory PDF tables of a launch.
template <class R>
struct SmPdf {
  PdfTable<R> tab[11];
};

template <class R> MC_D R xf_over_x(const PdfTable<R>& t, R x) { return pdf_interp_1d(t, m_log(x)) / x; }

struct EventOut {
  double f;
  int pass;
  int status;  // 0 or -5 (RAMBO rescaling failed)
};

MC_D void rec_put(double* rec, int off, double v) {
  if (rec) rec[off] = v;
}
template <class T> MC_D void rec_p4(double* rec, int slot, const v4<T>& p) {
  if (rec) {
    rec[49 + 4 * slot + 0] = double(p.e);
    rec[49 + 4 * slot + 1] = double(p.x);
    rec[49 + 4 * slot + 2] = double(p.y);
    rec[49 + 4 * slot + 3] = double(p.z);
  }
}

// gg -> t tbar g, split into the kinematic part (phase space, cuts, gluon
// luminosity) and the |M|^2 part so that the warp-specialised kernel can run
// them in different warps; the fused path calls the same three functions.
template <class R>
struct GgKin {
  v4<R> k[3];  // top, anti-top, gluon in the partonic frame
  R shat, rs;  // partonic s and its square root
  R lgg;       // g(x1) g(x2) / (x1 x2)
  R flux;      // gev2pb / (2 shat)
  double psw;  // phase-space weight
};

// Returns 1 when the event passes the cuts (kin filled), 0 when it fails
// them, -5 when RAMBO's rescaling did not converge.
template <int PROC, class R>
MC_D int gg_kinematics(const KernelArgs& a, const SmPdf<R>& pdf, const R* x, GgKin<R>* kin, double* rec) {
  const Params& p = a.prm;
  const double s = p.sqrt_s * p.sqrt_s;
  const R x1 = x[0], x2 = x[1];
  rec_put(rec, 77, x1); rec_put(rec, 78, x2);
  const R m = R(p.m_top);
  const R shat = sizeof(R) == 4 ? R(x1 * x2 * R(s)) : R(double(x1) * double(x2) * s);
  rec_put(rec, 79, shat);
  if (!(shat > R(4) * m * m)) return 0;
  const R rs = m_sqrt(shat);
  v4<R>* k = kin->k;
  double psw;
  int rc = 0;
  if constexpr (PROC == P_GG_TTBARG_7D) {
    v4<double> kd[3];
    hierarchical3<R>(double(m), double(rs), x + 2, kd, &psw);
    for (int i = 0; i < 3; ++i) k[i] = vcast<R>(kd[i]);
  } else if constexpr (sizeof(R) == 4) {
    // FP32 mode: FP64 only inside RAMBO's conformal transformation
    const float masses[3] = {m, m, 0.0f};
    rc = rambo_fp32<3>(masses, rs, a.w0_coef3, x + 2, k, &psw);
  } else {
    const double masses[3] = {double(m), double(m), 0.0};
    v4<double> kd[3];
    rc = rambo<R, 3>(masses, double(rs), a.w0_coef3, x + 2, kd, &psw);
    for (int i = 0; i < 3; ++i) k[i] = vcast<R>(kd[i]);
  }
  if (rec) {
    const v4<R> pa = {rs * R(0.5), R(0), R(0), rs * R(0.5)}, pb = {rs * R(0.5), R(0), R(0), -rs * R(0.5)};
    rec_p4(rec, 0, pa); rec_p4(rec, 1, pb); rec_p4(rec, 2, k[0]); rec_p4(rec, 3, k[1]); rec_p4(rec, 4, k[2]);
    rec_put(rec, 84, psw);
  }
  if (rc != 0) return -5;
  // gluon cuts in the lab frame: pT > cut and |eta_cm + y| < cut with
  // y = ln(x1/x2)/2, written without logarithms:
  // e^{-2c} (|p| - pz) x2 < (|p| + pz) x1 < e^{2c} (|p| - pz) x2.
  const v4<R>& g = k[2];
  const R pt2 = g.x * g.x + g.y * g.y;
  const R ptc = R(p.ptcut_g);
  if (!(pt2 > ptc * ptc)) return 0;
  const R pabs = m_sqrt(pt2 + g.z * g.z);
  const R fwd = (pabs + g.z) * x1, bwd = (pabs - g.z) * x2;
  const R e2 = R(a.e2eta);
  if (!(fwd < e2 * bwd && bwd < e2 * fwd)) return 0;
  kin->shat = shat;
  kin->rs = rs;
  kin->lgg = xf_over_x(pdf.tab[0], x1) * xf_over_x(pdf.tab[0], x2);
  kin->flux = sizeof(R) == 4 ? R(p.gev2pb) / (R(2) * shat) : R(0);
  kin->psw = psw;
  return 1;
}

// |M|^2 of an event that passed the cuts: packed FP32x2 arithmetic in FP32
// mode (me2_gg_ttbarg_rows with a shared-memory row store, me2_gg_ttbarg_p
// without), the precision-generic routine in FP64 mode.
template <class R, class Rows = NoRows>
MC_D R gg_me2(const KernelArgs& a, const GgKin<R>& kin, Rows rows = Rows{}) {
  const R h = kin.rs * R(0.5);
  const v4<R> pa = {h, R(0), R(0), h}, pb = {h, R(0), R(0), -h};
  const R m = R(a.prm.m_top), g2 = R(4.0 * kPi * a.prm.alpha_s);
  if constexpr (sizeof(R) == 4) {
    if constexpr (std::is_same<Rows, NoRows>::value)
      return me2_gg_ttbarg_p(pa, pb, kin.k[0], kin.k[1], kin.k[2], m, g2);
    else
      return me2_gg_ttbarg_rows(pa, pb, kin.k[0], kin.k[1], kin.k[2], m, g2, rows);
  } else {
    return me2_gg_ttbarg<R>(pa, pb, kin.k[0], kin.k[1], kin.k[2], m, g2);
  }
}

// f = L_gg <|M|^2> / (2 shat) * w_PS * gev2pb (the VEGAS Jacobian is applied
// by the caller).
template <class R>
MC_D double gg_weight(const KernelArgs& a, const GgKin<R>& kin, R me2) {
  if constexpr (sizeof(R) == 4)
    return double(kin.lgg * me2 * kin.flux) * kin.psw;
  else
    return double(kin.lgg) * double(me2) / (2.0 * double(kin.shat)) * kin.psw * a.prm.gev2pb;
}

// p p -> t tbar + parton, split like gg -> t tbar g for the warp-specialised
// kernel.  The kinematic part: every partonic channel at one point of the
// hierarchical three-body phase space (the light parton massless), the
// parton's cuts in the lab frame, and the seven channel luminosities summed
// over the five light flavours, lum = {gg, q qbar, qbar q, q g, g q,
// qbar g, g qbar}.  Returns 1 inside the cuts (kin and lum filled), else 0.
template <class R>
MC_D int ppj_kinematics(const KernelArgs& a, const SmPdf<R>& pdf, const R* x, GgKin<R>* kin, R* lum, double* rec) {
  const Params& p = a.prm;
  const double s = p.sqrt_s * p.sqrt_s;
  const R x1 = x[0], x2 = x[1];
  const R m = R(p.m_top);
  const R shat = sizeof(R) == 4 ? R(x1 * x2 * R(s)) : R(double(x1) * double(x2) * s);
  rec_put(rec, 77, x1); rec_put(rec, 78, x2); rec_put(rec, 79, shat);
  if (!(shat > R(4) * m * m)) return 0;
  const R rs = m_sqrt(shat);
  v4<double> kd[3];
  double psw;
  hierarchical3<R>(double(m), double(rs), x + 2, kd, &psw);
  for (int i = 0; i < 3; ++i) kin->k[i] = vcast<R>(kd[i]);
  kin->rs = rs;
  kin->shat = shat;
  kin->psw = psw;
  if (rec) {
    const v4<R> pa = {rs * R(0.5), R(0), R(0), rs * R(0.5)}, pb = {rs * R(0.5), R(0), R(0), -rs * R(0.5)};
    rec_p4(rec, 0, pa); rec_p4(rec, 1, pb); rec_p4(rec, 2, kin->k[0]); rec_p4(rec, 3, kin->k[1]);
    rec_p4(rec, 4, kin->k[2]);
    rec_put(rec, 84, psw);
  }
  // cuts on the light parton in the lab frame
  const v4<R>& pk = kin->k[2];
  const R pt2 = pk.x * pk.x + pk.y * pk.y, ptc = R(p.ptcut_g);
  const R pabs = m_sqrt(pt2 + pk.z * pk.z);
  const R fwd = (pabs + pk.z) * x1, bwd = (pabs - pk.z) * x2, e2 = R(a.e2eta);
  if (!(pt2 > ptc * ptc && fwd < e2 * bwd && bwd < e2 * fwd)) return 0;
  const R lx1 = m_log(x1), lx2 = m_log(x2);
  const R g1 = pdf_interp_1d(pdf.tab[0], lx1) / x1, g2x = pdf_interp_1d(pdf.tab[0], lx2) / x2;
  R q1 = R(0), qb1 = R(0), q2 = R(0), qb2 = R(0), lqq = R(0), lqbq = R(0);
#pragma unroll
  for (int f = 1; f <= 5; ++f) {
    const R a1 = pdf_interp_1d(pdf.tab[f], lx1) / x1, ab1 = pdf_interp_1d(pdf.tab[f + 5], lx1) / x1;
    const R a2 = pdf_interp_1d(pdf.tab[f], lx2) / x2, ab2 = pdf_interp_1d(pdf.tab[f + 5], lx2) / x2;
    q1 += a1; qb1 += ab1; q2 += a2; qb2 += ab2;
    lqq += a1 * ab2;
    lqbq += ab1 * a2;
  }
  lum[0] = g1 * g2x;
  lum[1] = lqq;
  lum[2] = lqbq;
  lum[3] = q1 * g2x;
  lum[4] = g1 * q2;
  lum[5] = qb1 * g2x;
  lum[6] = g1 * qb2;
  return 1;
}

// The |M|^2 part: gg -> t tbar g and the six light-quark channels at the
// event, weighted by the luminosities: f = sum_c lum_c <|M|^2>_c / (2 shat)
// * w_PS * gev2pb (the VEGAS Jacobian is applied by the caller).  me (may be
// null) receives the seven |M|^2 in the order of lum.
template <class R>
MC_D double ppj_weight(const KernelArgs& a, const GgKin<R>& kin, const R* lum, R* me) {
  const Params& p = a.prm;
  const R rs = kin.rs, m = R(p.m_top);
  const v4<R> pa = {rs * R(0.5), R(0), R(0), rs * R(0.5)}, pb = {rs * R(0.5), R(0), R(0), -rs * R(0.5)};
  const v4<R>& pt = kin.k[0];
  const v4<R>& ptb = kin.k[1];
  const v4<R>& pk = kin.k[2];
  const R g2c = R(4.0 * kPi * p.alpha_s);
  const R* cm;
  if constexpr (sizeof(R) == 4) cm = a.cqqf; else cm = a.cqq;
  const R me_gg = gg_me2<R>(a, kin);
  // the light-quark channels: packed complex arithmetic in FP32
  auto qline = [&](int kind, const v4<R>& x, const v4<R>& y) -> R {
    if constexpr (sizeof(R) == 4)
      return me2_qline_ttbarg_p(kind, x, y, pt, ptb, pk, m, g2c, cm);
    else
      return me2_qline_ttbarg<R>(kind, x, y, pt, ptb, pk, m, g2c, cm);
  };
  const R mq[6] = {qline(0, pa, pb), qline(0, pb, pa), qline(1, pa, pb),
                   qline(1, pb, pa), qline(2, pa, pb), qline(2, pb, pa)};
  const double sum = double(lum[0]) * double(me_gg) + double(lum[1]) * double(mq[0]) +
                     double(lum[2]) * double(mq[1]) + double(lum[3]) * double(mq[2]) + double(lum[4]) * double(mq[3]) +
                     double(lum[5]) * double(mq[4]) + double(lum[6]) * double(mq[5]);
  if (me) {
    me[0] = me_gg;
    for (int c = 0; c < 6; ++c) me[c + 1] = mq[c];
  }
  return sum / (2.0 * double(kin.shat)) * kin.psw * p.gev2pb;
}

// Integrand at the point x of the unit hypercube; rec (may be null) receives
// the intermediates in the MC_REC_* layout.
template <int PROC, class R>
MC_D EventOut integrand(const KernelArgs& a, const SmPdf<R>& pdf, const R* x, double* rec) {
  const Params& p = a.prm;
  EventOut out = {0.0, 1, 0};
  const double s = p.sqrt_s * p.sqrt_s;
  if constexpr (PROC == P_EE_MUMU) {
    const R e = R(p.sqrt_s * 0.5);
    v4<R> p1, p2;
    const R psw = two_body_equal<R>(R(p.sqrt_s), R(0), R(2) * x[0] - R(1), x[1], &p1, &p2);
    const v4<R> pa = {e, R(0), R(0), e}, pb = {e, R(0), R(0), -e};
    const R me2 = me2_eemumu<R>(pa, pb, p1, p2, R(s), R(4.0 * kPi * p.alpha), R(p.sw2), R(p.mz), R(p.gz));
    out.f = double(me2) / (2.0 * s) * double(psw) * p.gev2pb;
    if (rec) {
      rec_p4(rec, 0, pa); rec_p4(rec, 1, pb); rec_p4(rec, 2, p1); rec_p4(rec, 3, p2);
      rec_put(rec, 77, 1.0); rec_put(rec, 78, 1.0); rec_put(rec, 79, s); rec_put(rec, 80, 1.0);
      rec_put(rec, 82, me2); rec_put(rec, 84, psw);
    }
  } else if constexpr (PROC == P_PP_TTBAR) {
    const R x1 = x[0], x2 = x[1];
    const R shat = x1 * x2 * R(s);
    const R m = R(p.m_top);
    rec_put(rec, 77, x1); rec_put(rec, 78, x2); rec_put(rec, 79, shat);
    if (!(shat > R(4) * m * m)) {
      out.pass = 0;
      return out;
    }
    const R rs = m_sqrt(shat);
    v4<R> pt, ptb;
    const R psw = two_body_equal<R>(rs, m, R(2) * x[2] - R(1), x[3], &pt, &ptb);
    const v4<R> pa = {rs * R(0.5), R(0), R(0), rs * R(0.5)}, pb = {rs * R(0.5), R(0), R(0), -rs * R(0.5)};
    const R g2 = R(4.0 * kPi * p.alpha_s);
    // luminosities; flavour tables: 0 = gluon, 1..5 = quarks 1..5, 6..10 = antiquarks
    const R g1 = xf_over_x(pdf.tab[0], x1), g2x = xf_over_x(pdf.tab[0], x2);
    const R lx1 = m_log(x1), lx2 = m_log(x2);
    R lqq = R(0);
#pragma unroll
    for (int q = 1; q <= 5; ++q) {
      const R q1 = pdf_interp_1d(pdf.tab[q], lx1), qb2 = pdf_interp_1d(pdf.tab[q + 5], lx2);
      const R qb1 = pdf_interp_1d(pdf.tab[q + 5], lx1), q2 = pdf_interp_1d(pdf.tab[q], lx2);
      lqq += q1 * qb2 + qb1 * q2;
    }
    lqq = lqq / (x1 * x2);
    const R lgg = g1 * g2x;
    const R megg = me2_gg_ttbar<R>(pa, pb, pt, ptb, m, g2);
    const R meqq = me2_qqbar_ttbar<R>(pa, pb, pt, ptb, m, g2);
    out.f = (double(lgg) * double(megg) + double(lqq) * double(meqq)) / (2.0 * double(shat)) * double(psw) * p.gev2pb;
    if (rec) {
      rec_p4(rec, 0, pa); rec_p4(rec, 1, pb); rec_p4(rec, 2, pt); rec_p4(rec, 3, ptb);
      rec_put(rec, 80, lgg); rec_put(rec, 81, lqq); rec_put(rec, 82, megg); rec_put(rec, 83, meqq);
      rec_put(rec, 84, psw);
    }
  } else if constexpr (PROC == P_GG_TTBARG || PROC == P_GG_TTBARG_7D) {
    GgKin<R> kin;
    const int st = gg_kinematics<PROC, R>(a, pdf, x, &kin, rec);
    if (st != 1) {
      out.pass = 0;
      out.status = st;
      return out;
    }
    const R me2 = gg_me2<R>(a, kin);
    out.f = gg_weight<R>(a, kin, me2);
    if (rec) {
      rec_put(rec, 80, kin.lgg);
      rec_put(rec, 82, me2);
    }
  } else if constexpr (PROC == P_PP_TTBARJ) {
    GgKin<R> kin;
    R lum[7];
    if (ppj_kinematics<R>(a, pdf, x, &kin, lum, rec) != 1) {
      out.pass = 0;
      return out;
    }
    R me[7];
    out.f = ppj_weight<R>(a, kin, lum, rec ? me : nullptr);
    if (rec) {
      rec_put(rec, 80, lum[0]); rec_put(rec, 81, lum[1]); rec_put(rec, 82, me[0]); rec_put(rec, 83, me[1]);
      for (int c = 0; c < 5; ++c) rec_put(rec, 89 + c, me[c + 2]);
    }
  } else {  // Gaussian
    const R sg = R(p.gauss_sigma);
    const R norm = R(1) / (sg * R(2.5066282746310002));  // 1 / (sigma sqrt(2 pi))
    const R c = R(-0.5) / (sg * sg);
    R f = R(1);
#pragma unroll
    for (int d = 0; d < ProcTraits<P_GAUSS>::MAXD; ++d) {
      if (d < p.gauss_dim) {
        const R u = x[d] - R(0.5);
        f *= m_exp(c * u * u) * norm;
      }
    }
    out.f = double(f);
  }
  return out;
}

}  // namespace mc
