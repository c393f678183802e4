// The per-event integrand (thesis Sec. "The MadFlow event generator",
// eq. mc_master_formula) with the flux factor and the unit conversion made
// explicit:
//   f = sum_ab f_a(x1) f_b(x2) <|M_ab|^2> / (2 shat) * w_PS * gev2pb,
// f_a = (x f_a)(x, mu_F^2) / x.  The VEGAS event weight is f * J.
#pragma once
#include "matrix_elements.cuh"
#include "pdf.cuh"
#include "phasespace.cuh"
#include "sampling.cuh"

namespace mc {

enum : int { P_EE_MUMU = 0, P_PP_TTBAR = 1, P_GG_TTBARG = 2, P_GAUSS = 3, P_GG_TTBARG_7D = 4 };

template <int PROC> struct ProcTraits;
template <> struct ProcTraits<P_EE_MUMU> { static constexpr int MAXD = 2, NFL = 0; };
template <> struct ProcTraits<P_PP_TTBAR> { static constexpr int MAXD = 4, NFL = 11; };
template <> struct ProcTraits<P_GG_TTBARG> { static constexpr int MAXD = 14, NFL = 1; };
template <> struct ProcTraits<P_GAUSS> { static constexpr int MAXD = 16, NFL = 0; };
template <> struct ProcTraits<P_GG_TTBARG_7D> { static constexpr int MAXD = 7, NFL = 1; };

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
    // gg -> t tbar g: RAMBO (14 dims) or the hierarchical generator (7 dims)
    const R x1 = x[0], x2 = x[1];
    rec_put(rec, 77, x1); rec_put(rec, 78, x2);
    const R m = R(p.m_top);
    const R shat = sizeof(R) == 4 ? R(x1 * x2 * R(s)) : R(double(x1) * double(x2) * s);
    rec_put(rec, 79, shat);
    if (!(shat > R(4) * m * m)) {
      out.pass = 0;
      return out;
    }
    const R rs = m_sqrt(shat);
    v4<R> k[3];
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
    const v4<R> pa = {rs * R(0.5), R(0), R(0), rs * R(0.5)}, pb = {rs * R(0.5), R(0), R(0), -rs * R(0.5)};
    if (rec) {
      rec_p4(rec, 0, pa); rec_p4(rec, 1, pb); rec_p4(rec, 2, k[0]); rec_p4(rec, 3, k[1]); rec_p4(rec, 4, k[2]);
      rec_put(rec, 84, psw);
    }
    if (rc != 0) {
      out.pass = 0;
      out.status = -5;
      return out;
    }
    // gluon cuts in the lab frame: pT > cut and |eta_cm + y| < cut with
    // y = ln(x1/x2)/2, written without logarithms:
    // e^{-2c} (|p| - pz) x2 < (|p| + pz) x1 < e^{2c} (|p| - pz) x2.
    const v4<R>& g = k[2];
    const R pt2 = g.x * g.x + g.y * g.y;
    const R ptc = R(p.ptcut_g);
    if (!(pt2 > ptc * ptc)) {
      out.pass = 0;
      return out;
    }
    const R pabs = m_sqrt(pt2 + g.z * g.z);
    const R fwd = (pabs + g.z) * x1, bwd = (pabs - g.z) * x2;
    const R e2 = R(a.e2eta);
    if (!(fwd < e2 * bwd && bwd < e2 * fwd)) {
      out.pass = 0;
      return out;
    }
    const R me2 = me2_gg_ttbarg<R>(pa, pb, k[0], k[1], k[2], m, R(4.0 * kPi * p.alpha_s));
    const R lgg = xf_over_x(pdf.tab[0], x1) * xf_over_x(pdf.tab[0], x2);
    if (sizeof(R) == 4)
      out.f = double(lgg * me2 * (R(p.gev2pb) / (R(2) * shat))) * psw;
    else
      out.f = double(lgg) * double(me2) / (2.0 * double(shat)) * psw * p.gev2pb;
    if (rec) {
      rec_put(rec, 80, lgg);
      rec_put(rec, 82, me2);
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
