// Oracle: the per-event integrand, one VEGAS iteration and a full integration.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "The MadFlow event generator", eq. mc_master_formula:
// sigma = sum_ab int dPhi_n(x1, x2, p) L(x1, x2) |M(ab -> X)|^2, here with the
// flux factor 1/(2 shat) and the conversion GeV^-2 -> pb made explicit:
//   f = sum_ab f_a(x1) f_b(x2) <|M_ab|^2> / (2 shat) * w_PS * gev2pb,
// f_a = (x f_a)/x from the PDF grid at Q^2 = mu_F^2.  The VEGAS weight of an
// event is f times the grid Jacobian (eq. mc_est_is); the per-bin histogram
// accumulates the squared weight (Sec. "Adaptive Monte Carlo: VEGAS
// algorithm").  Sums run in long double per worker thread; workers own
// contiguous event ranges and are combined in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "oracle.h"

namespace orc {
double vegas_map_1d(const double* edges, int nbins, int bits, uint64_t k, int* bin, double* jac);
void vegas_refine_1d(const double* edges, int nbins, const double* hist, double alpha, double* out);
}  // namespace orc

extern "C" void orc_combine(int n, const double* e, const double* s2, double* mean, double* sigma,
                            double* chi2dof);
extern "C" void orc_iteration_estimate(double sum, double sum2, int64_t n, double* mean, double* var);

namespace orc {

static void put(double (*dst)[4], int i, const P4& p) {
  dst[i][0] = p.e;
  dst[i][1] = p.x;
  dst[i][2] = p.y;
  dst[i][3] = p.z;
}

int process_ndim(const orc_integrand& in) {
  switch (in.proc) {
    case EE_MUMU: return 2;
    case PP_TTBAR: return 4;
    case GG_TTBARG: return 14;
    case GAUSS: return in.gauss_dim;
    case GG_TTBARG_7D: return 7;
    case GG_TTBARG_MC: return 17;  // grid dimensions; 7 uniforms per event
    case PP_TTBARJ: return 7;
  }
  return -1;
}

// Integrand value at the point x of the unit hypercube (rec receives the
// intermediate quantities).
static double integrand_value(const orc_integrand& in, const Pdf* pdf, const double* x,
                              orc_event_record* rec) {
  const double pi = M_PI;
  const double s = in.sqrt_s * in.sqrt_s;
  rec->pass = 1;
  rec->status = 0;
  switch (in.proc) {
    case EE_MUMU: {
      // two-body massless phase space, eq. 2bodyps; cos(theta) = 2 x0 - 1
      const double c = 2.0 * x[0] - 1.0, phi = 2.0 * pi * x[1];
      P4 p[2];
      double w;
      two_body(in.sqrt_s, 0.0, 0.0, c, phi, p, &w);
      const double e = in.sqrt_s / 2.0;
      put(rec->p, 0, {e, 0.0, 0.0, e});
      put(rec->p, 1, {e, 0.0, 0.0, -e});
      put(rec->p, 2, p[0]);
      put(rec->p, 3, p[1]);
      rec->x1 = rec->x2 = 1.0;
      rec->shat = s;
      rec->lumi = 1.0;
      rec->me2 = me2_eemumu({in.alpha, in.mz, in.gz, in.sw2}, s, c);
      rec->ps_weight = w;
      return rec->me2 / (2.0 * s) * w * in.gev2pb;
    }
    case PP_TTBAR: {
      const double x1 = x[0], x2 = x[1], shat = x1 * x2 * s, m = in.m_top;
      rec->x1 = x1;
      rec->x2 = x2;
      rec->shat = shat;
      if (!(shat > 4.0 * m * m)) {
        rec->pass = 0;
        return 0.0;
      }
      const double rs = std::sqrt(shat);
      const double c = 2.0 * x[2] - 1.0, phi = 2.0 * pi * x[3];
      P4 p[2];
      double w;
      two_body(rs, m, m, c, phi, p, &w);
      const P4 pa = {rs / 2.0, 0.0, 0.0, rs / 2.0}, pb = {rs / 2.0, 0.0, 0.0, -rs / 2.0};
      put(rec->p, 0, pa);
      put(rec->p, 1, pb);
      put(rec->p, 2, p[0]);
      put(rec->p, 3, p[1]);
      const P4 d = sub(pa, p[0]);
      const double t = dot(d, d);
      const double q2 = in.mu_f * in.mu_f;
      const double g1 = pdf_xfxq2(*pdf, 21, x1, q2) / x1, g2 = pdf_xfxq2(*pdf, 21, x2, q2) / x2;
      double lqq = 0.0;
      for (int q = 1; q <= 5; ++q)
        lqq += pdf_xfxq2(*pdf, q, x1, q2) / x1 * pdf_xfxq2(*pdf, -q, x2, q2) / x2 +
               pdf_xfxq2(*pdf, -q, x1, q2) / x1 * pdf_xfxq2(*pdf, q, x2, q2) / x2;
      rec->lumi = g1 * g2;
      rec->lumi_qq = lqq;
      rec->me2 = me2_gg_ttbar(in.alpha_s, m, shat, t);
      rec->me2_qq = me2_qqbar_ttbar(in.alpha_s, m, shat, t);
      rec->ps_weight = w;
      return (rec->lumi * rec->me2 + lqq * rec->me2_qq) / (2.0 * shat) * w * in.gev2pb;
    }
    case GG_TTBARG:
    case GG_TTBARG_7D: {
      const double x1 = x[0], x2 = x[1], shat = x1 * x2 * s, m = in.m_top;
      rec->x1 = x1;
      rec->x2 = x2;
      rec->shat = shat;
      if (!(shat > 4.0 * m * m)) {
        rec->pass = 0;
        return 0.0;
      }
      const double rs = std::sqrt(shat);
      const double masses[3] = {m, m, 0.0};
      P4 p[5];
      p[0] = {rs / 2.0, 0.0, 0.0, rs / 2.0};
      p[1] = {rs / 2.0, 0.0, 0.0, -rs / 2.0};
      double w;
      // RAMBO (Sec. "RAMBO") or sequential branchings (table tab:hierarchical)
      const int rc = in.proc == GG_TTBARG ? rambo(3, masses, rs, x + 2, p + 2, &w)
                                          : hierarchical(3, masses, rs, x + 2, p + 2, &w);
      for (int i = 0; i < 5; ++i) put(rec->p, i, p[i]);
      rec->ps_weight = w;
      if (rc != 0) {
        rec->pass = 0;
        rec->status = rc;
        return 0.0;
      }
      // cuts on the gluon in the lab frame: pT is boost invariant along z;
      // the rapidity of the partonic frame is y = ln(x1/x2)/2.
      const P4& pg = p[4];
      const double pt = std::sqrt(pg.x * pg.x + pg.y * pg.y);
      const double pabs = std::sqrt(pt * pt + pg.z * pg.z);
      const double eta = 0.5 * std::log((pabs + pg.z) / (pabs - pg.z)) + 0.5 * std::log(x1 / x2);
      if (!(pt > in.ptcut_g) || !(std::fabs(eta) < in.etacut_g)) {
        rec->pass = 0;
        return 0.0;
      }
      const double q2 = in.mu_f * in.mu_f;
      rec->lumi = pdf_xfxq2(*pdf, 21, x1, q2) / x1 * pdf_xfxq2(*pdf, 21, x2, q2) / x2;
      rec->me2 = me2_gg_ttbarg(in.alpha_s, m, p);
      return rec->lumi * rec->me2 / (2.0 * shat) * w * in.gev2pb;
    }
    case PP_TTBARJ: {
      // p p -> t tbar + one parton at LO: every partonic channel at the same
      // point of the hierarchical three-body phase space (the light parton
      // massless, so the kinematics do not depend on the channel)
      const double x1 = x[0], x2 = x[1], shat = x1 * x2 * s, m = in.m_top;
      rec->x1 = x1;
      rec->x2 = x2;
      rec->shat = shat;
      if (!(shat > 4.0 * m * m)) {
        rec->pass = 0;
        return 0.0;
      }
      const double rs = std::sqrt(shat);
      const double masses[3] = {m, m, 0.0};
      P4 p[5];
      p[0] = {rs / 2.0, 0.0, 0.0, rs / 2.0};
      p[1] = {rs / 2.0, 0.0, 0.0, -rs / 2.0};
      double w;
      hierarchical(3, masses, rs, x + 2, p + 2, &w);
      for (int i = 0; i < 5; ++i) put(rec->p, i, p[i]);
      rec->ps_weight = w;
      // cuts on the light parton in the lab frame
      const P4& pk = p[4];
      const double pt = std::sqrt(pk.x * pk.x + pk.y * pk.y);
      const double pabs = std::sqrt(pt * pt + pk.z * pk.z);
      const double eta = 0.5 * std::log((pabs + pk.z) / (pabs - pk.z)) + 0.5 * std::log(x1 / x2);
      if (!(pt > in.ptcut_g) || !(std::fabs(eta) < in.etacut_g)) {
        rec->pass = 0;
        return 0.0;
      }
      const double q2 = in.mu_f * in.mu_f;
      auto f1 = [&](int pid) { return pdf_xfxq2(*pdf, pid, x1, q2) / x1; };
      auto f2 = [&](int pid) { return pdf_xfxq2(*pdf, pid, x2, q2) / x2; };
      double l[7] = {f1(21) * f2(21), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int q = 1; q <= 5; ++q) {
        l[1] += f1(q) * f2(-q);
        l[2] += f1(-q) * f2(q);
        l[3] += f1(q) * f2(21);
        l[4] += f1(21) * f2(q);
        l[5] += f1(-q) * f2(21);
        l[6] += f1(21) * f2(-q);
      }
      const P4 ab[5] = {p[0], p[1], p[2], p[3], p[4]};
      const P4 ba[5] = {p[1], p[0], p[2], p[3], p[4]};
      const P4 abc[5] = {p[0], p[1], p[3], p[2], p[4]};  // t and tbar exchanged (charge conjugation)
      const P4 bac[5] = {p[1], p[0], p[3], p[2], p[4]};
      double me[7];
      me[0] = me2_gg_ttbarg(in.alpha_s, m, p);
      me[1] = me2_qqbar_ttbarg(in.alpha_s, m, ab);
      me[2] = me2_qqbar_ttbarg(in.alpha_s, m, ba);
      me[3] = me2_qg_ttbarq(in.alpha_s, m, ab);
      me[4] = me2_qg_ttbarq(in.alpha_s, m, ba);
      // qbar g -> t tbar qbar is q g -> t tbar q with t and tbar exchanged
      me[5] = me2_qg_ttbarq(in.alpha_s, m, abc);
      me[6] = me2_qg_ttbarq(in.alpha_s, m, bac);
      double sum = 0.0;
      for (int c = 0; c < 7; ++c) {
        rec->lumi_x[c] = l[c];
        sum += l[c] * me[c];
      }
      for (int c = 0; c < 5; ++c) rec->me2_x[c] = me[c + 2];
      rec->lumi = l[0];
      rec->lumi_qq = l[1];
      rec->me2 = me[0];
      rec->me2_qq = me[1];
      return sum / (2.0 * shat) * w * in.gev2pb;
    }
    case GAUSS: {
      // normalised Gaussian of width sigma centred at 1/2 in every dimension
      double f = 1.0;
      const double sg = in.gauss_sigma;
      for (int d = 0; d < in.gauss_dim; ++d) {
        const double u = x[d] - 0.5;
        f *= std::exp(-u * u / (2.0 * sg * sg)) / (sg * std::sqrt(2.0 * pi));
      }
      return f;
    }
  }
  rec->status = -1;
  return 0.0;
}

void eval_event(const orc_integrand& in, const Pdf* pdf, int nbins, const double* edges, int prec,
                uint64_t seed, uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec) {
  if (in.proc == GG_TTBARG_MC) {  // channel choice and densities need the event and the grid
    double dens[3];
    channels_event(in, pdf, nbins, edges, prec, seed, iteration, gid, ev, rec, dens);
    return;
  }
  std::memset(rec, 0, sizeof(*rec));
  const int ndim = process_ndim(in);
  uint64_t k[16];
  event_uniform_ints(seed, iteration, gid, prec, ndim, ev, k);
  const int bits = uniform_bits(prec);
  double jac = 1.0;
  for (int d = 0; d < ndim; ++d) {
    int b;
    double jd;
    rec->x[d] = vegas_map_1d(edges + d * (nbins + 1), nbins, bits, k[d], &b, &jd);
    rec->bin[d] = b;
    jac *= jd;
  }
  rec->jac = jac;
  rec->f = integrand_value(in, pdf, rec->x, rec);
  rec->weight = rec->f * jac;
}

}  // namespace orc

extern "C" {

int orc_process_ndim(const orc_integrand* in) { return orc::process_ndim(*in); }

void orc_event(const orc_integrand* in, const void* pdf, int nbins, const double* edges, int prec,
               uint64_t seed, uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec) {
  orc::eval_event(*in, static_cast<const orc::Pdf*>(pdf), nbins, edges, prec, seed, iteration, gid,
                  ev, rec);
}

// Integrand at n given points x [n][ndim] of the unit hypercube (no VEGAS
// map): f[i] and the status of each evaluation (0, or negative on failure).
void orc_integrand_at(const orc_integrand* in, const void* pdf, int64_t n, const double* x, double* f,
                      int32_t* status) {
  const int ndim = orc::process_ndim(*in);
  for (int64_t i = 0; i < n; ++i) {
    orc_event_record rec;
    std::memset(&rec, 0, sizeof(rec));
    f[i] = orc::integrand_value(*in, static_cast<const orc::Pdf*>(pdf), x + i * ndim, &rec);
    status[i] = rec.status;
  }
}

// The weight w = f J of each event of [first, first + n) of one VEGAS
// iteration (thesis eq. mc_est_is: the terms of the estimate), in event order,
// on nthreads threads (0: one per core).
void orc_weights(const orc_integrand* in, const void* pdf_v, int nbins, const double* edges, int prec,
                 uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, int nthreads,
                 double* w) {
  const auto* pdf = static_cast<const orc::Pdf*>(pdf_v);
  if (nthreads <= 0) nthreads = int(std::max(1u, std::thread::hardware_concurrency()));
  nthreads = int(std::min<int64_t>(nthreads, std::max<int64_t>(n, 1)));
  auto work = [&](int tid) {
    const int64_t lo = n * tid / nthreads, hi = n * (tid + 1) / nthreads;
    orc_event_record rec;
    for (int64_t i = lo; i < hi; ++i) {
      orc::eval_event(*in, pdf, nbins, edges, prec, seed, iteration, gid, first + i, &rec);
      w[i] = rec.weight;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
}

// One VEGAS iteration over events [first, first + n): sums of w and w^2,
// the count of non-zero weights, the largest weight, and the per-dimension
// histograms of w^2 and of event counts (both accumulated into the outputs).
void orc_iterate(const orc_integrand* in, const void* pdf_v, int nbins, const double* edges,
                 int prec, uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first,
                 int64_t n, int nthreads, orc_iter_result* res, double* hist_w2,
                 uint32_t* hist_n) {
  const auto* pdf = static_cast<const orc::Pdf*>(pdf_v);
  const int ndim = orc::process_ndim(*in);
  if (nthreads <= 0) nthreads = int(std::max(1u, std::thread::hardware_concurrency()));
  nthreads = int(std::min<int64_t>(nthreads, std::max<int64_t>(n, 1)));
  struct Part {
    long double sum = 0, sum2 = 0;
    int64_t nz = 0;
    double wmax = 0;
    std::vector<long double> h;
    std::vector<uint32_t> c;
  };
  std::vector<Part> parts(nthreads);
  auto work = [&](int tid) {
    Part& p = parts[tid];
    p.h.assign(size_t(ndim) * nbins, 0.0L);
    p.c.assign(size_t(ndim) * nbins, 0u);
    const int64_t lo = first + n * tid / nthreads, hi = first + n * (tid + 1) / nthreads;
    orc_event_record rec;
    for (int64_t ev = lo; ev < hi; ++ev) {
      orc::eval_event(*in, pdf, nbins, edges, prec, seed, iteration, gid, ev, &rec);
      const double w = rec.weight;
      p.sum += w;
      p.sum2 += (long double)w * w;
      if (w != 0.0) ++p.nz;
      if (w > p.wmax) p.wmax = w;
      const bool mc = in->proc == orc::GG_TTBARG_MC;
      for (int d = 0; d < (mc ? 7 : ndim); ++d) {
        const int gd = mc ? orc::channel_grid_dim(d, rec.channel) : d;
        p.h[size_t(gd) * nbins + rec.bin[d]] += (long double)w * w;
        p.c[size_t(gd) * nbins + rec.bin[d]] += 1;
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nthreads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
  long double sum = 0, sum2 = 0;
  int64_t nz = 0;
  double wmax = 0;
  std::vector<long double> h(size_t(ndim) * nbins, 0.0L);
  for (auto& p : parts) {
    sum += p.sum;
    sum2 += p.sum2;
    nz += p.nz;
    wmax = std::max(wmax, p.wmax);
    for (size_t i = 0; i < h.size(); ++i) {
      h[i] += p.h[i];
      if (hist_n) hist_n[i] += p.c[i];
    }
  }
  if (hist_w2)
    for (size_t i = 0; i < h.size(); ++i) hist_w2[i] += double(h[i]);
  res->sum = double(sum);
  res->sum2 = double(sum2);
  res->n = n;
  res->n_nonzero = nz;
  res->wmax = wmax;
}

// Full integration: niter iterations of nevents each, refining the grid after
// every iteration (damping alpha), then the inverse-variance combination.
// edges (in/out) holds the grid; per_iter receives (E_i, S_i^2) pairs.
void orc_integrate(const orc_integrand* in, const void* pdf, int nbins, double* edges, int prec,
                   uint64_t seed, uint32_t gid, int niter, int64_t nevents, double alpha,
                   int nthreads, double* per_iter, double* mean, double* sigma, double* chi2dof) {
  const int ndim = orc::process_ndim(*in);
  std::vector<double> e(niter), s2(niter), hist(size_t(ndim) * nbins);
  std::vector<double> next(size_t(ndim) * (nbins + 1));
  for (int it = 0; it < niter; ++it) {
    std::fill(hist.begin(), hist.end(), 0.0);
    orc_iter_result r;
    orc_iterate(in, pdf, nbins, edges, prec, seed, uint32_t(it), gid, 0, nevents, nthreads, &r,
                hist.data(), nullptr);
    orc_iteration_estimate(r.sum, r.sum2, r.n, &e[it], &s2[it]);
    per_iter[2 * it] = e[it];
    per_iter[2 * it + 1] = s2[it];
    for (int d = 0; d < ndim; ++d)
      orc::vegas_refine_1d(edges + d * (nbins + 1), nbins, hist.data() + size_t(d) * nbins, alpha,
                           next.data() + size_t(d) * (nbins + 1));
    std::copy(next.begin(), next.end(), edges);
  }
  orc_combine(niter, e.data(), s2.data(), mean, sigma, chi2dof);
}
}
