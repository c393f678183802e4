// Oracle: algorithmic operation counts of the g g -> t tbar g event.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The per-event steps of g g -> t tbar g with RAMBO phase space (the fused
// integrand's benchmark workload), evaluated with the operation-counting
// scalar (counted.h) on the same Philox points as orc_iterate: the VEGAS map
// (thesis Sec. "Adaptive Monte Carlo: VEGAS algorithm"), RAMBO (Sec.
// "RAMBO", kinematics_t.h), the gluon cuts, the two gluon densities (Sec.
// "LHAPDF: the Les Houches Accord PDF", kinematics_t.h), |M|^2 from helicity
// amplitudes (formulation C, helicity_t.h; Sec. "The MadFlow event
// generator") and the weight (eq. mc_est_is).  The counts are those of the
// algorithm as the oracle states it: the Philox integers are not floating
// point, and grid properties (knots, knot slopes) are data.
#include <cmath>
#include <cstring>

#include "counted.h"
#include "helicity_t.h"
#include "kinematics_t.h"
#include "oracle.h"

namespace {
using orc::Counted;
using orc::OpCounts;

enum Step { kMap = 0, kRambo, kCuts, kPdf, kMe2, kWeight, kSteps };

OpCounts diff(const OpCounts& a, const OpCounts& b) {
  return {a.add - b.add, a.mul - b.mul, a.div - b.div, a.sqrt - b.sqrt, a.fn - b.fn};
}
void acc(OpCounts& t, const OpCounts& d) {
  t.add += d.add;
  t.mul += d.mul;
  t.div += d.div;
  t.sqrt += d.sqrt;
  t.fn += d.fn;
}
}  // namespace

extern "C" {

// Operation counts of events [first, first + n) of one iteration of
// g g -> t tbar g (RAMBO, 14 dimensions).  out[0] = events, out[1] = events
// inside the cuts, then for each step (map, RAMBO, cuts, PDF, |M|^2, weight)
// five totals: additions, multiplications, divisions, square roots, special
// functions (out[2 + 5 step + k]), and out[2 + 5 x 6] = the sum of the
// events' weights (equal to orc_iterate's sum over the same events: the
// counted arithmetic is the oracle's).  Steps after the cuts run only for
// the events inside them.
void orc_count_gg_ttbarg(const orc_integrand* in, const void* pdf_v, int nbins, const double* edges, int prec,
                         uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, double* out) {
  const auto* pdf = static_cast<const orc::Pdf*>(pdf_v);
  std::memset(out, 0, sizeof(double) * (3 + 5 * kSteps));
  long double wsum = 0.0L;
  OpCounts tot[kSteps];
  const int ndim = 14, bits = orc::uniform_bits(prec);
  const double s = in->sqrt_s * in->sqrt_s, m = in->m_top;
  const auto& ords = orc::ggg_orderings();
  const auto& cm = orc::ggg_colour_matrix();
  int64_t in_cuts = 0;
  for (int64_t ev = first; ev < first + n; ++ev) {
    uint64_t k[16];
    orc::event_uniform_ints(seed, iteration, gid, prec, ndim, ev, k);
    OpCounts c0 = orc::g_ops;
    // VEGAS map: x = lo + r (hi - lo), J = prod N_b (hi - lo)
    Counted x[16], jac = 1.0;
    for (int d = 0; d < ndim; ++d) {
      const uint64_t prod = k[d] * uint64_t(nbins);
      const uint64_t b = prod >> bits, mm = prod & ((uint64_t(1) << bits) - 1);
      const Counted r = Counted(double(2 * mm + 1)) * Counted(std::ldexp(1.0, -(bits + 1)));
      const Counted lo = edges[d * (nbins + 1) + b], hi = edges[d * (nbins + 1) + b + 1];
      const Counted w = hi - lo;
      x[d] = lo + r * w;
      jac *= Counted(double(nbins)) * w;
    }
    OpCounts c1 = orc::g_ops;
    acc(tot[kMap], diff(c1, c0));
    const Counted x1 = x[0], x2 = x[1], shat = x1 * x2 * Counted(s);
    if (!(shat > Counted(4.0 * m * m))) {
      acc(tot[kRambo], diff(orc::g_ops, c1));
      continue;
    }
    const Counted rs = sqrt(shat);
    const double masses[3] = {m, m, 0.0};
    orc::P4T<Counted> p[5];
    const Counted half = rs / Counted(2.0);
    p[0] = {half, 0.0, 0.0, half};
    p[1] = {half, 0.0, 0.0, -half};
    Counted wps;
    const int rc = orc::rambo_t<Counted>(3, masses, rs, x + 2, p + 2, &wps);
    OpCounts c2 = orc::g_ops;
    acc(tot[kRambo], diff(c2, c1));
    if (rc != 0) continue;
    const auto& pg = p[4];
    const Counted pt = sqrt(pg.x * pg.x + pg.y * pg.y);
    const Counted pabs = sqrt(pt * pt + pg.z * pg.z);
    const Counted eta = Counted(0.5) * log((pabs + pg.z) / (pabs - pg.z)) + Counted(0.5) * log(x1 / x2);
    OpCounts c3 = orc::g_ops;
    acc(tot[kCuts], diff(c3, c2));
    if (!(pt > Counted(in->ptcut_g)) || !(fabs(eta) < Counted(in->etacut_g))) continue;
    ++in_cuts;
    const Counted q2 = Counted(in->mu_f * in->mu_f);
    const Counted lumi = orc::pdf_xfxq2_t<Counted>(*pdf, 21, x1, q2) / x1 * orc::pdf_xfxq2_t<Counted>(*pdf, 21, x2, q2) / x2;
    OpCounts c4 = orc::g_ops;
    acc(tot[kPdf], diff(c4, c3));
    const Counted me2 = orc::me2_gg_ttbarg_helicity_t<Counted>(Counted(in->alpha_s), Counted(m), p, cm, ords);
    OpCounts c5 = orc::g_ops;
    acc(tot[kMe2], diff(c5, c4));
    const Counted w = lumi * me2 / (Counted(2.0) * shat) * wps * Counted(in->gev2pb) * jac;
    acc(tot[kWeight], diff(orc::g_ops, c5));
    wsum += orc::value(w);
  }
  out[0] = double(n);
  out[1] = double(in_cuts);
  for (int st = 0; st < kSteps; ++st) {
    double* o = out + 2 + 5 * st;
    o[0] = double(tot[st].add);
    o[1] = double(tot[st].mul);
    o[2] = double(tot[st].div);
    o[3] = double(tot[st].sqrt);
    o[4] = double(tot[st].fn);
  }
  out[2 + 5 * kSteps] = double(wsum);
}

}  // extern "C"
