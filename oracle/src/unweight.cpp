// Oracle: unweighting by acceptance-rejection.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "Unweighted event exporter" (after the acceptance-rejection
// paragraph of Sec. "Monte Carlo integration"): with w_max the largest weight
// of the sample, event i is accepted when w_i > r_i w_max, r_i uniform in
// (0, 1), so that it survives with probability w_i / w_max; the efficiency is
// N_accepted / N_total.  The thesis does not say where r_i comes from; here it
// is the event's own Philox stream at a call index the integrand never uses
// (255), so that any event's decision can be re-derived from (seed,
// iteration, integrand id, event index): counter (ev low, ev high, iteration,
// gid | 255 << 8), r = (2k + 1) / 2^53 with k the top 52 bits of words 0:1.
//
// The accepted events are exported in the laboratory frame, the frame of an
// LHE event record (Sec. "Unweighted event exporter"): the incoming partons
// carry x1 sqrt(s)/2 along +z and x2 sqrt(s)/2 along -z, and the outgoing
// momenta of the partonic centre-of-mass frame are boosted along z by the
// rapidity y = ln(x1/x2)/2 of the partonic system.
//
// Pins (tests/test_oracle_unweight.py): acceptance law for constant weights,
// the defining property of unweighting (the accepted events follow the
// weighted distribution), and for the exported records momentum conservation
// in the laboratory frame, the final-state masses, and the generation cuts,
// which are defined in the laboratory frame, evaluated on the exported
// momenta.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace orc {

double acceptance_uniform(uint64_t seed, uint32_t iteration, uint32_t gid, int64_t ev) {
  const uint32_t ctr[4] = {uint32_t(uint64_t(ev)), uint32_t(uint64_t(ev) >> 32), iteration,
                           (gid & 0xffu) | (255u << 8)};
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  const uint64_t k = ((uint64_t(w[0]) << 32) | w[1]) >> 12;
  return double(2 * k + 1) * 0x1p-53;
}

}  // namespace orc

extern "C" {

void orc_acceptance_uniforms(uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, double* r) {
  for (int64_t i = 0; i < n; ++i) r[i] = orc::acceptance_uniform(seed, iteration, gid, first + i);
}

// accept[i] = 1 when w[i] > r_i w_max.
// Evaluates events first .. first+n-1 (weights[i], may be NULL), takes
// w_max = wmax_in when wmax_in > 0 and the largest weight otherwise
// (*wmax_out), and writes the accepted events, in event order, to
// out[0 .. cap-1].  Returns the number accepted (which may exceed cap), or
// -1 for a process without an event record (p p -> t tbar, Gaussian).
int64_t orc_unweight_events(const orc_integrand* in, const void* pdf, int nbins, const double* edges, int prec,
                            uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, double wmax_in,
                            double* weights, orc_lab_event* out, int64_t cap, double* wmax_out) {
  int nout;
  switch (in->proc) {
    case orc::EE_MUMU: nout = 2; break;
    case orc::GG_TTBARG:
    case orc::GG_TTBARG_7D:
    case orc::GG_TTBARG_MC: nout = 3; break;
    default: return -1;
  }
  const orc::Pdf* P = static_cast<const orc::Pdf*>(pdf);
  std::vector<double> w(static_cast<size_t>(n));
  double wmax = 0.0;
  orc_event_record rec;
  for (int64_t i = 0; i < n; ++i) {
    orc::eval_event(*in, P, nbins, edges, prec, seed, iteration, gid, first + i, &rec);
    w[size_t(i)] = rec.weight;
    if (rec.weight > wmax) wmax = rec.weight;
    if (weights) weights[i] = rec.weight;
  }
  if (wmax_in > 0.0) wmax = wmax_in;
  if (wmax_out) *wmax_out = wmax;
  int64_t nacc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(w[size_t(i)] > orc::acceptance_uniform(seed, iteration, gid, first + i) * wmax)) continue;
    if (nacc < cap) {
      orc::eval_event(*in, P, nbins, edges, prec, seed, iteration, gid, first + i, &rec);
      orc_lab_event& e = out[nacc];
      std::memset(&e, 0, sizeof(e));
      e.event = first + i;
      e.weight = w[size_t(i)];
      e.x1 = rec.x1;
      e.x2 = rec.x2;
      e.proc = in->proc;
      e.nout = nout;
      const double half = in->sqrt_s / 2.0;
      const double pa[4] = {rec.x1 * half, 0.0, 0.0, rec.x1 * half};
      const double pb[4] = {rec.x2 * half, 0.0, 0.0, -rec.x2 * half};
      std::memcpy(e.p[0], pa, sizeof(pa));
      std::memcpy(e.p[1], pb, sizeof(pb));
      const double y = 0.5 * std::log(rec.x1 / rec.x2);
      const double ch = std::cosh(y), sh = std::sinh(y);
      for (int j = 0; j < nout; ++j) {
        const double* q = rec.p[2 + j];
        e.p[2 + j][0] = ch * q[0] + sh * q[3];
        e.p[2 + j][1] = q[1];
        e.p[2 + j][2] = q[2];
        e.p[2 + j][3] = sh * q[0] + ch * q[3];
      }
    }
    ++nacc;
  }
  return nacc;
}

void orc_unweight_accept(uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, const double* w,
                         double wmax, uint8_t* accept) {
  for (int64_t i = 0; i < n; ++i) accept[i] = w[i] > orc::acceptance_uniform(seed, iteration, gid, first + i) * wmax;
}
}
