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
// Pins (tests/test_oracle_unweight.py): acceptance law for constant weights,
// and the defining property of unweighting: the accepted events follow the
// weighted distribution.
#include <cstdint>

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
void orc_unweight_accept(uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, const double* w,
                         double wmax, uint8_t* accept) {
  for (int64_t i = 0; i < n; ++i) accept[i] = w[i] > orc::acceptance_uniform(seed, iteration, gid, first + i) * wmax;
}
}
