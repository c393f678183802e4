// Per-event uniforms and the VEGAS map, device side.
//
// Uniforms: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter-based
// so that every event draws its numbers from its own counter: no generator
// state lives in memory and any event can be regenerated from
// (seed, iteration, integrand id, event index).  The VEGAS map follows the
// thesis's Sec. "Adaptive Monte Carlo: VEGAS algorithm" (separable
// histogram importance sampler, inverse transform of the piecewise-constant
// density).
#pragma once
#include "common.cuh"

namespace mc {

// One Philox4x32-10 block: ten rounds; each multiplies counter words 0 and 2
// by the two published multipliers (__umulhi for the high halves) and mixes
// the high halves with the other two words and the round key; the key is
// advanced by the two published Weyl increments after every round.
MC_D uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Integer uniforms of dimensions [0, D) of event `ev`.  Counter = (ev lo,
// ev hi, iteration, gid | call << 8), key = (seed lo, seed hi).  FP32 mode:
// one 32-bit word per dimension, k = w >> 9 (23 bits).  FP64 mode: two words
// per dimension, k = (w_hi:w_lo) >> 12 (52 bits).
template <int MAXD, bool FP64>
MC_D void event_uniforms(uint64_t seed, uint32_t iteration, uint32_t gid, uint64_t ev, int ndim,
                         uint64_t (&k)[MAXD]) {
  const uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
  constexpr int PER = FP64 ? 2 : 4;
#pragma unroll
  for (int call = 0; call < (MAXD + PER - 1) / PER; ++call) {
    if (call * PER >= ndim) break;
    const uint4 w = philox4x32_10(
        make_uint4(uint32_t(ev), uint32_t(ev >> 32), iteration, (gid & 0xffu) | (uint32_t(call) << 8)), key);
    if (FP64) {
      if (call * 2 + 0 < MAXD) k[call * 2 + 0] = ((uint64_t(w.x) << 32) | w.y) >> 12;
      if (call * 2 + 1 < MAXD) k[call * 2 + 1] = ((uint64_t(w.z) << 32) | w.w) >> 12;
    } else {
      if (call * 4 + 0 < MAXD) k[call * 4 + 0] = w.x >> 9;
      if (call * 4 + 1 < MAXD) k[call * 4 + 1] = w.y >> 9;
      if (call * 4 + 2 < MAXD) k[call * 4 + 2] = w.z >> 9;
      if (call * 4 + 3 < MAXD) k[call * 4 + 3] = w.w >> 9;
    }
  }
}

// VEGAS map of one dimension: bin b = floor(u nbins) and the position r in
// the bin are taken from the integer k exactly (b = (k nbins) >> bits,
// r = (2 ((k nbins) mod 2^bits) + 1) / 2^(bits+1), exact in the working
// precision), then x = e_b + r (e_{b+1} - e_b) and J_d = nbins (e_{b+1} - e_b).
template <class R, bool FP64>
MC_D R vegas_map_1d(const R* edges, int nbins, uint64_t k, int* bin, R* jac) {
  constexpr int BITS = FP64 ? 52 : 23;
  const uint64_t prod = k * uint64_t(nbins);
  const int b = int(prod >> BITS);
  const uint64_t m = prod & ((uint64_t(1) << BITS) - 1);
  R r;
  if (FP64)
    r = R(double(2 * m + 1) * 0x1p-53);
  else
    r = R(float(uint32_t(2 * m + 1)) * 0x1p-24f);
  const R lo = edges[b], hi = edges[b + 1];
  *bin = b;
  *jac = R(nbins) * (hi - lo);
  return lo + r * (hi - lo);
}

}  // namespace mc
