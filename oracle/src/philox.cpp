// Oracle: Philox4x32-10 and the per-event integer uniforms.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Parity pin: tests/test_oracle_philox.py compares philox4x32_10 with the
// Philox4_32_10 generator of the cuRAND host library (run on the CPU).
#include "oracle.h"

namespace orc {

// Philox4x32-10 written from its published definition (Salmon et al., SC'11,
// Sec. 4.2): ten rounds of two 32x32->64 multiplications of counter words 0
// and 2 by fixed multipliers, the high halves xor-ed into the other counter
// words together with the round key; the key is bumped by the two Weyl
// constants between rounds.
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint64_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = kMul0 * uint64_t(c0);
    uint64_t prod1 = kMul1 * uint64_t(c2);
    uint32_t hi0 = uint32_t(prod0 >> 32), lo0 = uint32_t(prod0);
    uint32_t hi1 = uint32_t(prod1 >> 32), lo1 = uint32_t(prod1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int uniform_bits(int prec) { return prec == 0 ? 52 : 23; }

// The integer uniform k_d of dimension d for event `ev`.
// Counter = (ev low word, ev high word, iteration, gid | call << 8), key =
// (seed low word, seed high word); `call` numbers the Philox calls of one
// event.  FP64 mode (prec 0): two words per dimension, k = (hi:lo) >> 12
// (52 bits).  FP32 mode (prec 1): one word per dimension, k = w >> 9 (23
// bits).  The point in (0,1) is (2k+1) / 2^(bits+1), exact in both formats.
void event_uniform_ints(uint64_t seed, uint32_t iteration, uint32_t gid, int prec, int ndim,
                        int64_t ev, uint64_t* k) {
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  const int per_call = prec == 0 ? 2 : 4;
  for (int d = 0; d < ndim; ++d) {
    const int call = d / per_call;
    const uint32_t ctr[4] = {uint32_t(uint64_t(ev)), uint32_t(uint64_t(ev) >> 32), iteration,
                             (gid & 0xffu) | (uint32_t(call) << 8)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    const int slot = d % per_call;
    if (prec == 0) {
      const uint64_t hi = w[2 * slot], lo = w[2 * slot + 1];
      k[d] = ((hi << 32) | lo) >> 12;
    } else {
      k[d] = uint64_t(w[slot] >> 9);
    }
  }
}

}  // namespace orc

extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  orc::philox4x32_10(ctr, key, out);
}

void orc_uniform_ints(uint64_t seed, uint32_t iteration, uint32_t gid, int prec, int ndim,
                      int64_t first, int64_t n, uint64_t* k_out) {
  for (int64_t i = 0; i < n; ++i)
    orc::event_uniform_ints(seed, iteration, gid, prec, ndim, first + i, k_out + i * ndim);
}
}
