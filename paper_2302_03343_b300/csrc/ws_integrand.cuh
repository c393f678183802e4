// Warp-specialised fused integrand kernel for gg -> t tbar g and
// p p -> t tbar + parton in FP32 mode.
//
// The fused path of one event has two parts with very different hardware
// profiles: the kinematics (Philox, VEGAS map, RAMBO with its FP64 conformal
// boost, cuts, gluon luminosity) is bound by the FP64 pipe, whose B300
// throughput is about 1/64 of the FP32 rate, and about a fifth of the events
// fail the cuts; the |M|^2 (colour-ordered helicity amplitudes in packed
// FP32x2 arithmetic) is bound by the FMA pipe.  Run one after the other in
// every thread, a warp stalls for thousands of cycles in its FP64 section
// and carries idle lanes through the |M|^2 for the events that were cut.
//
// Here each block (one per SM) splits its warps into two roles (the shape
// given for gg -> t tbar g; per process below):
//  * 8 producer warps (two per SM sub-partition) walk the event range in
//    chunks of 32, evaluate the kinematics, add every event to the bin-count
//    histogram, and append the events that pass the cuts, compacted with a
//    warp ballot, to a shared-memory ring of slots of 32 event records;
//  * 8 consumer warps take full slots, evaluate |M|^2 on all 32 lanes, form
//    the weights w = f J, and keep the Kahan FP64 sums, w_max and the
//    shared-memory histogram of w^2.
// Slots pass between the roles through mbarriers (full: 32 producer-lane
// arrivals; empty: 32 consumer-lane arrivals).  Producer warp p owns the
// slots Sp .. Sp + S - 1 (S = ws_slots(process)), used in turn; with equal
// counts consumer warp c takes producer c's slots (the general mapping is
// below).  The assignment of
// events to lanes is fixed by the launch shape, so the sums are
// deterministic for a given grid.  A producer ends its stream with a partial
// slot and one end marker (count -1) for each consumer it feeds.  Sixteen
// warps of 128 registers at launch, rebalanced to 88 (producers) and 168
// (consumers) with setmaxnreg, measured fastest among the 4+8, 8+4 and 8+8
// shapes on B300 for that process.  ptxas allocates the code after each
// setmaxnreg within its count (the producers' within 88 registers, the
// consumers' within 168), and the consumers' |M|^2 still spills at 168, so
// the spills must stay in L1: the shared memory of a block is kept small for
// that (see ws_rows_in_smem).
//
// Every wait is bounded (kWsWaitNs of %globaltimer); a warp that gives up
// stops, the block poisons its partial sums with NaN and, when the launch
// carries a status word, sets it to MC_ETIMEOUT.
#pragma once
#include "event.cuh"
#include "tcgen05.cuh"

namespace mc {

// Launch shape, per process: ws_producer_warps producer warps and
// ws_consumer_warps consumer warps per block (each a multiple of 4, i.e.
// whole warpgroups, since the register split below is per warpgroup), one
// block per SM.  gg -> t tbar g: 8 + 8 (the description above).
// p p -> t tbar + parton: 4 + 8, a 12-warp launch of 168 registers a
// thread, so that the consumers' seven-channel |M|^2 compiles within 208
// registers instead of 168 and spills half as much (measured on B300: 19.0
// against 22.5 ms per 1e7 events with 8 + 8; the same 4 + 8 shape costs
// gg -> t tbar g 36 %: four producers cannot keep its consumers fed).
MC_HD constexpr int ws_producer_warps(int proc) { return proc == P_PP_TTBARJ ? 4 : 8; }
MC_HD constexpr int ws_consumer_warps(int) { return 8; }
MC_HD constexpr int ws_threads(int proc) { return 32 * (ws_producer_warps(proc) + ws_consumer_warps(proc)); }
// Slots per producer warp (a producer holds up to two at once, so at least
// three for the producer to work ahead of its consumer); 4 measured fastest
// on B300 for every process (3 and 2 return 24 and 47 KB to L1 but starve
// the three-channel consumers).
MC_HD constexpr int ws_slots(int) { return 4; }
// record words of one event (structure of arrays inside a slot: word j of
// lane e at [j][e]): k[3] (12), rs, lgg, flux, jac, psw (2 words), bins (4),
// the event's index in the launch (weights pass only), and for the
// three-channel process its channel and the ratios p_j / p (3); for
// p p -> t tbar + parton kWLgg holds the gg luminosity, kWFlux the partonic
// s and kWLum the other six channel luminosities
enum : int {
  kWK = 0, kWRs = 12, kWLgg = 13, kWFlux = 14, kWJac = 15, kWPsw = 16, kWBin = 18, kWIdx = 22, kWCh = 23,
  kWDens = 24, kWLum = 23
};
// words per record: 23, 27 for the three-channel process and 29 for
// p p -> t tbar + parton (the ring of the others stays at 23 words so their
// shared-memory carveout, and the L1 left for their register spills, does
// not change)
MC_HD constexpr int ws_words(int proc) {
  return proc == P_GG_TTBARG_MC ? 27 : (proc == P_PP_TTBARJ ? 29 : 23);
}
// flavour tables of the process in shared memory (the gluon, or all eleven)
MC_HD constexpr int ws_flavours(int proc) { return proc == P_PP_TTBARJ ? 11 : 1; }
constexpr unsigned long long kWsWaitNs = 2000000000ull;
// Registers per thread: the launch gets ws_regs (65536 / threads, rounded
// down to a multiple of 8); producers give up to ws_producer_regs, consumers
// take ws_consumer_regs, and the two together stay within the launch's
// registers, so the increase never waits on registers that are not there
// (ws_shape_ok, asserted in each kernel).
MC_HD constexpr int ws_regs(int proc) {
  return (65536 / ws_threads(proc)) / 8 * 8 > 248 ? 248 : (65536 / ws_threads(proc)) / 8 * 8;
}
MC_HD constexpr int ws_producer_regs(int) { return 88; }
MC_HD constexpr int ws_consumer_regs(int proc) { return proc == P_PP_TTBARJ ? 208 : 168; }
// Streams: producer p's slot sequence q = 0, 1, 2, ... goes to consumer
// (p mod C) + P ((q mod ws_classes)) when there are more consumers than
// producers (C = ws_classes P), and every consumer c serves the producers
// c, c + C, ... (ws_streams of them) when there are more producers.
MC_HD constexpr int ws_classes(int proc) {
  return ws_consumer_warps(proc) >= ws_producer_warps(proc) ? ws_consumer_warps(proc) / ws_producer_warps(proc) : 1;
}
MC_HD constexpr int ws_streams(int proc) {
  return ws_producer_warps(proc) >= ws_consumer_warps(proc) ? ws_producer_warps(proc) / ws_consumer_warps(proc) : 1;
}
// whole warpgroups, a register split within the launch's registers, warp
// counts that divide one another, at most two producers per consumer
MC_HD constexpr bool ws_shape_ok(int proc) {
  return ws_producer_warps(proc) % 4 == 0 && ws_consumer_warps(proc) % 4 == 0 &&
         32 * ws_producer_warps(proc) * ws_producer_regs(proc) +
                 32 * ws_consumer_warps(proc) * ws_consumer_regs(proc) <=
             ws_threads(proc) * ws_regs(proc) &&
         (ws_classes(proc) * ws_producer_warps(proc) == ws_consumer_warps(proc) ||
          ws_streams(proc) * ws_consumer_warps(proc) == ws_producer_warps(proc)) &&
         ws_streams(proc) <= 2;
}

MC_D unsigned long long ws_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the completion of the mbarrier phase of the given parity; false
// after kWsWaitNs.
MC_D bool ws_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = ws_clock_ns();
  while (!mbar_try_wait(bar, parity))
    if (ws_clock_ns() - t0 > kWsWaitNs) return false;
  return true;
}

// Dynamic shared memory of one block: the ring, then the histograms, the
// grid edges and the PDF tables (as in the per-thread fused kernel).
// With `rows`, each consumer thread also keeps the twelve row spinors of its
// current event's |M|^2 there (kWsRowBytes, after the ring) and evaluates it
// with me2_gg_ttbarg_rows, else with me2_gg_ttbarg_p.  Measured on B300, the
// rows pay for the three-channel process only (8 % faster there; for the
// others the L1 they take from the consumers' register spills costs more,
// 10 % with L2 flushed between launches), and only while the block's shared
// memory stays within kWsSmemRows (the histograms and edges grow with nbins).
constexpr int kWsRowBytes = 12 * 32;
constexpr size_t kWsSmemRows = 224 * 1024;  // 227 KB per block less the static shared memory
inline size_t ws_smem_bytes(int proc, int ndim, int nbins, int nx, bool rows) {
  const size_t ring = size_t(ws_slots(proc)) * ws_producer_warps(proc) * ws_words(proc) * 32 * 4 +
                      (rows ? size_t(ws_consumer_warps(proc)) * 32 * kWsRowBytes : 0);
  const size_t hist = ((size_t(ndim) * nbins * 8 + 15) / 16) * 16;
  return ring + hist + 4 * (size_t(ndim) * (nbins + 1) + size_t(nx) * (1 + 2 * ws_flavours(proc)));
}
inline bool ws_rows_in_smem(int proc, int ndim, int nbins, int nx) {
  return proc == P_GG_TTBARG_MC && ws_smem_bytes(proc, ndim, nbins, nx, true) <= kWsSmemRows;
}
inline size_t ws_smem_bytes(int proc, int ndim, int nbins, int nx) {
  return ws_smem_bytes(proc, ndim, nbins, nx, ws_rows_in_smem(proc, ndim, nbins, nx));
}

// Shared-memory ring of one block: ws_slots(PROC) x ws_producer_warps(PROC) slots of 32 event records, their
// full/empty mbarriers and counts (-1 = end marker).
struct WsRing {
  uint32_t* rec;   // [slots][ws_words(PROC)][32]
  uint64_t* full;  // [slots], arrival count 32 (the producer's lanes)
  uint64_t* empty;  // [slots], arrival count 32 (the consumer's lanes)
  int* count;      // [slots]
};

// Producer warp p (0 <= p < ws_producer_warps(PROC)): evaluates the kinematics of the
// events [lo, hi) of the integrand in chunks of 32 (chunk k = events
// lo + 32 k .. lo + 32 k + 31; this warp takes chunks k0, k0 + dk, ...), adds
// every event to the bin counts, appends the events that pass the cuts to its
// slots, and ends the stream with a partial slot and one end marker per
// consumer it feeds.  seq is the warp's slot sequence number and carries
// over between calls (the slot of seq is p S + seq % S, used for the
// (seq / S)-th time).  The Philox event index is a.first + i.  With WOUT the
// weights pass writes a.wout[i] = 0 for the events that are cut and passes i
// on in the record.  Returns false when a wait gave up.
template <int PROC, bool WOUT, bool PTS = false>
MC_D bool ws_produce(const KernelArgs& a, const SmPdf<float>& pdf, const float* sh_edges, unsigned int* sh_n,
                     const WsRing& ring, int p, long long lo, long long hi, long long k0, long long dk, int& seq,
                     Acc& acc) {
  constexpr int MAXD = ProcTraits<PROC>::MAXD;
  constexpr int NW = (MAXD + 3) / 4;
  const int lane = threadIdx.x & 31;
  const int ndim = a.ndim, nb = a.nbins;
  constexpr int S = ws_slots(PROC);
  auto slot_of = [&](int q) { return p * S + q % S; };
  auto acquire = [&](int q) -> bool {
    const int u = q / S;  // earlier uses of this slot
    return u == 0 || ws_wait(&ring.empty[slot_of(q)], uint32_t(u - 1) & 1u);
  };
  auto publish = [&](int q, int cnt) {
    if (lane == 0) ring.count[slot_of(q)] = cnt;
    mbar_arrive(&ring.full[slot_of(q)]);
  };
  const long long nchunks = (hi - lo + 31) / 32;
  int fill = 0;
  bool next_held = false;
  bool ok = acquire(seq);
  for (long long chunk = k0; ok && chunk < nchunks; chunk += dk) {
    const long long i = lo + chunk * 32 + lane;
    GgKin<float> kin;
    uint32_t binw[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) binw[j] = 0u;
    float jac = 1.0f;
    int st = 0, ch = 0;
    float dr[kChannels] = {0.0f, 0.0f, 0.0f};
    float lum[PROC == P_PP_TTBARJ ? 7 : 1];
    if constexpr (PROC == P_GG_TTBARG_MC) {
      if (i < hi) {
        McEvent<float> e;
        mc_prepare<false, float>(a, pdf, sh_edges, a.first + uint64_t(i), e);
#pragma unroll
        for (int d = 0; d < 7; ++d) {
          binw[d / 4] |= uint32_t(e.bin[d]) << (8 * (d % 4));
          atomicAdd(&sh_n[ch_grid_dim(d, e.ch) * nb + e.bin[d]], 1u);
        }
        ch = e.ch;
        jac = e.jx;
        kin = e.kin;
        st = e.pass;
        if (e.pass) {
#pragma unroll
          for (int j = 0; j < kChannels; ++j) dr[j] = float(e.dens[j] / e.pden);
        }
        if (WOUT && !e.pass) a.wout[i] = 0.0;
      }
    } else if (i < hi) {
      float x[MAXD];
      if constexpr (PTS) {
        // points input: x given; the record's Jacobian word carries log q(x)
#pragma unroll
        for (int dd = 0; dd < MAXD; ++dd) x[dd] = dd < ndim ? a.pts[size_t(i) * ndim + dd] : 0.5f;
        jac = a.pts_logq ? a.pts_logq[i] : 0.0f;
      } else {
        uint64_t k[MAXD];
        event_uniforms<MAXD, false>(a.seed, a.iteration, a.gid, a.first + uint64_t(i), ndim, k);
#pragma unroll
        for (int dd = 0; dd < MAXD; ++dd) {
          if (dd < ndim) {
            int b;
            float jd;
            x[dd] = vegas_map_1d<float, false>(sh_edges + dd * (nb + 1), nb, k[dd], &b, &jd);
            binw[dd / 4] |= uint32_t(b) << (8 * (dd % 4));
            jac *= jd;
            atomicAdd(&sh_n[dd * nb + b], 1u);
          }
        }
      }
      if constexpr (PROC == P_PP_TTBARJ) {
        st = ppj_kinematics<float>(a, pdf, x, &kin, lum, nullptr);
      } else {
        st = gg_kinematics<PROC, float>(a, pdf, x, &kin, nullptr);
      }
      if (st == -5) ++acc.nnoconv;
      if (WOUT && st != 1) a.wout[i] = 0.0;
    }
    const bool pass = st == 1;
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    const int tot = __popc(m);
    if (fill + tot > 32 && !next_held) {
      ok = acquire(seq + 1);
      next_held = true;
      if (!ok) break;
    }
    if (pass) {
      const int pos = fill + __popc(m & ((1u << lane) - 1u));
      uint32_t* r = ring.rec + size_t(slot_of(pos < 32 ? seq : seq + 1)) * ws_words(PROC) * 32 + (pos & 31);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        r[(kWK + 4 * j + 0) * 32] = __float_as_uint(kin.k[j].e);
        r[(kWK + 4 * j + 1) * 32] = __float_as_uint(kin.k[j].x);
        r[(kWK + 4 * j + 2) * 32] = __float_as_uint(kin.k[j].y);
        r[(kWK + 4 * j + 3) * 32] = __float_as_uint(kin.k[j].z);
      }
      r[kWRs * 32] = __float_as_uint(kin.rs);
      if constexpr (PROC == P_PP_TTBARJ) {
        r[kWLgg * 32] = __float_as_uint(lum[0]);
        r[kWFlux * 32] = __float_as_uint(kin.shat);
#pragma unroll
        for (int j = 0; j < 6; ++j) r[(kWLum + j) * 32] = __float_as_uint(lum[1 + j]);
      } else {
        r[kWLgg * 32] = __float_as_uint(kin.lgg);
        r[kWFlux * 32] = __float_as_uint(kin.flux);
      }
      r[kWJac * 32] = __float_as_uint(jac);
      r[kWPsw * 32] = __double2loint(kin.psw);
      r[(kWPsw + 1) * 32] = __double2hiint(kin.psw);
#pragma unroll
      for (int j = 0; j < NW; ++j) r[(kWBin + j) * 32] = binw[j];
      if (WOUT) r[kWIdx * 32] = uint32_t(i);
      if constexpr (PROC == P_GG_TTBARG_MC) {
        r[kWCh * 32] = uint32_t(ch);
#pragma unroll
        for (int j = 0; j < kChannels; ++j) r[(kWDens + j) * 32] = __float_as_uint(dr[j]);
      }
    }
    fill += tot;
    if (fill >= 32) {
      publish(seq, 32);
      ++seq;
      fill -= 32;
      if (!next_held) ok = acquire(seq);
      next_held = false;
    }
  }
  if (ok) {
    publish(seq, fill);  // the last, partial slot (possibly empty)
    for (int e = 1; e <= ws_classes(PROC) && ok; ++e) {
      ok = acquire(seq + e);
      if (ok) publish(seq + e, -1);
    }
    seq += ws_classes(PROC) + 1;
  }
  return ok;
}

// This consumer thread's row store in the block's array of
// ws_consumer_warps x 32 x kWsRowBytes bytes (word j of consumer thread t at
// 16 (j C + t), C the consumer threads).
template <int PROC>
MC_D SmemRows ws_rows(const unsigned char* sh_rows) {
  return {uint32_t(__cvta_generic_to_shared(sh_rows)) + 16u * uint32_t(threadIdx.x - 32 * ws_producer_warps(PROC)),
          16u * 32u * ws_consumer_warps(PROC)};
}

// Consumer warp c (0 <= c < ws_consumer_warps(PROC)): evaluates |M|^2 for the events
// of its producers' slots until every stream it serves has delivered an end
// marker, and adds the weights w = f J to the Kahan sums, w_max and the
// histogram of w^2.  q0, q1: the next slot sequence numbers of its (up to two)
// streams, carried over between calls.  With WOUT the weights pass writes
// a.wout[i] = w.  Returns false when a wait gave up.
template <int PROC, bool WOUT, class Rows, bool PTS = false>
MC_D bool ws_consume(const KernelArgs& a, float* sh_w2, const WsRing& ring, Rows rows, int c, int& q0, int& q1,
                     Acc& acc) {
  constexpr int MAXD = ProcTraits<PROC>::MAXD;
  constexpr int NW = (MAXD + 3) / 4;
  const int lane = threadIdx.x & 31;
  const int ndim = a.ndim, nb = a.nbins;
  constexpr int NP = ws_producer_warps(PROC), NC = ws_consumer_warps(PROC), NS = ws_streams(PROC);
  bool live0 = true, live1 = NS > 1;
  for (int si = 0; live0 || live1; si ^= (NS > 1)) {
    if (si == 0 ? !live0 : !live1) si ^= 1;
    const int p = (c % NP) + si * NC;
    int& q = si == 0 ? q0 : q1;
    constexpr int S = ws_slots(PROC);
    const int s = p * S + q % S;
    if (!ws_wait(&ring.full[s], uint32_t(q / S) & 1u)) return false;
    const int cnt = ring.count[s];
    q += ws_classes(PROC);
    if (cnt < 0) {
      // release the marker's slot too: a later call (the next tile of a
      // batch) reuses it
      mbar_arrive(&ring.empty[s]);
      if (si == 0)
        live0 = false;
      else
        live1 = false;
      continue;
    }
    if (lane < cnt) {
      const uint32_t* r = ring.rec + size_t(s) * ws_words(PROC) * 32 + lane;
      GgKin<float> kin;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        kin.k[j] = {__uint_as_float(r[(kWK + 4 * j + 0) * 32]), __uint_as_float(r[(kWK + 4 * j + 1) * 32]),
                    __uint_as_float(r[(kWK + 4 * j + 2) * 32]), __uint_as_float(r[(kWK + 4 * j + 3) * 32])};
      kin.rs = __uint_as_float(r[kWRs * 32]);
      const float jac = __uint_as_float(r[kWJac * 32]);  // log q(x) with a points input
      kin.psw = __hiloint2double(int(r[(kWPsw + 1) * 32]), int(r[kWPsw * 32]));
      uint32_t binw[NW];
#pragma unroll
      for (int j = 0; j < NW; ++j) binw[j] = r[(kWBin + j) * 32];
      double w;
      if constexpr (PROC == P_PP_TTBARJ) {
        kin.shat = __uint_as_float(r[kWFlux * 32]);
        float lum[7];
        lum[0] = __uint_as_float(r[kWLgg * 32]);
#pragma unroll
        for (int j = 0; j < 6; ++j) lum[1 + j] = __uint_as_float(r[(kWLum + j) * 32]);
        w = ppj_weight<float>(a, kin, lum, nullptr);
      } else {
        kin.lgg = __uint_as_float(r[kWLgg * 32]);
        kin.flux = __uint_as_float(r[kWFlux * 32]);
        const float me2 = gg_me2<float>(a, kin, rows);
        w = gg_weight<float>(a, kin, me2);
      }
      if constexpr (PTS)
        w *= exp(-double(jac));
      else
        w *= double(jac);
      if (!isfinite(w)) {
        ++acc.nbad;
        w = 0.0;
      }
      if (WOUT) a.wout[r[kWIdx * 32]] = w;
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
      if constexpr (PROC == P_GG_TTBARG_MC) {
        const int ch = int(r[kWCh * 32]);
        if (w != 0.0) {
#pragma unroll
          for (int j = 0; j < kChannels; ++j) acc.wch[j] += w2 * double(__uint_as_float(r[(kWDens + j) * 32]));
        }
#pragma unroll
        for (int d = 0; d < 7; ++d)
          atomicAdd(&sh_w2[ch_grid_dim(d, ch) * nb + int((binw[d / 4] >> (8 * (d % 4))) & 0xffu)], float(w2));
      } else if (!PTS) {
#pragma unroll
        for (int dd = 0; dd < MAXD; ++dd)
          if (dd < ndim) atomicAdd(&sh_w2[dd * nb + int((binw[dd / 4] >> (8 * (dd % 4))) & 0xffu)], float(w2));
      }
    }
    mbar_arrive(&ring.empty[s]);
  }
  return true;
}

// WOUT: the weights pass (a.wout receives every event's weight; launches of
// at most 2^32 - 1 events).  SMROWS: the consumers' row spinors in shared
// memory (ws_rows_in_smem).
template <int PROC, bool WOUT, bool SMROWS, bool PTS = false>
__global__ void __launch_bounds__(ws_threads(PROC), 1) ws_integrand_kernel(KernelArgs a) {
  static_assert(PROC == P_GG_TTBARG || PROC == P_GG_TTBARG_7D || PROC == P_GG_TTBARG_MC || PROC == P_PP_TTBARJ,
                "gg -> t tbar g and p p -> t tbar + parton only");
  static_assert(ws_shape_ok(PROC), "launch shape");
  constexpr int NP = ws_producer_warps(PROC), NC = ws_consumer_warps(PROC), SLOTS = ws_slots(PROC) * NP;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[SLOTS], empty[SLOTS];
  __shared__ int count[SLOTS];
  __shared__ int failed;
  __shared__ BlockPartial warp_part[NP + NC];
  const int ndim = a.ndim, nb = a.nbins;
  const int nedge = ndim * (nb + 1), nhist = ndim * nb;
  const WsRing ring = {reinterpret_cast<uint32_t*>(smem), full, empty, count};
  unsigned char* sh_rows = smem + size_t(SLOTS) * ws_words(PROC) * 32 * 4;
  unsigned char* rest = sh_rows + (SMROWS ? size_t(NC) * 32 * kWsRowBytes : 0);
  float* sh_w2 = reinterpret_cast<float*>(rest);
  unsigned int* sh_n = reinterpret_cast<unsigned int*>(rest + size_t(nhist) * 4);
  float* sh_edges = reinterpret_cast<float*>(rest + ((size_t(nhist) * 8 + 15) / 16) * 16);
  float* sh_pdf = sh_edges + nedge;

  if (!PTS)
    for (int i = threadIdx.x; i < nedge; i += blockDim.x) sh_edges[i] = a.edges32[i];
  for (int i = threadIdx.x; i < nhist; i += blockDim.x) {
    sh_w2[i] = 0.0f;
    sh_n[i] = 0u;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(&full[s], 32);
      mbar_init(&empty[s], 32);
    }
    failed = 0;
  }
  SmPdf<float> pdf;
  {
    constexpr int NFL = ws_flavours(PROC);
    const int nx = a.pdf.nx;
    float* t = sh_pdf;
    float* f = t + nx;
    float* d = f + NFL * nx;
    build_pdf_tables<float>(a.pdf, a.logq2_f, a.fl, NFL, t, f, d);  // ends with __syncthreads
    for (int k = 0; k < NFL; ++k) pdf.tab[k] = {t, f + k * nx, d + k * nx, nx};
  }

  Acc acc;
  const int warp = threadIdx.x >> 5;
  bool ok = true;
  if (warp < NP) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(ws_producer_regs(PROC)));
    int seq = 0;
    ok = ws_produce<PROC, WOUT, PTS>(a, pdf, sh_edges, sh_n, ring, warp, 0, a.n, (long long)blockIdx.x * NP + warp,
                                (long long)gridDim.x * NP, seq, acc);
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ws_regs(PROC)));
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ws_consumer_regs(PROC)));
    const int c = warp - NP;
    int q0 = c / NP, q1 = q0;
    if constexpr (SMROWS) {
      SmemRows rows = ws_rows<PROC>(sh_rows);
      ok = ws_consume<PROC, WOUT, SmemRows, PTS>(a, sh_w2, ring, rows, c, q0, q1, acc);
    } else {
      ok = ws_consume<PROC, WOUT, NoRows, PTS>(a, sh_w2, ring, NoRows{}, c, q0, q1, acc);
    }
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(ws_regs(PROC)));
  }
  if (!ok) atomicExch(&failed, 1);
  __syncthreads();
  if constexpr (PROC == P_GG_TTBARG_MC) channel_sums_add(acc, a.wch);
  block_reduce(acc, warp_part, &a.partials[blockIdx.x]);
  if (threadIdx.x == 0 && failed) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    a.partials[blockIdx.x].sum_hi = nan;
    a.partials[blockIdx.x].sum2_hi = nan;
    a.partials[blockIdx.x].n_bad += 1;
    if (a.status) atomicExch(a.status, MC_ETIMEOUT);
  }
  for (int i = threadIdx.x; i < nhist; i += blockDim.x) {
    if (sh_n[i]) {
      atomicAdd(&a.hist_n[i], sh_n[i]);
      atomicAdd(&a.hist_w2[i], double(sh_w2[i]));
    }
  }
}

}  // namespace mc
