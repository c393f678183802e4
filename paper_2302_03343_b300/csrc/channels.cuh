// Three-channel phase space for g g -> t tbar g (thesis Sec. "Multi-channel
// Monte Carlo"): each channel is a sequential splitting P -> c + Q,
// Q -> a + b (Sec. "Sequential splitting") whose variables flatten one peak
// of |M|^2, and the event weight is f / p with p = sum_j alpha_j p_j, every
// channel's density evaluated at the event's point.
//  * channel 0, initial-state radiation: c = g, (a, b) = (t, tbar); ln pT of
//    the gluon flat on [pTcut, E_max], E_max = (shat - 4 m^2) / (2 sqrt(shat)),
//    its rapidity flat in the window where |y + y_b| < eta_cut (the lab-frame
//    cut, y_b = ln(x1/x2)/2) and pT cosh y <= E_max, its azimuth flat;
//  * channels 1 and 2, radiation off the top (anti-top): c = tbar (t),
//    (a, b) = (t, g) ((tbar, g)); ln(s_Q - m^2 + Delta) flat on
//    [m^2, (sqrt(shat) - m)^2], Delta = m pTcut; c's direction flat;
//  * the direction of a in the rest frame of Q (axes of the partonic frame)
//    is flat.
// Weights w = dPhi_3 / du follow from dPhi_3 = d^3p_c / ((2 pi)^3 2 E_c)
// dPhi_2(Q -> a b) and eq. 2bodyps.  Each channel has its own VEGAS grid
// over its 5 variables and all share the (x1, x2) grid: 17 grid dimensions,
// used dimension d of a channel-ch event in grid dimension
// ch_grid_dim(d, ch).
#pragma once
#include "common.cuh"

namespace mc {

constexpr int kChannels = 3;
constexpr int kChannelGridDims = 2 + 5 * kChannels;

MC_HD int ch_grid_dim(int d, int ch) { return d < 2 ? d : 2 + 5 * ch + (d - 2); }

// Per-event constants of the channel maps.
template <class R>
struct ChCtx {
  R m, rs, s, etacut, yb;
  R lpt0, lpt1, emax;  // channel 0: ln pTcut, ln E_max, E_max
  R ls0, ls1, delta;   // channels 1, 2: ln Delta, ln(s_max - m^2 + Delta), Delta
  bool ok0, ok12;      // whether the channel can generate at this shat
};

template <class R>
MC_D ChCtx<R> ch_ctx(R m, R rs, R ptcut, R etacut, R yb) {
  ChCtx<R> c;
  c.m = m;
  c.rs = rs;
  c.s = rs * rs;
  c.etacut = etacut;
  c.yb = yb;
  c.emax = (c.s - R(4) * m * m) / (R(2) * rs);
  c.ok0 = c.emax > ptcut && ptcut > R(0);
  c.lpt0 = m_log(ptcut);
  c.lpt1 = m_log(c.ok0 ? c.emax : ptcut * R(2));
  c.delta = m * ptcut;
  const R smax = (rs - m) * (rs - m);
  c.ok12 = smax > m * m && c.delta > R(0);
  c.ls0 = m_log(c.delta);
  c.ls1 = m_log(c.ok12 ? smax - m * m + c.delta : R(2) * c.delta);
  return c;
}

// Rapidity window of channel 0's gluon at transverse momentum pt.
template <class R>
MC_D bool ch_ywin(const ChCtx<R>& c, R pt, R* lo, R* hi) {
  const R ymax = m_acosh(m_max(R(1), c.emax / pt));
  *lo = m_max(-c.etacut - c.yb, -ymax);
  *hi = m_min(c.etacut - c.yb, ymax);
  return *hi > *lo;
}

template <class R>
MC_D v4<R> boost_from_rest(const v4<R>& q, R mq, const v4<R>& v) {
  const R e = (q.e * v.e + q.x * v.x + q.y * v.y + q.z * v.z) / mq;
  const R f = (v.e + e) / (q.e + mq);
  return {e, v.x + f * q.x, v.y + f * q.y, v.z + f * q.z};
}
template <class R>
MC_D v4<R> boost_to_rest(const v4<R>& q, R mq, const v4<R>& v) {
  const R e = (q.e * v.e - q.x * v.x - q.y * v.y - q.z * v.z) / mq;
  const R f = (v.e + e) / (q.e + mq);
  return {e, v.x - f * q.x, v.y - f * q.y, v.z - f * q.z};
}

// dPhi_2(Q -> a b) factor |p*| dOmega* / (16 pi^2 M_Q) per unit square: a is
// a top quark, b the anti-top (channel 0) or the gluon (channels 1, 2).
template <class R>
MC_D R ch_decay_pabs(int ch, R m, R sq, R mq) {
  return ch == 0 ? R(0.5) * m_sqrt(m_max(R(0), sq - R(4) * m * m)) : (sq - m * m) / (R(2) * mq);
}

// Channel ch at u[5]: t, tbar, g in the partonic frame and w = dPhi_3/du;
// false when the channel cannot generate there.
template <class R>
MC_D bool ch_forward(int ch, const ChCtx<R>& c, const R* u, v4<R>* t, v4<R>* tb, v4<R>* g, R* w) {
  const R pi = R(kPi);
  R sp, cp;
  m_sincos2pi(u[2], &sp, &cp);
  R sq, wc;
  v4<R> pc;
  if (ch == 0) {
    if (!c.ok0) return false;
    const R pt = m_exp(c.lpt0 + u[0] * (c.lpt1 - c.lpt0));
    R ylo, yhi;
    if (!ch_ywin(c, pt, &ylo, &yhi)) return false;
    const R y = ylo + u[1] * (yhi - ylo);
    const R eg = pt * m_cosh(y);
    pc = {eg, pt * cp, pt * sp, pt * m_sinh(y)};
    sq = c.s - R(2) * c.rs * eg;
    wc = pt * pt * (c.lpt1 - c.lpt0) * (yhi - ylo) * (R(2) * pi) / (R(16) * pi * pi * pi);
  } else {
    if (!c.ok12) return false;
    const R tt = m_exp(c.ls0 + u[0] * (c.ls1 - c.ls0));
    sq = c.m * c.m - c.delta + tt;
    const R m2 = c.m * c.m;
    const R lam = c.s * c.s + sq * sq + m2 * m2 - R(2) * (c.s * sq + c.s * m2 + sq * m2);
    const R pca = m_sqrt(m_max(R(0), lam)) / (R(2) * c.rs);
    const R cth = R(2) * u[1] - R(1);
    const R sth = m_sqrt(m_max(R(0), (R(1) - cth) * (R(1) + cth)));
    pc = {m_sqrt(pca * pca + m2), pca * sth * cp, pca * sth * sp, pca * cth};
    wc = pca * tt * (c.ls1 - c.ls0) * (R(4) * pi) / (R(32) * pi * pi * pi * c.rs);
  }
  const R mb = ch == 0 ? c.m : R(0);
  if (!(sq > (c.m + mb) * (c.m + mb))) return false;
  const R mq = m_sqrt(sq);
  const v4<R> q = {c.rs - pc.e, -pc.x, -pc.y, -pc.z};
  const R ps = ch_decay_pabs(ch, c.m, sq, mq);
  R s2p, c2p;
  m_sincos2pi(u[4], &s2p, &c2p);
  const R c2 = R(2) * u[3] - R(1);
  const R s2 = m_sqrt(m_max(R(0), (R(1) - c2) * (R(1) + c2)));
  const v4<R> na = {m_sqrt(ps * ps + c.m * c.m), ps * s2 * c2p, ps * s2 * s2p, ps * c2};
  const v4<R> nb = {m_sqrt(ps * ps + mb * mb), -na.x, -na.y, -na.z};
  const v4<R> pa = boost_from_rest(q, mq, na), pb = boost_from_rest(q, mq, nb);
  if (ch == 0) {
    *t = pa; *tb = pb; *g = pc;
  } else if (ch == 1) {
    *t = pa; *g = pb; *tb = pc;
  } else {
    *tb = pa; *g = pb; *t = pc;
  }
  *w = wc * ps * (R(4) * pi) / (R(16) * pi * pi * mq);
  return true;
}

// The channel-ch variables u[5] of the point (t, tbar, g) and the channel's
// weight there; false outside the channel's support.
template <class R>
MC_D bool ch_inverse(int ch, const ChCtx<R>& c, const v4<R>& t, const v4<R>& tb, const v4<R>& g, R* u, R* w) {
  const R pi = R(kPi);
  const v4<R> pc = ch == 0 ? g : (ch == 1 ? tb : t);
  const v4<R> pa = ch == 2 ? tb : t;
  const v4<R> pb = ch == 0 ? tb : g;
  const v4<R> q = pa + pb;
  R sq, wc;
  if (ch == 0) {
    if (!c.ok0) return false;
    const R pt = m_sqrt(pc.x * pc.x + pc.y * pc.y);
    u[0] = (m_log(pt) - c.lpt0) / (c.lpt1 - c.lpt0);
    R ylo, yhi;
    if (!(u[0] >= R(0) && u[0] <= R(1)) || !ch_ywin(c, pt, &ylo, &yhi)) return false;
    const R pabs = m_sqrt(pt * pt + pc.z * pc.z);
    const R y = R(0.5) * m_log((pabs + pc.z) / (pabs - pc.z));
    u[1] = (y - ylo) / (yhi - ylo);
    sq = c.s - R(2) * c.rs * pc.e;
    wc = pt * pt * (c.lpt1 - c.lpt0) * (yhi - ylo) * (R(2) * pi) / (R(16) * pi * pi * pi);
  } else {
    if (!c.ok12) return false;
    const R a2 = R(2) * mdot(pa, pb);  // s_Q - m^2 for the massless gluon
    const R tt = a2 + c.delta;
    u[0] = (m_log(tt) - c.ls0) / (c.ls1 - c.ls0);
    sq = c.m * c.m + a2;
    const R pca = m_sqrt(pc.x * pc.x + pc.y * pc.y + pc.z * pc.z);
    u[1] = R(0.5) * (pc.z / pca + R(1));
    wc = pca * tt * (c.ls1 - c.ls0) * (R(4) * pi) / (R(32) * pi * pi * pi * c.rs);
  }
  const R ph = m_atan2(pc.y, pc.x) / (R(2) * pi);
  u[2] = ph < R(0) ? ph + R(1) : ph;
  if (!(sq > R(0))) return false;
  const R mq = m_sqrt(sq);
  const v4<R> na = boost_to_rest(q, mq, pa);
  const R naa = m_sqrt(na.x * na.x + na.y * na.y + na.z * na.z);
  u[3] = R(0.5) * (na.z / naa + R(1));
  const R ph2 = m_atan2(na.y, na.x) / (R(2) * pi);
  u[4] = ph2 < R(0) ? ph2 + R(1) : ph2;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (!(u[k] >= R(0) && u[k] <= R(1))) return false;
  const R ps = ch_decay_pabs(ch, c.m, sq, mq);
  *w = wc * ps * (R(4) * pi) / (R(16) * pi * pi * mq);
  return true;
}

// Density of one grid dimension at v (edges[0..nb], v = 1 in the last bin):
// 1 / (nb * width of the bin holding v), by bisection.
template <class R>
MC_D R grid_density(const R* e, int nb, R v) {
  int lo = 0, hi = nb;  // e[lo] <= v < e[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (v >= e[mid]) lo = mid; else hi = mid;
  }
  return R(1) / (R(nb) * (e[lo + 1] - e[lo]));
}

}  // namespace mc
