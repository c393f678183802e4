// Oracle: multi-channel sampling of g g -> t tbar g.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "Multi-channel Monte Carlo": with channel densities p_i and
// probabilities alpha_i (sum 1), points are drawn from channel i with
// probability alpha_i and weighted by f / p, p = sum_i alpha_i p_i; the
// alpha_i change only the variance, and are adjusted iteratively to reduce
// it (Kleiss & Pittau 1994, cited there).  The thesis proposes this as the
// remedy for RAMBO's flat sampling (Sec. "Unweighted event exporter").
//
// Readings (the thesis gives the method, not the channels):
//  * Three channels, each a sequential splitting (Sec. "Sequential
//    splitting") P -> c + Q, Q -> a + b, with a mapping that flattens one
//    peak of |M|^2:
//      0: c = g, (a, b) = (t, tbar): initial-state radiation; the gluon's
//         transverse momentum flat in ln pT on [pTcut, E_max], E_max =
//         (shat - 4 m^2) / (2 sqrt(shat)) (soft and collinear emission off
//         the beams go as dpT^2 / pT^2), its rapidity flat in the window
//         where it passes the lab-frame cut |y + y_b| < eta_cut (y_b =
//         ln(x1/x2)/2) and E_g = pT cosh y <= E_max, its azimuth flat: the
//         gluon cuts are built into the channel;
//      1: c = tbar, (a, b) = (t, g): radiation off the top; s_Q = (p_t +
//         p_g)^2 sampled flat in ln(s_Q - m^2 + Delta), Delta = m * pTcut,
//         on [m^2, (sqrt(shat) - m)^2]; the tbar direction flat;
//      2: as 1 with t and tbar exchanged.
//    The decay angles of Q in its rest frame (axes of the partonic frame)
//    are flat.  Final-state order t, tbar, g as everywhere.
//  * Weight of channel i at its point: w_i = dPhi_3 / du, from
//    dPhi_3 = d^3p_c / ((2 pi)^3 2 E_c) dPhi_2(Q -> a b) and eq. 2bodyps,
//    dPhi_2 = |p*| dOmega* / (16 pi^2 M_Q): channel 0 with d^3p/(2E) =
//    pT dpT dy dphi / 2, channels 1, 2 with d^3p_c/(2 E_c) = |p_c| ds_Q
//    dOmega_c / (4 sqrt(shat)).
//  * With VEGAS: every channel has its own grid over its 5 variables and the
//    channels share the grid of (x1, x2) (17 grid dimensions in all); an
//    event of channel i takes its 7 uniforms through the (x1, x2) grid and
//    channel i's grid.  Channel j's density at a point is rho_j(u_j) / w_j,
//    u_j the point's channel-j variables and rho_j channel j's grid density
//    there; the event weight is f J_x / sum_j alpha_j rho_j(u_j) / w_j, J_x
//    the Jacobian of the (x1, x2) grid.  The histograms of w^2 are filled in
//    the grids the event used, so channel i's grid adapts to the events it
//    draws, weighted by (f/p)^2: the density it aims for is |f| alpha_i p_i /
//    p, its share of the integrand.
//  * The channel is chosen by Philox call 254 of the event: u = (k + 0.5)
//    2^-24 with k the top 24 bits of word 0, channel i the first with
//    u < alpha_0 + ... + alpha_i.
//  * Where a channel cannot generate (channel 0 when E_max <= pTcut or the
//    rapidity window is empty) an event it draws has weight zero and its
//    density there is zero; the estimate stays unbiased, since p is the sum
//    of the densities the channels actually generate with.
//  * alpha update: alpha_i <- alpha_i W_i^beta / sum_j alpha_j W_j^beta,
//    W_i = (1/N) sum_events w^2 p_i / p (beta = 1/2), then a floor alpha_min
//    and renormalisation.
//
// Pins (tests/test_oracle_channels.py): forward then inverse map is the
// identity; every channel's mean weight is the three-body phase-space volume
// (Dalitz quadrature); each full-support channel's density integrates to one
// under the others; the multi-channel integral equals RAMBO's; the alpha
// update by hand and its fixed point on a two-peak toy.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace orc {

namespace {

constexpr double kPi = M_PI;

double kallen3(double x, double y, double z) { return x * x + y * y + z * z - 2.0 * x * y - 2.0 * x * z - 2.0 * y * z; }

P4 boost_from(const P4& q, double mq, const P4& v) {  // v given in the rest frame of q
  const double e = (q.e * v.e + q.x * v.x + q.y * v.y + q.z * v.z) / mq;
  const double f = (v.e + e) / (q.e + mq);
  return {e, v.x + f * q.x, v.y + f * q.y, v.z + f * q.z};
}

P4 boost_to(const P4& q, double mq, const P4& v) {  // v into the rest frame of q
  const double e = (q.e * v.e - q.x * v.x - q.y * v.y - q.z * v.z) / mq;
  const double f = (v.e + e) / (q.e + mq);
  return {e, v.x - f * q.x, v.y - f * q.y, v.z - f * q.z};
}

struct Roles {
  int c, a, b;  // recoiler and pair (indices into t, tbar, g)
};
Roles roles(int ch) {
  if (ch == 0) return {2, 0, 1};
  if (ch == 1) return {1, 0, 2};
  return {0, 1, 2};
}

double mass_of(int k, double m) { return k == 2 ? 0.0 : m; }

// Mapping of u0 (channel 0: ln pT range; channels 1, 2: range of
// ln(s_Q - m^2 + Delta), and Delta); false when the channel cannot generate
// at this shat.
struct SMap {
  double lo, hi, shift;
};

bool s_map(int ch, double m, double rs, double ptcut, SMap* sm) {
  const double s = rs * rs;
  if (ch == 0) {
    const double emax = (s - 4.0 * m * m) / (2.0 * rs);
    if (!(emax > ptcut) || !(ptcut > 0.0)) return false;
    *sm = {std::log(ptcut), std::log(emax), emax};
    return true;
  }
  const double delta = m * ptcut;
  const double smax = (rs - m) * (rs - m);
  if (!(smax > m * m) || !(delta > 0.0)) return false;
  *sm = {std::log(delta), std::log(smax - m * m + delta), delta};
  return true;
}

}  // namespace

// The cut geometry a channel needs: the gluon pT cut, |eta_lab| < etacut and
// the rapidity y_b = ln(x1/x2)/2 of the partonic frame.
struct Cuts {
  double ptcut, etacut, yb;
};

// Rapidity window of channel 0's gluon at transverse momentum pt; false if
// empty.
static bool y_window(double pt, double emax, const Cuts& k, double* lo, double* hi) {
  const double ymax = std::acosh(std::fmax(1.0, emax / pt));
  *lo = std::fmax(-k.etacut - k.yb, -ymax);
  *hi = std::fmin(k.etacut - k.yb, ymax);
  return *hi > *lo;
}

// Channel ch at the point u[5]: momenta p[3] (t, tbar, g, partonic frame)
// and weight dPhi_3/du; returns false when the channel cannot generate.
bool channel_forward(int ch, double m, double rs, const Cuts& k, const double* u, P4* p, double* w) {
  SMap sm;
  if (!s_map(ch, m, rs, k.ptcut, &sm)) return false;
  const Roles r = roles(ch);
  const double s = rs * rs;
  const double mc = mass_of(r.c, m), ma = mass_of(r.a, m), mb = mass_of(r.b, m);
  const double phi = 2.0 * kPi * u[2];
  double sq, wc;  // s_Q and the recoiler's factor d^3p_c / ((2 pi)^3 2 E_c) per du0 du1 du2
  if (ch == 0) {
    const double pt = std::exp(sm.lo + u[0] * (sm.hi - sm.lo));
    double ylo, yhi;
    if (!y_window(pt, sm.shift, k, &ylo, &yhi)) return false;
    const double y = ylo + u[1] * (yhi - ylo);
    const double eg = pt * std::cosh(y);
    p[r.c] = {eg, pt * std::cos(phi), pt * std::sin(phi), pt * std::sinh(y)};
    sq = s - 2.0 * rs * eg;
    wc = pt * (pt * (sm.hi - sm.lo)) * (yhi - ylo) * 2.0 * kPi / (16.0 * kPi * kPi * kPi);
  } else {
    const double t = std::exp(sm.lo + u[0] * (sm.hi - sm.lo));
    sq = m * m - sm.shift + t;
    const double ds_du = t * (sm.hi - sm.lo);
    const double pc = std::sqrt(std::fmax(0.0, kallen3(s, sq, m * m))) / (2.0 * rs);
    const double cth = 2.0 * u[1] - 1.0;
    const double sth = std::sqrt(std::fmax(0.0, (1.0 - cth) * (1.0 + cth)));
    p[r.c] = {std::sqrt(pc * pc + mc * mc), pc * sth * std::cos(phi), pc * sth * std::sin(phi), pc * cth};
    wc = pc * ds_du * (2.0 * 2.0 * kPi) / (32.0 * kPi * kPi * kPi * rs);
  }
  if (!(sq > (ma + mb) * (ma + mb))) return false;
  const double mq = std::sqrt(sq);
  const P4 q = {rs - p[r.c].e, -p[r.c].x, -p[r.c].y, -p[r.c].z};
  const double ps = std::sqrt(std::fmax(0.0, kallen3(sq, ma * ma, mb * mb))) / (2.0 * mq);
  const double c2 = 2.0 * u[3] - 1.0, s2 = std::sqrt(std::fmax(0.0, (1.0 - c2) * (1.0 + c2)));
  const double phi2 = 2.0 * kPi * u[4];
  const P4 na = {std::sqrt(ps * ps + ma * ma), ps * s2 * std::cos(phi2), ps * s2 * std::sin(phi2), ps * c2};
  const P4 nb = {std::sqrt(ps * ps + mb * mb), -na.x, -na.y, -na.z};
  p[r.a] = boost_from(q, mq, na);
  p[r.b] = boost_from(q, mq, nb);
  *w = wc * ps * (4.0 * kPi) / (16.0 * kPi * kPi * mq);
  return true;
}

// The point's channel-ch variables u[5] and that channel's weight there;
// false when the point lies outside the channel's support.
bool channel_inverse(int ch, double m, double rs, const Cuts& k, const P4* p, double* u, double* w) {
  SMap sm;
  if (!s_map(ch, m, rs, k.ptcut, &sm)) return false;
  const Roles r = roles(ch);
  const P4& c = p[r.c];
  const P4 q = add(p[r.a], p[r.b]);
  const double sq = dot(q, q);
  if (ch == 0) {
    const double pt = std::sqrt(c.x * c.x + c.y * c.y);
    u[0] = (std::log(pt) - sm.lo) / (sm.hi - sm.lo);
    double ylo, yhi;
    if (!(u[0] >= 0.0 && u[0] <= 1.0) || !y_window(pt, sm.shift, k, &ylo, &yhi)) return false;
    const double pabs = std::sqrt(pt * pt + c.z * c.z);
    const double y = 0.5 * std::log((pabs + c.z) / (pabs - c.z));
    u[1] = (y - ylo) / (yhi - ylo);
  } else {
    const double pc = std::sqrt(c.x * c.x + c.y * c.y + c.z * c.z);
    const double a2 = 2.0 * dot(p[r.a], p[r.b]);  // s_Q - m^2 for a massless b
    u[0] = (std::log(a2 + sm.shift) - sm.lo) / (sm.hi - sm.lo);
    u[1] = 0.5 * (c.z / pc + 1.0);
  }
  double ph = std::atan2(c.y, c.x) / (2.0 * kPi);
  u[2] = ph < 0.0 ? ph + 1.0 : ph;
  const double mq = std::sqrt(sq);
  const P4 na = boost_to(q, mq, p[r.a]);
  const double pa = std::sqrt(na.x * na.x + na.y * na.y + na.z * na.z);
  u[3] = 0.5 * (na.z / pa + 1.0);
  double ph2 = std::atan2(na.y, na.x) / (2.0 * kPi);
  u[4] = ph2 < 0.0 ? ph2 + 1.0 : ph2;
  for (int i = 0; i < 5; ++i)
    if (!(u[i] >= 0.0 && u[i] <= 1.0)) return false;
  P4 tmp[3];  // the weight of the channel at these variables (the forward formula)
  return channel_forward(ch, m, rs, k, u, tmp, w);
}

// Grid density at the point v of the unit interval: 1 / (N_b width of the
// bin holding v); v = 1 belongs to the last bin.
static double grid_density(const double* edges, int nbins, double v) {
  int b = 0;
  while (b < nbins - 1 && v >= edges[b + 1]) ++b;
  return 1.0 / (double(nbins) * (edges[b + 1] - edges[b]));
}

static double g_alpha[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};

// Multi-channel event: uniforms -> VEGAS map -> channel choice -> channel
// map -> densities of all channels -> weight.  rec as for the other
// processes, plus the channel and its three densities.
void channels_event(const orc_integrand& in, const Pdf* pdf, int nbins, const double* edges, int prec, uint64_t seed,
                    uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec, double* dens) {
  std::memset(rec, 0, sizeof(*rec));
  dens[0] = dens[1] = dens[2] = 0.0;
  // channel choice: Philox call 254
  const uint32_t ctr[4] = {uint32_t(uint64_t(ev)), uint32_t(uint64_t(ev) >> 32), iteration, (gid & 0xffu) | (254u << 8)};
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  uint32_t wd[4];
  philox4x32_10(ctr, key, wd);
  const double uc = (double(wd[0] >> 8) + 0.5) * 0x1p-24;
  int ch = 2;
  double cum = 0.0;
  for (int i = 0; i < 3; ++i) {
    cum += g_alpha[i];
    if (uc < cum) {
      ch = i;
      break;
    }
  }
  const int ndim = 7;
  uint64_t k[16];
  event_uniform_ints(seed, iteration, gid, prec, ndim, ev, k);
  const int bits = uniform_bits(prec);
  double jx = 1.0, jrest = 1.0;
  for (int d = 0; d < ndim; ++d) {
    int b;
    double jd;
    rec->x[d] = vegas_map_1d(edges + channel_grid_dim(d, ch) * (nbins + 1), nbins, bits, k[d], &b, &jd);
    rec->bin[d] = b;
    (d < 2 ? jx : jrest) *= jd;
  }
  rec->jac = jx * jrest;
  rec->status = 0;
  rec->pass = 0;
  rec->channel = ch;
  const double s = in.sqrt_s * in.sqrt_s, m = in.m_top;
  const double x1 = rec->x[0], x2 = rec->x[1], shat = x1 * x2 * s;
  rec->x1 = x1;
  rec->x2 = x2;
  rec->shat = shat;
  if (!(shat > 4.0 * m * m)) return;
  const double rs = std::sqrt(shat);
  P4 p[5];
  p[0] = {rs / 2.0, 0.0, 0.0, rs / 2.0};
  p[1] = {rs / 2.0, 0.0, 0.0, -rs / 2.0};
  const Cuts cuts = {in.ptcut_g, in.etacut_g, 0.5 * std::log(x1 / x2)};
  double wi;
  if (!channel_forward(ch, m, rs, cuts, rec->x + 2, p + 2, &wi)) return;
  for (int i = 0; i < 5; ++i) {
    rec->p[i][0] = p[i].e;
    rec->p[i][1] = p[i].x;
    rec->p[i][2] = p[i].y;
    rec->p[i][3] = p[i].z;
  }
  // densities of all channels at the point (rest of the grid: dims 2..6)
  double pden = 0.0;
  for (int j = 0; j < 3; ++j) {
    double uj[5], wj;
    if (j == ch) {
      dens[j] = 1.0 / (jrest * wi);
    } else if (channel_inverse(j, m, rs, cuts, p + 2, uj, &wj) && wj > 0.0) {
      double rho = 1.0;
      for (int d = 0; d < 5; ++d)
        rho *= grid_density(edges + channel_grid_dim(d + 2, j) * (nbins + 1), nbins, uj[d]);
      dens[j] = rho / wj;
    }
    pden += g_alpha[j] * dens[j];
  }
  rec->ps_weight = 1.0 / pden;  // dPhi per unit of the mixture's variables
  // the gluon cuts in the lab frame
  const P4& pg = p[4];
  const double pt = std::sqrt(pg.x * pg.x + pg.y * pg.y);
  const double pabs = std::sqrt(pt * pt + pg.z * pg.z);
  const double eta = 0.5 * std::log((pabs + pg.z) / (pabs - pg.z)) + 0.5 * std::log(x1 / x2);
  if (!(pt > in.ptcut_g) || !(std::fabs(eta) < in.etacut_g)) return;
  rec->pass = 1;
  const double q2 = in.mu_f * in.mu_f;
  rec->lumi = pdf_xfxq2(*pdf, 21, x1, q2) / x1 * pdf_xfxq2(*pdf, 21, x2, q2) / x2;
  rec->me2 = me2_gg_ttbarg(in.alpha_s, m, p);
  rec->f = rec->lumi * rec->me2 / (2.0 * shat) * in.gev2pb / pden;
  rec->weight = rec->f * jx;
}

}  // namespace orc

extern "C" {

void orc_set_channel_alpha(const double* alpha) {
  const double t = alpha[0] + alpha[1] + alpha[2];
  for (int i = 0; i < 3; ++i) orc::g_alpha[i] = alpha[i] / t;
}

int orc_channel_forward(int ch, double m, double rs, double ptcut, double etacut, double yb, const double* u, double* p,
                        double* w) {
  orc::P4 q[3];
  if (!orc::channel_forward(ch, m, rs, {ptcut, etacut, yb}, u, q, w)) return -1;
  for (int i = 0; i < 3; ++i) {
    p[4 * i] = q[i].e;
    p[4 * i + 1] = q[i].x;
    p[4 * i + 2] = q[i].y;
    p[4 * i + 3] = q[i].z;
  }
  return 0;
}

int orc_channel_inverse(int ch, double m, double rs, double ptcut, double etacut, double yb, const double* p, double* u,
                        double* w) {
  orc::P4 q[3];
  for (int i = 0; i < 3; ++i) q[i] = {p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]};
  return orc::channel_inverse(ch, m, rs, {ptcut, etacut, yb}, q, u, w) ? 0 : -1;
}

void orc_channels_event(const orc_integrand* in, const void* pdf, int nbins, const double* edges, int prec,
                        uint64_t seed, uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec,
                        double* dens) {
  orc::channels_event(*in, static_cast<const orc::Pdf*>(pdf), nbins, edges, prec, seed, iteration, gid, ev, rec, dens);
}

// One iteration of events first .. first+n-1: sums of w and w^2, w_max, and
// the alpha-update sums W_i = sum w^2 p_i / p (dens_i / sum_j alpha_j dens_j).
void orc_channels_iterate(const orc_integrand* in, const void* pdf, int nbins, const double* edges, int prec,
                          uint64_t seed, uint32_t iteration, uint32_t gid, int64_t first, int64_t n, double* sums,
                          double* wch) {
  long double s1 = 0, s2 = 0, c[3] = {0, 0, 0};
  double wmax = 0.0;
  orc_event_record rec;
  double dens[3];
  for (int64_t i = 0; i < n; ++i) {
    orc::channels_event(*in, static_cast<const orc::Pdf*>(pdf), nbins, edges, prec, seed, iteration, gid, first + i,
                        &rec, dens);
    const double w = rec.weight;
    s1 += w;
    s2 += (long double)w * w;
    if (w > wmax) wmax = w;
    if (w != 0.0) {
      const double pden = orc::g_alpha[0] * dens[0] + orc::g_alpha[1] * dens[1] + orc::g_alpha[2] * dens[2];
      for (int j = 0; j < 3; ++j) c[j] += (long double)w * w * dens[j] / pden;
    }
  }
  sums[0] = double(s1);
  sums[1] = double(s2);
  sums[2] = wmax;
  for (int j = 0; j < 3; ++j) wch[j] = double(c[j] / n);
}

// alpha_i <- alpha_i W_i^beta / sum_j alpha_j W_j^beta, floored at amin and
// renormalised.
void orc_channel_update(int n, const double* alpha, const double* w, double beta, double amin, double* out) {
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += (out[i] = alpha[i] * std::pow(w[i], beta));
  if (!(t > 0.0)) {
    for (int i = 0; i < n; ++i) out[i] = alpha[i];
    return;
  }
  double t2 = 0.0;
  for (int i = 0; i < n; ++i) t2 += (out[i] = std::fmax(out[i] / t, amin));
  for (int i = 0; i < n; ++i) out[i] /= t2;
}
}
