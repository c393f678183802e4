// Oracle: phase-space generators.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "Phase space generation from particle collisions":
// eq. phase-space (the measure), eq. 2bodyps (two-body element), table
// tab:hierarchical (sequential 1->2 branchings) and Sec. "RAMBO"
// (eq. rambo-transform, eq. rambo-w0 and the massive extension).
//
// Pins (tests/test_oracle_phasespace.py): momentum conservation and on-shell
// masses to 1e-12; massless RAMBO weight equal to the analytic volume; massive
// two-body volume beta/(8 pi); massive three-body volume from RAMBO,
// from the hierarchical generator and from quadrature of the Dalitz area.
#include <cmath>

#include "kinematics_t.h"
#include "oracle.h"

namespace orc {

static double kallen(double x, double y, double z) {
  return x * x + y * y + z * z - 2.0 * x * y - 2.0 * x * z - 2.0 * y * z;
}

// Two-body decay of P = (sqrt_s, 0) into masses m1, m2 at polar angle theta
// and azimuth phi of particle 1; eq. 2bodyps: dPhi_2 = lambda^(1/2) / ((2 pi)^2
// 8 s) dOmega.  The weight is per unit square of (cos(theta)+1)/2, phi/(2 pi):
// dOmega = 4 pi du1 du2.
void two_body(double sqrt_s, double m1, double m2, double cos_theta, double phi, P4* p, double* w) {
  const double s = sqrt_s * sqrt_s;
  const double lam = kallen(s, m1 * m1, m2 * m2);
  const double root = lam > 0.0 ? std::sqrt(lam) : 0.0;
  const double pabs = root / (2.0 * sqrt_s);
  const double sin_theta = std::sqrt(std::fmax(0.0, 1.0 - cos_theta * cos_theta));
  const double px = pabs * sin_theta * std::cos(phi);
  const double py = pabs * sin_theta * std::sin(phi);
  const double pz = pabs * cos_theta;
  p[0] = {std::sqrt(pabs * pabs + m1 * m1), px, py, pz};
  p[1] = {std::sqrt(pabs * pabs + m2 * m2), -px, -py, -pz};
  const double pi = M_PI;
  *w = root / ((2.0 * pi) * (2.0 * pi) * 8.0 * s) * 4.0 * pi;
}

// RAMBO (Sec. "RAMBO").  Massless step: isotropic q_i with energy density
// q0 exp(-q0) from four uniforms each, then the conformal transformation
// eq. rambo-transform to total momentum P, flat weight eq. rambo-w0.  Massive
// step: rescale three-momenta by xi solving sqrt(s) = sum_i sqrt(m_i^2 +
// xi^2 (p_i^0)^2) by Newton's method, k_i = (sqrt(m_i^2 + xi^2 (p_i^0)^2),
// xi p_i) and weight w_0 w_m.  Readings: the printed k_i^0 drops xi (it is
// restored, as the constraint on xi requires), and the first sum in w_m runs
// over all n particles.
int rambo(int n, const double* masses, double sqrt_s, const double* u, P4* p, double* w) {
  return rambo_t<double>(n, masses, sqrt_s, u, p, w);
}

// Boost v, given in the rest frame of q (mass mq), to the frame where q has
// its stated momentum.
static P4 boost_from_rest(const P4& q, double mq, const P4& v) {
  const double e = (q.e * v.e + q.x * v.x + q.y * v.y + q.z * v.z) / mq;
  const double f = (v.e + e) / (q.e + mq);
  return {e, v.x + f * q.x, v.y + f * q.y, v.z + f * q.z};
}

// Hierarchical generator, table tab:hierarchical, with three readings of
// garbled passages: cos(theta_i) = 2 u_i2 - 1; the intermediate mass step
// M_{i-1} = mu_{i-1} + u_i3 (M_i - mu_i) with mu_i = m_1 + ... + m_i; and the
// weight re-derived from eq. 2bodyps and eq. sequential-splitting (the printed
// eq. sequential-weight is not dimensionless for n = 2):
//   w = pi^(3-2n) 4^(1-n) / M_n * prod_{i=3..n} (M_i - mu_i) * prod_{i=2..n} |p*_i|
// with |p*_i| = lambda^(1/2)(M_i^2, M_{i-1}^2, m_i^2) / (2 M_i).  Uniforms are
// consumed for i = n, n-1, ..., 2 as (u_i1 -> phi, u_i2 -> cos theta, u_i3 ->
// mass for i >= 3).
int hierarchical(int n, const double* masses, double sqrt_s, const double* u, P4* p, double* w) {
  const double pi = M_PI;
  std::vector<double> mu(n + 1, 0.0);  // mu[i] = m_1 + ... + m_i (1-based)
  for (int i = 1; i <= n; ++i) mu[i] = mu[i - 1] + masses[i - 1];
  if (!(sqrt_s > mu[n])) return -1;
  P4 q = {sqrt_s, 0.0, 0.0, 0.0};
  double big_m = sqrt_s;  // M_i
  double weight = std::pow(pi, 3.0 - 2.0 * n) * std::pow(4.0, 1.0 - n) / sqrt_s;
  int iu = 0;
  for (int i = n; i >= 2; --i) {
    const double phi = 2.0 * pi * u[iu++];
    const double c = 2.0 * u[iu++] - 1.0;
    double m_prev;
    if (i >= 3) {
      const double span = big_m - mu[i];
      m_prev = mu[i - 1] + u[iu++] * span;
      weight *= span;
    } else {
      m_prev = masses[0];
    }
    const double mi = masses[i - 1];
    const double lam = kallen(big_m * big_m, m_prev * m_prev, mi * mi);
    const double pabs = (lam > 0.0 ? std::sqrt(lam) : 0.0) / (2.0 * big_m);
    weight *= pabs;
    const double st = std::sqrt(std::fmax(0.0, 1.0 - c * c));
    const P4 pi_rest = {std::sqrt(pabs * pabs + mi * mi), pabs * st * std::cos(phi),
                        pabs * st * std::sin(phi), pabs * c};
    const P4 qprev_rest = {std::sqrt(pabs * pabs + m_prev * m_prev), -pi_rest.x, -pi_rest.y,
                           -pi_rest.z};
    p[i - 1] = boost_from_rest(q, big_m, pi_rest);
    const P4 qprev = boost_from_rest(q, big_m, qprev_rest);
    if (i == 2) p[0] = qprev;
    q = qprev;
    big_m = m_prev;
  }
  *w = weight;
  return 0;
}

}  // namespace orc

extern "C" {

static void unpack(const orc::P4* p, int n, double* out) {
  for (int i = 0; i < n; ++i) {
    out[4 * i + 0] = p[i].e;
    out[4 * i + 1] = p[i].x;
    out[4 * i + 2] = p[i].y;
    out[4 * i + 3] = p[i].z;
  }
}

void orc_two_body(double sqrt_s, double m1, double m2, double cos_theta, double phi, double* p,
                  double* w) {
  orc::P4 q[2];
  orc::two_body(sqrt_s, m1, m2, cos_theta, phi, q, w);
  unpack(q, 2, p);
}

int orc_rambo(int n, const double* masses, double sqrt_s, const double* u, double* p, double* w) {
  std::vector<orc::P4> q(n);
  const int rc = orc::rambo(n, masses, sqrt_s, u, q.data(), w);
  unpack(q.data(), n, p);
  return rc;
}

int orc_hierarchical(int n, const double* masses, double sqrt_s, const double* u, double* p,
                     double* w) {
  std::vector<orc::P4> q(n);
  const int rc = orc::hierarchical(n, masses, sqrt_s, u, q.data(), w);
  unpack(q.data(), n, p);
  return rc;
}
}
