// Phase-space generators, device side (thesis Sec. "Phase space generation
// from particle collisions": eq. 2bodyps; Sec. "RAMBO": eq. rambo-transform,
// eq. rambo-w0 and the massive extension).
//
// RAMBO's isotropic massless momenta are drawn in the working precision; the
// conformal Lorentz transformation, the massive rescaling and the weights are
// taken in FP64 in both precision modes (the Newton iteration for xi runs in
// the working precision and is polished by one FP64 step).
#pragma once
#include "common.cuh"

namespace mc {

// Two-body decay of P = (sqrt_s, 0) into masses m1 = m2 = m at polar angle
// theta (cos theta = c) and azimuth phi = 2 pi u of particle 1.  Weight per
// unit square: lambda^(1/2) / ((2 pi)^2 8 s) * 4 pi = beta / (8 pi).
template <class R>
MC_D R two_body_equal(R sqrt_s, R m, R c, R uphi, v4<R>* p1, v4<R>* p2) {
  const R e = sqrt_s * R(0.5);
  const R beta = m > R(0) ? m_sqrt(m_max(R(0), R(1) - R(4) * m * m / (sqrt_s * sqrt_s))) : R(1);
  const R pabs = e * beta;
  const R st = m_sqrt(m_max(R(0), R(1) - c * c));
  R sp, cp;
  m_sincos2pi(uphi, &sp, &cp);
  const v4<R> k = {e, pabs * st * cp, pabs * st * sp, pabs * c};
  *p1 = k;
  *p2 = {e, -k.x, -k.y, -k.z};
  return beta / R(8.0 * kPi);
}

// RAMBO for N particles in the frame P = (sqrt_s, 0).  u: 4N uniforms
// (cos theta, phi, and two for the energy q0 = -log(u3 u4) per particle).
// w0_coef = (2 pi)^(4-3N) (pi/2)^(N-1) / (Gamma(N) Gamma(N-1)) so that
// w0 = w0_coef s^(N-2).  Returns 0, or -5 when the working-precision root of
// the rescaling equation misses by more than 1e-5 sqrt_s before the FP64 step.
template <class R, int N>
MC_D int rambo(const double* masses, double sqrt_s, double w0_coef, const R* u, v4<double>* p, double* w) {
  // isotropic massless momenta with energy density q0 exp(-q0)
  v4<double> q[N];
  v4<double> qs = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const R c = R(2) * u[4 * i] - R(1);
    R sp, cp;
    m_sincos2pi(u[4 * i + 1], &sp, &cp);
    const R q0 = -m_log(u[4 * i + 2] * u[4 * i + 3]);
    const R st = m_sqrt(m_max(R(0), R(1) - c * c));
    q[i] = {double(q0), double(q0 * st * cp), double(q0 * st * sp), double(q0 * c)};
    qs = qs + q[i];
  }
  // conformal transformation to total momentum P (FP64)
  const double mq = sqrt(mdot(qs, qs));
  const double inv_mq = 1.0 / mq;
  const double bx = -qs.x * inv_mq, by = -qs.y * inv_mq, bz = -qs.z * inv_mq;
  const double gamma = qs.e * inv_mq;
  const double a = 1.0 / (1.0 + gamma);
  const double x = sqrt_s * inv_mq;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double bq = bx * q[i].x + by * q[i].y + bz * q[i].z;
    p[i] = {x * (gamma * q[i].e + bq), x * (q[i].x + bx * q[i].e + a * bq * bx),
            x * (q[i].y + by * q[i].e + a * bq * by), x * (q[i].z + bz * q[i].e + a * bq * bz)};
  }
  const double s = sqrt_s * sqrt_s;
  double w0 = w0_coef;
#pragma unroll
  for (int i = 0; i < N - 2; ++i) w0 *= s;
  double msum = 0.0;
  bool massive = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    msum += masses[i];
    massive |= masses[i] != 0.0;
  }
  if (!massive) {
    *w = w0;
    return 0;
  }
  // massive rescaling: sqrt_s = sum_i sqrt(m_i^2 + xi^2 (p_i^0)^2), Newton in R
  R xi = R(sqrt(fmax(0.0, 1.0 - (msum / sqrt_s) * (msum / sqrt_s))));
  R e2[N], m2[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    e2[i] = R(p[i].e * p[i].e);
    m2[i] = R(masses[i] * masses[i]);
  }
  const R rs = R(sqrt_s);
  for (int it = 0; it < 40; ++it) {
    R f = -rs, fp = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const R k0 = m_sqrt(m2[i] + xi * xi * e2[i]);
      f += k0;
      fp += xi * e2[i] / k0;
    }
    const R step = f / fp;
    xi -= step;
    if (m_abs(step) <= (sizeof(R) == 4 ? R(2e-7) : R(1e-15)) * xi) break;
  }
  // one FP64 Newton step from the working-precision root
  double xd = double(xi), f = -sqrt_s, fp = 0.0;
  double k0[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    k0[i] = sqrt(masses[i] * masses[i] + xd * xd * p[i].e * p[i].e);
    f += k0[i];
    fp += xd * p[i].e * p[i].e / k0[i];
  }
  const double dxi = f / fp;
  const double xn = xd - dxi;
  // k0(xn) to first order in the (tiny) step
  double kabs[N];
  double sum_k = 0.0, prod_k = 1.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    k0[i] -= dxi * xd * p[i].e * p[i].e / k0[i];
    kabs[i] = xn * p[i].e;  // |p_i| = p_i^0 for the massless momenta
    sum_k += kabs[i];
    prod_k *= kabs[i];
  }
  if (!(fabs(f) <= 1e-5 * sqrt_s) || !(xn > 0.0)) return -5;
  // w_m = s^(2-N) (sum|k|)^(2N-3) prod(|k_i|/k_i^0) / sum(|k_i|^2 / k_i^0)
  double denom = 0.0;  // prod_j k_j^0 * sum_i |k_i|^2 / k_i^0, without divisions
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double others = 1.0;
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j != i) others *= k0[j];
    denom += kabs[i] * kabs[i] * others;
  }
  double num = prod_k;
#pragma unroll
  for (int i = 0; i < 2 * N - 3; ++i) num *= sum_k;
  double sp = 1.0;
#pragma unroll
  for (int i = 0; i < N - 2; ++i) sp *= s;
  const double wm = num / (sp * denom);
#pragma unroll
  for (int i = 0; i < N; ++i) p[i] = {k0[i], xn * p[i].x, xn * p[i].y, xn * p[i].z};
  *w = w0 * wm;
  return 0;
}

}  // namespace mc
