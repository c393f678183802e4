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

// Reciprocal and square root in FP64 from an FP32 seed plus one
// Newton-Raphson step (r <- r (2 - x r); y <- y + (x - y^2)/(2y)): about
// 1e-14 relative for arguments inside the FP32 range, at the cost of two or
// three FP64 operations instead of a full FP64 division or square root.
MC_D double rcp_nr(double x) {
  const double r = double(1.0f / float(x));
  return fma(r, fma(-x, r, 1.0), r);
}
MC_D double sqrt_nr(double x) {
  const float yf = sqrtf(float(x));
  const double y = double(yf);
  return fma(double(0.5f / yf), fma(-y, y, x), y);
}

// RAMBO in the FP32 mode: isotropic momenta in FP32, the conformal
// transformation (eq. rambo-transform) in FP64, the massive rescaling and the
// weights in FP32 on the accurately boosted momenta.  Same outputs as rambo()
// (momenta in FP32), returns 0 or -5.
template <int N>
MC_D int rambo_fp32(const float* masses, float sqrt_s, double w0_coef, const float* u, v4<float>* out, double* w) {
  float fe[N], fx[N], fy[N], fz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float c = 2.0f * u[4 * i] - 1.0f;
    float sp, cp;
    sincospif(2.0f * u[4 * i + 1], &sp, &cp);
    const float q0 = -logf(u[4 * i + 2] * u[4 * i + 3]);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    fe[i] = q0; fx[i] = q0 * st * cp; fy[i] = q0 * st * sp; fz[i] = q0 * c;
  }
  double qe[N], qx[N], qy[N], qz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) { qe[i] = fe[i]; qx[i] = fx[i]; qy[i] = fy[i]; qz[i] = fz[i]; }
  double se = qe[0], sx = qx[0], sy = qy[0], sz = qz[0];
#pragma unroll
  for (int i = 1; i < N; ++i) { se += qe[i]; sx += qx[i]; sy += qy[i]; sz += qz[i]; }
  // 1/M by one FP64 Newton step on the FP32 rsqrt seed: r (3 - M^2 r^2) / 2
  const double m2q = se * se - sx * sx - sy * sy - sz * sz;
  const double r0 = double(rsqrtf(float(m2q)));
  const double inv_mq = r0 * fma(-0.5 * m2q, r0 * r0, 1.5);
  const double bx = -sx * inv_mq, by = -sy * inv_mq, bz = -sz * inv_mq;
  const double gamma = se * inv_mq;
  const double a = rcp_nr(1.0 + gamma);
  const double x = double(sqrt_s) * inv_mq;
  float pe[N], px[N], py[N], pz[N];
  double de = double(sqrt_s), dx = 0.0, dy = 0.0, dz = 0.0;
#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
    const double bq = bx * qx[i] + by * qy[i] + bz * qz[i];
    const double t = qe[i] + a * bq;
    const double e = x * (gamma * qe[i] + bq), vx = x * (qx[i] + bx * t), vy = x * (qy[i] + by * t),
                 vz = x * (qz[i] + bz * t);
    pe[i] = float(e); px[i] = float(vx); py[i] = float(vy); pz[i] = float(vz);
    de -= e; dx -= vx; dy -= vy; dz -= vz;
  }
  // the last momentum by conservation: P - sum of the others
  pe[N - 1] = float(de); px[N - 1] = float(dx); py[N - 1] = float(dy); pz[N - 1] = float(dz);
  const float s = sqrt_s * sqrt_s;
  float w0 = float(w0_coef);
#pragma unroll
  for (int i = 0; i < N - 2; ++i) w0 *= s;
  float msum = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) msum += masses[i];
  float xi = sqrtf(fmaxf(0.0f, 1.0f - (msum / sqrt_s) * (msum / sqrt_s)));
  float k0[N];
  float resid = 0.0f;
  for (int it = 0; it < 16; ++it) {
    float f = -sqrt_s, fp = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      k0[i] = sqrtf(masses[i] * masses[i] + xi * xi * pe[i] * pe[i]);
      f += k0[i];
      fp += xi * pe[i] * pe[i] / k0[i];
    }
    resid = f;
    const float step = f / fp;
    xi -= step;
    if (fabsf(step) <= 4e-7f * xi) break;  // a few ulps: the FP32 root is reached
  }
  // accept the root when the residual is at FP32 rounding level of sqrt_s
  if (!(xi > 0.0f) || !(fabsf(resid) <= 1e-5f * sqrt_s)) return -5;
  float sum_k = 0.0f, prod_k = 1.0f, denom = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    k0[i] = sqrtf(masses[i] * masses[i] + xi * xi * pe[i] * pe[i]);
    const float kabs = xi * pe[i];
    sum_k += kabs;
    prod_k *= kabs;
    float others = 1.0f;
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j != i) others *= k0[j];
    denom += kabs * kabs * others;
  }
  // w_m = s^(2-N) (sum|k|)^(2N-3) prod|k_i| / (prod k_j^0 sum |k_i|^2/k_i^0)
  float num = prod_k;
#pragma unroll
  for (int i = 0; i < 2 * N - 3; ++i) num *= sum_k;
  float sp = 1.0f;
#pragma unroll
  for (int i = 0; i < N - 2; ++i) sp *= s;
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = {k0[i], xi * px[i], xi * py[i], xi * pz[i]};
  *w = double(w0) * double(num / (sp * denom));
  return 0;
}

// Three-body phase space by sequential two-body branchings (thesis table
// tab:hierarchical, n = 3): P -> p3 (massless gluon) + q2 (mass M2), then
// q2 -> p2 + p1 (top pair of mass m each) in the rest frame of q2, boosted
// back.  Uniforms: u0 -> phi_3, u1 -> cos theta_3, u2 -> M2 in [2m, sqrt_s],
// u3 -> phi_2, u4 -> cos theta_2.  Weight per unit hypercube (re-derived from
// eq. 2bodyps and eq. sequential-splitting, the printed eq. sequential-weight
// not being dimensionless):
//   w = pi^-3 4^-2 / sqrt_s * (sqrt_s - 2m) * |p*_2| |p*_3|.
// p[0] = top, p[1] = anti-top, p[2] = gluon, FP64.
template <class R>
MC_D void hierarchical3(double m, double sqrt_s, const R* u, v4<double>* p, double* w) {
  R s3, c3p, s2, c2p;
  m_sincos2pi(u[0], &s3, &c3p);
  m_sincos2pi(u[3], &s2, &c2p);
  const double c3 = 2.0 * double(u[1]) - 1.0, c2 = 2.0 * double(u[4]) - 1.0;
  const double st3 = sqrt(fmax(0.0, 1.0 - c3 * c3)), st2 = sqrt(fmax(0.0, 1.0 - c2 * c2));
  const double s = sqrt_s * sqrt_s;
  const double m2 = 2.0 * m + double(u[2]) * (sqrt_s - 2.0 * m);
  const double p3 = (s - m2 * m2) / (2.0 * sqrt_s);
  const double n3x = st3 * double(c3p), n3y = st3 * double(s3), n3z = c3;
  p[2] = {p3, p3 * n3x, p3 * n3y, p3 * n3z};
  const v4<double> q = {sqrt(p3 * p3 + m2 * m2), -p3 * n3x, -p3 * n3y, -p3 * n3z};
  const double p2 = 0.5 * m2 * sqrt(fmax(0.0, 1.0 - 4.0 * m * m / (m2 * m2)));
  const double e2 = sqrt(p2 * p2 + m * m);
  const double n2x = st2 * double(c2p), n2y = st2 * double(s2), n2z = c2;
  // boost (e, +-p2 n2) from the rest frame of q (mass m2) to the lab
  const double qn = q.x * n2x + q.y * n2y + q.z * n2z;
  const double inv_m2 = 1.0 / m2;
  const double ea = (q.e * e2 + p2 * qn) * inv_m2, eb = (q.e * e2 - p2 * qn) * inv_m2;
  const double fa = (e2 + ea) / (q.e + m2), fb = (e2 + eb) / (q.e + m2);
  p[1] = {ea, p2 * n2x + fa * q.x, p2 * n2y + fa * q.y, p2 * n2z + fa * q.z};
  p[0] = {eb, -p2 * n2x + fb * q.x, -p2 * n2y + fb * q.y, -p2 * n2z + fb * q.z};
  *w = (sqrt_s - 2.0 * m) * p2 * p3 / (kPi * kPi * kPi * 16.0 * sqrt_s);
}

}  // namespace mc
