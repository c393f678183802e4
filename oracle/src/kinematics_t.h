// Oracle: RAMBO and the log-bicubic PDF interpolation over a scalar type T.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The arithmetic of rambo() (phasespace.cpp) and pdf_xfxq2() (pdf.cpp),
// which are these templates at T = double, written over T so that an
// operation-counting type (counted.h) can measure their work.  Grid values
// and knots stay double: they are data, not per-event arithmetic.
#pragma once
#include <cmath>
#include <vector>

#include "counted.h"
#include "oracle.h"

namespace orc {

// Sec. "RAMBO": eq. rambo-transform, eq. rambo-w0 and the massive extension
// (see phasespace.cpp for the readings).  u has 4n entries.  Returns 0, -1
// below threshold, or -5 if the equation for xi did not converge.
template <class T>
int rambo_t(int n, const double* masses, T sqrt_s, const T* u, P4T<T>* p, T* w) {
  using std::cos;
  using std::log;
  using std::pow;
  using std::sin;
  using std::sqrt;
  using std::fabs;
  using std::fmax;
  const double pi = M_PI;
  const T s = sqrt_s * sqrt_s;
  std::vector<P4T<T>> q(n);
  P4T<T> qsum;
  for (int i = 0; i < n; ++i) {
    const T c = T(2.0) * u[4 * i + 0] - T(1.0);
    const T phi = T(2.0 * pi) * u[4 * i + 1];
    const T q0 = -log(u[4 * i + 2] * u[4 * i + 3]);
    const T st = sqrt(fmax(T(0.0), T(1.0) - c * c));
    q[i] = {q0, q0 * st * cos(phi), q0 * st * sin(phi), q0 * c};
    qsum = add(qsum, q[i]);
  }
  const T mq = sqrt(dot(qsum, qsum));
  const T bx = -qsum.x / mq, by = -qsum.y / mq, bz = -qsum.z / mq;
  const T gamma = qsum.e / mq;
  const T a = T(1.0) / (T(1.0) + gamma);
  const T x = sqrt_s / mq;
  for (int i = 0; i < n; ++i) {
    const T bq = bx * q[i].x + by * q[i].y + bz * q[i].z;
    p[i].e = x * (gamma * q[i].e + bq);
    p[i].x = x * (q[i].x + bx * q[i].e + a * bq * bx);
    p[i].y = x * (q[i].y + by * q[i].e + a * bq * by);
    p[i].z = x * (q[i].z + bz * q[i].e + a * bq * bz);
  }
  const T w0 = T(std::pow(2.0 * pi, 4.0 - 3.0 * n) * std::pow(pi / 2.0, n - 1.0)) * pow(s, T(n - 2.0)) /
               T(std::tgamma(double(n)) * std::tgamma(n - 1.0));
  double msum = 0.0;
  bool massive = false;
  for (int i = 0; i < n; ++i) {
    msum += masses[i];
    if (masses[i] != 0.0) massive = true;
  }
  if (!massive) {
    *w = w0;
    return 0;
  }
  if (!(sqrt_s > T(msum))) return -1;
  T xi = sqrt(T(1.0) - (T(msum) / sqrt_s) * (T(msum) / sqrt_s));
  bool converged = false;
  for (int it = 0; it < 100; ++it) {
    T f = -sqrt_s, fp = T(0.0);
    for (int i = 0; i < n; ++i) {
      const T e = sqrt(T(masses[i] * masses[i]) + xi * xi * p[i].e * p[i].e);
      f += e;
      fp += xi * p[i].e * p[i].e / e;
    }
    const T step = f / fp;
    xi -= step;
    if (fabs(step) <= T(1e-15) * xi) {
      converged = true;
      break;
    }
  }
  if (!converged) return -5;
  T sum_k = T(0.0), prod = T(1.0), sum_k2_e = T(0.0);
  for (int i = 0; i < n; ++i) {
    const T e = sqrt(T(masses[i] * masses[i]) + xi * xi * p[i].e * p[i].e);
    P4T<T> k = {e, xi * p[i].x, xi * p[i].y, xi * p[i].z};
    const T kabs = sqrt(k.x * k.x + k.y * k.y + k.z * k.z);
    sum_k += kabs;
    prod *= kabs / k.e;
    sum_k2_e += kabs * kabs / k.e;
    p[i] = k;
  }
  const T wm = pow(s, T(2.0 - n)) * pow(sum_k, T(2.0 * n - 3.0)) * prod / sum_k2_e;
  *w = w0 * wm;
  return 0;
}

namespace pdf_detail {
template <class T>
T hermite(T tau, double h, T f0, T f1, T d0, T d1) {
  const T tau2 = tau * tau, tau3 = tau2 * tau;
  const T h00 = T(2.0) * tau3 - T(3.0) * tau2 + T(1.0);
  const T h10 = tau3 - T(2.0) * tau2 + tau;
  const T h01 = T(-2.0) * tau3 + T(3.0) * tau2;
  const T h11 = tau3 - tau2;
  return h00 * f0 + h10 * T(h) * d0 + h01 * f1 + h11 * T(h) * d1;
}
// Slope at knot i of values fv[] sampled at coordinates t[] (n knots): the
// mean of the two adjacent divided differences, one-sided at the ends.
template <class V>
V knot_slope(const double* t, int n, const V* fv, int i) {
  if (i == 0) return (fv[1] - fv[0]) / V(t[1] - t[0]);
  if (i == n - 1) return (fv[n - 1] - fv[n - 2]) / V(t[n - 1] - t[n - 2]);
  return V(0.5) * ((fv[i + 1] - fv[i]) / V(t[i + 1] - t[i]) + (fv[i] - fv[i - 1]) / V(t[i] - t[i - 1]));
}
inline int locate(const std::vector<double>& knots, double v) {
  const int n = int(knots.size());
  int i = 0;
  while (i + 1 < n - 1 && knots[i + 1] <= v) ++i;
  return i;
}
}  // namespace pdf_detail

// Sec. "LHAPDF: the Les Houches Accord PDF": x f(x, Q^2) by cubic Hermite
// interpolation in log x at the Q knots of the 4-knot stencil, then in
// log Q^2 (see pdf.cpp).  Slopes along x at the knots are properties of the
// grid (double); everything that depends on the query point is T.
template <class T>
T pdf_xfxq2_t(const Pdf& pdf, int pid, T x, T q2) {
  using std::log;
  const int fl = pdf.flavour_index(pid);
  const double nan = std::nan("");
  if (fl < 0) return T(nan);
  const double q2min = pdf.q[0] * pdf.q[0], q2max = pdf.q[pdf.nq - 1] * pdf.q[pdf.nq - 1];
  const double xv = value(x), q2v = value(q2);
  if (!(xv >= pdf.x[0] && xv <= pdf.x[pdf.nx - 1] && q2v >= q2min && q2v <= q2max)) return T(nan);
  std::vector<double> q2knots(pdf.nq);
  for (int j = 0; j < pdf.nq; ++j) q2knots[j] = pdf.q[j] * pdf.q[j];
  const int ix = pdf_detail::locate(pdf.x, xv);
  const int iq = pdf_detail::locate(q2knots, q2v);
  const T t = log(x), s = log(q2);
  const double hx = pdf.logx[ix + 1] - pdf.logx[ix];
  const T tau_x = (t - T(pdf.logx[ix])) / T(hx);
  std::vector<double> along_x(pdf.nx);
  std::vector<T> v(pdf.nq, T(0.0));
  const int jlo = iq > 0 ? iq - 1 : 0;
  const int jhi = iq + 2 < pdf.nq ? iq + 2 : pdf.nq - 1;
  for (int j = jlo; j <= jhi; ++j) {
    for (int i = 0; i < pdf.nx; ++i) along_x[i] = pdf.node(i, j, fl);
    const double d0 = pdf_detail::knot_slope(pdf.logx.data(), pdf.nx, along_x.data(), ix);
    const double d1 = pdf_detail::knot_slope(pdf.logx.data(), pdf.nx, along_x.data(), ix + 1);
    v[j] = pdf_detail::hermite(tau_x, hx, T(along_x[ix]), T(along_x[ix + 1]), T(d0), T(d1));
  }
  const double hq = pdf.logq2[iq + 1] - pdf.logq2[iq];
  const T tau_q = (s - T(pdf.logq2[iq])) / T(hq);
  const T e0 = pdf_detail::knot_slope(pdf.logq2.data(), pdf.nq, v.data(), iq);
  const T e1 = pdf_detail::knot_slope(pdf.logq2.data(), pdf.nq, v.data(), iq + 1);
  return pdf_detail::hermite(tau_q, hq, v[iq], v[iq + 1], e0, e1);
}

}  // namespace orc
