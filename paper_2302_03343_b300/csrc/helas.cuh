// Helicity-amplitude building blocks in the chiral (Weyl) representation.
//
// The thesis evaluates |M|^2 by summing helicity amplitudes of external
// wave functions joined by vertex and propagator routines (HELAS / ALOHA,
// Sec. "The MadFlow event generator").  Here a Dirac spinor is the pair of
// two-component spinors (L, R); gamma^mu a_mu acts as
//   (aslash psi)_L = (a.sigma) psi_R,  (aslash psi)_R = (a.sigmabar) psi_L,
//   a.sigma    = [[a0 - a3, -(a1 - i a2)], [-(a1 + i a2), a0 + a3]],
//   a.sigmabar = [[a0 + a3,   a1 - i a2 ], [  a1 + i a2,  a0 - a3]].
// A barred (row) spinor is stored already conjugated: rbar psi =
// rbar.L . psi_L + rbar.R . psi_R, so ubar(p) has L = conj(u_R), R = conj(u_L).
// Gluon polarisations are real linear vectors, so every gluon current and
// every slashed vector on the fermion line has real components.
#pragma once
#include "common.cuh"

namespace mc {

template <class R>
struct sp4 {
  cx<R> l0, l1, r0, r1;
};

template <class R> MC_D cx<R> dot(const sp4<R>& bar, const sp4<R>& col) {
  return bar.l0 * col.l0 + bar.l1 * col.l1 + bar.r0 * col.r0 + bar.r1 * col.r1;
}
template <class R> MC_D sp4<R> operator+(const sp4<R>& a, const sp4<R>& b) {
  return {a.l0 + b.l0, a.l1 + b.l1, a.r0 + b.r0, a.r1 + b.r1};
}
template <class R> MC_D sp4<R> operator-(const sp4<R>& a, const sp4<R>& b) {
  return {a.l0 - b.l0, a.l1 - b.l1, a.r0 - b.r0, a.r1 - b.r1};
}
template <class R> MC_D sp4<R> scale(const sp4<R>& a, R s) {
  return {a.l0 * s, a.l1 * s, a.r0 * s, a.r1 * s};
}

// (real a)slash applied to a column spinor.
template <class R> MC_D sp4<R> slash_col(const v4<R>& a, const sp4<R>& p) {
  const R A = a.e - a.z, D = a.e + a.z;
  const cx<R> B = mkc(a.x, -a.y), C = mkc(a.x, a.y);  // a1 - i a2, a1 + i a2
  sp4<R> o;
  o.l0 = A * p.r0 - B * p.r1;
  o.l1 = D * p.r1 - C * p.r0;
  o.r0 = D * p.l0 + B * p.l1;
  o.r1 = C * p.l0 + A * p.l1;
  return o;
}
// Row spinor times (real a)slash: (bar aslash).L = bar.R (a.sigmabar),
// (bar aslash).R = bar.L (a.sigma).
template <class R> MC_D sp4<R> slash_row(const sp4<R>& b, const v4<R>& a) {
  const R A = a.e - a.z, D = a.e + a.z;
  const cx<R> B = mkc(a.x, -a.y), C = mkc(a.x, a.y);
  sp4<R> o;
  o.l0 = D * b.r0 + C * b.r1;
  o.l1 = B * b.r0 + A * b.r1;
  o.r0 = A * b.l0 - C * b.l1;
  o.r1 = D * b.l1 - B * b.l0;
  return o;
}
// Fermion propagator numerator (pslash + m) times inv = 1/(p^2 - m^2).
template <class R> MC_D sp4<R> prop_col(const v4<R>& p, R m, R inv, const sp4<R>& s) {
  sp4<R> o = slash_col(p, s);
  o.l0 = (o.l0 + m * s.l0) * inv;
  o.l1 = (o.l1 + m * s.l1) * inv;
  o.r0 = (o.r0 + m * s.r0) * inv;
  o.r1 = (o.r1 + m * s.r1) * inv;
  return o;
}
template <class R> MC_D sp4<R> prop_row(const sp4<R>& s, const v4<R>& p, R m, R inv) {
  sp4<R> o = slash_row(s, p);
  o.l0 = (o.l0 + m * s.l0) * inv;
  o.l1 = (o.l1 + m * s.l1) * inv;
  o.r0 = (o.r0 + m * s.r0) * inv;
  o.r1 = (o.r1 + m * s.r1) * inv;
  return o;
}

// Two-component helicity eigenstates chi_+, chi_- along the direction of p.
// a = |p| + p_z is formed as p_T^2 / (|p| - p_z) when p_z < 0, so that it
// keeps full relative precision for momenta close to the -z axis (the direct
// sum cancels there).
template <class R> MC_D void helicity_states(const v4<R>& p, cx<R>* chip, cx<R>* chim) {
  const R pt2 = p.x * p.x + p.y * p.y;
  const R pabs = m_sqrt(pt2 + p.z * p.z);
  const R a = p.z >= R(0) ? pabs + p.z : pt2 / (pabs - p.z);
  if (!(a > R(0))) {  // along -z (or p = 0)
    chip[0] = mkc(R(0), R(0)); chip[1] = mkc(R(1), R(0));
    chim[0] = mkc(R(-1), R(0)); chim[1] = mkc(R(0), R(0));
    return;
  }
  const R inv = R(1) / m_sqrt(R(2) * pabs * a);
  chip[0] = mkc(a * inv, R(0));
  chip[1] = mkc(p.x * inv, p.y * inv);
  chim[0] = mkc(-p.x * inv, p.y * inv);
  chim[1] = mkc(a * inv, R(0));
}

// sqrt(E + |p|) and sqrt(E - |p|) without cancellation (E - |p| = m^2/(E + |p|)).
template <class R> MC_D void energy_roots(const v4<R>& p, R m, R* plus, R* minus) {
  const R pabs = m_sqrt(p.x * p.x + p.y * p.y + p.z * p.z);
  const R ep = p.e + pabs;
  *plus = m_sqrt(ep);
  *minus = m > R(0) ? m / *plus : R(0);
}

// u(p, lambda) = (sqrt(E - lambda|p|) chi_lambda, sqrt(E + lambda|p|) chi_lambda);
// returned as the barred row ubar.
template <class R> MC_D sp4<R> ubar_spinor(const v4<R>& p, R m, int hel) {
  cx<R> cp[2], cm[2];
  helicity_states(p, cp, cm);
  R sp, sm;
  energy_roots(p, m, &sp, &sm);
  const cx<R>* c = hel > 0 ? cp : cm;
  const R wl = hel > 0 ? sm : sp, wr = hel > 0 ? sp : sm;
  sp4<R> b;  // L = conj(u_R), R = conj(u_L)
  b.l0 = conj(c[0]) * wr; b.l1 = conj(c[1]) * wr;
  b.r0 = conj(c[0]) * wl; b.r1 = conj(c[1]) * wl;
  return b;
}
// v(p, lambda) = (sqrt(E + lambda|p|) chi_{-lambda}, -sqrt(E - lambda|p|) chi_{-lambda}).
template <class R> MC_D sp4<R> v_spinor(const v4<R>& p, R m, int hel) {
  cx<R> cp[2], cm[2];
  helicity_states(p, cp, cm);
  R sp, sm;
  energy_roots(p, m, &sp, &sm);
  const cx<R>* c = hel > 0 ? cm : cp;
  const R wl = hel > 0 ? sp : sm, wr = hel > 0 ? -sm : -sp;
  return {c[0] * wl, c[1] * wl, c[0] * wr, c[1] * wr};
}
template <class R> MC_D sp4<R> u_spinor(const v4<R>& p, R m, int hel) {
  cx<R> cp[2], cm[2];
  helicity_states(p, cp, cm);
  R sp, sm;
  energy_roots(p, m, &sp, &sm);
  const cx<R>* c = hel > 0 ? cp : cm;
  const R wl = hel > 0 ? sm : sp, wr = hel > 0 ? sp : sm;
  return {c[0] * wl, c[1] * wl, c[0] * wr, c[1] * wr};
}
// Barred v: vbar = v^dagger gamma^0.
template <class R> MC_D sp4<R> vbar_spinor(const v4<R>& p, R m, int hel) {
  const sp4<R> v = v_spinor(p, m, hel);
  return {conj(v.r0), conj(v.r1), conj(v.l0), conj(v.l1)};
}

// Vector current J^mu = rbar gamma^mu c of a barred row spinor and a column
// spinor (the components of rbar (a-slash) c = J^mu a_mu, read off
// slash_col): J^0 = L0 r0 + L1 r1 + R0 l0 + R1 l1,
// J^1 = L0 r1 + L1 r0 - R0 l1 - R1 l0, J^2 = -i (L0 r1 - L1 r0 - R0 l1 + R1 l0),
// J^3 = L0 r0 - L1 r1 - R0 l0 + R1 l1 (L, R the row's parts, l, r the column's).
template <class R> MC_D void vector_current(const sp4<R>& b, const sp4<R>& c, cx<R>* j) {
  const cx<R> a = b.l0 * c.r0, d = b.l1 * c.r1, e = b.r0 * c.l0, f = b.r1 * c.l1;
  const cx<R> g = b.l0 * c.r1, h = b.l1 * c.r0, k = b.r0 * c.l1, l = b.r1 * c.l0;
  j[0] = a + d + e + f;
  j[1] = g + h - k - l;
  const cx<R> t = g - h - k + l;
  j[2] = mkc(t.im, -t.re);  // -i t
  j[3] = a - d - e + f;
}
template <class R> MC_D cx<R> cdot4(const cx<R>* a, const cx<R>* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
template <class R> MC_D cx<R> cdot4(const cx<R>* a, const v4<R>& b) {
  return a[0] * b.e - a[1] * b.x - a[2] * b.y - a[3] * b.z;
}

// Two real transverse polarisation vectors of a massless momentum:
// eps1 = (0, cos th cos ph, cos th sin ph, -sin th), eps2 = (0, -sin ph, cos ph, 0).
template <class R> MC_D void linear_polarisations(const v4<R>& k, v4<R>* e1, v4<R>* e2) {
  const R kt2 = k.x * k.x + k.y * k.y;
  const R kabs = m_sqrt(kt2 + k.z * k.z);
  const R kt = m_sqrt(kt2);
  R cph = R(1), sph = R(0);
  if (kt > kabs * R(1e-7)) {
    cph = k.x / kt;
    sph = k.y / kt;
  }
  const R cth = k.z / kabs, sth = kt / kabs;
  *e1 = {R(0), cth * cph, cth * sph, -sth};
  *e2 = {R(0), -sph, cph, R(0)};
}

// Colour-ordered off-shell gluon current of an adjacent pair (coupling g = 1):
// W(X, Y) = -V(X, Y) / (qX + qY)^2 with the three-gluon vertex stripped of
// f^{abc}: V = (X.Y)(qX - qY) + Y (X.(qX + 2 qY)) - X (Y.(2 qX + qY)).
template <class R>
MC_D v4<R> gluon_current(const v4<R>& x, const v4<R>& qx, const v4<R>& y, const v4<R>& qy, R inv_q2) {
  const R xy = mdot(x, y);
  const R xq = mdot(x, qx) + R(2) * mdot(x, qy);
  const R yq = R(2) * mdot(y, qx) + mdot(y, qy);
  const R s = -inv_q2;
  return {s * (xy * (qx.e - qy.e) + y.e * xq - x.e * yq), s * (xy * (qx.x - qy.x) + y.x * xq - x.x * yq),
          s * (xy * (qx.y - qy.y) + y.y * xq - x.y * yq), s * (xy * (qx.z - qy.z) + y.z * xq - x.z * yq)};
}
// Colour-ordered four-gluon contact current of the string (x y z):
// [2 (X.Z) Y - (Y.Z) X - (X.Y) Z] / Q^2.
template <class R>
MC_D v4<R> gluon_contact(const v4<R>& x, const v4<R>& y, const v4<R>& z, R inv_q2) {
  const R a = R(2) * mdot(x, z) * inv_q2, b = -mdot(y, z) * inv_q2, c = -mdot(x, y) * inv_q2;
  return {a * y.e + b * x.e + c * z.e, a * y.x + b * x.x + c * z.x, a * y.y + b * x.y + c * z.y,
          a * y.z + b * x.z + c * z.z};
}

}  // namespace mc
