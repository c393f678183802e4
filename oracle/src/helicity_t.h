// Oracle: g g -> t tbar g from helicity amplitudes (formulation C), over a
// scalar type T.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "The MadFlow event generator": |M|^2 as a sum over helicity
// configurations of squared colour-ordered amplitudes contracted with the
// colour matrix.  The same colour-ordered Feynman rules as formulation A
// (matrix_elements.cpp: vertex i g gamma^mu, quark propagator
// (k-slash + m)/(k^2 - m^2), gluon currents J(ab), J(abc) of Berends and
// Giele with the three- and four-gluon vertices), applied to spinors instead
// of Dirac matrices:
//   A_s(ordering abc) = ubar_s(t) [ eps_a S_a ( i g^3 eps_b X_c - i g^2 J(bc) v )
//                                  - i g^2 J(ab) X_c + i g J(abc) v ],
//   X_c = S_ab eps_c v,  S_a = S(p_t - q_a),  S_ab = S(p_t - q_a - q_b) = S(q_c - p_tbar),
// in the Dirac representation with spinors in the z spin basis and real
// linear gluon polarisations (so every gluon current is a real
// four-vector).  Spins: the sum over gluon polarisations and top spins at a
// fixed antitop spin is half the full sum (the antitop's polarisation is zero
// at tree level in QCD: the term linear in its spin vector is parity-odd or
// time-reversal-odd, and there is no absorptive part), so one antitop spin is
// evaluated and the sum doubled.  Averages: 1/4 (spins), 1/64 (colours).
//
// Pins (tests/test_oracle_me.py): equal to formulations A and B to 1e-12 at
// the same phase-space points.  Instantiated with Counted (counted.h) it
// gives the algorithmic operation count of the |M|^2 (tests/golden/ and the
// roofline of the fused integrand kernel).
#pragma once
#include <array>
#include <cmath>
#include <vector>

#include "counted.h"
#include "oracle.h"

namespace orc {
namespace hel {

template <class T>
struct Cx {
  T re = 0, im = 0;
};
template <class T>
inline Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
inline Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
inline Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T>
inline Cx<T> rmul(const T& s, const Cx<T>& a) { return {s * a.re, s * a.im}; }
template <class T>
inline Cx<T> conj(const Cx<T>& a) { return {a.re, -a.im}; }

template <class T>
using Spinor = std::array<Cx<T>, 4>;

// k-slash psi for a real four-vector k (Dirac representation):
// [[k^0, -S], [S, -k^0]] with S = sigma.k = [[k^z, k^x - i k^y], [k^x + i k^y, -k^z]].
template <class T>
Spinor<T> slash(const P4T<T>& k, const Spinor<T>& p) {
  // (k^x -+ i k^y) c
  auto minus_i = [&](const Cx<T>& c) -> Cx<T> { return {k.x * c.re + k.y * c.im, k.x * c.im - k.y * c.re}; };
  auto plus_i = [&](const Cx<T>& c) -> Cx<T> { return {k.x * c.re - k.y * c.im, k.x * c.im + k.y * c.re}; };
  const Cx<T> sl0 = rmul(k.z, p[2]) + minus_i(p[3]);
  const Cx<T> sl1 = plus_i(p[2]) - rmul(k.z, p[3]);
  const Cx<T> su0 = rmul(k.z, p[0]) + minus_i(p[1]);
  const Cx<T> su1 = plus_i(p[0]) - rmul(k.z, p[1]);
  return {rmul(k.e, p[0]) - sl0, rmul(k.e, p[1]) - sl1, su0 - rmul(k.e, p[2]), su1 - rmul(k.e, p[3])};
}
template <class T>
Spinor<T> sadd(const Spinor<T>& a, const Spinor<T>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2], a[3] + b[3]}; }
template <class T>
Spinor<T> ssub(const Spinor<T>& a, const Spinor<T>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2], a[3] - b[3]}; }
template <class T>
Spinor<T> sscale(const T& s, const Spinor<T>& a) { return {rmul(s, a[0]), rmul(s, a[1]), rmul(s, a[2]), rmul(s, a[3])}; }
// i s a for a real s
template <class T>
Spinor<T> sscale_i(const T& s, const Spinor<T>& a) {
  Spinor<T> r;
  for (int k = 0; k < 4; ++k) r[k] = {-(s * a[k].im), s * a[k].re};
  return r;
}
// (k-slash + m) psi / (k^2 - m^2), the reciprocal denominator given
template <class T>
Spinor<T> prop(const P4T<T>& k, const T& m, const T& inv, const Spinor<T>& p) {
  return sscale(inv, sadd(slash(k, p), sscale(m, p)));
}
// ubar psi for the adjoint row ubar = u^dagger gamma^0
template <class T>
Cx<T> row_dot(const Spinor<T>& ubar, const Spinor<T>& p) {
  return ubar[0] * p[0] + ubar[1] * p[1] + ubar[2] * p[2] + ubar[3] * p[3];
}

// Dirac spinors (Dirac representation, spin along z): chi_0 = (1, 0), chi_1 = (0, 1),
// u = (sqrt(E+m) chi; sigma.p chi / sqrt(E+m)), v = (sigma.p chi / sqrt(E+m); sqrt(E+m) chi).
template <class T>
Spinor<T> u_spinor(const P4T<T>& p, const T& m, int s) {
  using std::sqrt;
  const T r = sqrt(p.e + m), ir = T(1.0) / r;
  // sigma.p chi_0 = (p^z, p^x + i p^y), sigma.p chi_1 = (p^x - i p^y, -p^z)
  const Cx<T> a = s == 0 ? Cx<T>{p.z, T(0.0)} : Cx<T>{p.x, -p.y};
  const Cx<T> b = s == 0 ? Cx<T>{p.x, p.y} : Cx<T>{-p.z, T(0.0)};
  const Cx<T> up0 = s == 0 ? Cx<T>{r, T(0.0)} : Cx<T>{T(0.0), T(0.0)};
  const Cx<T> up1 = s == 0 ? Cx<T>{T(0.0), T(0.0)} : Cx<T>{r, T(0.0)};
  return {up0, up1, rmul(ir, a), rmul(ir, b)};
}
template <class T>
Spinor<T> v_spinor(const P4T<T>& p, const T& m, int s) {
  using std::sqrt;
  const T r = sqrt(p.e + m), ir = T(1.0) / r;
  const Cx<T> a = s == 0 ? Cx<T>{p.z, T(0.0)} : Cx<T>{p.x, -p.y};
  const Cx<T> b = s == 0 ? Cx<T>{p.x, p.y} : Cx<T>{-p.z, T(0.0)};
  const Cx<T> lo0 = s == 0 ? Cx<T>{r, T(0.0)} : Cx<T>{T(0.0), T(0.0)};
  const Cx<T> lo1 = s == 0 ? Cx<T>{T(0.0), T(0.0)} : Cx<T>{r, T(0.0)};
  return {rmul(ir, a), rmul(ir, b), lo0, lo1};
}
// ubar = u^dagger gamma^0 = (u0*, u1*, -u2*, -u3*)
template <class T>
Spinor<T> adjoint(const Spinor<T>& u) {
  return {conj(u[0]), conj(u[1]), Cx<T>{-u[2].re, u[2].im}, Cx<T>{-u[3].re, u[3].im}};
}

// Two real transverse polarisation vectors of a massless momentum k.
template <class T>
void linear_pols(const P4T<T>& k, P4T<T>* e1, P4T<T>* e2) {
  using std::sqrt;
  const T kabs = sqrt(k.x * k.x + k.y * k.y + k.z * k.z);
  const T n[3] = {k.x / kabs, k.y / kabs, k.z / kabs};
  T a[3];
  const T perp = sqrt(n[0] * n[0] + n[1] * n[1]);
  if (perp > T(1e-6)) {  // a = n x z / |n x z|
    a[0] = n[1] / perp;
    a[1] = -n[0] / perp;
    a[2] = T(0.0);
  } else {
    a[0] = T(1.0);
    a[1] = T(0.0);
    a[2] = T(0.0);
  }
  const T b[3] = {n[1] * a[2] - n[2] * a[1], n[2] * a[0] - n[0] * a[2], n[0] * a[1] - n[1] * a[0]};
  *e1 = {T(0.0), a[0], a[1], a[2]};
  *e2 = {T(0.0), b[0], b[1], b[2]};
}

// Three-gluon vertex contracted with two currents, as in formulation A:
// g [(x.y)(qx - qy) + y (x.(qx + 2 qy)) - x (y.(2 qx + qy))]; the current of
// two gluons is -V / (qx + qy)^2, and the contact term of the ordered string
// x y z is g^2 / Q^2 [2 (x.z) y - (y.z) x - (x.y) z].
template <class T>
P4T<T> vertex3(const T& g, const P4T<T>& x, const P4T<T>& qx, const P4T<T>& y, const P4T<T>& qy) {
  const T xy = dot(x, y);
  const T xq = dot(x, add(qx, scale(qy, T(2.0))));
  const T yq = dot(y, add(scale(qx, T(2.0)), qy));
  const P4T<T> d = sub(qx, qy);
  return scale(sub(add(scale(d, xy), scale(y, xq)), scale(x, yq)), g);
}
template <class T>
P4T<T> current2(const T& g, const P4T<T>& x, const P4T<T>& qx, const P4T<T>& y, const P4T<T>& qy) {
  const P4T<T> q = add(qx, qy);
  return scale(vertex3(g, x, qx, y, qy), T(-1.0) / dot(q, q));
}
template <class T>
P4T<T> current4(const T& g, const P4T<T>& x, const P4T<T>& y, const P4T<T>& z, const P4T<T>& q) {
  const T c = g * g / dot(q, q);
  const T xz = dot(x, z), yz = dot(y, z), xy = dot(x, y);
  return scale(sub(sub(scale(y, T(2.0) * xz), scale(x, yz)), scale(z, xy)), c);
}

}  // namespace hel

// Formulation C.  p[0], p[1]: incoming gluons; p[2]: top; p[3]: anti-top;
// p[4]: outgoing gluon.  cm: the 6 x 6 colour matrix of the orderings
// `ords` (formulation A's, from explicit SU(3) traces).
template <class T>
T me2_gg_ttbarg_helicity_t(const T& alpha_s, const T& mt, const P4T<T>* p, const std::vector<double>& cm,
                           const std::vector<std::array<int, 3>>& ords) {
  using namespace hel;
  using std::sqrt;
  const T g = sqrt(T(4.0 * M_PI) * alpha_s);
  const P4T<T> q[3] = {p[0], p[1], scale(p[4], T(-1.0))};
  P4T<T> pol[3][2];
  for (int i = 0; i < 3; ++i) linear_pols(i < 2 ? p[i] : p[4], &pol[i][0], &pol[i][1]);
  // propagator momenta and reciprocal denominators: S_a = S(p_t - q_a) and
  // S(q_c - p_tbar) (= S_ab for the pair ab without c)
  P4T<T> ka[3], kc[3];
  T ia[3], ic[3];
  const T m2 = mt * mt;
  for (int a = 0; a < 3; ++a) {
    ka[a] = sub(p[2], q[a]);
    ia[a] = T(1.0) / (dot(ka[a], ka[a]) - m2);
    kc[a] = sub(q[a], p[3]);
    ic[a] = T(1.0) / (dot(kc[a], kc[a]) - m2);
  }
  const Spinor<T> ubar[2] = {adjoint(u_spinor(p[2], mt, 0)), adjoint(u_spinor(p[2], mt, 1))};
  const Spinor<T> v = v_spinor(p[3], mt, 0);
  const T g2 = g * g, g3 = g2 * g;
  const int no = int(ords.size());
  T total = T(0.0);
  for (int h = 0; h < 8; ++h) {
    P4T<T> e[3];
    for (int i = 0; i < 3; ++i) e[i] = pol[i][(h >> i) & 1];
    // pair currents J(ab) for a < b (J(ba) = -J(ab)) and the column spinors X_c
    P4T<T> jp[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b) {
        jp[a][b] = current2(g, e[a], q[a], e[b], q[b]);
        jp[b][a] = scale(jp[a][b], T(-1.0));
      }
    Spinor<T> X[3];
    for (int c = 0; c < 3; ++c) X[c] = prop(kc[c], mt, ic[c], slash(e[c], v));
    std::vector<Cx<T>> amp(2 * no);
    for (int o = 0; o < no; ++o) {
      const int a = ords[o][0], b = ords[o][1], c = ords[o][2];
      const P4T<T> qab = add(q[a], q[b]), qbc = add(q[b], q[c]), qabc = add(qab, q[c]);
      const P4T<T> jabc = add(add(current2(g, jp[a][b], qab, e[c], q[c]), current2(g, e[a], q[a], jp[b][c], qbc)),
                              current4(g, e[a], e[b], e[c], qabc));
      // eps_a S_a (i g^3 eps_b X_c - i g^2 J(bc) v) - i g^2 J(ab) X_c + i g J(abc) v
      const Spinor<T> inner = ssub(sscale_i(g3, slash(e[b], X[c])), sscale_i(g2, slash(jp[b][c], v)));
      const Spinor<T> col = sadd(ssub(slash(e[a], prop(ka[a], mt, ia[a], inner)), sscale_i(g2, slash(jp[a][b], X[c]))),
                                 sscale_i(g, slash(jabc, v)));
      for (int st = 0; st < 2; ++st) amp[st * no + o] = row_dot(ubar[st], col);
    }
    for (int st = 0; st < 2; ++st)
      for (int s = 0; s < no; ++s)
        for (int sp = 0; sp < no; ++sp) {
          const Cx<T> pr = amp[st * no + s] * conj(amp[st * no + sp]);
          total += T(cm[s * no + sp]) * pr.re;
        }
  }
  // the other antitop spin gives the same sum; average over 2 x 2 gluon
  // polarisations and 8 x 8 colours
  return T(2.0) * total / T(256.0);
}

}  // namespace orc
