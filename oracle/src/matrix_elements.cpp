// Oracle: tree-level squared matrix elements.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "The MadFlow event generator" (master formula
// eq. mc_master_formula; helicity amplitudes and colour decomposition; the
// pp -> tt diagrams of fig. pp_ttx).  The thesis prints no amplitude, so:
//  * e+e- -> mu+mu- (gamma + Z), qq -> tt and gg -> tt use the textbook
//    spin- and colour-averaged closed forms (their plain definition), and each
//    is cross-checked by an explicit numerical Dirac trace of the Feynman
//    amplitude built from 4x4 gamma matrices;
//  * gg -> ttg has no closed form: formulation A evaluates the six
//    colour-ordered partial amplitudes as Dirac matrices (colour-ordered
//    Feynman rules derived from the standard QCD rules) and contracts them
//    with the colour matrix obtained from explicit SU(3) generator traces;
//    formulation B sums all 16 Feynman diagrams at every explicit colour
//    assignment.
// Pins (tests/test_oracle_me.py): closed form vs numerical trace; partonic
// total cross sections; A vs B; gauge invariance; Bose symmetry; the soft
// gluon limit of the colour-ordered amplitudes; gg -> tt colour-ordered vs
// closed form.
#include <algorithm>
#include <cmath>

#include "dirac.h"
#include "helicity_t.h"

namespace orc {

static const cplx I(0.0, 1.0);

// ------------------------------------------------------------ e+e- -> mu+mu-
// Massless leptons, photon + Z exchange with a fixed-width Breit-Wigner:
// <|M|^2> = e^4 [A0 (1 + c^2) + A1 c], c = cos(theta(e-, mu-)),
// chi = s / (s - MZ^2 + i MZ GZ) / (4 sW^2 cW^2), v = -1/2 + 2 sW^2, a = -1/2,
// A0 = 1 + 2 v^2 Re chi + (v^2 + a^2)^2 |chi|^2,  A1 = 4 a^2 Re chi + 8 v^2 a^2 |chi|^2.
double me2_eemumu(const EWParams& ew, double s, double c) {
  const double cw2 = 1.0 - ew.sw2;
  const cplx chi = cplx(s, 0.0) / cplx(s - ew.mz * ew.mz, ew.mz * ew.gz) / (4.0 * ew.sw2 * cw2);
  const double v = -0.5 + 2.0 * ew.sw2, a = -0.5;
  const double re = chi.real(), ab2 = std::norm(chi);
  const double a0 = 1.0 + 2.0 * v * v * re + (v * v + a * a) * (v * v + a * a) * ab2;
  const double a1 = 4.0 * a * a * re + 8.0 * v * v * a * a * ab2;
  const double e2 = 4.0 * M_PI * ew.alpha;
  return e2 * e2 * (a0 * (1.0 + c * c) + a1 * c);
}

// Numerical trace of the same amplitude: lepton currents with the vertex
// -i e Q gamma^mu (photon) and -i e/(sW cW) gamma^mu (gL PL + gR PR) (Z),
// photon propagator -i g/s, Z propagator -i g/(s - MZ^2 + i MZ GZ) (the
// k^mu k^nu term vanishes for massless leptons).  p[0] = e-, p[1] = e+,
// p[2] = mu-, p[3] = mu+.
double me2_eemumu_trace(const EWParams& ew, const P4* p) {
  const auto& g = gammas();
  Mat4 g5 = mmul(mmul(g[0], g[1]), mmul(g[2], g[3]));
  g5 = mscale(g5, I);
  const Mat4 pl = mscale(madd(meye(), mscale(g5, -1.0)), 0.5);
  const Mat4 pr = mscale(madd(meye(), g5), 0.5);
  const double e = std::sqrt(4.0 * M_PI * ew.alpha);
  const double sw = std::sqrt(ew.sw2), cw = std::sqrt(1.0 - ew.sw2);
  const double q = -1.0, t3 = -0.5;
  const double gl = t3 - q * ew.sw2, gr = -q * ew.sw2;
  const double s = dot(add(p[0], p[1]), add(p[0], p[1]));
  const cplx prop_a = -I / s;
  const cplx prop_z = -I / cplx(s - ew.mz * ew.mz, ew.mz * ew.gz);
  // Vertex matrices Gamma_mu for photon and Z.
  std::array<Mat4, 4> va, vz;
  for (int mu = 0; mu < 4; ++mu) {
    va[mu] = mscale(g[mu], -I * e * q);
    vz[mu] = mscale(mmul(g[mu], madd(mscale(pl, gl), mscale(pr, gr))), -I * e / (sw * cw));
  }
  const double metric[4] = {1.0, -1.0, -1.0, -1.0};
  // sum over spins of |vbar(e+) V^mu u(e-) P_mu,nu ubar(mu-) V^nu v(mu+)|^2
  //  = sum_{mu,nu,rho,sigma} L^{mu rho} M^{nu sigma} (props...)
  // with L^{mu rho} = Tr[p1slash V^mu p0slash bar(V^rho)] etc.
  const Mat4 s0 = slash(p[0]), s1 = slash(p[1]), s2 = slash(p[2]), s3 = slash(p[3]);
  double total = 0.0;
  // Amplitude = sum_X prop_X J_e^X . J_mu^X; square summed over spins.
  for (int xa = 0; xa < 2; ++xa)
    for (int xb = 0; xb < 2; ++xb) {
      const auto& v1 = xa == 0 ? va : vz;
      const auto& v2 = xb == 0 ? va : vz;
      const cplx pa = xa == 0 ? prop_a : prop_z;
      const cplx pb = xb == 0 ? prop_a : prop_z;
      cplx acc = 0.0;
      for (int mu = 0; mu < 4; ++mu)
        for (int rho = 0; rho < 4; ++rho) {
          const cplx lt = mtrace(mmul(mmul(s1, v1[mu]), mmul(s0, dirac_bar(v2[rho]))));
          const cplx mt = mtrace(mmul(mmul(s2, v1[mu]), mmul(s3, dirac_bar(v2[rho]))));
          acc += lt * mt * metric[mu] * metric[rho];
        }
      total += (pa * std::conj(pb) * acc).real();
    }
  return total / 4.0;
}

// ------------------------------------------------------------ q qbar -> t tbar
// Spin/colour averaged (Combridge 1979; Ellis-Stirling-Webber):
// g^4 (4/9) (tau1^2 + tau2^2 + rho/2), tau1 = (m^2 - t)/s, tau2 = 1 - tau1,
// rho = 4 m^2 / s.
double me2_qqbar_ttbar(double alpha_s, double mt, double s, double t) {
  const double g2 = 4.0 * M_PI * alpha_s;
  const double tau1 = (mt * mt - t) / s, tau2 = 1.0 - tau1, rho = 4.0 * mt * mt / s;
  return g2 * g2 * (4.0 / 9.0) * (tau1 * tau1 + tau2 * tau2 + rho / 2.0);
}

// g g -> t tbar: g^4 (1/(6 tau1 tau2) - 3/8) (tau1^2 + tau2^2 + rho - rho^2/(4 tau1 tau2)).
double me2_gg_ttbar(double alpha_s, double mt, double s, double t) {
  const double g2 = 4.0 * M_PI * alpha_s;
  const double tau1 = (mt * mt - t) / s, tau2 = 1.0 - tau1, rho = 4.0 * mt * mt / s;
  return g2 * g2 * (1.0 / (6.0 * tau1 * tau2) - 3.0 / 8.0) *
         (tau1 * tau1 + tau2 * tau2 + rho - rho * rho / (4.0 * tau1 * tau2));
}

// Numerical Dirac trace of q(p0) qbar(p1) -> t(p2) tbar(p3) via one s-channel
// gluon: vertex i g gamma^mu t^a, propagator -i g_{mu nu} delta^{ab} / s.
// Colour sum sum_{ab} tr(t^a t^b)^2 = 2; average 1/4 (spin) x 1/9 (colour).
double me2_qqbar_ttbar_trace(double alpha_s, double mt, const P4* p) {
  const auto& g = gammas();
  const double g2 = 4.0 * M_PI * alpha_s;
  const double s = dot(add(p[0], p[1]), add(p[0], p[1]));
  const double metric[4] = {1.0, -1.0, -1.0, -1.0};
  const Mat4 sq = slash(p[0]), sqb = slash(p[1]);
  const Mat4 st = madd(slash(p[2]), mscale(meye(), mt));
  const Mat4 stb = madd(slash(p[3]), mscale(meye(), -mt));
  cplx acc = 0.0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      const cplx lt = mtrace(mmul(mmul(sqb, g[mu]), mmul(sq, g[nu])));
      const cplx ht = mtrace(mmul(mmul(st, g[mu]), mmul(stb, g[nu])));
      acc += lt * ht * metric[mu] * metric[nu];
    }
  return (g2 * g2 / (s * s) * acc.real()) * 2.0 / 36.0;
}

// ------------------------------------------------------------ colour algebra
// SU(3) generators t^a = lambda^a / 2 (Gell-Mann matrices), tr(t^a t^b) = delta/2.
using Mat3 = std::array<cplx, 9>;
static const std::array<Mat3, 8>& generators() {
  static const std::array<Mat3, 8> t = [] {
    std::array<Mat3, 8> l;
    for (auto& m : l) m.fill(0.0);
    l[0][1] = l[0][3] = 1.0;
    l[1][1] = -I; l[1][3] = I;
    l[2][0] = 1.0; l[2][4] = -1.0;
    l[3][2] = l[3][6] = 1.0;
    l[4][2] = -I; l[4][6] = I;
    l[5][5] = l[5][7] = 1.0;
    l[6][5] = -I; l[6][7] = I;
    l[7][0] = l[7][4] = 1.0 / std::sqrt(3.0);
    l[7][8] = -2.0 / std::sqrt(3.0);
    for (auto& m : l)
      for (auto& x : m) x *= 0.5;
    return l;
  }();
  return t;
}
static Mat3 m3mul(const Mat3& a, const Mat3& b) {
  Mat3 c;
  c.fill(0.0);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) c[i * 3 + j] += a[i * 3 + k] * b[k * 3 + j];
  return c;
}
// f^{abc} = -2 i tr([t^a, t^b] t^c).
static const std::vector<double>& structure_constants() {
  static const std::vector<double> f = [] {
    const auto& t = generators();
    std::vector<double> r(512);
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int c = 0; c < 8; ++c) {
          const Mat3 ab = m3mul(t[a], t[b]), ba = m3mul(t[b], t[a]);
          Mat3 comm;
          for (int i = 0; i < 9; ++i) comm[i] = ab[i] - ba[i];
          const Mat3 x = m3mul(comm, t[c]);
          r[(a * 8 + b) * 8 + c] = (-2.0 * I * (x[0] + x[4] + x[8])).real();
        }
    return r;
  }();
  return f;
}
static double fabc(int a, int b, int c) { return structure_constants()[(a * 8 + b) * 8 + c]; }

// Colour matrix of ordered generator strings: C[s][s'] = sum over gluon
// colours of tr(t^{s1}..t^{sn} (t^{s'1}..t^{s'n})^dagger), for n = 2 or 3 and
// the orderings listed in `perms`.
static std::vector<double> colour_matrix(int n, const std::vector<std::array<int, 3>>& perms) {
  const auto& t = generators();
  const int np = int(perms.size());
  std::vector<double> c(np * np, 0.0);
  int total = 1;
  for (int i = 0; i < n; ++i) total *= 8;
  for (int cfg = 0; cfg < total; ++cfg) {
    int col[3] = {cfg % 8, (cfg / 8) % 8, (cfg / 64) % 8};
    std::vector<Mat3> str(np);
    for (int s = 0; s < np; ++s) {
      Mat3 m = t[col[perms[s][0]]];
      for (int k = 1; k < n; ++k) m = m3mul(m, t[col[perms[s][k]]]);
      str[s] = m;
    }
    for (int s = 0; s < np; ++s)
      for (int sp = 0; sp < np; ++sp) {
        cplx tr = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) tr += str[s][i * 3 + j] * std::conj(str[sp][i * 3 + j]);
        c[s * np + sp] += tr.real();
      }
  }
  return c;
}

// ------------------------------------------------------------ gluon currents
// Standard QCD rules (vertex i g gamma^mu t^a, quark propagator
// i (pslash + m)/(p^2 - m^2), gluon propagator -i g_{mu nu}/k^2, three-gluon
// vertex g f^{abc}[g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu]
// with all momenta incoming, and the four-gluon vertex).  Stripping f^{xye}
// and using f^{xye} t^e = -i [t^x, t^y] gives the colour-ordered current of
// an adjacent pair W(X, Y) = -V(X, Y) / Q^2 with
// V(X, Y) = g [(X.Y)(qX - qY) + Y (X.(qX + 2 qY)) - X (Y.(2 qX + qY))].
static CVec4 vertex3(double g, const CVec4& x, const P4& qx, const CVec4& y, const P4& qy) {
  const CVec4 cqx = cv(qx), cqy = cv(qy);
  const cplx xy = cdot(x, y);
  const cplx x_q = cdot(x, cadd(cqx, cscale(cqy, 2.0)));
  const cplx y_q = cdot(y, cadd(cscale(cqx, 2.0), cqy));
  CVec4 r;
  for (int mu = 0; mu < 4; ++mu) r[mu] = g * (xy * (cqx[mu] - cqy[mu]) + y[mu] * x_q - x[mu] * y_q);
  return r;
}
static CVec4 current2(double g, const CVec4& x, const P4& qx, const CVec4& y, const P4& qy) {
  const P4 q = add(qx, qy);
  return cscale(vertex3(g, x, qx, y, qy), -1.0 / dot(q, q));
}
// Colour-ordered four-gluon contact term of the string t^x t^y t^z:
// g^2 / Q^2 [2 (X.Z) Y - (Y.Z) X - (X.Y) Z].
static CVec4 current4(double g, const CVec4& x, const CVec4& y, const CVec4& z, const P4& q) {
  const double q2 = dot(q, q);
  CVec4 r;
  const cplx xz = cdot(x, z), yz = cdot(y, z), xy = cdot(x, y);
  for (int mu = 0; mu < 4; ++mu) r[mu] = g * g / q2 * (2.0 * xz * y[mu] - yz * x[mu] - xy * z[mu]);
  return r;
}

static Mat4 quark_prop(const P4& p, double m) {
  return mscale(madd(slash(p), mscale(meye(), m)), 1.0 / (dot(p, p) - m * m));
}

// Dirac matrix (between ubar(top) and v(antitop)) of the colour-ordered
// partial amplitude for the gluon ordering `ord` (gluons with incoming
// momenta q[i] and polarisations eps[i]).
static Mat4 partial_dirac(double g, double mt, const P4& ptop, const P4* q, const CVec4* eps,
                          const int* ord, int n) {
  if (n == 2) {
    const int a = ord[0], b = ord[1];
    const Mat4 line = mmul(mmul(slash(eps[a]), quark_prop(sub(ptop, q[a]), mt)), slash(eps[b]));
    const CVec4 jab = current2(g, eps[a], q[a], eps[b], q[b]);
    // (i g)^2 i = -i g^2 ; (i g) for the single vertex with the current.
    return madd(mscale(line, -I * g * g), mscale(slash(jab), I * g));
  }
  const int a = ord[0], b = ord[1], c = ord[2];
  const P4 qab = add(q[a], q[b]), qbc = add(q[b], q[c]), qabc = add(qab, q[c]);
  const Mat4 sa = quark_prop(sub(ptop, q[a]), mt);
  const Mat4 sab = quark_prop(sub(ptop, qab), mt);
  const CVec4 jab = current2(g, eps[a], q[a], eps[b], q[b]);
  const CVec4 jbc = current2(g, eps[b], q[b], eps[c], q[c]);
  CVec4 jabc = cadd(current2(g, jab, qab, eps[c], q[c]), current2(g, eps[a], q[a], jbc, qbc));
  jabc = cadd(jabc, current4(g, eps[a], eps[b], eps[c], qabc));
  // three single emissions: (i g)^3 i^2 = i g^3
  const Mat4 t1 = mscale(mmul(mmul(mmul(mmul(slash(eps[a]), sa), slash(eps[b])), sab), slash(eps[c])),
                         I * g * g * g);
  // one pair current and one emission: (i g)^2 i = -i g^2
  const Mat4 t2 = mscale(mmul(mmul(slash(jab), sab), slash(eps[c])), -I * g * g);
  const Mat4 t3 = mscale(mmul(mmul(slash(eps[a]), sa), slash(jbc)), -I * g * g);
  // triple current: i g
  const Mat4 t4 = mscale(slash(jabc), I * g);
  return madd(madd(t1, t2), madd(t3, t4));
}

// Two real transverse polarisation vectors of a massless momentum k.
static void linear_pols(const P4& k, CVec4* e1, CVec4* e2) {
  const double kabs = std::sqrt(k.x * k.x + k.y * k.y + k.z * k.z);
  const double n[3] = {k.x / kabs, k.y / kabs, k.z / kabs};
  double a[3];
  const double perp = std::sqrt(n[0] * n[0] + n[1] * n[1]);
  if (perp > 1e-6) {  // a = n x z / |n x z|
    a[0] = n[1] / perp; a[1] = -n[0] / perp; a[2] = 0.0;
  } else {
    a[0] = 1.0; a[1] = 0.0; a[2] = 0.0;
  }
  const double b[3] = {n[1] * a[2] - n[2] * a[1], n[2] * a[0] - n[0] * a[2], n[0] * a[1] - n[1] * a[0]};
  *e1 = {0.0, a[0], a[1], a[2]};
  *e2 = {0.0, b[0], b[1], b[2]};
}

static std::vector<std::array<int, 3>> orderings(int n) {
  std::vector<std::array<int, 3>> r;
  std::array<int, 3> p = {0, 1, 2};
  do {
    r.push_back(p);
  } while (std::next_permutation(p.begin(), p.begin() + n));
  return r;
}

// Formulation A for n gluons (n = 2: gg -> tt, n = 3: gg -> ttg).
// p[0], p[1] incoming gluons; p[2] top; p[3] anti-top; p[4] outgoing gluon.
static double me2_colour_ordered(double alpha_s, double mt, const P4* p, int n) {
  const double g = std::sqrt(4.0 * M_PI * alpha_s);
  P4 q[3];
  q[0] = p[0];
  q[1] = p[1];
  if (n == 3) q[2] = scale(p[4], -1.0);
  CVec4 pol[3][2];
  for (int i = 0; i < n; ++i) linear_pols(i < 2 ? p[i] : p[4], &pol[i][0], &pol[i][1]);
  const auto perms = orderings(n);
  const int np = int(perms.size());
  static const std::vector<double> c2 = colour_matrix(2, orderings(2));
  static const std::vector<double> c3 = colour_matrix(3, orderings(3));
  const std::vector<double>& cm = n == 2 ? c2 : c3;
  const Mat4 ptop = madd(slash(p[2]), mscale(meye(), mt));
  const Mat4 pbar = madd(slash(p[3]), mscale(meye(), -mt));
  double total = 0.0;
  const int npol = 1 << n;
  for (int h = 0; h < npol; ++h) {
    CVec4 eps[3];
    for (int i = 0; i < n; ++i) eps[i] = pol[i][(h >> i) & 1];
    std::vector<Mat4> left(np), right(np);
    for (int s = 0; s < np; ++s) {
      const Mat4 gam = partial_dirac(g, mt, p[2], q, eps, perms[s].data(), n);
      left[s] = mmul(ptop, gam);
      right[s] = mmul(pbar, dirac_bar(gam));
    }
    for (int s = 0; s < np; ++s)
      for (int sp = 0; sp < np; ++sp) {
        // Tr[(ptop + m) Gamma_s (pbar - m) bar(Gamma_s')]
        cplx tr = 0.0;
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) tr += left[s][i * 4 + j] * right[sp][j * 4 + i];
        total += cm[s * np + sp] * tr.real();
      }
  }
  return total / 256.0;  // average over 2x2 gluon polarisations and 8x8 colours
}

double me2_gg_ttbar_colour_ordered(double alpha_s, double mt, const P4* p) {
  return me2_colour_ordered(alpha_s, mt, p, 2);
}
double me2_gg_ttbarg(double alpha_s, double mt, const P4* p) {
  return me2_colour_ordered(alpha_s, mt, p, 3);
}

const std::vector<std::array<int, 3>>& ggg_orderings() {
  static const std::vector<std::array<int, 3>> o = orderings(3);
  return o;
}
const std::vector<double>& ggg_colour_matrix() {
  static const std::vector<double> c = colour_matrix(3, ggg_orderings());
  return c;
}
// Formulation C: helicity amplitudes on spinors (helicity_t.h) at T = double.
double me2_gg_ttbarg_helicity(double alpha_s, double mt, const P4* p) {
  return me2_gg_ttbarg_helicity_t<double>(alpha_s, mt, p, ggg_colour_matrix(), ggg_orderings());
}

// Formulation B: the 16 Feynman diagrams of g g -> t tbar g at every explicit
// colour assignment (a1, a2, a3, i, j), spins summed by Dirac traces.
double me2_gg_ttbarg_brute(double alpha_s, double mt, const P4* p) {
  const double g = std::sqrt(4.0 * M_PI * alpha_s);
  const auto& t = generators();
  P4 q[3] = {p[0], p[1], scale(p[4], -1.0)};
  CVec4 pol[3][2];
  for (int i = 0; i < 3; ++i) linear_pols(i < 2 ? p[i] : p[4], &pol[i][0], &pol[i][1]);
  const Mat4 ptop = madd(slash(p[2]), mscale(meye(), mt));
  const Mat4 pbar = madd(slash(p[3]), mscale(meye(), -mt));
  const auto perms = orderings(3);
  const int pairs[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};  // (x, y | z)
  double total = 0.0;
  for (int h = 0; h < 8; ++h) {
    CVec4 eps[3];
    for (int i = 0; i < 3; ++i) eps[i] = pol[i][(h >> i) & 1];
    // Dirac structures.
    Mat4 d1[6];  // three emissions in order perms[k]
    for (int k = 0; k < 6; ++k) {
      const int a = perms[k][0], b = perms[k][1], c = perms[k][2];
      const Mat4 m = mmul(mmul(mmul(mmul(slash(eps[a]), quark_prop(sub(p[2], q[a]), mt)),
                                    slash(eps[b])),
                               quark_prop(sub(sub(p[2], q[a]), q[b]), mt)),
                          slash(eps[c]));
      d1[k] = mscale(m, I * g * g * g);
    }
    Mat4 d2a[3], d2b[3], d3[3];
    CVec4 exy[3];
    for (int k = 0; k < 3; ++k) {
      const int x = pairs[k][0], y = pairs[k][1], z = pairs[k][2];
      const P4 qxy = add(q[x], q[y]);
      // internal gluon: E = -i V / Q^2 (f^{xye} stripped)
      exy[k] = cscale(vertex3(g, eps[x], q[x], eps[y], q[y]), -I / dot(qxy, qxy));
      // current next to the top, emission z next to the anti-top
      d2a[k] = mscale(mmul(mmul(slash(exy[k]), quark_prop(sub(p[2], qxy), mt)), slash(eps[z])),
                      -I * g * g);
      // emission z next to the top, current next to the anti-top
      d2b[k] = mscale(mmul(mmul(slash(eps[z]), quark_prop(sub(p[2], q[z]), mt)), slash(exy[k])),
                      -I * g * g);
      const P4 qall = add(qxy, q[z]);
      const CVec4 e3 = cscale(vertex3(g, exy[k], qxy, eps[z], q[z]), -I / dot(qall, qall));
      d3[k] = mscale(slash(e3), I * g);
    }
    // four-gluon vertex pieces (legs x=0, y=1, z=2, internal w): the three
    // Lorentz structures, each multiplied later by its colour factor.
    const P4 qall = add(add(q[0], q[1]), q[2]);
    const double q2 = dot(qall, qall);
    const cplx pref = (-I) * (-I * g * g) / q2;  // vertex -i g^2 [...], propagator -i/Q^2
    const cplx e01 = cdot(eps[0], eps[1]), e02 = cdot(eps[0], eps[2]), e12 = cdot(eps[1], eps[2]);
    CVec4 s4[3];
    for (int mu = 0; mu < 4; ++mu) {
      s4[0][mu] = pref * (e02 * eps[1][mu] - e12 * eps[0][mu]);  // f^{xye} f^{zwe}
      s4[1][mu] = pref * (e01 * eps[2][mu] - e12 * eps[0][mu]);  // f^{xze} f^{ywe}
      s4[2][mu] = pref * (e01 * eps[2][mu] - e02 * eps[1][mu]);  // f^{xwe} f^{yze}
    }
    Mat4 d4[3];
    for (int k = 0; k < 3; ++k) d4[k] = mscale(slash(s4[k]), I * g);

    for (int a0 = 0; a0 < 8; ++a0)
      for (int a1 = 0; a1 < 8; ++a1)
        for (int a2 = 0; a2 < 8; ++a2) {
          const int col[3] = {a0, a1, a2};
          for (int ci = 0; ci < 3; ++ci)
            for (int cj = 0; cj < 3; ++cj) {
              Mat4 amp = mzero();
              auto tt = [&](int a, int b, int c) {  // (t^a t^b t^c)_{ij}
                const Mat3 m = m3mul(m3mul(t[a], t[b]), t[c]);
                return m[ci * 3 + cj];
              };
              for (int k = 0; k < 6; ++k) {
                const cplx cf = tt(col[perms[k][0]], col[perms[k][1]], col[perms[k][2]]);
                if (cf != 0.0) amp = madd(amp, mscale(d1[k], cf));
              }
              for (int k = 0; k < 3; ++k) {
                const int x = pairs[k][0], y = pairs[k][1], z = pairs[k][2];
                cplx ca = 0.0, cb = 0.0, c3 = 0.0;
                for (int e = 0; e < 8; ++e) {
                  const double f = fabc(col[x], col[y], e);
                  if (f == 0.0) continue;
                  const Mat3 ez = m3mul(t[e], t[col[z]]), ze = m3mul(t[col[z]], t[e]);
                  ca += f * ez[ci * 3 + cj];
                  cb += f * ze[ci * 3 + cj];
                  for (int w = 0; w < 8; ++w) c3 += f * fabc(e, col[z], w) * t[w][ci * 3 + cj];
                }
                amp = madd(amp, mscale(d2a[k], ca));
                amp = madd(amp, mscale(d2b[k], cb));
                amp = madd(amp, mscale(d3[k], c3));
              }
              cplx c4[3] = {0.0, 0.0, 0.0};
              for (int w = 0; w < 8; ++w)
                for (int e = 0; e < 8; ++e) {
                  const cplx tw = t[w][ci * 3 + cj];
                  if (tw == 0.0) continue;
                  c4[0] += fabc(col[0], col[1], e) * fabc(col[2], w, e) * tw;
                  c4[1] += fabc(col[0], col[2], e) * fabc(col[1], w, e) * tw;
                  c4[2] += fabc(col[0], w, e) * fabc(col[1], col[2], e) * tw;
                }
              for (int k = 0; k < 3; ++k) amp = madd(amp, mscale(d4[k], c4[k]));
              total += mtrace(mmul(mmul(ptop, amp), mmul(pbar, dirac_bar(amp)))).real();
            }
        }
  }
  return total / 256.0;
}

// Colour-ordered partial amplitudes ubar Gamma_sigma v for given external
// wave functions (used by the gauge-invariance and soft-limit pins).
void ggttg_partial_amplitudes(double alpha_s, double mt, const P4* q_in, const cplx (*eps_in)[4],
                              int ngluon, const cplx* ubar, const cplx* v, cplx* amps) {
  const double g = std::sqrt(4.0 * M_PI * alpha_s);
  P4 ptop = q_in[ngluon];
  P4 q[3];
  CVec4 eps[3];
  for (int i = 0; i < ngluon; ++i) {
    q[i] = q_in[i];
    eps[i] = {eps_in[i][0], eps_in[i][1], eps_in[i][2], eps_in[i][3]};
  }
  const auto perms = orderings(ngluon);
  for (size_t s = 0; s < perms.size(); ++s) {
    const Mat4 gam = partial_dirac(g, mt, ptop, q, eps, perms[s].data(), ngluon);
    cplx a = 0.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a += ubar[i] * gam[i * 4 + j] * v[j];
    amps[s] = a;
  }
}

// ------------------------------------------------------------ q qbar -> t tbar g
// The five Feynman diagrams of q(p0) qbar(p1) -> t(p2) tbar(p3) g(p4), with
// the rules above: gluon emission off the quark, the antiquark, the top, the
// anti-top, and off the s-channel gluon (three-gluon vertex).  Each diagram
// d is written as sum_alpha [vbar(p1) Lambda_d^alpha u(p0)] [ubar(p2)
// Theta_{d,alpha} v(p3)] times a colour factor c_d(i, j, k, l, a) (quark,
// antiquark, top, anti-top, gluon colours), so that the spin sum is
//   sum_{d,d'} C_{dd'} sum_{alpha,alpha'} tr[Lambda_d p0slash Lambdabar_d' p1slash]
//                                          tr[Theta_d (p3slash - m) Thetabar_d' (p2slash + m)]
// with the colour matrix C_{dd'} = sum over colours of c_d c_d'^* (complex)
// and the real part of the double sum taken at the end.  The
// gluon polarisation is summed over the two real transverse vectors, or
// replaced by `eps_override` (the gauge-invariance pin sets it to p4).
// Average: 1/4 (spins) x 1/9 (colours).
static double me2_qqbar_ttbarg_impl(double alpha_s, double mt, const P4* p, const CVec4* eps_override) {
  const double g = std::sqrt(4.0 * M_PI * alpha_s);
  const auto& gm = gammas();
  const double metric[4] = {1.0, -1.0, -1.0, -1.0};
  // colour matrix of the five diagrams (complex: the three-gluon diagram's
  // colour factor is i times a combination of the others')
  static const std::vector<cplx> cmat = [] {
    const auto& tt = generators();
    std::vector<cplx> c(25, 0.0);
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
              cplx cf[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
              for (int b = 0; b < 8; ++b) {
                const Mat3 ba = m3mul(tt[b], tt[a]), ab = m3mul(tt[a], tt[b]);
                cf[0] += ba[j * 3 + i] * tt[b][k * 3 + l];
                cf[1] += ab[j * 3 + i] * tt[b][k * 3 + l];
                cf[2] += tt[b][j * 3 + i] * ab[k * 3 + l];
                cf[3] += tt[b][j * 3 + i] * ba[k * 3 + l];
                for (int c3 = 0; c3 < 8; ++c3) cf[4] += tt[b][j * 3 + i] * tt[c3][k * 3 + l] * fabc(b, c3, a);
              }
              for (int d = 0; d < 5; ++d)
                for (int e = 0; e < 5; ++e) c[d * 5 + e] += cf[d] * std::conj(cf[e]);
            }
    return c;
  }();
  const P4 pp = add(p[0], p[1]), qq = add(p[2], p[3]);
  const double P2 = dot(pp, pp), Q2 = dot(qq, qq);
  const Mat4 s0 = slash(p[0]), s1 = slash(p[1]);
  const Mat4 h2 = madd(slash(p[2]), mscale(meye(), mt)), h3 = madd(slash(p[3]), mscale(meye(), -mt));
  CVec4 pol[2];
  linear_pols(p[4], &pol[0], &pol[1]);
  const int npol = eps_override ? 1 : 2;
  double total = 0.0;
  for (int h = 0; h < npol; ++h) {
    const CVec4 eps = eps_override ? *eps_override : pol[h];
    const Mat4 se = slash(eps);
    const Mat4 sq1 = quark_prop(sub(p[0], p[4]), 0.0), sq2 = quark_prop(sub(p[4], p[1]), 0.0);
    const Mat4 st3 = quark_prop(add(p[2], p[4]), mt), st4 = quark_prop(scale(add(p[3], p[4]), -1.0), mt);
    // lower-index eps and the momenta of the three-gluon vertex (incoming P, -Q, -p4)
    const CVec4 ce = eps;
    const CVec4 kp = cv(add(pp, qq));                      // k - p = P + Q
    const CVec4 pq = cv(sub(p[4], qq));                    // p - q = -Q + p4
    const CVec4 qk = cv(scale(add(p[4], pp), -1.0));      // q - k = -p4 - P
    const cplx kpe = cdot(kp, ce);
    Mat4 L[5][4], H[5][4];
    for (int al = 0; al < 4; ++al) {
      const Mat4& ga = gm[al];
      L[0][al] = mscale(mmul(mmul(ga, sq1), se), -I * g * g * g / Q2);
      L[1][al] = mscale(mmul(mmul(se, sq2), ga), -I * g * g * g / Q2);
      L[2][al] = mscale(ga, -I * g * g * g / P2);
      L[3][al] = mscale(ga, -I * g * g * g / P2);
      L[4][al] = mscale(ga, g * g * g / (P2 * Q2));
      H[0][al] = mscale(ga, metric[al]);
      H[1][al] = mscale(ga, metric[al]);
      H[2][al] = mscale(mmul(mmul(se, st3), ga), metric[al]);
      H[3][al] = mscale(mmul(mmul(ga, st4), se), metric[al]);
      // Theta_{5,alpha} = sum_beta T_{alpha beta} gamma^beta,
      // T_{ab} = g_ab (k-p).eps + eps_b (p-q)_a + eps_a (q-k)_b (lower indices)
      Mat4 th = mzero();
      for (int be = 0; be < 4; ++be) {
        cplx tab = (al == be ? metric[al] : 0.0) * kpe + metric[be] * ce[be] * metric[al] * pq[al] +
                   metric[al] * ce[al] * metric[be] * qk[be];
        if (tab != 0.0) th = madd(th, mscale(gm[be], tab));
      }
      H[4][al] = th;
    }
    for (int d = 0; d < 5; ++d)
      for (int e = 0; e < 5; ++e) {
        const cplx c = cmat[d * 5 + e];
        if (c == 0.0) continue;
        cplx acc = 0.0;
        for (int al = 0; al < 4; ++al)
          for (int ap = 0; ap < 4; ++ap) {
            const cplx tl = mtrace(mmul(mmul(L[d][al], s0), mmul(dirac_bar(L[e][ap]), s1)));
            if (tl == 0.0) continue;
            const cplx th = mtrace(mmul(mmul(H[d][al], h3), mmul(dirac_bar(H[e][ap]), h2)));
            acc += tl * th;
          }
        total += (c * acc).real();
      }
  }
  return total / 36.0;
}

double me2_qqbar_ttbarg(double alpha_s, double mt, const P4* p) { return me2_qqbar_ttbarg_impl(alpha_s, mt, p, nullptr); }

// q(p0) g(p1) -> t(p2) tbar(p3) q(p4) by crossing: the antiquark of
// q qbar -> t tbar g becomes the outgoing quark and the outgoing gluon the
// incoming one, |M|^2(qg) = -|M|^2(q qbar)(p0, -p4; p2, p3, -p1) summed over
// spins and colours (one fermion crossed), averaged 1/(4 x 3 x 8) instead of
// 1/(4 x 9).
double me2_qg_ttbarq(double alpha_s, double mt, const P4* p) {
  const P4 q[5] = {p[0], scale(p[4], -1.0), p[2], p[3], scale(p[1], -1.0)};
  return -me2_qqbar_ttbarg(alpha_s, mt, q) * 36.0 / 96.0;
}

}  // namespace orc

extern "C" {

static void pack(const double* in, int n, orc::P4* p) {
  for (int i = 0; i < n; ++i) p[i] = {in[4 * i], in[4 * i + 1], in[4 * i + 2], in[4 * i + 3]};
}

double orc_me2_eemumu(double alpha, double mz, double gz, double sw2, double s, double c) {
  return orc::me2_eemumu({alpha, mz, gz, sw2}, s, c);
}
double orc_me2_eemumu_trace(double alpha, double mz, double gz, double sw2, const double* p) {
  orc::P4 q[4];
  pack(p, 4, q);
  return orc::me2_eemumu_trace({alpha, mz, gz, sw2}, q);
}
double orc_me2_qqbar_ttbar(double alpha_s, double mt, double s, double t) {
  return orc::me2_qqbar_ttbar(alpha_s, mt, s, t);
}
double orc_me2_qqbar_ttbar_trace(double alpha_s, double mt, const double* p) {
  orc::P4 q[4];
  pack(p, 4, q);
  return orc::me2_qqbar_ttbar_trace(alpha_s, mt, q);
}
double orc_me2_gg_ttbar(double alpha_s, double mt, double s, double t) {
  return orc::me2_gg_ttbar(alpha_s, mt, s, t);
}
double orc_me2_gg_ttbar_colour_ordered(double alpha_s, double mt, const double* p) {
  orc::P4 q[4];
  pack(p, 4, q);
  return orc::me2_gg_ttbar_colour_ordered(alpha_s, mt, q);
}
double orc_me2_gg_ttbarg(double alpha_s, double mt, const double* p) {
  orc::P4 q[5];
  pack(p, 5, q);
  return orc::me2_gg_ttbarg(alpha_s, mt, q);
}
double orc_me2_gg_ttbarg_helicity(double alpha_s, double mt, const double* p) {
  orc::P4 q[5];
  pack(p, 5, q);
  return orc::me2_gg_ttbarg_helicity(alpha_s, mt, q);
}
double orc_me2_gg_ttbarg_brute(double alpha_s, double mt, const double* p) {
  orc::P4 q[5];
  pack(p, 5, q);
  return orc::me2_gg_ttbarg_brute(alpha_s, mt, q);
}
// q_in: ngluon incoming gluon momenta then the top momentum ([ngluon+1][4]);
// eps: [ngluon][4][2] (re, im); ubar, v: [4][2]; amps out: [n!][2].
void orc_ggttg_partial_amplitudes(double alpha_s, double mt, const double* q_in, const double* eps,
                                  int ngluon, const double* ubar, const double* v, double* amps) {
  orc::P4 q[4];
  pack(q_in, ngluon + 1, q);
  orc::cplx e[3][4];
  for (int i = 0; i < ngluon; ++i)
    for (int mu = 0; mu < 4; ++mu) e[i][mu] = {eps[(i * 4 + mu) * 2], eps[(i * 4 + mu) * 2 + 1]};
  orc::cplx ub[4], vv[4];
  for (int i = 0; i < 4; ++i) {
    ub[i] = {ubar[2 * i], ubar[2 * i + 1]};
    vv[i] = {v[2 * i], v[2 * i + 1]};
  }
  orc::cplx out[6];
  orc::ggttg_partial_amplitudes(alpha_s, mt, q, e, ngluon, ub, vv, out);
  const int np = ngluon == 2 ? 2 : 6;
  for (int s = 0; s < np; ++s) {
    amps[2 * s] = out[s].real();
    amps[2 * s + 1] = out[s].imag();
  }
}
double orc_me2_qqbar_ttbarg(double alpha_s, double mt, const double* p) {
  orc::P4 q[5];
  pack(p, 5, q);
  return orc::me2_qqbar_ttbarg(alpha_s, mt, q);
}
double orc_me2_qg_ttbarq(double alpha_s, double mt, const double* p) {
  orc::P4 q[5];
  pack(p, 5, q);
  return orc::me2_qg_ttbarq(alpha_s, mt, q);
}
// |M|^2 with the gluon polarisation replaced by eps[4] (complex, pairs re/im).
double orc_me2_qqbar_ttbarg_eps(double alpha_s, double mt, const double* p, const double* eps) {
  orc::P4 q[5];
  pack(p, 5, q);
  const orc::CVec4 e = {orc::cplx(eps[0], eps[1]), orc::cplx(eps[2], eps[3]), orc::cplx(eps[4], eps[5]),
                        orc::cplx(eps[6], eps[7])};
  return orc::me2_qqbar_ttbarg_impl(alpha_s, mt, q, &e);
}
}
