// Oracle: an LHAPDF-style PDF set with sub-grids, members, extrapolation,
// and the alpha_s(Q) interpolation.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "LHAPDF: the Les Houches Accord PDF" and Sec. "PDFFlow:
// interpolating PDFs on GPUs":
//  * a grid may be split into sub-grids at quark-mass thresholds; adjacent
//    sub-grids share the threshold Q knot and a query exactly on it belongs
//    to the upper sub-grid;
//  * inside a sub-grid the values x f are interpolated by cubic Hermite
//    splines in (log x, log Q^2) from the 4 x 4 neighbouring knots (knot
//    slopes: mean of the adjacent divided differences, one-sided at the
//    sub-grid's first and last knot); where a sub-grid has fewer than 4 knots
//    in a direction the interpolation is bilinear in (log x, log Q^2);
//  * below x_min, x f is extrapolated linearly in log x from the two lowest x
//    knots, in log(x f) when both values exceed 1e-3 and in x f otherwise;
//    above Q_max the same, in log Q^2, from the two highest Q knots;
//  * below Q_min: x f(x, Q^2) = x f(x, Q^2_min) (Q^2 / Q^2_min)^(gamma r + 1 - r),
//    r = Q^2 / Q^2_min, gamma the anomalous dimension d ln(x f) / d ln Q^2 at
//    Q^2_min from the two lowest Q knots (1 when either value is not
//    positive); where x and Q are both outside, the x rule runs first and its
//    values enter the Q rule; the continuation knots are evaluated in their
//    own sub-grid (the first one below Q_min, the last one above Q_max);
//  * alpha_s: cubic Hermite in log Q^2 on segments between repeated
//    (threshold) knots, alpha_s(Q_max) above the grid, and below it ln alpha_s
//    continued linearly in ln Q^2 from the two lowest knots.
// The thesis writes the anomalous dimension as a derivative with respect to
// Q^2; the exponent of the continuation is dimensionless only for the
// derivative with respect to ln Q^2, which is the reading taken here.
//
// Pins (tests/test_oracle_pdfset.py): node reproduction in every sub-grid,
// exact reproduction of quadratic (bicubic sub-grids) and bilinear functions
// of (log x, log Q^2), exact power-law extrapolation, the two limits of the
// low-Q continuation that the thesis prints, one-loop running alpha_s.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "oracle.h"

namespace orc {
namespace {

struct SubGrid {
  int nx = 0, nq = 0;
  std::vector<double> logx, logq2;
  size_t off = 0;  // offset of this sub-grid's block in a member's values
};

struct PdfSet {
  int nflav = 0, nmem = 0;
  std::vector<int> pids;
  std::vector<SubGrid> sub;
  std::vector<double> xf;  // [member][sub-grid block: [x][q][flav]]
  size_t member_size = 0;

  int flavour_index(int pid) const {
    for (int i = 0; i < nflav; ++i)
      if (pids[i] == pid) return i;
    return -1;
  }
  double node(int m, int s, int ix, int iq, int fl) const {
    const SubGrid& g = sub[s];
    return xf[size_t(m) * member_size + g.off + (size_t(ix) * g.nq + iq) * nflav + fl];
  }
};

double hermite(double tau, double h, double f0, double f1, double d0, double d1) {
  const double tau2 = tau * tau, tau3 = tau2 * tau;
  return (2.0 * tau3 - 3.0 * tau2 + 1.0) * f0 + (tau3 - 2.0 * tau2 + tau) * h * d0 + (-2.0 * tau3 + 3.0 * tau2) * f1 +
         (tau3 - tau2) * h * d1;
}

double slope(const std::vector<double>& t, const std::vector<double>& f, int i) {
  const int n = int(t.size());
  if (i == 0) return (f[1] - f[0]) / (t[1] - t[0]);
  if (i == n - 1) return (f[n - 1] - f[n - 2]) / (t[n - 1] - t[n - 2]);
  return 0.5 * ((f[i + 1] - f[i]) / (t[i + 1] - t[i]) + (f[i] - f[i - 1]) / (t[i] - t[i - 1]));
}

// cell i with t[i] <= v < t[i+1] (the last cell includes its upper knot)
int cell(const std::vector<double>& t, double v) {
  int i = 0;
  while (i + 2 < int(t.size()) && t[i + 1] <= v) ++i;
  return i;
}

// Interpolation inside sub-grid s, (lx, lq) within its bounds.
double interp(const PdfSet& p, int m, int s, int fl, double lx, double lq) {
  const SubGrid& g = p.sub[s];
  const int ix = cell(g.logx, lx), iq = cell(g.logq2, lq);
  const double tx = (lx - g.logx[ix]) / (g.logx[ix + 1] - g.logx[ix]);
  const double tq = (lq - g.logq2[iq]) / (g.logq2[iq + 1] - g.logq2[iq]);
  if (g.nx < 4 || g.nq < 4) {
    return (1.0 - tx) * (1.0 - tq) * p.node(m, s, ix, iq, fl) + tx * (1.0 - tq) * p.node(m, s, ix + 1, iq, fl) +
           (1.0 - tx) * tq * p.node(m, s, ix, iq + 1, fl) + tx * tq * p.node(m, s, ix + 1, iq + 1, fl);
  }
  // Hermite in log x at the Q knots the log Q^2 slopes need (iq-1 .. iq+2),
  // from the x knots its own slopes need (ix-1 .. ix+2), then in log Q^2
  std::vector<double> along_x(g.nx, 0.0), at_q(g.nq, 0.0);
  for (int j = std::max(iq - 1, 0); j <= std::min(iq + 2, g.nq - 1); ++j) {
    for (int i = std::max(ix - 1, 0); i <= std::min(ix + 2, g.nx - 1); ++i) along_x[i] = p.node(m, s, i, j, fl);
    at_q[j] = hermite(tx, g.logx[ix + 1] - g.logx[ix], along_x[ix], along_x[ix + 1], slope(g.logx, along_x, ix),
                      slope(g.logx, along_x, ix + 1));
  }
  return hermite(tq, g.logq2[iq + 1] - g.logq2[iq], at_q[iq], at_q[iq + 1], slope(g.logq2, at_q, iq),
                 slope(g.logq2, at_q, iq + 1));
}

// Linear continuation from (t0, f0), (t1, f1) to t: in log f when both exceed 1e-3.
double continue_linear(double t, double t0, double t1, double f0, double f1) {
  const double u = (t - t0) / (t1 - t0);
  if (f0 > 1e-3 && f1 > 1e-3) return std::exp(std::log(f0) + u * (std::log(f1) - std::log(f0)));
  return f0 + u * (f1 - f0);
}

int subgrid_of(const PdfSet& p, double lq) {
  const int ns = int(p.sub.size());
  for (int s = 0; s < ns; ++s)
    if (lq < p.sub[s].logq2.back() || s == ns - 1) return s;
  return ns - 1;
}

// x f at (lx, lq) in sub-grid s (lq inside it): the x rule below x_min.
double at_q_in(const PdfSet& p, int m, int fl, double lx, double lq, int s) {
  const SubGrid& g = p.sub[s];
  if (lx >= g.logx[0]) return interp(p, m, s, fl, lx, lq);
  const double f0 = interp(p, m, s, fl, g.logx[0], lq), f1 = interp(p, m, s, fl, g.logx[1], lq);
  return continue_linear(lx, g.logx[0], g.logx[1], f0, f1);
}

double at_q_inside(const PdfSet& p, int m, int fl, double lx, double lq) {
  return at_q_in(p, m, fl, lx, lq, subgrid_of(p, lq));
}

double xfxq2(const PdfSet& p, int m, int pid, double x, double q2) {
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const int fl = p.flavour_index(pid);
  if (fl < 0 || m < 0 || m >= p.nmem || !(x > 0.0) || !(q2 > 0.0)) return nan;
  const double lx = std::log(x), lq = std::log(q2);
  if (lx > p.sub[0].logx.back()) return nan;  // above x_max: no rule
  const SubGrid& first = p.sub.front();
  const SubGrid& last = p.sub.back();
  if (lq >= first.logq2.front() && lq <= last.logq2.back()) return at_q_inside(p, m, fl, lx, lq);
  // the continuation knots are the last sub-grid's two highest (above Q_max)
  // and the first sub-grid's two lowest (below Q_min), each in its sub-grid
  const int sl = int(p.sub.size()) - 1;
  if (lq > last.logq2.back()) {
    const double t0 = last.logq2[last.nq - 2], t1 = last.logq2[last.nq - 1];
    return continue_linear(lq, t0, t1, at_q_in(p, m, fl, lx, t0, sl), at_q_in(p, m, fl, lx, t1, sl));
  }
  // low Q: anomalous-dimension continuation
  const double t0 = first.logq2[0], t1 = first.logq2[1];
  const double f0 = at_q_in(p, m, fl, lx, t0, 0), f1 = at_q_in(p, m, fl, lx, t1, 0);
  const double gamma = (f0 > 0.0 && f1 > 0.0) ? std::log(f1 / f0) / (t1 - t0) : 1.0;
  const double r = std::exp(lq - t0);
  return f0 * std::pow(r, gamma * r + 1.0 - r);
}

struct AlphaS {
  std::vector<double> lq, a;
};

double alphas_q2(const AlphaS& s, double q2) {
  const int n = int(s.lq.size());
  if (!(q2 > 0.0)) return std::numeric_limits<double>::quiet_NaN();
  const double lq = std::log(q2);
  if (lq >= s.lq[n - 1]) return s.a[n - 1];
  if (lq < s.lq[0])
    return std::exp(std::log(s.a[0]) + (lq - s.lq[0]) / (s.lq[1] - s.lq[0]) * (std::log(s.a[1]) - std::log(s.a[0])));
  // segment [b, e) between repeated knots containing lq (upper at a threshold)
  int b = 0;
  for (int i = 1; i < n; ++i)
    if (s.lq[i] == s.lq[i - 1] && lq >= s.lq[i]) b = i;
  int e = b + 1;
  while (e < n && s.lq[e] != s.lq[e - 1]) ++e;
  const std::vector<double> t(s.lq.begin() + b, s.lq.begin() + e), f(s.a.begin() + b, s.a.begin() + e);
  const int i = cell(t, lq);
  const double h = t[i + 1] - t[i];
  return hermite((lq - t[i]) / h, h, f[i], f[i + 1], slope(t, f, i), slope(t, f, i + 1));
}

}  // namespace
}  // namespace orc

extern "C" {

void* orc_pdfset_new(int nsub, const int* nx, const int* nq, const double* x, const double* q, int nflav,
                     const int* pids, int nmem, const double* xf) {
  auto* p = new orc::PdfSet;
  p->nflav = nflav;
  p->nmem = nmem;
  p->pids.assign(pids, pids + nflav);
  size_t xo = 0, qo = 0, off = 0;
  for (int s = 0; s < nsub; ++s) {
    orc::SubGrid g;
    g.nx = nx[s];
    g.nq = nq[s];
    for (int i = 0; i < nx[s]; ++i) g.logx.push_back(std::log(x[xo + i]));
    for (int j = 0; j < nq[s]; ++j) g.logq2.push_back(std::log(q[qo + j] * q[qo + j]));
    g.off = off;
    off += size_t(nx[s]) * nq[s] * nflav;
    xo += nx[s];
    qo += nq[s];
    p->sub.push_back(g);
  }
  p->member_size = off;
  p->xf.assign(xf, xf + off * size_t(nmem));
  return p;
}

void orc_pdfset_free(void* p) { delete static_cast<orc::PdfSet*>(p); }

double orc_pdfset_xfxq2(const void* p, int member, int pid, double x, double q2) {
  return orc::xfxq2(*static_cast<const orc::PdfSet*>(p), member, pid, x, q2);
}

void* orc_alphas_new(int n, const double* q, const double* a) {
  auto* s = new orc::AlphaS;
  for (int i = 0; i < n; ++i) {
    s->lq.push_back(std::log(q[i] * q[i]));
    s->a.push_back(a[i]);
  }
  return s;
}

void orc_alphas_free(void* s) { delete static_cast<orc::AlphaS*>(s); }

double orc_alphas_q2(const void* s, double q2) { return orc::alphas_q2(*static_cast<const orc::AlphaS*>(s), q2); }
}
