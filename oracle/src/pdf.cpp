// Oracle: LHAPDF-style grid and its log-bicubic interpolation.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "LHAPDF: the Les Houches Accord PDF" and Sec. "Software design
// and benchmarks" (PDFFlow): values x f(x, Q^2) stored at knots of the
// (x, Q^2) plane, interpolated by cubic Hermite splines in (log x, log Q^2)
// from the 4 x 4 neighbouring knots.  Knot slopes are the mean of the two
// adjacent divided differences, one-sided at the first and last knot (where
// the thesis says the 4-knot stencil is unavailable).  Log Q or log Q^2 give
// the same interpolant because the slopes are divided differences.
//
// Pins (tests/test_oracle_pdf.py): exact reproduction of every stored node;
// exact reproduction of a function quadratic in (log x, log Q^2) inside
// interior cells; relative-difference metric eq. pdfflow-diff.
#include <cmath>
#include <limits>

#include "oracle.h"

namespace orc {

int Pdf::flavour_index(int pid) const {
  for (int i = 0; i < nflav; ++i)
    if (pids[i] == pid) return i;
  return -1;
}

static double hermite(double tau, double h, double f0, double f1, double d0, double d1) {
  const double tau2 = tau * tau, tau3 = tau2 * tau;
  const double h00 = 2.0 * tau3 - 3.0 * tau2 + 1.0;
  const double h10 = tau3 - 2.0 * tau2 + tau;
  const double h01 = -2.0 * tau3 + 3.0 * tau2;
  const double h11 = tau3 - tau2;
  return h00 * f0 + h10 * h * d0 + h01 * f1 + h11 * h * d1;
}

// Slope at knot i of values fv[] sampled at coordinates t[] (n knots).
static double knot_slope(const double* t, int n, const double* fv, int i) {
  if (i == 0) return (fv[1] - fv[0]) / (t[1] - t[0]);
  if (i == n - 1) return (fv[n - 1] - fv[n - 2]) / (t[n - 1] - t[n - 2]);
  return 0.5 * ((fv[i + 1] - fv[i]) / (t[i + 1] - t[i]) + (fv[i] - fv[i - 1]) / (t[i] - t[i - 1]));
}

static int locate(const std::vector<double>& knots, double v) {
  const int n = int(knots.size());
  int i = 0;
  while (i + 1 < n - 1 && knots[i + 1] <= v) ++i;
  return i;
}

double pdf_xfxq2(const Pdf& pdf, int pid, double x, double q2) {
  const int fl = pdf.flavour_index(pid);
  const double nan = std::numeric_limits<double>::quiet_NaN();
  if (fl < 0) return nan;
  const double q2min = pdf.q[0] * pdf.q[0], q2max = pdf.q[pdf.nq - 1] * pdf.q[pdf.nq - 1];
  if (!(x >= pdf.x[0] && x <= pdf.x[pdf.nx - 1] && q2 >= q2min && q2 <= q2max)) return nan;
  std::vector<double> q2knots(pdf.nq);
  for (int j = 0; j < pdf.nq; ++j) q2knots[j] = pdf.q[j] * pdf.q[j];
  const int ix = locate(pdf.x, x);
  const int iq = locate(q2knots, q2);
  const double t = std::log(x), s = std::log(q2);
  const double hx = pdf.logx[ix + 1] - pdf.logx[ix];
  const double tau_x = (t - pdf.logx[ix]) / hx;
  // x-interpolation at every Q knot of the 4-knot stencil that exists.
  std::vector<double> along_x(pdf.nx), v(pdf.nq, 0.0);
  const int jlo = iq > 0 ? iq - 1 : 0;
  const int jhi = iq + 2 < pdf.nq ? iq + 2 : pdf.nq - 1;
  for (int j = jlo; j <= jhi; ++j) {
    for (int i = 0; i < pdf.nx; ++i) along_x[i] = pdf.node(i, j, fl);
    const double d0 = knot_slope(pdf.logx.data(), pdf.nx, along_x.data(), ix);
    const double d1 = knot_slope(pdf.logx.data(), pdf.nx, along_x.data(), ix + 1);
    v[j] = hermite(tau_x, hx, along_x[ix], along_x[ix + 1], d0, d1);
  }
  const double hq = pdf.logq2[iq + 1] - pdf.logq2[iq];
  const double tau_q = (s - pdf.logq2[iq]) / hq;
  const double e0 = knot_slope(pdf.logq2.data(), pdf.nq, v.data(), iq);
  const double e1 = knot_slope(pdf.logq2.data(), pdf.nq, v.data(), iq + 1);
  return hermite(tau_q, hq, v[iq], v[iq + 1], e0, e1);
}

}  // namespace orc

extern "C" {

void* orc_pdf_new(int nx, const double* x, int nq, const double* q, int nflav, const int* pids,
                  const double* xf) {
  auto* pdf = new orc::Pdf;
  pdf->nx = nx;
  pdf->nq = nq;
  pdf->nflav = nflav;
  pdf->x.assign(x, x + nx);
  pdf->q.assign(q, q + nq);
  pdf->pids.assign(pids, pids + nflav);
  pdf->xf.assign(xf, xf + size_t(nx) * nq * nflav);
  for (int i = 0; i < nx; ++i) pdf->logx.push_back(std::log(x[i]));
  for (int j = 0; j < nq; ++j) pdf->logq2.push_back(std::log(q[j] * q[j]));
  return pdf;
}

void orc_pdf_free(void* pdf) { delete static_cast<orc::Pdf*>(pdf); }

double orc_pdf_xfxq2(const void* pdf, int pid, double x, double q2) {
  return orc::pdf_xfxq2(*static_cast<const orc::Pdf*>(pdf), pid, x, q2);
}
}
