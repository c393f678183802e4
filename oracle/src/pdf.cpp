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

#include "kinematics_t.h"
#include "oracle.h"

namespace orc {

int Pdf::flavour_index(int pid) const {
  for (int i = 0; i < nflav; ++i)
    if (pids[i] == pid) return i;
  return -1;
}

double pdf_xfxq2(const Pdf& pdf, int pid, double x, double q2) { return pdf_xfxq2_t<double>(pdf, pid, x, q2); }

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
