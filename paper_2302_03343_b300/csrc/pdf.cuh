// Log-bicubic PDF interpolation, device side (thesis Sec. "LHAPDF: the Les
// Houches Accord PDF"; PDFFlow, Sec. "Software design and benchmarks").
//
// Grid layout in device memory: values [nflav][nq][nx] (x contiguous), knot
// coordinates log x and log Q^2 in FP64.  Interpolation is cubic Hermite in
// log x on the cell [i, i+1] at the Q knots j-1..j+2, then cubic Hermite in
// log Q^2 on [j, j+1]; knot slopes are the mean of the adjacent divided
// differences, one-sided at the first and last knot.
//
// The Q step is linear in the four Q-knot values, with weights that depend
// on Q alone.  For a fixed factorisation scale the fused kernel therefore
// contracts the grid over Q once per block (the "Q-collapsed" table, staged
// in shared memory with its log-x slopes) and each event then pays one 1D
// Hermite step per flavour.  This is the same interpolant up to rounding.
#pragma once
#include "common.cuh"

namespace mc {

struct PdfDev {
  int nx, nq, nflav;
  const double* logx;   // [nx]
  const double* logq2;  // [nq]
  const double* xf64;   // [nflav][nq][nx]
  const float* xf32;    // same, FP32
  double x_lo, x_hi, q2_lo, q2_hi;  // the grid's range (first and last knots)
  const float* xf32t;  // FP32, [nq][nx][nfp]: the flavours of a knot together, padded to nfp (a multiple of 4)
  int nfp;
};

MC_HD int knot_cell(const double* t, int n, double v) {
  // largest i in [0, n-2] with t[i] <= v (binary search)
  int lo = 0, hi = n - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t[mid] <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Weights w[0..3] of the Q knots j0 .. j0+3 (j0 = iq - 1; weights of knots
// outside the grid are 0) such that the Q step equals sum_t w[t] v[j0 + t].
MC_HD void q_weights(const double* lq, int nq, double s, int* j0_out, double* w) {
  const int iq = knot_cell(lq, nq, s);
  const double h = lq[iq + 1] - lq[iq];
  const double tau = (s - lq[iq]) / h;
  const double t2 = tau * tau, t3 = t2 * tau;
  const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + tau, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  for (int t = 0; t < 4; ++t) w[t] = 0.0;
  // value terms
  w[1] += h00;
  w[2] += h01;
  // slope at iq: d = (v[iq+1]-v[iq])/dr averaged with (v[iq]-v[iq-1])/dl
  auto add_slope = [&](int k, double coef) {  // coef * slope at knot k
    const int b = k - (iq - 1);             // stencil position of knot k
    if (k == 0) {
      const double d = lq[1] - lq[0];
      w[b] -= coef / d;
      w[b + 1] += coef / d;
    } else if (k == nq - 1) {
      const double d = lq[k] - lq[k - 1];
      w[b] += coef / d;
      w[b - 1] -= coef / d;
    } else {
      const double dr = lq[k + 1] - lq[k], dl = lq[k] - lq[k - 1];
      w[b + 1] += 0.5 * coef / dr;
      w[b] += 0.5 * coef * (-1.0 / dr + 1.0 / dl);
      w[b - 1] -= 0.5 * coef / dl;
    }
  };
  add_slope(iq, h10 * h);
  add_slope(iq + 1, h11 * h);
  *j0_out = iq - 1;
}

// q_weights in the working precision R: the knots are read in FP64 and
// rounded, the weights formed in R.
template <class R>
MC_D void q_weights_r(const double* lq, int nq, R s, int* j0_out, R* w) {
  const int iq = knot_cell(lq, nq, double(s));
  const R h = R(lq[iq + 1] - lq[iq]);
  const R tau = (s - R(lq[iq])) / h;
  const R t2 = tau * tau, t3 = t2 * tau;
  const R h00 = R(2) * t3 - R(3) * t2 + R(1), h10 = t3 - R(2) * t2 + tau, h01 = R(-2) * t3 + R(3) * t2,
          h11 = t3 - t2;
  for (int t = 0; t < 4; ++t) w[t] = R(0);
  w[1] += h00;
  w[2] += h01;
  auto add_slope = [&](int k, R coef) {
    const int b = k - (iq - 1);
    if (k == 0) {
      const R d = R(lq[1] - lq[0]);
      w[b] -= coef / d;
      w[b + 1] += coef / d;
    } else if (k == nq - 1) {
      const R d = R(lq[k] - lq[k - 1]);
      w[b] += coef / d;
      w[b - 1] -= coef / d;
    } else {
      const R dr = R(lq[k + 1] - lq[k]), dl = R(lq[k] - lq[k - 1]);
      w[b + 1] += R(0.5) * coef / dr;
      w[b] += R(0.5) * coef * (R(-1) / dr + R(1) / dl);
      w[b - 1] -= R(0.5) * coef / dl;
    }
  };
  add_slope(iq, h10 * h);
  add_slope(iq + 1, h11 * h);
  *j0_out = iq - 1;
}

template <class R>
MC_D R hermite(R tau, R h, R f0, R f1, R d0, R d1) {
  const R t2 = tau * tau, t3 = t2 * tau;
  return (R(2) * t3 - R(3) * t2 + R(1)) * f0 + (t3 - R(2) * t2 + tau) * h * d0 + (R(-2) * t3 + R(3) * t2) * f1 +
         (t3 - t2) * h * d1;
}

// Shared-memory table of one Q-collapsed flavour: values f[i] and log-x
// slopes d[i] at the x knots.
template <class R>
struct PdfTable {
  const R* t;  // log x knots [nx]
  const R* f;  // [nx]
  const R* d;  // [nx]
  int nx;
};

// 1D Hermite interpolation of x f(x) on a Q-collapsed table.
template <class R>
MC_D R pdf_interp_1d(const PdfTable<R>& tb, R logx) {
  int lo = 0, hi = tb.nx - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tb.t[mid] <= logx)
      lo = mid;
    else
      hi = mid - 1;
  }
  const R h = tb.t[lo + 1] - tb.t[lo];
  const R tau = (logx - tb.t[lo]) / h;
  return hermite(tau, h, tb.f[lo], tb.f[lo + 1], tb.d[lo], tb.d[lo + 1]);
}

// Block-cooperative construction of the Q-collapsed tables of `nfl` flavours
// (flavour indices fl[]) at log Q^2 = s into shared memory:
// sm_t[nx], then per flavour sm_f[nx], sm_d[nx].  Ends with __syncthreads.
template <class R>
__device__ void build_pdf_tables(const PdfDev& pdf, double s, const int* fl, int nfl, R* sm_t, R* sm_f, R* sm_d) {
  int j0;
  double w[4];
  q_weights(pdf.logq2, pdf.nq, s, &j0, w);
  const int nx = pdf.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) sm_t[i] = R(pdf.logx[i]);
  for (int idx = threadIdx.x; idx < nfl * nx; idx += blockDim.x) {
    const int k = idx / nx, i = idx % nx;
    const double* base = pdf.xf64 + size_t(fl[k]) * pdf.nq * nx;
    double v = 0.0;
    for (int t = 0; t < 4; ++t) {
      const int j = j0 + t;
      if (j >= 0 && j < pdf.nq && w[t] != 0.0) v += w[t] * base[size_t(j) * nx + i];
    }
    sm_f[k * nx + i] = R(v);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nfl * nx; idx += blockDim.x) {
    const int k = idx / nx, i = idx % nx;
    const R* f = sm_f + k * nx;
    R d;
    if (i == 0)
      d = (f[1] - f[0]) / (sm_t[1] - sm_t[0]);
    else if (i == nx - 1)
      d = (f[nx - 1] - f[nx - 2]) / (sm_t[nx - 1] - sm_t[nx - 2]);
    else
      d = R(0.5) * ((f[i + 1] - f[i]) / (sm_t[i + 1] - sm_t[i]) + (f[i] - f[i - 1]) / (sm_t[i] - sm_t[i - 1]));
    sm_d[k * nx + i] = d;
  }
  __syncthreads();
}

}  // namespace mc
