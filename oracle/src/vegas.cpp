// Oracle: the VEGAS map, grid refinement and iteration combination.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Thesis Sec. "Adaptive Monte Carlo: VEGAS algorithm": a separable
// histogram importance sampler whose bins keep their number and change their
// widths; the per-iteration estimates are combined with inverse-variance
// weights and checked with eq. vegas-check.  The thesis cites Lepage (1978)
// for the refinement but prints no refinement formula; the rule below is
// Lepage's (smoothing, damping exponent alpha, equal-importance rebinning).
//
// Pins (tests/test_oracle_vegas.py): a hand-made histogram refined by hand;
// convergence of a separable peaked integrand to its analytic quantile grid;
// Gaussian closed form; chi2/dof ~ 1.
#include <cmath>
#include <cstring>

#include "oracle.h"

namespace orc {

// Map the integer uniform k of one dimension through the grid: bin index
// b = floor(u * nbins) taken in integers, position r in the bin, and
// x = e_b + r (e_{b+1} - e_b) with Jacobian nbins (e_{b+1} - e_b).
// (Sec. "Adaptive Monte Carlo: VEGAS algorithm"; inverse transform method of
// Sec. "Inverse transform method" applied to the piecewise-constant p(x).)
double vegas_map_1d(const double* edges, int nbins, int bits, uint64_t k, int* bin, double* jac) {
  const uint64_t prod = k * uint64_t(nbins);
  const uint64_t b = prod >> bits;
  const uint64_t m = prod & ((uint64_t(1) << bits) - 1);
  const double r = double(2 * m + 1) * std::ldexp(1.0, -(bits + 1));
  const double lo = edges[b], hi = edges[b + 1];
  *bin = int(b);
  *jac = double(nbins) * (hi - lo);
  return lo + r * (hi - lo);
}

// Refinement of one dimension from its histogram d_b = sum over events in bin
// b of (f J)^2.  Smoothing with nearest neighbours, normalisation r_b =
// d_b / sum d, damped importance m_b = ((r_b - 1) / ln r_b)^alpha, then new
// edges placed at equal cumulative importance by linear interpolation inside
// the old bins.  A dimension with an empty histogram keeps its grid.
void vegas_refine_1d(const double* edges, int nbins, const double* hist, double alpha,
                     double* out) {
  std::vector<double> smooth(nbins), imp(nbins), cum(nbins + 1);
  if (nbins == 1) {
    out[0] = edges[0];
    out[1] = edges[1];
    return;
  }
  for (int b = 0; b < nbins; ++b) {
    if (b == 0)
      smooth[b] = (hist[0] + hist[1]) / 2.0;
    else if (b == nbins - 1)
      smooth[b] = (hist[nbins - 2] + hist[nbins - 1]) / 2.0;
    else
      smooth[b] = (hist[b - 1] + hist[b] + hist[b + 1]) / 3.0;
  }
  double total = 0.0;
  for (int b = 0; b < nbins; ++b) total += smooth[b];
  if (!(total > 0.0)) {
    std::memcpy(out, edges, sizeof(double) * (nbins + 1));
    return;
  }
  for (int b = 0; b < nbins; ++b) {
    const double r = smooth[b] / total;
    if (r <= 0.0)
      imp[b] = 0.0;
    else if (r == 1.0)
      imp[b] = 1.0;
    else
      imp[b] = std::pow((r - 1.0) / std::log(r), alpha);
  }
  cum[0] = 0.0;
  for (int b = 0; b < nbins; ++b) cum[b + 1] = cum[b] + imp[b];
  const double per_bin = cum[nbins] / nbins;
  out[0] = edges[0];
  out[nbins] = edges[nbins];
  for (int k = 1; k < nbins; ++k) {
    const double target = k * per_bin;
    int b = 0;
    while (b + 1 < nbins && cum[b + 1] < target) ++b;
    const double frac = (target - cum[b]) / imp[b];
    out[k] = edges[b] + frac * (edges[b + 1] - edges[b]);
  }
}

}  // namespace orc

extern "C" {

void orc_vegas_map(int ndim, int nbins, const double* edges, int prec, const uint64_t* k, double* x,
                   int32_t* bins, double* jac) {
  const int bits = orc::uniform_bits(prec);
  double j = 1.0;
  for (int d = 0; d < ndim; ++d) {
    int b;
    double jd;
    x[d] = orc::vegas_map_1d(edges + d * (nbins + 1), nbins, bits, k[d], &b, &jd);
    bins[d] = b;
    j *= jd;
  }
  *jac = j;
}

void orc_vegas_refine(int ndim, int nbins, const double* edges, const double* hist_w2, double alpha,
                      double* new_edges) {
  for (int d = 0; d < ndim; ++d)
    orc::vegas_refine_1d(edges + d * (nbins + 1), nbins, hist_w2 + d * nbins, alpha,
                         new_edges + d * (nbins + 1));
}

// Per-iteration estimate (eq. mc_est_is) and variance of the estimate: the
// unbiased sample variance of the weights divided by N (reading of the two
// unequal forms printed in eq. var-en-est; the first, unbiased one is used).
void orc_iteration_estimate(double sum, double sum2, int64_t n, double* mean, double* var) {
  const double nn = double(n);
  *mean = sum / nn;
  *var = n > 1 ? (sum2 / nn - (*mean) * (*mean)) / (nn - 1.0) : 0.0;
}

// Inverse-variance combination of M iterations and chi^2 per degree of
// freedom (Sec. "Adaptive Monte Carlo: VEGAS algorithm", eq. vegas-check).
// Iterations with zero variance are skipped unless all have zero variance.
void orc_combine(int n, const double* e, const double* s2, double* mean, double* sigma,
                 double* chi2dof) {
  double inv = 0.0, acc = 0.0;
  int used = 0;
  for (int i = 0; i < n; ++i)
    if (s2[i] > 0.0) {
      inv += 1.0 / s2[i];
      acc += e[i] / s2[i];
      ++used;
    }
  if (used == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m += e[i];
    *mean = n ? m / n : 0.0;
    *sigma = 0.0;
    *chi2dof = 0.0;
    return;
  }
  const double s2bar = 1.0 / inv;
  *mean = s2bar * acc;
  *sigma = std::sqrt(s2bar);
  double chi = 0.0;
  for (int i = 0; i < n; ++i)
    if (s2[i] > 0.0) chi += (e[i] - *mean) * (e[i] - *mean) / s2[i];
  *chi2dof = used > 1 ? chi / (used - 1) : 0.0;
}
}
