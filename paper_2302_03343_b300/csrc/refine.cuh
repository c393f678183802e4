// VEGAS grid refinement of one dimension, executed by one warp (thesis
// Sec. "Adaptive Monte Carlo: VEGAS algorithm", refinement after Lepage 1978):
// smooth the histogram of w^2 with nearest neighbours, normalise, damp
// m_b = ((r_b - 1)/ln r_b)^alpha, and place the new edges at equal cumulative
// importance by linear interpolation inside the old bins; then clear the
// histogram.  Lanes own bins, a warp prefix sum forms the cumulative
// importance and each new edge finds its old bin by binary search.  An empty
// histogram keeps the grid.  `work` holds 3 nbins + 2 doubles.
#pragma once
#include "common.cuh"

namespace mc {

__device__ inline void refine_dimension(double* e, float* e32, double* h, unsigned int* hn, int nbins, double alpha,
                                        double* work) {
  const int lane = threadIdx.x & 31;
  double* sh_imp = work;
  double* sh_cum = sh_imp + nbins;
  double* sh_old = sh_cum + nbins + 1;
  double part = 0.0;
  for (int b = lane; b < nbins; b += 32) {
    double sm;
    if (b == 0)
      sm = (h[0] + h[1]) / 2.0;
    else if (b == nbins - 1)
      sm = (h[nbins - 2] + h[nbins - 1]) / 2.0;
    else
      sm = (h[b - 1] + h[b] + h[b + 1]) / 3.0;
    sh_imp[b] = sm;
    part += sm;
  }
  for (int b = lane; b <= nbins; b += 32) sh_old[b] = e[b];
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  const double total = part;
  __syncwarp();
  if (total > 0.0) {
    for (int b = lane; b < nbins; b += 32) {
      const double r = sh_imp[b] / total;
      sh_imp[b] = r <= 0.0 ? 0.0 : (r == 1.0 ? 1.0 : pow((r - 1.0) / log(r), alpha));
    }
    __syncwarp();
    double carry = 0.0;  // inclusive prefix sums in chunks of 32 bins
    if (lane == 0) sh_cum[0] = 0.0;
    for (int base = 0; base < nbins; base += 32) {
      const int b = base + lane;
      double v = b < nbins ? sh_imp[b] : 0.0;
      for (int off = 1; off < 32; off <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += t;
      }
      if (b < nbins) sh_cum[b + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    __syncwarp();
    const double per_bin = sh_cum[nbins] / nbins;
    for (int k = 1 + lane; k < nbins; k += 32) {
      const double target = k * per_bin;
      int lo = 0, hi = nbins - 1;  // first old bin b with cum[b+1] >= target
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sh_cum[mid + 1] < target)
          lo = mid + 1;
        else
          hi = mid;
      }
      e[k] = sh_old[lo] + (target - sh_cum[lo]) / sh_imp[lo] * (sh_old[lo + 1] - sh_old[lo]);
    }
  }
  __syncwarp();
  for (int b = lane; b <= nbins; b += 32) e32[b] = float(e[b]);
  for (int b = lane; b < nbins; b += 32) {
    h[b] = 0.0;
    hn[b] = 0u;
  }
}

}  // namespace mc
