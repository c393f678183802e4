// Internal: definitions of the opaque handles of include/mcint.h, shared by
// the translation units of the C ABI.
#pragma once
#include <vector>

#include "../../include/mcint.h"
#include "launch.h"

namespace mc {
void set_last_error(const char* msg);  // api.cu
// Validates a process description and fills KernelArgs::prm, pdf, fl,
// logq2_f, w0_coef3 and e2eta (the rest zeroed); MC_OK or an MC_E* code with
// the message set (api.cu).
int fill_process_args(const mc_integrand* itg, mc_pdf pdf, KernelArgs* a);
int process_dim(const mc_integrand* itg);  // sampled dimensions of the process, -1 if unknown
// Inverse-variance combination of per-iteration estimates e[i] with
// variances s2[i] (thesis Sec. VEGAS, eq. vegas-check): mean, sigma, chi2/dof.
void combine_iterations(const std::vector<double>& e, const std::vector<double>& s2, mc_result* r);
}

struct mc_pdf_s {
  int device = 0, nx = 0, nq = 0, nflav = 0;
  std::vector<int> pids;
  std::vector<double> logq2;  // host copy of the Q^2 knots (log)
  double* d_logx = nullptr;
  double* d_logq2 = nullptr;
  double* d_xf64 = nullptr;
  float* d_xf32 = nullptr;
  double x_lo = 0, x_hi = 0, q2_lo = 0, q2_hi = 0;  // first and last knots
  float* d_xf32t = nullptr;  // [nq][nx][nfp], flavours innermost, padded with zeros
  int nfp = 0;
  mc::PdfDev dev() const {
    return {nx, nq, nflav, d_logx, d_logq2, d_xf64, d_xf32, x_lo, x_hi, q2_lo, q2_hi, d_xf32t, nfp};
  }
  int index(int pid) const {
    for (int i = 0; i < nflav; ++i)
      if (pids[i] == pid) return i;
    return -1;
  }
};

struct mc_vegas_s {
  int device = 0, ndim = 0, nbins = 0, prec = 0;
  uint64_t seed = 0;
  uint32_t iteration = 0, gid = 0;
  double* d_edges = nullptr;
  float* d_edges32 = nullptr;
  double* d_hist_w2 = nullptr;
  unsigned int* d_hist_n = nullptr;
  mc::BlockPartial* d_partials = nullptr;
  int max_partials = 0;
  mc::BlockPartial* d_total = nullptr;
  mc::BlockPartial* h_total = nullptr;  // pinned
  cudaEvent_t k0 = nullptr, k1 = nullptr;  // around the last integrand launch
  bool timed = false;
  // the last iteration's events (what mc_unweight selects from): its
  // iteration counter and size; false once the grid has changed since
  bool last_valid = false;
  uint32_t last_iteration = 0;
  int64_t last_n = 0;
  // unweighting: device scratch (grow-only), pinned count, timing events
  void* d_uw = nullptr;
  size_t uw_bytes = 0;
  unsigned long long* h_count = nullptr;
  cudaEvent_t u0 = nullptr, u1 = nullptr;
  bool uw_timed = false;
  // three-channel process: probabilities and the last iteration's update sums
  double alpha[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
  double wch[3] = {0.0, 0.0, 0.0};
  double* d_wch = nullptr;
};

