// C ABI of the library (declared in include/mcint.h): handles, argument
// validation, launch shapes and the host-side VEGAS driver.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mcint.h"
#include "launch.h"

using mc::BlockPartial;
using mc::KernelArgs;

namespace {
// the reduced sums of a launch followed by its status word (MC_ETIMEOUT or 0)
constexpr size_t kTotalBytes = sizeof(BlockPartial) + 16;

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define MC_CUDA(call)                                                                      \
  do {                                                                                     \
    const cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return fail(MC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int current_device(int* dev) {
  const cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return fail(MC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  return MC_OK;
}

int process_ndim(const mc_integrand* itg) {
  switch (itg->proc) {
    case MC_EE_MUMU: return 2;
    case MC_PP_TTBAR: return 4;
    case MC_GG_TTBARG: return 14;
    // the Gaussian kernels loop over at most 16 dimensions
    case MC_GAUSS: return itg->gauss_dim >= 1 && itg->gauss_dim <= 16 ? itg->gauss_dim : -1;
    case MC_GG_TTBARG_7D: return 7;
    case MC_GG_TTBARG_MC: return mc::kChannelGridDims;
    case MC_PP_TTBARJ: return 7;
  }
  return -1;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  return n;
}

// Colour matrix C_de = sum over the colours of the quark, antiquark, top,
// anti-top and gluon of c_d c_e^* for the five diagrams of me2_qline_ttbarg:
// c_1 = (T^b T^a)_ji T^b_kl, c_2 = (T^a T^b)_ji T^b_kl, c_3 = T^b_ji (T^a T^b)_kl,
// c_4 = T^b_ji (T^b T^a)_kl, c_5 = f^bca T^b_ji T^c_kl, with the Gell-Mann
// generators T^a = lambda^a / 2 and f^abc = -2 i tr([T^a, T^b] T^c).
// Re/im pairs, row-major.
void light_line_colour(double* out) {
  using C = std::complex<double>;
  C t[8][3][3] = {};
  const C i1(0.0, 1.0);
  t[0][0][1] = t[0][1][0] = 0.5;
  t[1][0][1] = -0.5 * i1; t[1][1][0] = 0.5 * i1;
  t[2][0][0] = 0.5; t[2][1][1] = -0.5;
  t[3][0][2] = t[3][2][0] = 0.5;
  t[4][0][2] = -0.5 * i1; t[4][2][0] = 0.5 * i1;
  t[5][1][2] = t[5][2][1] = 0.5;
  t[6][1][2] = -0.5 * i1; t[6][2][1] = 0.5 * i1;
  t[7][0][0] = t[7][1][1] = 0.5 / std::sqrt(3.0); t[7][2][2] = -1.0 / std::sqrt(3.0);
  auto prod = [&](int a, int b, int r, int c) {  // (T^a T^b)_rc
    C v = 0.0;
    for (int k = 0; k < 3; ++k) v += t[a][r][k] * t[b][k][c];
    return v;
  };
  double f[8][8][8];
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        C tr = 0.0;
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) tr += (prod(a, b, r, s) - prod(b, a, r, s)) * t[c][s][r];
        f[a][b][c] = (-2.0 * i1 * tr).real();
      }
  C acc[25] = {};
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            C c[5] = {};
            for (int b = 0; b < 8; ++b) {
              c[0] += prod(b, a, j, i) * t[b][k][l];
              c[1] += prod(a, b, j, i) * t[b][k][l];
              c[2] += t[b][j][i] * prod(a, b, k, l);
              c[3] += t[b][j][i] * prod(b, a, k, l);
              for (int e = 0; e < 8; ++e) c[4] += f[b][e][a] * t[b][j][i] * t[e][k][l];
            }
            for (int d = 0; d < 5; ++d)
              for (int e = 0; e < 5; ++e) acc[d * 5 + e] += c[d] * std::conj(c[e]);
          }
  for (int n = 0; n < 25; ++n) {
    out[2 * n] = acc[n].real();
    out[2 * n + 1] = acc[n].imag();
  }
}

}  // namespace

#include "handles.h"
#include "tc_gemm.h"

namespace mc {
// Message returned by mc_last_error() for the calling thread.
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace mc

extern "C" {

const char* mc_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ PDF
int mc_pdf_load(const double* x, int nx, const double* q, int nq, const int32_t* pids, int nflav, const double* xf,
                mc_pdf* out) {
  if (!out) return fail(MC_EINVAL, "mc_pdf_load: out is NULL");
  *out = nullptr;
  if (!x || !q || !pids || !xf) return fail(MC_EINVAL, "mc_pdf_load: NULL array");
  if (nx < 4 || nq < 4 || nflav < 1 || nflav > 64) return fail(MC_EINVAL, "mc_pdf_load: bad shape");
  for (int i = 0; i < nx; ++i) {
    if (!(x[i] > 0.0 && x[i] <= 1.0)) return fail(MC_EINVAL, "mc_pdf_load: x knot %d outside (0,1]", i);
    if (i && !(x[i] > x[i - 1])) return fail(MC_EINVAL, "mc_pdf_load: x knots not increasing at %d", i);
  }
  for (int j = 0; j < nq; ++j) {
    if (!(q[j] > 0.0 && std::isfinite(q[j]))) return fail(MC_EINVAL, "mc_pdf_load: bad Q knot %d", j);
    if (j && !(q[j] > q[j - 1])) return fail(MC_EINVAL, "mc_pdf_load: Q knots not increasing at %d", j);
  }
  const size_t nval = size_t(nx) * nq * nflav;
  for (size_t i = 0; i < nval; ++i)
    if (!std::isfinite(xf[i])) return fail(MC_EINVAL, "mc_pdf_load: non-finite value at %zu", i);
  auto* p = new mc_pdf_s;
  int rc = current_device(&p->device);
  if (rc) {
    delete p;
    return rc;
  }
  p->nx = nx;
  p->nq = nq;
  p->nflav = nflav;
  p->pids.assign(pids, pids + nflav);
  p->x_lo = x[0];
  p->x_hi = x[nx - 1];
  p->q2_lo = q[0] * q[0];
  p->q2_hi = q[nq - 1] * q[nq - 1];
  std::vector<double> lx(nx), lq(nq), v64(nval);
  p->logq2.resize(nq);
  std::vector<float> v32(nval);
  p->nfp = (nflav + 3) / 4 * 4;
  std::vector<float> v32t(size_t(nq) * nx * p->nfp, 0.0f);
  for (int i = 0; i < nx; ++i) lx[i] = std::log(x[i]);
  for (int j = 0; j < nq; ++j) lq[j] = p->logq2[j] = std::log(q[j] * q[j]);
  // device layout [flavour][Q][x]
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nq; ++j)
      for (int f = 0; f < nflav; ++f) {
        const double v = xf[(size_t(i) * nq + j) * nflav + f];
        v64[(size_t(f) * nq + j) * nx + i] = v;
        v32[(size_t(f) * nq + j) * nx + i] = float(v);
        v32t[(size_t(j) * nx + i) * p->nfp + f] = float(v);
      }
  auto cleanup = [&](int code, const char* what, cudaError_t e) {
    mc_pdf_free(p);
    return fail(code, "mc_pdf_load: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_logx, sizeof(double) * nx)) != cudaSuccess) return cleanup(MC_ENOMEM, "cudaMalloc", e);
  if ((e = cudaMalloc(&p->d_logq2, sizeof(double) * nq)) != cudaSuccess) return cleanup(MC_ENOMEM, "cudaMalloc", e);
  if ((e = cudaMalloc(&p->d_xf64, sizeof(double) * nval)) != cudaSuccess) return cleanup(MC_ENOMEM, "cudaMalloc", e);
  if ((e = cudaMalloc(&p->d_xf32, sizeof(float) * nval)) != cudaSuccess) return cleanup(MC_ENOMEM, "cudaMalloc", e);
  if ((e = cudaMalloc(&p->d_xf32t, sizeof(float) * v32t.size())) != cudaSuccess)
    return cleanup(MC_ENOMEM, "cudaMalloc", e);
  if ((e = cudaMemcpy(p->d_logx, lx.data(), sizeof(double) * nx, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(MC_ECUDA, "cudaMemcpy", e);
  if ((e = cudaMemcpy(p->d_logq2, lq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(MC_ECUDA, "cudaMemcpy", e);
  if ((e = cudaMemcpy(p->d_xf64, v64.data(), sizeof(double) * nval, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(MC_ECUDA, "cudaMemcpy", e);
  if ((e = cudaMemcpy(p->d_xf32, v32.data(), sizeof(float) * nval, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(MC_ECUDA, "cudaMemcpy", e);
  if ((e = cudaMemcpy(p->d_xf32t, v32t.data(), sizeof(float) * v32t.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cleanup(MC_ECUDA, "cudaMemcpy", e);
  *out = p;
  return MC_OK;
}

int mc_pdf_free(mc_pdf p) {
  if (!p) return MC_OK;
  cudaFree(p->d_logx);
  cudaFree(p->d_logq2);
  cudaFree(p->d_xf64);
  cudaFree(p->d_xf32);
  cudaFree(p->d_xf32t);
  delete p;
  return MC_OK;
}

int mc_pdf_xfxq2(mc_pdf p, int prec, int64_t n, const double* x, const double* q2, double* out, void* stream) {
  if (!p) return fail(MC_EINVAL, "mc_pdf_xfxq2: pdf is NULL");
  if (n < 0 || (n > 0 && (!x || !q2 || !out))) return fail(MC_EINVAL, "mc_pdf_xfxq2: bad arguments");
  if (prec != MC_FP64 && prec != MC_FP32_KAHAN) return fail(MC_EINVAL, "mc_pdf_xfxq2: bad precision");
  int dev;
  if (int rc = current_device(&dev)) return rc;
  if (dev != p->device) return fail(MC_EINVAL, "mc_pdf_xfxq2: pdf lives on device %d", p->device);
  MC_CUDA(mc::launch_pdf_xfxq2(p->dev(), prec == MC_FP64, n, x, q2, out, (cudaStream_t)stream));
  return MC_OK;
}

// ---------------------------------------------------------------- VEGAS
int mc_vegas_free(mc_vegas v) {
  if (!v) return MC_OK;
  cudaFree(v->d_edges);
  cudaFree(v->d_edges32);
  cudaFree(v->d_hist_w2);
  cudaFree(v->d_hist_n);
  cudaFree(v->d_partials);
  cudaFree(v->d_total);
  if (v->h_total) cudaFreeHost(v->h_total);
  if (v->k0) cudaEventDestroy(v->k0);
  if (v->k1) cudaEventDestroy(v->k1);
  if (v->d_uw) cudaFree(v->d_uw);
  if (v->d_wch) cudaFree(v->d_wch);
  if (v->h_count) cudaFreeHost(v->h_count);
  if (v->u0) cudaEventDestroy(v->u0);
  if (v->u1) cudaEventDestroy(v->u1);
  delete v;
  return MC_OK;
}

static int upload_grid(mc_vegas v, const double* edges) {
  const size_t ne = size_t(v->ndim) * (v->nbins + 1);
  std::vector<float> e32(ne);
  for (size_t i = 0; i < ne; ++i) e32[i] = float(edges[i]);
  MC_CUDA(cudaMemcpy(v->d_edges, edges, sizeof(double) * ne, cudaMemcpyHostToDevice));
  MC_CUDA(cudaMemcpy(v->d_edges32, e32.data(), sizeof(float) * ne, cudaMemcpyHostToDevice));
  return MC_OK;
}

int mc_vegas_init(int ndim, int nbins, uint64_t seed, int prec, mc_vegas* out) {
  if (!out) return fail(MC_EINVAL, "mc_vegas_init: out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > MC_MAX_DIM) return fail(MC_EINVAL, "mc_vegas_init: ndim %d outside 1..%d", ndim, MC_MAX_DIM);
  if (nbins < 2 || nbins > MC_MAX_BINS)
    return fail(MC_EINVAL, "mc_vegas_init: nbins %d outside 2..%d", nbins, MC_MAX_BINS);
  if (prec != MC_FP64 && prec != MC_FP32_KAHAN) return fail(MC_EINVAL, "mc_vegas_init: bad precision %d", prec);
  auto* v = new mc_vegas_s;
  if (int rc = current_device(&v->device)) {
    delete v;
    return rc;
  }
  v->ndim = ndim;
  v->nbins = nbins;
  v->prec = prec;
  v->seed = seed;
  v->max_partials = num_sms() * 32;
  const size_t ne = size_t(ndim) * (nbins + 1), nh = size_t(ndim) * nbins;
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&v->d_edges, sizeof(double) * ne)) != cudaSuccess ||
      (e = cudaMalloc(&v->d_edges32, sizeof(float) * ne)) != cudaSuccess ||
      (e = cudaMalloc(&v->d_hist_w2, sizeof(double) * nh)) != cudaSuccess ||
      (e = cudaMalloc(&v->d_hist_n, sizeof(unsigned int) * nh)) != cudaSuccess ||
      (e = cudaMalloc(&v->d_partials, sizeof(BlockPartial) * v->max_partials)) != cudaSuccess ||
      (e = cudaMalloc(&v->d_total, kTotalBytes)) != cudaSuccess ||
      (e = cudaMallocHost(&v->h_total, kTotalBytes)) != cudaSuccess ||
      (e = cudaEventCreate(&v->k0)) != cudaSuccess || (e = cudaEventCreate(&v->k1)) != cudaSuccess) {
    mc_vegas_free(v);
    return fail(MC_ENOMEM, "mc_vegas_init: allocation failed: %s", cudaGetErrorString(e));
  }
  std::vector<double> edges(ne);
  for (int d = 0; d < ndim; ++d)
    for (int b = 0; b <= nbins; ++b) edges[size_t(d) * (nbins + 1) + b] = b == nbins ? 1.0 : double(b) / nbins;
  int rc = upload_grid(v, edges.data());
  if (!rc && (e = cudaMemset(v->d_hist_w2, 0, sizeof(double) * nh)) != cudaSuccess)
    rc = fail(MC_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
  if (!rc && (e = cudaMemset(v->d_hist_n, 0, sizeof(unsigned int) * nh)) != cudaSuccess)
    rc = fail(MC_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
  if (rc) {
    mc_vegas_free(v);
    return rc;
  }
  *out = v;
  return MC_OK;
}

int mc_vegas_set_grid(mc_vegas v, const double* edges) {
  if (!v || !edges) return fail(MC_EINVAL, "mc_vegas_set_grid: NULL argument");
  for (int d = 0; d < v->ndim; ++d) {
    const double* e = edges + size_t(d) * (v->nbins + 1);
    if (e[0] != 0.0 || e[v->nbins] != 1.0) return fail(MC_EINVAL, "mc_vegas_set_grid: dim %d not on [0,1]", d);
    for (int b = 1; b <= v->nbins; ++b)
      if (!(e[b] > e[b - 1])) return fail(MC_EINVAL, "mc_vegas_set_grid: dim %d edges not increasing", d);
  }
  MC_CUDA(cudaDeviceSynchronize());
  v->last_valid = false;
  return upload_grid(v, edges);
}

int mc_vegas_get_grid(mc_vegas v, double* edges) {
  if (!v || !edges) return fail(MC_EINVAL, "mc_vegas_get_grid: NULL argument");
  MC_CUDA(cudaDeviceSynchronize());
  MC_CUDA(cudaMemcpy(edges, v->d_edges, sizeof(double) * v->ndim * (v->nbins + 1), cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_vegas_get_hist(mc_vegas v, double* w2, uint32_t* counts) {
  if (!v) return fail(MC_EINVAL, "mc_vegas_get_hist: NULL handle");
  MC_CUDA(cudaDeviceSynchronize());
  const size_t nh = size_t(v->ndim) * v->nbins;
  if (w2) MC_CUDA(cudaMemcpy(w2, v->d_hist_w2, sizeof(double) * nh, cudaMemcpyDeviceToHost));
  if (counts) MC_CUDA(cudaMemcpy(counts, v->d_hist_n, sizeof(uint32_t) * nh, cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_vegas_set_iteration(mc_vegas v, uint32_t it) {
  if (!v) return fail(MC_EINVAL, "mc_vegas_set_iteration: NULL handle");
  v->iteration = it;
  return MC_OK;
}
int mc_vegas_get_iteration(mc_vegas v, uint32_t* it) {
  if (!v || !it) return fail(MC_EINVAL, "mc_vegas_get_iteration: NULL argument");
  *it = v->iteration;
  return MC_OK;
}
int mc_vegas_set_channels(mc_vegas v, const double* alpha) {
  if (!v || !alpha) return fail(MC_EINVAL, "mc_vegas_set_channels: NULL argument");
  const double t = alpha[0] + alpha[1] + alpha[2];
  if (!(alpha[0] >= 0.0 && alpha[1] >= 0.0 && alpha[2] >= 0.0) || !(t > 0.0) || !std::isfinite(t))
    return fail(MC_EINVAL, "mc_vegas_set_channels: alpha must be non-negative with a positive sum");
  for (int i = 0; i < 3; ++i) v->alpha[i] = alpha[i] / t;
  return MC_OK;
}

int mc_vegas_get_channels(mc_vegas v, double* alpha, double* w) {
  if (!v) return fail(MC_EINVAL, "mc_vegas_get_channels: NULL handle");
  for (int i = 0; i < 3; ++i) {
    if (alpha) alpha[i] = v->alpha[i];
    if (w) w[i] = v->wch[i];
  }
  return MC_OK;
}

int mc_channel_update(int n, const double* alpha, const double* w, double beta, double amin, double* out) {
  if (n < 1 || n > 16 || !alpha || !w || !out || !(beta >= 0.0) || !(amin >= 0.0) || !(amin * n < 1.0))
    return fail(MC_EINVAL, "mc_channel_update: bad arguments");
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += (out[i] = alpha[i] * std::pow(w[i], beta));
  if (!(t > 0.0) || !std::isfinite(t)) {
    for (int i = 0; i < n; ++i) out[i] = alpha[i];
    return MC_OK;
  }
  double t2 = 0.0;
  for (int i = 0; i < n; ++i) t2 += (out[i] = std::fmax(out[i] / t, amin));
  for (int i = 0; i < n; ++i) out[i] /= t2;
  return MC_OK;
}

int mc_vegas_set_gid(mc_vegas v, uint32_t gid) {
  if (!v || gid > 255) return fail(MC_EINVAL, "mc_vegas_set_gid: bad argument");
  v->gid = gid;
  return MC_OK;
}

}  // extern "C"

// Validates an integrand and fills the process part of the kernel arguments
// (parameters, PDF tables and flavours, constants); shared with the flow
// sampler (flow.cu).
int mc::fill_process_args(const mc_integrand* itg, mc_pdf pdf, KernelArgs* a) {
  if (!itg) return fail(MC_EINVAL, "NULL integrand");
  if (itg->proc < MC_EE_MUMU || itg->proc > MC_PP_TTBARJ) return fail(MC_EINVAL, "unknown process %d", itg->proc);
  if (itg->proc == MC_GAUSS && process_ndim(itg) < 1)
    return fail(MC_EINVAL, "gauss_dim %d outside 1..16", itg->gauss_dim);
  const bool hadronic = itg->proc == MC_PP_TTBAR || itg->proc == MC_GG_TTBARG || itg->proc == MC_GG_TTBARG_7D ||
                        itg->proc == MC_GG_TTBARG_MC || itg->proc == MC_PP_TTBARJ;
  if ((itg->proc == MC_GG_TTBARG_MC || itg->proc == MC_PP_TTBARJ) && !(itg->ptcut_g > 0.0))
    return fail(MC_EINVAL, "process %d needs ptcut_g > 0", itg->proc);
  if (!(itg->sqrt_s > 0.0) && itg->proc != MC_GAUSS) return fail(MC_EINVAL, "sqrt_s must be positive");
  if (itg->proc == MC_GAUSS && !(itg->gauss_sigma > 0.0)) return fail(MC_EINVAL, "gauss_sigma must be positive");
  int dev;
  if (int rc = current_device(&dev)) return rc;
  std::memset(a, 0, sizeof(*a));
  a->prm = {itg->proc, itg->gauss_dim, itg->sqrt_s, itg->m_top, itg->alpha, itg->alpha_s, itg->mz, itg->gz,
            itg->sw2, itg->mu_f, itg->ptcut_g, itg->etacut_g, itg->gauss_sigma, itg->gev2pb};
  if (hadronic) {
    if (!pdf) return fail(MC_EINVAL, "process %d needs a PDF", itg->proc);
    if (pdf->device != dev) return fail(MC_EINVAL, "pdf lives on device %d", pdf->device);
    const double q = itg->mu_f;
    // mu_F must lie inside the Q range of the grid (no extrapolation on the hot path)
    const double lq = std::log(q * q);
    if (!(lq >= pdf->logq2.front() && lq <= pdf->logq2.back())) return fail(MC_EINVAL, "mu_f outside the PDF grid");
    a->pdf = pdf->dev();
    a->logq2_f = lq;
    const int g = pdf->index(21);
    if (g < 0) return fail(MC_EINVAL, "PDF has no gluon (pid 21)");
    a->fl[0] = g;
    if (itg->proc == MC_PP_TTBARJ) {
      static const std::vector<double> cq = [] {
        std::vector<double> c(50);
        light_line_colour(c.data());
        return c;
      }();
      for (int n = 0; n < 50; ++n) {
        a->cqq[n] = cq[n];
        a->cqqf[n] = float(cq[n]);
      }
    }
    if (itg->proc == MC_PP_TTBAR || itg->proc == MC_PP_TTBARJ)
      for (int qf = 1; qf <= 5; ++qf) {
        a->fl[qf] = pdf->index(qf);
        a->fl[qf + 5] = pdf->index(-qf);
        if (a->fl[qf] < 0 || a->fl[qf + 5] < 0) return fail(MC_EINVAL, "PDF lacks quark flavour %d", qf);
      }
  }
  // three-particle RAMBO coefficient (2 pi)^(4-3n) (pi/2)^(n-1) / (Gamma(n) Gamma(n-1)), n = 3
  a->w0_coef3 = std::pow(2.0 * M_PI, -5.0) * std::pow(M_PI / 2.0, 2.0) / (std::tgamma(3.0) * std::tgamma(2.0));
  a->e2eta = std::exp(2.0 * itg->etacut_g);
  return MC_OK;
}

int mc::process_dim(const mc_integrand* itg) { return process_ndim(itg); }

extern "C" {

// Validates an integrand against a grid and fills the kernel arguments.
static int prepare(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, KernelArgs* a) {
  if (!v || !itg) return fail(MC_EINVAL, "NULL handle or integrand");
  const int nd = process_ndim(itg);
  if (nd < 1) return fail(MC_EINVAL, "process %d: bad dimension (gauss_dim %d)", itg->proc, itg->gauss_dim);
  if (nd != v->ndim) return fail(MC_EINVAL, "process needs %d dimensions, grid has %d", nd, v->ndim);
  int dev;
  if (int rc = current_device(&dev)) return rc;
  if (dev != v->device) return fail(MC_EINVAL, "grid lives on device %d, current device is %d", v->device, dev);
  if (int rc = mc::fill_process_args(itg, pdf, a)) return rc;
  a->ndim = v->ndim;
  a->nbins = v->nbins;
  a->edges64 = v->d_edges;
  a->edges32 = v->d_edges32;
  a->seed = v->seed;
  a->iteration = v->iteration;
  a->gid = v->gid;
  a->hist_w2 = v->d_hist_w2;
  a->hist_n = v->d_hist_n;
  a->partials = v->d_partials;
  // channel probabilities (three-channel process): cumulative sums in the
  // order the channel choice compares them
  for (int i = 0; i < 3; ++i) a->alpha[i] = v->alpha[i];
  a->alpha_cum[0] = v->alpha[0];
  a->alpha_cum[1] = v->alpha[0] + v->alpha[1];
  a->alpha_cum[2] = a->alpha_cum[1] + v->alpha[2];
  if (itg->proc == MC_GG_TTBARG_MC) {
    if (!v->d_wch && cudaMalloc(&v->d_wch, 3 * sizeof(double)) != cudaSuccess)
      return fail(MC_ENOMEM, "channel sums");
    a->wch = v->d_wch;
  }
  return MC_OK;
}

static int launch_grid(int proc, bool fp64, int64_t n, size_t smem, int max_blocks) {
  const int per_sm = mc::integrand_max_blocks_per_sm(proc, fp64, smem);
  long long grid = (long long)num_sms() * per_sm;
  const int per_block = mc::integrand_block_events(proc, fp64);
  const long long need = (n + per_block - 1) / per_block;
  if (grid > need) grid = need;
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  return int(grid);
}

int mc_launch_shape(const mc_integrand* itg, int prec, int64_t nevents, int* blocks, int* threads) {
  if (!itg || !blocks || !threads) return fail(MC_EINVAL, "mc_launch_shape: NULL argument");
  const int nd = process_ndim(itg);
  if (nd < 1) return fail(MC_EINVAL, "mc_launch_shape: bad process");
  const size_t smem = mc::integrand_smem(itg->proc, prec == MC_FP64, nd, 50, 100);
  *blocks = launch_grid(itg->proc, prec == MC_FP64, nevents, smem, num_sms() * 32);
  *threads = mc::integrand_threads(itg->proc, prec == MC_FP64);
  return MC_OK;
}

// One iteration (weights: optional per-event weight output, device).
static int iterate_impl(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, double* weights,
                        void* stream, mc_iter_result* out, int64_t first = 0) {
  if (!out) return fail(MC_EINVAL, "mc_vegas_iterate: out is NULL");
  std::memset(out, 0, sizeof(*out));
  if (nevents < 0) return fail(MC_EINVAL, "mc_vegas_iterate: negative event count");
  if (first < 0 || nevents > INT64_MAX - first) return fail(MC_EINVAL, "mc_vegas_iterate: bad event range");
  KernelArgs a;
  if (int rc = prepare(v, itg, pdf, &a)) return rc;
  a.wout = weights;
  v->last_valid = false;
  const cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = v->prec == MC_FP64;
  out->n = nevents;
  if (nevents > 0) {
    const size_t smem = mc::integrand_smem(itg->proc, fp64, v->ndim, v->nbins, pdf ? pdf->nx : 0);
    const int grid = launch_grid(itg->proc, fp64, nevents, smem, v->max_partials);
    a.first = uint64_t(first);
    a.n = nevents;
    int* d_status = reinterpret_cast<int*>(v->d_total + 1);
    a.status = d_status;
    MC_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    if (a.wch) MC_CUDA(cudaMemsetAsync(a.wch, 0, 3 * sizeof(double), st));
    MC_CUDA(cudaEventRecord(v->k0, st));
    MC_CUDA(mc::launch_integrand(itg->proc, fp64, a, grid, smem, st));
    MC_CUDA(cudaEventRecord(v->k1, st));
    v->timed = true;
    MC_CUDA(mc::launch_finalize(v->d_partials, grid, v->d_total, st));
    MC_CUDA(cudaMemcpyAsync(v->h_total, v->d_total, kTotalBytes, cudaMemcpyDeviceToHost, st));
    MC_CUDA(cudaStreamSynchronize(st));
    if (*reinterpret_cast<const int*>(v->h_total + 1) != 0)
      return fail(MC_ETIMEOUT, "mc_vegas_iterate: a bounded wait inside the integrand kernel gave up");
    const BlockPartial& t = *v->h_total;
    out->sum = t.sum_hi + t.sum_lo;
    out->sum2 = t.sum2_hi + t.sum2_lo;
    out->wmax = t.wmax;
    out->n_nonzero = t.n_nonzero;
    out->n_bad = t.n_bad + t.n_noconv;
    out->status = t.n_bad ? MC_ENAN : (t.n_noconv ? MC_ENOCONV : MC_OK);
    if (a.wch) {
      MC_CUDA(cudaMemcpy(v->wch, a.wch, 3 * sizeof(double), cudaMemcpyDeviceToHost));
      for (int j = 0; j < 3; ++j) v->wch[j] /= double(nevents);
    }
  }
  v->last_iteration = v->iteration;
  v->last_n = nevents;
  v->last_valid = true;
  ++v->iteration;
  return MC_OK;
}

int mc_vegas_iterate(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, void* stream,
                     mc_iter_result* out) {
  return iterate_impl(v, itg, pdf, nevents, nullptr, stream, out);
}

int mc_vegas_iterate_shard(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t count,
                           void* stream, mc_iter_result* out) {
  return iterate_impl(v, itg, pdf, count, nullptr, stream, out, first);
}

int mc_vegas_set_hist(mc_vegas v, const double* w2, const uint32_t* counts) {
  if (!v || !w2 || !counts) return fail(MC_EINVAL, "mc_vegas_set_hist: NULL argument");
  const size_t nh = size_t(v->ndim) * v->nbins;
  for (size_t i = 0; i < nh; ++i)
    if (!(w2[i] >= 0.0) || !std::isfinite(w2[i])) return fail(MC_EINVAL, "mc_vegas_set_hist: bad w2 at %zu", i);
  MC_CUDA(cudaDeviceSynchronize());
  MC_CUDA(cudaMemcpy(v->d_hist_w2, w2, sizeof(double) * nh, cudaMemcpyHostToDevice));
  MC_CUDA(cudaMemcpy(v->d_hist_n, counts, sizeof(uint32_t) * nh, cudaMemcpyHostToDevice));
  return MC_OK;
}

int mc_vegas_iterate_weights(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, double* weights,
                             void* stream, mc_iter_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  if (nevents > 0 && !weights) return fail(MC_EINVAL, "mc_vegas_iterate_weights: weights is NULL");
  if (nevents >= (int64_t(1) << 32)) return fail(MC_EINVAL, "mc_vegas_iterate_weights: nevents >= 2^32");
  return iterate_impl(v, itg, pdf, nevents, weights, stream, out);
}

int mc_unweight(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, const double* weights, int64_t nevents, double wmax,
                mc_event* events, int64_t capacity, int64_t* n_accepted, void* stream) {
  if (!n_accepted) return fail(MC_EINVAL, "mc_unweight: n_accepted is NULL");
  *n_accepted = 0;
  if (!v || !itg) return fail(MC_EINVAL, "mc_unweight: NULL handle or integrand");
  if (itg->proc != MC_EE_MUMU && itg->proc != MC_GG_TTBARG && itg->proc != MC_GG_TTBARG_7D &&
      itg->proc != MC_GG_TTBARG_MC)
    return fail(MC_EINVAL, "mc_unweight: process %d has no event record", itg->proc);
  if (!v->last_valid) return fail(MC_EINVAL, "mc_unweight: no iteration on the current grid");
  if (nevents != v->last_n) return fail(MC_EINVAL, "mc_unweight: nevents differs from the last iteration's");
  if (capacity < 0 || (capacity > 0 && !events) || (nevents > 0 && !weights) || !std::isfinite(wmax))
    return fail(MC_EINVAL, "mc_unweight: bad arguments");
  if (nevents == 0 || !(wmax > 0.0)) return MC_OK;
  KernelArgs a;
  if (int rc = prepare(v, itg, pdf, &a)) return rc;
  a.iteration = v->last_iteration;
  a.first = 0;
  a.n = nevents;
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t need = mc::unweight_scratch_bytes(nevents, capacity);
  if (need > v->uw_bytes) {
    if (v->d_uw) {
      MC_CUDA(cudaStreamSynchronize(st));
      cudaFree(v->d_uw);
      v->d_uw = nullptr;
      v->uw_bytes = 0;
    }
    if (cudaMalloc(&v->d_uw, need) != cudaSuccess) return fail(MC_ENOMEM, "mc_unweight: scratch of %zu bytes", need);
    v->uw_bytes = need;
  }
  if (!v->h_count && cudaMallocHost(&v->h_count, sizeof(unsigned long long)) != cudaSuccess)
    return fail(MC_ENOMEM, "mc_unweight: pinned count");
  if (!v->u0) {
    MC_CUDA(cudaEventCreate(&v->u0));
    MC_CUDA(cudaEventCreate(&v->u1));
  }
  const auto* counts = static_cast<const unsigned long long*>(v->d_uw);
  MC_CUDA(cudaEventRecord(v->u0, st));
  MC_CUDA(mc::unweight_launch(itg->proc, v->prec == MC_FP64, a, weights, wmax, v->d_uw, events, capacity, num_sms(),
                              st));
  MC_CUDA(cudaEventRecord(v->u1, st));
  v->uw_timed = true;
  MC_CUDA(cudaMemcpyAsync(v->h_count, counts + mc::kUwMaxChunks, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          st));
  MC_CUDA(cudaStreamSynchronize(st));
  *n_accepted = int64_t(*v->h_count);
  return MC_OK;
}

int mc_unweight_ms(mc_vegas v, float* ms) {
  if (!v || !ms) return fail(MC_EINVAL, "mc_unweight_ms: NULL argument");
  *ms = 0.0f;
  if (!v->uw_timed) return MC_OK;
  MC_CUDA(cudaEventSynchronize(v->u1));
  MC_CUDA(cudaEventElapsedTime(ms, v->u0, v->u1));
  return MC_OK;
}

int mc_vegas_kernel_ms(mc_vegas v, float* ms) {
  if (!v || !ms) return fail(MC_EINVAL, "mc_vegas_kernel_ms: NULL argument");
  *ms = 0.0f;
  if (!v->timed) return MC_OK;
  MC_CUDA(cudaEventSynchronize(v->k1));
  MC_CUDA(cudaEventElapsedTime(ms, v->k0, v->k1));
  return MC_OK;
}

int mc_vegas_refine(mc_vegas v, double alpha, void* stream) {
  if (!v) return fail(MC_EINVAL, "mc_vegas_refine: NULL handle");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(MC_EINVAL, "mc_vegas_refine: bad alpha");
  v->last_valid = false;
  MC_CUDA(mc::launch_refine(v->d_edges, v->d_edges32, v->d_hist_w2, v->d_hist_n, v->ndim, v->nbins, alpha,
                            (cudaStream_t)stream));
  return MC_OK;
}

int mc_debug_events(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t k, double* out,
                    void* stream) {
  if (k < 0 || first < 0 || (k > 0 && !out)) return fail(MC_EINVAL, "mc_debug_events: bad arguments");
  KernelArgs a;
  if (int rc = prepare(v, itg, pdf, &a)) return rc;
  if (k == 0) return MC_OK;
  const bool fp64 = v->prec == MC_FP64;
  const size_t smem = mc::integrand_smem(itg->proc, fp64, v->ndim, v->nbins, pdf ? pdf->nx : 0);
  a.first = uint64_t(first);
  a.n = k;
  a.record = out;
  const long long grid = (k + mc::kBlock - 1) / mc::kBlock;
  MC_CUDA(mc::launch_integrand_record(itg->proc, fp64, a, int(grid), smem, (cudaStream_t)stream));
  return MC_OK;
}

// Inverse-variance combination and chi^2/dof (thesis eq. vegas-check); an
// iteration with zero variance is left out unless every iteration has zero
// variance.
}  // extern "C"

void mc::combine_iterations(const std::vector<double>& e, const std::vector<double>& s2, mc_result* r) {
  double inv = 0.0, acc = 0.0;
  int used = 0;
  for (size_t i = 0; i < e.size(); ++i)
    if (s2[i] > 0.0) {
      inv += 1.0 / s2[i];
      acc += e[i] / s2[i];
      ++used;
    }
  if (!used) {
    double m = 0.0;
    for (double x : e) m += x;
    r->mean = e.empty() ? 0.0 : m / double(e.size());
    r->sigma = 0.0;
    r->chi2_dof = 0.0;
    return;
  }
  r->mean = acc / inv;
  r->sigma = std::sqrt(1.0 / inv);
  double chi = 0.0;
  for (size_t i = 0; i < e.size(); ++i)
    if (s2[i] > 0.0) chi += (e[i] - r->mean) * (e[i] - r->mean) / s2[i];
  r->chi2_dof = used > 1 ? chi / (used - 1) : 0.0;
}

extern "C" {

static void combine(const std::vector<double>& e, const std::vector<double>& s2, mc_result* r) {
  mc::combine_iterations(e, s2, r);
}

int mc_integrate(const mc_integrand* itg, mc_pdf pdf, int niter, int64_t nevents, int nbins, uint64_t seed,
                 uint32_t gid, int prec, double alpha, double target, void* stream, mc_result* out,
                 mc_iter_result* per_iter) {
  if (!out || !itg) return fail(MC_EINVAL, "mc_integrate: NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (niter < 1 || nevents < 2) return fail(MC_EINVAL, "mc_integrate: need niter >= 1 and nevents >= 2");
  const int nd = process_ndim(itg);
  if (nd < 1 || nd > MC_MAX_DIM) return fail(MC_EINVAL, "mc_integrate: bad process dimension");
  mc_vegas v = nullptr;
  if (int rc = mc_vegas_init(nd, nbins, seed, prec, &v)) return rc;
  if (int rc = mc_vegas_set_gid(v, gid)) {
    mc_vegas_free(v);
    return rc;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<double> es, s2s;
  int rc = MC_OK;
  float total_ms = 0.0f;
  for (int it = 0; it < niter; ++it) {
    mc_iter_result r;
    cudaEventRecord(e0, st);
    rc = mc_vegas_iterate(v, itg, pdf, nevents, stream, &r);
    if (rc) break;
    if (itg->proc == MC_GG_TTBARG_MC) {  // Kleiss-Pittau step of the channel probabilities
      double al[3], w[3], next[3];
      mc_vegas_get_channels(v, al, w);
      mc_channel_update(3, al, w, 0.5, 0.02, next);
      mc_vegas_set_channels(v, next);
    }
    rc = mc_vegas_refine(v, alpha, stream);
    if (rc) break;
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    total_ms += ms;
    if (per_iter) per_iter[it] = r;
    if (r.status && !out->status) out->status = r.status;
    const double n = double(r.n);
    const double mean = r.sum / n;
    es.push_back(mean);
    s2s.push_back((r.sum2 / n - mean * mean) / (n - 1.0));
    combine(es, s2s, out);
    out->n_iter = it + 1;
    if (target > 0.0 && out->mean != 0.0 && out->sigma / std::fabs(out->mean) <= target) break;
  }
  out->gpu_ms = total_ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  mc_vegas_free(v);
  return rc;
}

int mc_gemm_bf16(int M, int N, int K, int bn, int epilogue, const void* a, int lda, const void* b, int ldb,
                 const float* bias, void* c, int ldc, const void* mask, int ld_mask, int splits, int* err,
                 void* stream) {
  if (!a || !b || !c || !err || epilogue < 0 || epilogue > 4 || (epilogue == 2 && !mask))
    return fail(MC_EINVAL, "mc_gemm_bf16: bad arguments");
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.bn = bn;
  g.epilogue = epilogue;
  g.bias = bias;
  g.ldc = ldc;
  if (epilogue == 1 || epilogue >= 3)
    g.c_f32 = static_cast<float*>(c);
  else
    g.c_bf16 = static_cast<__nv_bfloat16*>(c);
  g.mask = static_cast<const __nv_bfloat16*>(mask);
  g.ld_mask = ld_mask;
  g.error = err;
  const cudaError_t e = mc::tc_gemm(g, static_cast<const __nv_bfloat16*>(a), lda, static_cast<const __nv_bfloat16*>(b),
                                    ldb, splits, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(MC_EINVAL, "mc_gemm_bf16: unsupported shape or alignment");
  if (e != cudaSuccess) return fail(MC_ECUDA, "mc_gemm_bf16: %s", cudaGetErrorString(e));
  return MC_OK;
}

int mc_gemm_bf16_tn(int M, int N, int K, int bn, int epilogue, const void* x, int ldx, const void* y, int ldy,
                    float* c, int ldc, int splits, int* err, void* stream) {
  if (!x || !y || !c || !err || (epilogue != 1 && epilogue != 3 && epilogue != 4))
    return fail(MC_EINVAL, "mc_gemm_bf16_tn: bad arguments");
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.bn = bn;
  g.epilogue = epilogue;
  g.c_f32 = c;
  g.ldc = ldc;
  g.error = err;
  const cudaError_t e = mc::tc_gemm_tn(g, static_cast<const __nv_bfloat16*>(x), ldx,
                                       static_cast<const __nv_bfloat16*>(y), ldy, splits,
                                       static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(MC_EINVAL, "mc_gemm_bf16_tn: unsupported shape or alignment");
  if (e != cudaSuccess) return fail(MC_ECUDA, "mc_gemm_bf16_tn: %s", cudaGetErrorString(e));
  return MC_OK;
}

int mc_gemm_bf16_xn(int M, int N, int K, int bn, int epilogue, const void* x, int ldx, const void* b, int ldb,
                    float* c, int ldc, int splits, int* err, void* stream) {
  if (!x || !b || !c || !err || (epilogue != 1 && epilogue != 3 && epilogue != 4))
    return fail(MC_EINVAL, "mc_gemm_bf16_xn: bad arguments");
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.bn = bn;
  g.epilogue = epilogue;
  g.c_f32 = c;
  g.ldc = ldc;
  g.error = err;
  const cudaError_t e = mc::tc_gemm_xn(g, static_cast<const __nv_bfloat16*>(x), ldx,
                                       static_cast<const __nv_bfloat16*>(b), ldb, splits,
                                       static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(MC_EINVAL, "mc_gemm_bf16_xn: unsupported shape or alignment");
  if (e != cudaSuccess) return fail(MC_ECUDA, "mc_gemm_bf16_xn: %s", cudaGetErrorString(e));
  return MC_OK;
}

int mc_gemm_bf16_rs(int M, int N, int K, int bn, int epilogue, const void* a, int lda, const void* b, int ldb,
                    const float* bias, void* c, int ldc, void* c_t, int ldt, const void* mask, int ld_mask, int* err,
                    void* stream) {
  if (!a || !b || (!c && !c_t) || !err || epilogue < 0 || epilogue > 2 || (epilogue == 2 && !mask))
    return fail(MC_EINVAL, "mc_gemm_bf16_rs: bad arguments");
  mc::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.bn = bn;
  g.epilogue = epilogue;
  g.bias = bias;
  g.ldc = ldc;
  g.ldt = ldt;
  if (epilogue == 1) {
    g.c_f32 = static_cast<float*>(c);
    g.c_t_f32 = static_cast<float*>(c_t);
  } else {
    g.c_bf16 = static_cast<__nv_bfloat16*>(c);
    g.c_t_bf16 = static_cast<__nv_bfloat16*>(c_t);
  }
  g.mask = static_cast<const __nv_bfloat16*>(mask);
  g.ld_mask = ld_mask;
  g.error = err;
  const cudaError_t e = mc::tc_gemm_rs(g, static_cast<const __nv_bfloat16*>(a), lda,
                                       static_cast<const __nv_bfloat16*>(b), ldb, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(MC_EINVAL, "mc_gemm_bf16_rs: unsupported shape or alignment");
  if (e != cudaSuccess) return fail(MC_ECUDA, "mc_gemm_bf16_rs: %s", cudaGetErrorString(e));
  return MC_OK;
}

}  // extern "C"
