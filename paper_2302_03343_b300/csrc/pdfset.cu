// PDF sets with sub-grids, members and extrapolation, and alpha_s(Q)
// interpolation, on the GPU (C ABI: mc_pdfset_*, mc_alphas_* in
// include/mcint.h).
//
// Thesis Sec. "LHAPDF: the Les Houches Accord PDF" and Sec. "PDFFlow:
// interpolating PDFs on GPUs" (multi-member evaluation: Table tab:fktable).
// A set holds nsub sub-grids that cover adjacent Q ranges (the threshold
// knot is shared; a query exactly on it belongs to the upper sub-grid) and
// nmem members on the same knots.  Inside a sub-grid x f is a cubic Hermite
// spline in log x and then in log Q^2 (knot slopes the mean of the adjacent
// divided differences, one-sided at the sub-grid's ends), bilinear in
// (log x, log Q^2) where the sub-grid has fewer than 4 knots in a direction.
// Outside: below x_min and above Q_max, linear continuation in log x (log Q^2)
// from the two edge knots, of log(x f) when both values exceed 1e-3 and of
// x f otherwise; below Q_min, x f(Q^2_min) (Q^2/Q^2_min)^(gamma r + 1 - r) with
// r = Q^2/Q^2_min and gamma = d ln(x f)/d ln Q^2 from the two lowest Q knots
// (1 when either value is not positive); x rules first when both are out.
// x above x_max, x <= 0 or Q^2 <= 0 give NaN.
//
// Device layout: values [member][sub-grid][flavour][Q][x] (x contiguous), in
// FP64 and FP32; knots as log x and log Q^2 per sub-grid.  In the kernel
// the weights of each query point are formed once per point (the bicubic
// spline is linear in the stored values: weights w_Q x w_x over a 4 x 4
// stencil); then each output (member, point, flavour) is 16 loads and 16 FMAs
// plus the continuation rules, and [member][point][flavour] is written
// contiguously through shared memory.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mcint.h"
#include "common.cuh"
#include "handles.h"

namespace mc {
namespace {

constexpr int kMaxSub = 8;
constexpr int kMaxFlav = 16;

struct SubInfo {
  int nx, nq;
  int kx, kq;     // offsets of this sub-grid's knots in the knot arrays
  long long off;  // offset of this sub-grid's block in a member's values
};

struct SetDev {
  int nsub, nflav, nmem;
  long long msize;  // values per member
  SubInfo sub[kMaxSub];
  const double* lx64;
  const double* lq64;
  const float* lx32;
  const float* lq32;
  const double* v64;
  const float* v32;
};

template <class R> MC_D const R* knots_x(const SetDev& s);
template <class R> MC_D const R* knots_q(const SetDev& s);
template <class R> MC_D const R* values(const SetDev& s);
template <> MC_D const double* knots_x<double>(const SetDev& s) { return s.lx64; }
template <> MC_D const float* knots_x<float>(const SetDev& s) { return s.lx32; }
template <> MC_D const double* knots_q<double>(const SetDev& s) { return s.lq64; }
template <> MC_D const float* knots_q<float>(const SetDev& s) { return s.lq32; }
template <> MC_D const double* values<double>(const SetDev& s) { return s.v64; }
template <> MC_D const float* values<float>(const SetDev& s) { return s.v32; }

// largest c in [0, n-2] with t[c] <= v
template <class R>
MC_D int cell_of(const R* t, int n, R v) {
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

template <class R>
MC_D R herm(R tau, R h, R f0, R f1, R d0, R d1) {
  const R t2 = tau * tau, t3 = t2 * tau;
  return (R(2) * t3 - R(3) * t2 + R(1)) * f0 + (t3 - R(2) * t2 + tau) * h * d0 + (R(3) * t2 - R(2) * t3) * f1 +
         (t3 - t2) * h * d1;
}

// Cubic Hermite on the cell [k, k+1] of n knots t[] with values f(k-1..k+2)
// given as g[0..3] (g[0] unused when k == 0, g[3] when k + 1 == n - 1).
template <class R>
MC_D R herm_cell(const R* t, int n, int k, const R* g, R u) {
  const R h = t[k + 1] - t[k];
  const R dd = (g[2] - g[1]) / h;
  const R d0 = k == 0 ? dd : R(0.5) * (dd + (g[1] - g[0]) / (t[k] - t[k - 1]));
  const R d1 = k + 1 == n - 1 ? dd : R(0.5) * (dd + (g[3] - g[2]) / (t[k + 2] - t[k + 1]));
  return herm((u - t[k]) / h, h, g[1], g[2], d0, d1);
}

// The Hermite spline on cell k with divided-difference slopes is linear in
// the values at knots k-1 .. k+2: w[0..3] with f(u) = sum_b w[b] g[b].
// Bilinear (w = (0, 1 - tau, tau, 0)) for fewer than 4 knots.
template <class R>
MC_D void herm_weights(const R* t, int n, int k, R u, bool linear, R* w) {
  const R h = t[k + 1] - t[k];
  const R tau = (u - t[k]) / h;
  if (linear) {
    w[0] = R(0);
    w[1] = R(1) - tau;
    w[2] = tau;
    w[3] = R(0);
    return;
  }
  const R t2 = tau * tau, t3 = t2 * tau;
  const R h00 = R(2) * t3 - R(3) * t2 + R(1), h10 = t3 - R(2) * t2 + tau, h01 = R(3) * t2 - R(2) * t3,
          h11 = t3 - t2;
  // slope at k: a0 dd + b0 (g1 - g0)/hl, at k+1: a1 dd + b1 (g3 - g2)/hr, dd = (g2 - g1)/h
  const bool left = k > 0, right = k + 1 < n - 1;
  const R a0 = left ? R(0.5) : R(1), a1 = right ? R(0.5) : R(1);
  const R c0 = left ? R(0.5) * h * h10 / (t[k] - t[k - 1]) : R(0);
  const R c3 = right ? R(0.5) * h * h11 / (t[k + 2] - t[k + 1]) : R(0);
  w[0] = -c0;
  w[1] = h00 - a0 * h10 + c0 - a1 * h11;
  w[2] = h01 + a0 * h10 + a1 * h11 - c3;
  w[3] = c3;
}

// What one query point needs from the set, computed once per point: the
// sub-grid, the 4 x 4 stencil origin, the x weights of up to two x positions
// (the point, or the two lowest x knots below x_min) and the Q weights of up
// to two Q positions (the point, or the two edge knots outside [Q_min, Q_max]),
// and the parameters of the continuation rules.
enum : int { kQInside = 0, kQHigh = 1, kQLow = 2 };
template <class R>
struct PointW {
  bool nan, xlow;
  int qmode, s, ix, iq;
  R wx[2][4], wq[2][4];
  R ux, uq;      // continuation coordinates (u = (t - t0) / (t1 - t0))
  R lnr, r, dq;  // low Q: ln(Q^2 / Q^2_min), Q^2 / Q^2_min, t1 - t0
};

template <class R>
MC_D PointW<R> point_weights(const SetDev& S, double x, double q2) {
  PointW<R> P;
  P.nan = !(x > 0.0) || !(q2 > 0.0);
  P.xlow = false;
  P.qmode = kQInside;
  P.s = 0;
  P.ix = P.iq = 0;
  P.ux = P.uq = P.lnr = P.r = P.dq = R(0);
  if (P.nan) return P;
  // FP32 mode takes the logarithms of the FP32-rounded inputs (an FP64 log
  // costs about 64 FP32 ones on B300)
  const R lx = sizeof(R) == 4 ? R(logf(float(x))) : R(log(x));
  const R lq = sizeof(R) == 4 ? R(logf(float(q2))) : R(log(q2));
  const SubInfo& first = S.sub[0];
  const SubInfo& last = S.sub[S.nsub - 1];
  const R* q0 = knots_q<R>(S) + first.kq;
  const R* qn = knots_q<R>(S) + last.kq;
  if (lx > knots_x<R>(S)[first.kx + first.nx - 1]) {
    P.nan = true;
    return P;
  }
  if (lq > qn[last.nq - 1]) {
    P.qmode = kQHigh;
    P.s = S.nsub - 1;
  } else if (lq < q0[0]) {
    P.qmode = kQLow;
    P.s = 0;
  } else {
    int s = 0;
    while (s + 1 < S.nsub && !(lq < knots_q<R>(S)[S.sub[s].kq + S.sub[s].nq - 1])) ++s;
    P.s = s;
  }
  const SubInfo& g = S.sub[P.s];
  const R* tx = knots_x<R>(S) + g.kx;
  const R* tq = knots_q<R>(S) + g.kq;
  const bool linear = g.nx < 4 || g.nq < 4;
  if (P.qmode == kQInside) {
    P.iq = cell_of(tq, g.nq, lq);
    herm_weights(tq, g.nq, P.iq, lq, linear, P.wq[0]);
  } else {
    P.iq = P.qmode == kQHigh ? g.nq - 2 : 0;
    const R t0 = tq[P.iq], t1 = tq[P.iq + 1];
    herm_weights(tq, g.nq, P.iq, t0, linear, P.wq[0]);
    herm_weights(tq, g.nq, P.iq, t1, linear, P.wq[1]);
    P.uq = (lq - t0) / (t1 - t0);
    P.lnr = lq - t0;
    P.r = m_exp(P.lnr);
    P.dq = t1 - t0;
  }
  if (lx >= tx[0]) {
    P.ix = cell_of(tx, g.nx, lx);
    herm_weights(tx, g.nx, P.ix, lx, linear, P.wx[0]);
  } else {
    P.xlow = true;
    P.ix = 0;
    herm_weights(tx, g.nx, 0, tx[0], linear, P.wx[0]);
    herm_weights(tx, g.nx, 0, tx[1], linear, P.wx[1]);
    P.ux = (lx - tx[0]) / (tx[1] - tx[0]);
  }
  return P;
}

template <class R>
MC_D R cont(R u, R f0, R f1) {
  if (f0 > R(1e-3) && f1 > R(1e-3)) return m_exp(m_log(f0) + u * (m_log(f1) - m_log(f0)));
  return f0 + u * (f1 - f0);
}

// x f of member m, flavour fl at the point described by P; rows[a] and
// cols[b] are the clamped element offsets of the 4 x 4 stencil inside a
// (member, flavour) block of sub-grid P.s, base that block's first value.
template <class R>
MC_D R point_value(const PointW<R>& P, const R* base, const int* rows, const int* cols) {
  R st[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) st[a][b] = base[rows[a] + cols[b]];
  auto F = [&](int xs, int qs) {
    R acc = R(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      R row = R(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) row += P.wx[xs][b] * st[a][b];
      acc += P.wq[qs][a] * row;
    }
    return acc;
  };
  auto X = [&](int qs) { return P.xlow ? cont(P.ux, F(0, qs), F(1, qs)) : F(0, qs); };
  if (P.qmode == kQInside) return X(0);
  const R f0 = X(0), f1 = X(1);
  if (P.qmode == kQHigh) return cont(P.uq, f0, f1);
  const R gamma = (f0 > R(0) && f1 > R(0)) ? m_log(f1 / f0) / P.dq : R(1);
  return f0 * m_exp((gamma * P.r + R(1) - P.r) * P.lnr);
}

// Block: 32 points (lane) x all flavours (warp = flavour), for a chunk of
// kMembersPerBlock members.  Warp 0 forms the 32 points' weights once into
// shared memory; then every round produces kMembersPerRound members' 32 x
// nflav outputs, staged in shared memory and written as contiguous runs of
// out[m][p0 .. p0+31][flavour].
constexpr int kMembersPerBlock = 32;
constexpr int kMembersPerRound = 8;

template <class R>
__global__ void __launch_bounds__(32 * kMaxFlav, 2)
    pdfset_kernel(SetDev S, int m0, int nm, long long n, const double* x, const double* q2, R* out) {
  __shared__ PointW<R> pts[32];
  __shared__ R tile[kMembersPerRound][32 * kMaxFlav];
  const int lane = threadIdx.x & 31, fl = threadIdx.x >> 5;
  const int nfl = S.nflav;
  const long long p0 = (long long)blockIdx.x * 32, p = p0 + lane;
  const int np = int(min(32LL, n - p0));
  if (fl == 0 && p < n) pts[lane] = point_weights<R>(S, x[p], q2[p]);
  __syncthreads();
  PointW<R> P;
  int rows[4], cols[4];
  long long off = 0;
  if (p < n) {
    P = pts[lane];
    const SubInfo& g = S.sub[P.s];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      rows[a] = min(max(P.iq - 1 + a, 0), g.nq - 1) * g.nx;
      cols[a] = min(max(P.ix - 1 + a, 0), g.nx - 1);
    }
    off = g.off + (long long)fl * g.nq * g.nx;
  }
  const int mb = int(blockIdx.y) * kMembersPerBlock;
  const int me = min(nm, mb + kMembersPerBlock);
  for (int mr = mb; mr < me; mr += kMembersPerRound) {
    const int nr = min(kMembersPerRound, me - mr);
    if (p < n) {
#pragma unroll
      for (int k = 0; k < kMembersPerRound; ++k) {
        if (k < nr) {
          const R* base = values<R>(S) + (long long)(m0 + mr + k) * S.msize + off;
          tile[k][lane * nfl + fl] =
              P.nan ? R(__longlong_as_double(0x7ff8000000000000LL)) : point_value<R>(P, base, rows, cols);
        }
      }
    }
    __syncthreads();
    for (int k = 0; k < nr; ++k) {
      R* o = out + ((long long)(mr + k) * n + p0) * nfl;
      for (int e = threadIdx.x; e < np * nfl; e += blockDim.x) o[e] = tile[k][e];
    }
    __syncthreads();
  }
}

struct AlphasDev {
  int n;
  const double* lq;  // log Q^2 knots [n]
  const double* a;   // values [n]
};

__global__ void alphas_kernel(AlphasDev A, long long n, const double* q2, double* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = q2[i];
    if (!(v > 0.0)) {
      out[i] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const double lq = log(v);
    const int k = A.n;
    if (lq >= A.lq[k - 1]) {
      out[i] = A.a[k - 1];
      continue;
    }
    if (lq < A.lq[0]) {
      out[i] = exp(log(A.a[0]) + (lq - A.lq[0]) / (A.lq[1] - A.lq[0]) * (log(A.a[1]) - log(A.a[0])));
      continue;
    }
    // the segment between repeated knots that holds lq (the upper one at a threshold)
    int b = 0;
    for (int j = 1; j < k; ++j)
      if (A.lq[j] == A.lq[j - 1] && lq >= A.lq[j]) b = j;
    int e = b + 1;
    while (e < k && A.lq[e] != A.lq[e - 1]) ++e;
    const int c = b + cell_of(A.lq + b, e - b, lq);
    double g[4];
    for (int t = 0; t < 4; ++t) {
      const int j = c - 1 + t;
      g[t] = (j >= b && j < e) ? A.a[j] : 0.0;
    }
    out[i] = herm_cell(A.lq + b, e - b, c - b, g, lq);
  }
}

}  // namespace
}  // namespace mc

struct mc_pdfset_s {
  int device = 0;
  mc::SetDev dev{};
  double xmax = 1.0;
  void* mem = nullptr;  // one allocation for knots and values
};

struct mc_alphas_s {
  int device = 0;
  mc::AlphasDev dev{};
  void* mem = nullptr;
};

namespace {

int pfail(int code, const char* msg) {
  mc::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" {

int mc_pdfset_load(int nsub, const int* nx, const int* nq, const double* x, const double* q, int nflav,
                   const int* pids, int nmem, const double* xf, mc_pdfset* out) {
  if (!out) return pfail(MC_EINVAL, "mc_pdfset_load: out is NULL");
  *out = nullptr;
  if (nsub < 1 || nsub > mc::kMaxSub || !nx || !nq || !x || !q || !xf || !pids)
    return pfail(MC_EINVAL, "mc_pdfset_load: need 1..8 sub-grids and non-NULL arrays");
  if (nflav < 1 || nflav > mc::kMaxFlav || nmem < 1) return pfail(MC_EINVAL, "mc_pdfset_load: bad flavour or member count");
  long long tx = 0, tq = 0, msize = 0;
  for (int s = 0; s < nsub; ++s) {
    if (nx[s] < 2 || nq[s] < 2) return pfail(MC_EINVAL, "mc_pdfset_load: a sub-grid needs 2 knots in each direction");
    for (int i = 0; i < nx[s]; ++i)
      if (!(x[tx + i] > 0.0) || (i && !(x[tx + i] > x[tx + i - 1])))
        return pfail(MC_EINVAL, "mc_pdfset_load: x knots must be positive and increasing");
    for (int j = 0; j < nq[s]; ++j)
      if (!(q[tq + j] > 0.0) || (j && !(q[tq + j] > q[tq + j - 1])))
        return pfail(MC_EINVAL, "mc_pdfset_load: Q knots must be positive and increasing");
    if (s && q[tq] != q[tq - 1]) return pfail(MC_EINVAL, "mc_pdfset_load: adjacent sub-grids must share their threshold knot");
    tx += nx[s];
    tq += nq[s];
    msize += (long long)nx[s] * nq[s] * nflav;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return pfail(MC_ECUDA, "mc_pdfset_load: no device");
  // host images: log knots (FP64, FP32), values reordered to [member][sub][flav][q][x]
  std::vector<double> lx(tx), lq(tq);
  std::vector<float> lx32(tx), lq32(tq);
  for (long long i = 0; i < tx; ++i) {
    lx[i] = std::log(x[i]);
    lx32[i] = float(lx[i]);
  }
  for (long long j = 0; j < tq; ++j) {
    lq[j] = std::log(q[j] * q[j]);
    lq32[j] = float(lq[j]);
  }
  std::vector<double> v((size_t)(msize * nmem));
  mc::SetDev d{};
  d.nsub = nsub;
  d.nflav = nflav;
  d.nmem = nmem;
  d.msize = msize;
  {
    long long kx = 0, kq = 0, off = 0;
    for (int s = 0; s < nsub; ++s) {
      d.sub[s] = {nx[s], nq[s], int(kx), int(kq), off};
      for (int m = 0; m < nmem; ++m)
        for (int i = 0; i < nx[s]; ++i)
          for (int j = 0; j < nq[s]; ++j)
            for (int f = 0; f < nflav; ++f)
              v[size_t(m * msize + off + ((long long)f * nq[s] + j) * nx[s] + i)] =
                  xf[size_t(m * msize + off + ((long long)i * nq[s] + j) * nflav + f)];
      kx += nx[s];
      kq += nq[s];
      off += (long long)nx[s] * nq[s] * nflav;
    }
  }
  const size_t b_l64 = sizeof(double) * size_t(tx + tq), b_l32 = sizeof(float) * size_t(tx + tq);
  const size_t b_v64 = sizeof(double) * v.size(), b_v32 = sizeof(float) * v.size();
  auto up16 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t total = up16(b_l64) + up16(b_l32) + up16(b_v64) + up16(b_v32);
  void* mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) return pfail(MC_ENOMEM, "mc_pdfset_load: device allocation failed");
  char* p = static_cast<char*>(mem);
  double* d_l64 = reinterpret_cast<double*>(p);
  float* d_l32 = reinterpret_cast<float*>(p + up16(b_l64));
  double* d_v64 = reinterpret_cast<double*>(p + up16(b_l64) + up16(b_l32));
  float* d_v32 = reinterpret_cast<float*>(p + up16(b_l64) + up16(b_l32) + up16(b_v64));
  std::vector<double> l64(lx);
  l64.insert(l64.end(), lq.begin(), lq.end());
  std::vector<float> l32(lx32);
  l32.insert(l32.end(), lq32.begin(), lq32.end());
  std::vector<float> v32(v.begin(), v.end());
  if (cudaMemcpy(d_l64, l64.data(), b_l64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_l32, l32.data(), b_l32, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_v64, v.data(), b_v64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_v32, v32.data(), b_v32, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return pfail(MC_ECUDA, "mc_pdfset_load: upload failed");
  }
  d.lx64 = d_l64;
  d.lq64 = d_l64 + tx;
  d.lx32 = d_l32;
  d.lq32 = d_l32 + tx;
  d.v64 = d_v64;
  d.v32 = d_v32;
  auto* h = new mc_pdfset_s;
  h->device = dev;
  h->dev = d;
  h->mem = mem;
  (void)pids;  // the output follows the flavour order given here
  *out = h;
  return MC_OK;
}

int mc_pdfset_free(mc_pdfset s) {
  if (!s) return MC_OK;
  cudaFree(s->mem);
  delete s;
  return MC_OK;
}

int mc_pdfset_xfxq2(mc_pdfset s, int prec, int member0, int nmem, int64_t n, const double* x, const double* q2,
                    void* out, void* stream) {
  if (!s) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: NULL handle");
  if (prec != MC_FP64 && prec != MC_FP32_KAHAN) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: bad precision");
  if (member0 < 0 || nmem < 1 || member0 + nmem > s->dev.nmem) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: bad member range");
  if (n < 0 || (n > 0 && (!x || !q2 || !out))) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: bad arguments");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: set lives on another device");
  if (n == 0) return MC_OK;
  const long long tiles = (n + 31) / 32;
  if (tiles > 0x7fffffffLL) return pfail(MC_EINVAL, "mc_pdfset_xfxq2: too many points for one launch");
  const dim3 grid(unsigned(tiles), unsigned((nmem + mc::kMembersPerBlock - 1) / mc::kMembersPerBlock));
  const int block = 32 * s->dev.nflav;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // half of the unified L1/shared memory as shared memory, so that several
  // blocks (up to 5 of 11 warps) are resident per SM; left to itself the
  // runtime picks a carveout that holds one
  (void)cudaGetLastError();
  if (cudaFuncSetAttribute(mc::pdfset_kernel<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 50) !=
          cudaSuccess ||
      cudaFuncSetAttribute(mc::pdfset_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 50) != cudaSuccess)
    return pfail(MC_ECUDA, "mc_pdfset_xfxq2: kernel attribute");
  if (prec == MC_FP64)
    mc::pdfset_kernel<double><<<grid, block, 0, st>>>(s->dev, member0, nmem, n, x, q2, static_cast<double*>(out));
  else
    mc::pdfset_kernel<float><<<grid, block, 0, st>>>(s->dev, member0, nmem, n, x, q2, static_cast<float*>(out));
  if (cudaGetLastError() != cudaSuccess) return pfail(MC_ECUDA, "mc_pdfset_xfxq2: launch failed");
  return MC_OK;
}

int mc_alphas_load(int n, const double* q, const double* alphas, mc_alphas* out) {
  if (!out) return pfail(MC_EINVAL, "mc_alphas_load: out is NULL");
  *out = nullptr;
  if (n < 2 || !q || !alphas) return pfail(MC_EINVAL, "mc_alphas_load: need at least 2 knots");
  for (int i = 0; i < n; ++i) {
    if (!(q[i] > 0.0) || !(alphas[i] > 0.0)) return pfail(MC_EINVAL, "mc_alphas_load: knots and values must be positive");
    if (i && !(q[i] >= q[i - 1])) return pfail(MC_EINVAL, "mc_alphas_load: Q knots must not decrease");
    if (i >= 2 && q[i] == q[i - 1] && q[i - 1] == q[i - 2]) return pfail(MC_EINVAL, "mc_alphas_load: a knot repeats more than twice");
  }
  if (q[1] == q[0] || q[n - 1] == q[n - 2]) return pfail(MC_EINVAL, "mc_alphas_load: the first and last segments need 2 knots");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return pfail(MC_ECUDA, "mc_alphas_load: no device");
  std::vector<double> h(2 * size_t(n));
  for (int i = 0; i < n; ++i) {
    h[i] = std::log(q[i] * q[i]);
    h[n + i] = alphas[i];
  }
  void* mem = nullptr;
  if (cudaMalloc(&mem, sizeof(double) * h.size()) != cudaSuccess) return pfail(MC_ENOMEM, "mc_alphas_load: allocation failed");
  if (cudaMemcpy(mem, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return pfail(MC_ECUDA, "mc_alphas_load: upload failed");
  }
  auto* a = new mc_alphas_s;
  a->device = dev;
  a->dev = {n, static_cast<double*>(mem), static_cast<double*>(mem) + n};
  a->mem = mem;
  *out = a;
  return MC_OK;
}

int mc_alphas_free(mc_alphas a) {
  if (!a) return MC_OK;
  cudaFree(a->mem);
  delete a;
  return MC_OK;
}

int mc_alphas_q2(mc_alphas a, int64_t n, const double* q2, double* out, void* stream) {
  if (!a) return pfail(MC_EINVAL, "mc_alphas_q2: NULL handle");
  if (n < 0 || (n > 0 && (!q2 || !out))) return pfail(MC_EINVAL, "mc_alphas_q2: bad arguments");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != a->device) return pfail(MC_EINVAL, "mc_alphas_q2: knots live on another device");
  if (n == 0) return MC_OK;
  const long long blocks = (n + 255) / 256;
  (void)cudaGetLastError();
  mc::alphas_kernel<<<int(blocks < 148 * 16 ? blocks : 148 * 16), 256, 0, static_cast<cudaStream_t>(stream)>>>(a->dev, n,
                                                                                                           q2, out);
  if (cudaGetLastError() != cudaSuccess) return pfail(MC_ECUDA, "mc_alphas_q2: launch failed");
  return MC_OK;
}

}  // extern "C"
