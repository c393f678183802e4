// Piecewise-quadratic coupling transform (Mueller et al., "Neural Importance
// Sampling"): per transformed coordinate, K bin widths W = softmax(a) and K+1
// vertex heights V = exp(e) / A with A = sum_k (exp e_k + exp e_{k+1})/2 W_k,
// so that the piecewise-linear density c integrates to one and the CDF C is
// piecewise quadratic.  Forward: y = C(x); inverse: x = C^-1(y) by the stable
// root of the bin's quadratic; backward of the inverse for training.  FP32;
// the 2K+1 exponentials of a coordinate use the hardware exponential
// (__expf: a few ulp for the logits' range, two instructions instead of the
// range-reduced expf) in every path, so the fused and layer-by-layer kernels
// agree bit for bit.
//
// Every loop runs over the compile-time maximum kFlowMaxBins with a K guard
// and every array is indexed with compile-time indices only, so a Spline and
// the gradient arrays live in registers; the bin is selected by predication.
#pragma once
#include "common.cuh"

namespace mc {

constexpr int kFlowMaxBins = 32;

struct Spline {
  float W[kFlowMaxBins], V[kFlowMaxBins + 1];
};

// Widths and normalised heights from the 2K+1 logits of one coordinate,
// logit k at lg[k * ld] (ld = 1 for a contiguous row, n for a transposed
// [logit][event] layout).
MC_D void spline_load(const float* lg, size_t ld, int K, Spline& s) {
  float a[kFlowMaxBins];
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k)
    if (k < K) {
      a[k] = lg[size_t(k) * ld];
      mx = fmaxf(mx, a[k]);
    }
  float sw = 0.0f;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) {
    s.W[k] = k < K ? __expf(a[k] - mx) : 0.0f;
    sw += s.W[k];
  }
  const float isw = 1.0f / sw;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) s.W[k] *= isw;
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) s.V[k] = k <= K ? __expf(lg[size_t(K + k) * ld]) : 0.0f;
  float area = 0.0f;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k)
    if (k < K) area += 0.5f * (s.V[k] + s.V[k + 1]) * s.W[k];
  const float ia = 1.0f / area;
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) s.V[k] *= ia;
}

// The same from logits held in registers (lg[0 .. 2K]), K fixed at compile
// time so that every index is static.
template <int K, int NL>
MC_D void spline_load_regs(const float (&lg)[NL], Spline& s) {
  static_assert(K <= kFlowMaxBins && 2 * K + 1 <= NL, "logit count");
  float mx = lg[0];
#pragma unroll
  for (int k = 1; k < K; ++k) mx = fmaxf(mx, lg[k]);
  float sw = 0.0f;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) {
    s.W[k] = k < K ? __expf(lg[k < K ? k : 0] - mx) : 0.0f;
    sw += s.W[k];
  }
  const float isw = 1.0f / sw;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) s.W[k] *= isw;
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) s.V[k] = k <= K ? __expf(lg[k <= K ? K + k : 0]) : 0.0f;
  float area = 0.0f;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k)
    if (k < K) area += 0.5f * (s.V[k] + s.V[k + 1]) * s.W[k];
  const float ia = 1.0f / area;
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) s.V[k] *= ia;
}

// The bin of a point: Xb, Cb (left edge and CDF there), Wb, Vb, Vb1.  With
// by_cdf the point is a CDF value y (inverse), otherwise a coordinate x.
struct SplineBin {
  int b;
  float Xb, Cb, Wb, Vb, Vb1;
};
MC_D SplineBin spline_bin(const Spline& s, int K, float p, bool by_cdf) {
  SplineBin r = {K - 1, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float xacc = 0.0f, cacc = 0.0f;
  bool found = false;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) {
    if (k < K) {
      const float seg = 0.5f * (s.V[k] + s.V[k + 1]) * s.W[k];
      const bool take = !found && (k == K - 1 || (by_cdf ? p < cacc + seg : p < xacc + s.W[k]));
      if (take) {
        r.b = k;
        r.Xb = xacc;
        r.Cb = cacc;
        r.Wb = s.W[k];
        r.Vb = s.V[k];
        r.Vb1 = s.V[k + 1];
        found = true;
      }
      xacc += s.W[k];
      cacc += seg;
    }
  }
  return r;
}

// y = C(x) and log c(x).
MC_D float spline_fwd(const Spline& s, int K, float x, float* logc) {
  const SplineBin q = spline_bin(s, K, x, false);
  const float d = x - q.Xb, dv = q.Vb1 - q.Vb;
  *logc = logf(q.Vb + d / q.Wb * dv);
  return q.Cb + d * q.Vb + d * d / (2.0f * q.Wb) * dv;
}

// x = C^-1(y) and log c(x).
MC_D float spline_inv(const Spline& s, int K, float y, float* logc) {
  const SplineBin q = spline_bin(s, K, y, true);
  const float r = fmaxf(0.0f, (y - q.Cb) / q.Wb);
  const float dv = q.Vb1 - q.Vb;
  const float t = 2.0f * r / (q.Vb + sqrtf(fmaxf(0.0f, q.Vb * q.Vb + 2.0f * dv * r)));
  *logc = logf(q.Vb + t * dv);
  return q.Xb + t * q.Wb;
}

// Backward of (x, ld) = (C^-1(y), -log c(x)) given gx = dL/dx and gl = dL/dld:
// returns dL/dy and writes dL/d(width logits) to gw[0..K) and dL/d(height
// logits) to gv[0..K].  With G = gx - gl c'/c: dL/dy = G/c and
// dL/dtheta = -(G dC/dtheta + gl dc/dtheta)/c at fixed x, chained through the
// normalisation of V and the softmax of W.
MC_D float spline_inv_bwd(const Spline& s, int K, float y, float gx, float gl, float (&gw)[kFlowMaxBins],
                          float (&gv)[kFlowMaxBins + 1]) {
  const SplineBin q = spline_bin(s, K, y, true);
  const int b = q.b;
  const float Wb = q.Wb, Vb = q.Vb, dv = q.Vb1 - q.Vb;
  const float r = fmaxf(0.0f, (y - q.Cb) / Wb);
  const float t = 2.0f * r / (Vb + sqrtf(fmaxf(0.0f, Vb * Vb + 2.0f * dv * r)));
  const float d = t * Wb;
  const float c = Vb + t * dv;
  const float ic = 1.0f / c;
  const float G = gx - gl * (dv / Wb) * ic;
  const float gy = G * ic;
  // derivatives at fixed normalisation: bins left of b move the edge and the
  // CDF offset; bin b enters through its width and its two vertex heights
  const float gW_left = gl * dv / Wb;
  const float gW_b = -ic * (-G * 0.5f * t * t * dv - gl * t * dv / Wb);
  const float gVb_in = G * (d - d * d / (2.0f * Wb)) + gl * (1.0f - t);
  const float gVb1 = -ic * (G * d * d / (2.0f * Wb) + gl * t);
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) {
    const float wl = k > 0 ? s.W[k - 1] : 0.0f;
    if (k < b) {
      gw[k] = -ic * (G * (0.5f * (s.V[k] + s.V[k + 1]) - c) - gW_left);
      gv[k] = -ic * G * 0.5f * (wl + s.W[k]);
    } else if (k == b) {
      gw[k] = gW_b;
      gv[k] = -ic * (G * 0.5f * wl + gVb_in);
    } else {
      gw[k] = 0.0f;
      gv[k] = k == b + 1 ? gVb1 : 0.0f;
    }
  }
  gv[kFlowMaxBins] = kFlowMaxBins == b + 1 ? gVb1 : 0.0f;
  // normalisation V = exp(e) / A: S = sum_j gV_j V_j
  float S = 0.0f;
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) S += gv[k] * s.V[k];
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) gw[k] -= S * 0.5f * (s.V[k] + s.V[k + 1]);
#pragma unroll
  for (int k = 0; k <= kFlowMaxBins; ++k) {
    const float dA = 0.5f * ((k > 0 ? s.W[k - 1] : 0.0f) + (k < kFlowMaxBins ? s.W[k] : 0.0f));
    gv[k] = s.V[k] * (gv[k] - S * dA);
  }
  // softmax of the widths
  float sg = 0.0f;
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) sg += s.W[k] * gw[k];
#pragma unroll
  for (int k = 0; k < kFlowMaxBins; ++k) gw[k] = s.W[k] * (gw[k] - sg);
  return gy;
}

}  // namespace mc
