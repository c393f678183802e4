// Piecewise-quadratic coupling transform (Mueller et al., "Neural Importance
// Sampling"): per transformed coordinate, K bin widths W = softmax(a) and K+1
// vertex heights V = exp(e) / A with A = sum_k (exp e_k + exp e_{k+1})/2 W_k,
// so that the piecewise-linear density c integrates to one and the CDF C is
// piecewise quadratic.  Forward: y = C(x); inverse: x = C^-1(y) by the stable
// root of the bin's quadratic; backward of the inverse for training.  FP32.
#pragma once
#include "common.cuh"

namespace mc {

constexpr int kFlowMaxBins = 32;

struct SplineCoef {
  float W[kFlowMaxBins], V[kFlowMaxBins + 1];
};

// Widths and normalised heights from the 2K+1 logits of one coordinate.
MC_D void spline_coef(const float* lg, int K, SplineCoef& s) {
  float mx = lg[0];
  for (int k = 1; k < K; ++k) mx = fmaxf(mx, lg[k]);
  float sw = 0.0f;
  for (int k = 0; k < K; ++k) {
    s.W[k] = expf(lg[k] - mx);
    sw += s.W[k];
  }
  const float isw = 1.0f / sw;
  for (int k = 0; k < K; ++k) s.W[k] *= isw;
  for (int k = 0; k <= K; ++k) s.V[k] = expf(lg[K + k]);
  float area = 0.0f;
  for (int k = 0; k < K; ++k) area += 0.5f * (s.V[k] + s.V[k + 1]) * s.W[k];
  const float ia = 1.0f / area;
  for (int k = 0; k <= K; ++k) s.V[k] *= ia;
}

// y = C(x) and log c(x).
MC_D float spline_fwd(const SplineCoef& s, int K, float x, float* logc) {
  float xb = 0.0f, cb = 0.0f;
  int b = 0;
  for (; b < K - 1; ++b) {
    if (x < xb + s.W[b]) break;
    cb += 0.5f * (s.V[b] + s.V[b + 1]) * s.W[b];
    xb += s.W[b];
  }
  const float d = x - xb, dv = s.V[b + 1] - s.V[b];
  const float c = s.V[b] + d / s.W[b] * dv;
  *logc = logf(c);
  return cb + d * s.V[b] + d * d / (2.0f * s.W[b]) * dv;
}

// Bin b, its left edge X_b and CDF C_b for the inverse at y.
MC_D int spline_locate_inv(const SplineCoef& s, int K, float y, float* xb, float* cb) {
  float x0 = 0.0f, c0 = 0.0f;
  int b = 0;
  for (; b < K - 1; ++b) {
    const float seg = 0.5f * (s.V[b] + s.V[b + 1]) * s.W[b];
    if (y < c0 + seg) break;
    c0 += seg;
    x0 += s.W[b];
  }
  *xb = x0;
  *cb = c0;
  return b;
}

// x = C^-1(y) and log c(x).
MC_D float spline_inv(const SplineCoef& s, int K, float y, float* logc) {
  float xb, cb;
  const int b = spline_locate_inv(s, K, y, &xb, &cb);
  const float r = fmaxf(0.0f, (y - cb) / s.W[b]);
  const float dv = s.V[b + 1] - s.V[b];
  const float t = 2.0f * r / (s.V[b] + sqrtf(fmaxf(0.0f, s.V[b] * s.V[b] + 2.0f * dv * r)));
  *logc = logf(s.V[b] + t * dv);
  return xb + t * s.W[b];
}

// Backward of (x, ld) = (C^-1(y), -log c(x)) given gx = dL/dx and gl = dL/dld:
// returns dL/dy and writes dL/d(logits) (2K+1 values) to glog.
// With G = gx - gl c'/c: dL/dy = G/c and dL/dtheta = -(G dC/dtheta + gl dc/dtheta)/c
// at fixed x, chained through the normalisation of V and the softmax of W.
MC_D float spline_inv_bwd(const SplineCoef& s, int K, float y, float gx, float gl, float* glog) {
  float xb, cb;
  const int b = spline_locate_inv(s, K, y, &xb, &cb);
  const float Wb = s.W[b], Vb = s.V[b], Vb1 = s.V[b + 1], dv = Vb1 - Vb;
  const float r = fmaxf(0.0f, (y - cb) / Wb);
  const float t = 2.0f * r / (Vb + sqrtf(fmaxf(0.0f, Vb * Vb + 2.0f * dv * r)));
  const float d = t * Wb;
  const float c = Vb + t * dv;
  const float ic = 1.0f / c;
  const float G = gx - gl * (dv / Wb) * ic;
  const float gy = G * ic;
  float gW[kFlowMaxBins], gV[kFlowMaxBins + 1];
  for (int k = 0; k < K; ++k) gW[k] = 0.0f;
  for (int k = 0; k <= K; ++k) gV[k] = 0.0f;
  for (int k = 0; k < b; ++k) {
    gW[k] = -ic * (G * (0.5f * (s.V[k] + s.V[k + 1]) - c) - gl * dv / Wb);
    gV[k] = -ic * G * 0.5f * ((k > 0 ? s.W[k - 1] : 0.0f) + s.W[k]);
  }
  gW[b] = -ic * (-G * 0.5f * t * t * dv - gl * t * dv / Wb);
  gV[b] = -ic * (G * ((b > 0 ? 0.5f * s.W[b - 1] : 0.0f) + d - d * d / (2.0f * Wb)) + gl * (1.0f - t));
  gV[b + 1] = -ic * (G * d * d / (2.0f * Wb) + gl * t);
  // normalisation V = exp(e) / A: S = sum_j gV_j V_j
  float S = 0.0f;
  for (int k = 0; k <= K; ++k) S += gV[k] * s.V[k];
  for (int k = 0; k < K; ++k) gW[k] -= S * 0.5f * (s.V[k] + s.V[k + 1]);
  for (int k = 0; k <= K; ++k) {
    const float dA = 0.5f * ((k > 0 ? s.W[k - 1] : 0.0f) + (k < K ? s.W[k] : 0.0f));
    glog[K + k] = s.V[k] * (gV[k] - S * dA);
  }
  // softmax of the widths
  float sg = 0.0f;
  for (int k = 0; k < K; ++k) sg += s.W[k] * gW[k];
  for (int k = 0; k < K; ++k) glog[k] = s.W[k] * (gW[k] - sg);
  return gy;
}

}  // namespace mc
