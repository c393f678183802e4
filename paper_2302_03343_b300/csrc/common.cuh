// Device-side basic types: precision-generic math, complex numbers and
// Lorentz vectors used by every stage of the fused integrand kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MC_HD __host__ __device__ __forceinline__
#define MC_D __device__ __forceinline__

namespace mc {

constexpr double kPi = 3.14159265358979323846;

// Precision-generic scalar helpers (FP32 calls the single-precision CUDA
// math functions, FP64 the double ones).
MC_D float m_sqrt(float x) { return sqrtf(x); }
MC_D double m_sqrt(double x) { return sqrt(x); }
MC_D float m_log(float x) { return logf(x); }
MC_D double m_log(double x) { return log(x); }
MC_D float m_exp(float x) { return expf(x); }
MC_D double m_exp(double x) { return exp(x); }
MC_D float m_abs(float x) { return fabsf(x); }
MC_D double m_abs(double x) { return fabs(x); }
MC_D float m_max(float a, float b) { return fmaxf(a, b); }
MC_D double m_max(double a, double b) { return fmax(a, b); }
MC_D float m_cosh(float x) { return coshf(x); }
MC_D double m_cosh(double x) { return cosh(x); }
MC_D float m_sinh(float x) { return sinhf(x); }
MC_D double m_sinh(double x) { return sinh(x); }
MC_D float m_acosh(float x) { return acoshf(x); }
MC_D double m_acosh(double x) { return acosh(x); }
MC_D float m_atan2(float y, float x) { return atan2f(y, x); }
MC_D double m_atan2(double y, double x) { return atan2(y, x); }
MC_D float m_min(float a, float b) { return fminf(a, b); }
MC_D double m_min(double a, double b) { return fmin(a, b); }
// sin and cos of 2 pi u for u in (0, 1)
MC_D void m_sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
MC_D void m_sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }

template <class R>
struct cx {
  R re, im;
};
template <class R> MC_HD cx<R> mkc(R a, R b) { return {a, b}; }
template <class R> MC_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> MC_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> MC_HD cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R> MC_HD cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> MC_HD cx<R> operator*(cx<R> a, R s) { return {a.re * s, a.im * s}; }
template <class R> MC_HD cx<R> operator*(R s, cx<R> a) { return {a.re * s, a.im * s}; }
template <class R> MC_HD cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <class R> MC_HD R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// a * conj(b)
template <class R> MC_HD cx<R> mul_conj(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}

// Real Lorentz vector (E, px, py, pz), metric (+, -, -, -).
template <class R>
struct v4 {
  R e, x, y, z;
};
template <class R> MC_HD R mdot(const v4<R>& a, const v4<R>& b) {
  return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z;
}
template <class R> MC_HD v4<R> operator+(const v4<R>& a, const v4<R>& b) {
  return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z};
}
template <class R> MC_HD v4<R> operator-(const v4<R>& a, const v4<R>& b) {
  return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z};
}
template <class R> MC_HD v4<R> operator-(const v4<R>& a) { return {-a.e, -a.x, -a.y, -a.z}; }
template <class R> MC_HD v4<R> operator*(const v4<R>& a, R s) { return {a.e * s, a.x * s, a.y * s, a.z * s}; }
template <class T, class R> MC_HD v4<T> vcast(const v4<R>& a) { return {T(a.e), T(a.x), T(a.y), T(a.z)}; }

// Process-independent parameters of one integrand, passed by value.
struct Params {
  int proc, gauss_dim;
  double sqrt_s, m_top, alpha, alpha_s, mz, gz, sw2, mu_f, ptcut_g, etacut_g, gauss_sigma, gev2pb;
};

}  // namespace mc
