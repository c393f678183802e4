// Oracle: explicit 4x4 Dirac-matrix algebra (Dirac representation).
// TEST INFRASTRUCTURE ONLY (see oracle.h).
#pragma once
#include <array>

#include "oracle.h"

namespace orc {

using Mat4 = std::array<cplx, 16>;  // row-major
using CVec4 = std::array<cplx, 4>;  // contravariant components (E, x, y, z)

inline Mat4 mzero() {
  Mat4 m;
  m.fill(cplx(0.0, 0.0));
  return m;
}
inline Mat4 meye() {
  Mat4 m = mzero();
  for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0;
  return m;
}
inline Mat4 mmul(const Mat4& a, const Mat4& b) {
  Mat4 c = mzero();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      const cplx aik = a[i * 4 + k];
      for (int j = 0; j < 4; ++j) c[i * 4 + j] += aik * b[k * 4 + j];
    }
  return c;
}
inline Mat4 madd(const Mat4& a, const Mat4& b) {
  Mat4 c;
  for (int i = 0; i < 16; ++i) c[i] = a[i] + b[i];
  return c;
}
inline Mat4 mscale(const Mat4& a, cplx s) {
  Mat4 c;
  for (int i = 0; i < 16; ++i) c[i] = a[i] * s;
  return c;
}
inline cplx mtrace(const Mat4& a) { return a[0] + a[5] + a[10] + a[15]; }

// gamma^mu, mu = 0..3, Dirac representation.
inline const std::array<Mat4, 4>& gammas() {
  static const std::array<Mat4, 4> g = [] {
    std::array<Mat4, 4> r;
    for (auto& m : r) m = mzero();
    const cplx I(0.0, 1.0);
    // gamma^0 = diag(1, 1, -1, -1)
    r[0][0] = 1.0; r[0][5] = 1.0; r[0][10] = -1.0; r[0][15] = -1.0;
    // gamma^k = [[0, sigma_k], [-sigma_k, 0]]
    const cplx sig[3][4] = {{0.0, 1.0, 1.0, 0.0}, {0.0, -I, I, 0.0}, {1.0, 0.0, 0.0, -1.0}};
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          r[k + 1][a * 4 + (b + 2)] = sig[k][a * 2 + b];
          r[k + 1][(a + 2) * 4 + b] = -sig[k][a * 2 + b];
        }
    return r;
  }();
  return g;
}

// v-slash = gamma^mu v_mu = gamma^0 v^0 - gamma^k v^k.
inline Mat4 slash(const CVec4& v) {
  const auto& g = gammas();
  Mat4 m = mscale(g[0], v[0]);
  for (int k = 1; k < 4; ++k) m = madd(m, mscale(g[k], -v[k]));
  return m;
}
inline CVec4 cv(const P4& p) { return {p.e, p.x, p.y, p.z}; }
inline Mat4 slash(const P4& p) { return slash(cv(p)); }

// Dirac adjoint bar(G) = gamma^0 G^dagger gamma^0.
inline Mat4 dirac_bar(const Mat4& a) {
  Mat4 h;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) h[i * 4 + j] = std::conj(a[j * 4 + i]);
  const auto& g = gammas();
  return mmul(mmul(g[0], h), g[0]);
}

inline cplx cdot(const CVec4& a, const CVec4& b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
inline CVec4 cadd(const CVec4& a, const CVec4& b) {
  return {a[0] + b[0], a[1] + b[1], a[2] + b[2], a[3] + b[3]};
}
inline CVec4 cscale(const CVec4& a, cplx s) { return {a[0] * s, a[1] * s, a[2] * s, a[3] * s}; }

}  // namespace orc
