// Packed FP32x2 arithmetic (PTX add/sub/mul/fma .f32x2, sm_100 and later):
// one instruction operates on a pair of floats held in a 64-bit register
// pair.  A complex number is stored as the pair (re, im); complex products
// use the swapped pair (im, re) and broadcast scalars (s, s).
#pragma once
#include "common.cuh"

namespace mc {

struct f2 {
  unsigned long long v;
};
MC_D f2 pk2(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
MC_D f2 bc2(float s) { return pk2(s, s); }
MC_D float lo2(f2 a) {
  float l;
  asm("mov.b64 {%0, _}, %1;" : "=f"(l) : "l"(a.v));
  return l;
}
MC_D float hi2(f2 a) {
  float h;
  asm("mov.b64 {_, %0}, %1;" : "=f"(h) : "l"(a.v));
  return h;
}
MC_D f2 swp2(f2 a) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
  return pk2(h, l);
}
MC_D f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
MC_D f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
MC_D f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
MC_D f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}

// Dirac spinor in the chiral representation, components as packed complex.
struct sp4p {
  f2 l0, l1, r0, r1;
};
MC_D sp4p operator+(const sp4p& a, const sp4p& b) {
  return {add2(a.l0, b.l0), add2(a.l1, b.l1), add2(a.r0, b.r0), add2(a.r1, b.r1)};
}
MC_D sp4p operator-(const sp4p& a, const sp4p& b) {
  return {sub2(a.l0, b.l0), sub2(a.l1, b.l1), sub2(a.r0, b.r0), sub2(a.r1, b.r1)};
}
MC_D sp4p to_p(const sp4<float>& s) {
  return {pk2(s.l0.re, s.l0.im), pk2(s.l1.re, s.l1.im), pk2(s.r0.re, s.r0.im), pk2(s.r1.re, s.r1.im)};
}

// A real four-vector prepared for slashing: A = a0 - a3, D = a0 + a3, a1 and
// the sign pair P = (a2, -a2); with N = swap(P) = (-a2, a2),
// (a1 - i a2) z = a1 z + P swap(z) and (a1 + i a2) z = a1 z + N swap(z).
struct sv {
  float A, D, x;
  f2 P;
};
MC_D sv make_sv(const v4<float>& a) { return {a.e - a.z, a.e + a.z, a.x, pk2(a.y, -a.y)}; }
MC_D sv make_sv(const v4<float>& a, float s) {  // the vector a s
  return make_sv(v4<float>{a.e * s, a.x * s, a.y * s, a.z * s});
}

// (a-slash) p for a column spinor p
MC_D sp4p slash_colp(const sv& a, const sp4p& p) {
  const f2 N = swp2(a.P);
  sp4p o;
  o.l0 = fma2(N, swp2(p.r1), fma2(bc2(-a.x), p.r1, mul2(bc2(a.A), p.r0)));
  o.l1 = fma2(a.P, swp2(p.r0), fma2(bc2(-a.x), p.r0, mul2(bc2(a.D), p.r1)));
  o.r0 = fma2(a.P, swp2(p.l1), fma2(bc2(a.x), p.l1, mul2(bc2(a.D), p.l0)));
  o.r1 = fma2(N, swp2(p.l0), fma2(bc2(a.x), p.l0, mul2(bc2(a.A), p.l1)));
  return o;
}
// (k-slash + m) p with the propagator denominator folded into k and m
MC_D sp4p prop_colp(const sv& k, float m, const sp4p& p) {
  const f2 N = swp2(k.P);
  sp4p o;
  o.l0 = fma2(N, swp2(p.r1), fma2(bc2(-k.x), p.r1, fma2(bc2(k.A), p.r0, mul2(bc2(m), p.l0))));
  o.l1 = fma2(k.P, swp2(p.r0), fma2(bc2(-k.x), p.r0, fma2(bc2(k.D), p.r1, mul2(bc2(m), p.l1))));
  o.r0 = fma2(k.P, swp2(p.l1), fma2(bc2(k.x), p.l1, fma2(bc2(k.D), p.l0, mul2(bc2(m), p.r0))));
  o.r1 = fma2(N, swp2(p.l0), fma2(bc2(k.x), p.l0, fma2(bc2(k.A), p.l1, mul2(bc2(m), p.r1))));
  return o;
}

// Row spinor times (a-slash): (b aslash).L = b.R (a.sigmabar),
// (b aslash).R = b.L (a.sigma), with the same prepared vector as slash_colp.
MC_D sp4p slash_rowp(const sp4p& b, const sv& a) {
  const f2 N = swp2(a.P);
  sp4p o;
  o.l0 = fma2(N, swp2(b.r1), fma2(bc2(a.x), b.r1, mul2(bc2(a.D), b.r0)));
  o.l1 = fma2(a.P, swp2(b.r0), fma2(bc2(a.x), b.r0, mul2(bc2(a.A), b.r1)));
  o.r0 = fma2(a.P, swp2(b.l1), fma2(bc2(-a.x), b.l1, mul2(bc2(a.A), b.l0)));
  o.r1 = fma2(N, swp2(b.l0), fma2(bc2(-a.x), b.l0, mul2(bc2(a.D), b.l1)));
  return o;
}
// b (k-slash + m) for a row spinor, the denominator folded as in prop_colp
MC_D sp4p prop_rowp(const sp4p& b, const sv& k, float m) {
  const f2 N = swp2(k.P);
  sp4p o;
  o.l0 = fma2(N, swp2(b.r1), fma2(bc2(k.x), b.r1, fma2(bc2(k.D), b.r0, mul2(bc2(m), b.l0))));
  o.l1 = fma2(k.P, swp2(b.r0), fma2(bc2(k.x), b.r0, fma2(bc2(k.A), b.r1, mul2(bc2(m), b.l1))));
  o.r0 = fma2(k.P, swp2(b.l1), fma2(bc2(-k.x), b.l1, fma2(bc2(k.A), b.l0, mul2(bc2(m), b.r0))));
  o.r1 = fma2(N, swp2(b.l0), fma2(bc2(-k.x), b.l0, fma2(bc2(k.D), b.l1, mul2(bc2(m), b.r1))));
  return o;
}

// bar . col for a barred row spinor with scalar parts: the real parts of the
// row times col plus the imaginary parts times swap(col), combined with the
// sign pair (-1, 1) at the end.
MC_D f2 dotp(const sp4<float>& b, const sp4p& c) {
  f2 ra = mul2(bc2(b.l0.re), c.l0);
  f2 ia = mul2(bc2(b.l0.im), swp2(c.l0));
  ra = fma2(bc2(b.l1.re), c.l1, ra);
  ia = fma2(bc2(b.l1.im), swp2(c.l1), ia);
  ra = fma2(bc2(b.r0.re), c.r0, ra);
  ia = fma2(bc2(b.r0.im), swp2(c.r0), ia);
  ra = fma2(bc2(b.r1.re), c.r1, ra);
  ia = fma2(bc2(b.r1.im), swp2(c.r1), ia);
  return fma2(pk2(-1.0f, 1.0f), ia, ra);
}

// The same product for a packed row spinor.
MC_D f2 dotpp(const sp4p& b, const sp4p& c) {
  f2 ra = mul2(bc2(lo2(b.l0)), c.l0);
  f2 ia = mul2(bc2(hi2(b.l0)), swp2(c.l0));
  ra = fma2(bc2(lo2(b.l1)), c.l1, ra);
  ia = fma2(bc2(hi2(b.l1)), swp2(c.l1), ia);
  ra = fma2(bc2(lo2(b.r0)), c.r0, ra);
  ia = fma2(bc2(hi2(b.r0)), swp2(c.r0), ia);
  ra = fma2(bc2(lo2(b.r1)), c.r1, ra);
  ia = fma2(bc2(hi2(b.r1)), swp2(c.r1), ia);
  return fma2(pk2(-1.0f, 1.0f), ia, ra);
}

// Stores of packed row spinors that an amplitude routine forms once per
// event and reads back inside its helicity loops.  Row i is the pair of
// 16-byte words 2i, 2i + 1 ((l0, l1) and (r0, r1)).
// In shared memory: word j of this thread at byte base + j * step, so that
// with step = 16 x (threads sharing the array) and consecutive threads at
// consecutive 16-byte offsets a warp's access covers one contiguous 512 bytes.
struct SmemRows {
  uint32_t base, step;
  MC_D void put(int i, const sp4p& r) const {
    const uint32_t ad = base + uint32_t(2 * i) * step;
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(ad), "l"(r.l0.v), "l"(r.l1.v) : "memory");
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(ad + step), "l"(r.r0.v), "l"(r.r1.v) : "memory");
  }
  MC_D sp4p get(int i) const {
    const uint32_t ad = base + uint32_t(2 * i) * step;
    sp4p r;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(r.l0.v), "=l"(r.l1.v) : "r"(ad));
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(r.r0.v), "=l"(r.r1.v) : "r"(ad + step));
    return r;
  }
};
// No store: the routine forms each row where it is used.
struct NoRows {};

}  // namespace mc
