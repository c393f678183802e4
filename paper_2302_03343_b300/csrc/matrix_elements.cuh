// Tree-level |M|^2 from helicity amplitudes (thesis Sec. "The MadFlow event
// generator": helicity amplitudes joined by vertex/propagator routines and
// gathered into colour-ordered, gauge-invariant groups; fig. pp_ttx for the
// pp -> tt diagrams).  All functions return the spin- and colour-averaged
// |M|^2 for momenta in the partonic centre-of-mass frame.
#pragma once
#include <type_traits>

#include "helas.cuh"
#include "packed.cuh"

namespace mc {

// ------------------------------------------------------------- e+e- -> mu+mu-
// s-channel photon and Z (fixed-width Breit-Wigner) between massless lepton
// currents J^mu = g_L x_L^dag sigmabar^mu y_L + g_R x_R^dag sigma^mu y_R.
template <class R>
MC_D void lepton_current(const cx<R>* xl, const cx<R>* xr, const cx<R>* yl, const cx<R>* yr, R gl, R gr,
                         cx<R>* j) {
  // x^dag sigma^mu y for mu = 0..3 (sigmabar^mu = (1, -sigma^k))
  auto sandwich = [](const cx<R>* x, const cx<R>* y, cx<R>* s) {
    const cx<R> a = mul_conj(y[0], x[0]), b = mul_conj(y[1], x[1]);  // x0* y0, x1* y1
    const cx<R> c = mul_conj(y[1], x[0]), d = mul_conj(y[0], x[1]);  // x0* y1, x1* y0
    s[0] = a + b;
    s[1] = c + d;
    s[2] = mkc(c.im - d.im, d.re - c.re);  // -i x0* y1 + i x1* y0
    s[3] = a - b;
  };
  cx<R> sl[4], sr[4];
  sandwich(xl, yl, sl);
  sandwich(xr, yr, sr);
  j[0] = sl[0] * gl + sr[0] * gr;
  for (int k = 1; k < 4; ++k) j[k] = sr[k] * gr - sl[k] * gl;
}

template <class R>
MC_D R me2_eemumu(const v4<R>& pem, const v4<R>& pep, const v4<R>& pmm, const v4<R>& pmp, R s, R e2,
                  R sw2, R mz, R gz) {
  const R cw2 = R(1) - sw2;
  const R q = R(-1), t3 = R(-0.5);
  const R gl = t3 - q * sw2, gr = -q * sw2;
  const R zc = R(1) / (sw2 * cw2);
  // 1/(s - MZ^2 + i MZ GZ)
  const R dre = s - mz * mz, dim = mz * gz, dn = R(1) / (dre * dre + dim * dim);
  const cx<R> zprop = mkc(dre * dn, -dim * dn);
  R total = R(0);
  for (int h1 = -1; h1 <= 1; h1 += 2)
    for (int h2 = -1; h2 <= 1; h2 += 2) {
      const sp4<R> u1 = u_spinor(pem, R(0), h1);
      const sp4<R> v2 = v_spinor(pep, R(0), h2);
      const cx<R> v2l[2] = {v2.l0, v2.l1}, v2r[2] = {v2.r0, v2.r1};
      const cx<R> u1l[2] = {u1.l0, u1.l1}, u1r[2] = {u1.r0, u1.r1};
      cx<R> jev[4], jez[4];
      lepton_current(v2l, v2r, u1l, u1r, R(1), R(1), jev);  // vbar gamma u
      lepton_current(v2l, v2r, u1l, u1r, gl, gr, jez);
      for (int h3 = -1; h3 <= 1; h3 += 2)
        for (int h4 = -1; h4 <= 1; h4 += 2) {
          const sp4<R> u3 = u_spinor(pmm, R(0), h3);
          const sp4<R> v4s = v_spinor(pmp, R(0), h4);
          const cx<R> u3l[2] = {u3.l0, u3.l1}, u3r[2] = {u3.r0, u3.r1};
          const cx<R> v4l[2] = {v4s.l0, v4s.l1}, v4r[2] = {v4s.r0, v4s.r1};
          cx<R> jmv[4], jmz[4];
          lepton_current(u3l, u3r, v4l, v4r, R(1), R(1), jmv);  // ubar gamma v
          lepton_current(u3l, u3r, v4l, v4r, gl, gr, jmz);
          cx<R> dv = jev[0] * jmv[0], dz = jez[0] * jmz[0];
          for (int k = 1; k < 4; ++k) {
            dv = dv - jev[k] * jmv[k];
            dz = dz - jez[k] * jmz[k];
          }
          const cx<R> amp = dv * (q * q / s) + dz * zprop * zc;
          total += norm2(amp);
        }
    }
  return e2 * e2 * total * R(0.25);
}

// ------------------------------------------------------------- q qbar -> t tbar
// One s-channel gluon: |M|^2 = g^4 / s^2 |J_q . J_t|^2 summed over helicities,
// colour sum tr(t^a t^b) tr(t^a t^b) = 2, average 1/4 x 1/9.
template <class R>
MC_D R me2_qqbar_ttbar(const v4<R>& pq, const v4<R>& pqb, const v4<R>& pt, const v4<R>& ptb, R m, R g2) {
  const R s = mdot(pq + pqb, pq + pqb);
  R total = R(0);
  for (int h1 = -1; h1 <= 1; h1 += 2)
    for (int h2 = -1; h2 <= 1; h2 += 2) {
      const sp4<R> u = u_spinor(pq, R(0), h1);
      const sp4<R> vb = vbar_spinor(pqb, R(0), h2);
      // J_q^mu = vbar gamma^mu u for mu = 0..3 via slashing the basis vectors
      cx<R> jq[4];
      const v4<R> basis[4] = {{R(1), R(0), R(0), R(0)}, {R(0), R(1), R(0), R(0)},
                              {R(0), R(0), R(1), R(0)}, {R(0), R(0), R(0), R(1)}};
      for (int mu = 0; mu < 4; ++mu) {
        // gamma^mu = gamma^nu (e_mu)_nu with (e_mu)_nu = g_{mu nu}: slash(a) uses a^mu,
        // so gamma^0 = slash(1,0,0,0) and gamma^k = -slash(e_k).
        const cx<R> val = dot(vb, slash_col(basis[mu], u));
        jq[mu] = mu == 0 ? val : -val;
      }
      for (int h3 = -1; h3 <= 1; h3 += 2)
        for (int h4 = -1; h4 <= 1; h4 += 2) {
          const sp4<R> ub = ubar_spinor(pt, m, h3);
          const sp4<R> v = v_spinor(ptb, m, h4);
          cx<R> jt[4];
          for (int mu = 0; mu < 4; ++mu) {
            const cx<R> val = dot(ub, slash_col(basis[mu], v));
            jt[mu] = mu == 0 ? val : -val;
          }
          cx<R> d = jq[0] * jt[0] - jq[1] * jt[1] - jq[2] * jt[2] - jq[3] * jt[3];
          total += norm2(d);
        }
    }
  return g2 * g2 / (s * s) * total * R(2) / R(36);
}

// ------------------------------------------------------------- g g -> t tbar
// Two colour-ordered partial amplitudes (gluon order along the quark line)
// A(ab) = ubar [ -epsa S(pt - qa) epsb + J(ab) ] v (common factor i g^2
// dropped), colour matrix of the strings t^a t^b, t^b t^a:
// [[16/3, -2/3], [-2/3, 16/3]]; average 1/4 (spins) x 1/64 (colours).
template <class R>
MC_D R me2_gg_ttbar(const v4<R>& pa, const v4<R>& pb, const v4<R>& pt, const v4<R>& ptb, R m, R g2) {
  const v4<R> q[2] = {pa, pb};
  v4<R> eps[2][2];
  linear_polarisations(pa, &eps[0][0], &eps[0][1]);
  linear_polarisations(pb, &eps[1][0], &eps[1][1]);
  const v4<R> k0 = pt - pa, k1 = pt - pb;
  const R inv0 = R(1) / (mdot(k0, k0) - m * m), inv1 = R(1) / (mdot(k1, k1) - m * m);
  const v4<R> qab = pa + pb;
  const R invq = R(1) / mdot(qab, qab);
  R total = R(0);
  // spin-flip symmetry (see me2_gg_ttbarg): the antitop spin +1/2 half, doubled
  for (int ht = -1; ht <= 1; ht += 2) {
    const sp4<R> ub = ubar_spinor(pt, m, ht);
    {
      const sp4<R> v = v_spinor(ptb, m, +1);
      for (int h = 0; h < 4; ++h) {
        const v4<R> e0 = eps[0][h & 1], e1 = eps[1][h >> 1];
        const v4<R> j01 = gluon_current(e0, q[0], e1, q[1], invq);
        const sp4<R> r0 = slash_col(e0, v), r1 = slash_col(e1, v);
        const cx<R> cur = dot(ub, slash_col(j01, v));
        // A(01) = -ubar e0 S0 e1 v + J01 ;  A(10) = -ubar e1 S1 e0 v - J01
        const cx<R> a01 = cur - dot(slash_row(ub, e0), prop_col(k0, m, inv0, r1));
        const cx<R> a10 = -cur - dot(slash_row(ub, e1), prop_col(k1, m, inv1, r0));
        const R d = norm2(a01) + norm2(a10);
        const R o = a01.re * a10.re + a01.im * a10.im;
        total += (R(16) / R(3)) * d - (R(4) / R(3)) * o;
      }
    }
  }
  return g2 * g2 * total * R(2) / R(256);
}

// ------------------------------------------------------------- g g -> t tbar g
// Six colour-ordered partial amplitudes A(abc) of the strings t^a t^b t^c
// (gluons with incoming momenta q_a; the outgoing gluon is crossed) built
// right to left on the anti-top spinor:
//   Gamma(abc) v = epsa S_a epsb S_ab epsc v - J(ab) S_ab epsc v
//                - epsa S_a J(bc) v + J(abc) v,
// S_a = S(pt - q_a), S_ab = S(pt - q_a - q_b) (its momentum depends only on
// the remaining gluon c), J(ab) = W(eps_a, eps_b), J(abc) = W(J(ab), eps_c) +
// W(eps_a, J(bc)) + contact term (common factor i g^3 dropped).
// Orderings are indexed lexicographically: 012, 021, 102, 120, 201, 210.
// Colour matrix (x 1/27) = sum over gluon colours of tr(t^{s1} t^{s2} t^{s3}
// (t^{s'1} t^{s'2} t^{s'3})^dagger), tr(t^a t^b) = delta/2, evaluated with
// the Fierz identity sum_a t^a_ij t^a_kl = (delta_il delta_kj - delta_ij delta_kl / 3) / 2:
// 192 on the diagonal (C_F^3 N), 30 for the reversed string, 3 for its two
// cyclic shifts, -24 for the two adjacent transpositions.
__constant__ float kColour3[36] = {
    192, -24, -24, 3,   3,   30,  -24, 192, 3,   30,  -24, 3,   -24, 3,   192, -24, 30,  3,
    3,   30,  -24, 192, 3,   -24, 3,   -24, 30,  3,   192, -24, 30,  3,   3,   -24, -24, 192};

template <class R>
MC_D R me2_gg_ttbarg(const v4<R>& pa, const v4<R>& pb, const v4<R>& pt, const v4<R>& ptb, const v4<R>& pg,
                     R m, R g2) {
  const v4<R> q[3] = {pa, pb, -pg};
  v4<R> eps[3][2];
  linear_polarisations(pa, &eps[0][0], &eps[0][1]);
  linear_polarisations(pb, &eps[1][0], &eps[1][1]);
  linear_polarisations(pg, &eps[2][0], &eps[2][1]);
  // fermion propagators: single gluon a next to the top, and the pair
  // complementary to gluon c
  v4<R> ka[3], kc[3];
  R inva[3], invc[3];
  for (int a = 0; a < 3; ++a) {
    ka[a] = pt - q[a];
    inva[a] = R(1) / (mdot(ka[a], ka[a]) - m * m);
    kc[a] = q[a] - ptb;  // pt - q_b - q_c with {b, c} the other two gluons
    invc[a] = R(1) / (mdot(kc[a], kc[a]) - m * m);
  }
  // gluon propagators of the pairs (01), (02), (12) and of all three
  const v4<R> q01 = q[0] + q[1], q02 = q[0] + q[2], q12 = q[1] + q[2];
  const R i01 = R(1) / mdot(q01, q01), i02 = R(1) / mdot(q02, q02), i12 = R(1) / mdot(q12, q12);
  const v4<R> qall = q01 + q[2];
  const R iall = R(1) / mdot(qall, qall);

  // Spin-flip symmetry: with real momenta and real (linear) polarisation
  // vectors the antilinear map psi -> gamma^5 gamma^2 psi^* turns every
  // helicity spinor into the opposite-helicity one up to a phase and leaves
  // the slashed real vectors and the propagators invariant, so
  // A_sigma(-s_t, -s_tbar) = c A_sigma(s_t, s_tbar)^* with one phase c for all
  // orderings.  The colour-summed square is then equal for the two spin
  // assignments: only the anti-top spin +1/2 is evaluated and the sum doubled.
  sp4<R> ubar[2];
  ubar[0] = ubar_spinor(pt, m, -1);
  ubar[1] = ubar_spinor(pt, m, +1);
  const sp4<R> v = v_spinor(ptb, m, +1);

  R total = R(0);
  // polarisation loops nested so that X_0, X_1, J(01) and S_2 J(01) v are
  // formed once per outer configuration
#pragma unroll 1
  for (int h0 = 0; h0 < 2; ++h0) {
   const v4<R> e0 = eps[0][h0];
   const sp4<R> x0 = prop_col(kc[0], m, invc[0], slash_col(e0, v));
#pragma unroll 1
   for (int h1 = 0; h1 < 2; ++h1) {
    const v4<R> e1 = eps[1][h1];
    const sp4<R> x1 = prop_col(kc[1], m, invc[1], slash_col(e1, v));
    const v4<R> j01 = gluon_current(e0, q[0], e1, q[1], i01);
    const sp4<R> s2j01 = prop_col(ka[2], m, inva[2], slash_col(j01, v));
#pragma unroll 1
    for (int h2 = 0; h2 < 2; ++h2) {
    const v4<R> e2 = eps[2][h2];
    // pair currents J(ab) for a < b (J(ba) = -J(ab))
    const v4<R> j02 = gluon_current(e0, q[0], e2, q[2], i02);
    const v4<R> j12 = gluon_current(e1, q[1], e2, q[2], i12);
    // triple currents, J(cba) = J(abc): J012 = J210, J021 = J120, J102 = J201
    const v4<R> j012 = gluon_current(j01, q01, e2, q[2], iall) + gluon_current(e0, q[0], j12, q12, iall) +
                       gluon_contact(e0, e1, e2, iall);
    const v4<R> j021 = gluon_current(j02, q02, e1, q[1], iall) + gluon_current(e0, q[0], -j12, q12, iall) +
                       gluon_contact(e0, e2, e1, iall);
    const v4<R> j102 = gluon_current(-j01, q01, e2, q[2], iall) + gluon_current(e1, q[1], j02, q02, iall) +
                       gluon_contact(e1, e0, e2, iall);
    {
      // X_c = S_{pair != c} eps_c v
      const sp4<R> x[3] = {x0, x1, prop_col(kc[2], m, invc[2], slash_col(e2, v))};
      // column spinors Gamma(sigma) v for the six orderings
      sp4<R> col[6];
      // term 1: eps_a S_a eps_b X_c
      // (a,b,c): 012 021 102 120 201 210
      col[0] = slash_col(e0, prop_col(ka[0], m, inva[0], slash_col(e1, x[2])));
      col[1] = slash_col(e0, prop_col(ka[0], m, inva[0], slash_col(e2, x[1])));
      col[2] = slash_col(e1, prop_col(ka[1], m, inva[1], slash_col(e0, x[2])));
      col[3] = slash_col(e1, prop_col(ka[1], m, inva[1], slash_col(e2, x[0])));
      col[4] = slash_col(e2, prop_col(ka[2], m, inva[2], slash_col(e0, x[1])));
      col[5] = slash_col(e2, prop_col(ka[2], m, inva[2], slash_col(e1, x[0])));
      // term 2: -J(ab) X_c
      const sp4<R> y2 = slash_col(j01, x[2]), y1 = slash_col(j02, x[1]), y0 = slash_col(j12, x[0]);
      col[0] = col[0] - y2;
      col[2] = col[2] + y2;
      col[1] = col[1] - y1;
      col[4] = col[4] + y1;
      col[3] = col[3] - y0;
      col[5] = col[5] + y0;
      // term 3: -eps_a S_a J(bc) v
      const sp4<R> z0 = slash_col(e0, prop_col(ka[0], m, inva[0], slash_col(j12, v)));
      const sp4<R> z1 = slash_col(e1, prop_col(ka[1], m, inva[1], slash_col(j02, v)));
      const sp4<R> z2 = slash_col(e2, s2j01);
      col[0] = col[0] - z0;
      col[1] = col[1] + z0;
      col[2] = col[2] - z1;
      col[3] = col[3] + z1;
      col[4] = col[4] - z2;
      col[5] = col[5] + z2;
      // term 4: J(abc) v
      const sp4<R> w012 = slash_col(j012, v), w021 = slash_col(j021, v), w102 = slash_col(j102, v);
      col[0] = col[0] + w012;
      col[5] = col[5] + w012;
      col[1] = col[1] + w021;
      col[3] = col[3] + w021;
      col[2] = col[2] + w102;
      col[4] = col[4] + w102;
#pragma unroll
      for (int ht = 0; ht < 2; ++ht) {
        cx<R> amp[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) amp[s] = dot(ubar[ht], col[s]);
        R acc = R(0);
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          acc += R(kColour3[s * 6 + s]) * norm2(amp[s]);
#pragma unroll
          for (int t = s + 1; t < 6; ++t)
            acc += R(2) * R(kColour3[s * 6 + t]) * (amp[s].re * amp[t].re + amp[s].im * amp[t].im);
        }
        total += acc;
      }
    }
    }
   }
  }
  return g2 * g2 * g2 * total * R(2) / (R(27) * R(256));
}

// ------------------------------------------ light-quark line -> t tbar g
// q qbar -> t tbar g and its crossings with a light-quark line and one
// external gluon, from helicity amplitudes of the five diagrams (emission
// off the light line before and after the internal gluon, off the top and
// the anti-top, and off the internal gluon through the three-gluon vertex),
// with vertices i g gamma T, quark propagators i (pslash + m)/(p^2 - m^2),
// gluon propagators -i g / k^2 and the three-gluon vertex
// g f [g (k - p) + g (p - q) + g (q - k)] (momenta incoming).  The light line
// is the column spinor `col` entering with fermion-flow momentum Pin and the
// row spinor `row` leaving with Pout; the gluon has outgoing-convention
// momentum k:
//   kind 0, q(pa) qbar(pb) -> t tbar g(pk): col u(pa), row vbar(pb), Pin pa,
//           Pout -pb, k pk, average 1/36;
//   kind 1, q(pa) g(pb) -> t tbar q(pk): col u(pa), row ubar(pk), Pin pa,
//           Pout pk, k -pb, average 1/96;
//   kind 2, qbar(pa) g(pb) -> t tbar qbar(pk): col v(pk), row vbar(pa),
//           Pin -pk, Pout -pa, k -pb, average 1/96.
// Colour-stripped amplitudes A_d (d: emission before / after on the light
// line, off t, off tbar, three-gluon) combine with the colour matrix
// C_de = sum over colours of c_d c_e^* (Hermitian, complex), passed as
// re/im pairs: |M|^2 = sum_d C_dd |A_d|^2 + 2 sum_{d<e} Re(C_de A_d A_e^*).
// The light-line currents depend only on the light helicities and the gluon
// polarisation, the heavy-line ones only on the top spins and the
// polarisation: both are formed once (the light side for the two helicity
// pairs the massless line allows, kept; the heavy side per top-spin
// configuration) and contracted for every combination.
template <class R>
MC_D R me2_qline_ttbarg(int kind, const v4<R>& pa, const v4<R>& pb, const v4<R>& pt, const v4<R>& ptb,
                        const v4<R>& pk, R m, R g2, const R* cmat) {
  const v4<R> k = kind == 0 ? pk : -pb;
  const v4<R> kphys = kind == 0 ? pk : pb;
  const v4<R> pin = kind == 2 ? -pk : pa;
  const v4<R> pout = kind == 0 ? -pb : (kind == 1 ? pk : -pa);
  const v4<R> q = pt + ptb, pl = pin - pout;
  const R iq2 = R(1) / mdot(q, q), ip2 = R(1) / mdot(pl, pl);
  const v4<R> s1 = pin - k, s2 = pout + k, s3 = pt + k, s4 = -(ptb + k);
  const R i1 = R(1) / mdot(s1, s1), i2 = R(1) / mdot(s2, s2);
  const R i3 = R(1) / (mdot(s3, s3) - m * m), i4 = R(1) / (mdot(s4, s4) - m * m);
  const v4<R> kpq = pl + q, kmq = k - q, mkp = -(k + pl);
  v4<R> eps[2];
  linear_polarisations(kphys, &eps[0], &eps[1]);
  const R g3 = g2 * m_sqrt(g2);
  // light side: a massless line keeps its chirality through an odd number of
  // gamma matrices, so u(h) pairs with vbar(-h) and ubar(h), v(h) with vbar(h)
  cx<R> vl[2][4], v1[2][2][4], v2[2][2][4];  // [helicity pair][polarisation][mu]
#pragma unroll 1
  for (int ip = 0; ip < 2; ++ip) {
    const int h1 = 2 * ip - 1, h2 = kind == 0 ? -h1 : h1;
    const sp4<R> col = kind == 2 ? v_spinor(pk, R(0), h1) : u_spinor(pa, R(0), h1);
    const sp4<R> row = kind == 0 ? vbar_spinor(pb, R(0), h2)
                                 : (kind == 1 ? ubar_spinor(pk, R(0), h2) : vbar_spinor(pa, R(0), h2));
    vector_current(row, col, vl[ip]);
#pragma unroll
    for (int lam = 0; lam < 2; ++lam) {
      vector_current(row, prop_col(s1, R(0), i1, slash_col(eps[lam], col)), v1[ip][lam]);
      vector_current(prop_row(slash_row(row, eps[lam]), s2, R(0), i2), col, v2[ip][lam]);
    }
  }
  cx<R> vlk[2], vle[2][2];  // vl . (k - q), vl . eps
#pragma unroll
  for (int ip = 0; ip < 2; ++ip) {
    vlk[ip] = cdot4(vl[ip], kmq);
#pragma unroll
    for (int lam = 0; lam < 2; ++lam) vle[ip][lam] = cdot4(vl[ip], eps[lam]);
  }
  const cx<R> mi = mkc(R(0), -g3);  // -i g^3
  R total = R(0);
#pragma unroll 1
  for (int h3 = -1; h3 <= 1; h3 += 2) {
    const sp4<R> ut = ubar_spinor(pt, m, h3);
#pragma unroll 1
    for (int h4 = -1; h4 <= 1; h4 += 2) {
      const sp4<R> vt = v_spinor(ptb, m, h4);
      cx<R> hh[4];
      vector_current(ut, vt, hh);
      const cx<R> hhm = cdot4(hh, mkp);
#pragma unroll
      for (int lam = 0; lam < 2; ++lam) {
        const v4<R>& e = eps[lam];
        cx<R> h3v[4], h4v[4];
        vector_current(prop_row(slash_row(ut, e), s3, m, i3), vt, h3v);
        vector_current(ut, prop_col(s4, m, i4, slash_col(e, vt)), h4v);
        const cx<R> hhe = cdot4(hh, e);
        const R ke = mdot(kpq, e);
#pragma unroll
        for (int ip = 0; ip < 2; ++ip) {
          cx<R> amp[5];
          amp[0] = mi * (cdot4(v1[ip][lam], hh) * iq2);
          amp[1] = mi * (cdot4(v2[ip][lam], hh) * iq2);
          amp[2] = mi * (cdot4(vl[ip], h3v) * ip2);
          amp[3] = mi * (cdot4(vl[ip], h4v) * ip2);
          amp[4] = (cdot4(vl[ip], hh) * ke + vlk[ip] * hhe + vle[ip][lam] * hhm) * (g3 * ip2 * iq2);
#pragma unroll
          for (int d = 0; d < 5; ++d) {
            total += cmat[2 * (d * 5 + d)] * norm2(amp[d]);
#pragma unroll
            for (int f = d + 1; f < 5; ++f) {
              const cx<R> x = mul_conj(amp[d], amp[f]);  // A_d A_f^*
              total += R(2) * (cmat[2 * (d * 5 + f)] * x.re - cmat[2 * (d * 5 + f) + 1] * x.im);
            }
          }
        }
      }
    }
  }
  return total / (kind == 0 ? R(36) : R(96));
}

// ---- packed complex helpers of me2_qline_ttbarg_p (FP32): a complex
// number is the pair (re, im); x y = re(x) y + im(x) (i y), i y =
// (-1, 1) * swap(y), so sums of products gather the re(x) y and the
// im(x) swap(y) terms apart and combine them once.
MC_D f2 cx_i(f2 ra, f2 ia) { return fma2(pk2(-1.0f, 1.0f), ia, ra); }
MC_D f2 cmul2(f2 x, f2 y) { return cx_i(mul2(bc2(lo2(x)), y), mul2(bc2(hi2(x)), swp2(y))); }
// J^mu = rbar gamma^mu c (vector_current) for packed spinors
MC_D void vcur_p(const sp4p& b, const sp4p& c, f2* j) {
  const float L0r = lo2(b.l0), L0i = hi2(b.l0), L1r = lo2(b.l1), L1i = hi2(b.l1);
  const float R0r = lo2(b.r0), R0i = hi2(b.r0), R1r = lo2(b.r1), R1i = hi2(b.r1);
  const f2 sr0 = swp2(c.r0), sr1 = swp2(c.r1), sl0 = swp2(c.l0), sl1 = swp2(c.l1);
  // J0 = a + d + e + f, J3 = a - d - e + f, J1 = g + h - k - l, J2 = -i (g - h - k + l)
  // with a = L0 r0, d = L1 r1, e = R0 l0, f = R1 l1, g = L0 r1, h = L1 r0, k = R0 l1, l = R1 l0
  const f2 ad_r = fma2(bc2(L0r), c.r0, mul2(bc2(L1r), c.r1)), ad_i = fma2(bc2(L0i), sr0, mul2(bc2(L1i), sr1));
  const f2 ef_r = fma2(bc2(R0r), c.l0, mul2(bc2(R1r), c.l1)), ef_i = fma2(bc2(R0i), sl0, mul2(bc2(R1i), sl1));
  const f2 af_r = fma2(bc2(L0r), c.r0, mul2(bc2(R1r), c.l1)), af_i = fma2(bc2(L0i), sr0, mul2(bc2(R1i), sl1));
  const f2 de_r = fma2(bc2(L1r), c.r1, mul2(bc2(R0r), c.l0)), de_i = fma2(bc2(L1i), sr1, mul2(bc2(R0i), sl0));
  j[0] = cx_i(add2(ad_r, ef_r), add2(ad_i, ef_i));
  j[3] = cx_i(sub2(af_r, de_r), sub2(af_i, de_i));
  const f2 gh_r = fma2(bc2(L0r), c.r1, mul2(bc2(L1r), c.r0)), gh_i = fma2(bc2(L0i), sr1, mul2(bc2(L1i), sr0));
  const f2 kl_r = fma2(bc2(R0r), c.l1, mul2(bc2(R1r), c.l0)), kl_i = fma2(bc2(R0i), sl1, mul2(bc2(R1i), sl0));
  j[1] = cx_i(sub2(gh_r, kl_r), sub2(gh_i, kl_i));
  const f2 gl_r = fma2(bc2(L0r), c.r1, mul2(bc2(R1r), c.l0)), gl_i = fma2(bc2(L0i), sr1, mul2(bc2(R1i), sl0));
  const f2 hk_r = fma2(bc2(L1r), c.r0, mul2(bc2(R0r), c.l1)), hk_i = fma2(bc2(L1i), sr0, mul2(bc2(R0i), sl1));
  const f2 t = cx_i(sub2(gl_r, hk_r), sub2(gl_i, hk_i));
  j[2] = mul2(pk2(1.0f, -1.0f), swp2(t));  // -i t
}
// a . b for complex four-vectors
MC_D f2 cdot4_p(const f2* a, const f2* b) {
  const f2 ra = fma2(bc2(lo2(a[0])), b[0], fma2(bc2(-lo2(a[1])), b[1],
                fma2(bc2(-lo2(a[2])), b[2], mul2(bc2(-lo2(a[3])), b[3]))));
  const f2 ia = fma2(bc2(hi2(a[0])), swp2(b[0]), fma2(bc2(-hi2(a[1])), swp2(b[1]),
                fma2(bc2(-hi2(a[2])), swp2(b[2]), mul2(bc2(-hi2(a[3])), swp2(b[3])))));
  return cx_i(ra, ia);
}
// a . v for a complex four-vector and a real one
MC_D f2 cdot4_pr(const f2* a, const v4<float>& v) {
  return fma2(bc2(v.e), a[0], fma2(bc2(-v.x), a[1], fma2(bc2(-v.y), a[2], mul2(bc2(-v.z), a[3]))));
}

// me2_qline_ttbarg in FP32 with packed complex arithmetic: the same
// amplitudes, currents formed once per channel as there, and the colour sum
// as sum_d Re(A_d conj(sum_e conj(C_de) ... )) written out below.
MC_D float me2_qline_ttbarg_p(int kind, const v4<float>& pa, const v4<float>& pb, const v4<float>& pt,
                              const v4<float>& ptb, const v4<float>& pk, float m, float g2, const float* cmat) {
  const v4<float> k = kind == 0 ? pk : -pb;
  const v4<float> kphys = kind == 0 ? pk : pb;
  const v4<float> pin = kind == 2 ? -pk : pa;
  const v4<float> pout = kind == 0 ? -pb : (kind == 1 ? pk : -pa);
  const v4<float> q = pt + ptb, pl = pin - pout;
  const float iq2 = 1.0f / mdot(q, q), ip2 = 1.0f / mdot(pl, pl);
  const v4<float> s1 = pin - k, s2 = pout + k, s3 = pt + k, s4 = -(ptb + k);
  const float i1 = 1.0f / mdot(s1, s1), i2 = 1.0f / mdot(s2, s2);
  const float i3 = 1.0f / (mdot(s3, s3) - m * m), i4 = 1.0f / (mdot(s4, s4) - m * m);
  const sv S1 = make_sv(s1, i1), S2 = make_sv(s2, i2), S3 = make_sv(s3, i3), S4 = make_sv(s4, i4);
  const float m3 = m * i3, m4 = m * i4;
  const v4<float> kpq = pl + q, kmq = k - q, mkp = -(k + pl);
  v4<float> eps[2];
  linear_polarisations(kphys, &eps[0], &eps[1]);
  const sv E[2] = {make_sv(eps[0]), make_sv(eps[1])};
  const float g3 = g2 * sqrtf(g2);
  // -i g^3 iq2 z = (g3 iq2 im z, -g3 iq2 re z): the swap of z times this pair
  const f2 mq = pk2(g3 * iq2, -g3 * iq2), mp = pk2(g3 * ip2, -g3 * ip2);
  const float c4 = g3 * ip2 * iq2;
  f2 vl[2][4], v1[2][2][4], v2[2][2][4];
#pragma unroll 1
  for (int ip = 0; ip < 2; ++ip) {
    const int h1 = 2 * ip - 1, h2 = kind == 0 ? -h1 : h1;
    const sp4p col = to_p(kind == 2 ? v_spinor(pk, 0.0f, h1) : u_spinor(pa, 0.0f, h1));
    const sp4p row = to_p(kind == 0 ? vbar_spinor(pb, 0.0f, h2)
                                    : (kind == 1 ? ubar_spinor(pk, 0.0f, h2) : vbar_spinor(pa, 0.0f, h2)));
    vcur_p(row, col, vl[ip]);
#pragma unroll
    for (int lam = 0; lam < 2; ++lam) {
      vcur_p(row, prop_colp(S1, 0.0f, slash_colp(E[lam], col)), v1[ip][lam]);
      vcur_p(prop_rowp(slash_rowp(row, E[lam]), S2, 0.0f), col, v2[ip][lam]);
    }
  }
  f2 vlk[2], vle[2][2];
#pragma unroll
  for (int ip = 0; ip < 2; ++ip) {
    vlk[ip] = cdot4_pr(vl[ip], kmq);
#pragma unroll
    for (int lam = 0; lam < 2; ++lam) vle[ip][lam] = cdot4_pr(vl[ip], eps[lam]);
  }
  float total = 0.0f;
#pragma unroll 1
  for (int h3 = -1; h3 <= 1; h3 += 2) {
    const sp4p ut = to_p(ubar_spinor(pt, m, h3));
#pragma unroll 1
    for (int h4 = -1; h4 <= 1; h4 += 2) {
      const sp4p vt = to_p(v_spinor(ptb, m, h4));
      f2 hh[4];
      vcur_p(ut, vt, hh);
      const f2 hhm = cdot4_pr(hh, mkp);
#pragma unroll
      for (int lam = 0; lam < 2; ++lam) {
        f2 h3v[4], h4v[4];
        vcur_p(prop_rowp(slash_rowp(ut, E[lam]), S3, m3), vt, h3v);
        vcur_p(ut, prop_colp(S4, m4, slash_colp(E[lam], vt)), h4v);
        const f2 hhe = cdot4_pr(hh, eps[lam]);
        const float ke = mdot(kpq, eps[lam]);
#pragma unroll
        for (int ip = 0; ip < 2; ++ip) {
          f2 amp[5];
          amp[0] = mul2(mq, swp2(cdot4_p(v1[ip][lam], hh)));
          amp[1] = mul2(mq, swp2(cdot4_p(v2[ip][lam], hh)));
          amp[2] = mul2(mp, swp2(cdot4_p(vl[ip], h3v)));
          amp[3] = mul2(mp, swp2(cdot4_p(vl[ip], h4v)));
          amp[4] = mul2(bc2(c4), fma2(bc2(ke), cdot4_p(vl[ip], hh),
                                      add2(cmul2(vlk[ip], hhe), cmul2(vle[ip][lam], hhm))));
          // sum_d C_dd |A_d|^2 + 2 sum_{d<f} Re(C_df A_d conj(A_f)):
          // per d, s_d = sum_{f>d} C_df conj(A_f), then Re(A_d s_d)
#pragma unroll
          for (int d = 0; d < 5; ++d) {
            const f2 sq = mul2(amp[d], amp[d]);
            total += cmat[2 * (d * 5 + d)] * (lo2(sq) + hi2(sq));
            if (d < 4) {
              // C conj(A) = (Cr ar + Ci ai, Ci ar - Cr ai) = Cr (ar, -ai) + Ci (ai, ar)
              f2 sr = bc2(0.0f), si = bc2(0.0f);
#pragma unroll
              for (int f = d + 1; f < 5; ++f) {
                sr = fma2(bc2(cmat[2 * (d * 5 + f)]), amp[f], sr);
                si = fma2(bc2(cmat[2 * (d * 5 + f) + 1]), swp2(amp[f]), si);
              }
              // s = conj-combination: s = (sr.re + si.re, si.im - sr.im)
              const f2 sd = fma2(pk2(1.0f, -1.0f), sr, si);
              const f2 p = mul2(amp[d], pk2(lo2(sd), -hi2(sd)));  // (ar sr, -ai si)
              total += 2.0f * (lo2(p) + hi2(p));
            }
          }
        }
      }
    }
  }
  return total / (kind == 0 ? 36.0f : 96.0f);
}

// Unroll factors of the helicity loops of me2_gg_ttbarg_p (1: a rolled loop,
// which keeps the consumer warps' register count down).
#ifndef MC_ME_UNROLL_H0
#define MC_ME_UNROLL_H0 1
#define MC_ME_UNROLL_H1 1
#define MC_ME_UNROLL_H2 1
#endif
#define MC_PRAGMA(x) _Pragma(#x)
#define MC_UNROLL_(n) MC_PRAGMA(unroll n)
#define MC_UNROLL(n) MC_UNROLL_(n)

// Products used by me2_gg_ttbarg_p.  A gluon's linear polarisation vector
// has no time component and is orthogonal to the gluon's momentum.
// a . T for a real four-vector a and a complex one T (packed components)
MC_D f2 rdot_c(const v4<float>& a, const f2* T) {
  return fma2(bc2(a.e), T[0], fma2(bc2(-a.x), T[1], fma2(bc2(-a.y), T[2], mul2(bc2(-a.z), T[3]))));
}
// the same for a polarisation vector e (e^0 = 0)
MC_D f2 pdot_c(const v4<float>& e, const f2* T) {
  return fma2(bc2(-e.x), T[1], fma2(bc2(-e.y), T[2], mul2(bc2(-e.z), T[3])));
}
// a . e for a polarisation vector e
MC_D float pdot(const v4<float>& a, const v4<float>& e) { return -(a.x * e.x + a.y * e.y + a.z * e.z); }
// The pair current gluon_current(ea, qa, eb, qb, inv) of two external gluons:
// with ea . qa = eb . qb = 0 the vertex reduces to
// (ea . eb)(qa - qb) + 2 (ea . qb) eb - 2 (eb . qa) ea.
MC_D v4<float> pair_current(const v4<float>& ea, const v4<float>& eb, const v4<float>& dq, float eaqb, float ebqa,
                            float inv) {
  const float c1 = -inv * pdot(ea, eb), c2 = -2.0f * inv * eaqb, c3 = 2.0f * inv * ebqa;
  return {c1 * dq.e, c1 * dq.x + c2 * eb.x + c3 * ea.x, c1 * dq.y + c2 * eb.y + c3 * ea.y,
          c1 * dq.z + c2 * eb.z + c3 * ea.z};
}

// FP32 gg -> t tbar g with packed (re, im) complex arithmetic: the same
// colour-ordered amplitudes as me2_gg_ttbarg, regrouped per ordering (abc):
//   Gamma(abc) v = eps_a S_a [eps_b X_c - J(bc) v] - J(ab) X_c + J(abc) v,
// with ubar J(abc)-slash v = J(abc) . T, T^mu = ubar gamma^mu v; each column
// spinor is contracted with both top spinors as soon as it is formed.  The
// pair currents use e_a . q_a = 0 (pair_current), and the three triple
// currents share four three-gluon vertices and the products of the contact
// terms (the decomposition written out above me2_gg_ttbarg_rows), which
// removes two fifths of the scalar work of the currents without adding
// per-event state: this routine runs where registers, not operations, are
// the limit.
MC_D float me2_gg_ttbarg_p(const v4<float>& pa, const v4<float>& pb, const v4<float>& pt, const v4<float>& ptb,
                           const v4<float>& pg, float m, float g2) {
  const v4<float> q[3] = {pa, pb, -pg};
  v4<float> eps[3][2];
  linear_polarisations(pa, &eps[0][0], &eps[0][1]);
  linear_polarisations(pb, &eps[1][0], &eps[1][1]);
  linear_polarisations(pg, &eps[2][0], &eps[2][1]);
  sv ka[3], kc[3];
  float ma[3], mc_[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const v4<float> k1 = pt - q[a];
    const float i1 = 1.0f / (mdot(k1, k1) - m * m);
    ka[a] = make_sv(k1, i1);
    ma[a] = m * i1;
    const v4<float> k2 = q[a] - ptb;
    const float i2 = 1.0f / (mdot(k2, k2) - m * m);
    kc[a] = make_sv(k2, i2);
    mc_[a] = m * i2;
  }
  const v4<float> q01 = q[0] + q[1], q02 = q[0] + q[2], q12 = q[1] + q[2];
  const float i01 = 1.0f / mdot(q01, q01), i02 = 1.0f / mdot(q02, q02), i12 = 1.0f / mdot(q12, q12);
  const v4<float> qall = q01 + q[2];
  const float iall = 1.0f / mdot(qall, qall);
  const sp4<float> ub[2] = {ubar_spinor(pt, m, -1), ubar_spinor(pt, m, +1)};
  const sp4p v = to_p(v_spinor(ptb, m, +1));
  // T[ht][mu] = ubar gamma^mu v, gamma^0 = slash(1,0,0,0), gamma^k = slash(-e_k)
  f2 T[2][4];
  {
    const sp4p g0 = slash_colp(make_sv(v4<float>{1.0f, 0.0f, 0.0f, 0.0f}), v);
    const sp4p g1 = slash_colp(make_sv(v4<float>{0.0f, -1.0f, 0.0f, 0.0f}), v);
    const sp4p g2v = slash_colp(make_sv(v4<float>{0.0f, 0.0f, -1.0f, 0.0f}), v);
    const sp4p g3 = slash_colp(make_sv(v4<float>{0.0f, 0.0f, 0.0f, -1.0f}), v);
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      T[ht][0] = dotp(ub[ht], g0);
      T[ht][1] = dotp(ub[ht], g1);
      T[ht][2] = dotp(ub[ht], g2v);
      T[ht][3] = dotp(ub[ht], g3);
    }
  }
  f2 total0 = bc2(0.0f), total1 = bc2(0.0f);
  MC_UNROLL(MC_ME_UNROLL_H0)
  for (int h0 = 0; h0 < 2; ++h0) {
    const v4<float> e0 = eps[0][h0];
    const sp4p x0 = prop_colp(kc[0], mc_[0], slash_colp(make_sv(e0), v));
    MC_UNROLL(MC_ME_UNROLL_H1)
    for (int h1 = 0; h1 < 2; ++h1) {
      const v4<float> e1 = eps[1][h1];
      const sp4p x1 = prop_colp(kc[1], mc_[1], slash_colp(make_sv(e1), v));
      const v4<float> j01 = pair_current(e0, e1, q[0] - q[1], pdot(q[1], e0), pdot(q[0], e1), i01);
      const sp4p u01 = slash_colp(make_sv(j01), v);
      MC_UNROLL(MC_ME_UNROLL_H2)
      for (int h2 = 0; h2 < 2; ++h2) {
        const v4<float> e2 = eps[2][h2];
        const v4<float> j02 = pair_current(e0, e2, q[0] - q[2], pdot(q[2], e0), pdot(q[0], e2), i02);
        const v4<float> j12 = pair_current(e1, e2, q[1] - q[2], pdot(q[2], e1), pdot(q[1], e2), i12);
        const sp4p x2 = prop_colp(kc[2], mc_[2], slash_colp(make_sv(e2), v));
        f2 amp[2][6];
        // orderings 012 021 102 120 201 210
#define MC_PUT(S, EA, A, B)                                                  \
  {                                                                          \
    const sp4p c_ = slash_colp(make_sv(EA), prop_colp(ka[A], ma[A], B));     \
    amp[0][S] = dotp(ub[0], c_);                                             \
    amp[1][S] = dotp(ub[1], c_);                                             \
  }
        {
          const sp4p u12 = slash_colp(make_sv(j12), v);
          MC_PUT(0, e0, 0, slash_colp(make_sv(e1), x2) - u12)
          MC_PUT(1, e0, 0, slash_colp(make_sv(e2), x1) + u12)
        }
        {
          const sp4p u02 = slash_colp(make_sv(j02), v);
          MC_PUT(2, e1, 1, slash_colp(make_sv(e0), x2) - u02)
          MC_PUT(3, e1, 1, slash_colp(make_sv(e2), x0) + u02)
        }
        MC_PUT(4, e2, 2, slash_colp(make_sv(e0), x1) - u01)
        MC_PUT(5, e2, 2, slash_colp(make_sv(e1), x0) + u01)
#undef MC_PUT
        // -J(ab) X_c, with J(ba) = -J(ab)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const sp4p y = c == 2 ? slash_colp(make_sv(j01), x2) : (c == 1 ? slash_colp(make_sv(j02), x1)
                                                                         : slash_colp(make_sv(j12), x0));
          const int sm = c == 2 ? 0 : (c == 1 ? 1 : 3), sp = c == 2 ? 2 : (c == 1 ? 4 : 5);
#pragma unroll
          for (int ht = 0; ht < 2; ++ht) {
            const f2 d = dotp(ub[ht], y);
            amp[ht][sm] = sub2(amp[ht][sm], d);
            amp[ht][sp] = add2(amp[ht][sp], d);
          }
        }
        // J(abc) v contracted with ubar: J . T ; J(012) = J(210), J(021) = J(120), J(102) = J(201)
        {
          // four shared vertices V(x, qx, y, qy) (gluon_current without -1/Q^2)
          const float a1 = pdot(j01, e2), b1 = mdot(j01, q01 + q[2] * 2.0f), c1 = 2.0f * pdot(q01, e2);
          const v4<float> V1 = (q01 - q[2]) * a1 + e2 * b1 - j01 * c1;  // V(j01, q01, e2, q2)
          const float a2 = pdot(j12, e0), b2 = 2.0f * pdot(q12, e0), c2 = mdot(j12, q[0] * 2.0f + q12);
          const v4<float> V2 = (q[0] - q12) * a2 + j12 * b2 - e0 * c2;  // V(e0, q0, j12, q12)
          const float a3 = pdot(j02, e1), b3 = mdot(j02, q02 + q[1] * 2.0f), c3 = 2.0f * pdot(q02, e1);
          const v4<float> V3 = (q02 - q[1]) * a3 + e1 * b3 - j02 * c3;  // V(j02, q02, e1, q1)
          const v4<float> V4 = (q[1] - q02) * a3 + j02 * c3 - e1 * b3;  // V(e1, q1, j02, q02)
          // contact terms C(x, y, z) Q^2 = 2 (x.z) y - (y.z) x - (x.y) z from
          // P0 = -(e1.e2) e0, P1 = -(e0.e2) e1, P2 = -(e0.e1) e2, S = P0 + P1 + P2:
          // C(012) = S - 3 P1, C(021) = S - 3 P2, C(102) = S - 3 P0
          const v4<float> P0 = e0 * -pdot(e1, e2), P1 = e1 * -pdot(e0, e2), P2 = e2 * -pdot(e0, e1);
          const v4<float> S = P0 + P1 + P2;
          const v4<float> j012 = (S - P1 * 3.0f - V1 - V2) * iall;
          const v4<float> j021 = (S - P2 * 3.0f - V3 + V2) * iall;
          const v4<float> j102 = (S - P0 * 3.0f + V1 - V4) * iall;
#pragma unroll
          for (int ht = 0; ht < 2; ++ht) {
            const f2 wa = fma2(bc2(j012.e), T[ht][0], fma2(bc2(-j012.x), T[ht][1],
                          fma2(bc2(-j012.y), T[ht][2], mul2(bc2(-j012.z), T[ht][3]))));
            const f2 wb = fma2(bc2(j021.e), T[ht][0], fma2(bc2(-j021.x), T[ht][1],
                          fma2(bc2(-j021.y), T[ht][2], mul2(bc2(-j021.z), T[ht][3]))));
            const f2 wc = fma2(bc2(j102.e), T[ht][0], fma2(bc2(-j102.x), T[ht][1],
                          fma2(bc2(-j102.y), T[ht][2], mul2(bc2(-j102.z), T[ht][3]))));
            amp[ht][0] = add2(amp[ht][0], wa);
            amp[ht][5] = add2(amp[ht][5], wa);
            amp[ht][1] = add2(amp[ht][1], wb);
            amp[ht][3] = add2(amp[ht][3], wb);
            amp[ht][2] = add2(amp[ht][2], wc);
            amp[ht][4] = add2(amp[ht][4], wc);
          }
        }
#pragma unroll
        for (int ht = 0; ht < 2; ++ht) {
#pragma unroll
          for (int s = 0; s < 6; ++s) {
            f2 c = mul2(bc2(kColour3[s * 6 + s]), amp[ht][s]);
#pragma unroll
            for (int t = s + 1; t < 6; ++t) c = fma2(bc2(2.0f * kColour3[s * 6 + t]), amp[ht][t], c);
            if (ht == 0)
              total0 = fma2(amp[ht][s], c, total0);
            else
              total1 = fma2(amp[ht][s], c, total1);
          }
        }
      }
    }
  }
  const f2 total = add2(total0, total1);
  return g2 * g2 * g2 * (lo2(total) + hi2(total)) * 2.0f / (27.0f * 256.0f);
}

// The same |M|^2 as me2_gg_ttbarg_p with fewer operations and more per-event
// state, for a kernel that can hold that state in shared memory:
//   ubar Gamma(abc) v = R(a) [eps_b X_c - J(bc) v] - ubar J(ab) X_c + J(abc) . T,
// with the row spinors R(a) = ubar eps_a S_a and the column spinors
// X_c = S_{pair != c} eps_c v, T^mu = ubar gamma^mu v.  The twelve rows
// R(a, h_a, s_t) depend on one gluon's polarisation only: they are formed
// once per event, kept in the row store (index (2a + h_a) 2 + s_t) and read
// back in the helicity loops, which then cost one slash and two products per
// ordering instead of two slashes, a propagator and two products.
// The triple currents enter only through J(abc) . T.  Each is a sum of two
// three-gluon vertices and a contact term, all bilinear in the currents they
// join, so J(abc) . T is assembled from scalar products instead of the
// four-vector: with V(x, qx, y, qy) = (x.y)(qx - qy) + y (x.(qx + 2 qy))
// - x (y.(2 qx + qy)) (the vertex of gluon_current without -1/Q^2),
//   V . T = (x.y)((qx - qy).T) + (y.T)(x.(qx + 2 qy)) - (x.T)(y.(2 qx + qy)),
// and V(-x, ...) = -V(x, ...) lets the three orderings share four vertices:
//   J(012) = -[V(j01, q01, e2, q2) + V(e0, q0, j12, q12)]/Q^2 + C(0, 1, 2),
//   J(021) = -[V(j02, q02, e1, q1) - V(e0, q0, j12, q12)]/Q^2 + C(0, 2, 1),
//   J(102) = -[-V(j01, q01, e2, q2) + V(e1, q1, j02, q02)]/Q^2 + C(1, 0, 2),
// with the contact terms C(x, y, z) = [2 (x.z) y - (y.z) x - (x.y) z]/Q^2
// (gluon_contact) and Q the sum of the three gluon momenta.
template <class Rows>
MC_D float me2_gg_ttbarg_rows(const v4<float>& pa, const v4<float>& pb, const v4<float>& pt, const v4<float>& ptb,
                           const v4<float>& pg, float m, float g2, Rows rows) {
  const v4<float> q[3] = {pa, pb, -pg};
  v4<float> eps[3][2];
  linear_polarisations(pa, &eps[0][0], &eps[0][1]);
  linear_polarisations(pb, &eps[1][0], &eps[1][1]);
  linear_polarisations(pg, &eps[2][0], &eps[2][1]);
  const sp4<float> ub[2] = {ubar_spinor(pt, m, -1), ubar_spinor(pt, m, +1)};
  const sp4p v = to_p(v_spinor(ptb, m, +1));
  sv kc[3];
  float mc_[3];
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    const v4<float> k1 = pt - q[a];
    const float i1 = 1.0f / (mdot(k1, k1) - m * m);
    const sv ka = make_sv(k1, i1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const sv e = make_sv(eps[a][h]);
#pragma unroll
      for (int ht = 0; ht < 2; ++ht) rows.put((2 * a + h) * 2 + ht, prop_rowp(slash_rowp(to_p(ub[ht]), e), ka, m * i1));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const v4<float> k2 = q[a] - ptb;
    const float i2 = 1.0f / (mdot(k2, k2) - m * m);
    kc[a] = make_sv(k2, i2);
    mc_[a] = m * i2;
  }
  const v4<float> q01 = q[0] + q[1], q02 = q[0] + q[2], q12 = q[1] + q[2];
  const float i01 = 1.0f / mdot(q01, q01), i02 = 1.0f / mdot(q02, q02), i12 = 1.0f / mdot(q12, q12);
  const v4<float> qall = q01 + q[2];
  const float iall = 1.0f / mdot(qall, qall);
  const v4<float> d01 = q[0] - q[1], d02 = q[0] - q[2], d12 = q[1] - q[2];
  // T[ht][mu] = ubar gamma^mu v / Q^2, gamma^0 = slash(1,0,0,0), gamma^k = slash(-e_k)
  f2 T[2][4];
  {
    const sp4p g0 = slash_colp(make_sv(v4<float>{iall, 0.0f, 0.0f, 0.0f}), v);
    const sp4p g1 = slash_colp(make_sv(v4<float>{0.0f, -iall, 0.0f, 0.0f}), v);
    const sp4p g2v = slash_colp(make_sv(v4<float>{0.0f, 0.0f, -iall, 0.0f}), v);
    const sp4p g3 = slash_colp(make_sv(v4<float>{0.0f, 0.0f, 0.0f, -iall}), v);
#pragma unroll
    for (int ht = 0; ht < 2; ++ht) {
      T[ht][0] = dotp(ub[ht], g0);
      T[ht][1] = dotp(ub[ht], g1);
      T[ht][2] = dotp(ub[ht], g2v);
      T[ht][3] = dotp(ub[ht], g3);
    }
  }
  // (qx - qy) . T of the vertices V1 = V(j01, q01, e2, q2), V2 = V(e0, q0, j12, q12),
  // V3 = V(j02, q02, e1, q1) and V4 = V(e1, q1, j02, q02) (the last is -DT[.][2])
  f2 DT[2][3];
#pragma unroll
  for (int ht = 0; ht < 2; ++ht) {
    DT[ht][0] = rdot_c(q01 - q[2], T[ht]);
    DT[ht][1] = rdot_c(q[0] - q12, T[ht]);
    DT[ht][2] = rdot_c(q02 - q[1], T[ht]);
  }
  const v4<float> A1 = q01 + q[2] * 2.0f, B2 = q[0] * 2.0f + q12, A3 = q02 + q[1] * 2.0f, B4 = q[1] * 2.0f + q02;
  f2 total0 = bc2(0.0f), total1 = bc2(0.0f);
  MC_UNROLL(MC_ME_UNROLL_H0)
  for (int h0 = 0; h0 < 2; ++h0) {
    const v4<float> e0 = eps[0][h0];
    const sp4p x0 = prop_colp(kc[0], mc_[0], slash_colp(make_sv(e0), v));
    const float e0q1 = pdot(q[1], e0), e0q2 = pdot(q[2], e0);
    const float e0A2 = 2.0f * pdot(q12, e0);  // e0 . (q0 + 2 q12)
    const f2 e0T[2] = {pdot_c(e0, T[0]), pdot_c(e0, T[1])};
    MC_UNROLL(MC_ME_UNROLL_H1)
    for (int h1 = 0; h1 < 2; ++h1) {
      const v4<float> e1 = eps[1][h1];
      const sp4p x1 = prop_colp(kc[1], mc_[1], slash_colp(make_sv(e1), v));
      const float e1q2 = pdot(q[2], e1);
      const float e1B3 = 2.0f * pdot(q02, e1);  // e1 . (2 q02 + q1) = e1 . (q1 + 2 q02)
      const float e0e1 = pdot(e0, e1);
      const v4<float> j01 = pair_current(e0, e1, d01, e0q1, pdot(q[0], e1), i01);
      const sp4p u01 = slash_colp(make_sv(j01), v);
      const float j01A1 = mdot(j01, A1);
      const f2 j01T[2] = {rdot_c(j01, T[0]), rdot_c(j01, T[1])};
      const f2 e1T[2] = {pdot_c(e1, T[0]), pdot_c(e1, T[1])};
      MC_UNROLL(MC_ME_UNROLL_H2)
      for (int h2 = 0; h2 < 2; ++h2) {
        const v4<float> e2 = eps[2][h2];
        const float e2q0 = pdot(q[0], e2), e2q1 = pdot(q[1], e2);
        const v4<float> j02 = pair_current(e0, e2, d02, e0q2, e2q0, i02);
        const v4<float> j12 = pair_current(e1, e2, d12, e1q2, e2q1, i12);
        const sp4p x2 = prop_colp(kc[2], mc_[2], slash_colp(make_sv(e2), v));
        f2 amp[2][6];
        // orderings 012 021 102 120 201 210: (a, b, c) with the row of a
        // times eps_b X_c -/+ J(bc) v
#define MC_PUT2(S0, S1, A, HA, COL0, COL1)                           \
  {                                                                 \
    const sp4p r0_ = rows.get((2 * A + HA) * 2 + 0);                \
    const sp4p r1_ = rows.get((2 * A + HA) * 2 + 1);                \
    const sp4p c0_ = COL0;                                          \
    amp[0][S0] = dotpp(r0_, c0_);                                   \
    amp[1][S0] = dotpp(r1_, c0_);                                   \
    const sp4p c1_ = COL1;                                          \
    amp[0][S1] = dotpp(r0_, c1_);                                   \
    amp[1][S1] = dotpp(r1_, c1_);                                   \
  }
        {
          const sp4p u12 = slash_colp(make_sv(j12), v);
          MC_PUT2(0, 1, 0, h0, slash_colp(make_sv(e1), x2) - u12, slash_colp(make_sv(e2), x1) + u12)
        }
        {
          const sp4p u02 = slash_colp(make_sv(j02), v);
          MC_PUT2(2, 3, 1, h1, slash_colp(make_sv(e0), x2) - u02, slash_colp(make_sv(e2), x0) + u02)
        }
        MC_PUT2(4, 5, 2, h2, slash_colp(make_sv(e0), x1) - u01, slash_colp(make_sv(e1), x0) + u01)
#undef MC_PUT2
        // -J(ab) X_c, with J(ba) = -J(ab)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const sp4p y = c == 2 ? slash_colp(make_sv(j01), x2) : (c == 1 ? slash_colp(make_sv(j02), x1)
                                                                         : slash_colp(make_sv(j12), x0));
          const int sm = c == 2 ? 0 : (c == 1 ? 1 : 3), sp = c == 2 ? 2 : (c == 1 ? 4 : 5);
#pragma unroll
          for (int ht = 0; ht < 2; ++ht) {
            const f2 d = dotp(ub[ht], y);
            amp[ht][sm] = sub2(amp[ht][sm], d);
            amp[ht][sp] = add2(amp[ht][sp], d);
          }
        }
        // J(abc) v contracted with ubar: J(abc) . T ; J(012) = J(210), J(021) = J(120), J(102) = J(201)
        {
          const float j01e2 = pdot(j01, e2), e0j12 = pdot(j12, e0), j12B2 = mdot(j12, B2);
          const float j02e1 = pdot(j02, e1), j02A3 = mdot(j02, A3), j02B4 = mdot(j02, B4);
          const float e2B1 = 2.0f * (e2q0 + e2q1);  // e2 . (2 q01 + q2)
          const float e0e2 = pdot(e0, e2), e1e2 = pdot(e1, e2);
#pragma unroll
          for (int ht = 0; ht < 2; ++ht) {
            const f2 e2T = pdot_c(e2, T[ht]), j12T = rdot_c(j12, T[ht]), j02T = rdot_c(j02, T[ht]);
            const f2 v1 = fma2(bc2(j01e2), DT[ht][0], fma2(bc2(j01A1), e2T, mul2(bc2(-e2B1), j01T[ht])));
            const f2 v2 = fma2(bc2(e0j12), DT[ht][1], fma2(bc2(e0A2), j12T, mul2(bc2(-j12B2), e0T[ht])));
            const f2 v3 = fma2(bc2(j02e1), DT[ht][2], fma2(bc2(j02A3), e1T[ht], mul2(bc2(-e1B3), j02T)));
            const f2 v4_ = fma2(bc2(-j02e1), DT[ht][2], fma2(bc2(e1B3), j02T, mul2(bc2(-j02B4), e1T[ht])));
            // contact terms: with P0 = -(e1.e2) e0T, P1 = -(e0.e2) e1T, P2 = -(e0.e1) e2T
            // and S = P0 + P1 + P2: C(012) = S - 3 P1, C(021) = S - 3 P2, C(102) = S - 3 P0
            const f2 p0 = mul2(bc2(-e1e2), e0T[ht]), p1 = mul2(bc2(-e0e2), e1T[ht]), p2 = mul2(bc2(-e0e1), e2T);
            const f2 sc = add2(add2(p0, p1), p2);
            const f2 wa = sub2(fma2(bc2(-3.0f), p1, sc), add2(v1, v2));
            const f2 wb = add2(fma2(bc2(-3.0f), p2, sc), sub2(v2, v3));
            const f2 wc = add2(fma2(bc2(-3.0f), p0, sc), sub2(v1, v4_));
            amp[ht][0] = add2(amp[ht][0], wa);
            amp[ht][5] = add2(amp[ht][5], wa);
            amp[ht][1] = add2(amp[ht][1], wb);
            amp[ht][3] = add2(amp[ht][3], wb);
            amp[ht][2] = add2(amp[ht][2], wc);
            amp[ht][4] = add2(amp[ht][4], wc);
          }
        }
#pragma unroll
        for (int ht = 0; ht < 2; ++ht) {
#pragma unroll
          for (int s = 0; s < 6; ++s) {
            f2 c = mul2(bc2(kColour3[s * 6 + s]), amp[ht][s]);
#pragma unroll
            for (int t = s + 1; t < 6; ++t) c = fma2(bc2(2.0f * kColour3[s * 6 + t]), amp[ht][t], c);
            if (ht == 0)
              total0 = fma2(amp[ht][s], c, total0);
            else
              total1 = fma2(amp[ht][s], c, total1);
          }
        }
      }
    }
  }
  const f2 total = add2(total0, total1);
  return g2 * g2 * g2 * (lo2(total) + hi2(total)) * 2.0f / (27.0f * 256.0f);
}

}  // namespace mc
