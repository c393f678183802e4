// FP64 CPU oracle for the per-event LO cross-section integrand.
//
// TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
// the CUDA path is checked against; it shares no code with the CUDA path.
// Only the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark may load it.  Every function cites the thesis passage
// (arxiv 2302.03343) it restates: section titles and equation labels as
// they appear in the thesis source.
//
// Parity pins: every function here is pinned by at least one test in
// tests/test_oracle_*.py against a closed form, an invariant, an external
// library routine or brute force.  See the per-function comments.
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <vector>

namespace orc {

using cplx = std::complex<double>;

// ---------------------------------------------------------------- Philox
// Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11.  The thesis uses random uniforms throughout
// (Sec. "Sample generation") but names no generator.
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

// Integer uniform per dimension for event `ev` (see uniform_ints in philox.cpp
// for the counter layout).  prec 0 = 52-bit integers, prec 1 = 23-bit.
void event_uniform_ints(uint64_t seed, uint32_t iteration, uint32_t gid, int prec,
                        int ndim, int64_t ev, uint64_t* k);
int uniform_bits(int prec);

// ---------------------------------------------------------------- Lorentz
// Four-vectors over a scalar type T (double, or an operation-counting type).
template <class T>
struct P4T {
  T e = 0, x = 0, y = 0, z = 0;
};
using P4 = P4T<double>;
template <class T>
inline T dot(const P4T<T>& a, const P4T<T>& b) { return a.e * b.e - a.x * b.x - a.y * b.y - a.z * b.z; }
template <class T>
inline P4T<T> add(const P4T<T>& a, const P4T<T>& b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
inline P4T<T> sub(const P4T<T>& a, const P4T<T>& b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T>
inline P4T<T> scale(const P4T<T>& a, T s) { return {a.e * s, a.x * s, a.y * s, a.z * s}; }

// ---------------------------------------------------------------- phase space
// Sec. "Phase space generation from particle collisions", eq. 2bodyps.
void two_body(double sqrt_s, double m1, double m2, double cos_theta, double phi, P4* p, double* w);
// Sec. "RAMBO": eq. rambo-transform, eq. rambo-w0 and the massive extension.
// u has 4n entries.  Returns 0, or -5 if the xi equation did not converge.
int rambo(int n, const double* masses, double sqrt_s, const double* u, P4* p, double* w);
// Sec. "Hierarchical approach": table tab:hierarchical (see phasespace.cpp for
// the readings of the garbled mass step and weight).  u has 3n-4 entries.
int hierarchical(int n, const double* masses, double sqrt_s, const double* u, P4* p, double* w);

// ---------------------------------------------------------------- PDF
struct Pdf {
  int nx = 0, nq = 0, nflav = 0;
  std::vector<double> x, q, logx, logq2;
  std::vector<int> pids;
  std::vector<double> xf;  // [nx][nq][nflav]  (LHAPDF data-block order)
  int flavour_index(int pid) const;
  double node(int ix, int iq, int fl) const { return xf[(size_t(ix) * nq + iq) * nflav + fl]; }
};
// Sec. "LHAPDF: the Les Houches Accord PDF": log-bicubic cubic-Hermite
// interpolation in (log x, log Q^2).  Returns x*f(x, Q^2).
double pdf_xfxq2(const Pdf& pdf, int pid, double x, double q2);

// ---------------------------------------------------------------- |M|^2
// Spin- and colour-averaged squared matrix elements (GeV^-2 units free).
struct EWParams {
  double alpha, mz, gz, sw2;
};
double me2_eemumu(const EWParams& ew, double s, double cos_theta);
double me2_qqbar_ttbar(double alpha_s, double mt, double s, double t);
double me2_gg_ttbar(double alpha_s, double mt, double s, double t);
// Colour-ordered numerical evaluation with explicit Dirac matrices
// (formulation A).  p[0], p[1]: incoming gluons; p[2]: top; p[3]: anti-top;
// p[4]: outgoing gluon (gg->ttg only).
double me2_gg_ttbar_colour_ordered(double alpha_s, double mt, const P4* p);
double me2_gg_ttbarg(double alpha_s, double mt, const P4* p);
// Feynman diagrams with explicit SU(3) colour indices (formulation B).
double me2_gg_ttbarg_brute(double alpha_s, double mt, const P4* p);
// Helicity amplitudes on spinors (formulation C, helicity_t.h), and the
// gluon orderings and colour matrix it shares with formulation A.
double me2_gg_ttbarg_helicity(double alpha_s, double mt, const P4* p);
const std::vector<std::array<int, 3>>& ggg_orderings();
const std::vector<double>& ggg_colour_matrix();
// q(p0) qbar(p1) -> t(p2) tbar(p3) g(p4) (five diagrams, explicit colours, Dirac
// traces) and q(p0) g(p1) -> t(p2) tbar(p3) q(p4) by crossing; spin- and
// colour-averaged.
double me2_qqbar_ttbarg(double alpha_s, double mt, const P4* p);
double me2_qg_ttbarq(double alpha_s, double mt, const P4* p);
// Colour-ordered partial amplitudes A(sigma) for given gluon polarisation
// vectors and explicit spinor pair (for gauge and soft-limit pins).
void ggttg_partial_amplitudes(double alpha_s, double mt, const P4* q_in, const cplx (*eps)[4],
                              int ngluon, const cplx* ubar, const cplx* v, cplx* amps);

// ---------------------------------------------------------------- integrand
enum Process { EE_MUMU = 0, PP_TTBAR = 1, GG_TTBARG = 2, GAUSS = 3, GG_TTBARG_7D = 4, GG_TTBARG_MC = 5,
               PP_TTBARJ = 6 };

}  // namespace orc

extern "C" {

// Plain-old-data views used by the ctypes wrapper (oracle/__init__.py).
typedef struct {
  int32_t proc, gauss_dim;
  double sqrt_s, m_top, alpha, alpha_s, mz, gz, sw2, mu_f, ptcut_g, etacut_g, gauss_sigma, gev2pb;
} orc_integrand;

typedef struct {
  double x[16];
  int32_t bin[16];
  double jac;        // VEGAS Jacobian
  double p[7][4];    // incoming a, b then outgoing momenta, partonic CM frame
  double x1, x2, shat;
  double lumi;       // f_g(x1) f_g(x2) (gluon-initiated channels)
  double lumi_qq;    // sum_q f_q(x1) f_qbar(x2) + f_qbar(x1) f_q(x2) (pp->tt only)
  double me2;        // averaged |M|^2 (e+e- channel, or the gg channel)
  double me2_qq;     // averaged |M|^2 of the q qbar channel (pp->tt only)
  double ps_weight;  // phase-space weight per unit hypercube
  double f;          // integrand value (pb) before the VEGAS Jacobian
  double weight;     // f * jac
  int32_t pass;      // 1 = inside the cuts/threshold, 0 = zero weight
  int32_t status;
  int32_t channel;   // multi-channel process: the channel that generated the event
  int32_t pad_;
  // p p -> t tbar + parton: |M|^2 of q qbar with the quark from beam b, of
  // q g, g q, qbar g, g qbar (quark or antiquark from beam a or b), and the
  // luminosities of the seven partonic channels in the order gg, q qbar,
  // qbar q, q g, g q, qbar g, g qbar
  double me2_x[5];
  double lumi_x[7];
} orc_event_record;

typedef struct {
  double sum, sum2;
  int64_t n, n_nonzero;
  double wmax;
} orc_iter_result;

void* orc_pdf_new(int nx, const double* x, int nq, const double* q, int nflav, const int* pids,
                  const double* xf);
void orc_pdf_free(void* pdf);

// An accepted event of the unweighted sample in the laboratory frame.
typedef struct {
  int64_t event;    // Philox event index
  double weight;    // its weight in the weighted sample
  double x1, x2;    // momentum fractions (1, 1 for e+e-)
  double p[5][4];   // incoming a, b, outgoing 1..nout: (E, px, py, pz)
  int32_t proc, nout;
} orc_lab_event;
}

namespace orc {
// Uniforms -> VEGAS map -> integrand of one event (integrand.cpp).
void eval_event(const orc_integrand& in, const Pdf* pdf, int nbins, const double* edges, int prec, uint64_t seed,
                uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec);
double acceptance_uniform(uint64_t seed, uint32_t iteration, uint32_t gid, int64_t ev);
// Multi-channel g g -> t tbar g (channels.cpp): 7 uniforms per event, a
// 17-dimension grid (x1, x2, then 5 dimensions per channel); used dimension
// d of an event of channel ch lives in grid dimension channel_grid_dim(d, ch).
// dens[3] receives the three channel densities at the event's point.
inline int channel_grid_dim(int d, int ch) { return d < 2 ? d : 2 + 5 * ch + (d - 2); }
void channels_event(const orc_integrand& in, const Pdf* pdf, int nbins, const double* edges, int prec, uint64_t seed,
                    uint32_t iteration, uint32_t gid, int64_t ev, orc_event_record* rec, double* dens);
double vegas_map_1d(const double* edges, int nbins, int bits, uint64_t k, int* bin, double* jac);
}  // namespace orc
