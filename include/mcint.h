/*
 * mcint.h - C ABI of the B300 per-event Monte Carlo cross-section library.
 *
 * The library evaluates, one event per thread inside a single fused CUDA
 * kernel, the leading-order collider cross-section integrand of the thesis
 * arXiv:2302.03343 (Part II, "MadFlow" chapter, master formula
 * eq. mc_master_formula):
 *
 *     sigma = sum_ab int dPhi_n(x1, x2, p) L(x1, x2) |M(ab -> X)|^2
 *
 * sampled with the VEGAS importance sampler (Sec. "Adaptive Monte Carlo:
 * VEGAS algorithm"): each event draws counter-based Philox4x32-10 uniforms,
 * maps them through the VEGAS grid, builds phase space (two-body or RAMBO,
 * Sec. "RAMBO"), interpolates the PDFs log-bicubically (Sec. "LHAPDF"),
 * evaluates |M|^2 from helicity amplitudes and accumulates the weighted sum,
 * the sum of squares and the per-bin VEGAS histograms.
 *
 * Conventions for every entry point:
 *  - Return value: MC_OK (0) or a negative MC_E* code; nothing throws across
 *    the ABI.  mc_last_error() returns a message for the calling thread's
 *    last failure (valid until the next call from that thread).
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    device memory of the current device.  Input arrays are caller-owned
 *    and are copied (or only read) before the call returns.
 *  - Handles (mc_pdf, mc_vegas) are library-owned; free them with the
 *    matching *_free call.  A handle belongs to the device that was current
 *    when it was created.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that return results to the host synchronise that stream
 *    before returning; other calls are asynchronous on it.
 *  - Energies in GeV, cross sections in pb.
 */
#ifndef MCINT_H
#define MCINT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define MC_OK 0
#define MC_EINVAL (-1)   /* invalid argument (shape, range, NaN input)          */
#define MC_ENOMEM (-2)   /* device or pinned-host allocation failed             */
#define MC_ECUDA (-3)    /* a CUDA runtime call failed                          */
#define MC_ENAN (-4)     /* non-finite event weights were produced (counted)    */
#define MC_ENOCONV (-5)  /* RAMBO's massive rescaling did not converge (counted) */
#define MC_ETIMEOUT (-6) /* a bounded device wait gave up (result invalid)      */
#define MC_EIO (-7)      /* a file could not be created or written              */

/* -------------------------------------------------------------- enums */
#define MC_FP64 0        /* integrand in FP64, 52-bit uniforms                   */
#define MC_FP32_KAHAN 1  /* integrand in FP32, 23-bit uniforms, FP64 reductions  */

#define MC_EE_MUMU 0    /* e+e- -> mu+mu- (gamma + Z), 2 dims                    */
#define MC_PP_TTBAR 1   /* p p -> t tbar (gg + q qbar), 4 dims                   */
#define MC_GG_TTBARG 2  /* g g -> t tbar g, RAMBO, 14 dims (7 physical)          */
#define MC_GAUSS 3      /* normalised Gaussian centred at 1/2, gauss_dim dims     */
#define MC_GG_TTBARG_7D 4 /* g g -> t tbar g, hierarchical 2->3 generator, 7 dims */
#define MC_GG_TTBARG_MC 5 /* g g -> t tbar g, three-channel sampling: 7 uniforms  */
                          /* per event, 17 grid dimensions (see below)           */
#define MC_PP_TTBARJ 6    /* p p -> t tbar + parton (gg, q qbar, q g, qbar g and  */
                          /* the beam-swapped channels), hierarchical 2 -> 3,     */
                          /* 7 dims; the parton with pT > ptcut_g (> 0),          */
                          /* |eta| < etacut_g                                     */

#define MC_MAX_DIM 17   /* grid dimensions: 16, or 17 for MC_GG_TTBARG_MC */
#define MC_MAX_BINS 256

typedef struct mc_pdf_s* mc_pdf;
typedef struct mc_vegas_s* mc_vegas;

/* One integrand.  Field order is part of the ABI. */
typedef struct {
  int32_t proc;        /* MC_EE_MUMU ... MC_GG_TTBARG_7D                         */
  int32_t gauss_dim;   /* dimension of MC_GAUSS (1..16), ignored otherwise       */
  double sqrt_s;       /* collider (or e+e-) centre-of-mass energy              */
  double m_top;        /* top-quark mass                                         */
  double alpha;        /* QED coupling (e+e- -> mu+mu-)                          */
  double alpha_s;      /* strong coupling, fixed                                 */
  double mz, gz, sw2;  /* Z mass, width, sin^2(theta_W)                          */
  double mu_f;         /* factorisation scale: PDFs are read at Q = mu_f         */
  double ptcut_g;      /* gg -> ttg: gluon pT > ptcut_g                          */
  double etacut_g;     /* gg -> ttg: |eta_gluon| < etacut_g (lab frame)          */
  double gauss_sigma;  /* width of MC_GAUSS                                      */
  double gev2pb;       /* GeV^-2 -> pb conversion (0.3893794e9)                  */
} mc_integrand;

/* Result of one VEGAS iteration (thesis eq. mc_est_is / eq. var_is inputs). */
typedef struct {
  double sum;          /* sum of event weights w = f * J (Kahan, FP64)           */
  double sum2;         /* sum of w^2                                             */
  int64_t n;           /* events evaluated                                       */
  int64_t n_nonzero;   /* events with w != 0                                     */
  double wmax;         /* largest weight (unweighting efficiency = mean / wmax)  */
  int64_t n_bad;       /* events dropped as non-finite or non-converged          */
  int32_t status;      /* MC_OK, MC_ENAN or MC_ENOCONV                           */
  int32_t pad_;
} mc_iter_result;

/* Combined result (thesis Sec. "Adaptive Monte Carlo: VEGAS algorithm":
 * inverse-variance mean, its error, and eq. vegas-check chi^2/dof). */
typedef struct {
  double mean, sigma, chi2_dof;
  int32_t n_iter;      /* iterations actually run                                */
  int32_t status;
  double gpu_ms;       /* device time of all iterations (CUDA events)            */
} mc_result;

/* Thread-local message for the last failing call of this thread. */
const char* mc_last_error(void);

/* ------------------------------------------------------------------ PDF
 * mc_pdf_load: an LHAPDF-style grid (thesis Sec. "LHAPDF: the Les Houches
 * Accord PDF"; PDFFlow's mkPDF/Subgrid of Sec. "Software design and
 * benchmarks").  x_knots[nx] strictly increasing in (0, 1], q_knots[nq]
 * strictly increasing (GeV), pids[nflav] PDG codes (21 = gluon), xf
 * [nx][nq][nflav] values x*f(x, Q) in the LHAPDF data-block order (x outer,
 * Q, then flavour), FP64, all host.  nx, nq >= 4.  Values must be finite.
 * The grid is copied to the device in FP64 and FP32.  EINVAL on bad shapes,
 * non-monotone knots or non-finite values; ENOMEM / ECUDA on device failure.
 */
int mc_pdf_load(const double* x_knots, int nx, const double* q_knots, int nq,
                const int32_t* pids, int nflav, const double* xf, mc_pdf* out);
int mc_pdf_free(mc_pdf pdf);

/* mc_pdf_xfxq2: PDFFlow's xfxQ2 over a batch (thesis Sec. "Software design
 * and benchmarks"): for n query points (x[i], q2[i]) (device arrays, FP64)
 * writes all flavours, xf_out[i][nflav] (device, FP64), by log-bicubic
 * Hermite interpolation in (log x, log Q^2); points outside the grid give
 * NaN.  prec selects FP64 or FP32 arithmetic.  Asynchronous on `stream`.
 */
int mc_pdf_xfxq2(mc_pdf pdf, int prec, int64_t n, const double* x, const double* q2,
                 double* xf_out, void* stream);

/* ---------------------------------------------------------- PDF sets
 * A PDF set of several sub-grids and members with LHAPDF's interpolation and
 * extrapolation rules (thesis Sec. "LHAPDF: the Les Houches Accord PDF";
 * multi-member evaluation: Sec. "PDFFlow: interpolating PDFs on GPUs",
 * Table tab:fktable).  Sub-grids cover adjacent Q ranges split at quark-mass
 * thresholds; the threshold knot is the last Q knot of one sub-grid and the
 * first of the next, and a query exactly on it uses the upper sub-grid.
 * Inside a sub-grid: cubic Hermite splines in log x, then in log Q^2, knot
 * slopes the mean of the adjacent divided differences (one-sided at the
 * sub-grid's ends); bilinear in (log x, log Q^2) where the sub-grid has
 * fewer than 4 knots in a direction.  Below x_min and above Q_max: linear
 * continuation in log x (log Q^2) from the two edge knots, of log(x f) when
 * both values exceed 1e-3 and of x f otherwise.  Below Q_min:
 * x f(Q^2_min) (Q^2/Q^2_min)^(gamma r + 1 - r), r = Q^2/Q^2_min, gamma =
 * d ln(x f)/d ln Q^2 from the two lowest Q knots (1 when either value is not
 * positive).  When x and Q are both outside, the x rule runs first.
 *
 * mc_pdfset_load: nsub (1..8) sub-grids with nx[s], nq[s] (>= 2) knots;
 * x: the x knots of all sub-grids concatenated (positive, increasing within
 * a sub-grid); q: the Q knots (GeV) concatenated, adjacent sub-grids sharing
 * the threshold knot; nflav (1..16) flavours with PDG ids pids[] (the output
 * follows this order); nmem (>= 1) members; xf: for each member, for each
 * sub-grid, nx[s] x nq[s] x nflav values in [x][q][flavour] order (LHAPDF's
 * data blocks).  All host arrays are caller-owned, FP64, copied; the set is
 * held on the current device in FP64 and FP32 until mc_pdfset_free.
 * EINVAL on bad shapes or knots, ENOMEM when the device allocation fails.
 */
typedef struct mc_pdfset_s* mc_pdfset;
int mc_pdfset_load(int nsub, const int* nx, const int* nq, const double* x, const double* q, int nflav,
                   const int* pids, int nmem, const double* xf, mc_pdfset* out);
int mc_pdfset_free(mc_pdfset set);
/* mc_pdfset_xfxq2: x f of every flavour of members member0 .. member0+nmem-1
 * at n points (x[i], q2[i]) (device arrays, FP64): out[m][i][flavour]
 * (device, caller-owned), double for prec = MC_FP64, float for
 * MC_FP32_KAHAN (FP32 arithmetic on the FP32 copy of the set).  x > x_max,
 * x <= 0 and q2 <= 0 give NaN.  Asynchronous on `stream`; EINVAL on a bad
 * member range or arguments, or when the set lives on another device. */
int mc_pdfset_xfxq2(mc_pdfset set, int prec, int member0, int nmem, int64_t n, const double* x, const double* q2,
                    void* out, void* stream);

/* alpha_s(Q) on LHAPDF-style knots (thesis Sec. "LHAPDF: the Les Houches
 * Accord PDF"): cubic Hermite in log Q^2 on the segments between repeated
 * (threshold) knots, alpha_s(Q_max) above the knots, and below them
 * ln alpha_s continued linearly in ln Q^2 from the two lowest knots.
 * mc_alphas_load: n (>= 2) knots q[] (GeV, non-decreasing; a value repeated
 * twice marks a threshold; the first and last segments need two distinct
 * knots) and alphas[] (> 0), host, FP64, copied to the current device.
 * mc_alphas_q2: alpha_s at n values q2[] (device, FP64) into out[] (device,
 * FP64); q2 <= 0 gives NaN; asynchronous on `stream`. */
typedef struct mc_alphas_s* mc_alphas;
int mc_alphas_load(int n, const double* q, const double* alphas, mc_alphas* out);
int mc_alphas_free(mc_alphas a);
int mc_alphas_q2(mc_alphas a, int64_t n, const double* q2, double* out, void* stream);

/* ---------------------------------------------------------------- VEGAS
 * mc_vegas_init: a VEGAS grid of ndim (1..16) dimensions with nbins
 * (2..256) equal bins each, the Philox seed, and the precision (MC_FP64 or
 * MC_FP32_KAHAN).  The iteration counter starts at 0; it enters the Philox
 * counter so every iteration draws fresh, reproducible uniforms.
 */
int mc_vegas_init(int ndim, int nbins, uint64_t seed, int prec, mc_vegas* out);
int mc_vegas_free(mc_vegas v);
/* Grid edges [ndim][nbins+1], host, FP64; set requires edges[d][0] = 0,
 * edges[d][nbins] = 1 and strictly increasing edges. */
int mc_vegas_set_grid(mc_vegas v, const double* edges);
int mc_vegas_get_grid(mc_vegas v, double* edges);
/* Accumulated histograms since the last refine: w2[ndim][nbins] (sum of w^2)
 * and counts[ndim][nbins] (events), host outputs; synchronises the device. */
int mc_vegas_get_hist(mc_vegas v, double* w2, uint32_t* counts);
/* mc_vegas_set_hist: replace the accumulated histograms (same layout as
 * mc_vegas_get_hist, host inputs, copied) -- the sums over the ranks of a
 * sharded iteration, before mc_vegas_refine.  EINVAL on NULL or on a
 * negative or non-finite w2 entry; synchronises the device. */
int mc_vegas_set_hist(mc_vegas v, const double* w2, const uint32_t* counts);
int mc_vegas_set_iteration(mc_vegas v, uint32_t iteration);
int mc_vegas_get_iteration(mc_vegas v, uint32_t* iteration);
/* Integrand id (0..255) mixed into the Philox counter (batched runs). */
int mc_vegas_set_gid(mc_vegas v, uint32_t gid);

/* mc_vegas_iterate: one VEGAS iteration of nevents events (eq. mc_est_is):
 * launches the fused integrand kernel over events 0..nevents-1 of the
 * current iteration, accumulates the histograms, advances the iteration
 * counter and returns the sums in *out (host; the stream is synchronised).
 * pdf may be NULL for processes without hadrons.  ndim of the grid must
 * equal the process dimension.  Events with a non-finite weight, or whose
 * RAMBO rescaling failed, contribute zero and are counted in out->n_bad;
 * out->status is then MC_ENAN or MC_ENOCONV while the call itself returns
 * MC_OK (the sums stay valid).
 */
int mc_vegas_iterate(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t nevents,
                     void* stream, mc_iter_result* out);

/* mc_vegas_iterate_shard: the events first .. first+count-1 of the current
 * iteration (Philox event indices first + i; the same points as those events
 * of an mc_vegas_iterate over the whole range), for one device of several
 * that split an iteration (thesis Sec. VEGAS: the iteration's estimate and
 * its histogram are sums over its events, so the parts' sums add up to the
 * whole's).  out holds the part's sums (out->n = count); the histograms
 * accumulate the part's events.  The caller adds the parts' sums and
 * histograms across devices (mc_vegas_get_hist / mc_vegas_set_hist) before
 * mc_vegas_refine, which then yields the same grid on every device.  Like
 * mc_vegas_iterate it advances the iteration counter.  For the three-channel
 * process the channel sums W_i are the part's means.  EINVAL on first < 0,
 * count < 0 or first + count beyond 2^63 - 1; otherwise as mc_vegas_iterate.
 */
int mc_vegas_iterate_shard(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t count,
                           void* stream, mc_iter_result* out);

/* mc_vegas_refine: rebins every dimension from the accumulated histograms
 * (smoothing, damping exponent alpha, equal-importance rebinning after
 * Lepage 1978, the reference of the thesis's VEGAS section) and clears the
 * histograms.  Asynchronous on `stream`. */
int mc_vegas_refine(mc_vegas v, double alpha, void* stream);

/* mc_integrate: full VEGAS integration from a uniform grid: up to niter
 * iterations of nevents events, refining with damping alpha after each, and
 * the inverse-variance combination with chi^2/dof.  target_rel_err > 0 stops
 * at the first iteration whose combined sigma/|mean| <= target_rel_err.
 * per_iter (host, may be NULL) receives niter results.  gid as in
 * mc_vegas_set_gid.  The stream is synchronised once per iteration.
 */
int mc_integrate(const mc_integrand* itg, mc_pdf pdf, int niter, int64_t nevents, int nbins,
                 uint64_t seed, uint32_t gid, int prec, double alpha, double target_rel_err,
                 void* stream, mc_result* out, mc_iter_result* per_iter);

/* -------------------------------------------- multi-channel sampling
 * Thesis Sec. "Multi-channel Monte Carlo": points are drawn from channel i
 * with probability alpha_i and weighted by f / p, p = sum_i alpha_i p_i; the
 * alpha_i leave the estimate unchanged and are adjusted to reduce its
 * variance (Kleiss & Pittau, cited there).  MC_GG_TTBARG_MC has three
 * channels, each a sequential splitting whose variables flatten one peak of
 * |M|^2: 0, initial-state radiation (gluon first: ln pT flat from the pT cut,
 * rapidity flat inside the lab-frame eta cut); 1 and 2, radiation off the
 * top and off the anti-top (t g or tbar g pair first, ln(s_pair - m^2 +
 * m pTcut) flat).  Every channel has its own VEGAS grid over its 5 variables
 * and all share the (x1, x2) grid: a 17-dimension grid (dims 0-1 x1, x2;
 * 2-6 channel 0; 7-11 channel 1; 12-16 channel 2), of which an event uses
 * and fills the 7 of its channel.  The channel of an event is Philox call
 * 254: u = (k + 0.5) 2^-24, k the top 24 bits of word 0, channel i the first
 * with u < alpha_0 + ... + alpha_i.  Needs ptcut_g > 0.
 *
 * mc_vegas_set_channels: alpha[3] (host, non-negative, positive sum;
 * normalised), default 1/3 each.  mc_vegas_get_channels: the current
 * alpha[3] and (w, may be NULL) the last iteration's update sums
 * W_i = (1/N) sum_events w^2 p_i / p.  mc_channel_update: one update
 * alpha_i <- alpha_i W_i^beta / sum_j alpha_j W_j^beta, then a floor amin
 * and renormalisation (host arithmetic, n <= 16).  mc_integrate applies it
 * (beta = 1/2, amin = 0.02) after every iteration of MC_GG_TTBARG_MC.
 */
int mc_vegas_set_channels(mc_vegas v, const double* alpha);
int mc_vegas_get_channels(mc_vegas v, double* alpha, double* w);
int mc_channel_update(int n, const double* alpha, const double* w, double beta, double amin, double* alpha_out);

/* ------------------------------------------------- unweighted events
 * Thesis Sec. "Unweighted event exporter" (acceptance-rejection as in
 * Sec. "Monte Carlo integration"): from a weighted sample with largest
 * weight w_max, event i is kept when w_i > r_i w_max, i.e. with probability
 * w_i / w_max; the kept events follow the integrand's distribution with unit
 * weight, and the efficiency is N_accepted / N_total.  r_i is Philox call 255
 * of the event's counter (ev lo, ev hi, iteration, gid | 255 << 8):
 * r = (2k + 1) / 2^53, k the top 52 bits of words 0:1.
 *
 * mc_event: one accepted event in the laboratory frame, the content of an
 * LHE <event> record.  Incoming a (+z) and b (-z) carry x1 sqrt(s)/2 and
 * x2 sqrt(s)/2; the outgoing momenta are the partonic-frame momenta boosted
 * along z by the rapidity ln(x1/x2)/2.  e+e- -> mu+mu-: a = e-, b = e+,
 * outgoing mu-, mu+, x1 = x2 = 1.  gg -> t tbar g: a = b = g, outgoing
 * t, tbar, g.  200 bytes, field order part of the ABI.
 */
typedef struct {
  int64_t event;     /* Philox event index within its iteration                */
  double weight;     /* its weight w = f J in the weighted sample (pb)         */
  double x1, x2;     /* momentum fractions of the incoming partons             */
  double p[5][4];    /* (E, px, py, pz) in GeV: a, b, outgoing 1..nout; rest 0 */
  int32_t proc;      /* MC_EE_MUMU, MC_GG_TTBARG or MC_GG_TTBARG_7D            */
  int32_t nout;      /* outgoing particles: 2 or 3                             */
} mc_event;

/* mc_vegas_iterate_weights: mc_vegas_iterate that also writes the weight of
 * every event to weights[0 .. nevents-1] (device, FP64; 0 for events outside
 * the cuts or with non-finite weight).  nevents < 2^32.  The sums, histograms
 * and iteration counter behave as in mc_vegas_iterate. */
int mc_vegas_iterate_weights(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, double* weights,
                             void* stream, mc_iter_result* out);

/* mc_unweight: the unweighted sample of the last iteration of v, which must
 * have been made by mc_vegas_iterate_weights with the same integrand and
 * nevents, and the grid unchanged since (no refine or set_grid in between;
 * EINVAL otherwise).  weights: that call's output (device).  wmax > 0: the
 * normalisation (normally out->wmax of that call; a smaller value keeps
 * every event above it, with its weight truncated).  The accepted events are
 * written in event order to events[0 .. capacity-1] (device); *n_accepted
 * (host) receives their number, which may exceed capacity (the surplus is
 * not written).  Supported: MC_EE_MUMU, MC_GG_TTBARG, MC_GG_TTBARG_7D (EINVAL
 * for other processes).  Device scratch, kept in the handle: 8 KB, one bit
 * per event and 4 bytes per event up to capacity.  Synchronises `stream` to
 * read the count. */
int mc_unweight(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, const double* weights, int64_t nevents, double wmax,
                mc_event* events, int64_t capacity, int64_t* n_accepted, void* stream);
/* Device time (ms) of the last mc_unweight's passes (CUDA events around them
 * on its stream). */
int mc_unweight_ms(mc_vegas v, float* ms);

/* Les Houches Event files (LHE 3.0: <LesHouchesEvents version="3.0">, an
 * <init> block and one <event> block per event), written by a native writer
 * thread so that the caller (and the GPU) never wait on text formatting or
 * the disk, as the thesis's LheWriter gathers events in a separate CPU
 * thread.  Events carry unit weight (IDWTUP = 3, XWGTUP = 1); the colour flow
 * of gg -> t tbar g is the leading-colour line g1(501,502) g2(503,504) ->
 * t(501,0) tbar(0,504) g(503,502); particle masses are the nominal ones
 * (m_top, 0).  Each event ends with a comment line "# mcint <event index>
 * <weight>".
 *
 * mc_lhe_open: creates the file (header and a placeholder <init> block) and
 * starts the writer with `threads` (1..64) formatting threads.
 * mc_lhe_write: queues n host events (copied before return).
 * mc_lhe_write_device: queues n device events: an asynchronous copy on
 * `stream` into a pinned buffer of the writer, formatted once the copy has
 * completed; returns without waiting for it.  Later work on `stream` is
 * ordered after the copy, so the device buffer may be reused by it.
 * Both block only while 4 batches are already queued.
 * mc_lhe_close: drains the queue, writes the closing tag, fills the <init>
 * block with the cross-section, its error and the largest weight (pb), and
 * closes the file; *n_written (may be NULL) receives the number of events.
 * The handle is freed even on error.
 */
typedef struct mc_lhe_s* mc_lhe;
int mc_lhe_open(const char* path, const mc_integrand* itg, int threads, mc_lhe* out);
int mc_lhe_write(mc_lhe w, const mc_event* events, int64_t n);
int mc_lhe_write_device(mc_lhe w, const mc_event* events, int64_t n, void* stream);
int mc_lhe_close(mc_lhe w, double xsec, double xerr, double wmax, int64_t* n_written);

/* mc_generate_lhe: event generation as the thesis's MadFlow run: ntrain
 * VEGAS iterations of nevents that adapt the grid (refinement with damping
 * alpha), then niter iterations of nevents on the frozen grid, each one a
 * weights pass, its unweighting with that iteration's w_max, and the export
 * of the accepted events to the LHE file `path` while the next iteration
 * runs.  out: the inverse-variance combination of the niter frozen
 * iterations (the cross-section written to <init>).  stats (may be NULL):
 * events evaluated and written, device times, host wall time. */
typedef struct {
  int64_t n_weighted;   /* events evaluated in the export iterations           */
  int64_t n_accepted;   /* unweighted events written                           */
  double iterate_ms;    /* device time of the weights passes                   */
  double unweight_ms;   /* device time of the unweighting passes               */
  double wall_ms;       /* host time of the export iterations until closed     */
} mc_gen_stats;
int mc_generate_lhe(const mc_integrand* itg, mc_pdf pdf, int ntrain, int niter, int64_t nevents, int nbins,
                    uint64_t seed, int prec, double alpha, const char* path, int threads, void* stream,
                    mc_result* out, mc_gen_stats* stats);

/* ------------------------------------------------------------ debugging
 * mc_debug_events: per-event intermediates of events first..first+k-1 of
 * the current iteration (the counter is not advanced and no sums or
 * histograms change), written to out (device, FP64, [k][MC_REC_STRIDE]).
 * Used by the parity tests.
 */
#define MC_REC_K 0        /* 16: integer uniforms (exact in FP64)               */
#define MC_REC_X 16       /* 16: mapped point x                                 */
#define MC_REC_BIN 32     /* 16: VEGAS bin per dimension                        */
#define MC_REC_JAC 48     /* VEGAS Jacobian                                     */
#define MC_REC_P 49       /* 7 x 4: incoming a, b, outgoing momenta, CM frame    */
#define MC_REC_X1 77
#define MC_REC_X2 78
#define MC_REC_SHAT 79
#define MC_REC_LUMI 80    /* f_g(x1) f_g(x2), or 1 for e+e-                      */
#define MC_REC_LUMI_QQ 81 /* sum_q f_q f_qbar + f_qbar f_q (pp -> tt)            */
#define MC_REC_ME2 82     /* averaged |M|^2 (gg channel for pp -> tt)            */
#define MC_REC_ME2_QQ 83  /* averaged |M|^2 of q qbar -> tt                      */
#define MC_REC_PSW 84     /* phase-space weight per unit hypercube               */
#define MC_REC_F 85       /* integrand value, pb                                 */
#define MC_REC_W 86       /* event weight f * J                                  */
#define MC_REC_PASS 87    /* 1 inside cuts and thresholds, else 0                */
#define MC_REC_STATUS 88  /* 0, or MC_ENAN / MC_ENOCONV                          */
#define MC_REC_CHANNEL 89 /* three-channel process: the event's channel          */
#define MC_REC_DENS 90    /* 3: the channels' densities at the event's point     */
#define MC_REC_ME2_X 89   /* p p -> t tbar + parton: 5 averaged |M|^2 of q qbar   */
                          /* (quark from beam b), q g, g q, qbar g, g qbar         */
                          /* (slots 89.. shared with the three-channel entries)   */
#define MC_REC_STRIDE 96
int mc_debug_events(mc_vegas v, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t k,
                    double* out, void* stream);

/* Device time (ms) of the fused integrand kernel launched by the last
 * mc_vegas_iterate on this handle, from CUDA events recorded on the caller's
 * stream immediately around that launch (0 if no events were evaluated). */
int mc_vegas_kernel_ms(mc_vegas v, float* ms);

/* Number of SMs of the current device and the kernel launch shape the
 * library would use for a process (blocks, threads per block). */
int mc_launch_shape(const mc_integrand* itg, int prec, int64_t nevents, int* blocks, int* threads);

/* FMA throughput of the CUDA cores, the denominator of the integrand
 * kernels' roofline (measured rather than derived from unit counts; the
 * thesis has no counterpart).  Launches, asynchronously on `stream`, a
 * full-occupancy grid (SMs x max threads per SM / 256 blocks of 256 threads)
 * whose every thread runs 8 independent chains of `iters` dependent fused
 * multiply-adds: kind 0 fma.rn.f32, kind 1 fma.rn.f32x2 (packed pairs),
 * kind 2 fma.rn.f64.  *flop receives the launch's floating-point operations
 * (2 per FMA lane operation); the caller times the launch with events on
 * `stream`.  out (device, caller-owned) receives one float per thread:
 * out_len must be at least the grid's thread count (EINVAL otherwise). */
int mc_fma_peak(int kind, int iters, float* out, int64_t out_len, double* flop, void* stream);

/* ---------------------------------------------------------------- batches
 * Many integrands of uneven dimension and event count in one persistent
 * launch per iteration.  The thesis evaluates one integrand at a time over
 * vectors of events (Sec. "Software design and benchmarks"); here every
 * integrand keeps its own VEGAS grid, Philox stream (gid = its index) and
 * histograms, and one iteration of all of them is: the persistent kernel
 * (blocks pull (integrand, event range) tiles from an atomic counter,
 * heaviest integrands first), a fixed-order reduction per integrand, the
 * refinement of every grid, and the advance of the iteration counter, all
 * captured once in a CUDA graph and replayed.  The first mc_batch_iterate
 * autotunes the launch: it times one pass for each block size in {64, 128,
 * 256} and events per thread in {2, 8, 32} (results discarded) and keeps the
 * fastest.
 *
 * mc_batch_create: n (1..256) integrands itgs[n] and event counts nevents[n]
 * (host), the PDF (needed if any integrand is hadronic; all hadronic
 * integrands must share mu_f), nbins, seed, precision.  Grids start uniform.
 * mc_batch_iterate: one iteration of all integrands with damping alpha;
 * out[n] (host) receives the sums; synchronises `stream`.  Do not call it
 * while `stream` is being captured.
 * mc_batch_get_grid: the current grid of integrand i, [ndim_i][nbins+1] host.
 * mc_batch_shape: the launch shape chosen by the autotuner.
 * mc_batch_kernel_ms: device time of the last persistent launch.
 */
typedef struct mc_batch_s* mc_batch;
int mc_batch_create(int n, const mc_integrand* itgs, const int64_t* nevents, mc_pdf pdf, int nbins, uint64_t seed,
                    int prec, mc_batch* out);
int mc_batch_iterate(mc_batch b, double alpha, void* stream, mc_iter_result* out);
int mc_batch_get_grid(mc_batch b, int i, double* edges);
int mc_batch_shape(mc_batch b, int* block, int* events_per_thread, int* grid, int* ntiles);
int mc_batch_kernel_ms(mc_batch b, float* ms);
int mc_batch_free(mc_batch b);

/* ------------------------------------------------ tensor-core dense layer
 * mc_gemm_bf16: the dense-layer contraction of the flow sampler's
 * conditioner (thesis Sec. "Deep learning": dense layer y = phi(W x + b)) on
 * the tcgen05 tensor cores: C[M x N] (+)= A[M x K] . B[N x K]^T with A and B
 * BF16 row-major (device; leading dimensions lda, ldb multiples of 8,
 * 16-byte aligned), FP32 accumulation, and the epilogue:
 *   0: C (BF16) = relu(acc + bias)      1: C (FP32) = acc + bias (bias may be NULL)
 *   2: C (BF16) = acc * [mask > 0]       3: C (FP32) += acc (split-K over `splits`)
 *   4: C (FP32) [splits][M][ldc]: the partial product of each K split
 * M % 128 == 0, K % 64 == 0, bn (the N tile) a multiple of 16 <= 256 that
 * divides N.  err: device int set non-zero if a bounded wait inside the kernel
 * timed out (the result is then invalid).  Asynchronous on `stream`.
 */
int mc_gemm_bf16(int M, int N, int K, int bn, int epilogue, const void* a, int lda, const void* b, int ldb,
                 const float* bias, void* c, int ldc, const void* mask, int ld_mask, int splits, int* err,
                 void* stream);
/* mc_gemm_bf16_tn: C[M x N] (+)= X^T Y with X [K x M] and Y [K x N]
 * row-major BF16 (device; leading dimensions ldx >= M, ldy >= N, multiples
 * of 8): the weight gradient of a dense layer from row-major activations and
 * gradients, both operands read MN-major by the tensor cores.  Epilogue 1
 * (C = acc), 3 (C += acc, split-K) or 4 (per-split partials as above);
 * M % 128 == 0, K % 64 == 0, bn a multiple of 64 <= 256 dividing N.
 * Asynchronous on `stream`. */
int mc_gemm_bf16_tn(int M, int N, int K, int bn, int epilogue, const void* x, int ldx, const void* y, int ldy,
                    float* c, int ldc, int splits, int* err, void* stream);
/* mc_gemm_bf16_xn: C[M x N] (+)= X^T B^T with X [K x M] row-major (ldx >= M)
 * and B [N x K] row-major (ldb >= K), BF16 on the device (leading dimensions
 * multiples of 8, 16-byte aligned): the weight gradient of a dense layer from
 * row-major activations X and transposed gradients B, X read MN-major and B
 * K-major by the tensor cores.  Epilogues 1, 3, 4 as for mc_gemm_bf16_tn;
 * M % 128 == 0, K % 64 == 0, bn a multiple of 16 <= 256 dividing N.
 * Asynchronous on `stream`. */
int mc_gemm_bf16_xn(int M, int N, int K, int bn, int epilogue, const void* x, int ldx, const void* b, int ldb,
                    float* c, int ldc, int splits, int* err, void* stream);
/* mc_gemm_bf16_rs: the same product for a long A and a short B (a dense
 * layer applied to a batch): a persistent kernel keeps B in shared memory
 * (bn * K * 2 bytes, K <= 320) and streams the 128-row tiles of A, with the
 * epilogue of one tile overlapping the MMAs of the next.  Epilogues 0-2 as
 * above.  c (row-major, ldc) and/or c_t (the transpose, c_t[col * ldt + row],
 * ldt >= M) receive the result; either may be NULL, not both.  Asynchronous. */
int mc_gemm_bf16_rs(int M, int N, int K, int bn, int epilogue, const void* a, int lda, const void* b, int ldb,
                    const float* bias, void* c, int ldc, void* c_t, int ldt, const void* mask, int ld_mask, int* err,
                    void* stream);

/* ------------------------------------------- allocation-free iteration
 * mc_vegas_iterate_noalloc: the same fused iteration as mc_vegas_iterate, for
 * callers that must not allocate device memory while they run: code whose
 * device memory is owned by another pool (an application or framework
 * allocator that has reserved the device), and latency-critical loops where
 * a cudaMalloc/cudaFree could synchronise the device.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  The thesis has no
 * counterpart; this is an operational variant of the same kernel.
 *
 * Scratch: the per-block partial sums live in a file-scope device array of
 * MC_NOALLOC_MAX_BLOCKS entries (64 B each, 256 KiB) that every device which
 * loads this library holds until the process exits.  The first call on a
 * device looks up the array's device address with that device current
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array: calls whose launches overlap on the GPU race
 * (serialise them on one stream).  Each launch writes every slot it later
 * reads, so nothing in the array needs clearing between calls.
 *
 * Processes: MC_EE_MUMU, MC_PP_TTBAR, MC_GG_TTBARG, MC_GAUSS,
 * MC_GG_TTBARG_7D and MC_PP_TTBARJ, validated exactly as mc_vegas_iterate
 * validates them.  MC_GG_TTBARG_MC is rejected with EINVAL: its channel
 * probabilities and update sums belong to a VEGAS handle.
 *
 * Inputs (caller-owned): itg (host), pdf (an mc_pdf loaded earlier, or NULL
 * for processes without hadrons), the grid as device arrays edges64 (FP64)
 * and, for MC_FP32_KAHAN, edges32 (FP32), both [ndim][nbins+1]; seed,
 * iteration and gid form the Philox counter as in mc_vegas_iterate.
 * blocks = 0 lets the library choose the launch (at most
 * MC_NOALLOC_MAX_BLOCKS blocks); a larger request is rejected with EINVAL.
 * Outputs (device, caller-owned): hist_w2[ndim][nbins] and
 * hist_n[ndim][nbins] are accumulated into (zero them to start a fresh
 * histogram); *sums receives the compensated sums of the launch.
 * Asynchronous on `stream`; the outputs are valid once the stream reaches
 * the end of the call.  There is no status word: if a bounded wait inside
 * the warp-specialised FP32 gg -> t tbar g kernel gives up (where
 * mc_vegas_iterate returns MC_ETIMEOUT), the call still returns MC_OK and
 * the timeout shows in *sums as sum_hi = sum2_hi = NaN with n_bad increased
 * by one per block that gave up.
 */
#define MC_NOALLOC_MAX_BLOCKS 4096
typedef struct {
  double sum_hi, sum_lo;    /* sum of w = sum_hi + sum_lo                       */
  double sum2_hi, sum2_lo;  /* sum of w^2                                       */
  double wmax;
  int64_t n_nonzero, n_bad, n_noconv;
} mc_device_sums;
int mc_vegas_iterate_noalloc(const mc_integrand* itg, mc_pdf pdf, int ndim, int nbins, const double* edges64,
                             const float* edges32, int prec, uint64_t seed, uint32_t iteration, uint32_t gid,
                             int64_t nevents, int blocks, double* hist_w2, uint32_t* hist_n, mc_device_sums* sums,
                             void* stream);

/* ------------------------------------------------ normalizing-flow sampler
 * Importance sampling with a trained density q (thesis Sec. "Importance
 * sampling": E = (1/N) sum f(x_i)/q(x_i), variance minimal for q ~ |f|), the
 * density being a normalizing flow built from dense layers y = phi(W x + b)
 * (Sec. "Deep learning") and trained with Adam (Sec. "Optimizers").  The
 * flow is a stack of piecewise-quadratic coupling layers on the unit cube:
 * layer l transforms the coordinates d with d % 2 == l % 2; its conditioner
 * maps u = 2 x_A - 1 through dense layers of `hidden` units with ReLU to
 * 2 * bins + 1 logits per transformed coordinate (bins width logits ->
 * softmax; bins + 1 vertex-height logits -> exp, normalised to unit area).
 * Every dense layer runs on the tcgen05 tensor cores with BF16 weights and
 * activations and FP32 accumulation; the first layer's bias b1 enters as a
 * BF16 weight on a constant input of one (b2..b4 are added in FP32); the
 * splines and log-determinants are FP32.
 *
 * Parameters (host, packed FP32): for each layer in order, W1 [hidden x n_A],
 * b1 [hidden], W2 [hidden x hidden], b2, W3 [hidden x hidden], b3,
 * W4 [n_B (2 bins + 1) x hidden], b4 [n_B (2 bins + 1)], matrices row-major
 * [out x in]; n_B = number of transformed coordinates, n_A = ndim - n_B.
 * mc_flow_param_count gives the total.
 */
typedef struct mc_flow_s* mc_flow;
typedef struct {
  int ndim;    /* 2..16 */
  int layers;  /* 1..16 coupling layers */
  int bins;    /* 2..32 spline bins */
  int hidden;  /* must be 256 */
} mc_flow_cfg;

/* Number of FP32 parameters of a flow of configuration cfg. */
int mc_flow_param_count(const mc_flow_cfg* cfg, int64_t* n);
/* Creates a flow on the current device with parameters `init` (host, packed,
 * copied), workspace for batches of up to max_batch events, and `seed` as
 * the Philox key of its uniforms; 1 <= max_batch <= 2^21.  Device memory: about
 * max_batch * layers * (6 hidden + 4 * 2 * ndim * (2 bins + 1)) bytes. */
int mc_flow_create(const mc_flow_cfg* cfg, const float* init, int64_t max_batch, uint64_t seed, mc_flow* out);
int mc_flow_free(mc_flow f);
/* Replace / read the parameters (host, packed).  Set resets nothing else
 * (Adam moments and the step counter are kept).  Both synchronise. */
int mc_flow_set_params(mc_flow f, const float* host);
int mc_flow_get_params(mc_flow f, float* host);
/* Choose between the fused and the layer-by-layer kernels of the flow.
 * mask bit 0: the forward direction (mc_flow_forward, mc_flow_iterate and
 * the sampling half of mc_flow_train) runs each coupling layer as one fused
 * kernel (dense layers on the tensor cores with the activations kept in
 * shared and tensor memory, spline in the epilogue); bit 1: the backward
 * (mc_flow_loss_grad, mc_flow_train) runs the spline and activation
 * gradients of each layer as one fused kernel.  Both apply where bins == 32
 * and a layer transforms at most 6 coordinates; elsewhere, or with the bit
 * clear, the layer-by-layer kernels run.  Default 3.  Both implementations
 * compute the same numbers. */
int mc_flow_set_fused(mc_flow f, int mask);
/* Sampling direction: z [n x ndim] (device, uniform in the unit cube) ->
 * x [n x ndim] (device) and log q(x) [n] (device); n <= max_batch.
 * Synchronises (to read the tensor-core error flag). */
int mc_flow_forward(mc_flow f, int64_t n, const float* z, float* x, float* log_q, void* stream);
/* Loss L = -sum w_i log q(x_i) / sum w_i at fixed points x [n x ndim] and
 * weights w [n] (device), q evaluated through the inverse pass; *loss
 * (host, may be NULL) receives L and grads (host, packed like the
 * parameters, may be NULL) dL/dtheta.  Leaves the gradients in place for
 * mc_flow_adam_step.  Synchronises. */
int mc_flow_loss_grad(mc_flow f, int64_t n, const float* x, const float* w, double* loss, float* grads,
                      void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * gradients of the last loss evaluation, then refreshes the BF16 weights. */
int mc_flow_adam_step(mc_flow f, double lr, void* stream);
/* `steps` online training steps on the integrand: each samples `batch`
 * events from the current flow (Philox counter iteration 0x10000 + step),
 * evaluates f in FP32 at them, forms w = |f| / q, and takes one loss
 * gradient and Adam step.  losses (host, may be NULL) receives each step's
 * loss; without it the call is asynchronous except for a final error-flag
 * check.  The flow's ndim must equal the process's. */
int mc_flow_train(mc_flow f, const mc_integrand* itg, mc_pdf pdf, int steps, int64_t batch, double lr,
                  void* stream, double* losses);
/* One training step of mc_flow_train split across devices (data parallel;
 * the loss is a sum over the batch's events, so its gradient is a sum of
 * per-device parts, thesis Sec. "Optimizers" applied to the importance-
 * sampling loss).  Every rank holds a flow with the same parameters, seed
 * and step count; rank r of W:
 *   1. mc_flow_step_sample(f, itg, pdf, first, count, stream, &wsum):
 *      samples events [first, first + count) of the step's batch (the same
 *      Philox counters as mc_flow_train's single-device batch), keeps the
 *      activations, evaluates f and w = |f| / q; *wsum (host) receives this
 *      share's sum of w.  Synchronises.  count <= max_batch.
 *   2. the ranks add their wsum (an all-reduce of one double);
 *   3. mc_flow_step_grads(f, wsum_total, grads, stream): the gradient of
 *      this share's part of L = -sum w log q / wsum_total into grads (device,
 *      caller-owned, mc_flow_grad_count floats in the library's internal
 *      parameter order; NULL keeps it in place).  Asynchronous.
 *   4. the ranks add their grads (an all-reduce of mc_flow_grad_count floats);
 *   5. mc_flow_step_apply(f, grads, lr, stream): installs the summed
 *      gradient (NULL: the one in place) and takes the Adam step, advancing
 *      the step counter.  Asynchronous.
 * With one rank (first 0, count = batch, wsum_total = wsum, grads NULL) the
 * three calls perform exactly the arithmetic of one mc_flow_train step. */
int mc_flow_grad_count(mc_flow f, int64_t* n);
int mc_flow_step_sample(mc_flow f, const mc_integrand* itg, mc_pdf pdf, int64_t first, int64_t count, void* stream,
                        double* wsum);
int mc_flow_step_grads(mc_flow f, double wsum_total, float* grads, void* stream);
int mc_flow_step_apply(mc_flow f, const float* grads, double lr, void* stream);
/* One sampling pass of nevents events from the flow (Philox counter
 * iteration 0x20000 + iteration), in chunks of max_batch: weights
 * w = f(x)/q(x) accumulated in compensated FP64 into *out (host); events
 * whose integrand failed or is non-finite count in n_bad with w = 0. */
int mc_flow_iterate(mc_flow f, const mc_integrand* itg, mc_pdf pdf, int64_t nevents, uint32_t iteration,
                    void* stream, mc_iter_result* out);

/* mc_integrate_flow: the integral with the flow as importance sampler and
 * plain VEGAS as its judge and fallback.  One FP32 VEGAS iteration of
 * nevents on a fresh nbins grid (then refined) measures VEGAS's variance per
 * event; the flow (configuration cfg, parameters init) is trained online
 * (train_steps Adam steps of train_batch events, learning rate lr) and runs
 * one iteration of nevents.  The flow is used (*sampler = 1) when its
 * training loss and its iteration are finite and its relative variance per
 * event does not exceed VEGAS's; otherwise VEGAS continues (*sampler = 0).
 * Iterations of the chosen sampler follow until the combined relative error
 * is at most target (0: no target) or niter of them have run; every
 * iteration, the judge's included, enters the inverse-variance combination
 * (each is unbiased).  out->gpu_ms covers everything from the first launch
 * (the judge's iteration) to the end; the set-up before it (the judge's grid,
 * the flow's buffers and initial parameters) is not timed, as in
 * mc_integrate.  Synchronises. */
int mc_integrate_flow(const mc_integrand* itg, mc_pdf pdf, const mc_flow_cfg* cfg, const float* init,
                      int train_steps, int64_t train_batch, double lr, int niter, int64_t nevents, int nbins,
                      uint64_t seed, double target_rel_err, void* stream, mc_result* out, int* sampler);

#ifdef __cplusplus
}
#endif
#endif /* MCINT_H */
