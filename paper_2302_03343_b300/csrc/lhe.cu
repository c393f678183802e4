// Les Houches Event output (LHE 3.0) with a native writer thread, and the
// event-generation driver (thesis Sec. "Unweighted event exporter": the
// weighted events are gathered asynchronously to the |M|^2 computation and
// dumped as LHE tags by a separate CPU thread, so that the host-device
// traffic and the text formatting do not hold up the device).
//
// The writer owns a queue of at most kLhePending batches.  A batch is either
// host events (copied when queued) or device events copied on the caller's
// stream into one of kLhePending pinned staging buffers; the writer thread
// waits for that copy with a blocking-sync CUDA event, formats the batch in
// parallel slices (one string per formatting thread) and appends the slices
// to the file in order, so the file does not depend on the thread count.
// The <init> block's cross-section line is written as a fixed-width
// placeholder when the file is opened and filled in place when it is closed.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mcint.h"
#include "handles.h"

namespace {

constexpr int kLhePending = 4;
constexpr int kInitWidth = 80;  // characters of the placeholder cross-section line, before its newline

int lfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  mc::set_last_error(buf);
  return code;
}

struct LheBatch {
  std::vector<mc_event> host;  // host batch
  int pinned = -1;             // or the index of the staging buffer
  int64_t n = 0;
};

struct Staging {
  mc_event* p = nullptr;
  size_t cap = 0;
  bool busy = false;
  cudaEvent_t ready = nullptr;
};

// Writes v in the layout of printf's "%+.10e" (sign, d.dddddddddd, 'e',
// exponent sign, at least two exponent digits) and returns the end.  The
// eleven significant digits are llround(|v| 10^(10 - e)) with e the decimal
// exponent, the scaling done in double precision by exact powers of ten
// (|e| <= 22), so the last digit can differ from exact decimal rounding when
// |v| lies within a few units of 1e-16 (relative) of a rounding boundary.
// Non-finite values go through snprintf.
char* put_e10(char* o, double v) {
  static const double p10[23] = {1e0,  1e1,  1e2,  1e3,  1e4,  1e5,  1e6,  1e7,  1e8,  1e9,  1e10, 1e11,
                                 1e12, 1e13, 1e14, 1e15, 1e16, 1e17, 1e18, 1e19, 1e20, 1e21, 1e22};
  if (!std::isfinite(v)) return o + snprintf(o, 32, "%+.10e", v);
  *o++ = std::signbit(v) ? '-' : '+';
  const double a = std::fabs(v);
  if (a == 0.0) {
    std::memcpy(o, "0.0000000000e+00", 16);
    return o + 16;
  }
  int e = int(std::floor(std::log10(a)));
  auto digits = [&](int ex) {
    int k = 10 - ex;  // |v| 10^k has eleven digits before the point
    double m = a;
    if (k > 22 || k < -22) {  // outside the exact powers: steps of at most 10^200, no overflow
      while (k > 200) {
        m *= 1e200;
        k -= 200;
      }
      while (k < -200) {
        m /= 1e200;
        k += 200;
      }
      m = k >= 0 ? m * std::pow(10.0, k) : m / std::pow(10.0, -k);
    } else {
      m = k >= 0 ? m * p10[k] : m / p10[-k];
    }
    return (unsigned long long)std::llround(m);
  };
  unsigned long long d = digits(e);
  if (d >= 100000000000ull) d = digits(++e);  // log10 fell short, or rounding carried
  if (d < 10000000000ull) d = digits(--e);    // log10 overshot
  if (d >= 100000000000ull) {                 // the carry case of the retry: 9.99...95 -> 10
    d = 10000000000ull;
    ++e;
  }
  char dig[11];
  for (int i = 10; i >= 0; --i) {
    dig[i] = char('0' + d % 10);
    d /= 10;
  }
  *o++ = dig[0];
  *o++ = '.';
  std::memcpy(o, dig + 1, 10);
  o += 10;
  *o++ = 'e';
  *o++ = e < 0 ? '-' : '+';
  const int ae = e < 0 ? -e : e;
  if (ae >= 100) *o++ = char('0' + ae / 100);
  *o++ = char('0' + (ae / 10) % 10);
  *o++ = char('0' + ae % 10);
  return o;
}

// One particle line: IDUP ISTUP MOTHUP(1,2) ICOLUP(1,2) PUP(1..5) VTIMUP
// SPINUP; the integer part of a particle slot is fixed and formatted once.
struct ParticleSlot {
  char head[48];
  int len;
  ParticleSlot(int id, int status, int m1, int m2, int c1, int c2) {
    len = snprintf(head, sizeof(head), " %8d %2d %4d %4d %4d %4d", id, status, m1, m2, c1, c2);
  }
};

void put_particle(std::string& s, const ParticleSlot& slot, const double* p, double mass) {
  char line[160];
  char* o = line;
  std::memcpy(o, slot.head, size_t(slot.len));
  o += slot.len;
  const double v[5] = {p[1], p[2], p[3], p[0], mass};
  for (double x : v) {
    *o++ = ' ';
    o = put_e10(o, x);
  }
  std::memcpy(o, " 0. 9.\n", 7);
  o += 7;
  s.append(line, size_t(o - line));
}

}  // namespace

struct mc_lhe_s {
  FILE* f = nullptr;
  long init_pos = 0;
  int threads = 1, device = 0;
  int proc = 0;
  double scale = 0.0, aqed = 0.0, aqcd = 0.0, m_top = 0.0;
  std::thread writer;
  std::mutex m;
  std::condition_variable cv_work, cv_space;
  std::deque<LheBatch> q;
  bool closing = false;
  int in_flight = 0;  // batches queued or being formatted
  Staging pool[kLhePending];
  int64_t written = 0;
  int error = MC_OK;
  std::string err_msg;
  std::vector<std::string> parts;  // formatted slices of the current batch (writer thread only)

  void append_event(std::string& s, const mc_event& e) const {
    // e+e- -> mu+mu-, and g g -> t tbar g with the leading-colour flow
    // g1(501,502) g2(503,504) -> t(501,0) tbar(0,504) g(503,502)
    static const ParticleSlot ee[4] = {{11, -1, 0, 0, 0, 0}, {-11, -1, 0, 0, 0, 0}, {13, 1, 1, 2, 0, 0},
                                       {-13, 1, 1, 2, 0, 0}};
    static const ParticleSlot gg[5] = {{21, -1, 0, 0, 501, 502}, {21, -1, 0, 0, 503, 504}, {6, 1, 1, 2, 501, 0},
                                       {-6, 1, 1, 2, 0, 504}, {21, 1, 1, 2, 503, 502}};
    char line[160];
    int k = snprintf(line, sizeof(line), "<event>\n %d 1 +1.0000000000e+00", 2 + e.nout);
    char* o = line + k;
    for (double x : {scale, aqed, aqcd}) {
      *o++ = ' ';
      o = put_e10(o, x);
    }
    *o++ = '\n';
    s.append(line, size_t(o - line));
    if (proc == MC_EE_MUMU) {
      for (int i = 0; i < 4; ++i) put_particle(s, ee[i], e.p[i], 0.0);
    } else {
      for (int i = 0; i < 5; ++i) put_particle(s, gg[i], e.p[i], i == 2 || i == 3 ? m_top : 0.0);
    }
    k = snprintf(line, sizeof(line), "# mcint %lld ", (long long)e.event);
    o = put_e10(line + k, e.weight);
    std::memcpy(o, "\n</event>\n", 10);
    o += 10;
    s.append(line, size_t(o - line));
  }

  // Formats events[0 .. n) in `threads` slices, one string each (kept
  // between batches), and appends them in order; slice t is written while
  // the slices after it are still being formatted.
  void format_and_write(const mc_event* ev, int64_t n) {
    const int T = int(std::min<int64_t>(threads, std::max<int64_t>(1, n / 256)));
    if (int(parts.size()) < T) parts.resize(size_t(T));
    auto work = [&](int t) {
      const int64_t lo = n * t / T, hi = n * (t + 1) / T;
      std::string& s = parts[size_t(t)];
      s.clear();
      s.reserve(size_t(hi - lo) * 1024);
      for (int64_t i = lo; i < hi; ++i) append_event(s, ev[i]);
    };
    auto put = [&](const std::string& s) {
      if (fwrite(s.data(), 1, s.size(), f) != s.size()) {
        std::lock_guard<std::mutex> lk(m);
        if (!error) {
          error = MC_EIO;
          err_msg = "mc_lhe: short write";
        }
      }
    };
    std::vector<std::thread> pool_threads;
    for (int t = 1; t < T; ++t) pool_threads.emplace_back(work, t);
    work(0);
    put(parts[0]);
    for (int t = 1; t < T; ++t) {
      pool_threads[size_t(t - 1)].join();
      put(parts[size_t(t)]);
    }
  }

  void run() {
    bool on_device = false;  // the CUDA device is selected for this thread at the first device batch
    for (;;) {
      LheBatch b;
      {
        std::unique_lock<std::mutex> lk(m);
        cv_work.wait(lk, [&] { return closing || !q.empty(); });
        if (q.empty()) break;
        b = std::move(q.front());
        q.pop_front();
      }
      const mc_event* ev = b.host.data();
      bool ok = true;
      if (b.pinned >= 0) {
        if (!on_device) on_device = cudaSetDevice(device) == cudaSuccess;
        const cudaError_t e = cudaEventSynchronize(pool[b.pinned].ready);
        if (e != cudaSuccess) {
          ok = false;
          std::lock_guard<std::mutex> lk(m);
          if (!error) {
            error = MC_ECUDA;
            err_msg = std::string("mc_lhe: device copy: ") + cudaGetErrorString(e);
          }
        }
        ev = pool[b.pinned].p;
      }
      if (ok && b.n > 0) format_and_write(ev, b.n);
      {
        std::lock_guard<std::mutex> lk(m);
        if (b.pinned >= 0) pool[b.pinned].busy = false;
        if (ok) written += b.n;
        --in_flight;
      }
      cv_space.notify_all();
    }
  }
};

namespace {

void write_init_line(FILE* f, double xsec, double xerr, double wmax) {
  char line[kInitWidth + 2];
  int k = snprintf(line, sizeof(line), " %+.10e %+.10e %+.10e 1", xsec, xerr, wmax);
  if (k < 0) k = 0;
  for (; k < kInitWidth; ++k) line[k] = ' ';
  line[kInitWidth] = '\n';
  fwrite(line, 1, kInitWidth + 1, f);
}

}  // namespace

extern "C" {

int mc_lhe_open(const char* path, const mc_integrand* itg, int threads, mc_lhe* out) {
  if (!out) return lfail(MC_EINVAL, "mc_lhe_open: out is NULL");
  *out = nullptr;
  if (!path || !itg || threads < 1 || threads > 64) return lfail(MC_EINVAL, "mc_lhe_open: bad arguments");
  if (itg->proc != MC_EE_MUMU && itg->proc != MC_GG_TTBARG && itg->proc != MC_GG_TTBARG_7D &&
      itg->proc != MC_GG_TTBARG_MC)
    return lfail(MC_EINVAL, "mc_lhe_open: process %d has no event record", itg->proc);
  FILE* f = fopen(path, "wb");
  if (!f) return lfail(MC_EIO, "mc_lhe_open: cannot create %s", path);
  auto* w = new mc_lhe_s;
  w->f = f;
  w->threads = threads;
  if (cudaGetDevice(&w->device) != cudaSuccess) w->device = 0;
  w->proc = itg->proc;
  w->m_top = itg->m_top;
  const bool ee = itg->proc == MC_EE_MUMU;
  w->scale = ee ? itg->sqrt_s : itg->mu_f;
  w->aqed = itg->alpha;
  w->aqcd = ee ? 0.0 : itg->alpha_s;
  const double eb = itg->sqrt_s / 2.0;
  fprintf(f, "<LesHouchesEvents version=\"3.0\">\n<header>\n<!--\n");
  if (ee)
    fprintf(f, " process: e- e+ > mu- mu+ (gamma + Z), sqrt(s) = %.6g GeV, alpha = %.8g, MZ = %.6g, GZ = %.6g\n",
            itg->sqrt_s, itg->alpha, itg->mz, itg->gz);
  else
    fprintf(f,
            " process: g g > t t~ g (%s), sqrt(s) = %.6g GeV, m_top = %.6g, alpha_s = %.6g, mu_F = %.6g,\n"
            " gluon pT > %.6g GeV, |eta| < %.6g\n",
            itg->proc == MC_GG_TTBARG ? "RAMBO" : (itg->proc == MC_GG_TTBARG_7D ? "hierarchical 2 -> 3" : "three channels"),
            itg->sqrt_s, itg->m_top, itg->alpha_s,
            itg->mu_f, itg->ptcut_g, itg->etacut_g);
  fprintf(f, " unweighted events: w_i > r_i w_max (acceptance-rejection), unit weights\n-->\n</header>\n<init>\n");
  fprintf(f, " %d %d %+.10e %+.10e 0 0 0 0 3 1\n", ee ? 11 : 2212, ee ? -11 : 2212, eb, eb);
  w->init_pos = ftell(f);
  write_init_line(f, 0.0, 0.0, 0.0);
  fprintf(f, "</init>\n");
  if (ferror(f)) {
    fclose(f);
    delete w;
    return lfail(MC_EIO, "mc_lhe_open: write failed on %s", path);
  }
  w->writer = std::thread([w] { w->run(); });
  *out = w;
  return MC_OK;
}

int mc_lhe_write(mc_lhe w, const mc_event* events, int64_t n) {
  if (!w || n < 0 || (n > 0 && !events)) return lfail(MC_EINVAL, "mc_lhe_write: bad arguments");
  if (n == 0) return MC_OK;
  LheBatch b;
  b.host.assign(events, events + n);
  b.n = n;
  {
    std::unique_lock<std::mutex> lk(w->m);
    w->cv_space.wait(lk, [&] { return w->in_flight < kLhePending; });
    if (w->error) return lfail(w->error, "%s", w->err_msg.c_str());
    ++w->in_flight;
    w->q.push_back(std::move(b));
  }
  w->cv_work.notify_one();
  return MC_OK;
}

int mc_lhe_write_device(mc_lhe w, const mc_event* events, int64_t n, void* stream) {
  if (!w || n < 0 || (n > 0 && !events)) return lfail(MC_EINVAL, "mc_lhe_write_device: bad arguments");
  if (n == 0) return MC_OK;
  int slot = -1;
  {
    std::unique_lock<std::mutex> lk(w->m);
    w->cv_space.wait(lk, [&] { return w->in_flight < kLhePending; });
    if (w->error) return lfail(w->error, "%s", w->err_msg.c_str());
    // in_flight < kLhePending batches hold staging buffers, so one is free
    for (int i = 0; i < kLhePending; ++i)
      if (!w->pool[i].busy) {
        slot = i;
        break;
      }
    w->pool[slot].busy = true;
    ++w->in_flight;
  }
  Staging& sg = w->pool[slot];
  auto release = [&](int code, const char* what, cudaError_t e) {
    {
      std::lock_guard<std::mutex> lk(w->m);
      sg.busy = false;
      --w->in_flight;
    }
    w->cv_space.notify_all();
    return lfail(code, "mc_lhe_write_device: %s: %s", what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if (size_t(n) > sg.cap) {
    if (sg.p) cudaFreeHost(sg.p);
    sg.p = nullptr;
    sg.cap = 0;
    if ((e = cudaMallocHost(&sg.p, sizeof(mc_event) * size_t(n))) != cudaSuccess)
      return release(MC_ENOMEM, "pinned staging", e);
    sg.cap = size_t(n);
  }
  if (!sg.ready && (e = cudaEventCreateWithFlags(&sg.ready, cudaEventBlockingSync | cudaEventDisableTiming)) !=
                       cudaSuccess)
    return release(MC_ECUDA, "cudaEventCreate", e);
  const cudaStream_t st = (cudaStream_t)stream;
  if ((e = cudaMemcpyAsync(sg.p, events, sizeof(mc_event) * size_t(n), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return release(MC_ECUDA, "cudaMemcpyAsync", e);
  if ((e = cudaEventRecord(sg.ready, st)) != cudaSuccess) return release(MC_ECUDA, "cudaEventRecord", e);
  LheBatch b;
  b.pinned = slot;
  b.n = n;
  {
    std::lock_guard<std::mutex> lk(w->m);
    w->q.push_back(std::move(b));
  }
  w->cv_work.notify_one();
  return MC_OK;
}

int mc_lhe_close(mc_lhe w, double xsec, double xerr, double wmax, int64_t* n_written) {
  if (n_written) *n_written = 0;
  if (!w) return lfail(MC_EINVAL, "mc_lhe_close: NULL handle");
  {
    std::lock_guard<std::mutex> lk(w->m);
    w->closing = true;
  }
  w->cv_work.notify_one();
  if (w->writer.joinable()) w->writer.join();
  int rc = w->error;
  std::string msg = w->err_msg;
  fprintf(w->f, "</LesHouchesEvents>\n");
  if (fseek(w->f, w->init_pos, SEEK_SET) == 0)
    write_init_line(w->f, xsec, xerr, wmax);
  else if (!rc) {
    rc = MC_EIO;
    msg = "mc_lhe_close: cannot seek to <init>";
  }
  if (ferror(w->f) && !rc) {
    rc = MC_EIO;
    msg = "mc_lhe_close: write failed";
  }
  if (fclose(w->f) != 0 && !rc) {
    rc = MC_EIO;
    msg = "mc_lhe_close: close failed";
  }
  if (n_written) *n_written = w->written;
  for (auto& sg : w->pool) {
    if (sg.p) cudaFreeHost(sg.p);
    if (sg.ready) cudaEventDestroy(sg.ready);
  }
  delete w;
  if (rc) return lfail(rc, "%s", msg.c_str());
  return MC_OK;
}

int mc_generate_lhe(const mc_integrand* itg, mc_pdf pdf, int ntrain, int niter, int64_t nevents, int nbins,
                    uint64_t seed, int prec, double alpha, const char* path, int threads, void* stream,
                    mc_result* out, mc_gen_stats* stats) {
  if (!out || !itg || !path) return lfail(MC_EINVAL, "mc_generate_lhe: NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (ntrain < 0 || niter < 1 || nevents < 2) return lfail(MC_EINVAL, "mc_generate_lhe: bad iteration counts");
  if (itg->proc != MC_EE_MUMU && itg->proc != MC_GG_TTBARG && itg->proc != MC_GG_TTBARG_7D &&
      itg->proc != MC_GG_TTBARG_MC)
    return lfail(MC_EINVAL, "mc_generate_lhe: process %d has no event record", itg->proc);
  const int nd = mc::process_dim(itg);
  mc_vegas v = nullptr;
  if (int rc = mc_vegas_init(nd, nbins, seed, prec, &v)) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  double* d_w = nullptr;
  mc_event* d_ev = nullptr;
  mc_lhe lhe = nullptr;
  int rc = MC_OK;
  mc_iter_result r;
  for (int it = 0; it < ntrain && !rc; ++it) {
    rc = mc_vegas_iterate(v, itg, pdf, nevents, stream, &r);
    if (!rc) rc = mc_vegas_refine(v, alpha, stream);
  }
  if (!rc && (cudaMalloc(&d_w, sizeof(double) * size_t(nevents)) != cudaSuccess ||
              cudaMalloc(&d_ev, sizeof(mc_event) * size_t(nevents)) != cudaSuccess))
    rc = lfail(MC_ENOMEM, "mc_generate_lhe: device buffers for %lld events", (long long)nevents);
  if (!rc) rc = mc_lhe_open(path, itg, threads, &lhe);
  std::vector<double> es, s2s;
  double wmax_all = 0.0, it_ms = 0.0, uw_ms = 0.0;
  int64_t nacc_all = 0;
  const auto t0 = std::chrono::steady_clock::now();
  for (int it = 0; it < niter && !rc; ++it) {
    rc = mc_vegas_iterate_weights(v, itg, pdf, nevents, d_w, stream, &r);
    if (rc) break;
    float ms = 0.0f;
    mc_vegas_kernel_ms(v, &ms);
    it_ms += ms;
    if (r.status && !out->status) out->status = r.status;
    const double n = double(r.n), mean = r.sum / n;
    es.push_back(mean);
    s2s.push_back((r.sum2 / n - mean * mean) / (n - 1.0));
    int64_t nacc = 0;
    rc = mc_unweight(v, itg, pdf, d_w, nevents, r.wmax, d_ev, nevents, &nacc, stream);
    if (rc) break;
    mc_unweight_ms(v, &ms);
    uw_ms += ms;
    rc = mc_lhe_write_device(lhe, d_ev, nacc, stream);
    wmax_all = std::max(wmax_all, r.wmax);
    nacc_all += nacc;
  }
  if (!es.empty()) {
    mc::combine_iterations(es, s2s, out);
    out->n_iter = int(es.size());
  }
  if (lhe) {
    int64_t nw = 0;
    const int crc = mc_lhe_close(lhe, out->mean, out->sigma, wmax_all, &nw);
    if (!rc) rc = crc;
    if (!rc && nw != nacc_all) rc = lfail(MC_EIO, "mc_generate_lhe: %lld of %lld events written", (long long)nw,
                                          (long long)nacc_all);
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->n_weighted = int64_t(es.size()) * nevents;
    stats->n_accepted = nacc_all;
    stats->iterate_ms = it_ms;
    stats->unweight_ms = uw_ms;
    stats->wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  out->gpu_ms = it_ms + uw_ms;
  cudaStreamSynchronize(st);
  cudaFree(d_w);
  cudaFree(d_ev);
  mc_vegas_free(v);
  return rc;
}

}  // extern "C"
