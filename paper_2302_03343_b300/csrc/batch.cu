// Many integrands in one persistent launch (C ABI: mc_batch_* in
// include/mcint.h).
//
// Work is cut into tiles (integrand i, a range of its events); blocks take
// tiles from a global atomic counter, the heaviest integrands first, and keep
// the current integrand's grid and shared-memory histogram until they move
// to a tile of another integrand.  Each tile writes one compensated partial;
// a second kernel reduces the partials of every integrand in a fixed order,
// a third refines all grids, a fourth advances the iteration counter (held in
// device memory) and resets the tile counter, so one iteration is a fixed
// sequence of launches that is captured once in a CUDA graph and replayed.
// Block size and events per thread are chosen by timing candidate launch
// shapes on the batch itself (autotune()).
//
// In FP32 mode the batch runs batch_ws_kernel instead: one block of
// ws_threads(P_GG_TTBARG) per SM; a tile of gg -> t tbar g events goes through the
// warp-specialised producer/consumer path of ws_integrand.cuh (each tile
// ends every producer stream with end markers, so the ring is empty between
// tiles), any other tile through all threads of the block one event each.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "event.cuh"
#include "handles.h"
#include "refine.cuh"
#include "ws_integrand.cuh"

namespace mc {

struct BatchItem {
  KernelArgs args;  // per-integrand arguments (grid pointers, gid, process parameters)
  int proc;
  long long nevents;
  int first_tile, ntiles;
  size_t edge_off, hist_off;
};

struct BatchArgs {
  const BatchItem* items;
  const int* tile_item;
  int ntiles;
  int tile_events;            // events per tile = events per thread x block
  unsigned int* counter;      // next tile
  const unsigned int* iteration;
  int nbins;
  int has_pdf;
  PdfDev pdf;
  double logq2_f;
  int fl[11];
  BlockPartial* tile_partials;
  int* status;  // MC_ETIMEOUT when a bounded wait of the launch gave up (warp-specialised kernel)
};

template <bool FP64, int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_kernel(BatchArgs b) {
  using R = typename std::conditional<FP64, double, float>::type;
  using H = typename std::conditional<FP64, double, float>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nb = b.nbins;
  const int nhist = MC_MAX_DIM * nb, nedge = MC_MAX_DIM * (nb + 1);
  H* sh_w2 = reinterpret_cast<H*>(smem);
  unsigned int* sh_n = reinterpret_cast<unsigned int*>(smem + size_t(nhist) * 8);
  R* sh_edges = reinterpret_cast<R*>(smem + ((size_t(nhist) * 12 + 15) / 16) * 16);
  R* sh_pdf = sh_edges + nedge;
  __shared__ KernelArgs ka;
  __shared__ int sh_tile;
  __shared__ BlockPartial warp_part[BLOCK / 32];

  SmPdf<R> pdf;
  if (b.has_pdf) {
    const int nx = b.pdf.nx;
    R* t = sh_pdf;
    R* f = t + nx;
    R* d = f + 11 * nx;
    build_pdf_tables<R>(b.pdf, b.logq2_f, b.fl, 11, t, f, d);
#pragma unroll
    for (int k = 0; k < 11; ++k) pdf.tab[k] = {t, f + k * nx, d + k * nx, nx};
  }
  for (int i = threadIdx.x; i < nhist; i += BLOCK) {
    sh_w2[i] = H(0);
    sh_n[i] = 0u;
  }
  const unsigned int iteration = *b.iteration;
  int cur = -1;
  auto flush = [&](int item) {
    const BatchItem& it = b.items[item];
    const int n = it.args.ndim * nb;
    for (int i = threadIdx.x; i < n; i += BLOCK) {
      if (sh_n[i]) {
        atomicAdd(&it.args.hist_n[i], sh_n[i]);
        atomicAdd(&it.args.hist_w2[i], double(sh_w2[i]));
      }
      sh_w2[i] = H(0);
      sh_n[i] = 0u;
    }
  };
  for (;;) {
    if (threadIdx.x == 0) sh_tile = int(atomicAdd(b.counter, 1u));
    __syncthreads();
    const int tile = sh_tile;
    if (tile >= b.ntiles) break;
    const int item = b.tile_item[tile];
    if (item != cur) {
      if (cur >= 0) flush(cur);
      const BatchItem& it = b.items[item];
      if (threadIdx.x == 0) {
        ka = it.args;
        ka.iteration = iteration;
      }
      const R* ge = FP64 ? reinterpret_cast<const R*>(it.args.edges64) : reinterpret_cast<const R*>(it.args.edges32);
      const int ne = it.args.ndim * (nb + 1);
      for (int i = threadIdx.x; i < ne; i += BLOCK) sh_edges[i] = ge[i];
      cur = item;
    }
    __syncthreads();
    const BatchItem& it = b.items[item];
    const long long start = (long long)(tile - it.first_tile) * b.tile_events;
    const long long end = min(start + (long long)b.tile_events, it.nevents);
    Acc acc;
    switch (it.proc) {
      case P_EE_MUMU:
        for (long long i = start + threadIdx.x; i < end; i += BLOCK)
          process_event<P_EE_MUMU, FP64, false, R, H>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr, acc);
        break;
      case P_PP_TTBAR:
        for (long long i = start + threadIdx.x; i < end; i += BLOCK)
          process_event<P_PP_TTBAR, FP64, false, R, H>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr, acc);
        break;
      case P_GG_TTBARG:
        for (long long i = start + threadIdx.x; i < end; i += BLOCK)
          process_event<P_GG_TTBARG, FP64, false, R, H>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr, acc);
        break;
      case P_GG_TTBARG_7D:
        for (long long i = start + threadIdx.x; i < end; i += BLOCK)
          process_event<P_GG_TTBARG_7D, FP64, false, R, H>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr,
                                                           acc);
        break;
      default:
        for (long long i = start + threadIdx.x; i < end; i += BLOCK)
          process_event<P_GAUSS, FP64, false, R, H>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr, acc);
    }
    block_reduce(acc, warp_part, &b.tile_partials[tile]);  // ends with __syncthreads
  }
  if (cur >= 0) flush(cur);
}

// FP32 batch kernel with the warp-specialised path for gg -> t tbar g tiles
// (both processes share the launch shape and the ring of P_GG_TTBARG: 23
// words, ws_slots slots).
constexpr int kBwProducers = ws_producer_warps(P_GG_TTBARG), kBwThreads = ws_threads(P_GG_TTBARG);
__global__ void __launch_bounds__(kBwThreads, 1) batch_ws_kernel(BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kSlots = ws_slots(P_GG_TTBARG) * kBwProducers;
  static_assert(ws_slots(P_GG_TTBARG) == ws_slots(P_GG_TTBARG_7D) && ws_words(P_GG_TTBARG) == ws_words(P_GG_TTBARG_7D) &&
                    ws_producer_warps(P_GG_TTBARG) == ws_producer_warps(P_GG_TTBARG_7D) &&
                    ws_consumer_warps(P_GG_TTBARG) == ws_consumer_warps(P_GG_TTBARG_7D) &&
                    ws_producer_regs(P_GG_TTBARG) == ws_producer_regs(P_GG_TTBARG_7D) &&
                    ws_consumer_regs(P_GG_TTBARG) == ws_consumer_regs(P_GG_TTBARG_7D),
                "the two processes share one ring and one launch shape");
  static_assert(ws_shape_ok(P_GG_TTBARG), "launch shape");
  __shared__ __align__(8) uint64_t full[kSlots], empty[kSlots];
  __shared__ int count[kSlots];
  __shared__ int failed;
  __shared__ KernelArgs ka;
  __shared__ int sh_tile;
  __shared__ BlockPartial warp_part[kBwThreads / 32];
  const int nb = b.nbins;
  const int nhist = MC_MAX_DIM * nb, nedge = MC_MAX_DIM * (nb + 1);
  const WsRing ring = {reinterpret_cast<uint32_t*>(smem), full, empty, count};
  unsigned char* rest = smem + size_t(kSlots) * ws_words(P_GG_TTBARG) * 32 * 4;
  float* sh_w2 = reinterpret_cast<float*>(rest);
  unsigned int* sh_n = reinterpret_cast<unsigned int*>(rest + size_t(nhist) * 4);
  float* sh_edges = reinterpret_cast<float*>(rest + ((size_t(nhist) * 8 + 15) / 16) * 16);
  float* sh_pdf = sh_edges + nedge;

  for (int i = threadIdx.x; i < nhist; i += kBwThreads) {
    sh_w2[i] = 0.0f;
    sh_n[i] = 0u;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&full[s], 32);
      mbar_init(&empty[s], 32);
    }
    failed = 0;
  }
  SmPdf<float> pdf;
  if (b.has_pdf) {
    const int nx = b.pdf.nx;
    float* t = sh_pdf;
    float* f = t + nx;
    float* d = f + 11 * nx;
    build_pdf_tables<float>(b.pdf, b.logq2_f, b.fl, 11, t, f, d);  // ends with __syncthreads
#pragma unroll
    for (int k = 0; k < 11; ++k) pdf.tab[k] = {t, f + k * nx, d + k * nx, nx};
  } else {
    __syncthreads();
  }
  const unsigned int iteration = *b.iteration;
  const int warp = threadIdx.x >> 5;
  int cur = -1;
  auto flush = [&](int item) {
    const BatchItem& it = b.items[item];
    const int n = it.args.ndim * nb;
    for (int i = threadIdx.x; i < n; i += kBwThreads) {
      if (sh_n[i]) {
        atomicAdd(&it.args.hist_n[i], sh_n[i]);
        atomicAdd(&it.args.hist_w2[i], double(sh_w2[i]));
      }
      sh_w2[i] = 0.0f;
      sh_n[i] = 0u;
    }
  };
  // slot sequence numbers, carried over from tile to tile
  int seq = 0;
  int q0 = (warp - kBwProducers) / kBwProducers, q1 = q0;
  for (;;) {
    if (threadIdx.x == 0) sh_tile = int(atomicAdd(b.counter, 1u));
    __syncthreads();
    const int tile = sh_tile;
    if (tile >= b.ntiles) break;
    const int item = b.tile_item[tile];
    if (item != cur) {
      if (cur >= 0) flush(cur);
      const BatchItem& it = b.items[item];
      if (threadIdx.x == 0) {
        ka = it.args;
        ka.iteration = iteration;
      }
      const int ne = it.args.ndim * (nb + 1);
      for (int i = threadIdx.x; i < ne; i += kBwThreads) sh_edges[i] = it.args.edges32[i];
      cur = item;
    }
    __syncthreads();
    const BatchItem& it = b.items[item];
    const long long start = (long long)(tile - it.first_tile) * b.tile_events;
    const long long end = min(start + (long long)b.tile_events, it.nevents);
    Acc acc;
    bool ok = true;
    if (it.proc == P_GG_TTBARG || it.proc == P_GG_TTBARG_7D) {
      if (warp < kBwProducers) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(ws_producer_regs(P_GG_TTBARG)));
        ok = it.proc == P_GG_TTBARG
                 ? ws_produce<P_GG_TTBARG, false>(ka, pdf, sh_edges, sh_n, ring, warp, start, end, warp,
                                                  kBwProducers, seq, acc)
                 : ws_produce<P_GG_TTBARG_7D, false>(ka, pdf, sh_edges, sh_n, ring, warp, start, end, warp,
                                                     kBwProducers, seq, acc);
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ws_regs(P_GG_TTBARG)));
      } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ws_consumer_regs(P_GG_TTBARG)));
        const int c = warp - kBwProducers;
        ok = it.proc == P_GG_TTBARG ? ws_consume<P_GG_TTBARG, false>(ka, sh_w2, ring, NoRows{}, c, q0, q1, acc)
                                    : ws_consume<P_GG_TTBARG_7D, false>(ka, sh_w2, ring, NoRows{}, c, q0, q1, acc);
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(ws_regs(P_GG_TTBARG)));
      }
    } else {
      switch (it.proc) {
        case P_EE_MUMU:
          for (long long i = start + threadIdx.x; i < end; i += kBwThreads)
            process_event<P_EE_MUMU, false, false, float, float>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr,
                                                                 acc);
          break;
        case P_PP_TTBAR:
          for (long long i = start + threadIdx.x; i < end; i += kBwThreads)
            process_event<P_PP_TTBAR, false, false, float, float>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i),
                                                                  nullptr, acc);
          break;
        default:
          for (long long i = start + threadIdx.x; i < end; i += kBwThreads)
            process_event<P_GAUSS, false, false, float, float>(ka, pdf, sh_edges, sh_w2, sh_n, uint64_t(i), nullptr,
                                                               acc);
      }
    }
    if (!ok) atomicExch(&failed, 1);
    block_reduce(acc, warp_part, &b.tile_partials[tile]);  // ends with __syncthreads
    if (failed) {
      if (threadIdx.x == 0) {
        b.tile_partials[tile].sum_hi = __longlong_as_double(0x7ff8000000000000LL);
        if (b.status) atomicExch(b.status, MC_ETIMEOUT);
      }
      break;  // the ring is no longer consistent: stop this block
    }
  }
  if (cur >= 0) flush(cur);
}

cudaError_t launch_batch_ws(const BatchArgs& b, int grid, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(batch_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  batch_ws_kernel<<<grid, kBwThreads, smem, st>>>(b);
  return cudaGetLastError();
}

// One block per integrand: fixed-order reduction of its tile partials.
__global__ void batch_finalize_kernel(const BatchItem* items, const BlockPartial* parts, BlockPartial* out) {
  __shared__ BlockPartial sh[256];
  const BatchItem& it = items[blockIdx.x];
  BlockPartial b = {0.0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0};
  for (int i = threadIdx.x; i < it.ntiles; i += blockDim.x) partial_add(b, parts[it.first_tile + i]);
  sh[threadIdx.x] = b;
  __syncthreads();
  for (int width = blockDim.x / 2; width > 0; width >>= 1) {
    if (int(threadIdx.x) < width) partial_add(sh[threadIdx.x], sh[threadIdx.x + width]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// One block per integrand, one warp per dimension.
__global__ void batch_refine_kernel(const BatchItem* items, const double* alpha, int nbins) {
  extern __shared__ double refine_work[];
  const BatchItem& it = items[blockIdx.x];
  const int d = threadIdx.x >> 5;
  if (d >= it.args.ndim) return;
  double* e = const_cast<double*>(it.args.edges64) + size_t(d) * (nbins + 1);
  float* e32 = const_cast<float*>(it.args.edges32) + size_t(d) * (nbins + 1);
  refine_dimension(e, e32, it.args.hist_w2 + size_t(d) * nbins, it.args.hist_n + size_t(d) * nbins, nbins, *alpha,
                   refine_work + size_t(d) * (3 * nbins + 2));
}

__global__ void batch_advance_kernel(unsigned int* counter, unsigned int* iteration) {
  *counter = 0u;
  *iteration += 1u;
}

template <bool FP64, int BLOCK>
cudaError_t launch_batch_t(const BatchArgs& b, int grid, size_t smem, cudaStream_t st) {
  auto k = batch_kernel<FP64, BLOCK>;
  (void)cudaGetLastError();  // report only this launch's error below
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k<<<grid, BLOCK, smem, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_batch(bool fp64, int block, const BatchArgs& b, int grid, size_t smem, cudaStream_t st) {
  switch (block) {
    case 64: return fp64 ? launch_batch_t<true, 64>(b, grid, smem, st) : launch_batch_t<false, 64>(b, grid, smem, st);
    case 256:
      return fp64 ? launch_batch_t<true, 256>(b, grid, smem, st) : launch_batch_t<false, 256>(b, grid, smem, st);
    default:
      return fp64 ? launch_batch_t<true, 128>(b, grid, smem, st) : launch_batch_t<false, 128>(b, grid, smem, st);
  }
}

int batch_blocks_per_sm(bool fp64, int block, size_t smem) {
  int n = 0;
  cudaError_t e;
  switch (block) {
    case 64:
      e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<true, 64>, 64, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<false, 64>, 64, smem);
      break;
    case 256:
      e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<true, 256>, 256, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<false, 256>, 256, smem);
      break;
    default:
      e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<true, 128>, 128, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<false, 128>, 128, smem);
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

// Relative cost of one event of each process, used to order the tiles
// (heaviest integrands first) so the launch ends with cheap tiles.
double event_cost(int proc) {
  switch (proc) {
    case P_GG_TTBARG:
    case P_GG_TTBARG_7D: return 100.0;
    case P_PP_TTBAR: return 10.0;
    case P_EE_MUMU: return 2.0;
  }
  return 1.0;
}

}  // namespace mc

using mc::BatchArgs;
using mc::BatchItem;
using mc::BlockPartial;

struct mc_batch_s {
  int device = 0, n = 0, nbins = 0, prec = 0;
  uint64_t seed = 0;
  std::vector<mc_integrand> itg;
  std::vector<long long> nevents;
  std::vector<int> ndim;
  mc_pdf pdf = nullptr;
  // device state
  double* d_edges = nullptr;
  float* d_edges32 = nullptr;
  double* d_hist_w2 = nullptr;
  unsigned int* d_hist_n = nullptr;
  BatchItem* d_items = nullptr;
  int* d_tile_item = nullptr;
  BlockPartial* d_tile_partials = nullptr;
  BlockPartial* d_results = nullptr;
  BlockPartial* h_results = nullptr;  // pinned
  unsigned int* d_counter = nullptr;
  unsigned int* d_iteration = nullptr;
  double* d_alpha = nullptr;
  double* h_alpha = nullptr;  // pinned
  size_t edges_total = 0, hist_total = 0;
  int max_tiles = 0;
  // launch shape (autotuned)
  int block = 128, events_per_thread = 8, ntiles = 0, grid = 0;
  bool ws = false;  // FP32: the warp-specialised batch kernel
  size_t smem = 0;
  BatchArgs args{};
  std::vector<BatchItem> h_items;
  // graph of one iteration
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t k0 = nullptr, k1 = nullptr;
  cudaStream_t capture = nullptr;  // private stream the iteration graph is captured on
  bool tuned = false;
};

namespace {

int bfail(int code, const char* msg) {
  mc::set_last_error(msg);
  return code;
}

// Tiles for a launch shape: per integrand ceil(N / (ept * block)) tiles,
// integrands ordered by decreasing total cost.
int build_tiles(mc_batch b) {
  const int te = b->events_per_thread * b->block;
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return mc::event_cost(b->itg[x].proc) * double(b->nevents[x]) >
           mc::event_cost(b->itg[y].proc) * double(b->nevents[y]);
  });
  std::vector<int> tile_item;
  for (int i : order) {
    BatchItem& it = b->h_items[i];
    it.first_tile = int(tile_item.size());
    it.ntiles = int((b->nevents[i] + te - 1) / te);
    for (int t = 0; t < it.ntiles; ++t) tile_item.push_back(i);
  }
  if (int(tile_item.size()) > b->max_tiles) return bfail(MC_EINVAL, "mc_batch: too many tiles for the launch shape");
  b->ntiles = int(tile_item.size());
  if (cudaMemcpy(b->d_tile_item, tile_item.data(), sizeof(int) * tile_item.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_items, b->h_items.data(), sizeof(BatchItem) * b->n, cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: upload of the tile table failed");
  const bool fp64 = b->prec == MC_FP64;
  const size_t r = fp64 ? 8 : 4;
  const size_t nhist = size_t(MC_MAX_DIM) * b->nbins;
  b->smem = ((nhist * 12 + 15) / 16) * 16 + r * (size_t(MC_MAX_DIM) * (b->nbins + 1)) +
            (b->pdf ? r * size_t(b->pdf->nx) * 23 : 0);
  if (b->ws)
    b->smem = size_t(mc::ws_slots(mc::P_GG_TTBARG)) * mc::kBwProducers * mc::ws_words(mc::P_GG_TTBARG) * 32 * 4 +
              ((nhist * 8 + 15) / 16) * 16 + 4 * (size_t(MC_MAX_DIM) * (b->nbins + 1)) +
              (b->pdf ? 4 * size_t(b->pdf->nx) * 23 : 0);
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int per_sm = b->ws ? 1 : mc::batch_blocks_per_sm(fp64, b->block, b->smem);
  b->grid = std::max(1, std::min(sms * per_sm, b->ntiles));
  BatchArgs& a = b->args;
  a.items = b->d_items;
  a.tile_item = b->d_tile_item;
  a.ntiles = b->ntiles;
  a.tile_events = te;
  a.counter = b->d_counter;
  a.iteration = b->d_iteration;
  a.nbins = b->nbins;
  a.tile_partials = b->d_tile_partials;
  a.status = reinterpret_cast<int*>(b->d_results + b->n);
  return MC_OK;
}

void drop_graph(mc_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// The launches of one iteration on `st`.
// `captured`: the events become event-record nodes of the graph.
int enqueue_iteration(mc_batch b, cudaStream_t st, bool with_refine, bool captured) {
  const bool fp64 = b->prec == MC_FP64;
  const unsigned int flags = captured ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (cudaMemsetAsync(b->args.status, 0, sizeof(int), st) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: status reset failed");
  if (cudaEventRecordWithFlags(b->k0, st, flags) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: event record failed");
  const cudaError_t le = b->ws ? mc::launch_batch_ws(b->args, b->grid, b->smem, st)
                               : mc::launch_batch(fp64, b->block, b->args, b->grid, b->smem, st);
  if (le != cudaSuccess) return bfail(MC_ECUDA, "mc_batch: batch kernel launch failed");
  if (cudaEventRecordWithFlags(b->k1, st, flags) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: event record failed");
  mc::batch_finalize_kernel<<<b->n, 256, 0, st>>>(b->d_items, b->d_tile_partials, b->d_results);
  if (with_refine) {
    const size_t smem = sizeof(double) * MC_MAX_DIM * (3 * b->nbins + 2);
    mc::batch_refine_kernel<<<b->n, 32 * MC_MAX_DIM, smem, st>>>(b->d_items, b->d_alpha, b->nbins);
  }
  mc::batch_advance_kernel<<<1, 1, 0, st>>>(b->d_counter, b->d_iteration);
  if (cudaMemcpyAsync(b->h_results, b->d_results, sizeof(BlockPartial) * (b->n + 1), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: result copy failed");
  if (cudaGetLastError() != cudaSuccess) return bfail(MC_ECUDA, "mc_batch: launch failed");
  return MC_OK;
}

// Autotuner: time one batch launch (no refinement, results discarded, the
// histograms restored afterwards) for each candidate (block size, events per
// thread) and keep the fastest.
int autotune(mc_batch b, cudaStream_t st) {
  static const int kBlocks[] = {64, 128, 256};
  static const int kEpt[] = {2, 8, 32};
  float best = 1e30f;
  int best_b = b->ws ? mc::kBwThreads : 128, best_e = b->ws ? 16 : 8;
  unsigned int it0 = 0;
  cudaMemcpy(&it0, b->d_iteration, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  const size_t smem_r = sizeof(double) * MC_MAX_DIM * (3 * b->nbins + 2);
  if (smem_r > 48 * 1024 &&
      cudaFuncSetAttribute(mc::batch_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_r)) !=
          cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch: refine kernel attribute");
  // warp-specialised kernel: one block shape, tiles of 4, 16 or 64 events per thread
  static const int kBlocksWs[] = {mc::kBwThreads};
  static const int kEptWs[] = {4, 16, 64};
  const int nbl = b->ws ? 1 : 3, nep = 3;
  const int* blocks = b->ws ? kBlocksWs : kBlocks;
  const int* epts = b->ws ? kEptWs : kEpt;
  for (int pass = 0; pass < 2; ++pass) {  // pass 0 warms up the first shape
    for (int ib = 0; ib < nbl; ++ib)
      for (int ie = 0; ie < nep; ++ie) {
        const int bl = blocks[ib], ep = epts[ie];
        if (pass == 0 && !(ib == nbl / 2 && ie == 1)) continue;
        b->block = bl;
        b->events_per_thread = ep;
        if (int rc = build_tiles(b)) return rc;
        if (int rc = enqueue_iteration(b, st, false, false)) return rc;
        if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(MC_ECUDA, "mc_batch: autotune launch failed");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, b->k0, b->k1);
        if (pass == 1 && ms < best) {
          best = ms;
          best_b = bl;
          best_e = ep;
        }
        cudaMemcpy(b->d_iteration, &it0, sizeof(unsigned int), cudaMemcpyHostToDevice);
      }
  }
  cudaMemset(b->d_hist_w2, 0, sizeof(double) * b->hist_total);
  cudaMemset(b->d_hist_n, 0, sizeof(unsigned int) * b->hist_total);
  b->block = best_b;
  b->events_per_thread = best_e;
  b->tuned = true;
  return build_tiles(b);
}

}  // namespace

extern "C" {

int mc_batch_free(mc_batch b) {
  if (!b) return MC_OK;
  drop_graph(b);
  cudaFree(b->d_edges);
  cudaFree(b->d_edges32);
  cudaFree(b->d_hist_w2);
  cudaFree(b->d_hist_n);
  cudaFree(b->d_items);
  cudaFree(b->d_tile_item);
  cudaFree(b->d_tile_partials);
  cudaFree(b->d_results);
  cudaFree(b->d_counter);
  cudaFree(b->d_iteration);
  cudaFree(b->d_alpha);
  if (b->h_results) cudaFreeHost(b->h_results);
  if (b->h_alpha) cudaFreeHost(b->h_alpha);
  if (b->k0) cudaEventDestroy(b->k0);
  if (b->k1) cudaEventDestroy(b->k1);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
  return MC_OK;
}

int mc_batch_create(int n, const mc_integrand* itgs, const int64_t* nevents, mc_pdf pdf, int nbins, uint64_t seed,
                    int prec, mc_batch* out) {
  if (!out) return bfail(MC_EINVAL, "mc_batch_create: out is NULL");
  *out = nullptr;
  if (n < 1 || n > 256 || !itgs || !nevents) return bfail(MC_EINVAL, "mc_batch_create: need 1..256 integrands");
  if (nbins < 2 || nbins > MC_MAX_BINS) return bfail(MC_EINVAL, "mc_batch_create: bad nbins");
  if (prec != MC_FP64 && prec != MC_FP32_KAHAN) return bfail(MC_EINVAL, "mc_batch_create: bad precision");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bfail(MC_ECUDA, "mc_batch_create: no device");
  auto* b = new mc_batch_s;
  b->device = dev;
  b->n = n;
  b->nbins = nbins;
  b->prec = prec;
  b->seed = seed;
  b->pdf = pdf;
  b->ws = prec == MC_FP32_KAHAN;
  if (b->ws) {
    b->block = mc::kBwThreads;
    b->events_per_thread = 16;
  }
  b->itg.assign(itgs, itgs + n);
  double logq2 = 0.0;
  bool have_mu = false;
  for (int i = 0; i < n; ++i) {
    const mc_integrand& t = itgs[i];
    // the batch kernels run these five processes (Gaussian: gauss_dim 1..16)
    const bool supported = t.proc == MC_EE_MUMU || t.proc == MC_PP_TTBAR || t.proc == MC_GG_TTBARG ||
                           t.proc == MC_GAUSS || t.proc == MC_GG_TTBARG_7D;
    const int nd = supported ? mc::process_dim(&t) : -1;
    if (nd < 1 || nd > MC_MAX_DIM || nevents[i] < 0) {
      mc_batch_free(b);
      return bfail(MC_EINVAL, "mc_batch_create: bad integrand or event count");
    }
    if (t.proc == MC_PP_TTBAR || t.proc == MC_GG_TTBARG || t.proc == MC_GG_TTBARG_7D) {
      if (!pdf || pdf->device != dev) {
        mc_batch_free(b);
        return bfail(MC_EINVAL, "mc_batch_create: hadronic integrands need a PDF on this device");
      }
      const double lq = std::log(t.mu_f * t.mu_f);
      if (!(lq >= pdf->logq2.front() && lq <= pdf->logq2.back()) || (have_mu && lq != logq2)) {
        mc_batch_free(b);
        return bfail(MC_EINVAL, "mc_batch_create: mu_f must be inside the grid and common to all integrands");
      }
      logq2 = lq;
      have_mu = true;
    }
    b->ndim.push_back(nd);
    b->nevents.push_back(nevents[i]);
    b->edges_total += size_t(nd) * (nbins + 1);
    b->hist_total += size_t(nd) * nbins;
  }
  long long maxt = 0;
  for (int i = 0; i < n; ++i) maxt += (b->nevents[i] + 2 * 64 - 1) / (2 * 64);  // smallest tile: 2 x 64 events
  b->max_tiles = int(std::min<long long>(maxt + n, 1LL << 28));
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&b->d_edges, sizeof(double) * b->edges_total)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_edges32, sizeof(float) * b->edges_total)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_hist_w2, sizeof(double) * b->hist_total)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_hist_n, sizeof(unsigned int) * b->hist_total)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_items, sizeof(BatchItem) * n)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_tile_item, sizeof(int) * b->max_tiles)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_tile_partials, sizeof(BlockPartial) * b->max_tiles)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_results, sizeof(BlockPartial) * (n + 1))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_counter, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_iteration, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_alpha, sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_results, sizeof(BlockPartial) * (n + 1))) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_alpha, sizeof(double))) != cudaSuccess ||
      (e = cudaEventCreate(&b->k0)) != cudaSuccess || (e = cudaEventCreate(&b->k1)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) != cudaSuccess) {
    mc_batch_free(b);
    return bfail(MC_ENOMEM, (std::string("mc_batch_create: allocation failed: ") + cudaGetErrorString(e)).c_str());
  }
  // uniform grids, zero histograms and counters
  std::vector<double> edges(b->edges_total);
  std::vector<float> e32(b->edges_total);
  size_t eo = 0, ho = 0;
  b->h_items.resize(n);
  for (int i = 0; i < n; ++i) {
    const int nd = b->ndim[i];
    for (int d = 0; d < nd; ++d)
      for (int k = 0; k <= nbins; ++k) {
        const double v = k == nbins ? 1.0 : double(k) / nbins;
        edges[eo + size_t(d) * (nbins + 1) + k] = v;
        e32[eo + size_t(d) * (nbins + 1) + k] = float(v);
      }
    BatchItem& it = b->h_items[i];
    std::memset(&it, 0, sizeof(it));
    const mc_integrand& t = itgs[i];
    mc::KernelArgs& a = it.args;
    a.prm = {t.proc, t.gauss_dim, t.sqrt_s, t.m_top, t.alpha, t.alpha_s, t.mz, t.gz, t.sw2, t.mu_f, t.ptcut_g,
             t.etacut_g, t.gauss_sigma, t.gev2pb};
    a.ndim = nd;
    a.nbins = nbins;
    a.edges64 = b->d_edges + eo;
    a.edges32 = b->d_edges32 + eo;
    a.w0_coef3 = std::pow(2.0 * M_PI, -5.0) * std::pow(M_PI / 2.0, 2.0) / 2.0;
    a.e2eta = std::exp(2.0 * t.etacut_g);
    a.seed = seed;
    a.gid = uint32_t(i);
    a.hist_w2 = b->d_hist_w2 + ho;
    a.hist_n = b->d_hist_n + ho;
    it.proc = t.proc;
    it.nevents = b->nevents[i];
    it.edge_off = eo;
    it.hist_off = ho;
    eo += size_t(nd) * (nbins + 1);
    ho += size_t(nd) * nbins;
  }
  BatchArgs& ba = b->args;
  std::memset(&ba, 0, sizeof(ba));
  if (have_mu) {
    ba.has_pdf = 1;
    ba.pdf = pdf->dev();
    ba.logq2_f = logq2;
    ba.fl[0] = pdf->index(21);
    for (int q = 1; q <= 5; ++q) {
      ba.fl[q] = pdf->index(q);
      ba.fl[q + 5] = pdf->index(-q);
    }
    for (int k = 0; k < 11; ++k)
      if (ba.fl[k] < 0) {
        mc_batch_free(b);
        return bfail(MC_EINVAL, "mc_batch_create: the PDF needs the gluon and quarks 1..5");
      }
  }
  const unsigned int zero = 0;
  if (cudaMemcpy(b->d_edges, edges.data(), sizeof(double) * b->edges_total, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_edges32, e32.data(), sizeof(float) * b->edges_total, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_hist_w2, 0, sizeof(double) * b->hist_total) != cudaSuccess ||
      cudaMemset(b->d_hist_n, 0, sizeof(unsigned int) * b->hist_total) != cudaSuccess ||
      cudaMemcpy(b->d_counter, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_iteration, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_batch_free(b);
    return bfail(MC_ECUDA, "mc_batch_create: initialisation failed");
  }
  if (int rc = build_tiles(b)) {
    mc_batch_free(b);
    return rc;
  }
  *out = b;
  return MC_OK;
}

int mc_batch_iterate(mc_batch b, double alpha, void* stream, mc_iter_result* out) {
  if (!b || !out) return bfail(MC_EINVAL, "mc_batch_iterate: NULL argument");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return bfail(MC_EINVAL, "mc_batch_iterate: bad alpha");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
    return bfail(MC_EINVAL, "mc_batch_iterate: batch lives on another device");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->tuned) {
    drop_graph(b);
    if (int rc = autotune(b, st)) return rc;
  }
  if (!b->exec) {
    // capture one iteration (batch kernel, finalize, refine, advance, copy
    // back) on the private stream; the graph is then launched on `stream`
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bfail(MC_ECUDA, "mc_batch_iterate: stream capture failed to start");
    const int rc = enqueue_iteration(b, b->capture, true, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return bfail(MC_ECUDA, "mc_batch_iterate: stream capture failed");
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      drop_graph(b);
      return bfail(MC_ECUDA, "mc_batch_iterate: graph instantiation failed");
    }
  }
  *b->h_alpha = alpha;
  if (cudaMemcpyAsync(b->d_alpha, b->h_alpha, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch_iterate: alpha upload failed");
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return bfail(MC_ECUDA, "mc_batch_iterate: graph launch failed");
  if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(MC_ECUDA, "mc_batch_iterate: iteration failed");
  if (*reinterpret_cast<const int*>(b->h_results + b->n) != 0)
    return bfail(MC_ETIMEOUT, "mc_batch_iterate: a bounded wait inside the batch kernel gave up");
  for (int i = 0; i < b->n; ++i) {
    const BlockPartial& t = b->h_results[i];
    mc_iter_result& r = out[i];
    std::memset(&r, 0, sizeof(r));
    r.n = b->nevents[i];
    r.sum = t.sum_hi + t.sum_lo;
    r.sum2 = t.sum2_hi + t.sum2_lo;
    r.wmax = t.wmax;
    r.n_nonzero = t.n_nonzero;
    r.n_bad = t.n_bad + t.n_noconv;
    r.status = t.n_bad ? MC_ENAN : (t.n_noconv ? MC_ENOCONV : MC_OK);
  }
  return MC_OK;
}

int mc_batch_get_grid(mc_batch b, int i, double* edges) {
  if (!b || !edges || i < 0 || i >= b->n) return bfail(MC_EINVAL, "mc_batch_get_grid: bad argument");
  if (cudaDeviceSynchronize() != cudaSuccess) return bfail(MC_ECUDA, "mc_batch_get_grid: device error");
  const BatchItem& it = b->h_items[i];
  if (cudaMemcpy(edges, b->d_edges + it.edge_off, sizeof(double) * b->ndim[i] * (b->nbins + 1),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(MC_ECUDA, "mc_batch_get_grid: copy failed");
  return MC_OK;
}

int mc_batch_shape(mc_batch b, int* block, int* events_per_thread, int* grid, int* ntiles) {
  if (!b) return bfail(MC_EINVAL, "mc_batch_shape: NULL handle");
  if (block) *block = b->block;
  if (events_per_thread) *events_per_thread = b->events_per_thread;
  if (grid) *grid = b->grid;
  if (ntiles) *ntiles = b->ntiles;
  return MC_OK;
}

int mc_batch_kernel_ms(mc_batch b, float* ms) {
  if (!b || !ms) return bfail(MC_EINVAL, "mc_batch_kernel_ms: NULL argument");
  if (cudaEventElapsedTime(ms, b->k0, b->k1) != cudaSuccess) {
    (void)cudaGetLastError();
    *ms = 0.0f;
  }
  return MC_OK;
}

}  // extern "C"
