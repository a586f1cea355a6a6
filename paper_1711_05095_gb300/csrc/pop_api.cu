// Host side of the C ABI declared in include/pop.h.
//
// A handle owns only host state; every device buffer is carved out of the
// caller's workspace.  Layout of the workspace (each region 256-byte aligned):
//   PopDesc[P]  PopState[P]  tile_pop[ntiles]  wtab[P][4096] u64  qtab, qm1tab[P][4096] f64
//   inv_rate[P][129] f32  logtab[64] f32x2  hist[P][4096] u32  thist[64][ntiles] u32
//   tile_sum, tile_excl[ntiles] u64
//   beta  ksum[P]
//   X[2], Y lattices [nslots][W] u64   KX[2], KY, dK[2], anc [nslots] i32   A[2] [nslots] f32
// where every population starts on a 1024-slot tile and nslots is the padded total.
//
// One interval = k_evolve, k_weights, k_gather on the caller's stream.  pop_run fuses
// the cloning stage of each interval with the dynamical stage of the next where it can
// (k_gather<FUSE>), captures kGraphIntervals of its repeated part into a CUDA graph once
// (on a private capture stream) and replays it on the caller's stream; the kernels read
// the interval number and every other changing quantity from device memory, so replays
// need no new arguments.  The evolved lattices, K, dK and A are double-buffered by the
// parity of the interval, so one interval's dynamical stage never overwrites the
// population its cloning stage is still reading.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pop.h"
#include "pop_kernels.cuh"

using namespace popgpu;

// pop_run's chains (see pop_batch::nch): at most POP_RUN_CHAINS for a batch that fits
// in two waves of the fused kernel, at most POP_RUN_CHAINS_LARGE for a larger one
#ifndef POP_RUN_CHAINS
#define POP_RUN_CHAINS 8
#endif
#ifndef POP_RUN_CHAINS_LARGE
#define POP_RUN_CHAINS_LARGE 2
#endif
constexpr int kMaxChains = 8;
// clones each lane of the fused kernel advances together (1 or 2)
#ifndef POP_FUSE_CLONES
#define POP_FUSE_CLONES 1
#endif
constexpr int kFuseClones = POP_FUSE_CLONES;
static_assert(POP_RUN_CHAINS >= 1 && POP_RUN_CHAINS <= kMaxChains &&
              POP_RUN_CHAINS_LARGE >= 1 && POP_RUN_CHAINS_LARGE <= kMaxChains, "1 to 8 chains");


namespace {

constexpr int kGraphIntervals = 32;
// the separate cloning stage uses 256-thread blocks above this many tiles (several
// waves; at one wave, 128-thread blocks finish first)
constexpr int kGatherWideTiles = 4096;
#ifndef POP_GATHER_WIDE_THREADS
#define POP_GATHER_WIDE_THREADS 256
#endif

struct Layout {
  int32_t P = 0, W = 0, ntiles = 0, nunits = 0;
  int64_t nslots = 0;
  size_t o_pops, o_st, o_tile_pop, o_wtab, o_qtab, o_qm1tab, o_inv, o_logtab, o_exp2, o_A, o_S, o_cs, o_tacc, o_hist, o_thist, o_tile_sum, o_tile_excl, o_beta, o_phi, o_gtab, o_gdu, o_gq, o_gcar,
      o_ksum, o_X, o_Y, o_KX, o_KY, o_dK, o_anc, total;
};

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

bool valid_params(const pop_params* params, int32_t n_pops) {
  if (params == nullptr || n_pops < 1 || n_pops > (1 << 20)) return false;
  for (int32_t p = 0; p < n_pops; ++p) {
    const pop_params& q = params[p];
    if (q.L < 3 || q.L > POP_MAX_L) return false;
    if (q.N < 0 || q.N > q.L) return false;
    if (q.n_clones < 1 || q.n_clones > POP_MAX_CLONES) return false;
    if (q.weight_mode != POP_PLAIN && q.weight_mode != POP_MODIFIED &&
        q.weight_mode != POP_GUIDED)
      return false;
    if (q.selection != POP_EQ && q.selection != POP_IID) return false;
    // GUIDED: one clone per thread with 18-site windows, and the whole batch guided
    if ((q.weight_mode == POP_GUIDED) != (params[0].weight_mode == POP_GUIDED)) return false;
    if (q.weight_mode == POP_GUIDED && (q.L < 18 || q.L > kMaxL || n_pops > 65535)) return false;
  }
  return true;
}

bool make_layout(const pop_params* params, int32_t n_pops, Layout* lay) {
  if (!valid_params(params, n_pops)) return false;
  Layout l;
  l.P = n_pops;
  int32_t maxL = 0;
  int64_t ntiles = 0;
  for (int32_t p = 0; p < n_pops; ++p) {
    maxL = params[p].L > maxL ? params[p].L : maxL;
    ntiles += (params[p].n_clones + kTile - 1) / kTile;
  }
  if (ntiles > (int64_t)INT32_MAX / 2) return false;
  l.W = (maxL + 63) / 64;
  l.ntiles = (int32_t)ntiles;
  l.nslots = ntiles * kTile;
  l.nunits = (int32_t)(l.nslots / kUnit);
  const size_t P = (size_t)n_pops, ns = (size_t)l.nslots, nt = (size_t)l.ntiles;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  l.o_pops = take(P * sizeof(PopDesc));
  l.o_st = take(P * sizeof(PopState));
  l.o_tile_pop = take(nt * sizeof(int32_t));
  l.o_wtab = take(P * kKcap * sizeof(unsigned long long));
  l.o_qtab = take(P * kKcap * sizeof(double));
  l.o_qm1tab = take(P * kKcap * sizeof(double));
  l.o_inv = take(P * kInvStride * sizeof(float));
  l.o_logtab = take(64 * sizeof(float2));
  l.o_exp2 = take(64 * sizeof(float));
  l.o_hist = take(P * kKcap * sizeof(unsigned int));
  l.o_thist = take((size_t)kTH * nt * sizeof(unsigned int));
  l.o_tile_sum = take(nt * sizeof(unsigned long long));
  l.o_tile_excl = take(nt * sizeof(unsigned long long));
  l.o_beta = take((1 + kMaxChains) * sizeof(unsigned int));   // the interval counter, one per chain
  l.o_ksum = take(P * sizeof(long long));
  l.o_phi = take(P * 512 * sizeof(int32_t));
  l.o_gtab = take((kGuideTabA + kGuideTabB) * sizeof(unsigned long long));
  // GUIDED batches: the per-population bond tables (dU and its rate Q by segment)
  const bool guided = params[0].weight_mode == POP_GUIDED;
  l.o_gdu = take(guided ? P * kGuideSeg * sizeof(int32_t) : 0);
  l.o_gq = take(guided ? P * kGuideSeg * sizeof(unsigned long long) : 0);
  l.o_gcar = take(guided ? 2 * ns * (size_t)(8 * l.W) * sizeof(unsigned long long) : 0);
  l.o_X = take(2 * ns * (size_t)l.W * sizeof(unsigned long long));
  l.o_Y = take(ns * (size_t)l.W * sizeof(unsigned long long));
  l.o_KX = take(2 * ns * sizeof(int32_t));
  l.o_KY = take(ns * sizeof(int32_t));
  l.o_dK = take(2 * ns * sizeof(int32_t));
  l.o_anc = take(ns * sizeof(int32_t));
  l.o_A = take(2 * ns * sizeof(float));
  l.o_S = take(ns * sizeof(unsigned long long));
  l.o_cs = take(P * kInvStride * sizeof(float2));
  l.o_tacc = take(nt * sizeof(double));
  l.total = o;
  *lay = l;
  return true;
}

int ceil_log2(int64_t x) {
  int c = 0;
  while (((int64_t)1 << c) < x) ++c;
  return c;
}

enum Phase { kReady = 0, kEvolved = 1 };

}  // namespace

namespace {
// Split ntiles into K chains of whole populations, K the largest number up to want for
// which each chain holds at least half of its equal share: boundary k is the population
// start nearest k ntiles / K.  Returns K; bounds[0..K] are the chains' first tiles and
// ntiles.
int choose_chains(const std::vector<PopDesc>& desc, int32_t ntiles, int want, int32_t* bounds) {
  for (int K = want; K >= 2; --K) {
    bool ok = true;
    bounds[0] = 0;
    for (int k = 1; k < K && ok; ++k) {
      int32_t best = -1;
      for (size_t p = 1; p < desc.size(); ++p) {
        const int64_t t = desc[p].first_tile;
        if (best < 0 || std::llabs(K * t - (int64_t)k * ntiles) < std::llabs((int64_t)K * best - (int64_t)k * ntiles))
          best = (int32_t)t;
      }
      ok = best >= 0;
      bounds[k] = best;
    }
    bounds[K] = ntiles;
    for (int k = 0; k < K && ok; ++k) ok = 2 * (int64_t)K * (bounds[k + 1] - bounds[k]) >= ntiles;
    if (ok) return K;
  }
  bounds[0] = 0;
  bounds[1] = ntiles;
  return 1;
}
}  // namespace

struct pop_batch {
  Layout lay;
  std::vector<pop_params> params;
  std::vector<PopDesc> desc;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  // pop_run's fused loop as nch chains of whole populations, each on its own stream,
  // so the latency-bound phases of one chain overlap the dynamical stage of another
  int32_t nch = 1;
  int32_t chain_tile[kMaxChains + 1] = {};   // chain c: tiles [chain_tile[c], chain_tile[c + 1])
  int32_t chain_pop[kMaxChains + 1] = {};    // and populations [chain_pop[c], chain_pop[c + 1])
  cudaStream_t aux_stream[kMaxChains - 1] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxChains - 1] = {};
  Batch chain[kMaxChains]{};                 // the batch with each chain's own interval counter
  // launch configuration (rule-based at pop_init; pop_autotune or pop_set_tuning may change it)
  int fuse_threads = 128;                    // fused kernel: threads per block (128 or 256)
  int fuse_clones = kFuseClones;             // fused kernel: clones per lane (1 or 2)
  int gather_threads = 0;                    // separate cloning stage: 128, 256, or 0 for the rule
  int hist_mode = -1;                        // tile activity histograms: 1 on, 0 off, -1 the rule
  int max_L = 0;
  // the last dynamical stage was a fused launch that filled the tile histograms, so the
  // next cloning stage takes its weights from them (k_tile_scan<true>)
  bool hist_pending = false;
  int graph_hist = -1;                       // hist_on of the captured graph
  float tuned_default_us = 0.0f, tuned_us = 0.0f;
  cudaGraphExec_t graph = nullptr;
  float graph_dt = 0.0f;
  unsigned char* ws = nullptr;
  Batch B{};
  bool any_mod = false;
  bool guided = false;       // every population GUIDED
  bool guided_q_stale = true; // GUIDED: the rate tables need (re)building once s is fixed
  int guided_split = 1;       // GUIDED: blocks per tile of the dynamical stage (1, 2, 4, 8)
  int evolve_grid = 0;
  int evolve_grid_cap = 0;  // persistent grid at full occupancy
  size_t evolve_smem = 0;
  bool s_fixed = false;
  std::vector<double> s;
  Phase phase = kReady;
  int64_t intervals = 0;
  double t_obs = 0.0;
  // kernels launched, by kind; launches made during graph capture go to graph_counts
  // and are added to launches at every replay
  uint64_t launches[POP_NKINDS] = {};
  uint64_t graph_counts[POP_NKINDS] = {};
  uint64_t* count = launches;
  // pop_kernel_times: events recorded around every launch while set
  std::vector<cudaEvent_t>* timer_events = nullptr;
  std::vector<int>* timer_kinds = nullptr;
  std::vector<int>* timer_intervals = nullptr;
  int timer_interval = 0;
  int timer_base = -1;        // run_chains tags interval i of its call timer_base + i (if >= 0)
  bool timer_capture = false; // the timed launches are being captured into a graph
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? POP_OK : POP_ERR_CUDA; }

#define POP_CUDA(call)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return POP_ERR_CUDA;     \
  } while (0)

// GUIDED: Q(clamp(dU - s_q)) of every segment of every population, rebuilt after s is
// fixed and after a potential changes (outside any capture: a launch of its own).
int guided_rate_tables(pop_t* h) {
  if (!h->guided || !h->guided_q_stale) return POP_OK;
  const dim3 grid((unsigned)(kGuideSeg / kThreads), (unsigned)h->lay.P);
  h->launches[POP_K_OTHER] += 1;
  k_guided_qtab<<<grid, kThreads, 0, h->stream>>>(h->B);
  if (cudaGetLastError() != cudaSuccess) return POP_ERR_CUDA;
  h->guided_q_stale = false;
  return POP_OK;
}

int fix_biases(pop_t* h, const double* s) {
  if (s == nullptr) return POP_ERR_ARG;
  for (int32_t p = 0; p < h->lay.P; ++p)
    if (!std::isfinite(s[p])) return POP_ERR_ARG;
  if (h->s_fixed) {
    for (int32_t p = 0; p < h->lay.P; ++p)
      if (s[p] != h->s[p]) return POP_ERR_STATE;
    return guided_rate_tables(h);
  }
  // Fixed-point weights (64-bit): F = 61 - ceil(log2 N_c), so N_c weights of at most
  // 2^F sum to at most 2^61; wtab[k] = nearest integer to 2^F exp(-|s| k).  The psi
  // term uses exp(-|s| k) and expm1(-|s| k) in FP64 (qtab, qm1tab).
  const size_t n = (size_t)h->lay.P * kKcap;
  std::vector<unsigned long long> wtab(n);
  std::vector<double> qtab(n), qm1tab(n);
  for (int32_t p = 0; p < h->lay.P; ++p) {
    const int F = 61 - ceil_log2(h->params[p].n_clones);
    const double a = std::fabs(s[p]);
    for (int k = 0; k < kKcap; ++k) {
      const double x = -a * (double)k;
      const double q = std::exp(x);
      wtab[(size_t)p * kKcap + k] = (unsigned long long)std::nearbyint(std::ldexp(q, F));
      qtab[(size_t)p * kKcap + k] = q;
      qm1tab[(size_t)p * kKcap + k] = std::expm1(x);
    }
    h->desc[p].s = s[p];
    h->desc[p].abs_s = a;
    h->desc[p].s_neg = s[p] < 0.0 ? 1 : 0;
    h->desc[p].c_f = (float)(-std::expm1(-s[p]));
    h->desc[p].s_q = (int32_t)std::nearbyint(std::ldexp(s[p], 17));
    h->desc[p].c_s = (float)(std::ldexp((double)h->desc[p].s_q, -17) - s[p]);
  }
  // MODIFIED dynamics: every rate times e^-s, so the waiting-time factor is e^s / r
  std::vector<float> inv_mod;
  for (int32_t p = 0; p < h->lay.P; ++p) {
    if (!h->desc[p].modified || h->desc[p].guided) continue;
    inv_mod.assign(kInvStride, 0.0f);
    const double es = std::exp(s[p]);
    for (int r = 1; r <= h->params[p].L; ++r) inv_mod[r] = (float)(es / (double)r);
    POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_inv + (size_t)p * kInvStride * sizeof(float),
                             inv_mod.data(), kInvStride * sizeof(float), cudaMemcpyHostToDevice,
                             h->stream));
    POP_CUDA(cudaStreamSynchronize(h->stream));
  }
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_wtab, wtab.data(), n * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice, h->stream));
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_qtab, qtab.data(), n * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_qm1tab, qm1tab.data(), n * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_pops, h->desc.data(),
                           h->desc.size() * sizeof(PopDesc), cudaMemcpyHostToDevice, h->stream));
  POP_CUDA(cudaStreamSynchronize(h->stream));
  h->s.assign(s, s + h->lay.P);
  h->s_fixed = true;
  return guided_rate_tables(h);
}

bool valid_dt(double dt) { return std::isfinite(dt) && dt > 0.0 && dt < 1e30; }

// Bookkeeping around one kernel launch: the per-kind count and, under
// pop_kernel_times, an event pair on the launching stream.
// pop_kernel_times: an event before and after each launch (while a graph is being
// captured, as an event-record node of the graph)
void timer_record(pop_t* h, cudaStream_t st) {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  if (h->timer_capture) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
  h->timer_events->push_back(e);
}

void kernel_begin(pop_t* h, cudaStream_t st, int kind) {
  h->count[kind] += 1;
  if (h->timer_events != nullptr) {
    timer_record(h, st);
    h->timer_kinds->push_back(kind);
    if (h->timer_intervals) h->timer_intervals->push_back(h->timer_interval);
  }
}

void kernel_end(pop_t* h, cudaStream_t st) {
  if (h->timer_events != nullptr) timer_record(h, st);
}

int launch_evolve(pop_t* h, cudaStream_t st, float dt_f) {
  const unsigned grid = (unsigned)h->evolve_grid;
  const size_t sm = h->evolve_smem;
  kernel_begin(h, st, POP_K_EVOLVE);
  if (h->guided) {
    // a tile per block, or a half, quarter or eighth of one for a batch of fewer tiles
    // than two waves of blocks
    const int spb = kTile / h->guided_split;
    const unsigned gg = (unsigned)((int64_t)h->lay.ntiles * h->guided_split);
    if (h->lay.W == 1) k_evolve_guided<1><<<gg, kGuideThreads, 0, st>>>(h->B, dt_f, spb);
    else k_evolve_guided<2><<<gg, kGuideThreads, 0, st>>>(h->B, dt_f, spb);
  } else if (h->any_mod) {
    if (h->lay.W == 1) k_evolve<1, true><<<grid, kThreads, sm, st>>>(h->B, dt_f);
    else if (h->lay.W == 2) k_evolve<2, true><<<grid, kThreads, sm, st>>>(h->B, dt_f);
    else k_evolve_wide<true><<<grid, kThreads, 0, st>>>(h->B, dt_f);
  } else {
    if (h->lay.W == 1) k_evolve<1, false><<<grid, kThreads, sm, st>>>(h->B, dt_f);
    else if (h->lay.W == 2) k_evolve<2, false><<<grid, kThreads, sm, st>>>(h->B, dt_f);
    else k_evolve_wide<false><<<grid, kThreads, 0, st>>>(h->B, dt_f);
  }
  kernel_end(h, st);
  return cuda_status(cudaGetLastError());
}

// The tile prefixes and totals of the populations [pop0, pop1); hist: the tile sums and
// activity histograms too, from the tile histograms of the fused stage.
void launch_tile_scan(pop_t* h, cudaStream_t st, const Batch& Bx, int pop0, int pop1, bool hist = false) {
  kernel_begin(h, st, hist ? POP_K_WEIGHTS : POP_K_OTHER);
  if (hist) k_tile_scan<true><<<(unsigned)(pop1 - pop0), kScanThreads, 0, st>>>(Bx, pop0);
  else k_tile_scan<false><<<(unsigned)(pop1 - pop0), kScanThreads, 0, st>>>(Bx, pop0);
  kernel_end(h, st);
}

// k_weights over the tiles [tile0, tile0 + ntiles), one block per tile
void launch_weights_range(pop_t* h, cudaStream_t st, const Batch& Bx, int tile0, int ntiles) {
  kernel_begin(h, st, POP_K_WEIGHTS);
  k_weights<<<(unsigned)ntiles, kThreads, 0, st>>>(Bx, tile0);
  kernel_end(h, st);
}

void launch_weights(pop_t* h, cudaStream_t st) {
  launch_weights_range(h, st, h->B, 0, h->lay.ntiles);
  launch_tile_scan(h, st, h->B, 0, h->lay.P);
}

int launch_resample(pop_t* h, cudaStream_t st) {
  const unsigned grid = (unsigned)h->lay.ntiles;
  if (h->hist_pending) launch_tile_scan(h, st, h->B, 0, h->lay.P, true);
  else launch_weights(h, st);
  h->hist_pending = false;
  constexpr int GT = POP_GATHER_THREADS;
  kernel_begin(h, st, POP_K_GATHER);
  const bool wide_blocks = h->gather_threads == 0 ? h->lay.ntiles > kGatherWideTiles : h->gather_threads == 256;
  if (wide_blocks) {
    // many waves of tiles: 256-thread blocks keep more bytes in flight (measured
    // 4567 against 4379 GB/s on 2^25 two-word clones)
    constexpr int GW = POP_GATHER_WIDE_THREADS;
    if (h->lay.W == 1) k_gather<1, GW><<<grid, GW, 0, st>>>(h->B, 0.0f, 0);
    else if (h->lay.W == 2) k_gather<2, GW><<<grid, GW, 0, st>>>(h->B, 0.0f, 0);
    else k_gather<0, GW><<<grid, GW, 0, st>>>(h->B, 0.0f, 0);
  } else if (h->lay.W == 1) {
    k_gather<1, GT><<<grid, GT, 0, st>>>(h->B, 0.0f, 0);
  } else if (h->lay.W == 2) {
    k_gather<2, GT><<<grid, GT, 0, st>>>(h->B, 0.0f, 0);
  } else {
    k_gather<0, GT><<<grid, GT, 0, st>>>(h->B, 0.0f, 0);
  }
  kernel_end(h, st);
  if (h->B.any_iid) {
    kernel_begin(h, st, POP_K_GATHER);
    if (h->lay.W == 1) k_select_iid<1><<<grid, kThreads, 0, st>>>(h->B);
    else if (h->lay.W == 2) k_select_iid<2><<<grid, kThreads, 0, st>>>(h->B);
    else k_select_iid<0><<<grid, kThreads, 0, st>>>(h->B);
    kernel_end(h, st);
  }
  return cuda_status(cudaGetLastError());
}

// The fused kernel in the handle's configuration: 128 threads per block with one or two
// clones per lane, or 256 threads with one.
template <int W, bool MOD, bool SCAN, bool FULL>
void launch_fused_form(pop_t* h, unsigned grid, cudaStream_t st, const Batch& Bx, float dt_f, int tile0) {
  if (h->fuse_threads == 256)
    k_gather<W, 256, true, MOD, SCAN, 1, FULL><<<grid, 256, 0, st>>>(Bx, dt_f, tile0);
  else if (h->fuse_clones == 2)
    k_gather<W, 128, true, MOD, SCAN, 2, FULL><<<grid, 128, 0, st>>>(Bx, dt_f, tile0);
  else
    k_gather<W, 128, true, MOD, SCAN, 1, FULL><<<grid, 128, 0, st>>>(Bx, dt_f, tile0);
}

// full: every population of the launch has L = 64 W (the ring fills the lattice words)
template <int W, bool MOD, bool SCAN>
void launch_fused(pop_t* h, unsigned grid, cudaStream_t st, const Batch& Bx, float dt_f, int tile0, bool full) {
  if (full) launch_fused_form<W, MOD, SCAN, true>(h, grid, st, Bx, dt_f, tile0);
  else launch_fused_form<W, MOD, SCAN, false>(h, grid, st, Bx, dt_f, tile0);
}

// pop_run fuses the cloning stage of one interval with the dynamical stage of
// the next when every population uses [eq] selection on a ring of at most 128 sites.
bool fusable(const pop_t* h) {
  return h->lay.W >= 1 && h->lay.W <= 2 && !h->B.any_iid && !h->guided;
}

// Cloning stage of the current interval and dynamical stage of the next one, for
// the tiles [tile0, tile0 + ntiles) (whole populations) with the batch view Bx.
// after_fused: the current interval's dynamical stage was a fused launch of this
// configuration, so with Bx.hist_on its tile histograms stand in for k_weights.
int launch_resample_evolve_range(pop_t* h, cudaStream_t st, float dt_f, const Batch& Bx,
                                 int tile0, int ntiles, int pop0, int pop1, bool after_fused) {
  const unsigned grid = (unsigned)ntiles;
  bool scan = true;
  if (after_fused && Bx.hist_on) {
    launch_tile_scan(h, st, Bx, pop0, pop1, true);
  } else {
    launch_weights_range(h, st, Bx, tile0, ntiles);
    // the tile prefixes from k_tile_scan when every population here has many tiles; a
    // population of a few tiles is cheaper to sum inside the fused kernel than to scan
    // in one more launch per interval
    for (int p = pop0; p < pop1; ++p) scan = scan && h->desc[p].ntiles > kScanTiles;
    if (scan) launch_tile_scan(h, st, Bx, pop0, pop1);
  }
  bool full = true;
  for (int p = pop0; p < pop1; ++p) full = full && h->desc[p].L == 64 * h->lay.W;
  kernel_begin(h, st, POP_K_GATHER_EVOLVE);
  if (h->lay.W == 1) {
    if (h->any_mod) {
      if (scan) launch_fused<1, true, true>(h, grid, st, Bx, dt_f, tile0, full);
      else launch_fused<1, true, false>(h, grid, st, Bx, dt_f, tile0, full);
    } else {
      if (scan) launch_fused<1, false, true>(h, grid, st, Bx, dt_f, tile0, full);
      else launch_fused<1, false, false>(h, grid, st, Bx, dt_f, tile0, full);
    }
  } else {
    if (h->any_mod) {
      if (scan) launch_fused<2, true, true>(h, grid, st, Bx, dt_f, tile0, full);
      else launch_fused<2, true, false>(h, grid, st, Bx, dt_f, tile0, full);
    } else {
      if (scan) launch_fused<2, false, true>(h, grid, st, Bx, dt_f, tile0, full);
      else launch_fused<2, false, false>(h, grid, st, Bx, dt_f, tile0, full);
    }
  }
  kernel_end(h, st);
  return cuda_status(cudaGetLastError());
}


// pop_run's chains: the largest K <= want of choose_chains, each chain a copy of the
// batch with its own interval counter (the counter word after the batch's own).
void set_chains(pop_t* h, int want) {
  h->nch = 1;
  h->chain_tile[0] = 0;
  h->chain_tile[1] = h->lay.ntiles;
  if (fusable(h) && want > 1) h->nch = choose_chains(h->desc, h->lay.ntiles, want, h->chain_tile);
  for (int c = 0, p = 0; c <= h->nch; ++c) {  // chains hold whole populations
    while (p < h->lay.P && h->desc[p].first_tile < h->chain_tile[c]) ++p;
    h->chain_pop[c] = p;
  }
  for (int c = 0; c < h->nch; ++c) {
    h->chain[c] = h->B;
    h->chain[c].beta = h->B.beta + 1 + c;
  }
}

// Whether the fused stage fills the tile histograms for this dt (pop_tuning hist_mode):
// only without MODIFIED weights, and by the rule when every population has more than
// kScanTiles tiles (so the tile scan runs in every interval anyway; for fewer tiles
// k_weights' many short blocks and the fused stage's own tile sums are faster than one
// scan block per population) and dt * (largest L) <= 16, where the number of hops of a
// clone in one interval stays far below 64 (the escape rate is at most L).
void set_hist(pop_t* h, float dt_f) {
  bool many_tiles = true;
  for (const PopDesc& d : h->desc) many_tiles = many_tiles && d.ntiles > kScanTiles;
  const bool on = fusable(h) && !h->any_mod &&
                  (h->hist_mode == 1 ||
                   (h->hist_mode == -1 && many_tiles && (double)dt_f * h->max_L <= 16.0));
  h->B.hist_on = on ? 1 : 0;
  for (int c = 0; c < kMaxChains; ++c) h->chain[c].hist_on = h->B.hist_on;
}

// The rule pop_init starts from: in a batch of at most two waves of the fused kernel
// the drain at the end of each launch and the k_weights between launches are a large
// part of an interval, and more chains fill them; in a larger batch more chains only
// compete.
int size_chains(pop_t* h) {
  int want = 1;
  if (fusable(h)) {
    const void* f = h->lay.W == 1
                        ? (h->any_mod ? (const void*)k_gather<1, 128, true, true, false, 1>
                                      : (const void*)k_gather<1, 128, true, false, false, 1>)
                        : (h->any_mod ? (const void*)k_gather<2, 128, true, true, false, 1>
                                      : (const void*)k_gather<2, 128, true, false, false, 1>);
    int per_sm = 0, sms = 0;
    POP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 128, 0));
    POP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const long long wave = (long long)(per_sm < 1 ? 1 : per_sm) * sms;
    want = h->lay.ntiles <= 2 * wave ? POP_RUN_CHAINS : POP_RUN_CHAINS_LARGE;
  }
  set_chains(h, want);
  return POP_OK;
}

// Persistent evolve grid: as many blocks as fit on the device at once, each
// owning an equal share of the 256-slot units.
template <int W, bool MOD>
int size_evolve_grid(pop_t* h) {
  const size_t smem = sizeof(EvolveSmem<W>);
  POP_CUDA(cudaFuncSetAttribute(k_evolve<W, MOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int per_sm = 0, sms = 0;
  POP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_evolve<W, MOD>, kThreads, smem));
  POP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  if (per_sm < 1) per_sm = 1;
  const long long want = (long long)per_sm * sms;
  h->evolve_grid = (int)(want < h->lay.nunits ? want : h->lay.nunits);
  h->evolve_grid_cap = h->evolve_grid;
  h->evolve_smem = smem;
  h->B.unit_q = h->lay.nunits / h->evolve_grid;
  h->B.unit_r = h->lay.nunits % h->evolve_grid;
  return POP_OK;
}

// Re-split the units over a different persistent grid (k_evolve only).
void set_evolve_grid(pop_t* h, int grid) {
  if (grid < 1) grid = 1;
  if (h->lay.W <= 2 && grid > h->lay.nunits) grid = h->lay.nunits;
  h->evolve_grid = grid;
  h->B.unit_q = h->lay.nunits / grid;
  h->B.unit_r = h->lay.nunits % grid;
}

// Rings longer than 128 sites: one warp per clone, a grid-stride loop over slots.
template <bool MOD>
int size_evolve_grid_wide(pop_t* h) {
  int per_sm = 0, sms = 0;
  POP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_evolve_wide<MOD>, kThreads, 0));
  POP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  if (per_sm < 1) per_sm = 1;
  const long long want = (long long)per_sm * sms;
  const long long need = (h->lay.nslots + kWarps - 1) / kWarps;
  h->evolve_grid = (int)(want < need ? want : need);
  h->evolve_grid_cap = h->evolve_grid;
  h->evolve_smem = 0;
  return POP_OK;
}

// n fused intervals over the chains: chain 0 on st, the others on the auxiliary
// streams forked from st and joined back into it, each chain with its own interval
// counter (copy_chain_counters brings them in line with the batch's counter before and
// the batch's back from chain 0 after).  after_fused: the interval before the first
// was itself a fused one (its tile histograms are pending).
int run_chains(pop_t* h, cudaStream_t st, float dt_f, int64_t n, bool after_fused) {
  if (n > 0) h->hist_pending = h->B.hist_on != 0;
  if (h->nch == 1) {
    int lr = POP_OK;
    for (int64_t i = 0; i < n && lr == POP_OK; ++i) {
      if (h->timer_base >= 0) h->timer_interval = h->timer_base + (int)i;
      lr = launch_resample_evolve_range(h, st, dt_f, h->chain[0], 0, h->lay.ntiles, 0, h->lay.P,
                                        after_fused || i > 0);
    }
    return lr;
  }
  if (cudaEventRecord(h->ev_fork, st) != cudaSuccess) return POP_ERR_CUDA;
  for (int c = 0; c + 1 < h->nch; ++c)
    if (cudaStreamWaitEvent(h->aux_stream[c], h->ev_fork, 0) != cudaSuccess) return POP_ERR_CUDA;
  int lr = POP_OK;
  for (int64_t i = 0; i < n && lr == POP_OK; ++i)
    for (int c = 0; c < h->nch && lr == POP_OK; ++c) {
      if (h->timer_base >= 0) h->timer_interval = h->timer_base + (int)i;
      lr = launch_resample_evolve_range(h, c == 0 ? st : h->aux_stream[c - 1], dt_f, h->chain[c],
                                        h->chain_tile[c], h->chain_tile[c + 1] - h->chain_tile[c],
                                        h->chain_pop[c], h->chain_pop[c + 1], after_fused || i > 0);
    }
  // the joins are made even after a failed launch, so a capture can end cleanly
  for (int c = 0; c + 1 < h->nch; ++c)
    if (cudaEventRecord(h->ev_join[c], h->aux_stream[c]) != cudaSuccess ||
        cudaStreamWaitEvent(st, h->ev_join[c], 0) != cudaSuccess)
      return POP_ERR_CUDA;
  return lr;
}

cudaError_t copy_chain_counters(pop_t* h, bool to_chains) {
  for (int c = 0; c < h->nch; ++c) {
    if (!to_chains && c > 0) break;
    const cudaError_t e = to_chains ? cudaMemcpyAsync(h->chain[c].beta, h->B.beta, sizeof(unsigned int),
                                                      cudaMemcpyDeviceToDevice, h->stream)
                                    : cudaMemcpyAsync(h->B.beta, h->chain[0].beta, sizeof(unsigned int),
                                                      cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int check_device_errors(pop_t* h, std::vector<PopState>* out) {
  std::vector<PopState> st((size_t)h->lay.P);
  POP_CUDA(cudaMemcpyAsync(st.data(), h->ws + h->lay.o_st, st.size() * sizeof(PopState),
                           cudaMemcpyDeviceToHost, h->stream));
  POP_CUDA(cudaStreamSynchronize(h->stream));
  for (const PopState& q : st)
    if (q.err != 0) return q.err;
  if (out) *out = std::move(st);
  return POP_OK;
}

}  // namespace

extern "C" {

size_t pop_workspace_bytes(const pop_params* params, int32_t n_pops) {
  Layout l;
  if (!make_layout(params, n_pops, &l)) return 0;
  return l.total;
}

int32_t pop_lattice_words(const pop_params* params, int32_t n_pops) {
  Layout l;
  if (!make_layout(params, n_pops, &l)) return 0;
  return l.W;
}

int pop_init(pop_t** out, const pop_params* params, int32_t n_pops, void* d_workspace,
             size_t workspace_bytes, void* cuda_stream) {
  if (out == nullptr) return POP_ERR_ARG;
  *out = nullptr;
  Layout lay;
  if (!make_layout(params, n_pops, &lay)) return POP_ERR_ARG;
  if (d_workspace == nullptr || workspace_bytes < lay.total) return POP_ERR_ARG;
  if (((uintptr_t)d_workspace & 255u) != 0) return POP_ERR_ARG;

  pop_t* h = new (std::nothrow) pop_batch();
  if (h == nullptr) return POP_ERR_ARG;
  h->lay = lay;
  h->params.assign(params, params + n_pops);
  for (int32_t p = 0; p < n_pops; ++p) h->max_L = std::max(h->max_L, (int)params[p].L);
  h->stream = (cudaStream_t)cuda_stream;
  h->ws = (unsigned char*)d_workspace;
  auto fail = [&](int rc) { pop_free(h); return rc; };
  if (cudaGetDevice(&h->device) != cudaSuccess) return fail(POP_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(POP_ERR_CUDA);

  // per-population descriptors and the tile map
  std::vector<int32_t> tile_pop((size_t)lay.ntiles);
  h->desc.resize((size_t)n_pops);
  int32_t tile = 0;
  for (int32_t p = 0; p < n_pops; ++p) {
    PopDesc& d = h->desc[p];
    d.L = params[p].L;
    d.N = params[p].N;
    d.nc = params[p].n_clones;
    d.seed = params[p].seed;
    d.first_tile = tile;
    d.ntiles = (int32_t)((params[p].n_clones + kTile - 1) / kTile);
    d.off = (int64_t)tile * kTile;
    d.s = 0.0;
    d.abs_s = 0.0;
    d.s_neg = 0;
    d.guided = params[p].weight_mode == POP_GUIDED ? 1 : 0;
    // GUIDED weights take the continuous-weight path of MODIFIED (log weight in A)
    d.modified = (params[p].weight_mode == POP_MODIFIED || d.guided) ? 1 : 0;
    d.iid = params[p].selection == POP_IID ? 1 : 0;
    d.F = 61 - ceil_log2(params[p].n_clones);
    d.c_f = 0.0f;
    d.s_q = 0;
    d.c_s = 0.0f;
    h->guided = d.guided != 0;
    h->any_mod = h->any_mod || d.modified;
    h->B.any_iid = h->B.any_iid || d.iid;
    for (int32_t t = 0; t < d.ntiles; ++t) tile_pop[(size_t)tile + t] = p;
    tile += d.ntiles;
  }
  // float(1/r): the plain SSEP escape rate is the number r of active bonds
  std::vector<float> inv((size_t)n_pops * kInvStride, 0.0f);
  for (int32_t p = 0; p < n_pops; ++p)
    for (int r = 1; r <= params[p].L; ++r) inv[(size_t)p * kInvStride + r] = 1.0f / (float)r;
  // waiting-time logarithm: c_i = 1 + (i + 1/2)/64, (float(1/c_i), float(ln c_i))
  std::vector<float2> logtab(64);
  for (int i = 0; i < 64; ++i) {
    const double c = 1.0 + ((double)i + 0.5) / 64.0;
    logtab[i] = make_float2((float)(1.0 / c), (float)std::log(c));
  }
  std::vector<PopState> st((size_t)n_pops);
  for (PopState& q : st) {
    std::memset(&q, 0, sizeof q);
    for (int par = 0; par < 2; ++par) {
      q.dk_min[par] = INT_MAX;
      q.dk_max[par] = INT_MIN;
      q.a_min[par] = INT_MAX;
      q.a_max[par] = INT_MIN;
    }
  }
  // GUIDED rate tables: TA[a] = nearest(2^44 exp(a/64 - 8)), TB[c] = nearest(2^40 exp(c/2^17))
  std::vector<unsigned long long> gtab((size_t)(kGuideTabA + kGuideTabB));
  for (int a = 0; a < kGuideTabA; ++a)
    gtab[(size_t)a] = (unsigned long long)std::nearbyint(std::ldexp(std::exp(a / 64.0 - 8.0), 44));
  for (int c = 0; c < kGuideTabB; ++c)
    gtab[(size_t)kGuideTabA + c] =
        (unsigned long long)std::nearbyint(std::ldexp(std::exp(c / 131072.0), 40));
  // MODIFIED weight exponential: 2^(i/64)
  std::vector<float> exp2tab(64);
  for (int i = 0; i < 64; ++i) exp2tab[i] = (float)std::exp2((double)i / 64.0);
  const unsigned int beta0 = 1u;

  unsigned char* ws = h->ws;
  if (cudaMemsetAsync(ws, 0, lay.total, h->stream) != cudaSuccess) return fail(POP_ERR_CUDA);
  if (cudaMemcpyAsync(ws + lay.o_pops, h->desc.data(), h->desc.size() * sizeof(PopDesc),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_st, st.data(), st.size() * sizeof(PopState),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_tile_pop, tile_pop.data(), tile_pop.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_inv, inv.data(), inv.size() * sizeof(float),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_logtab, logtab.data(), logtab.size() * sizeof(float2),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_exp2, exp2tab.data(), exp2tab.size() * sizeof(float),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_gtab, gtab.data(), gtab.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(ws + lay.o_beta, &beta0, sizeof beta0, cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return fail(POP_ERR_CUDA);

  Batch& B = h->B;
  B.pops = (const PopDesc*)(ws + lay.o_pops);
  B.st = (PopState*)(ws + lay.o_st);
  B.tile_pop = (const int32_t*)(ws + lay.o_tile_pop);
  B.wtab = (const unsigned long long*)(ws + lay.o_wtab);
  B.qtab = (const double*)(ws + lay.o_qtab);
  B.qm1tab = (const double*)(ws + lay.o_qm1tab);
  B.inv_rate = (const float*)(ws + lay.o_inv);
  B.logtab = (const float2*)(ws + lay.o_logtab);
  B.exp2tab = (const float*)(ws + lay.o_exp2);
  B.Ab[0] = (float*)(ws + lay.o_A);
  B.Ab[1] = B.Ab[0] + lay.nslots;
  B.S = (unsigned long long*)(ws + lay.o_S);
  B.hist = (unsigned int*)(ws + lay.o_hist);
  B.thist = (unsigned int*)(ws + lay.o_thist);
  B.tile_sum = (unsigned long long*)(ws + lay.o_tile_sum);
  B.tile_excl = (unsigned long long*)(ws + lay.o_tile_excl);
  B.beta = (unsigned int*)(ws + lay.o_beta);
  B.phi = (const int32_t*)(ws + lay.o_phi);
  B.gtab = (const unsigned long long*)(ws + lay.o_gtab);
  B.gdu = (int32_t*)(ws + lay.o_gdu);
  B.gq = (unsigned long long*)(ws + lay.o_gq);
  B.gcar[0] = (unsigned long long*)(ws + lay.o_gcar);
  B.gcar[1] = B.gcar[0] + (size_t)lay.nslots * (8 * lay.W);
  B.ksum = (long long*)(ws + lay.o_ksum);
  B.Xb[0] = (unsigned long long*)(ws + lay.o_X);
  B.Xb[1] = B.Xb[0] + lay.nslots * lay.W;
  B.Y = (unsigned long long*)(ws + lay.o_Y);
  B.KXb[0] = (int32_t*)(ws + lay.o_KX);
  B.KXb[1] = B.KXb[0] + lay.nslots;
  B.KY = (int32_t*)(ws + lay.o_KY);
  B.dKb[0] = (int32_t*)(ws + lay.o_dK);
  B.dKb[1] = B.dKb[0] + lay.nslots;
  B.anc = (int32_t*)(ws + lay.o_anc);
  B.ntiles = lay.ntiles;
  B.nunits = lay.nunits;
  B.nslots = lay.nslots;
  B.W = lay.W;
  if (size_chains(h) != POP_OK) return fail(POP_ERR_CUDA);
  for (int c = 0; c + 1 < kMaxChains; ++c)
    if (cudaStreamCreateWithFlags(&h->aux_stream[c], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join[c], cudaEventDisableTiming) != cudaSuccess)
      return fail(POP_ERR_CUDA);
  const bool mod = h->any_mod;
  const int grc = lay.W == 1 ? (mod ? size_evolve_grid<1, true>(h) : size_evolve_grid<1, false>(h))
                  : lay.W == 2 ? (mod ? size_evolve_grid<2, true>(h) : size_evolve_grid<2, false>(h))
                               : (mod ? size_evolve_grid_wide<true>(h) : size_evolve_grid_wide<false>(h));
  if (grc != POP_OK) return fail(POP_ERR_CUDA);
  if (h->guided) {
    int per_sm = 0, sms = 0;
    const void* f = lay.W == 1 ? (const void*)k_evolve_guided<1> : (const void*)k_evolve_guided<2>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kGuideThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
      return fail(POP_ERR_CUDA);
    const long long want = 2ll * (per_sm < 1 ? 1 : per_sm) * sms;
    while (h->guided_split < 8 && (long long)lay.ntiles * h->guided_split < want) h->guided_split *= 2;
  }

  const unsigned grid = (unsigned)(lay.nslots / kThreads);
  h->launches[POP_K_OTHER] += 1;
  if (lay.W == 1) k_init<1><<<grid, kThreads, 0, h->stream>>>(B);
  else if (lay.W == 2) k_init<2><<<grid, kThreads, 0, h->stream>>>(B);
  else k_init<0><<<grid, kThreads, 0, h->stream>>>(B);
  if (cudaGetLastError() != cudaSuccess) return fail(POP_ERR_CUDA);
  // host tables above are stack vectors: wait until their copies have landed
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(POP_ERR_CUDA);
  *out = h;
  return POP_OK;
}

int pop_set_state(pop_t* h, int32_t p, const uint64_t* h_lattice, const int32_t* h_K) {
  if (h == nullptr || p < 0 || p >= h->lay.P || h_lattice == nullptr) return POP_ERR_ARG;
  if (h->intervals != 0 || h->phase != kReady) return POP_ERR_STATE;
  const pop_params& q = h->params[p];
  const int W = h->lay.W;
  for (int64_t j = 0; j < q.n_clones; ++j) {
    int n = 0;
    for (int w = 0; w < W; ++w) {
      uint64_t v = h_lattice[j * W + w];
      const int lo = 64 * w;
      if (q.L < lo + 64) {
        const int keep = q.L - lo;
        const uint64_t mask = keep <= 0 ? 0ull : (keep >= 64 ? ~0ull : ((1ull << keep) - 1ull));
        if (v & ~mask) return POP_ERR_ARG;
      }
      n += __builtin_popcountll(v);
    }
    if (n != q.N) return POP_ERR_ARG;
  }
  const PopDesc& d = h->desc[p];
  POP_CUDA(cudaMemcpyAsync(h->B.Y + d.off * W, h_lattice, (size_t)q.n_clones * W * 8u,
                           cudaMemcpyHostToDevice, h->stream));
  if (h_K != nullptr) {
    POP_CUDA(cudaMemcpyAsync(h->B.KY + d.off, h_K, (size_t)q.n_clones * 4u,
                             cudaMemcpyHostToDevice, h->stream));
  } else {
    POP_CUDA(cudaMemsetAsync(h->B.KY + d.off, 0, (size_t)q.n_clones * 4u, h->stream));
  }
  POP_CUDA(cudaStreamSynchronize(h->stream));
  return POP_OK;
}

int pop_evolve(pop_t* h, double dt, const double* s) {
  if (h == nullptr || !valid_dt(dt)) return POP_ERR_ARG;
  if (h->phase != kReady) return POP_ERR_STATE;
  const int rc = fix_biases(h, s);
  if (rc != POP_OK) return rc;
  const int lr = launch_evolve(h, h->stream, (float)dt);
  if (lr != POP_OK) return lr;
  h->phase = kEvolved;
  h->t_obs += dt;
  return POP_OK;
}

int pop_resample(pop_t* h) {
  if (h == nullptr) return POP_ERR_ARG;
  if (h->phase != kEvolved) return POP_ERR_STATE;
  const int lr = launch_resample(h, h->stream);
  if (lr != POP_OK) return lr;
  h->phase = kReady;
  h->intervals += 1;
  return POP_OK;
}

int pop_run(pop_t* h, double dt, const double* s, int64_t n_intervals) {
  if (h == nullptr || !valid_dt(dt) || n_intervals < 0) return POP_ERR_ARG;
  if (h->phase != kReady) return POP_ERR_STATE;
  int rc = fix_biases(h, s);
  if (rc != POP_OK) return rc;
  if (n_intervals == 0) return POP_OK;
  const float dt_f = (float)dt;
  // fused: evolve, then (n - 1) x [weights, gather + next evolve] over the chains, then
  // weights, gather; otherwise n x [evolve, weights, gather].  The graph holds
  // kGraphIntervals of the repeated part.  The first fused interval follows the
  // separate dynamical stage, so it runs before the graph, whose intervals all follow
  // a fused one (with tile histograms, their weights come from those).
  const bool fuse = fusable(h);
  set_hist(h, dt_f);
  if (fuse) {
    rc = launch_evolve(h, h->stream, dt_f);
    if (rc != POP_OK) return rc;
    POP_CUDA(copy_chain_counters(h, true));
    if (n_intervals > 1) {
      rc = run_chains(h, h->stream, dt_f, 1, false);
      if (rc != POP_OK) return rc;
    }
  }
  const int64_t n_rep = fuse ? (n_intervals > 1 ? n_intervals - 2 : 0) : n_intervals;
  const int64_t n_graph = n_rep / kGraphIntervals;
  const int64_t n_rest = n_rep % kGraphIntervals;
  auto block = [&](cudaStream_t st, int64_t n) {
    if (fuse) return run_chains(h, st, dt_f, n, true);
    int lr = POP_OK;
    for (int64_t i = 0; i < n && lr == POP_OK; ++i) {
      lr = launch_evolve(h, st, dt_f);
      if (lr == POP_OK) lr = launch_resample(h, st);
    }
    return lr;
  };
  if (n_graph > 0 && (h->graph == nullptr || h->graph_dt != dt_f || h->graph_hist != h->B.hist_on)) {
    if (h->graph != nullptr) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    POP_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    for (uint64_t& c : h->graph_counts) c = 0;
    h->count = h->graph_counts;
    const int lr = block(h->capture_stream, kGraphIntervals);
    h->count = h->launches;
    const cudaError_t ec = cudaStreamEndCapture(h->capture_stream, &g);
    if (lr != POP_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return POP_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->graph = nullptr;
      return POP_ERR_CUDA;
    }
    h->graph_dt = dt_f;
    h->graph_hist = h->B.hist_on;
  }
  for (int64_t i = 0; i < n_graph; ++i) {
    POP_CUDA(cudaGraphLaunch(h->graph, h->stream));
    for (int k = 0; k < POP_NKINDS; ++k) h->launches[k] += h->graph_counts[k];
  }
  if (n_rest > 0) {
    rc = block(h->stream, n_rest);
    if (rc != POP_OK) return rc;
  }
  if (fuse) {
    POP_CUDA(copy_chain_counters(h, false));
    rc = launch_resample(h, h->stream);
    if (rc != POP_OK) return rc;
  }
  h->intervals += n_intervals;
  h->t_obs += (double)n_intervals * dt;
  return POP_OK;
}

int pop_kernel_times(pop_t* h, double dt, const double* s, int64_t n_intervals, int32_t per_step,
                     double* h_us, int64_t* h_n, uint64_t* h_hops) {
  if (h == nullptr || !valid_dt(dt) || n_intervals < 1) return POP_ERR_ARG;
  if (h->phase != kReady) return POP_ERR_STATE;
  int rc = fix_biases(h, s);
  if (rc != POP_OK) return rc;
  auto total_hops = [&](uint64_t* out) {
    std::vector<PopState> st;
    const int r = check_device_errors(h, &st);
    uint64_t sum = 0;
    for (const PopState& q : st) sum += q.events;
    *out = sum;
    return r;
  };
  uint64_t hops0 = 0, hops1 = 0, hops2 = 0;
  rc = total_hops(&hops0);
  if (rc != POP_OK) return rc;
  std::vector<cudaEvent_t> events;
  std::vector<int> kinds, ivs;
  events.reserve((size_t)(6 * (n_intervals + 2) * h->nch));
  cudaEvent_t origin = nullptr;
  POP_CUDA(cudaEventCreate(&origin));
  POP_CUDA(cudaEventRecord(origin, h->stream));
  h->timer_events = &events;
  h->timer_kinds = &kinds;
  h->timer_intervals = &ivs;
  h->timer_interval = 0;
  const float dt_f = (float)dt;
  const bool fuse = per_step == 0 && fusable(h);
  set_hist(h, dt_f);
  // the same launches, in the same order and on the same streams, as pop_run (or the
  // per-step calls), each interval's launches tagged with its index
  if (fuse) {
    rc = launch_evolve(h, h->stream, dt_f);
    if (rc == POP_OK) rc = total_hops(&hops1);
    if (rc == POP_OK) rc = copy_chain_counters(h, true) == cudaSuccess ? POP_OK : POP_ERR_CUDA;
    // the first fused interval as pop_run launches it; the others as one captured graph
    // of run_chains, as pop_run replays them, with event-record nodes around each launch
    if (n_intervals > 1 && rc == POP_OK) {
      h->timer_interval = 1;
      rc = run_chains(h, h->stream, dt_f, 1, false);
    }
    if (n_intervals > 2 && rc == POP_OK) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = POP_ERR_CUDA;
      } else {
        h->timer_capture = true;
        h->timer_base = 2;
        const int lc = run_chains(h, h->capture_stream, dt_f, n_intervals - 2, true);
        h->timer_base = -1;
        h->timer_capture = false;
        const cudaError_t ec = cudaStreamEndCapture(h->capture_stream, &g);
        if (lc != POP_OK || ec != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess ||
            cudaGraphLaunch(ge, h->stream) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess)
          rc = POP_ERR_CUDA;
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
      }
    }
    h->timer_interval = (int)n_intervals;
    if (rc == POP_OK) rc = copy_chain_counters(h, false) == cudaSuccess ? POP_OK : POP_ERR_CUDA;
    if (rc == POP_OK) rc = launch_resample(h, h->stream);
  } else {
    for (int64_t i = 0; i < n_intervals && rc == POP_OK; ++i) {
      h->timer_interval = (int)i;
      rc = launch_evolve(h, h->stream, dt_f);
      if (rc == POP_OK) rc = launch_resample(h, h->stream);
    }
  }
  h->timer_events = nullptr;
  h->timer_kinds = nullptr;
  h->timer_intervals = nullptr;
  if (rc == POP_OK) rc = total_hops(&hops2);
  // per kind: the time during which at least one of its launches runs (the union of
  // the launches' [start, end] from the common origin event; the chains' launches run
  // side by side and drift apart over the graph), per interval that launches the kind
  std::vector<std::vector<std::pair<double, double>>> runs(POP_NKINDS);
  std::vector<std::vector<char>> seen(POP_NKINDS, std::vector<char>((size_t)n_intervals + 1, 0));
  int64_t cnt[POP_NKINDS] = {};
  for (size_t i = 0; i < kinds.size() && rc == POP_OK; ++i) {
    float a = 0.0f, b = 0.0f;
    if (cudaEventElapsedTime(&a, origin, events[2 * i]) != cudaSuccess ||
        cudaEventElapsedTime(&b, origin, events[2 * i + 1]) != cudaSuccess) {
      rc = POP_ERR_CUDA;
      break;
    }
    runs[kinds[i]].emplace_back((double)a, (double)b);
    seen[kinds[i]][ivs[i]] = 1;
    cnt[kinds[i]] += 1;
  }
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  cudaEventDestroy(origin);
  if (rc != POP_OK) return rc;
  h->intervals += n_intervals;
  h->t_obs += (double)n_intervals * dt;
  for (int k = 0; k < POP_NKINDS; ++k) {
    std::vector<std::pair<double, double>>& r = runs[k];
    std::sort(r.begin(), r.end());
    double sum = 0.0, lo = 0.0, hi = -1e300;
    for (const auto& x : r) {
      if (x.first > hi) {
        if (hi > lo) sum += hi - lo;
        lo = x.first;
        hi = x.second;
      } else {
        hi = std::max(hi, x.second);
      }
    }
    if (hi > lo) sum += hi - lo;
    int64_t groups = 0;
    for (char c : seen[k]) groups += c;
    if (h_us) h_us[k] = groups ? 1e3 * sum / (double)groups : 0.0;
    if (h_n) h_n[k] = cnt[k];
    if (h_hops) h_hops[k] = 0;
  }
  if (h_hops) {
    if (fuse) {
      h_hops[POP_K_EVOLVE] = hops1 - hops0;
      h_hops[POP_K_GATHER_EVOLVE] = hops2 - hops1;
    } else {
      h_hops[POP_K_EVOLVE] = hops2 - hops0;
    }
  }
  return POP_OK;
}

int32_t pop_run_chains(pop_t* h, int32_t* h_first_tiles) {
  if (h == nullptr) return -1;
  const int32_t n = fusable(h) ? h->nch : 0;
  if (h_first_tiles != nullptr && n > 0)
    for (int c = 0; c <= n; ++c) h_first_tiles[c] = h->chain_tile[c];
  return n;
}

int pop_launch_count(pop_t* h, uint64_t* h_n) {
  if (h == nullptr || h_n == nullptr) return POP_ERR_ARG;
  for (int k = 0; k < POP_NKINDS; ++k) h_n[k] = h->launches[k];
  return POP_OK;
}

int pop_estimate_psi(pop_t* h, double* psi, double* k_hat, double* t_obs) {
  if (h == nullptr) return POP_ERR_ARG;
  if (h->phase != kReady || h->intervals == 0) return POP_ERR_STATE;
  POP_CUDA(cudaMemsetAsync(h->B.ksum, 0, (size_t)h->lay.P * sizeof(long long), h->stream));
  h->launches[POP_K_OTHER] += 1;
  k_ksum<<<(unsigned)(h->lay.nslots / kThreads), kThreads, 0, h->stream>>>(h->B);
  POP_CUDA(cudaGetLastError());
  std::vector<long long> ks((size_t)h->lay.P);
  POP_CUDA(cudaMemcpyAsync(ks.data(), h->B.ksum, ks.size() * sizeof(long long),
                           cudaMemcpyDeviceToHost, h->stream));
  std::vector<PopState> st;
  const int rc = check_device_errors(h, &st);
  if (rc != POP_OK) return rc;
  for (int32_t p = 0; p < h->lay.P; ++p) {
    const pop_params& q = h->params[p];
    if (psi) psi[p] = st[p].psi_acc / h->t_obs;
    if (k_hat) k_hat[p] = (double)ks[p] / ((double)q.n_clones * (double)q.L * h->t_obs);
  }
  if (t_obs) *t_obs = h->t_obs;
  return POP_OK;
}

int pop_copy_state(pop_t* h, int32_t p, uint64_t* h_lattice, int32_t* h_K, int32_t* h_anc,
                   int32_t* h_dK) {
  if (h == nullptr || p < 0 || p >= h->lay.P) return POP_ERR_ARG;
  const PopDesc& d = h->desc[p];
  const int W = h->lay.W;
  const bool evolved = h->phase == kEvolved;
  // the interval most recently evolved and its buffer parity
  const int64_t last = h->intervals + (evolved ? 1 : 0);
  const int par = (int)(last & 1);
  const unsigned long long* lat = evolved ? h->B.Xb[par] : h->B.Y;
  const int32_t* K = evolved ? h->B.KXb[par] : h->B.KY;
  if (h_lattice)
    POP_CUDA(cudaMemcpyAsync(h_lattice, lat + d.off * W, (size_t)d.nc * W * 8u,
                             cudaMemcpyDeviceToHost, h->stream));
  if (h_K)
    POP_CUDA(cudaMemcpyAsync(h_K, K + d.off, (size_t)d.nc * 4u, cudaMemcpyDeviceToHost,
                             h->stream));
  if (h_anc)
    POP_CUDA(cudaMemcpyAsync(h_anc, h->B.anc + d.off, (size_t)d.nc * 4u,
                             cudaMemcpyDeviceToHost, h->stream));
  if (h_dK)
    POP_CUDA(cudaMemcpyAsync(h_dK, h->B.dKb[par] + d.off, (size_t)d.nc * 4u, cudaMemcpyDeviceToHost,
                             h->stream));
  return check_device_errors(h, nullptr);
}

int pop_set_potential(pop_t* h, int32_t p, const float* h_phi) {
  if (h == nullptr || p < 0 || p >= h->lay.P || h_phi == nullptr) return POP_ERR_ARG;
  if (!h->desc[p].guided || h->phase != kReady) return POP_ERR_STATE;
  std::vector<int32_t> q(512);
  for (int i = 0; i < 512; ++i) {
    if (!(std::fabs(h_phi[i]) <= 64.0f)) return POP_ERR_ARG;
    q[i] = (int32_t)std::nearbyint(std::ldexp((double)h_phi[i], 16));
  }
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_phi + (size_t)p * 512 * sizeof(int32_t), q.data(),
                           512 * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  // the clones' carried rate sums were those of the old potential
  const int32_t zero = 0;
  POP_CUDA(cudaMemcpyAsync(h->ws + h->lay.o_st + (size_t)p * sizeof(PopState) + offsetof(PopState, gcarry),
                           &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
  // the bond table of this population, and (once s is fixed) every rate table
  h->launches[POP_K_OTHER] += 1;
  k_guided_table<<<(unsigned)(kGuideSeg / kThreads), kThreads, 0, h->stream>>>(h->B, p);
  POP_CUDA(cudaGetLastError());
  h->guided_q_stale = true;
  if (h->s_fixed) {
    const int rc = guided_rate_tables(h);
    if (rc != POP_OK) return rc;
  }
  POP_CUDA(cudaStreamSynchronize(h->stream));
  return POP_OK;
}

int pop_lineage(pop_t* h, const int32_t* d_in, int32_t* d_out) {
  if (h == nullptr || d_in == nullptr || d_out == nullptr || d_in == d_out) return POP_ERR_ARG;
  if (h->intervals == 0 || h->phase != kReady) return POP_ERR_STATE;
  h->launches[POP_K_OTHER] += 1;
  k_lineage<<<(unsigned)(h->lay.nslots / kThreads), kThreads, 0, h->stream>>>(h->B, d_in, d_out);
  return cuda_status(cudaGetLastError());
}

int64_t pop_slots(pop_t* h) { return h == nullptr ? -1 : h->lay.nslots; }

int64_t pop_first_slot(pop_t* h, int32_t p) {
  if (h == nullptr || p < 0 || p >= h->lay.P) return -1;
  return h->desc[p].off;
}

int pop_events(pop_t* h, uint64_t* h_events) {
  if (h == nullptr || h_events == nullptr) return POP_ERR_ARG;
  std::vector<PopState> st;
  const int rc = check_device_errors(h, &st);
  if (rc != POP_OK) return rc;
  for (int32_t p = 0; p < h->lay.P; ++p) h_events[p] = st[p].events;
  return POP_OK;
}

int pop_autotune(pop_t* h, double dt, const double* s, int32_t trials, int32_t* h_evolve_grid) {
  if (h == nullptr || !valid_dt(dt) || trials < 1) return POP_ERR_ARG;
  if (h->phase != kReady || h->intervals != 0) return POP_ERR_STATE;
  int rc = fix_biases(h, s);
  if (rc != POP_OK) return rc;
  // Every trial runs from interval 1 on the initial population (the fused intervals and
  // the dynamical stage write only the evolved buffers; a trial of the separate cloning
  // stage writes the population, which is kept in the free evolved buffers of the even
  // parity meanwhile); the per-population counters, the interval counters and the
  // activities are put back afterwards, so tuning changes no result.
  std::vector<PopState> saved((size_t)h->lay.P);
  POP_CUDA(cudaMemcpyAsync(saved.data(), h->ws + h->lay.o_st, saved.size() * sizeof(PopState),
                           cudaMemcpyDeviceToHost, h->stream));
  POP_CUDA(cudaStreamSynchronize(h->stream));
  const unsigned int beta1 = 1u;
  set_hist(h, (float)dt);
  auto restore = [&]() {
    if (cudaMemcpyAsync(h->ws + h->lay.o_st, saved.data(), saved.size() * sizeof(PopState),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return false;
    for (int c = 0; c <= kMaxChains; ++c)
      if (cudaMemcpyAsync(h->B.beta + c, &beta1, sizeof beta1, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return false;
    h->hist_pending = false;  // a trial may end with its tile histograms filled
    return cudaMemsetAsync(h->B.dKb[0], 0, 2 * (size_t)h->lay.nslots * sizeof(int32_t), h->stream) == cudaSuccess &&
           cudaMemsetAsync(h->B.thist, 0, (size_t)kTH * h->lay.ntiles * sizeof(unsigned int), h->stream) ==
               cudaSuccess &&
           cudaStreamSynchronize(h->stream) == cudaSuccess;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  POP_CUDA(cudaEventCreate(&e0));
  POP_CUDA(cudaEventCreate(&e1));
  const float dt_f = (float)dt;
  // time of `reps` repetitions of a launch sequence after one untimed one, ms per repetition
  auto timed = [&](auto&& seq, int reps, float* ms_out) {
    if (!restore()) return (int)POP_ERR_CUDA;
    int lr = seq(true);
    if (lr == POP_OK && cudaEventRecord(e0, h->stream) != cudaSuccess) lr = POP_ERR_CUDA;
    for (int i = 0; i < reps && lr == POP_OK; ++i) lr = seq(false);
    if (lr == POP_OK && (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      lr = POP_ERR_CUDA;
    float ms = 0.0f;
    if (lr == POP_OK) cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / (float)reps;
    return lr;
  };

  uint64_t launches_before[POP_NKINDS];
  for (int k = 0; k < POP_NKINDS; ++k) launches_before[k] = h->launches[k];
  // (1) the persistent grid of the separate dynamical stage (first interval of a fused
  // run, every interval otherwise): 1 .. the resident blocks per SM, times the SM count
  int sms = 0;
  POP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const int cap = h->evolve_grid_cap;
  const int per_sm = cap / (sms > 0 ? sms : 1);
  int best = cap;
  float best_ms = 1e30f;
  for (int b = per_sm > 0 ? per_sm : 1; b >= 1 && rc == POP_OK; --b) {
    const int grid = per_sm > 0 ? b * sms : cap;
    set_evolve_grid(h, grid);
    float ms = 0.0f;
    rc = timed([&](bool) { return launch_evolve(h, h->stream, dt_f); }, trials, &ms);
    if (rc == POP_OK && ms < best_ms) { best_ms = ms; best = grid; }
    if (per_sm <= 0) break;
  }
  set_evolve_grid(h, best);

  // (2) fused batches: the fused kernel's form (threads per block, clones per lane),
  // the chains of pop_run and, where activities of 64 or more are very unlikely
  // (dt * (largest L) <= 16, no MODIFIED weights), whether the fused stage counts them
  // per tile, by the time per interval of `trials` fused intervals
  if (rc == POP_OK && fusable(h)) {
    const int forms[3][2] = {{128, 1}, {128, 2}, {256, 1}};
    const int wants[4] = {1, 2, 4, 8};
    const int def_threads = h->fuse_threads, def_clones = h->fuse_clones, def_nch = h->nch;
    const int def_hist = h->hist_mode;
    const bool def_on = h->B.hist_on != 0;
    const bool hist_ok = !h->any_mod && (double)dt_f * h->max_L <= 16.0;
    int bt = def_threads, bc = def_clones, bw = def_nch, bh = def_hist;
    float bms = 1e30f, def_ms = 0.0f;
    int last_nch = -1;
    for (int hm = 0; hm < (hist_ok ? 2 : 1) && rc == POP_OK; ++hm)
    for (int f = 0; f < 3 && rc == POP_OK; ++f) {
      last_nch = -1;
      for (int w = 0; w < 4 && rc == POP_OK; ++w) {
        h->fuse_threads = forms[f][0];
        h->fuse_clones = forms[f][1];
        h->hist_mode = hist_ok ? hm : def_hist;
        set_chains(h, wants[w]);
        set_hist(h, dt_f);
        if (h->nch == last_nch) continue;  // the same split as the smaller want
        last_nch = h->nch;
        // `trials` fused intervals captured as a graph, as pop_run replays them (launched
        // one by one, many short chains would be timed by their launch overhead); each
        // follows a fused interval, as in pop_run's graph
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          rc = POP_ERR_CUDA;
          break;
        }
        uint64_t* const count = h->count;
        h->count = h->graph_counts;  // launches made while tuning are not the batch's
        const int lc = run_chains(h, h->capture_stream, dt_f, trials, true);
        h->count = count;
        const cudaError_t ec = cudaStreamEndCapture(h->capture_stream, &g);
        if (lc != POP_OK || ec != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          rc = POP_ERR_CUDA;
          break;
        }
        cudaGraphDestroy(g);
        float ms = 0.0f;
        rc = timed([&](bool first) {
              int lr = POP_OK;
              if (first) {  // as pop_run: the first fused interval follows the dynamical stage
                lr = launch_evolve(h, h->stream, dt_f);
                if (lr == POP_OK && copy_chain_counters(h, true) != cudaSuccess) lr = POP_ERR_CUDA;
                if (lr == POP_OK) lr = run_chains(h, h->stream, dt_f, 1, false);
              }
              if (lr == POP_OK && cudaGraphLaunch(ge, h->stream) != cudaSuccess) lr = POP_ERR_CUDA;
              return lr;
            }, 3, &ms);
        cudaGraphExecDestroy(ge);
        ms /= (float)trials;
        if (rc != POP_OK) break;
        if (forms[f][0] == def_threads && forms[f][1] == def_clones && h->nch == def_nch &&
            (h->B.hist_on != 0) == def_on)
          def_ms = ms;
        if (ms < bms) { bms = ms; bt = forms[f][0]; bc = forms[f][1]; bw = wants[w]; bh = h->hist_mode; }
      }
    }
    h->fuse_threads = bt;
    h->fuse_clones = bc;
    h->hist_mode = bh;
    set_chains(h, bw);
    set_hist(h, dt_f);
    h->tuned_default_us = 1e3f * def_ms;
    h->tuned_us = 1e3f * bms;
  }

  // (3) batches that do not fuse: the separate cloning stage's block size, by the time
  // of whole intervals; the population is kept in the even-parity evolved buffers
  if (rc == POP_OK && !fusable(h)) {
    const size_t lat = (size_t)h->lay.nslots * h->lay.W * sizeof(unsigned long long);
    const size_t ks = (size_t)h->lay.nslots * sizeof(int32_t);
    POP_CUDA(cudaMemcpyAsync(h->B.Xb[0], h->B.Y, lat, cudaMemcpyDeviceToDevice, h->stream));
    POP_CUDA(cudaMemcpyAsync(h->B.KXb[0], h->B.KY, ks, cudaMemcpyDeviceToDevice, h->stream));
    const int def = h->gather_threads;
    float def_ms = 0.0f, bms = 1e30f;
    int bg = def;
    for (int g : {0, 128, 256}) {
      h->gather_threads = g;
      float ms = 0.0f;
      rc = timed([&](bool) {
            int lr = cudaMemcpyAsync(h->B.Y, h->B.Xb[0], lat, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess &&
                             cudaMemcpyAsync(h->B.KY, h->B.KXb[0], ks, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess
                         ? POP_OK : POP_ERR_CUDA;
            if (lr == POP_OK) lr = launch_evolve(h, h->stream, dt_f);
            if (lr == POP_OK) lr = launch_resample(h, h->stream);
            if (lr == POP_OK) {  // the next repetition evolves interval 1 again, from the start
              for (int c = 0; c <= kMaxChains && lr == POP_OK; ++c)
                if (cudaMemcpyAsync(h->B.beta + c, &beta1, sizeof beta1, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                  lr = POP_ERR_CUDA;
              if (lr == POP_OK && cudaMemcpyAsync(h->ws + h->lay.o_st, saved.data(), saved.size() * sizeof(PopState),
                                                  cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                lr = POP_ERR_CUDA;
            }
            return lr;
          }, trials, &ms);
      if (rc != POP_OK) break;
      if (g == def) def_ms = ms;
      if (ms < bms) { bms = ms; bg = g; }
    }
    h->gather_threads = bg;
    POP_CUDA(cudaMemcpyAsync(h->B.Y, h->B.Xb[0], lat, cudaMemcpyDeviceToDevice, h->stream));
    POP_CUDA(cudaMemcpyAsync(h->B.KY, h->B.KXb[0], ks, cudaMemcpyDeviceToDevice, h->stream));
    h->tuned_default_us = 1e3f * def_ms;
    h->tuned_us = 1e3f * bms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int k = 0; k < POP_NKINDS; ++k) h->launches[k] = launches_before[k];
  if (h->graph != nullptr) {  // a captured graph holds the old launch configuration
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (!restore()) return POP_ERR_CUDA;
  if (rc != POP_OK) return rc;
  if (h_evolve_grid) *h_evolve_grid = best;
  return POP_OK;
}

int pop_get_tuning(pop_t* h, pop_tuning* out) {
  if (h == nullptr || out == nullptr) return POP_ERR_ARG;
  out->evolve_grid = h->evolve_grid;
  out->fuse_threads = h->fuse_threads;
  out->fuse_clones = h->fuse_clones;
  out->chains = h->nch;
  out->gather_threads = h->gather_threads;
  out->hist_mode = h->hist_mode;
  out->default_us_per_interval = h->tuned_default_us;
  out->tuned_us_per_interval = h->tuned_us;
  return POP_OK;
}

int pop_set_tuning(pop_t* h, const pop_tuning* cfg) {
  if (h == nullptr || cfg == nullptr) return POP_ERR_ARG;
  if (cfg->evolve_grid < 1 || (cfg->fuse_threads != 128 && cfg->fuse_threads != 256) ||
      (cfg->fuse_clones != 1 && cfg->fuse_clones != 2) || (cfg->fuse_threads == 256 && cfg->fuse_clones != 1) ||
      cfg->chains < 1 || cfg->chains > kMaxChains ||
      (cfg->gather_threads != 0 && cfg->gather_threads != 128 && cfg->gather_threads != 256) ||
      cfg->hist_mode < -1 || cfg->hist_mode > 1)
    return POP_ERR_ARG;
  if (h->phase != kReady) return POP_ERR_STATE;
  set_evolve_grid(h, cfg->evolve_grid);
  h->fuse_threads = cfg->fuse_threads;
  h->fuse_clones = cfg->fuse_clones;
  h->gather_threads = cfg->gather_threads;
  h->hist_mode = cfg->hist_mode;
  set_chains(h, cfg->chains);
  if (h->graph != nullptr) {  // the captured graph holds the old launch configuration
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return POP_OK;
}

int pop_density_mode(pop_t* h, int32_t n, double* h_mean) {
  if (h == nullptr || h_mean == nullptr || n < 0) return POP_ERR_ARG;
  if (h->phase != kReady) return POP_ERR_STATE;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<float2> cs((size_t)h->lay.P * kInvStride, make_float2(0.0f, 0.0f));
  for (int32_t p = 0; p < h->lay.P; ++p) {
    const int L = h->params[p].L;
    for (int x = 0; x < L; ++x) {
      const double th = two_pi * (double)((int64_t)n * x % L) / (double)L;
      cs[(size_t)p * kInvStride + x] = make_float2((float)std::cos(th), (float)std::sin(th));
    }
  }
  float2* d_cs = (float2*)(h->ws + h->lay.o_cs);
  double* d_tacc = (double*)(h->ws + h->lay.o_tacc);
  POP_CUDA(cudaMemcpyAsync(d_cs, cs.data(), cs.size() * sizeof(float2), cudaMemcpyHostToDevice,
                           h->stream));
  const unsigned grid = (unsigned)h->lay.ntiles;
  h->launches[POP_K_OTHER] += 1;
  if (h->lay.W == 1) k_density<1><<<grid, kThreads, 0, h->stream>>>(h->B, d_cs, d_tacc);
  else if (h->lay.W == 2) k_density<2><<<grid, kThreads, 0, h->stream>>>(h->B, d_cs, d_tacc);
  else k_density<0><<<grid, kThreads, 0, h->stream>>>(h->B, d_cs, d_tacc);
  POP_CUDA(cudaGetLastError());
  std::vector<double> tacc((size_t)h->lay.ntiles);
  POP_CUDA(cudaMemcpyAsync(tacc.data(), d_tacc, tacc.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  POP_CUDA(cudaStreamSynchronize(h->stream));
  for (int32_t p = 0; p < h->lay.P; ++p) {
    double sum = 0.0;
    for (int32_t t = 0; t < h->desc[p].ntiles; ++t) sum += tacc[(size_t)h->desc[p].first_tile + t];
    h_mean[p] = sum / (double)h->params[p].n_clones;
  }
  return POP_OK;
}

const char* pop_strerror(int status) {
  switch (status) {
    case POP_OK: return "ok";
    case POP_ERR_ARG: return "invalid argument";
    case POP_ERR_CUDA: return "CUDA runtime error";
    case POP_ERR_RANGE: return "interval activity outside the weight table, or step limit reached";
    case POP_ERR_STATE: return "call out of order or bias changed during a run";
    default: return "unknown status";
  }
}

void pop_free(pop_t* h) {
  if (h == nullptr) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (int c = 0; c + 1 < kMaxChains; ++c) {
    if (h->aux_stream[c]) cudaStreamDestroy(h->aux_stream[c]);
    if (h->ev_join[c]) cudaEventDestroy(h->ev_join[c]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  delete h;
}

}  // extern "C"
