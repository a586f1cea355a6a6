// pop_select_noalloc: the cloning-stage selection of one population for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a process whose device memory is all
// reserved by another allocator (a framework's caching pool), a latency-critical
// loop where an allocation and the synchronisation it implies are not allowed, or
// an embedded runtime without a device allocator.  For them this entry point computes
// the [eq] ancestors and the psi term of one interval from device buffers the
// caller already owns (the interval activities in, the ancestors out).  Its scratch
// (the fixed-point weight table, the FP64 exp/expm1 tables, the activity
// histogram, per-tile weight sums and a few scalars) lives in one file-scope
// static __device__ array of kScratchBytes (120 KiB), held by every GPU that loads
// the library until the process exits.  Every call shares that array: the
// histogram and scalars are cleared at the start of each call, the tables are uploaded
// only when the bias or the weight scale differs from the last upload on that device,
// and calls that overlap on the GPU (two streams, or two host threads) race on it.
// A call synchronises its stream and copies from pageable host memory, so it cannot
// be made on a stream that is being captured into a CUDA graph.
//
// The same arithmetic as k_weights / k_gather of the batch path (pop_kernels.cuh),
// restricted to one population and without the lattice copy, so its ancestors and
// psi term equal those of pop_resample for the same activities.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "pop.h"
#include "pop_common.cuh"

using namespace popgpu;

namespace {

constexpr int64_t kMaxClones = (int64_t)1 << 20;           // POP_NOALLOC_MAX_CLONES
constexpr int kMaxTiles = (int)(kMaxClones / kTile);        // 1024
constexpr int kMaxDevices = 64;

struct SelState {
  int32_t dk_min, dk_max, kref, err;
  uint32_t U, pad;
  double psi_term;
};

// byte offsets into the scratch array
constexpr size_t kOffWtab = 0;
constexpr size_t kOffQ = kOffWtab + (size_t)kKcap * 8;
constexpr size_t kOffQm1 = kOffQ + (size_t)kKcap * 8;
constexpr size_t kOffHist = kOffQm1 + (size_t)kKcap * 8;
constexpr size_t kOffTileSum = kOffHist + (size_t)kKcap * 4;
constexpr size_t kOffState = kOffTileSum + (size_t)kMaxTiles * 8;
constexpr size_t kScratchBytes = kOffState + 256;

static __device__ __align__(256) unsigned char g_select_scratch[kScratchBytes];

// device address of g_select_scratch per device, set on the first call on that device
static unsigned char* g_scratch_ptr[kMaxDevices];

// the bias and weight scale whose tables the array of each device holds (the tables
// depend on nothing else), so a call with the same s and N_c skips their upload
struct TableKey {
  bool valid;
  double s;
  int F;
};
static TableKey g_tables[kMaxDevices];

// host copies of the tables, built per thread outside the stack (96 KiB)
struct HostTables {
  unsigned long long wtab[kKcap];
  double qtab[kKcap], qm1tab[kKcap];
};
static thread_local HostTables t_host;

struct SelArgs {
  const int32_t* dK;
  int32_t* anc;
  unsigned long long* wtab;
  double* qtab;
  double* qm1tab;
  unsigned int* hist;
  unsigned long long* tile_sum;
  SelState* st;
  uint32_t nc;
  int32_t ntiles;
  int32_t s_neg;
  uint32_t beta;
  uint64_t seed;
  double s;
};

__global__ void __launch_bounds__(kThreads) k_sel_range(SelArgs A) {
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  int mn = INT_MAX, mx = INT_MIN;
  for (int i = tid; i < kTile; i += kThreads) {
    if (base + i < (int64_t)A.nc) {
      const int v = A.dK[base + i];
      mn = min(mn, v);
      mx = max(mx, v);
    }
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((tid & 31) == 0 && mn != INT_MAX) {
    atomicMin(&A.st->dk_min, mn);
    atomicMax(&A.st->dk_max, mx);
  }
}

__global__ void __launch_bounds__(kThreads) k_sel_weights(SelArgs A) {
  __shared__ unsigned long long s_red[kWarps];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int64_t base = (int64_t)tile * kTile;
  const int kref = A.s_neg ? A.st->dk_max : A.st->dk_min;
  unsigned long long sum = 0ull;
  bool range_err = false;
  for (int i = tid; i < kTile; i += kThreads) {
    if (base + i < (int64_t)A.nc) {
      const unsigned int k = abs_diff(A.dK[base + i], kref);
      if (k >= (unsigned int)kKcap) {
        range_err = true;
      } else {
        sum += A.wtab[k];
        atomicAdd(&A.hist[k], 1u);
      }
    }
  }
  if (range_err) A.st->err = kErrRange;
  const unsigned long long total = block_sum_u64(sum, s_red);
  if (tid == 0) {
    A.tile_sum[tile] = total;
    if (tile == 0) {
      A.st->kref = kref;
      A.st->U = philox4x32_10(make_uint4(0u, A.beta, 0u, kTagResample), (uint32_t)A.seed,
                              (uint32_t)(A.seed >> 32)).x;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_sel_ancestors(SelArgs A) {
  __shared__ uint32_t s_jlo[kTile + 1];
  __shared__ unsigned long long s_red[kWarps];
  __shared__ unsigned long long s_wsum[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = blockIdx.x;
  const int64_t base = (int64_t)tile * kTile;
  const int kref = A.st->kref;
  const unsigned long long c = 2ull * (unsigned long long)A.st->U + 1ull;
  const uint32_t nc = A.nc;

  unsigned long long tT = 0ull, tE = 0ull;
  for (int i = tid; i < A.ntiles; i += kThreads) {
    const unsigned long long v = A.tile_sum[i];
    tT += v;
    if (i < tile) tE += v;
  }
  unsigned long long w[kItems];
  unsigned long long tsum = 0ull;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t j = base + (int64_t)tid * kItems + i;
    w[i] = 0ull;
    if (j < (int64_t)nc) {
      const unsigned int k = abs_diff(A.dK[j], kref);
      if (k < (unsigned int)kKcap) w[i] = A.wtab[k];
    }
    tsum += w[i];
  }
  unsigned long long xs = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, xs, o);
    if (lane >= o) xs += y;
  }
  if (lane == 31) s_wsum[wid] = xs;
  const unsigned long long T = block_sum_u64(tT, s_red);
  const unsigned long long excl = block_sum_u64(tE, s_red);
  const int sh = max(0, 64 - __clzll((long long)T) - 24);
  const float ratio = __fdiv_rn((float)nc, __uint2float_rn((uint32_t)(T >> sh)));
  unsigned long long run = excl + xs - tsum;
  for (int q = 0; q < wid; ++q) run += s_wsum[q];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    s_jlo[tid * kItems + i] = j_lo(run, T, c, nc, sh, ratio);
    run += w[i];
  }
  if (tid == kThreads - 1) s_jlo[kTile] = j_lo(run, T, c, nc, sh, ratio);
  __syncthreads();
  // old clone k of this tile is the ancestor of new clones [s_jlo[k], s_jlo[k+1])
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int k = tid * kItems + i;
    for (uint32_t jj = s_jlo[k]; jj < s_jlo[k + 1]; ++jj) A.anc[jj] = (int32_t)(base + k);
  }

  // psi term of this interval (same arithmetic as the batch path)
  if (tile == 0 && wid == 0) {
    const int R = hist_bins(A.st->dk_min, A.st->dk_max, kKcap);
    double a = 0.0, q = 0.0;
    for (int b = lane; b < R; b += 32) {
      const unsigned int cnt = A.hist[b];
      if (cnt) {
        a = fma((double)cnt, A.qm1tab[b], a);
        q = fma((double)cnt, A.qtab[b], q);
      }
    }
    a = warp_sum_f64(a);
    q = warp_sum_f64(q);
    if (lane == 0) {
      const double ncd = (double)nc;
      const double mean_q = q / ncd;
      const double ln_mean = (mean_q > 0.5) ? log1p(a / ncd) : log(mean_q);
      A.st->psi_term = -A.s * (double)kref + ln_mean;
    }
  }
}

int ceil_log2(int64_t x) {
  int c = 0;
  while (((int64_t)1 << c) < x) ++c;
  return c;
}

}  // namespace

extern "C" int pop_select_noalloc(const int32_t* d_dK, int64_t n_clones, double s, uint64_t seed,
                                  uint32_t interval, int32_t* d_anc, double* h_psi_term,
                                  void* cuda_stream) {
  if (d_dK == nullptr || d_anc == nullptr || n_clones < 1 || n_clones > kMaxClones ||
      !std::isfinite(s) || interval < 1u)
    return POP_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return POP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return POP_ERR_ARG;
  // set-up, once per device, with that device current: the device address of the
  // scratch array (its host-side name is only a stand-in for the symbol)
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || p == nullptr)
      return POP_ERR_CUDA;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  unsigned char* scratch = g_scratch_ptr[dev];
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // tables of this bias (the same definitions as the batch path); uploaded only when
  // the array does not already hold those of this (s, F)
  const int F = 61 - ceil_log2(n_clones);
  const bool upload = !(g_tables[dev].valid && g_tables[dev].s == s && g_tables[dev].F == F);
  if (upload) {
    const double a = std::fabs(s);
    for (int k = 0; k < kKcap; ++k) {
      const double x = -a * (double)k;
      const double q = std::exp(x);
      t_host.wtab[k] = (unsigned long long)std::nearbyint(std::ldexp(q, F));
      t_host.qtab[k] = q;
      t_host.qm1tab[k] = std::expm1(x);
    }
  }
  SelState st0;
  std::memset(&st0, 0, sizeof st0);
  st0.dk_min = INT_MAX;
  st0.dk_max = INT_MIN;

  SelArgs A;
  A.dK = d_dK;
  A.anc = d_anc;
  A.wtab = (unsigned long long*)(scratch + kOffWtab);
  A.qtab = (double*)(scratch + kOffQ);
  A.qm1tab = (double*)(scratch + kOffQm1);
  A.hist = (unsigned int*)(scratch + kOffHist);
  A.tile_sum = (unsigned long long*)(scratch + kOffTileSum);
  A.st = (SelState*)(scratch + kOffState);
  A.nc = (uint32_t)n_clones;
  A.ntiles = (int32_t)((n_clones + kTile - 1) / kTile);
  A.s_neg = s < 0.0 ? 1 : 0;
  A.beta = interval;
  A.seed = seed;
  A.s = s;

  if (upload) {
    // pageable sources: each copy has read its source when it returns
    g_tables[dev].valid = false;
    if (cudaMemcpyAsync(A.wtab, t_host.wtab, sizeof t_host.wtab, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(A.qtab, t_host.qtab, sizeof t_host.qtab, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(A.qm1tab, t_host.qm1tab, sizeof t_host.qm1tab, cudaMemcpyHostToDevice,
                        stream) != cudaSuccess)
      return POP_ERR_CUDA;
    g_tables[dev] = TableKey{true, s, F};
  }
  if (cudaMemsetAsync(A.hist, 0, (size_t)kKcap * 4, stream) != cudaSuccess ||
      cudaMemcpyAsync(A.st, &st0, sizeof st0, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return POP_ERR_CUDA;
  k_sel_range<<<A.ntiles, kThreads, 0, stream>>>(A);
  k_sel_weights<<<A.ntiles, kThreads, 0, stream>>>(A);
  k_sel_ancestors<<<A.ntiles, kThreads, 0, stream>>>(A);
  if (cudaGetLastError() != cudaSuccess) return POP_ERR_CUDA;
  SelState out;
  if (cudaMemcpyAsync(&out, A.st, sizeof out, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return POP_ERR_CUDA;
  if (out.err != 0) return out.err;
  if (h_psi_term) *h_psi_term = out.psi_term;
  return POP_OK;
}
