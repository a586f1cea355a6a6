// Device code of the SSEP cloning library (sm_103a).
//
// One interval of the cloning algorithm (arXiv:1711.05095, Sec. 2.3) is three
// kernels over a batch of populations laid out back to back in "slots":
//   k_evolve   dynamical stage (Sec. 4: BKL continuous-time Monte Carlo of the SSEP,
//              Sec. 3.1 rates), one clone per thread, lattice in registers as a
//              bitmask; epilogue: per-population min/max of the interval activity.
//   k_scan     weights exp(-s dK) in 64-bit fixed point, exact single-pass prefix
//              sum per population (decoupled look-back), histogram of the activity;
//              the last tile of a population adds the psi term of eq. (psihat).
//   k_gather   [eq] selection (Sec. 4.1, eq. alpha-Ups) inverted per old clone in
//              exact integers, then a warp-cooperative coalesced pull copy of the
//              lattices and carried activities (eq. khat).
// All arithmetic that decides an integer result (waiting times, bond choice,
// weights, ancestors) is specified bit for bit; see pop_api.cu for the contract.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace popgpu {

constexpr uint32_t kTagInit = 1u;
constexpr uint32_t kTagEvolve = 2u;
constexpr uint32_t kTagResample = 3u;

constexpr int kThreads = 256;             // threads per block of every kernel
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 1024;               // slots per scan tile; populations start on a tile
constexpr int kItems = kTile / kThreads;  // slots per scan thread
constexpr int kKcap = 4096;               // fixed-point weight table size
constexpr int kHistSmem = 512;            // activity bins kept in shared memory
constexpr int kMaxL = 128;                // one-clone-per-thread lattices: W <= 2 words
constexpr int kInvStride = kMaxL + 1;     // per-population 1/r table stride

constexpr unsigned long long kStatusAgg = 1ull << 62;  // tile aggregate published
constexpr unsigned long long kStatusPre = 2ull << 62;  // tile inclusive prefix published
constexpr unsigned long long kValueMask = (1ull << 62) - 1ull;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kStepLimit = 1u << 24;  // BKL steps per clone per interval

constexpr int32_t kErrRange = -3;
constexpr int32_t kErrTimeout = -4;

// Constant per run.
struct PopDesc {
  int32_t L, N;
  int64_t nc;        // clones N_c
  int64_t off;       // first slot of the population (a multiple of kTile)
  uint64_t seed;     // Philox key
  int32_t first_tile, ntiles;
  double s;          // bias
  double abs_s;
};

// Mutable per population.
struct PopState {
  int32_t dk_min, dk_max;      // interval activity range (evolve epilogue; reset by k_scan)
  uint32_t done;               // scan tiles finished this interval
  uint32_t U;                  // [eq] offset word of this interval
  unsigned long long T;        // total fixed-point weight of this interval
  double psi_acc;              // sum of psi terms (eq. psihat numerator)
  unsigned long long events;   // executed hops since init
  int32_t err;                 // sticky kernel-side error
  int32_t pad;
};

struct Batch {
  const PopDesc* pops;
  PopState* st;
  const int32_t* tile_pop;              // tile -> population
  const unsigned long long* wtab;       // [P][kKcap] fixed-point weights
  const float* inv_rate;                // [P][kInvStride] float(1/r)
  unsigned int* hist;                   // [P][kKcap] activity histogram (kept zero between intervals)
  unsigned long long* tile_status;      // [2][ntiles] look-back words, by interval parity
  unsigned int* ticket;                 // [2] scan tile tickets, by interval parity
  unsigned int* beta;                   // interval being evolved (1-based)
  unsigned long long* X;                // evolved lattices  [slots][W]
  unsigned long long* Y;                // population lattices between intervals [slots][W]
  int32_t* KX;                          // evolved cumulative activity
  int32_t* KY;                          // population cumulative activity
  int32_t* dK;                          // activity of the last interval
  unsigned long long* S;                // exclusive prefix sums of the weights
  int32_t* anc;                         // ancestors of the last cloning stage
  long long* ksum;                      // [P] sum of K (estimates)
  int32_t ntiles;
  int64_t nslots;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the published multipliers; the key is bumped by the published
// Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = c.x * 0xD2511F53u;
    const uint32_t hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u;
    const uint32_t hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// ---------------------------------------------------------------------------
// E = -ln(u), u = (2w+1)/2^33, as a fixed sequence of IEEE-754 float operations:
// v = 2w+1 rounded once to float, v = m 2^e with m folded into (sqrt(1/2), sqrt(2)],
// ln u = (e-33) ln2 + 2 atanh(f), f = (m-1)/(m+1), and 2 atanh(f) by its odd series
// f (2 + 2/3 z + 2/5 z^2 + 2/7 z^3 + 2/9 z^4), z = f^2 (|f| <= 0.1716).  ln 2 is a
// 15-bit head (exact products for |e-33| <= 33) plus a float tail.  Every step is
// an explicitly rounded intrinsic, so no contraction can change the bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float neg_ln_u(uint32_t w) {
  const unsigned long long v = 2ull * (unsigned long long)w + 1ull;
  const float vf = __ull2float_rn(v);
  const uint32_t bits = __float_as_uint(vf);
  int e = (int)((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float z = __fmul_rn(f, f);
  float p = __fmaf_rn(0x1.c71c72p-3f, z, 0x1.24924ap-2f);
  p = __fmaf_rn(p, z, 0x1.99999ap-2f);
  p = __fmaf_rn(p, z, 0x1.555556p-1f);
  p = __fmaf_rn(p, z, 2.0f);
  const float ln_m = __fmul_rn(f, p);
  const float n = (float)(e - 33);
  float ln_u = __fmaf_rn(n, 0x1.7f7d1cp-20f, ln_m);
  ln_u = __fmaf_rn(n, 0x1.62e4p-1f, ln_u);
  return -ln_u;
}

// ---------------------------------------------------------------------------
// Lattice helpers.  A clone is W 64-bit words; site i is bit i%64 of word i/64.
// Bond i joins sites i and (i+1) mod L; it is active (a hop across it is
// possible) when exactly one end is occupied: a = x XOR rot(x), rot(x)_i = x_{i+1}.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void active_bonds(const unsigned long long (&x)[W], int L,
                                             unsigned long long (&a)[W]) {
  if constexpr (W == 1) {
    const unsigned long long rot = (x[0] >> 1) | ((x[0] & 1ull) << (L - 1));
    a[0] = x[0] ^ rot;
  } else {
    if (L <= 64) {
      const unsigned long long rot = (x[0] >> 1) | ((x[0] & 1ull) << (L - 1));
      a[0] = x[0] ^ rot;
      a[1] = 0ull;
    } else {
      const unsigned long long r0 = (x[0] >> 1) | (x[1] << 63);
      const unsigned long long r1 = (x[1] >> 1) | ((x[0] & 1ull) << (L - 65));
      a[0] = x[0] ^ r0;
      a[1] = x[1] ^ r1;
    }
  }
}

template <int W>
__device__ __forceinline__ int popc_lat(const unsigned long long (&a)[W]) {
  if constexpr (W == 1) return __popcll(a[0]);
  else return __popcll(a[0]) + __popcll(a[1]);
}

// Position of the k-th (0-based) set bit of a, k < popc(a): binary descent on
// population counts of halves.
__device__ __forceinline__ int kth_set_bit64(unsigned long long a, uint32_t k) {
  uint32_t x = (uint32_t)a;
  int pos = 0;
  uint32_t c = (uint32_t)__popc(x);
  if (k >= c) { k -= c; x = (uint32_t)(a >> 32); pos = 32; }
  c = (uint32_t)__popc(x & 0xffffu);
  if (k >= c) { k -= c; x >>= 16; pos += 16; }
  c = (uint32_t)__popc(x & 0xffu);
  if (k >= c) { k -= c; x >>= 8; pos += 8; }
  c = (uint32_t)__popc(x & 0xfu);
  if (k >= c) { k -= c; x >>= 4; pos += 4; }
  c = (uint32_t)__popc(x & 0x3u);
  if (k >= c) { k -= c; x >>= 2; pos += 2; }
  c = x & 1u;
  if (k >= c) { pos += 1; }
  return pos;
}

template <int W>
__device__ __forceinline__ int kth_bond(const unsigned long long (&a)[W], uint32_t k) {
  if constexpr (W == 1) {
    return kth_set_bit64(a[0], k);
  } else {
    const uint32_t c0 = (uint32_t)__popcll(a[0]);
    const bool lo = k < c0;
    return kth_set_bit64(lo ? a[0] : a[1], lo ? k : k - c0) + (lo ? 0 : 64);
  }
}

// A hop across bond b swaps the occupations of sites b and (b+1) mod L, which
// differ, so both bits flip.
template <int W>
__device__ __forceinline__ void hop(unsigned long long (&x)[W], int b, int L) {
  const int b1 = (b + 1 == L) ? 0 : b + 1;
  if constexpr (W == 1) {
    x[0] ^= (1ull << b) | (1ull << b1);
  } else {
    unsigned long long m0 = 0ull, m1 = 0ull;
    if (b < 64) m0 |= 1ull << b; else m1 |= 1ull << (b - 64);
    if (b1 < 64) m0 |= 1ull << b1; else m1 |= 1ull << (b1 - 64);
    x[0] ^= m0;
    x[1] ^= m1;
  }
}

template <int W>
__device__ __forceinline__ void load_lat(const unsigned long long* base, int64_t slot,
                                         unsigned long long (&x)[W]) {
  if constexpr (W == 1) {
    x[0] = base[slot];
  } else {
    const ulonglong2 v = reinterpret_cast<const ulonglong2*>(base)[slot];
    x[0] = v.x;
    x[1] = v.y;
  }
}

template <int W>
__device__ __forceinline__ void store_lat(unsigned long long* base, int64_t slot,
                                          const unsigned long long (&x)[W]) {
  if constexpr (W == 1) {
    base[slot] = x[0];
  } else {
    reinterpret_cast<ulonglong2*>(base)[slot] = make_ulonglong2(x[0], x[1]);
  }
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Initial state: a uniform N-subset of the L sites by selection sampling; site t is
// taken iff floor(U64 (L-t) / 2^64) < N - taken, U64 from draw (t, 0, j, init).
// Padded slots get an empty lattice.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_init(Batch B) {
  const int64_t slot = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int p = B.tile_pop[(blockIdx.x * kThreads) / kTile];
  const PopDesc d = B.pops[p];
  const int64_t j = slot - d.off;
  unsigned long long x[W];
#pragma unroll
  for (int q = 0; q < W; ++q) x[q] = 0ull;
  if (j < d.nc) {
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    int taken = 0;
    for (int t = 0; t < d.L; ++t) {
      const int need = d.N - taken;
      if (need <= 0) break;
      const uint4 r = philox4x32_10(make_uint4((uint32_t)t, 0u, (uint32_t)j, kTagInit), k0, k1);
      const unsigned long long u = ((unsigned long long)r.y << 32) | r.x;
      if (__umul64hi(u, (unsigned long long)(d.L - t)) < (unsigned long long)need) {
        if (W == 1 || t < 64) x[0] |= 1ull << (t & 63);
        else x[W - 1] |= 1ull << (t & 63);
        ++taken;
      }
    }
  }
  store_lat<W>(B.Y, slot, x);
  B.KY[slot] = 0;
  B.dK[slot] = 0;
}

// ---------------------------------------------------------------------------
// Dynamical stage (Sec. 4 BKL; Sec. 3.1 rates 1 per possible hop).
// Per step e of the interval: r = active bonds (escape rate); if r = 0 stop.
// Draw q = e/2 of (q, beta, j, evolve) gives (wa, wb) = words (0,1) or (2,3).
// tau = E(wa) * float(1/r); t_new = t + tau; stop if t_new >= dt (the residual
// waiting time is dropped, which the exponential law's memorylessness allows);
// else hop across the floor(wb r / 2^32)-th active bond.
// All lanes of a warp that are still running are at the same step e, so the
// draw on even steps is taken uniformly by the warp.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_evolve(Batch B, float dt_f) {
  __shared__ float s_inv[kInvStride];
  __shared__ int s_min[kWarps], s_max[kWarps];
  __shared__ unsigned int s_ev[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t slot = (int64_t)blockIdx.x * kThreads + tid;
  const int p = B.tile_pop[(blockIdx.x * kThreads) / kTile];
  const PopDesc d = B.pops[p];
  for (int r = tid; r <= d.L; r += kThreads) s_inv[r] = B.inv_rate[p * kInvStride + r];
  __syncthreads();
  const int64_t j = slot - d.off;
  const bool valid = j < d.nc;
  const uint32_t beta = *B.beta;
  int hops = 0;
  if (valid) {
    unsigned long long x[W];
    load_lat<W>(B.Y, slot, x);
    const int L = d.L;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    float t = 0.0f;
    uint32_t e = 0u, wc = 0u, wd = 0u;
    for (;;) {
      if (e >= kStepLimit) {  // guard: the interval must end; report instead of spinning
        B.st[p].err = kErrRange;
        break;
      }
      unsigned long long a[W];
      active_bonds<W>(x, L, a);
      const int r = popc_lat<W>(a);
      if (r == 0) break;
      uint32_t wa, wb;
      if ((e & 1u) == 0u) {
        const uint4 q = philox4x32_10(make_uint4(e >> 1, beta, (uint32_t)j, kTagEvolve), k0, k1);
        wa = q.x; wb = q.y; wc = q.z; wd = q.w;
      } else {
        wa = wc; wb = wd;
      }
      ++e;
      const float E = neg_ln_u(wa);
      const float t_new = __fadd_rn(t, __fmul_rn(E, s_inv[r]));
      if (t_new >= dt_f) break;
      t = t_new;
      const uint32_t k = __umulhi(wb, (uint32_t)r);
      hop<W>(x, kth_bond<W>(a, k), L);
      ++hops;
    }
    store_lat<W>(B.X, slot, x);
    B.KX[slot] = B.KY[slot] + hops;
    B.dK[slot] = hops;
  }
  const int mn = __reduce_min_sync(0xffffffffu, valid ? hops : INT_MAX);
  const int mx = __reduce_max_sync(0xffffffffu, valid ? hops : INT_MIN);
  const unsigned int ev = __reduce_add_sync(0xffffffffu, (unsigned int)hops);
  if (lane == 0) { s_min[wid] = mn; s_max[wid] = mx; s_ev[wid] = ev; }
  __syncthreads();
  if (tid == 0) {
    int bmn = s_min[0], bmx = s_max[0];
    unsigned long long bev = s_ev[0];
    for (int w = 1; w < kWarps; ++w) {
      bmn = min(bmn, s_min[w]);
      bmx = max(bmx, s_max[w]);
      bev += s_ev[w];
    }
    if (bmn != INT_MAX) {
      atomicMin(&B.st[p].dk_min, bmn);
      atomicMax(&B.st[p].dk_max, bmx);
      atomicAdd(&B.st[p].events, bev);
    }
  }
}

// ---------------------------------------------------------------------------
// Weights and exact prefix sums.  F = 61 - ceil(log2 N_c), so the total T <= 2^61
// and a look-back word holds a 62-bit value plus a 2-bit status.  One tile of
// kTile slots per block; tiles are taken in ticket order, so every predecessor a
// tile waits on is already running.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_scan(Batch B) {
  __shared__ unsigned int s_hist[kHistSmem];
  __shared__ unsigned long long s_warp[kWarps];
  __shared__ unsigned long long s_agg, s_excl;
  __shared__ int s_tile, s_last;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t beta = *B.beta;
  const int par = (int)(beta & 1u);
  if (tid == 0) s_tile = (int)atomicAdd(&B.ticket[par], 1u);
  for (int i = tid; i < kHistSmem; i += kThreads) s_hist[i] = 0u;
  __syncthreads();
  const int tile = s_tile;
  const int p = B.tile_pop[tile];
  const PopDesc d = B.pops[p];
  PopState* st = B.st + p;
  const int64_t base = (int64_t)tile * kTile;
  const int64_t j0 = base - d.off + (int64_t)tid * kItems;
  const int dk_min = st->dk_min, dk_max = st->dk_max;
  const int kref = (d.s >= 0.0) ? dk_min : dk_max;
  const int4 dk4 = reinterpret_cast<const int4*>(B.dK + base)[tid];
  const int dkv[kItems] = {dk4.x, dk4.y, dk4.z, dk4.w};
  unsigned long long w[kItems];
  unsigned long long tsum = 0ull;
  bool range_err = false;
  const unsigned long long* wt = B.wtab + (size_t)p * kKcap;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    w[i] = 0ull;
    if (j0 + i < d.nc) {
      const int k = abs(dkv[i] - kref);
      if (k >= kKcap) {
        range_err = true;
      } else {
        w[i] = __ldg(wt + k);
        if (k < kHistSmem) atomicAdd(&s_hist[k], 1u);
        else atomicAdd(&B.hist[(size_t)p * kKcap + k], 1u);
      }
    }
    tsum += w[i];
  }
  if (range_err) st->err = kErrRange;

  // block-wide exclusive scan of the per-thread sums
  unsigned long long x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const unsigned long long v = (lane < kWarps) ? s_warp[lane] : 0ull;
    unsigned long long vi = v;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < kWarps) s_warp[lane] = vi - v;
    if (lane == kWarps - 1) s_agg = vi;
  }
  __syncthreads();
  const unsigned long long thread_excl = x - tsum + s_warp[wid];
  const unsigned long long agg = s_agg;

  // decoupled look-back across the tiles of this population
  unsigned long long* status = B.tile_status + (size_t)par * B.ntiles;
  if (wid == 0) {
    unsigned long long excl = 0ull;
    if (tile == d.first_tile) {
      if (lane == 0) st_release(&status[tile], kStatusPre | agg);
    } else {
      if (lane == 0) st_release(&status[tile], kStatusAgg | agg);
      int look = tile - 1;
      bool timed_out = false;
      for (;;) {
        const int t = look - lane;
        const bool in = t >= d.first_tile;
        unsigned long long v = 0ull;
        if (in) {
          uint32_t spins = 0;
          do {
            v = ld_acquire(&status[t]);
          } while ((v >> 62) == 0ull && ++spins < kSpinLimit);
          if ((v >> 62) == 0ull) timed_out = true;
        }
        const unsigned int pre = __ballot_sync(0xffffffffu, in && (v >> 62) == 2ull);
        if (pre != 0u) {
          const int first = __ffs(pre) - 1;
          excl += warp_sum_u64((in && lane <= first) ? (v & kValueMask) : 0ull);
          break;
        }
        excl += warp_sum_u64(in ? (v & kValueMask) : 0ull);
        look -= 32;
        if (look < d.first_tile || __any_sync(0xffffffffu, timed_out)) break;
      }
      if (__any_sync(0xffffffffu, timed_out) && lane == 0) st->err = kErrTimeout;
      if (lane == 0) st_release(&status[tile], kStatusPre | (excl + agg));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();

  // exclusive prefix sums of this thread's slots
  unsigned long long run = s_excl + thread_excl;
  unsigned long long sv[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) { sv[i] = run; run += w[i]; }
  ulonglong2* sdst = reinterpret_cast<ulonglong2*>(B.S + base + (int64_t)tid * kItems);
  sdst[0] = make_ulonglong2(sv[0], sv[1]);
  sdst[1] = make_ulonglong2(sv[2], sv[3]);

  // histogram to global memory
  const int nb = min(dk_max - dk_min + 1, kHistSmem);
  for (int b = tid; b < nb; b += kThreads) {
    const unsigned int c = s_hist[b];
    if (c) atomicAdd(&B.hist[(size_t)p * kKcap + b], c);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int prev = atomicAdd(&st->done, 1u);
    s_last = (prev == (unsigned int)(d.ntiles - 1));
    // this tile's look-back word for the next interval of the same parity
    B.tile_status[(size_t)(par ^ 1) * B.ntiles + tile] = 0ull;
  }
  __syncthreads();
  if (!s_last || wid != 0) return;

  // Last tile of the population: psi term of eq. (psihat) from the histogram,
  //   term = -s k_ref + ln( (1/N_c) sum_k n_k exp(-|s| k) ),
  // taken as log1p of the expm1 sum when the mean is above 1/2.
  __threadfence();
  const unsigned long long T =
      ld_acquire(&status[d.first_tile + d.ntiles - 1]) & kValueMask;
  const int R = min(dk_max - dk_min + 1, kKcap);
  double a = 0.0, q = 0.0;
  unsigned int* h = B.hist + (size_t)p * kKcap;
  for (int b = lane; b < R; b += 32) {
    const unsigned int c = __ldcg(h + b);
    if (c) {
      const double xk = -d.abs_s * (double)b;
      a += (double)c * expm1(xk);
      q += (double)c * exp(xk);
      h[b] = 0u;
    }
  }
  a = warp_sum_f64(a);
  q = warp_sum_f64(q);
  if (lane == 0) {
    const double ncd = (double)d.nc;
    const double mean_q = q / ncd;
    const double ln_mean = (mean_q > 0.5) ? log1p(a / ncd) : log(mean_q);
    st->psi_acc += -d.s * (double)kref + ln_mean;
    st->T = T;
    st->U = philox4x32_10(make_uint4(0u, beta, 0u, kTagResample),
                          (uint32_t)d.seed, (uint32_t)(d.seed >> 32)).x;
    st->done = 0u;
    st->dk_min = INT_MAX;
    st->dk_max = INT_MIN;
  }
}

// 128-bit unsigned products and comparison.
struct U128 { unsigned long long hi, lo; };
__device__ __forceinline__ U128 mul128(unsigned long long a, unsigned long long b) {
  return U128{__umul64hi(a, b), a * b};
}
__device__ __forceinline__ bool lt128(const U128& a, const U128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// First new slot whose [eq] point falls at or beyond the prefix sum S:
//   j_lo(S) = min{ j : (2^33 j + c) T >= S 2^33 N_c },  c = 2U + 1,
// i.e. alpha_j = floor((2^33 j + c) T / (2^33 N_c)) >= S (eq. alpha-Ups with
// d = c/2^33).  A float estimate is corrected with exact 128-bit comparisons.
__device__ __forceinline__ uint32_t j_lo(unsigned long long S, unsigned long long T,
                                         unsigned long long c, uint32_t nc, float nc_over_T) {
  if (S == 0ull) return 0u;
  if (S >= T) return nc;
  const U128 R = mul128(S, (unsigned long long)nc << 33);
  const float est = __fmaf_rn(__ull2float_rn(S), nc_over_T, -__ull2float_rn(c) * 0x1p-33f);
  long long j = (long long)ceilf(est);
  j = j < 0 ? 0 : (j > (long long)nc ? (long long)nc : j);
  while (j < (long long)nc && lt128(mul128(((unsigned long long)j << 33) + c, T), R)) ++j;
  while (j > 0 && !lt128(mul128(((unsigned long long)(j - 1) << 33) + c, T), R)) --j;
  return (uint32_t)j;
}

// ---------------------------------------------------------------------------
// Cloning stage: old clone k owns new slots [j_lo(S_k), j_lo(S_{k+1})).  Each warp
// owns 32 consecutive old clones, hence one contiguous run of new slots; lanes
// walk that run 32 at a time (coalesced stores), find their source lane by a
// binary search over the warp's j_lo values and take the clone by shuffles.
// The last block also advances the interval counter.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_gather(Batch B) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t slot = (int64_t)blockIdx.x * kThreads + tid;
  const int p = B.tile_pop[(blockIdx.x * kThreads) / kTile];
  const PopDesc d = B.pops[p];
  const PopState* st = B.st + p;
  const unsigned long long T = st->T;
  const unsigned long long c = 2ull * (unsigned long long)st->U + 1ull;
  const uint32_t nc = (uint32_t)d.nc;
  const float nc_over_T = __fdiv_rn((float)nc, __ull2float_rn(T));
  const int64_t k = slot - d.off;
  const bool valid = k < d.nc;
  uint32_t jlo = nc;
  unsigned long long x[W];
  int32_t Kv = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) x[q] = 0ull;
  if (valid) {
    jlo = j_lo(B.S[slot], T, c, nc, nc_over_T);
    load_lat<W>(B.X, slot, x);
    Kv = B.KX[slot];
  }
  uint32_t jhi = __shfl_down_sync(0xffffffffu, jlo, 1);
  if (lane == 31) jhi = (k + 1 < d.nc) ? j_lo(B.S[slot + 1], T, c, nc, nc_over_T) : nc;
  const uint32_t J0 = __shfl_sync(0xffffffffu, jlo, 0);
  const uint32_t J1 = __shfl_sync(0xffffffffu, jhi, 31);
  const int64_t k_first = slot - lane - d.off;
  for (uint32_t base = J0; base < J1; base += 32u) {
    const uint32_t jj = base + (uint32_t)lane;
    int src = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const uint32_t v = __shfl_sync(0xffffffffu, jlo, src + step);
      if (v <= jj) src += step;
    }
    unsigned long long xs[W];
#pragma unroll
    for (int q = 0; q < W; ++q) xs[q] = __shfl_sync(0xffffffffu, x[q], src);
    const int32_t Ks = __shfl_sync(0xffffffffu, Kv, src);
    if (jj < J1) {
      const int64_t dst = d.off + (int64_t)jj;
      store_lat<W>(B.Y, dst, xs);
      B.KY[dst] = Ks;
      B.anc[dst] = (int32_t)(k_first + src);
    }
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) {
    const unsigned int b = *B.beta;
    B.ticket[(b + 1u) & 1u] = 0u;
    *B.beta = b + 1u;
  }
}

// Sum of the carried activities of each population (for k_hat, eq. khat).
__global__ void __launch_bounds__(kThreads) k_ksum(Batch B) {
  __shared__ long long s_part[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t slot = (int64_t)blockIdx.x * kThreads + tid;
  const int p = B.tile_pop[(blockIdx.x * kThreads) / kTile];
  const PopDesc d = B.pops[p];
  long long v = (slot - d.off < d.nc) ? (long long)B.KY[slot] : 0ll;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_part[wid] = v;
  __syncthreads();
  if (tid == 0) {
    long long t = 0;
    for (int w = 0; w < kWarps; ++w) t += s_part[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(&B.ksum[p]), (unsigned long long)t);
  }
}

}  // namespace popgpu
