// Device-side definitions shared by the SSEP cloning kernels (sm_103a).
//
// One interval of the cloning algorithm (arXiv:1711.05095, Sec. 2.3) is three
// kernels over a batch of populations laid out back to back in "slots" (every
// population starts on a 1024-slot tile):
//   k_evolve   dynamical stage (Sec. 4: BKL continuous-time Monte Carlo of the SSEP,
//              Sec. 3.1 rates).  A persistent grid; each block owns an equal range of
//              256-slot units, stages the clones in shared memory and advances them in
//              rounds of one BKL step per running clone, compacting the running clones
//              after each round so that every lane does useful work.  Epilogue: the
//              per-population min/max of the interval activity.
//   k_weights  fixed-point weights exp(-s dK) (64-bit), their per-tile sums and the
//              histogram of the interval activity.
//   k_gather   per tile: the exclusive prefix sums of the weights (tile sums, then a
//              block scan), [eq] selection (Sec. 4.1, eq. alpha-Ups) inverted per old
//              clone in exact integers, and a pull copy of lattices and carried
//              activities (eq. khat) staged through shared memory.  The first tile of
//              each population adds the psi term of eq. (psihat).
// All arithmetic that decides an integer result (waiting times, bond choice,
// weights, ancestors) is specified bit for bit; pop_api.cu states the contract.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace popgpu {

constexpr uint32_t kTagInit = 1u;
constexpr uint32_t kTagEvolve = 2u;
constexpr uint32_t kTagResample = 3u;
constexpr uint32_t kTagIid = 4u;

constexpr int kThreads = 256;             // threads per block of every kernel
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 1024;               // slots per tile; populations start on a tile
constexpr int kItems = kTile / kThreads;  // slots per thread in the tile kernels
constexpr int kUnit = 256;                // slots per evolve work unit (one population)
constexpr int kChunkUnits = 7;            // at most this many units staged in shared memory
constexpr int kChunk = kUnit * kChunkUnits;
constexpr int kKcap = 4096;               // fixed-point weight table size
constexpr int kHistSmem = 512;            // activity bins kept in shared memory
constexpr int kTH = 64;                   // per-tile activity histogram bins (activities 0 .. 63)
constexpr int kMap = 2048;                // new slots of one tile mapped in shared memory
#ifndef POP_SCAN_TILES
#define POP_SCAN_TILES 64
#endif
constexpr int kScanTiles = POP_SCAN_TILES; // fused stage: k_tile_scan when every population
                                           // of the launch has more tiles
constexpr int kMaxL = 128;                // one clone per lane: W <= 2 words
constexpr int kMaxLWide = 4096;           // one clone per warp: 2 words per lane
constexpr int kInvStride = kMaxLWide + 1; // per-population 1/r table stride
constexpr uint32_t kStepLimit = 1u << 24; // BKL steps per clone per interval

constexpr int32_t kErrRange = -3;

// GUIDED dynamics: hop rates 2^-40 Q(k), Q(k) = 2^40 exp(k 2^-17), |k| <= kGuideKmax.
constexpr int kGuideKmax = 1 << 20;
constexpr int kGuideTabA = 1025, kGuideTabB = 2048;
constexpr uint32_t kTagGuided = 5u;

// Constant per run.
struct PopDesc {
  int32_t L, N;
  int64_t nc;        // clones N_c
  int64_t off;       // first slot of the population (a multiple of kTile)
  uint64_t seed;     // Philox key
  int32_t first_tile, ntiles;
  int32_t s_neg;     // s < 0: the reference activity is the maximum
  int32_t modified;  // MODIFIED dynamics and weights (Sec. 3.2, eq. def-ups-ssep)
  int32_t iid;       // [iid] selection (Sec. 4.1)
  int32_t F;         // fixed-point weight scale, 61 - ceil(log2 N_c)
  float c_f;         // float(1 - e^-s), the MODIFIED weight coefficient
  int32_t guided;    // GUIDED dynamics and weights (local potential; modified is also set)
  double s;          // bias
  double abs_s;
  int32_t s_q;       // GUIDED: s in units of 2^-17 (nearest integer)
  float c_s;         // GUIDED: float(s_q 2^-17 - s)
};

// Mutable per population.
struct PopState {
  int32_t dk_min[2], dk_max[2];  // interval activity range by interval parity
                                 // (k_evolve; reset by k_gather of the same interval)
  int32_t kref;                // reference activity of this interval (k_weights)
  uint32_t U;                  // [eq] offset word of this interval (k_weights)
  double psi_acc;              // sum of psi terms (eq. psihat numerator)
  unsigned long long events;   // executed hops since init
  int32_t err;                 // sticky kernel-side error
  int32_t a_min[2], a_max[2];  // MODIFIED: range of the rate integral A by interval parity
                               // (float bits, A >= 0)
  float a_ref;                 // MODIFIED: reference A of this interval (k_weights)
  uint32_t beta;               // interval being resampled (k_weights)
  int32_t gcarry;              // GUIDED: the clones' rate sums of the last interval are
                               // carried (set by the cloning stage, cleared by the host
                               // when the potential changes)
  int32_t hovf;                // some activity of this interval is >= kTH, so the tile
                               // histograms do not hold every clone (set by the fused
                               // stage, cleared by k_tile_scan<true>)
  unsigned long long T;        // total weight of this interval (k_tile_scan or k_gather)
};

struct Batch {
  const PopDesc* pops;
  PopState* st;
  const int32_t* tile_pop;              // tile -> population
  const unsigned long long* wtab;       // [P][kKcap] fixed-point weights
  const double* qtab;                   // [P][kKcap] exp(-|s| k)
  const double* qm1tab;                 // [P][kKcap] expm1(-|s| k)
  const float* inv_rate;                // [P][kInvStride] float(1/r)
  const float2* logtab;                 // [64] (1/c_i, ln c_i) of the waiting-time log
  const float* exp2tab;                 // [64] 2^(i/64) of the MODIFIED weight exponential
  const int32_t* phi;                   // GUIDED: [P][512] potential, fixed point phi 2^16
  const unsigned long long* gtab;       // GUIDED: TA[1025] then TB[2048], the rate tables
  int32_t* gdu;                         // GUIDED: [P][2^17] dU of an active bond by its segment
  unsigned long long* gq;               // GUIDED: [P][2^17] its rate Q(clamp(dU - s_q))
  unsigned long long* gcar[2];          // GUIDED: each clone's final rate sums [slots][8 W], by
                                        // interval parity
  float* Ab[2];                         // MODIFIED: rate integral, by interval parity
  unsigned long long* S;                // [iid]: exclusive prefix sums of the weights
  unsigned int* hist;                   // [P][kKcap] activity histogram (zero between intervals)
  unsigned int* thist;                  // [kTH][ntiles] activity histogram of each tile, filled
                                        // by the fused stage when hist_on (zero between uses)
  int32_t hist_on;                      // the fused stage fills thist
  unsigned long long* tile_sum;         // [ntiles] weight sum of each tile
  unsigned long long* tile_excl;        // [ntiles] sum of the population's earlier tiles
                                        // (k_tile_scan)
  unsigned int* beta;                   // interval being evolved (1-based)
  unsigned long long* Xb[2];            // evolved lattices [slots][W], by interval parity
  unsigned long long* Y;                // population lattices between intervals [slots][W]
  int32_t* KXb[2];                      // evolved cumulative activity, by interval parity
  int32_t* KY;                          // population cumulative activity
  int32_t* dKb[2];                      // interval activity, by interval parity
  int32_t* anc;                         // ancestors of the last cloning stage
  long long* ksum;                      // [P] sum of K (estimates)
  int32_t ntiles;
  int32_t nunits;
  int64_t nslots;
  int32_t W;                            // lattice words per clone
  int32_t unit_q, unit_r;               // k_evolve: nunits = unit_q * grid + unit_r
  int32_t any_iid;                      // some population selects [iid]: k_select_iid runs last
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

// The same generator with the key schedule given: rk[r] = (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85) mod 2^32, the key of round r.  A block whose clones share one
// key (one population per tile) computes the schedule once instead of per draw.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint2* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint2 k = rk[r];
    const uint32_t lo0 = c.x * 0xD2511F53u;
    const uint32_t hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u;
    const uint32_t hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ---------------------------------------------------------------------------
// E = -ln(u), u = (2w+1)/2^33, in FP32 with a fixed sequence of operations:
// v = 2w+1 truncated to its 24 leading bits, v' = m 2^p with m in [1, 2) and p the
// position of the leading one; ln u' = (p-33) ln 2 + ln c_i + ln(1+r), where
// c_i = 1 + (i + 1/2)/64 for the top 6 fraction bits i of m, r = m/c_i - 1
// (|r| <= 1/128) and ln(1+r) ~ r (1 - r/2 + r^2/3).  tab[i] = (float(1/c_i),
// float(ln c_i)).  ln 2 is a 15-bit head (exact products with 33-p) plus a float
// tail.  Every float step is an explicitly rounded intrinsic, so no contraction
// can change the bits; the integer work stays in 32 bits (no 64-bit shifts or
// conversions): the leading one of v = 2w+1 is one above that of w, and for p >= 24
// the head of v is w >> (p - 24) (the trailing 1 of v is shifted out).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float neg_ln_u(uint32_t w, const float2* tab) {
  const int p = 32 - __clz((int)w);  // leading one of 2w+1: 0..32
  const uint32_t t = (p >= 24) ? (w >> (p - 24)) : ((2u * w + 1u) << (23 - p));
  const float m = __uint_as_float(0x3f800000u | (t & 0x007fffffu));
  const float2 cl = tab[(t >> 17) & 63u];
  const float r = __fmaf_rn(m, cl.x, -1.0f);
  float q = __fmaf_rn(r, 0x1.555556p-2f, -0.5f);
  q = __fmaf_rn(q, r, 1.0f);
  const float ln_m = __fadd_rn(cl.y, __fmul_rn(q, r));
  // float(33 - p) exactly: 1.5*2^23 + n has n in its low mantissa bits
  const float n = __fsub_rn(__int_as_float(0x4B400000 + (33 - p)), 12582912.0f);
  const float E = __fmaf_rn(n, 0x1.7f7d1cp-20f, -ln_m);
  return __fmaf_rn(n, 0x1.62e4p-1f, E);
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

// Position of the k-th (0-based) set bit of a, k < popc(a): binary descent on the
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
// differ, so both bits flip: bits b, b+1 (or b and 0 for the closing bond L-1).
template <int W>
__device__ __forceinline__ void hop(unsigned long long (&x)[W], int b, int L) {
  if constexpr (W == 1) {
    x[0] ^= (b + 1 == L) ? ((1ull << b) | 1ull) : (3ull << b);
  } else {
    unsigned long long m0, m1;
    if (b + 1 == L) {
      m0 = 1ull | (b < 64 ? (1ull << b) : 0ull);
      m1 = b >= 64 ? (1ull << (b - 64)) : 0ull;
    } else if (b < 63) {
      m0 = 3ull << b;
      m1 = 0ull;
    } else if (b == 63) {
      m0 = 1ull << 63;
      m1 = 1ull;
    } else {
      m0 = 0ull;
      m1 = 3ull << (b - 64);
    }
    x[0] ^= m0;
    x[1] ^= m1;
  }
}

// The same lattice operations on 32-bit words (u[j] holds sites [32j, 32j + 32)),
// the ALU's native width.  Shifts that may fall outside a word use the clamped
// funnel shift: __funnelshift_lc(0, v, n) = v << min(n, 32), which is 0 for n >= 32
// and, with n formed in unsigned arithmetic, for "negative" n too.
template <int W>
__device__ __forceinline__ void split32(const unsigned long long (&x)[W], uint32_t (&u)[2 * W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) {
    u[2 * w] = (uint32_t)x[w];
    u[2 * w + 1] = (uint32_t)(x[w] >> 32);
  }
}

template <int W>
__device__ __forceinline__ void join32(const uint32_t (&u)[2 * W], unsigned long long (&x)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = ((unsigned long long)u[2 * w + 1] << 32) | u[2 * w];
}

// a = x XOR rot(x) on 2W words; lm1 = L - 1 (site L-1's right neighbour is site 0).
// p[j] = popc(a[j]).  FULL: L = 32 NW, the ring fills the words, and rot is a
// rotation of the words' concatenation by one bit.
template <int NW, bool FULL = false>
__device__ __forceinline__ void active_bonds32(const uint32_t (&u)[NW], uint32_t lm1, uint32_t (&a)[NW],
                                               uint32_t (&p)[NW]) {
  const uint32_t c0 = u[0] & 1u;
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    uint32_t rot;
    if constexpr (FULL) {
      rot = __funnelshift_r(u[j], u[(j + 1) % NW], 1);
    } else {
      const uint32_t nxt = (j + 1 < NW) ? u[j + 1] : 0u;
      rot = __funnelshift_r(u[j], nxt, 1) | __funnelshift_lc(0u, c0, lm1 - 32u * (uint32_t)j);
    }
    a[j] = u[j] ^ rot;
    p[j] = (uint32_t)__popc(a[j]);
  }
}

// Position of the k-th (0-based) set bit of the 2W-word mask a (k < sum p, p[j] =
// popc(a[j])): the word by the prefix of the word counts, then halves of 16 and 8
// bits, then the byte table kth8[8 v + k] (the k-th set bit of the byte v).  For
// a = 0 and k = 0 it returns a position inside the lattice words without reading
// outside the table.
template <int NW>
__device__ __forceinline__ uint32_t kth_bond32(const uint32_t (&a)[NW], const uint32_t (&p)[NW], uint32_t k,
                                               const uint8_t* kth8) {
  uint32_t w, pos;
  if constexpr (NW == 2) {
    const bool h = k >= p[0];
    k = h ? k - p[0] : k;
    w = h ? a[1] : a[0];
    pos = h ? 32u : 0u;
  } else {
    const uint32_t p01 = p[0] + p[1];
    const bool h2 = k >= p01;
    k = h2 ? k - p01 : k;
    const uint32_t w0 = h2 ? a[2] : a[0], w1 = h2 ? a[3] : a[1], q0 = h2 ? p[2] : p[0];
    const bool h1 = k >= q0;
    k = h1 ? k - q0 : k;
    w = h1 ? w1 : w0;
    pos = (h2 ? 64u : 0u) + (h1 ? 32u : 0u);
  }
  uint32_t c = (uint32_t)__popc(w & 0xffffu);
  if (k >= c) { k -= c; w >>= 16; pos += 16u; }
  c = (uint32_t)__popc(w & 0xffu);
  if (k >= c) { k -= c; w >>= 8; pos += 8u; }
  return pos + kth8[((w & 0xffu) << 3) | (k & 7u)];
}

// A hop across bond b flips sites b and c = (b + 1) mod L (lm1 = L - 1); b >= 32 NW
// (with b != lm1) flips nothing, which is the predicated step's "no hop".
template <int NW>
__device__ __forceinline__ void hop32(uint32_t (&u)[NW], uint32_t b, uint32_t lm1) {
  const uint32_t c = (b == lm1) ? 0u : b + 1u;
#pragma unroll
  for (int j = 0; j < NW; ++j)
    u[j] ^= __funnelshift_lc(0u, 1u, b - 32u * (uint32_t)j) ^ __funnelshift_lc(0u, 1u, c - 32u * (uint32_t)j);
}

// kth8 as 512 words (4 table bytes per word, little-endian), built at compile time.
struct Kth8Table {
  uint32_t w[512];
};
constexpr Kth8Table make_kth8() {
  Kth8Table t{};
  for (int v = 0; v < 256; ++v) {
    int k = 0;
    for (int i = 0; i < 8; ++i)
      if ((v >> i) & 1) {
        const int e = 8 * v + k;
        t.w[e >> 2] |= (uint32_t)i << (8 * (e & 3));
        ++k;
      }
  }
  return t;
}
__device__ __align__(16) const Kth8Table g_kth8 = make_kth8();

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

// Block-wide sum of one 64-bit value per thread for blocks of NW warps (result
// valid in every thread).
template <int NW>
__device__ __forceinline__ unsigned long long block_sum_u64_n(unsigned long long v,
                                                              unsigned long long* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_u64(v);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  unsigned long long t = 0ull;
#pragma unroll
  for (int w = 0; w < NW; ++w) t += scratch[w];
  __syncthreads();
  return t;
}

// Block-wide sum of one 64-bit value per thread (result valid in every thread).
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_u64(v);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  unsigned long long t = 0ull;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += scratch[w];
  __syncthreads();
  return t;
}

// |a - b| as an unsigned magnitude (no overflow for any pair of ints), so that an
// out-of-range activity is rejected by the table-size check instead of indexing.
__device__ __forceinline__ unsigned int abs_diff(int a, int b) {
  const long long d = (long long)a - (long long)b;
  const unsigned long long m = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
  return m > 0xffffffffull ? 0xffffffffu : (unsigned int)m;
}

// Number of histogram bins in use, clamped to [0, cap].
__device__ __forceinline__ int hist_bins(int dk_min, int dk_max, int cap) {
  const long long n = (long long)dk_max - (long long)dk_min + 1;
  return n < 0 ? 0 : (n > cap ? cap : (int)n);
}

// 128-bit unsigned products and comparison.
struct U128 { unsigned long long hi, lo; };
__device__ __forceinline__ U128 mul128(unsigned long long a, unsigned long long b) {
  return U128{__umul64hi(a, b), a * b};
}
__device__ __forceinline__ bool lt128(const U128& a, const U128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// First new slot whose [eq] point lies at or beyond the prefix sum S:
//   j_lo(S) = min{ j : (2^33 j + c) T >= S 2^33 N_c },  c = 2U + 1,
// i.e. alpha_j = floor((2^33 j + c) T / (2^33 N_c)) >= S (eq. alpha-Ups with
// d = c / 2^33).  A float estimate of S N_c / T (from the top 24 bits of S and T)
// starts the search; exact 128-bit comparisons settle it.
__device__ __forceinline__ uint32_t j_lo(unsigned long long S, unsigned long long T,
                                         unsigned long long c, uint32_t nc, int sh,
                                         float ratio) {
  if (S == 0ull) return 0u;
  if (S >= T) return nc;
  const U128 R = mul128(S, (unsigned long long)nc << 33);
  const float est = __fmul_rn(__uint2float_rn((uint32_t)(S >> sh)), ratio);
  unsigned long long j = (unsigned long long)min((float)nc, floorf(est));
  while (j < nc && lt128(mul128((j << 33) + c, T), R)) ++j;
  while (j > 0 && !lt128(mul128(((j - 1ull) << 33) + c, T), R)) --j;
  return (uint32_t)j;
}

// j_lo of the prefix sums S0, S0 + w[0], ..., S0 + w[0] + ... + w[n-1] (n + 1
// values): the first exactly as above, the rest by walking j forward, since
// (2^33 (j+1) + c) T = (2^33 j + c) T + 2^33 T.
template <int n>
__device__ __forceinline__ void j_lo_run(unsigned long long S0, const unsigned long long (&w)[n],
                                         unsigned long long T, unsigned long long c, uint32_t nc,
                                         int sh, float ratio, uint32_t (&out)[n + 1]) {
  unsigned long long j = j_lo(S0, T, c, nc, sh, ratio);
  out[0] = (uint32_t)j;
  U128 X = mul128((j << 33) + c, T);
  const unsigned long long step_hi = T >> 31, step_lo = T << 33;  // 2^33 T
  const unsigned long long nc33 = (unsigned long long)nc << 33;
  unsigned long long S = S0;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    S += w[i];
    const U128 R = mul128(S, nc33);
    while (j < nc && lt128(X, R)) {
      ++j;
      const unsigned long long lo = X.lo + step_lo;
      X.hi += step_hi + (lo < X.lo ? 1ull : 0ull);
      X.lo = lo;
    }
    out[i + 1] = (uint32_t)j;
  }
}

// ---------------------------------------------------------------------------
// MODIFIED weights: floor(2^F exp(x)) for x <= 0 in FP32 with a fixed sequence of
// rounded operations.  x = (k/64) ln 2 + r, k = floor(64 x / ln 2), r formed in
// two fma steps with ln2/64 split into a 9-bit head (exact products for |k| < 2^15)
// and a float tail; exp(x) = 2^n 2^(i/64) e^r (k = 64 n + i), 2^(i/64) from tab2,
// e^r ~ 1 + r (1 + r (1/2 + r/6)).  The weight is the 24-bit mantissa of
// y = 2^(i/64) e^r shifted by (exponent of y) + n + F - 23.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long weight_exp(float x, int F, const float* tab2) {
  if (!(x >= -87.0f)) return 0ull;
  const int k = (int)floorf(__fmul_rn(x, 0x1.715476p+6f));
  const float kf = (float)k;
  float r = __fmaf_rn(-kf, 0x1.62p-7f, x);
  r = __fmaf_rn(-kf, 0x1.c85fe0p-16f, r);
  float q = __fmaf_rn(r, 0x1.555556p-3f, 0.5f);
  q = __fmaf_rn(q, r, 1.0f);
  q = __fmaf_rn(q, r, 1.0f);
  const int i = k & 63, n = k >> 6;
  const float y = __fmul_rn(tab2[i], q);
  const uint32_t bits = __float_as_uint(y);
  const int ey = (int)((bits >> 23) & 0xffu) - 127;
  const unsigned long long mant = (unsigned long long)((bits & 0x007fffffu) | 0x00800000u);
  const int sa = ey + n + F - 23;
  if (sa >= 0) return mant << sa;
  if (sa <= -64) return 0ull;
  return mant >> (-sa);
}

// Float bits mapped to an int of the same order (an involution), so that atomic
// integer min/max order any floats, negative ones included.
__device__ __forceinline__ int float_order(float f) {
  const int i = __float_as_int(f);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float order_float(int i) {
  return __int_as_float(i ^ ((i >> 31) & 0x7fffffff));
}

// The weight of one clone: plain (table of 2^F exp(-|s| k), k = |dK - k_ref|),
// MODIFIED (weight_exp of -c (A - A_ref)) or GUIDED (weight_exp of X - X_ref, X the
// clone's log weight held in A, X_ref the maximum).  Returns false on a plain range error.
__device__ __forceinline__ bool clone_weight(const PopDesc& d, int dk, int kref, float a,
                                            float a_ref, const unsigned long long* wt,
                                            const float* tab2, unsigned long long& w,
                                            unsigned int& k_out) {
  if (d.guided) {
    w = weight_exp(__fsub_rn(a, a_ref), d.F, tab2);
    k_out = 0u;
    return true;
  }
  if (d.modified) {
    w = weight_exp(__fmul_rn(-d.c_f, __fsub_rn(a, a_ref)), d.F, tab2);
    k_out = 0u;
    return true;
  }
  const unsigned int k = abs_diff(dk, kref);
  k_out = k;
  if (k >= (unsigned int)kKcap) { w = 0ull; return false; }
  w = __ldg(wt + k);
  return true;
}

}  // namespace popgpu
