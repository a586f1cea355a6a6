// Kernels of the SSEP cloning library (sm_103a); see pop_common.cuh for the
// interval structure, the data layout and the arithmetic they share.
#pragma once

#include "pop_common.cuh"

namespace popgpu {

// ---------------------------------------------------------------------------
// Initial state: a uniform N-subset of the L sites by selection sampling; site t is
// taken iff floor(U64 (L-t) / 2^64) < N - taken, U64 from draw (t, 0, j, init).
// Padded slots get an empty lattice.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_init(Batch B) {
  const int64_t slot = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int p = B.tile_pop[slot / kTile];
  const PopDesc d = B.pops[p];
  const int64_t j = slot - d.off;
  if constexpr (W == 0) {
    // wide lattices: words are written as soon as their 64 sites are decided
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    const bool valid = j < d.nc;
    int taken = 0;
    unsigned long long word = 0ull;
    for (int t = 0; t < 64 * B.W; ++t) {
      if (valid && t < d.L && d.N - taken > 0) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)t, 0u, (uint32_t)j, kTagInit), k0, k1);
        const unsigned long long u = ((unsigned long long)r.y << 32) | r.x;
        if (__umul64hi(u, (unsigned long long)(d.L - t)) < (unsigned long long)(d.N - taken)) {
          word |= 1ull << (t & 63);
          ++taken;
        }
      }
      if ((t & 63) == 63) {
        B.Y[slot * B.W + (t >> 6)] = word;
        word = 0ull;
      }
    }
  } else {
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
  }
  B.KY[slot] = 0;
  B.dKb[0][slot] = 0;
  B.dKb[1][slot] = 0;
}

// Shared-memory state of k_evolve: one chunk of up to kChunk clones.
template <int W>
struct EvolveSmem {
  unsigned long long x[kChunk][W];  // lattices (in, then out)
  int32_t hops[kChunk];             // activity of the interval
  float a[kChunk];                  // MODIFIED: integral of the escape rate over the interval
  float inv[kChunkUnits][kMaxL + 1];
  float2 logtab[64];
  __align__(16) uint32_t kth8[512];  // the byte table of kth_bond32
  uint2 u_key[kChunkUnits];         // Philox key of the unit's population
  int32_t u_j0[kChunkUnits];        // population-local index of the unit's first slot
  int32_t u_pop[kChunkUnits], u_L[kChunkUnits], u_valid[kChunkUnits];
  int32_t u_min[kChunkUnits], u_max[kChunkUnits];
  int32_t u_amin[kChunkUnits], u_amax[kChunkUnits];
  unsigned int u_ev[kChunkUnits];
  int take;                         // next unclaimed clone of the chunk
};

// One BKL step (Sec. 4 BKL; Sec. 3.1 rates 1 per possible hop) with the step's
// exponential variate E = -ln u(wa) and bond word wb, on the lattice as 2W 32-bit
// words u (lm1 = L - 1): r = active bonds (escape rate; r = 0 ends the interval);
// tau = E * float(1/r); t_new = t + tau; t_new >= dt ends the interval (the residual
// waiting time is dropped, as the exponential law's memorylessness allows);
// otherwise hop across the floor(wb r / 2^32)-th active bond (kth8: the byte table of
// kth_bond32).  Returns true if the clone hopped (and is still running).
// MODIFIED dynamics (Sec. 3.2): inv holds float(e^s / r) and the integral of the
// unmodified escape rate is accumulated, A <- fma(r, tau, A) per hop and
// A <- fma(r, dt - t, A) for the last segment.
template <int W, bool MOD>
__device__ __forceinline__ bool bkl_step(uint32_t (&u)[2 * W], float& t, float& acc, uint32_t lm1,
                                         const float* inv, float E, uint32_t wb, float dt_f,
                                         const uint8_t* kth8) {
  constexpr int NW = 2 * W;
  uint32_t a[NW], pc[NW];
  active_bonds32<NW>(u, lm1, a, pc);
  uint32_t r = 0u;
#pragma unroll
  for (int j = 0; j < NW; ++j) r += pc[j];
  if (r == 0u) return false;
  const float tau = __fmul_rn(E, inv[r]);
  const float t_new = __fadd_rn(t, tau);
  if (t_new >= dt_f) {
    if (MOD) acc = __fmaf_rn((float)r, __fsub_rn(dt_f, t), acc);
    return false;
  }
  if (MOD) acc = __fmaf_rn((float)r, tau, acc);
  t = t_new;
  hop32<NW>(u, kth_bond32<NW>(a, pc, __umulhi(wb, r), kth8), lm1);
  return true;
}

// The same step without branches, for a clone that is `live` (else nothing changes):
// the rate, waiting time and bond are computed in any case and applied under the
// step's predicate, so the lanes of a warp stay together.  r = 0 or t_new >= dt ends
// the interval as in bkl_step (MOD: the last segment r (dt - t) is added when r > 0;
// for r = 0 it adds nothing).  A step that does not hop passes bond 1024, which
// hop32 turns into no change.  FULL: L = 64 W (see active_bonds32).
template <int W, bool MOD, bool FULL = false>
__device__ __forceinline__ bool bkl_step_pred(uint32_t (&u)[2 * W], float& t, float& acc, uint32_t lm1,
                                              const float* inv, float E, uint32_t wb, float dt_f,
                                              bool live, const uint8_t* kth8) {
  constexpr int NW = 2 * W;
  uint32_t a[NW], pc[NW];
  active_bonds32<NW, FULL>(u, lm1, a, pc);
  uint32_t r = 0u;
#pragma unroll
  for (int j = 0; j < NW; ++j) r += pc[j];
  const float tau = __fmul_rn(E, inv[r]);
  const float t_new = __fadd_rn(t, tau);
  const bool moving = live && r != 0u;
  const bool hopped = moving && t_new < dt_f;
  if (MOD) {
    const float seg = hopped ? tau : __fsub_rn(dt_f, t);
    acc = moving ? __fmaf_rn((float)r, seg, acc) : acc;
  }
  t = hopped ? t_new : t;
  const uint32_t b = kth_bond32<NW>(a, pc, __umulhi(wb, r), kth8);
  hop32<NW>(u, hopped ? b : 1024u, lm1);
  return hopped;
}

// ---------------------------------------------------------------------------
// Dynamical stage.  A persistent grid; each block stages an equal share of the
// clones in shared memory.  Every lane holds one clone in registers and advances
// it two BKL steps per iteration from one Philox draw (draw q of the clone serves
// its steps 2q and 2q+1); a lane whose clone has ended takes the next clone of
// the block from a shared-memory counter, so lanes stay busy until the block's
// clones run out and no block-wide barrier is needed during the interval.
// ---------------------------------------------------------------------------
#ifndef POP_EVOLVE_MIN_BLOCKS
#define POP_EVOLVE_MIN_BLOCKS 4  // two-word staging (~48 KB) allows 4 blocks per SM anyway:
                                 // 64 registers and no spills (5: 48 registers, 2.5 % slower)
#endif
template <int W, bool MOD>
__global__ void __launch_bounds__(kThreads, POP_EVOLVE_MIN_BLOCKS) k_evolve(Batch B, float dt_f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EvolveSmem<W>& S = *reinterpret_cast<EvolveSmem<W>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t beta = *B.beta;
  const int par = (int)(beta & 1u);
  unsigned long long* const Xo = B.Xb[par];
  int32_t* const KXo = B.KXb[par];
  int32_t* const dKo = B.dKb[par];
  float* const Ao = B.Ab[par];
  if (tid < 64) S.logtab[tid] = B.logtab[tid];
  if (tid < 128) reinterpret_cast<uint4*>(S.kth8)[tid] = reinterpret_cast<const uint4*>(g_kth8.w)[tid];
  const uint8_t* const kth8 = reinterpret_cast<const uint8_t*>(S.kth8);
  // this block's units: an even split of B.nunits over the grid, B.unit_q units each
  // and one more for the first B.unit_r blocks (no divisions on the device)
  const int bx = (int)blockIdx.x;
  const int u_begin = bx * B.unit_q + min(bx, B.unit_r);
  const int len = B.unit_q + (bx < B.unit_r ? 1 : 0);
  const int nchunks = (len + kChunkUnits - 1) / kChunkUnits;
  const int cq = len / nchunks, cr = len - cq * nchunks;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int uc = u_begin + ch * cq + min(ch, cr);
    const int nu = cq + (ch < cr ? 1 : 0);
    const int64_t chunk_slot0 = (int64_t)uc * kUnit;
    if (tid < nu) {
      const int64_t slot0 = chunk_slot0 + (int64_t)tid * kUnit;
      const int p = B.tile_pop[slot0 / kTile];
      const PopDesc d = B.pops[p];
      const int64_t j0 = slot0 - d.off;
      S.u_pop[tid] = p;
      S.u_L[tid] = d.L;
      S.u_j0[tid] = (int32_t)j0;
      S.u_key[tid] = make_uint2((uint32_t)d.seed, (uint32_t)(d.seed >> 32));
      S.u_valid[tid] = (int)max((int64_t)0, min((int64_t)kUnit, d.nc - j0));
      S.u_min[tid] = INT_MAX;
      S.u_max[tid] = INT_MIN;
      S.u_amin[tid] = INT_MAX;
      S.u_amax[tid] = INT_MIN;
      S.u_ev[tid] = 0u;
    }
    if (tid == 0) S.take = 0;
    // this thread's cumulative activities, needed at write-back
    int32_t ky[kChunkUnits];
#pragma unroll
    for (int m = 0; m < kChunkUnits; ++m)
      if (m < nu) ky[m] = B.KY[chunk_slot0 + m * kUnit + tid];
    __syncthreads();
    for (int uu = 0; uu < nu; ++uu) {
      const float* src = B.inv_rate + (size_t)S.u_pop[uu] * kInvStride;
      for (int r = tid; r <= kMaxL; r += kThreads) S.inv[uu][r] = (r <= S.u_L[uu]) ? src[r] : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < kChunkUnits; ++m) {
      if (m < nu) {
        const int i = m * kUnit + tid;
        if (tid < S.u_valid[m]) {
          unsigned long long x[W];
          load_lat<W>(B.Y, chunk_slot0 + i, x);
#pragma unroll
          for (int q = 0; q < W; ++q) S.x[i][q] = x[q];
        }
        S.hops[i] = 0;
      }
    }
    __syncthreads();

    const int n = nu * kUnit;
    int c = -1;  // the lane's clone (chunk index), -1 when it has none
    unsigned long long x[W];
    float t = 0.0f, acc = 0.0f;
    int h = 0, L = 3;
    uint32_t q = 0u, j = 0u;
    uint2 key = make_uint2(0u, 0u);
    const float* inv = S.inv[0];
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = 0ull;
    for (;;) {
      // one read of the counter per warp keeps every branch below warp-uniform
      int taken = 0;
      if (lane == 0) taken = *(volatile int*)&S.take;
      taken = __shfl_sync(0xffffffffu, taken, 0);
      const bool need = c < 0;
      const unsigned int m = __ballot_sync(0xffffffffu, need);
      if (m != 0u && taken < n) {
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&S.take, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) {
          const int idx = base + __popc(m & ((1u << lane) - 1u));
          if (idx < n) {
            const int uu = idx / kUnit;
            if ((idx % kUnit) < S.u_valid[uu]) {
              c = idx;
#pragma unroll
              for (int w = 0; w < W; ++w) x[w] = S.x[c][w];
              t = 0.0f;
              acc = 0.0f;
              h = 0;
              q = 0u;
              L = S.u_L[uu];
              key = S.u_key[uu];
              j = (uint32_t)(S.u_j0[uu] + (idx % kUnit));
              inv = S.inv[uu];
            }
          }
        }
      }
      if (__ballot_sync(0xffffffffu, c >= 0) == 0u) {
        if (lane == 0) taken = *(volatile int*)&S.take;
        if (__shfl_sync(0xffffffffu, taken, 0) >= n) break;
      }
      if (c >= 0) {
        const uint4 d4 = philox4x32_10(make_uint4(q, beta, j, kTagEvolve), key.x, key.y);
        // both waiting-time variates up front: independent of the lattice, so the two
        // logarithms overlap
        const float E1 = neg_ln_u(d4.x, S.logtab), E2 = neg_ln_u(d4.z, S.logtab);
        bool run = false;
        uint32_t u[2 * W];
        split32<W>(x, u);
        if (bkl_step<W, MOD>(u, t, acc, (uint32_t)L - 1u, inv, E1, d4.y, dt_f, kth8)) {
          ++h;
          if (bkl_step<W, MOD>(u, t, acc, (uint32_t)L - 1u, inv, E2, d4.w, dt_f, kth8)) {
            ++h;
            run = true;
          }
        }
        join32<W>(u, x);
        ++q;
        if (run && q >= kStepLimit / 2u) {  // guard: an interval must end; report, never spin
          B.st[S.u_pop[c / kUnit]].err = kErrRange;
          run = false;
        }
        if (!run) {
#pragma unroll
          for (int w = 0; w < W; ++w) S.x[c][w] = x[w];
          S.hops[c] = h;
          if (MOD) S.a[c] = acc;
          c = -1;
        }
      }
    }
    __syncthreads();

    // write back (coalesced) and reduce the activity per unit
#pragma unroll
    for (int m = 0; m < kChunkUnits; ++m) {
      if (m < nu) {
        const int i = m * kUnit + tid;
        const bool valid = tid < S.u_valid[m];
        const int64_t slot = chunk_slot0 + i;
        const int hh = S.hops[i];
        if (valid) {
          unsigned long long xo[W];
#pragma unroll
          for (int w = 0; w < W; ++w) xo[w] = S.x[i][w];
          store_lat<W>(Xo, slot, xo);
          KXo[slot] = ky[m] + hh;
          dKo[slot] = hh;
          if (MOD) Ao[slot] = S.a[i];
        }
        if (MOD) {
          // A >= 0, so its float bits order like the values
          const int ab = valid ? __float_as_int(S.a[i]) : 0;
          const int amn = __reduce_min_sync(0xffffffffu, valid ? ab : INT_MAX);
          const int amx = __reduce_max_sync(0xffffffffu, valid ? ab : INT_MIN);
          if (lane == 0) {
            atomicMin(&S.u_amin[m], amn);
            atomicMax(&S.u_amax[m], amx);
          }
        }
        const int mn = __reduce_min_sync(0xffffffffu, valid ? hh : INT_MAX);
        const int mx = __reduce_max_sync(0xffffffffu, valid ? hh : INT_MIN);
        const unsigned int ev = __reduce_add_sync(0xffffffffu, valid ? (unsigned int)hh : 0u);
        if (lane == 0) {
          atomicMin(&S.u_min[m], mn);
          atomicMax(&S.u_max[m], mx);
          atomicAdd(&S.u_ev[m], ev);
        }
      }
    }
    __syncthreads();
    if (tid < nu && S.u_min[tid] != INT_MAX) {
      PopState* st = B.st + S.u_pop[tid];
      atomicMin(&st->dk_min[par], S.u_min[tid]);
      atomicMax(&st->dk_max[par], S.u_max[tid]);
      atomicAdd(&st->events, (unsigned long long)S.u_ev[tid]);
      if (MOD) {
        atomicMin(&st->a_min[par], S.u_amin[tid]);
        atomicMax(&st->a_max[par], S.u_amax[tid]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Weights: F = 61 - ceil(log2 N_c); w = wtab[|dK - k_ref|] with k_ref the min (s >= 0)
// or max (s < 0) activity, so every weight is at most 2^F and the total at most 2^61.
// Per tile: the weight sum and the histogram of |dK - k_ref|.  The first tile of a
// population also records k_ref and the [eq] offset word U of the interval.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_weights(Batch B, int tile0) {
  __shared__ unsigned int s_hist[kHistSmem];
  __shared__ unsigned long long s_red[kWarps];
  const int tid = threadIdx.x;
  const int tile = tile0 + (int)blockIdx.x;
  const int p = B.tile_pop[tile];
  const PopDesc d = B.pops[p];
  PopState* st = B.st + p;
  const int64_t base = (int64_t)tile * kTile;
  const int64_t j0 = base - d.off + (int64_t)tid * kItems;
  const uint32_t beta = *B.beta;  // the interval being resampled (no kernel advances it meanwhile)
  const int par = (int)(beta & 1u);
  const int4 dk4 = reinterpret_cast<const int4*>(B.dKb[par] + base)[tid];
  float av[kItems] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (d.modified) {
    const float4 a4 = reinterpret_cast<const float4*>(B.Ab[par] + base)[tid];
    av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
  }
  for (int i = tid; i < kHistSmem; i += kThreads) s_hist[i] = 0u;
  const int dk_min = st->dk_min[par], dk_max = st->dk_max[par];
  const int kref = d.s_neg ? dk_max : dk_min;
  // MODIFIED reference: the smallest (s >= 0) or largest (s < 0) rate integral;
  // GUIDED: the largest log weight (held as an order-preserving int)
  const float a_ref = d.guided ? order_float(st->a_max[par])
                               : __int_as_float(d.s_neg ? st->a_max[par] : st->a_min[par]);
  __syncthreads();
  const int dkv[kItems] = {dk4.x, dk4.y, dk4.z, dk4.w};
  const unsigned long long* wt = B.wtab + (size_t)p * kKcap;
  unsigned long long sum = 0ull;
  bool range_err = false;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (j0 + i < d.nc) {
      unsigned long long w;
      unsigned int k;
      if (!clone_weight(d, dkv[i], kref, av[i], a_ref, wt, B.exp2tab, w, k)) {
        range_err = true;
      } else {
        sum += w;
        if (!d.modified) {
          if (k < (unsigned int)kHistSmem) atomicAdd(&s_hist[k], 1u);
          else atomicAdd(&B.hist[(size_t)p * kKcap + k], 1u);
        }
      }
    }
  }
  if (range_err) st->err = kErrRange;
  const unsigned long long total = block_sum_u64(sum, s_red);
  if (!d.modified) {
    const int nb = hist_bins(dk_min, dk_max, kHistSmem);
    for (int b = tid; b < nb; b += kThreads) {
      const unsigned int c = s_hist[b];
      if (c) atomicAdd(&B.hist[(size_t)p * kKcap + b], c);
    }
  }
  if (tid == 0) {
    B.tile_sum[tile] = total;
    if (tile == d.first_tile) {
      st->kref = kref;
      st->a_ref = a_ref;
      st->beta = beta;
      st->U = philox4x32_10(make_uint4(0u, beta, 0u, kTagResample), (uint32_t)d.seed,
                            (uint32_t)(d.seed >> 32)).x;
    }
  }
}

// ---------------------------------------------------------------------------
// One block per population scans its tile sums once (each tile's exclusive prefix and
// the total T), so each block of the cloning stage reads two numbers instead of summing
// all the population's tile sums, work that grows with the square of its tile count
// (integer sums: the order of addition is immaterial).
//
// HIST: the interval's dynamical stage was the fused one with hist_on, so this kernel
// also does k_weights' work for the population.  With every activity below kTH the
// tile sums are sum_b n_tile(b) wtab[|b - k_ref|] over the tile histograms, which
// count the clones of each activity b; the population histogram of |dK - k_ref| is the
// sum of the tile histograms (both exact integer sums, so equal to the per-clone ones).
// Otherwise the weights of every clone are formed as in k_weights.  The histograms
// read are cleared for the next use.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
static_assert(kScanThreads == kTile, "the fallback of k_tile_scan<true> takes a tile per pass");
template <bool HIST>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(Batch B, int pop0) {
  __shared__ unsigned long long s_part[kScanThreads / 32];
  __shared__ unsigned int s_hb[HIST ? kTH : 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int p = pop0 + (int)blockIdx.x;
  const PopDesc d = B.pops[p];
  if constexpr (HIST) {
    PopState* st = B.st + p;
    const uint32_t beta = *B.beta;  // the interval being resampled
    const int par = (int)(beta & 1u);
    const int dk_min = st->dk_min[par], dk_max = st->dk_max[par];
    const int kref = d.s_neg ? dk_max : dk_min;
    const bool ovf = st->hovf != 0 || dk_min < 0 || dk_max >= kTH;
    for (int b = tid; b < kTH; b += kScanThreads) s_hb[b] = 0u;
    __syncthreads();  // every thread has read hovf before it is cleared
    if (tid == 0) {
      st->kref = kref;
      st->a_ref = __int_as_float(d.s_neg ? st->a_max[par] : st->a_min[par]);
      st->beta = beta;
      st->U = philox4x32_10(make_uint4(0u, beta, 0u, kTagResample), (uint32_t)d.seed,
                            (uint32_t)(d.seed >> 32)).x;
      st->hovf = 0;
    }
    const unsigned long long* wt = B.wtab + (size_t)p * kKcap;
    unsigned int* const th = B.thist + d.first_tile;
    if (!ovf) {
      const int b0 = dk_min, b1 = dk_max;  // 0 <= b0 <= b1 < kTH
      for (int i0 = 0; i0 < d.ntiles; i0 += kScanThreads) {
        const int i = i0 + tid;
        const bool in = i < d.ntiles;
        unsigned long long v = 0ull;
        for (int b = b0; b <= b1; ++b) {
          unsigned int c = 0u;
          if (in) {
            unsigned int* cell = th + (size_t)b * B.ntiles + i;
            c = *cell;
            if (c) {
              v += (unsigned long long)c * wt[abs_diff(b, kref)];
              *cell = 0u;
            }
          }
          const unsigned int cs = __reduce_add_sync(0xffffffffu, c);
          if (lane == 0 && cs) atomicAdd(&s_hb[b - b0], cs);
        }
        if (in) B.tile_sum[d.first_tile + i] = v;
      }
      __syncthreads();
      for (int b = b0 + tid; b <= b1; b += kScanThreads)
        B.hist[(size_t)p * kKcap + abs_diff(b, kref)] = s_hb[b - b0];
    } else {
      // an activity at or above kTH: the weight of every clone, a tile per pass
      for (int i = 0; i < d.ntiles; ++i) {
        const int64_t j = (int64_t)i * kTile + tid;
        unsigned long long w = 0ull;
        if (j < d.nc) {
          unsigned int k;
          if (!clone_weight(d, B.dKb[par][d.off + j], kref, 0.0f, 0.0f, wt, B.exp2tab, w, k))
            st->err = kErrRange;
          else
            atomicAdd(&B.hist[(size_t)p * kKcap + k], 1u);
        }
        const unsigned long long t = block_sum_u64_n<kScanThreads / 32>(w, s_part);
        if (tid == 0) B.tile_sum[d.first_tile + i] = t;
      }
      for (int64_t e = tid; e < (int64_t)kTH * d.ntiles; e += kScanThreads)
        th[(e / d.ntiles) * B.ntiles + e % d.ntiles] = 0u;
    }
    __syncthreads();  // the tile sums written above are read back below
  }
  unsigned long long run = 0ull;
  for (int i0 = 0; i0 < d.ntiles; i0 += kScanThreads) {
    const int i = i0 + tid;
    const unsigned long long v = (i < d.ntiles) ? B.tile_sum[d.first_tile + i] : 0ull;
    unsigned long long xs = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, xs, o);
      if (lane >= o) xs += y;
    }
    if (lane == 31) s_part[wid] = xs;
    __syncthreads();
    unsigned long long before = run + xs - v, chunk = 0ull;
#pragma unroll
    for (int q = 0; q < kScanThreads / 32; ++q) {
      const unsigned long long t = s_part[q];
      if (q < wid) before += t;
      chunk += t;
    }
    if (i < d.ntiles) B.tile_excl[d.first_tile + i] = before;
    run += chunk;
    __syncthreads();
  }
  if (tid == 0) B.st[p].T = run;
}

// ---------------------------------------------------------------------------
// Cloning stage for one tile of old clones.  The tile's exclusive prefix and the
// population total come from k_tile_scan (or the tile sums); a block scan gives S_k
// for its clones; old clone k owns the new
// slots [j_lo(S_k), j_lo(S_{k+1})).  The old clones are staged in shared memory, a
// map from new slot to old clone is scattered there, and every new slot of the
// tile's range is written once, coalesced.  The first tile of each population adds
// the psi term; the last block advances the interval counter (no block of this
// kernel reads it).
//
// FUSE: the cloning stage of interval beta and the dynamical stage of interval
// beta + 1 in one pass (pop_run, [eq] populations of at most 128 sites).  Each new
// clone is taken straight from its staged ancestor and evolved (the same BKL steps,
// draws and write-back as k_evolve, into the buffers of the other parity), so the
// population between the two stages never goes through global memory.  Lanes take
// new slots from a shared counter as their clones end, as in k_evolve.
// ---------------------------------------------------------------------------
#ifndef POP_GATHER_THREADS
#define POP_GATHER_THREADS 128
#endif
#ifndef POP_FUSE_THREADS
#define POP_FUSE_THREADS 128
#endif
#ifndef POP_FUSE_MIN_BLOCKS
#define POP_FUSE_MIN_BLOCKS 8  // 64 registers, no spills; pop_run's chains keep more than one launch resident
#endif
#ifndef POP_FUSE2_MIN_BLOCKS
#define POP_FUSE2_MIN_BLOCKS 6  // two clones per lane: up to 80 registers
#endif
// SCAN: the population totals and tile prefixes come from k_tile_scan; otherwise each
// block sums its population's tile sums (cheaper for a few tiles per population, but
// the extra path costs registers and scheduling when compiled into the same kernel).
// NCL (FUSE only): clones each lane advances together in the dynamical stage, 1 or 2
// (two independent Philox and bit-select chains in flight per lane).
// FULL (FUSE only): every population of the launch has L = 64 W, so the ring fills
// the lattice words (active_bonds32<.., true>).
template <int W, int NT, bool FUSE = false, bool MOD = false, bool SCAN = true, int NCL = 1, bool FULL = false>
__global__ void __launch_bounds__(NT, FUSE ? (NCL == 1 ? POP_FUSE_MIN_BLOCKS * 128 / NT : POP_FUSE2_MIN_BLOCKS)
                                           : (NT == 128 ? 11 : (NT == 256 ? 6 : 3)))
    k_gather(Batch B, float dt_f, int tile0) {
  constexpr int NI = kTile / NT;   // old clones per thread
  constexpr int NWARP = NT / 32;
  constexpr int WS = W > 0 ? W : 1;  // W == 0: wide lattices, copied without staging
  static_assert(!FUSE || W > 0, "the fused stage needs staged lattices");
  static_assert(NI % 4 == 0 && NI * NT == kTile, "whole int4 loads of activities per thread");
  static_assert(NCL == 1 || NCL == 2, "one or two clones per lane");
  __shared__ unsigned long long s_x[W > 0 ? kTile : 1][WS];
  // the old clones' cumulative activities (the fused stage reads each new clone's from
  // global memory when the clone is taken, keeping shared memory for more blocks)
  __shared__ int32_t s_K[FUSE ? 1 : kTile];
  // the new slots of the tile's old clones: the map from new slot to old clone
  // (uint16, kMap entries) or, when one old clone has more copies than the map holds,
  // the ranges j_lo (uint32, kTile + 1 entries) searched instead; one buffer
  static_assert(kMap * sizeof(uint16_t) <= (kTile + 1) * sizeof(uint32_t), "map fits the range buffer");
  __shared__ __align__(16) uint32_t s_rng[kTile + 1];
  uint32_t* const s_jlo = s_rng;
  uint16_t* const s_src = reinterpret_cast<uint16_t*>(s_rng);
  __shared__ uint32_t s_J[2];
  __shared__ unsigned long long s_red[SCAN ? 1 : NWARP];
  __shared__ unsigned long long s_wsum[NWARP];
  // FUSE only: the population's waiting-time factors, the log table, the Philox key
  // schedule, the slot counter and the block's activity range of the next interval
  __shared__ float s_inv[FUSE ? kMaxL + 1 : 1];
  __shared__ float2 s_logtab[FUSE ? 64 : 1];
  __shared__ uint2 s_keys[FUSE ? 10 : 1];
  // FUSE: the first kWStage entries of the population's weight table (the activity
  // spreads of nearly every interval), read from shared memory instead of a dependent
  // global load (the separate cloning stage measured faster without the extra barrier)
  constexpr int kWStage = 64;
  __shared__ unsigned long long s_wt[FUSE ? kWStage : 1];
  __shared__ __align__(16) uint32_t s_kth8[FUSE ? 512 : 1];
  // FUSE, plain weights: activity histograms of the first three tiles the new clones
  // fall in (the rest go straight to global memory)
  __shared__ unsigned int s_th[(FUSE && !MOD) ? 3 * kTH : 1];
  __shared__ int s_take;
  __shared__ unsigned int s_pack[2];  // FUSE: clones packed in the current / next tail round
  __shared__ int s_nmin, s_nmax, s_namin, s_namax;
  __shared__ unsigned int s_nev;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = tile0 + (int)blockIdx.x;
  const int p = B.tile_pop[tile];
  const PopDesc d = B.pops[p];
  PopState* st = B.st + p;
  const int lt = tile - d.first_tile;
  const uint32_t nc = (uint32_t)d.nc;
  const int64_t base = (int64_t)tile * kTile;
  const int64_t j0 = base - d.off + (int64_t)tid * NI;
  // the interval being resampled, as recorded by k_weights: the device counter is
  // advanced by this kernel's last block and may not be read here
  const uint32_t beta = st->beta;
  const int par = (int)(beta & 1u);
  const unsigned long long* const Xo = B.Xb[par];
  const int32_t* const KXo = B.KXb[par];
  if constexpr (FUSE) {
    const float* src = B.inv_rate + (size_t)p * kInvStride;
    for (int r = tid; r <= kMaxL; r += NT) s_inv[r] = (r <= d.L) ? src[r] : 0.0f;
    if (tid < 64) s_logtab[tid] = B.logtab[tid];
    if (tid < 128) reinterpret_cast<uint4*>(s_kth8)[tid] = reinterpret_cast<const uint4*>(g_kth8.w)[tid];
    if constexpr (!MOD)
      for (int e = tid; e < 3 * kTH; e += NT) s_th[e] = 0u;
    if (tid < 10)
      s_keys[tid] = make_uint2((uint32_t)d.seed + (uint32_t)tid * 0x9E3779B9u,
                               (uint32_t)(d.seed >> 32) + (uint32_t)tid * 0xBB67AE85u);
    if (tid == 0) {
      s_take = 0;
      s_pack[0] = 0u;
      s_pack[1] = 0u;
      s_nmin = INT_MAX;
      s_nmax = INT_MIN;
      s_namin = INT_MAX;
      s_namax = INT_MIN;
      s_nev = 0u;
    }
  }

  const unsigned long long* wt = B.wtab + (size_t)p * kKcap;
  if (FUSE && tid < kWStage) s_wt[tid] = wt[tid];
  // independent loads first: activities and the old clones of this tile
  int dkv[NI];
#pragma unroll
  for (int v = 0; v < NI / 4; ++v) {
    const int4 dk4 = reinterpret_cast<const int4*>(B.dKb[par] + base)[tid * (NI / 4) + v];
    dkv[4 * v] = dk4.x; dkv[4 * v + 1] = dk4.y; dkv[4 * v + 2] = dk4.z; dkv[4 * v + 3] = dk4.w;
  }
#pragma unroll
  for (int m = 0; m < NI; ++m) {
    const int i = m * NT + tid;
    if (base - d.off + i < d.nc) {
      if constexpr (W > 0) {
        unsigned long long x[W];
        load_lat<W>(Xo, base + i, x);
#pragma unroll
        for (int q = 0; q < W; ++q) s_x[i][q] = x[q];
      }
      if constexpr (!FUSE) s_K[i] = KXo[base + i];
    }
  }
  float av[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) av[i] = 0.0f;
  if (d.modified) {
#pragma unroll
    for (int v = 0; v < NI / 4; ++v) {
      const float4 a4 = reinterpret_cast<const float4*>(B.Ab[par] + base)[tid * (NI / 4) + v];
      av[4 * v] = a4.x; av[4 * v + 1] = a4.y; av[4 * v + 2] = a4.z; av[4 * v + 3] = a4.w;
    }
  }
  const int kref = st->kref;
  const float a_ref = st->a_ref;
  const unsigned long long c = 2ull * (unsigned long long)st->U + 1ull;

  // population total T and this tile's exclusive prefix
  unsigned long long T = 0ull, excl = 0ull, tT = 0ull, tE = 0ull;
  if constexpr (SCAN) {
    T = st->T;
    excl = B.tile_excl[tile];
  } else {
    for (int i = tid; i < d.ntiles; i += NT) {
      const unsigned long long v = B.tile_sum[d.first_tile + i];
      tT += v;
      if (i < lt) tE += v;
    }
  }

  // weights of this tile's clones and their scan within each warp
  if constexpr (FUSE) __syncthreads();  // s_wt
  unsigned long long w[NI];
  unsigned long long tsum = 0ull;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    w[i] = 0ull;
    if (j0 + i < d.nc) {
      if (FUSE && !d.modified) {  // plain: wtab[|dK - k_ref|] (0 beyond the table: k_weights reports it)
        const unsigned int k = abs_diff(dkv[i], kref);
        w[i] = k < (unsigned int)kWStage ? s_wt[k] : (k < (unsigned int)kKcap ? __ldg(wt + k) : 0ull);
      } else {
        unsigned int k;
        clone_weight(d, dkv[i], kref, av[i], a_ref, wt, B.exp2tab, w[i], k);
      }
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
  if constexpr (SCAN) {
    __syncthreads();
  } else {
    T = block_sum_u64_n<NWARP>(tT, s_red);
    excl = block_sum_u64_n<NWARP>(tE, s_red);
  }

  const int sh = max(0, 64 - __clzll((long long)T) - 24);
  const float ratio = __fdiv_rn((float)nc, __uint2float_rn((uint32_t)(T >> sh)));
  unsigned long long run = excl + xs - tsum;
  for (int q = 0; q < wid; ++q) run += s_wsum[q];
  if (d.iid) {
    // [iid]: publish this tile's prefix sums; k_select_iid draws the points
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      B.S[base + (int64_t)tid * NI + i] = run;
      run += w[i];
    }
    if (lt == 0 && tid == 0) st->T = T;
  } else {
  uint32_t jl[NI + 1];
  j_lo_run<NI>(run, w, T, c, nc, sh, ratio, jl);
  if (tid == 0) s_J[0] = jl[0];
  if (tid == NT - 1) s_J[1] = jl[NI];
  __syncthreads();

  const uint32_t J0 = s_J[0], J1 = s_J[1];
  const bool mapped = (J1 - J0) <= (uint32_t)kMap;
  if (FUSE && mapped) {
    // the thread's old clones own the new slots [jl[0], jl[NI]): a marker at the first
    // slot of each old clone with copies, then an inclusive max scan over the slots
    // (markers grow with the slot, and the first slot always has one); no divergent
    // loops, at the cost of two more barriers (the separate cloning stage, bound by
    // memory, measured faster with the loops below)
    constexpr int SP = kMap / NT;  // slots per thread in the scan
    static_assert(SP % 8 == 0, "whole 16-byte words of the map per thread");
    const int nsl = (int)(J1 - J0);
    for (int e = tid; e < kMap / 2; e += NT) s_rng[e] = 0u;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NI; ++i)
      if (jl[i + 1] > jl[i]) s_src[jl[i] - J0] = (uint16_t)(tid * NI + i);
    __syncthreads();
    uint4 pk[SP / 8];
    int m = 0;
#pragma unroll
    for (int v = 0; v < SP / 8; ++v) {
      pk[v] = reinterpret_cast<const uint4*>(s_src)[tid * (SP / 8) + v];
      const uint32_t wd[4] = {pk[v].x, pk[v].y, pk[v].z, pk[v].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) m = max(m, (int)max(wd[q] & 0xffffu, wd[q] >> 16));
    }
    int inc = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = max(inc, y);
    }
    __shared__ int s_mx[NWARP];
    if (lane == 31) s_mx[wid] = inc;
    int run = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) run = 0;
    __syncthreads();
    for (int q = 0; q < wid; ++q) run = max(run, s_mx[q]);
#pragma unroll
    for (int v = 0; v < SP / 8; ++v) {
      uint32_t wd[4] = {pk[v].x, pk[v].y, pk[v].z, pk[v].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        run = max(run, (int)(wd[q] & 0xffffu));
        const uint32_t lo = (uint32_t)run;
        run = max(run, (int)(wd[q] >> 16));
        wd[q] = lo | ((uint32_t)run << 16);
      }
      if (tid * SP + 8 * v < nsl) reinterpret_cast<uint4*>(s_src)[tid * (SP / 8) + v] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
  } else if (mapped) {
    // the thread's old clones own the new slots [jl[0], jl[NI]), held in its registers
#pragma unroll
    for (int i = 0; i < NI; ++i)
      for (uint32_t jj = jl[i]; jj < jl[i + 1]; ++jj) s_src[jj - J0] = (uint16_t)(tid * NI + i);
  } else {
#pragma unroll
    for (int i = 0; i < NI; ++i) s_jlo[tid * NI + i] = jl[i];
    if (tid == NT - 1) s_jlo[kTile] = jl[NI];
  }
  __syncthreads();
  auto source = [&](uint32_t jj) -> int {
    if (mapped) return s_src[jj - J0];
    int lo = 0, hi = kTile - 1;  // one old clone with very many copies: search j_lo
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_jlo[mid] <= jj) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  if constexpr (FUSE) {
    // dynamical stage of interval beta + 1 for the new slots [J0, J1): each lane holds
    // NCL clones; an empty clone slot takes the next new slot of the tile from the
    // shared counter (all of a warp's empty slots in one atomic), so lanes stay busy
    // until the tile's slots run out.  Every live clone takes one Philox draw (its next
    // two BKL steps) per iteration; the steps are predicated, without branches.
    const uint32_t beta1 = beta + 1u;
    const int pn = par ^ 1;
    unsigned long long* const Xn = B.Xb[pn];
    int32_t* const KXn = B.KXb[pn];
    int32_t* const dKn = B.dKb[pn];
    float* const An = B.Ab[pn];
    const int n = (int)(J1 - J0);
    const int L = d.L;
    // the tile of the new slot J0 (tiles of the next interval: 1024 slots, populations
    // tile-aligned), and whether an activity fell outside the histograms
    const int t0 = (int)((d.off + (int64_t)J0) >> 10);
    const bool hist_on = !MOD && B.hist_on != 0;
    bool ovf = false;
    const unsigned int lt_mask = (1u << lane) - 1u;
    int cl[NCL], h[NCL];              // the slot's new clone (offset from J0, -1: empty)
    int kold[NCL];                    // its ancestor's cumulative activity
    uint32_t q[NCL];
    float t[NCL], acc[NCL];
    unsigned long long x[NCL][W];
    int hmin = INT_MAX, hmax = INT_MIN, amin = INT_MAX, amax = INT_MIN;
    unsigned int ev = 0u;
#pragma unroll
    for (int k = 0; k < NCL; ++k) {
      cl[k] = -1;
      kold[k] = 0;
      h[k] = 0;
      q[k] = 0u;
      t[k] = 0.0f;
      acc[k] = 0.0f;
#pragma unroll
      for (int w = 0; w < W; ++w) x[k][w] = 0ull;
    }
    // one iteration of the lane's clones: a Philox draw each, two predicated BKL steps,
    // and the write-back of a clone whose interval ended
    auto iterate = [&]() {
      uint4 d4[NCL];
      float E1[NCL], E2[NCL];
#pragma unroll
      for (int k = 0; k < NCL; ++k)
        d4[k] = philox4x32_10_rk(make_uint4(q[k], beta1, J0 + (uint32_t)cl[k], kTagEvolve), s_keys);
#pragma unroll
      for (int k = 0; k < NCL; ++k) {
        E1[k] = neg_ln_u(d4[k].x, s_logtab);
        E2[k] = neg_ln_u(d4[k].z, s_logtab);
      }
#pragma unroll
      for (int k = 0; k < NCL; ++k) {
        const bool live = cl[k] >= 0;
        uint32_t u[2 * W];
        split32<W>(x[k], u);
        const uint8_t* kth8 = reinterpret_cast<const uint8_t*>(s_kth8);
        const bool h1 = bkl_step_pred<W, MOD, FULL>(u, t[k], acc[k], (uint32_t)L - 1u, s_inv, E1[k], d4[k].y,
                                                    dt_f, live, kth8);
        const bool h2 = bkl_step_pred<W, MOD, FULL>(u, t[k], acc[k], (uint32_t)L - 1u, s_inv, E2[k], d4[k].w,
                                                    dt_f, h1, kth8);
        join32<W>(u, x[k]);
        h[k] += (int)h1 + (int)h2;
        ++q[k];
        bool run = h2;
        if (run && q[k] >= kStepLimit / 2u) {  // guard: an interval must end; report, never spin
          st->err = kErrRange;
          run = false;
        }
        if (live && !run) {
          const int64_t dst = d.off + (int64_t)J0 + cl[k];
          store_lat<W>(Xn, dst, x[k]);
          KXn[dst] = kold[k] + h[k];
          dKn[dst] = h[k];
          if (MOD) {
            An[dst] = acc[k];
            amin = min(amin, __float_as_int(acc[k]));  // A >= 0: float bits order like values
            amax = max(amax, __float_as_int(acc[k]));
          }
          hmin = min(hmin, h[k]);
          hmax = max(hmax, h[k]);
          ev += (unsigned int)h[k];
          cl[k] = -1;
        }
      }
    };
    // lanes take new slots from the shared counter until it runs out
    for (;;) {
      unsigned int m[NCL];
      int tot = 0;
#pragma unroll
      for (int k = 0; k < NCL; ++k) {
        m[k] = __ballot_sync(0xffffffffu, cl[k] < 0);
        tot += __popc(m[k]);
      }
      if (tot != 0) {
        // one read of the counter per warp keeps every branch below warp-uniform
        int taken = 0;
        if (lane == 0) taken = *(volatile int*)&s_take;
        taken = __shfl_sync(0xffffffffu, taken, 0);
        if (taken >= n) break;  // the counter ran out: on to the packed rounds below
        int base_i = 0;
        if (lane == 0) base_i = atomicAdd(&s_take, tot);
        base_i = __shfl_sync(0xffffffffu, base_i, 0);
#pragma unroll
        for (int k = 0; k < NCL; ++k) {
          const int idx = base_i + __popc(m[k] & lt_mask);
          if (cl[k] < 0 && idx < n) {
            cl[k] = idx;
            const int sk = source(J0 + (uint32_t)idx);
            kold[k] = KXo[base + sk];
#pragma unroll
            for (int w = 0; w < W; ++w) x[k][w] = s_x[sk][w];
            t[k] = 0.0f;
            acc[k] = 0.0f;
            h[k] = 0;
            q[k] = 0u;
          }
          base_i += __popc(m[k]);
        }
        if (tot == 32 * NCL) {
          // every slot was empty and the claim may have come after the last clone
          bool any = false;
#pragma unroll
          for (int k = 0; k < NCL; ++k) any = any || cl[k] >= 0;
          if (__ballot_sync(0xffffffffu, any) == 0u) continue;
        }
      }
      iterate();
    }
    // The counter has run out.  Each round packs the block's remaining clones into the
    // lowest threads (through the staging buffer of the old clones, no longer read),
    // so that warps left without clones stop issuing, and runs one iteration.
    struct Packed {
      unsigned long long x[W];
      float t, acc;
      int cl, h, kold;
      uint32_t q;
    };
    static_assert(sizeof(Packed) * NT * NCL <= sizeof(s_x), "the packed clones fit the staging buffer");
    Packed* const s_packed = reinterpret_cast<Packed*>(&s_x[0][0]);
    for (int rnd = 0;; ++rnd) {
      __syncthreads();  // every warp is done with the staging buffer and the last round
      unsigned int* const cnt = &s_pack[rnd & 1];
#pragma unroll
      for (int k = 0; k < NCL; ++k) {
        if (cl[k] >= 0) {
          Packed& e = s_packed[atomicAdd(cnt, 1u)];
#pragma unroll
          for (int w = 0; w < W; ++w) e.x[w] = x[k][w];
          e.t = t[k];
          e.acc = acc[k];
          e.cl = cl[k];
          e.h = h[k];
          e.kold = kold[k];
          e.q = q[k];
        }
      }
      if (tid == 0) s_pack[(rnd + 1) & 1] = 0u;
      __syncthreads();
      const int count = (int)*cnt;
      if (count == 0) break;
      bool any = false;
#pragma unroll
      for (int k = 0; k < NCL; ++k) {
        const int i = tid + k * NT;
        cl[k] = -1;
        if (i < count) {
          const Packed& e = s_packed[i];
#pragma unroll
          for (int w = 0; w < W; ++w) x[k][w] = e.x[w];
          t[k] = e.t;
          acc[k] = e.acc;
          cl[k] = e.cl;
          h[k] = e.h;
          kold[k] = e.kold;
          q[k] = e.q;
          any = true;
        }
      }
      if (__ballot_sync(0xffffffffu, any) != 0u) iterate();
    }
    hmin = __reduce_min_sync(0xffffffffu, hmin);
    hmax = __reduce_max_sync(0xffffffffu, hmax);
    ev = __reduce_add_sync(0xffffffffu, ev);
    if (MOD) {
      amin = __reduce_min_sync(0xffffffffu, amin);
      amax = __reduce_max_sync(0xffffffffu, amax);
    }
    if (lane == 0 && hmin != INT_MAX) {
      atomicMin(&s_nmin, hmin);
      atomicMax(&s_nmax, hmax);
      atomicAdd(&s_nev, ev);
      if (MOD) {
        atomicMin(&s_namin, amin);
        atomicMax(&s_namax, amax);
      }
    }
    __syncthreads();
    if (tid == 0 && s_nmin != INT_MAX) {
      atomicMin(&st->dk_min[pn], s_nmin);
      atomicMax(&st->dk_max[pn], s_nmax);
      atomicAdd(&st->events, (unsigned long long)s_nev);
      if (MOD) {
        atomicMin(&st->a_min[pn], s_namin);
        atomicMax(&st->a_max[pn], s_namax);
      }
    }
    if (hist_on) {
      // count the new clones' activities by tile (after the loop, from the activities
      // just written: counting inside the loop costs the loop registers)
      for (int jj = tid; jj < n; jj += NT) {
        const int64_t dst = d.off + (int64_t)J0 + jj;
        const int hh = dKn[dst];
        if (hh < kTH) {
          const int tn = (int)(dst >> 10);
          if (tn - t0 < 3) atomicAdd(&s_th[(tn - t0) * kTH + hh], 1u);
          else atomicAdd(&B.thist[(size_t)hh * B.ntiles + tn], 1u);
        } else {
          ovf = true;
        }
      }
      __syncthreads();
      // a shared bin holds only clones of its tile, so a non-zero bin names a real tile
      for (int e = tid; e < 3 * kTH; e += NT) {
        const unsigned int v = s_th[e];
        if (v) atomicAdd(&B.thist[(size_t)(e % kTH) * B.ntiles + t0 + e / kTH], v);
      }
      if (ovf) st->hovf = 1;
    }
  } else if constexpr (W > 0) {
    for (uint32_t jj = J0 + (uint32_t)tid; jj < J1; jj += NT) {
      const int k = source(jj);
      unsigned long long x[W];
#pragma unroll
      for (int q = 0; q < W; ++q) x[q] = s_x[k][q];
      const int64_t dst = d.off + (int64_t)jj;
      store_lat<W>(B.Y, dst, x);
      B.KY[dst] = s_K[k];
      B.anc[dst] = lt * kTile + k;
    }
  } else {
    // one warp per new clone; its lanes copy the lattice words (coalesced)
    for (uint32_t jj = J0 + (uint32_t)wid; jj < J1; jj += NWARP) {
      const int k = source(jj);
      const int64_t dst = d.off + (int64_t)jj;
      for (int q = lane; q < B.W; q += 32)
        B.Y[dst * B.W + q] = Xo[(base + k) * B.W + q];
      if (lane == 0) {
        B.KY[dst] = s_K[k];
        B.anc[dst] = lt * kTile + k;
      }
    }
  }
  }  // [eq]

  // psi term of eq. (psihat) for this interval, once per population.
  // MODIFIED (reading of eq. def-ups-ssep): -c A_ref + log1p((T - N_c 2^F) / (N_c 2^F))
  // from the exact total T of the quantised weights.
  // GUIDED: X_ref + log1p(...) with X_ref the largest log weight.
  if (d.modified && lt == 0 && tid == 0) {
    const double base_w = ldexp((double)d.nc, d.F);
    const long long D = (long long)T - (long long)((unsigned long long)d.nc << d.F);
    const double ref = d.guided ? (double)a_ref : -(double)d.c_f * (double)a_ref;
    st->psi_acc += ref + log1p((double)D / base_w);
    st->dk_min[par] = INT_MAX;
    st->dk_max[par] = INT_MIN;
    st->a_min[par] = INT_MAX;
    st->a_max[par] = INT_MIN;
  }
  // plain: term = -s k_ref + ln( (1/N_c) sum_k n_k exp(-|s| k) ) from the exact
  // activity histogram, the log taken as log1p of the expm1 sum when the mean is > 1/2.
  if (!d.modified && lt == 0 && wid == 0) {
    const int dk_min = st->dk_min[par], dk_max = st->dk_max[par];
    const int R = hist_bins(dk_min, dk_max, kKcap);
    unsigned int* h = B.hist + (size_t)p * kKcap;
    const double* qt = B.qtab + (size_t)p * kKcap;
    const double* qm = B.qm1tab + (size_t)p * kKcap;
    double a = 0.0, q = 0.0;
    for (int b = lane; b < R; b += 32) {
      const unsigned int cnt = h[b];
      if (cnt) {
        a = fma((double)cnt, qm[b], a);
        q = fma((double)cnt, qt[b], q);
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
      st->dk_min[par] = INT_MAX;
      st->dk_max[par] = INT_MIN;
      st->a_min[par] = INT_MAX;
      st->a_max[par] = INT_MIN;
    }
  }
  // GUIDED: the new clones' ancestors are known, so the next dynamical stage can start
  // each new clone from its ancestor's rate sums
  if (d.guided && lt == 0 && tid == 0) st->gcarry = 1;
  // the interval ends here unless [iid] selection still has to run
  if (!B.any_iid && blockIdx.x == gridDim.x - 1 && tid == 0) *B.beta += 1u;
}

// ---------------------------------------------------------------------------
// [iid] selection (Sec. 4.1): new clone j of the population pulls old clone k with
// S_k <= alpha_j < S_{k+1}, alpha_j = floor(U64_j T / 2^64), U64_j from draw
// (j, beta, 0, 4).  The search runs in two levels over the same non-decreasing prefix
// sums: the last tile whose first prefix (k_tile_scan's tile_excl) is <= alpha_j,
// from a shared-memory copy of the population's tile prefixes, then the last k of
// that tile with S_k <= alpha_j.  One block per tile of new slots; populations with
// [eq] selection are skipped.  The last block advances the interval counter.
// ---------------------------------------------------------------------------
constexpr int kIidSmemTiles = 2048;  // tile prefixes kept in shared memory (16 KB)
template <int W>
__global__ void __launch_bounds__(kThreads) k_select_iid(Batch B) {
  __shared__ unsigned long long s_te[kIidSmemTiles];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = blockIdx.x;
  const int p = B.tile_pop[tile];
  const PopDesc d = B.pops[p];
  if (d.iid) {
    const unsigned long long* te = B.tile_excl + d.first_tile;
    const bool staged = d.ntiles <= kIidSmemTiles;
    if (staged)
      for (int i = tid; i < d.ntiles; i += kThreads) s_te[i] = te[i];
    __syncthreads();
    const PopState* st = B.st + p;
    const unsigned long long T = st->T;
    const uint32_t beta = st->beta;
    const int par = (int)(beta & 1u);
    const unsigned long long* const Xo = B.Xb[par];
    const int32_t* const KXo = B.KXb[par];
    const int lt = tile - d.first_tile;
    const unsigned long long* S = B.S + d.off;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    for (int i = (W > 0 ? tid : wid); i < kTile; i += (W > 0 ? kThreads : kWarps)) {
      const int64_t j = (int64_t)lt * kTile + i;
      if (j >= d.nc) break;
      const uint4 r = philox4x32_10(make_uint4((uint32_t)j, beta, 0u, kTagIid), k0, k1);
      const unsigned long long alpha = __umul64hi(((unsigned long long)r.y << 32) | r.x, T);
      int tlo = 0, thi = d.ntiles - 1;  // the last tile whose first prefix is <= alpha
      while (tlo < thi) {
        const int mid = (tlo + thi + 1) >> 1;
        if ((staged ? s_te[mid] : te[mid]) <= alpha) tlo = mid; else thi = mid - 1;
      }
      long long lo = (long long)tlo * kTile;  // the last k of the tile with S_k <= alpha
      long long hi = min((long long)d.nc, lo + kTile) - 1;
      while (lo < hi) {
        const long long mid = lo + (hi - lo + 1) / 2;
        if (S[mid] <= alpha) lo = mid; else hi = mid - 1;
      }
      const int64_t src = d.off + lo, dst = d.off + j;
      if constexpr (W > 0) {
        unsigned long long x[W];
        load_lat<W>(Xo, src, x);
        store_lat<W>(B.Y, dst, x);
        B.KY[dst] = KXo[src];
        B.anc[dst] = (int32_t)lo;
      } else {
        for (int q = lane; q < B.W; q += 32) B.Y[dst * B.W + q] = Xo[src * B.W + q];
        if (lane == 0) {
          B.KY[dst] = KXo[src];
          B.anc[dst] = (int32_t)lo;
        }
      }
    }
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) *B.beta += 1u;
}

// ---------------------------------------------------------------------------
// GUIDED dynamical stage (Sec. 2.2, eqs. modpdef and upsdef, with a local potential
// U(C) = sum_i phi(sites i-4..i+4) in place of the uniform e^-s of Sec. 3.2).  The hop
// across active bond b has rate 2^-40 Q(k_b), Q(k) = floor(TA[a] TB[c] / 2^44) =
// 2^40 exp(k 2^-17) to 3e-9 (k + 2^20 = 2^11 a + c), with the exponent
// k_b = clamp(dU_b - s_q, +-2^20): dU_b = U(C^b) - U(C) from the ten windows that
// contain the bond's sites (exact fixed-point integers), s_q = s in units of 2^-17.
// dU_b depends only on the 18 sites b-8..b+9, of which sites b and b+1 differ, so it is
// tabulated per population over the 17 free bits (k_guided_table, when the potential is
// set), and Q(k_b) likewise once s is fixed (k_guided_qtab): a bond's rate is one load.
// Step e uses draw (e, beta, j, 5): E = -ln u(w0); r'_f = float(R) 2^-40 with R = sum Q;
// tau = E / r'_f; the bond is the first whose cumulative Q exceeds
// floor((w2 2^32 + w1) R / 2^64).  Log weight in FP32, every term formed at its own size
// (no large terms that cancel):
//   X = sum_hops ((c_s - float(k_b + s_q) 2^-17) - eta) - sum_segments (r - r'_f) tau,
// c_s = float(s_q 2^-17 - s), eta = (2^40 r'_f - R) / R the rounding of the total rate;
// this is the weight of the rates simulated, so the estimate is unbiased for any
// potential.  Requires 18 <= L <= 128.
// ---------------------------------------------------------------------------
constexpr int kGuideThreads = 128;
constexpr int kGuideGroup = 8;              // bonds per rate-sum group
constexpr int kGuideSegBits = 17;
constexpr int kGuideSeg = 1 << kGuideSegBits;

// The table index of an active bond's segment: its bits 0..8 (sites b-8..b) and
// 10..17 (sites b+2..b+9); bit 9 (site b+1) is the complement of bit 8.
__device__ __forceinline__ uint32_t guided_index(uint32_t seg) {
  return (seg & 0x1FFu) | ((seg >> 10) << 9);
}

// Q(k) = floor(TA[a] TB[c] / 2^44).
__device__ __forceinline__ unsigned long long guided_q(int k, const unsigned long long* tab) {
  const uint32_t u = (uint32_t)(k + kGuideKmax);
  const unsigned long long ta = __ldg(tab + (u >> 11)), tb = __ldg(tab + kGuideTabA + (u & 2047u));
  return (__umul64hi(ta, tb) << 20) | ((ta * tb) >> 44);
}

// dU of the active bond whose segment has table index i, population p.
__global__ void __launch_bounds__(kThreads) k_guided_table(Batch B, int p) {
  const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= (uint32_t)kGuideSeg) return;
  const uint32_t b8 = (i >> 8) & 1u;
  const uint32_t seg = (i & 0x1FFu) | ((b8 ^ 1u) << 9) | ((i >> 9) << 10);
  const uint32_t seg2 = seg ^ (3u << 8);
  const int32_t* phi = B.phi + (size_t)p * 512;
  int dU = 0;
#pragma unroll
  for (int m = 0; m < 10; ++m) dU += phi[(seg2 >> m) & 511u] - phi[(seg >> m) & 511u];
  B.gdu[(size_t)p * kGuideSeg + i] = dU;
}

// Q(clamp(dU - s_q)) of every table index of every population (s fixed for the run).
__global__ void __launch_bounds__(kThreads) k_guided_qtab(Batch B) {
  const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
  const int p = (int)blockIdx.y;
  const int s_q = B.pops[p].s_q;
  const size_t at = (size_t)p * kGuideSeg + i;
  const int k = min(max(B.gdu[at] - s_q, -kGuideKmax), kGuideKmax);
  B.gq[at] = guided_q(k, B.gtab);
}

// Sites start, start+1, ..., start+63 (mod L) of a configuration as the bits of one
// word (bit k = site (start + k) mod L), 18 <= L, 0 <= start < L; bits of x at or
// above L are zero.
template <int W>
__device__ __forceinline__ unsigned long long ring_window(const unsigned long long (&x)[W], int L,
                                                         int start) {
  if (W == 1 || L <= 64) {
    const unsigned long long x0 = x[0];
    unsigned long long y = (start == 0) ? x0 : ((x0 >> start) | (x0 << (L - start)));
    if (L < 64) {
      y &= (1ull << L) - 1ull;
      y |= y << L;                       // 2L >= 36 sites
      if (2 * L < 64) y |= y << (2 * L);  // 4L >= 72 sites
    }
    return y;
  } else {
    const unsigned long long x0 = x[0], x1 = x[W - 1];
    unsigned long long y = (start == 0) ? x0 : (start < 64 ? ((x0 >> start) | (x1 << (64 - start)))
                                                           : (x1 >> (start - 64)));
    const int valid = L - start;  // sites before the wrap to site 0
    if (valid < 64) y |= x0 << valid;
    return y;
  }
}

// Rate of the bond whose 18-site segment starts at bit o of window v (its sites at bits
// o + 8 and o + 9): Q from the table if they differ, else 0 (the table is read only for
// an active bond).
__device__ __forceinline__ unsigned long long guided_q_at(unsigned long long v, int o,
                                                          const unsigned long long* qtab) {
  const uint32_t seg = (uint32_t)(v >> o) & 0x3FFFFu;
  const bool act = ((seg >> 8) ^ (seg >> 9)) & 1u;
  unsigned long long q = 0ull;
  if (act) q = __ldg(qtab + guided_index(seg));
  return q;
}

// float(v) rounded to nearest (ties to even) for a 64-bit unsigned v, in 32-bit integer
// arithmetic (the 64-bit integer <-> float conversions run on the narrow FP64 pipe):
// the 24 leading bits, rounded by the bits below them.
__device__ __forceinline__ float u64_to_float_rn(unsigned long long v) {
  if ((v >> 24) == 0ull) return __uint2float_rn((uint32_t)v);  // exact
  const int p = 63 - __clzll((long long)v);                        // leading one, >= 24
  const int sh = p - 23;
  uint32_t m = (uint32_t)(v >> sh);                                // 24 bits
  const unsigned long long rest = v & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  m += (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
  int e = p;
  if (m == (1u << 24)) { m >>= 1; ++e; }
  return __uint_as_float(((uint32_t)(e + 127) << 23) | (m & 0x007fffffu));
}

// The integer value of a float that holds an integer in [1, 2^64): mantissa shifted.
__device__ __forceinline__ unsigned long long float_to_u64_exact(float f) {
  const uint32_t bits = __float_as_uint(f);
  const int e = (int)((bits >> 23) & 0xffu) - 127;
  const unsigned long long m = (unsigned long long)((bits & 0x007fffffu) | 0x00800000u);
  return e >= 23 ? m << (e - 23) : m >> (23 - e);
}

__device__ __forceinline__ float i64_to_float_rn(long long v) {
  if (v >= -2147483647ll && v <= 2147483647ll) return __int2float_rn((int)v);
  const float f = u64_to_float_rn(v < 0 ? (unsigned long long)(-v) : (unsigned long long)v);
  return v < 0 ? -f : f;
}

// One lane per clone; a lane whose clone has ended takes the next clone of the block's
// share of a tile (spb slots: a whole tile, or a half, quarter or eighth of one for a
// batch of few tiles, so that it still fills the GPU).  The rate sums of a clone's
// groups of eight bonds live in shared memory
// (group-major: the lanes of a warp never share a bank); a newly taken clone's sums
// are formed by the whole warp (each lane four or two bonds), so refills stay uniform.
#ifndef POP_GUIDE_MIN_BLOCKS
#define POP_GUIDE_MIN_BLOCKS 8   // 64 registers, 32 warps per SM (5 blocks at 96 registers: 5 % slower)
#endif
#ifndef POP_GUIDE1_MIN_BLOCKS
#define POP_GUIDE1_MIN_BLOCKS 8  // one-word lattices too (1 block at 140 registers and
                                 // unpredicated table loads: 1.3x slower)
#endif

template <int W>
__global__ void __launch_bounds__(kGuideThreads, W == 1 ? POP_GUIDE1_MIN_BLOCKS : POP_GUIDE_MIN_BLOCKS)
    k_evolve_guided(Batch B, float dt_f, int spb) {
  constexpr int nb = 64 * W, ng = nb / kGuideGroup;
  constexpr int BPL = nb / 32;  // bonds per lane in the cooperative sums
  __shared__ unsigned long long s_g[ng][kGuideThreads];
  __shared__ float2 s_log[64];
  __shared__ int s_take;
  __shared__ int s_min, s_max, s_amin, s_amax;
  __shared__ unsigned int s_ev;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t base = (int64_t)blockIdx.x * spb;  // the block's first slot
  const int p = B.tile_pop[base / kTile];
  const PopDesc d = B.pops[p];
  if (tid < 64) s_log[tid] = B.logtab[tid];
  if (tid == 0) {
    s_take = 0;
    s_min = INT_MAX;
    s_max = INT_MIN;
    s_amin = INT_MAX;
    s_amax = INT_MIN;
    s_ev = 0u;
  }
  __syncthreads();
  const uint32_t beta = *B.beta;
  const int par = (int)(beta & 1u);
  const int n = (int)max((int64_t)0, min((int64_t)spb, d.nc - (base - d.off)));  // clones of the block
  const int L = d.L;
  const unsigned long long* const qtab = B.gq + (size_t)p * kGuideSeg;
  const int32_t* const dtab = B.gdu + (size_t)p * kGuideSeg;
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  const unsigned int lt_mask = (1u << lane) - 1u;
  // the rate sums of the clones' final configurations of the last interval, if carried:
  // a new clone starts from its ancestor's
  const bool carry = B.st[p].gcarry != 0;
  const unsigned long long* const gin = B.gcar[par ^ 1];
  unsigned long long* const gout = B.gcar[par];
  int cl = -1;  // the lane's clone (offset in the tile), -1 when it has none
  unsigned long long x[W], a[W];
  unsigned long long R = 0ull;
  int r = 0, h = 0;
  uint32_t e = 0u;
  float t = 0.0f, a_r = 0.0f, a_h = 0.0f;
  int hmin = INT_MAX, hmax = INT_MIN, xmin = INT_MAX, xmax = INT_MIN;
  unsigned int ev = 0u;
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = a[w] = 0ull;
  for (;;) {
    const unsigned int m = __ballot_sync(0xffffffffu, cl < 0);
    int taken = 0;
    if (lane == 0) taken = *(volatile int*)&s_take;
    taken = __shfl_sync(0xffffffffu, taken, 0);
    if (m != 0u && taken < n) {
      int base_i = 0;
      if (lane == 0) base_i = atomicAdd(&s_take, __popc(m));
      base_i = __shfl_sync(0xffffffffu, base_i, 0);
      const int idx = base_i + __popc(m & lt_mask);
      const bool got = cl < 0 && idx < n;
      if (got) {
        cl = idx;
        load_lat<W>(B.Y, base + idx, x);
        active_bonds<W>(x, L, a);
        r = popc_lat<W>(a);
        h = 0;
        e = 0u;
        t = a_r = a_h = 0.0f;
        if (carry) {
          const unsigned long long* src = gin + (d.off + (int64_t)B.anc[base + idx]) * ng;
          R = 0ull;
#pragma unroll
          for (int g = 0; g < ng; ++g) {
            const unsigned long long v = src[g];
            s_g[g][tid] = v;
            R += v;
          }
        }
      }
      // the rate sums of every new clone without carried ones, one clone at a time by
      // the whole warp
      unsigned int todo = __ballot_sync(0xffffffffu, got && !carry);
      while (todo != 0u) {
        const int o = __ffs(todo) - 1;
        todo &= todo - 1u;
        unsigned long long xo[W];
#pragma unroll
        for (int w = 0; w < W; ++w) xo[w] = __shfl_sync(0xffffffffu, x[w], o);
        // the lane's bonds b0 .. b0 + BPL - 1 (those below L): segments from one window
        const int b0 = lane * BPL;
        unsigned long long v = 0ull;
        if (b0 < L) {
          const int st0 = b0 >= 8 ? b0 - 8 : b0 - 8 + L;
          const unsigned long long win = ring_window<W>(xo, L, st0);
#pragma unroll
          for (int i = 0; i < BPL; ++i)
            if (b0 + i < L) v += guided_q_at(win, i, qtab);
        }
        // a group of eight bonds spans 8 / BPL lanes
#pragma unroll
        for (int off = 1; off < kGuideGroup / BPL; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane % (kGuideGroup / BPL) == 0) s_g[lane / (kGuideGroup / BPL)][(tid & ~31) + o] = v;
#pragma unroll
        for (int off = kGuideGroup / BPL; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == o) R = v;
      }
      __syncwarp();
    }
    if (__ballot_sync(0xffffffffu, cl >= 0) == 0u) {
      if (lane == 0) taken = *(volatile int*)&s_take;
      if (__shfl_sync(0xffffffffu, taken, 0) >= n) break;
      continue;
    }
    if (cl >= 0) {
      const uint32_t j = (uint32_t)(base - d.off + cl);
      const float Rf = u64_to_float_rn(R);
      const float rp = __fmul_rn(Rf, 0x1p-40f);
      const long long D = (long long)(float_to_u64_exact(Rf) - R);
      const float eta = __fdiv_rn(i64_to_float_rn(D), Rf);
      const float dr = __fsub_rn(__int2float_rn(r), rp);
      const uint4 w = philox4x32_10(make_uint4(e, beta, j, kTagGuided), k0, k1);
      const float E = neg_ln_u(w.x, s_log);
      const float tau = __fdiv_rn(E, rp);
      const float t_new = __fadd_rn(t, tau);
      bool run = r != 0;
      if (run && e >= kStepLimit) {  // guard: an interval must end; report, never spin
        B.st[p].err = kErrRange;
        run = false;
      }
      if (run && t_new >= dt_f) {
        a_r = __fmaf_rn(dr, __fsub_rn(dt_f, t), a_r);
        run = false;
      }
      if (run) {
        a_r = __fmaf_rn(dr, tau, a_r);
        t = t_new;
        const unsigned long long kk = __umul64hi(((unsigned long long)w.z << 32) | w.y, R);
        // the first bond whose inclusive cumulative rate exceeds kk < R: the group from the
        // group sums, then the bond inside it (the last group if the sums run out first)
        unsigned long long cum = 0ull;
        int g = ng - 1;
        bool found = false;
#pragma unroll
        for (int gg = 0; gg < ng - 1; ++gg) {
          const unsigned long long v = s_g[gg][tid];
          if (!found) {
            if (cum + v <= kk) cum += v;
            else { found = true; g = gg; }
          }
        }
        const int gb = g * kGuideGroup;  // < L: the group holds the bond kk falls on
        const unsigned long long gwin = ring_window<W>(x, L, gb >= 8 ? gb - 8 : gb - 8 + L);
        int b = gb + kGuideGroup - 1;
        uint32_t bseg = 0u;
        found = false;
#pragma unroll
        for (int i = 0; i < kGuideGroup; ++i) {
          const unsigned long long q = gb + i < L ? guided_q_at(gwin, i, qtab) : 0ull;
          if (!found) {
            cum += q;
            if (cum > kk) {
              found = true;
              b = gb + i;
              bseg = (uint32_t)(gwin >> i) & 0x3FFFFu;
            }
          }
        }
        const int kb = min(max(__ldg(dtab + guided_index(bseg)) - d.s_q, -kGuideKmax), kGuideKmax);
        a_h = __fadd_rn(a_h, __fsub_rn(__fsub_rn(d.c_s, __fmul_rn(__int2float_rn(kb + d.s_q), 0x1p-17f)), eta));
        // the bonds b-9 .. b+9, whose windows contain site b or b+1, change rate: their
        // segments (sites b-17 .. b+18) from one window before and one after the hop
        const int ws = b >= 17 ? b - 17 : b - 17 + L;
        const unsigned long long wo = ring_window<W>(x, L, ws);
        hop<W>(x, b, L);
        ++h;
        active_bonds<W>(x, L, a);
        r = popc_lat<W>(a);
        const unsigned long long wn = ring_window<W>(x, L, ws);
#pragma unroll
        for (int db = -9; db <= 9; ++db) {
          if (db == 9 && L <= 18) continue;  // on 18 sites bond b+9 is bond b-9
          int c = b + db;
          if (c < 0) c += L;
          if (c >= L) c -= L;
          const unsigned long long qo = guided_q_at(wo, db + 9, qtab);
          const unsigned long long qn = guided_q_at(wn, db + 9, qtab);
          if (qn != qo) {
            s_g[c / kGuideGroup][tid] += qn - qo;
            R += qn - qo;
          }
        }
      }
      ++e;
      if (!run) {
        const float X = __fsub_rn(a_h, a_r);
        const int64_t slot = base + cl;
#pragma unroll
        for (int g = 0; g < ng; ++g) gout[slot * ng + g] = s_g[g][tid];
        store_lat<W>(B.Xb[par], slot, x);
        B.KXb[par][slot] = B.KY[slot] + h;
        B.dKb[par][slot] = h;
        B.Ab[par][slot] = X;
        hmin = min(hmin, h);
        hmax = max(hmax, h);
        ev += (unsigned int)h;
        xmin = min(xmin, float_order(X));
        xmax = max(xmax, float_order(X));
        cl = -1;
      }
    }
  }
  hmin = __reduce_min_sync(0xffffffffu, hmin);
  hmax = __reduce_max_sync(0xffffffffu, hmax);
  ev = __reduce_add_sync(0xffffffffu, ev);
  xmin = __reduce_min_sync(0xffffffffu, xmin);
  xmax = __reduce_max_sync(0xffffffffu, xmax);
  if (lane == 0 && hmin != INT_MAX) {
    atomicMin(&s_min, hmin);
    atomicMax(&s_max, hmax);
    atomicAdd(&s_ev, ev);
    atomicMin(&s_amin, xmin);
    atomicMax(&s_amax, xmax);
  }
  __syncthreads();
  if (tid == 0 && s_min != INT_MAX) {
    PopState* st = B.st + p;
    atomicMin(&st->dk_min[par], s_min);
    atomicMax(&st->dk_max[par], s_max);
    atomicAdd(&st->events, (unsigned long long)s_ev);
    atomicMin(&st->a_min[par], s_amin);
    atomicMax(&st->a_max[par], s_amax);
  }
}

// ---------------------------------------------------------------------------
// Dynamical stage for rings longer than 128 sites: one warp per clone.  Lane l
// holds sites [128 l, 128 l + 128) in two words.  Active bonds are x XOR rot(x),
// where the site above a lane's top bit is bit 0 of the next lane and the site
// above L-1 is site 0.  The escape rate is a warp sum, the k-th active bond is
// found from an exclusive prefix of the lanes' counts, and the draw, the waiting
// time and the bond index are the same on every lane (the same arithmetic as the
// one-clone-per-lane kernel, so results are identical to the oracle's).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void wide_active(unsigned long long xl, unsigned long long xh, int L,
                                            int lane, unsigned long long& al,
                                            unsigned long long& ah) {
  const unsigned long long nb = __shfl_sync(0xffffffffu, xl, (lane + 1) & 31) & 1ull;
  const unsigned long long b0 = __shfl_sync(0xffffffffu, xl, 0) & 1ull;
  const int last = (L - 1) >> 7, pos = (L - 1) & 127;
  unsigned long long rl = (xl >> 1) | (xh << 63);
  unsigned long long rh = (xh >> 1) | (nb << 63);
  if (lane == last) {
    if (pos < 64) rl |= b0 << pos; else rh |= b0 << (pos - 64);
  }
  if (lane > last) { rl = 0ull; rh = 0ull; }
  al = xl ^ rl;
  ah = xh ^ rh;
}

// One BKL step of the warp's clone; returns true if it hopped (MOD: accumulate
// the rate integral as in bkl_step).
template <bool MOD>
__device__ __forceinline__ bool wide_step(unsigned long long& xl, unsigned long long& xh,
                                          float& t, float& acc, int L, int lane, const float* inv,
                                          const float2* tab, uint32_t wa, uint32_t wb,
                                          float dt_f) {
  unsigned long long al, ah;
  wide_active(xl, xh, L, lane, al, ah);
  const int cl = __popcll(al) + __popcll(ah);
  const int r = __reduce_add_sync(0xffffffffu, (unsigned int)cl);
  if (r == 0) return false;
  const float tau = __fmul_rn(neg_ln_u(wa, tab), inv[r]);
  const float t_new = __fadd_rn(t, tau);
  if (t_new >= dt_f) {
    if (MOD) acc = __fmaf_rn((float)r, __fsub_rn(dt_f, t), acc);
    return false;
  }
  if (MOD) acc = __fmaf_rn((float)r, tau, acc);
  t = t_new;
  const uint32_t k = __umulhi(wb, (uint32_t)r);
  int incl = cl;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int excl = incl - cl;
  const unsigned int owner_mask = __ballot_sync(0xffffffffu, (uint32_t)excl <= k && k < (uint32_t)incl);
  const int owner = __ffs(owner_mask) - 1;
  int bpos = 0;
  if (lane == owner) {
    const uint32_t kk = k - (uint32_t)excl;
    const uint32_t cl0 = (uint32_t)__popcll(al);
    bpos = (kk < cl0) ? kth_set_bit64(al, kk) : 64 + kth_set_bit64(ah, kk - cl0);
  }
  const int b = (owner << 7) + __shfl_sync(0xffffffffu, bpos, owner);
  const int b1 = (b + 1 == L) ? 0 : b + 1;
  if ((b >> 7) == lane) { const int q = b & 127; if (q < 64) xl ^= 1ull << q; else xh ^= 1ull << (q - 64); }
  if ((b1 >> 7) == lane) { const int q = b1 & 127; if (q < 64) xl ^= 1ull << q; else xh ^= 1ull << (q - 64); }
  return true;
}

template <bool MOD>
__global__ void __launch_bounds__(kThreads) k_evolve_wide(Batch B, float dt_f) {
  __shared__ float2 s_tab[64];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 64) s_tab[tid] = B.logtab[tid];
  __syncthreads();
  const uint32_t beta = *B.beta;
  const int par = (int)(beta & 1u);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  for (int64_t slot = (int64_t)blockIdx.x * kWarps + (tid >> 5); slot < B.nslots; slot += nwarps) {
    const int p = B.tile_pop[slot / kTile];
    const PopDesc d = B.pops[p];
    const int64_t j = slot - d.off;
    if (j >= d.nc) continue;  // padding (warp-uniform)
    const int W = B.W;
    unsigned long long xl = (2 * lane < W) ? B.Y[slot * W + 2 * lane] : 0ull;
    unsigned long long xh = (2 * lane + 1 < W) ? B.Y[slot * W + 2 * lane + 1] : 0ull;
    const float* inv = B.inv_rate + (size_t)p * kInvStride;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    float t = 0.0f, acc = 0.0f;
    int h = 0;
    for (uint32_t q = 0;; ++q) {
      if (q >= kStepLimit / 2u) {  // guard: an interval must end; report, never spin
        if (lane == 0) B.st[p].err = kErrRange;
        break;
      }
      const uint4 d4 = philox4x32_10(make_uint4(q, beta, (uint32_t)j, kTagEvolve), k0, k1);
      if (!wide_step<MOD>(xl, xh, t, acc, d.L, lane, inv, s_tab, d4.x, d4.y, dt_f)) break;
      ++h;
      if (!wide_step<MOD>(xl, xh, t, acc, d.L, lane, inv, s_tab, d4.z, d4.w, dt_f)) break;
      ++h;
    }
    if (2 * lane < W) B.Xb[par][slot * W + 2 * lane] = xl;
    if (2 * lane + 1 < W) B.Xb[par][slot * W + 2 * lane + 1] = xh;
    if (lane == 0) {
      B.KXb[par][slot] = B.KY[slot] + h;
      B.dKb[par][slot] = h;
      atomicMin(&B.st[p].dk_min[par], h);
      atomicMax(&B.st[p].dk_max[par], h);
      atomicAdd(&B.st[p].events, (unsigned long long)h);
      if (MOD) {
        B.Ab[par][slot] = acc;
        atomicMin(&B.st[p].a_min[par], __float_as_int(acc));
        atomicMax(&B.st[p].a_max[par], __float_as_int(acc));
      }
    }
  }
}

// Fourier density mode (eq. fourdens): per clone, C and S are the sums over the
// occupied sites in increasing order of float(cos), float(sin) of 2 pi n x / L
// (cs[x], from the host); |delta rho_n|^2 = (C^2 + S^2) / L in FP32; per tile the
// FP64 sum over its clones.
template <int W>
__global__ void __launch_bounds__(kThreads) k_density(Batch B, const float2* cs, double* tile_acc) {
  __shared__ double s_part[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = blockIdx.x;
  const int p = B.tile_pop[tile];
  const PopDesc d = B.pops[p];
  const float2* tab = cs + (size_t)p * kInvStride;
  const int64_t base = (int64_t)tile * kTile;
  const int nw = W > 0 ? W : B.W;
  double acc = 0.0;
  for (int i = tid; i < kTile; i += kThreads) {
    if (base - d.off + i >= d.nc) continue;
    float c = 0.0f, sn = 0.0f;
    for (int q = 0; q < nw; ++q) {
      unsigned long long bits = B.Y[(base + i) * nw + q];
      while (bits) {
        const int b = __ffsll((long long)bits) - 1;
        const float2 v = tab[64 * q + b];
        c = __fadd_rn(c, v.x);
        sn = __fadd_rn(sn, v.y);
        bits &= bits - 1ull;
      }
    }
    acc += (double)__fdiv_rn(__fadd_rn(__fmul_rn(c, c), __fmul_rn(sn, sn)), (float)d.L);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s_part[wid] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += s_part[w];
    tile_acc[tile] = t;
  }
}

// Sum of the carried activities of each population (for k_hat, eq. khat).
// Ancestry across the last cloning stage: out[off + j] = in[off + anc_j].
__global__ void __launch_bounds__(kThreads) k_lineage(Batch B, const int32_t* in, int32_t* out) {
  const int64_t slot = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const PopDesc d = B.pops[B.tile_pop[slot / kTile]];
  if (slot - d.off < d.nc) out[slot] = in[d.off + B.anc[slot]];
}

__global__ void __launch_bounds__(kThreads) k_ksum(Batch B) {
  __shared__ long long s_part[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t slot = (int64_t)blockIdx.x * kThreads + tid;
  const int p = B.tile_pop[slot / kTile];
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
