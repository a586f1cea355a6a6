/*
 * CPU oracle for the population-dynamics (cloning) estimator of psi(s) for the
 * activity of the symmetric simple exclusion process (SSEP) on a ring.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU path computes.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never does,
 * and this file shares no code, header, table or constant generator with it.
 *
 * What it follows (arXiv:1711.05095, Brewer, Clark, Bradford, Jack):
 *   - Sec. 2.3 "Cloning algorithm": N_c clones, M = t_obs/dt intervals, each a
 *     dynamical stage followed by a cloning stage; eq. (upsbdef) per-interval
 *     weight; eq. (psihat) estimator of psi.
 *   - Sec. 3.1: SSEP on a ring of L sites, N particles, every particle hops with
 *     rate 1 to each empty neighbour; the activity K counts successful hops.
 *   - Sec. 4 (first paragraph): BKL continuous-time Monte Carlo.
 *   - Sec. 4.1, eq. (alpha-Ups): [eq] clone selection with one shared d in (0,1).
 *   - Sec. 4.2, eq. (khat): the cumulative K is carried with the clone.
 *
 * The lattice is held here as one byte per site (n_i in {0,1}); the GPU path
 * uses packed bitmasks.  Conversion between the two is done by the tests.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   R1 random numbers: Philox4x32-10 (Salmon et al., SC'11) replaces the paper's
 *      Mersenne Twister.  key = 64-bit seed; counter = (c0, c1, c2, c3):
 *        init     (site t, 0,    slot j, 1)
 *        evolve   (draw q, beta, slot j, 2)   beta = 1..M, q = 0,1,... per interval
 *        resample (0,      beta, 0,      3)
 *      The slot j is the clone's position in the population, after resampling.
 *      One evolve draw serves two BKL steps: step e of the interval uses draw
 *      q = e/2, words (w0, w1) when e is even and (w2, w3) when e is odd.
 *   R2 exponential variate: u = (2*wa + 1) / 2^33 from the step's first word wa,
 *      with 2*wa+1 truncated to 24 significant bits; E = -ln(u) by the FP32
 *      logarithm defined in orc_neg_ln_u() below (ln(m 2^n) = n ln 2 + ln c +
 *      ln(1 + r) with c from a 64-entry table; no library log at run time).
 *   R3 time arithmetic in FP32: tau = E * (1/r) with 1/r rounded to float,
 *      t_new = t + tau; the interval ends when t_new >= (float)dt (no hop).
 *   R4 bond choice: k = floor(wb * r / 2^32) with wb the step's second word (a
 *      bias of at most r / 2^32 per bond); the hop is across the k-th active bond
 *      counted from bond 0; bond i joins sites i and (i+1) mod L and is active
 *      when exactly one of the two is occupied.
 *   R5 initial condition: a uniform N-subset of the L sites per clone, by
 *      selection sampling (site t taken iff floor(U64*(L-t)/2^64) < N - taken).
 *   R6 fixed-point weights: F = 61 - ceil(log2 N_c); k_ref = min dK (s >= 0) or
 *      max dK (s < 0); w = nearest-integer(2^F exp(-|s| |dK - k_ref|)), computed
 *      with FP64 exp; |dK - k_ref| >= 4096 is a range error.  The quantised
 *      weights only steer selection; the psi term uses exact FP64 (eq. psihat).
 *   R7 [eq] selection with exact integers: d = (2U+1)/2^33 with U the resample
 *      word; alpha_j = floor((2^33 j + 2U + 1) T / (2^33 N_c)) for j = 0..N_c-1;
 *      the ancestor is the 0-based k with S_k <= alpha_j < S_{k+1}, S the
 *      exclusive prefix sums of the weights (the printed index is off by one).
 *   R13 MODIFIED dynamics (Sec. 3.2, eq. def-ups-ssep): every rate times e^-s, so
 *      tau = E * float(e^s / r); the weight exponent A = integral of the unmodified
 *      escape rate r over the interval, accumulated in FP32 as A <- fma(r, tau, A)
 *      per hop and A <- fma(r, dt - t, A) for the last segment.  Upsilon =
 *      exp(-c A) with c = float(1 - e^-s).  A_ref = min A (s >= 0) or max A (s < 0);
 *      w = floor(2^F exp_spec(-c (A - A_ref))) with exp_spec the FP32 exponential
 *      of orc_weight_exp() below; the psi term is -c A_ref + log1p((T - N_c 2^F)/(N_c 2^F))
 *      from the exact integer total T of those weights.
 *   R14 [iid] selection (Sec. 4.1): alpha_j = floor(U64_j T / 2^64), U64_j = w1 2^32 + w0
 *      of draw (j, beta, 0, 4); the ancestor is the k with S_k <= alpha_j < S_{k+1}.
 *   R15 GUIDED dynamics (Sec. 2.2, eqs. modpdef and upsdef, with a local potential
 *      in place of the uniform e^-s of Sec. 3.2).  U(C) = sum_i phi(window_i), window_i
 *      the 9 sites i-4..i+4 (mod L) read as a 9-bit number (bit k = site i-4+k);
 *      phi is given as 512 floats and used as fixed point phi_q = nearest(phi 2^16)
 *      (|phi| <= 64), so every sum of U is an exact integer.  Requires 10 <= L.
 *      Rate of the hop across active bond b, ~ e^-s e^{dU_b/2}, with an exactly known
 *      logarithm:
 *        dU_b = U(C^b) - U(C) = sum_{m=0..9} phi_q(seg' >> m & 511) - phi_q(seg >> m & 511),
 *        seg = the 18 sites b-8..b+9 (bit k = site b-8+k), seg' = seg with bits 8, 9 flipped;
 *        exponent k_b = clamp(dU_b - s_q, -2^20, 2^20) in units of 2^-17, s_q = nearest(s 2^17)
 *        (dU_b in units of 2^-16 is dU/2 in units of 2^-17);
 *        Q_b = floor(TA[a] TB[c] / 2^44), k_b + 2^20 = 2^11 a + c, with the tables
 *        TA[a] = nearest(2^44 exp(a/64 - 8)), TB[c] = nearest(2^40 exp(c/2^17)) (FP64 exp),
 *      so Q_b = 2^40 exp(k_b 2^-17) (1 + d), |d| < 3e-9.  R' = sum_b Q_b (64-bit, exact).
 *      Step e of the interval uses draw (e, beta, j, 5): E = -ln u(w0) as in R2;
 *      r'_f = float(R') 2^-40 (one rounding); tau = E / r'_f; t_new >= dt ends the
 *      interval; otherwise the hop is across the first active bond (increasing b) whose
 *      inclusive cumulative Q exceeds floor((w2 2^32 + w1) R' / 2^64).
 *      Weight (eq. upsdef with the P-hat of the simulated process: waiting rate r'_f,
 *      bond b with probability Q_b / R', i.e. hop rate 2^-40 Q_b (1 + eta), eta =
 *      (2^40 r'_f - R') / R' from the rounding of r'_f, computed from exact integers):
 *        ln Upsilon = sum_hops (-s - ln(2^-40 Q_b) - eta) - integral (r - r'_f) dt,
 *      with ln(2^-40 Q_b) taken as k_b 2^-17 (the table error d is below 3e-9) and
 *      -s = -s_q 2^-17 + c_s, c_s = float(s_q 2^-17 - s) (|c_s| <= 2^-18), in FP32:
 *        per hop      a_h <- a_h + ((c_s - float(k_b + s_q) 2^-17) - eta),
 *        per segment  a_r <- fma(float(r) - r'_f, tau, a_r)  (last: dt - t in place of tau);
 *      X = a_h - a_r.  Each term is computed from quantities of its own size, so no
 *      rounding is repeated hop after hop into a systematic shift of psi; since the
 *      weight is that of the rates simulated, the estimate is unbiased for any potential.
 *      Selection weights w = floor(2^F exp_spec(X - X_ref)), X_ref = max X; psi term
 *      X_ref + log1p((T - N_c 2^F)/(N_c 2^F)).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (see oracle/build.py).
 * Contraction must stay off: every float operation below is a separately rounded
 * IEEE-754 operation, or an explicit fmaf().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_INIT 1u
#define ORC_TAG_EVOLVE 2u
#define ORC_TAG_RESAMPLE 3u
#define ORC_TAG_IID 4u
#define ORC_KCAP 4096

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_RANGE -3

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of the Philox S-box with the two published
 * round multipliers, the key advanced by the two Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
  uint32_t k1 = (uint32_t)(seed >> 32);
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_at(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint64_t seed, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  orc_philox(ctr, seed, out);
}

/* floor(a * b / 2^64) for 64-bit a, b */
static uint64_t mul_hi_64(uint64_t a, uint64_t b) {
  return (uint64_t)(((u128)a * (u128)b) >> 64);
}

/* ---------------------------------------------------------------------------
 * Reading R2: E = -ln(u), u = (2w+1)/2^33, in FP32.
 * v = 2w+1 (33 bits, odd) is truncated to its 24 leading bits: v' = t 2^(p-23)
 * with t in [2^23, 2^24) and p the position of the leading one, so
 * v' = m 2^p with m = t / 2^23 in [1, 2) (exact in float).  Then
 *   ln u' = (p - 33) ln 2 + ln m,
 *   ln m = ln c_i + ln(1 + r),   c_i = 1 + (i + 1/2)/64,  i = top 6 fraction bits of m,
 *   r = m / c_i - 1 (|r| <= 1/128),  ln(1 + r) ~ r (1 - r/2 + r^2/3)
 * (the first dropped term is below 1e-9).  The table holds float(1/c_i) and
 * float(ln c_i), each rounded once from FP64.  ln 2 is split into a 15-bit head
 * (exact products with the small integer 33 - p) and a float tail.
 * ------------------------------------------------------------------------- */
static const float ORC_LN2_HI = 0x1.62e4p-1f;
static const float ORC_LN2_LO = 0x1.7f7d1cp-20f;
static const float ORC_THIRD = 0x1.555556p-2f; /* 1/3 */

static float orc_tab_inv_c[64];
static float orc_tab_ln_c[64];
static int orc_tab_ready = 0;

static void orc_log_table(void) {
  for (int i = 0; i < 64; ++i) {
    double c = 1.0 + ((double)i + 0.5) / 64.0;
    orc_tab_inv_c[i] = (float)(1.0 / c);
    orc_tab_ln_c[i] = (float)log(c);
  }
  orc_tab_ready = 1;
}

float orc_neg_ln_u(uint32_t w) {
  if (!orc_tab_ready) orc_log_table();
  uint64_t v = 2u * (uint64_t)w + 1u;
  int p = 0;
  while ((v >> (p + 1)) != 0u) ++p;
  uint32_t t = (p >= 23) ? (uint32_t)(v >> (p - 23)) : (uint32_t)(v << (23 - p));
  uint32_t mbits = 0x3f800000u | (t & 0x007fffffu);
  float m;
  memcpy(&m, &mbits, sizeof m);
  int i = (int)((t >> 17) & 63u);
  float r = fmaf(m, orc_tab_inv_c[i], -1.0f);
  float q = fmaf(r, ORC_THIRD, -0.5f);
  q = fmaf(q, r, 1.0f);
  float ln_m = orc_tab_ln_c[i] + q * r;
  float n = (float)(33 - p);
  float E = fmaf(n, ORC_LN2_LO, -ln_m);
  E = fmaf(n, ORC_LN2_HI, E);
  return E;
}

/* ---------------------------------------------------------------------------
 * Reading R5: initial configurations, independent uniform N-subsets per clone
 * (steady state of the SSEP at fixed N: Sec. 2.1 takes the initial condition from
 * the steady state; Sec. 3.1 says that state is uniform).
 * sites: n_clones * L bytes, clone-major.  K is set to zero.
 * ------------------------------------------------------------------------- */
int orc_init(int32_t L, int32_t N, int64_t n_clones, uint64_t seed,
             uint8_t* sites, int32_t* K) {
  if (L < 3 || N < 0 || N > L || n_clones < 1) return ORC_ERR_ARG;
  for (int64_t j = 0; j < n_clones; ++j) {
    uint8_t* n = sites + j * (int64_t)L;
    int taken = 0;
    for (int t = 0; t < L; ++t) {
      n[t] = 0;
      int need = N - taken;
      if (need <= 0) continue;
      uint32_t r[4];
      philox_at((uint32_t)t, 0u, (uint32_t)j, ORC_TAG_INIT, seed, r);
      uint64_t u = ((uint64_t)r[1] << 32) | r[0];
      if (mul_hi_64(u, (uint64_t)(L - t)) < (uint64_t)need) {
        n[t] = 1;
        ++taken;
      }
    }
    K[j] = 0;
  }
  return ORC_OK;
}

/* number of active bonds: bond i joins sites i and (i+1) mod L */
static int count_active(const uint8_t* n, int L) {
  int r = 0;
  for (int i = 0; i < L; ++i) r += (n[i] != n[(i + 1) % L]);
  return r;
}

/* ---------------------------------------------------------------------------
 * Dynamical stage of interval beta for every clone (Sec. 2.3; Sec. 3.1 rates;
 * Sec. 4 BKL): plain SSEP rates (1 per active bond), so the escape rate is the
 * number of active bonds r.  Readings R2-R4 fix the arithmetic.
 * On return sites hold the configurations at the end of the interval, K the
 * cumulative activity and dK the activity K^beta of this interval.
 * ------------------------------------------------------------------------- */
int orc_evolve(int32_t L, int64_t n_clones, double dt, uint32_t beta, uint64_t seed,
               uint8_t* sites, int32_t* K, int32_t* dK) {
  if (L < 3 || n_clones < 1 || !(dt > 0.0)) return ORC_ERR_ARG;
  const float dt_f = (float)dt;
  for (int64_t j = 0; j < n_clones; ++j) {
    uint8_t* n = sites + j * (int64_t)L;
    float t = 0.0f;
    uint32_t e = 0;
    int32_t hops = 0;
    for (;;) {
      int r = count_active(n, L);
      if (r == 0) break;
      uint32_t w[4];
      philox_at(e / 2u, beta, (uint32_t)j, ORC_TAG_EVOLVE, seed, w);
      uint32_t wa = (e % 2u == 0u) ? w[0] : w[2];
      uint32_t wb = (e % 2u == 0u) ? w[1] : w[3];
      ++e;
      float E = orc_neg_ln_u(wa);
      float inv_r = 1.0f / (float)r;
      float tau = E * inv_r;
      float t_new = t + tau;
      if (t_new >= dt_f) break;
      t = t_new;
      uint64_t k = ((uint64_t)wb * (uint64_t)r) >> 32;
      /* the k-th active bond, counting from bond 0 */
      int b = -1;
      uint64_t seen = 0;
      for (int i = 0; i < L; ++i) {
        if (n[i] != n[(i + 1) % L]) {
          if (seen == k) { b = i; break; }
          ++seen;
        }
      }
      int b1 = (b + 1) % L;
      uint8_t tmp = n[b];
      n[b] = n[b1];
      n[b1] = tmp;
      ++hops;
    }
    dK[j] = hops;
    K[j] += hops;
  }
  return ORC_OK;
}

static int ceil_log2_i64(int64_t x) {
  int c = 0;
  while (((int64_t)1 << c) < x) ++c;
  return c;
}

/* Reading R6: the fixed-point weight scale F and the reference activity. */
int32_t orc_weight_scale(int64_t n_clones) { return 61 - ceil_log2_i64(n_clones); }

int32_t orc_k_ref(double s, int64_t n_clones, const int32_t* dK) {
  int32_t ref = dK[0];
  for (int64_t j = 1; j < n_clones; ++j) {
    if (s >= 0.0) { if (dK[j] < ref) ref = dK[j]; }
    else          { if (dK[j] > ref) ref = dK[j]; }
  }
  return ref;
}

/* ---------------------------------------------------------------------------
 * Weights Upsilon^beta = exp(-s K^beta) (eq. upsbdef with U = 0), quantised per
 * reading R6: Upsilon_j / Upsilon_max = exp(-|s| |dK_j - k_ref|).
 * ------------------------------------------------------------------------- */
int orc_weights(double s, int64_t n_clones, const int32_t* dK, uint64_t* w) {
  if (n_clones < 1) return ORC_ERR_ARG;
  const int F = orc_weight_scale(n_clones);
  const int32_t ref = orc_k_ref(s, n_clones, dK);
  int status = ORC_OK;
  for (int64_t j = 0; j < n_clones; ++j) {
    int64_t k = (int64_t)dK[j] - ref;
    if (k < 0) k = -k;
    if (k >= ORC_KCAP) { w[j] = 0; status = ORC_ERR_RANGE; continue; }
    double x = ldexp(exp(-fabs(s) * (double)k), F);
    w[j] = (uint64_t)nearbyint(x);
  }
  return status;
}

/* Compensated (Neumaier) summation: sum and running correction. */
typedef struct { double sum, comp; } orc_ksum;
static void ksum_add(orc_ksum* a, double x) {
  double t = a->sum + x;
  if (fabs(a->sum) >= fabs(x)) a->comp += (a->sum - t) + x;
  else a->comp += (x - t) + a->sum;
  a->sum = t;
}

/* ---------------------------------------------------------------------------
 * One term of eq. (psihat): ln( (1/N_c) sum_j exp(-s dK_j) ), in FP64.
 * Factoring out exp(-s k_ref), with q_j = exp(-|s| |dK_j - k_ref|) in (0, 1]:
 *   term = -s k_ref + ln( mean_j q_j ).
 * When mean q is near 1 the logarithm is taken as log1p(mean_j expm1(.)), which is
 * the same number without the cancellation of ln(1 + small).
 * ------------------------------------------------------------------------- */
double orc_psi_term(double s, int64_t n_clones, const int32_t* dK) {
  const int32_t ref = orc_k_ref(s, n_clones, dK);
  orc_ksum a = {0.0, 0.0}, b = {0.0, 0.0};
  for (int64_t j = 0; j < n_clones; ++j) {
    int64_t k = (int64_t)dK[j] - ref;
    if (k < 0) k = -k;
    double x = -fabs(s) * (double)k;
    ksum_add(&a, expm1(x));
    ksum_add(&b, exp(x));
  }
  double mean_q = (b.sum + b.comp) / (double)n_clones;
  double ln_mean = (mean_q > 0.5) ? log1p((a.sum + a.comp) / (double)n_clones) : log(mean_q);
  return -s * (double)ref + ln_mean;
}

/* The [eq] offset word U of interval beta (reading R7). */
uint32_t orc_resample_word(uint32_t beta, uint64_t seed) {
  uint32_t r[4];
  philox_at(0u, beta, 0u, ORC_TAG_RESAMPLE, seed, r);
  return r[0];
}

/* ---------------------------------------------------------------------------
 * [eq] clone selection, eq. (alpha-Ups) with reading R7, in exact integers.
 * anc[j] = 0-based index of the old clone that new clone j is pulled from.
 * Returns ORC_ERR_ARG if every weight is zero.
 * ------------------------------------------------------------------------- */
int orc_ancestors(int64_t n_clones, const uint64_t* w, uint32_t beta, uint64_t seed,
                  int32_t* anc) {
  if (n_clones < 1) return ORC_ERR_ARG;
  uint64_t* S = (uint64_t*)malloc((size_t)(n_clones + 1) * sizeof(uint64_t));
  if (!S) return ORC_ERR_ARG;
  S[0] = 0;
  for (int64_t k = 0; k < n_clones; ++k) S[k + 1] = S[k] + w[k];
  const uint64_t T = S[n_clones];
  if (T == 0) { free(S); return ORC_ERR_ARG; }
  const uint64_t U = orc_resample_word(beta, seed);
  const u128 c = 2 * (u128)U + 1;
  const u128 denom = ((u128)n_clones) << 33;
  for (int64_t j = 0; j < n_clones; ++j) {
    u128 num = ((((u128)j) << 33) + c) * (u128)T;
    uint64_t alpha = (uint64_t)(num / denom);
    /* largest k in [0, N_c) with S_k <= alpha; then alpha < S_{k+1} */
    int64_t lo = 0, hi = n_clones - 1;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo + 1) / 2;
      if (S[mid] <= alpha) lo = mid; else hi = mid - 1;
    }
    anc[j] = (int32_t)lo;
  }
  free(S);
  return ORC_OK;
}

/* Pull copy of the population (Sec. 6.1: new and old populations are separate). */
void orc_gather(int32_t L, int64_t n_clones, const int32_t* anc,
                const uint8_t* sites_old, const int32_t* K_old,
                uint8_t* sites_new, int32_t* K_new) {
  for (int64_t j = 0; j < n_clones; ++j) {
    memcpy(sites_new + j * (int64_t)L, sites_old + (int64_t)anc[j] * L, (size_t)L);
    K_new[j] = K_old[anc[j]];
  }
}

/* ---------------------------------------------------------------------------
 * Reading R13: the MODIFIED dynamics of Sec. 3.2 for one interval.  Same streams
 * and steps as orc_evolve; the waiting time uses the rate e^-s r, and A (the
 * integral of the unmodified escape rate over the interval) is returned per clone.
 * ------------------------------------------------------------------------- */
int orc_evolve_modified(int32_t L, int64_t n_clones, double dt, double s, uint32_t beta,
                        uint64_t seed, uint8_t* sites, int32_t* K, int32_t* dK, float* A) {
  if (L < 3 || n_clones < 1 || !(dt > 0.0)) return ORC_ERR_ARG;
  const float dt_f = (float)dt;
  const double es = exp(s);
  for (int64_t j = 0; j < n_clones; ++j) {
    uint8_t* n = sites + j * (int64_t)L;
    float t = 0.0f, a = 0.0f;
    uint32_t e = 0;
    int32_t hops = 0;
    for (;;) {
      int r = count_active(n, L);
      if (r == 0) break;
      uint32_t w[4];
      philox_at(e / 2u, beta, (uint32_t)j, ORC_TAG_EVOLVE, seed, w);
      uint32_t wa = (e % 2u == 0u) ? w[0] : w[2];
      uint32_t wb = (e % 2u == 0u) ? w[1] : w[3];
      ++e;
      float E = orc_neg_ln_u(wa);
      float inv_r = (float)(es / (double)r);
      float tau = E * inv_r;
      float t_new = t + tau;
      if (t_new >= dt_f) {
        a = fmaf((float)r, dt_f - t, a);
        break;
      }
      a = fmaf((float)r, tau, a);
      t = t_new;
      uint64_t k = ((uint64_t)wb * (uint64_t)r) >> 32;
      int b = -1;
      uint64_t seen = 0;
      for (int i = 0; i < L; ++i) {
        if (n[i] != n[(i + 1) % L]) {
          if (seen == k) { b = i; break; }
          ++seen;
        }
      }
      int b1 = (b + 1) % L;
      uint8_t tmp = n[b];
      n[b] = n[b1];
      n[b1] = tmp;
      ++hops;
    }
    dK[j] = hops;
    K[j] += hops;
    A[j] = a;
  }
  return ORC_OK;
}

/* 2^(i/64) for i = 0..63, rounded once from FP64 (reading R13). */
static float orc_tab_exp2[64];
static int orc_exp_ready = 0;
static void orc_exp_table(void) {
  for (int i = 0; i < 64; ++i) orc_tab_exp2[i] = (float)exp2((double)i / 64.0);
  orc_exp_ready = 1;
}

static const float ORC_64_LOG2E = 0x1.715476p+6f;   /* 64 / ln 2 */
static const float ORC_LN2_64_HI = 0x1.62p-7f;      /* ln2/64, 9-bit head */
static const float ORC_LN2_64_LO = 0x1.c85fe0p-16f; /* ln2/64 - head */
static const float ORC_SIXTH = 0x1.555556p-3f;      /* 1/6 */

/* floor(2^F exp(x)) for x <= 0 (reading R13).  x = (k/64) ln 2 + r with
 * k = floor(64 x / ln 2) and r = x - k ln2/64 formed exactly in two fma steps
 * (k ln2/64 split into a 9-bit head, exact for |k| < 2^15, and a float tail);
 * exp(x) = 2^n 2^(i/64) e^r with k = 64 n + i, 2^(i/64) from the table and
 * e^r ~ 1 + r (1 + r (1/2 + r/6)) for 0 <= r < ln2/64 (first dropped term below
 * 6e-10).  y = 2^(i/64) e^r is a float in [1, 2.02); the weight is its 24-bit
 * mantissa shifted by (exponent of y) + n + F - 23. */
uint64_t orc_weight_exp(float x, int F) {
  if (!orc_exp_ready) orc_exp_table();
  if (!(x >= -87.0f)) return 0;
  int k = (int)floorf(x * ORC_64_LOG2E);
  float r = fmaf(-(float)k, ORC_LN2_64_HI, x);
  r = fmaf(-(float)k, ORC_LN2_64_LO, r);
  float q = fmaf(r, ORC_SIXTH, 0.5f);
  q = fmaf(q, r, 1.0f);
  q = fmaf(q, r, 1.0f);
  int i = ((k % 64) + 64) % 64;
  int n = (k - i) / 64;
  float y = orc_tab_exp2[i] * q;
  uint32_t bits;
  memcpy(&bits, &y, sizeof bits);
  int ey = (int)((bits >> 23) & 0xffu) - 127;
  uint64_t mant = (uint64_t)((bits & 0x007fffffu) | 0x00800000u);
  int sa = ey + n + F - 23;
  if (sa >= 0) return mant << sa;
  if (sa <= -64) return 0;
  return mant >> (-sa);
}

float orc_a_ref(double s, int64_t n_clones, const float* A) {
  float ref = A[0];
  for (int64_t j = 1; j < n_clones; ++j) {
    if (s >= 0.0) { if (A[j] < ref) ref = A[j]; }
    else          { if (A[j] > ref) ref = A[j]; }
  }
  return ref;
}

int orc_weights_modified(double s, int64_t n_clones, const float* A, uint64_t* w) {
  if (n_clones < 1) return ORC_ERR_ARG;
  const int F = orc_weight_scale(n_clones);
  const float c = (float)(-expm1(-s));
  const float ref = orc_a_ref(s, n_clones, A);
  for (int64_t j = 0; j < n_clones; ++j) {
    float x = (-c) * (A[j] - ref);
    w[j] = orc_weight_exp(x, F);
  }
  return ORC_OK;
}

/* psi term of reading R13 from the exact total T of the quantised weights. */
double orc_psi_term_modified(double s, int64_t n_clones, const float* A) {
  const int F = orc_weight_scale(n_clones);
  const float c = (float)(-expm1(-s));
  const float ref = orc_a_ref(s, n_clones, A);
  uint64_t T = 0;
  for (int64_t j = 0; j < n_clones; ++j) T += orc_weight_exp((-c) * (A[j] - ref), F);
  const double base = ldexp((double)n_clones, F);
  const int64_t D = (int64_t)T - (int64_t)(((uint64_t)n_clones) << F);
  return -(double)c * (double)ref + log1p((double)D / base);
}

/* ---------------------------------------------------------------------------
 * Reading R15: GUIDED dynamics with a local potential (see the header).
 * ------------------------------------------------------------------------- */
#define ORC_TAG_GUIDED 5u
#define ORC_GUIDE_KMAX (1 << 20) /* exponent clamp, units of 2^-17: |ln rate + s| <= 8 */

/* phi (512 floats, |phi| <= 64) to the fixed point used by every U sum. */
int orc_phi_fixed(const float* phi, int32_t* phi_q) {
  for (int i = 0; i < 512; ++i) {
    if (!(fabsf(phi[i]) <= 64.0f)) return ORC_ERR_ARG;
    phi_q[i] = (int32_t)nearbyint(ldexp((double)phi[i], 16));
  }
  return ORC_OK;
}

/* U(C) = sum_i phi_q(window_i) as an exact integer. */
int64_t orc_potential(int32_t L, const uint8_t* n, const int32_t* phi_q) {
  int64_t U = 0;
  for (int i = 0; i < L; ++i) {
    int pat = 0;
    for (int k = 0; k < 9; ++k) pat |= (int)n[((i - 4 + k) % L + L) % L] << k;
    U += phi_q[pat];
  }
  return U;
}

/* The exponential tables of reading R15. */
static uint64_t orc_ta[1025], orc_tb[2048];
static int orc_guide_ready = 0;
static void orc_guide_tables(void) {
  for (int a = 0; a <= 1024; ++a) orc_ta[a] = (uint64_t)nearbyint(ldexp(exp(a / 64.0 - 8.0), 44));
  for (int c = 0; c < 2048; ++c) orc_tb[c] = (uint64_t)nearbyint(ldexp(exp(c / 131072.0), 40));
  orc_guide_ready = 1;
}

/* Q(k) = floor(TA[a] TB[c] / 2^44) = 2^40 exp(k 2^-17) (1 + d), for |k| <= 2^20. */
uint64_t orc_guided_q(int32_t k) {
  if (!orc_guide_ready) orc_guide_tables();
  const uint32_t u = (uint32_t)(k + ORC_GUIDE_KMAX);
  return (uint64_t)(((u128)orc_ta[u >> 11] * (u128)orc_tb[u & 2047u]) >> 44);
}

int32_t orc_s_q(double s) { return (int32_t)nearbyint(ldexp(s, 17)); }

static int32_t clamp_k(int64_t k) {
  if (k > ORC_GUIDE_KMAX) return ORC_GUIDE_KMAX;
  if (k < -ORC_GUIDE_KMAX) return -ORC_GUIDE_KMAX;
  return (int32_t)k;
}

/* Rate exponent k_b of the hop across active bond b under the LUT potential. */
int32_t orc_guided_k(int32_t L, const uint8_t* n, int b, const int32_t* phi_q, int32_t s_q) {
  uint32_t seg = 0;
  for (int k = 0; k < 18; ++k) seg |= (uint32_t)n[((b - 8 + k) % L + L) % L] << k;
  uint32_t seg2 = seg ^ (3u << 8);
  int32_t dU = 0;
  for (int m = 0; m < 10; ++m) dU += phi_q[(seg2 >> m) & 511u] - phi_q[(seg >> m) & 511u];
  return clamp_k((int64_t)dU - s_q);
}

/* A rate-exponent function for the guided step: the LUT potential above, or (for
 * pins only) an arbitrary potential given as a table over all 2^L configurations. */
typedef int32_t (*orc_rate_fn)(int32_t L, const uint8_t* n, int b, const void* ctx, int32_t s_q);

static int32_t rate_lut(int32_t L, const uint8_t* n, int b, const void* ctx, int32_t s_q) {
  return orc_guided_k(L, n, b, (const int32_t*)ctx, s_q);
}

/* Potential table over configurations (bit i of the index = site i): k_b =
 * nearest(dU / 2 2^17) - s_q, clamped. */
static int32_t rate_table(int32_t L, const uint8_t* n, int b, const void* ctx, int32_t s_q) {
  const double* U = (const double*)ctx;
  uint64_t c = 0;
  for (int i = 0; i < L; ++i) c |= (uint64_t)n[i] << i;
  int b1 = (b + 1) % L;
  uint64_t c2 = c ^ ((1ull << b) | (1ull << b1));
  return clamp_k((int64_t)nearbyint(ldexp((U[c2] - U[c]) / 2.0, 17)) - s_q);
}

static int guided_evolve(int32_t L, int64_t n_clones, double dt, double s, uint32_t beta,
                         uint64_t seed, orc_rate_fn rate, const void* ctx, uint8_t* sites,
                         int32_t* K, int32_t* dK, float* X) {
  if (L < 10 || n_clones < 1 || !(dt > 0.0)) return ORC_ERR_ARG;
  const float dt_f = (float)dt;
  const int32_t s_q = orc_s_q(s);
  const float c_s = (float)(ldexp((double)s_q, -17) - s);
  int32_t* kb = (int32_t*)malloc((size_t)L * sizeof(int32_t));
  uint64_t* q = (uint64_t*)malloc((size_t)L * sizeof(uint64_t));
  if (!kb || !q) { free(kb); free(q); return ORC_ERR_ARG; }
  for (int64_t j = 0; j < n_clones; ++j) {
    uint8_t* n = sites + j * (int64_t)L;
    float t = 0.0f, a_r = 0.0f, a_h = 0.0f;
    int32_t hops = 0;
    for (uint32_t e = 0;; ++e) {
      /* rates of every active bond of the current configuration */
      int r = 0;
      uint64_t R = 0;
      for (int b = 0; b < L; ++b) {
        if (n[b] != n[(b + 1) % L]) {
          kb[b] = rate(L, n, b, ctx, s_q);
          q[b] = orc_guided_q(kb[b]);
          R += q[b];
          ++r;
        } else {
          q[b] = 0;
        }
      }
      if (r == 0) break;
      const float Rf = (float)R;               /* one rounding */
      const float rp = ldexpf(Rf, -40);
      const int64_t D = (int64_t)((uint64_t)Rf - R);
      const float eta = (float)D / Rf;
      const float d = (float)r - rp;
      uint32_t w[4];
      philox_at(e, beta, (uint32_t)j, ORC_TAG_GUIDED, seed, w);
      const float E = orc_neg_ln_u(w[0]);
      const float tau = E / rp;
      const float t_new = t + tau;
      if (t_new >= dt_f) {
        a_r = fmaf(d, dt_f - t, a_r);
        break;
      }
      a_r = fmaf(d, tau, a_r);
      t = t_new;
      const uint64_t kk = mul_hi_64(((uint64_t)w[2] << 32) | w[1], R);
      uint64_t cum = 0;
      int b = -1;
      for (int i = 0; i < L; ++i) {
        cum += q[i];
        if (q[i] != 0 && cum > kk) { b = i; break; }
      }
      a_h = a_h + ((c_s - ldexpf((float)(kb[b] + s_q), -17)) - eta);
      const int b1 = (b + 1) % L;
      const uint8_t tmp = n[b];
      n[b] = n[b1];
      n[b1] = tmp;
      ++hops;
    }
    dK[j] = hops;
    K[j] += hops;
    X[j] = a_h - a_r;
  }
  free(kb);
  free(q);
  return ORC_OK;
}

/* Dynamical stage of one interval under the LUT potential (reading R15).
 * X receives each clone's log weight ln Upsilon for the interval. */
int orc_evolve_guided(int32_t L, int64_t n_clones, double dt, double s, uint32_t beta,
                      uint64_t seed, const int32_t* phi_q, uint8_t* sites, int32_t* K,
                      int32_t* dK, float* X) {
  return guided_evolve(L, n_clones, dt, s, beta, seed, rate_lut, phi_q, sites, K, dK, X);
}

/* The same with a potential table over all 2^L configurations (L <= 20); test pins only. */
int orc_evolve_guided_table(int32_t L, int64_t n_clones, double dt, double s, uint32_t beta,
                            uint64_t seed, const double* U, uint8_t* sites, int32_t* K,
                            int32_t* dK, float* X) {
  if (L > 20) return ORC_ERR_ARG;
  return guided_evolve(L, n_clones, dt, s, beta, seed, rate_table, U, sites, K, dK, X);
}

float orc_x_ref(int64_t n_clones, const float* X) {
  float ref = X[0];
  for (int64_t j = 1; j < n_clones; ++j) if (X[j] > ref) ref = X[j];
  return ref;
}

int orc_weights_guided(int64_t n_clones, const float* X, uint64_t* w) {
  if (n_clones < 1) return ORC_ERR_ARG;
  const int F = orc_weight_scale(n_clones);
  const float ref = orc_x_ref(n_clones, X);
  for (int64_t j = 0; j < n_clones; ++j) w[j] = orc_weight_exp(X[j] - ref, F);
  return ORC_OK;
}

double orc_psi_term_guided(int64_t n_clones, const float* X) {
  const int F = orc_weight_scale(n_clones);
  const float ref = orc_x_ref(n_clones, X);
  uint64_t T = 0;
  for (int64_t j = 0; j < n_clones; ++j) T += orc_weight_exp(X[j] - ref, F);
  const double base = ldexp((double)n_clones, F);
  const int64_t D = (int64_t)T - (int64_t)(((uint64_t)n_clones) << F);
  return (double)ref + log1p((double)D / base);
}

/* Reading R14: [iid] clone selection. */
int orc_ancestors_iid(int64_t n_clones, const uint64_t* w, uint32_t beta, uint64_t seed,
                      int32_t* anc) {
  if (n_clones < 1) return ORC_ERR_ARG;
  uint64_t* S = (uint64_t*)malloc((size_t)(n_clones + 1) * sizeof(uint64_t));
  if (!S) return ORC_ERR_ARG;
  S[0] = 0;
  for (int64_t k = 0; k < n_clones; ++k) S[k + 1] = S[k] + w[k];
  const uint64_t T = S[n_clones];
  if (T == 0) { free(S); return ORC_ERR_ARG; }
  for (int64_t j = 0; j < n_clones; ++j) {
    uint32_t r[4];
    philox_at((uint32_t)j, beta, 0u, ORC_TAG_IID, seed, r);
    uint64_t u = ((uint64_t)r[1] << 32) | r[0];
    uint64_t alpha = mul_hi_64(u, T);
    int64_t lo = 0, hi = n_clones - 1;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo + 1) / 2;
      if (S[mid] <= alpha) lo = mid; else hi = mid - 1;
    }
    anc[j] = (int32_t)lo;
  }
  free(S);
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Fourier density mode, eq. (fourdens): delta rho_n = L^-1/2 sum_j e^{-2 pi i n X_j / L}
 * over the occupied sites X_j.  Reading: per clone in FP32, |delta rho_n|^2 =
 * (C^2 + S^2) / L with C, S the sums (in increasing site order) of
 * float(cos(2 pi n x / L)) and float(sin(2 pi n x / L)) rounded once from FP64;
 * the population mean is taken in FP64.
 * ------------------------------------------------------------------------- */
double orc_density_mode(int32_t L, int64_t n_clones, const uint8_t* sites, int32_t n) {
  float* ct = (float*)malloc((size_t)L * sizeof(float));
  float* st = (float*)malloc((size_t)L * sizeof(float));
  if (!ct || !st) { free(ct); free(st); return -1.0; }
  const double two_pi = 6.283185307179586476925286766559;
  for (int x = 0; x < L; ++x) {
    double th = two_pi * (double)((int64_t)n * x % L) / (double)L;
    ct[x] = (float)cos(th);
    st[x] = (float)sin(th);
  }
  double acc = 0.0;
  for (int64_t j = 0; j < n_clones; ++j) {
    const uint8_t* occ = sites + j * (int64_t)L;
    float c = 0.0f, s = 0.0f;
    for (int x = 0; x < L; ++x) {
      if (occ[x]) { c = c + ct[x]; s = s + st[x]; }
    }
    float v = (c * c + s * s) / (float)L;
    acc += (double)v;
  }
  free(ct); free(st);
  return acc / (double)n_clones;
}

/* ---------------------------------------------------------------------------
 * A full run of the cloning algorithm (Sec. 2.3): init, then M intervals of
 * (dynamical stage, cloning stage).  psi_hat = (1/t_obs) sum_beta term_beta
 * (eq. psihat, all M intervals); k_hat = (1/(N_c L t_obs)) sum_j K_j over the
 * final population (eq. khat with the 1/N_c of eq. avedef).
 * events (optional) receives the number of hops executed by all clones.
 * If sites_out / K_out are given, the final population is written there.
 * ------------------------------------------------------------------------- */
int orc_run_ex(int32_t L, int32_t N, int64_t n_clones, uint64_t seed, double s, double dt,
               int64_t M, int32_t modified, int32_t iid, double* psi_hat, double* k_hat,
               uint64_t* events, uint8_t* sites_out, int32_t* K_out) {
  if (L < 3 || N < 0 || N > L || n_clones < 1 || !(dt > 0.0) || M < 1) return ORC_ERR_ARG;
  size_t nbytes = (size_t)n_clones * (size_t)L;
  uint8_t* a = (uint8_t*)malloc(nbytes);
  uint8_t* b = (uint8_t*)malloc(nbytes);
  int32_t* Ka = (int32_t*)malloc((size_t)n_clones * sizeof(int32_t));
  int32_t* Kb = (int32_t*)malloc((size_t)n_clones * sizeof(int32_t));
  int32_t* dK = (int32_t*)malloc((size_t)n_clones * sizeof(int32_t));
  uint64_t* w = (uint64_t*)malloc((size_t)n_clones * sizeof(uint64_t));
  int32_t* anc = (int32_t*)malloc((size_t)n_clones * sizeof(int32_t));
  float* A = (float*)malloc((size_t)n_clones * sizeof(float));
  int status = ORC_OK;
  if (!a || !b || !Ka || !Kb || !dK || !w || !anc || !A) { status = ORC_ERR_ARG; goto done; }
  orc_init(L, N, n_clones, seed, a, Ka);
  double acc = 0.0;
  uint64_t ev = 0;
  for (int64_t beta = 1; beta <= M; ++beta) {
    int st;
    if (modified) {
      orc_evolve_modified(L, n_clones, dt, s, (uint32_t)beta, seed, a, Ka, dK, A);
      acc += orc_psi_term_modified(s, n_clones, A);
      st = orc_weights_modified(s, n_clones, A, w);
    } else {
      orc_evolve(L, n_clones, dt, (uint32_t)beta, seed, a, Ka, dK);
      acc += orc_psi_term(s, n_clones, dK);
      st = orc_weights(s, n_clones, dK, w);
    }
    for (int64_t j = 0; j < n_clones; ++j) ev += (uint64_t)dK[j];
    if (st != ORC_OK) status = st;
    st = iid ? orc_ancestors_iid(n_clones, w, (uint32_t)beta, seed, anc)
             : orc_ancestors(n_clones, w, (uint32_t)beta, seed, anc);
    if (st != ORC_OK) {
      status = ORC_ERR_RANGE;
      goto done;
    }
    orc_gather(L, n_clones, anc, a, Ka, b, Kb);
    uint8_t* ts = a; a = b; b = ts;
    int32_t* tk = Ka; Ka = Kb; Kb = tk;
  }
  {
    double t_obs = (double)M * dt;
    double ksum = 0.0;
    for (int64_t j = 0; j < n_clones; ++j) ksum += (double)Ka[j];
    if (psi_hat) *psi_hat = acc / t_obs;
    if (k_hat) *k_hat = ksum / ((double)n_clones * (double)L * t_obs);
    if (events) *events = ev;
    if (sites_out) memcpy(sites_out, a, nbytes);
    if (K_out) memcpy(K_out, Ka, (size_t)n_clones * sizeof(int32_t));
  }
done:
  free(a); free(b); free(Ka); free(Kb); free(dK); free(w); free(anc); free(A);
  return status;
}

int orc_run(int32_t L, int32_t N, int64_t n_clones, uint64_t seed, double s, double dt,
            int64_t M, double* psi_hat, double* k_hat, uint64_t* events,
            uint8_t* sites_out, int32_t* K_out) {
  return orc_run_ex(L, N, n_clones, seed, s, dt, M, 0, 0, psi_hat, k_hat, events, sites_out, K_out);
}
