/*
 * pop.h -- C ABI of the GB300 population-dynamics (cloning) library.
 *
 * The library estimates the scaled cumulant generating function psi(s) of the
 * activity K (number of particle hops) of the symmetric simple exclusion process
 * (SSEP) on a ring by the cloning algorithm of arXiv:1711.05095:
 *   - Sec. 2.3: a population of N_c clones, M = t_obs/dt intervals, each a
 *     dynamical stage (independent evolution) followed by a cloning stage
 *     (resampling in proportion to the weights Upsilon, eq. upsbdef);
 *   - eq. (psihat): psi_hat = (1/t_obs) sum_beta ln( (1/N_c) sum_i Upsilon_i^beta );
 *   - Sec. 4.1, eq. (alpha-Ups): [eq] selection with equally spaced points;
 *   - eq. (khat): k_hat from the cumulative activity carried with each clone.
 * A handle holds a BATCH of independent populations (each its own L, N, N_c,
 * seed and bias s) that advance through the intervals together.
 *
 * Conventions
 *   - Every call returns an int status: POP_OK (0) or a negative POP_ERR_*.
 *   - Device memory is owned by the caller: pop_init carves one caller-allocated
 *     device workspace of pop_workspace_bytes() bytes; pop_free never frees it.
 *   - Work is enqueued on the CUDA stream given to pop_init.  pop_evolve,
 *     pop_resample and pop_run return once their kernels are enqueued; the
 *     host-reading calls (pop_estimate_psi, pop_copy_state, pop_events) wait for
 *     the stream.  Kernel-side errors (an activity outside the weight table, an
 *     interval that needed more than 2^24 BKL steps) are sticky in device memory and
 *     are returned by the next host-reading call.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Lattices: site i of a clone is bit (i mod 64) of 64-bit word (i div 64); a
 *     clone occupies W = ceil(max_p L_p / 64) consecutive words (bits >= L zero).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     population's 64-bit seed, counter (c0, c1, c2, c3) =
 *       initial state   (site t, 0,        clone slot j, 1)
 *       dynamical stage (draw q, interval, clone slot j, 2)  step e uses draw e/2
 *       cloning stage   (0,      interval, 0,            3)   [eq]
 *                       (new clone j, interval, 0,      4)   [iid]
 *     Intervals are numbered from 1.  Results are reproducible bit for bit for a
 *     given batch, independent of the launch configuration.
 */
#ifndef POP_H
#define POP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define POP_OK 0
#define POP_ERR_ARG (-1)     /* an argument is out of its documented range */
#define POP_ERR_CUDA (-2)    /* a CUDA runtime call failed (no device, launch failure) */
#define POP_ERR_RANGE (-3)   /* an interval activity differed from the reference by >= POP_KCAP,
                                or a clone's interval needed more than 2^24 BKL steps */
/* (-4) is not used: no kernel of this library waits on the device */
#define POP_ERR_STATE (-5)   /* call out of order, or s changed during a run */

/* weight modes (eq. upsdef) */
#define POP_PLAIN 0    /* unmodified SSEP rates, Upsilon = exp(-s dK) (eq. upsbdef, U = 0) */
#define POP_MODIFIED 1 /* every rate times e^-s, Upsilon = exp(-(1-e^-s) int r dt)
                          (Sec. 3.2, eq. def-ups-ssep); the integral is accumulated in
                          FP32 and the weights use a specified FP32 exponential */
#define POP_GUIDED 2   /* modified dynamics of Sec. 2.2 (eqs. modpdef, upsdef) with a
                          local potential U(C) = sum_i phi(sites i-4..i+4): the hop
                          across bond b has rate e^-s e^{(U(C^b) - U(C))/2}, the exponent
                          rounded to a multiple of 2^-17 and clamped to [-8, 8], held as
                          an integer in units of 2^-40 whose logarithm is known to 3e-9;
                          Upsilon = prod_hops (e^-s / rate) exp(-int (r - r') dt) of the
                          rates simulated, so the estimate is unbiased for any phi.
                          18 <= L <= 128, every population of the batch must be
                          GUIDED, and a GUIDED batch holds at most 65535 populations
                          (each with 1.5 MiB of rate tables in the workspace).  phi is
                          set by pop_set_potential (default 0) */

/* clone selection (Sec. 4.1) */
#define POP_EQ 0  /* equally spaced alpha_j, eq. (alpha-Ups) */
#define POP_IID 1 /* independent uniform alpha_j = floor(U64 T / 2^64), U64 from Philox
                     counter (new clone j, interval, 0, 4) */

#define POP_KCAP 4096     /* size of the fixed-point weight table */
#define POP_MAX_L 4096    /* largest ring; rings above 128 sites run one clone per warp */
#define POP_MAX_CLONES (1LL << 30)

/* One population of the batch. */
typedef struct pop_params {
  int32_t L;           /* ring length, 3 <= L <= POP_MAX_L (a batch with any L > 128
                          runs every population with the one-clone-per-warp evolve) */
  int32_t N;           /* particles, 0 <= N <= L */
  int64_t n_clones;    /* N_c, 1 <= N_c <= POP_MAX_CLONES */
  uint64_t seed;       /* Philox key of this population's streams */
  int32_t weight_mode; /* POP_PLAIN, POP_MODIFIED or POP_GUIDED */
  int32_t selection;   /* POP_EQ or POP_IID */
} pop_params;

typedef struct pop_batch pop_t;

/*
 * Device workspace needed for a batch of n_pops populations (bytes, a multiple of
 * 256).  Returns 0 if the parameters are invalid.  Host-only; touches no device.
 */
size_t pop_workspace_bytes(const pop_params* params, int32_t n_pops);

/*
 * Create a batch and draw its initial configurations (Sec. 2.1: initial condition
 * from the steady state, which for the SSEP at fixed N is a uniform N-subset of the
 * sites; Sec. 3.1).  params: host array of n_pops entries (copied).  d_workspace:
 * caller-owned device memory of at least pop_workspace_bytes(params, n_pops) bytes,
 * 256-byte aligned, that must outlive the handle.  cuda_stream: a cudaStream_t (NULL
 * = legacy default stream).  On success *out receives the handle; on failure *out is
 * NULL and nothing needs freeing.
 */
int pop_init(pop_t** out, const pop_params* params, int32_t n_pops, void* d_workspace,
             size_t workspace_bytes, void* cuda_stream);

/*
 * Replace the configurations of population p (0-based) by caller-supplied ones
 * (host memory): h_lattice holds N_c * W words (clone-major), h_K the N_c cumulative
 * activities (NULL = zeros).  Every clone must hold exactly N particles and no bit at
 * or above L (else POP_ERR_ARG, nothing copied).  Allowed before the first interval
 * only.  Waits for the copies.
 */
int pop_set_state(pop_t* pop, int32_t p, const uint64_t* h_lattice, const int32_t* h_K);

/*
 * Dynamical stage of the next interval (Sec. 2.3; Sec. 4: BKL continuous-time Monte
 * Carlo of the SSEP for a time dt).  s: host array of n_pops biases; the first call
 * fixes them for the run (a later call with a different s returns POP_ERR_STATE).
 * dt > 0 may change between intervals; t_obs is their sum.
 */
int pop_evolve(pop_t* pop, double dt, const double* s);

/*
 * Cloning stage of the interval just evolved (Sec. 2.3, Sec. 4.1): the weights, the
 * psi term ln((1/N_c) sum Upsilon) accumulated in FP64 (eq. psihat), exact 64-bit
 * fixed-point prefix sums, [eq] ancestors (eq. alpha-Ups) and the gather of lattices
 * and cumulative activities.  POP_ERR_STATE unless pop_evolve came just before.
 */
int pop_resample(pop_t* pop);

/*
 * n_intervals full intervals (dynamical stage then cloning stage), identical in
 * result to n_intervals pairs of pop_evolve/pop_resample, launched as captured CUDA
 * graphs.  Same rules for s and dt as pop_evolve.
 * When the batch fuses the cloning stage with the next dynamical stage (every
 * population [eq], not GUIDED, L <= 128), the fused intervals run as 1 to 8 chains of
 * kernels, each over a run of whole populations, on internal streams forked from and
 * joined back into the handle's stream (the chains share no data; results are the
 * same bit for bit); pop_run_chains gives the split.
 */
int pop_run(pop_t* pop, double dt, const double* s, int64_t n_intervals);

/*
 * The chains of pop_run: returns their number K (0 when the batch does not fuse, so
 * pop_run launches one sequence; -1 for a NULL handle) and, when h_first_tiles is not
 * NULL and K > 0, writes K + 1 entries: chain c runs the 1024-slot tiles
 * [h_first_tiles[c], h_first_tiles[c + 1]), whole populations, the last entry the
 * batch's tile count.  K is the largest number up to 8 (for a batch that fits in two
 * waves of the fused kernel on this device; up to 2 for a larger one) for which the
 * population starts nearest k/K of the tiles (k = 1 .. K-1) leave every chain at least
 * half of its equal share.
 */
int32_t pop_run_chains(pop_t* pop, int32_t* h_first_tiles);

/*
 * Estimates after the intervals run so far (host arrays of n_pops each; any may be
 * NULL): psi[p] = eq. (psihat); k_hat[p] = (1/(N_c L t_obs)) sum_i K_i over the
 * current population (eq. khat with the 1/N_c of eq. avedef); t_obs = sum of dt.
 * Waits for the stream.  POP_ERR_STATE before the first complete interval.
 */
int pop_estimate_psi(pop_t* pop, double* psi, double* k_hat, double* t_obs);

/*
 * Copy population p to host memory (any pointer may be NULL):
 *   h_lattice  N_c * W words   current configurations
 *   h_K        N_c             cumulative activities
 *   h_anc      N_c             ancestors of the last cloning stage (0-based)
 *   h_dK       N_c             activities of the last dynamical stage
 * Between pop_evolve and pop_resample the lattices/K are the evolved ones.
 * Waits for the stream.
 */
int pop_copy_state(pop_t* pop, int32_t p, uint64_t* h_lattice, int32_t* h_K,
                   int32_t* h_anc, int32_t* h_dK);

/*
 * Launch configuration of a batch (the paper has none: its codes had fixed thread
 * counts).  Every choice changes only speed, never a result:
 *   evolve_grid     persistent grid of the separate dynamical stage (the first interval
 *                   of a fused run; every interval of a batch that does not fuse)
 *   fuse_threads    threads per block of the fused cloning + dynamical stage: 128 or 256
 *   fuse_clones     clones each lane of the fused stage advances together: 1 or 2
 *                   (2 only with 128 threads)
 *   chains          chains of pop_run (1 .. 8; the split actually used may have fewer,
 *                   see pop_run_chains)
 *   gather_threads  threads per block of the separate cloning stage: 128, 256, or 0 for
 *                   the rule (256 above 4096 tiles)
 *   hist_mode       whether the fused stage of a batch without MODIFIED weights also
 *                   counts the new clones' activities per tile, so that the next
 *                   interval's tile weight sums and activity histogram come from those
 *                   counts instead of a pass over every clone: 1 on, 0 off, -1 the rule
 *                   (on when every population has more than 64 tiles of 1024 clones and
 *                   dt * (largest L) <= 16, where an activity of 64 or more in one
 *                   interval is very unlikely; such an activity is still handled, by a
 *                   slower pass over the population's clones)
 *   default_us_per_interval, tuned_us_per_interval: the times per interval pop_autotune
 *                   measured for the configuration pop_init chose and for its choice
 *                   (0 until it has run; ignored by pop_set_tuning)
 */
typedef struct pop_tuning {
  int32_t evolve_grid;
  int32_t fuse_threads;
  int32_t fuse_clones;
  int32_t chains;
  int32_t gather_threads;
  int32_t hist_mode;
  float default_us_per_interval;
  float tuned_us_per_interval;
} pop_tuning;

/*
 * Choose the launch configuration by timing on this batch's own shape.  Times `trials`
 * launches of the dynamical stage of the first interval for every candidate persistent
 * grid (1 .. the resident blocks per SM, times the SM count); for a batch that fuses,
 * three replays of `trials` fused intervals captured as a CUDA graph (as pop_run runs
 * them) for each fused-kernel form (128 threads with one or two clones per lane, 256
 * threads with one) and each chain split (up to 1, 2, 4, 8), with and without the
 * per-tile activity counts where dt * (largest L) <= 16 and no weights are MODIFIED
 * (the hist_mode chosen, 0 or 1, is for this dt); for a
 * batch that does not, `trials` whole intervals for each block size of the separate
 * cloning stage.  Keeps the fastest of each.  Every trial starts again from interval 1
 * and the counters, activities and (for the cloning-stage trials) the population are
 * put back, so results are identical with and without tuning.  Before the first interval
 * only (else POP_ERR_STATE); fixes s like pop_evolve.  h_evolve_grid (may be NULL)
 * receives the chosen grid; pop_get_tuning gives the whole choice.  Waits for the stream.
 */
int pop_autotune(pop_t* pop, double dt, const double* s, int32_t trials, int32_t* h_evolve_grid);

/* The current launch configuration (host struct). */
int pop_get_tuning(pop_t* pop, pop_tuning* out);

/* Set the launch configuration (values outside the ranges above: POP_ERR_ARG; between
 * pop_evolve and pop_resample: POP_ERR_STATE).  Results do not depend on it. */
int pop_set_tuning(pop_t* pop, const pop_tuning* cfg);

/*
 * Population mean of |delta rho_n|^2 over the current configurations (eq. fourdens:
 * delta rho_n = L^-1/2 sum_j exp(-2 pi i n X_j / L) over the occupied sites X_j;
 * Sec. 3.3 uses n = 1 to follow the clustering transition).  Per clone in FP32 from
 * float tables of cos and sin, the mean in FP64.  h_mean: host array of n_pops.
 * n >= 0.  POP_ERR_STATE between pop_evolve and pop_resample.  Waits for the stream.
 */
int pop_density_mode(pop_t* pop, int32_t n, double* h_mean);

/*
 * Potential of a GUIDED population p: h_phi is a host array of 512 floats, phi of
 * the 9-site window whose site i-4+k is bit k of the index (the compiled lookup
 * table of a learned potential).  |phi| <= 64, else POP_ERR_ARG; held as the
 * fixed-point integers nearest to phi 2^16, so every potential difference is exact.
 * POP_ERR_STATE for a population that is not GUIDED, or between pop_evolve and
 * pop_resample.  May change between intervals.  Waits for the stream.
 */
int pop_set_potential(pop_t* pop, int32_t p, const float* h_phi);

/*
 * Ancestry across the last cloning stage (Sec. 2.2: the ancestral population that
 * defines p_ave is found by following the clones' histories backwards): for every
 * clone j of every population, d_out[off + j] = d_in[off + anc_j], anc_j the
 * population-local ancestor written by the last pop_resample and off the
 * population's first slot.  d_in and d_out are device int32 arrays of
 * pop_slots() entries; starting from d_in[off + j] = j and applying this after every
 * cloning stage gives, for each current clone, its ancestor's index at the start.
 * Needs the per-step calls (pop_run does not record ancestors).  Asynchronous.
 */
int pop_lineage(pop_t* pop, const int32_t* d_in, int32_t* d_out);

/* Slots of the batch (populations padded to 1024-slot tiles) and the first slot of
 * population p; -1 for an invalid handle or p. */
int64_t pop_slots(pop_t* pop);
int64_t pop_first_slot(pop_t* pop, int32_t p);

/*
 * Learned guiding potential: a window network phi (MLP 9 -> 128 -> 128 -> 1, GELU)
 * trained on the GPU as a classifier of time-averaged (ancestral, label 1) against
 * end-of-interval (label 0) configurations (Sec. 2.2, eqs. Opave and Opend).  The
 * logit of a configuration is z = (1/2) sum_i phi(w_i) + c over its L windows w_i
 * (sites i-4..i+4, bit k = site i-4+k); the loss is the mean of softplus(z) - y z.
 * Products take BF16 operands with FP32 accumulation; parameters are FP32, in the
 * order W1[128][9], b1[128], W2[128][128], b2[128], W3[128], b3, c (POP_MLP_PARAMS
 * floats).  The trained phi, evaluated at the 512 window patterns, is the table that
 * pop_set_potential takes.
 */
#define POP_MLP_HIDDEN 128
#define POP_MLP_PARAMS 17922
typedef struct pop_mlp pop_mlp_t;

/* Device workspace of a trainer (bytes, a multiple of 256). */
size_t pop_mlp_workspace_bytes(void);

/* Create a trainer with parameters h_theta (host, POP_MLP_PARAMS floats) and zero
 * Adam state in the caller's 256-byte aligned workspace.  Waits for the stream. */
int pop_mlp_init(pop_mlp_t** out, const float* h_theta, void* d_workspace, size_t workspace_bytes,
                 void* cuda_stream);

/* Loss and gradient of a batch without updating: d_lattice (device, n x W words, the
 * configurations as pop_copy_state returns them, 1 <= W <= 2, 9 <= L <= 64 W),
 * d_labels (device, n bytes, 0 or 1).  h_loss (may be NULL): mean loss; h_grad (may
 * be NULL): POP_MLP_PARAMS floats.  Waits for the stream. */
int pop_mlp_grad(pop_mlp_t* mlp, const uint64_t* d_lattice, int32_t W, int32_t L,
                 const uint8_t* d_labels, int64_t n, double* h_loss, float* h_grad);

/* One Adam step (betas 0.9, 0.999, eps 1e-8) at learning rate lr > 0 on a batch as
 * above.  Asynchronous unless h_loss is given (then waits and stores the batch loss,
 * taken before the update). */
int pop_mlp_step(pop_mlp_t* mlp, const uint64_t* d_lattice, int32_t W, int32_t L,
                 const uint8_t* d_labels, int64_t n, float lr, double* h_loss);

/* Current parameters (host, POP_MLP_PARAMS floats).  Waits for the stream. */
int pop_mlp_params(pop_mlp_t* mlp, float* h_theta);

/* The compiled potential: phi at the 512 window patterns (host, 512 floats), from
 * the current parameters.  Waits for the stream. */
int pop_mlp_potential(pop_mlp_t* mlp, float* h_phi);

/* Release the trainer (never the caller's workspace). */
void pop_mlp_free(pop_mlp_t* mlp);

/* Executed hops (BKL events) per population since pop_init (host array of n_pops). */
int pop_events(pop_t* pop, uint64_t* h_events);

/* Kernel kinds of pop_kernel_times and pop_launch_count. */
#define POP_K_EVOLVE 0         /* dynamical stage (Sec. 2.3), one interval */
#define POP_K_WEIGHTS 1        /* cloning weights, tile sums, activity histogram
                                  (k_weights, or the tile scan that forms them from the
                                  fused stage's per-tile activity counts) */
#define POP_K_GATHER 2         /* cloning stage: [eq] copies, [iid] selection */
#define POP_K_GATHER_EVOLVE 3  /* cloning stage of one interval fused with the
                                  dynamical stage of the next (pop_run, [eq], L <= 128) */
#define POP_K_OTHER 4          /* initial state, estimates, density mode, ancestry
                                  (pop_lineage), and the scan of each population's tile
                                  sums before a cloning stage (when it does not also
                                  form the weights) */
#define POP_NKINDS 5

/*
 * Measurement.  Advances the batch by n_intervals >= 1 intervals with the launches
 * pop_run makes (per_step = 0: the same chains on the same streams, the intervals after
 * the first fused one as one captured graph, as pop_run replays them) or those of
 * pop_evolve + pop_resample (per_step = 1: the separate dynamical and cloning stages,
 * launched one by one), in the same order and so with the same results, with a CUDA
 * event recorded before and after every launch on its own stream (an event-record node
 * inside the graph).  Any output may be NULL; each is a host array of POP_NKINDS:
 *   h_us    per kind, the time during which at least one of its launches runs (the
 *           union of their start-to-end ranges), divided by the number of intervals
 *           that launch it, microseconds (one chain: the mean launch time; 0 if none)
 *   h_n     number of launches of each kind
 *   h_hops  hops executed by the launches of each kind (nonzero only for the kinds
 *           that run dynamical stages)
 * Between pop_evolve and pop_resample: POP_ERR_STATE.  Fixes s like pop_evolve.
 * Waits for the stream.
 */
int pop_kernel_times(pop_t* pop, double dt, const double* s, int64_t n_intervals, int32_t per_step,
                     double* h_us, int64_t* h_n, uint64_t* h_hops);

/*
 * Kernels launched by this handle since pop_init, by kind (host array of
 * POP_NKINDS); a replay of pop_run's captured graph counts every kernel it holds.
 */
int pop_launch_count(pop_t* pop, uint64_t* h_n);

/*
 * Cloning-stage selection of ONE population without allocating anything.  The
 * paper has no counterpart: this exists for callers that cannot call cudaMalloc
 * and so cannot provide pop_init's workspace: a process whose device memory is
 * all reserved by another allocator (a framework's caching pool), a
 * latency-critical loop where an allocation and the synchronisation it implies
 * are not allowed, or an embedded runtime without a device allocator.
 *   d_dK        device, n_clones int32: the interval activities K^beta (input)
 *   n_clones    1 <= N_c <= POP_NOALLOC_MAX_CLONES (larger: POP_ERR_ARG)
 *   s, seed     bias and Philox key of the population
 *   interval    beta >= 1, selects the [eq] offset word of that interval
 *   d_anc       device, n_clones int32: ancestors of the new clones (output)
 *   h_psi_term  host, may be NULL: ln((1/N_c) sum_i exp(-s K_i^beta)) (output)
 * Results equal those of pop_resample for the same activities.  Scratch lives in
 * a static device array of 120 KiB that every GPU which loads the library holds
 * until the process exits; each call clears what must start at zero, the array
 * keeps the last call's contents (the weight tables are re-sent only when s or the
 * weight scale of N_c changes), and calls that overlap on the GPU race on it.  The
 * array of the CURRENT device is used: the stream must belong to that device.  The
 * first call on a device looks up the array's device address (with that device
 * current).  Every call synchronises the stream and copies from pageable host
 * memory, so it must not be called on a stream that is being captured.  No
 * cudaMalloc, cudaFree or allocating library routine is called.
 */
#define POP_NOALLOC_MAX_CLONES (1LL << 20)
int pop_select_noalloc(const int32_t* d_dK, int64_t n_clones, double s, uint64_t seed,
                       uint32_t interval, int32_t* d_anc, double* h_psi_term, void* cuda_stream);

/* Lattice words per clone, W, of a batch (0 if the parameters are invalid). */
int32_t pop_lattice_words(const pop_params* params, int32_t n_pops);

/* Static description of a status code. */
const char* pop_strerror(int status);

/* Release the handle (host state and CUDA graphs); never the caller's workspace. */
void pop_free(pop_t* pop);

#ifdef __cplusplus
}
#endif
#endif /* POP_H */
