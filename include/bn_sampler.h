/*
 * bn_sampler.h — C ABI of the GB300 (sm_103a) screen-space blue-noise sampler optimizer.
 *
 * Method: Belcour & Heitz, "Lessons Learned and Improvements when Building Screen-Space
 * Samplers with Blue-Noise Error Distribution" (SIGGRAPH '21 Talks).
 *   - Sec. 2:   a screen-space sampler is a main sequence s^k scrambled per pixel by u_p; the
 *               tile U = {u_p} is optimised against the Eq. 1 loss over the map of test-
 *               integrand estimates I_p (random Heavisides, Fig. 1b).
 *   - Sec. 3.2: main sequence = rank-1 lattice s^k = mod(Phi(k) d, 1), scrambling =
 *               toroidal (Cranley-Patterson) shift mod(s^k + u_p, 1).
 *   - Sec. 3.4: parallel optimisation: many disjoint couples of pixels are tested for a swap
 *               in each pass; candidates come from a precomputed permutation of pixel indices
 *               XOR-scrambled with a per-pass value.
 *
 * Conventions
 *   - Every call returns BN_OK (0) or a negative BN_ERR_* code; bn_last_error() then returns a
 *     thread-local message.  No C++ exception crosses this boundary.
 *   - All device work of a sampler is enqueued on the CUDA stream given to bn_sampler_init
 *     (NULL = the legacy default stream).  Calls that return data to the host synchronise that
 *     stream; the others only enqueue.
 *   - The library owns all device state it allocates (cudaMalloc at init, cudaFree at destroy).
 *     Host output buffers are owned by the caller and must hold the stated number of elements.
 *   - Pixel p = y * width + x.  Per-pixel arrays are row-major [height][width].
 *   - One sampler holds n_pairs independent 2-D problems ("pairs of dimensions", Sec. 3.1):
 *     each pair has its own shifts, integrands, estimates and optimisation state; pair i uses
 *     Philox streams with pair index i.
 */
#ifndef BN_SAMPLER_H
#define BN_SAMPLER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------------ */
#define BN_OK 0
#define BN_ERR_INVALID_ARG (-1) /* a parameter is out of range or a pointer is NULL        */
#define BN_ERR_OOM (-2)         /* a device allocation failed                              */
#define BN_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed             */
#define BN_ERR_TIMEOUT (-4)     /* a bounded device-side wait ran out (grid barrier)       */
#define BN_ERR_BUSY (-5)        /* the server refused a request (memory budget / slots)    */
#define BN_ERR_BAD_STATE (-6)   /* the object is not in a state that allows this call      */

/* ---- optimisation options ----------------------------------------------------------------- */
/* Commit rule of one pass (Sec. 3.4).  NONINTERACTING keeps, among improving couples whose
 * pixels lie within the weight radius of each other, only the couple of highest priority, so
 * the kept changes add up exactly and the objective never gets worse.  CONCURRENT keeps every
 * improving couple, as the paper describes its GPU optimiser (the loss may then move the wrong
 * way early on, as the paper notes). */
#define BN_MODE_NONINTERACTING 0
#define BN_MODE_CONCURRENT 1

/* Direction of the optimisation of Eq. 1.  A swap keeps sum_p |I_p|^2 fixed, so raising Eq. 1
 * lowers the Gaussian-weighted correlation of neighbouring estimates: the error becomes blue
 * noise (BLUE, the default).  LITERAL reduces Eq. 1 as printed. */
#define BN_OBJECTIVE_BLUE (-1)
#define BN_OBJECTIVE_LITERAL 1

/* How sweeps are executed (results are identical; only speed differs). */
#define BN_SCHEDULE_AUTO 0       /* persistent when the tile allows it, else plain          */
#define BN_SCHEDULE_PLAIN 1      /* three launches per sweep, one warp per couple           */
#define BN_SCHEDULE_PERSISTENT 2 /* one cooperative launch for many sweeps, SMEM-blocked    */
#define BN_SCHEDULE_TENSOR 3     /* five launches per sweep, the stencil of Eq. 1 as products */
                                 /* on the 5th-generation tensor cores (N <= 512 and         */
                                 /* radius <= 8, tile sides >= 2 radius + 1)                 */

typedef struct bn_config {
    int32_t width, height;     /* toroidal tile, 2..4096 each, width*height <= 2^22          */
    int32_t n_points;          /* N = 2^m lattice points per pixel, 2..1024                  */
    int32_t generator_g;       /* Korobov generator, odd, < N; 0 = max-min-distance choice   */
    int32_t n_pairs;           /* 1 (2-D) or 2 (4-D as two independent pairs, Sec. 3.1)      */
    int32_t n_integrands;      /* T Heavisides per pair, 1..4096                             */
    float sigma;               /* Eq. 1 weight exp(-d^2 / sigma^2); the paper uses 2.1       */
    int32_t radius;            /* weight cut-off: pairs with d^2 <= radius^2, 1..8           */
    int32_t couples_per_sweep; /* couples tested per pass; 0 = 2^ceil(log2 P) / 8 (N/4 px)   */
    int32_t mode;              /* BN_MODE_*                                                  */
    int32_t objective;         /* BN_OBJECTIVE_*; 0 = BN_OBJECTIVE_BLUE                      */
    int32_t schedule;          /* BN_SCHEDULE_*                                              */
    uint64_t seed;             /* key of every Philox stream of this sampler                 */
} bn_config;
/* Further limit: 24 * T * N^2 < 2^31 (exact int32 accumulation of the swap energy terms). */

typedef struct bn_sweep_stats {
    int64_t sweeps;     /* passes run by the call (per pair)                                  */
    int64_t proposals;  /* valid couples evaluated, all pairs                                 */
    int64_t improving;  /* couples whose swap improves the objective                          */
    int64_t committed;  /* swaps applied                                                       */
    int64_t ties;       /* couples with |dL| < 1e-6 * sum of |per-distance terms| (fp32 view) */
} bn_sweep_stats;

typedef struct bn_info {
    int32_t generator_g;     /* g actually used                                              */
    int32_t log2_padded;     /* L: candidate indices live in [0, 2^L), 2^L >= P              */
    int32_t couples;         /* couples per pass (M)                                         */
    int32_t count_bytes;     /* 1 (N <= 64) or 2 bytes per stored count                      */
    int32_t row_bytes;       /* bytes of one pixel's count vector (T padded to 128 B)        */
    int32_t n_offsets;       /* distinct neighbours within the radius                        */
    int32_t n_classes;       /* distinct squared distances among them                        */
    int32_t schedule;        /* schedule that optimize_sweeps will use                       */
    int64_t sweep;           /* passes done so far (per pair)                                */
    int64_t device_bytes;    /* device memory held by the sampler                            */
    int64_t reset_h2d_bytes; /* host->device bytes copied by bn_sampler_reset                */
} bn_info;

typedef struct bn_sampler bn_sampler;

/* Create a sampler and run its initialisation on the stream (Sec. 2, Sec. 3.2): pick g, draw
 * the shifts u_p, the Heaviside bank and the candidate permutation, and count, for every pixel
 * and integrand, the lattice points under the Heaviside (k_p[t], estimate k/N).
 * cfg: read only, copied.  cuda_stream: a cudaStream_t or NULL.  out: receives the handle. */
int bn_sampler_init(const bn_config *cfg, void *cuda_stream, bn_sampler **out);

/* Eq. 1 for every pair: L = sum_p sum_{q != p, d(p,q) <= r} exp(-d^2/sigma^2) |I_p - I_q|^2
 * over ordered pairs, distances on the torus.  Exact integer sums per squared distance, then
 * an fp32 compensated weighted sum.  energy_per_pair: host, n_pairs doubles.  Synchronises. */
int bn_evaluate_energy(bn_sampler *s, double *energy_per_pair);

/* Same as bn_evaluate_energy, enqueued only: writes n_pairs doubles to device memory. */
int bn_evaluate_energy_device(bn_sampler *s, double *energy_per_pair_device);

/* Run n_sweeps passes of the parallel swap optimiser (Sec. 3.4) on every pair; the pass
 * counter persists, so two calls of a and b passes equal one call of a + b.  stats: host,
 * nullable; when given the call synchronises and fills it. */
int bn_optimize_sweeps(bn_sampler *s, int32_t n_sweeps, bn_sweep_stats *stats);

/* The optimised tile u_p as float [n_pairs][height][width][2] (exact: 24-bit fixed point).
 * out: host (out_is_device = 0, synchronises) or device (1, enqueued) buffer of n_floats >=
 * n_pairs * width * height * 2 floats. */
int bn_fetch_shifts(bn_sampler *s, float *out, size_t n_floats, int out_is_device);

/* Re-run the initialisation with a new seed (same geometry), without allocating: the problem
 * descriptors are copied from pinned host memory, then shifts, integrands, permutation and
 * counts are rebuilt and the pass counter returns to 0.  Enqueued only. */
int bn_sampler_reset(bn_sampler *s, uint64_t seed);

/* Free all device state.  Synchronises the sampler's stream first.  NULL is allowed. */
void bn_sampler_destroy(bn_sampler *s);

/* Message of the last failed call on this thread ("" if none). */
const char *bn_last_error(void);

/* ---- inspection, parity and checkpoint -------------------------------------------------- */
int bn_get_info(bn_sampler *s, bn_info *info);

/* The shifted lattice s^k_p of one pixel (Sec. 3.2, Fig. 1a) as float [N][2] in [0, 1).
 * Computed on the device from the same fixed-point values the counting kernel uses.  Host
 * buffer of n_floats >= 2 N.  Synchronises. */
int bn_fetch_points(bn_sampler *s, int32_t pair, int32_t pixel, float *out, size_t n_floats);

/* Counts k_p[t] of one pair as int32 [P][T] (host, n >= P*T).  Synchronises. */
int bn_fetch_counts(bn_sampler *s, int32_t pair, int32_t *out, size_t n);

/* The Heaviside bank of one pair: a[T], b[T] (int32) and C[T] (int64, c * 2^24); the
 * integrand is [a x + b y < c].  Host buffers of T elements.  Synchronises. */
int bn_fetch_integrands(bn_sampler *s, int32_t pair, int32_t *a, int32_t *b, int64_t *C,
                        size_t T);

/* Candidate permutation of one pair: int32 [2^L] (host).  Synchronises. */
int bn_fetch_permutation(bn_sampler *s, int32_t pair, int32_t *out, size_t n);

/* Log of the last pass of one pair: per couple j < M the change dL_j of Eq. 1 (float; 0 for
 * dropped couples), flags (1 valid, 2 improving, 4 committed, 8 tie in fp32) and the couple's
 * pixels (int32 [M][2]).  Any pointer may be NULL.  cap >= M.  Synchronises. */
int bn_fetch_sweep_log(bn_sampler *s, int32_t pair, float *dE, uint8_t *flags,
                       int32_t *couples, size_t cap);

/* Checkpoint: the pass counter and, per pair, the index of the initial shift now at each
 * pixel (int32 [n_pairs][P]).  get synchronises; set re-derives the counts from the shifts
 * and enqueues. */
int bn_get_state(bn_sampler *s, int64_t *sweep, int32_t *shift_index, size_t n);
int bn_set_state(bn_sampler *s, int64_t sweep, const int32_t *shift_index, size_t n);

/* Self-test of the kernels' bounded waits: runs the grid barrier (which = 0, waiting for one
 * more block than exists) or an mbarrier wait (which = 1, nobody arrives) with a budget of
 * budget_cycles SM clock cycles (1000 .. 2^31) on a condition that cannot occur.  Returns
 * BN_ERR_TIMEOUT when the wait gave up and reported it, as it must; the GPU context stays
 * usable.  Synchronises the legacy default stream. */
int bn_selftest_wait_timeout(int32_t which, int64_t budget_cycles);

/* Number of kernels this library has launched in this process (all samplers). */
int64_t bn_launch_counter(void);

/* ---- kernel timing ------------------------------------------------------------------------ */
/* enable = 1: the evaluation kernel of every pass launched for this sampler (or a batch containing
 * it) is bracketed by CUDA events on its stream; 2: every kernel of a pass; 0: none.
 * bn_kernel_times then returns, per kernel name, the number of launches and their summed device
 * time since the last read (and resets them).  Synchronises. */
typedef struct bn_kernel_time {
    char name[32];
    int64_t launches;
    double total_ms;
} bn_kernel_time;
int bn_set_kernel_timing(bn_sampler *s, int enable);
int bn_kernel_times(bn_sampler *s, bn_kernel_time *out, int32_t cap, int32_t *n_out);

/* ---- execution schedule (speed only; results do not depend on it) ------------------------ */
/* kind: BN_SCHEDULE_*.  For the persistent kernel, block_x x block_y pixels per work unit,
 * threads per CTA and proposed pixels per compute warp per round must name an instantiated
 * shape (8x8/256/4, 16x8/512/4, 8x16/512/4; a shape that does not fit the tiles, i.e. tiles
 * narrower than block_x + 2 radius, gives way to the first one that does); tsplit = chunk
 * ranges per block (1..4, 0 = auto).  block_x = 0 keeps the default shape.
 * BN_SCHEDULE_TENSOR ignores the other fields; for every problem it needs counts below 1024
 * (N <= 512), radius <= 8 and tile sides of at least 2 radius + 1 (BN_ERR_INVALID_ARG
 * otherwise); the centred products are summed exactly in f32 per accumulator round of at most
 * 2^25 / (64 N^2) stages of 64 integrands, the rounds as integers; its plan holds the couples' per-pass f16 deltas (1/4 of the count bytes for 8-bit counts, 1/8 for 16-bit) and one TMA
 * tensor map per problem, released with the plan.  set synchronises the stream. */
typedef struct bn_schedule {
    int32_t kind;
    int32_t block_x, block_y;
    int32_t threads;
    int32_t slots_per_warp;   /* proposed pixels per compute warp per round */
    int32_t tsplit;
} bn_schedule;
int bn_sampler_set_schedule(bn_sampler *s, const bn_schedule *sc);
int bn_sampler_get_schedule(bn_sampler *s, bn_schedule *out);

/* Plain and tensor-core schedules: sweeps run as replays of a CUDA graph that holds
 * passes_per_graph passes (three or five kernels each), captured on first use; 0 launches every
 * kernel directly.  Default 32.
 * Results are identical either way; per-kernel timing (bn_set_kernel_timing) bypasses the
 * graphs.  Synchronises the stream and drops graphs already captured. */
int bn_sampler_set_graph_passes(bn_sampler *s, int32_t passes_per_graph);

/* Autotuner: time every instantiated schedule (CTA shape x chunk split, the tensor-core
 * schedule where every tile allows it, plain as fallback) for
 * trial_sweeps passes on a scratch copy of the device state, keep the fastest, and cache the
 * choice per workload signature (tile sizes, N, T, couples, radius, SM count) in the process and,
 * when the environment variable BN_AUTOTUNE_CACHE names a file, in that file.  The caller's
 * tiles are not modified; results never depend on the schedule.  chosen: nullable.
 * Synchronises. */
int bn_sampler_autotune(bn_sampler *s, int32_t trial_sweeps, bn_schedule *chosen);

/* ---- evaluation of a tile (Sec. 3.3, Sec. 3.5) ------------------------------------------------
 * Criterion of Fig. 1c: for each integrand the error tile (estimate minus exact integral) is
 * filtered by a Gaussian of standard deviation sigma (pixels) and the RMSE over integrands and
 * pixels is returned per sigma: rmse = sqrt(mean_t mean_p ((k_sigma * e_t)(p))^2).
 * The filter is the sampled Gaussian exp(-d^2 / (2 sigma^2)) wrapped around the toroidal tile
 * and normalised to sum 1, applied along x then y; sigma <= 0 leaves the error unfiltered.
 *   integrands  BN_INTEGRANDS_HEAVISIDE: the first n_integrands Heavisides of the pair's bank
 *               (estimate k_p[t] / N, reference the exact area within the unit square);
 *               BN_INTEGRANDS_GAUSSIAN: n_integrands (<= 4096) smooth bumps
 *               exp(-|x - c|^2 / (2 s^2)), c uniform in [0,1)^2 and s uniform in [0.05, 0.5)
 *               from Philox tag 7 (estimate: mean over the pixel's N shifted lattice points;
 *               reference: closed form with erf).  The Sec. 3.5 check: the optimiser never
 *               sees these, yet their filtered error drops too.
 *   sigmas      host, n_sigma (1..64) floats; rmse_out: host, n_sigma doubles.
 * FP64 throughout.  Uses temporary device memory (stream-ordered); synchronises. */
#define BN_INTEGRANDS_HEAVISIDE 0
#define BN_INTEGRANDS_GAUSSIAN 1
int bn_evaluate_criterion(bn_sampler *s, int32_t pair, int32_t integrands, int32_t n_integrands,
                          const float *sigmas, int32_t n_sigma, double *rmse_out);

/* ---- error spectrum (Fig. 1b) -----------------------------------------------------------------
 * Radially averaged power spectrum of the pair's error tiles e_t(p) = I_p - I_ref, for the same
 * integrands as bn_evaluate_criterion.  F_t is the 2-D DFT of e_t over the W x H tile; the power
 * of frequency (u, v) is |F_t(u, v)|^2 / (W H), so white error of variance s^2 has power s^2 at
 * every frequency and the rings' power x count sums to the mean squared error per pixel (times
 * W H / W H: Parseval).  Ring of (u, v): f_x = u, or u - W when 2u > W (likewise f_y with H),
 * rho = sqrt((f_x / W)^2 + (f_y / H)^2) cycles per pixel, ring = floor(rho min(W, H) + 1/2),
 * decided in exact integer arithmetic; ring 0 holds the mean error (0, 0).
 *   power_out    host, n_rings doubles: mean over the integrands and over the ring's
 *                frequencies; null = only report the ring count in *n_rings_out.
 *   counts_out   host, n_rings int64 (nullable): frequencies per ring.
 *   n_rings_out  (nullable) receives the ring count, floor(sqrt(1/2) min(W, H) + 1/2) + 1 for a
 *                square tile; n_rings below it is BN_ERR_INVALID_ARG.
 * Tile sides at most 1024.  FP64 throughout (direct DFT sums, twiddles computed on the host).
 * Uses temporary device memory (stream-ordered); synchronises. */
int bn_error_spectrum(bn_sampler *s, int32_t pair, int32_t integrands, int32_t n_integrands,
                      double *power_out, int64_t *counts_out, int32_t n_rings,
                      int32_t *n_rings_out);

/* ---- renderer lookup (Sec. 3.1, Sec. 3.2) ---------------------------------------------------
 * bn_export_shift_table writes the pair's current per-pixel shifts (uint32 [height][width][2],
 * 0.32 fixed point) to device memory (enqueued only), for the device function bn_sample() of
 * include/bn_sample.cuh that a renderer's kernels call.
 * bn_generate_samples fills out[r][i][j][d] = sample first_sample + j of screen pixel
 * (x0 + i, y0 + r) in dimension d: the tile repeats over the screen (negative coordinates
 * wrap too), dimension d reads coordinate d % 2 of pair d / 2, so n_dims <= 2 n_pairs; an odd
 * n_dims leaves out the second coordinate of the last pair (the padding of Sec. 3.1).  Values
 * are multiples of 2^-24 in [0, 1).  first_sample + n_samples <= n_points.  out: device when
 * out_is_device, else host (then the call synchronises). */
int bn_export_shift_table(bn_sampler *s, int32_t pair, uint32_t *out_device, size_t n_words);
int bn_generate_samples(bn_sampler *s, int32_t x0, int32_t y0, int32_t width, int32_t height,
                        int32_t first_sample, int32_t n_samples, int32_t n_dims, float *out,
                        size_t n_floats, int32_t out_is_device);

/* ---- batches: many samplers swept together in one launch sequence ------------------------- */
typedef struct bn_batch bn_batch;

/* Group samplers (all created on the same device) so that their sweeps run fused: every pair
 * of every sampler becomes one problem of a single launch.  The batch sweeps on its own stream
 * (cuda_stream): a sweep call first waits for each member's stream to finish its queued work,
 * and work enqueued later on a member's stream waits for the batch's sweeps (event). */
int bn_batch_create(bn_sampler *const *samplers, int32_t n, void *cuda_stream, bn_batch **out);
int bn_batch_optimize(bn_batch *b, int32_t n_sweeps, bn_sweep_stats *stats);
/* As bn_batch_optimize, with a pass budget per member sampler (host array, one entry per sampler
 * in the order given to bn_batch_create); members stop at their own budget inside the launch. */
int bn_batch_optimize_each(bn_batch *b, const int32_t *n_sweeps_per_member,
                           bn_sweep_stats *stats);
int bn_batch_set_schedule(bn_batch *b, const bn_schedule *sc);
int bn_batch_autotune(bn_batch *b, int32_t trial_sweeps, bn_schedule *chosen);
int bn_batch_get_schedule(bn_batch *b, bn_schedule *out);
int bn_batch_set_graph_passes(bn_batch *b, int32_t passes_per_graph);
void bn_batch_destroy(bn_batch *b);

/* ---- serving: continuous batching of sampler-generation requests --------------------------
 * The paper runs one optimisation at a time; this is the serving loop around it.  A server owns
 * one GPU and a background host thread.  Each request is one sampler configuration plus a pass
 * budget.  The thread admits queued requests (first come, first served) while a slot is free and
 * their device memory fits the budget, initialises their samplers on a side stream, sweeps all
 * resident requests together in fused batches of at most sweeps_per_chunk passes each (each
 * request stops at its own budget inside the launch): one batch on the tensor-core schedule for
 * the requests whose signature (count width, N, T, radius, pairs, tile sides rounded up to
 * powers of two) the autotuner assigned to it, timed once per signature on a scratch copy of the
 * first such request and cached for the server's lifetime, and one batch for the rest.  It
 * retires finished requests (final Eq. 1 and
 * the optimised shifts copied to host, device memory released).  A request's result is identical
 * to running it alone through bn_sampler_init + bn_optimize_sweeps with the same pass budget.
 * All functions are thread-safe; none waits for the GPU except bn_server_drain/destroy. */
typedef struct bn_server bn_server;

typedef struct bn_server_config {
    int32_t device;               /* CUDA device index                                       */
    int32_t max_slots;            /* resident requests at most (1..4096)                     */
    int32_t sweeps_per_chunk;     /* passes per fused launch sequence (1..500)               */
    int32_t tensor_policy;        /* BN_SERVE_TENSOR_*: which requests join the tensor batch */
    int64_t memory_budget_bytes;  /* device bytes for resident requests; 0 = 80% of free     */
} bn_server_config;

#define BN_SERVE_TENSOR_TUNED 0   /* the autotuner's choice per request signature (default)  */
#define BN_SERVE_TENSOR_ALWAYS 1  /* every request that supports the schedule, no trials     */
#define BN_SERVE_TENSOR_NEVER 2   /* none: one fused batch on the other schedules            */

typedef struct bn_request {
    bn_config cfg;                /* the sampler to build (schedule is ignored)              */
    int32_t n_sweeps;             /* pass budget (>= 1)                                      */
    int32_t reserved;
    int64_t user_tag;             /* returned unchanged in the result                        */
} bn_request;

typedef struct bn_result {
    int64_t request_id, user_tag;
    int32_t status;               /* BN_OK, BN_ERR_BAD_STATE when cancelled, else the error  */
    int32_t n_pairs, width, height;
    double energy[2];             /* Eq. 1 of each pair after the budget                     */
    double t_submit, t_admit, t_done;  /* seconds since the server was created              */
} bn_result;

typedef struct bn_server_stats {
    int64_t submitted, admitted, completed, rejected, cancelled, failed;
    int64_t pending, active;      /* queued / resident right now                             */
    int64_t chunks;               /* fused launch sequences run                              */
    int64_t proposals;            /* couples proposed (pairs x couples x passes)             */
    int64_t memory_in_use, memory_budget;
    int64_t tensor_chunks;        /* chunks that ran a batch on the tensor-core schedule     */
    int64_t tunes;                /* request signatures timed by the autotuner               */
} bn_server_stats;

int bn_server_create(const bn_server_config *cfg, bn_server **out);
/* Queue a request; request_id (nullable) receives its id.  BN_ERR_INVALID_ARG for an invalid
 * configuration, BN_ERR_BUSY (counted as rejected) when it alone exceeds the memory budget. */
int bn_server_submit(bn_server *sv, const bn_request *req, int64_t *request_id);
/* Cancel a queued or resident request; it is reported with status BN_ERR_BAD_STATE. */
int bn_server_cancel(bn_server *sv, int64_t request_id);
/* Move up to cap finished results (in completion order) into out; *n_out = how many. */
int bn_server_poll(bn_server *sv, bn_result *out, int32_t cap, int32_t *n_out);
/* Copy a completed request's shifts (host floats [n_pairs][height][width][2], the layout of
 * bn_fetch_shifts) and release them; each request's shifts can be taken once. */
int bn_server_take_shifts(bn_server *sv, int64_t request_id, float *out, size_t n_floats);
int bn_server_get_stats(bn_server *sv, bn_server_stats *out);
/* Wait until no request is queued or resident (BN_ERR_BUSY at the timeout). */
int bn_server_drain(bn_server *sv, double timeout_s);
/* Stop the thread after its current chunk; resident and queued requests are dropped. */
void bn_server_destroy(bn_server *sv);

/* ---- Eq. 1 without device allocation -------------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory (code running inside another framework's memory pool or arena, real-time loops that
 * must not stall on the allocator, plug-ins that are only handed pre-allocated buffers).  It
 * computes the same Eq. 1 as bn_evaluate_energy, for n_fields count fields given by the caller,
 * and allocates nothing: its only scratch is a fixed 16 KiB array of the library (per-class
 * sums of up to 64 fields) that every GPU loading the library keeps until the process exits.
 *   counts   device, int32 [n_fields][height][width][n_integrands]; values in [0, n_points]
 *   energy   device, n_fields doubles (written)
 *   n_fields 1..64 (more is rejected with BN_ERR_INVALID_ARG: the scratch holds 64 fields)
 *   width, height, n_points, n_integrands, sigma, radius: as in bn_config (radius 1..8)
 * Enqueued on cuda_stream; returns without waiting.  The first call on each device looks up
 * the device address of the scratch array (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  That address is kept for the life of the process: after a reset
 * of the device's context (cudaDeviceReset, or a primary-context reset by the host framework)
 * the module is reloaded and the cached address is stale, so do not call this entry point
 * again after such a reset.  Every call shares the scratch array: a call clears what it uses
 * before accumulating, but calls whose work overlaps on the GPU race on it.  A CUDA error
 * already pending on the calling thread is reported (BN_ERR_CUDA) before anything is launched,
 * and is left pending for the caller. */
int bn_evaluate_energy_noalloc(const int32_t *counts, int32_t n_fields, int32_t width,
                               int32_t height, int32_t n_points, int32_t n_integrands,
                               float sigma, int32_t radius, double *energy, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BN_SAMPLER_H */
