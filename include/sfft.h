/*
 * sfft.h -- C ABI of the GB300-native flat-window voting sparse FFT.
 *
 * The library computes, for a length-N complex signal x whose spectrum is
 * (approximately) K-sparse, the K largest Fourier coefficients
 *
 *     xhat_f = (1/N) sum_j x_j exp(-2 pi i f j / N)          (Eq. 2)
 *
 * with the voting framework of sFFT1.0 as surveyed in "Empirical Evaluation of
 * Typical Sparse Fast Fourier Transform Algorithms" (arXiv:2012.08238).  Per
 * location loop l < L it
 *   a0  draws a random odd scaling sigma_l and shift tau_l (scaling method,
 *       Eq. 6-7) from Philox4x64-10 keyed by the plan seed;
 *   a1  gathers x[(sigma_l m + tau_l) mod N] for window positions
 *       m in [-w/2, w/2), multiplies by the flat window g (sinc x Gaussian,
 *       Eq. 12-13) and folds the product into B buckets (Eq. 11);
 *   a2  takes a B-point FFT of the fold (bucket values, Eq. 14);
 *   a3  keeps the c*K buckets of largest energy (probability-and-statistics
 *       location method: "2K large buckets");
 *   a4  hashes every frequency f to bucket round(sigma_l f B / N) mod B;
 *   a5  votes: frequencies hashed into kept buckets in at least T loops are
 *       candidates;
 *   a6  estimates each candidate per loop by energy concentration, undoing
 *       the time-shift phase and the window gain, and takes the median over
 *       loops (real and imaginary parts separately);
 *   a7  returns the K candidates of largest magnitude, sorted by frequency.
 *
 * Conventions shared by every entry point:
 *   - complex64 arrays are interleaved (re, im) float pairs;
 *   - x_dev / outputs are DEVICE pointers owned by the caller unless the
 *     function name ends in _host; the library never frees caller memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued asynchronously and results are valid once
 *     the stream reaches that point;
 *   - every call returns an sfft_status; no call aborts or throws.  A failed
 *     call writes a one-line reason readable with sfft_last_error();
 *   - a plan owns device scratch: one plan must not be executed by two
 *     streams at once (use separate plans, sfft_execute_batch or the server).
 *
 * Sizes (checked, SFFT_EINVAL otherwise): N a power of two in [2, 2^30];
 * B a power of two in [2, min(N, 16384)]; w a multiple of B in [B, N];
 * 1 <= L <= 32; 1 <= K <= min(N, 16384); c >= 1; 1 <= T <= L.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFFT_OK = 0,
    SFFT_EINVAL = 1,    /* invalid argument or size */
    SFFT_ENOMEM = 2,    /* device or host allocation failed */
    SFFT_ECUDA = 3,     /* a CUDA runtime call failed (see sfft_last_error) */
    SFFT_EBUSY = 4,     /* admission refused: server budget or slots exhausted */
    SFFT_ETIMEDOUT = 5, /* a bounded wait expired */
    SFFT_EPENDING = 6,  /* request not finished yet (sfft_poll) */
    SFFT_ENOTIMPL = 7   /* option not implemented in this build */
} sfft_status;

typedef struct sfft_plan sfft_plan;
typedef struct sfft_server sfft_server;

/* Plan options.  Zero-initialised fields take the defaults listed. */
typedef struct {
    int32_t c;         /* buckets kept per loop = min(c*K, B); 0 -> 2 ("2K large buckets") */
    int32_t T;         /* vote threshold; 0 -> ceil(L/2) */
    int32_t precision; /* B-point transform (a2): 0 -> FP32 radix-2 FFT; 1 -> split-BF16 DFT on the
                          tensor cores (voting and comb methods, 64 <= B <= 4096; see below) */
    int32_t method;    /* SFFT_METHOD_VOTING (0, default), SFFT_METHOD_PHASE, SFFT_METHOD_COMB or
                          SFFT_METHOD_SEARCH */
    int32_t comb;      /* SFFT_METHOD_COMB: residue classes Bc (power of two); 0 -> default
                          min(2^ceil(log2(16 c K)), 8192, N, 32 N / B for 32 <= B <= 512) */
    int32_t estimator; /* SFFT_ESTIMATOR_MEDIAN (0, default) or SFFT_ESTIMATOR_MEAN (voting
                          and comb methods) */
    int32_t refine;    /* iterative-framework refinement passes over the found set, 0..8
                          (0, default: none; voting and comb methods, K <= 4096) */
    int32_t search_bits; /* SFFT_METHOD_SEARCH: bits per search digit, 1..4; 0 -> 1 (binary
                            search); b > 1: multi-scale search with l = 2^b */
    int32_t residual;  /* 1: final residual-energy check in FP64 after the output (voting and
                          comb methods; 4 <= B <= 8192), read with sfft_plan_last_stats;
                          0 (default): none */
    int32_t mode;      /* how step a1 reads the signal: SFFT_GATHER_AUTO (0, default),
                          SFFT_GATHER_PERMUTED or SFFT_GATHER_STREAM (see below) */
} sfft_opts;

/* Location methods.
   SFFT_METHOD_VOTING: L loops of flat-window bucketization, top-2K buckets,
     voting, median estimate ("Method of probability and statistics", sFFT1.0).
   SFFT_METHOD_PHASE: iterative framework with phase-encoding location
     ("Phase encoding method", "The iterative framework"; Table 1, sFFT3.0):
     up to L iterations, each bucketizing the signal at shifts tau and tau+1
     under a new permutation, subtracting the coefficients found so far, and
     reading every bucket above 1e-6 of iteration 0's largest bucket energy as
     a lone coefficient at f = arg(zhat' / zhat) N / 2 pi (kept when f hashes
     back to the bucket), valued by energy concentration.  For exactly sparse
     signals (Table 2: robustness "none"); c and T are ignored. */
#define SFFT_METHOD_VOTING 0
#define SFFT_METHOD_PHASE 1
/* SFFT_METHOD_COMB: voting behind the spike-train pre-filter (sFFT2.0-style;
   Eq. 10, 15-16; Table 1 sFFT2.0): two subsamplings of the signal at stride
   N/Bc (shifts tau of loops L and L+1) alias it into Bc residue classes;
   their energies keep the min(cK, Bc) largest classes, and only frequencies
   of kept classes are voted on, estimated and output (L <= 30). */
#define SFFT_METHOD_COMB 2

/* SFFT_METHOD_SEARCH: location by binary or multi-scale search (sFFT4.0 /
   MPFFT-style; "The method of binary search or multi-scale search"; Table 1)
   in the iterative framework of SFFT_METHOD_PHASE (L = iterations; found
   coefficients subtracted before each bucketization; top K of the found
   set; threshold: the larger of 1e-6 of the largest and 20 times the median
   bucket energy of iteration 0, so that a noisy signal stops once nothing
   above its noise floor remains).  Iteration
   r bucketizes the signal at the shifts tau_r + N / 2^m, m = b, 2b, ..., up
   to bits = min(log2(N/B) + 1, log2 N) (b = search_bits), besides tau_r: a
   coefficient f turns by exp(2 pi i f / 2^m) at shift N / 2^m, so each
   shifted bucket decides one digit of f (the candidate whose predicted turn
   best matches; candidates lie 1/2^b of a turn apart); the bits fix
   sigma f to one value in a window of two buckets around the bucket.  A
   located f is kept when it hashes back to the bucket and every shifted
   bucket matches the lone-coefficient prediction within a residual of 1/4
   of its energy, valued by energy estimation.  More robust to noise than
   phase encoding (whose one-sample phase must resolve f to 1 of N); needs
   1 + ceil(bits / b) bucketizations per iteration, whose buffers and the
   top-K ranks must fit one CTA's shared memory (160 KB); c and T are
   ignored. */
#define SFFT_METHOD_SEARCH 3

/* Combination of a candidate's L per-loop estimates (step a6; "The method of
   estimating the value").  MEDIAN: the coordinate-wise median, robust to
   collisions in a minority of loops; candidates whose median cannot reach the
   top K are pruned exactly before they are estimated.  MEAN: the average of
   the L estimates (the paper's remark that averaging several buckets is more
   accurate): lower variance under noise, but a collision in one loop biases
   it by 1/L of the colliding coefficient, and no bound on a mean prunes the
   candidates, so every candidate is estimated (slower). */
#define SFFT_ESTIMATOR_MEDIAN 0
#define SFFT_ESTIMATOR_MEAN 1

/* sfft_opts.mode: how the bucketization (step a1, "The analysis of
   bucketization through the flat filter") reads the signal; both give the
   same bucket sums up to FP32 rounding order.
   PERMUTED: each window tap reads its sample at the permuted position
     (sigma m + tau) mod N, one 8-byte read (a 32-byte sector) per tap: L w
     reads per signal, the whole signal from DRAM when L w >~ N/4.
   STREAM: the signal is read once, in order (8 N bytes, coalesced); per
     loop, one thread per segment visits the samples the window reads in
     sample order through the three-gap return map of the permutation
     (sfft_window_walk), and the taps are added into shared-memory bins
     (FP32 atomics: the order of the additions, hence the last bits, may
     differ from run to run).  Voting and comb methods, N >= 2^12,
     B <= 4096; plans with L B > 6144 take their loops in groups, each
     reading the signal again (mostly from L2).  Keeps a table of 4 L
     N / seglen bytes (segment starts, seglen = N / (8 V nclu)).
   AUTO: the permuted gather, which measured faster on GB300 at every size
   tried (N = 2^14 .. 2^26; 3.6x at N = 2^20, B = 512): its reads are L2
   hits for signals within L2, and where the window is sparse its sector
   traffic is below 8 N bytes, while the stream gather pays a few shared-
   memory operations per tap. */
#define SFFT_GATHER_AUTO 0
#define SFFT_GATHER_PERMUTED 1
#define SFFT_GATHER_STREAM 2

/* sfft_opts.refine > 0: after the top K, the iterative framework's
   subtraction ("Four algorithmic frameworks") refines the K output values.
   Each pass re-estimates every found coefficient f in every loop from its
   bucket after subtracting the other found coefficients that hash to the same
   or a neighbouring bucket (by the bucket identity with the filter's gain;
   further out the gain is below the flat window's stop-band floor), using the
   previous pass's values, and combines the L estimates by the plan's
   estimator.  The support is not changed.  Removes the collision bias that
   the mean estimator otherwise carries. */
#define SFFT_MAX_REFINE 8

/* sfft_opts.precision = 1: the B-point DFT of step a2 (Eq. 2) as a matrix
   product on the tensor cores.  Every (signal, loop) row of bucket sums z
   (interleaved re, im) is multiplied by the real 2B x 2B DFT matrix W
   (cos / sin of 2 pi j k / B); z and W are split into BF16 hi and lo parts and
   zhat = z_hi W_hi + z_lo W_hi + z_hi W_lo with FP32 accumulation (the
   dropped z_lo W_lo is ~2^-16 of the result): relative error ~1e-5, within
   the 1e-3 tolerance stated for it.  The rows of a batch that share B form
   one GEMM.  The W table (16 B^2 bytes) is built once per device and B. */

/* sfft_opts.residual = 1: the final residual-energy check (the error that
   Eq. 5 bounds, seen through the buckets).  After the output (and any
   refinement) the k_out recovered coefficients are subtracted in FP64 from
   the L loops' bucket values by the bucket identity
       zhat_l[k] = sum_f xhat_f exp(+2 pi i tau_l f / N) G~(sigma_l f - k N/B)
   (each coefficient from its own and both neighbouring buckets; further out
   the flat window's gain is below 1e-7 of its passband), and the energy left,
   sum_l sum_k |residual_l[k]|^2, is reported beside the buckets' energy
   sum_l sum_k |zhat_l[k]|^2 (sfft_exec_stats).  A small ratio says the output
   explains the buckets; a planted miss or a wrong value leaves that
   coefficient's bucket energy. */

/* Read-only description of a plan (host struct filled by sfft_plan_get_info). */
typedef struct {
    int64_t N, w;
    int32_t K, B, L, c, T, nsel; /* nsel = min(c*K, B) */
    uint64_t seed;
    int64_t samples_touched;     /* distinct sample indices read per execute (Table 2; counted
                                    on the host at the first sfft_plan_get_info of a seed) */
    int64_t candidate_capacity;  /* min(N, (L-T+1)*nsel*N/B): bound on the candidate set */
    size_t device_bytes;         /* device memory held by the plan itself (its scratch; the
                                    tables it shares with plans of the same N, B, w are apart) */
    int32_t method;              /* SFFT_METHOD_* */
    int32_t estimator;           /* SFFT_ESTIMATOR_* */
    int32_t refine;              /* refinement passes */
} sfft_plan_info;

/* ------------------------------------------------------------------ plans */

/* Create a plan: validates sizes, derives sigma_l, tau_l (a0), and allocates
   scratch on the current CUDA device.  The seed-independent tables (window
   taps, gain tables, FFT twiddles; a0') are computed on the GPU in FP64 for
   the first plan of each (device, N, B, w) and shared, reference-counted, by
   every later plan of that shape (kept for reuse after their last plan goes).
   *plan is NULL on failure.  Blocks until its set-up (and any table build)
   has finished.  Errors: SFFT_EINVAL, SFFT_ENOMEM, SFFT_ECUDA. */
sfft_status sfft_plan_create(sfft_plan **plan, int64_t N, int32_t K, int32_t B, int64_t w,
                             int32_t L, uint64_t seed);

/* As sfft_plan_create with explicit options (opts may be NULL). */
sfft_status sfft_plan_create_ex(sfft_plan **plan, int64_t N, int32_t K, int32_t B, int64_t w,
                                int32_t L, uint64_t seed, const sfft_opts *opts);

/* Release a plan and its device memory (NULL is a no-op).  The caller must
   ensure no enqueued work still uses it. */
void sfft_plan_destroy(sfft_plan *plan);

/* Re-draw the plan's loop parameters for another seed (a0; the scratch and
   the shared tables stay): sigma_l, tau_l as sfft_plan_create would draw them
   for `seed`, uploaded on `stream`, so work enqueued on that stream afterwards
   uses them (cached batch graphs of the plan stay valid).  The caller must
   ensure no work of the plan is in flight on another stream.  Errors:
   SFFT_EINVAL, SFFT_ECUDA. */
sfft_status sfft_plan_reseed(sfft_plan *plan, uint64_t seed, void *stream);

sfft_status sfft_plan_get_info(const sfft_plan *plan, sfft_plan_info *info);

/* Copy the L loop parameters (host arrays of length L; any may be NULL):
   sigma (odd), tau, and sigma^-1 mod N.  Pure host call. */
sfft_status sfft_plan_get_loops(const sfft_plan *plan, uint32_t *sigma, uint32_t *tau,
                                uint32_t *sigma_inv);

/* Counters of the plan's most recent execution (host struct).  Reads device
   memory synchronously: call after the stream that ran the plan has reached
   the end of that execution. */
typedef struct {
    int64_t candidates;  /* |{f : votes >= T}| when the fallback pass ran (it counts
                            them); -1 otherwise (then at least K exist) */
    int64_t estimated;   /* frequencies the median bound could not exclude */
    int64_t recorded;    /* estimates kept for the top-K (candidates, key >= theta) */
    int32_t fallback;    /* 1 if the unpruned pass ran (fewer than K recorded) */
    float theta;         /* prune threshold: 1/4 of the K-th largest bucket energy
                            (phase encoding: the bucket-energy threshold) */
    int32_t iterations;  /* phase encoding: iterations run; voting: L */
    double residual_energy;  /* sfft_opts.residual: energy left in the buckets after
                                subtracting the output (FP64); else -1 */
    double bucket_energy;    /* sfft_opts.residual: energy of the buckets (FP64); else -1 */
    int32_t device_error;    /* 0, or the code of a bounded device-side wait that gave up
                                (tensor-core DFT: 1 operand load, 2 accumulator) */
} sfft_exec_stats;

sfft_status sfft_plan_last_stats(const sfft_plan *plan, sfft_exec_stats *stats);

/* Loop parameters without a plan (host only, no GPU needed): block
   Philox4x64-10(counter = (l,0,0,0), key = (seed,0)) gives words r0, r1;
   sigma_l = 2 (r0 mod N/2) + 1, tau_l = r1 mod N.  Errors: SFFT_EINVAL. */
sfft_status sfft_loop_params(int64_t N, int32_t L, uint64_t seed, uint32_t *sigma, uint32_t *tau,
                             uint32_t *sigma_inv);

/* Plan sizes for a signal shape (host only, no GPU needed).  When a loaded
   tuning cache (sfft_tuning_load) has a class covering (log2 N, K, SNR), its
   measured choice is used: B = the smallest power of two >= B_per_K K
   (bounded as below), w = B (log2 N + w_extra), its L.  Otherwise the fixed
   size-class rule:
     B = the smallest power of two >= max(64, 4K) (so the 2K kept buckets
         are at most half of them), at most min(16384, N/64) (which keeps the
         window inside the signal) and at least 2; a cap below 2K is refused
         (SFFT_EINVAL): the rule plans K <= min(8192, N/128) only;
     w = B (log2 N + 21) (the flat window's width; Eq. 13's Gaussian at
         sigma_g = B sqrt(log2 N) falls below its stop-band floor at its edge),
         lowered to the largest multiple of B <= N;
     L = 8 for a noiseless signal (snr_db NaN: exactly sparse) and 12 else.
   The rule gives the named workloads' B (K = 10: 64; K = 100: 512;
   K = 1000: 4096).  Errors: SFFT_EINVAL (N not a power of two in
   [2, 2^30], K not in [1, N], K beyond the rule's range, NULL outputs). */
sfft_status sfft_suggest_params(int64_t N, int32_t K, double snr_db, int32_t *B, int64_t *w, int32_t *L);

/* Sampling geometry of one loop of the stream gather (host only; for tests
   and tools).  The loop with permutation (sigma odd, tau) reads sample p with
   window tap q(p) = (sigma^-1 (p - tau) + floor(w/2)) mod N whenever
   q(p) < w (2 <= w <= N, N a power of two in [2, 2^30], p0 < N).  out[0]:
   the first sample p >= p0 the loop reads (cyclically, mod N); out[1]: its
   tap; out[2..5]: the return map {k+, alpha, k-, beta} (three-distance
   theorem): after the read with tap q the next read is p + k+ (tap
   q + alpha) if q + alpha < w, else p + k- (tap q - beta) if q >= beta,
   else p + k+ + k- (tap q + alpha - beta).  SFFT_EINVAL on bad arguments. */
sfft_status sfft_window_walk(int64_t N, int64_t w, uint64_t sigma, uint64_t tau, int64_t p0, int64_t out[6]);

/* Load the autotuner's cache (JSON written by paper_2012_08238_gb300/tune.py,
   which measures per size class the fastest B/K ratio, window width and L
   whose L1 error and support recall match the fixed rule's):
     {"version": 1, "classes": [{"logN": n, "K_lo": a, "K_hi": b, "snr_lo": s0,
       "snr_hi": s1, "B_per_K": r, "w_extra": e, "L": l, ...}, ...]}
   A class covers N = 2^n, a <= K <= b and s0 <= SNR < s1 (snr_lo null: the
   noiseless class).  Replaces any loaded classes (process-wide; host only).
   Errors: SFFT_EINVAL (unreadable file, malformed JSON, values out of range;
   the previously loaded classes stay). */
sfft_status sfft_tuning_load(const char *path);
/* Forget the loaded classes (the fixed rule applies again). */
void sfft_tuning_clear(void);
/* Number of loaded classes. */
int32_t sfft_tuning_classes(void);

/* ---------------------------------------------------------------- execute */

/* Whole hot path a1..a7 on one signal.
   x_dev:     complex64[N], device.
   idx_dev:   int32[K], device; the k_out recovered frequencies, ascending;
              entries past k_out are left untouched.
   val_dev:   complex64[K], device; estimates of xhat_f (Eq. 2 scale).
   k_out_dev: int32[1], device; k_out = min(K, number of candidates).
   Errors: SFFT_EINVAL (NULL pointer), SFFT_ECUDA (launch failure). */
sfft_status sfft_execute(sfft_plan *plan, const float *x_dev, int32_t *idx_dev, float *val_dev,
                         int32_t *k_out_dev, void *stream);

/* The same with HOST buffers: copies x_host (complex64[N]) to a device buffer
   owned by the plan, executes, copies the outputs back and synchronises the
   stream.  Pinned host memory gives the fastest copies. */
sfft_status sfft_execute_host(sfft_plan *plan, const float *x_host, int32_t *idx_host,
                              float *val_host, int32_t *k_out_host, void *stream);

/* Many signals in one pass: every stage is one launch over all `count` jobs
   (plans may differ in N, K, B, w, L).  Arrays have `count` entries; plans
   must be distinct (each owns its scratch).  k_out_dev is int32[count] on the
   device.  A job list seen before replays a cached CUDA graph.
   Errors: SFFT_EINVAL, SFFT_ENOMEM, SFFT_ECUDA. */
sfft_status sfft_execute_batch(sfft_plan *const *plans, const float *const *x_dev,
                               int32_t *const *idx_dev, float *const *val_dev, int32_t *k_out_dev,
                               int32_t count, void *stream);

/* Measurement form of sfft_execute_batch: enqueues `steps` back-to-back runs
   of the batch on `stream` (no graph) with CUDA events recorded on that
   stream around each of its six stages (gather-fold, FFT+select, vote scan,
   survivor estimate, refinement, residual check; the top-K and any fallback
   pass run in the last estimate CTA of each job, so the fourth stage holds
   them; the fifth holds the refinement passes of plans with
   sfft_opts.refine > 0 and the sixth the residual check of plans with
   sfft_opts.residual, else they are empty), waits for the last
   one, and returns the device time from the first event to the last
   (*total_ms) and the summed time of each stage over all steps
   (stage_ms[6]).  Errors as for sfft_execute_batch. */
sfft_status sfft_execute_batch_timed(sfft_plan *const *plans, const float *const *x_dev,
                                     int32_t *const *idx_dev, float *const *val_dev,
                                     int32_t *k_out_dev, int32_t count, int32_t steps,
                                     float *total_ms, float *stage_ms, void *stream);

/* Batch with HOST buffers: copies each x_host[i] (complex64[N_i]) into a
   device buffer owned by plans[i] (on an internal copy stream, in up to 8
   chunks of jobs; each chunk's batch runs on `stream` once its copies have
   landed, beside the next chunk's copies), copies idx/val/k_out back to the
   host arrays (k_out_host int32[count]) with one device-to-host copy, and
   synchronises the stream.  Pinned host memory gives the full link rate. */
sfft_status sfft_execute_batch_host(sfft_plan *const *plans, const float *const *x_host,
                                    int32_t *const *idx_host, float *const *val_host,
                                    int32_t *k_out_host, int32_t count, void *stream);

/* ------------------------------------------------- single stages (tests) */
/* Each runs one step on caller buffers; the plan's scratch is used for the
   rest.  They exist so that every kernel can be checked on its own. */

/* a1+a2: zhat_dev = complex64[L][B], bucket values of every loop. */
sfft_status sfft_bucketize(sfft_plan *plan, const float *x_dev, float *zhat_dev, void *stream);

/* a3: sel_dev = int32[L][nsel], per loop the kept buckets in rank order
   (energy descending, ties to the lower bucket); zhat_dev as above. */
sfft_status sfft_select(sfft_plan *plan, const float *zhat_dev, int32_t *sel_dev, void *stream);

/* a4+a5: candidates {f : votes >= T} from the kept buckets sel_dev
   (int32[L][nsel]); cand_dev int32[cap] receives them in no particular
   order and n_cand_dev int32[1] their count.  The count never exceeds
   candidate_capacity; cap must be at least that (SFFT_EINVAL otherwise). */
sfft_status sfft_vote(sfft_plan *plan, const int32_t *sel_dev, int32_t *cand_dev,
                      int32_t *n_cand_dev, int64_t cap, void *stream);

/* a6: est_dev complex64[n_cand] = median estimates of the n_cand frequencies
   cand_dev (any order) from bucket values zhat_dev (complex64[L][B]). */
sfft_status sfft_estimate(sfft_plan *plan, const float *zhat_dev, const int32_t *cand_dev,
                          int64_t n_cand, float *est_dev, void *stream);

/* Bucket values (a1+a2, same output as sfft_bucketize) for callers that
   cannot allocate device memory.  The paper has no counterpart: this exists
   for processes whose device memory belongs to another allocator (a
   framework's caching pool, a fixed arena reserved at start-up) or whose
   steady state cannot afford an allocation that may block, and which
   therefore cannot create a plan.  Takes the plan sizes and seed directly;
   x_dev complex64[N] and zhat_dev complex64[L][B] are the caller's device
   buffers.  Calls no cudaMalloc/cudaFree and no allocating library routine:
   its only scratch is a 2 MiB array in the library's static device memory
   (2^18 complex64 partial sums; every device that loads the library holds
   it until the process exits).  Sizes as for plans, plus L*B <= 262144
   (SFFT_EINVAL otherwise, with the reason in sfft_last_error).  The first
   call on each device looks up that array's device address; make that first
   call before any stream capture.  All calls share the array: calls whose
   work overlaps on the GPU (different streams, different host threads) race
   and must be serialised by the caller.  Every scratch entry a call reads
   is written earlier in the same call, so no clearing is needed. */
sfft_status sfft_bucketize_noalloc(int64_t N, int32_t B, int64_t w, int32_t L, uint64_t seed,
                                   const float *x_dev, float *zhat_dev, void *stream);

/* ---------------------------------------------------------------- serving */

typedef struct {
    int64_t N, w;
    int32_t K, B, L;
    uint64_t seed;
    sfft_opts opts;        /* zero -> defaults */
    const float *x_dev;    /* complex64[N], device, caller-owned, valid until done */
    int32_t *idx_dev;      /* int32[K], device */
    float *val_dev;        /* complex64[K], device */
    int32_t count_samples; /* 1: sfft_result.samples_touched is counted (O(L w) host work
                              on the thread that takes the result); 0: it is -1 */
} sfft_request;

typedef struct {
    int32_t k_out;          /* number of frequencies written */
    int32_t status;         /* sfft_status of the request */
    int64_t samples_touched;
    int64_t latency_ns;     /* submit -> completion observed by the server */
} sfft_result;

/* Start a serving loop on the current device: a host thread admits submitted
   requests while their plans fit in hbm_budget_bytes and at most max_slots
   are in flight, batches whatever is admitted (one location method per
   batch), and launches it while earlier batches still run (continuous
   batching: requests arriving meanwhile join the next batch).  Plans are
   cached by shape (N, B, w, L, options and, for voting, K rounded up to a
   power of two) and rebound to each request's own K and seed, so distinct
   seeds reuse them; a shape without an idle plan is built by a second host
   thread while admission goes on, and idle plans are evicted least recently
   used to fit the budget.  max_slots = 1 serves one request at a time (the
   plain per-signal path through the same machinery). */
sfft_status sfft_server_create(sfft_server **srv, size_t hbm_budget_bytes, int32_t max_slots);

/* Queue one request; *ticket identifies it.  SFFT_EBUSY if its plan alone
   exceeds the budget; SFFT_EINVAL for bad sizes. */
sfft_status sfft_submit(sfft_server *srv, const sfft_request *req, uint64_t *ticket);

/* SFFT_EPENDING until the request has finished, then SFFT_OK (result filled;
   the ticket is released) or the request's error. */
sfft_status sfft_poll(sfft_server *srv, uint64_t ticket, sfft_result *result);

/* Block until the ticket finishes or timeout_ms passes (SFFT_ETIMEDOUT). */
sfft_status sfft_wait(sfft_server *srv, uint64_t ticket, int64_t timeout_ms, sfft_result *result);

/* Pause (paused != 0) or resume admission: paused requests stay queued.
   Used to drain a server or to hold requests back deliberately. */
sfft_status sfft_server_set_paused(sfft_server *srv, int32_t paused);

/* Drain outstanding work and stop the loop (NULL is a no-op). */
void sfft_server_destroy(sfft_server *srv);

/* ------------------------------------------------------------------ misc */
const char *sfft_status_string(sfft_status s);
/* Reason for the calling thread's most recent failure ("" if none). */
const char *sfft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H */
