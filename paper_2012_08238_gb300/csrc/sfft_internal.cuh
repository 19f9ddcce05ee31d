// Internal declarations of the CUDA sparse-FFT library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sfft.h"

namespace sfft {

constexpr int kMaxL = 32;
constexpr int kMaxB = 16384;
constexpr int kMaxK = 16384;
constexpr int kMaxLogN = 30;
constexpr int kFlagsSmemBytes = 96 * 1024;
constexpr int kClusterMaxB = 16384;    // clustered FFT/select up to this B (when a cluster of L fits)
constexpr uint32_t kMethodVoting = 0;  // sFFT1.0-style voting (the default)
constexpr uint32_t kMethodPhase = 1;   // sFFT3.0-style phase encoding, iterative framework
constexpr uint32_t kPeSmemFound = 2048;  // phase encoding: found lists up to this size live in shared memory
constexpr uint32_t kMethodComb = 2;     // voting behind the spike-train pre-filter
constexpr uint32_t kMethodSearch = 3;   // sFFT4.0 / MPFFT-style location by binary or multi-scale search
constexpr float kSearchRho = 0.25f;     // search: residual bound of a lone coefficient (relative)
constexpr float kSearchKappa = 20.0f;   // search: threshold at least this many median bucket energies
constexpr uint32_t kSearchSmemMax = 160 * 1024;  // search: bucket buffers of one job in shared memory
constexpr uint32_t kCombShifts = 2;     // comb subsamplings (shifts tau of loops L, L+1)
constexpr uint32_t kMaxComb = 8192;     // largest number of residue classes
constexpr uint32_t kEstMedian = 0;      // a6: coordinate-wise median of the per-loop estimates
constexpr uint32_t kEstMean = 1;        // a6: their mean (every candidate estimated)
constexpr uint32_t kRefineMaxK = 4096;  // refinement: the found set lives in shared memory
constexpr int kVoteTileF = 4096;        // frequencies per vote tile (= survivor queue capacity)
constexpr int kEstimateCtas = 64;       // most CTAs per job of the survivor-estimate kernels
constexpr uint32_t kDynMaxJobs = 2048;  // groups of at most this many jobs share survivor chunks dynamically
constexpr int kEstTabCtasPerSm = 3;     // resident staged-table estimate CTAs per SM (72 KB each)
constexpr int kEstSurvCtasPerSm = 4;    // resident estimate CTAs per SM with the tables in L2 (64 registers)
constexpr uint32_t kEstTabMaxBytes = 72 * 1024;  // staged estimate tables: up to 3 CTAs per SM
constexpr uint32_t kResidualMaxB = 8192;  // residual check: a loop's B residuals (FP64) in shared memory
constexpr uint32_t kDftMaxB = 4096;       // split-BF16 tensor-core DFT: B in [64, 4096]
constexpr uint32_t kDftRowTile = 128;     // its GEMM's row tile (rows padded to a multiple)
constexpr uint32_t kGatherPermuted = 0;   // a1 read at the permuted positions, sample by sample
constexpr uint32_t kGatherStream = 1;     // a1 read once in sample order (stream gather)
constexpr uint32_t kStreamCluster = 8;    // stream gather: CTAs per cluster (bins summed through DSMEM)
constexpr uint32_t kStreamStages = 4;     // stream gather: cp.async ring depth
constexpr uint32_t kStreamStageSamples = 2048;  // stream gather: samples per stage (V pieces)
constexpr uint32_t kStreamBins = 6144;    // stream gather: L B bins of one loop group (48 KB)
constexpr uint32_t kStreamMinLogN = 12;   // stream gather: N >= 2^12

// Shared-memory bytes of a job's staged estimate tables: zhat (L B complex),
// 1/G~ (N/B complex), kept bits (L B / 8 bytes); 0 when B < 32 (whole bit words).
inline uint32_t estimate_tab_bytes(uint64_t N, uint32_t B, uint32_t L) {
    if (B < 32) return 0;
    const uint64_t b = 8ull * L * B + 8ull * (N / B) + (uint64_t)L * B / 8;
    return b <= kEstTabMaxBytes ? (uint32_t)((b + 15) / 16 * 16) : 0;
}

// Per-plan counters in device memory (uint32 slots).
enum Counter : int {
    kNCand = 0,    // candidates (score >= T), counted by the fallback pass only
    kNSurv = 1,    // survivors of the median bound listed by the pruned scan
    kNGe = 2,      // their estimates with key >= theta (records of the pruned pass)
    kSelDone = 4,  // loops finished by the FFT/select kernel (last-block pattern)
    kTheta = 5,    // prune threshold theta (float bits)
    kErr = 6,      // device-side error word (0 = none)
    kNRec2 = 7,    // records written by the unpruned fallback pass (in the top-K step)
    kEstDone = 8,  // estimate CTAs of the job finished (last-CTA ticket for the top-K step)
    kPeIter = 10,  // phase encoding: iterations run
    kFbPend = 11,  // 1 when the job's pruned records could not certify the top K (fallback pass due)
    kFbDone = 12,  // fallback CTAs of the job finished (last-CTA ticket for its top-K step)
    kNumCounters = 16
};

// Everything a kernel needs to know about one plan; lives in device memory and
// is copied into shared memory by every CTA that works on the plan.
struct PlanDev {
    uint32_t N, mask, logN;
    uint32_t B, logB;
    uint32_t shift;   // log2(N/B)
    uint32_t half;    // (N/B)/2 : round-half-up offset of the hash
    uint32_t w, halfw;
    uint32_t L, K, Kl;  // Kl = min(K, B)
    uint32_t nsel, T, M;  // M = ceil(L/2): strong loops needed by the median bound
    uint32_t nchunk, rounds, rpc, tb, tiles;  // gather decomposition
    uint32_t vtiles;                          // vote tiles per job (<= kVoteTileF frequencies each)
    uint32_t use_bits;                        // register-table scan (32 <= B <= 4096, B <= 512 for comb; T = M for the mean)
    uint32_t cap;                             // candidate capacity
    float ginv2max;                           // max_o |1/G~(o)|^2 (rounded up)
    uint32_t method;                          // kMethodVoting, kMethodPhase, kMethodComb or kMethodSearch
    uint32_t srch_b;                          // search: bits per digit (1: binary search)
    uint32_t Bc, logBc, ncls;                 // comb: residue classes, kept classes
    uint32_t estimator;                       // kEstMedian or kEstMean
    uint32_t refine;                          // refinement passes (0: none)
    uint32_t residual;                        // final residual-energy check (0: none)
    uint32_t precision;                       // 0: FP32 radix-2 FFT; 1: split-BF16 tensor-core DFT
    uint32_t gmode;                           // a1: kGatherPermuted or kGatherStream
    // stream gather: loops per CTA group, loop groups, walkers (segments) per
    // loop and CTA, samples per stage piece, log2 segment length, clusters
    // per loop group (= nchunk)
    uint32_t slg, sgrp, sV, spiece, sseg, snclu;
    uint32_t sigma[kMaxL], tau[kMaxL];
    const float *taps;     // [w]
    const float2 *tw;      // [B/2] exp(-2 pi i k / B)
    const float2 *twst;    // [B - 1] by FFT stage: exp(-2 pi i k / (2h)) at h - 1 + k, k < h
    const float2 *ginv;    // [N/B] 1 / G~(o), o + half
    const float2 *gext;    // phase encoding, refinement: [3N/B] G~(nu) for nu + 3N/2B in [0, 3N/B)
    const float2 *ctw;     // comb: [Bc/2] exp(-2 pi i k / Bc)
    uint32_t *cls;         // comb: [ncls] kept residue classes, ascending
    uint32_t *keptc;       // comb: [Bc/32] kept-class bitmap
    float2 *partial;       // [nchunk][L][B]
    float2 *zhat;          // [L][B]
    float *energy;         // [L][B]
    float *loopkth;        // [L] ceil(K/L)-th largest energy of each loop
    uint32_t *packed;      // [L][E][32]: lane j's strong bits, kept bits for the mean (register-table scan;
                           // E = B/1024 words per lane for B >= 1024, else 1)
    int32_t *sel;          // [L][nsel]
    uint16_t *flags;       // [L][B]: 1 = kept, +256 = strong
    uint32_t *bits2;       // [L][B/16]: the same as 2 bits per bucket (kept, strong), when the
                           // u16 table exceeds the scan's shared memory (else NULL)
    uint32_t *survf;       // [N] with use_bits (survivors of the median bound), else [cap] (candidates)
    uint4 *surv;           // [cap] records {f, key bits, re bits, im bits}
    float2 *rscr;          // refinement: [K][L] per-loop estimates of a pass
    const double2 *gext64; // residual check: [3N/B] G~(nu) in FP64, as gext
    double *resid;         // residual check: [L][2] energy left, bucket energy per loop
    const uint4 *walk;     // stream gather: [L] return map {k+, alpha, k-, beta} (walk.cuh)
    uint32_t *wq;          // stream gather: [L][N >> sseg] tap of each segment's first read
    uint32_t *ctr;         // [kNumCounters]
};

// One signal of a launch: which plan, which input, where the outputs go.
struct Job {
    const PlanDev *p;
    const float2 *x;
    int32_t *idx;
    float2 *val;
    int32_t *kout;
    uint32_t rpc, nchunk;  // gather split of this launch: rounds per chunk, chunks (<= plan's nchunk)
    uint32_t vctas;        // pruned-scan CTAs of this job (each takes every vctas-th vote tile)
    uint32_t ectas;        // survivor-estimate CTAs of this job
};

// Launch descriptor shared by all stage kernels: either one job passed by
// value, or `njobs` jobs in device memory with, per kernel, a CTA-offset
// prefix and a CTA -> job map.
struct Launch {
    const Job *jobs;        // nullptr -> use `one`
    const uint32_t *offs;   // [njobs + 1] CTA prefix for this kernel (batch only)
    const uint32_t *map;    // [total CTAs] job of each CTA (batch only)
    int njobs;
    uint32_t cta0;          // batch: CTA of the map that this launch's block 0 is (a group's first)
    uint32_t *gctr;         // batch group (estimate, fallback): 8 words, zero between launches:
                            // the estimate's {next chunk, finished CTAs}, the fallback's, and
                            // the count of jobs flagged for the fallback (nullptr: static shares)
    Job one;
};

enum VoteMode : int { kVotePrune = 0, kVoteCandidates = 2 };

// ---------------------------------------------------------------- host side
void set_error(const std::string &msg);
sfft_status cuda_fail(cudaError_t e, const char *what);
// Plan creation with scratch for up to K_cap output coefficients (K <= K_cap;
// K_cap != K only for the voting method), and the rebinding of an idle plan
// to another K <= K_cap and seed on stream s (api.cu).
sfft_status plan_create(sfft_plan **plan, int64_t N, int32_t K, int32_t K_cap, int64_t B, int64_t w, int32_t L,
                        uint64_t seed, const sfft_opts *opts);
sfft_status plan_rebind(sfft_plan *p, int32_t K, uint64_t seed, cudaStream_t s);
// The loaded tuning class of a signal shape (tuning.cu): B = pow2 >= B_per_K K,
// w = B (log2 N + w_extra), L.  False when no class covers it.
bool tuning_lookup(int logN, int64_t K, double snr_db, int64_t *B_per_K, int64_t *w_extra, int32_t *L);
// Distinct samples a plan of these sizes, options and seed reads (host count).
int64_t samples_touched_of(int64_t N, int32_t B, int64_t w, int32_t L, uint64_t seed, const sfft_opts &o);

// Kernel launchers (stream-ordered, no synchronisation).
cudaError_t launch_gather(const Launch &ln, uint32_t total_ctas, cudaStream_t s);
// Stream gather (gather_stream.cu): every job has gmode = kGatherStream and
// kStreamCluster * sgrp * snclu CTAs, starting at a multiple of
// kStreamCluster; smem: the largest stream_smem_bytes of the jobs.  The
// per-plan table of segment starts is written by launch_walk_start (sinv:
// sigma_l^-1 mod N) whenever sigma, tau change.
cudaError_t launch_gather_stream(const Launch &ln, uint32_t total_ctas, uint32_t smem, cudaStream_t s);
cudaError_t launch_walk_start(const PlanDev &P, const uint32_t *sinv, cudaStream_t s);
uint32_t stream_smem_bytes(uint32_t lg, uint32_t B, uint32_t V, uint32_t piece);
// cluster_L > 0: every job has L = cluster_L and the job's CTAs form one
// thread-block cluster (fft_select_cluster_ok(cluster_L, max_B) must hold).
// dftC != NULL: the bucket values are the tensor-core DFT's partial planes
// (dft_partials) instead of gather partials + FFT; dft_err its error word.
cudaError_t launch_fft_select(const Launch &ln, uint32_t total_ctas, uint32_t max_B, int select_only,
                              uint32_t cluster_L, cudaStream_t s, const float *dftC = nullptr, uint32_t dft_mpad = 0,
                              const uint32_t *dft_err = nullptr);
// Split-BF16 tensor-core DFT (dft_tc.cu): scratch bytes for `rows` rows of B
// buckets; the W table of B (built once per device, at plan creation);
// the DFT of a group's rows (ln: the FFT/select prefix, one CTA per row) into
// the scratch's partial planes, waits bounded (error word *err).
size_t dft_scratch_bytes(uint32_t rows, uint32_t B);
sfft_status dft_table_prepare(uint32_t B);
cudaError_t launch_dft(const Launch &ln, uint32_t rows, uint32_t B, void *scratch, uint32_t *err, cudaStream_t s);
const float *dft_partials(void *scratch, uint32_t rows, uint32_t B);
// Whether clusters of L FFT/select CTAs with B <= max_B can be launched here.
bool fft_select_cluster_ok(uint32_t L, uint32_t max_B);
// The pruned scan uses the register table of strong bits when every job has
// use_bits and they share L in {8, 12, 16}.
inline bool scan_uses_bits(uint32_t L_uniform, bool bits) {
    return bits && (L_uniform == 8 || L_uniform == 12 || L_uniform == 16);
}

// L_uniform: common L of every job (0 when they differ); bits: every job has
// use_bits (the pruned scan then uses the register table of strong bits).
// max_B: the largest B of the jobs (register-table jobs of one launch share
// its number of table words per lane, B/1024 for B >= 1024).
cudaError_t launch_vote(const Launch &ln, uint32_t total_ctas, int mode, uint32_t L_uniform, bool bits,
                        uint32_t max_flags_bytes, uint32_t max_B, int32_t *cand_out, int32_t *ncand_out,
                        cudaStream_t s);
// Pruned-pass estimates, each job's Job::ectas CTAs (total_ctas in all; ln's
// prefix array must match); the job's last CTA to finish then takes the
// job's top K or flags its fallback pass.  tab_smem > 0: every job's tables
// fit that many bytes of shared memory (estimate_tab_bytes) and L is uniform
// in {8, 12, 16}; they are then staged there.
cudaError_t launch_estimate(const Launch &ln, uint32_t total_ctas, uint32_t L_uniform, uint32_t tab_smem,
                            uint32_t max_K, cudaStream_t s);
// Unpruned fallback pass of the jobs whose pruned records could not certify
// the top K (the estimate's last CTA flags them): fb_ctas(N) CTAs per job
// (ln's prefix array must match), each scanning a share of the frequencies
// and recording every candidate; the job's last one takes the top K.  CTAs
// of jobs without a pending fallback return at once.
cudaError_t launch_fallback(const Launch &ln, uint32_t total_ctas, uint32_t L_uniform, uint32_t max_K,
                            cudaStream_t s);
// CTAs per job of the fallback pass: one per 2^18 frequencies, 1..64 (few:
// most launches only read the flag).
__host__ __device__ inline uint32_t fallback_ctas(uint32_t N) {
    const uint32_t c = (N + 262143u) >> 18;
    return c < 1 ? 1u : (c > 64 ? 64u : c);
}
// Spike-train pre-filter of comb plans: one CTA per job (max_Bc: the largest
// number of residue classes).
cudaError_t launch_comb(const Launch &ln, uint32_t njobs, uint32_t max_Bc, cudaStream_t s);
// Phase-encoding variant: one CTA per job runs all its iterations and writes
// its top K.
// max_cap: the largest found-list capacity of the jobs (lists of at most
// kPeSmemFound entries stay in shared memory).
cudaError_t launch_pe(const Launch &ln, uint32_t njobs, uint32_t max_B, uint32_t max_K, uint32_t max_cap,
                      cudaStream_t s);
// Search-location variant: one CTA per job runs all its iterations (max_nbuf:
// the largest count of bucket buffers, 1 + ceil(bits / b) rounded up to even).
cudaError_t launch_bs(const Launch &ln, uint32_t njobs, uint32_t max_B, uint32_t max_K, uint32_t max_cap,
                      uint32_t max_nbuf, cudaStream_t s);
// Bucket buffers of a search plan: 1 + ceil(min(log2(N/B) + 1, log2 N) / b), rounded up to even.
inline uint32_t search_nbuf(uint32_t logN, uint32_t logB, uint32_t b) {
    const uint32_t bits = logN - logB + 1 < logN ? logN - logB + 1 : logN;
    const uint32_t S = 1 + (bits + b - 1) / b;
    return (S + 1) & ~1u;
}
// Iterative-framework refinement of the jobs' outputs: one CTA per job (ln:
// one per job) runs all the job's passes; jobs with refine = 0 return at
// once.  max_K: the largest K of the refining jobs (<= kRefineMaxK);
// L_uniform: the jobs' common L (0 when they differ).
cudaError_t launch_refine(const Launch &ln, uint32_t njobs, uint32_t max_K, uint32_t L_uniform, cudaStream_t s);
// Final residual-energy check: one CTA per (job, loop) (ln: the FFT/select
// prefix, L CTAs per job); jobs without the option return at once.  max_B:
// the largest B of the checking jobs (<= kResidualMaxB).
cudaError_t launch_residual(const Launch &ln, uint32_t total_ctas, uint32_t max_B, cudaStream_t s);
cudaError_t launch_estimate_list(const PlanDev *p, uint32_t L, const float2 *zhat, const int32_t *cand,
                                 uint32_t n, float2 *est, cudaStream_t s);
cudaError_t launch_flags_from_sel(const PlanDev *p, uint32_t L, const int32_t *sel, cudaStream_t s);

// Seed-independent tables of one (device, N, B, w), shared by plans
// (tables.cu).  gext / gext64 are NULL unless requested.
struct TableSet {
    const float *taps;      // [w]
    const float2 *tw;       // [B/2]
    const float2 *twst;     // [B - 1] the twiddles by FFT stage (PlanDev::twst)
    const float2 *ginv;     // [N/B]
    const float2 *gext;     // [3N/B] or NULL
    const double2 *gext64;  // [3N/B] or NULL
    float ginv2max;         // max_o |1/G~(o)|^2, rounded up
    size_t bytes;           // device bytes of the entry
};
// The current device's tables of this shape (built and waited for on first
// use; ext: G~ over three buckets in FP32, ext64: in FP64).  *handle is
// released by tables_release when the plan goes.
sfft_status tables_acquire(uint32_t N, uint32_t B, uint32_t w, bool ext, bool ext64, const void **handle,
                           TableSet *out);
void tables_release(const void *handle);

// Plan-time FP64 kernels (plan.cu).
// gext (phase-encoding plans, else NULL): G~ over three buckets around 0.
// gext64 (residual-checking plans, else NULL): the same three buckets in FP64.
cudaError_t plan_tables(uint32_t N, uint32_t B, uint32_t w, float *taps, float2 *tw, float2 *twst, float2 *ginv,
                        double *ginv2, float2 *gext, double2 *gext64, cudaStream_t s);
cudaError_t plan_max_bits(const double *v, uint32_t n, unsigned long long *out, cudaStream_t s);
// exp(-2 pi i k / n), k < n/2 (FP64 -> FP32)
cudaError_t plan_twiddles(uint32_t n, float2 *tw, cudaStream_t s);

}  // namespace sfft

#define SFFT_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return sfft::cuda_fail(_e, #expr); \
    } while (0)
