// Host side of the C ABI: plans, execute, batched execute with cached CUDA
// graphs, single-stage entry points, errors.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <list>
#include <mutex>
#include <string>
#include <vector>

#include "sfft_internal.cuh"
#include "walk.cuh"

struct sfft_plan {
    uint64_t id;  // unique per plan, keys the batch-graph cache
    int device;
    int64_t N, w;
    int32_t K, B, L, c, T, nsel;
    int32_t K_cap;           // largest K the scratch was sized for (>= K)
    uint64_t seed;
    uint32_t sigma_inv[sfft::kMaxL];
    mutable int64_t samples_touched;  // -1 until first asked for (host count)
    int64_t cap;
    size_t device_bytes;     // this plan's scratch (the shared tables not included)
    sfft::PlanDev h;         // host mirror of the device descriptor
    sfft::PlanDev *d;        // device descriptor
    void *dmem;              // single allocation holding the descriptor and the scratch
    const void *tables;      // shared seed-independent tables (tables_acquire)
    void *dft;               // precision 1: scratch of the tensor-core DFT of this plan's L rows
    // staging for sfft_execute_host (allocated on first use)
    void *stage;
};

namespace sfft {

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_next_id{1};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

uint32_t ilog2(uint64_t v) {
    uint32_t r = 0;
    while ((1ull << r) < v) ++r;
    return r;
}

// Philox4x64-10 block function (Salmon et al., SC'11): ten rounds of two
// 64x64->128-bit multiplies with the published multipliers, the key bumped by
// the published Weyl increments after every round.
void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * c[0];
        const unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ULL * c[2];
        const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c[1] ^ k0;
        const uint64_t n1 = (uint64_t)p1;
        const uint64_t n2 = (uint64_t)(p0 >> 64) ^ c[3] ^ k1;
        const uint64_t n3 = (uint64_t)p0;
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
}

// inverse of an odd number modulo 2^32 by Newton's iteration x <- x (2 - a x)
uint32_t inv_odd_u32(uint32_t a) {
    uint32_t x = a;  // correct to 3 bits
    for (int i = 0; i < 4; ++i) x *= 2u - a * x;
    return x;
}

void loop_params_host(int64_t N, int32_t L, uint64_t seed, uint32_t *sigma, uint32_t *tau, uint32_t *sinv) {
    const uint64_t half = (uint64_t)N / 2;
    for (int32_t l = 0; l < L; ++l) {
        uint64_t c[4] = {(uint64_t)l, 0, 0, 0};
        philox4x64_10(c, seed, 0);
        const uint32_t s = (uint32_t)(2 * (c[0] % half) + 1);
        if (sigma) sigma[l] = s;
        if (tau) tau[l] = (uint32_t)(c[1] % (uint64_t)N);
        if (sinv) sinv[l] = inv_odd_u32(s) & (uint32_t)(N - 1);
    }
}

sfft_status check_sizes(int64_t N, int32_t K, int32_t B, int64_t w, int32_t L, int32_t c, int32_t T) {
    if (!is_pow2(N) || N < 2 || N > (1ll << kMaxLogN)) {
        set_error("N must be a power of two in [2, 2^30]");
        return SFFT_EINVAL;
    }
    if (!is_pow2(B) || B < 2 || B > kMaxB || B > N) {
        set_error("B must be a power of two in [2, min(N, 16384)]");
        return SFFT_EINVAL;
    }
    if (w < B || w > N || w % B) {
        set_error("w must be a multiple of B in [B, N]");
        return SFFT_EINVAL;
    }
    if (L < 1 || L > kMaxL) {
        set_error("L must lie in [1, 32]");
        return SFFT_EINVAL;
    }
    if (K < 1 || K > kMaxK || K > N) {
        set_error("K must lie in [1, min(N, 16384)]");
        return SFFT_EINVAL;
    }
    if (c < 1 || T < 1 || T > L) {
        set_error("c must be >= 1 and T in [1, L]");
        return SFFT_EINVAL;
    }
    if (N / B > (1ll << 24) || (double)(N / B) * (double)w > 68719476736.0) {
        set_error("plan too large: N/B must be <= 2^24 and (N/B)*w <= 2^36");
        return SFFT_EINVAL;
    }
    return SFFT_OK;
}

constexpr int kNumSms = 152;  // GB300; only shapes the default work split
constexpr int kHostChunks = 8;  // host-buffer batches: copies of chunk c+1 overlap chunk c's batch
constexpr int kScanCtasPerSm = 8;  // resident 256-thread scan CTAs per SM
constexpr int kScanWaves = 1;

// Methods of the iterative framework: one CTA per job runs every iteration.
inline bool iterative(uint32_t method) { return method == kMethodPhase || method == kMethodSearch; }

// Work split of one plan for the gather and vote kernels.
void decompose(PlanDev &P) {
    P.tb = std::min<uint32_t>(P.B, 256);
    P.tiles = P.B / P.tb;
    P.rounds = P.w / P.B;
    // about one CTA per SM per signal (measured best of 76..600 at the
    // N = 2^20, B = 512, L = 12 workload: longer CTAs amortise the set-up,
    // fewer chunks leave fewer partials to sum)
    // (phase encoding and the search gather one loop per launch)
    const uint32_t loops = iterative(P.method) ? 1u : P.L;
    uint32_t want = (kNumSms + P.tiles * loops - 1) / (P.tiles * loops);
    want = std::max<uint32_t>(1, std::min<uint32_t>(want, P.rounds));
    P.rpc = (P.rounds + want - 1) / want;
    P.nchunk = (P.rounds + P.rpc - 1) / P.rpc;
    P.vtiles = (P.N + kVoteTileF - 1) / kVoteTileF;  // each tile's survivors fit the CTA's queue
    // comb: only the kept classes' N/Bc frequencies each are scanned
    if (P.method == kMethodComb)
        P.vtiles = (uint32_t)(((uint64_t)P.ncls * (P.N / P.Bc) + kVoteTileF - 1) / kVoteTileF);
    // (mean: the register table counts kept bits against M, so T must be M)
    P.use_bits = (P.B >= 32 && (P.B <= 512 || (P.B <= 4096 && P.method != kMethodComb)) &&
                  (P.estimator == kEstMedian || P.T == P.M))
                     ? 1u
                     : 0u;
    if (P.gmode == kGatherStream) {
        // stream gather: loop groups whose L B bins fit kStreamBins; walkers
        // per loop and CTA a power of two (V lg <= 256, V <= 64); CTAs of
        // min(N/8, 2^15) samples, eight per cluster, one cluster per 2^18
        // samples and loop group (a partial chunk each); V segments per CTA,
        // streamed in pieces of kStreamStageSamples / V samples
        const uint32_t lmax = std::max<uint32_t>(1, kStreamBins / P.B);
        P.sgrp = (P.L + lmax - 1) / lmax;
        P.slg = (P.L + P.sgrp - 1) / P.sgrp;
        uint32_t V = 1;
        while (V < 64 && 2 * V * P.slg <= 256) V *= 2;
        P.sV = V;
        P.snclu = std::max<uint32_t>(1, P.N >> 18);
        const uint32_t seglen = P.N / (kStreamCluster * P.snclu) / V;
        P.sseg = ilog2(seglen);
        P.spiece = std::min<uint32_t>(kStreamStageSamples / V, seglen);
        P.nchunk = P.snclu;
    }
}

// Plans whose pruned scan reads the 2-bit table: no register table, and a
// u16 table beyond the scan's shared memory.
bool needs_bits2(const PlanDev &P) {
    return !iterative(P.method) && !P.use_bits && (size_t)P.L * P.B * 2 > (size_t)kFlagsSmemBytes;
}

struct Layout {
    size_t plan, ctw, cls, keptc, part, zhat, en, lkth, topk, sel, flags, bits2, survf, surv, rscr, resid, dft, walk,
        wq, ctr, total;
};

Layout layout_of(const PlanDev &P, int64_t cap) {
    Layout o;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align256(bytes);
        return at;
    };
    const bool phase = iterative(P.method);
    // phase encoding keeps the two shifts' partials and bucket values in rows 0 and 1
    const size_t L = phase ? std::max<uint32_t>(P.L, 2) : P.L, B = P.B;
    o.plan = take(sizeof(PlanDev));
    const bool comb = P.method == kMethodComb;
    o.ctw = take(comb ? sizeof(float2) * (P.Bc / 2) : 0);
    o.cls = take(comb ? sizeof(uint32_t) * P.ncls : 0);
    o.keptc = take(comb ? sizeof(uint32_t) * ((P.Bc + 31) / 32) : 0);
    o.part = take(sizeof(float2) * P.nchunk * L * B);
    o.zhat = take(sizeof(float2) * L * B);
    o.en = take(sizeof(float) * L * B);
    o.lkth = take(sizeof(float) * L);
    o.topk = take(sizeof(uint32_t) * L * 32 * (B > 1024 ? B / 1024 : 1));
    o.sel = take(sizeof(int32_t) * L * P.nsel);
    o.flags = take(sizeof(uint16_t) * L * B);
    o.bits2 = take(needs_bits2(P) ? sizeof(uint32_t) * L * B / 16 : 0);
    // the register-table scan lists survivors of the median bound before their
    // candidacy is checked: each frequency at most once, up to N of them; the
    // other scans list candidates only (at most cap)
    o.survf = take(sizeof(uint32_t) * (P.use_bits ? (size_t)P.N : (size_t)cap));
    o.surv = take(sizeof(uint4) * (size_t)cap);
    o.rscr = take(P.refine ? sizeof(float2) * P.K * P.L : 0);
    o.resid = take(P.residual ? sizeof(double) * 2 * P.L : 0);
    o.dft = take(P.precision ? dft_scratch_bytes(P.L, P.B) + 256 : 0);  // (+ its error word)
    const bool stream = P.gmode == kGatherStream;
    o.walk = take(stream ? sizeof(uint4) * P.L : 0);
    o.wq = take(stream ? sizeof(uint32_t) * P.L * (size_t)(P.N >> P.sseg) : 0);
    o.ctr = take(sizeof(uint32_t) * kNumCounters);
    o.total = off;
    return o;
}

// Sizes and work split of a plan, without touching the device.
void fill_plan_dev(PlanDev &P, int64_t N, int32_t K, int32_t B, int64_t w, int32_t L, int32_t c, int32_t T,
                   int64_t *cap, uint32_t method, uint32_t Bc, uint32_t estimator = kEstMedian,
                   uint32_t refine = 0, uint32_t srch_b = 1, uint32_t residual = 0, uint32_t precision = 0,
                   uint32_t gmode = kGatherPermuted) {
    memset(&P, 0, sizeof(P));
    const int32_t nsel = (int32_t)std::min<int64_t>((int64_t)c * K, B);
    P.N = (uint32_t)N;
    P.mask = (uint32_t)(N - 1);
    P.logN = ilog2(N);
    P.B = (uint32_t)B;
    P.logB = ilog2(B);
    P.shift = P.logN - P.logB;
    P.half = (uint32_t)((N / B) / 2);
    P.w = (uint32_t)w;
    P.halfw = (uint32_t)(w / 2);
    P.L = (uint32_t)L;
    P.K = (uint32_t)K;
    P.Kl = (uint32_t)std::min<int32_t>(K, B);
    P.nsel = (uint32_t)nsel;
    P.T = (uint32_t)T;
    P.M = (uint32_t)((L + 1) / 2);
    P.method = method;
    P.estimator = estimator;
    P.refine = refine;
    P.srch_b = srch_b;
    P.residual = residual;
    P.precision = precision;
    P.gmode = gmode;
    if (method == kMethodComb) {
        P.Bc = Bc;
        P.logBc = ilog2(Bc);
        P.ncls = (uint32_t)std::min<int64_t>((int64_t)c * K, Bc);
    }
    decompose(P);
    *cap = std::min<int64_t>(N, (int64_t)(L - T + 1) * nsel * (N / B));
    // phase encoding, search: each iteration adds at most B found coefficients
    if (iterative(method)) *cap = std::min<int64_t>(N, (int64_t)L * B);
    P.cap = (uint32_t)*cap;
}

// A voting plan's descriptor fields that depend on K (scratch already sized
// for a K at least this large).
void set_K(PlanDev &P, int32_t K, int64_t *cap, int32_t c) {
    P.K = (uint32_t)K;
    P.Kl = (uint32_t)std::min<int32_t>(K, (int32_t)P.B);
    P.nsel = (uint32_t)std::min<int64_t>((int64_t)c * K, P.B);
    *cap = std::min<int64_t>(P.N, (int64_t)(P.L - P.T + 1) * P.nsel * (P.N / P.B));
    P.cap = (uint32_t)*cap;
}

// Distinct sample indices the plan's loops read (Table 2's sampling count),
// counted on the host with an N-bit map: the gather's indices
// (sigma m + tau) mod N, plus for phase encoding the sample one past each and
// for the search the samples at every search shift.
int64_t samples_touched_host(const PlanDev &P) {
    const uint32_t N = P.N, w = P.w, mask = N - 1;
    std::vector<uint64_t> bits(((size_t)N + 63) / 64, 0);
    auto mark = [&](uint32_t i) { bits[i >> 6] |= 1ull << (i & 63); };
    uint32_t nsh = 1, bb = 0, sbits = 0;
    if (P.method == kMethodSearch) {
        bb = P.srch_b;
        sbits = P.logN - P.logB + 1 < P.logN ? P.logN - P.logB + 1 : P.logN;
        nsh = 1 + (sbits + bb - 1) / bb;
    }
    for (uint32_t l = 0; l < P.L; ++l)
        for (uint32_t q = 0; q < w; ++q) {
            const uint32_t i = (P.sigma[l] * (q - w / 2) + P.tau[l]) & mask;
            mark(i);
            if (P.method == kMethodPhase) mark((i + 1) & mask);
            for (uint32_t j = 1; j < nsh; ++j) mark((i + (N >> std::min(j * bb, sbits))) & mask);
        }
    int64_t n = 0;
    for (uint64_t v : bits) n += __builtin_popcountll(v);
    return n;
}

// The calling thread's non-blocking stream for plan set-up on the current device.
cudaError_t setup_stream(cudaStream_t &out) {
    thread_local int dev = -1;
    thread_local cudaStream_t st = nullptr;
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (dev != d) {
        // a stream of another device is left to process teardown
        st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        dev = d;
    }
    out = st;
    return cudaSuccess;
}

}  // namespace

int64_t samples_touched_of(int64_t N, int32_t B, int64_t w, int32_t L, uint64_t seed, const sfft_opts &o) {
    PlanDev P;
    int64_t cap;
    const uint32_t method = o.method == SFFT_METHOD_PHASE    ? kMethodPhase
                            : o.method == SFFT_METHOD_SEARCH ? kMethodSearch
                            : o.method == SFFT_METHOD_COMB   ? kMethodComb
                                                             : kMethodVoting;
    fill_plan_dev(P, N, 1, B, w, L, 1, 1, &cap, method, method == kMethodComb ? 2u : 0u, kEstMedian, 0,
                  (uint32_t)std::max<int32_t>(o.search_bits, 1));
    loop_params_host(N, L, seed, P.sigma, P.tau, nullptr);
    return samples_touched_host(P);
}

size_t plan_device_bytes(int64_t N, int32_t K, int32_t B, int64_t w, int32_t L, int32_t c, int32_t T,
                         const sfft_opts &o) {
    const int32_t method = o.method;
    if (method == SFFT_METHOD_PHASE || method == SFFT_METHOD_SEARCH) c = T = 1;
    if (check_sizes(N, K, B, w, L, c, T) != SFFT_OK) return 0;
    PlanDev P;
    int64_t cap;
    // (a comb plan's residue tables are a few KB; sized here at the largest default)
    fill_plan_dev(P, N, K, B, w, L, c, T, &cap,
                  method == SFFT_METHOD_PHASE    ? kMethodPhase
                  : method == SFFT_METHOD_COMB   ? kMethodComb
                  : method == SFFT_METHOD_SEARCH ? kMethodSearch
                                                 : kMethodVoting,
                  (uint32_t)std::min<int64_t>(N, kMaxComb),
                  o.estimator == SFFT_ESTIMATOR_MEAN ? kEstMean : kEstMedian,
                  (uint32_t)std::max<int32_t>(o.refine, 0), (uint32_t)std::max<int32_t>(o.search_bits, 1),
                  o.residual ? 1u : 0u, o.precision ? 1u : 0u,
                  o.mode == SFFT_GATHER_STREAM ? kGatherStream : kGatherPermuted);
    return layout_of(P, cap).total;
}

void set_error(const std::string &msg) { g_err = msg; }

sfft_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return SFFT_ENOMEM;
    return SFFT_ECUDA;
}

// ------------------------------------------------------------ launch helpers
namespace {

struct Sizes {
    uint32_t gather = 0, select = 0, vote = 0, jobs = 0;
    uint32_t fb = 0;  // fallback-pass CTAs
    uint32_t max_B = 0, max_flags = 0, L_uniform = 0, max_K = 0;
    uint32_t est_smem = 0;  // pruned estimate: staged table bytes
    bool bits = true;
    bool phase = false;    // every job uses the phase-encoding method
    uint32_t max_L = 0;    // phase encoding: iterations to launch
    uint32_t max_cap = 0;  // phase encoding: largest found-list capacity
    bool comb = false;     // every job votes behind the spike-train pre-filter
    uint32_t max_Bc = 0;   // comb: largest number of residue classes
    bool search = false;   // every job locates by binary / multi-scale search
    uint32_t max_nbuf = 0; // search: largest count of bucket buffers
    bool refine = false;   // some job refines its output
    uint32_t max_rK = 0;   // refinement: largest K of the refining jobs
    uint32_t max_resB = 0; // residual check: largest B of the checking jobs (0: none checks)
    uint32_t dft_B = 0;    // split-BF16 tensor-core DFT of B buckets (0: the FP32 FFT)
    bool stream = false;   // the job's a1 is the stream gather (groups: every job's)
    uint32_t stream_smem = 0;  // stream gather: largest dynamic shared memory of the jobs
    uint64_t sum_N = 0;    // the jobs' N summed
};

Sizes plan_sizes(const sfft_plan *p) {
    Sizes z;
    z.max_L = p->h.L;
    if (iterative(p->h.method)) {
        // one CTA per job (the select slot of the batch maps)
        z.phase = true;
        z.search = p->h.method == kMethodSearch;
        z.max_nbuf = z.search ? search_nbuf(p->h.logN, p->h.logB, p->h.srch_b) : 0u;
        z.max_cap = p->h.cap;
        z.gather = 0;
        z.select = 1;
        z.vote = 0;
        z.jobs = 1;
        z.max_B = p->h.B;
        z.max_K = p->h.K;
        z.L_uniform = p->h.L;
        z.bits = false;
        return z;
    }
    z.comb = p->h.method == kMethodComb;
    z.max_Bc = p->h.Bc;
    z.sum_N = p->h.N;
    z.gather = p->h.tiles * p->h.L * p->h.nchunk;
    if (p->h.gmode == kGatherStream) {
        z.stream = true;
        z.gather = kStreamCluster * p->h.sgrp * p->h.snclu;
        z.stream_smem = stream_smem_bytes(p->h.slg, p->h.B, p->h.sV, p->h.spiece);
    }
    z.select = p->h.L;
    z.fb = fallback_ctas(p->h.N);
    z.vote = p->h.vtiles;
    z.jobs = 1;
    z.max_B = p->h.B;
    z.max_K = p->h.K;
    z.max_flags = p->h.L * p->h.B * 2;
    z.L_uniform = p->h.L;
    z.bits = p->h.use_bits != 0;
    z.est_smem = estimate_tab_bytes(p->h.N, p->h.B, p->h.L);
    z.refine = p->h.refine > 0;
    z.max_rK = z.refine ? p->h.K : 0u;
    z.max_resB = p->h.residual ? p->h.B : 0u;
    z.dft_B = p->h.precision ? p->h.B : 0u;
    return z;
}

// Phase-encoding method: one launch, one CTA per job over all its iterations.
// With ev: bracketed as the first stage; the other stages are empty.
cudaError_t launch_phase(const Launch &lj, const Sizes &z, cudaStream_t s, cudaEvent_t *ev = nullptr) {
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    if ((e = z.search ? launch_bs(lj, z.jobs, z.max_B, z.max_K, z.max_cap, z.max_nbuf, s)
                      : launch_pe(lj, z.jobs, z.max_B, z.max_K, z.max_cap, s)) != cudaSuccess)
        return e;
    for (int i = 1; ev && i <= 6; ++i)
        if ((e = cudaEventRecord(ev[i], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Per-thread side stream of the comb pre-filter (for the thread's current
// device) with its fork and join events.  The stream has the highest priority
// so the comb CTAs are placed while the gather's many short CTAs run.
struct SideRes {
    int device = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

cudaError_t side_res(SideRes *&out) {
    thread_local SideRes r;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (r.device != device) {
        // resources of another device are left to process teardown
        r = SideRes();
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&r.s, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        r.device = device;
    }
    out = &r;
    return cudaSuccess;
}

// Jobs of a batch that share every kernel variant (they are contiguous in
// the batch's job order): their sizes and, per kernel slot, the group's first
// CTA in the slot's CTA map and its CTA count.
struct Group {
    Sizes z;
    uint32_t cta0[6] = {0, 0, 0, 0, 0, 0}, ctas[6] = {0, 0, 0, 0, 0, 0};
};

// gather -> FFT/select -> scan -> estimate (whose last CTA per job takes the
// top K, running the job's fallback pass first when needed), all
// stream-ordered.  lk[k] is the launch of kernel slot k (0 gather, 1
// FFT/select, 2 scan, 3 one CTA per job, 5 estimate); the gather runs over
// every job at once, the FFT/select, scan and estimate once per group of
// jobs with common variants.  With ev (kStages + 1 events) the events
// bracket the stages: gather, FFT/select (and the wait for the comb kernel
// of comb plans), scan, estimate + top-K, refinement (empty unless a plan
// refines), residual check (empty unless a plan checks).
cudaError_t launch_pipeline(const Launch *lk, const Sizes &all, const std::vector<Group> &gs, void *dft_scratch,
                            cudaStream_t s, cudaEvent_t *ev = nullptr, uint32_t *gctr = nullptr) {
    cudaError_t e;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    auto at = [&](int k, const Group &g) {
        Launch l = lk[k];
        l.cta0 = g.cta0[k];
        return l;
    };
    if ((e = mark(0)) != cudaSuccess) return e;
    // comb plans: the kept residue classes (one CTA per job).  The comb
    // kernel reads only the signal, so it runs on the side stream beside the
    // gather and FFT/select and is joined before the scan.
    SideRes *sr = nullptr;
    if (all.comb) {
        if ((e = side_res(sr)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(sr->fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sr->s, sr->fork, 0)) != cudaSuccess) return e;
        if ((e = launch_comb(lk[3], all.jobs, all.max_Bc, sr->s)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(sr->join, sr->s)) != cudaSuccess) return e;
    }
    {
        // a1: the permuted gather over its jobs (a prefix of the slot's map:
        // stream-gather groups sort last), then the stream gather
        uint32_t perm = 0, str = 0, smem = 0;
        for (const Group &g : gs) {
            if (g.z.stream) {
                str += g.ctas[0];
                smem = std::max(smem, g.z.stream_smem);
            } else {
                perm += g.ctas[0];
            }
        }
        if ((e = launch_gather(lk[0], perm, s)) != cudaSuccess) return e;
        if (str) {
            Launch l = lk[0];
            l.cta0 = perm;
            if ((e = launch_gather_stream(l, str, smem, s)) != cudaSuccess) return e;
        }
    }
    if ((e = mark(1)) != cudaSuccess) return e;
    for (const Group &g : gs) {
        const uint32_t cl = fft_select_cluster_ok(g.z.L_uniform, g.z.max_B) ? g.z.L_uniform : 0u;
        if (g.z.dft_B) {
            // split-BF16 tensor-core DFT of the group's rows, then select on its partial planes
            const uint32_t rows = g.ctas[1], Bd = g.z.dft_B;
            uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<char *>(dft_scratch) + dft_scratch_bytes(rows, Bd));
            if ((e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
            if ((e = launch_dft(at(1, g), rows, Bd, dft_scratch, err, s)) != cudaSuccess) return e;
            const uint32_t mpad = (rows + kDftRowTile - 1) / kDftRowTile * kDftRowTile;
            if ((e = launch_fft_select(at(1, g), rows, Bd, 0, cl, s, dft_partials(dft_scratch, rows, Bd), mpad, err)) !=
                cudaSuccess)
                return e;
            continue;
        }
        if ((e = launch_fft_select(at(1, g), g.ctas[1], g.z.max_B, 0, cl, s)) != cudaSuccess) return e;
    }
    if (all.comb && (e = cudaStreamWaitEvent(s, sr->join, 0)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    for (const Group &g : gs)
        if ((e = launch_vote(at(2, g), g.ctas[2], kVotePrune, g.z.L_uniform, g.z.bits, g.z.max_flags, g.z.max_B,
                             nullptr, nullptr, s)) != cudaSuccess)
            return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        const Group &g = gs[gi];
        // (batch groups of up to kDynMaxJobs jobs share their survivors' chunks
        // dynamically; their counts and chunk sums are 32-bit: N summed < 2^31)
        Launch le = at(5, g);
        le.gctr = gctr && g.z.jobs <= kDynMaxJobs && g.z.sum_N < (1ull << 31) ? gctr + 8 * gi : nullptr;
        if ((e = launch_estimate(le, g.ctas[5], g.z.L_uniform, g.z.est_smem, g.z.max_K, s)) != cudaSuccess)
            return e;
        // jobs whose pruned records could not certify their top K
        Launch lf = at(4, g);
        lf.gctr = le.gctr;  // (words 2, 3: the fallback's chunk counters; 4: jobs flagged for it)
        if ((e = launch_fallback(lf, g.ctas[4], g.z.L_uniform, g.z.max_K, s)) != cudaSuccess) return e;
    }
    if ((e = mark(4)) != cudaSuccess) return e;
    // refining jobs: the iterative framework's subtraction over the found set
    if (all.refine && (e = launch_refine(lk[3], all.jobs, all.max_rK, all.L_uniform, s)) != cudaSuccess) return e;
    if ((e = mark(5)) != cudaSuccess) return e;
    // checking jobs: FP64 energy left after subtracting the final output
    if (all.max_resB && (e = launch_residual(lk[1], all.select, all.max_resB, s)) != cudaSuccess) return e;
    return mark(6);
}

// One plan's launch: a single group covering its CTAs (dft: the plan's own
// tensor-core DFT scratch, precision 1).
cudaError_t launch_single(const Launch &ln, const Sizes &z, void *dft, cudaStream_t s, cudaEvent_t *ev = nullptr) {
    Launch lk[6] = {ln, ln, ln, ln, ln, ln};
    std::vector<Group> gs(1);
    gs[0].z = z;
    gs[0].ctas[0] = z.gather;
    gs[0].ctas[1] = z.select;
    gs[0].ctas[2] = z.vote;
    gs[0].ctas[4] = z.fb;
    gs[0].ctas[5] = kEstimateCtas;
    return launch_pipeline(lk, z, gs, dft, s, ev);
}

Job make_job(const sfft_plan *p, const float *x, int32_t *idx, float *val, int32_t *kout) {
    Job j;
    j.p = p->d;
    j.x = reinterpret_cast<const float2 *>(x);
    j.idx = idx;
    j.val = reinterpret_cast<float2 *>(val);
    j.kout = kout;
    j.rpc = p->h.rpc;
    j.nchunk = p->h.nchunk;
    j.vctas = p->h.vtiles;
    j.ectas = kEstimateCtas;
    return j;
}


Launch single(const Job &j) {
    Launch ln;
    ln.jobs = nullptr;
    ln.offs = nullptr;
    ln.map = nullptr;
    ln.njobs = 1;
    ln.cta0 = 0;
    ln.gctr = nullptr;
    ln.one = j;
    return ln;
}

// ---- batch buffers: a small ring of (pinned host, device) pairs for one-off
// job lists, and a cache of captured graphs for job lists seen again.
struct Slot {
    void *host = nullptr;
    void *dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    int device = -1;
};

struct GraphEntry {
    std::vector<uint64_t> key;
    void *dev = nullptr;
    cudaGraphExec_t exec = nullptr;
    int seen = 0;
    int device = -1;
};

std::mutex g_batch_mu;
Slot g_slots[4];
int g_next_slot = 0;
std::list<GraphEntry> g_graphs;  // most recent first
constexpr size_t kMaxGraphs = 16;

void drop_entry(GraphEntry &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.dev) cudaFree(e.dev);
    e.exec = nullptr;
    e.dev = nullptr;
}

}  // namespace

void forget_plan_graphs(uint64_t id) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        bool uses = false;
        for (size_t i = 1; i < it->key.size(); i += 4)
            if (it->key[i] == id) uses = true;
        if (uses) {
            drop_entry(*it);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace sfft

using namespace sfft;

// ------------------------------------------------------------------- plans
extern "C" sfft_status sfft_loop_params(int64_t N, int32_t L, uint64_t seed, uint32_t *sigma, uint32_t *tau,
                                        uint32_t *sigma_inv) {
    if (!is_pow2(N) || N < 2 || N > (1ll << kMaxLogN) || L < 1 || L > kMaxL) {
        set_error("N must be a power of two in [2, 2^30] and L in [1, 32]");
        return SFFT_EINVAL;
    }
    loop_params_host(N, L, seed, sigma, tau, sigma_inv);
    return SFFT_OK;
}

extern "C" sfft_status sfft_window_walk(int64_t N, int64_t w, uint64_t sigma, uint64_t tau, int64_t p0,
                                        int64_t out[6]) {
    if (!out || !is_pow2(N) || N < 2 || N > (1ll << kMaxLogN) || w < 2 || w > N || !(sigma & 1) ||
        sigma >= (uint64_t)N || tau >= (uint64_t)N || p0 < 0 || p0 >= N) {
        set_error("sfft_window_walk: N a power of two in [2, 2^30], 2 <= w <= N, sigma odd < N, tau, p0 < N");
        return SFFT_EINVAL;
    }
    const uint32_t n = (uint32_t)N, s = inv_odd_u32((uint32_t)sigma) & (n - 1);
    const WindowWalk wk = window_walk(n, s, (uint32_t)w);
    uint32_t k = 0, q = 0;
    window_first_read(n, s, (uint32_t)tau, (uint32_t)w, (uint32_t)(w / 2), (uint32_t)p0, &k, &q);
    out[0] = (int64_t)(((uint64_t)p0 + k) % (uint64_t)N);
    out[1] = q;
    out[2] = wk.kp;
    out[3] = wk.alpha;
    out[4] = wk.km;
    out[5] = wk.beta;
    return SFFT_OK;
}

extern "C" sfft_status sfft_suggest_params(int64_t N, int32_t K, double snr_db, int32_t *B, int64_t *w,
                                           int32_t *L) {
    if (!is_pow2(N) || N < 2 || N > (1ll << kMaxLogN) || K < 1 || K > N || !B || !w || !L) {
        set_error("N must be a power of two in [2, 2^30], K in [1, N], outputs non-NULL");
        return SFFT_EINVAL;
    }
    // a loaded tuning class for this shape overrides the rule's ratios
    int64_t bpk = 4, wex = 21;
    int32_t Lt = 0;
    const bool tuned = tuning_lookup((int)ilog2((uint64_t)N), K, snr_db, &bpk, &wex, &Lt);
    int64_t b = 64;
    while (b < bpk * K) b <<= 1;
    b = std::min<int64_t>(b, std::min<int64_t>(kMaxB, N / 64));  // B (log2 N + 21) < N
    b = std::max<int64_t>(2, std::min<int64_t>(b, N));
    if (b < 2ll * K) {
        // the 2K kept buckets would be all of them: no bucket is left empty to
        // tell the large ones apart, and the flat window needs N/B >= 64
        set_error("K too large for N: the size-class rule needs B >= 2K with B <= min(16384, N/64), i.e. "
                  "K <= min(8192, N/128)");
        return SFFT_EINVAL;
    }
    int64_t ww = b * (int64_t)(ilog2((uint64_t)N) + wex);
    if (ww > N) ww = N / b * b;
    *B = (int32_t)b;
    *w = ww;
    *L = tuned ? Lt : (std::isnan(snr_db) ? 8 : 12);
    return SFFT_OK;
}

extern "C" sfft_status sfft_plan_create(sfft_plan **plan, int64_t N, int32_t K, int32_t B, int64_t w, int32_t L,
                                        uint64_t seed) {
    return sfft_plan_create_ex(plan, N, K, B, w, L, seed, nullptr);
}

namespace sfft {

// Plan creation with scratch sized for up to K_cap output coefficients (K <=
// K_cap; the serving loop rebinds cached voting plans to other K and seeds).
sfft_status plan_create(sfft_plan **plan, int64_t N, int32_t K, int32_t K_cap, int64_t B, int64_t w, int32_t L,
                        uint64_t seed, const sfft_opts *opts) {
    if (!plan) {
        set_error("plan pointer is NULL");
        return SFFT_EINVAL;
    }
    *plan = nullptr;
    sfft_opts o = {};
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) {
        set_error("sfft_opts.precision must be 0 (FP32 FFT) or 1 (split-BF16 tensor-core DFT)");
        return SFFT_EINVAL;
    }
    if (o.method != SFFT_METHOD_VOTING && o.method != SFFT_METHOD_PHASE && o.method != SFFT_METHOD_COMB &&
        o.method != SFFT_METHOD_SEARCH) {
        set_error("sfft_opts.method must be SFFT_METHOD_VOTING, SFFT_METHOD_PHASE, SFFT_METHOD_COMB or "
                  "SFFT_METHOD_SEARCH");
        return SFFT_EINVAL;
    }
    const bool search = o.method == SFFT_METHOD_SEARCH;
    const bool phase = o.method == SFFT_METHOD_PHASE || search;  // the iterative-framework methods
    const bool comb = o.method == SFFT_METHOD_COMB;
    if (!search && o.search_bits != 0) {
        set_error("sfft_opts.search_bits applies to SFFT_METHOD_SEARCH only");
        return SFFT_EINVAL;
    }
    const int32_t sb = search ? (o.search_bits > 0 ? o.search_bits : 1) : 1;
    if (sb < 1 || sb > 4) {
        set_error("sfft_opts.search_bits must be 1..4 (1: binary search)");
        return SFFT_EINVAL;
    }
    if (!comb && o.comb != 0) {
        set_error("sfft_opts.comb applies to SFFT_METHOD_COMB only");
        return SFFT_EINVAL;
    }
    if (o.estimator != SFFT_ESTIMATOR_MEDIAN && o.estimator != SFFT_ESTIMATOR_MEAN) {
        set_error("sfft_opts.estimator must be SFFT_ESTIMATOR_MEDIAN or SFFT_ESTIMATOR_MEAN");
        return SFFT_EINVAL;
    }
    if (phase && o.estimator != SFFT_ESTIMATOR_MEDIAN) {
        set_error("sfft_opts.estimator applies to the voting and comb methods");
        return SFFT_EINVAL;
    }
    if (K_cap < K || (K_cap != K && o.method != SFFT_METHOD_VOTING)) {
        set_error("plan capacity below K (or a capacity for a method other than voting)");
        return SFFT_EINVAL;
    }
    if (o.refine < 0 || o.refine > SFFT_MAX_REFINE || (o.refine && (phase || K_cap > (int32_t)kRefineMaxK))) {
        set_error("sfft_opts.refine must be 0..8 passes, for the voting and comb methods with K <= 4096");
        return SFFT_EINVAL;
    }
    if (o.precision == 1 && (phase || B < 64 || B > (int64_t)kDftMaxB)) {
        set_error("sfft_opts.precision 1 (split-BF16 tensor-core DFT) is for the voting and comb methods with "
                  "64 <= B <= 4096");
        return SFFT_EINVAL;
    }
    if (o.residual != 0 && (o.residual != 1 || phase || B < 4 || B > (int32_t)kResidualMaxB)) {
        set_error("sfft_opts.residual must be 0 or 1, for the voting and comb methods with 4 <= B <= 8192");
        return SFFT_EINVAL;
    }
    if (o.mode != SFFT_GATHER_AUTO && o.mode != SFFT_GATHER_PERMUTED && o.mode != SFFT_GATHER_STREAM) {
        set_error("sfft_opts.mode must be SFFT_GATHER_AUTO, SFFT_GATHER_PERMUTED or SFFT_GATHER_STREAM");
        return SFFT_EINVAL;
    }
    const bool stream = o.mode == SFFT_GATHER_STREAM;
    if (stream && (phase || N < (1ll << kStreamMinLogN) || B > 4096)) {
        set_error("sfft_opts.mode SFFT_GATHER_STREAM is for the voting and comb methods with N >= 2^12 and "
                  "B <= 4096");
        return SFFT_EINVAL;
    }
    // (phase encoding reads no c or T)
    const int32_t c = phase ? 1 : (o.c > 0 ? o.c : 2);
    const int32_t T = phase ? 1 : (o.T > 0 ? o.T : (L + 1) / 2);
    sfft_status st = check_sizes(N, K_cap, (int32_t)B, w, L, c, T);
    if (st != SFFT_OK) return st;
    if (K < 1) {
        set_error("K must lie in [1, min(N, 16384)]");
        return SFFT_EINVAL;
    }
    uint32_t Bc = 0;
    if (comb) {
        // residue classes: a power of two dividing N/G (G = B/32 frequencies per
        // register-table scan thread must share one class), at most kMaxComb
        int64_t lim = std::min<int64_t>(N, kMaxComb);
        if (B >= 32 && B <= 512) lim = std::min<int64_t>(lim, 32 * N / B);
        int64_t bc = o.comb;
        if (bc == 0) {
            bc = 1;
            while (bc < 16ll * c * K) bc <<= 1;
            bc = std::min(bc, lim);
        }
        if (bc < 2 || (bc & (bc - 1)) || bc > lim || L + (int32_t)kCombShifts > kMaxL) {
            set_error("SFFT_METHOD_COMB needs comb a power of two in [2, min(N, 8192, 32N/B for 32 <= B <= 512)] "
                      "and L <= 30");
            return SFFT_EINVAL;
        }
        Bc = (uint32_t)bc;
    }

    if (search) {
        // one CTA holds the job's bucket buffers and its top-K ranks
        const uint32_t logN = ilog2(N), logB = ilog2(B);
        uint64_t rank = 1024;
        while (rank < (uint64_t)K) rank <<= 1;
        const uint64_t fcap = std::min<int64_t>(N, (int64_t)L * B);  // found-list capacity
        const uint64_t tail = std::max<uint64_t>(std::max<uint64_t>(12ull * rank, fcap <= kPeSmemFound ? 16ull * fcap : 0ull),
                                                 4ull * B);
        const uint64_t bytes = 8ull * search_nbuf(logN, logB, (uint32_t)sb) * B + 8ull * (B / 2 + 1) + tail;
        if (bytes > kSearchSmemMax) {
            set_error("SFFT_METHOD_SEARCH: the bucket buffers (1 + ceil((log2(N/B) + 1) / search_bits) of B each) "
                      "and the top-K ranks exceed one CTA's shared memory");
            return SFFT_EINVAL;
        }
    }

    sfft_plan *p = new (std::nothrow) sfft_plan();
    if (!p) {
        set_error("host allocation failed");
        return SFFT_ENOMEM;
    }
    p->id = g_next_id.fetch_add(1);
    cudaGetDevice(&p->device);
    p->N = N;
    p->w = w;
    p->K = K;
    p->K_cap = K_cap;
    p->B = (int32_t)B;
    p->L = L;
    p->c = c;
    p->T = T;
    p->seed = seed;
    p->samples_touched = -1;

    // scratch sized for K_cap, then the descriptor set to K
    PlanDev &P = p->h;
    fill_plan_dev(P, N, K_cap, (int32_t)B, w, L, c, T, &p->cap, (uint32_t)o.method, Bc,
                  o.estimator == SFFT_ESTIMATOR_MEAN ? kEstMean : kEstMedian, (uint32_t)o.refine, (uint32_t)sb,
                  (uint32_t)o.residual, (uint32_t)o.precision, stream ? kGatherStream : kGatherPermuted);
    const Layout lay = layout_of(P, p->cap);
    if (K != K_cap) set_K(P, K, &p->cap, c);
    p->nsel = (int32_t)P.nsel;
    // (comb plans: loops L and L+1 give the comb shifts)
    loop_params_host(N, L + (comb ? (int32_t)kCombShifts : 0), seed, P.sigma, P.tau, p->sigma_inv);

    if (P.precision && (st = dft_table_prepare(P.B)) != SFFT_OK) {
        delete p;
        return st;
    }
    TableSet tab;
    st = tables_acquire(P.N, P.B, P.w, phase || P.refine, P.residual != 0, &p->tables, &tab);
    if (st != SFFT_OK) {
        delete p;
        return st;
    }
    p->device_bytes = lay.total;
    cudaError_t e = cudaMalloc(&p->dmem, lay.total);
    if (e != cudaSuccess) {
        tables_release(p->tables);
        delete p;
        return cuda_fail(e, "cudaMalloc(plan)");
    }
    char *base = static_cast<char *>(p->dmem);
    p->d = reinterpret_cast<PlanDev *>(base + lay.plan);
    P.taps = tab.taps;
    P.tw = tab.tw;
    P.twst = tab.twst;
    P.ginv = tab.ginv;
    P.gext = tab.gext;
    P.gext64 = tab.gext64;
    P.ginv2max = tab.ginv2max;
    P.rscr = P.refine ? reinterpret_cast<float2 *>(base + lay.rscr) : nullptr;
    P.resid = P.residual ? reinterpret_cast<double *>(base + lay.resid) : nullptr;
    p->dft = P.precision ? static_cast<void *>(base + lay.dft) : nullptr;
    P.ctw = comb ? reinterpret_cast<float2 *>(base + lay.ctw) : nullptr;
    P.cls = comb ? reinterpret_cast<uint32_t *>(base + lay.cls) : nullptr;
    P.keptc = comb ? reinterpret_cast<uint32_t *>(base + lay.keptc) : nullptr;
    P.partial = reinterpret_cast<float2 *>(base + lay.part);
    P.zhat = reinterpret_cast<float2 *>(base + lay.zhat);
    P.energy = reinterpret_cast<float *>(base + lay.en);
    P.loopkth = reinterpret_cast<float *>(base + lay.lkth);
    P.packed = reinterpret_cast<uint32_t *>(base + lay.topk);
    P.sel = reinterpret_cast<int32_t *>(base + lay.sel);
    P.flags = reinterpret_cast<uint16_t *>(base + lay.flags);
    P.bits2 = needs_bits2(P) ? reinterpret_cast<uint32_t *>(base + lay.bits2) : nullptr;
    P.survf = reinterpret_cast<uint32_t *>(base + lay.survf);
    P.surv = reinterpret_cast<uint4 *>(base + lay.surv);
    P.walk = stream ? reinterpret_cast<const uint4 *>(base + lay.walk) : nullptr;
    P.wq = stream ? reinterpret_cast<uint32_t *>(base + lay.wq) : nullptr;
    P.ctr = reinterpret_cast<uint32_t *>(base + lay.ctr);

    // descriptor, counters, the comb twiddles and the stream gather's walk
    // tables on the thread's set-up stream
    auto fail = [&](cudaError_t err, const char *what) {
        cudaFree(p->dmem);
        tables_release(p->tables);
        delete p;
        return cuda_fail(err, what);
    };
    cudaStream_t s = nullptr;
    if ((e = setup_stream(s)) != cudaSuccess) return fail(e, "set-up stream");
    if ((e = cudaMemcpyAsync(p->d, &P, sizeof(PlanDev), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e, "upload plan");
    if ((e = cudaMemsetAsync(P.ctr, 0, sizeof(uint32_t) * kNumCounters, s)) != cudaSuccess)
        return fail(e, "clear counters");
    if (comb && (e = plan_twiddles(P.Bc, const_cast<float2 *>(P.ctw), s)) != cudaSuccess)
        return fail(e, "comb twiddles");
    if ((e = launch_walk_start(P, p->sigma_inv, s)) != cudaSuccess) return fail(e, "stream gather walk tables");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "plan set-up");
    *plan = p;
    return SFFT_OK;
}

// Rebinds an idle plan to another seed (new sigma, tau) and, for voting
// plans, another K <= K_cap: the descriptor is re-uploaded on stream s, so
// work enqueued on s afterwards sees the new parameters.  A changed K changes
// launch shapes, so the plan takes a new identity (cached batch graphs of
// the old one no longer match).
sfft_status plan_rebind(sfft_plan *p, int32_t K, uint64_t seed, cudaStream_t s) {
    if (K < 1 || K > p->K_cap || (K != p->K && p->h.method != kMethodVoting)) {
        set_error("rebind: K beyond the plan's capacity (or K changed on a plan other than voting)");
        return SFFT_EINVAL;
    }
    PlanDev &P = p->h;
    if (K != p->K) {
        set_K(P, K, &p->cap, p->c);
        p->K = K;
        p->nsel = (int32_t)P.nsel;
        p->id = g_next_id.fetch_add(1);
    }
    const bool comb = P.method == kMethodComb;
    loop_params_host(p->N, p->L + (comb ? (int32_t)kCombShifts : 0), seed, P.sigma, P.tau, p->sigma_inv);
    p->seed = seed;
    p->samples_touched = -1;
    // (from pageable memory: the descriptor is staged before the call returns)
    SFFT_CUDA_TRY(cudaMemcpyAsync(p->d, &P, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
    SFFT_CUDA_TRY(launch_walk_start(P, p->sigma_inv, s));
    return SFFT_OK;
}

}  // namespace sfft

extern "C" sfft_status sfft_plan_create_ex(sfft_plan **plan, int64_t N, int32_t K, int32_t B, int64_t w,
                                           int32_t L, uint64_t seed, const sfft_opts *opts) {
    return plan_create(plan, N, K, K, B, w, L, seed, opts);
}

extern "C" sfft_status sfft_plan_reseed(sfft_plan *p, uint64_t seed, void *stream) {
    if (!p) {
        set_error("NULL plan");
        return SFFT_EINVAL;
    }
    return plan_rebind(p, p->K, seed, static_cast<cudaStream_t>(stream));
}

extern "C" void sfft_plan_destroy(sfft_plan *plan) {
    if (!plan) return;
    forget_plan_graphs(plan->id);
    if (plan->stage) cudaFree(plan->stage);
    cudaFree(plan->dmem);
    tables_release(plan->tables);
    delete plan;
}

extern "C" sfft_status sfft_plan_get_info(const sfft_plan *p, sfft_plan_info *info) {
    if (!p || !info) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    info->N = p->N;
    info->w = p->w;
    info->K = p->K;
    info->B = p->B;
    info->L = p->L;
    info->c = p->c;
    info->T = p->T;
    info->nsel = p->nsel;
    info->seed = p->seed;
    if (p->samples_touched < 0) p->samples_touched = samples_touched_host(p->h);
    info->samples_touched = p->samples_touched;
    info->candidate_capacity = p->cap;
    info->device_bytes = p->device_bytes;
    info->method = (int32_t)p->h.method;
    info->estimator = (int32_t)p->h.estimator;
    info->refine = (int32_t)p->h.refine;
    return SFFT_OK;
}

extern "C" sfft_status sfft_plan_get_loops(const sfft_plan *p, uint32_t *sigma, uint32_t *tau,
                                           uint32_t *sigma_inv) {
    if (!p) {
        set_error("NULL plan");
        return SFFT_EINVAL;
    }
    for (int l = 0; l < p->L; ++l) {
        if (sigma) sigma[l] = p->h.sigma[l];
        if (tau) tau[l] = p->h.tau[l];
        if (sigma_inv) sigma_inv[l] = p->sigma_inv[l];
    }
    return SFFT_OK;
}

extern "C" sfft_status sfft_plan_last_stats(const sfft_plan *p, sfft_exec_stats *st) {
    if (!p || !st) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    uint32_t c[kNumCounters];
    SFFT_CUDA_TRY(cudaMemcpy(c, p->h.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    st->residual_energy = -1.0;
    st->bucket_energy = -1.0;
    st->device_error = (int32_t)c[kErr];
    if (p->h.residual) {
        // per-loop pairs summed in loop order
        std::vector<double> r(2 * (size_t)p->L);
        SFFT_CUDA_TRY(cudaMemcpy(r.data(), p->h.resid, sizeof(double) * r.size(), cudaMemcpyDeviceToHost));
        double er = 0.0, et = 0.0;
        for (int32_t l = 0; l < p->L; ++l) {
            er += r[2 * l];
            et += r[2 * l + 1];
        }
        st->residual_energy = er;
        st->bucket_energy = et;
    }
    if (iterative(p->h.method)) {
        // found coefficients (kNGe), iterations run, bucket-energy threshold
        st->candidates = -1;
        st->estimated = c[kNGe];
        st->recorded = c[kNGe];
        st->fallback = 0;
        memcpy(&st->theta, &c[kTheta], sizeof(float));
        st->iterations = (int32_t)c[kPeIter];
        return SFFT_OK;
    }
    st->iterations = p->L;
    const bool fb = c[kNGe] < (uint32_t)p->K;
    st->candidates = fb ? (int64_t)c[kNCand] : -1;
    st->estimated = fb ? c[kNCand] : c[kNSurv];  // the fallback pass estimates every candidate
    st->recorded = fb ? c[kNRec2] : c[kNGe];
    st->fallback = fb ? 1 : 0;
    float th;
    memcpy(&th, &c[kTheta], sizeof(th));
    st->theta = th;
    return SFFT_OK;
}

// ----------------------------------------------------------------- execute
extern "C" sfft_status sfft_execute(sfft_plan *p, const float *x_dev, int32_t *idx_dev, float *val_dev,
                                    int32_t *k_out_dev, void *stream) {
    if (!p || !x_dev || !idx_dev || !val_dev || !k_out_dev) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    const Launch ln = single(make_job(p, x_dev, idx_dev, val_dev, k_out_dev));
    if (iterative(p->h.method))
        SFFT_CUDA_TRY(launch_phase(ln, plan_sizes(p), static_cast<cudaStream_t>(stream)));
    else
        SFFT_CUDA_TRY(launch_single(ln, plan_sizes(p), p->dft, static_cast<cudaStream_t>(stream)));
    return SFFT_OK;
}

// Device staging of a plan's host-buffer calls: x, then idx, val and k_out.
static size_t stage_bytes(const sfft_plan *p) {
    return align256(sizeof(float2) * p->N) + align256(sizeof(int32_t) * p->K) + align256(sizeof(float2) * p->K) +
           256;
}

extern "C" sfft_status sfft_execute_host(sfft_plan *p, const float *x_host, int32_t *idx_host, float *val_host,
                                         int32_t *k_out_host, void *stream) {
    if (!p || !x_host || !idx_host || !val_host || !k_out_host) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    const size_t xb = align256(sizeof(float2) * p->N), ib = align256(sizeof(int32_t) * p->K),
                 vb = align256(sizeof(float2) * p->K);
    if (!p->stage) SFFT_CUDA_TRY(cudaMalloc(&p->stage, stage_bytes(p)));
    char *b = static_cast<char *>(p->stage);
    float *x = reinterpret_cast<float *>(b);
    int32_t *idx = reinterpret_cast<int32_t *>(b + xb);
    float *val = reinterpret_cast<float *>(b + xb + ib);
    int32_t *kout = reinterpret_cast<int32_t *>(b + xb + ib + vb);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SFFT_CUDA_TRY(cudaMemcpyAsync(x, x_host, sizeof(float2) * p->N, cudaMemcpyHostToDevice, s));
    sfft_status st = sfft_execute(p, x, idx, val, kout, stream);
    if (st != SFFT_OK) return st;
    SFFT_CUDA_TRY(cudaMemcpyAsync(k_out_host, kout, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SFFT_CUDA_TRY(cudaMemcpyAsync(idx_host, idx, sizeof(int32_t) * p->K, cudaMemcpyDeviceToHost, s));
    SFFT_CUDA_TRY(cudaMemcpyAsync(val_host, val, sizeof(float2) * p->K, cudaMemcpyDeviceToHost, s));
    SFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return SFFT_OK;
}

// ------------------------------------------------------------------- batch
namespace {

struct BatchLayout {
    std::vector<unsigned char> bytes;  // jobs, then per kernel a CTA prefix and a CTA -> job map,
                                       // then eight zero words per group (Launch::gctr)
    size_t off_offs[6], off_map[6], off_gctr = 0;
    Sizes z;                  // the whole batch
    std::vector<Group> groups;  // runs of jobs with common kernel variants
    size_t dft_bytes = 0;     // tensor-core DFT scratch after the bytes (largest group; groups run in turn)
    // device bytes of the batch buffer: the bytes (copied), then the DFT scratch (not copied)
    size_t dev_bytes() const { return align256(bytes.size()) + dft_bytes; }
};

// Accumulates job sizes s into batch sizes z (first: z is still empty).
void merge_sizes(Sizes &z, const Sizes &s, bool first) {
    z.max_B = std::max(z.max_B, s.max_B);
    z.max_K = std::max(z.max_K, s.max_K);
    z.bits = (first || z.bits) && s.bits;
    z.max_flags = std::max(z.max_flags, s.max_flags);
    if (first) z.L_uniform = s.L_uniform;
    else if (s.L_uniform != z.L_uniform) z.L_uniform = 0;
    z.est_smem = (first || z.est_smem) && s.est_smem ? std::max(z.est_smem, s.est_smem) : 0u;
    z.phase = first ? s.phase : z.phase;  // one method per batch (callers split mixed lists)
    z.search = first ? s.search : z.search;
    z.max_nbuf = std::max(z.max_nbuf, s.max_nbuf);
    z.max_L = std::max(z.max_L, s.max_L);
    z.max_cap = std::max(z.max_cap, s.max_cap);
    z.comb = first ? s.comb : z.comb;
    z.max_Bc = std::max(z.max_Bc, s.max_Bc);
    z.refine = z.refine || s.refine;
    z.max_rK = std::max(z.max_rK, s.max_rK);
    z.max_resB = std::max(z.max_resB, s.max_resB);
    z.dft_B = std::max(z.dft_B, s.dft_B);
    z.stream = first ? s.stream : (z.stream && s.stream);
    z.stream_smem = std::max(z.stream_smem, s.stream_smem);
    z.sum_N = (first ? 0 : z.sum_N) + s.sum_N;
    z.gather += s.gather;
    z.select += s.select;
    z.vote += s.vote;
    z.fb += s.fb;
    z.jobs += 1;
}

// Kernel variants a job runs (jobs with equal keys form one group): L, the
// scan's table kind, the estimate's table kind, a clusterable FFT/select.
uint32_t variant_key(const Sizes &s) {
    const uint32_t L = s.L_uniform;
    // (register-table jobs also by their table words per lane)
    const uint32_t scan = scan_uses_bits(L, s.bits) ? (s.max_B > 1024 ? s.max_B / 1024 : 0u)
                                                    : (s.max_flags <= (uint32_t)kFlagsSmemBytes ? 8u : 9u);
    const uint32_t est = (s.est_smem && (L == 8 || L == 12 || L == 16)) ? 0u : 1u;
    // (the FFT/select's shared memory and cluster check go by the group's largest B)
    const uint32_t cl = s.max_B <= 1024 ? 0u : s.max_B <= 4096 ? 1u : s.max_B <= 8192 ? 2u : 3u;
    const uint32_t dft = s.dft_B ? ilog2(s.dft_B) : 0u;  // tensor-core DFT groups share B
    // (stream-gather jobs sort last: their gather CTAs end the slot's map)
    return ((s.stream ? 1u : 0u) << 24) | (dft << 16) | (L << 8) | (scan << 4) | (est << 2) | cl;
}

// Expected estimate work of a job, for sharing the estimate's CTAs: N times
// the fraction of frequencies the pruned pass estimates.  A frequency
// survives the median bound with >= M strong loops, and a loop's bucket is
// strong about as often as it holds one of the K coefficients, so the
// fraction is about P[Bin(L, min(1, K/B)) >= M] (measured on the batched
// workload: 0.52 of N at N = 2^14, K/B ~ 1/2, against 0.015 at K/B ~ 1/5);
// the mean estimator estimates every candidate (kept in >= T loops,
// p = nsel/B); comb plans only the kept classes' share.  A floor of 0.5%
// stands for buckets made strong by noise.
double estimate_weight(const PlanDev &P) {
    const bool mean = P.estimator == kEstMean;
    const double p = std::min(1.0, (double)(mean ? P.nsel : P.K) / (double)P.B);
    const uint32_t need = mean ? P.T : P.M;
    double tail = 0.0, c = 1.0;  // c = C(L, k)
    for (uint32_t k = 0; k <= P.L; ++k) {
        if (k >= need) tail += c * std::pow(p, (double)k) * std::pow(1.0 - p, (double)(P.L - k));
        c = c * (double)(P.L - k) / (double)(k + 1);
    }
    double f = std::max(tail, 0.005);
    if (P.method == kMethodComb && P.Bc) f *= (double)P.ncls / (double)P.Bc;
    return (double)P.N * f;
}

BatchLayout build_batch(sfft_plan *const *plans, const float *const *x, int32_t *const *idx,
                        float *const *val, int32_t *kout, int32_t count) {
    BatchLayout b;
    std::vector<Sizes> ps(count);
    for (int32_t i = 0; i < count; ++i) ps[i] = plan_sizes(plans[i]);
    // jobs ordered by variant group (the iterative methods: one group, in
    // the caller's order); each job keeps its own output pointers
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    if (!ps[0].phase)
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t c) { return variant_key(ps[a]) < variant_key(ps[c]); });
    // CTA counts per job and kernel: gather, select, vote, one per job, fallback, estimate
    std::vector<uint32_t> cnt((size_t)count * 6);
    std::vector<Job> jobs(count);
    Sizes &z = b.z;
    for (int32_t r = 0; r < count; ++r) {
        const int32_t i = order[r];
        const sfft_plan *p = plans[i];
        jobs[r] = make_job(p, x[i], idx[i], val[i], kout + i);
        const Sizes &s = ps[i];
        uint32_t *c = &cnt[(size_t)r * 6];
        c[0] = s.gather;
        if (count > 1 && !s.phase && !s.stream) {
            // in a batch the other signals fill the GPU: a job's gather takes
            // about kNumSms CTAs per 2^20 samples of signal (the plan's split,
            // one CTA per SM, at N = 2^20), so small signals are not cut into
            // many CTAs of a few rounds each
            const PlanDev &P = p->h;
            const uint32_t per = P.tiles * P.L;
            const uint64_t want = ((uint64_t)kNumSms * P.N + (1u << 20) - 1) >> 20;
            uint32_t nc = (uint32_t)std::min<uint64_t>(P.nchunk, std::max<uint64_t>(1, (want + per - 1) / per));
            const uint32_t rpc = (P.rounds + nc - 1) / nc;
            nc = (P.rounds + rpc - 1) / rpc;
            jobs[r].rpc = rpc;
            jobs[r].nchunk = nc;
            c[0] = per * nc;
        }
        c[1] = s.select;
        c[2] = s.vote;
        c[3] = 1;
        c[4] = s.fb;
        c[5] = kEstimateCtas;
        merge_sizes(z, s, r == 0);
        bool start = r == 0;
        if (r > 0 && !ps[0].phase) start = variant_key(s) != variant_key(ps[order[r - 1]]);
        if (start) b.groups.push_back(Group());
        merge_sizes(b.groups.back().z, s, start);
    }
    // per group: the pruned scan takes as many vote tiles per CTA as keep
    // its CTAs within kScanWaves waves of resident CTAs (fewer CTAs amortise
    // the per-CTA set-up; a partial last wave costs a whole CTA lifetime);
    // the estimate takes one wave of resident CTAs, shared among the jobs in
    // proportion to their expected survivors (estimate_weight),
    // 1..kEstimateCtas each
    size_t r0 = 0;
    for (Group &g : b.groups) {
        Sizes &gz = g.z;
        if (gz.L_uniform != 8 && gz.L_uniform != 12 && gz.L_uniform != 16) gz.est_smem = 0;
        double sumW = 0.0;
        for (size_t r = r0; r < r0 + gz.jobs; ++r) sumW += estimate_weight(plans[order[r]]->h);
        const double wave = (double)kNumSms * (gz.est_smem ? kEstTabCtasPerSm : kEstSurvCtasPerSm);
        uint64_t vt = 0;
        for (size_t r = r0; r < r0 + gz.jobs; ++r) vt += cnt[r * 6 + 2];
        // (the fewest tiles per CTA that keep the group's scan within one wave of
        // resident CTAs, up to 32: 8 headline signals' scan 14.6 -> 12.6 us)
        uint32_t tpc = 1;
        while (tpc < 32 && vt > (uint64_t)tpc * kScanWaves * kNumSms * kScanCtasPerSm) tpc <<= 1;
        gz.vote = 0;
        for (size_t r = r0; r < r0 + gz.jobs; ++r) {
            // (rounded down: the group's CTAs stay within one wave)
            const double share = std::floor(wave * estimate_weight(plans[order[r]]->h) / sumW);
            const uint32_t ec = (uint32_t)std::max(1.0, std::min((double)kEstimateCtas, share));
            cnt[r * 6 + 5] = ec;
            jobs[r].ectas = ec;
            uint32_t &c2 = cnt[r * 6 + 2];
            c2 = (c2 + tpc - 1) / tpc;
            jobs[r].vctas = c2;
            gz.vote += c2;
        }
        r0 += gz.jobs;
    }
    uint64_t tot[6] = {0, 0, 0, 0, 0, 0};
    for (int32_t i = 0; i < count; ++i)
        for (int k = 0; k < 6; ++k) tot[k] += cnt[(size_t)i * 6 + k];
    const size_t jb = align256(sizeof(Job) * count), ob = align256(sizeof(uint32_t) * (count + 1));
    size_t off = jb;
    for (int k = 0; k < 6; ++k) {
        b.off_offs[k] = off;
        off += ob;
        b.off_map[k] = off;
        off += align256(sizeof(uint32_t) * tot[k]);
    }
    b.off_gctr = off;
    off += align256(8 * sizeof(uint32_t) * std::max<size_t>(1, b.groups.size()));
    b.bytes.assign(off, 0);
    memcpy(b.bytes.data(), jobs.data(), sizeof(Job) * count);
    for (int k = 0; k < 6; ++k) {
        uint32_t *offs = reinterpret_cast<uint32_t *>(b.bytes.data() + b.off_offs[k]);
        uint32_t *map = reinterpret_cast<uint32_t *>(b.bytes.data() + b.off_map[k]);
        offs[0] = 0;
        for (int32_t i = 0; i < count; ++i) {
            const uint32_t c = cnt[(size_t)i * 6 + k];
            offs[i + 1] = offs[i] + c;
            for (uint32_t t = 0; t < c; ++t) map[offs[i] + t] = (uint32_t)i;
        }
    }
    // each group's first CTA and CTA count per kernel
    {
        const uint32_t *o[6];
        for (int k = 0; k < 6; ++k) o[k] = reinterpret_cast<const uint32_t *>(b.bytes.data() + b.off_offs[k]);
        size_t first = 0;
        for (Group &g : b.groups) {
            for (int k = 0; k < 6; ++k) {
                g.cta0[k] = o[k][first];
                g.ctas[k] = o[k][first + g.z.jobs] - o[k][first];
            }
            first += g.z.jobs;
        }
    }
    for (const Group &g : b.groups)
        if (g.z.dft_B) b.dft_bytes = std::max(b.dft_bytes, dft_scratch_bytes(g.ctas[1], g.z.dft_B) + 256);
    z.gather = (uint32_t)tot[0];
    z.select = (uint32_t)tot[1];
    z.vote = (uint32_t)tot[2];
    z.jobs = (uint32_t)count;
    return b;
}

cudaError_t launch_batch(const BatchLayout &b, const void *dev, int32_t count, cudaStream_t s,
                         cudaEvent_t *ev = nullptr) {
    const char *base = static_cast<const char *>(dev);
    Launch ln[6];
    for (int k = 0; k < 6; ++k) {
        ln[k].jobs = reinterpret_cast<const Job *>(base);
        ln[k].offs = reinterpret_cast<const uint32_t *>(base + b.off_offs[k]);
        ln[k].map = reinterpret_cast<const uint32_t *>(base + b.off_map[k]);
        ln[k].njobs = count;
        ln[k].cta0 = 0;
        ln[k].gctr = nullptr;
        memset(&ln[k].one, 0, sizeof(Job));
    }
    if (b.z.phase) return launch_phase(ln[1], b.z, s, ev);
    void *dft = b.dft_bytes ? static_cast<void *>(const_cast<char *>(base) + align256(b.bytes.size())) : nullptr;
    uint32_t *gctr = reinterpret_cast<uint32_t *>(const_cast<char *>(base) + b.off_gctr);
    return launch_pipeline(ln, b.z, b.groups, dft, s, ev, gctr);
}

sfft_status check_batch_args(sfft_plan *const *plans, const void *const *x, const void *const *idx,
                             const void *const *val, const void *kout, int32_t count) {
    if (count < 0 || (count > 0 && (!plans || !x || !idx || !val || !kout))) {
        set_error("NULL argument or negative count");
        return SFFT_EINVAL;
    }
    for (int32_t i = 0; i < count; ++i) {
        if (!plans[i] || !x[i] || !idx[i] || !val[i]) {
            set_error("NULL entry in batch arrays");
            return SFFT_EINVAL;
        }
        for (int32_t j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("a plan appears twice in one batch (each plan owns its scratch)");
                return SFFT_EINVAL;
            }
        if (plans[i]->h.method != plans[0]->h.method) {
            set_error("a batch mixes location methods (each method runs as a separate batch)");
            return SFFT_EINVAL;
        }
    }
    return SFFT_OK;
}

}  // namespace

extern "C" sfft_status sfft_execute_batch(sfft_plan *const *plans, const float *const *x_dev,
                                          int32_t *const *idx_dev, float *const *val_dev, int32_t *k_out_dev,
                                          int32_t count, void *stream) {
    sfft_status st = check_batch_args(plans, (const void *const *)x_dev, (const void *const *)idx_dev,
                                      (const void *const *)val_dev, k_out_dev, count);
    if (st != SFFT_OK || count == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int device = 0;
    cudaGetDevice(&device);
    BatchLayout b = build_batch(plans, x_dev, idx_dev, val_dev, k_out_dev, count);

    // key: count, then (plan id, x, idx, val) per job, then k_out
    std::vector<uint64_t> key;
    key.reserve(2 + 4 * count);
    key.push_back((uint64_t)count);
    for (int32_t i = 0; i < count; ++i) {
        key.push_back(plans[i]->id);
        key.push_back((uint64_t)(uintptr_t)x_dev[i]);
        key.push_back((uint64_t)(uintptr_t)idx_dev[i]);
        key.push_back((uint64_t)(uintptr_t)val_dev[i]);
    }
    key.push_back((uint64_t)(uintptr_t)k_out_dev);

    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->device != device || it->key != key) continue;
        GraphEntry &ge = *it;
        if (!ge.exec) {
            // second sighting: keep a persistent job buffer and capture the pipeline
            cudaError_t e = cudaMalloc(&ge.dev, b.dev_bytes());
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch graph)");
            SFFT_CUDA_TRY(cudaMemcpy(ge.dev, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice));
            cudaStream_t cap = nullptr;
            SFFT_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                cudaError_t le = launch_batch(b, ge.dev, count, cap);
                e = cudaStreamEndCapture(cap, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) {
                drop_entry(ge);
                g_graphs.erase(it);
                return cuda_fail(e, "capture batch graph");
            }
        }
        g_graphs.splice(g_graphs.begin(), g_graphs, it);
        SFFT_CUDA_TRY(cudaGraphLaunch(g_graphs.front().exec, s));
        return SFFT_OK;
    }
    // first sighting: remember the key, run through a staging slot
    GraphEntry ne;
    ne.key = key;
    ne.device = device;
    g_graphs.push_front(ne);
    while (g_graphs.size() > kMaxGraphs) {
        drop_entry(g_graphs.back());
        g_graphs.pop_back();
    }
    Slot &sl = g_slots[g_next_slot];
    g_next_slot = (g_next_slot + 1) % 4;
    if (sl.done) SFFT_CUDA_TRY(cudaEventSynchronize(sl.done));
    if (sl.device != device || sl.cap < b.dev_bytes()) {
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.done) cudaEventDestroy(sl.done);
        sl = Slot();
        const size_t cap = std::max<size_t>(b.dev_bytes(), 64 * 1024);
        SFFT_CUDA_TRY(cudaMallocHost(&sl.host, cap));
        SFFT_CUDA_TRY(cudaMalloc(&sl.dev, cap));
        SFFT_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        sl.cap = cap;
        sl.device = device;
    }
    memcpy(sl.host, b.bytes.data(), b.bytes.size());
    SFFT_CUDA_TRY(cudaMemcpyAsync(sl.dev, sl.host, b.bytes.size(), cudaMemcpyHostToDevice, s));
    SFFT_CUDA_TRY(launch_batch(b, sl.dev, count, s));
    SFFT_CUDA_TRY(cudaEventRecord(sl.done, s));
    return SFFT_OK;
}

extern "C" sfft_status sfft_execute_batch_timed(sfft_plan *const *plans, const float *const *x_dev,
                                                int32_t *const *idx_dev, float *const *val_dev,
                                                int32_t *k_out_dev, int32_t count, int32_t steps,
                                                float *total_ms, float *stage_ms, void *stream) {
    sfft_status st = check_batch_args(plans, (const void *const *)x_dev, (const void *const *)idx_dev,
                                      (const void *const *)val_dev, k_out_dev, count);
    if (st != SFFT_OK) return st;
    if (count == 0 || steps < 1 || !total_ms || !stage_ms) {
        set_error("timed batch needs count >= 1, steps >= 1 and output pointers");
        return SFFT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchLayout b = build_batch(plans, x_dev, idx_dev, val_dev, k_out_dev, count);
    void *dev = nullptr;
    SFFT_CUDA_TRY(cudaMalloc(&dev, b.dev_bytes()));
    constexpr int kStages = 6;
    std::vector<cudaEvent_t> ev((size_t)steps * (kStages + 1), nullptr);
    cudaError_t e = cudaMemcpy(dev, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    for (int32_t k = 0; k < steps && e == cudaSuccess; ++k)
        e = launch_batch(b, dev, count, s, &ev[(size_t)k * (kStages + 1)]);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    if (e == cudaSuccess) {
        for (int i = 0; i < kStages; ++i) stage_ms[i] = 0.f;
        for (int32_t k = 0; k < steps && e == cudaSuccess; ++k)
            for (int i = 0; i < kStages && e == cudaSuccess; ++i) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, ev[(size_t)k * (kStages + 1) + i],
                                         ev[(size_t)k * (kStages + 1) + i + 1]);
                stage_ms[i] += ms;
            }
        if (e == cudaSuccess) e = cudaEventElapsedTime(total_ms, ev.front(), ev.back());
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(dev);
    if (e != cudaSuccess) return cuda_fail(e, "timed batch");
    return SFFT_OK;
}

namespace {

// Per-thread resources of the host-buffer batch call: a copy stream and one
// event per chunk (for the calling thread's current device), the contiguous
// device output region and its pinned host image.
struct HostBatchRes {
    int device = -1;
    cudaStream_t copy = nullptr;
    cudaEvent_t fork = nullptr, chunk[kHostChunks] = {};
    void *out_dev = nullptr, *out_host = nullptr;
    size_t out_cap = 0;
};

cudaError_t host_batch_res(HostBatchRes &r, int device, size_t out_bytes) {
    cudaError_t e = cudaSuccess;
    if (r.device != device) {
        // resources of another device are left to process teardown
        r = HostBatchRes();
        e = cudaStreamCreateWithFlags(&r.copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
        for (int i = 0; i < kHostChunks && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&r.chunk[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        r.device = device;
    }
    if (r.out_cap < out_bytes) {
        if (r.out_dev) cudaFree(r.out_dev);
        if (r.out_host) cudaFreeHost(r.out_host);
        r.out_dev = r.out_host = nullptr;
        r.out_cap = 0;
        const size_t cap = std::max<size_t>(out_bytes, 64 * 1024);
        if ((e = cudaMalloc(&r.out_dev, cap)) != cudaSuccess) return e;
        if ((e = cudaMallocHost(&r.out_host, cap)) != cudaSuccess) return e;
        r.out_cap = cap;
    }
    return cudaSuccess;
}

}  // namespace

// Host buffers in, host buffers out.  The inputs go to the plans' device
// staging buffers on a copy stream in up to kHostChunks chunks of jobs; each
// chunk's batch runs on `stream` as soon as its copies land (the next chunk's
// copies continue meanwhile); every job's outputs go to one contiguous
// device region read back by a single copy.
extern "C" sfft_status sfft_execute_batch_host(sfft_plan *const *plans, const float *const *x_host,
                                               int32_t *const *idx_host, float *const *val_host,
                                               int32_t *k_out_host, int32_t count, void *stream) {
    sfft_status st = check_batch_args(plans, (const void *const *)x_host, (const void *const *)idx_host,
                                      (const void *const *)val_host, k_out_host, count);
    if (st != SFFT_OK || count == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int device = 0;
    SFFT_CUDA_TRY(cudaGetDevice(&device));
    // output layout: per job idx int32[K] and val complex64[K], then k_out[count]
    std::vector<size_t> oi(count), ov(count);
    size_t out = 0;
    for (int32_t i = 0; i < count; ++i) {
        oi[i] = out;
        out += align256(sizeof(int32_t) * plans[i]->K);
        ov[i] = out;
        out += align256(sizeof(float2) * plans[i]->K);
    }
    const size_t ok = out;
    out += sizeof(int32_t) * count;
    static thread_local HostBatchRes res;
    SFFT_CUDA_TRY(host_batch_res(res, device, out));
    char *od = static_cast<char *>(res.out_dev);
    std::vector<const float *> xd(count);
    std::vector<int32_t *> id(count);
    std::vector<float *> vd(count);
    for (int32_t i = 0; i < count; ++i) {
        sfft_plan *p = plans[i];
        if (!p->stage) SFFT_CUDA_TRY(cudaMalloc(&p->stage, stage_bytes(p)));  // x first
        xd[i] = static_cast<const float *>(p->stage);
        id[i] = reinterpret_cast<int32_t *>(od + oi[i]);
        vd[i] = reinterpret_cast<float *>(od + ov[i]);
    }
    int32_t *kd = reinterpret_cast<int32_t *>(od + ok);
    const int chunks = std::min<int>(kHostChunks, count);
    // the copy stream follows the caller's earlier work
    SFFT_CUDA_TRY(cudaEventRecord(res.fork, s));
    SFFT_CUDA_TRY(cudaStreamWaitEvent(res.copy, res.fork, 0));
    for (int c = 0; c < chunks; ++c) {
        const int32_t f0 = (int32_t)((int64_t)count * c / chunks), f1 = (int32_t)((int64_t)count * (c + 1) / chunks);
        for (int32_t i = f0; i < f1; ++i)
            SFFT_CUDA_TRY(cudaMemcpyAsync(const_cast<float *>(xd[i]), x_host[i], sizeof(float2) * plans[i]->N,
                                          cudaMemcpyHostToDevice, res.copy));
        SFFT_CUDA_TRY(cudaEventRecord(res.chunk[c], res.copy));
    }
    for (int c = 0; c < chunks; ++c) {
        const int32_t f0 = (int32_t)((int64_t)count * c / chunks), f1 = (int32_t)((int64_t)count * (c + 1) / chunks);
        SFFT_CUDA_TRY(cudaStreamWaitEvent(s, res.chunk[c], 0));
        st = sfft_execute_batch(plans + f0, xd.data() + f0, id.data() + f0, vd.data() + f0, kd + f0, f1 - f0,
                                stream);
        if (st != SFFT_OK) return st;
    }
    SFFT_CUDA_TRY(cudaMemcpyAsync(res.out_host, od, out, cudaMemcpyDeviceToHost, s));
    SFFT_CUDA_TRY(cudaStreamSynchronize(s));
    const char *oh = static_cast<const char *>(res.out_host);
    memcpy(k_out_host, oh + ok, sizeof(int32_t) * count);
    for (int32_t i = 0; i < count; ++i) {
        memcpy(idx_host[i], oh + oi[i], sizeof(int32_t) * plans[i]->K);
        memcpy(val_host[i], oh + ov[i], sizeof(float2) * plans[i]->K);
    }
    return SFFT_OK;
}

// ------------------------------------------------------------ single stages
extern "C" sfft_status sfft_bucketize(sfft_plan *p, const float *x_dev, float *zhat_dev, void *stream) {
    if (!p || !x_dev || !zhat_dev) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Launch ln = single(make_job(p, x_dev, nullptr, nullptr, nullptr));
    const Sizes z = plan_sizes(p);
    SFFT_CUDA_TRY(z.stream ? launch_gather_stream(ln, z.gather, z.stream_smem, s) : launch_gather(ln, z.gather, s));
    if (z.dft_B) {
        // the plan's tensor-core DFT, as in the pipeline
        uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<char *>(p->dft) + dft_scratch_bytes(z.select, z.dft_B));
        SFFT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
        SFFT_CUDA_TRY(launch_dft(ln, z.select, z.dft_B, p->dft, err, s));
        const uint32_t mpad = (z.select + kDftRowTile - 1) / kDftRowTile * kDftRowTile;
        SFFT_CUDA_TRY(launch_fft_select(ln, z.select, z.max_B, 0, 0, s, dft_partials(p->dft, z.select, z.dft_B), mpad,
                                        err));
    } else {
        SFFT_CUDA_TRY(launch_fft_select(ln, z.select, z.max_B, 0, 0, s));
    }
    SFFT_CUDA_TRY(cudaMemcpyAsync(zhat_dev, p->h.zhat, sizeof(float2) * p->L * p->B, cudaMemcpyDeviceToDevice, s));
    return SFFT_OK;
}

extern "C" sfft_status sfft_select(sfft_plan *p, const float *zhat_dev, int32_t *sel_dev, void *stream) {
    if (!p || !zhat_dev || !sel_dev) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Launch ln = single(make_job(p, nullptr, nullptr, nullptr, nullptr));
    SFFT_CUDA_TRY(cudaMemcpyAsync(p->h.zhat, zhat_dev, sizeof(float2) * p->L * p->B, cudaMemcpyDeviceToDevice, s));
    SFFT_CUDA_TRY(launch_fft_select(ln, p->h.L, p->h.B, 1, 0, s));
    SFFT_CUDA_TRY(
        cudaMemcpyAsync(sel_dev, p->h.sel, sizeof(int32_t) * p->L * p->nsel, cudaMemcpyDeviceToDevice, s));
    return SFFT_OK;
}

extern "C" sfft_status sfft_vote(sfft_plan *p, const int32_t *sel_dev, int32_t *cand_dev, int32_t *n_cand_dev,
                                 int64_t cap, void *stream) {
    if (!p || !sel_dev || !cand_dev || !n_cand_dev) {
        set_error("NULL argument");
        return SFFT_EINVAL;
    }
    if (cap < p->cap) {
        set_error("candidate buffer smaller than the plan's candidate capacity");
        return SFFT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Launch ln = single(make_job(p, nullptr, nullptr, nullptr, nullptr));
    SFFT_CUDA_TRY(cudaMemsetAsync(n_cand_dev, 0, sizeof(int32_t), s));
    SFFT_CUDA_TRY(launch_flags_from_sel(p->d, p->h.L, sel_dev, s));
    SFFT_CUDA_TRY(launch_vote(ln, p->h.vtiles, kVoteCandidates, p->h.L, false, p->h.L * p->h.B * 2, p->h.B,
                              cand_dev, n_cand_dev, s));
    return SFFT_OK;
}

extern "C" sfft_status sfft_estimate(sfft_plan *p, const float *zhat_dev, const int32_t *cand_dev, int64_t n_cand,
                                     float *est_dev, void *stream) {
    if (!p || n_cand < 0 || (n_cand > 0 && (!zhat_dev || !cand_dev || !est_dev))) {
        set_error("NULL argument or negative count");
        return SFFT_EINVAL;
    }
    if (n_cand > (int64_t)p->N) {
        set_error("more candidates than frequencies");
        return SFFT_EINVAL;
    }
    SFFT_CUDA_TRY(launch_estimate_list(p->d, p->h.L, reinterpret_cast<const float2 *>(zhat_dev), cand_dev,
                                       (uint32_t)n_cand, reinterpret_cast<float2 *>(est_dev),
                                       static_cast<cudaStream_t>(stream)));
    return SFFT_OK;
}

// -------------------------------------------------------------------- misc
extern "C" const char *sfft_status_string(sfft_status s) {
    switch (s) {
        case SFFT_OK: return "ok";
        case SFFT_EINVAL: return "invalid argument";
        case SFFT_ENOMEM: return "out of memory";
        case SFFT_ECUDA: return "CUDA error";
        case SFFT_EBUSY: return "busy";
        case SFFT_ETIMEDOUT: return "timed out";
        case SFFT_EPENDING: return "pending";
        case SFFT_ENOTIMPL: return "not implemented";
    }
    return "unknown status";
}

extern "C" const char *sfft_last_error(void) { return g_err.c_str(); }
