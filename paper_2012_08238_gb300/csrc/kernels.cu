// Hot-path kernels of the flat-window voting sparse FFT (steps a1..a7).
//
// Every kernel takes a Launch descriptor: one job by value (plain execute) or
// an array of jobs in device memory with a per-kernel CTA prefix (batched
// execute).  A CTA locates its job, copies the job's PlanDev into shared
// memory and works on one tile of that job.
//
// Pipeline per job: k_gather (a1) -> k_fft_select (a2, a3; its last CTA also
// builds the vote tables) -> k_scan_bits or k_vote_scan (a4, a5: survivors of
// the median bound) -> k_estimate_tab or k_estimate_surv (a6: estimates,
// keeps key >= theta; the job's last CTA then takes the top K, a7, running
// the unpruned fallback pass first when fewer than K estimates reached theta).
#include <cooperative_groups.h>
#include <mutex>
#include <math_constants.h>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

constexpr int kThreads = 256;  // every kernel but the comb
constexpr int kCombThreads = 1024;
constexpr uint32_t kTwSmemMaxB = 8192;  // FFT twiddles staged in shared memory up to this B

__device__ __forceinline__ void locate(const Launch &ln, uint32_t bid, Job &job, uint32_t &local) {
    if (ln.jobs == nullptr) {
        job = ln.one;
        local = bid;
        return;
    }
    const uint32_t jid = __ldg(ln.map + bid);
    job = ln.jobs[jid];
    local = bid - __ldg(ln.offs + jid);
}

// Copy the job's plan descriptor into shared memory (call from all threads,
// then __syncthreads()).
__device__ __forceinline__ void load_plan(PlanDev &dst, const PlanDev *src) {
    static_assert(sizeof(PlanDev) % 8 == 0, "PlanDev must be 8-byte sized");
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(&dst);
    for (uint32_t i = threadIdx.x; i < sizeof(PlanDev) / 8; i += blockDim.x) d[i] = __ldg(s + i);
}

// Locate + load in one call; every kernel starts with it.
__device__ __forceinline__ void enter(const Launch &ln, PlanDev &P, Job &J, uint32_t &s_local) {
    if (threadIdx.x == 0) {
        Job j;
        uint32_t loc;
        locate(ln, blockIdx.x, j, loc);
        J = j;
        s_local = loc;
    }
    __syncthreads();
    load_plan(P, J.p);
    __syncthreads();
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// sigma^-1 mod 32 for odd sigma: sigma^2 = 1 (mod 8) holds 3 bits, one
// Newton step doubles them
__device__ __forceinline__ uint32_t inv_mod32(uint32_t sigma) { return sigma * (2u - sigma * sigma); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// True when the pruned pass could not certify the top K: fewer than K
// candidates reached theta.  The fallback pass then records (and counts)
// every candidate.
__device__ __forceinline__ bool needs_fallback(const PlanDev &P) { return __ldcg(P.ctr + kNGe) < P.K; }

// Inclusive sum over a block of NW warps (warp shuffles + NW warp totals).
template <int NW>
__device__ __forceinline__ uint32_t block_incl_scan_n(uint32_t v, uint32_t *wsum) {
    static_assert(NW >= 1 && NW <= 32, "one warp scans the warp totals");
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < (uint32_t)NW ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= (uint32_t)o) s += y;
        }
        if (lane < (uint32_t)NW) wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t r = x + (wid ? wsum[wid - 1] : 0u);
    __syncthreads();  // wsum free again
    return r;
}

// Inclusive sum over a 256-thread block.
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *wsum) {
    return block_incl_scan_n<kThreads / 32>(v, wsum);
}

// k-th largest (1 <= k <= n) of n 32-bit keys by four 8-bit radix passes over
// a 256-bin histogram whose suffix sums come from one block scan per pass.
// Returns the key; *s_need is how many keys equal to it rank within the top k.
// Called by all NT threads of the block (NT a multiple of 256, at most 1024;
// wsum holds NT / 32 words).
template <int NT, bool kGlobal>
__device__ uint32_t block_kth_largest(const uint32_t *v, uint32_t n, uint32_t k, uint32_t *hist, uint32_t *wsum,
                                      uint32_t *s_prefix, uint32_t *s_need) {
    static_assert(NT % 256 == 0 && NT <= 1024, "256 bins, one per thread of the first 256");
    if (threadIdx.x == 0) {
        *s_prefix = 0;
        *s_need = k;
    }
    __syncthreads();
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 24 - 8 * pass;
        const uint32_t pmask = pass == 0 ? 0u : (0xFFFFFFFFu << (sh + 8));
        const uint32_t prefix = *s_prefix, need = *s_need;
        if (threadIdx.x < 256) hist[threadIdx.x] = 0;
        __syncthreads();
        // one atomic per distinct bin and warp (equal exponents are common)
        for (uint32_t i0 = threadIdx.x & ~31u; i0 < n; i0 += NT) {
            const uint32_t i = i0 + (threadIdx.x & 31u);
            uint32_t bin = 256u;  // none
            if (i < n) {
                const uint32_t u = kGlobal ? __ldcg(v + i) : v[i];
                if ((u & pmask) == prefix) bin = (u >> sh) & 255u;
            }
            const uint32_t m = __match_any_sync(0xFFFFFFFFu, bin);
            if (bin < 256u && (threadIdx.x & 31u) == (uint32_t)(__ffs(m) - 1)) atomicAdd(&hist[bin], __popc(m));
        }
        __syncthreads();
        const uint32_t c = threadIdx.x < 256 ? hist[255 - threadIdx.x] : 0u;  // thread t scans bins from the top
        const uint32_t incl = block_incl_scan_n<NT / 32>(c, wsum);
        const uint32_t excl = incl - c;
        if (c > 0 && excl < need && need <= incl) {
            *s_prefix = prefix | ((255u - threadIdx.x) << sh);
            *s_need = need - excl;
        }
        __syncthreads();
    }
    return *s_prefix;
}

// The k1-th and k2-th largest of n 32-bit keys (1 <= k1, k2 <= n < 65536) in
// one sequence of four radix passes: two 256-bin histograms per pass, their
// counts packed into 16-bit halves of one word for a single block scan.
// Returns the k1-th key (*s_need: keys equal to it within the top k1) and
// stores the k2-th in *kth2.  hist holds 256 words.  Called by all 256 threads.
__device__ uint32_t block_kth_largest2(const uint32_t *v, uint32_t n, uint32_t k1, uint32_t k2, uint32_t *hist,
                                       uint32_t *wsum, uint32_t *s_prefix, uint32_t *s_need, uint32_t *kth2) {
    __shared__ uint32_t s_prefix2, s_need2;
    if (threadIdx.x == 0) {
        *s_prefix = 0;
        *s_need = k1;
        s_prefix2 = 0;
        s_need2 = k2;
    }
    __syncthreads();
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 24 - 8 * pass;
        const uint32_t pmask = pass == 0 ? 0u : (0xFFFFFFFFu << (sh + 8));
        const uint32_t p1 = *s_prefix, need1 = *s_need, p2 = s_prefix2, need2 = s_need2;
        hist[threadIdx.x] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
            const uint32_t u = v[i];
            const uint32_t add = ((u & pmask) == p1 ? 1u : 0u) | ((u & pmask) == p2 ? 0x10000u : 0u);
            if (add) atomicAdd(&hist[(u >> sh) & 255u], add);
        }
        __syncthreads();
        const uint32_t c = hist[255 - threadIdx.x];  // thread t scans bins from the top
        const uint32_t incl = block_incl_scan(c, wsum);
        const uint32_t excl = incl - c;
        const uint32_t c1 = c & 0xFFFFu, i1 = incl & 0xFFFFu, e1 = excl & 0xFFFFu;
        const uint32_t c2 = c >> 16, i2 = incl >> 16, e2 = excl >> 16;
        if (c1 > 0 && e1 < need1 && need1 <= i1) {
            *s_prefix = p1 | ((255u - threadIdx.x) << sh);
            *s_need = need1 - e1;
        }
        if (c2 > 0 && e2 < need2 && need2 <= i2) {
            s_prefix2 = p2 | ((255u - threadIdx.x) << sh);
            s_need2 = need2 - e2;
        }
        __syncthreads();
    }
    *kth2 = s_prefix2;
    return *s_prefix;
}

// Round-half-up flat-filter hash of frequency f in loop l: bucket h and the
// offset o from the bucket centre, returned as o + half in [0, N/B).
__device__ __forceinline__ void hash_freq(const PlanDev &P, uint32_t sigma, uint32_t f, uint32_t &h,
                                          uint32_t &opos) {
    const uint32_t p = (sigma * f) & P.mask;
    const uint32_t hh = (p + P.half) >> P.shift;  // in [0, B]
    opos = p + P.half - (hh << P.shift);
    h = hh & (P.B - 1);
}

// ------------------------------------------------------------------ a1
// z_l[j] partial sums: sum over the rounds of one chunk of
// g(m) * x[(sigma_l m + tau_l) mod N] for the window positions m = j (mod B).
// The job chooses the chunking (rpc rounds per chunk).
__global__ void __launch_bounds__(kThreads) k_gather(Launch ln) {
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ float2 red[kThreads];
    enter(ln, P, J, s_local);

    const uint32_t local = s_local;
    const uint32_t tile = local % P.tiles;
    const uint32_t rest = local / P.tiles;
    const uint32_t l = rest % P.L;
    const uint32_t chunk = rest / P.L;
    const uint32_t TB = P.tb;
    const uint32_t PP = kThreads / TB;  // threads sharing one bucket
    const uint32_t jt = threadIdx.x & (TB - 1);
    const uint32_t s = threadIdx.x / TB;
    const uint32_t j = tile * TB + jt;
    const uint32_t r0 = chunk * J.rpc;
    const uint32_t r1 = min(P.rounds, r0 + J.rpc);
    const uint32_t sig = P.sigma[l], tau = P.tau[l], mask = P.mask, B = P.B, halfw = P.halfw;
    const uint32_t jq = (j + halfw) & (B - 1);  // position of bucket j inside a round
    const float2 *__restrict__ x = J.x;
    const float *__restrict__ taps = P.taps;

    float ar = 0.f, ai = 0.f;
#pragma unroll 8
    for (uint32_t r = r0 + s; r < r1; r += PP) {
        const uint32_t q = r * B + jq;
        const uint32_t i = (sig * (q - halfw) + tau) & mask;  // uint32 wrap: exact mod N
        const float g = __ldg(taps + q);
        const float2 v = __ldg(x + i);
        ar = fmaf(g, v.x, ar);
        ai = fmaf(g, v.y, ai);
    }
    float2 *dst = P.partial + ((size_t)chunk * P.L + l) * B + j;
    if (PP == 1) {
        *dst = make_float2(ar, ai);
        return;
    }
    red[threadIdx.x] = make_float2(ar, ai);
    __syncthreads();
    if (s == 0) {
        float2 acc = red[jt];
        for (uint32_t k = 1; k < PP; ++k) {
            acc.x += red[jt + k * TB].x;
            acc.y += red[jt + k * TB].y;
        }
        *dst = acc;
    }
}

// Bitonic sort of n (power of two) 64-bit keys in shared memory, descending.
__device__ void bitonic_desc(unsigned long long *a, uint32_t n) {
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = a[i], y = a[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (x < y) : (x > y)) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Same, for (key, payload) pairs; ascending when asc is set.
__device__ void bitonic_pairs(unsigned long long *a, uint32_t *pay, uint32_t n, bool asc) {
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = a[i], y = a[ixj];
                    const bool up = ((i & k) == 0) == asc;
                    if (up ? (x > y) : (x < y)) {
                        a[i] = y;
                        a[ixj] = x;
                        const uint32_t t = pay[i];
                        pay[i] = pay[ixj];
                        pay[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Strong-bit threshold of the vote tables: a loop is "strong" for f when
// |zhat|^2 * max|1/G~|^2 >= theta/2; with fewer than M strong loops the median
// estimate is provably below theta.
__device__ __forceinline__ bool strong_energy(float en, float gmul, float thr) { return en * gmul >= thr; }

// theta = 1/4 of a lower bound of the K-th largest bucket energy over all
// loops (the minimum over loops of each loop's ceil(K/L)-th largest energy):
// a guess at a lower bound of the K-th largest estimate.  Exactness never
// depends on it; a guess that is too high only sends the job to the fallback
// pass.
__device__ __forceinline__ float theta_from(float min_kth) {
    float theta = 0.25f * min_kth;
    if (!(theta >= 0.f) || isinf(theta)) theta = 0.f;
    return theta;
}

// Loop l's packed bits for the register-table scan: lane word j holds the
// bit of every bucket h = j (mod 32) at (sigma^-1 (h >> (log2 B - 5))) mod
// 32, so that the scan's one rotate puts the bit of f + kN/G (G = B/32) at
// position k 32/G.  bit(h) is bucket h's bit: strong for the median
// estimator, kept for the mean.
template <class Bit>
__device__ __forceinline__ uint32_t packed_word(const PlanDev &P, uint32_t l, uint32_t j, Bit bit) {
    const uint32_t sh = P.logB - 5, si = inv_mod32(P.sigma[l]);
    uint32_t word = 0;
#pragma unroll
    for (uint32_t m = 0; m < 16; ++m) {
        const uint32_t h = j + 32 * m;
        if (h < P.B) word |= (uint32_t)bit(h) << ((si * (h >> sh)) & 31u);
    }
    return word;
}

// Clustered tail of k_fft_select for loop l (all threads of every CTA of the
// job's cluster): theta from the loops' ceil(K/L)-th energies read through
// distributed shared memory, then this loop's flags (kept | strong << 8) and
// packed strong bits.  Cluster rank 0 publishes theta and resets the job's
// counters.
__device__ void cluster_tables(const PlanDev &P, uint32_t l, uint32_t kqv, const uint32_t *en_s,
                               const uint8_t *kept_s, uint16_t *frow) {
    namespace cg = cooperative_groups;
    __shared__ float s_kq, s_th;
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) s_kq = __uint_as_float(kqv);
    cl.sync();
    if (threadIdx.x < 32) {
        float mn = INFINITY;
        for (uint32_t ll = threadIdx.x; ll < P.L; ll += 32) mn = fminf(mn, *cl.map_shared_rank(&s_kq, ll));
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        if (threadIdx.x == 0) {
            const float theta = theta_from(mn);
            s_th = theta;
            if (l == 0) {
                P.ctr[kTheta] = __float_as_uint(theta);
                P.ctr[kSelDone] = 0;
                P.ctr[kNCand] = 0;
                P.ctr[kNSurv] = 0;
                P.ctr[kNGe] = 0;
                P.ctr[kNRec2] = 0;
                P.ctr[kEstDone] = 0;
            }
        }
    }
    cl.sync();  // no CTA leaves while another still reads its s_kq
    const float thr = 0.5f * s_th;
    const float gmul = P.ginv2max * (1.0f + 1.0f / 1024.0f);
    const uint32_t B = P.B;
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x)
        frow[k] = (uint16_t)(kept_s[k] | (strong_energy(__uint_as_float(en_s[k]), gmul, thr) ? 256u : 0u));
    const bool mean = P.estimator == kEstMean;
    if (P.use_bits && threadIdx.x < 32)
        P.packed[l * 32 + threadIdx.x] = packed_word(P, l, threadIdx.x, [&](uint32_t h) {
            return mean ? kept_s[h] != 0 : strong_energy(__uint_as_float(en_s[h]), gmul, thr);
        });
}

// -------------------------------------------------------------- a2 + a3
// One CTA per (job, loop): sum the gather partials, B-point radix-2 FFT in
// shared memory, bucket energies, and the nsel kept buckets (energy
// descending, ties to the lower bucket).  The last CTA of a job derives the
// prune threshold theta and the kept/strong tables for all loops.
// select_only: the bucket values are already in P.zhat; the kept buckets are
// also listed in rank order in P.sel.
// clustered: the launch groups each job's L CTAs into one thread-block
// cluster (every job has this L and B <= kClusterMaxB); then, instead of a
// last CTA building every loop's tables, each CTA reads the other loops'
// order statistics from their shared memory, derives theta and builds its
// own loop's tables.
__global__ void __launch_bounds__(kThreads, 6) k_fft_select(Launch ln, int select_only, int clustered) {
    // B values, B energies, B/2 twiddles (B <= kTwSmemMaxB), B kept bytes (clustered)
    extern __shared__ unsigned long long sm[];
    float2 *buf = reinterpret_cast<float2 *>(sm);
    uint32_t *en_s;
    const float2 *tw;
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ int s_last;
    __shared__ float s_theta;
    __shared__ uint32_t s_hist[256], s_wsum[8], s_prefix, s_need;
    enter(ln, P, J, s_local);

    const uint32_t l = s_local, B = P.B, logB = P.logB;
    en_s = reinterpret_cast<uint32_t *>(buf + B);
    float2 *tw_s = B <= kTwSmemMaxB ? reinterpret_cast<float2 *>(en_s + B) : nullptr;
    tw = tw_s ? tw_s : P.tw;
    float2 *zrow = P.zhat + (size_t)l * B;
    float *erow = P.energy + (size_t)l * B;
    uint16_t *frow = P.flags + (size_t)l * B;
    if (!select_only) {
        const uint32_t nchunk = J.nchunk;
        if (tw_s)
            for (uint32_t k = threadIdx.x; k < B / 2; k += blockDim.x) tw_s[k] = __ldg(P.tw + k);
        const size_t cstride = (size_t)P.L * B;
        for (uint32_t j = threadIdx.x; j < B; j += blockDim.x) {
            // chunk order, up to 8 chunk loads in flight at once
            float2 acc = make_float2(0.f, 0.f);
            const float2 *src = P.partial + (size_t)l * B + j;
            for (uint32_t c0 = 0; c0 < nchunk; c0 += 8) {
                float2 v[8];
#pragma unroll
                for (uint32_t k = 0; k < 8; ++k)
                    v[k] = c0 + k < nchunk ? __ldcg(src + (c0 + k) * cstride) : make_float2(0.f, 0.f);
#pragma unroll
                for (uint32_t k = 0; k < 8; ++k) {
                    if (c0 + k < nchunk) {
                        acc.x += v[k].x;
                        acc.y += v[k].y;
                    }
                }
            }
            buf[__brev(j) >> (32 - logB)] = acc;
        }
        __syncthreads();
        // iterative radix-2 decimation in time, twiddles exp(-2 pi i k / (2h))
        for (uint32_t hs = 0; hs < logB; ++hs) {
            const uint32_t h = 1u << hs;
            for (uint32_t bf = threadIdx.x; bf < B / 2; bf += blockDim.x) {
                const uint32_t k = bf & (h - 1);
                const uint32_t i0 = ((bf >> hs) << (hs + 1)) + k;
                const uint32_t i1 = i0 + h;
                const float2 w = tw[k << (logB - 1 - hs)];
                const float2 a = buf[i0];
                const float2 t = cmul(w, buf[i1]);
                buf[i0] = make_float2(a.x + t.x, a.y + t.y);
                buf[i1] = make_float2(a.x - t.x, a.y - t.y);
            }
            __syncthreads();
        }
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z = buf[k];
            const float e = z.x * z.x + z.y * z.y;
            zrow[k] = z;
            erow[k] = e;
            en_s[k] = __float_as_uint(e);
        }
    } else {
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z = zrow[k];
            const float e = z.x * z.x + z.y * z.y;
            erow[k] = e;
            en_s[k] = __float_as_uint(e);
        }
    }
    __syncthreads();
    if (select_only) {
        // rank-ordered list for the single-stage entry point
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x)
            sm[k] = ((unsigned long long)en_s[k] << 32) | (uint32_t)(~k);
        __syncthreads();
        bitonic_desc(sm, B);
        for (uint32_t s = threadIdx.x; s < P.nsel; s += blockDim.x)
            P.sel[(size_t)l * P.nsel + s] = (int32_t)(~(uint32_t)sm[s]);
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) frow[k] = 0;
        __syncthreads();
        for (uint32_t s = threadIdx.x; s < P.nsel; s += blockDim.x) frow[~(uint32_t)sm[s]] = 1;
    } else {
        // kept = energy above the nsel-th largest, plus the lowest-index ties;
        // also this loop's ceil(K/L)-th largest energy: their minimum over
        // loops is at most the K-th largest energy of all loops (each loop has
        // ceil(K/L) values at or above it)
        const uint32_t kq = (P.K + P.L - 1) / P.L;
        uint32_t kqv = 0;
        const uint32_t kth = block_kth_largest2(en_s, B, P.nsel, min(kq, B), s_hist, s_wsum, &s_prefix, &s_need,
                                                &kqv);
        if (kq > B) kqv = 0;
        const uint32_t need_eq = s_need;
        const uint32_t per = (B + kThreads - 1) / kThreads;
        const uint32_t k0 = min(B, threadIdx.x * per), k1 = min(B, k0 + per);
        uint32_t eq = 0;
        for (uint32_t k = k0; k < k1; ++k) eq += en_s[k] == kth;
        uint32_t r = block_incl_scan(eq, s_wsum) - eq;  // equal keys before k0
        uint8_t *kept_s = reinterpret_cast<uint8_t *>(tw_s + B / 2);  // clustered only
        for (uint32_t k = k0; k < k1; ++k) {
            const uint32_t e = en_s[k];
            bool keep = e > kth;
            if (e == kth) keep = r++ < need_eq;
            if (clustered)
                kept_s[k] = keep ? 1 : 0;
            else
                frow[k] = keep ? 1 : 0;
        }
        if (clustered) {
            cluster_tables(P, l, kqv, en_s, kept_s, frow);
            return;
        }
        if (threadIdx.x == 0) P.loopkth[l] = __uint_as_float(kqv);
    }

    // ---- last CTA of the job: theta and the kept/strong tables
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(P.ctr + kSelDone, 1u) == P.L - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t total = P.L * B;
    // theta = 1/4 of a lower bound of the K-th largest bucket energy over all
    // loops: a guess at a lower bound of the K-th largest estimate.  Exactness
    // never depends on it; a guess that is too high only sends the job to the
    // fallback pass.
    if (threadIdx.x < 32) {
        float mn = INFINITY;
        for (uint32_t ll = threadIdx.x; ll < P.L; ll += 32) mn = fminf(mn, __ldcg(P.loopkth + ll));
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        if (threadIdx.x == 0) {
            const float theta = select_only ? 0.f : theta_from(mn);  // single-stage select: no pruning downstream
            s_theta = theta;
            P.ctr[kTheta] = __float_as_uint(theta);
        }
    }
    __syncthreads();
    // a loop is "strong" for f when |zhat|^2 * max|1/G~|^2 >= theta/2; with
    // fewer than M strong loops the median estimate is provably below theta
    const float thr = 0.5f * s_theta;
    const float gmul = P.ginv2max * (1.0f + 1.0f / 1024.0f);
    if ((total & 3u) == 0) {
        // four buckets per thread and step, four steps' loads issued together
        const float4 *e4 = reinterpret_cast<const float4 *>(P.energy);
        uint2 *f4 = reinterpret_cast<uint2 *>(P.flags);
        const uint32_t n4 = total / 4;
        for (uint32_t b0 = threadIdx.x; b0 < n4; b0 += 4 * kThreads) {
            float4 en[4];
            uint2 fl[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint32_t i = b0 + u * kThreads;
                if (i < n4) {
                    en[u] = __ldcg(e4 + i);
                    fl[u] = __ldcg(f4 + i);
                }
            }
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint32_t i = b0 + u * kThreads;
                if (i < n4) {
                    const uint32_t s0 = (fl[u].x & 1u) | (strong_energy(en[u].x, gmul, thr) ? 256u : 0u);
                    const uint32_t s1 = ((fl[u].x >> 16) & 1u) | (strong_energy(en[u].y, gmul, thr) ? 256u : 0u);
                    const uint32_t s2 = (fl[u].y & 1u) | (strong_energy(en[u].z, gmul, thr) ? 256u : 0u);
                    const uint32_t s3 = ((fl[u].y >> 16) & 1u) | (strong_energy(en[u].w, gmul, thr) ? 256u : 0u);
                    f4[i] = make_uint2(s0 | (s1 << 16), s2 | (s3 << 16));
                }
            }
        }
    } else {
        for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
            const float en = __ldcg(P.energy + e);
            uint16_t f = __ldcg(reinterpret_cast<const unsigned short *>(P.flags) + e) & 1u;
            if (strong_energy(en, gmul, thr)) f |= 256;
            P.flags[e] = f;
        }
    }
    if (P.use_bits) {
        __syncthreads();  // the flags above are complete
        const bool mean = P.estimator == kEstMean;
        for (uint32_t idx = threadIdx.x; idx < P.L * 32; idx += blockDim.x) {
            const uint32_t ll = idx >> 5;
            const float *er = P.energy + (size_t)ll * B;
            const unsigned short *fr = reinterpret_cast<const unsigned short *>(P.flags) + (size_t)ll * B;
            P.packed[idx] = packed_word(P, ll, idx & 31, [&](uint32_t h) {
                return mean ? (__ldcg(fr + h) & 1u) != 0 : strong_energy(__ldcg(er + h), gmul, thr);
            });
        }
    }
    if (threadIdx.x == 0) {
        P.ctr[kSelDone] = 0;
        P.ctr[kNCand] = 0;
        P.ctr[kNSurv] = 0;
        P.ctr[kNGe] = 0;
        P.ctr[kNRec2] = 0;
        P.ctr[kEstDone] = 0;
    }
}

// ------------------------------------------------------------------ a6
// Batcher's odd-even merge sort on the next power-of-two number of slots, with
// every comparator that touches a slot >= N dropped (those slots would hold
// +inf and never move): 24 comparators for N = 8, 42 for 12, 63 for 16.
template <int N>
__device__ __forceinline__ void sort_net(float *a) {
    constexpr int S = N <= 8 ? 8 : (N <= 16 ? 16 : 32);
#pragma unroll
    for (int p = 1; p < S; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
#pragma unroll
            for (int j = k % p; j <= S - 1 - k; j += 2 * k) {
#pragma unroll
                for (int i = 0; i < k; ++i) {
                    if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                        const float x = a[i + j], y = a[i + j + k];
                        a[i + j] = fminf(x, y);
                        a[i + j + k] = fmaxf(x, y);
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ float median_sorted(const float *a, uint32_t n) {
    return (n & 1) ? a[n / 2] : 0.5f * (a[n / 2 - 1] + a[n / 2]);
}

// Bucket value z of a frequency turned by exp(-2 pi i tau f / N) and scaled by
// g = 1/G~(o); ph = (tau f mod N) 2^(32 - log2 N) is the turn as a 32-bit
// fraction.
__device__ __forceinline__ float2 turn_scale(float2 z, float2 g, uint32_t ph) {
    float sn, cs;
    // the signed fraction is an angle in [-pi, pi), where the fast intrinsic's
    // absolute error (~2^-21) is far inside the value tolerance
    __sincosf((float)(int32_t)ph * (2.0f * CUDART_PI_F / 4294967296.0f), &sn, &cs);
    const float2 zp = make_float2(z.x * cs + z.y * sn, z.y * cs - z.x * sn);
    return cmul(zp, g);
}

// Per-loop energy-concentration estimate of frequency f in loop l:
// zhat_l[h] * exp(-2 pi i tau_l f / N) / G~(o).
__device__ __forceinline__ float2 loop_estimate(const PlanDev &P, const float2 *zhat, uint32_t l, uint32_t f) {
    uint32_t h, opos;
    hash_freq(P, P.sigma[l], f, h, opos);
    const float2 z = zhat[(size_t)l * P.B + h];
    const float2 g = __ldg(P.ginv + opos);
    return turn_scale(z, g, (P.tau[l] << (32 - P.logN)) * f);
}

template <int LT>
__device__ float2 median_estimate(const PlanDev &P, const float2 *zhat, uint32_t f) {
    if constexpr (LT > 0) {
        float re[LT], im[LT];
#pragma unroll
        for (int l = 0; l < LT; ++l) {
            const float2 v = loop_estimate(P, zhat, l, f);
            re[l] = v.x;
            im[l] = v.y;
        }
        sort_net<LT>(re);
        sort_net<LT>(im);
        return make_float2(median_sorted(re, LT), median_sorted(im, LT));
    } else {
        float re[kMaxL], im[kMaxL];
        const uint32_t L = P.L;
        for (uint32_t l = 0; l < L; ++l) {
            const float2 v = loop_estimate(P, zhat, l, f);
            // insertion into the sorted prefixes
            uint32_t a = l, b = l;
            while (a > 0 && re[a - 1] > v.x) {
                re[a] = re[a - 1];
                --a;
            }
            re[a] = v.x;
            while (b > 0 && im[b - 1] > v.y) {
                im[b] = im[b - 1];
                --b;
            }
            im[b] = v.y;
        }
        return make_float2(median_sorted(re, L), median_sorted(im, L));
    }
}

// The plan's combination of the L per-loop estimates: the coordinate-wise
// median, or the mean (summed in loop order).
template <int LT>
__device__ float2 combined_estimate(const PlanDev &P, const float2 *zhat, uint32_t f) {
    if (P.estimator == kEstMean) {
        const uint32_t L = LT > 0 ? (uint32_t)LT : P.L;
        float sr = 0.f, si = 0.f;
        for (uint32_t l = 0; l < L; ++l) {
            const float2 v = loop_estimate(P, zhat, l, f);
            sr += v.x;
            si += v.y;
        }
        return make_float2(sr / (float)L, si / (float)L);
    }
    return median_estimate<LT>(P, zhat, f);
}

// kept in at least T loops (the candidate test the register-table scan defers)
template <int LT>
__device__ __forceinline__ bool is_candidate(const PlanDev &P, uint32_t f) {
    const uint32_t cv = P.half << (32 - P.logN), top = 32 - P.logB;
    uint32_t score = 0;
    if constexpr (LT > 0) {
#pragma unroll
        for (int l = 0; l < LT; ++l)
            score += __ldg(P.flags + (size_t)l * P.B + (((P.sigma[l] << (32 - P.logN)) * f + cv) >> top)) & 1u;
    } else {
        for (uint32_t l = 0; l < P.L; ++l)
            score += __ldg(P.flags + (size_t)l * P.B + (((P.sigma[l] << (32 - P.logN)) * f + cv) >> top)) & 1u;
    }
    return score >= P.T;
}

// Pruned-pass estimate of survivor f with L = LT, appended to the records at
// *cnt when f is a candidate whose key reaches theta.  One hash word per loop
// feeds the bucket and gain loads, all issued before any is used.  Before the
// candidacy test and the sort, f is dropped when neither median component can reach
// a = sqrt(theta/2) (1 - 2^-10) in magnitude: a median >= a needs at least
// M = ceil(L/2) values >= a, one <= -a as many <= -a, and with both medians
// inside (-a, a) the computed key stays below theta.  Kept records are
// bit-identical to median_estimate's.  Mean plans: every survivor is a
// candidate and is estimated by the mean of its L values (summed in loop
// order, bit-identical to combined_estimate's).
// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory loads by 32-bit shared address (the staged estimate tables).
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Tables: the plan's in global memory (SM false), or copies in shared memory
// (zt: zhat [L][B], gt: 1/G~ [N/B], kt: kept bits [L][B/32]).
template <int LT, bool SM>
__device__ __forceinline__ void estimate_pruned(const PlanDev &P, uint32_t f, float theta, float a,
                                                uint32_t *cnt, const float2 *zt, const float2 *gt,
                                                const uint32_t *kt) {
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB;
    const uint32_t cv = P.half << sN;
    const uint32_t osh = P.logB + sN;  // offset in the bucket: the word's bits below the bucket bits
    const uint32_t B = P.B;
    float2 z[LT], g[LT];
    uint32_t ph[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) {
        const uint32_t t = (P.sigma[l] << sN) * f + cv;
        const uint32_t h = t >> top;
        const uint32_t opos = osh < 32 ? (t << P.logB) >> osh : 0u;
        if constexpr (SM) {
            const uint32_t zb = (uint32_t)__cvta_generic_to_shared(zt);
            const uint32_t gb = (uint32_t)__cvta_generic_to_shared(gt);
            z[l] = lds_f2(zb + 8 * (l * B + h));
            g[l] = lds_f2(gb + 8 * opos);
        } else {
            z[l] = __ldg(P.zhat + l * B + h);
            g[l] = __ldg(P.ginv + opos);
        }
        ph[l] = (P.tau[l] << sN) * f;
    }
    bool keep = true;
    const bool mean = P.estimator == kEstMean;
    float re[LT], im[LT];
    {
        uint32_t rp = 0, rn = 0, ip = 0, in = 0;
#pragma unroll
        for (int l = 0; l < LT; ++l) {
            const float2 v = turn_scale(z[l], g[l], ph[l]);
            re[l] = v.x;
            im[l] = v.y;
            rp += v.x >= a;
            rn += v.x <= -a;
            ip += v.y >= a;
            in += v.y <= -a;
        }
        constexpr uint32_t M = (LT + 1) / 2;
        keep = mean || rp >= M || rn >= M || ip >= M || in >= M;
    }
    if (keep && !mean) {
        // candidacy (kept in >= T loops), only for the few that pass (the
        // mean's survivors are the candidates already)
        uint32_t kept = 0;
#pragma unroll
        for (int l = 0; l < LT; ++l) {
            const uint32_t h = ((P.sigma[l] << sN) * f + cv) >> top;
            if constexpr (SM)
                kept += (lds_u32((uint32_t)__cvta_generic_to_shared(kt) + 4 * ((l * B + h) >> 5)) >> (h & 31u)) & 1u;
            else
                kept += __ldg(P.flags + l * B + h) & 1u;
        }
        keep = kept >= P.T;
    }
    float2 v = make_float2(0.f, 0.f);
    float key = 0.f;
    if (keep) {
        if (mean) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int l = 0; l < LT; ++l) {
                sr += re[l];
                si += im[l];
            }
            v = make_float2(sr / (float)LT, si / (float)LT);
        } else {
            sort_net<LT>(re);
            sort_net<LT>(im);
            v = make_float2(median_sorted(re, LT), median_sorted(im, LT));
        }
        key = v.x * v.x + v.y * v.y;
        keep = key >= theta;
    }
    const uint32_t act = __activemask();
    const uint32_t bal = __ballot_sync(act, keep);
    if (bal) {
        const int leader = __ffs(bal) - 1;
        uint32_t b0 = 0;
        if ((threadIdx.x & 31) == (uint32_t)leader) b0 = atomicAdd(cnt, __popc(bal));
        b0 = __shfl_sync(act, b0, leader);
        if (keep)
            P.surv[b0 + __popc(bal & lanemask_lt())] =
                make_uint4(f, __float_as_uint(key), __float_as_uint(v.x), __float_as_uint(v.y));
    }
}

// Estimate of f (the plan's combination), appended to the job's records {f, key bits, re bits,
// im bits} at *cnt when kept: by the pruned pass when f is a candidate whose
// key reaches theta, by the fallback pass always (f is a listed candidate).
template <int LT>
__device__ __forceinline__ void estimate_record(const PlanDev &P, uint32_t f, bool prune, float theta,
                                                uint32_t *cnt) {
    bool keep = !prune || is_candidate<LT>(P, f);
    float2 v = make_float2(0.f, 0.f);
    float key = 0.f;
    if (keep) {
        v = combined_estimate<LT>(P, P.zhat, f);
        key = v.x * v.x + v.y * v.y;
        keep = !prune || key >= theta;
    }
    const uint32_t act = __activemask();
    const uint32_t bal = __ballot_sync(act, keep);
    if (bal) {
        const int leader = __ffs(bal) - 1;
        uint32_t b0 = 0;
        if ((threadIdx.x & 31) == (uint32_t)leader) b0 = atomicAdd(cnt, __popc(bal));
        b0 = __shfl_sync(act, b0, leader);
        if (keep)
            P.surv[b0 + __popc(bal & lanemask_lt())] =
                make_uint4(f, __float_as_uint(key), __float_as_uint(v.x), __float_as_uint(v.y));
    }
}

// --------------------------------------------------------------- a4 + a5
// Vote scan over the tiles of frequencies of a job.
//
// Pruned pass: only frequencies with at least M strong loops can reach the top
// K (median bound), so they are queued per tile in shared memory and appended
// to the job's survivor list (k_scan_bits below does the same with a register
// table and estimates them itself).  Fallback pass and candidate listing: the
// u16 kept/strong table (shared or global memory); every candidate is
// counted and listed.
//
// The bucket comes from t = (sigma_l << (32 - log2 N)) f + (half << (32 - log2 N))
// mod 2^32, whose top log2 B bits are round-half-up(sigma_l f B / N) mod B.
enum TableKind : int { kTabGlobal = 0, kTabSmem = 1 };

// Full adder over 32 bit-lanes: a + b + c = s + 2 cy.
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &sum, uint32_t &cy) {
    sum = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

// Bit-sliced population count of N words: pl[i] holds bit i of the per-position
// count.  One column of N words of equal weight is reduced to one word by
// full adders (a half adder for an even remainder); the floor(N/2) carries
// form the next column.
template <int N, int P, int AT = 0>
__device__ __forceinline__ void count_planes(const uint32_t (&col)[N], uint32_t (&pl)[P]) {
    constexpr int NC = N / 2;
    uint32_t cy[NC > 0 ? NC : 1];
    uint32_t acc = col[0];
#pragma unroll
    for (int k = 0; k < (N - 1) / 2; ++k) full_add(acc, col[1 + 2 * k], col[2 + 2 * k], acc, cy[k]);
    if constexpr (N > 1 && (N - 1) % 2 == 1) {
        cy[NC - 1] = acc & col[N - 1];
        acc ^= col[N - 1];
    }
    pl[AT] = acc;
    if constexpr (NC > 0) count_planes<NC, P, AT + 1>(cy, pl);
}

// Positions whose count (planes pl, least significant first) is >= M.
template <int M, int P>
__device__ __forceinline__ uint32_t count_at_least(const uint32_t (&pl)[P]) {
    uint32_t ge = 0, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int b = P - 1; b >= 0; --b) {
        if ((M >> b) & 1) {
            eq &= pl[b];
        } else {
            ge |= eq & pl[b];
            eq &= ~pl[b];
        }
    }
    return ge | eq;
}

constexpr int bit_length(int v) { return v > 0 ? 1 + bit_length(v >> 1) : 0; }

// Bits k * 32/G, k < G = 2^lgG (lgG <= 5): the member counters.
__device__ __forceinline__ uint32_t member_mask(uint32_t lgG) {
    uint32_t m = 1u;
    for (uint32_t w = 32u >> lgG; w < 32u; w <<= 1) m |= m << w;
    return m;
}

template <int LT, int TAB>
__global__ void __launch_bounds__(kThreads) k_vote_scan(Launch ln, int mode, int32_t *cand_out, int32_t *ncand_out) {
    extern __shared__ uint16_t tab_s[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_qn, s_base;
    __shared__ uint32_t queue[kVoteTileF];
    enter(ln, P, J, s_local);
    if (threadIdx.x == 0) s_qn = 0;
    __syncthreads();

    const uint32_t L = LT > 0 ? (uint32_t)LT : P.L;
    const uint32_t B = P.B;
    const uint32_t lane = threadIdx.x & 31;
    const uint16_t *tab = P.flags;
    if constexpr (TAB == kTabSmem) {
        const uint32_t nw = (L * B) / 2;  // B is even
        const uint32_t *src = reinterpret_cast<const uint32_t *>(P.flags);
        uint32_t *dst = reinterpret_cast<uint32_t *>(tab_s);
        for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = __ldcg(src + i);
        __syncthreads();
        tab = tab_s;
    }
    constexpr int LR = LT > 0 ? LT : 1;
    uint32_t av[LR];
    if constexpr (LT > 0) {
#pragma unroll
        for (int l = 0; l < LT; ++l) av[l] = P.sigma[l] << (32 - P.logN);
    }
    const uint32_t cv = P.half << (32 - P.logN);
    const uint32_t top = 32 - P.logB;
    const uint32_t M = P.M, T = P.T, N = P.N;
    const bool mean = P.estimator == kEstMean;

    // comb plans (pruned pass) scan only the kept classes: index v -> class
    // cls[v >> lm], f = class + (v & (2^lm - 1)) Bc with 2^lm = N / Bc
    const bool comb = P.method == kMethodComb && mode == kVotePrune;
    const uint32_t lm = comb ? P.logN - P.logBc : 0u;
    const uint32_t vspan = comb ? P.ncls << lm : N;
    uint32_t per = (vspan + P.vtiles - 1) / P.vtiles;
    per = (per + kThreads - 1) / kThreads * kThreads;  // <= kVoteTileF
    const uint32_t stride = mode == kVotePrune ? J.vctas : P.vtiles;

    auto enqueue = [&](uint32_t f, bool take) {
        const uint32_t bs = __ballot_sync(0xFFFFFFFFu, take);
        if (bs) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(&s_qn, __popc(bs));
            b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
            if (take) queue[b0 + __popc(bs & lanemask_lt())] = f;  // < kVoteTileF: one slot per f of the tile
        }
    };

    for (uint32_t tile = s_local; tile < P.vtiles; tile += stride) {
        const uint32_t f0 = tile * per;
        const uint32_t f1 = min(vspan, f0 + per);
        for (uint32_t base = f0; base < f1; base += kThreads) {
            const uint32_t v = base + threadIdx.x;
            const bool valid = v < f1;
            const uint32_t f = comb ? (valid ? __ldg(P.cls + (v >> lm)) + ((v & ((1u << lm) - 1)) << P.logBc) : 0u) : v;
            {
                uint32_t acc = 0;  // score | strong << 8
                if constexpr (LT > 0) {
#pragma unroll
                    for (int l = 0; l < LT; ++l) acc += tab[l * B + ((av[l] * f + cv) >> top)];
                } else {
                    for (uint32_t l = 0; l < L; ++l)
                        acc += tab[l * B + (((P.sigma[l] << (32 - P.logN)) * f + cv) >> top)];
                }
                const bool cand = valid && (acc & 0xFFu) >= T;
                if (mode == kVoteCandidates) {
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, cand);
                    if (bal) {
                        uint32_t b0 = 0;
                        if (lane == 0) b0 = atomicAdd(reinterpret_cast<uint32_t *>(ncand_out), __popc(bal));
                        b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
                        if (cand) cand_out[b0 + __popc(bal & lanemask_lt())] = (int32_t)f;
                    }
                    continue;
                }
                enqueue(f, cand && (mean || (acc >> 8) >= M));  // the mean has no strong-loop bound
            }
        }
        if (mode == kVoteCandidates) continue;
        __syncthreads();
        const uint32_t qn = s_qn;
        if (qn) {
            if (threadIdx.x == 0) s_base = atomicAdd(P.ctr + kNSurv, qn);
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < qn; i += blockDim.x) P.survf[s_base + i] = queue[i];
            __syncthreads();
            if (threadIdx.x == 0) s_qn = 0;
            __syncthreads();
        }
    }
}


// Pruned scan with the register table of strong bits (32 <= B <= 512, L in
// {8, 12, 16}).  Mean plans (T = M) pack kept bits instead, so the survivors
// are exactly the candidates.
//
// A thread takes the G = B/32 frequencies f + kN/G.  Their hash words differ
// by k sigma_l 2^32/G, so their buckets h + k sigma_l 32 share the lane
// h mod 32 of the packed table, and one warp shuffle fetches the word holding
// all G strong bits.  A rotate by sigma^-1 (h >> (log2 B - 5)) (the table's
// positions are scaled by sigma^-1 to match) puts member k's bit at position
// k 32/G in every loop, so carry-save adders over the L rotated words count
// the strong loops of all 32 positions at once (bit-sliced counters).
// Frequencies with at least M = ceil(L/2) strong loops are queued in shared
// memory (overflow goes straight to the job's survivor list) and appended to
// the list when the CTA ends; candidacy is checked when they are estimated.
template <int LT>
__global__ void __launch_bounds__(kThreads) k_scan_bits(Launch ln) {
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_qn, s_base;
    __shared__ uint32_t queue[kVoteTileF];
    enter(ln, P, J, s_local);
    if (threadIdx.x == 0) s_qn = 0;

    const uint32_t lane = threadIdx.x & 31;
    // per loop: sigma << (32 - log2 N), the lane's table word, and sigma^-1
    // mod 32 packed six 5-bit fields to a word (fewer live registers)
    constexpr int NSW = (LT + 5) / 6;
    uint32_t av[LT], pw[LT], sip[NSW];
#pragma unroll
    for (int k = 0; k < NSW; ++k) sip[k] = 0;
#pragma unroll
    for (int l = 0; l < LT; ++l) {
        av[l] = P.sigma[l] << (32 - P.logN);
        pw[l] = __ldcg(P.packed + l * 32 + lane);
        sip[l / 6] |= (inv_mod32(P.sigma[l]) & 31u) << (5 * (l % 6));
    }
    const uint32_t cv = P.half << (32 - P.logN);
    const uint32_t top = 32 - P.logB;
    // G = 2^lgG frequencies f + k span per thread, member k's counter at bit k << gsh
    const uint32_t lgG = P.logB - 5;
    const uint32_t gsh = 5 - lgG;
    const uint32_t span = P.N >> lgG;
    const uint32_t members = member_mask(lgG);
    // comb plans scan only the kept classes: index v -> class cls[v >> lm],
    // f = class + (v & (2^lm - 1)) Bc with 2^lm = span / Bc (members f + k span
    // stay in the class: Bc divides span)
    const bool comb = P.method == kMethodComb;
    const uint32_t lm = comb ? (P.logN - lgG) - P.logBc : 0u;
    const uint32_t vspan = comb ? P.ncls << lm : span;
    uint32_t per = (vspan + P.vtiles - 1) / P.vtiles;
    per = (per + kThreads - 1) / kThreads * kThreads;
    __syncthreads();

    // survivors go to the CTA's queue; once it is full, straight to the job's
    // list (no barrier until the CTA's last tile)
    for (uint32_t tile = s_local; tile < P.vtiles; tile += J.vctas) {
        const uint32_t f0 = tile * per;
        const uint32_t f1 = min(vspan, f0 + per);
        for (uint32_t base = f0; base < f1; base += kThreads) {
            const uint32_t v = base + threadIdx.x;
            const bool valid = v < f1;
            const uint32_t f = comb ? (valid ? __ldg(P.cls + (v >> lm)) + ((v & ((1u << lm) - 1)) << P.logBc) : 0u) : v;
            uint32_t x[LT];
#pragma unroll
            for (int l = 0; l < LT; ++l) {
                const uint32_t t = av[l] * f + cv;
                const uint32_t w = __shfl_sync(0xFFFFFFFFu, pw[l], t >> top);  // lane = bucket mod 32
                const uint32_t si = (sip[l / 6] >> (5 * (l % 6))) & 31u;
                x[l] = __funnelshift_r(w, w, (t >> 27) * si);
            }
            constexpr int NP = bit_length(LT);
            uint32_t pl[NP];
            count_planes<LT, NP>(x, pl);
            uint32_t m = valid ? count_at_least<(LT + 1) / 2, NP>(pl) & members : 0u;
            if (m) {
                const uint32_t n = __popc(m);
                uint32_t q = atomicAdd(&s_qn, n);
                uint32_t g = q + n > (uint32_t)kVoteTileF ? atomicAdd(P.ctr + kNSurv, q + n - max(q, (uint32_t)kVoteTileF))
                                                          : 0u;
                do {
                    const uint32_t b = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t fs = f + (b >> gsh) * span;
                    if (q < (uint32_t)kVoteTileF)
                        queue[q++] = fs;
                    else
                        P.survf[g++] = fs;
                } while (m);
            }
        }
    }
    __syncthreads();
    const uint32_t qn = min(s_qn, (uint32_t)kVoteTileF);
    if (qn) {
        if (threadIdx.x == 0) s_base = atomicAdd(P.ctr + kNSurv, qn);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < qn; i += blockDim.x) P.survf[s_base + i] = queue[i];
    }
}

// ------------------------------------------------------------------ a6

// ------------------------------------------------------------------ a7
__device__ __forceinline__ unsigned long long surv_key(uint4 r) {
    return ((unsigned long long)r.y << 32) | (uint32_t)(~r.x);  // key desc, then f asc
}

// Records up to this many are ranked by counting comparisons.
constexpr uint32_t kRankMax = 1024;

// Fallback pass of one job inside its top-K CTA, taken when fewer than K
// pruned records reached theta: every candidate (kept in >= T loops) is
// counted, estimated and recorded (kNCand, kNRec2).  A single CTA scans all N
// frequencies, so such a job is slow, but the pass is exact and the common
// case launches nothing for it.
__device__ void fallback_pass(const PlanDev &P, uint32_t *s_cnt) {
    if (threadIdx.x == 0) *s_cnt = 0;
    __syncthreads();
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB, cv = P.half << sN;
    uint32_t cand = 0;
    for (uint32_t base = 0; base < P.N; base += blockDim.x) {
        const uint32_t f = base + threadIdx.x;
        bool c = false;
        // comb plans: only frequencies of kept residue classes
        const bool eligible = P.method != kMethodComb ||
                              ((__ldg(P.keptc + ((f & (P.Bc - 1)) >> 5)) >> (f & (P.Bc - 1) & 31u)) & 1u);
        if (f < P.N && eligible) {
            uint32_t score = 0;
            for (uint32_t l = 0; l < P.L; ++l)
                score += __ldg(P.flags + (size_t)l * P.B + (((P.sigma[l] << sN) * f + cv) >> top)) & 1u;
            c = score >= P.T;
        }
        cand += c;
        if (c) estimate_record<0>(P, f, false, 0.f, P.ctr + kNRec2);
    }
    cand = __reduce_add_sync(0xFFFFFFFFu, cand);
    if ((threadIdx.x & 31) == 0 && cand) atomicAdd(s_cnt, cand);
    __syncthreads();
    if (threadIdx.x == 0) P.ctr[kNCand] = *s_cnt;
    __syncthreads();
}

// Top-K of one job: the k_out = min(K, candidates) recorded estimates of
// largest magnitude (ties to the lower f), written sorted by f.  Records are
// those of the pruned pass (candidates with key >= theta) when at least K of
// them exist; otherwise those of the fallback pass (every candidate).  Pruned
// candidates have key < theta, so either set contains the top K.
// Run by all threads of the job's last estimate CTA (the other CTAs' records
// are visible: they fenced before taking their ticket).  tk: shared memory for
// cap keys + cap payloads (cap a power of two >= max(kRankMax, K)).
__device__ void rank_records(const PlanDev &P, const Job &J, unsigned long long *tk, uint32_t cap, uint32_t S,
                             uint32_t kout);

__device__ void topk_job(const PlanDev &P, const Job &J, unsigned long long *tk, uint32_t cap) {
    __shared__ uint32_t s_S, s_kout, s_cnt;
    __shared__ int s_fb;
    if (threadIdx.x == 0) s_fb = needs_fallback(P);
    __syncthreads();
    if (s_fb) fallback_pass(P, &s_cnt);
    if (threadIdx.x == 0) {
        s_S = __ldcg(P.ctr + (s_fb ? kNRec2 : kNGe));
        s_kout = s_fb ? min(P.K, __ldcg(P.ctr + kNCand)) : P.K;  // without fallback >= K candidates exist
    }
    __syncthreads();
    rank_records(P, J, tk, cap, s_S, s_kout);
}

// The kout (<= S) records {f, key bits, re bits, im bits} of largest key (ties
// to the lower f) among the S in P.surv, written to the job's outputs sorted
// by f (all threads of one CTA).
__device__ void rank_records(const PlanDev &P, const Job &J, unsigned long long *tk, uint32_t cap, uint32_t S,
                             uint32_t kout) {
    uint32_t *pay = reinterpret_cast<uint32_t *>(tk + cap);
    __shared__ uint32_t s_hist[256], s_need, s_cnt;
    __shared__ unsigned long long s_prefix, s_pmask;
    const uint4 *surv = P.surv;
    if (S <= kRankMax) {
        // ranks by counting: record i wins when fewer than kout keys exceed
        // its key (keys are distinct: f breaks ties); winners are then placed
        // by the number of winning frequencies below theirs
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) tk[i] = surv_key(__ldcg(surv + i));
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
            const unsigned long long k = tk[i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < S; ++j) r += tk[j] > k;
            pay[i] = r < kout ? ~(uint32_t)k : 0xFFFFFFFFu;  // the winner's f, else above every f
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
            const uint32_t f = pay[i];
            if (f == 0xFFFFFFFFu) continue;
            uint32_t pos = 0;
            for (uint32_t j = 0; j < S; ++j) pos += pay[j] < f;
            const uint4 r = __ldcg(surv + i);
            J.idx[pos] = (int32_t)f;
            J.val[pos] = make_float2(__uint_as_float(r.z), __uint_as_float(r.w));
        }
        if (threadIdx.x == 0) *J.kout = (int32_t)kout;
        return;
    }
    if (S <= cap) {
        uint32_t n2 = 1;
        while (n2 < S) n2 <<= 1;
        for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
            if (i < S) {
                tk[i] = surv_key(__ldcg(surv + i));
                pay[i] = i;
            } else {
                tk[i] = 0ull;  // ranks below every real entry (~f > 0)
                pay[i] = 0xFFFFFFFFu;
            }
        }
        __syncthreads();
        bitonic_pairs(tk, pay, n2, false);
    } else {
        // rare path (the unpruned fallback over many candidates): exact radix
        // select of the kout-th largest key, 8 bits per pass
        if (threadIdx.x == 0) {
            s_prefix = 0ull;
            s_pmask = 0ull;
            s_need = kout;
        }
        for (int pass = 0; pass < 8; ++pass) {
            const int sh = 56 - 8 * pass;
            for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_hist[i] = 0;
            __syncthreads();
            const unsigned long long pre = s_prefix, pm = s_pmask;
            for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
                const unsigned long long k = surv_key(__ldcg(surv + i));
                if ((k & pm) == pre) atomicAdd(&s_hist[(k >> sh) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0 && s_need > 0) {
                uint32_t need = s_need, cum = 0;
                int d = 255;
                for (; d > 0; --d) {
                    if (cum + s_hist[d] >= need) break;
                    cum += s_hist[d];
                }
                s_need = need - cum;
                s_prefix = pre | ((unsigned long long)d << sh);
                s_pmask = pm | (255ull << sh);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const unsigned long long kth = s_prefix;
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
            const unsigned long long k = surv_key(__ldcg(surv + i));
            if (kout > 0 && k >= kth) {
                const uint32_t pos = atomicAdd(&s_cnt, 1u);
                if (pos < cap) {
                    tk[pos] = k;
                    pay[pos] = i;
                }
            }
        }
        __syncthreads();
    }
    // winners are tk[0..kout): re-key by frequency and sort ascending
    uint32_t n2k = 1;
    while (n2k < kout) n2k <<= 1;
    for (uint32_t i = threadIdx.x; i < n2k; i += blockDim.x) {
        if (i < kout) tk[i] = (unsigned long long)(~(uint32_t)tk[i]);
        else tk[i] = ~0ull;
    }
    __syncthreads();
    if (kout > 1) bitonic_pairs(tk, pay, n2k, true);
    for (uint32_t s = threadIdx.x; s < kout; s += blockDim.x) {
        const uint4 r = __ldcg(surv + pay[s]);
        J.idx[s] = (int32_t)r.x;
        J.val[s] = make_float2(__uint_as_float(r.z), __uint_as_float(r.w));
    }
    if (threadIdx.x == 0) *J.kout = (int32_t)kout;
}

// True in every thread of the job's last CTA of this launch to finish (each
// CTA fences its records first); that CTA also re-arms the ticket.
__device__ bool last_of_job(const PlanDev &P, uint32_t ctas_per_job) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last = atomicAdd(P.ctr + kEstDone, 1u) == ctas_per_job - 1;
        if (s_last) atomicExch(P.ctr + kEstDone, 0u);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Pruned-pass median estimates of the job's survivors, ctas_per_job CTAs per
// job: candidates whose key reaches theta are recorded as {f, key bits, re
// bits, im bits}.  The job's last CTA to finish (atomic ticket after a fence)
// then takes the job's top K (a7).
template <int LT>
__global__ void __launch_bounds__(kThreads) k_estimate_surv(Launch ln, uint32_t ctas_per_job, uint32_t cap) {
    extern __shared__ unsigned long long est_topk[];  // top-K buffer of the job's last CTA
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    enter(ln, P, J, s_local);
    const uint32_t n = P.ctr[kNSurv];
    const float theta = __uint_as_float(P.ctr[kTheta]);
    uint32_t *cnt = P.ctr + kNGe;
    const uint32_t stride = ctas_per_job * kThreads;
    if constexpr (LT > 0) {
        const float a = sqrtf(0.5f * theta) * (1.0f - 1.0f / 1024.0f);
        // the next survivor's frequency is fetched while this one is estimated
        uint32_t i = s_local * kThreads + threadIdx.x;
        uint32_t fn = i < n ? __ldg(P.survf + i) : 0u;
        for (; i < n; i += stride) {
            const uint32_t f = fn;
            if (i + stride < n) fn = __ldg(P.survf + i + stride);
            estimate_pruned<LT, false>(P, f, theta, a, cnt, nullptr, nullptr, nullptr);
        }
    } else {
        for (uint32_t i = s_local * kThreads + threadIdx.x; i < n; i += stride)
            estimate_record<LT>(P, P.survf[i], true, theta, cnt);
    }
    if (last_of_job(P, ctas_per_job)) topk_job(P, J, est_topk, cap);
}

template <int LT>
__device__ void estimate_tab_part(const PlanDev &P, uint32_t s_local, uint32_t ctas_per_job, uint32_t n,
                                  float4 *est_tab) {
    const uint32_t LB = LT * P.B, NB = P.N >> P.logB;
    float2 *zs = reinterpret_cast<float2 *>(est_tab);
    float2 *gs = zs + LB;
    uint32_t *ks = reinterpret_cast<uint32_t *>(gs + NB);
    {
        // zhat and 1/G~ by asynchronous 16-byte copies (all in flight at once;
        // both tables start 256-byte aligned, LB is even)
        const uint32_t zb = (uint32_t)__cvta_generic_to_shared(zs);
        const uint32_t gb = (uint32_t)__cvta_generic_to_shared(gs);
        for (uint32_t i = threadIdx.x; i < LB / 2; i += kThreads) cp_async16(zb + 16 * i, P.zhat + 2 * i);
        for (uint32_t i = threadIdx.x; i < NB / 2; i += kThreads) cp_async16(gb + 16 * i, P.ginv + 2 * i);
        if ((NB & 1u) && threadIdx.x == 0) gs[NB - 1] = __ldg(P.ginv + NB - 1);
        // kept bits: word w from flags [32 w, 32 w + 32) (64 bytes, four 16-byte loads)
        for (uint32_t w = threadIdx.x; w < LB / 32; w += kThreads) {
            const uint4 *src = reinterpret_cast<const uint4 *>(P.flags + 32 * w);
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = __ldcg(src + k);
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t c[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int b = 8 * k + 2 * j;
                    word |= (c[j] & 1u) << b;
                    word |= ((c[j] >> 16) & 1u) << (b + 1);
                }
            }
            ks[w] = word;
        }
        cp_async_wait_all();
    }
    __syncthreads();
    const float theta = __uint_as_float(P.ctr[kTheta]);
    const float a = sqrtf(0.5f * theta) * (1.0f - 1.0f / 1024.0f);
    // the next survivor's frequency is fetched while this one is estimated
    const uint32_t stride = ctas_per_job * kThreads;
    uint32_t i = s_local * kThreads + threadIdx.x;
    uint32_t fn = i < n ? __ldg(P.survf + i) : 0u;
    for (; i < n; i += stride) {
        const uint32_t f = fn;
        if (i + stride < n) fn = __ldg(P.survf + i + stride);
        estimate_pruned<LT, true>(P, f, theta, a, P.ctr + kNGe, zs, gs, ks);
    }
}

// Pruned-pass estimates with the job's tables staged in shared memory: zhat
// (L B complex), 1/G~ (N/B complex) and the kept flags as bits.  A few CTAs
// per job, each over a strided share of the survivors, so every lookup is a
// shared-memory load.
template <int LT>
__global__ void __launch_bounds__(kThreads) k_estimate_tab(Launch ln, uint32_t ctas_per_job, uint32_t cap) {
    extern __shared__ float4 est_tab[];  // the job's tables, then the last CTA's top-K buffer
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    enter(ln, P, J, s_local);
    const uint32_t n = P.ctr[kNSurv];
    if (s_local * kThreads < n) estimate_tab_part<LT>(P, s_local, ctas_per_job, n, est_tab);
    if (last_of_job(P, ctas_per_job)) topk_job(P, J, reinterpret_cast<unsigned long long *>(est_tab), cap);
}


// ------------------------------------------------- spike-train pre-filter
// Radix-4 pass over a bit-reversed buffer: the DIT stages hs and hs + 1 of the
// group at i0 (distance h = 2^hs).  Same twiddles as two radix-2 stages; the
// second stage's odd pair takes W_{4h}^{k+h} = -i W_{4h}^k.
__device__ __forceinline__ void r4_pass(float2 *b, uint32_t i0, uint32_t h, float2 w1, float2 w2) {
    const float2 x0 = b[i0], x1 = b[i0 + h], x2 = b[i0 + 2 * h], x3 = b[i0 + 3 * h];
    const float2 t1 = cmul(w1, x1), t3 = cmul(w1, x3);
    const float2 a0 = make_float2(x0.x + t1.x, x0.y + t1.y), a1 = make_float2(x0.x - t1.x, x0.y - t1.y);
    const float2 a2 = make_float2(x2.x + t3.x, x2.y + t3.y), a3 = make_float2(x2.x - t3.x, x2.y - t3.y);
    const float2 u2 = cmul(w2, a2), v3 = cmul(w2, a3), u3 = make_float2(v3.y, -v3.x);
    b[i0] = make_float2(a0.x + u2.x, a0.y + u2.y);
    b[i0 + 2 * h] = make_float2(a0.x - u2.x, a0.y - u2.y);
    b[i0 + h] = make_float2(a1.x + u3.x, a1.y + u3.y);
    b[i0 + 3 * h] = make_float2(a1.x - u3.x, a1.y - u3.y);
}

// Per-pass twiddles of fft2_smem_r4, contiguous in k so that a warp's
// lookups hit distinct banks: the radix-4 pass at hs (distance h = 2^hs)
// takes W_{2h}^k from tws[o + k] and W_{4h}^k from tws[o + h + k], k < h,
// where o sums 2h over the earlier passes (at most 2B/3 entries in all).
// tw: exp(-2 pi i k / B), k < B/2.  All threads; ends with a barrier.
__device__ void r4_twiddles(float2 *tws, uint32_t logB, const float2 *tw) {
    uint32_t o = 0;
    for (uint32_t hs = logB & 1; hs + 1 < logB; hs += 2) {
        const uint32_t h = 1u << hs;
        for (uint32_t k = threadIdx.x; k < h; k += blockDim.x) {
            tws[o + k] = __ldg(tw + (k << (logB - 1 - hs)));
            tws[o + h + k] = __ldg(tw + (k << (logB - 2 - hs)));
        }
        o += 2 * h;
    }
    __syncthreads();
}

// Two B-point FFTs of bit-reversed buffers in shared memory (per-pass
// twiddles from r4_twiddles), two stages per barrier.  All threads; ends with
// a barrier.
__device__ void fft2_smem_r4(float2 *b0, float2 *b1, uint32_t B, uint32_t logB, const float2 *tws) {
    uint32_t hs = 0;
    if (logB & 1) {  // odd log2 B: one radix-2 stage (h = 1, twiddle 1) first
        for (uint32_t q = threadIdx.x; q < B / 2; q += blockDim.x) {
            float2 *b = b0;
#pragma unroll
            for (int t = 0; t < 2; ++t, b = b1) {
                const float2 a = b[2 * q], c = b[2 * q + 1];
                b[2 * q] = make_float2(a.x + c.x, a.y + c.y);
                b[2 * q + 1] = make_float2(a.x - c.x, a.y - c.y);
            }
        }
        __syncthreads();
        hs = 1;
    }
    for (uint32_t o = 0; hs + 1 < logB; hs += 2) {
        const uint32_t h = 1u << hs;
        for (uint32_t q = threadIdx.x; q < B / 4; q += blockDim.x) {
            const uint32_t k = q & (h - 1);
            const uint32_t i0 = ((q >> hs) << (hs + 2)) + k;
            const float2 w1 = tws[o + k], w2 = tws[o + h + k];
            r4_pass(b0, i0, h, w1, w2);
            r4_pass(b1, i0, h, w1, w2);
        }
        o += 2 * h;
        __syncthreads();
    }
}

// One CTA per job (sFFT2.0-style; Eq. 10, 15-16): kCombShifts = 2
// subsamplings at stride N/Bc (shifts tau of loops L, L+1), each a Bc-point
// FFT scaled by 1/Bc, so class i holds the sum over f = i (mod Bc) of
// x^_f e^{+2 pi i tau f/N}; the energies summed over the shifts keep the ncls
// largest classes (ties to the lower class), listed ascending in P.cls and
// marked in P.keptc.  Shared memory: both spectra, then Bc entries for the
// per-pass twiddles (whose room takes the energies once the FFTs are done).
// kCombThreads threads: the job's whole work is one CTA, latency-bound, so
// it runs with many warps.
__global__ void __launch_bounds__(kCombThreads) k_comb(Launch ln) {
    constexpr uint32_t NT = kCombThreads, NW = NT / 32;
    extern __shared__ float2 cb[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_hist[256], s_wsum[NW], s_prefix, s_need;
    enter(ln, P, J, s_local);
    const uint32_t Bc = P.Bc, logBc = P.logBc, stride = P.N >> logBc, mask = P.mask;
    const uint32_t tau0 = P.tau[P.L], tau1 = P.tau[P.L + 1];
    float2 *b0 = cb, *b1 = cb + Bc, *tws = cb + 2 * Bc;
    // both subsamplings, kU samples of each in flight per thread; consecutive
    // threads read consecutive samples j (addresses N/Bc apart, spread over
    // the memory channels) and store them at the bit-reversed positions
    constexpr int kU = 4;
    for (uint32_t j0 = threadIdx.x; j0 < Bc; j0 += kU * NT) {
        float2 v0[kU], v1[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t j = j0 + u * NT;
            if (j < Bc) {
                v0[u] = __ldg(J.x + ((tau0 + j * stride) & mask));
                v1[u] = __ldg(J.x + ((tau1 + j * stride) & mask));
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t j = j0 + u * NT;
            if (j < Bc) {
                const uint32_t r = __brev(j) >> (32 - logBc);
                b0[r] = v0[u];
                b1[r] = v1[u];
            }
        }
    }
    r4_twiddles(tws, logBc, P.ctw);  // (its barrier also covers the stores above)
    fft2_smem_r4(b0, b1, Bc, logBc, tws);
    const float scale = 1.0f / (float)Bc;
    float *en = reinterpret_cast<float *>(tws);  // Bc floats: the twiddles' room
    for (uint32_t i = threadIdx.x; i < Bc; i += NT) {
        const float2 y0 = make_float2(b0[i].x * scale, b0[i].y * scale);
        const float2 y1 = make_float2(b1[i].x * scale, b1[i].y * scale);
        en[i] = (y0.x * y0.x + y0.y * y0.y) + (y1.x * y1.x + y1.y * y1.y);
    }
    __syncthreads();
    // kept = energy above the ncls-th largest, plus the lowest-index ties
    const uint32_t *keys = reinterpret_cast<const uint32_t *>(en);  // non-negative floats: monotone bits
    const uint32_t kth = block_kth_largest<NT, false>(keys, Bc, P.ncls, s_hist, s_wsum, &s_prefix, &s_need);
    const uint32_t need_eq = s_need;
    // each warp takes a contiguous range of bitmap words; ballots give the
    // words, the ties' ranks and the list positions in class order
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t words = (Bc + 31) / 32, wpw = (words + NW - 1) / NW;
    const uint32_t w0 = min(words, wid * wpw), w1 = min(words, w0 + wpw);
    uint32_t neq = 0;
    for (uint32_t wd = w0; wd < w1; ++wd) {
        const uint32_t k = wd * 32 + lane;
        neq += __popc(__ballot_sync(0xFFFFFFFFu, k < Bc && keys[k] == kth));
    }
    uint32_t rank = block_incl_scan_n<NW>(lane == 0 ? neq : 0u, s_wsum);  // ties in earlier warps, inclusive
    rank = __shfl_sync(0xFFFFFFFFu, rank, 0) - neq;
    uint32_t *bm = reinterpret_cast<uint32_t *>(b0);  // the kept-class bitmap
    uint32_t nk = 0;
    for (uint32_t wd = w0; wd < w1; ++wd) {
        const uint32_t k = wd * 32 + lane;
        const uint32_t e = k < Bc ? keys[k] : 0u;
        const bool tie = k < Bc && e == kth;
        const uint32_t tm = __ballot_sync(0xFFFFFFFFu, tie);
        const bool keep = (k < Bc && e > kth) || (tie && rank + __popc(tm & lt) < need_eq);
        const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) {
            bm[wd] = km;
            P.keptc[wd] = km;
        }
        rank += __popc(tm);
        nk += __popc(km);
    }
    uint32_t pos = block_incl_scan_n<NW>(lane == 0 ? nk : 0u, s_wsum);  // kept classes before this warp
    pos = __shfl_sync(0xFFFFFFFFu, pos, 0) - nk;
    for (uint32_t wd = w0; wd < w1; ++wd) {
        const uint32_t km = bm[wd];  // written by this warp's lane 0 (block_incl_scan's barriers order it)
        if ((km >> lane) & 1u) P.cls[pos + __popc(km & lt)] = wd * 32 + lane;
        pos += __popc(km);
    }
}

// ------------------------------------------------------ phase encoding
// sFFT3.0-style variant: iteration r bucketizes the signal under loop
// parameters r at shifts tau_r and tau_r + 1 ("Phase encoding method"),
// subtracts the coefficients found so far ("The iterative framework"), and
// reads every bucket above the threshold as a lone coefficient.  The found
// coefficients are kept as records {f, 0, re bits, im bits} in P.surv
// (count in kNGe); values of a frequency found again accumulate.

// Radix-2 FFT of two B-point bit-reversed buffers in shared memory, the same
// stages as k_fft_select (all threads; ends with a barrier).
__device__ void fft2_smem(float2 *b0, float2 *b1, uint32_t B, uint32_t logB, const float2 *tw) {
    for (uint32_t hs = 0; hs < logB; ++hs) {
        const uint32_t h = 1u << hs;
        for (uint32_t bf = threadIdx.x; bf < B / 2; bf += blockDim.x) {
            const uint32_t k = bf & (h - 1);
            const uint32_t i0 = ((bf >> hs) << (hs + 1)) + k, i1 = i0 + h;
            const float2 w = tw[k << (logB - 1 - hs)];
            const float2 a = b0[i0], t = cmul(w, b0[i1]);
            b0[i0] = make_float2(a.x + t.x, a.y + t.y);
            b0[i1] = make_float2(a.x - t.x, a.y - t.y);
            const float2 c = b1[i0], u = cmul(w, b1[i1]);
            b1[i0] = make_float2(c.x + u.x, c.y + u.y);
            b1[i1] = make_float2(c.x - u.x, c.y - u.y);
        }
        __syncthreads();
    }
}

// exp(+2 pi i ph / 2^32) for a 32-bit turn ph
__device__ __forceinline__ float2 turn_pos(uint32_t ph) {
    float sn, cs;
    __sincosf((float)(int32_t)ph * (2.0f * CUDART_PI_F / 4294967296.0f), &sn, &cs);
    return make_float2(cs, sn);
}

// One job per CTA, all iterations: bucket values of both shifts (gathered and
// folded straight into shared memory), subtraction of the found coefficients
// from their own and both neighbouring buckets (G~ of the plan's three-bucket
// table; the flat window's gain further out is below its stop-band floor),
// threshold (1e-6 of iteration 0's largest bucket energy), location and
// estimate of lone coefficients; stops after the first iteration with no
// bucket above the threshold, then writes the K largest found coefficients.
__global__ void __launch_bounds__(kThreads) k_pe_job(Launch ln, uint32_t cap, uint32_t fcap) {
    // bucket values of both shifts [B] [B], twiddles [B/2]; then the found
    // list when it fits fcap entries (else it stays in P.surv), or the top-K
    // buffer at the end
    extern __shared__ float2 pe_s[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_active, s_n;
    __shared__ float s_thr, s_wmax[kThreads / 32];
    __shared__ float2 red0[kThreads], red1[kThreads];
    enter(ln, P, J, s_local);
    const uint32_t B = P.B, logB = P.logB, N = P.N, NB = N >> logB;
    float2 *b0 = pe_s, *b1 = pe_s + B, *tw = pe_s + 2 * B;
    for (uint32_t k = threadIdx.x; k < B / 2; k += blockDim.x) tw[k] = __ldg(P.tw + k);
    if (threadIdx.x == 0) s_n = 0;
    const uint32_t TB = P.tb, PP = kThreads / TB;
    const uint32_t jt = threadIdx.x & (TB - 1), sidx = threadIdx.x / TB;
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB, cv = P.half << sN;
    const float2 *__restrict__ x = J.x;
    uint4 *F = P.cap <= fcap ? reinterpret_cast<uint4 *>(pe_s + 2 * B + B / 2 + (B & 1)) : P.surv;
    uint32_t iters = 0;
    for (uint32_t r = 0; r < P.L; ++r) {
        const uint32_t sig = P.sigma[r], tau = P.tau[r];
        // a1 for both shifts, bucket tile by bucket tile
        for (uint32_t tile = 0; tile < P.tiles; ++tile) {
            const uint32_t j = tile * TB + jt, jq = (j + P.halfw) & (B - 1);
            float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll 8
            for (uint32_t rr = sidx; rr < P.rounds; rr += PP) {
                const uint32_t q = rr * B + jq;
                const uint32_t i = (sig * (q - P.halfw) + tau) & P.mask;
                const float g = __ldg(P.taps + q);
                const float2 v0 = __ldg(x + i), v1 = __ldg(x + ((i + 1) & P.mask));
                a0r = fmaf(g, v0.x, a0r);
                a0i = fmaf(g, v0.y, a0i);
                a1r = fmaf(g, v1.x, a1r);
                a1i = fmaf(g, v1.y, a1i);
            }
            red0[threadIdx.x] = make_float2(a0r, a0i);
            red1[threadIdx.x] = make_float2(a1r, a1i);
            __syncthreads();
            if (sidx == 0) {
                float2 c0 = red0[jt], c1 = red1[jt];
                for (uint32_t k = 1; k < PP; ++k) {
                    c0.x += red0[jt + k * TB].x;
                    c0.y += red0[jt + k * TB].y;
                    c1.x += red1[jt + k * TB].x;
                    c1.y += red1[jt + k * TB].y;
                }
                const uint32_t br = __brev(j) >> (32 - logB);
                b0[br] = c0;
                b1[br] = c1;
            }
            __syncthreads();
        }
        fft2_smem(b0, b1, B, logB, tw);
        const uint32_t nprev = s_n;
        // subtraction, bucket by bucket over the found list (a fixed order)
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            float2 z0 = b0[k], z1 = b1[k];
            for (uint32_t e = 0; e < nprev; ++e) {
                const uint4 rec = F[e];
                const uint32_t f = rec.x;
                const uint32_t h = ((sig << sN) * f + cv) >> top;
                const uint32_t d = (k - h) & (B - 1);
                if (d != 0 && d != 1 && d != B - 1) continue;
                // nu = (sigma f mod N) - k N/B, wrapped into [-N/2, N/2)
                const int32_t nu = (int32_t)((((sig * f) & P.mask) - k * NB + N / 2) & P.mask) - (int32_t)(N / 2);
                const float2 G = __ldg(P.gext + (nu + (int32_t)(3 * NB / 2)));
                const float2 c0 = cmul(cmul(make_float2(__uint_as_float(rec.z), __uint_as_float(rec.w)),
                                            turn_pos((tau << sN) * f)),
                                       G);
                const float2 c1 = cmul(c0, turn_pos((1u << sN) * f));
                z0.x -= c0.x;
                z0.y -= c0.y;
                z1.x -= c1.x;
                z1.y -= c1.y;
            }
            b0[k] = z0;
            b1[k] = z1;
        }
        if (threadIdx.x == 0) s_active = 0;
        __syncthreads();
        if (r == 0) {
            float m = 0.f;
            for (uint32_t k = threadIdx.x; k < B; k += blockDim.x)
                m = fmaxf(m, b0[k].x * b0[k].x + b0[k].y * b0[k].y);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if ((threadIdx.x & 31) == 0) s_wmax[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                float mm = 0.f;
                for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2) mm = fmaxf(mm, s_wmax[w2]);
                s_thr = 1e-6f * mm;
            }
            __syncthreads();
        }
        const float thr = s_thr;
        uint32_t active = 0;
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z0 = b0[k], z1 = b1[k];
            const float e = z0.x * z0.x + z0.y * z0.y;
            if (!(e >= thr) || e == 0.f) continue;
            ++active;
            // a lone coefficient at f turns by exp(+2 pi i f / N) per unit shift
            const float2 rt = make_float2(z1.x * z0.x + z1.y * z0.y, z1.y * z0.x - z1.x * z0.y);
            const double phi = atan2((double)rt.y, (double)rt.x);
            const long long fl = llrint(phi * (double)N / (2.0 * CUDART_PI));
            const uint32_t f = (uint32_t)fl & P.mask;
            const uint32_t t = (sig << sN) * f + cv;
            if ((t >> top) != k) continue;  // not a lone coefficient of this bucket
            const uint32_t opos = P.logB < P.logN ? (t << P.logB) >> (P.logB + sN) : 0u;
            const float2 v = turn_scale(z0, __ldg(P.ginv + opos), (tau << sN) * f);
            bool merged = false;
            for (uint32_t e2 = 0; e2 < nprev; ++e2) {
                const uint4 rec = F[e2];
                if (rec.x == f) {  // f has one home bucket: one writer per iteration
                    F[e2] = make_uint4(f, 0u, __float_as_uint(__uint_as_float(rec.z) + v.x),
                                            __float_as_uint(__uint_as_float(rec.w) + v.y));
                    merged = true;
                    break;
                }
            }
            if (!merged) {
                const uint32_t pos = atomicAdd(&s_n, 1u);  // < cap: at most B per iteration
                F[pos] = make_uint4(f, 0u, __float_as_uint(v.x), __float_as_uint(v.y));
            }
        }
        active = __reduce_add_sync(0xFFFFFFFFu, active);
        if ((threadIdx.x & 31) == 0 && active) atomicAdd(&s_active, active);
        __threadfence_block();
        __syncthreads();
        iters = r + 1;
        if (s_active == 0) break;  // uniform
    }
    const uint32_t S = s_n;
    if (threadIdx.x == 0) {
        P.ctr[kNGe] = S;
        P.ctr[kPeIter] = iters;
        P.ctr[kTheta] = __float_as_uint(s_thr);
    }
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
        uint4 rec = F[i];
        const float re = __uint_as_float(rec.z), im = __uint_as_float(rec.w);
        rec.y = __float_as_uint(re * re + im * im);
        P.surv[i] = rec;
    }
    __threadfence_block();
    __syncthreads();
    unsigned long long *tk = reinterpret_cast<unsigned long long *>(pe_s + 2 * B + B / 2 + (B & 1));
    rank_records(P, J, tk, cap, S, min(S, P.K));
}

// ------------------------------------- location by binary / multi-scale search
// sFFT4.0 / MPFFT-style variant ("The method of binary search or multi-scale
// search"): the iterative framework of k_pe_job, but iteration r bucketizes
// the signal at the S shifts tau_r + s_j (s_0 = 0, s_{j+1} = N / 2^m_j) and
// reads each bucket above the threshold digit by digit: a coefficient f
// turns by exp(2 pi i f / 2^m) at shift N / 2^m, so with the lower digits r
// known, digit j (b bits) is the d whose predicted turn of f = r + d 2^(jb)
// best matches z_{j+1} conj(z_0) (threshold: the larger of 1e-6 of the
// largest and kSearchKappa times the median bucket energy of iteration 0).
// The bits = min(log2(N/B) + 1, log2 N)
// decoded bits fix p = sigma f modulo 2^bits, one value in the window of two
// bucket widths centred on the bucket; f is kept when it hashes back there
// and every shifted bucket is z_0 turned by exp(2 pi i s_j f / N) up to a
// residual of rho (S - 1) |z_0|^2 (a lone coefficient).

// sigma^-1 mod 2^32 for odd sigma (so also mod N): sigma^2 = 1 (mod 8) holds
// 3 bits, each Newton step doubles them
__device__ __forceinline__ uint32_t inv_mod_2p32(uint32_t sigma) {
    uint32_t x = sigma;
#pragma unroll
    for (int i = 0; i < 4; ++i) x *= 2u - sigma * x;
    return x;
}

// k_bs_job's block: with B >= 256 (one bucket tile of 256 columns) 1024
// threads, four partitions of the gather rounds per column and many warps
// for the latency-bound sample loads; smaller B keep 256 threads (several
// partitions already, more resident CTAs).
constexpr uint32_t kBsWideB = 256;

__device__ __forceinline__ uint32_t bs_bits(const PlanDev &P) {
    return min(P.logN - P.logB + 1u, P.logN);
}

// shift of search step j (0 for the base bucketization j = 0)
__device__ __forceinline__ uint32_t bs_shift(const PlanDev &P, uint32_t j) {
    if (j == 0) return 0u;
    return P.N >> min(j * P.srch_b, bs_bits(P));
}

template <int kBsThreads>
__global__ void __launch_bounds__(kBsThreads) k_bs_job(Launch ln, uint32_t cap, uint32_t fcap, uint32_t nbuf) {
    // nbuf bucket buffers [B] (S rounded up to even), twiddles [B/2]; then
    // the found list when it fits fcap entries (else it stays in P.surv), or
    // the top-K buffer at the end
    extern __shared__ float2 bs_s[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_active, s_n;
    __shared__ float s_thr, s_wmax[kBsThreads / 32];
    __shared__ float2 red0[kBsThreads], red1[kBsThreads];
    __shared__ uint32_t s_hist[256], s_wsum[kBsThreads / 32], s_prefix, s_need;
    enter(ln, P, J, s_local);
    const uint32_t B = P.B, logB = P.logB, N = P.N, NB = N >> logB;
    const uint32_t bits = bs_bits(P), W = 1u << bits, b = P.srch_b;
    const uint32_t S = 1 + (bits + b - 1) / b;  // bucketizations per iteration (<= nbuf)
    float2 *tw = bs_s + (size_t)nbuf * B;
    for (uint32_t k = threadIdx.x; k < B / 2; k += blockDim.x) tw[k] = __ldg(P.tw + k);
    if (threadIdx.x == 0) s_n = 0;
    const uint32_t TB = P.tb, PP = kBsThreads / TB;
    const uint32_t jt = threadIdx.x & (TB - 1), sidx = threadIdx.x / TB;
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB, cv = P.half << sN;
    const float2 *__restrict__ x = J.x;
    uint4 *F = P.cap <= fcap ? reinterpret_cast<uint4 *>(tw + B / 2 + (B & 1)) : P.surv;
    uint32_t iters = 0;
    for (uint32_t r = 0; r < P.L; ++r) {
        const uint32_t sig = P.sigma[r], tau = P.tau[r];
        // a1 at the shifts, two at a time, bucket tile by bucket tile
        for (uint32_t sh = 0; sh < S; sh += 2) {
            const uint32_t t0 = (tau + bs_shift(P, sh)) & P.mask;
            const uint32_t t1 = sh + 1 < S ? (tau + bs_shift(P, sh + 1)) & P.mask : t0;
            float2 *b0 = bs_s + (size_t)sh * B, *b1 = b0 + B;
            for (uint32_t tile = 0; tile < P.tiles; ++tile) {
                const uint32_t j = tile * TB + jt, jq = (j + P.halfw) & (B - 1);
                float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll 4
                for (uint32_t rr = sidx; rr < P.rounds; rr += PP) {
                    const uint32_t q = rr * B + jq;
                    const uint32_t i = sig * (q - P.halfw);
                    const float g = __ldg(P.taps + q);
                    const float2 v0 = __ldg(x + ((i + t0) & P.mask)), v1 = __ldg(x + ((i + t1) & P.mask));
                    a0r = fmaf(g, v0.x, a0r);
                    a0i = fmaf(g, v0.y, a0i);
                    a1r = fmaf(g, v1.x, a1r);
                    a1i = fmaf(g, v1.y, a1i);
                }
                red0[threadIdx.x] = make_float2(a0r, a0i);
                red1[threadIdx.x] = make_float2(a1r, a1i);
                __syncthreads();
                if (sidx == 0) {
                    float2 c0 = red0[jt], c1 = red1[jt];
                    for (uint32_t k = 1; k < PP; ++k) {
                        c0.x += red0[jt + k * TB].x;
                        c0.y += red0[jt + k * TB].y;
                        c1.x += red1[jt + k * TB].x;
                        c1.y += red1[jt + k * TB].y;
                    }
                    const uint32_t br = __brev(j) >> (32 - logB);
                    b0[br] = c0;
                    b1[br] = c1;
                }
                __syncthreads();
            }
            fft2_smem(b0, b1, B, logB, tw);
        }
        const uint32_t nprev = s_n;
        // subtraction of the found list from every shift's bucket (a fixed order)
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            for (uint32_t e = 0; e < nprev; ++e) {
                const uint4 rec = F[e];
                const uint32_t f = rec.x;
                const uint32_t h = ((sig << sN) * f + cv) >> top;
                const uint32_t d = (k - h) & (B - 1);
                if (d != 0 && d != 1 && d != B - 1) continue;
                // nu = (sigma f mod N) - k N/B, wrapped into [-N/2, N/2)
                const int32_t nu = (int32_t)((((sig * f) & P.mask) - k * NB + N / 2) & P.mask) - (int32_t)(N / 2);
                const float2 G = __ldg(P.gext + (nu + (int32_t)(3 * NB / 2)));
                const float2 c0 = cmul(cmul(make_float2(__uint_as_float(rec.z), __uint_as_float(rec.w)),
                                            turn_pos((tau << sN) * f)),
                                       G);
                for (uint32_t sh = 0; sh < S; ++sh) {
                    const float2 c = sh ? cmul(c0, turn_pos((bs_shift(P, sh) * f) << sN)) : c0;
                    float2 &z = bs_s[(size_t)sh * B + k];
                    z.x -= c.x;
                    z.y -= c.y;
                }
            }
        }
        if (threadIdx.x == 0) s_active = 0;
        __syncthreads();
        if (r == 0) {
            // 1e-6 of the largest bucket energy, and at least kSearchKappa times
            // the median one (the ceil(B/2)-th largest: the noise floor of a
            // noisy signal); the energies' bits go through the tail area (the
            // found list is still empty, the top-K buffer not yet in use)
            uint32_t *ek = reinterpret_cast<uint32_t *>(tw + B / 2 + (B & 1));
            float m = 0.f;
            for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
                const float e = bs_s[k].x * bs_s[k].x + bs_s[k].y * bs_s[k].y;
                m = fmaxf(m, e);
                ek[k] = __float_as_uint(e);
            }
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if ((threadIdx.x & 31) == 0) s_wmax[threadIdx.x >> 5] = m;
            __syncthreads();
            const float emed = __uint_as_float(
                block_kth_largest<kBsThreads, false>(ek, B, (B + 1) / 2, s_hist, s_wsum, &s_prefix, &s_need));
            if (threadIdx.x == 0) {
                float mm = 0.f;
                for (uint32_t w2 = 0; w2 < blockDim.x / 32; ++w2) mm = fmaxf(mm, s_wmax[w2]);
                s_thr = fmaxf(1e-6f * mm, kSearchKappa * emed);
            }
            __syncthreads();
        }
        const float thr = s_thr;
        uint32_t active = 0;
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z0 = bs_s[k];
            const float e0 = z0.x * z0.x + z0.y * z0.y;
            if (!(e0 >= thr) || e0 == 0.f) continue;
            ++active;
            // digits of f, low to high: rb = f mod 2^lo so far
            uint32_t rb = 0;
            for (uint32_t j = 0, lo = 0; lo < bits; ++j, lo += b) {
                const uint32_t m = min(lo + b, bits);
                const float2 zj = bs_s[(size_t)(j + 1) * B + k];
                const float2 rj = make_float2(zj.x * z0.x + zj.y * z0.y, zj.y * z0.x - zj.x * z0.y);  // zj conj(z0)
                uint32_t best = 0;
                float bestv = -INFINITY;
                for (uint32_t dd = 0; dd < (1u << (m - lo)); ++dd) {
                    const uint32_t cand = rb + (dd << lo);
                    // Re(rj exp(-2 pi i cand / 2^m))
                    const float2 u = turn_pos(cand << (32 - m));
                    const float v = rj.x * u.x + rj.y * u.y;
                    if (v > bestv) {
                        bestv = v;
                        best = dd;
                    }
                }
                rb += best << lo;
            }
            // p = sigma f (mod N): p = sigma rb (mod W) in [k N/B - W/2, k N/B + W/2)
            const uint32_t pr = (sig * rb) & (W - 1);
            const uint32_t lo_p = (k * NB - W / 2) & P.mask;
            const uint32_t p = (lo_p + ((pr - lo_p) & (W - 1))) & P.mask;
            const uint32_t f = (inv_mod_2p32(sig) * p) & P.mask;
            const uint32_t t = (sig << sN) * f + cv;
            if ((t >> top) != k) continue;  // a neighbour's leakage
            float res = 0.f;
            for (uint32_t sh = 1; sh < S; ++sh) {
                const float2 zj = bs_s[(size_t)sh * B + k];
                const float2 pz = cmul(z0, turn_pos((bs_shift(P, sh) * f) << sN));
                res += (zj.x - pz.x) * (zj.x - pz.x) + (zj.y - pz.y) * (zj.y - pz.y);
            }
            if (res > kSearchRho * (float)(S - 1) * e0) continue;  // not a lone coefficient
            const uint32_t opos = P.logB < P.logN ? (t << P.logB) >> (P.logB + sN) : 0u;
            const float2 v = turn_scale(z0, __ldg(P.ginv + opos), (tau << sN) * f);
            bool merged = false;
            for (uint32_t e2 = 0; e2 < nprev; ++e2) {
                const uint4 rec = F[e2];
                if (rec.x == f) {  // f has one home bucket: one writer per iteration
                    F[e2] = make_uint4(f, 0u, __float_as_uint(__uint_as_float(rec.z) + v.x),
                                       __float_as_uint(__uint_as_float(rec.w) + v.y));
                    merged = true;
                    break;
                }
            }
            if (!merged) {
                const uint32_t pos = atomicAdd(&s_n, 1u);  // < cap: at most B per iteration
                F[pos] = make_uint4(f, 0u, __float_as_uint(v.x), __float_as_uint(v.y));
            }
        }
        active = __reduce_add_sync(0xFFFFFFFFu, active);
        if ((threadIdx.x & 31) == 0 && active) atomicAdd(&s_active, active);
        __threadfence_block();
        __syncthreads();
        iters = r + 1;
        if (s_active == 0) break;  // uniform
    }
    const uint32_t Sn = s_n;
    if (threadIdx.x == 0) {
        P.ctr[kNGe] = Sn;
        P.ctr[kPeIter] = iters;
        P.ctr[kTheta] = __float_as_uint(s_thr);
    }
    for (uint32_t i = threadIdx.x; i < Sn; i += blockDim.x) {
        uint4 rec = F[i];
        const float re = __uint_as_float(rec.z), im = __uint_as_float(rec.w);
        rec.y = __float_as_uint(re * re + im * im);
        P.surv[i] = rec;
    }
    __threadfence_block();
    __syncthreads();
    unsigned long long *tk = reinterpret_cast<unsigned long long *>(tw + B / 2 + (B & 1));
    rank_records(P, J, tk, cap, Sn, min(Sn, P.K));
}

// Stage kernels for the single-step entry points.
template <int LT>
__global__ void k_estimate_list(const PlanDev *pd, const float2 *zhat, const int32_t *cand, uint32_t n,
                                float2 *est) {
    __shared__ PlanDev P;
    load_plan(P, pd);
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        est[i] = combined_estimate<LT>(P, zhat, (uint32_t)cand[i]);
}

__global__ void k_flags_from_sel(const PlanDev *pd, const int32_t *sel) {
    __shared__ PlanDev P;
    load_plan(P, pd);
    __syncthreads();
    const uint32_t l = blockIdx.x;
    uint16_t *frow = P.flags + (size_t)l * P.B;
    for (uint32_t k = threadIdx.x; k < P.B; k += blockDim.x) frow[k] = 0;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < P.nsel; s += blockDim.x) {
        const int32_t k = sel[(size_t)l * P.nsel + s];
        if (k >= 0 && (uint32_t)k < P.B) frow[k] = 1;
    }
}

// ------------------------------------------ iterative-framework refinement
// After the top K ("Four algorithmic frameworks", its iterative framework,
// applied to the voting output): P.refine passes, each re-estimating every
// found coefficient f in every loop from its bucket after subtracting the
// other found coefficients that hash to the same or a neighbouring bucket
// (their gain from the three-bucket table gext; further out the flat
// window's gain is below its stop-band floor), with the previous pass's
// values, then combining the L estimates as the plan does.  One CTA of
// kRefineThreads per job runs all passes, the (f, l) pairs spread over its
// threads.  The found set sits in shared memory (previous and current
// values [K], frequencies [K]), the per-loop estimates of a pass in P.rscr.
// Neighbours: with L B <= kRefineBinMax and n L <= kRefineSortMax the
// found coefficients are counting-sorted once into the L B (loop, bucket)
// bins (the buckets do not change between passes; each bin ordered by index,
// so the subtraction order is fixed) and a pair reads its three bins
// directly; otherwise it compares every other coefficient's bucket.  LT = L
// in {8, 12, 16} combines with sorting networks in registers.
constexpr int kRefineThreads = 1024;
constexpr uint32_t kRefineSortMax = 4096;   // (f, l) pairs of the binned lists
constexpr uint32_t kRefineBinMax = 16384;   // bins: L B

template <int LT>
__global__ void __launch_bounds__(kRefineThreads) k_refine(Launch ln) {
    extern __shared__ float2 rq_s[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_wsum[kRefineThreads / 32];
    enter(ln, P, J, s_local);
    if (P.refine == 0) return;  // (uniform over the CTA)
    const uint32_t K = P.K, L = LT > 0 ? (uint32_t)LT : P.L, B = P.B, N = P.N, NB = N >> P.logB;
    const uint32_t n = min((uint32_t)max(__ldcg(J.kout), 0), K);
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB, cv = P.half << sN;
    float2 *cur = rq_s, *nxt = rq_s + K;
    uint32_t *fi = reinterpret_cast<uint32_t *>(rq_s + 2 * K);
    uint32_t *bend = fi + K;                                          // [L B] end of each bin
    uint16_t *ord = reinterpret_cast<uint16_t *>(bend + kRefineBinMax);  // [n L] indices by bin
    for (uint32_t i = threadIdx.x; i < n; i += kRefineThreads) {
        fi[i] = (uint32_t)__ldcg(J.idx + i);
        cur[i] = __ldcg(J.val + i);
    }
    const uint32_t nbin = L * B;
    const bool binned = nbin <= kRefineBinMax && n * L <= kRefineSortMax;
    if (binned) {
        for (uint32_t b = threadIdx.x; b < nbin; b += kRefineThreads) bend[b] = 0;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < n * L; j += kRefineThreads) {
            const uint32_t l = j / n, i = j - l * n;
            atomicAdd(&bend[l * B + (((P.sigma[l] << sN) * fi[i] + cv) >> top)], 1u);
        }
        __syncthreads();
        // exclusive starts: each thread scans a contiguous run of bins
        const uint32_t per = (nbin + kRefineThreads - 1) / kRefineThreads;
        const uint32_t b0 = min(nbin, threadIdx.x * per), b1 = min(nbin, b0 + per);
        uint32_t run = 0;
        for (uint32_t b = b0; b < b1; ++b) run += bend[b];
        uint32_t st = block_incl_scan_n<kRefineThreads / 32>(run, s_wsum) - run;
        for (uint32_t b = b0; b < b1; ++b) {
            const uint32_t c = bend[b];
            bend[b] = st;  // start, advanced to the end by the scatter below
            st += c;
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < n * L; j += kRefineThreads) {
            const uint32_t l = j / n, i = j - l * n;
            const uint32_t b = l * B + (((P.sigma[l] << sN) * fi[i] + cv) >> top);
            ord[atomicAdd(&bend[b], 1u)] = (uint16_t)i;
        }
        __syncthreads();
        // each bin in index order (bins hold a few entries)
        for (uint32_t b = threadIdx.x; b < nbin; b += kRefineThreads) {
            const uint32_t e = bend[b], s0 = b ? bend[b - 1] : 0u;
            for (uint32_t x = s0 + 1; x < e; ++x) {
                const uint16_t v = ord[x];
                uint32_t y = x;
                while (y > s0 && ord[y - 1] > v) {
                    ord[y] = ord[y - 1];
                    --y;
                }
                ord[y] = v;
            }
        }
    }
    __syncthreads();
    for (uint32_t pass = 0; pass < P.refine; ++pass) {
        for (uint32_t w = threadIdx.x; w < n * L; w += kRefineThreads) {
            const uint32_t i = w / L, l = w - i * L;
            const uint32_t sig = P.sigma[l], tau = P.tau[l], a = sig << sN;
            const uint32_t f = fi[i], h = (a * f + cv) >> top;
            float2 r = __ldcg(P.zhat + (size_t)l * B + h);
            auto subtract = [&](uint32_t d) {
                const uint32_t g = fi[d];
                // nu = (sigma g mod N) - h N/B, wrapped into [-N/2, N/2): within +-3N/2B
                const int32_t nu =
                    (int32_t)((((sig * g) & P.mask) - h * NB + N / 2) & P.mask) - (int32_t)(N / 2);
                const float2 G = __ldg(P.gext + (nu + (int32_t)(3 * NB / 2)));
                const float2 c = cmul(cmul(cur[d], turn_pos((tau << sN) * g)), G);
                r.x -= c.x;
                r.y -= c.y;
            };
            if (binned) {
                const uint32_t nb = B < 3 ? B : 3;  // buckets h - 1, h, h + 1 (distinct ones)
                for (uint32_t q = 0; q < nb; ++q) {
                    const uint32_t b = l * B + ((B >= 3 ? h + B - 1 + q : h + q) & (B - 1));
                    const uint32_t e = bend[b];
                    for (uint32_t x = b ? bend[b - 1] : 0u; x < e; ++x) {
                        const uint32_t d = ord[x];
                        if (d != i) subtract(d);
                    }
                }
            } else {
                for (uint32_t d = 0; d < n; ++d) {
                    const uint32_t dd = (((a * fi[d] + cv) >> top) - h) & (B - 1);
                    if (d != i && (dd == 0 || dd == 1 || dd == B - 1)) subtract(d);
                }
            }
            uint32_t hh, opos;
            hash_freq(P, sig, f, hh, opos);
            P.rscr[(size_t)i * L + l] = turn_scale(r, __ldg(P.ginv + opos), (tau << sN) * f);
        }
        __syncthreads();  // the pass's (f, l) estimates are written
        for (uint32_t i = threadIdx.x; i < n; i += kRefineThreads) {
            const float2 *v = P.rscr + (size_t)i * L;
            if (P.estimator == kEstMean) {
                float sr = 0.f, si = 0.f;
                for (uint32_t l = 0; l < L; ++l) {
                    const float2 e = __ldcg(v + l);
                    sr += e.x;
                    si += e.y;
                }
                nxt[i] = make_float2(sr / (float)L, si / (float)L);
            } else if constexpr (LT > 0) {
                float re[LT], im[LT];
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    const float2 e = __ldcg(v + l);
                    re[l] = e.x;
                    im[l] = e.y;
                }
                sort_net<LT>(re);
                sort_net<LT>(im);
                nxt[i] = make_float2(median_sorted(re, LT), median_sorted(im, LT));
            } else {
                float re[kMaxL], im[kMaxL];
                for (uint32_t l = 0; l < L; ++l) {
                    const float2 e = __ldcg(v + l);
                    uint32_t a = l, b = l;
                    while (a > 0 && re[a - 1] > e.x) {
                        re[a] = re[a - 1];
                        --a;
                    }
                    re[a] = e.x;
                    while (b > 0 && im[b - 1] > e.y) {
                        im[b] = im[b - 1];
                        --b;
                    }
                    im[b] = e.y;
                }
                nxt[i] = make_float2(median_sorted(re, L), median_sorted(im, L));
            }
        }
        __syncthreads();  // (the next pass reads nxt and rewrites P.rscr)
        float2 *t = cur;
        cur = nxt;
        nxt = t;
    }
    for (uint32_t i = threadIdx.x; i < n; i += kRefineThreads) J.val[i] = cur[i];
}

template <int LT, int TAB>
cudaError_t scan_variant(const Launch &ln, uint32_t ctas, int mode, uint32_t smem, int32_t *cand_out,
                         int32_t *ncand_out, cudaStream_t s) {
    auto kern = k_vote_scan<LT, TAB>;
    if (TAB == kTabSmem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<ctas, kThreads, TAB == kTabSmem ? smem : 0, s>>>(ln, mode, cand_out, ncand_out);
    return cudaGetLastError();
}

template <int TAB>
cudaError_t scan_dispatch_l(const Launch &ln, uint32_t ctas, int mode, uint32_t L, uint32_t smem, int32_t *cand_out,
                            int32_t *ncand_out, cudaStream_t s) {
    switch (L) {
        case 8: return scan_variant<8, TAB>(ln, ctas, mode, smem, cand_out, ncand_out, s);
        case 12: return scan_variant<12, TAB>(ln, ctas, mode, smem, cand_out, ncand_out, s);
        case 16: return scan_variant<16, TAB>(ln, ctas, mode, smem, cand_out, ncand_out, s);
        default: return scan_variant<0, TAB>(ln, ctas, mode, smem, cand_out, ncand_out, s);
    }
}

}  // namespace

cudaError_t launch_gather(const Launch &ln, uint32_t total_ctas, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    k_gather<<<total_ctas, kThreads, 0, s>>>(ln);
    return cudaGetLastError();
}

cudaError_t launch_fft_select(const Launch &ln, uint32_t total_ctas, uint32_t max_B, int select_only,
                              uint32_t cluster_L, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    const int smem = (int)(max_B * (sizeof(float2) + sizeof(uint32_t)) +
                           (max_B <= kTwSmemMaxB ? max_B / 2 * sizeof(float2) : 0) + (cluster_L ? max_B : 0));
    cudaError_t e = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (!cluster_L) {
        k_fft_select<<<total_ctas, kThreads, smem, s>>>(ln, select_only, 0);
        return cudaGetLastError();
    }
    if (cluster_L > 8) {
        e = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total_ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster_L;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fft_select, ln, select_only, 1);
}

bool fft_select_cluster_ok(uint32_t L, uint32_t max_B) {
    if (L < 2 || L > 16 || max_B > (uint32_t)kClusterMaxB) return false;
    static std::mutex mu;
    static int known[17][2] = {};  // [L][B > 1024]: 0 unknown, 1 yes, 2 no
    const int bb = max_B > 1024 ? 1 : 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!known[L][bb]) {
        const uint32_t qB = bb ? (uint32_t)kClusterMaxB : 1024u;
        const int smem = (int)(qB * (sizeof(float2) + sizeof(uint32_t)) + qB / 2 * sizeof(float2) + qB);
        bool ok = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
        if (ok && L > 8)
            ok = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
        int n = 0;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(L);
            cfg.blockDim = dim3(kThreads);
            cfg.dynamicSmemBytes = (size_t)smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = L;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            ok = cudaOccupancyMaxActiveClusters(&n, k_fft_select, &cfg) == cudaSuccess && n > 0;
        }
        cudaGetLastError();  // a refused query leaves no sticky error
        known[L][bb] = ok ? 1 : 2;
    }
    return known[L][bb] == 1;
}

cudaError_t launch_vote(const Launch &ln, uint32_t total_ctas, int mode, uint32_t L_uniform, bool bits,
                        uint32_t max_flags_bytes, int32_t *cand_out, int32_t *ncand_out, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    if (mode == kVotePrune && scan_uses_bits(L_uniform, bits)) {
        switch (L_uniform) {
            case 8: k_scan_bits<8><<<total_ctas, kThreads, 0, s>>>(ln); break;
            case 12: k_scan_bits<12><<<total_ctas, kThreads, 0, s>>>(ln); break;
            default: k_scan_bits<16><<<total_ctas, kThreads, 0, s>>>(ln); break;
        }
        return cudaGetLastError();
    }
    if (max_flags_bytes <= (uint32_t)kFlagsSmemBytes)
        return scan_dispatch_l<kTabSmem>(ln, total_ctas, mode, L_uniform, max_flags_bytes, cand_out, ncand_out, s);
    return scan_dispatch_l<kTabGlobal>(ln, total_ctas, mode, L_uniform, 0, cand_out, ncand_out, s);
}

cudaError_t launch_estimate(const Launch &ln, uint32_t njobs, uint32_t L_uniform, uint32_t per, uint32_t tab_smem,
                            uint32_t max_K, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const uint32_t ctas = njobs * per;
    uint32_t cap = kRankMax;
    while (cap < max_K) cap <<= 1;  // the top-K buffer holds the K winners (and up to kRankMax records)
    const uint32_t topk_smem = cap * (uint32_t)(sizeof(unsigned long long) + sizeof(uint32_t));
    if (tab_smem && (L_uniform == 8 || L_uniform == 12 || L_uniform == 16)) {
        auto kern = L_uniform == 8 ? k_estimate_tab<8> : (L_uniform == 12 ? k_estimate_tab<12> : k_estimate_tab<16>);
        const uint32_t smem = max(tab_smem, topk_smem);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<ctas, kThreads, smem, s>>>(ln, per, cap);
        return cudaGetLastError();
    }
    auto kern = L_uniform == 8    ? k_estimate_surv<8>
                : L_uniform == 12 ? k_estimate_surv<12>
                : L_uniform == 16 ? k_estimate_surv<16>
                                  : k_estimate_surv<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)topk_smem);
    if (e != cudaSuccess) return e;
    kern<<<ctas, kThreads, topk_smem, s>>>(ln, per, cap);
    return cudaGetLastError();
}


cudaError_t launch_comb(const Launch &ln, uint32_t njobs, uint32_t max_Bc, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const int smem = (int)(sizeof(float2) * 3 * max_Bc);  // two spectra, per-pass twiddles
    cudaError_t e = cudaFuncSetAttribute(k_comb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_comb<<<njobs, kCombThreads, smem, s>>>(ln);
    return cudaGetLastError();
}

cudaError_t launch_pe(const Launch &ln, uint32_t njobs, uint32_t max_B, uint32_t max_K, uint32_t max_cap,
                      cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    uint32_t cap = kRankMax;
    while (cap < max_K) cap <<= 1;
    const size_t tables = (sizeof(float2) * (2 * max_B + max_B / 2 + 1) + 15) & ~(size_t)15;
    const size_t rank = cap * (sizeof(unsigned long long) + sizeof(uint32_t));
    // found list in shared memory when every job's fits kPeSmemFound entries
    const uint32_t fcap = max_cap <= kPeSmemFound ? max_cap : 0u;
    const int smem = (int)(tables + std::max<size_t>(rank, sizeof(uint4) * fcap));
    cudaError_t e = cudaFuncSetAttribute(k_pe_job, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_pe_job<<<njobs, kThreads, smem, s>>>(ln, cap, fcap);
    return cudaGetLastError();
}

cudaError_t launch_refine(const Launch &ln, uint32_t njobs, uint32_t max_K, uint32_t L_uniform, cudaStream_t s) {
    if (njobs == 0 || max_K == 0) return cudaSuccess;
    // values [2][K], frequencies [K], bin ends [kRefineBinMax], binned indices [kRefineSortMax]
    const int smem = (int)((2 * sizeof(float2) + sizeof(uint32_t)) * max_K + sizeof(uint32_t) * kRefineBinMax +
                           sizeof(uint16_t) * kRefineSortMax);
    auto kern = L_uniform == 8 ? k_refine<8> : L_uniform == 12 ? k_refine<12> : L_uniform == 16 ? k_refine<16>
                                                                                                    : k_refine<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<njobs, kRefineThreads, smem, s>>>(ln);
    return cudaGetLastError();
}

cudaError_t launch_bs(const Launch &ln, uint32_t njobs, uint32_t max_B, uint32_t max_K, uint32_t max_cap,
                      uint32_t max_nbuf, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    uint32_t cap = kRankMax;
    while (cap < max_K) cap <<= 1;
    const size_t tables = (sizeof(float2) * ((size_t)max_nbuf * max_B + max_B / 2 + 1) + 15) & ~(size_t)15;
    const size_t rank = cap * (sizeof(unsigned long long) + sizeof(uint32_t));
    const uint32_t fcap = max_cap <= kPeSmemFound ? max_cap : 0u;
    // tail: the top-K ranks or the found list, and the energies' bits of the threshold
    const size_t tail = std::max<size_t>(std::max<size_t>(rank, sizeof(uint4) * fcap), sizeof(uint32_t) * max_B);
    const int smem = (int)(tables + tail);
    auto kern = max_B >= kBsWideB ? k_bs_job<1024> : k_bs_job<256>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<njobs, max_B >= kBsWideB ? 1024 : 256, smem, s>>>(ln, cap, fcap, max_nbuf);
    return cudaGetLastError();
}

cudaError_t launch_estimate_list(const PlanDev *p, uint32_t L, const float2 *zhat, const int32_t *cand,
                                 uint32_t n, float2 *est, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = min((n + 255) / 256, 4096u);
    switch (L) {
        case 8: k_estimate_list<8><<<blocks, 256, 0, s>>>(p, zhat, cand, n, est); break;
        case 12: k_estimate_list<12><<<blocks, 256, 0, s>>>(p, zhat, cand, n, est); break;
        case 16: k_estimate_list<16><<<blocks, 256, 0, s>>>(p, zhat, cand, n, est); break;
        default: k_estimate_list<0><<<blocks, 256, 0, s>>>(p, zhat, cand, n, est); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_flags_from_sel(const PlanDev *p, uint32_t L, const int32_t *sel, cudaStream_t s) {
    k_flags_from_sel<<<L, 256, 0, s>>>(p, sel);
    return cudaGetLastError();
}

}  // namespace sfft
