// Hot-path kernels of the flat-window voting sparse FFT (steps a1..a7).
//
// Every kernel takes a Launch descriptor: one job by value (plain execute) or
// an array of jobs in device memory with a per-kernel CTA prefix (batched
// execute).  A CTA locates its job, copies the job's PlanDev into shared
// memory and works on one tile of that job.
#include <math_constants.h>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

constexpr int kGatherThreads = 256;
constexpr int kSelectThreads = 256;
constexpr int kVoteThreads = 256;
constexpr int kTopkThreads = 1024;

__device__ __forceinline__ void locate(const Launch &ln, uint32_t bid, Job &job, uint32_t &local) {
    if (ln.jobs == nullptr) {
        job = ln.one;
        local = bid;
        return;
    }
    int lo = 0, hi = ln.njobs;  // offs[lo] <= bid < offs[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(ln.offs + mid) <= bid) lo = mid;
        else hi = mid;
    }
    job = ln.jobs[lo];
    local = bid - __ldg(ln.offs + lo);
}

// Copy the job's plan descriptor into shared memory (call from all threads,
// then __syncthreads()).
__device__ __forceinline__ void load_plan(PlanDev &dst, const PlanDev *src) {
    static_assert(sizeof(PlanDev) % 8 == 0, "PlanDev must be 8-byte sized");
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(&dst);
    for (uint32_t i = threadIdx.x; i < sizeof(PlanDev) / 8; i += blockDim.x) d[i] = __ldg(s + i);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Round-half-up flat-filter hash of frequency f in loop l: bucket h and the
// offset o from the bucket centre, returned as o + half in [0, N/B).
__device__ __forceinline__ void hash_freq(const PlanDev &P, uint32_t sigma, uint32_t f, uint32_t &h,
                                          uint32_t &opos) {
    uint32_t p = (sigma * f) & P.mask;
    uint32_t hh = (p + P.half) >> P.shift;  // in [0, B]
    opos = p + P.half - (hh << P.shift);
    h = hh & (P.B - 1);
}

// ------------------------------------------------------------------ a1
// z_l[j] partial sums: sum over the rounds of one chunk of
// g(m) * x[(sigma_l m + tau_l) mod N] for the window positions m = j (mod B).
__global__ void __launch_bounds__(kGatherThreads) k_gather(Launch ln) {
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ float2 red[kGatherThreads];
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

    const uint32_t local = s_local;
    const uint32_t tile = local % P.tiles;
    const uint32_t rest = local / P.tiles;
    const uint32_t l = rest % P.L;
    const uint32_t chunk = rest / P.L;
    const uint32_t TB = P.tb;
    const uint32_t PP = kGatherThreads / TB;  // threads sharing one bucket
    const uint32_t jt = threadIdx.x & (TB - 1);
    const uint32_t s = threadIdx.x / TB;
    const uint32_t j = tile * TB + jt;
    const uint32_t r0 = chunk * P.rpc;
    const uint32_t r1 = min(P.rounds, r0 + P.rpc);
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
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long x = a[i], y = a[ixj];
                    bool desc = (i & k) == 0;
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
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long x = a[i], y = a[ixj];
                    bool up = ((i & k) == 0) == asc;
                    if (up ? (x > y) : (x < y)) {
                        a[i] = y;
                        a[ixj] = x;
                        uint32_t t = pay[i];
                        pay[i] = pay[ixj];
                        pay[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// K-th largest of n non-negative floats (as bit patterns) by four 8-bit radix
// passes over a 256-bin shared histogram; called by all threads of a block.
__device__ uint32_t radix_kth_largest(const float *v, uint32_t n, uint32_t k, uint32_t *hist,
                                      uint32_t *s_prefix, uint32_t *s_need) {
    if (threadIdx.x == 0) {
        *s_prefix = 0;
        *s_need = k;
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 24 - 8 * pass;
        const uint32_t pmask = pass == 0 ? 0u : (0xFFFFFFFFu << (sh + 8));
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = *s_prefix;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t u = __float_as_uint(__ldcg(v + i));
            if ((u & pmask) == prefix) atomicAdd(&hist[(u >> sh) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t need = *s_need, cum = 0;
            int d = 255;
            for (; d > 0; --d) {
                if (cum + hist[d] >= need) break;
                cum += hist[d];
            }
            *s_need = need - cum;
            *s_prefix = prefix | ((uint32_t)d << sh);
        }
        __syncthreads();
    }
    return *s_prefix;
}

// -------------------------------------------------------------- a2 + a3
// One CTA per (job, loop): sum the gather partials, B-point radix-2 FFT in
// shared memory, bucket energies, top-nsel selection (energy descending,
// ties to the lower bucket).  The last CTA of a job derives the prune
// threshold theta and the strong-bucket flags for all loops.
__global__ void __launch_bounds__(kSelectThreads) k_fft_select(Launch ln, int select_only) {
    extern __shared__ unsigned long long sm[];  // B entries
    float2 *buf = reinterpret_cast<float2 *>(sm);
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ int s_last;
    __shared__ float s_theta;
    __shared__ uint32_t s_hist[256], s_prefix, s_need;
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

    const uint32_t l = s_local, B = P.B, logB = P.logB;
    float2 *zrow = P.zhat + (size_t)l * B;
    float *erow = P.energy + (size_t)l * B;
    if (!select_only) {
        for (uint32_t j = threadIdx.x; j < B; j += blockDim.x) {
            float2 acc = make_float2(0.f, 0.f);
            for (uint32_t c = 0; c < P.nchunk; ++c) {
                float2 v = P.partial[((size_t)c * P.L + l) * B + j];
                acc.x += v.x;
                acc.y += v.y;
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
                const float2 w = __ldg(P.tw + (k << (logB - 1 - hs)));
                const float2 a = buf[i0];
                const float2 t = cmul(w, buf[i1]);
                buf[i0] = make_float2(a.x + t.x, a.y + t.y);
                buf[i1] = make_float2(a.x - t.x, a.y - t.y);
            }
            __syncthreads();
        }
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z = buf[k];
            zrow[k] = z;
            erow[k] = z.x * z.x + z.y * z.y;
        }
    } else {
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z = zrow[k];
            erow[k] = z.x * z.x + z.y * z.y;
        }
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x)
        sm[k] = ((unsigned long long)__float_as_uint(erow[k]) << 32) | (uint32_t)(~k);
    __syncthreads();
    bitonic_desc(sm, B);
    for (uint32_t s = threadIdx.x; s < P.nsel; s += blockDim.x)
        P.sel[(size_t)l * P.nsel + s] = (int32_t)(~(uint32_t)sm[s]);
    uint16_t *frow = P.flags + (size_t)l * B;
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) frow[k] = 0;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < P.nsel; s += blockDim.x) frow[~(uint32_t)sm[s]] = 1;

    // ---- last CTA of the job: theta and the kept/strong tables
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(P.ctr + kSelDone, 1u) == P.L - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t total = P.L * B;
    // theta = 1/4 of the K-th largest bucket energy over all loops: a guess at
    // a lower bound of the K-th largest estimate.  Exactness never depends on
    // it; a guess that is too high only sends the job to the fallback pass.
    if (P.K <= total) {
        const uint32_t kth = radix_kth_largest(P.energy, total, P.K, s_hist, &s_prefix, &s_need);
        if (threadIdx.x == 0) {
            float theta = 0.25f * __uint_as_float(kth);
            if (!(theta >= 0.f) || isinf(theta)) theta = 0.f;
            s_theta = theta;
        }
    } else if (threadIdx.x == 0) {
        s_theta = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) P.ctr[kTheta] = __float_as_uint(s_theta);
    // a loop is "strong" for f when |zhat|^2 * max|1/G~|^2 >= theta/2; with
    // fewer than M strong loops the median estimate is provably below theta
    const float thr = 0.5f * s_theta;
    const float gmul = P.ginv2max * (1.0f + 1.0f / 1024.0f);
    for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
        const float en = __ldcg(P.energy + e);
        uint16_t f = __ldcg(reinterpret_cast<const unsigned short *>(P.flags) + e) & 1u;
        if (en * gmul >= thr) f |= 256;
        P.flags[e] = f;
    }
    if (P.use_shfl) {
        __syncthreads();
        const uint32_t bpl = 1u << P.lbpl;
        for (uint32_t idx = threadIdx.x; idx < P.L * 32; idx += blockDim.x) {
            const uint32_t ll = idx >> 5, j = idx & 31;
            const uint16_t *fr = P.flags + (size_t)ll * B + j * bpl;
            uint32_t word = 0;
            for (uint32_t b = 0; b < bpl; ++b) {
                const uint32_t fl = fr[b];
                word |= (fl & 1u) << b;
                word |= ((fl >> 8) & 1u) << (16 + b);
            }
            P.packed[idx] = word;
        }
    }
    if (threadIdx.x == 0) {
        P.ctr[kSelDone] = 0;
        P.ctr[kNCand] = 0;
        P.ctr[kNSurv] = 0;
        P.ctr[kNGe] = 0;
        P.ctr[kNSurv2] = 0;
    }
}

// ------------------------------------------------------------------ a6
template <int N>
__device__ __forceinline__ void sort_net(float *a) {
#pragma unroll
    for (int pass = 0; pass < N; ++pass) {
#pragma unroll
        for (int i = pass & 1; i + 1 < N; i += 2) {
            const float x = a[i], y = a[i + 1];
            a[i] = fminf(x, y);
            a[i + 1] = fmaxf(x, y);
        }
    }
}

__device__ __forceinline__ float median_sorted(const float *a, uint32_t n) {
    return (n & 1) ? a[n / 2] : 0.5f * (a[n / 2 - 1] + a[n / 2]);
}

// Per-loop energy-concentration estimate of frequency f in loop l:
// zhat_l[h] * exp(-2 pi i tau_l f / N) / G~(o).
__device__ __forceinline__ float2 loop_estimate(const PlanDev &P, const float2 *zhat, uint32_t l,
                                                uint32_t f) {
    uint32_t h, opos;
    hash_freq(P, P.sigma[l], f, h, opos);
    const float2 z = zhat[(size_t)l * P.B + h];
    const float2 g = __ldg(P.ginv + opos);
    const uint32_t r = (P.tau[l] * f) & P.mask;
    const int32_t rs = (int32_t)(r << (32 - P.logN)) >> (32 - P.logN);  // in [-N/2, N/2)
    float sn, cs;
    sincospif(2.0f * (float)rs / (float)P.N, &sn, &cs);
    const float2 zp = make_float2(z.x * cs + z.y * sn, z.y * cs - z.x * sn);
    return cmul(zp, g);
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

// --------------------------------------------------------------- a4 + a5
// Vote scan over all f of a job tile: score(f) = #{l : h_l(f) kept} and the
// number of strong loops, both from one table lookup per loop.  Candidates
// (score >= T) are counted.  Candidates that can still reach the top K
// (strong count >= M in the pruned pass; every candidate in the fallback
// pass) are queued in shared memory and estimated by all threads together;
// the pruned pass records only estimates with key >= theta, the fallback
// pass records all.
template <int LT>
__device__ void flush_queue(const PlanDev &P, const uint32_t *queue, uint32_t qn, int mode, float theta,
                            uint32_t &my_rec) {
    for (uint32_t i = threadIdx.x; i < qn; i += blockDim.x) {
        const uint32_t f = queue[i];
        const float2 v = median_estimate<LT>(P, P.zhat, f);
        const float key = v.x * v.x + v.y * v.y;
        if (mode == kVoteFallback || key >= theta) {
            const uint32_t pos = atomicAdd(P.ctr + (mode == kVotePrune ? kNGe : kNSurv2), 1u);
            P.surv[pos] = make_uint4(f, __float_as_uint(key), __float_as_uint(v.x), __float_as_uint(v.y));
            ++my_rec;
        }
    }
}

enum TableKind : int { kTabGlobal = 0, kTabSmem = 1, kTabShfl = 2 };

template <int LT, int TAB>
__global__ void __launch_bounds__(kVoteThreads) k_vote(Launch ln, int mode, uint32_t fb_ctas, int32_t *cand_out,
                                                       int32_t *ncand_out) {
    extern __shared__ uint16_t tab_s[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_cand, s_est, s_qn;
    __shared__ int s_skip;
    __shared__ uint32_t queue[kVoteTileF];
    if (threadIdx.x == 0) {
        Job j;
        uint32_t loc;
        locate(ln, blockIdx.x, j, loc);
        J = j;
        s_local = loc;
        s_cand = 0;
        s_est = 0;
        s_qn = 0;
    }
    __syncthreads();
    load_plan(P, J.p);
    __syncthreads();
    if (threadIdx.x == 0) {
        int skip = 0;
        if (mode == kVoteFallback) {
            const uint32_t nge = P.ctr[kNGe], nc = P.ctr[kNCand];
            skip = (nge >= P.K) || (nge >= nc);  // the recorded set already decides the top K
        }
        s_skip = skip;
    }
    __syncthreads();
    if (s_skip) return;

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
    // register copies of the loop scalings and (shuffle table) of this lane's bucket bits
    constexpr int LR = LT > 0 ? LT : 1;
    uint32_t sg[LR], pw[LR];
    if constexpr (LT > 0) {
#pragma unroll
        for (int l = 0; l < LT; ++l) {
            sg[l] = P.sigma[l];
            pw[l] = TAB == kTabShfl ? __ldcg(P.packed + l * 32 + lane) : 0u;
        }
    }
    const float theta = mode == kVotePrune ? __uint_as_float(P.ctr[kTheta]) : 0.f;
    const uint32_t Mreq = mode == kVotePrune ? P.M : 0u;
    const uint32_t T = P.T, N = P.N, mask = P.mask, half = P.half, shift = P.shift;
    const uint32_t lshift = shift + P.lbpl, bmask = (1u << P.lbpl) - 1u;
    // fields of the per-frequency accumulator: score | strong << sfield
    constexpr uint32_t sfield = TAB == kTabShfl ? 16 : 8;
    constexpr uint32_t smask = (1u << sfield) - 1u;

    uint32_t per = (N + P.vtiles - 1) / P.vtiles;
    per = (per + kVoteThreads - 1) / kVoteThreads * kVoteThreads;  // <= kVoteTileF
    const uint32_t stride = mode == kVoteFallback ? fb_ctas : P.vtiles;
    uint32_t my_cand = 0, my_rec = 0;
    for (uint32_t tile = s_local; tile < P.vtiles; tile += stride) {
        const uint32_t f0 = tile * per;
        const uint32_t f1 = min(N, f0 + per);
        for (uint32_t base = f0; base < f1; base += kVoteThreads) {
            const uint32_t f = base + threadIdx.x;
            const bool valid = f < f1;
            uint32_t acc = 0;
            if constexpr (TAB == kTabShfl) {
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    // bits [logN-5, logN) of q pick the lane, the next lbpl bits down the bucket in it
                    const uint32_t q = sg[l] * f + half;
                    const uint32_t w = __shfl_sync(0xFFFFFFFFu, pw[l], q >> lshift);
                    acc += (w >> ((q >> shift) & bmask)) & 0x10001u;
                }
            } else if constexpr (LT > 0) {
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    const uint32_t h = ((sg[l] * f + half) & mask) >> shift;
                    acc += tab[l * B + h];
                }
            } else {
                for (uint32_t l = 0; l < L; ++l) {
                    const uint32_t h = ((P.sigma[l] * f + half) & mask) >> shift;
                    acc += tab[l * B + h];
                }
            }
            const bool cand = valid && (acc & smask) >= T;
            my_cand += cand;
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
            const bool surv = cand && (acc >> sfield) >= Mreq;
            const uint32_t bs = __ballot_sync(0xFFFFFFFFu, surv);
            if (bs) {
                uint32_t b0 = 0;
                if (lane == 0) b0 = atomicAdd(&s_qn, __popc(bs));
                b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
                if (surv) queue[b0 + __popc(bs & lanemask_lt())] = f;  // < kVoteTileF: one slot per f of the tile
            }
        }
        if (mode == kVoteCandidates) continue;
        __syncthreads();
        const uint32_t qn = s_qn;
        flush_queue<LT>(P, queue, qn, mode, theta, my_rec);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_est += qn;
            s_qn = 0;
        }
        __syncthreads();
    }
    if (mode == kVoteCandidates) return;
    // block totals
    my_cand = __reduce_add_sync(0xFFFFFFFFu, my_cand);
    if (lane == 0 && my_cand) atomicAdd(&s_cand, my_cand);
    __syncthreads();
    if (threadIdx.x == 0 && mode == kVotePrune) {
        if (s_cand) atomicAdd(P.ctr + kNCand, s_cand);
        atomicAdd(P.ctr + kNSurv, s_est);
    }
}

// ------------------------------------------------------------------ a7
__device__ __forceinline__ unsigned long long surv_key(uint4 r) {
    return ((unsigned long long)r.y << 32) | (uint32_t)(~r.x);  // key desc, then f asc
}

// One CTA per job: the k_out = min(K, candidates) recorded estimates of
// largest magnitude (ties to the lower f), written sorted by f.  Records are
// those of the pruned pass (key >= theta) when at least K of them exist or
// they are all the candidates; otherwise those of the fallback pass (every
// candidate).  Pruned candidates have key < theta, so either set contains
// the top K of all candidates.
__global__ void __launch_bounds__(kTopkThreads) k_topk(Launch ln) {
    extern __shared__ unsigned long long tk[];  // kTopkSmem keys + kTopkSmem payloads
    uint32_t *pay = reinterpret_cast<uint32_t *>(tk + kTopkSmem);
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_S, s_kout, s_hist[256], s_need, s_cnt;
    __shared__ unsigned long long s_prefix, s_pmask;
    if (threadIdx.x == 0) {
        Job j;
        uint32_t loc;
        locate(ln, blockIdx.x, j, loc);
        J = j;
    }
    __syncthreads();
    load_plan(P, J.p);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t nge = P.ctr[kNGe], nc = P.ctr[kNCand];
        const bool fallback = (nge < P.K) && (nge < nc);
        s_S = fallback ? P.ctr[kNSurv2] : nge;
        s_kout = min(P.K, nc);
    }
    __syncthreads();
    const uint32_t S = s_S, kout = s_kout;
    const uint4 *surv = P.surv;
    if (S <= (uint32_t)kTopkSmem) {
        uint32_t n2 = 1;
        while (n2 < S) n2 <<= 1;
        for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
            if (i < S) {
                tk[i] = surv_key(surv[i]);
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
                const unsigned long long k = surv_key(surv[i]);
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
            const unsigned long long k = surv_key(surv[i]);
            if (kout > 0 && k >= kth) {
                const uint32_t pos = atomicAdd(&s_cnt, 1u);
                if (pos < (uint32_t)kTopkSmem) {
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
        const uint4 r = surv[pay[s]];
        J.idx[s] = (int32_t)r.x;
        J.val[s] = make_float2(__uint_as_float(r.z), __uint_as_float(r.w));
    }
    if (threadIdx.x == 0) *J.kout = (int32_t)kout;
}

// Stage kernels for the single-step entry points.
template <int LT>
__global__ void k_estimate_list(const PlanDev *pd, const float2 *zhat, const int32_t *cand,
                                uint32_t n, float2 *est) {
    __shared__ PlanDev P;
    load_plan(P, pd);
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        est[i] = median_estimate<LT>(P, zhat, (uint32_t)cand[i]);
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

template <int LT, int TAB>
cudaError_t vote_variant(const Launch &ln, uint32_t ctas, int mode, uint32_t smem, uint32_t fb_ctas,
                         int32_t *cand_out, int32_t *ncand_out, cudaStream_t s) {
    auto kern = k_vote<LT, TAB>;
    if (TAB == kTabSmem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<ctas, kVoteThreads, TAB == kTabSmem ? smem : 0, s>>>(ln, mode, fb_ctas, cand_out, ncand_out);
    return cudaGetLastError();
}

template <int TAB>
cudaError_t vote_dispatch_l(const Launch &ln, uint32_t ctas, int mode, uint32_t L, uint32_t smem, uint32_t fb_ctas,
                            int32_t *cand_out, int32_t *ncand_out, cudaStream_t s) {
    switch (L) {
        case 8: return vote_variant<8, TAB>(ln, ctas, mode, smem, fb_ctas, cand_out, ncand_out, s);
        case 12: return vote_variant<12, TAB>(ln, ctas, mode, smem, fb_ctas, cand_out, ncand_out, s);
        case 16: return vote_variant<16, TAB>(ln, ctas, mode, smem, fb_ctas, cand_out, ncand_out, s);
        default:
            if (TAB == kTabShfl) return cudaErrorInvalidValue;
            return vote_variant<0, TAB == kTabShfl ? kTabGlobal : TAB>(ln, ctas, mode, smem, fb_ctas, cand_out,
                                                                      ncand_out, s);
    }
}

}  // namespace

cudaError_t launch_gather(const Launch &ln, uint32_t total_ctas, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    k_gather<<<total_ctas, kGatherThreads, 0, s>>>(ln);
    return cudaGetLastError();
}

cudaError_t launch_fft_select(const Launch &ln, uint32_t total_ctas, uint32_t max_B, int select_only,
                              cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    const int smem = (int)(max_B * sizeof(unsigned long long));
    cudaError_t e = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_fft_select<<<total_ctas, kSelectThreads, smem, s>>>(ln, select_only);
    return cudaGetLastError();
}

cudaError_t launch_vote(const Launch &ln, uint32_t total_ctas, int mode, uint32_t L_uniform, bool shfl,
                        uint32_t max_flags_bytes, uint32_t fb_ctas, int32_t *cand_out, int32_t *ncand_out,
                        cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    if (shfl && (L_uniform == 8 || L_uniform == 12 || L_uniform == 16))
        return vote_dispatch_l<kTabShfl>(ln, total_ctas, mode, L_uniform, 0, fb_ctas, cand_out, ncand_out, s);
    if (max_flags_bytes <= (uint32_t)kFlagsSmemBytes)
        return vote_dispatch_l<kTabSmem>(ln, total_ctas, mode, L_uniform, max_flags_bytes, fb_ctas, cand_out,
                                         ncand_out, s);
    return vote_dispatch_l<kTabGlobal>(ln, total_ctas, mode, L_uniform, 0, fb_ctas, cand_out, ncand_out, s);
}

cudaError_t launch_topk(const Launch &ln, uint32_t njobs, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const int smem = kTopkSmem * (int)(sizeof(unsigned long long) + sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_topk<<<njobs, kTopkThreads, smem, s>>>(ln);
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
