// Device helpers shared by the kernel files (kernels.cu: the voting
// pipeline; kernels_variants.cu: the pre-filter, the iterative-framework
// methods and the refinement).  Everything sits in an unnamed namespace:
// each file compiles its own copies.
#pragma once

#include <cooperative_groups.h>
#include <math_constants.h>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

constexpr int kThreads = 256;  // every kernel but the comb
constexpr int kCombThreads = 1024;
constexpr uint32_t kTwSmemMaxB = 8192;  // FFT twiddles staged in shared memory up to this B

// Launch of a pipeline kernel after the stream's previous kernel with
// programmatic dependent launch (the kernel's CTAs may start while that
// kernel finishes and wait in enter()), in clusters of `cluster` CTAs when
// nonzero.  The kernel must wait (enter() or grid_dep_wait()) before it
// reads anything an earlier kernel of the stream wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), uint32_t grid, uint32_t block, size_t smem, cudaStream_t s,
                       uint32_t cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    unsigned n = 0;
    at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (cluster) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = cluster;
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

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

// Programmatic dependent launch: wait for the stream's previous kernel to
// complete (its writes visible; a no-op when this launch does not overlap
// it), and allow the stream's next kernel to start its prologue.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Locate + load in one call; every kernel starts with it.  The job list and
// the plan descriptor are written before a pipeline's first kernel, so they
// are read before the wait for the previous kernel (launch_pdl overlaps this
// prologue with that kernel's tail).
__device__ __forceinline__ void enter(const Launch &ln, PlanDev &P, Job &J, uint32_t &s_local) {
    if (threadIdx.x == 0) {
        Job j;
        uint32_t loc;
        locate(ln, ln.cta0 + blockIdx.x, j, loc);
        J = j;
        s_local = loc;
    }
    __syncthreads();
    load_plan(P, J.p);
    __syncthreads();
    grid_dep_wait();
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

__device__ __forceinline__ unsigned long long surv_key(uint4 r) {
    return ((unsigned long long)r.y << 32) | (uint32_t)(~r.x);  // key desc, then f asc
}

// Records up to this many are ranked by counting comparisons.
constexpr uint32_t kRankMax = 1024;

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

}  // namespace

}  // namespace sfft
