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

#include <cstddef>
#include <mutex>
#include <math_constants.h>

#include "device_common.cuh"
#include "sfft_internal.cuh"

namespace sfft {

namespace {

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
    // the FFT/select may be placed once every gather CTA has started (its CTAs
    // take the slots the gather's last, partial wave leaves and wait there)
    grid_dep_launch();

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

// Words per lane and loop of the register table: B/1024 for B >= 1024, else 1.
__host__ __device__ __forceinline__ uint32_t table_words(uint32_t logB) { return logB > 10 ? 1u << (logB - 10) : 1u; }

// Loop l's packed bits for the register-table scan: word c of lane j holds
// the bit of every bucket h = j + 32 m (m = c mod E, E = table_words) at
// (sigma^-1 (h >> (log2 B - 5))) mod 32, so that the scan's one rotate puts
// the bit of f + kN/G (G = min(B/32, 32)) at position k 32/G.  bit(h) is
// bucket h's bit: strong for the median estimator, kept for the mean.
template <class Bit>
__device__ __forceinline__ uint32_t packed_word(const PlanDev &P, uint32_t l, uint32_t c, uint32_t j, Bit bit) {
    const uint32_t sh = P.logB - 5, si = inv_mod32(P.sigma[l]), E = table_words(P.logB);
    uint32_t word = 0;
    for (uint32_t m = c; 32 * m < P.B; m += E) {
        const uint32_t h = j + 32 * m;
        word |= (uint32_t)bit(h) << ((si * (h >> sh)) & 31u);
    }
    return word;
}

// Words [w0, w1) of the 2-bit table: word w packs the entries 16 w .. 16 w + 15
// (flag(e) = kept | strong << 8 of table entry e = l B + h) as kept at bit
// 2k and strong at bit 2k + 1.
template <class Flag>
__device__ __forceinline__ void pack_bits2(const PlanDev &P, uint32_t w0, uint32_t w1, Flag flag) {
    for (uint32_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        uint32_t word = 0;
#pragma unroll
        for (uint32_t k = 0; k < 16; ++k) {
            const uint32_t f = flag(16 * w + k);
            word |= ((f & 1u) | (((f >> 8) & 1u) << 1)) << (2 * k);
        }
        P.bits2[w] = word;
    }
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
    if (P.bits2)
        pack_bits2(P, l * (B >> 4), (l + 1) * (B >> 4), [&](uint32_t e) {
            const uint32_t k = e - l * B;
            return kept_s[k] | (strong_energy(__uint_as_float(en_s[k]), gmul, thr) ? 256u : 0u);
        });
    const bool mean = P.estimator == kEstMean;
    const uint32_t E = table_words(P.logB);
    if (P.use_bits)
        for (uint32_t i = threadIdx.x; i < 32 * E; i += blockDim.x)
            P.packed[(l * E + (i >> 5)) * 32 + (i & 31)] = packed_word(P, l, i >> 5, i & 31, [&](uint32_t h) {
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
// dftC (precision 1): the bucket values come from the tensor-core DFT's three
// FP32 partial planes C[3][dft_mpad][B] (complex), row blockIdx.x, summed in
// product order instead of the gather partials and the radix-2 FFT.
__global__ void __launch_bounds__(kThreads, 6) k_fft_select(Launch ln, int select_only, int clustered,
                                                            const float2 *dftC, uint32_t dft_mpad,
                                                            const uint32_t *dft_err) {
    // B values, B energies, B kept bytes (clustered)
    extern __shared__ unsigned long long sm[];
    float2 *buf = reinterpret_cast<float2 *>(sm);
    uint32_t *en_s;
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ int s_last;
    __shared__ float s_theta;
    __shared__ uint32_t s_hist[256], s_wsum[8], s_prefix, s_need;
    enter(ln, P, J, s_local);

    const uint32_t l = s_local, B = P.B, logB = P.logB;
    en_s = reinterpret_cast<uint32_t *>(buf + B);
    // the FFT's values sit at sw(i): the low four bits XOR the top four, so the
    // bit-reversed stores of a half-warp (top bits differing) and the
    // butterflies' runs of consecutive indices both fall in distinct banks
    const uint32_t swsh = logB >= 8 ? logB - 4 : 31u;
    auto sw = [&](uint32_t i) { return swsh < 31u ? i ^ ((i >> swsh) & 15u) : i; };
    float2 *zrow = P.zhat + (size_t)l * B;
    float *erow = P.energy + (size_t)l * B;
    uint16_t *frow = P.flags + (size_t)l * B;
    if (!select_only && dftC) {
        const size_t plane = (size_t)dft_mpad * B;
        const float2 *c0 = dftC + (size_t)blockIdx.x * B;
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 a = __ldcg(c0 + k), b = __ldcg(c0 + plane + k), c = __ldcg(c0 + 2 * plane + k);
            const float2 z = make_float2((a.x + b.x) + c.x, (a.y + b.y) + c.y);
            const float e = z.x * z.x + z.y * z.y;
            zrow[k] = z;
            erow[k] = e;
            en_s[k] = __float_as_uint(e);
        }
        if (threadIdx.x == 0 && *dft_err) P.ctr[kErr] = *dft_err;  // a tensor-core wait gave up
    } else if (!select_only) {
        const uint32_t nchunk = J.nchunk;
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
            buf[sw(__brev(j) >> (32 - logB))] = acc;
        }
        __syncthreads();
        // iterative radix-2 decimation in time, twiddles exp(-2 pi i k / (2h))
        // read by stage from the table whose stage h holds them at h - 1 + k
        // (consecutive butterflies, consecutive entries)
        const float2 *__restrict__ twst = P.twst;
        for (uint32_t hs = 0; hs < logB; ++hs) {
            const uint32_t h = 1u << hs;
            for (uint32_t bf = threadIdx.x; bf < B / 2; bf += blockDim.x) {
                const uint32_t k = bf & (h - 1);
                const uint32_t i0 = ((bf >> hs) << (hs + 1)) + k;
                const uint32_t i1 = i0 + h;
                const float2 w = __ldg(twst + (h - 1) + k);
                const float2 a = buf[sw(i0)];
                const float2 t = cmul(w, buf[sw(i1)]);
                buf[sw(i0)] = make_float2(a.x + t.x, a.y + t.y);
                buf[sw(i1)] = make_float2(a.x - t.x, a.y - t.y);
            }
            __syncthreads();
        }
        for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
            const float2 z = buf[sw(k)];
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
        uint8_t *kept_s = reinterpret_cast<uint8_t *>(en_s + B);  // clustered only
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
    if (P.bits2) {
        __syncthreads();  // the flags above are complete
        pack_bits2(P, 0, P.L * (B >> 4), [&](uint32_t e) { return __ldcg(reinterpret_cast<const unsigned short *>(P.flags) + e); });
    }
    if (P.use_bits) {
        __syncthreads();  // the flags above are complete
        const bool mean = P.estimator == kEstMean;
        const uint32_t E = table_words(P.logB);
        for (uint32_t idx = threadIdx.x; idx < P.L * E * 32; idx += blockDim.x) {
            const uint32_t ll = idx / (32 * E), c = (idx >> 5) % E;
            const float *er = P.energy + (size_t)ll * B;
            const unsigned short *fr = reinterpret_cast<const unsigned short *>(P.flags) + (size_t)ll * B;
            P.packed[idx] = packed_word(P, ll, c, idx & 31, [&](uint32_t h) {
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

// Tables: the plan's in global memory (SM 0), the gains' copy in shared
// memory (SM 1: gt, 1/G~ [N/B]) or copies of all three (SM 2: zt, zhat
// [L][B]; gt; kt, kept bits [L][B/32]).
template <int LT, int SM>
__device__ __forceinline__ void estimate_pruned(const PlanDev &P, uint32_t f, float theta, float a,
                                                uint32_t *cnt, const float2 *zt, const float2 *gt,
                                                const uint32_t *kt) {
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB;
    const uint32_t cv = P.half << sN;
    const uint32_t osh = P.logB + sN;  // offset in the bucket: the word's bits below the bucket bits
    const uint32_t B = P.B;
    // loop l's bucket value and gain (one hash word feeds both loads) and its turn
    auto fetch = [&](int l, float2 &z, float2 &g, uint32_t &ph) {
        const uint32_t t = (P.sigma[l] << sN) * f + cv;
        const uint32_t h = t >> top;
        const uint32_t opos = osh < 32 ? (t << P.logB) >> osh : 0u;
        if constexpr (SM == 2) {
            const uint32_t zb = (uint32_t)__cvta_generic_to_shared(zt);
            const uint32_t gb = (uint32_t)__cvta_generic_to_shared(gt);
            z = lds_f2(zb + 8 * (l * B + h));
            g = lds_f2(gb + 8 * opos);
        } else if constexpr (SM == 1) {
            z = __ldg(P.zhat + l * B + h);
            g = lds_f2((uint32_t)__cvta_generic_to_shared(gt) + 8 * opos);
        } else {
            z = __ldg(P.zhat + l * B + h);
            g = __ldg(P.ginv + opos);
        }
        ph = (P.tau[l] << sN) * f;
    };
    // pass 1, in batches of GB loops (a batch's loads issued together): the
    // reject's counts and, for the mean, the sums in loop order.  Tables in
    // shared memory: one batch of all L (their CTAs are limited by shared
    // memory, not registers); tables in L2: batches of four, so that four
    // CTAs per SM fit 64 registers and hide the L2 latency
    constexpr int GB = SM == 2 ? LT : (LT % 4 == 0 ? 4 : 1);
    // (shared-memory tables also keep the L values for the medians; tables in
    // L2 fetch them again in pass 2, for the few that pass)
    constexpr bool KEEP = SM == 2;
    bool keep = true;
    const bool mean = P.estimator == kEstMean;
    float sr = 0.f, si = 0.f;
    float re[LT], im[LT];
    {
        uint32_t rp = 0, rn = 0, ip = 0, in = 0;
#pragma unroll
        for (int l0 = 0; l0 < LT; l0 += GB) {
            float2 z[GB], g[GB];
            uint32_t ph[GB];
#pragma unroll
            for (int k = 0; k < GB; ++k) fetch(l0 + k, z[k], g[k], ph[k]);
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const float2 v = turn_scale(z[k], g[k], ph[k]);
                if constexpr (KEEP) {
                    re[l0 + k] = v.x;
                    im[l0 + k] = v.y;
                }
                rp += v.x >= a;
                rn += v.x <= -a;
                ip += v.y >= a;
                in += v.y <= -a;
                if (mean) {
                    sr += v.x;
                    si += v.y;
                }
            }
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
            if constexpr (SM == 2)
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
            v = make_float2(sr / (float)LT, si / (float)LT);
        } else {
            if constexpr (!KEEP) {
                // pass 2 (the few that passed): the L values again, for the medians
#pragma unroll
                for (int l = 0; l < LT; ++l) {
                    float2 z, g;
                    uint32_t ph;
                    fetch(l, z, g, ph);
                    const float2 w = turn_scale(z, g, ph);
                    re[l] = w.x;
                    im[l] = w.y;
                }
            }
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
// kTabBits2: the 2-bit table (kept, strong) of tables too large for the u16
// one in shared memory, staged there (L B / 4 bytes).
enum TableKind : int { kTabGlobal = 0, kTabSmem = 1, kTabBits2 = 2 };

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
    const uint32_t *tab2 = reinterpret_cast<const uint32_t *>(tab_s);
    const uint32_t wpl = B >> 4;  // 2-bit table: words per loop
    if constexpr (TAB == kTabBits2) {
        uint32_t *dst = reinterpret_cast<uint32_t *>(tab_s);
        for (uint32_t i = threadIdx.x; i < L * wpl; i += blockDim.x) dst[i] = __ldcg(P.bits2 + i);
        __syncthreads();
    }
    // score | strong << 8 of loop l's bucket h
    auto entry = [&](uint32_t l, uint32_t h) -> uint32_t {
        if constexpr (TAB == kTabBits2) {
            const uint32_t v = (tab2[l * wpl + (h >> 4)] >> ((h & 15u) << 1)) & 3u;
            return (v & 1u) | ((v >> 1) << 8);
        } else {
            return tab[l * B + h];
        }
    };
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
                    for (int l = 0; l < LT; ++l) acc += entry(l, (av[l] * f + cv) >> top);
                } else {
                    for (uint32_t l = 0; l < L; ++l) acc += entry(l, ((P.sigma[l] << (32 - P.logN)) * f + cv) >> top);
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


// Pruned scan with the register table of strong bits (32 <= B <= 4096, L in
// {8, 12, 16}).  Mean plans (T = M) pack kept bits instead, so the survivors
// are exactly the candidates.
//
// A thread takes the G = min(B/32, 32) frequencies f + kN/G.  Their hash
// words differ by k sigma_l 2^32/G, so their buckets h + k sigma_l B/G share
// the lane h mod 32 of the packed table, and for B >= 1024 also the word
// c = (h >> 5) mod E of the lane's E = B/1024 words; E warp shuffles (one per
// word, the thread keeping word c) fetch the word holding all G strong bits.
// A rotate by sigma^-1 (h >> (log2 B - 5)) (the table's positions are scaled
// by sigma^-1 to match) puts member k's bit at position k 32/G in every loop,
// so carry-save adders over the L rotated words count the strong loops of
// all 32 positions at once (bit-sliced counters).  Frequencies with at least
// M = ceil(L/2) strong loops are queued in shared memory (overflow goes
// straight to the job's survivor list) and appended to the list when the CTA
// ends; candidacy is checked when they are estimated.
template <int LT, int E>
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
    uint32_t av[LT], pw[LT][E], sip[NSW];
#pragma unroll
    for (int k = 0; k < NSW; ++k) sip[k] = 0;
#pragma unroll
    for (int l = 0; l < LT; ++l) {
        av[l] = P.sigma[l] << (32 - P.logN);
#pragma unroll
        for (int c = 0; c < E; ++c) pw[l][c] = __ldcg(P.packed + (l * E + c) * 32 + lane);
        sip[l / 6] |= (inv_mod32(P.sigma[l]) & 31u) << (5 * (l % 6));
    }
    const uint32_t cv = P.half << (32 - P.logN);
    const uint32_t top = 32 - P.logB;
    // G = 2^lgG frequencies f + k span per thread, member k's counter at bit k << gsh
    const uint32_t lgG = min(P.logB - 5, 5u);
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
                const uint32_t h = t >> top;
                uint32_t w = __shfl_sync(0xFFFFFFFFu, pw[l][0], h);  // lane = bucket mod 32
                if constexpr (E > 1) {
                    const uint32_t c = (h >> 5) & (E - 1);
#pragma unroll
                    for (int cc = 1; cc < E; ++cc) {
                        const uint32_t v = __shfl_sync(0xFFFFFFFFu, pw[l][cc], h);
                        w = c == (uint32_t)cc ? v : w;
                    }
                }
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
// Fallback share of one job, taken when fewer than K pruned records reached
// theta: every candidate (kept in >= T loops) among the frequencies [f0, f1)
// is counted (kNCand), estimated and recorded (kNRec2).  Each of the job's
// fallback CTAs scans one share, so the pass is exact and parallel; jobs that
// need none launch CTAs that return at once.
template <int LT>
__device__ void fallback_share(const PlanDev &P, uint32_t f0, uint32_t f1, uint32_t *s_cnt) {
    if (threadIdx.x == 0) *s_cnt = 0;
    __syncthreads();
    const uint32_t sN = 32 - P.logN, top = 32 - P.logB, cv = P.half << sN;
    const uint32_t L = LT > 0 ? (uint32_t)LT : P.L;
    uint32_t cand = 0;
    for (uint32_t base = f0; base < f1; base += blockDim.x) {
        const uint32_t f = base + threadIdx.x;
        bool c = false;
        // comb plans: only frequencies of kept residue classes
        const bool eligible = P.method != kMethodComb ||
                              ((__ldg(P.keptc + ((f & (P.Bc - 1)) >> 5)) >> (f & (P.Bc - 1) & 31u)) & 1u);
        if (f < f1 && eligible) {
            uint32_t score = 0;
#pragma unroll
            for (uint32_t l = 0; l < L; ++l)
                score += __ldg(P.flags + (size_t)l * P.B + (((P.sigma[l] << sN) * f + cv) >> top)) & 1u;
            c = score >= P.T;
        }
        cand += c;
        if (c) estimate_record<LT>(P, f, false, 0.f, P.ctr + kNRec2);
    }
    cand = __reduce_add_sync(0xFFFFFFFFu, cand);
    if ((threadIdx.x & 31) == 0 && cand) atomicAdd(s_cnt, cand);
    __syncthreads();
    if (threadIdx.x == 0 && *s_cnt) atomicAdd(P.ctr + kNCand, *s_cnt);
}

// Top-K of one job: the k_out = min(K, candidates) recorded estimates of
// largest magnitude (ties to the lower f), written sorted by f.  Records are
// those of the pruned pass (candidates with key >= theta) when at least K of
// them exist; otherwise those of the fallback pass (every candidate).  Pruned
// candidates have key < theta, so either set contains the top K.
// Run by all threads of the job's last CTA (the other CTAs' records are
// visible: they fenced before taking their ticket).  tk: shared memory for
// cap keys + cap payloads (cap a power of two >= max(kRankMax, K)).
__device__ void rank_records(const PlanDev &P, const Job &J, unsigned long long *tk, uint32_t cap, uint32_t S,
                             uint32_t kout);

// The estimate's last CTA of a job: the top K of the pruned records, or, when
// they cannot certify it, the flag that hands the job to the fallback pass.
// gctr (batch groups): a flagged job also counts itself in gctr[4], which the
// group's fallback CTAs read first.
__device__ void topk_job(const PlanDev &P, const Job &J, unsigned long long *tk, uint32_t cap,
                         uint32_t *gctr = nullptr) {
    __shared__ int s_fb;
    if (threadIdx.x == 0) {
        s_fb = needs_fallback(P);
        P.ctr[kFbPend] = s_fb ? 1u : 0u;
        if (s_fb && gctr) atomicAdd(gctr + 4, 1u);
    }
    __syncthreads();
    if (!s_fb) rank_records(P, J, tk, cap, __ldcg(P.ctr + kNGe), P.K);  // >= K candidates exist
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

// CTAs of a job's estimate launch that take survivors: one per kEstChunk of
// them, at most the job's CTAs (the rest only take their ticket), so few
// survivors are not spread over CTAs that each stage the tables.  (Measured
// on 8-128 headline signals per batch: 512 against 2048 took 8 signals'
// estimate from 31.0 to 21.5 us and left 64 and 128 unchanged; 256 was no
// faster.)
constexpr uint32_t kEstChunk = 512;
// Shared memory of the survivor-estimate kernel with its tables in L2: at
// least this much, where the gains (N/B complex) are staged when they fit.
constexpr uint32_t kSurvGainSmem = 16384;
__device__ __forceinline__ uint32_t est_active(uint32_t n, uint32_t ctas_per_job) {
    const uint32_t a = (n + kEstChunk - 1) / kEstChunk;
    return a < 1 ? 1u : (a > ctas_per_job ? ctas_per_job : a);
}

// Stages the job's gains (N/B complex) in shared memory (all threads).
__device__ __forceinline__ void stage_gains(const PlanDev &P, float2 *gsm) {
    const uint32_t NB = P.N >> P.logB;
    const uint32_t gb = (uint32_t)__cvta_generic_to_shared(gsm);
    for (uint32_t k = threadIdx.x; k < NB / 2; k += kThreads) cp_async16(gb + 16 * k, P.ginv + 2 * k);
    if ((NB & 1u) && threadIdx.x == 0) gsm[NB - 1] = __ldg(P.ginv + NB - 1);
    cp_async_wait_all();
    __syncthreads();
}

// Survivor estimates of a batch group with the survivors of all its jobs
// shared out dynamically: every CTA reads the jobs' survivor counts (the
// scan's), cuts each job's list into chunks of C survivors (C sized so the
// group has about two chunks per CTA, 256..2048) and takes chunks in job
// order from the group's counter gctr[0], loading a job's descriptor (and
// staging its gains) when its chunk is another job's; the CTA that finishes
// a job's last chunk (per-job ticket after a fence) takes that job's top K.
// The group's last CTA to finish resets the counters for the next launch.
// Balances jobs whose survivors differ by orders of magnitude (low SNR,
// dense windows), which fixed per-job shares cannot.
template <int LT>
__device__ void estimate_dynamic(const Launch &ln, PlanDev &P, Job &J, uint32_t cap, uint32_t gain_max,
                                 unsigned long long *smem) {
    __shared__ uint32_t s_pre[kDynMaxJobs + 1];  // chunk prefix over the group's jobs
    __shared__ uint32_t s_wsum[kThreads / 32], s_tot, s_c;
    __shared__ int s_last;
    const uint32_t j0 = __ldg(ln.map + ln.cta0), j1 = __ldg(ln.map + ln.cta0 + gridDim.x - 1) + 1;
    const uint32_t nj = j1 - j0;
    // each thread's jobs: survivor counts (three dependent loads per job, a thread's jobs in flight together)
    constexpr uint32_t kPer = kDynMaxJobs / kThreads;
    uint32_t cnt[kPer];
    uint32_t mysum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
        const uint32_t k = threadIdx.x * kPer + q;
        cnt[q] = 0;
        if (k < nj) {
            const PlanDev *pd = ln.jobs[j0 + k].p;
            const uint32_t *ctr = *reinterpret_cast<uint32_t *const *>(reinterpret_cast<const char *>(pd) +
                                                                       offsetof(PlanDev, ctr));
            cnt[q] = __ldcg(ctr + kNSurv);
        }
        mysum += cnt[q];
    }
    const uint32_t allsurv = block_incl_scan(mysum, s_wsum);
    if (threadIdx.x == kThreads - 1) s_tot = allsurv;
    __syncthreads();
    uint32_t C = s_tot / (2 * gridDim.x);
    C = C < 256 ? 256u : (C > 2048 ? 2048u : C);
    uint32_t mych = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q)
        if (threadIdx.x * kPer + q < nj) mych += cnt[q] > 0 ? (cnt[q] + C - 1) / C : 1u;
    const uint32_t incl = block_incl_scan(mych, s_wsum);
    uint32_t run = incl - mych;
    if (threadIdx.x == 0) s_pre[0] = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
        const uint32_t k = threadIdx.x * kPer + q;
        if (k < nj) {
            run += cnt[q] > 0 ? (cnt[q] + C - 1) / C : 1u;
            s_pre[k + 1] = run;
        }
    }
    if (threadIdx.x == kThreads - 1) s_tot = incl;
    uint32_t nxt = 0;  // thread 0: the next chunk's ticket
    if (threadIdx.x == 0) nxt = atomicAdd(ln.gctr, 1u);
    __syncthreads();
    const uint32_t total = s_tot;
    float2 *gsm = reinterpret_cast<float2 *>(smem);
    uint32_t cur = 0xFFFFFFFFu;
    bool staged = false;
    for (;;) {
        if (threadIdx.x == 0) s_c = nxt;
        __syncthreads();
        const uint32_t c = s_c;
        if (c >= total) break;
        if (threadIdx.x == 0) nxt = atomicAdd(ln.gctr, 1u);  // (in flight while this chunk is estimated)
        // the chunk's job: s_pre[jr] <= c < s_pre[jr + 1]
        uint32_t lo = 0, hi = nj;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pre[mid] <= c) lo = mid;
            else hi = mid;
        }
        const uint32_t jr = lo, nch = s_pre[jr + 1] - s_pre[jr], cj = c - s_pre[jr];
        if (jr != cur) {
            __syncthreads();  // (everyone is done with the previous descriptor)
            if (threadIdx.x == 0) J = ln.jobs[j0 + jr];
            __syncthreads();
            load_plan(P, J.p);
            __syncthreads();
            staged = (P.N >> P.logB) <= gain_max;
            if (staged) stage_gains(P, gsm);
            cur = jr;
        }
        const uint32_t n = __ldcg(P.ctr + kNSurv);
        const float theta = __uint_as_float(__ldcg(P.ctr + kTheta));
        const float a = sqrtf(0.5f * theta) * (1.0f - 1.0f / 1024.0f);
        const uint32_t e1 = min(n, (cj + 1) * C);
        for (uint32_t i = cj * C + threadIdx.x; i < e1; i += kThreads) {
            const uint32_t f = __ldg(P.survf + i);
            if (staged)
                estimate_pruned<LT, 1>(P, f, theta, a, P.ctr + kNGe, nullptr, gsm, nullptr);
            else
                estimate_pruned<LT, 0>(P, f, theta, a, P.ctr + kNGe, nullptr, nullptr, nullptr);
        }
        // the job's chunk ticket; the last chunk's CTA takes the top K
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(P.ctr + kEstDone, 1u) == nch - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            topk_job(P, J, smem, cap, ln.gctr);  // (overwrites the staged gains)
            __syncthreads();
            if (threadIdx.x == 0) P.ctr[kEstDone] = 0;
            cur = 0xFFFFFFFFu;
        }
    }
    if (threadIdx.x == 0 && atomicAdd(ln.gctr + 1, 1u) == gridDim.x - 1) {
        // every CTA has taken its last ticket: re-arm the group for the next launch
        ln.gctr[0] = 0;
        ln.gctr[1] = 0;
        __threadfence();
    }
}

// Pruned-pass median estimates of the job's survivors, ctas_per_job CTAs per
// job: candidates whose key reaches theta are recorded as {f, key bits, re
// bits, im bits}.  The job's last CTA to finish (atomic ticket after a fence)
// then takes the job's top K (a7).  Batch groups with ln.gctr share their
// survivors out dynamically instead (estimate_dynamic).
template <int LT>
__global__ void __launch_bounds__(kThreads, 4) k_estimate_surv(Launch ln, uint32_t cap, uint32_t gain_max) {
    // the job's 1/G~ when N/B <= gain_max (survivor CTAs), then the top-K
    // buffer of the job's last CTA
    extern __shared__ unsigned long long est_topk[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    enter(ln, P, J, s_local);
    if constexpr (LT > 0) {
        if (ln.gctr) {
            estimate_dynamic<LT>(ln, P, J, cap, gain_max, est_topk);
            return;
        }
    }
    const uint32_t ctas_per_job = J.ectas;
    const uint32_t n = P.ctr[kNSurv];
    const float theta = __uint_as_float(P.ctr[kTheta]);
    uint32_t *cnt = P.ctr + kNGe;
    // CTAs past the job's active count take no survivors (their strides would overlap)
    const uint32_t active = est_active(n, ctas_per_job);
    const uint32_t stride = active * kThreads;
    const uint32_t i0 = s_local < active ? s_local * kThreads + threadIdx.x : n;
    if constexpr (LT > 0) {
        const float a = sqrtf(0.5f * theta) * (1.0f - 1.0f / 1024.0f);
        // gains staged in shared memory when they fit (uniform over the CTA)
        const uint32_t NB = P.N >> P.logB;
        float2 *gsm = reinterpret_cast<float2 *>(est_topk);
        const bool staged = NB <= gain_max && s_local < active;
        if (staged) stage_gains(P, gsm);
        // the next survivor's frequency is fetched while this one is estimated
        uint32_t i = i0;
        uint32_t fn = i < n ? __ldg(P.survf + i) : 0u;
        for (; i < n; i += stride) {
            const uint32_t f = fn;
            if (i + stride < n) fn = __ldg(P.survf + i + stride);
            if (staged)
                estimate_pruned<LT, 1>(P, f, theta, a, cnt, nullptr, gsm, nullptr);
            else
                estimate_pruned<LT, 0>(P, f, theta, a, cnt, nullptr, nullptr, nullptr);
        }
    } else {
        for (uint32_t i = i0; i < n; i += stride) estimate_record<LT>(P, P.survf[i], true, theta, cnt);
    }
    if (last_of_job(P, ctas_per_job)) topk_job(P, J, est_topk, cap, ln.gctr);
}

template <int LT>
__device__ void estimate_tab_part(const PlanDev &P, uint32_t s_local, uint32_t active, uint32_t n,
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
    const uint32_t stride = active * kThreads;
    uint32_t i = s_local * kThreads + threadIdx.x;
    uint32_t fn = i < n ? __ldg(P.survf + i) : 0u;
    for (; i < n; i += stride) {
        const uint32_t f = fn;
        if (i + stride < n) fn = __ldg(P.survf + i + stride);
        estimate_pruned<LT, 2>(P, f, theta, a, P.ctr + kNGe, zs, gs, ks);
    }
}

// Pruned-pass estimates with the job's tables staged in shared memory: zhat
// (L B complex), 1/G~ (N/B complex) and the kept flags as bits.  A few CTAs
// per job, each over a strided share of the survivors, so every lookup is a
// shared-memory load.
template <int LT>
__global__ void __launch_bounds__(kThreads) k_estimate_tab(Launch ln, uint32_t cap) {
    extern __shared__ float4 est_tab[];  // the job's tables, then the last CTA's top-K buffer
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    enter(ln, P, J, s_local);
    const uint32_t ctas_per_job = J.ectas;
    const uint32_t n = P.ctr[kNSurv];
    // only the CTAs with a share of at least kEstChunk survivors stage the tables
    const uint32_t active = est_active(n, ctas_per_job);
    if (s_local < active) estimate_tab_part<LT>(P, s_local, active, n, est_tab);
    if (last_of_job(P, ctas_per_job))
        topk_job(P, J, reinterpret_cast<unsigned long long *>(est_tab), cap, ln.gctr);
}


// Frequencies per chunk of the dynamic fallback pass.
constexpr uint32_t kFbChunk = 16384;

// The fallback pass of a batch group with the pending jobs' frequencies
// shared out dynamically over every CTA of the group (most jobs have no
// pending fallback; one that has, at low SNR, may hold most of its N as
// candidates): each CTA reads the jobs' flags and sizes, cuts each pending
// job's frequencies into chunks of kFbChunk and takes chunks in job order
// from the group's counter gctr[2]; the CTA that finishes a job's last chunk
// ranks its records.  Nothing pending: every CTA returns after the flags.
template <int LT>
__device__ void fallback_dynamic(const Launch &ln, PlanDev &P, Job &J, uint32_t cap, unsigned long long *smem) {
    __shared__ uint32_t s_pre[kDynMaxJobs + 1];  // chunk prefix over the group's jobs
    __shared__ uint32_t s_wsum[kThreads / 32], s_tot, s_c, s_cnt;
    __shared__ int s_last, s_any;
    uint32_t *gc = ln.gctr + 2;
    // jobs the estimate flagged (gctr[4]): none, the common case, ends every CTA here
    if (threadIdx.x == 0) s_any = __ldcg(ln.gctr + 4) != 0;
    __syncthreads();
    if (!s_any) return;
    const uint32_t j0 = __ldg(ln.map + ln.cta0), j1 = __ldg(ln.map + ln.cta0 + gridDim.x - 1) + 1;
    const uint32_t nj = j1 - j0;
    constexpr uint32_t kPer = kDynMaxJobs / kThreads;
    uint32_t nch[kPer];
    uint32_t mych = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
        const uint32_t k = threadIdx.x * kPer + q;
        nch[q] = 0;
        if (k < nj) {
            const char *pd = reinterpret_cast<const char *>(ln.jobs[j0 + k].p);
            const uint32_t *ctr = *reinterpret_cast<uint32_t *const *>(pd + offsetof(PlanDev, ctr));
            const uint32_t N = *reinterpret_cast<const uint32_t *>(pd + offsetof(PlanDev, N));
            if (__ldcg(ctr + kFbPend)) nch[q] = (N + kFbChunk - 1) / kFbChunk;
        }
        mych += nch[q];
    }
    const uint32_t incl = block_incl_scan(mych, s_wsum);
    uint32_t run = incl - mych;
    if (threadIdx.x == 0) s_pre[0] = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
        const uint32_t k = threadIdx.x * kPer + q;
        if (k < nj) {
            run += nch[q];
            s_pre[k + 1] = run;
        }
    }
    if (threadIdx.x == kThreads - 1) s_tot = incl;
    __syncthreads();
    const uint32_t total = s_tot;
    if (total == 0) return;  // (uniform: no job of the group is pending)
    uint32_t nxt = 0;  // thread 0: the next chunk's ticket
    if (threadIdx.x == 0) nxt = atomicAdd(gc, 1u);
    uint32_t cur = 0xFFFFFFFFu;
    for (;;) {
        if (threadIdx.x == 0) s_c = nxt;
        __syncthreads();
        const uint32_t c = s_c;
        if (c >= total) break;
        if (threadIdx.x == 0) nxt = atomicAdd(gc, 1u);  // (in flight while this chunk runs)
        // the chunk's job: the last jr with s_pre[jr] <= c (jobs without chunks have s_pre[jr] == s_pre[jr + 1])
        uint32_t lo = 0, hi = nj;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pre[mid] <= c) lo = mid;
            else hi = mid;
        }
        const uint32_t jr = lo, cj = c - s_pre[jr], jn = s_pre[jr + 1] - s_pre[jr];
        if (jr != cur) {
            __syncthreads();
            if (threadIdx.x == 0) J = ln.jobs[j0 + jr];
            __syncthreads();
            load_plan(P, J.p);
            __syncthreads();
            cur = jr;
        }
        const uint32_t f0 = cj * kFbChunk, f1 = min(P.N, f0 + kFbChunk);
        fallback_share<LT>(P, f0, f1, &s_cnt);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(P.ctr + kFbDone, 1u) == jn - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            const uint32_t S = __ldcg(P.ctr + kNRec2), kout = min(P.K, __ldcg(P.ctr + kNCand));
            rank_records(P, J, smem, cap, S, kout);
            __syncthreads();
            if (threadIdx.x == 0) P.ctr[kFbDone] = 0;
        }
    }
    if (threadIdx.x == 0 && atomicAdd(gc + 1, 1u) == gridDim.x - 1) {
        gc[0] = 0;  // every CTA has taken its last ticket: re-arm for the next launch
        gc[1] = 0;
        ln.gctr[4] = 0;
        __threadfence();
    }
}

// Unpruned fallback pass, fallback_ctas(N) CTAs per job: a CTA of a job with
// no pending fallback returns after reading one flag; otherwise it records
// the candidates of its share of the frequencies, and the job's last CTA to
// finish (atomic ticket after a fence) ranks them (top K of every candidate).
// Batch groups with ln.gctr share the pending jobs' chunks dynamically
// instead (fallback_dynamic).
template <int LT>
__global__ void __launch_bounds__(kThreads) k_fallback(Launch ln, uint32_t cap) {
    extern __shared__ unsigned long long fb_topk[];
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local, s_cnt;
    __shared__ int s_go, s_last;
    grid_dep_wait();  // (the flag and records come from the estimate kernel)
    if (ln.gctr) {
        fallback_dynamic<LT>(ln, P, J, cap, fb_topk);
        return;
    }
    if (threadIdx.x == 0) {
        Job j;
        uint32_t loc;
        locate(ln, ln.cta0 + blockIdx.x, j, loc);
        J = j;
        s_local = loc;
        // the descriptor's counter pointer, then the job's flag (one load each)
        const uint32_t *ctr = *reinterpret_cast<uint32_t *const *>(reinterpret_cast<const char *>(j.p) +
                                                                   offsetof(PlanDev, ctr));
        s_go = __ldcg(ctr + kFbPend) != 0;
    }
    __syncthreads();
    if (!s_go) return;
    load_plan(P, J.p);
    __syncthreads();
    const uint32_t n = fallback_ctas(P.N);
    const uint32_t per = ((P.N + n - 1) / n + kThreads - 1) / kThreads * kThreads;
    const uint32_t f0 = min(P.N, s_local * per), f1 = min(P.N, f0 + per);
    fallback_share<LT>(P, f0, f1, &s_cnt);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last = atomicAdd(P.ctr + kFbDone, 1u) == n - 1;
        if (s_last) atomicExch(P.ctr + kFbDone, 0u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t S = __ldcg(P.ctr + kNRec2), kout = min(P.K, __ldcg(P.ctr + kNCand));
    rank_records(P, J, fb_topk, cap, S, kout);
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

template <int LT, int TAB>
cudaError_t scan_variant(const Launch &ln, uint32_t ctas, int mode, uint32_t smem, int32_t *cand_out,
                         int32_t *ncand_out, cudaStream_t s) {
    auto kern = k_vote_scan<LT, TAB>;
    if (TAB != kTabGlobal) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(kern, ctas, kThreads, TAB != kTabGlobal ? smem : 0, s, 0, ln, mode, cand_out, ncand_out);
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
                              uint32_t cluster_L, cudaStream_t s, const float *dftC, uint32_t dft_mpad,
                              const uint32_t *dft_err) {
    if (total_ctas == 0) return cudaSuccess;
    const int smem = (int)(max_B * (sizeof(float2) + sizeof(uint32_t)) + (cluster_L ? max_B : 0));
    cudaError_t e = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (!cluster_L)
        return launch_pdl(k_fft_select, total_ctas, kThreads, smem, s, 0, ln, select_only, 0,
                          reinterpret_cast<const float2 *>(dftC), dft_mpad, dft_err);
    if (cluster_L > 8) {
        e = cudaFuncSetAttribute(k_fft_select, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k_fft_select, total_ctas, kThreads, (size_t)smem, s, cluster_L, ln, select_only, 1,
                      reinterpret_cast<const float2 *>(dftC), dft_mpad, dft_err);
}

bool fft_select_cluster_ok(uint32_t L, uint32_t max_B) {
    if (L < 2 || L > 16 || max_B > (uint32_t)kClusterMaxB) return false;
    static std::mutex mu;
    static int known[17][4] = {};  // [L][B class: <= 1024, 4096, 8192, 16384]: 0 unknown, 1 yes, 2 no
    const int bb = max_B <= 1024 ? 0 : max_B <= 4096 ? 1 : max_B <= 8192 ? 2 : 3;
    std::lock_guard<std::mutex> lk(mu);
    if (!known[L][bb]) {
        const uint32_t qB = bb == 0 ? 1024u : bb == 1 ? 4096u : bb == 2 ? 8192u : 16384u;
        const int smem = (int)(qB * (sizeof(float2) + sizeof(uint32_t)) + qB);
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
                        uint32_t max_flags_bytes, uint32_t max_B, int32_t *cand_out, int32_t *ncand_out,
                        cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    if (mode == kVotePrune && scan_uses_bits(L_uniform, bits)) {
        // words per lane and loop of the largest B (every job's B in the group is the same class)
        const uint32_t E = table_words(31 - __builtin_clz(max_B));
        cudaError_t e = cudaSuccess;
        switch (L_uniform * 8 + E) {
            case 8 * 8 + 1: e = launch_pdl(k_scan_bits<8, 1>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 8 * 8 + 2: e = launch_pdl(k_scan_bits<8, 2>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 8 * 8 + 4: e = launch_pdl(k_scan_bits<8, 4>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 12 * 8 + 1: e = launch_pdl(k_scan_bits<12, 1>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 12 * 8 + 2: e = launch_pdl(k_scan_bits<12, 2>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 12 * 8 + 4: e = launch_pdl(k_scan_bits<12, 4>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 16 * 8 + 1: e = launch_pdl(k_scan_bits<16, 1>, total_ctas, kThreads, 0, s, 0, ln); break;
            case 16 * 8 + 2: e = launch_pdl(k_scan_bits<16, 2>, total_ctas, kThreads, 0, s, 0, ln); break;
            default: e = launch_pdl(k_scan_bits<16, 4>, total_ctas, kThreads, 0, s, 0, ln); break;
        }
        return e;
    }
    if (max_flags_bytes <= (uint32_t)kFlagsSmemBytes)
        return scan_dispatch_l<kTabSmem>(ln, total_ctas, mode, L_uniform, max_flags_bytes, cand_out, ncand_out, s);
    // the pruned pass stages the 2-bit table (L B / 4 bytes, an eighth of the u16 one)
    if (mode == kVotePrune)
        return scan_dispatch_l<kTabBits2>(ln, total_ctas, mode, L_uniform, max_flags_bytes / 8, cand_out, ncand_out,
                                          s);
    return scan_dispatch_l<kTabGlobal>(ln, total_ctas, mode, L_uniform, 0, cand_out, ncand_out, s);
}

cudaError_t launch_estimate(const Launch &ln, uint32_t total_ctas, uint32_t L_uniform, uint32_t tab_smem,
                            uint32_t max_K, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    const uint32_t ctas = total_ctas;
    uint32_t cap = kRankMax;
    while (cap < max_K) cap <<= 1;  // the top-K buffer holds the K winners (and up to kRankMax records)
    const uint32_t topk_smem = cap * (uint32_t)(sizeof(unsigned long long) + sizeof(uint32_t));
    if (tab_smem && (L_uniform == 8 || L_uniform == 12 || L_uniform == 16)) {
        auto kern = L_uniform == 8 ? k_estimate_tab<8> : (L_uniform == 12 ? k_estimate_tab<12> : k_estimate_tab<16>);
        const uint32_t smem = max(tab_smem, topk_smem);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return launch_pdl(kern, ctas, kThreads, smem, s, 0, ln, cap);
    }
    auto kern = L_uniform == 8    ? k_estimate_surv<8>
                : L_uniform == 12 ? k_estimate_surv<12>
                : L_uniform == 16 ? k_estimate_surv<16>
                                  : k_estimate_surv<0>;
    // at least kSurvGainSmem, so the gains of N/B <= 2048 are staged (eight
    // CTAs per SM stay resident)
    const uint32_t smem = max(topk_smem, kSurvGainSmem);
    uint32_t gain_max = 1;
    while (2 * gain_max * (uint32_t)sizeof(float2) <= smem) gain_max <<= 1;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, ctas, kThreads, smem, s, 0, ln, cap, gain_max);
}


cudaError_t launch_fallback(const Launch &ln, uint32_t total_ctas, uint32_t L_uniform, uint32_t max_K,
                            cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    uint32_t cap = kRankMax;
    while (cap < max_K) cap <<= 1;
    const uint32_t smem = cap * (uint32_t)(sizeof(unsigned long long) + sizeof(uint32_t));
    auto kern = L_uniform == 8    ? k_fallback<8>
                : L_uniform == 12 ? k_fallback<12>
                : L_uniform == 16 ? k_fallback<16>
                                  : k_fallback<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, total_ctas, kThreads, smem, s, 0, ln, cap);
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
