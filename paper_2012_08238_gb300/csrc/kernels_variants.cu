// Kernels of the method variants: the spike-train pre-filter (sFFT2.0-style),
// the iterative-framework methods (phase encoding, sFFT3.0-style; binary or
// multi-scale search, sFFT4.0 / MPFFT-style) and the iterative-framework
// refinement of the voting output, with their launchers.
#include <algorithm>

#include "device_common.cuh"
#include "sfft_internal.cuh"

namespace sfft {

namespace {

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

}  // namespace

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
    return launch_pdl(kern, njobs, kRefineThreads, smem, s, 0, ln);
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

}  // namespace sfft
