// Stream gather: step a1 (permuted gather, window, fold) with the signal read
// once, in order, instead of sample by sample at the permuted positions.
//
// The loops' reads are the samples p whose window tap q(p) = (sigma_l^-1
// (p - tau_l) + w/2) mod N is below w (walk.cuh).  The signal is cut into
// segments; per loop, one walker thread visits the reads of one segment in
// sample order, from the segment's first read (a per-plan table) by the
// three-gap return map, so no sample is tested.  A CTA owns V segments of
// each of its loops: it streams their samples into shared memory (cp.async,
// a ring of stages of one piece per segment), its walkers add
// taps[q] x[p] into the loops' B bins in shared memory (atomics), and the
// eight CTAs of a thread-block cluster, which cover adjacent segments, sum
// their bins through distributed shared memory into one partial per cluster
// ([chunk][L][B], as the permuted gather's).  Plans with L B > 6144 take the
// loops in groups (the bins of a group fit 48 KB); each group reads the
// signal again, mostly from L2 (the groups' clusters of one range of samples
// run next to each other).
//
// Bucket sums equal the permuted gather's up to the order of the FP32
// additions, which here depends on the run (shared-memory atomics).
#include <cooperative_groups.h>

#include "device_common.cuh"
#include "sfft_internal.cuh"
#include "walk.cuh"

namespace sfft {

namespace {

// k_walk_start: for every (loop, segment) the tap of the segment's first read;
// the first L threads also write the loops' return maps.
struct WalkArgs {
    uint32_t N, w, halfw, L, nseg, seglog;
    uint32_t sinv[kMaxL], tau[kMaxL];
    uint4 *walk;
    uint32_t *wq;
};

__global__ void __launch_bounds__(kThreads) k_walk_start(WalkArgs a) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.L) {
        const WindowWalk wk = window_walk(a.N, a.sinv[t], a.w);
        a.walk[t] = make_uint4(wk.kp, wk.alpha, wk.km, wk.beta);
    }
    if (t >= a.L * a.nseg) return;
    const uint32_t l = t / a.nseg, seg = t % a.nseg;
    uint32_t k, q;
    window_first_read(a.N, a.sinv[l], a.tau[l], a.w, a.halfw, seg << a.seglog, &k, &q);
    a.wq[t] = q;
}

__device__ __forceinline__ void cp_async16_s(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8_s(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Reads a walker handles per round: their tap and sample loads are all
// issued before the first of their additions.
constexpr int kWalkBatch = 4;

__global__ void __launch_bounds__(kThreads, 2) k_gather_stream(Launch ln) {
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    extern __shared__ __align__(16) float2 sdyn[];
    enter(ln, P, J, s_local);
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();

    // local CTA = ((cluster * groups) + group) * 8 + rank: the groups of one
    // range of segments are adjacent clusters
    const uint32_t rank = s_local % kStreamCluster;
    const uint32_t grp = (s_local / kStreamCluster) % P.sgrp;
    const uint32_t clu = s_local / kStreamCluster / P.sgrp;
    const uint32_t B = P.B, lg = P.slg, l0 = grp * lg, nl = min(lg, P.L - l0);
    const uint32_t V = P.sV, piece = P.spiece, seglog = P.sseg;
    const uint32_t nseg = P.N >> seglog, nstage = (1u << seglog) / piece;
    const uint32_t seg0 = (clu * kStreamCluster + rank) * V;  // this CTA's first segment
    const uint32_t nb = nl * B;
    float2 *bins = sdyn;              // [nl][B]
    float2 *stg = sdyn + (size_t)lg * B;  // [kStreamStages][V][piece]
    for (uint32_t i = threadIdx.x; i < nb; i += kThreads) bins[i] = make_float2(0.f, 0.f);

    // walker t: loop l0 + t / V, segment seg0 + t % V; rel = its next read's
    // distance from the segment start (>= the segment length: none left)
    const uint32_t t = threadIdx.x;
    const bool walker = t < nl * V;
    const uint32_t wl = l0 + (walker ? t / V : 0u), wv = t % V;
    WindowWalk wk = {0u, 0u, 0u, 0u};
    uint32_t q = 0, rel = 0xFFFFFFFFu;
    if (walker) {
        const uint4 m = __ldg(P.walk + wl);
        wk.kp = m.x;
        wk.alpha = m.y;
        wk.km = m.z;
        wk.beta = m.w;
        q = __ldg(P.wq + (size_t)wl * nseg + seg0 + wv);
        const uint32_t p = (P.sigma[wl] * (q - P.halfw) + P.tau[wl]) & P.mask;
        rel = (p - ((seg0 + wv) << seglog)) & P.mask;
    }
    const uint32_t kpm = wk.kp + wk.km, amb = wk.alpha - wk.beta;  // (unsigned wrap: q + amb >= 0)
    float2 *mybins = bins + (size_t)(wl - l0) * B;
    const float *__restrict__ taps = P.taps;
    const uint32_t w = P.w, halfw = P.halfw, bmask = B - 1;

    // stage st: samples [st piece, (st + 1) piece) of each of the V segments,
    // copied in units of 16 bytes (8 when the signal is only 8-byte aligned);
    // this thread's units u = t + 256 i keep their offsets from stage to stage
    const float2 *x = J.x;
    const bool a16 = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    const uint32_t ub = a16 ? 2u : 1u, per = piece / ub, nunit = V * per;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stg), bufbytes = 8u * V * piece;
    constexpr int kMaxUnits = kStreamStageSamples / kThreads;  // (8-byte units)
    size_t soff[kMaxUnits];
    uint32_t doff[kMaxUnits];
#pragma unroll
    for (int i = 0; i < kMaxUnits; ++i) {
        const uint32_t u = threadIdx.x + kThreads * i, v = u / per, o = (u % per) * ub;
        soff[i] = ((size_t)(seg0 + v) << seglog) + o;
        doff[i] = 8u * (v * piece + o);
    }
    auto issue = [&](uint32_t st) {
        if (st < nstage) {
            const float2 *xs = x + (size_t)st * piece;
            const uint32_t d0 = sbase + (st % kStreamStages) * bufbytes;
#pragma unroll
            for (int i = 0; i < kMaxUnits; ++i) {
                if (threadIdx.x + kThreads * i >= nunit) break;
                if (a16) cp_async16_s(d0 + doff[i], xs + soff[i]);
                else cp_async8_s(d0 + doff[i], xs + soff[i]);
            }
        }
        cp_async_commit();  // (an empty group past the last stage keeps the counting uniform)
    };
#pragma unroll
    for (uint32_t st = 0; st < kStreamStages - 1; ++st) issue(st);

    for (uint32_t st = 0; st < nstage; ++st) {
        cp_async_wait_group<kStreamStages - 2>();  // this thread's copies of stage st landed
        __syncthreads();                           // everyone's, and stage st - 1's buffer is free
        issue(st + kStreamStages - 1);
        if (!walker) continue;
        const uint32_t base = st * piece, end = base + piece;
        const float2 *buf = stg + ((size_t)(st % kStreamStages) * V + wv) * piece;
        while (rel < end) {
            uint32_t qk[kWalkBatch], rk[kWalkBatch];
#pragma unroll
            for (int k = 0; k < kWalkBatch; ++k) {
                qk[k] = q;
                rk[k] = rel;
                if (rel < end) {
                    // the return map (walk.cuh), with k+ + k- and alpha - beta precomputed
                    const bool up = q + wk.alpha < w, down = q >= wk.beta;
                    rel += up ? wk.kp : (down ? wk.km : kpm);
                    q = up ? q + wk.alpha : (down ? q - wk.beta : q + amb);
                }
            }
            float gk[kWalkBatch];
            float2 vk[kWalkBatch];
#pragma unroll
            for (int k = 0; k < kWalkBatch; ++k) {
                const bool ok = rk[k] < end;
                gk[k] = ok ? __ldg(taps + qk[k]) : 0.f;
                vk[k] = ok ? buf[rk[k] - base] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kWalkBatch; ++k)
                if (rk[k] < end) {
                    float2 *b = mybins + ((qk[k] - halfw) & bmask);
                    atomicAdd(&b->x, gk[k] * vk[k].x);
                    atomicAdd(&b->y, gk[k] * vk[k].y);
                }
        }
    }
    cp_async_wait_group<0>();
    // the cluster's bins, summed in rank order: CTA r writes the r-th eighth
    cl.sync();
    const uint32_t share = (nb + kStreamCluster - 1) / kStreamCluster;
    const uint32_t i0 = rank * share, i1 = min(nb, i0 + share);
    float2 *dst = P.partial + ((size_t)clu * P.L + l0) * B;
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (uint32_t r = 0; r < kStreamCluster; ++r) {
            const float2 *rb = cl.map_shared_rank(bins, r);
            const float2 v = rb[i];
            acc.x += v.x;
            acc.y += v.y;
        }
        dst[i] = acc;
    }
    cl.sync();  // (no CTA leaves while its peers read its bins)
}

}  // namespace

cudaError_t launch_walk_start(const PlanDev &P, const uint32_t *sinv, cudaStream_t s) {
    if (!P.gmode) return cudaSuccess;
    WalkArgs a;
    a.N = P.N;
    a.w = P.w;
    a.halfw = P.halfw;
    a.L = P.L;
    a.seglog = P.sseg;
    a.nseg = P.N >> P.sseg;
    for (uint32_t l = 0; l < kMaxL; ++l) {
        a.sinv[l] = l < P.L ? sinv[l] : 0u;
        a.tau[l] = l < P.L ? P.tau[l] : 0u;
    }
    a.walk = const_cast<uint4 *>(P.walk);
    a.wq = P.wq;
    const uint32_t n = P.L * a.nseg;
    k_walk_start<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

uint32_t stream_smem_bytes(uint32_t lg, uint32_t B, uint32_t V, uint32_t piece) {
    return (uint32_t)(sizeof(float2) * ((size_t)lg * B + (size_t)kStreamStages * V * piece));
}

cudaError_t launch_gather_stream(const Launch &ln, uint32_t total_ctas, uint32_t smem, cudaStream_t s) {
    if (total_ctas == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_gather_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total_ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kStreamCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gather_stream, ln);
}

}  // namespace sfft
