// Final residual-energy check in FP64 (problem statement, Eq. 5: the error
// left after recovery, seen through the buckets).
//
// After the output (and any refinement), every recovered coefficient f with
// value v is subtracted from loop l's bucket values by the bucket identity
//     zhat_l[k] = sum_f xhat_f exp(+2 pi i tau_l f / N) G~(sigma_l f - k N/B)
// (from its own bucket and both neighbours: further out the flat window's
// gain is below 1e-7 of its passband), and the energy left is summed.  One
// CTA per (job, loop); the loop's B residuals sit in shared memory as FP64
// and receive the subtractions by FP64 shared-memory atomics.  Each CTA
// writes its loop's (energy left, bucket energy) pair; the host sums the L
// pairs in loop order.
#include "device_common.cuh"
#include "sfft_internal.cuh"

namespace sfft {

namespace {

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Sum over the block of two doubles (all threads call; result in thread 0).
__device__ __forceinline__ double2 block_sum2(double a, double b, double2 *ws) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = make_double2(a, b);
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (uint32_t i = 0; i < blockDim.x / 32; ++i) {
            t.x += ws[i].x;
            t.y += ws[i].y;
        }
    return t;
}

__global__ void __launch_bounds__(kThreads) k_residual(Launch ln) {
    extern __shared__ double2 rbuf[];  // [B] residual of this loop's buckets
    __shared__ PlanDev P;
    __shared__ Job J;
    __shared__ uint32_t s_local;
    __shared__ double2 s_ws[kThreads / 32];
    enter(ln, P, J, s_local);
    if (!P.residual) return;
    const uint32_t l = s_local, B = P.B;
    const float2 *zrow = P.zhat + (size_t)l * B;
    double et = 0.0;
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) {
        const float2 z = zrow[k];
        const double zr = z.x, zi = z.y;
        rbuf[k] = make_double2(zr, zi);
        et += zr * zr + zi * zi;
    }
    __syncthreads();
    const uint32_t n = (uint32_t)*J.kout;
    const uint32_t NB = P.N >> P.logB, sigma = P.sigma[l], tau = P.tau[l];
    for (uint32_t c = threadIdx.x; c < n; c += blockDim.x) {
        const uint32_t f = (uint32_t)J.idx[c];
        const float2 vf = J.val[c];
        // bucket and offset from the bucket centre (round half up), as a4
        const uint32_t p = (sigma * f) & P.mask;
        const uint32_t hh = (p + P.half) >> P.shift;
        const int32_t o = (int32_t)(p + P.half - (hh << P.shift)) - (int32_t)P.half;  // [-N/2B, N/2B)
        // exp(+2 pi i tau f / N) from the exact turn (tau f) mod N
        const uint32_t t = (tau * f) & P.mask;
        double sn, cs;
        sincospi(2.0 * (double)t / (double)P.N, &sn, &cs);
        const double2 vt = cmul64(make_double2((double)vf.x, (double)vf.y), make_double2(cs, sn));
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            // G~(sigma f - (hh + d) N/B) = G~(o - d N/B), stored at nu + 3N/2B
            const int32_t nu = o - d * (int32_t)NB;
            const double2 g = P.gext64[(uint32_t)(nu + (int32_t)(3 * NB / 2))];
            const double2 ct = cmul64(vt, g);
            const uint32_t k = (hh + (uint32_t)d) & (B - 1);
            atomicAdd(&rbuf[k].x, -ct.x);
            atomicAdd(&rbuf[k].y, -ct.y);
        }
    }
    __syncthreads();
    double er = 0.0;
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) er += rbuf[k].x * rbuf[k].x + rbuf[k].y * rbuf[k].y;
    const double2 tot = block_sum2(er, et, s_ws);
    if (threadIdx.x == 0) {
        P.resid[2 * l] = tot.x;
        P.resid[2 * l + 1] = tot.y;
    }
}

}  // namespace

cudaError_t launch_residual(const Launch &ln, uint32_t total_ctas, uint32_t max_B, cudaStream_t s) {
    if (total_ctas == 0 || max_B == 0) return cudaSuccess;
    const int smem = (int)(sizeof(double2) * max_B);
    cudaError_t e = cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_residual, total_ctas, kThreads, smem, s, 0, ln);
}

}  // namespace sfft
