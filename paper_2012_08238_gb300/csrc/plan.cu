// Plan-time kernels: flat-window taps, window gain tables and FFT twiddles in
// FP64 (step a0').
#include <math_constants.h>

#include <algorithm>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

// Eq. 12 (sinc of width B with centre value 1/B) times Eq. 13 (Gaussian of
// width sigma_g = B sqrt(log2 N)), window position m = q - w/2.
__device__ double flat_tap(int64_t m, uint32_t B, double sg) {
    const double sinc = (m == 0) ? 1.0 / (double)B : sinpi((double)m / (double)B) / (CUDART_PI * (double)m);
    const double t = (double)m / sg;
    return sinc * exp(-0.5 * t * t);
}

__global__ void k_taps(uint32_t N, uint32_t B, uint32_t w, double sg, double *g64, float *g32) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < w; q += gridDim.x * blockDim.x) {
        const double g = flat_tap((int64_t)q - (int64_t)(w / 2), B, sg);
        g64[q] = g;
        g32[q] = (float)g;
    }
}

// G~(o) = sum_m g(m) exp(+2 pi i m o / N), one CTA per offset o in
// [-N/2B, N/2B); stores 1/G~(o) (FP32) and |1/G~(o)|^2 (FP64).
__global__ void k_gain(uint32_t N, uint32_t B, uint32_t w, const double *g64, float2 *ginv, double *ginv2) {
    __shared__ double sre[256], sim[256];
    const uint32_t NB = N / B, half = NB / 2;
    const int64_t o = (int64_t)blockIdx.x - (int64_t)half;
    double re = 0.0, im = 0.0;
    for (uint32_t q = threadIdx.x; q < w; q += blockDim.x) {
        const int64_t m = (int64_t)q - (int64_t)(w / 2);
        int64_t r = (m * o) % (int64_t)N;
        if (r < 0) r += N;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)N, &sn, &cs);
        re += g64[q] * cs;
        im += g64[q] * sn;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (uint32_t s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sre[threadIdx.x] += sre[threadIdx.x + s];
            sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double gr = sre[0], gi = sim[0], n2 = gr * gr + gi * gi;
        ginv[blockIdx.x] = make_float2((float)(gr / n2), (float)(-gi / n2));
        ginv2[blockIdx.x] = 1.0 / n2;
    }
}

// G~(nu) itself for nu in [-3N/2B, 3N/2B): the gains of a coefficient in its
// own bucket and both neighbours, used by the phase-encoding and refinement
// subtractions (FP32, gext) and the residual check (FP64, gext64; either may
// be NULL).  One CTA per offset.
__global__ void k_gain_ext(uint32_t N, uint32_t B, uint32_t w, const double *g64, float2 *gext, double2 *gext64) {
    __shared__ double sre[256], sim[256];
    const uint32_t NB = N / B;
    const int64_t o = (int64_t)blockIdx.x - (int64_t)(3 * NB / 2);
    double re = 0.0, im = 0.0;
    for (uint32_t q = threadIdx.x; q < w; q += blockDim.x) {
        const int64_t m = (int64_t)q - (int64_t)(w / 2);
        int64_t r = (m * o) % (int64_t)N;
        if (r < 0) r += N;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)N, &sn, &cs);
        re += g64[q] * cs;
        im += g64[q] * sn;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (uint32_t s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sre[threadIdx.x] += sre[threadIdx.x + s];
            sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (gext) gext[blockIdx.x] = make_float2((float)sre[0], (float)sim[0]);
        if (gext64) gext64[blockIdx.x] = make_double2(sre[0], sim[0]);
    }
}

__global__ void k_twiddle(uint32_t B, float2 *tw) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < B / 2; k += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)B, &sn, &cs);
        tw[k] = make_float2((float)cs, (float)sn);
    }
}

// The same twiddles by FFT stage: entry h - 1 + k (h = 1, 2, ..., B/2, k < h)
// is exp(-2 pi i k / (2h)) = exp(-2 pi i (k B / 2h) / B), bit-identical to
// k_twiddle's entry k B / 2h (the FP64 arguments are equal); a stage's
// butterflies read consecutive entries.
__global__ void k_twiddle_stages(uint32_t B, float2 *twst) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i + 1 < B; i += gridDim.x * blockDim.x) {
        const uint32_t h = 1u << (31 - __clz(i + 1)), k = i + 1 - h;
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)(2 * h), &sn, &cs);
        twst[i] = make_float2((float)cs, (float)sn);
    }
}

// max of non-negative doubles through their (monotone) bit patterns
__global__ void k_max_bits(const double *v, uint32_t n, unsigned long long *out) {
    unsigned long long m = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = v[i];
        const unsigned long long b = (d >= 0.0) ? (unsigned long long)__double_as_longlong(d) : 0ull;
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xFFFFFFFFu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

cudaError_t plan_max_bits(const double *v, uint32_t n, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_max_bits<<<std::min<uint32_t>((n + 255) / 256, 4096), 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t plan_tables(uint32_t N, uint32_t B, uint32_t w, float *taps, float2 *tw, float2 *twst, float2 *ginv,
                        double *ginv2, float2 *gext, double2 *gext64, cudaStream_t s) {
    double *g64 = nullptr;
    cudaError_t e = cudaMallocAsync(&g64, sizeof(double) * w, s);
    if (e != cudaSuccess) return e;
    const uint32_t logN = 31 - __builtin_clz(N);
    const double sg = (double)B * sqrt((double)logN);
    k_taps<<<(w + 255) / 256, 256, 0, s>>>(N, B, w, sg, g64, taps);
    k_gain<<<N / B, 256, 0, s>>>(N, B, w, g64, ginv, ginv2);
    if (gext || gext64) k_gain_ext<<<3 * (N / B), 256, 0, s>>>(N, B, w, g64, gext, gext64);
    k_twiddle<<<(B / 2 + 255) / 256, 256, 0, s>>>(B, tw);
    if (B > 1) k_twiddle_stages<<<(B + 255) / 256, 256, 0, s>>>(B, twst);
    e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(g64, s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t plan_twiddles(uint32_t n, float2 *tw, cudaStream_t s) {
    k_twiddle<<<(n / 2 + 255) / 256, 256, 0, s>>>(n, tw);
    return cudaGetLastError();
}

}  // namespace sfft
