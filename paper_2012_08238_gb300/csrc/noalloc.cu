// Bucketization (steps a1 + a2) without any allocation: the gather partial
// sums live in a fixed file-scope device array instead of plan scratch.
//
// Some callers cannot allocate device memory once they are running: a
// process whose device memory is owned by another allocator (a framework's
// caching pool, a fixed arena handed out at start-up) must not call
// cudaMalloc behind that allocator's back, and a latency-bound loop cannot
// afford an allocation that may block for milliseconds.  Such callers cannot
// create a plan (a plan allocates its tables and scratch), so this entry
// point takes the plan parameters directly, derives sigma/tau on the host,
// evaluates the window taps and FFT twiddles inside the kernels, and keeps
// its only scratch in g_static_partial below.
#include <math_constants.h>

#include <mutex>

#include "sfft_internal.cuh"

namespace {

// Capacity of the shared scratch: 2^18 complex64 partial sums (2 MiB), held by
// every device that loads the library until the process exits.
constexpr uint32_t kStaticPartialEntries = 1u << 18;

__device__ __align__(256) float2 g_static_partial[kStaticPartialEntries];

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

struct StaticArgs {
    uint32_t N, mask, B, logB, w, halfw, L;
    uint32_t tb, tiles, rounds, rpc, nchunk;
    double sg;  // Gaussian width B sqrt(log2 N)
    uint32_t sigma[sfft::kMaxL], tau[sfft::kMaxL];
    const float2 *x;
    float2 *partial;  // device address of g_static_partial
    float2 *zhat;     // caller's output [L][B]
};

// Eq. 12 (sinc of width B, centre value 1/B) times Eq. 13 (Gaussian), in
// FP64 then rounded, as the plan tables do.
__device__ float window_tap(int64_t m, uint32_t B, double sg) {
    const double sinc = (m == 0) ? 1.0 / (double)B : sinpi((double)m / (double)B) / (CUDART_PI * (double)m);
    const double t = (double)m / sg;
    return (float)(sinc * exp(-0.5 * t * t));
}

// a1: partial folds of one (bucket tile, loop, chunk of rounds); every partial
// entry of the call is written exactly once, so nothing needs clearing.
__global__ void __launch_bounds__(kThreads) k_gather_noalloc(StaticArgs a) {
    __shared__ float2 red[kThreads];
    const uint32_t local = blockIdx.x;
    const uint32_t tile = local % a.tiles;
    const uint32_t rest = local / a.tiles;
    const uint32_t l = rest % a.L;
    const uint32_t chunk = rest / a.L;
    const uint32_t TB = a.tb, PP = kThreads / TB;
    const uint32_t jt = threadIdx.x & (TB - 1), s = threadIdx.x / TB;
    const uint32_t j = tile * TB + jt;
    const uint32_t r0 = chunk * a.rpc, r1 = min(a.rounds, r0 + a.rpc);
    const uint32_t sig = a.sigma[l], tau = a.tau[l];
    const uint32_t jq = (j + a.halfw) & (a.B - 1);
    float ar = 0.f, ai = 0.f;
    for (uint32_t r = r0 + s; r < r1; r += PP) {
        const uint32_t q = r * a.B + jq;
        const uint32_t i = (sig * (q - a.halfw) + tau) & a.mask;
        const float g = window_tap((int64_t)q - (int64_t)a.halfw, a.B, a.sg);
        const float2 v = __ldg(a.x + i);
        ar = fmaf(g, v.x, ar);
        ai = fmaf(g, v.y, ai);
    }
    float2 *dst = a.partial + ((size_t)chunk * a.L + l) * a.B + j;
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

// a2: one CTA per loop sums the partials in chunk order and runs the radix-2
// FFT in shared memory with FP64-derived twiddles.
__global__ void __launch_bounds__(kThreads) k_fft_noalloc(StaticArgs a) {
    extern __shared__ float2 sm2[];  // B values, then B/2 twiddles
    float2 *buf = sm2;
    float2 *tw = sm2 + a.B;
    const uint32_t l = blockIdx.x, B = a.B, logB = a.logB;
    for (uint32_t k = threadIdx.x; k < B / 2; k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)B, &sn, &cs);
        tw[k] = make_float2((float)cs, (float)sn);
    }
    for (uint32_t j = threadIdx.x; j < B; j += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        for (uint32_t c = 0; c < a.nchunk; ++c) {
            const float2 v = a.partial[((size_t)c * a.L + l) * B + j];
            acc.x += v.x;
            acc.y += v.y;
        }
        buf[__brev(j) >> (32 - logB)] = acc;
    }
    __syncthreads();
    for (uint32_t hs = 0; hs < logB; ++hs) {
        const uint32_t h = 1u << hs;
        for (uint32_t bf = threadIdx.x; bf < B / 2; bf += blockDim.x) {
            const uint32_t k = bf & (h - 1);
            const uint32_t i0 = ((bf >> hs) << (hs + 1)) + k, i1 = i0 + h;
            const float2 w = tw[k << (logB - 1 - hs)];
            const float2 x0 = buf[i0], x1 = buf[i1];
            const float2 t = make_float2(w.x * x1.x - w.y * x1.y, w.x * x1.y + w.y * x1.x);
            buf[i0] = make_float2(x0.x + t.x, x0.y + t.y);
            buf[i1] = make_float2(x0.x - t.x, x0.y - t.y);
        }
        __syncthreads();
    }
    for (uint32_t k = threadIdx.x; k < B; k += blockDim.x) a.zhat[(size_t)l * B + k] = buf[k];
}

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};  // multiprocessor count of each device (shapes the chunk split)

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

uint32_t log2u(uint64_t v) {
    uint32_t r = 0;
    while ((1ull << r) < v) ++r;
    return r;
}

}  // namespace

extern "C" sfft_status sfft_bucketize_noalloc(int64_t N, int32_t B, int64_t w, int32_t L, uint64_t seed,
                                              const float *x_dev, float *zhat_dev, void *stream) {
    if (!x_dev || !zhat_dev) {
        sfft::set_error("NULL argument");
        return SFFT_EINVAL;
    }
    if (!pow2(N) || N < 2 || N > (1ll << sfft::kMaxLogN) || !pow2(B) || B < 2 || B > sfft::kMaxB || B > N ||
        w < B || w > N || w % B || L < 1 || L > sfft::kMaxL) {
        sfft::set_error("invalid size: need N a power of two in [2, 2^30], B a power of two in "
                        "[2, min(N, 16384)], w a multiple of B in [B, N], L in [1, 32]");
        return SFFT_EINVAL;
    }
    if ((uint64_t)L * (uint64_t)B > kStaticPartialEntries) {
        sfft::set_error("L*B exceeds the static scratch of sfft_bucketize_noalloc (at most 262144 partial sums)");
        return SFFT_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sfft::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        sfft::set_error("device ordinal out of range for the static scratch table");
        return SFFT_EINVAL;
    }
    void *partial = nullptr;
    int sms = 0;
    {
        // once per device, with that device current: the array's device
        // address and the multiprocessor count (neither query allocates)
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_partial);
            if (e != cudaSuccess) return sfft::cuda_fail(e, "cudaGetSymbolAddress(g_static_partial)");
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return sfft::cuda_fail(e, "cudaDeviceGetAttribute(multiprocessors)");
            g_sms[dev] = n > 0 ? n : 1;
            g_addr[dev] = p;
        }
        partial = g_addr[dev];
        sms = g_sms[dev];
    }

    StaticArgs a;
    a.N = (uint32_t)N;
    a.mask = (uint32_t)(N - 1);
    a.B = (uint32_t)B;
    a.logB = log2u(B);
    a.w = (uint32_t)w;
    a.halfw = (uint32_t)(w / 2);
    a.L = (uint32_t)L;
    a.sg = (double)B * sqrt((double)log2u(N));
    const sfft_status st = sfft_loop_params(N, L, seed, a.sigma, a.tau, nullptr);
    if (st != SFFT_OK) return st;
    // same work split as a plan, with the chunk count capped by the scratch
    a.tb = B < kThreads ? (uint32_t)B : (uint32_t)kThreads;
    a.tiles = a.B / a.tb;
    a.rounds = a.w / a.B;
    uint32_t want = (2 * (uint32_t)sms + a.tiles * a.L - 1) / (a.tiles * a.L);
    const uint32_t fit = kStaticPartialEntries / (a.L * a.B);
    want = want < a.rounds ? want : a.rounds;
    want = want < fit ? want : fit;
    want = want > 0 ? want : 1;
    a.rpc = (a.rounds + want - 1) / want;
    a.nchunk = (a.rounds + a.rpc - 1) / a.rpc;
    a.x = reinterpret_cast<const float2 *>(x_dev);
    a.partial = static_cast<float2 *>(partial);
    a.zhat = reinterpret_cast<float2 *>(zhat_dev);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_gather_noalloc<<<a.tiles * a.L * a.nchunk, kThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return sfft::cuda_fail(e, "k_gather_noalloc");
    const int smem = (int)(sizeof(float2) * (B + B / 2));
    if ((e = cudaFuncSetAttribute(k_fft_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return sfft::cuda_fail(e, "k_fft_noalloc attribute");
    k_fft_noalloc<<<L, kThreads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return sfft::cuda_fail(e, "k_fft_noalloc");
    return SFFT_OK;
}
