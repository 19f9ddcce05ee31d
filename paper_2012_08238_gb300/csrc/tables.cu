// Seed-independent plan tables, shared by every plan of one (device, N, B, w).
//
// The window taps (Eq. 12-13), the FFT twiddles, 1/G~ over one bucket and,
// when a plan needs them, G~ over three buckets in FP32 and FP64 depend only
// on the signal length, the bucket count and the window width; sigma and tau
// (the seed) do not enter them.  Building them is the dominant plan-time
// cost (the gain tables are O(N/B w) FP64 sums), so they are built once per
// shape, reference-counted by the plans that use them, and kept for reuse
// (least recently used first out) after their last plan is destroyed.
#include <string.h>

#include <cmath>
#include <list>
#include <mutex>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

struct Entry {
    int device;
    uint32_t N, B, w;
    bool ext, ext64;
    void *mem;
    TableSet t;
    int refs;
    uint64_t last_use;
};

std::mutex g_mu;
std::list<Entry> g_entries;
uint64_t g_clock = 0;
constexpr size_t kMaxIdle = 64;  // unreferenced entries kept for reuse

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

void drop_idle_beyond(size_t keep) {
    size_t idle = 0;
    for (const Entry &e : g_entries) idle += e.refs == 0;
    while (idle > keep) {
        auto victim = g_entries.end();
        for (auto it = g_entries.begin(); it != g_entries.end(); ++it)
            if (it->refs == 0 && (victim == g_entries.end() || it->last_use < victim->last_use)) victim = it;
        if (victim == g_entries.end()) return;
        int cur = 0;
        cudaGetDevice(&cur);
        if (victim->device != cur) cudaSetDevice(victim->device);
        cudaFree(victim->mem);
        if (victim->device != cur) cudaSetDevice(cur);
        g_entries.erase(victim);
        --idle;
    }
}

// Builds the tables of one shape on a private stream and waits for them.
cudaError_t build(Entry &en) {
    const uint32_t N = en.N, B = en.B, w = en.w, NB = N / B;
    const size_t b_taps = a256(sizeof(float) * w), b_tw = a256(sizeof(float2) * (B / 2 > 0 ? B / 2 : 1)),
                 b_twst = a256(sizeof(float2) * (B > 1 ? B - 1 : 1)), b_ginv = a256(sizeof(float2) * NB), b_gext = en.ext ? a256(sizeof(float2) * 3 * NB) : 0,
                 b_gx64 = en.ext64 ? a256(sizeof(double2) * 3 * NB) : 0;
    // scratch for the build: FP64 |1/G~|^2 and its maximum
    const size_t b_g2 = a256(sizeof(double) * NB), b_max = 256;
    const size_t keep = b_taps + b_tw + b_twst + b_ginv + b_gext + b_gx64;
    cudaError_t e = cudaMalloc(&en.mem, keep + b_g2 + b_max);
    if (e != cudaSuccess) return e;
    char *base = static_cast<char *>(en.mem);
    float *taps = reinterpret_cast<float *>(base);
    float2 *tw = reinterpret_cast<float2 *>(base + b_taps);
    float2 *twst = reinterpret_cast<float2 *>(base + b_taps + b_tw);
    float2 *ginv = reinterpret_cast<float2 *>(base + b_taps + b_tw + b_twst);
    float2 *gext = en.ext ? reinterpret_cast<float2 *>(base + b_taps + b_tw + b_twst + b_ginv) : nullptr;
    double2 *gx64 =
        en.ext64 ? reinterpret_cast<double2 *>(base + b_taps + b_tw + b_twst + b_ginv + b_gext) : nullptr;
    double *g2 = reinterpret_cast<double *>(base + keep);
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(base + keep + b_g2);
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    unsigned long long hmax = 0;
    e = plan_tables(N, B, w, taps, tw, twst, ginv, g2, gext, gx64, s);
    if (e == cudaSuccess) e = plan_max_bits(g2, NB, mx, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hmax, mx, sizeof(hmax), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaFree(en.mem);
        en.mem = nullptr;
        return e;
    }
    double gmax;
    memcpy(&gmax, &hmax, sizeof(double));
    float gf = (float)gmax;  // rounded up: the strong-loop bound must not shrink
    if ((double)gf < gmax) gf = nextafterf(gf, INFINITY);
    en.t.taps = taps;
    en.t.tw = tw;
    en.t.twst = twst;
    en.t.ginv = ginv;
    en.t.gext = gext;
    en.t.gext64 = gx64;
    en.t.ginv2max = gf;
    en.t.bytes = keep + b_g2 + b_max;
    return cudaSuccess;
}

}  // namespace

sfft_status tables_acquire(uint32_t N, uint32_t B, uint32_t w, bool ext, bool ext64, const void **handle,
                           TableSet *out) {
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    for (Entry &en : g_entries) {
        if (en.device == device && en.N == N && en.B == B && en.w == w && (en.ext || !ext) && (en.ext64 || !ext64)) {
            ++en.refs;
            en.last_use = ++g_clock;
            *handle = &en;
            *out = en.t;
            return SFFT_OK;
        }
    }
    drop_idle_beyond(kMaxIdle - 1);
    Entry en{};
    en.device = device;
    en.N = N;
    en.B = B;
    en.w = w;
    en.ext = ext;
    en.ext64 = ext64;
    // (the mutex is held while building: plans of one shape wait for one build)
    if ((e = build(en)) != cudaSuccess) return cuda_fail(e, "plan tables");
    en.refs = 1;
    en.last_use = ++g_clock;
    g_entries.push_back(en);
    *handle = &g_entries.back();
    *out = en.t;
    return SFFT_OK;
}

void tables_release(const void *handle) {
    if (!handle) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (Entry &en : g_entries)
        if (&en == handle) {
            if (en.refs > 0) --en.refs;
            en.last_use = ++g_clock;
            break;
        }
    drop_idle_beyond(kMaxIdle);
}

}  // namespace sfft
