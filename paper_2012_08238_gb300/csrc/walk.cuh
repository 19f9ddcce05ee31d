// Sampling geometry of the flat-window bucketization (step a1) read in sample
// order, for the stream gather.
//
// Loop (sigma, tau) of a plan reads sample p with window tap q(p) =
// (sigma^-1 (p - tau) + w/2) mod N whenever q(p) < w (tap q weights
// m = q - w/2 of the permuted signal, folded into bucket (q - w/2) mod B).
// As p advances by one, q advances by s = sigma^-1 mod N, so the samples a
// loop reads are the visits of the rotation q -> q + s of Z_N to the interval
// [0, w).  By the three-distance theorem for first returns to an interval
// (N. B. Slater, 1950/1967) the gaps between consecutive reads take at most
// three values: with k+ (k-) the least k >= 1 whose displacement k s mod N
// lies in (0, w) (in (-w, 0)), alpha = k+ s mod N and beta = -(k- s) mod N
// (so alpha + beta >= w), the read after the one with tap q is
//   p + k+         with tap q + alpha           when q + alpha < w,
//   p + k-         with tap q - beta            when q >= beta,
//   p + k+ + k-    with tap q + alpha - beta    otherwise.
// A reader that walks a range of samples therefore needs only the first read
// at or after the range's start and these four numbers per loop.
#pragma once

#include <stdint.h>

namespace sfft {

constexpr uint64_t kNoMult = ~0ull;

// Least k >= 0 with lo <= (a k mod m) <= hi, for 0 <= lo <= hi < m, or
// kNoMult when there is none.  Euclid-like: if no multiple of a lies in
// [lo, hi], a solution a k = m y + t (t in [lo, hi]) needs the least y >= 1
// with (m y mod a) in [a - hi mod a, a - lo mod a], the same problem for
// (m mod a, a); then k = ceil((lo + m y) / a).  The reductions follow
// Euclid's algorithm on (a, m), at most ~1.44 log2(m) of them (an explicit
// stack, no recursion).  m < 2^31 keeps every product below 2^62.
__host__ __device__ inline uint64_t least_mult_in(uint64_t a, uint64_t m, uint64_t lo, uint64_t hi) {
    constexpr int kDepth = 64;
    uint64_t fa[kDepth], fm[kDepth], fl[kDepth];
    int d = 0;
    uint64_t k = 0;
    for (;;) {
        if (lo == 0) {
            k = 0;
            break;
        }
        a %= m;
        if (a == 0) return kNoMult;
        const uint64_t c = (lo + a - 1) / a;
        if (a * c <= hi) {
            k = c;
            break;
        }
        if (d == kDepth) return kNoMult;  // (unreachable for m < 2^31)
        fa[d] = a;
        fm[d] = m;
        fl[d] = lo;
        ++d;
        const uint64_t nlo = a - hi % a, nhi = a - lo % a;
        const uint64_t na = m % a;
        m = a;
        a = na;
        lo = nlo;
        hi = nhi;
    }
    while (d > 0) {
        --d;
        k = (fl[d] + fm[d] * k + fa[d] - 1) / fa[d];
    }
    return k;
}

// The return map of one loop: {k+, alpha, k-, beta} for the rotation by
// s = sigma^-1 mod N and the window's w taps (2 <= w <= N; s odd, so both
// sides have a solution).
struct WindowWalk {
    uint32_t kp, alpha, km, beta;
};

__host__ __device__ inline WindowWalk window_walk(uint32_t N, uint32_t s, uint32_t w) {
    WindowWalk r;
    const uint64_t kp = least_mult_in(s, N, 1, w - 1);
    const uint64_t km = least_mult_in(s, N, (uint64_t)N - w + 1, N - 1);
    r.kp = (uint32_t)kp;
    r.alpha = (uint32_t)((kp * s) % N);
    r.km = (uint32_t)km;
    r.beta = (uint32_t)(N - (km * s) % N);
    return r;
}

// Tap of sample p in the loop with sigma^-1 = s and shift tau (>= w: not read).
__host__ __device__ inline uint32_t window_tap_of(uint32_t N, uint32_t s, uint32_t tau, uint32_t halfw, uint32_t p) {
    return (s * (p - tau) + halfw) & (N - 1);  // (uint32 wrap: exact mod N)
}

// First sample at or after p0 (cyclically) that the loop reads: its distance
// k from p0 (< N) and its tap q.
__host__ __device__ inline void window_first_read(uint32_t N, uint32_t s, uint32_t tau, uint32_t w, uint32_t halfw,
                                                  uint32_t p0, uint32_t *k, uint32_t *q) {
    const uint32_t q0 = window_tap_of(N, s, tau, halfw, p0);
    if (q0 < w) {
        *k = 0;
        *q = q0;
        return;
    }
    // (q0 + k s) mod N in [0, w)  <=>  k s mod N in [N - q0, N - q0 + w - 1] (no wrap: q0 >= w)
    const uint64_t kk = least_mult_in(s, N, (uint64_t)N - q0, (uint64_t)N - q0 + w - 1);
    *k = (uint32_t)kk;
    *q = (uint32_t)((q0 + kk * s) % N);
}

// The step of the return map from a read with tap q: returns the distance to
// the next read and updates q.
__host__ __device__ __forceinline__ uint32_t window_step(const WindowWalk &wk, uint32_t w, uint32_t &q) {
    const bool up = q + wk.alpha < w, down = q >= wk.beta;
    const uint32_t dp = up ? wk.kp : (down ? wk.km : wk.kp + wk.km);
    q = up ? q + wk.alpha : (down ? q - wk.beta : q + wk.alpha - wk.beta);
    return dp;
}

}  // namespace sfft
