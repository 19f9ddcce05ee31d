/*
 * FP64 CPU oracle for the flat-window voting sparse FFT.  TEST INFRASTRUCTURE
 * ONLY: see sfft_oracle.h.  Plain C99, single-threaded, no blocking or fusion
 * beyond what each step's definition states.
 */
#include "sfft_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- Philox */
/* Philox4x64 round function and key schedule as published by Salmon, Moraes,
   Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
   two 64x64->128 multiplies per round, outputs permuted and xored with the
   round key, key bumped by the Weyl constants between rounds. */
static void philox_mulhilo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        philox_mulhilo(M0, x0, &hi0, &lo0);
        philox_mulhilo(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------ arithmetic */
static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static int64_t mod_pos(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

int64_t oracle_modinv(int64_t a, int64_t N)
{
    /* extended Euclid on (a, N) */
    int64_t r0 = N, r1 = mod_pos(a, N), s0 = 0, s1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    if (r0 != 1) return -1; /* not invertible */
    return mod_pos(s0, N);
}

/* ------------------------------------------------------- a0: parameters */
/* Random odd scaling sigma ("Scaling method") and shift tau (Eq. 6-7). */
int oracle_loop_params(int64_t N, int L, uint64_t seed, int64_t *sigma, int64_t *tau,
                       int64_t *sigma_inv)
{
    if (!is_pow2(N) || N < 2) return -1;
    for (int l = 0; l < L; ++l) {
        uint64_t ctr[4] = {(uint64_t)l, 0, 0, 0}, key[2] = {seed, 0}, out[4];
        oracle_philox4x64_10(ctr, key, out);
        int64_t s = 2 * (int64_t)(out[0] % (uint64_t)(N / 2)) + 1;
        sigma[l] = s;
        tau[l] = (int64_t)(out[1] % (uint64_t)N);
        if (sigma_inv) sigma_inv[l] = oracle_modinv(s, N);
    }
    return 0;
}

/* --------------------------------------------------- a0': flat window */
/* Eq. 12 (sinc of width B, centre value 1/B) times Eq. 13 (Gaussian with
   sigma_g = B sqrt(log2 N)), both centred at Omega/2 = w/2. */
void oracle_window_taps(int64_t N, int64_t B, int64_t w, double *g)
{
    double sg = (double)B * sqrt(log2((double)N));
    for (int64_t q = 0; q < w; ++q) {
        int64_t m = q - w / 2;
        double sinc = (m == 0) ? 1.0 / (double)B
                               : sin(M_PI * (double)m / (double)B) / (M_PI * (double)m);
        double t = (double)m / sg;
        g[q] = sinc * exp(-0.5 * t * t);
    }
}

/* exp(+2 pi i r / N) with the integer r reduced first (exact argument) */
static double complex unit_root(int64_t r, int64_t N)
{
    double a = 2.0 * M_PI * (double)mod_pos(r, N) / (double)N;
    return cos(a) + I * sin(a);
}

void oracle_filter_gain_at(int64_t N, int64_t w, const double *g, int64_t o, double out[2])
{
    double complex s = 0;
    for (int64_t q = 0; q < w; ++q) {
        int64_t m = q - w / 2;
        s += g[q] * unit_root(mod_pos(m * o, N), N);
    }
    out[0] = creal(s);
    out[1] = cimag(s);
}

void oracle_filter_gain(int64_t N, int64_t B, int64_t w, const double *g, double *Gt)
{
    int64_t NB = N / B, half = NB / 2;
    for (int64_t i = 0; i < NB; ++i) oracle_filter_gain_at(N, w, g, i - half, Gt + 2 * i);
}

/* ----------------------------------------------------------- a4: hash */
/* Bucket of frequency f after scaling: round-half-up of (sigma f mod N)/(N/B),
   the rule of the worked example (bucket 1 = round(64/128)). */
void oracle_hash(int64_t N, int64_t B, int64_t sigma, int64_t f, int64_t *h, int64_t *o)
{
    int64_t NB = N / B, half = NB / 2;
    int64_t p = mod_pos(sigma * f, N);
    int64_t hh = (p + half) / NB; /* in [0, B] */
    *o = p - hh * NB;             /* in [-half, NB - half) */
    *h = hh % B;
}

void oracle_permute(int64_t N, int64_t sigma, int64_t tau, const double *x, double *out)
{
    for (int64_t m = 0; m < N; ++m) {
        int64_t i = mod_pos(sigma * m + tau, N);
        out[2 * m] = x[2 * i];
        out[2 * m + 1] = x[2 * i + 1];
    }
}

/* ------------------------------------------------------ a1 + a2 */
void oracle_bucketize(int64_t N, int64_t B, int64_t w, int L, const int64_t *sigma,
                      const int64_t *tau, const double *g, const double *x, double *z,
                      double *zhat)
{
    double complex *zl = (double complex *)malloc(sizeof(double complex) * (size_t)B);
    double complex *wB = (double complex *)malloc(sizeof(double complex) * (size_t)B);
    for (int64_t t = 0; t < B; ++t) {
        double a = -2.0 * M_PI * (double)t / (double)B;
        wB[t] = cos(a) + I * sin(a); /* omega_B^t */
    }
    for (int l = 0; l < L; ++l) {
        for (int64_t j = 0; j < B; ++j) zl[j] = 0;
        /* multiply by the window and fold (Eq. 11) the permuted signal */
        for (int64_t q = 0; q < w; ++q) {
            int64_t m = q - w / 2;
            int64_t i = mod_pos(sigma[l] * m + tau[l], N);
            int64_t j = mod_pos(m, B);
            zl[j] += g[q] * (x[2 * i] + I * x[2 * i + 1]);
        }
        if (z) {
            for (int64_t j = 0; j < B; ++j) {
                z[2 * (l * B + j)] = creal(zl[j]);
                z[2 * (l * B + j) + 1] = cimag(zl[j]);
            }
        }
        /* B-point DFT, unnormalised */
        for (int64_t k = 0; k < B; ++k) {
            double complex s = 0;
            for (int64_t j = 0; j < B; ++j) s += zl[j] * wB[(j * k) % B];
            zhat[2 * (l * B + k)] = creal(s);
            zhat[2 * (l * B + k) + 1] = cimag(s);
        }
    }
    free(zl);
    free(wB);
}

/* ---------------------------------------------------------- a3: select */
typedef struct {
    float key;
    int64_t id;  /* tie-break: smaller id ranks first */
    int64_t pos; /* where the entry came from */
} keyed;

/* larger key first, then smaller id */
static int keyed_cmp(const void *a, const void *b)
{
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key > y->key) return -1;
    if (x->key < y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

int64_t oracle_select(int64_t B, int64_t cK, const double *zhat_loop, int32_t *sel)
{
    keyed *k = (keyed *)malloc(sizeof(keyed) * (size_t)B);
    for (int64_t j = 0; j < B; ++j) {
        double re = zhat_loop[2 * j], im = zhat_loop[2 * j + 1];
        k[j].key = (float)(re * re + im * im);
        k[j].id = j;
        k[j].pos = j;
    }
    qsort(k, (size_t)B, sizeof(keyed), keyed_cmp);
    int64_t n = cK < B ? cK : B;
    for (int64_t s = 0; s < n; ++s) sel[s] = (int32_t)k[s].id;
    free(k);
    return n;
}

/* ------------------------------------------------------ a4 + a5: vote */
/* Every frequency hashed (via sigma^-1) into one of the selected buckets of a
   loop receives one vote; candidates are those with at least T votes. */
int64_t oracle_vote(int64_t N, int64_t B, int L, int64_t nsel, int T, const int64_t *sigma_inv,
                    const int32_t *sel, int32_t *score, int32_t *cand)
{
    int64_t NB = N / B, half = NB / 2;
    int32_t *sc = score ? score : (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    memset(sc, 0, sizeof(int32_t) * (size_t)N);
    for (int l = 0; l < L; ++l) {
        for (int64_t s = 0; s < nsel; ++s) {
            int64_t j = sel[l * nsel + s];
            for (int64_t o = -half; o < NB - half; ++o) {
                int64_t p = mod_pos(j * NB + o, N);
                int64_t f = mod_pos(sigma_inv[l] * p, N);
                sc[f] += 1;
            }
        }
    }
    int64_t n = 0;
    for (int64_t f = 0; f < N; ++f)
        if (sc[f] >= T) cand[n++] = (int32_t)f;
    if (!score) free(sc);
    return n;
}

/* ------------------------------------------------------ a6: estimate */
static int dbl_cmp(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double median_of(double *v, int n)
{
    qsort(v, (size_t)n, sizeof(double), dbl_cmp);
    if (n % 2) return v[n / 2];
    return 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

/* combine = ORACLE_MEDIAN: the coordinate-wise median of the L per-loop
   estimates; ORACLE_MEAN: their average ("the average value of multiple
   buckets", § "The method of estimating the value"). */
void oracle_estimate_ex(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                        const double *Gt, const double *zhat, int64_t ncand, const int32_t *cand,
                        int combine, double *est, double *per_loop)
{
    int64_t half = (N / B) / 2;
    double *re = (double *)malloc(sizeof(double) * (size_t)L);
    double *im = (double *)malloc(sizeof(double) * (size_t)L);
    for (int64_t c = 0; c < ncand; ++c) {
        int64_t f = cand[c];
        for (int l = 0; l < L; ++l) {
            int64_t h, o;
            oracle_hash(N, B, sigma[l], f, &h, &o);
            double complex zb = zhat[2 * (l * B + h)] + I * zhat[2 * (l * B + h) + 1];
            double complex G = Gt[2 * (o + half)] + I * Gt[2 * (o + half) + 1];
            /* undo the time-shift phase exp(+2 pi i tau f / N) and the
               filter's gain at offset o */
            double complex v = zb * unit_root(-(tau[l] * f), N) / G;
            re[l] = creal(v);
            im[l] = cimag(v);
            if (per_loop) {
                per_loop[2 * (c * L + l)] = re[l];
                per_loop[2 * (c * L + l) + 1] = im[l];
            }
        }
        if (combine == ORACLE_MEAN) {
            double sr = 0.0, si = 0.0;
            for (int l = 0; l < L; ++l) {
                sr += re[l];
                si += im[l];
            }
            est[2 * c] = sr / (double)L;
            est[2 * c + 1] = si / (double)L;
        } else {
            est[2 * c] = median_of(re, L);
            est[2 * c + 1] = median_of(im, L);
        }
    }
    free(re);
    free(im);
}

void oracle_estimate(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                     const double *Gt, const double *zhat, int64_t ncand, const int32_t *cand,
                     double *est, double *per_loop)
{
    oracle_estimate_ex(N, B, L, sigma, tau, Gt, zhat, ncand, cand, ORACLE_MEDIAN, est, per_loop);
}

/* --------------------------------------------------------- a7: top-K */
int64_t oracle_topk(int64_t ncand, const int32_t *cand, const double *est, int64_t K,
                    int32_t *idx, double *val)
{
    keyed *k = (keyed *)malloc(sizeof(keyed) * (size_t)(ncand > 0 ? ncand : 1));
    for (int64_t c = 0; c < ncand; ++c) {
        double re = est[2 * c], im = est[2 * c + 1];
        k[c].key = (float)(re * re + im * im);
        k[c].id = cand[c];
        k[c].pos = c;
    }
    qsort(k, (size_t)ncand, sizeof(keyed), keyed_cmp);
    int64_t n = K < ncand ? K : ncand;
    /* the n winners, back in increasing f */
    keyed *win = (keyed *)malloc(sizeof(keyed) * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) {
        win[s] = k[s];
        win[s].key = 0.0f; /* equal keys: the comparator falls back to id = f */
    }
    qsort(win, (size_t)n, sizeof(keyed), keyed_cmp);
    for (int64_t s = 0; s < n; ++s) {
        idx[s] = (int32_t)win[s].id;
        val[2 * s] = est[2 * win[s].pos];
        val[2 * s + 1] = est[2 * win[s].pos + 1];
    }
    free(win);
    free(k);
    return n;
}

/* ---------------------------------------------------- sampling ratio */
int64_t oracle_samples_touched(int64_t N, int64_t w, int L, const int64_t *sigma,
                               const int64_t *tau)
{
    unsigned char *seen = (unsigned char *)calloc((size_t)N, 1);
    int64_t n = 0;
    for (int l = 0; l < L; ++l)
        for (int64_t q = 0; q < w; ++q) {
            int64_t i = mod_pos(sigma[l] * (q - w / 2) + tau[l], N);
            if (!seen[i]) {
                seen[i] = 1;
                ++n;
            }
        }
    free(seen);
    return n;
}

/* ------------------------------------------------------------- Eq. 2 */
void oracle_dft(int64_t N, const double *x, double *xhat)
{
    for (int64_t i = 0; i < N; ++i) {
        double complex s = 0;
        for (int64_t j = 0; j < N; ++j)
            s += (x[2 * j] + I * x[2 * j + 1]) * unit_root(-mod_pos(i * j, N), N);
        s /= (double)N;
        xhat[2 * i] = creal(s);
        xhat[2 * i + 1] = cimag(s);
    }
}

/* --------------------------------------------------------- pipeline */
int64_t oracle_sfft(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T,
                    uint64_t seed, const double *g, const double *Gt, const double *x,
                    int32_t *idx, double *val, double *zhat_out, int32_t *sel_out,
                    int32_t *cand_out, double *est_out, int64_t *ncand_out)
{
    return oracle_sfft_ex(N, K, B, w, L, c, T, seed, g, Gt, x, ORACLE_MEDIAN, idx, val, zhat_out, sel_out,
                          cand_out, est_out, ncand_out);
}

int64_t oracle_sfft_ex(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T,
                       uint64_t seed, const double *g, const double *Gt, const double *x, int combine,
                       int32_t *idx, double *val, double *zhat_out, int32_t *sel_out,
                       int32_t *cand_out, double *est_out, int64_t *ncand_out)
{
    if (!is_pow2(N) || N < 2 || !is_pow2(B) || B > N || w < B || w > N || w % B || L < 1 ||
        K < 1 || c < 1 || T < 1 || T > L)
        return -1;
    int64_t *sigma = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    int64_t *sinv = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    oracle_loop_params(N, L, seed, sigma, tau, sinv);

    double *zhat = zhat_out ? zhat_out : (double *)malloc(sizeof(double) * 2 * (size_t)(L * B));
    oracle_bucketize(N, B, w, L, sigma, tau, g, x, NULL, zhat);

    int64_t cK = (int64_t)c * K;
    int64_t nsel = cK < B ? cK : B;
    int32_t *sel = sel_out ? sel_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)(L * nsel));
    for (int l = 0; l < L; ++l) oracle_select(B, cK, zhat + 2 * l * B, sel + l * nsel);

    int32_t *cand = cand_out ? cand_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t ncand = oracle_vote(N, B, L, nsel, T, sinv, sel, NULL, cand);

    double *est = est_out ? est_out : (double *)malloc(sizeof(double) * 2 * (size_t)(ncand ? ncand : 1));
    oracle_estimate_ex(N, B, L, sigma, tau, Gt, zhat, ncand, cand, combine, est, NULL);

    int64_t kout = oracle_topk(ncand, cand, est, K, idx, val);
    if (ncand_out) *ncand_out = ncand;

    if (!est_out) free(est);
    if (!cand_out) free(cand);
    if (!sel_out) free(sel);
    if (!zhat_out) free(zhat);
    free(sigma);
    free(tau);
    free(sinv);
    return kout;
}

/* ==================================================================
 * sFFT3.0-style location: phase encoding ("Phase encoding method") inside
 * the iterative framework ("The iterative framework"; Table 1, sFFT3.0:
 * flat filter, phase encoding, energy estimation, iteration, exactly sparse).
 * ================================================================== */

/* Textbook iterative radix-2 FFT (decimation in time), in place:
   a[k] <- sum_n a[n] exp(s 2 pi i n k / n_len), s = +1 or -1. */
static void fft_radix2(int64_t n, double complex *a, int s)
{
    for (int64_t i = 1, j = 0; i < n; ++i) { /* bit reversal */
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < len / 2; ++k) {
                double ang = (double)s * 2.0 * M_PI * (double)k / (double)len;
                double complex wk = cos(ang) + I * sin(ang);
                double complex u = a[i + k], v = a[i + k + len / 2] * wk;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

void oracle_filter_gain_full(int64_t N, int64_t w, const double *g, double *Gfull)
{
    double complex *a = (double complex *)calloc((size_t)N, sizeof(double complex));
    for (int64_t q = 0; q < w; ++q) a[mod_pos(q - w / 2, N)] += g[q]; /* g(m) at index m mod N */
    fft_radix2(N, a, +1);
    for (int64_t v = 0; v < N; ++v) {
        Gfull[2 * v] = creal(a[v]);
        Gfull[2 * v + 1] = cimag(a[v]);
    }
    free(a);
}

void oracle_pe_subtract(int64_t N, int64_t B, int64_t sigma, int64_t tau, const double *Gfull, int64_t nf,
                        const int32_t *fidx, const double *fval, double *zhat)
{
    int64_t NB = N / B;
    for (int64_t c = 0; c < nf; ++c) {
        int64_t f = fidx[c];
        double complex v = fval[2 * c] + I * fval[2 * c + 1];
        double complex vt = v * unit_root(tau * f, N); /* x^_f exp(+2 pi i tau f / N) */
        int64_t p = mod_pos(sigma * f, N);
        for (int64_t k = 0; k < B; ++k) {
            int64_t nu = mod_pos(p - k * NB, N);
            double complex G = Gfull[2 * nu] + I * Gfull[2 * nu + 1];
            double complex d = vt * G;
            zhat[2 * k] -= creal(d);
            zhat[2 * k + 1] -= cimag(d);
        }
    }
}

int64_t oracle_pe_locate(int64_t N, int64_t B, int64_t sigma, int64_t tau, const double *Gfull,
                         const double *zhat0, const double *zhat1, double thr, int32_t *f_out,
                         double *v_out, int64_t *active_out)
{
    int64_t n = 0, active = 0;
    for (int64_t k = 0; k < B; ++k) {
        double complex z0 = zhat0[2 * k] + I * zhat0[2 * k + 1];
        double complex z1 = zhat1[2 * k] + I * zhat1[2 * k + 1];
        double e = creal(z0) * creal(z0) + cimag(z0) * cimag(z0);
        if (!(e >= thr) || e == 0.0) continue;
        ++active;
        /* a lone coefficient at f turns by exp(+2 pi i f / N) per unit shift */
        double complex r = z1 * conj(z0);
        double phi = atan2(cimag(r), creal(r));
        int64_t f = mod_pos(llround(phi * (double)N / (2.0 * M_PI)), N);
        int64_t h, o;
        oracle_hash(N, B, sigma, f, &h, &o);
        if (h != k) continue; /* not a lone coefficient of this bucket */
        double complex G = Gfull[2 * mod_pos(o, N)] + I * Gfull[2 * mod_pos(o, N) + 1];
        double complex v = z0 * unit_root(-tau * f, N) / G;
        f_out[n] = (int32_t)f;
        v_out[2 * n] = creal(v);
        v_out[2 * n + 1] = cimag(v);
        ++n;
    }
    *active_out = active;
    return n;
}

int64_t oracle_sfft_pe(int64_t N, int64_t K, int64_t B, int64_t w, int R, double eta, uint64_t seed,
                       const double *g, const double *Gfull, const double *x, int32_t *idx, double *val,
                       int *iters_out, int64_t *nfound_out)
{
    if (!is_pow2(N) || N < 2 || !is_pow2(B) || B > N || w < B || w % B || R < 1 || K < 0) return -1;
    int64_t *sigma = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    int64_t *sinv = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    oracle_loop_params(N, R, seed, sigma, tau, sinv);
    double *found = (double *)calloc(2 * (size_t)N, sizeof(double)); /* accumulated values */
    char *seen = (char *)calloc((size_t)N, 1);
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *lval = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    int64_t nf = 0;
    double *z0 = (double *)malloc(sizeof(double) * 2 * (size_t)B);
    double *z1 = (double *)malloc(sizeof(double) * 2 * (size_t)B);
    int32_t *nfi = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
    double *nfv = (double *)malloc(sizeof(double) * 2 * (size_t)B);
    double thr = 0.0;
    int iters = 0;
    for (int r = 0; r < R; ++r) {
        int64_t t0 = tau[r], t1 = mod_pos(tau[r] + 1, N);
        oracle_bucketize(N, B, w, 1, &sigma[r], &t0, g, x, NULL, z0); /* shift tau_r */
        oracle_bucketize(N, B, w, 1, &sigma[r], &t1, g, x, NULL, z1); /* shift tau_r + 1 */
        for (int64_t c = 0; c < nf; ++c) {
            lval[2 * c] = found[2 * list[c]];
            lval[2 * c + 1] = found[2 * list[c] + 1];
        }
        oracle_pe_subtract(N, B, sigma[r], t0, Gfull, nf, list, lval, z0);
        oracle_pe_subtract(N, B, sigma[r], t1, Gfull, nf, list, lval, z1);
        if (r == 0) {
            double emax = 0.0;
            for (int64_t k = 0; k < B; ++k) {
                double e = z0[2 * k] * z0[2 * k] + z0[2 * k + 1] * z0[2 * k + 1];
                if (e > emax) emax = e;
            }
            thr = eta * emax;
        }
        int64_t active = 0;
        int64_t n = oracle_pe_locate(N, B, sigma[r], t0, Gfull, z0, z1, thr, nfi, nfv, &active);
        iters = r + 1;
        if (active == 0) break;
        for (int64_t c = 0; c < n; ++c) {
            int64_t f = nfi[c];
            found[2 * f] += nfv[2 * c];
            found[2 * f + 1] += nfv[2 * c + 1];
            if (!seen[f]) {
                seen[f] = 1;
                list[nf++] = (int32_t)f;
            }
        }
    }
    for (int64_t c = 0; c < nf; ++c) {
        lval[2 * c] = found[2 * list[c]];
        lval[2 * c + 1] = found[2 * list[c] + 1];
    }
    int64_t kout = oracle_topk(nf, list, lval, K, idx, val);
    if (iters_out) *iters_out = iters;
    if (nfound_out) *nfound_out = nf;
    free(sigma);
    free(tau);
    free(sinv);
    free(found);
    free(seen);
    free(list);
    free(lval);
    free(z0);
    free(z1);
    free(nfi);
    free(nfv);
    return kout;
}

/* ==================================================================
 * sFFT2.0-style spike-train pre-filter (Eq. 10 subsampling, Eq. 15 spike
 * train, Eq. 16 bucket composition; Table 1 sFFT2.0: spike train + flat
 * filters, statistics, energy, voting).
 * ================================================================== */

int64_t oracle_comb(int64_t N, int64_t Bc, int C, const int64_t *tau_c, int64_t nkeep, const double *x,
                    uint8_t *kept, double *E)
{
    int64_t stride = N / Bc;
    double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)Bc);
    double complex *y = (double complex *)malloc(sizeof(double complex) * (size_t)Bc);
    for (int64_t i = 0; i < Bc; ++i) E[i] = 0.0;
    for (int c = 0; c < C; ++c) {
        /* subsample (Eq. 10) at a shift: one sample per N/Bc */
        for (int64_t j = 0; j < Bc; ++j) {
            int64_t n = mod_pos(tau_c[c] + j * stride, N);
            w[j] = x[2 * n] + I * x[2 * n + 1];
        }
        /* Bc-point DFT with 1/Bc: y[i] = sum over f = i (mod Bc) of x^_f e^{+2 pi i tau f / N} (Eq. 16) */
        for (int64_t i = 0; i < Bc; ++i) {
            double complex s = 0;
            for (int64_t j = 0; j < Bc; ++j) {
                double a = -2.0 * M_PI * (double)((i * j) % Bc) / (double)Bc;
                s += w[j] * (cos(a) + I * sin(a));
            }
            y[i] = s / (double)Bc;
        }
        for (int64_t i = 0; i < Bc; ++i) E[i] += creal(y[i]) * creal(y[i]) + cimag(y[i]) * cimag(y[i]);
    }
    /* kept classes: the nkeep largest energies (key rounded to binary32), ties to the lower class */
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)Bc);
    double *Ez = (double *)malloc(sizeof(double) * 2 * (size_t)Bc); /* as |z|^2 with z = sqrt(E) */
    for (int64_t i = 0; i < Bc; ++i) {
        Ez[2 * i] = sqrt(E[i]);
        Ez[2 * i + 1] = 0.0;
    }
    int64_t n = oracle_select(Bc, nkeep, Ez, sel);
    memset(kept, 0, (size_t)Bc);
    for (int64_t s = 0; s < n; ++s) kept[sel[s]] = 1;
    free(sel);
    free(Ez);
    free(w);
    free(y);
    return n;
}

int64_t oracle_sfft2(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T, int64_t Bc, int C,
                     uint64_t seed, const double *g, const double *Gt, const double *x, int32_t *idx, double *val,
                     uint8_t *kept_out, int64_t *ncand_out)
{
    return oracle_sfft2_ex(N, K, B, w, L, c, T, Bc, C, seed, g, Gt, x, ORACLE_MEDIAN, idx, val, kept_out,
                           ncand_out, NULL);
}

int64_t oracle_sfft2_ex(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T, int64_t Bc, int C,
                        uint64_t seed, const double *g, const double *Gt, const double *x, int combine,
                        int32_t *idx, double *val, uint8_t *kept_out, int64_t *ncand_out, double *zhat_out)
{
    if (!is_pow2(N) || N < 2 || !is_pow2(B) || B > N || w < B || w % B || L < 1 || c < 1 || T < 1 || T > L ||
        !is_pow2(Bc) || Bc > N || C < 1)
        return -1;
    int64_t *sigma = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L + C));
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L + C));
    int64_t *sinv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L + C));
    oracle_loop_params(N, L + C, seed, sigma, tau, sinv); /* loops 0..L-1 vote; L..L+C-1 give the comb shifts */

    uint8_t *kept = kept_out ? kept_out : (uint8_t *)malloc((size_t)Bc);
    double *E = (double *)malloc(sizeof(double) * (size_t)Bc);
    oracle_comb(N, Bc, C, tau + L, (int64_t)c * K < Bc ? (int64_t)c * K : Bc, x, kept, E);

    double *zhat = zhat_out ? zhat_out : (double *)malloc(sizeof(double) * 2 * (size_t)(L * B));
    oracle_bucketize(N, B, w, L, sigma, tau, g, x, NULL, zhat);
    int64_t cK = (int64_t)c * K;
    int64_t nsel = cK < B ? cK : B;
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L * nsel));
    for (int l = 0; l < L; ++l) oracle_select(B, cK, zhat + 2 * l * B, sel + l * nsel);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t nc = oracle_vote(N, B, L, nsel, T, sinv, sel, NULL, cand);
    /* only frequencies of kept residue classes stay candidates */
    int64_t ncand = 0;
    for (int64_t q = 0; q < nc; ++q)
        if (kept[mod_pos(cand[q], Bc)]) cand[ncand++] = cand[q];
    double *est = (double *)malloc(sizeof(double) * 2 * (size_t)(ncand ? ncand : 1));
    oracle_estimate_ex(N, B, L, sigma, tau, Gt, zhat, ncand, cand, combine, est, NULL);
    int64_t kout = oracle_topk(ncand, cand, est, K, idx, val);
    if (ncand_out) *ncand_out = ncand;
    if (!kept_out) free(kept);
    free(E);
    if (!zhat_out) free(zhat);
    free(sel);
    free(cand);
    free(est);
    free(sigma);
    free(tau);
    free(sinv);
    return kout;
}

/* ==================================================================
 * Iterative-framework refinement of a found set (§ "Four algorithmic
 * frameworks", its iterative framework, applied to the voting output).
 * ================================================================== */

void oracle_refine(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau, const double *Gfull,
                   const double *zhat, int64_t n, const int32_t *idx, int combine, int passes, double *val)
{
    int64_t NB = N / B;
    double *cur = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double *re = (double *)malloc(sizeof(double) * (size_t)L);
    double *im = (double *)malloc(sizeof(double) * (size_t)L);
    for (int p = 0; p < passes; ++p) {
        for (int64_t q = 0; q < 2 * n; ++q) cur[q] = val[q];
        for (int64_t c = 0; c < n; ++c) {
            int64_t f = idx[c];
            for (int l = 0; l < L; ++l) {
                int64_t h, o;
                oracle_hash(N, B, sigma[l], f, &h, &o);
                double complex r = zhat[2 * (l * B + h)] + I * zhat[2 * (l * B + h) + 1];
                /* the other found coefficients' share of this bucket, by the
                   identity zhat_l[k] = sum_g x^_g e^{+2 pi i tau g / N} G~(sigma g - k N/B) */
                for (int64_t d = 0; d < n; ++d) {
                    if (d == c) continue;
                    int64_t gq = idx[d];
                    double complex v = cur[2 * d] + I * cur[2 * d + 1];
                    int64_t nu = mod_pos(sigma[l] * gq - h * NB, N);
                    double complex G = Gfull[2 * nu] + I * Gfull[2 * nu + 1];
                    r -= v * unit_root(tau[l] * gq, N) * G;
                }
                double complex Gf = Gfull[2 * mod_pos(o, N)] + I * Gfull[2 * mod_pos(o, N) + 1];
                double complex e = r * conj(unit_root(tau[l] * f, N)) / Gf; /* undo the turn of f */
                re[l] = creal(e);
                im[l] = cimag(e);
            }
            if (combine == ORACLE_MEDIAN) {
                val[2 * c] = median_of(re, L);
                val[2 * c + 1] = median_of(im, L);
            } else {
                double sr = 0.0, si = 0.0;
                for (int l = 0; l < L; ++l) {
                    sr += re[l];
                    si += im[l];
                }
                val[2 * c] = sr / (double)L;
                val[2 * c + 1] = si / (double)L;
            }
        }
    }
    free(cur);
    free(re);
    free(im);
}

/* ==================================================================
 * sFFT4.0 / MPFFT-style location by binary or multi-scale search (§ "The
 * method of binary search or multi-scale search"; Table 1: flat filter,
 * binary or multi-scale search, energy estimation, iterative framework).
 * ================================================================== */

/* The search decodes the low log2(N/B) + 1 bits of f (capped at log2 N):
   they fix p = sigma f modulo 2N/B, which picks one value in the window of
   two bucket widths centred on bucket k, so a coefficient that leaks into a
   neighbouring bucket is located there too and fails the hash-back test.
   Digit j covers bits [j b, min((j+1) b, bits)); at shift N / 2^m (m = the
   digit's top bit + 1) a coefficient f turns by exp(2 pi i f / 2^m), which
   depends on f mod 2^m only. */
static int64_t bs_bits(int64_t N, int64_t B)
{
    int64_t bits = 1, logN = 0;
    for (int64_t q = N / B; q > 1; q >>= 1) ++bits;
    for (int64_t q = N; q > 1; q >>= 1) ++logN;
    return bits < logN ? bits : logN;
}

static int64_t bs_steps(int64_t N, int64_t B, int b)
{
    int64_t J = 0, bits = bs_bits(N, B);
    for (int64_t lo = 0; lo < bits; lo += b) ++J;
    return J;
}

int64_t oracle_bs_nshifts(int64_t N, int64_t B, int b) { return 1 + bs_steps(N, B, b); }

void oracle_bs_shifts(int64_t N, int64_t B, int b, int64_t *s)
{
    int64_t bits = bs_bits(N, B);
    int64_t J = bs_steps(N, B, b);
    s[0] = 0;
    for (int64_t j = 0; j < J; ++j) {
        int64_t m = (j + 1) * b < bits ? (j + 1) * b : bits;
        s[j + 1] = N >> m;
    }
}

int64_t oracle_bs_locate(int64_t N, int64_t B, int b, int64_t sigma, int64_t sigma_inv, int64_t tau,
                         const double *Gfull, const double *zhat, double thr, double rho, int32_t *f_out,
                         double *v_out, int64_t *active_out)
{
    int64_t NB = N / B, bits = bs_bits(N, B);
    int64_t W = (int64_t)1 << bits; /* p is decoded modulo W = 2N/B (N when B = 1) */
    int64_t J = bs_steps(N, B, b);
    int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)(J + 1));
    oracle_bs_shifts(N, B, b, s);
    int64_t n = 0, active = 0;
    for (int64_t k = 0; k < B; ++k) {
        double complex z0 = zhat[2 * k] + I * zhat[2 * k + 1];
        double e0 = creal(z0) * creal(z0) + cimag(z0) * cimag(z0);
        if (!(e0 >= thr) || e0 == 0.0) continue;
        ++active;
        /* digit by digit: r = f mod 2^lo so far */
        int64_t r = 0;
        for (int64_t j = 0; j < J; ++j) {
            int64_t lo = j * b, m = (j + 1) * b < bits ? (j + 1) * b : bits;
            double complex zj = zhat[2 * ((j + 1) * B + k)] + I * zhat[2 * ((j + 1) * B + k) + 1];
            double complex rho_j = zj * conj(z0); /* |z0|^2 exp(2 pi i f / 2^m) for a lone f */
            int64_t best = 0;
            double bestv = -INFINITY;
            for (int64_t d = 0; d < ((int64_t)1 << (m - lo)); ++d) {
                int64_t cand = r + (d << lo);
                double v = creal(rho_j * unit_root(-cand * (N >> m), N));
                if (v > bestv) {
                    bestv = v;
                    best = d;
                }
            }
            r += best << lo;
        }
        /* p = sigma f mod N: the value with p = sigma r (mod W) in the window
           [k N/B - W/2, k N/B + W/2) */
        int64_t pr = mod_pos(sigma * r, W);
        int64_t lo_p = k * NB - W / 2;
        int64_t p = lo_p + mod_pos(pr - lo_p, W);
        int64_t f = mod_pos(sigma_inv * mod_pos(p, N), N);
        int64_t h, o;
        oracle_hash(N, B, sigma, f, &h, &o);
        if (h != k) continue; /* located in a neighbouring bucket: leakage */
        /* a lone coefficient: every shifted bucket is z0 turned by exp(2 pi i s_j f / N) */
        double res = 0.0;
        for (int64_t j = 1; j <= J; ++j) {
            double complex zj = zhat[2 * (j * B + k)] + I * zhat[2 * (j * B + k) + 1];
            double complex dlt = zj - z0 * unit_root(s[j] * f, N);
            res += creal(dlt) * creal(dlt) + cimag(dlt) * cimag(dlt);
        }
        if (res > rho * (double)J * e0) continue;
        double complex G = Gfull[2 * mod_pos(o, N)] + I * Gfull[2 * mod_pos(o, N) + 1];
        double complex v = z0 * conj(unit_root(tau * f, N)) / G; /* energy estimation */
        f_out[n] = (int32_t)f;
        v_out[2 * n] = creal(v);
        v_out[2 * n + 1] = cimag(v);
        ++n;
    }
    free(s);
    *active_out = active;
    return n;
}
static int flt_desc(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x < y) - (x > y);
}

int64_t oracle_sfft_bs(int64_t N, int64_t K, int64_t B, int64_t w, int R, int b, double eta, double kappa,
                       double rho, uint64_t seed, const double *g, const double *Gfull, const double *x,
                       int32_t *idx, double *val, int *iters_out, int64_t *nfound_out)
{
    if (!is_pow2(N) || N < 2 || !is_pow2(B) || B > N || w < B || w % B || R < 1 || K < 0 || b < 1 || b > 4)
        return -1;
    int64_t *sigma = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    int64_t *sinv = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    oracle_loop_params(N, R, seed, sigma, tau, sinv);
    int64_t S = oracle_bs_nshifts(N, B, b);
    int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
    oracle_bs_shifts(N, B, b, s);
    double *found = (double *)calloc(2 * (size_t)N, sizeof(double));
    char *seen = (char *)calloc((size_t)N, 1);
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *lval = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    int64_t nf = 0;
    double *z = (double *)malloc(sizeof(double) * 2 * (size_t)(S * B));
    int32_t *nfi = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
    double *nfv = (double *)malloc(sizeof(double) * 2 * (size_t)B);
    double thr = 0.0;
    int iters = 0;
    for (int r = 0; r < R; ++r) {
        for (int64_t c = 0; c < nf; ++c) {
            lval[2 * c] = found[2 * list[c]];
            lval[2 * c + 1] = found[2 * list[c] + 1];
        }
        /* bucketize at tau_r + s_j, minus the coefficients found so far */
        for (int64_t j = 0; j < S; ++j) {
            int64_t tj = mod_pos(tau[r] + s[j], N);
            oracle_bucketize(N, B, w, 1, &sigma[r], &tj, g, x, NULL, z + 2 * j * B);
            oracle_pe_subtract(N, B, sigma[r], tj, Gfull, nf, list, lval, z + 2 * j * B);
        }
        if (r == 0) {
            /* eta of the largest bucket energy, and at least kappa times the
               median one (the noise floor of a noisy signal; leakage-level
               for an exactly sparse one) */
            double emax = 0.0;
            float *ek = (float *)malloc(sizeof(float) * (size_t)B);
            for (int64_t k = 0; k < B; ++k) {
                double e = z[2 * k] * z[2 * k] + z[2 * k + 1] * z[2 * k + 1];
                if (e > emax) emax = e;
                ek[k] = (float)e;
            }
            qsort(ek, (size_t)B, sizeof(float), flt_desc);
            double emed = (double)ek[(B + 1) / 2 - 1]; /* the ceil(B/2)-th largest, as binary32 */
            free(ek);
            thr = eta * emax;
            if (kappa * emed > thr) thr = kappa * emed;
        }
        int64_t active = 0;
        int64_t n = oracle_bs_locate(N, B, b, sigma[r], sinv[r], tau[r], Gfull, z, thr, rho, nfi, nfv, &active);
        iters = r + 1;
        if (active == 0) break;
        for (int64_t c = 0; c < n; ++c) {
            int64_t f = nfi[c];
            found[2 * f] += nfv[2 * c];
            found[2 * f + 1] += nfv[2 * c + 1];
            if (!seen[f]) {
                seen[f] = 1;
                list[nf++] = (int32_t)f;
            }
        }
    }
    for (int64_t c = 0; c < nf; ++c) {
        lval[2 * c] = found[2 * list[c]];
        lval[2 * c + 1] = found[2 * list[c] + 1];
    }
    int64_t kout = oracle_topk(nf, list, lval, K, idx, val);
    if (iters_out) *iters_out = iters;
    if (nfound_out) *nfound_out = nf;
    free(sigma);
    free(tau);
    free(sinv);
    free(s);
    free(found);
    free(seen);
    free(list);
    free(lval);
    free(z);
    free(nfi);
    free(nfv);
    return kout;
}

/* ==================================================================
 * Final residual-energy check (problem statement, Eq. 5: the error left
 * after recovery).  Energy of every loop's buckets after the recovered
 * coefficients are subtracted by the exact bucket identity.
 * ================================================================== */

void oracle_residual_energy(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                            const double *Gfull, const double *zhat, int64_t n, const int32_t *idx,
                            const double *val, double *e_res, double *e_tot)
{
    double *r = (double *)malloc(sizeof(double) * 2 * (size_t)B);
    double er = 0.0, et = 0.0;
    for (int l = 0; l < L; ++l) {
        for (int64_t k = 0; k < 2 * B; ++k) r[k] = zhat[2 * (int64_t)l * B + k];
        for (int64_t k = 0; k < B; ++k) et += r[2 * k] * r[2 * k] + r[2 * k + 1] * r[2 * k + 1];
        oracle_pe_subtract(N, B, sigma[l], tau[l], Gfull, n, idx, val, r);
        for (int64_t k = 0; k < B; ++k) er += r[2 * k] * r[2 * k] + r[2 * k + 1] * r[2 * k + 1];
    }
    free(r);
    *e_res = er;
    *e_tot = et;
}
