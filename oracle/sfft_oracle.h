/*
 * FP64 CPU oracle for the flat-window voting sparse FFT (sFFT1.0-style), its
 * phase-encoding, iterative variant (sFFT3.0-style), the spike-train
 * pre-filter in front of voting (sFFT2.0-style), the averaging estimator,
 * the iterative-framework refinement of the voting output, the location
 * by binary or multi-scale search (sFFT4.0 / MPFFT-style), and the final
 * residual-energy check.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link or
 * call this code: only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA implementation.
 *
 * Every routine is a plain, slow restatement of one step of the method, in the
 * order the paper describes it ("Empirical Evaluation of Typical Sparse Fast
 * Fourier Transform Algorithms", arXiv:2012.08238):
 *   Eq. 2          forward DFT with the 1/N factor (oracle_dft)
 *   Eq. 6-7        time shift / time scaling -> the permuted gather
 *   Eq. 11         time-domain aliasing (fold into B buckets)
 *   Eq. 12-13      flat window = sinc x Gaussian (oracle_window_taps)
 *   Eq. 14         flat-filter bucket composition, rounding rule of the
 *                  worked example (oracle_hash)
 *   "Method of probability and statistics": top-2K buckets + voting
 *   "Energy concentration method": per-loop estimate, combined by median
 *                  (or by the mean: oracle_estimate_ex)
 *   "Scaling method": random odd sigma
 *   Table 2        sampling complexity (oracle_samples_touched)
 *
 * Conventions.  Complex arrays are interleaved (re, im) doubles.  Window index
 * q in [0, w) stands for window position m = q - w/2.  Loop parameters are
 * sigma (odd), tau, and sigma^-1 mod N.  All indices are int64.
 */
#ifndef SFFT_ORACLE_H
#define SFFT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x64-10 block (Salmon et al., SC'11): 4x64-bit counter, 2x64 key. */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Per-loop parameters: block = Philox(ctr=(l,0,0,0), key=(seed,0));
   sigma_l = 2*(out0 mod N/2) + 1, tau_l = out1 mod N, sigma_inv_l by the
   extended Euclidean algorithm.  Returns 0, or -1 if N is not a power of two
   >= 2. */
int oracle_loop_params(int64_t N, int L, uint64_t seed, int64_t *sigma, int64_t *tau,
                       int64_t *sigma_inv);

/* Multiplicative inverse of odd a modulo N (power of two), extended Euclid. */
int64_t oracle_modinv(int64_t a, int64_t N);

/* Eq. 12 x Eq. 13 taps g[q], q in [0,w). */
void oracle_window_taps(int64_t N, int64_t B, int64_t w, double *g);

/* Flat-filter gain G~(o) = sum_m g(m) exp(+2 pi i m o / N) for one offset o. */
void oracle_filter_gain_at(int64_t N, int64_t w, const double *g, int64_t o, double out[2]);

/* All N/B gains, o in [-N/2B, N/2B) stored at index o + N/2B. */
void oracle_filter_gain(int64_t N, int64_t B, int64_t w, const double *g, double *Gt);

/* Flat-filter hash (Eq. 14 rounding): p = sigma f mod N,
   h = round_half_up(p B / N) mod B, o = p - round_half_up(p B / N) * N/B. */
void oracle_hash(int64_t N, int64_t B, int64_t sigma, int64_t f, int64_t *h, int64_t *o);

/* out[m'] = x[(sigma m' + tau) mod N] for m' in [0, N): Eq. 6-7 composed. */
void oracle_permute(int64_t N, int64_t sigma, int64_t tau, const double *x, double *out);

/* Steps a1+a2: z[l][j] (fold of the windowed permuted signal, Eq. 11) and
   zhat[l][k] = sum_j z[l][j] exp(-2 pi i j k / B).  z may be NULL. */
void oracle_bucketize(int64_t N, int64_t B, int64_t w, int L, const int64_t *sigma,
                      const int64_t *tau, const double *g, const double *x, double *z,
                      double *zhat);

/* Step a3: the cK buckets of one loop with largest |zhat|^2 (key rounded to
   binary32), ties to the lower bucket.  Writes min(cK, B) indices in rank
   order and returns that count. */
int64_t oracle_select(int64_t B, int64_t cK, const double *zhat_loop, int32_t *sel);

/* Steps a4+a5: explicit score[N] histogram of hashed-back votes; writes the
   candidates {f : score >= T} in increasing f and returns their count.
   sel is [L][nsel]. score may be NULL (then allocated internally). */
int64_t oracle_vote(int64_t N, int64_t B, int L, int64_t nsel, int T, const int64_t *sigma_inv,
                    const int32_t *sel, int32_t *score, int32_t *cand);

/* Step a6: v_l(f) = zhat_l[h_l(f)] exp(-2 pi i tau_l f / N) / G~(o_l(f)),
   combined by coordinate-wise median (even L: mean of the two middle values).
   per_loop ([ncand][L] complex) may be NULL. */
void oracle_estimate(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                     const double *Gt, const double *zhat, int64_t ncand, const int32_t *cand,
                     double *est, double *per_loop);

/* Combinations of the L per-loop estimates: the coordinate-wise median
   (sFFT1.0's robust choice), or their mean ("the average value of multiple
   buckets is more accurate", § "The method of estimating the value"). */
#define ORACLE_MEDIAN 0
#define ORACLE_MEAN 1

/* oracle_estimate with the combination chosen by combine. */
void oracle_estimate_ex(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                        const double *Gt, const double *zhat, int64_t ncand, const int32_t *cand,
                        int combine, double *est, double *per_loop);

/* Step a7: the K candidates with largest |est|^2 (key rounded to binary32),
   ties to the lower f, returned sorted by f.  Returns min(K, ncand). */
int64_t oracle_topk(int64_t ncand, const int32_t *cand, const double *est, int64_t K,
                    int32_t *idx, double *val);

/* Distinct sample indices touched by all L loops (Table 2 sampling). */
int64_t oracle_samples_touched(int64_t N, int64_t w, int L, const int64_t *sigma,
                               const int64_t *tau);

/* Eq. 2: xhat_i = (1/N) sum_j x_j exp(-2 pi i i j / N), O(N^2). */
void oracle_dft(int64_t N, const double *x, double *xhat);

/* Whole pipeline a0..a7 for one signal.  g (w taps) and Gt (N/B gains) come
   from oracle_window_taps / oracle_filter_gain.  Intermediates may be NULL:
   zhat [L][B] complex, sel [L][min(cK,B)], cand/est (capacity N).
   Returns k_out = min(K, |I|), or -1 on invalid parameters. */
int64_t oracle_sfft(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T,
                    uint64_t seed, const double *g, const double *Gt, const double *x,
                    int32_t *idx, double *val, double *zhat_out, int32_t *sel_out,
                    int32_t *cand_out, double *est_out, int64_t *ncand_out);

/* oracle_sfft with the a6 combination chosen by combine (ORACLE_MEDIAN or
   ORACLE_MEAN). */
int64_t oracle_sfft_ex(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T,
                       uint64_t seed, const double *g, const double *Gt, const double *x, int combine,
                       int32_t *idx, double *val, double *zhat_out, int32_t *sel_out,
                       int32_t *cand_out, double *est_out, int64_t *ncand_out);

/* ---- sFFT3.0-style phase-encoding location, iterative framework ---- */

/* G~(nu) for every offset nu in [0, N) (nu and nu - N name the same offset):
   Gfull[nu] = sum_m g(m) exp(+2 pi i m nu / N), one length-N radix-2 FFT of
   the zero-padded window. */
void oracle_filter_gain_full(int64_t N, int64_t w, const double *g, double *Gfull);

/* The iterative framework's subtraction: removes from the B bucket values of
   one bucketization (sigma, tau) the contributions of nf known coefficients
   (fidx, fval complex), by the exact identity
   zhat[k] = sum_f x^_f exp(+2 pi i tau f / N) G~(sigma f - k N/B). */
void oracle_pe_subtract(int64_t N, int64_t B, int64_t sigma, int64_t tau, const double *Gfull, int64_t nf,
                        const int32_t *fidx, const double *fval, double *zhat);

/* Phase-encoding location ("Phase encoding method"): for every bucket k with
   |zhat0[k]|^2 >= thr (and > 0) -- counted in *active_out -- the time shift
   by one sample turns a lone coefficient f by exp(+2 pi i f / N), so
   f = round(arg(zhat1[k] conj(zhat0[k])) N / 2 pi) mod N; f is kept when it
   hashes back to bucket k, valued zhat0[k] exp(-2 pi i tau f / N) / G~(o).
   Writes the kept (f, value) pairs and returns their number. */
int64_t oracle_pe_locate(int64_t N, int64_t B, int64_t sigma, int64_t tau, const double *Gfull,
                         const double *zhat0, const double *zhat1, double thr, int32_t *f_out,
                         double *v_out, int64_t *active_out);

/* Whole sFFT3.0-style pipeline for one exactly sparse signal.  Iteration r
   uses loop parameters r (oracle_loop_params(N, R, seed)) and bucketizes the
   signal at shifts tau_r and tau_r + 1; the coefficients found so far are
   subtracted from both; the located (f, value) pairs are added to the found
   set (values of a frequency found again accumulate).  The threshold is eta
   times the largest bucket energy of iteration 0; the loop stops after R
   iterations or when no bucket reaches it.  Output: the K found coefficients
   of largest magnitude (ties to the lower f), sorted by f.  Returns k_out, or
   -1 on invalid parameters. */
int64_t oracle_sfft_pe(int64_t N, int64_t K, int64_t B, int64_t w, int R, double eta, uint64_t seed,
                       const double *g, const double *Gfull, const double *x, int32_t *idx, double *val,
                       int *iters_out, int64_t *nfound_out);

/* ---- sFFT2.0-style spike-train pre-filter ---- */

/* Residue classes kept by the spike-train filter.  Comb c samples the signal
   at x[(tau_c[c] + j N/Bc) mod N], j < Bc (Eq. 10 at a shift); its Bc-point
   DFT with 1/Bc gives y_c[i] = sum over f = i (mod Bc) of x^_f e^{+2 pi i tau_c f/N}
   (Eq. 16); E[i] = sum_c |y_c[i]|^2.  kept[i] = 1 for the nkeep classes of
   largest E (key rounded to binary32, ties to the lower class).  Returns the
   number kept. */
int64_t oracle_comb(int64_t N, int64_t Bc, int C, const int64_t *tau_c, int64_t nkeep, const double *x,
                    uint8_t *kept, double *E);

/* Voting pipeline behind the spike-train pre-filter (sFFT2.0-style): loop
   parameters 0..L-1 vote as in oracle_sfft; loops L..L+C-1 give the comb
   shifts; min(cK, Bc) residue classes are kept; a frequency is a candidate
   when its score reaches T and its class f mod Bc is kept.  Estimate and
   top-K as in oracle_sfft.  kept_out (Bc bytes) may be NULL.  Returns k_out,
   or -1 on invalid parameters. */
int64_t oracle_sfft2(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T, int64_t Bc, int C,
                     uint64_t seed, const double *g, const double *Gt, const double *x, int32_t *idx, double *val,
                     uint8_t *kept_out, int64_t *ncand_out);

/* oracle_sfft2 with the a6 combination chosen by combine. */
int64_t oracle_sfft2_ex(int64_t N, int64_t K, int64_t B, int64_t w, int L, int c, int T, int64_t Bc, int C,
                        uint64_t seed, const double *g, const double *Gt, const double *x, int combine,
                        int32_t *idx, double *val, uint8_t *kept_out, int64_t *ncand_out, double *zhat_out);

/* Iterative-framework refinement of the n found coefficients idx[] with
   values val[] (in: the pipeline's estimates; out: refined).  Each of the
   passes re-estimates every found f in every loop from its bucket
   zhat_l[h_l(f)] after subtracting the other found coefficients by the exact
   bucket identity (Gfull: G~ at every offset, oracle_filter_gain_full), using
   the previous pass's values, and combines the L estimates by combine. */
void oracle_refine(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau, const double *Gfull,
                   const double *zhat, int64_t n, const int32_t *idx, int combine, int passes, double *val);

/* ---- sFFT4.0 / MPFFT-style location by binary or multi-scale search ---- */

/* Number of bucketizations per iteration, 1 + ceil(bits / b) with bits =
   min(log2(N/B) + 1, log2 N), and their shifts s[0] = 0, s[j+1] =
   N / 2^min((j+1) b, bits): search step j decides digit j (b bits, the last
   one possibly fewer) of f. */
int64_t oracle_bs_nshifts(int64_t N, int64_t B, int b);
void oracle_bs_shifts(int64_t N, int64_t B, int b, int64_t *s);

/* Location in the buckets of one loop (zhat: the nshifts bucketizations,
   row j at tau + s[j]).  For a bucket with |zhat_0[k]|^2 >= thr, digit j of f
   is the d whose predicted turn exp(2 pi i (r + d 2^(jb)) s_j / N) best
   matches zhat_j[k] conj(zhat_0[k]) (largest real part of their product;
   r: the lower digits).  The bits fix p = sigma f modulo W = 2^bits: p is
   the one value with p = sigma r (mod W) in [k N/B - W/2, k N/B + W/2) and
   f = sigma^-1 p.  Kept when f hashes back to bucket k (else the bucket only
   holds a neighbour's leakage) and sum_j |zhat_j[k] - zhat_0[k]
   exp(2 pi i s_j f / N)|^2 <= rho (nshifts - 1) |zhat_0[k]|^2 (a lone
   coefficient), valued zhat_0[k] exp(-2 pi i tau f/N) / G~(o).  Returns the
   number kept; *active_out = buckets above thr. */
int64_t oracle_bs_locate(int64_t N, int64_t B, int b, int64_t sigma, int64_t sigma_inv, int64_t tau,
                         const double *Gfull, const double *zhat, double thr, double rho, int32_t *f_out,
                         double *v_out, int64_t *active_out);

/* Whole pipeline: as oracle_sfft_pe (iterations r with loop parameters r,
   subtraction of the found set, accumulation of values found again, top K),
   with the location by search in radix 2^b (b = 1: binary search; b > 1:
   multi-scale search) over the shifts tau_r + s[j].  Threshold: the larger
   of eta times the largest and kappa times the median (the ceil(B/2)-th
   largest, as binary32) bucket energy of iteration 0. */
int64_t oracle_sfft_bs(int64_t N, int64_t K, int64_t B, int64_t w, int R, int b, double eta, double kappa,
                       double rho, uint64_t seed, const double *g, const double *Gfull, const double *x,
                       int32_t *idx, double *val, int *iters_out, int64_t *nfound_out);

/* ---- final residual-energy check (Eq. 5, problem statement) ---- */

/* Energy left in the L loops' bucket values zhat ([L][B] complex) after the
   n recovered coefficients (idx, val complex) are subtracted from every
   bucket of every loop by the exact identity of oracle_pe_subtract:
   *e_res = sum_l sum_k |zhat_l[k] - sum_f v_f e^{+2 pi i tau_l f / N}
   G~(sigma_l f - k N/B)|^2; *e_tot = sum_l sum_k |zhat_l[k]|^2. */
void oracle_residual_energy(int64_t N, int64_t B, int L, const int64_t *sigma, const int64_t *tau,
                            const double *Gfull, const double *zhat, int64_t n, const int32_t *idx,
                            const double *val, double *e_res, double *e_tot);

#ifdef __cplusplus
}
#endif
#endif
