/*
 * hp_oracle.c -- plain, slow CPU definition of the single-pulse search hot
 * path of Heimdall++ (arXiv 2512.00398), used ONLY as test infrastructure.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and
 * its --impl reference arm) may load this code.  The CUDA library never links,
 * includes or calls it, and it shares no code with the library.
 *
 * Every step follows the pipeline of Section II-B (stage list) and Algorithm 1
 * (per-trial loop: baseline removal, normalisation, matched filtering, peak
 * detection; then merging/clustering).  The paper names the stages but prints
 * no formulas except the DM integral (Eq. 1); the reading used where it is
 * silent is written out next to each function.
 *
 * Arithmetic: exact integers (int64) for every sum; FP64 for sigma, the
 * threshold and S/N.  Build with -ffp-contract=off so that no multiply-add
 * is fused (the decisions S >= thr*sigma*sqrt(W) must be reproducible).
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   hpo_delays            pinned: closed form, hand-worked values, invariants
 *   hpo_dedisperse_rows   pinned: impulse response, DM-0 channel sum, brute force
 *   hpo_remedian/baseline pinned: ramp reproduction, constant, spike rejection,
 *                                 brute-force recursion, monotone-input median
 *   hpo_baseline_mean     pinned: brute-force window mean
 *   hpo_mad               pinned: numpy sort median, Gaussian unit RMS
 *   hpo_detect_trial      pinned: naive window sums, rectangular pulse, brute-force runs
 *   hpo_merge             pinned: brute-force O(N^2) components, permutation invariance
 *   hpo_raw_snr           pinned: reproduces the S/N of every raw candidate a search
 *                                 found, hand-worked values
 *   hpo_subband_delays    pinned: two-stage brute force, S = 1 / G = 1 / S = nchans
 *                                 reductions, closed-form error bound
 *   hpo_width_sigma       pinned: numpy brute force, W = 1 reduction to the MAD,
 *                                 sqrt(W) law on white noise, random-walk growth,
 *                                 rectangular pulse S/N by hand
 *   decimated boxcars     pinned: numpy brute force on the scrunched series, R >= Wmax
 *                                 reduction to every start
 *   hpo_detect_window     pinned: brute-force runs with window and carry, whole-series
 *                                 window = plain detection, carry chains across gulps
 *   hpo_rfi_clean         pinned: an independent numpy formulation on small inputs,
 *                                 planted tones and spikes found exactly, clean noise and
 *                                 dispersed pulses left alone
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HPO_OK 0
#define HPO_ERR_ARG -1
#define HPO_ERR_OVERFLOW -4
#define HPO_ERR_SHORT -6

/* Cold-plasma dispersion constant, s MHz^2 pc^-1 cm^3. */
static const double HPO_KDM = 4148.808;
/* Consistency factor of the median absolute deviation for Gaussian noise,
 * 1 / Phi^-1(3/4). */
static const double HPO_MAD_TO_SIGMA = 1.482602218505602;

int hpo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Step c1: per-channel, per-trial delay in samples (Section II-B, Eq. 1 and
 * the cold-plasma law).  Channel c is at f_c = f_top + c*chan_bw MHz, the
 * reference frequency is f_top (so channel 0 has zero delay), and the delay
 * in seconds K*DM*(f_c^-2 - f_top^-2) is divided by tsamp and rounded to the
 * nearest integer, halves to even (rint).
 * ---------------------------------------------------------------------- */
int hpo_delays(int nchans, double f_top, double chan_bw, double tsamp,
               const float* dm_list, int ndm, int32_t* out /* [ndm][nchans] */) {
    if (nchans <= 0 || ndm <= 0 || !(tsamp > 0.0) || !(f_top > 0.0)) return HPO_ERR_ARG;
    double inv_top2 = 1.0 / (f_top * f_top);
    for (int d = 0; d < ndm; ++d) {
        double dm = (double)dm_list[d];
        for (int c = 0; c < nchans; ++c) {
            double f = f_top + (double)c * chan_bw;
            double sec = HPO_KDM * dm * (1.0 / (f * f) - inv_top2);
            out[(int64_t)d * nchans + c] = (int32_t)rint(sec / tsamp);
        }
    }
    return HPO_OK;
}

/* Largest delay of the table (the last usable input sample offset). */
int32_t hpo_max_delay(const int32_t* delays, int ndm, int nchans) {
    int32_t m = 0;
    for (int64_t i = 0; i < (int64_t)ndm * nchans; ++i)
        if (delays[i] > m) m = delays[i];
    return m;
}

/* ------------------------------------------------------------------------
 * Variant of step c2 that the paper does not use: two-stage (sub-band)
 * dedispersion, the classic way of trading sensitivity for work.  Channels
 * are cut into sub-bands of S consecutive channels (sub-band s = c / S, its
 * first, highest-frequency channel top(s) = s*S) and trials into groups of G
 * consecutive trials (group g = d / G, of size len(g) = min(G, ndm - g*G))
 * whose nominal trial is n(g) = g*G + (len(g) - 1) / 2.
 *   stage 1, per sub-band and group:
 *     B[s][g][u] = sum over c in s of x[u + delay(c,n(g)) - delay(top(s),n(g))][c]
 *   stage 2, per trial:
 *     D~[d][t]   = sum over s of B[s][g(d)][t + delay(top(s),d)]
 * Putting stage 1 into stage 2, D~ is direct dedispersion (step c2) with the
 * effective delay table
 *     e(c,d) = delay(top(s),d) + delay(c,n(g(d))) - delay(top(s),n(g(d))),
 * which this function writes; the variant's nout is nsamps - max e.  S = 1
 * or G = 1 give e = delay; S >= nchans gives e(c,d) = delay(c,n(g(d))).
 * ---------------------------------------------------------------------- */
int hpo_subband_delays(const int32_t* delays /* [ndm][nchans] */, int ndm, int nchans,
                       int S, int G, int32_t* out /* [ndm][nchans] */) {
    if (ndm <= 0 || nchans <= 0 || S < 1 || G < 1) return HPO_ERR_ARG;
    for (int d = 0; d < ndm; ++d) {
        int g = d / G;
        int len = ndm - g * G < G ? ndm - g * G : G;
        int n = g * G + (len - 1) / 2;
        const int32_t* at_d = delays + (int64_t)d * nchans;
        const int32_t* at_n = delays + (int64_t)n * nchans;
        for (int c = 0; c < nchans; ++c) {
            int top = (c / S) * S;
            out[(int64_t)d * nchans + c] = at_d[top] + at_n[c] - at_n[top];
        }
    }
    return HPO_OK;
}

/* ------------------------------------------------------------------------
 * Step c2: incoherent dedispersion (Section II-B): for every trial d and
 * output sample t in [0, nout), D[d][t] = sum_c x[t + delay(c,d)][c].
 * Only samples whose every term lies inside the input are produced
 * (nout = nsamps - max delay).  Rows d_begin..d_end-1 are written to
 * out[(d - d_begin)][t].  The sum is formed in int64 and must fit int32.
 * ---------------------------------------------------------------------- */
int hpo_dedisperse_rows(const uint8_t* x, int64_t nsamps, int nchans,
                        const int32_t* delays, int d_begin, int d_end,
                        int64_t nout, int32_t* out) {
    if (nout < 0 || d_end < d_begin) return HPO_ERR_ARG;
    int nrows = d_end - d_begin;
    const int64_t TB = 4096;
    int64_t ntb = (nout + TB - 1) / TB;
    int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic) reduction(| : bad)
    for (int r = 0; r < nrows; ++r) {
        for (int64_t tb = 0; tb < ntb; ++tb) {
            const int32_t* dl = delays + (int64_t)(d_begin + r) * nchans;
            int64_t t1 = (tb + 1) * TB < nout ? (tb + 1) * TB : nout;
            for (int64_t t = tb * TB; t < t1; ++t) {
                int64_t acc = 0;
                for (int c = 0; c < nchans; ++c) {
                    int64_t row = t + dl[c];
                    if (row < 0 || row >= nsamps) { bad = 1; continue; }
                    acc += x[row * nchans + c];
                }
                if (acc > INT32_MAX) bad = 1;
                out[(int64_t)r * nout + t] = (int32_t)acc;
            }
        }
    }
    return bad ? HPO_ERR_ARG : HPO_OK;
}

/* One dedispersed sample, for sampled checks of large runs. */
int64_t hpo_dedisperse_point(const uint8_t* x, int nchans, const int32_t* delay_row, int64_t t) {
    int64_t acc = 0;
    for (int c = 0; c < nchans; ++c) acc += x[(t + delay_row[c]) * nchans + c];
    return acc;
}

/* ------------------------------------------------------------------------
 * Helpers: exact lower median of r <= 5 values, floor division.
 * ---------------------------------------------------------------------- */
static int64_t lower_median_small(const int64_t* v, int r) {
    int64_t s[5];
    for (int i = 0; i < r; ++i) s[i] = v[i];
    for (int i = 1; i < r; ++i) {            /* insertion sort */
        int64_t key = s[i];
        int j = i - 1;
        while (j >= 0 && s[j] > key) { s[j + 1] = s[j]; --j; }
        s[j + 1] = key;
    }
    return s[(r - 1) / 2];
}

static int64_t floor_div(int64_t a, int64_t b) {     /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && (a < 0)) --q;
    return q;
}

/* Number of remedian levels for a window of `win` samples: the largest L with
 * 5^L <= win (integer form of floor(log5(win))). */
int hpo_remedian_levels(int64_t win) {
    int L = 0;
    int64_t p = 1;
    while (win >= 1 && p <= win / 5) { p *= 5; ++L; }
    return L;
}

/* ------------------------------------------------------------------------
 * Step c3 (median mode): baseline removal by a running median (Section II-B,
 * "Baseline Removal"; the paper only names a moving average, the running
 * median is the robust reading).  The running median is the remedian of
 * Rousseeuw & Bassett (1990): level 0 is the series, level l+1 holds the
 * medians of consecutive groups of five level-l values, a trailing group of
 * r < 5 values taking its lower median.  After L levels value m_j stands for
 * input samples [5^L j, 5^L (j+1)) and is placed at the centre
 * c_j = 5^L j + (5^L - 1)/2.
 * Writes the level-L values to m (capacity >= ceil(n / 5^L)) and returns
 * their count.
 * ---------------------------------------------------------------------- */
int64_t hpo_remedian(const int32_t* D, int64_t n, int L, int64_t* m) {
    if (n <= 0) return 0;
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!cur) return -1;
    for (int64_t i = 0; i < n; ++i) cur[i] = D[i];
    int64_t cn = n;
    for (int l = 0; l < L; ++l) {
        int64_t nn = (cn + 4) / 5;
        for (int64_t j = 0; j < nn; ++j) {
            int64_t a = 5 * j;
            int r = (int)((cn - a) < 5 ? (cn - a) : 5);
            cur[j] = lower_median_small(cur + a, r);   /* j <= a: in place is safe */
        }
        cn = nn;
    }
    memcpy(m, cur, sizeof(int64_t) * (size_t)cn);
    free(cur);
    return cn;
}

/* Baseline b(t) from the level-L values: linear between neighbouring centres,
 *   b(t) = m_j + floor((m_{j+1} - m_j) * (t - c_j) / 5^L)   for c_j <= t < c_{j+1},
 * held at m_0 before the first centre and at m_{M-1} after the last. */
int hpo_baseline_median(const int32_t* D, int64_t n, int L, int64_t* b) {
    if (n <= 0) return HPO_OK;
    int64_t P = 1;
    for (int l = 0; l < L; ++l) P *= 5;
    int64_t M = (n + P - 1) / P;
    int64_t* m = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    if (!m) return HPO_ERR_ARG;
    int64_t got = hpo_remedian(D, n, L, m);
    if (got != M) { free(m); return HPO_ERR_ARG; }
    int64_t half = (P - 1) / 2;
    int64_t c_first = half, c_last = P * (M - 1) + half;
    for (int64_t t = 0; t < n; ++t) {
        if (t <= c_first) { b[t] = m[0]; continue; }
        if (t >= c_last) { b[t] = m[M - 1]; continue; }
        int64_t j = (t - half) / P;                   /* c_j <= t < c_{j+1} */
        int64_t cj = P * j + half;
        b[t] = m[j] + floor_div((m[j + 1] - m[j]) * (t - cj), P);
    }
    free(m);
    return HPO_OK;
}

/* Step c3 (mean mode): the paper's "moving average subtraction" taken
 * literally: b(t) = floor( sum_{|i-t| <= H, 0 <= i < n} D[i] / count ). */
int hpo_baseline_mean(const int32_t* D, int64_t n, int64_t H, int64_t* b) {
    if (n <= 0) return HPO_OK;
    int64_t* pre = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!pre) return HPO_ERR_ARG;
    pre[0] = 0;
    for (int64_t i = 0; i < n; ++i) pre[i + 1] = pre[i] + D[i];
    for (int64_t t = 0; t < n; ++t) {
        int64_t lo = t - H < 0 ? 0 : t - H;
        int64_t hi = t + H > n - 1 ? n - 1 : t + H;
        b[t] = floor_div(pre[hi + 1] - pre[lo], hi - lo + 1);
    }
    free(pre);
    return HPO_OK;
}

/* ------------------------------------------------------------------------
 * Step c4: normalisation by a robust RMS (Section II-B, "Normalization").
 * MAD = lower median of |y| (element (n-1)/2 of the sorted values, exact);
 * sigma = 1.482602218505602 * MAD.
 * ---------------------------------------------------------------------- */
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int64_t hpo_mad(const int64_t* y, int64_t n) {
    if (n <= 0) return 0;
    int64_t* a = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!a) return -1;
    for (int64_t i = 0; i < n; ++i) a[i] = y[i] < 0 ? -y[i] : y[i];
    qsort(a, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t v = a[(n - 1) / 2];
    free(a);
    return v;
}

double hpo_sigma_from_mad(int64_t mad) { return HPO_MAD_TO_SIGMA * (double)mad; }

/* ------------------------------------------------------------------------
 * Variant of step c4 that the paper does not use (per-width normalisation,
 * as Heimdall does for its boxcar bank): every width W_k gets its own robust
 * sigma from the boxcar series itself,
 *   MAD_k = lower median of |S_k(t)| over the starts 0 <= t <= n - W_k,
 *   sigma_k = 1.482602218505602 * MAD_k,
 * with S_k(t) = sum_{i<W_k} y(t+i) as in step c5.  The threshold becomes
 * S >= thr * sigma_k and snr = S / sigma_k (no sqrt(W) scaling); sigma_k = 0
 * gives no candidates for that width.  On white noise sigma_k ~ sigma sqrt(W_k);
 * on correlated (red) noise sigma_k grows faster, which lowers false
 * detections at wide widths.  W_1 = 1 gives MAD_1 = MAD (step c4).
 * ---------------------------------------------------------------------- */
int hpo_width_sigma(const int64_t* y, int64_t n, const int32_t* widths, int nw,
                    int64_t* mad_w, double* sigma_w) {
    int64_t* a = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!a || !P) { free(a); free(P); return HPO_ERR_ARG; }
    P[0] = 0;
    for (int64_t i = 0; i < n; ++i) P[i + 1] = P[i] + y[i];
    for (int k = 0; k < nw; ++k) {
        int64_t W = widths[k];
        int64_t m = n - W + 1;          /* number of starts */
        int64_t mad = 0;
        if (m > 0) {
            for (int64_t t = 0; t < m; ++t) {
                int64_t S = P[t + W] - P[t];
                a[t] = S < 0 ? -S : S;
            }
            qsort(a, (size_t)m, sizeof(int64_t), cmp_i64);
            mad = a[(m - 1) / 2];
        }
        if (mad_w) mad_w[k] = mad;
        sigma_w[k] = HPO_MAD_TO_SIGMA * (double)mad;
    }
    free(a);
    free(P);
    return HPO_OK;
}

/* ------------------------------------------------------------------------
 * Steps c5 + c6: matched filtering by a boxcar bank and peak detection
 * (Section II-B, "Matched Filtering and Peak Detection").
 * For width W: S(t) = sum_{i=t}^{t+W-1} y(i), 0 <= t <= n - W (int64, formed
 * by differences of an exact prefix sum).  Sample t is above threshold iff
 * S(t) >= thr * sigma * sqrt(W) (FP64, products in that order).  Each maximal
 * run of consecutive above-threshold t gives one candidate at the argmax of
 * S over the run, ties to the smallest t.  snr = S / (sigma * sqrt(W)).
 * sigma == 0 gives no candidates.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t dm_idx;
    int32_t width_idx;
    int64_t sample;
    int64_t S;
    double snr;
} hpo_raw;

typedef struct {
    int32_t dm_idx;
    int32_t width_idx;
    int64_t sample;
    double snr;
    int32_t members;
    int32_t dm_lo;
    int32_t dm_hi;
    int32_t pad_;
    int64_t t_lo;
    int64_t t_hi;
} hpo_cluster;

typedef struct {
    hpo_raw* v;
    int64_t n, cap;
} raw_vec;

static int raw_push(raw_vec* rv, hpo_raw r) {
    if (rv->n == rv->cap) {
        int64_t nc = rv->cap ? 2 * rv->cap : 64;
        hpo_raw* nv = (hpo_raw*)realloc(rv->v, sizeof(hpo_raw) * (size_t)nc);
        if (!nv) return -1;
        rv->v = nv;
        rv->cap = nc;
    }
    rv->v[rv->n++] = r;
    return 0;
}

/* Decimated boxcars, a variant the paper does not use (Heimdall scrunches the
 * series for its wide boxcars): with a decimation R > 0, a width W > R that is
 * a multiple of R is evaluated only at the starts t = m q, q = W / R, which is
 * the boxcar of R samples on the series summed in blocks of q; its runs are
 * maximal sets of consecutive grid starts above threshold.  Other widths keep
 * every start (q = 1).  The sigmas are not changed by it. */
static int64_t decim_step(int64_t W, int R) { return (R > 0 && W > R && W % R == 0) ? W / R : 1; }

/* sigma_w: NULL for the paper's reading (one sigma per trial, scaled by
 * sqrt(W)), else the per-width sigmas of hpo_width_sigma: then the limit is
 * thr * sigma_w[k] and snr = S / sigma_w[k].  decimate: R of decim_step. */
static int detect_into(const int64_t* y, int64_t n, int d, double sigma,
                       const int32_t* widths, int nw, float thr, const double* sigma_w,
                       int decimate, raw_vec* rv) {
    if (!sigma_w && !(sigma > 0.0)) return 0;
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!P) return -1;
    P[0] = 0;
    for (int64_t i = 0; i < n; ++i) P[i + 1] = P[i] + y[i];
    double thr_d = (double)thr;
    for (int k = 0; k < nw; ++k) {
        int64_t W = widths[k];
        if (W > n) continue;
        if (sigma_w && !(sigma_w[k] > 0.0)) continue;
        double sw = sqrt((double)W);
        double lim = sigma_w ? thr_d * sigma_w[k] : thr_d * sigma * sw;
        int64_t last = n - W;
        int64_t q = decim_step(W, decimate);   /* start grid step */
        int64_t t = 0;
        while (t <= last) {
            int64_t S = P[t + W] - P[t];
            if ((double)S >= lim) {
                int64_t best_t = t, best_S = S;
                t += q;
                while (t <= last) {
                    int64_t S2 = P[t + W] - P[t];
                    if (!((double)S2 >= lim)) break;
                    if (S2 > best_S) { best_S = S2; best_t = t; }
                    t += q;
                }
                hpo_raw r;
                r.dm_idx = d;
                r.width_idx = k;
                r.sample = best_t;
                r.S = best_S;
                r.snr = sigma_w ? (double)best_S / sigma_w[k] : (double)best_S / (sigma * sw);
                if (raw_push(rv, r)) { free(P); return -1; }
            } else {
                t += q;
            }
        }
    }
    free(P);
    return 0;
}

/* S/N of raw candidates (step c5, the paper's reading: one sigma per trial,
 * scaled by sqrt(W)) from their exact sums and the per-trial sigmas: the same
 * FP64 expression as detect_into, snr = S / (sigma_d * sqrt(W)).  Used to
 * merge raw candidates that come with sums and sigmas only. */
void hpo_raw_snr(hpo_raw* c, int64_t n, const double* sigma, const int32_t* widths) {
    for (int64_t i = 0; i < n; ++i) {
        double sw = sqrt((double)widths[c[i].width_idx]);
        c[i].snr = (double)c[i].S / (sigma[c[i].dm_idx] * sw);
    }
}

/* Detection on one baseline-subtracted series y (length n) of trial d. */
int hpo_detect_trial(const int64_t* y, int64_t n, int d, double sigma,
                     const int32_t* widths, int nw, float thr,
                     hpo_raw* out, int64_t cap, int64_t* nout) {
    raw_vec rv = {0, 0, 0};
    if (detect_into(y, n, d, sigma, widths, nw, thr, NULL, 0, &rv)) { free(rv.v); return HPO_ERR_ARG; }
    *nout = rv.n;
    int64_t m = rv.n < cap ? rv.n : cap;
    if (m > 0) memcpy(out, rv.v, sizeof(hpo_raw) * (size_t)m);
    free(rv.v);
    return rv.n > cap ? HPO_ERR_OVERFLOW : HPO_OK;
}

/* ------------------------------------------------------------------------
 * Step c9a: detection inside one gulp's window (streamed search).
 * Section III-B explains that a long observation is searched chunk by chunk
 * and that neighbouring chunks must overlap in time to keep a dispersed
 * signal whole across a chunk boundary; Section V-C searches a long file in
 * chunks of 256K samples.  The paper gives no rule for the overlap or for
 * candidates near a boundary.  The reading used here (also in
 * hpo_search_window below): the searched buffer's boxcar starts [0, nwin)
 * form this gulp's window; later starts are look-ahead.  The runs of
 * above-threshold starts are found exactly as in hpo_detect_trial over every
 * valid start [0, n - W], and a run is reported iff its first start lies in
 * the window, unless it begins at start 0 while carry_in[k] says that the
 * previous window ended inside a run (that run was reported by the previous
 * gulp).  carry_out[k] = 1 iff start nwin - 1 is above threshold.  Reported
 * samples are shifted by t_offset (the buffer's first dedispersed sample in
 * the stream).
 * ---------------------------------------------------------------------- */
static int detect_window_into(const int64_t* y, int64_t n, int d, double sigma,
                              const int32_t* widths, int nw, float thr, int64_t nwin,
                              const uint8_t* carry_in, uint8_t* carry_out, int64_t t_offset,
                              const double* sigma_w, raw_vec* rv) {
    for (int k = 0; k < nw; ++k) carry_out[k] = 0;
    if (!sigma_w && !(sigma > 0.0)) return 0;
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!P) return -1;
    P[0] = 0;
    for (int64_t i = 0; i < n; ++i) P[i + 1] = P[i] + y[i];
    for (int k = 0; k < nw; ++k) {
        int64_t W = widths[k];
        if (W > n) continue;
        if (sigma_w && !(sigma_w[k] > 0.0)) continue;
        double lim = sigma_w ? (double)thr * sigma_w[k] : (double)thr * sigma * sqrt((double)W);
        int64_t last = n - W;
        if (nwin >= 1 && nwin - 1 <= last)
            carry_out[k] = (double)(P[nwin - 1 + W] - P[nwin - 1]) >= lim;
        int64_t t = 0;
        while (t <= last) {
            int64_t S = P[t + W] - P[t];
            if (!((double)S >= lim)) { ++t; continue; }
            int64_t first = t, best_t = t, best_S = S;
            for (++t; t <= last; ++t) {
                int64_t S2 = P[t + W] - P[t];
                if (!((double)S2 >= lim)) break;
                if (S2 > best_S) { best_S = S2; best_t = t; }
            }
            if (first >= nwin) break;                        /* past the window */
            if (first == 0 && carry_in && carry_in[k]) continue;   /* reported before */
            hpo_raw r;
            r.dm_idx = d;
            r.width_idx = k;
            r.sample = best_t + t_offset;
            r.S = best_S;
            r.snr = sigma_w ? (double)best_S / sigma_w[k] : (double)best_S / (sigma * sqrt((double)W));
            if (raw_push(rv, r)) { free(P); return -1; }
        }
    }
    free(P);
    return 0;
}

int hpo_detect_window(const int64_t* y, int64_t n, int d, double sigma, const int32_t* widths,
                      int nw, float thr, int64_t nwin, const uint8_t* carry_in,
                      uint8_t* carry_out, int64_t t_offset, hpo_raw* out, int64_t cap,
                      int64_t* nout) {
    raw_vec rv = {0, 0, 0};
    if (detect_window_into(y, n, d, sigma, widths, nw, thr, nwin, carry_in, carry_out, t_offset, NULL,
                           &rv)) {
        free(rv.v);
        return HPO_ERR_ARG;
    }
    *nout = rv.n;
    int64_t m = rv.n < cap ? rv.n : cap;
    if (m > 0) memcpy(out, rv.v, sizeof(hpo_raw) * (size_t)m);
    free(rv.v);
    return rv.n > cap ? HPO_ERR_OVERFLOW : HPO_OK;
}

/* ------------------------------------------------------------------------
 * Step c7: candidate merging and clustering (Section II-B, "Candate Merging
 * and Clustering"; Algorithm 1, last stage).  Candidates are ordered by
 * (dm_idx, sample, width_idx).  Two candidates are friends iff
 * |d_i - d_j| <= dm_tol, |k_i - k_j| <= w_tol and their windows
 * [t, t + W) lie within t_gap samples of each other:
 *   max(t_i, t_j) - min(t_i + W_i, t_j + W_j) <= t_gap.
 * Clusters are the connected components of the friendship graph.  Each
 * cluster reports its member with maximum snr (ties: smallest key), the member
 * count, the DM-index range and the time range [min t, max(t + W)).  Clusters
 * are listed in order of their smallest member key.
 * ---------------------------------------------------------------------- */
static int cmp_raw(const void* a, const void* b) {
    const hpo_raw* x = (const hpo_raw*)a;
    const hpo_raw* y = (const hpo_raw*)b;
    if (x->dm_idx != y->dm_idx) return x->dm_idx < y->dm_idx ? -1 : 1;
    if (x->sample != y->sample) return x->sample < y->sample ? -1 : 1;
    if (x->width_idx != y->width_idx) return x->width_idx < y->width_idx ? -1 : 1;
    return 0;
}

static int64_t uf_find(int64_t* parent, int64_t i) {
    while (parent[i] != i) {
        parent[i] = parent[parent[i]];
        i = parent[i];
    }
    return i;
}

static void uf_union(int64_t* parent, int64_t a, int64_t b) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) parent[b] = a; else parent[a] = b;   /* root = smallest index */
}

void hpo_sort_raw(hpo_raw* c, int64_t n) {
    if (n > 1) qsort(c, (size_t)n, sizeof(hpo_raw), cmp_raw);
}

int hpo_merge(hpo_raw* c /* sorted in place */, int64_t n, const int32_t* widths,
              int dm_tol, int64_t t_gap, int w_tol,
              hpo_cluster* out, int64_t cap, int64_t* nclusters) {
    *nclusters = 0;
    if (n <= 0) return HPO_OK;
    hpo_sort_raw(c, n);
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!parent) return HPO_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        int64_t ti = c[i].sample, ei = ti + widths[c[i].width_idx];
        for (int64_t j = i + 1; j < n && c[j].dm_idx <= c[i].dm_idx + dm_tol; ++j) {
            int dk = c[i].width_idx - c[j].width_idx;
            if (dk < 0) dk = -dk;
            if (dk > w_tol) continue;
            int64_t tj = c[j].sample, ej = tj + widths[c[j].width_idx];
            int64_t gap = (ti > tj ? ti : tj) - (ei < ej ? ei : ej);
            if (gap <= t_gap) uf_union(parent, i, j);
        }
    }
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!slot) { free(parent); return HPO_ERR_ARG; }
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = uf_find(parent, i);
        int64_t e = c[i].sample + widths[c[i].width_idx];
        if (r == i) {
            slot[i] = nc;
            if (nc < cap) {
                hpo_cluster* o = &out[nc];
                o->dm_idx = c[i].dm_idx;
                o->width_idx = c[i].width_idx;
                o->sample = c[i].sample;
                o->snr = c[i].snr;
                o->members = 1;
                o->dm_lo = o->dm_hi = c[i].dm_idx;
                o->pad_ = 0;
                o->t_lo = c[i].sample;
                o->t_hi = e;
            }
            ++nc;
        } else {
            int64_t s = slot[r];                    /* r < i: already assigned */
            if (s < cap) {
                hpo_cluster* o = &out[s];
                o->members += 1;
                if (c[i].dm_idx < o->dm_lo) o->dm_lo = c[i].dm_idx;
                if (c[i].dm_idx > o->dm_hi) o->dm_hi = c[i].dm_idx;
                if (c[i].sample < o->t_lo) o->t_lo = c[i].sample;
                if (e > o->t_hi) o->t_hi = e;
                if (c[i].snr > o->snr) {            /* strict: ties keep the earlier key */
                    o->dm_idx = c[i].dm_idx;
                    o->width_idx = c[i].width_idx;
                    o->sample = c[i].sample;
                    o->snr = c[i].snr;
                }
            }
        }
    }
    free(slot);
    free(parent);
    *nclusters = nc;
    return nc > cap ? HPO_ERR_OVERFLOW : HPO_OK;
}

/* ------------------------------------------------------------------------
 * The whole hot path for one filterbank (Algorithm 1 without RFI mitigation):
 * delays -> dedispersion -> per trial {baseline, MAD sigma, boxcars, peaks}
 * -> merge.  Trials run in parallel (OpenMP) only for speed; each trial is
 * independent, as Algorithm 1's per-thread split of the trial loop shows.
 *
 * baseline_mode: 0 = running median (remedian), 1 = moving mean.
 * Window: N = floor(baseline_s / tsamp + 0.5) samples; median mode uses
 * L = floor(log5 N) levels, mean mode the half-width H = floor(N/2).
 * Optional outputs (NULL to skip): sigma[ndm], mad[ndm].
 * ---------------------------------------------------------------------- */
typedef struct {
    int nchans;
    double f_top, chan_bw, tsamp;
    const float* dm_list;
    int ndm;
    const int32_t* widths;
    int nw;
    float thr;
    int baseline_mode;
    double baseline_s;
    int dm_tol;
    int64_t t_gap;
    int w_tol;
    int subband_chans;   /* S of the sub-band variant; 0 = direct dedispersion */
    int subband_group;   /* G of the sub-band variant */
    int width_sigma;     /* 1 = per-width sigmas (hpo_width_sigma) */
    int decimate;        /* R of the decimated boxcars (decim_step); 0 = every start */
} hpo_params;

/* The delay table a search dedisperses with: step c1's, or the sub-band
 * variant's effective table when subband_chans > 0. */
static int search_delays(const hpo_params* p, int32_t* delays) {
    int rc = hpo_delays(p->nchans, p->f_top, p->chan_bw, p->tsamp, p->dm_list, p->ndm, delays);
    if (rc || p->subband_chans <= 0) return rc;
    size_t n = (size_t)p->ndm * (size_t)p->nchans;
    int32_t* e = (int32_t*)malloc(sizeof(int32_t) * n);
    if (!e) return HPO_ERR_ARG;
    rc = hpo_subband_delays(delays, p->ndm, p->nchans, p->subband_chans, p->subband_group, e);
    if (!rc) memcpy(delays, e, sizeof(int32_t) * n);
    free(e);
    return rc;
}

int64_t hpo_baseline_window(double baseline_s, double tsamp) {
    return (int64_t)floor(baseline_s / tsamp + 0.5);
}

/* Baseline-subtracted series of one trial: y = D - b. */
int hpo_subtract_baseline(const int32_t* D, int64_t n, int baseline_mode, int64_t win,
                          int64_t* y) {
    int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!b) return HPO_ERR_ARG;
    int rc = baseline_mode == 0 ? hpo_baseline_median(D, n, hpo_remedian_levels(win), b)
                                : hpo_baseline_mean(D, n, win / 2, b);
    if (rc == HPO_OK)
        for (int64_t t = 0; t < n; ++t) y[t] = (int64_t)D[t] - b[t];
    free(b);
    return rc;
}

/* Per-trial stage of Algorithm 1 on an already dedispersed block of rows. */
int hpo_search_trials(const int32_t* D /* [nrows][nout] */, int64_t nout, int d_begin, int nrows,
                      const hpo_params* p, hpo_raw* raw, int64_t raw_cap, int64_t* nraw,
                      double* sigma_out, int64_t* mad_out) {
    int64_t win = hpo_baseline_window(p->baseline_s, p->tsamp);
    raw_vec* per = (raw_vec*)calloc((size_t)nrows, sizeof(raw_vec));
    if (!per) return HPO_ERR_ARG;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int r = 0; r < nrows; ++r) {
        int64_t* y = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nout > 0 ? nout : 1));
        if (!y) { bad = 1; continue; }
        if (hpo_subtract_baseline(D + (int64_t)r * nout, nout, p->baseline_mode, win, y)) bad = 1;
        int64_t mad = hpo_mad(y, nout);
        double sigma = hpo_sigma_from_mad(mad);
        if (sigma_out) sigma_out[r] = sigma;
        if (mad_out) mad_out[r] = mad;
        double* sw = NULL;
        if (p->width_sigma) {
            sw = (double*)malloc(sizeof(double) * (size_t)(p->nw > 0 ? p->nw : 1));
            if (!sw || hpo_width_sigma(y, nout, p->widths, p->nw, NULL, sw)) bad = 1;
        }
        if (!bad && detect_into(y, nout, d_begin + r, sigma, p->widths, p->nw, p->thr, sw,
                                p->decimate, &per[r]))
            bad = 1;
        free(sw);
        free(y);
    }
    int64_t tot = 0;
    for (int r = 0; r < nrows; ++r) {
        for (int64_t i = 0; i < per[r].n; ++i) {
            if (tot < raw_cap) raw[tot] = per[r].v[i];
            ++tot;
        }
        free(per[r].v);
    }
    free(per);
    *nraw = tot;
    if (bad) return HPO_ERR_ARG;
    return tot > raw_cap ? HPO_ERR_OVERFLOW : HPO_OK;
}

int hpo_search(const uint8_t* x, int64_t nsamps, const hpo_params* p,
               hpo_raw* raw, int64_t raw_cap, int64_t* nraw,
               hpo_cluster* cl, int64_t cl_cap, int64_t* ncl,
               double* sigma_out, int64_t* mad_out) {
    *nraw = 0;
    *ncl = 0;
    int32_t* delays = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->ndm * (size_t)p->nchans);
    if (!delays) return HPO_ERR_ARG;
    int rc = search_delays(p, delays);
    if (rc) { free(delays); return rc; }
    int32_t maxd = hpo_max_delay(delays, p->ndm, p->nchans);
    int wmax = 0;
    for (int k = 0; k < p->nw; ++k) if (p->widths[k] > wmax) wmax = p->widths[k];
    if (nsamps <= (int64_t)maxd + wmax) { free(delays); return HPO_ERR_SHORT; }
    int64_t nout = nsamps - maxd;
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->ndm * (size_t)nout);
    if (!D) { free(delays); return HPO_ERR_ARG; }
    rc = hpo_dedisperse_rows(x, nsamps, p->nchans, delays, 0, p->ndm, nout, D);
    free(delays);
    if (rc) { free(D); return rc; }
    rc = hpo_search_trials(D, nout, 0, p->ndm, p, raw, raw_cap, nraw, sigma_out, mad_out);
    free(D);
    if (rc) return rc;
    return hpo_merge(raw, *nraw, p->widths, p->dm_tol, p->t_gap, p->w_tol, cl, cl_cap, ncl);
}

/* ------------------------------------------------------------------------
 * Step c9b: one gulp of a streamed search (Sections III-B, V-C; reading as
 * in detect_window_into).  x holds the searched buffer: input samples
 * [B0, E) of the beam, nsamps = E - B0 = nwin + maxd + Wmax - 1 (or fewer
 * leading samples for the first gulps, B0 = 0).  The buffer is searched as a
 * plain series (dedispersion, per-trial baseline, MAD sigma, boxcars), runs
 * are kept by the window rule, samples are shifted by t_offset = B0, and the
 * gulp's raw candidates are merged on their own.  carry_in / carry_out are
 * [ndm][nw] flags (carry_in may be NULL for the first searched gulp).
 * ---------------------------------------------------------------------- */
int hpo_search_window(const uint8_t* x, int64_t nsamps, const hpo_params* p, int64_t nwin,
                      int64_t t_offset, const uint8_t* carry_in, uint8_t* carry_out,
                      hpo_raw* raw, int64_t raw_cap, int64_t* nraw,
                      hpo_cluster* cl, int64_t cl_cap, int64_t* ncl) {
    *nraw = 0;
    *ncl = 0;
    int32_t* delays = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->ndm * (size_t)p->nchans);
    if (!delays) return HPO_ERR_ARG;
    int rc = search_delays(p, delays);
    if (rc) { free(delays); return rc; }
    int32_t maxd = hpo_max_delay(delays, p->ndm, p->nchans);
    int wmax = 0;
    for (int k = 0; k < p->nw; ++k) if (p->widths[k] > wmax) wmax = p->widths[k];
    int64_t nout = nsamps - maxd;
    if (nwin < 1 || nout != nwin + wmax - 1) { free(delays); return HPO_ERR_ARG; }
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->ndm * (size_t)nout);
    if (!D) { free(delays); return HPO_ERR_ARG; }
    rc = hpo_dedisperse_rows(x, nsamps, p->nchans, delays, 0, p->ndm, nout, D);
    free(delays);
    if (rc) { free(D); return rc; }
    int64_t win = hpo_baseline_window(p->baseline_s, p->tsamp);
    raw_vec* per = (raw_vec*)calloc((size_t)p->ndm, sizeof(raw_vec));
    if (!per) { free(D); return HPO_ERR_ARG; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int d = 0; d < p->ndm; ++d) {
        int64_t* y = (int64_t*)malloc(sizeof(int64_t) * (size_t)nout);
        if (!y) { bad = 1; continue; }
        if (hpo_subtract_baseline(D + (int64_t)d * nout, nout, p->baseline_mode, win, y)) bad = 1;
        double sigma = hpo_sigma_from_mad(hpo_mad(y, nout));
        double* sw = NULL;
        if (p->width_sigma) {
            sw = (double*)malloc(sizeof(double) * (size_t)(p->nw > 0 ? p->nw : 1));
            if (!sw || hpo_width_sigma(y, nout, p->widths, p->nw, NULL, sw)) bad = 1;
        }
        if (!bad && detect_window_into(y, nout, d, sigma, p->widths, p->nw, p->thr, nwin,
                                       carry_in ? carry_in + (int64_t)d * p->nw : NULL,
                                       carry_out + (int64_t)d * p->nw, t_offset, sw, &per[d]))
            bad = 1;
        free(sw);
        free(y);
    }
    free(D);
    int64_t tot = 0;
    for (int d = 0; d < p->ndm; ++d) {
        for (int64_t i = 0; i < per[d].n; ++i) {
            if (tot < raw_cap) raw[tot] = per[d].v[i];
            ++tot;
        }
        free(per[d].v);
    }
    free(per);
    *nraw = tot;
    if (bad) return HPO_ERR_ARG;
    if (tot > raw_cap) return HPO_ERR_OVERFLOW;
    return hpo_merge(raw, tot, p->widths, p->dm_tol, p->t_gap, p->w_tol, cl, cl_cap, ncl);
}

/* ------------------------------------------------------------------------
 * Step c0: RFI mitigation before dedispersion (Section II-B "RFI
 * Mitigation": broadband interference spans all channels, narrowband
 * interference a few; corrupted regions are masked.  Section III-C: broadband
 * RFI is found on the DM = 0 series, since it is not dispersed).  The paper
 * gives no statistic or threshold; the reading used here:
 *   - per channel c, m_c = lower median of x[.][c] and s_c = lower median of
 *     |x[.][c] - m_c| over all samples (exact, by counting the 256 values);
 *   - across channels, M_m = lower median of m_c, D_m = lower median of
 *     |m_c - M_m| (likewise M_s, D_s for s_c); channel c is narrowband RFI iff
 *     |m_c - M_m| > nb_k * max(D_m, 1) or |s_c - M_s| > nb_k * max(D_s, 1);
 *   - z[t] = sum over channels of x[t][c], with flagged channels taking m_c;
 *     y = z - baseline(z) (the search's baseline, step c3), sigma_z =
 *     1.482602218505602 * median|y| (step c4); sample t is broadband RFI iff
 *     |y[t]| >= bb_k * sigma_z (FP64; never when sigma_z = 0);
 *   - out[t][c] = m_c where channel c or sample t is flagged, else x[t][c].
 * ---------------------------------------------------------------------- */
static int32_t median_of_counts(const int64_t* h, int nbins, int64_t n) {
    /* lower median (element (n-1)/2 of the sorted values) from value counts */
    int64_t k = (n - 1) / 2, c = 0;
    for (int v = 0; v < nbins; ++v) {
        c += h[v];
        if (c > k) return v;
    }
    return nbins - 1;
}

int hpo_rfi_clean(const uint8_t* x, int64_t nsamps, int nchans, int nb_k, float bb_k,
                  int baseline_mode, double baseline_s, double tsamp, uint8_t* out,
                  uint8_t* chan_flag, uint8_t* samp_flag, int32_t* chan_median,
                  double* sigma_z) {
    if (nsamps < 1 || nchans < 1 || nb_k < 0 || !(bb_k > 0.0f)) return HPO_ERR_ARG;
    int32_t* m = (int32_t*)malloc(sizeof(int32_t) * (size_t)nchans);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)nchans);
    int32_t* z = (int32_t*)malloc(sizeof(int32_t) * (size_t)nsamps);
    int64_t* y = (int64_t*)malloc(sizeof(int64_t) * (size_t)nsamps);
    if (!m || !s || !z || !y) { free(m); free(s); free(z); free(y); return HPO_ERR_ARG; }
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < nchans; ++c) {
        int64_t h[256] = {0}, ha[256] = {0};
        for (int64_t t = 0; t < nsamps; ++t) h[x[t * nchans + c]]++;
        m[c] = median_of_counts(h, 256, nsamps);
        for (int v = 0; v < 256; ++v) ha[v > m[c] ? v - m[c] : m[c] - v] += h[v];
        s[c] = median_of_counts(ha, 256, nsamps);
    }
    int64_t hm[256] = {0}, hs[256] = {0}, hdm[256] = {0}, hds[256] = {0};
    for (int c = 0; c < nchans; ++c) { hm[m[c]]++; hs[s[c]]++; }
    const int32_t Mm = median_of_counts(hm, 256, nchans), Ms = median_of_counts(hs, 256, nchans);
    for (int c = 0; c < nchans; ++c) {
        hdm[m[c] > Mm ? m[c] - Mm : Mm - m[c]]++;
        hds[s[c] > Ms ? s[c] - Ms : Ms - s[c]]++;
    }
    const int64_t Dm = median_of_counts(hdm, 256, nchans), Ds = median_of_counts(hds, 256, nchans);
    for (int c = 0; c < nchans; ++c) {
        const int64_t dm = m[c] > Mm ? m[c] - Mm : Mm - m[c];
        const int64_t ds = s[c] > Ms ? s[c] - Ms : Ms - s[c];
        chan_flag[c] = dm > (int64_t)nb_k * (Dm > 1 ? Dm : 1) ||
                       ds > (int64_t)nb_k * (Ds > 1 ? Ds : 1);
        if (chan_median) chan_median[c] = m[c];
    }
#pragma omp parallel for
    for (int64_t t = 0; t < nsamps; ++t) {
        int64_t acc = 0;
        for (int c = 0; c < nchans; ++c) acc += chan_flag[c] ? m[c] : x[t * nchans + c];
        z[t] = (int32_t)acc;
    }
    int rc = hpo_subtract_baseline(z, nsamps, baseline_mode,
                                   hpo_baseline_window(baseline_s, tsamp), y);
    double sg = 0.0;
    if (!rc) {
        sg = hpo_sigma_from_mad(hpo_mad(y, nsamps));
#pragma omp parallel for
        for (int64_t t = 0; t < nsamps; ++t) {
            const int64_t a = y[t] < 0 ? -y[t] : y[t];
            samp_flag[t] = sg > 0.0 && (double)a >= (double)bb_k * sg;
            for (int c = 0; c < nchans; ++c)
                out[t * nchans + c] = (chan_flag[c] || samp_flag[t]) ? (uint8_t)m[c]
                                                                    : x[t * nchans + c];
        }
    }
    if (sigma_z) *sigma_z = sg;
    free(m); free(s); free(z); free(y);
    return rc ? HPO_ERR_ARG : HPO_OK;
}
