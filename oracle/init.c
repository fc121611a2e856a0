/*
 * Initialisation: log-matched filter, peak picking and the initial point cloud.
 * TEST INFRASTRUCTURE ONLY -- see rt3d_oracle.h.
 *
 * The paper initialises every pixel independently and in parallel (Methods,
 * "3D Reconstruction algorithm"); the details are in its Supplementary Note 3,
 * which is not available.  The reading implemented here:
 *   1. a log-matched filter: correlate the histogram with
 *      K_s = round(2^f log(1 + h_s / delta)),  delta = delta_rel max_s h_s,
 *      the log-likelihood of a single return over a background floor, shifted to
 *      be >= 0 and quantised so that the correlation is integer-exact;
 *   2. candidates are strict-left / non-strict-right local maxima of the filter
 *      output over +-sep bins with at least min_photons counts in the IRF
 *      window; the K largest (ties to the earlier bin) become points, stored in
 *      slots by increasing depth;
 *   3. b0 = counts outside all kept windows / (bins outside g), and
 *      r0 = max(window counts / g - b0 |window|, r_min).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "rt3d_oracle.h"

void or_lmf_kernel(const or_irf* irf, double delta_rel, int frac_bits, int32_t* kern)
{
    double hmax = 0.0;
    for (int s = 0; s < irf->len; ++s)
        if (irf->h[s] > hmax) hmax = irf->h[s];
    const double delta = delta_rel * hmax;
    const double scale = ldexp(1.0, frac_bits);
    for (int s = 0; s < irf->len; ++s)
        kern[s] = (int32_t)nearbyint(scale * log1p(irf->h[s] / delta));
}

/* y(tau) = sum_s z(tau + s - origin) K_s and the window count
 * w(tau) = sum_s z(tau + s - origin), with z = 0 outside [0, T). */
void or_lmf(const uint16_t* z, int t, const int32_t* kern, int len, int origin,
            int64_t* y, int64_t* wcount)
{
    for (int tau = 0; tau < t; ++tau) {
        int64_t acc = 0, cnt = 0;
        for (int s = 0; s < len; ++s) {
            const int tb = tau + s - origin;
            if (tb < 0 || tb >= t) continue;
            acc += (int64_t)z[tb] * kern[s];
            cnt += z[tb];
        }
        y[tau] = acc;
        wcount[tau] = cnt;
    }
}

/* Peak picking as described at the top of the file; returns how many peaks
 * were kept and writes their bins in increasing order. */
int or_peaks(const int64_t* y, const int64_t* wcount, int t, int sep, int min_photons,
             int kmax, int32_t* taus)
{
    int32_t best_tau[16];
    int64_t best_y[16];
    int nbest = 0;
    for (int tau = 0; tau < t; ++tau) {
        if (y[tau] <= 0 || wcount[tau] < min_photons) continue;
        int is_peak = 1;
        for (int q = tau - sep; q < tau && is_peak; ++q)
            if (q >= 0 && !(y[tau] > y[q])) is_peak = 0;
        for (int q = tau + 1; q <= tau + sep && is_peak; ++q)
            if (q < t && !(y[tau] >= y[q])) is_peak = 0;
        if (!is_peak) continue;
        /* insert into the list ordered by (y descending, tau ascending) */
        int pos = nbest;
        while (pos > 0 && best_y[pos - 1] < y[tau]) --pos;
        if (pos >= kmax) continue;
        const int last = nbest < kmax ? nbest : kmax - 1;
        for (int q = last; q > pos; --q) {
            best_y[q] = best_y[q - 1];
            best_tau[q] = best_tau[q - 1];
        }
        best_y[pos] = y[tau];
        best_tau[pos] = tau;
        if (nbest < kmax) ++nbest;
    }
    /* slots by increasing depth */
    for (int a = 0; a < nbest; ++a)
        for (int c = a + 1; c < nbest; ++c)
            if (best_tau[c] < best_tau[a]) {
                int32_t tmp = best_tau[a];
                best_tau[a] = best_tau[c];
                best_tau[c] = tmp;
            }
    for (int a = 0; a < nbest; ++a) taus[a] = best_tau[a];
    return nbest;
}

/* Initialisation with per-pixel instrument responses: pixel p uses
 * irf_set[irf_idx[p]] for its matched filter and windows (irf_idx NULL: every
 * pixel uses irf_set[0]). */
void or_init_idx(const uint16_t* dense, const double* gain, const uint8_t* irf_idx, int h, int w, int t,
                 const or_irf* irf_set, const or_params* prm, or_state* s)
{
    const int64_t npix = (int64_t)h * w;
    const int up = prm->upsample > 1 ? prm->upsample : 1;
    const int64_t wnpix = npix * up * up;
    int n_irf = 1;
    if (irf_idx)
        for (int64_t p = 0; p < npix; ++p)
            if (irf_idx[p] + 1 > n_irf) n_irf = irf_idx[p] + 1;
    int32_t* kerns[256];
    for (int i = 0; i < n_irf; ++i) {
        kerns[i] = (int32_t*)malloc(sizeof(int32_t) * irf_set[i].len);
        or_lmf_kernel(&irf_set[i], prm->lmf_delta_rel, prm->lmf_frac_bits, kerns[i]);
    }
#pragma omp parallel
    {
        int64_t* y = (int64_t*)malloc(sizeof(int64_t) * t);
        int64_t* wc = (int64_t*)malloc(sizeof(int64_t) * t);
        uint8_t* inwin = (uint8_t*)malloc((size_t)t);
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npix; ++p) {
            const uint16_t* z = dense + p * t;
            const double g = gain[p];
            const int which = irf_idx ? irf_idx[p] : 0;
            const or_irf* irf = &irf_set[which];
            const int32_t* kern = kerns[which];
            int32_t taus[16];
            int n = 0;
            if (g > 0.0) {
                or_lmf(z, t, kern, irf->len, irf->origin, y, wc);
                n = or_peaks(y, wc, t, prm->peak_sep, prm->peak_min_photons, s->k, taus);
            }
            /* background from the counts outside every kept window */
            memset(inwin, 0, (size_t)t);
            for (int a = 0; a < n; ++a)
                for (int sidx = 0; sidx < irf->len; ++sidx) {
                    const int tb = taus[a] + sidx - irf->origin;
                    if (tb >= 0 && tb < t) inwin[tb] = 1;
                }
            int64_t n_out = 0, t_out = 0;
            for (int tb = 0; tb < t; ++tb)
                if (!inwin[tb]) {
                    n_out += z[tb];
                    ++t_out;
                }
            double b0 = prm->b_floor;
            if (g > 0.0 && t_out > 0) {
                const double v = (double)n_out / ((double)t_out * g);
                b0 = v > prm->b_floor ? v : prm->b_floor;
            }
            s->b[p] = b0;
            /* with super-resolution (upsample u > 1) every world pixel of the
             * lidar pixel's u x u block starts from the pixel's peaks, each with
             * 1/u^2 of the intensity (reading: the block's points then give the
             * pixel the same lambda as the peaks) */
            const int64_t pi = p / w, pj = p % w, ww = (int64_t)w * up;
            for (int a = 0; a < up * up; ++a) {
                const int64_t q = (pi * up + a / up) * ww + (pj * up + a % up);
                for (int k = 0; k < s->k; ++k) {
                    const int64_t idx = (int64_t)k * wnpix + q;
                    if (k < n) {
                        int win = 0;
                        for (int sidx = 0; sidx < irf->len; ++sidx) {
                            const int tb = taus[k] + sidx - irf->origin;
                            if (tb >= 0 && tb < t) ++win;
                        }
                        const double r0 = (double)wc[taus[k]] / g - b0 * win;
                        s->t[idx] = (double)taus[k];
                        s->r[idx] = (r0 > prm->r_min ? r0 : prm->r_min) / (up * up);
                        s->alive[idx] = 1;
                    } else {
                        s->t[idx] = 0.0;
                        s->r[idx] = 0.0;
                        s->alive[idx] = 0;
                    }
                }
            }
        }
        free(y);
        free(wc);
        free(inwin);
    }
    for (int i = 0; i < n_irf; ++i) free(kerns[i]);
}

void or_init(const uint16_t* dense, const double* gain, int h, int w, int t,
             const or_irf* irf, const or_params* prm, or_state* s)
{
    or_init_idx(dense, gain, NULL, h, w, t, irf, prm, s);
}
