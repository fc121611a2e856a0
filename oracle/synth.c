/*
 * Synthetic photon histograms (test and benchmark input; not the method).
 * TEST INFRASTRUCTURE ONLY -- see rt3d_oracle.h.
 *
 * Counts follow the Poisson observation model of the paper (Results,
 * "Observation model"): each surface returns Poisson-many photons spread by the
 * instrument response, plus Poisson background spread uniformly over the bins.
 */
#include "rt3d_oracle.h"

/* Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit multiplications
 * with a Weyl-sequence key schedule.  Written from the published definition. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key increments */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t prod0 = (uint64_t)M0 * c0;
        uint64_t prod1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Poisson draw by inversion of the CDF in 2^-62 fixed point.
 *   p0 = round(exp(-mu) 2^62), mu_fx = round(mu 2^32)
 *   p_k = p_{k-1} * mu / k  (integer recurrence), F_k = sum_{j<=k} p_j
 *   result = min{k : u 2^30 < F_k}; stops early if p_k underflows to zero. */
uint32_t or_poisson_fixed(uint32_t u, uint64_t p0, uint64_t mu_fx)
{
    const uint64_t target = (uint64_t)u << 30;
    uint64_t p = p0, cdf = p0;
    uint32_t k = 0;
    while (target >= cdf && k < 4096u) {
        ++k;
        p = (uint64_t)(((unsigned __int128)p * mu_fx) >> 32) / k;
        if (p == 0) break;
        cdf += p;
    }
    return k;
}

/* Histogram of one scene.  Philox counters: (pixel, component, part, 1) for the
 * count of Poisson part `part`, (pixel, component, photon, 2) for a photon;
 * the key is the 64-bit seed.  Background is component 255.  A photon of
 * surface s lands in bin floor(d_s) + (offset index - origin) + [w1 < split_s],
 * a background photon in bin floor(w0 * T / 2^32).  Bins outside [0, T) are lost;
 * counts saturate at 65535. */
void or_synthesize(int h, int w, int t, int n_comp,
                   const int32_t* depth_int, const uint32_t* depth_split,
                   const uint32_t* n_parts, const uint64_t* p0, const uint64_t* mu,
                   const uint32_t* irf_cdf, int irf_len, int irf_origin,
                   uint64_t seed, uint16_t* dense)
{
    const int64_t npix = (int64_t)h * w;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        uint16_t* row = dense + p * t;
        for (int b = 0; b < t; ++b) row[b] = 0;
        for (int c = 0; c <= n_comp; ++c) {
            const int bg = (c == n_comp);
            const uint32_t comp_id = bg ? 255u : (uint32_t)c;
            const int64_t e = (int64_t)c * npix + p;
            uint32_t count = 0;
            for (uint32_t part = 0; part < n_parts[e]; ++part) {
                uint32_t ctr[4] = {(uint32_t)p, comp_id, part, 1u}, rnd[4];
                or_philox4x32_10(ctr, key, rnd);
                count += or_poisson_fixed(rnd[0], p0[e], mu[e]);
            }
            for (uint32_t j = 0; j < count; ++j) {
                uint32_t ctr[4] = {(uint32_t)p, comp_id, j, 2u}, rnd[4];
                or_philox4x32_10(ctr, key, rnd);
                int64_t bin;
                if (bg) {
                    bin = (int64_t)(((uint64_t)rnd[0] * (uint64_t)t) >> 32);
                } else {
                    int off = 0;
                    for (int s = 0; s < irf_len - 1; ++s)
                        if (irf_cdf[s] <= rnd[0]) ++off;
                    bin = (int64_t)depth_int[e] + off - irf_origin
                        + (rnd[1] < depth_split[e] ? 1 : 0);
                }
                if (bin >= 0 && bin < t && row[bin] < 65535u) row[bin]++;
            }
        }
    }
}
