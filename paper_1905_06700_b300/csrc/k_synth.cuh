// k_synth.cuh -- photon synthesis on the device (benchmark and test input).
//
// Integer-only: Philox4x32-10 words drive a fixed-point Poisson inversion for
// the counts and table look-ups for the photon bins, so the histogram is
// bit-reproducible.  One warp per pixel accumulates photons in a shared-memory
// row of 32-bit counters and then writes the row out with 16-byte stores.
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplier S-box with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Poisson(mu) by inversion in 2^-62 fixed point: p_k = p_{k-1} mu / k.
__device__ __forceinline__ uint32_t poisson_fixed(uint32_t u, uint64_t p0, uint64_t mu_fx)
{
    const uint64_t target = (uint64_t)u << 30;
    uint64_t p = p0, cdf = p0;
    uint32_t k = 0;
    while (target >= cdf && k < 4096u) {
        ++k;
        // (p * mu_fx) >> 32 from the 128-bit product
        const uint64_t lo = p * mu_fx, hi = __umul64hi(p, mu_fx);
        p = ((hi << 32) | (lo >> 32)) / k;
        if (p == 0) break;
        cdf += p;
    }
    return k;
}

struct SynthArgs {
    int h, w, t, n_comp;
    const int32_t* depth_int;
    const uint32_t* depth_split;
    const uint32_t* n_parts;
    const uint64_t* p0;
    const uint64_t* mu;
    const uint32_t* irf_cdf;
    int irf_len, irf_origin;
    uint2 key;
    uint16_t* out;
};

constexpr int kSynthWarps = 4;

__global__ void __launch_bounds__(kSynthWarps * 32)
k_synth(const __grid_constant__ SynthArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cdf = reinterpret_cast<uint32_t*>(smem);             // [irf_len - 1]
    const int n_thr = a.irf_len - 1;
    const int cdf_words = (n_thr + 3) & ~3;
    for (int i = threadIdx.x; i < n_thr; i += blockDim.x) s_cdf[i] = a.irf_cdf[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long npix = (long long)a.h * a.w;
    const long long p = (long long)blockIdx.x * kSynthWarps + warp;
    if (p >= npix) return;
    const int T = a.t;
    const int t_words = (T + 3) & ~3;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem) + cdf_words + warp * t_words;
    for (int i = lane; i < T; i += 32) cnt[i] = 0;
    __syncwarp();

    for (int c = 0; c <= a.n_comp; ++c) {
        const bool bg = (c == a.n_comp);
        const uint32_t comp_id = bg ? 255u : (uint32_t)c;
        const long long e = (long long)c * npix + p;
        const uint32_t parts = a.n_parts[e];
        uint32_t count = 0;
        for (uint32_t q = lane; q < parts; q += 32) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)p, comp_id, q, 1u), a.key);
            count += poisson_fixed(r.x, a.p0[e], a.mu[e]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
        const int d0 = bg ? 0 : a.depth_int[e];
        const uint32_t split = bg ? 0u : a.depth_split[e];
        for (uint32_t j = lane; j < count; j += 32) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)p, comp_id, j, 2u), a.key);
            long long bin;
            if (bg) {
                bin = (long long)(((uint64_t)r.x * (uint64_t)T) >> 32);
            } else {
                int lo = 0, hi = n_thr;            // number of thresholds <= r.x
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_cdf[mid] <= r.x) lo = mid + 1; else hi = mid;
                }
                bin = (long long)d0 + lo - a.irf_origin + (r.y < split ? 1 : 0);
            }
            if (bin >= 0 && bin < T) atomicAdd(&cnt[bin], 1u);
        }
    }
    __syncwarp();
    uint16_t* row = a.out + p * T;
    if ((T & 7) == 0) {
        for (int v = lane; v < T / 8; v += 32) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t lo = min(cnt[8 * v + 2 * q], 65535u);
                const uint32_t hi = min(cnt[8 * v + 2 * q + 1], 65535u);
                w[q] = lo | (hi << 16);
            }
            reinterpret_cast<uint4*>(row)[v] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        for (int i = lane; i < T; i += 32) row[i] = (uint16_t)min(cnt[i], 65535u);
    }
}

}  // namespace rt3d
