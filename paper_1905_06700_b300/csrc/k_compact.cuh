// k_compact.cuh -- dense histogram to a standard offsets + entries sparse list
// (rt3d_compact): count nonzero bins per pixel, exclusive scan, emit.  The
// reconstruction itself compacts inside the initialisation kernel; this path
// serves callers that want to keep or transmit the sparse form.
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {

constexpr int kCompactWarps = 8;

__global__ void __launch_bounds__(kCompactWarps * 32)
k_count_nnz(const uint16_t* dense, int npix, int T, uint32_t* cnt)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * kCompactWarps + (threadIdx.x >> 5);
    if (p >= npix) return;
    const uint16_t* row = dense + (long long)p * T;
    uint32_t c = 0;
    for (int b = lane; b < T; b += 32) c += row[b] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[p] = c;
}

// Single-CTA exclusive scan of n counts into off[0..n] (off[n] = total).
__global__ void __launch_bounds__(1024) k_exclusive_scan(const uint32_t* cnt, int n, uint32_t* off)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < n ? cnt[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t ws = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += u;
            }
            warp_sums[lane] = ws;
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0u) + carry;
        if (i < n) off[i] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void __launch_bounds__(kCompactWarps * 32)
k_emit(const uint16_t* dense, int npix, int T, const uint32_t* off, uint32_t* ent)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * kCompactWarps + (threadIdx.x >> 5);
    if (p >= npix) return;
    const uint16_t* row = dense + (long long)p * T;
    uint32_t cursor = off[p];
    for (int b0 = 0; b0 < T; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t z = b < T ? row[b] : 0u;
        const unsigned m = __ballot_sync(0xffffffffu, z != 0);
        if (z) ent[cursor + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)b << 16) | z;
        cursor += __popc(m);
    }
}

}  // namespace rt3d
