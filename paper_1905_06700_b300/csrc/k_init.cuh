// k_init.cuh -- per-pixel initialisation (Methods, "3D Reconstruction
// algorithm": the initialisation processes each pixel independently).
//
// One warp per pixel:
//   1. dense histogram: stream the row (16-byte loads), count nonzero bins,
//      reserve space in the workspace entry buffer with one atomic, re-read the
//      row (L2-resident by then) and emit packed (bin << 16 | count) entries in
//      bin order -- the sparse form the PALM loop iterates over;
//      sparse input: take the caller's list as is;
//   2. log-matched filter by scatter: every nonzero bin adds count * K_s to
//      y(bin + origin - s) for the L taps (lanes over taps), together with a
//      saturating window count; integer arithmetic, so exact;
//   3. peak picking: strict-left / non-strict-right local maxima over +-sep
//      with enough photons in the IRF window; the K largest (ties to the
//      earlier bin) by a K-round warp arg-max; slots by increasing depth;
//   4. b0 from the counts outside the kept windows, r0 from the window counts.
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {

constexpr int kInitWarps = 4;                 // upper bound; fewer for long histograms
constexpr int kInitSmemBudget = 200 * 1024;

__host__ __device__ constexpr int init_warp_bytes(int tmax)
{
    // int32 filter output + uint8 window counts, 16-byte aligned
    return ((tmax * 4 + 15) & ~15) + ((tmax + 15) & ~15);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

template <bool kDumpY, bool kCompactOnly>
__global__ void __launch_bounds__(kInitWarps * 32)
k_init(const __grid_constant__ KParams P, const __grid_constant__ Batch B, const Work W)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int* sK = reinterpret_cast<int*>(smem);
    const int L = P.irf_len, O = P.irf_origin;
    const int k_bytes = (L * 4 + 15) & ~15;
    for (int i = threadIdx.x; i < L; i += blockDim.x) sK[i] = P.lmf[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pix = blockIdx.x * (int)(blockDim.x >> 5) + warp;
    if (pix >= B.total_pix) return;
    const FrameDesc& F = B.f[frame_of_pixel(B, pix)];
    const int lp = pix - F.pix_base;
    const int T = F.nt;
    const float g = F.gain ? F.gain[lp] : 1.0f;

    // ---- 1. sparse entries -------------------------------------------------
    uint32_t start = 0, nnz = 0;
    unsigned long long total = 0;
    const uint32_t* ent;
    if (F.csr_off) {
        start = F.csr_off[lp];
        nnz = F.csr_off[lp + 1] - start;
        ent = F.ent;
        for (uint32_t e = lane; e < nnz; e += 32) total += ent[start + e] & 0xffffu;
    } else {
        const uint16_t* row = F.dense + (long long)lp * T;
        const bool vec = (T & 7) == 0;
        uint32_t my = 0;
        if (vec) {
            for (int v = lane; v < T / 8; v += 32) {
                const uint4 q = reinterpret_cast<const uint4*>(row)[v];
                const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    my += ((w4[c] & 0xffffu) != 0) + ((w4[c] >> 16) != 0);
                    total += (w4[c] & 0xffffu) + (w4[c] >> 16);
                }
            }
        } else {
            for (int b = lane; b < T; b += 32) {
                const uint32_t z = row[b];
                my += z != 0;
                total += z;
            }
        }
        uint32_t tot_nnz = my;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot_nnz += __shfl_xor_sync(0xffffffffu, tot_nnz, o);
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd(W.ent_count, (unsigned long long)tot_nnz);
            if (base + tot_nnz > (unsigned long long)W.ent_cap) {
                atomicOr(W.status, kStatusCapacity);
                base = ~0ull;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base == ~0ull) {
            nnz = 0;
            start = 0;
        } else {
            start = (uint32_t)base;
            nnz = tot_nnz;
            uint32_t cursor = start;
            // re-read in the same order and emit bins in increasing order
            if (vec) {
                for (int v0 = 0; v0 < T / 8; v0 += 32) {
                    const int v = v0 + lane;
                    uint32_t w4[4] = {0, 0, 0, 0};
                    if (v < T / 8) {
                        const uint4 q = reinterpret_cast<const uint4*>(row)[v];
                        w4[0] = q.x; w4[1] = q.y; w4[2] = q.z; w4[3] = q.w;
                    }
                    uint32_t c = 0;
#pragma unroll
                    for (int s = 0; s < 4; ++s) c += ((w4[s] & 0xffffu) != 0) + ((w4[s] >> 16) != 0);
                    uint32_t incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += n;
                    }
                    uint32_t pos = cursor + incl - c;
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint32_t zl = w4[s] & 0xffffu, zh = w4[s] >> 16;
                        const uint32_t b = 8u * v + 2u * s;
                        if (zl) W.ent[pos++] = (b << 16) | zl;
                        if (zh) W.ent[pos++] = ((b + 1) << 16) | zh;
                    }
                    cursor += __shfl_sync(0xffffffffu, incl, 31);
                }
            } else {
                for (int b0 = 0; b0 < T; b0 += 32) {
                    const int b = b0 + lane;
                    const uint32_t z = b < T ? row[b] : 0u;
                    const unsigned m = __ballot_sync(0xffffffffu, z != 0);
                    if (z) W.ent[cursor + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)b << 16) | z;
                    cursor += __popc(m);
                }
            }
        }
        ent = W.ent;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) W.seg[pix] = make_uint2(start, nnz);
    if (kCompactOnly) return;
    __syncwarp();   // entries written by this warp are read back below

    // exact-arithmetic guard: every filter value must fit in int32
    const bool in_range = total * (unsigned long long)P.lmf_kmax < (1ull << 31);
    if (!in_range && lane == 0) atomicOr(W.status, kStatusRange);
    const bool active = in_range && g > 0.0f;

    // ---- 2. log-matched filter (scatter) -----------------------------------
    unsigned char* wbase = smem + k_bytes + warp * init_warp_bytes(B.max_t);
    int* Y = reinterpret_cast<int*>(wbase);
    uint8_t* Wc = wbase + ((B.max_t * 4 + 15) & ~15);
    {
        int4* y4 = reinterpret_cast<int4*>(Y);
        for (int i = lane; i < (T + 3) / 4; i += 32) y4[i] = make_int4(0, 0, 0, 0);
        uint4* w4 = reinterpret_cast<uint4*>(Wc);
        for (int i = lane; i < (T + 15) / 16; i += 32) w4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
    if (active || kDumpY) {
        for (uint32_t e0 = 0; e0 < nnz; e0 += 32) {
            const uint32_t mine = (e0 + lane < nnz) ? ent[start + e0 + lane] : 0u;
            const int cnt = (int)min(32u, nnz - e0);
            for (int j = 0; j < cnt; ++j) {
                const uint32_t v = __shfl_sync(0xffffffffu, mine, j);
                const int bin = (int)(v >> 16), z = (int)(v & 0xffffu);
                for (int s = lane; s < L; s += 32) {
                    const int tau = bin + O - s;
                    if (tau >= 0 && tau < T) {
                        Y[tau] += z * sK[s];
                        Wc[tau] = (uint8_t)min((int)Wc[tau] + z, 255);
                    }
                }
                __syncwarp();
            }
        }
    }
    if (kDumpY) {
        for (int i = lane; i < T; i += 32) W.y_out[(long long)lp * T + i] = Y[i];
        return;
    }

    // ---- 3. peak picking ---------------------------------------------------
    const int K = P.k, sep = P.peak_sep;
    int by[kMaxK], bt[kMaxK];
    int nb = 0;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) { by[k] = 0; bt[k] = 0; }
    if (active) {
        for (int tau = lane; tau < T; tau += 32) {
            const int y = Y[tau];
            if (y <= 0 || (int)Wc[tau] < P.peak_min_photons) continue;
            bool ok = true;
            const int qlo = max(0, tau - sep), qhi = min(T - 1, tau + sep);
            for (int q = tau - 1; q >= qlo; --q)
                if (Y[q] >= y) { ok = false; break; }
            if (ok)
                for (int q = tau + 1; q <= qhi; ++q)
                    if (Y[q] > y) { ok = false; break; }
            if (!ok) continue;
            // insert into this lane's list (y descending; equal y keeps the earlier bin first)
            int pos = nb;
#pragma unroll
            for (int k = kMaxK - 1; k >= 0; --k)
                if (k < nb && by[k] < y) pos = k;
            if (pos >= K) continue;
#pragma unroll
            for (int k = kMaxK - 1; k > 0; --k)
                if (k > pos && k < K) { by[k] = by[k - 1]; bt[k] = bt[k - 1]; }
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)
                if (k == pos) { by[k] = y; bt[k] = tau; }
            if (nb < K) ++nb;
        }
    }
    // K-round warp arg-max: key = (y << 32) | ~tau  (largest y, then smallest tau)
    int sel[kMaxK];
    int nsel = 0;
    int head = 0;
    for (int r = 0; r < K; ++r) {
        unsigned long long key = 0;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
            if (k == head && head < nb)
                key = ((unsigned long long)(unsigned)by[k] << 32) | (0xffffffffu - (unsigned)bt[k]);
        const unsigned long long best = warp_max_u64(key);
        if (best == 0) break;
        if (key == best) ++head;
        sel[nsel++] = (int)(0xffffffffu - (unsigned)(best & 0xffffffffu));
    }
    // slots by increasing depth
    for (int a = 0; a < nsel; ++a)
        for (int c = a + 1; c < nsel; ++c)
            if (sel[c] < sel[a]) { const int tmp = sel[a]; sel[a] = sel[c]; sel[c] = tmp; }

    // ---- 4. initial intensities and background ------------------------------
    unsigned long long inside = 0;
    unsigned long long wsum[kMaxK] = {0, 0, 0, 0};
    for (uint32_t e = lane; e < nnz; e += 32) {
        const uint32_t v = ent[start + e];
        const int bin = (int)(v >> 16);
        const unsigned z = v & 0xffffu;
        bool any = false;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
            if (k < nsel && bin >= sel[k] - O && bin <= sel[k] - O + L - 1) {
                wsum[k] += z;
                any = true;
            }
        if (any) inside += z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        inside += __shfl_xor_sync(0xffffffffu, inside, o);
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) wsum[k] += __shfl_xor_sync(0xffffffffu, wsum[k], o);
    }
    // bins covered by the union of the kept windows (windows sorted by start)
    int covered = 0, cur_lo = 0, cur_hi = -1;
    int winlen[kMaxK];
    for (int k = 0; k < nsel; ++k) {
        const int lo = max(sel[k] - O, 0), hi = min(sel[k] - O + L - 1, T - 1);
        winlen[k] = max(hi - lo + 1, 0);
        if (hi < lo) continue;
        if (lo > cur_hi) {
            covered += max(cur_hi - cur_lo + 1, 0);
            cur_lo = lo;
            cur_hi = hi;
        } else if (hi > cur_hi) {
            cur_hi = hi;
        }
    }
    covered += max(cur_hi - cur_lo + 1, 0);
    const long long t_out = (long long)T - covered;
    const long long n_out = (long long)total - (long long)inside;
    float b0 = P.b_floor;
    if (g > 0.0f && t_out > 0) b0 = fmaxf((float)n_out / ((float)t_out * g), P.b_floor);
    if (!active) nsel = 0;

    const int np = F.npix;
    if (lane < K) {
        const int k = lane;
        float tt = 0.0f, rr = 0.0f;
        uint8_t al = 0;
#pragma unroll
        for (int q = 0; q < kMaxK; ++q)
            if (q == k && q < nsel) {
                tt = (float)sel[q];
                rr = fmaxf((float)wsum[q] / g - b0 * (float)winlen[q], P.r_min);
                al = 1;
            }
        F.t[(long long)k * np + lp] = tt;
        F.r[(long long)k * np + lp] = rr;
        F.alive[(long long)k * np + lp] = al;
    }
    if (lane == 0) F.b[lp] = b0;
}

}  // namespace rt3d
