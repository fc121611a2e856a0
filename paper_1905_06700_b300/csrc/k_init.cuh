// k_init.cuh -- per-pixel initialisation (Methods, "3D Reconstruction
// algorithm": the initialisation processes each pixel independently).
//
// One warp per pixel, bounded by the dense read (2 T bytes per pixel):
//   1. stream the histogram row once with 16-byte loads; one vote per load
//      finds the few 16-byte words holding a nonzero bin, which 8 lanes unpack
//      into packed (bin << 16 | count) entries in a per-warp shared staging
//      list, in bin order; one atomic reserves the pixel's span of the
//      workspace entry buffer -- the sparse form the PALM loop iterates over.
//      Rows with more nonzero bins than the staging list holds are re-read
//      and emitted straight to global memory.  A caller's sparse list is used
//      as is;
//   2. log-matched filter by scatter, cluster by cluster: entries more than
//      L - 1 + 2 sep bins apart cannot affect each other's filter values,
//      peak tests or window counts, so the sorted entries split into
//      independent clusters; a cluster with fewer photons than the peak
//      threshold cannot hold a peak and is skipped (most isolated background
//      photons).  For the others, the filter output of up to 256 positions
//      plus a +-sep halo lives in shared memory; each entry adds count * K_s
//      at bin + origin - s for the L taps (lanes over taps).  Integer
//      arithmetic, so the output is exact;
//   3. peak picking: strict-left / non-strict-right local maxima over +-sep
//      (immediate neighbours first, then the window) with enough photons in
//      the IRF window (summed from the chunk's entries); each lane keeps its K
//      best, a K-round warp arg-max keeps the overall K largest (ties to the
//      earlier bin); slots by increasing depth;
//   4. b0 from the counts outside the kept windows, r0 from the window counts.
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {

constexpr int kInitWarps = 2;        // warps (pixels) per CTA: small CTAs, 20 per SM
constexpr int kInitChunk = 256;      // filter positions per chunk
constexpr int kInitStage = 256;      // staged entries per warp
constexpr int kInitSmemBudget = 200 * 1024;

__host__ __device__ constexpr int init_buf(int sep) { return kInitChunk + 2 * sep; }

__host__ __device__ constexpr int init_warp_bytes(int sep)
{
    // staging list + int32 filter chunk, 16-byte aligned
    return kInitStage * 4 + ((init_buf(sep) * 4 + 15) & ~15);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Variants (kVar bits): kInitIdx -- some frame of the launch names a response
// per pixel (rt3d_frame.irf_index); kInitUp -- super-resolution (the points
// go to the world grid).
constexpr int kInitIdx = 1, kInitUp = 2;

template <bool kDumpY, bool kCompactOnly, int kVar = 0>
__global__ void __launch_bounds__(kInitWarps * 32, 20)
k_init(const CallRecord* __restrict__ rec, const Work W, int pix0, int pix_end)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    extern __shared__ __align__(16) unsigned char smem[];
    int* sK_all = reinterpret_cast<int*>(smem);
    const int sep = P.peak_sep;
    const int min_photons = P.peak_min_photons;
    // every response's taps (a pixel uses its own response's)
    constexpr bool kIdx = (kVar & kInitIdx) != 0;
    const int n_taps = kIdx ? P.irf_offs[P.n_irf - 1] + P.irf_lens[P.n_irf - 1] : P.irf_len;
    const int k_bytes = (n_taps * 4 + 15) & ~15;
    for (int i = threadIdx.x; i < n_taps; i += blockDim.x) sK_all[i] = P.lmf[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this launch covers the batch's pixels [pix0, pix_end)
    const int pix = pix0 + (int)blockIdx.x * (int)(blockDim.x >> 5) + warp;
    if (pix >= pix_end) return;
    // lidar pixels: the histograms' grid
    const FrameDesc& F = B.f[frame_of_lpixel(B, pix)];
    // frames whose cold start runs in the tensor-core init
    if (!kCompactOnly && F.tc) return;
    const int lp = pix - F.lpix_base;
    const int T = F.nt;
    if (lp == 0 && lane == 0 && F.n_points) *F.n_points = 0;   // counted by the finaliser
    const float g = F.gain ? F.gain[lp] : 1.0f;
    // the pixel's instrument response: taps, length and origin (response 0
    // unless the frame names one per pixel)
    const int which = kIdx ? pixel_irf(P, F, lp) : 0;
    const int L = kIdx ? P.irf_lens[which] : P.irf_len, O = kIdx ? P.irf_origins[which] : P.irf_origin;
    const int* sK = kIdx ? sK_all + P.irf_offs[which] : sK_all;

    unsigned char* wbase = smem + k_bytes + warp * init_warp_bytes(sep);
    uint32_t* stage = reinterpret_cast<uint32_t*>(wbase);
    int* Y = reinterpret_cast<int*>(wbase + kInitStage * 4);

    // ---- 1. sparse entries -------------------------------------------------
    uint32_t start = 0, nnz = 0;
    unsigned long long total = 0;
    const uint32_t* ent;                 // generic pointer: shared stage or global list
    if (F.csr_off) {
        start = F.csr_off[lp];
        nnz = F.csr_off[lp + 1] - start;
        ent = F.ent + start;
    } else {
        const uint16_t* row = F.dense + (long long)lp * T;
        uint32_t n_stage = 0;
        bool overflow = false;
        if ((T & 7) == 0) {
            const uint4* row4 = reinterpret_cast<const uint4*>(row);
            const int nv = T >> 3;
            for (int v0 = 0; v0 < nv; v0 += 128) {
                uint4 q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int v = v0 + u * 32 + lane;
                    q[u] = v < nv ? row4[v] : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    unsigned words = __ballot_sync(0xffffffffu, (q[u].x | q[u].y | q[u].z | q[u].w) != 0u);
                    while (words) {
                        // one nonzero 16-byte word (8 bins) of lane src: lanes 0..7 unpack a bin each
                        const int src = __ffs(words) - 1;
                        words &= words - 1;
                        const uint32_t wx = __shfl_sync(0xffffffffu, q[u].x, src);
                        const uint32_t wy = __shfl_sync(0xffffffffu, q[u].y, src);
                        const uint32_t wz = __shfl_sync(0xffffffffu, q[u].z, src);
                        const uint32_t ww = __shfl_sync(0xffffffffu, q[u].w, src);
                        const int j = lane & 7;
                        const uint32_t word = j < 2 ? wx : (j < 4 ? wy : (j < 6 ? wz : ww));
                        const uint32_t val = (j & 1) ? (word >> 16) : (word & 0xffffu);
                        const unsigned m = __ballot_sync(0xffffffffu, lane < 8 && val != 0u);
                        const uint32_t bin = 8u * (uint32_t)(v0 + u * 32 + src) + (uint32_t)j;
                        if (lane < 8 && val != 0u) {
                            const uint32_t pos = n_stage + __popc(m & ((1u << lane) - 1u));
                            if (pos < (uint32_t)kInitStage) stage[pos] = (bin << 16) | val;
                        }
                        n_stage += __popc(m);
                    }
                }
            }
            overflow = n_stage > (uint32_t)kInitStage;
        } else {
            for (int b0 = 0; b0 < T; b0 += 32) {
                const int b = b0 + lane;
                const uint32_t val = b < T ? (uint32_t)row[b] : 0u;
                const unsigned m = __ballot_sync(0xffffffffu, val != 0u);
                if (val) {
                    const uint32_t pos = n_stage + __popc(m & ((1u << lane) - 1u));
                    if (pos < (uint32_t)kInitStage) stage[pos] = ((uint32_t)b << 16) | val;
                }
                n_stage += __popc(m);
            }
            overflow = n_stage > (uint32_t)kInitStage;
        }
        nnz = n_stage;
        unsigned long long base = 0;
        if (lane == 0) {
            base = (unsigned long long)B.ent_base_int + atomicAdd(W.ent_count, (unsigned long long)nnz);
            if (base + nnz > (unsigned long long)W.ent_cap) {
                atomicOr(W.status, kStatusCapacity);
                base = ~0ull;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base == ~0ull) {
            nnz = 0;
            start = 0;
            ent = stage;
        } else if (!overflow) {
            start = (uint32_t)base;
            for (uint32_t e = lane; e < nnz; e += 32) W.ent[start + e] = stage[e];
            ent = stage;
        } else {
            // more nonzero bins than the stage holds: re-read and emit to global
            start = (uint32_t)base;
            uint32_t cursor = start;
            for (int b0 = 0; b0 < T; b0 += 32) {
                const int b = b0 + lane;
                const uint32_t z = b < T ? row[b] : 0u;
                const unsigned m = __ballot_sync(0xffffffffu, z != 0);
                if (z) W.ent[cursor + __popc(m & ((1u << lane) - 1u))] = ((uint32_t)b << 16) | z;
                cursor += __popc(m);
            }
            ent = W.ent + start;
        }
    }
    if (lane == 0) W.seg[pix] = make_uint2(start, nnz);
    if (kCompactOnly) return;
    __syncwarp();   // entries written by this warp are read back below

    // photons of the pixel
    for (uint32_t e = lane; e < nnz; e += 32) total += ent[e] & 0xffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);

    // exact-arithmetic guard: every filter value must fit in int32
    const bool in_range = total * (unsigned long long)P.lmf_kmax < (1ull << 31);
    if (!in_range && lane == 0) atomicOr(W.status, kStatusRange);
    const bool active = in_range && g > 0.0f;

    // ---- 2 + 3. chunked matched filter and peak candidates ------------------
    const int K = P.k;
    int by[kMaxK], bt[kMaxK];
    int nb = 0;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) { by[k] = 0; bt[k] = 0; }
    const int nbuf = init_buf(sep);
    const int gap = L - 1 + 2 * sep;     // entries farther apart never interact
    if (kDumpY)
        for (int i = lane; i < T; i += 32) W.y_out[(long long)lp * T + i] = 0;
    uint32_t c_lo = (active || kDumpY) ? 0u : nnz;
    // up to 32 entries: one lane per entry, the breaks between clusters in one vote
    const bool small = nnz <= 32u;
    uint32_t v_small = 0u;
    unsigned brk_small = 0u;
    if (small) {
        v_small = (uint32_t)lane < nnz ? ent[lane] : 0u;
        const uint32_t nxt = __shfl_down_sync(0xffffffffu, v_small, 1);
        brk_small = __ballot_sync(0xffffffffu, (uint32_t)lane + 1u < nnz &&
                                                   (int)(nxt >> 16) - (int)(v_small >> 16) > gap);
    }
    while (c_lo < nnz) {
        // the cluster [c_lo, c_hi): consecutive entries at most `gap` bins apart
        uint32_t c_hi = c_lo;
        unsigned long long cl_tot = 0;
        if (small) {
            const unsigned after = brk_small >> c_lo;   // breaks at or after entry c_lo
            c_hi = after ? c_lo + (uint32_t)__ffs(after) : nnz;
            const bool mine = (uint32_t)lane >= c_lo && (uint32_t)lane < c_hi;
            cl_tot = __reduce_add_sync(0xffffffffu, mine ? (v_small & 0xffffu) : 0u);
        } else {
            while (true) {
                const uint32_t e = c_hi + lane;
                const bool in = e < nnz;
                const uint32_t v = in ? ent[e] : 0u;
                const bool brk = in && e + 1 < nnz && (int)(ent[e + 1] >> 16) - (int)(v >> 16) > gap;
                const unsigned mb = __ballot_sync(0xffffffffu, brk);
                const unsigned mi = __ballot_sync(0xffffffffu, in);
                // entries up to and including the first break belong to the cluster
                const int take = mb ? (__ffs(mb)) : __popc(mi);
                cl_tot += __reduce_add_sync(0xffffffffu, (lane < take) ? (v & 0xffffu) : 0u);
                c_hi += take;
                if (mb || take < 32) break;
            }
        }
        const uint32_t e_first = c_lo, e_last = c_hi - 1;
        c_lo = c_hi;
        if (!kDumpY && cl_tot < (unsigned long long)min_photons) continue;
        const int lo = max(0, (int)(ent[e_first] >> 16) + O - L + 1);
        const int hi = min(T - 1, (int)(ent[e_last] >> 16) + O);
        uint32_t e_lo = e_first;
        const bool one_chunk = hi - lo < kInitChunk;
        for (int cbase = lo; cbase <= hi; cbase += kInitChunk) {
            // cluster entries reaching [cbase - sep, cbase + chunk + sep): all of
            // them when the cluster's positions fit one chunk
            const int lo_b = cbase - sep - O;
            const int hi_b = cbase + kInitChunk - 1 + sep - O + L - 1;
            while (!one_chunk && e_lo <= e_last) {
                const uint32_t e = e_lo + lane;
                const bool below = e <= e_last && (int)(ent[e] >> 16) < lo_b;
                const unsigned m = __ballot_sync(0xffffffffu, below);
                e_lo += __popc(m);
                if (m != 0xffffffffu) break;
            }
            uint32_t e_hi = one_chunk ? e_last + 1 : e_lo;
            while (e_hi <= e_last) {
                const uint32_t e = e_hi + lane;
                const bool in = e <= e_last && (int)(ent[e] >> 16) <= hi_b;
                const unsigned m = __ballot_sync(0xffffffffu, in);
                e_hi += __popc(m);
                if (m != 0xffffffffu) break;
            }
            const int cend = min(cbase + kInitChunk, hi + 1);
            // positions the scatter below can reach and the scan reads
            const int nclr = min(nbuf, cend - cbase + 2 * sep);
            for (int i = lane; i < nclr; i += 32) Y[i] = 0;
            __syncwarp();
            const int blo = max(0, cbase - sep), bhi = min(T, cend + sep);
            for (uint32_t e = e_lo; e < e_hi; ++e) {
                const uint32_t v = ent[e];
                const int bin = (int)(v >> 16), z = (int)(v & 0xffffu);
                for (int s = lane; s < L; s += 32) {
                    const int tau = bin + O - s;
                    if (tau >= blo && tau < bhi) Y[tau - cbase + sep] += z * sK[s];
                }
                __syncwarp();
            }
            if constexpr (kDumpY) {
                for (int i = lane; cbase + i < cend; i += 32)
                    W.y_out[(long long)lp * T + cbase + i] = Y[i + sep];
                __syncwarp();
                continue;
            } else {
            for (int i0 = 0; cbase + i0 < cend; i0 += 32) {
                // local maxima against the immediate neighbours, 32 positions per vote
                const int i = i0 + lane, yi = i + sep;
                bool cand = false;
                if (cbase + i < cend) {
                    const int y = Y[yi];
                    cand = y > 0 && (sep == 0 || (Y[yi - 1] < y && Y[yi + 1] <= y));
                }
                unsigned cm = __ballot_sync(0xffffffffu, cand);
                while (cm) {
                    // one candidate at a time, in bin order, tested by the whole warp
                    const int ci = i0 + __ffs(cm) - 1;
                    cm &= cm - 1;
                    const int cyi = ci + sep, tau = cbase + ci;
                    const int y = Y[cyi];
                    // strict-left / non-strict-right maximum over +-sep: lanes over offsets
                    bool ok = true;
                    for (int q = 2 + lane; q <= sep; q += 32) ok = ok && Y[cyi - q] < y && Y[cyi + q] <= y;
                    if (!__all_sync(0xffffffffu, ok)) continue;
                    // photons in the IRF window [tau - origin, tau - origin + L): lanes over entries
                    // (photon counts of an active pixel are below 2^31: 32-bit sums are exact)
                    uint32_t wcount = 0;
                    for (uint32_t e = e_first + lane; e <= e_last; e += 32) {
                        const uint32_t v = ent[e];
                        const int bin = (int)(v >> 16);
                        if (bin >= tau - O && bin <= tau - O + L - 1) wcount += v & 0xffffu;
                    }
                    wcount = __reduce_add_sync(0xffffffffu, wcount);
                    if ((long long)wcount < (long long)min_photons) continue;
                    // the warp's list of the K best (y descending; candidates arrive in
                    // bin order, so equal y keeps the earlier bin first)
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
            __syncwarp();
            }
        }
    }
    if (kDumpY) return;

    // the K largest filter values (ties to the earlier bin), the same in every lane
    int sel[kMaxK];
    int nsel = nb;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) sel[k] = bt[k];
    // slots by increasing depth
#pragma unroll
    for (int a = 0; a < kMaxK; ++a)
#pragma unroll
        for (int c = a + 1; c < kMaxK; ++c)
            if (c < nsel && sel[c] < sel[a]) { const int tmp = sel[a]; sel[a] = sel[c]; sel[c] = tmp; }

    // ---- 4. initial intensities and background ------------------------------
    // window sums of an active pixel are below 2^31 (an inactive one keeps none)
    uint32_t inside = 0;
    uint32_t wsum[kMaxK] = {0, 0, 0, 0};
    for (uint32_t e = lane; e < nnz; e += 32) {
        const uint32_t v = ent[e];
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
    inside = __reduce_add_sync(0xffffffffu, inside);
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) wsum[k] = __reduce_add_sync(0xffffffffu, wsum[k]);
    // bins covered by the union of the kept windows (windows sorted by start)
    int covered = 0, cur_lo = 0, cur_hi = -1;
    int winlen[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        winlen[k] = 0;
        if (k >= nsel) continue;
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

    // the points: with super-resolution (u > 1) every world pixel of the
    // lidar pixel's u x u block starts from the pixel's peaks, each with
    // 1/u^2 of the intensity; lanes over (world pixel a, slot k)
    const int np = F.npix;
    const int up = (kVar & kInitUp) ? P.up : 1;
    if (lane < K * up * up) {
        // lane = a K + k: world pixel a of the block (a = 0 without super-resolution), slot k
        const int k = up == 1 ? lane : lane % K, a = up == 1 ? 0 : lane / K;
        float tt = 0.0f, rr = 0.0f;
        uint8_t al = 0;
#pragma unroll
        for (int q = 0; q < kMaxK; ++q)
            if (q == k && q < nsel) {
                tt = (float)sel[q];
                rr = fmaxf((float)wsum[q] / g - b0 * (float)winlen[q], P.r_min);
                al = 1;
            }
        long long wq = lp;
        if (up > 1) {
            const int i = lp / F.lw, j = lp - i * F.lw;
            wq = (long long)(i * up + a / up) * F.w + (j * up + a % up);
            rr /= (float)(up * up);
        }
        F.t[(long long)k * np + wq] = tt;
        F.r[(long long)k * np + wq] = rr;
        F.alive[(long long)k * np + wq] = al;
    }
    if ((kVar & kInitUp) && up > 2) {
        // blocks of more than 32 points: the rest (u = 3, 4 with K > 3 or u = 4)
        for (int e = lane + 32; e < K * up * up; e += 32) {
            const int k = e % K, a = e / K;
            float tt = 0.0f, rr = 0.0f;
            uint8_t al = 0;
#pragma unroll
            for (int q = 0; q < kMaxK; ++q)
                if (q == k && q < nsel) {
                    tt = (float)sel[q];
                    rr = fmaxf((float)wsum[q] / g - b0 * (float)winlen[q], P.r_min);
                    al = 1;
                }
            const int i = lp / F.lw, j = lp - i * F.lw;
            const long long wq = (long long)(i * up + a / up) * F.w + (j * up + a % up);
            rr /= (float)(up * up);
            F.t[(long long)k * np + wq] = tt;
            F.r[(long long)k * np + wq] = rr;
            F.alive[(long long)k * np + wq] = al;
        }
    }
    if (lane == 0) F.b[lp] = b0;
}

}  // namespace rt3d
