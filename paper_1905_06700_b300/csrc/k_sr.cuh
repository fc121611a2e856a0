// k_sr.cuh -- gradient steps of the super-resolved observation model.
//
// With the point-to-cube mapping f of Results, "Observation model" sending a
// u x u window of world pixels to one lidar pixel (Results, "3D Dynamic
// scenes": 32 x 32 pixels reconstructed on a 96 x 96 world grid), the mean
// count of lidar pixel (i, j) sums the alive points of its block:
//   lambda_t = g (sum_{a < u^2, k < K} r_ak h(t - t_ak) + b).
// The depth, intensity and background steps therefore run per lidar pixel:
// one warp per pixel, its lanes over the pixel's nonzero bins.  The
// denoisers run on the world grid in the tile kernels of k_loop.cuh.
#pragma once
#include "k_loop.cuh"

namespace rt3d {

constexpr int kSrMaxPts = kMaxK * 16;   // u <= 4
constexpr int kSrWarps = 4;

struct SrWarp {
    float t[kSrMaxPts];                 // the block's alive points, in (world pixel, slot) order
    float rr[kSrMaxPts];
    int base[kSrMaxPts];
    float u[kSrMaxPts];
    int idx[kSrMaxPts];                 // a K + k of each alive point
    float part[kSrMaxPts][33];          // per-lane partial sums (padded row)
};

// MODE 0: background denoiser of the previous iteration (unless `first`),
//         alive flags of the previous pruning into the result, depth step
//         into t_half;
// MODE 1: intensity step into r_half (depths after the depth denoiser);
// MODE 2: background step into b_half (intensities and flags after the
//         intensity denoiser, pruning and merging).
template <int K, int MODE>
__global__ void __launch_bounds__(kSrWarps * 32)
k_sr_step(const CallRecord* __restrict__ rec, const Work W, int first, int lpix0, int lpix_end)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float4 coef[kCoefLen];
    __shared__ SrWarp sw[kSrWarps];
    load_irf_coef(pad, coef, P);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lpix = lpix0 + (int)blockIdx.x * kSrWarps + warp;
    if (lpix >= lpix_end) return;
    SrWarp& S = sw[warp];
    const FrameDesc& F = B.f[frame_of_lpixel(B, lpix)];
    const int lp = lpix - F.lpix_base;
    const int i = lp / F.lw, j = lp - (lp / F.lw) * F.lw;
    const int up = P.up, np = F.npix, T = F.nt, stride = W.stride;
    const int npts = up * up * K;
    const float g = F.gain ? F.gain[lp] : 1.0f;
    const IrfRef ir = irf_ref(P, pixel_irf(P, F, lp));
    float b;
    if (MODE == 0 && !first) {
        b = bkg_filter(P, W.b_half + F.lpix_base, F.lh, F.lw, i, j);
        if (lane == 0) F.b[lp] = b;
    } else {
        b = F.b[lp];
    }

    // the block's points (lanes over (world pixel a, slot k)); compact the alive ones
    int n_alive = 0;
    for (int e0 = 0; e0 < npts; e0 += 32) {
        const int e = e0 + lane;
        bool al = false;
        float tv = 0.0f, rv = 0.0f;
        long long q = 0;
        int k = 0;
        if (e < npts) {
            k = e % K;
            const int a = e / K;
            q = (long long)(i * up + a / up) * F.w + (j * up + a % up);
            uint8_t a8;
            if (MODE == 0)
                a8 = first ? F.alive[(long long)k * np + q] : W.alive_b[(long long)k * stride + F.pix_base + q];
            else if (MODE == 1)
                a8 = F.alive[(long long)k * np + q];
            else
                a8 = W.alive_b[(long long)k * stride + F.pix_base + q];
            if (MODE == 0 && !first) F.alive[(long long)k * np + q] = a8;
            al = a8 != 0;
            tv = F.t[(long long)k * np + q];
            rv = F.r[(long long)k * np + q];
        }
        const unsigned m = __ballot_sync(0xffffffffu, al);
        if (al) {
            const int pos = n_alive + __popc(m & ((1u << lane) - 1u));
            int base;
            float u;
            slot_frame(ir.origin, tv, base, u);
            S.t[pos] = tv;
            S.rr[pos] = rv;
            S.base[pos] = base;
            S.u[pos] = u;
            S.idx[pos] = e;
        }
        n_alive += __popc(m);
    }
    __syncwarp();

    // bin sums: lane l takes the pixel's nonzero bins l, l + 32, ... in order
    const uint2 sg = W.seg[lpix];
    const uint32_t* ent = F.ent + sg.x;
    const unsigned coff = (unsigned)ir.coef_off, cmax = (unsigned)(ir.len + 4);
    for (int p = 0; p < n_alive; ++p) S.part[p][lane] = 0.0f;
    float sz = 0.0f;
    for (uint32_t e = lane; e < sg.y; e += 32) {
        const uint32_t v = ent[e];
        const int tb = (int)(v >> 16);
        const float z = (float)(v & 0xffffu);
        float acc = b;
        for (int p = 0; p < n_alive; ++p) {
            const float4 c = coef[coff + min((unsigned)(tb + S.base[p]), cmax)];
            const float u = S.u[p];
            acc += S.rr[p] * (c.x + u * (c.y + u * (c.z + u * c.w)));
        }
        const float inv = __fdividef(z, fmaxf(g * acc, P.lam_floor));
        if (MODE == 2) {
            sz += inv;
        } else {
            for (int p = 0; p < n_alive; ++p) {
                const float4 c = coef[coff + min((unsigned)(tb + S.base[p]), cmax)];
                const float u = S.u[p];
                const float hv = MODE == 0 ? c.y + u * (2.0f * c.z + 3.0f * c.w * u)
                                           : c.x + u * (c.y + u * (c.z + u * c.w));
                S.part[p][lane] += hv * inv;
            }
        }
    }
    __syncwarp();

    if constexpr (MODE == 2) {
        sz = group_sum<32>(sz, 0xffffffffu);
        if (lane == 0) {
            float bn = b;
            if (g > 0.0f) bn = fmaxf(b - P.b_step * (b + P.eps_b) * (1.0f - sz / (float)T), P.b_floor);
            W.b_half[F.lpix_base + lp] = bn;
        }
        return;
    }

    // per point: its sum over the lanes' pieces in lane order, then the step
    if constexpr (MODE != 2)
    for (int e = lane; e < npts; e += 32) {
        const int k = e % K, a = e / K;
        const long long q = (long long)(i * up + a / up) * F.w + (j * up + a % up);
        const float tv = F.t[(long long)k * np + q];
        const float rv = F.r[(long long)k * np + q];
        int p = -1;
        for (int x = 0; x < n_alive; ++x)
            if (S.idx[x] == e) p = x;
        float out = MODE == 0 ? tv : rv;
        if (p >= 0 && g > 0.0f) {
            float s = 0.0f;
            for (int l = 0; l < 32; ++l) s += S.part[p][l];
            float H, dH;
            support_sums(pad, ir, T, tv, H, dH);
            if (MODE == 0) {
                const float grad = g * rv * (-dH + s);
                const float beta = P.t_step / (g * rv + P.eps_r);
                const float step = clampf(-beta * grad, -P.dt_max, P.dt_max);
                out = clampf(tv + step, 0.0f, (float)(T - 1));
            } else {
                out = fmaxf(rv - P.r_step * (rv + P.eps_r) * (H - s), 0.0f);
            }
        }
        if (MODE == 0)
            W.t_half[(long long)k * stride + F.pix_base + q] = out;
        else
            W.r_half[(long long)k * stride + F.pix_base + q] = out;
    }
}

}  // namespace rt3d
