// k_loop.cuh -- the PALM iteration (Results, "Reconstruction algorithm",
// Fig. 2) as three fused kernels per iteration plus a finaliser.
//
// Each neighbourhood step (APSS, intensity low-pass, background low-pass)
// needs the preceding per-pixel step finished on its halo, so the per-pixel
// gradient steps ride at the tail (or head) of the neighbourhood kernels:
//   A: [b <- background denoiser(b_half); alive <- alive_b]  + depth step
//   B: APSS(t_half)                                           + intensity step
//   C: intensity low-pass + pruning                           + background step
// A CTA owns an 8 x 16 pixel tile of one frame.  Neighbourhood work runs one
// thread per pixel (or per alive point) over a shared-memory copy of the tile
// and its halo; the per-pixel gradient steps run one thread per pixel over the
// pixel's nonzero bins (cost linear in active bins, Methods and Fig. 5).
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {


struct TileCtx {
    int fi, i0, j0, li, lj, gi, gj;
    bool inb;
};

__device__ __forceinline__ TileCtx tile_ctx(const Batch& B)
{
    TileCtx c;
    c.fi = frame_of_tile(B, blockIdx.x);
    const FrameDesc& F = B.f[c.fi];
    const int lt = blockIdx.x - F.tile_base;
    c.i0 = (lt / F.tiles_w) * kTileH;
    c.j0 = (lt % F.tiles_w) * kTileW;
    c.li = threadIdx.x / kTileW;
    c.lj = threadIdx.x % kTileW;
    c.gi = c.i0 + c.li;
    c.gj = c.j0 + c.lj;
    c.inb = c.gi < F.h && c.gj < F.w;
    return c;
}

__device__ __forceinline__ void load_irf(float* pad, const KParams& P)
{
    for (int i = threadIdx.x; i < P.irf_len + 2 * kIrfPad; i += blockDim.x) {
        const int k = i - kIrfPad;
        pad[i] = (k >= 0 && k < P.irf_len) ? P.irf[k] : 0.0f;
    }
}

// Sums over the nonzero bins of one pixel, by one thread:
//   sh[k] = sum z h(t - t_k)/lambda, sdh[k] = sum z h'(t - t_k)/lambda,
//   sz = sum z/lambda, lambda = max(g (sum_alive r_k h(t - t_k) + b), lam_floor).
// Every slot is evaluated (a dead slot enters lambda with r = 0), so lanes of
// a warp do not diverge on which slots are alive; the next entry is fetched
// while the current one is computed.
__device__ __forceinline__ void pixel_sums(const uint32_t* ent, uint2 sg, const float* pad,
                                           const KParams& P, const float* tk, const float* rk,
                                           const bool* ak, float b, float g, float* sh, float* sdh,
                                           float& sz)
{
    const int K = P.k, L = P.irf_len, O = P.irf_origin;
    float rr[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        sh[k] = 0.0f;
        sdh[k] = 0.0f;
        rr[k] = ak[k] ? rk[k] : 0.0f;
    }
    sz = 0.0f;
    const float lam_floor = P.lam_floor;
    uint32_t v = sg.y ? ent[sg.x] : 0u;
    for (uint32_t e = 0; e < sg.y; ++e) {
        const uint32_t cur = v;
        if (e + 1 < sg.y) v = ent[sg.x + e + 1];
        const float tb = (float)(cur >> 16), z = (float)(cur & 0xffffu);
        float hv[kMaxK], dv[kMaxK];
        float acc = b;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            hv[k] = 0.0f;
            dv[k] = 0.0f;
            if (k < K) {
                irf_eval(pad, L, O, tb - tk[k], hv[k], dv[k]);
                acc += rr[k] * hv[k];
            }
        }
        const float lam = fmaxf(g * acc, lam_floor);
        const float inv = __fdividef(z, lam);
        sz += inv;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            sh[k] += hv[k] * inv;
            sdh[k] += dv[k] * inv;
        }
    }
}

// Background denoiser at pixel (i, j): periodic separable Gaussian over the
// frame (equal to the FFT low-pass with the kernel's DFT), or identity.
__device__ __forceinline__ float bkg_filter(const KParams& P, const float* bh, int h, int w,
                                            int i, int j)
{
    if (P.bkg_mode != RT3D_BKG_LOWPASS) return bh[i * w + j];
    const int R = P.bkg_rad;
    float acc = 0.0f;
    for (int di = -R; di <= R; ++di) {
        int ii = (i + di) % h;
        if (ii < 0) ii += h;
        float row = 0.0f;
        for (int dj = -R; dj <= R; ++dj) {
            int jj = (j + dj) % w;
            if (jj < 0) jj += w;
            row += P.bkg_ker[dj + R] * bh[ii * w + jj];
        }
        acc += P.bkg_ker[di + R] * row;
    }
    return acc;
}

// ----------------------------------------------------------------------------
// Phase A: background denoiser of the previous iteration + depth gradient step,
// one thread per pixel.
__global__ void __launch_bounds__(kTileThreads)
k_phase_a(const CallRecord* __restrict__ rec, const Work W, int first)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    load_irf(pad, P);
    __syncthreads();
    const TileCtx c = tile_ctx(B);
    const FrameDesc& F = B.f[c.fi];
    if (!c.inb) return;
    const int np = F.npix, S = W.stride, K = P.k;
    const int lp = c.gi * F.w + c.gj, wp = F.pix_base + lp;
    float b;
    if (first) {
        b = F.b[lp];
    } else {
        b = bkg_filter(P, W.b_half + F.pix_base, F.h, F.w, c.gi, c.gj);
        F.b[lp] = b;
    }
    const float g = F.gain ? F.gain[lp] : 1.0f;
    float tk[kMaxK], rk[kMaxK];
    bool ak[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        tk[k] = 0.0f;
        rk[k] = 0.0f;
        ak[k] = false;
        if (k < K) {
            uint8_t a;
            if (first) {
                a = F.alive[(long long)k * np + lp];
            } else {
                a = W.alive_b[(long long)k * S + wp];
                F.alive[(long long)k * np + lp] = a;
            }
            ak[k] = a != 0;
            tk[k] = F.t[(long long)k * np + lp];
            rk[k] = F.r[(long long)k * np + lp];
        }
    }
    float sh[kMaxK], sdh[kMaxK], sz;
    pixel_sums(F.ent, W.seg[wp], pad, P, tk, rk, ak, b, g, sh, sdh, sz);
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        if (k >= K) continue;
        float tn = tk[k];
        if (ak[k] && g > 0.0f) {
            float H, dH;
            support_sums(pad, P, F.nt, tk[k], H, dH);
            const float grad = g * rk[k] * (-dH + sdh[k]);
            const float beta = P.t_step / (g * rk[k] + P.eps_r);
            const float step = clampf(-beta * grad, -P.dt_max, P.dt_max);
            tn = clampf(tk[k] + step, 0.0f, (float)(F.nt - 1));
        }
        W.t_half[(long long)k * S + wp] = tn;
    }
}

// ----------------------------------------------------------------------------
constexpr int kHaloH = kTileH + 2 * kMaxWinR, kHaloW = kTileW + 2 * kMaxWinR;
constexpr int kHalo = kHaloH * kHaloW;

// APSS projection of one point (Results, "Depth update"; Guennebaud & Gross):
// weighted algebraic-sphere fit s(x) = u0 + u1 x + u2 y + z + u4 |x|^2 over
// the window (local coordinates scaled by 1/h), solved in centred form --
// the 3x3 normal equations of (x, y, |x|^2) against z, then u0 from the
// weighted means -- and projection along the line of sight onto s = 0.
// The accumulation is branch-free: dead or absent slots hold a far sentinel
// depth, so their weight is exactly zero; window offsets outside the lateral
// radius are skipped uniformly across the warp.
__device__ float apss_point(const float* st, int hstride, int R, int K, int ci, int cj, float tn,
                            const KParams& P, int T)
{
    const float inv_h = 1.0f / P.apss_h;
    const float px = P.pitch * inv_h;
    float S0 = 0.f, Sx = 0.f, Sy = 0.f, Sz = 0.f, Sq = 0.f;
    float Sxx = 0.f, Sxy = 0.f, Syy = 0.f, Sxq = 0.f, Syq = 0.f, Sqq = 0.f;
    float Sxz = 0.f, Syz = 0.f, Sqz = 0.f;
    // indicator sums of the pixel offsets of weighted neighbours (exact integers)
    float nw = 0.f, si = 0.f, sj = 0.f, sii = 0.f, sjj = 0.f, sij = 0.f;
    for (int di = -R; di <= R; ++di) {
        const float y = (float)di * px;
        for (int dj = -R; dj <= R; ++dj) {
            const float x = (float)dj * px;
            const float r2 = x * x + y * y;
            if (!(r2 < 1.0f)) continue;
            const int q = (ci + di) * hstride + (cj + dj);
            float cnt = 0.0f;
            for (int m = 0; m < K; ++m) {
                const float z = (st[m * kHalo + q] - tn) * inv_h;
                const float d2 = r2 + z * z;
                const bool in = d2 < 1.0f;
                float w = 1.0f - d2;
                w *= w;
                w = in ? w * w : 0.0f;
                cnt += in ? 1.0f : 0.0f;
                const float wx = w * x, wy = w * y, wq = w * d2;
                S0 += w; Sx += wx; Sy += wy; Sz += w * z; Sq += wq;
                Sxx += wx * x; Sxy += wx * y; Syy += wy * y;
                Sxq += wx * d2; Syq += wy * d2; Sqq += wq * d2;
                Sxz += wx * z; Syz += wy * z; Sqz += wq * z;
            }
            nw += cnt;
            si += cnt * (float)di;
            sj += cnt * (float)dj;
            sii += cnt * (float)(di * di);
            sjj += cnt * (float)(dj * dj);
            sij += cnt * (float)(di * dj);
        }
    }
    const long long n = (long long)nw;
    if (n < P.apss_min_nb) return tn;
    const long long vii = n * (long long)sii - (long long)si * (long long)si;
    const long long vjj = n * (long long)sjj - (long long)sj * (long long)sj;
    const long long vij = n * (long long)sij - (long long)si * (long long)sj;
    if (vii * vjj - vij * vij == 0) return tn;      // collinear pixel offsets
    const float iw = 1.0f / S0;
    const float mx = Sx * iw, my = Sy * iw, mz = Sz * iw, mq = Sq * iw;
    const float cxx = Sxx * iw - mx * mx, cxy = Sxy * iw - mx * my, cyy = Syy * iw - my * my;
    const float cxq = Sxq * iw - mx * mq, cyq = Syq * iw - my * mq, cqq = Sqq * iw - mq * mq;
    const float dx = Sxz * iw - mx * mz, dy = Syz * iw - my * mz, dq = Sqz * iw - mq * mz;
    // Cholesky of the 3x3 covariance
    if (!(cxx > 0.0f)) return tn;
    const float l11 = sqrtf(cxx);
    const float l21 = cxy / l11, l31 = cxq / l11;
    const float d22 = cyy - l21 * l21;
    if (!(d22 > 0.0f)) return tn;
    const float l22 = sqrtf(d22);
    const float l32 = (cyq - l31 * l21) / l22;
    const float d33 = cqq - l31 * l31 - l32 * l32;
    if (!(d33 > 0.0f)) return tn;
    const float l33 = sqrtf(d33);
    const float y1 = -dx / l11;
    const float y2 = (-dy - l21 * y1) / l22;
    const float y3 = (-dq - l31 * y1 - l32 * y2) / l33;
    const float u4 = y3 / l33;
    const float u2 = (y2 - l32 * u4) / l22;
    const float u1 = (y1 - l21 * u2 - l31 * u4) / l11;
    const float u0 = -mz - u1 * mx - u2 * my - u4 * mq;
    const float disc = 1.0f - 4.0f * u0 * u4;
    float zs = -2.0f * u0 / (1.0f + sqrtf(fmaxf(disc, 0.0f)));
    zs = clampf(zs, -1.0f, 1.0f);
    return clampf(tn + P.apss_h * zs, 0.0f, (float)(T - 1));
}

constexpr float kDeadDepth = -1.0e12f;   // sentinel depth of dead or absent slots

// Depths of the tile plus halo R; dead slots and pixels outside the frame get
// the sentinel depth.
__device__ __forceinline__ void load_halo_depth(const TileCtx& c, const FrameDesc& F, int R, int K,
                                                const float* src, long long src_stride, int src_off,
                                                const uint8_t* asrc, long long a_stride, float* st)
{
    const int hh = kTileH + 2 * R, hw = kTileW + 2 * R;
    for (int idx = threadIdx.x; idx < hh * hw; idx += blockDim.x) {
        const int hi = idx / hw, hj = idx % hw;
        const int gi = c.i0 - R + hi, gj = c.j0 - R + hj;
        const bool in = gi >= 0 && gi < F.h && gj >= 0 && gj < F.w;
        const int lp = in ? gi * F.w + gj : 0;
        for (int m = 0; m < K; ++m) {
            float v = kDeadDepth;
            if (in && asrc[(long long)m * a_stride + lp]) v = src[(long long)m * src_stride + src_off + lp];
            st[m * kHalo + idx] = v;
        }
    }
}

// Alive points of the tile's own pixels, as (local pixel << 2 | slot).
__device__ __forceinline__ int compact_points(const float* st, int R, int K, bool inb, int li, int lj,
                                              unsigned short* pts, int* s_warp)
{
    const int hstride = kTileW + 2 * R;
    const int q0 = (li + R) * hstride + (lj + R);
    int mine = 0;
    if (inb)
        for (int k = 0; k < K; ++k) mine += st[k * kHalo + q0] != kDeadDepth;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
        if (w < warp) before += s_warp[w];
        total += s_warp[w];
    }
    int pos = before + incl - mine;
    if (inb)
        for (int k = 0; k < K; ++k)
            if (st[k * kHalo + q0] != kDeadDepth) pts[pos++] = (unsigned short)((threadIdx.x << 2) | k);
    return total;
}

// ----------------------------------------------------------------------------
// Phase B: APSS depth denoiser + intensity gradient step.
__global__ void __launch_bounds__(kTileThreads)
k_phase_b(const CallRecord* __restrict__ rec, const Work W)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float st[kMaxK * kHalo];
    __shared__ float s_tn[kMaxK][kTileThreads];
    __shared__ unsigned short s_pts[kMaxK * kTileThreads];
    __shared__ int s_warp[kTileThreads / 32];
    load_irf(pad, P);
    const TileCtx c = tile_ctx(B);
    const FrameDesc& F = B.f[c.fi];
    const int np = F.npix, S = W.stride, R = P.win_r, K = P.k;
    load_halo_depth(c, F, R, K, W.t_half, S, F.pix_base, F.alive, np, st);
    __syncthreads();
    const int hstride = kTileW + 2 * R;
    const int q0 = (c.li + R) * hstride + (c.lj + R);
    for (int k = 0; k < K; ++k) s_tn[k][threadIdx.x] = st[k * kHalo + q0];
    const int n_pts = compact_points(st, R, K, c.inb, c.li, c.lj, s_pts, s_warp);
    __syncthreads();
    if (P.depth_den == RT3D_DEPTH_APSS) {
        for (int i = threadIdx.x; i < n_pts; i += kTileThreads) {
            const int px = s_pts[i] >> 2, k = s_pts[i] & 3;
            const int ci = px / kTileW + R, cj = px % kTileW + R;
            s_tn[k][px] = apss_point(st, hstride, R, K, ci, cj, st[k * kHalo + ci * hstride + cj], P, F.nt);
        }
    } else if (P.depth_den == RT3D_DEPTH_LEARNED) {
        // the network's move where it stays within the fallback bound, APSS elsewhere
        for (int i = threadIdx.x; i < n_pts; i += kTileThreads) {
            const int px = s_pts[i] >> 2, k = s_pts[i] & 3;
            const int ci = px / kTileW + R, cj = px % kTileW + R;
            const float t0 = st[k * kHalo + ci * hstride + cj];
            if (k < 2) {
                const int gi = c.i0 + px / kTileW, gj = c.j0 + px % kTileW;
                const float d = W.net_y[((long long)F.pix_base + gi * F.w + gj) * 2 + k] * P.net_scale;
                if (fabsf(d) <= P.net_fallback) {
                    s_tn[k][px] = clampf(t0 + d, 0.0f, (float)(F.nt - 1));
                    continue;
                }
            }
            s_tn[k][px] = apss_point(st, hstride, R, K, ci, cj, t0, P, F.nt);
        }
    }
    __syncthreads();
    if (c.inb) {
        const int lp = c.gi * F.w + c.gj;
        for (int k = 0; k < K; ++k) {
            const float v = s_tn[k][threadIdx.x];
            // dead slots keep the depth they had
            F.t[(long long)k * np + lp] = v == kDeadDepth ? W.t_half[(long long)k * S + F.pix_base + lp] : v;
        }
    }

    if (!c.inb) return;
    {
        const int lp = c.gi * F.w + c.gj, wp = F.pix_base + lp;
        float tk[kMaxK], rk[kMaxK];
        bool ak[kMaxK];
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            const bool in = k < K;
            const float v = in ? s_tn[k][threadIdx.x] : kDeadDepth;
            ak[k] = v != kDeadDepth;
            tk[k] = ak[k] ? v : 0.0f;
            rk[k] = in ? F.r[(long long)k * np + lp] : 0.0f;
        }
        const float g = F.gain ? F.gain[lp] : 1.0f;
        float sh[kMaxK], sdh[kMaxK], sz;
        pixel_sums(F.ent, W.seg[wp], pad, P, tk, rk, ak, F.b[lp], g, sh, sdh, sz);
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            if (k >= K) continue;
            float rn = rk[k];
            if (ak[k] && g > 0.0f) {
                float H, dH;
                support_sums(pad, P, F.nt, tk[k], H, dH);
                rn = fmaxf(rk[k] - P.r_step * (rk[k] + P.eps_r) * (H - sh[k]), 0.0f);
            }
            W.r_half[(long long)k * S + wp] = rn;
        }
    }
}

// ----------------------------------------------------------------------------
// Phase C: intensity low-pass on the surface + pruning + background gradient step.
__global__ void __launch_bounds__(kTileThreads)
k_phase_c(const CallRecord* __restrict__ rec, const Work W)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float st[kMaxK * kHalo];
    __shared__ float sr[kMaxK * kHalo];
    __shared__ float s_rn[kMaxK][kTileThreads];
    __shared__ uint8_t s_an[kMaxK][kTileThreads];
    __shared__ unsigned short s_pts[kMaxK * kTileThreads];
    __shared__ int s_warp[kTileThreads / 32];
    load_irf(pad, P);
    const TileCtx c = tile_ctx(B);
    const FrameDesc& F = B.f[c.fi];
    const int np = F.npix, S = W.stride, R = P.win_r, K = P.k;
    load_halo_depth(c, F, R, K, F.t, np, 0, F.alive, np, st);
    {
        const int hh = kTileH + 2 * R, hw = kTileW + 2 * R;
        for (int idx = threadIdx.x; idx < hh * hw; idx += blockDim.x) {
            const int hi = idx / hw, hj = idx % hw;
            const int gi = c.i0 - R + hi, gj = c.j0 - R + hj;
            const bool in = gi >= 0 && gi < F.h && gj >= 0 && gj < F.w;
            const int lp = in ? gi * F.w + gj : 0;
            for (int m = 0; m < K; ++m)
                sr[m * kHalo + idx] = in ? W.r_half[(long long)m * S + F.pix_base + lp] : 0.0f;
        }
    }
    __syncthreads();
    const int hstride = kTileW + 2 * R;
    const int q0 = (c.li + R) * hstride + (c.lj + R);
    for (int k = 0; k < K; ++k) {
        const bool al = st[k * kHalo + q0] != kDeadDepth;
        s_an[k][threadIdx.x] = 0;
        s_rn[k][threadIdx.x] = al ? sr[k * kHalo + q0] : (c.inb ? F.r[(long long)k * np + c.gi * F.w + c.gj] : 0.0f);
    }
    const int n_pts = compact_points(st, R, K, c.inb, c.li, c.lj, s_pts, s_warp);
    __syncthreads();
    {
        const float inv_h = 1.0f / P.int_h, px = P.pitch * inv_h;
        for (int i = threadIdx.x; i < n_pts; i += kTileThreads) {
            const int pxl = s_pts[i] >> 2, k = s_pts[i] & 3;
            const int ci = pxl / kTileW + R, cj = pxl % kTileW + R;
            const int qc = ci * hstride + cj;
            float rbar = sr[k * kHalo + qc];
            if (P.int_den) {
                const float tn = st[k * kHalo + qc];
                float num = 0.0f, den = 0.0f;
                for (int di = -R; di <= R; ++di) {
                    const float y = (float)di * px;
                    for (int dj = -R; dj <= R; ++dj) {
                        const float x = (float)dj * px;
                        const float r2 = x * x + y * y;
                        if (!(r2 < 1.0f)) continue;
                        const int q = (ci + di) * hstride + (cj + dj);
                        for (int m = 0; m < K; ++m) {
                            const float z = (st[m * kHalo + q] - tn) * inv_h;
                            const float d2 = r2 + z * z;
                            float w = 1.0f - d2;
                            w *= w;
                            w = d2 < 1.0f ? w * w : 0.0f;
                            num += w * sr[m * kHalo + q];
                            den += w;
                        }
                    }
                }
                rbar = num / den;
            }
            s_rn[k][pxl] = rbar;
            s_an[k][pxl] = rbar >= P.r_min ? 1 : 0;
        }
    }
    __syncthreads();
    if (c.inb) {
        const int lp = c.gi * F.w + c.gj, wp = F.pix_base + lp;
        // same-pixel points closer than merge_dist are one surface: the weaker
        // (the later slot on a tie) is removed and its intensity added to the other
        for (int a = 0; a < K; ++a)
            for (int b2 = a + 1; b2 < K; ++b2) {
                if (!s_an[a][threadIdx.x] || !s_an[b2][threadIdx.x]) continue;
                const float ta = st[a * kHalo + q0], tb = st[b2 * kHalo + q0];
                if (!(fabsf(ta - tb) < P.merge_dist)) continue;
                const int keep = s_rn[b2][threadIdx.x] > s_rn[a][threadIdx.x] ? b2 : a;
                const int drop = keep == a ? b2 : a;
                s_rn[keep][threadIdx.x] += s_rn[drop][threadIdx.x];
                s_an[drop][threadIdx.x] = 0;
            }
        for (int k = 0; k < K; ++k) {
            if (st[k * kHalo + q0] != kDeadDepth) F.r[(long long)k * np + lp] = s_rn[k][threadIdx.x];
            W.alive_b[(long long)k * S + wp] = s_an[k][threadIdx.x];
        }
    }
    __syncthreads();

    if (!c.inb) return;
    {
        const int lp = c.gi * F.w + c.gj, wp = F.pix_base + lp;
        float tk[kMaxK], rk[kMaxK];
        bool ak[kMaxK];
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            const bool in = k < K;
            ak[k] = in && s_an[k][threadIdx.x];
            tk[k] = ak[k] ? st[k * kHalo + q0] : 0.0f;
            rk[k] = in ? s_rn[k][threadIdx.x] : 0.0f;
        }
        const float g = F.gain ? F.gain[lp] : 1.0f;
        const float b = F.b[lp];
        float sh[kMaxK], sdh[kMaxK], sz;
        pixel_sums(F.ent, W.seg[wp], pad, P, tk, rk, ak, b, g, sh, sdh, sz);
        float bn = b;
        if (g > 0.0f) bn = fmaxf(b - P.b_step * (b + P.eps_b) * (1.0f - sz / (float)F.nt), P.b_floor);
        W.b_half[wp] = bn;
    }
}

// ----------------------------------------------------------------------------
// Finaliser: the last iteration's pruning and background denoiser land in the
// result buffers; alive points are counted per frame.
__global__ void __launch_bounds__(kTileThreads)
k_final(const CallRecord* __restrict__ rec, const Work W, int ran)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const TileCtx c = tile_ctx(B);
    const FrameDesc& F = B.f[c.fi];
    int mine = 0;
    if (c.inb) {
        const int lp = c.gi * F.w + c.gj, wp = F.pix_base + lp;
        for (int k = 0; k < P.k; ++k) {
            uint8_t a;
            if (ran) {
                a = W.alive_b[(long long)k * W.stride + wp];
                F.alive[(long long)k * F.npix + lp] = a;
            } else {
                a = F.alive[(long long)k * F.npix + lp];
            }
            mine += a;
        }
        if (ran) F.b[lp] = bkg_filter(P, W.b_half + F.pix_base, F.h, F.w, c.gi, c.gj);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt && F.n_points) atomicAdd(F.n_points, s_cnt);
}

}  // namespace rt3d
