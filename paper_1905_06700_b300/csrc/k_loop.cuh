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

// Tile of this CTA: tile0 + blockIdx.x of the batch (a launch may cover a
// contiguous range of the batch's tiles).
__device__ __forceinline__ TileCtx tile_ctx(const Batch& B, int tile0)
{
    TileCtx c;
    const int tile = tile0 + (int)blockIdx.x;
    c.fi = frame_of_tile(B, tile);
    const FrameDesc& F = B.f[c.fi];
    const int lt = tile - F.tile_base;
    c.i0 = (lt / F.tiles_w) * kTileH;
    c.j0 = (lt % F.tiles_w) * kTileW;
    c.li = threadIdx.x / kTileW;
    c.lj = threadIdx.x % kTileW;
    c.gi = c.i0 + c.li;
    c.gj = c.j0 + c.lj;
    c.inb = c.gi < F.h && c.gj < F.w;
    return c;
}

// The responses' samples with kIrfPad zeros on each side, one region per
// response (IrfRef::pad_off).
__device__ __forceinline__ void load_irf(float* pad, const KParams& P)
{
    for (int i = 0; i < P.n_irf; ++i) {
        const IrfRef R = irf_ref(P, i);
        const float* src = P.irf + P.irf_offs[i];
        for (int q = threadIdx.x; q < R.len + 2 * kIrfPad; q += blockDim.x) {
            const int k = q - kIrfPad;
            pad[R.pad_off + q] = (k >= 0 && k < R.len) ? src[k] : 0.0f;
        }
    }
}

// Catmull-Rom intervals of the IRF, for the bin sums.  Entry i of a
// response's region (IrfRef::coef_off) holds the interval that starts at
// sample k = i - 3,
//   h(k + u) = c.x + u (c.y + u (c.z + u c.w)),   h'(k + u) = c.y + u (2 c.z + 3 c.w u),
// the interpolant of irf_eval with its factor 1/2 folded into the coefficients
// (an exact scaling).  Entries 0 and L + 4 (k = -3 and k = L + 1) are zero: an
// argument outside the support (-2, L + 1) lands on them and gives h = h' = 0.
constexpr int kCoefLen = kMaxIrf + 5;

__device__ __forceinline__ void load_irf_coef(float* pad, float4* coef, const KParams& P)
{
    load_irf(pad, P);
    for (int r = 0; r < P.n_irf; ++r) {
        const IrfRef R = irf_ref(P, r);
        const int L = R.len;
        const float* h = P.irf + P.irf_offs[r];
        for (int i = threadIdx.x; i < L + 5; i += blockDim.x) {
            const int k = i - 3;
            float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (k >= -2 && k <= L) {
                const float pm = k - 1 >= 0 && k - 1 < L ? h[k - 1] : 0.0f;
                const float p0 = k >= 0 && k < L ? h[k] : 0.0f;
                const float p1 = k + 1 >= 0 && k + 1 < L ? h[k + 1] : 0.0f;
                const float p2 = k + 2 >= 0 && k + 2 < L ? h[k + 2] : 0.0f;
                const float c1 = p1 - pm;
                const float c2 = 2.0f * pm - 5.0f * p0 + 4.0f * p1 - p2;
                const float c3 = -pm + 3.0f * p0 - 3.0f * p1 + p2;
                c = make_float4(p0, 0.5f * c1, 0.5f * c2, 0.5f * c3);
            }
            coef[R.coef_off + i] = c;
        }
    }
}

// One (pixel, slot) of the bin sums: a bin tb lies in IRF interval
// tb + base - 3 at fraction u, both fixed by the slot's depth (bins are
// integers): y = tb - t + origin = tb + (origin - t).
__device__ __forceinline__ void slot_frame(int origin, float t, int& base, float& u)
{
    const float y0 = (float)origin - t;
    const float f = floorf(y0);
    base = (int)f + 3;
    u = y0 - f;
}

// Per-pixel record of the bin sums: u[K], base[K], rr[K], b, g and the
// response's coefficient region (offset << 16 | last entry), packed in
// 16-byte words.
template <int K>
struct PixRec {
    static constexpr int NW = (3 * K + 3 + 3) / 4;
    float4 q[NW];
};

// Per-warp scratch of warp_pixel_sums: the 32 pixels' bin ranges and records,
// and the partial sums of pixels whose bins are split between lanes.
template <int K, int NS>
struct WarpSums {
    PixRec<K> rec[32];
    float acc[NS][32], first[NS][32], last[NS][32];
    uint32_t start[32];
    int excl[32], incl[32], nextp[32];
};

// Sums over the nonzero bins of the warp's 32 pixels (one pixel per lane, `on`
// false for lanes outside the frame):
//   MODE 0: out[k] = sum z h'(t - t_k)/lambda          (depth step)
//   MODE 1: out[k] = sum z h(t - t_k)/lambda           (intensity step)
//   MODE 2: out[0] = sum z/lambda                      (background step)
// with lambda = max(g (sum_k rr_k h(t - t_k) + b), lam_floor) and rr_k the
// intensity of an alive slot, 0 for a dead one.
// Work is balanced over lanes, not pixels: the warp's bins, concatenated in
// pixel order, are cut into 32 contiguous runs of equal length (+-1) and lane
// l sums run l.  A pixel whose bins fall in one run is summed in bin order by
// one lane; a pixel split over lanes l1..l2 is the sum of its per-lane pieces
// added in lane order.  The grouping depends only on the 32 pixels' bin counts,
// so the result is deterministic and independent of the rest of the batch.
template <int K, int MODE, int NSX>
__device__ __forceinline__ void warp_pixel_sums(const uint32_t* __restrict__ ent, uint2 sg, bool on,
                                                const float4* coef, const KParams& P, const IrfRef& ir,
                                                const float* tk, const float* rr, float b, float g,
                                                WarpSums<K, NSX>& S, float* out)
{
    constexpr int NS = MODE == 2 ? 1 : K;
    static_assert(NSX >= NS, "scratch too small for the sums");
    constexpr int NW = PixRec<K>::NW;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int cnt = on ? (int)sg.y : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += n;
    }
    const int E = __shfl_sync(full, incl, 31);
    const int excl = incl - cnt;
    const unsigned nz = __ballot_sync(full, cnt > 0);
    const unsigned above = lane == 31 ? 0u : nz & (full << (lane + 1));
    {
        float w[4 * NW];
#pragma unroll
        for (int i = 0; i < 4 * NW; ++i) w[i] = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int base;
            slot_frame(ir.origin, tk[k], base, w[k]);
            w[K + k] = __int_as_float(base);
            w[2 * K + k] = rr[k];
        }
        w[3 * K] = b;
        w[3 * K + 1] = g;
        w[3 * K + 2] = __int_as_float((ir.coef_off << 16) | (ir.len + 4));
#pragma unroll
        for (int i = 0; i < NW; ++i) S.rec[lane].q[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    }
    S.start[lane] = on ? sg.x : 0u;
    S.excl[lane] = excl;
    S.incl[lane] = incl;
    S.nextp[lane] = above ? __ffs(above) - 1 : 32;
    __syncwarp();

    const float lam_floor = P.lam_floor;
    const int lo = (lane * E) >> 5, hi = ((lane + 1) * E) >> 5;
    if (lo < hi) {
        // the pixel holding bin lo: the first with incl > lo (it is nonempty)
        int p = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1)
            if (S.incl[p + s - 1] <= lo) p += s;
        float up[K], rp[K], bp, gp;
        int basep[K];
        unsigned coffp, cmaxp;   // the pixel's coefficient region and its last (zero) entry
        auto load_pixel = [&](int q) {
            float w[4 * NW];
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const float4 v = S.rec[q].q[i];
                w[4 * i] = v.x;
                w[4 * i + 1] = v.y;
                w[4 * i + 2] = v.z;
                w[4 * i + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                up[k] = w[k];
                basep[k] = __float_as_int(w[K + k]);
                rp[k] = w[2 * K + k];
            }
            bp = w[3 * K];
            gp = w[3 * K + 1];
            const unsigned cw = __float_as_uint(w[3 * K + 2]);
            coffp = cw >> 16;
            cmaxp = cw & 0xffffu;
        };
        float part[NS];
        // a piece of pixel q ends: a lane's first piece of a pixel begun in an
        // earlier run goes to first, a piece that continues into the next run
        // to last, a whole pixel to acc
        auto flush = [&](int q, bool starts_in, bool ends_in) {
            float* dst = !starts_in ? &S.first[0][lane] : (!ends_in ? &S.last[0][lane] : &S.acc[0][q]);
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                dst[32 * j] = part[j];
                part[j] = 0.0f;
            }
        };
#pragma unroll
        for (int j = 0; j < NS; ++j) part[j] = 0.0f;
        load_pixel(p);
        int p_incl = S.incl[p];
        bool starts_in = S.excl[p] == lo;
        bool open = true;
        uint32_t addr = S.start[p] + (uint32_t)(lo - S.excl[p]);
        uint32_t v = ent[addr];
        for (int e = lo; e < hi; ++e) {
            const uint32_t cur = v;
            const bool cross = e + 1 == p_incl;
            const bool more = e + 1 < hi;
            int q = p;
            uint32_t naddr = addr + 1;
            if (cross && more) {
                q = S.nextp[p];
                naddr = S.start[q];
            }
            if (more) v = ent[naddr];
            const int tb = (int)(cur >> 16);
            const float z = (float)(cur & 0xffffu);
            float hv[K], dv[K];
            float acc = bp;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float4 c = coef[coffp + min((unsigned)(tb + basep[k]), cmaxp)];
                const float u = up[k];
                hv[k] = c.x + u * (c.y + u * (c.z + u * c.w));
                dv[k] = c.y + u * (2.0f * c.z + 3.0f * c.w * u);
                acc += rp[k] * hv[k];
            }
            const float lam = fmaxf(gp * acc, lam_floor);
            const float inv = __fdividef(z, lam);
            if (MODE == 2) {
                part[0] += inv;
            } else {
#pragma unroll
                for (int k = 0; k < NS; ++k) part[k] += (MODE == 0 ? dv[k] : hv[k]) * inv;
            }
            if (cross) {
                flush(p, starts_in, true);
                open = false;
                if (more) {
                    p = q;
                    load_pixel(p);
                    p_incl = S.incl[p];
                    starts_in = true;
                    open = true;
                }
            }
            addr = naddr;
        }
        if (open) flush(p, starts_in, false);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NS; ++j) out[j] = 0.0f;
    if (cnt > 0) {
        // lanes holding this pixel's first and last bin
        const int l1 = (32 * excl + 31) / E, l2 = (32 * incl - 1) / E;
        if (l1 == l2) {
#pragma unroll
            for (int j = 0; j < NS; ++j) out[j] = S.acc[j][lane];
        } else {
#pragma unroll
            for (int j = 0; j < NS; ++j) out[j] = S.last[j][l1];
            for (int l = l1 + 1; l <= l2; ++l) {
                if (((l * E) >> 5) == (((l + 1) * E) >> 5)) continue;   // empty run
#pragma unroll
                for (int j = 0; j < NS; ++j) out[j] += S.first[j][l];
            }
        }
    }
    __syncwarp();
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

// Depth gradient step of one pixel's slots (Results, "Depth update": a scaled
// gradient step on the negative log-likelihood, clamped to dt_max and to the
// histogram) from its bin sums sdh[k] = sum z h'(t - t_k)/lambda.
template <int K>
__device__ __forceinline__ void depth_step(const float* pad, const KParams& P, const IrfRef& ir, int T,
                                           const float* tk, const float* rk, const bool* ak, float g,
                                           const float* sdh, float* t_half, long long stride)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float tn = tk[k];
        if (ak[k] && g > 0.0f) {
            float H, dH;
            support_sums(pad, ir, T, tk[k], H, dH);
            const float grad = g * rk[k] * (-dH + sdh[k]);
            const float beta = P.t_step / (g * rk[k] + P.eps_r);
            const float step = clampf(-beta * grad, -P.dt_max, P.dt_max);
            tn = clampf(tk[k] + step, 0.0f, (float)(T - 1));
        }
        t_half[(long long)k * stride] = tn;
    }
}

// ----------------------------------------------------------------------------
// Phase A: background denoiser of the previous iteration + depth gradient step,
// one thread per pixel (the bin sums shared out over the warp).
template <int K>
__global__ void __launch_bounds__(kTileThreads)
k_phase_a(const CallRecord* __restrict__ rec, const Work W, int first, int tile0)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float4 coef[kCoefLen];
    __shared__ WarpSums<K, K> ws[kTileThreads / 32];
    load_irf_coef(pad, coef, P);
    __syncthreads();
    const TileCtx c = tile_ctx(B, tile0);
    const FrameDesc& F = B.f[c.fi];
    const int np = F.npix, S = W.stride;
    const int lp = c.inb ? c.gi * F.w + c.gj : 0, wp = F.pix_base + lp;
    const uint2 sg = c.inb ? W.seg[wp] : make_uint2(0u, 0u);
    const IrfRef ir = irf_ref(P, c.inb ? pixel_irf(P, F, lp) : 0);
    float b = 0.0f, g = 0.0f;
    float tk[K], rk[K], rr[K];
    bool ak[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        tk[k] = 0.0f;
        rk[k] = 0.0f;
        ak[k] = false;
    }
    if (c.inb) {
        // every load before the first store (one memory round trip)
        uint8_t a[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a[k] = first ? F.alive[(long long)k * np + lp] : W.alive_b[(long long)k * S + wp];
            tk[k] = F.t[(long long)k * np + lp];
            rk[k] = F.r[(long long)k * np + lp];
        }
        g = F.gain ? F.gain[lp] : 1.0f;
        b = first ? F.b[lp] : bkg_filter(P, W.b_half + F.pix_base, F.h, F.w, c.gi, c.gj);
        if (!first) {
            F.b[lp] = b;
#pragma unroll
            for (int k = 0; k < K; ++k) F.alive[(long long)k * np + lp] = a[k];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) ak[k] = a[k] != 0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) rr[k] = ak[k] ? rk[k] : 0.0f;
    float sdh[K];
    warp_pixel_sums<K, 0>(F.ent, sg, c.inb, coef, P, ir, tk, rr, b, g, ws[threadIdx.x >> 5], sdh);
    if (!c.inb) return;
    depth_step<K>(pad, P, ir, F.nt, tk, rk, ak, g, sdh, W.t_half + wp, S);
}

// ----------------------------------------------------------------------------
constexpr int kHaloH = kTileH + 2 * kMaxWinR, kHaloW = kTileW + 2 * kMaxWinR;
constexpr int kHalo = kHaloH * kHaloW;

// Window cells inside the lateral radius.  A neighbourhood sum (APSS moments,
// intensity low-pass) runs over the cells (di, dj) of the (2R+1)^2 window whose
// lateral distance, in units of the kernel radius h, is below one: the unit
// disk.  The cells are listed once per tile, row-major (the order the sums run
// in), with what the sums need of them, so the per-point loops carry no window
// index arithmetic and no radius test.  The first three warps build the list:
// win_vote (one vote per warp, before the tile's first barrier) and win_fill
// (entries at their ranks, after it; readable after the next barrier).
constexpr int kMaxWinCells = (2 * kMaxWinR + 1) * (2 * kMaxWinR + 1);
static_assert(kMaxWinCells <= 96 && kTileThreads >= 96, "three warps vote over the window cells");

__device__ __forceinline__ void win_cell(int t, int R, float px, int& di, int& dj, float& x, float& y,
                                         float& r2)
{
    const int n = 2 * R + 1;
    di = t / n - R;
    dj = t % n - R;
    y = (float)di * px;
    x = (float)dj * px;
    r2 = x * x + y * y;
}

__device__ __forceinline__ void win_vote(unsigned* vote, int R, float px)
{
    if (threadIdx.x >= 96) return;
    const int t = threadIdx.x;
    bool in = false;
    if (t < (2 * R + 1) * (2 * R + 1)) {
        int di, dj;
        float x, y, r2;
        win_cell(t, R, px, di, dj, x, y, r2);
        in = r2 < 1.0f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if ((t & 31) == 0) vote[t >> 5] = m;
}

// Cell list entries.  APSS (kApss): {x, y, r2, halo offset} and the cell's
// packed indicator words -- (di+4) | (dj+4) << 12, di^2 | dj^2 << 13 and
// 1 | (di dj + 16) << 9 -- whose multiples by a slot count sum, field by field
// and without carries (at most 4 slots x 81 cells), to the exact pixel-offset
// moments of the weighted neighbours, then the cell's depth bound
// h sqrt(1 - r2) (bins) of the window test.  Low-pass: {r2, halo offset}.
template <bool kApss>
__device__ __forceinline__ int win_fill(const unsigned* vote, int R, float px, int hstride, float4* g4,
                                        uint4* ind, float2* g2, float h = 0.0f)
{
    const unsigned v0 = vote[0], v1 = vote[1], v2 = vote[2];
    const int t = threadIdx.x;
    if (t < 96) {
        const int w = t >> 5, l = t & 31;
        const unsigned mw = w == 0 ? v0 : (w == 1 ? v1 : v2);
        if ((mw >> l) & 1u) {
            const int rank = (w > 0 ? __popc(v0) : 0) + (w > 1 ? __popc(v1) : 0) + __popc(mw & ((1u << l) - 1u));
            int di, dj;
            float x, y, r2;
            win_cell(t, R, px, di, dj, x, y, r2);
            const int q = di * hstride + dj;
            if constexpr (kApss) {
                g4[rank] = make_float4(x, y, r2, __int_as_float(q));
                ind[rank] = make_uint4((unsigned)(di + 4) | ((unsigned)(dj + 4) << 12),
                                       (unsigned)(di * di) | ((unsigned)(dj * dj) << 13),
                                       1u | ((unsigned)(di * dj + 16) << 9),
                                       __float_as_uint(h * sqrtf(1.0f - r2)));
            } else {
                g2[rank] = make_float2(r2, __int_as_float(q));
            }
        }
    }
    return __popc(v0) + __popc(v1) + __popc(v2);
}

// Depth denoiser variants of phase B (template argument V):
constexpr int kDenApss = 0;       // APSS, solve in FP32
constexpr int kDenApss64 = 1;     // APSS, solve in FP64
constexpr int kDenPlane = 2;      // local plane fit
constexpr int kDenBilateral = 3;  // bilateral depth filter

// FP64 reciprocal and reciprocal square root for the FP64 solve: the
// single-precision hardware approximation refined by one Newton-Raphson step
// in double, y <- y (2 - x y) and y <- y (3 - x y^2) / 2, which squares the
// seed's relative error (about 2^-22) to about 2^-44.
__device__ __forceinline__ double rcp64(double x)
{
    const double y = (double)__frcp_rn((float)x);
    return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ double rsqrt64(double x)
{
    const double y = (double)rsqrtf((float)x);
    return y * fma(-0.5 * x, y * y, 1.5);
}

// Depth denoiser of one point (Results, "Depth update"), over the window
// cells of the unit disk (win_fill's list; qc is the point's halo index).
// Dead or absent slots hold a far sentinel depth, so their weight is exactly
// zero; each thread accumulates only the slots inside the window (in slot
// order).  Local coordinates are scaled by 1/h and taken about the point
// itself; weights (1 - d^2)^4.
//   APSS (Guennebaud & Gross): the weighted algebraic-sphere fit
//     s(x) = u0 + u1 x + u2 y + z + u4 |x|^2, solved as the 3x3 normal
//     equations of (x, y, |x|^2) against z about the weighted means
//     (covariances from the raw moments, E[ab] - E[a] E[b]), then u0 from the
//     means; projection along the line of sight onto s = 0.  kDenApss64 takes
//     the covariances, the Cholesky solve and the projection in FP64 from the
//     FP32 moments.
//   Plane fit: the same without the sphere term (2x2 system), z* = -u0.
//   Bilateral: z* = sum w z / sum w.
// A point with fewer than apss_min_nb weighted neighbours (or, for the fits,
// collinear pixel offsets) keeps its depth.
template <int K, int V>
__device__ float apss_point(const float* st, const float4* wg, const uint4* wi, int n_off, int qc, float tn,
                            const KParams& P, int T)
{
    constexpr bool kSphere = V == kDenApss || V == kDenApss64;
    constexpr bool kFit = V != kDenBilateral;
    const float inv_h = 1.0f / P.apss_h;
    float S0 = 0.f, Sx = 0.f, Sy = 0.f, Sz = 0.f, Sq = 0.f;
    float Sxx = 0.f, Sxy = 0.f, Syy = 0.f, Sxq = 0.f, Syq = 0.f, Sqq = 0.f;
    float Sxz = 0.f, Syz = 0.f, Sqz = 0.f;
    // packed indicator sums of the pixel offsets of weighted neighbours (exact)
    unsigned ia = 0u, ib = 0u, ic = 0u;
    for (int o = 0; o < n_off; ++o) {
        const float4 gc = wg[o];
        const float x = gc.x, y = gc.y, r2 = gc.z;
        const int q = qc + __float_as_int(gc.w);
        const uint4 pk = wi[o];
        // inside the window iff d^2 = r2 + (dt / h)^2 < 1, i.e. |dt| < h sqrt(1 - r2),
        // the cell's depth bound: one subtraction and one compare per slot;
        // only the slots inside accumulate, the others have weight exactly
        // zero and would leave every sum unchanged
        const float dlim = __uint_as_float(pk.w);
        float dk[K];
        unsigned in = 0u;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            dk[m] = st[m * kHalo + q] - tn;
            if (fabsf(dk[m]) < dlim) in |= 1u << m;
        }
        const unsigned cnt = __popc(in);
        while (in) {
            const int m = __ffs(in) - 1;
            in &= in - 1u;
            float dd = dk[0];
#pragma unroll
            for (int j = 1; j < K; ++j)
                if (m == j) dd = dk[j];
            const float z = dd * inv_h;
            const float d2 = r2 + z * z;
            float w = 1.0f - d2;
            w *= w;
            w = w * w;
            if constexpr (kSphere) {
                const float wx = w * x, wy = w * y, wq = w * d2;
                S0 += w; Sx += wx; Sy += wy; Sz += w * z; Sq += wq;
                Sxx += wx * x; Sxy += wx * y; Syy += wy * y;
                Sxq += wx * d2; Syq += wy * d2; Sqq += wq * d2;
                Sxz += wx * z; Syz += wy * z; Sqz += wq * z;
            } else if constexpr (kFit) {
                const float wx = w * x, wy = w * y;
                S0 += w; Sx += wx; Sy += wy; Sz += w * z;
                Sxx += wx * x; Sxy += wx * y; Syy += wy * y;
                Sxz += wx * z; Syz += wy * z;
            } else {
                S0 += w; Sz += w * z;
            }
        }
        ia += cnt * pk.x;
        ib += cnt * pk.y;
        ic += cnt * pk.z;
    }
    const long long n = (long long)(ic & 511u);
    if (n < P.apss_min_nb) return tn;
    float zs = 0.0f;
    if constexpr (V == kDenBilateral) {
        zs = Sz / S0;
    } else {
        const long long si = (long long)(ia & 4095u) - 4 * n, sj = (long long)(ia >> 12) - 4 * n;
        const long long sii = (long long)(ib & 8191u), sjj = (long long)(ib >> 13);
        const long long sij = (long long)(ic >> 9) - 16 * n;
        const long long vii = n * sii - si * si;
        const long long vjj = n * sjj - sj * sj;
        const long long vij = n * sij - si * sj;
        if (vii * vjj - vij * vij == 0) return tn;      // collinear pixel offsets
        if constexpr (V == kDenApss64) {
            const double iw = rcp64((double)S0);
            const double mx = Sx * iw, my = Sy * iw, mz = Sz * iw, mq = Sq * iw;
            const double cxx = fma((double)Sxx, iw, -mx * mx), cxy = fma((double)Sxy, iw, -mx * my);
            const double cyy = fma((double)Syy, iw, -my * my), cxq = fma((double)Sxq, iw, -mx * mq);
            const double cyq = fma((double)Syq, iw, -my * mq), cqq = fma((double)Sqq, iw, -mq * mq);
            const double dx = fma((double)Sxz, iw, -mx * mz), dy = fma((double)Syz, iw, -my * mz);
            const double dq = fma((double)Sqz, iw, -mq * mz);
            // Cholesky of the 3x3 covariance, with the reciprocal pivots
            if (!(cxx > 0.0)) return tn;
            const double r11 = rsqrt64(cxx);
            const double l21 = cxy * r11, l31 = cxq * r11;
            const double d22 = cyy - l21 * l21;
            if (!(d22 > 0.0)) return tn;
            const double r22 = rsqrt64(d22);
            const double l32 = (cyq - l31 * l21) * r22;
            const double d33 = cqq - l31 * l31 - l32 * l32;
            if (!(d33 > 0.0)) return tn;
            const double r33 = rsqrt64(d33);
            const double y1 = -dx * r11;
            const double y2 = (-dy - l21 * y1) * r22;
            const double y3 = (-dq - l31 * y1 - l32 * y2) * r33;
            const double u4 = y3 * r33;
            const double u2 = (y2 - l32 * u4) * r22;
            const double u1 = (y1 - l21 * u2 - l31 * u4) * r11;
            const double u0 = -mz - u1 * mx - u2 * my - u4 * mq;
            const double disc = 1.0 - 4.0 * u0 * u4;
            const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
            double z64 = -2.0 * u0 * rcp64(1.0 + sq);
            z64 = fmin(fmax(z64, -1.0), 1.0);
            const double t64 = (double)tn + (double)P.apss_h * z64;
            return (float)fmin(fmax(t64, 0.0), (double)(T - 1));
        } else if constexpr (kSphere) {
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
            zs = -2.0f * u0 / (1.0f + sqrtf(fmaxf(disc, 0.0f)));
        } else {
            // plane: the 2x2 covariance of (x, y) against z
            const float iw = 1.0f / S0;
            const float mx = Sx * iw, my = Sy * iw, mz = Sz * iw;
            const float cxx = Sxx * iw - mx * mx, cxy = Sxy * iw - mx * my, cyy = Syy * iw - my * my;
            const float dx = Sxz * iw - mx * mz, dy = Syz * iw - my * mz;
            if (!(cxx > 0.0f)) return tn;
            const float l11 = sqrtf(cxx);
            const float l21 = cxy / l11;
            const float d22 = cyy - l21 * l21;
            if (!(d22 > 0.0f)) return tn;
            const float l22 = sqrtf(d22);
            const float y1 = -dx / l11;
            const float y2 = (-dy - l21 * y1) / l22;
            const float u2 = y2 / l22;
            const float u1 = (y1 - l21 * u2) / l11;
            const float u0 = -mz - u1 * mx - u2 * my;
            zs = -u0;
        }
    }
    zs = clampf(zs, -1.0f, 1.0f);
    return clampf(tn + P.apss_h * zs, 0.0f, (float)(T - 1));
}

constexpr float kDeadDepth = -1.0e12f;   // sentinel depth of dead or absent slots

constexpr int kHaloIters = (kHalo + kTileThreads - 1) / kTileThreads;

// Depths of the tile plus halo R (dead slots and pixels outside the frame get
// the sentinel depth) and, with kWithR, a second per-slot field (0 outside the
// frame).  Every global load is issued before the first shared store, so the
// halo costs one memory round trip.
template <int K, bool kWithR>
__device__ __forceinline__ void load_halo(const TileCtx& c, const FrameDesc& F, int R,
                                          const float* src, long long src_stride, int src_off,
                                          const uint8_t* asrc, long long a_stride, float* st,
                                          const float* rsrc, long long r_stride, int r_off, float* sr)
{
    const int hh = kTileH + 2 * R, hw = kTileW + 2 * R, n = hh * hw;
    float tv[kHaloIters][K], rv[kHaloIters][K];
    uint8_t av[kHaloIters][K];
    bool inn[kHaloIters];
#pragma unroll
    for (int it = 0; it < kHaloIters; ++it) {
        const int idx = threadIdx.x + it * kTileThreads;
        const int hi = idx / hw, hj = idx % hw;
        const int gi = c.i0 - R + hi, gj = c.j0 - R + hj;
        const bool in = idx < n && gi >= 0 && gi < F.h && gj >= 0 && gj < F.w;
        const int lp = in ? gi * F.w + gj : 0;
        inn[it] = in;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            av[it][m] = 0;
            tv[it][m] = 0.0f;
            rv[it][m] = 0.0f;
            if (in) {
                av[it][m] = asrc[(long long)m * a_stride + lp];
                tv[it][m] = src[(long long)m * src_stride + src_off + lp];
                if (kWithR) rv[it][m] = rsrc[(long long)m * r_stride + r_off + lp];
            }
        }
    }
#pragma unroll
    for (int it = 0; it < kHaloIters; ++it) {
        const int idx = threadIdx.x + it * kTileThreads;
        if (idx >= n) continue;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            st[m * kHalo + idx] = inn[it] && av[it][m] ? tv[it][m] : kDeadDepth;
            if (kWithR) sr[m * kHalo + idx] = inn[it] ? rv[it][m] : 0.0f;
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
// Phase B: depth denoiser (variant V of apss_point; the learned network with
// V as its fallback) + intensity gradient step.  alive_from_b: the previous
// phase C ran this iteration's depth step, so the alive flags are still in
// alive_b; they land in the frame here (phase C reads them there).
template <int K, int V>
__global__ void __launch_bounds__(kTileThreads, 7)
k_phase_b(const CallRecord* __restrict__ rec, const Work W, int alive_from_b, int tile0)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float st[K * kHalo];
    __shared__ float s_tn[K][kTileThreads];
    __shared__ unsigned short s_pts[K * kTileThreads];
    __shared__ int s_warp[kTileThreads / 32];
    __shared__ float4 coef[kCoefLen];
    __shared__ WarpSums<K, K> ws[kTileThreads / 32];
    __shared__ float4 s_wg[kMaxWinCells];
    __shared__ uint4 s_wi[kMaxWinCells];
    __shared__ unsigned s_vote[3];
    load_irf_coef(pad, coef, P);
    const TileCtx c = tile_ctx(B, tile0);
    const FrameDesc& F = B.f[c.fi];
    const int np = F.npix, S = W.stride, R = P.win_r;
    const int lp = c.inb ? c.gi * F.w + c.gj : 0, wp = F.pix_base + lp;
    // with super-resolution this kernel runs the depth denoiser on the world
    // grid only (the intensity step is per lidar pixel: k_sr_step)
    const bool sres = P.up > 1;
    const uint2 sg = c.inb && !sres ? W.seg[wp] : make_uint2(0u, 0u);
    const IrfRef ir = irf_ref(P, c.inb && !sres ? pixel_irf(P, F, lp) : 0);
    const bool apss = P.depth_den != RT3D_DEPTH_NONE;
    const float apss_px = P.pitch * (1.0f / P.apss_h);
    if (apss) win_vote(s_vote, R, apss_px);
    if (alive_from_b)
        load_halo<K, false>(c, F, R, W.t_half, S, F.pix_base, W.alive_b + F.pix_base, S, st, nullptr, 0, 0,
                            nullptr);
    else
        load_halo<K, false>(c, F, R, W.t_half, S, F.pix_base, F.alive, np, st, nullptr, 0, 0, nullptr);
    __syncthreads();
    const int hstride = kTileW + 2 * R;
    const int q0 = (c.li + R) * hstride + (c.lj + R);
    const int n_off = apss ? win_fill<true>(s_vote, R, apss_px, hstride, s_wg, s_wi, nullptr, P.apss_h) : 0;
    for (int k = 0; k < K; ++k) s_tn[k][threadIdx.x] = st[k * kHalo + q0];
    if (alive_from_b && c.inb)
        for (int k = 0; k < K; ++k) F.alive[(long long)k * np + lp] = st[k * kHalo + q0] != kDeadDepth ? 1 : 0;
    const int n_pts = compact_points(st, R, K, c.inb, c.li, c.lj, s_pts, s_warp);
    __syncthreads();
    if (apss && P.depth_den != RT3D_DEPTH_LEARNED) {
        for (int i = threadIdx.x; i < n_pts; i += kTileThreads) {
            const int px = s_pts[i] >> 2, k = s_pts[i] & 3;
            const int ci = px / kTileW + R, cj = px % kTileW + R;
            const int qc = ci * hstride + cj;
            s_tn[k][px] = apss_point<K, V>(st, s_wg, s_wi, n_off, qc, st[k * kHalo + qc], P, F.nt);
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
            s_tn[k][px] = apss_point<K, V>(st, s_wg, s_wi, n_off, ci * hstride + cj, t0, P, F.nt);
        }
    }
    __syncthreads();
    float tk[K], rk[K], rr[K], tn[K];
    bool ak[K];
    float g = 0.0f, b = 0.0f;
    // every load before the first store (one memory round trip)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float v = c.inb ? s_tn[k][threadIdx.x] : kDeadDepth;
        ak[k] = v != kDeadDepth;
        tk[k] = ak[k] ? v : 0.0f;
        rk[k] = c.inb ? F.r[(long long)k * np + lp] : 0.0f;
        rr[k] = ak[k] ? rk[k] : 0.0f;
        // dead slots keep the depth they had
        tn[k] = v;
        if (c.inb && !ak[k]) tn[k] = W.t_half[(long long)k * S + wp];
    }
    if (c.inb) {
        g = F.gain && !sres ? F.gain[lp] : 1.0f;
        b = sres ? 0.0f : F.b[lp];
#pragma unroll
        for (int k = 0; k < K; ++k) F.t[(long long)k * np + lp] = tn[k];
    }
    if (sres) return;
    float sh[K];
    warp_pixel_sums<K, 1>(F.ent, sg, c.inb, coef, P, ir, tk, rr, b, g, ws[threadIdx.x >> 5], sh);
    if (!c.inb) return;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float rn = rk[k];
        if (ak[k] && g > 0.0f) {
            float H, dH;
            support_sums(pad, ir, F.nt, tk[k], H, dH);
            rn = fmaxf(rk[k] - P.r_step * (rk[k] + P.eps_r) * (H - sh[k]), 0.0f);
        }
        W.r_half[(long long)k * S + wp] = rn;
    }
}

// ----------------------------------------------------------------------------
// Phase C: intensity low-pass on the surface + pruning + background gradient step.
// fuse_next (background denoiser = identity): the next iteration's phase A
// follows on the state each thread holds -- b <- b_half, alive <- alive_b (it
// reaches the frame in the next phase B, since neighbours read the frame's
// alive flags here), depth step into t_half.
template <int K>
__global__ void __launch_bounds__(kTileThreads)
k_phase_c(const CallRecord* __restrict__ rec, const Work W, int fuse_next, int tile0)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ float pad[kMaxIrf + 2 * kIrfPad];
    __shared__ float st[K * kHalo];
    __shared__ float sr[K * kHalo];
    __shared__ float s_rn[K][kTileThreads];
    __shared__ uint8_t s_an[K][kTileThreads];
    __shared__ unsigned short s_pts[K * kTileThreads];
    __shared__ int s_warp[kTileThreads / 32];
    __shared__ float4 coef[kCoefLen];
    __shared__ WarpSums<K, K> ws[kTileThreads / 32];
    __shared__ float2 s_wg[kMaxWinCells];
    __shared__ unsigned s_vote[3];
    load_irf_coef(pad, coef, P);
    const TileCtx c = tile_ctx(B, tile0);
    const FrameDesc& F = B.f[c.fi];
    const int np = F.npix, S = W.stride, R = P.win_r;
    const int lp = c.inb ? c.gi * F.w + c.gj : 0, wp = F.pix_base + lp;
    // with super-resolution this kernel runs the intensity denoiser on the
    // world grid only (the background step is per lidar pixel: k_sr_step)
    const bool sres = P.up > 1;
    const uint2 sg = c.inb && !sres ? W.seg[wp] : make_uint2(0u, 0u);
    const IrfRef ir = irf_ref(P, c.inb && !sres ? pixel_irf(P, F, lp) : 0);
    const float int_px = P.pitch * (1.0f / P.int_h);
    if (P.int_den) win_vote(s_vote, R, int_px);
    // own pixel state read with the halo (one memory round trip)
    float r_own[K];
#pragma unroll
    for (int k = 0; k < K; ++k) r_own[k] = c.inb ? F.r[(long long)k * np + lp] : 0.0f;
    const float g_own = c.inb && !sres ? (F.gain ? F.gain[lp] : 1.0f) : 0.0f;
    const float b_own = c.inb && !sres ? F.b[lp] : 0.0f;
    load_halo<K, true>(c, F, R, F.t, np, 0, F.alive, np, st, W.r_half, S, F.pix_base, sr);
    __syncthreads();
    const int hstride = kTileW + 2 * R;
    const int q0 = (c.li + R) * hstride + (c.lj + R);
    const int n_off = P.int_den ? win_fill<false>(s_vote, R, int_px, hstride, nullptr, nullptr, s_wg) : 0;
    for (int k = 0; k < K; ++k) {
        const bool al = st[k * kHalo + q0] != kDeadDepth;
        s_an[k][threadIdx.x] = 0;
        s_rn[k][threadIdx.x] = al ? sr[k * kHalo + q0] : r_own[k];
    }
    const int n_pts = compact_points(st, R, K, c.inb, c.li, c.lj, s_pts, s_warp);
    __syncthreads();
    {
        const float inv_h = 1.0f / P.int_h;
        for (int i = threadIdx.x; i < n_pts; i += kTileThreads) {
            const int pxl = s_pts[i] >> 2, k = s_pts[i] & 3;
            const int ci = pxl / kTileW + R, cj = pxl % kTileW + R;
            const int qc = ci * hstride + cj;
            float rbar = sr[k * kHalo + qc];
            if (P.int_den) {
                const float tn = st[k * kHalo + qc];
                float num = 0.0f, den = 0.0f;
                // the cells of the unit disk (win_fill's list)
                for (int o = 0; o < n_off; ++o) {
                    const float2 gc = s_wg[o];
                    const float r2 = gc.x;
                    const int q = qc + __float_as_int(gc.y);
#pragma unroll
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
                rbar = num / den;
            }
            s_rn[k][pxl] = rbar;
            s_an[k][pxl] = rbar >= P.r_min ? 1 : 0;
        }
    }
    __syncthreads();
    if (c.inb) {
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
    if (sres) return;
    __syncthreads();

    float tk[K], rr[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool ak = c.inb && s_an[k][threadIdx.x];
        tk[k] = ak ? st[k * kHalo + q0] : 0.0f;
        rr[k] = ak ? s_rn[k][threadIdx.x] : 0.0f;
    }
    const float g = g_own, b = b_own;
    float sz;
    warp_pixel_sums<K, 2>(F.ent, sg, c.inb, coef, P, ir, tk, rr, b, g, ws[threadIdx.x >> 5], &sz);
    float bn = b;
    if (c.inb) {
        if (g > 0.0f) bn = fmaxf(b - P.b_step * (b + P.eps_b) * (1.0f - sz / (float)F.nt), P.b_floor);
        W.b_half[wp] = bn;
    }
    if (!fuse_next) return;

    // next iteration: background denoiser (identity) and depth step
    float tka[K], rka[K], rra[K];
    bool aka[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float ts = st[k * kHalo + q0];
        aka[k] = c.inb && s_an[k][threadIdx.x];
        tka[k] = ts != kDeadDepth ? ts : (c.inb ? F.t[(long long)k * np + lp] : 0.0f);
        rka[k] = c.inb ? s_rn[k][threadIdx.x] : 0.0f;
        rra[k] = aka[k] ? rka[k] : 0.0f;
    }
    if (c.inb) F.b[lp] = bn;
    float sdh[K];
    warp_pixel_sums<K, 0>(F.ent, sg, c.inb, coef, P, ir, tka, rra, bn, g, ws[threadIdx.x >> 5], sdh);
    if (!c.inb) return;
    depth_step<K>(pad, P, ir, F.nt, tka, rka, aka, g, sdh, W.t_half + wp, S);
}

// ----------------------------------------------------------------------------
// Finaliser: the last iteration's pruning and background denoiser land in the
// result buffers; alive points are counted per frame.
__global__ void __launch_bounds__(kTileThreads)
k_final(const CallRecord* __restrict__ rec, const Work W, int ran, int tile0)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const TileCtx c = tile_ctx(B, tile0);
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
        if (ran) {
            if (P.up == 1) {
                F.b[lp] = bkg_filter(P, W.b_half + F.pix_base, F.h, F.w, c.gi, c.gj);
            } else if (c.gi % P.up == 0 && c.gj % P.up == 0) {
                // one world pixel per lidar pixel writes that pixel's background
                const int i = c.gi / P.up, j = c.gj / P.up;
                F.b[i * F.lw + j] = bkg_filter(P, W.b_half + F.lpix_base, F.lh, F.lw, i, j);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt && F.n_points) atomicAdd(F.n_points, s_cnt);
}

}  // namespace rt3d
