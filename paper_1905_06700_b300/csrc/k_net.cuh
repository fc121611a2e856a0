// k_net.cuh -- learned depth denoiser (an extension of the method: a small
// convolutional network standing in for the APSS depth step of Results,
// "Depth update"; APSS stays as the per-point fallback).
//
// Network: four 3x3 convolutions, 6 -> 48 -> 48 -> 48 -> 2 channels, zero
// padding, bias, ReLU after the first three.  Input features per pixel, for
// the first two point slots k (dead or absent points give 0): with n the
// alive points of any slot in the 8 neighbouring pixels whose depth lies
// within 4 scale of t_k (the point's surface) and m their mean depth,
//   f_t = clamp((t_k - m) / scale, -4, 4) (0 when n = 0),
//   f_r = log(1 + r_k), f_a = (1 + n) / 9;
// channels (f_t0, f_r0, f_a0, f_t1, f_r1, f_a1).
// Output: y = (dt_0, dt_1) / scale.
//
// Precision: the parameters are FP32 masters; the convolutions use their
// bfloat16 rounding (nearest even), every layer input is stored in bfloat16
// (activations NHWC), sums and the output are FP32.  Training (backward,
// AdamW) is FP32 and treats the roundings as identity.
//
// Tiling: one CTA per 8 x 16 pixel tile of a frame (the loop kernels' tiles),
// one thread per output pixel; the input tile with its one-pixel halo and the
// layer's weights (all input channels, a block of output channels) sit in
// shared memory as FP32; per-pixel rows are padded by one word so that
// neighbouring threads hit different banks.
#pragma once
#include "rt3d_device.cuh"
#include "k_init_tc.cuh"   // tcgen05 / mbarrier helpers

namespace rt3d {

constexpr int kNetLayers = 4;
__host__ __device__ constexpr int net_cin(int l) { return l == 0 ? 6 : 48; }
__host__ __device__ constexpr int net_cout(int l) { return l == 3 ? 2 : 48; }
__host__ __device__ constexpr long net_woff(int l)
{
    return l == 0 ? 0 : net_woff(l - 1) + (long)net_cout(l - 1) * net_cin(l - 1) * 9 + net_cout(l - 1);
}
__host__ __device__ constexpr long net_boff(int l) { return net_woff(l) + (long)net_cout(l) * net_cin(l) * 9; }
constexpr long kNetParams = net_woff(kNetLayers);
static_assert(kNetParams == 45074, "parameter count");
// FP32 copies of the rounded weights, per layer: forward [ci][k][co] and
// backward-data [co][8 - k][ci] (flipped taps, transposed channels)
__host__ __device__ constexpr long net_wfoff(int l)
{
    return l == 0 ? 0 : net_wfoff(l - 1) + (long)net_cout(l - 1) * net_cin(l - 1) * 9;
}
constexpr long kNetWeights = net_wfoff(kNetLayers);
constexpr int kNetCh = 48;                    // widest layer
constexpr int kNetHaloH = kTileH + 2, kNetHaloW = kTileW + 2, kNetHalo = kNetHaloH * kNetHaloW;

__device__ __forceinline__ float bf16_bits_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// round to bfloat16, nearest even (no NaN or infinity reaches here)
__device__ __forceinline__ uint16_t f_to_bf16_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ float bf16_round(float f) { return bf16_bits_to_f(f_to_bf16_bits(f)); }

// Pixel of a tile of the batch (the loop kernels' 8 x 16 tiling).
struct NetPix {
    int fi, gi, gj, lp, pix;   // frame, row, column, pixel in frame, pixel in batch
    bool in;
};

__device__ __forceinline__ NetPix net_pix(const Batch& B, int tile, int li, int lj)
{
    NetPix q;
    q.fi = frame_of_tile(B, tile);
    const FrameDesc& F = B.f[q.fi];
    const int t = tile - F.tile_base;
    q.gi = (t / F.tiles_w) * kTileH + li;
    q.gj = (t % F.tiles_w) * kTileW + lj;
    q.in = q.gi < F.h && q.gj < F.w;
    q.lp = q.gi * F.w + q.gj;
    q.pix = F.pix_base + q.lp;
    return q;
}

// ---------------------------------------------------------------- features

// Depth, intensity and liveness of slot k at pixel q of a frame: a view of
// either the loop's state (half-step depths in the workspace) or a caller's
// [k][h][w] arrays.
struct NetStateView {
    const float* t;     // slot k of pixel lp at t[k * t_slot + t_base + lp]
    const float* r;
    const uint8_t* alive;
    long long t_slot, r_slot, a_slot;
    long long t_base, r_base, a_base;
};

__device__ __forceinline__ void net_features_at(const NetStateView& v, int K, int h, int w, int gi, int gj,
                                                float scale, float (&x)[6])
{
    const int lp = gi * w + gj;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float ft = 0.0f, fr = 0.0f, fa = 0.0f;
        if (k < K && v.alive[k * v.a_slot + v.a_base + lp]) {
            const float tk = v.t[k * v.t_slot + v.t_base + lp];
            const float reach = 4.0f * scale;
            float sum = 0.0f;
            int n = 0;
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj) {
                    if (di == 0 && dj == 0) continue;
                    const int ii = gi + di, jj = gj + dj;
                    if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                    const int q = ii * w + jj;
                    for (int kk = 0; kk < K; ++kk) {
                        if (!v.alive[kk * v.a_slot + v.a_base + q]) continue;
                        const float tq = v.t[kk * v.t_slot + v.t_base + q];
                        if (!(fabsf(tq - tk) <= reach)) continue;
                        sum += tq;
                        ++n;
                    }
                }
            if (n > 0) ft = clampf((tk - sum / (float)n) / scale, -4.0f, 4.0f);
            fr = log1pf(fmaxf(v.r[k * v.r_slot + v.r_base + lp], 0.0f));
            fa = (float)(1 + n) / 9.0f;
        }
        x[3 * k] = ft;
        x[3 * k + 1] = fr;
        x[3 * k + 2] = fa;
    }
}

// Features of the loop's half-step state (t_half, r, alive) -> x [pix][8] bf16
// (channels 6 and 7 zero: the chunk-planar input of the pipelined convolution).
__global__ void __launch_bounds__(kTileThreads)
k_net_features_loop(const CallRecord* __restrict__ rec, const Work W, uint16_t* __restrict__ x, float scale,
                    int alive_from_b)
{
    const Batch& B = rec->B;
    const int K = rec->P.k;
    // the tile's depths and alive flags with a one-pixel margin, read once
    // (every load issued before the first shared store); a neighbour outside
    // the frame is not alive
    __shared__ float s_t[kMaxK][kNetHalo];
    __shared__ uint8_t s_a[kMaxK][kNetHalo];
    const int tile = (int)blockIdx.x;
    const int fi = frame_of_tile(B, tile);
    const FrameDesc& F = B.f[fi];
    const int tl = tile - F.tile_base;
    const int i0 = (tl / F.tiles_w) * kTileH - 1, j0 = (tl % F.tiles_w) * kTileW - 1;
    // after a phase C that ran the depth step the alive flags are still in alive_b
    const uint8_t* alive = alive_from_b ? W.alive_b + F.pix_base : F.alive;
    const long long a_slot = alive_from_b ? (long long)W.stride : (long long)F.npix;
    constexpr int kIters = (kNetHalo + kTileThreads - 1) / kTileThreads;
    float tv[kIters][kMaxK];
    uint8_t av[kIters][kMaxK];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        const int e = (int)threadIdx.x + it * kTileThreads;
        const int gi = i0 + e / kNetHaloW, gj = j0 + e % kNetHaloW;
        const bool in = e < kNetHalo && gi >= 0 && gi < F.h && gj >= 0 && gj < F.w;
        const int lp = in ? gi * F.w + gj : 0;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            av[it][k] = 0;
            tv[it][k] = 0.0f;
            if (in && k < K) {
                av[it][k] = alive[k * a_slot + lp];
                tv[it][k] = W.t_half[(long long)k * W.stride + F.pix_base + lp];
            }
        }
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
        const int e = (int)threadIdx.x + it * kTileThreads;
        if (e >= kNetHalo) continue;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k) {
            s_a[k][e] = av[it][k];
            s_t[k][e] = tv[it][k];
        }
    }
    __syncthreads();
    const int li = (int)threadIdx.x / kTileW, lj = (int)threadIdx.x % kTileW;
    const int gi = i0 + 1 + li, gj = j0 + 1 + lj;
    if (gi >= F.h || gj >= F.w) return;
    const int lp = gi * F.w + gj;
    const int c0 = (li + 1) * kNetHaloW + (lj + 1);
    // the features of net_features_at, in the same order of operations
    float f[6];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float ft = 0.0f, fr = 0.0f, fa = 0.0f;
        if (k < K && s_a[k][c0]) {
            const float tk = s_t[k][c0];
            const float reach = 4.0f * scale;
            float sum = 0.0f;
            int n = 0;
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj) {
                    if (di == 0 && dj == 0) continue;
                    const int q = c0 + di * kNetHaloW + dj;
                    for (int kk = 0; kk < K; ++kk) {
                        if (!s_a[kk][q]) continue;
                        const float tq = s_t[kk][q];
                        if (!(fabsf(tq - tk) <= reach)) continue;
                        sum += tq;
                        ++n;
                    }
                }
            if (n > 0) ft = clampf((tk - sum / (float)n) / scale, -4.0f, 4.0f);
            fr = log1pf(fmaxf(F.r[(long long)k * F.npix + lp], 0.0f));
            fa = (float)(1 + n) / 9.0f;
        }
        f[3 * k] = ft;
        f[3 * k + 1] = fr;
        f[3 * k + 2] = fa;
    }
    // chunk-planar with 8 channels (the last two zero): one 16-byte row per pixel
    const uint32_t w0 = (uint32_t)f_to_bf16_bits(f[0]) | ((uint32_t)f_to_bf16_bits(f[1]) << 16);
    const uint32_t w1 = (uint32_t)f_to_bf16_bits(f[2]) | ((uint32_t)f_to_bf16_bits(f[3]) << 16);
    const uint32_t w2 = (uint32_t)f_to_bf16_bits(f[4]) | ((uint32_t)f_to_bf16_bits(f[5]) << 16);
    *reinterpret_cast<uint4*>(x + (long long)(F.pix_base + lp) * 8) = make_uint4(w0, w1, w2, 0u);
}

// Features of n caller images, state [n][K][h][w] -> x [n][6][h][w] (FP32
// holding the bf16-rounded values).
__global__ void k_net_features_images(int n, int K, int h, int w, const float* __restrict__ t,
                                      const float* __restrict__ r, const uint8_t* __restrict__ alive,
                                      float scale, float* __restrict__ x)
{
    const long long npix = (long long)h * w;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * npix) return;
    const int im = (int)(idx / npix);
    const int lp = (int)(idx % npix);
    const long long base = (long long)im * K * npix;
    NetStateView v{t, r, alive, npix, npix, npix, base, base, base};
    float f[6];
    net_features_at(v, K, h, w, lp / w, lp % w, scale, f);
#pragma unroll
    for (int c = 0; c < 6; ++c) x[((long long)im * 6 + c) * npix + lp] = bf16_round(f[c]);
}

// x [n][6][h][w] FP32 -> NHWC bf16
__global__ void k_net_pack_input(long long npix, int n, const float* __restrict__ x, uint16_t* __restrict__ a0)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * npix) return;
    const long long im = idx / npix, p = idx % npix;
#pragma unroll
    for (int c = 0; c < 6; ++c) a0[idx * 6 + c] = f_to_bf16_bits(x[(im * 6 + c) * npix + p]);
}

// ------------------------------------------------------------- convolution

enum NetConvMode { kConvHidden = 0, kConvOut = 1, kConvBackData = 2 };

__host__ __device__ constexpr int net_conv_smem(int ci, int co_blk)
{
    return (kNetHalo * (ci + 1) + ci * 9 * co_blk) * 4;
}

// One 3x3 convolution over the batch's tiles.  blockIdx.y selects a block of
// CO_BLK output channels.
//   kConvHidden:   in bf16 [pix][CI] -> relu(conv + b) as bf16 [pix][CO]
//   kConvOut:      in bf16 [pix][CI] -> conv + b as FP32 [pix][CO]
//   kConvBackData: in FP32 gradients [pix][CI] -> conv * (ref > 0) as FP32
//                  [pix][CO] (ref: the stored activations of the layer input)
// wt: FP32 [CI][9][CO] (flipped and transposed for kConvBackData).
template <int CI, int CO, int CO_BLK, int MODE>
__global__ void __launch_bounds__(kTileThreads)
k_net_conv(const Batch* __restrict__ Bp, const void* __restrict__ in, const float* __restrict__ wt,
           const float* __restrict__ bias, void* __restrict__ out, const uint16_t* __restrict__ ref)
{
    const Batch& B = *Bp;
    extern __shared__ float net_smem[];
    float* s_in = net_smem;                                  // [halo px][CI + 1]
    float* s_w = net_smem + kNetHalo * (CI + 1);             // [CI][9][CO_BLK]
    const int co0 = blockIdx.y * CO_BLK;
    const int tile = blockIdx.x;
    const int fi = frame_of_tile(B, tile);
    const FrameDesc& F = B.f[fi];
    const int t = tile - F.tile_base;
    const int gi0 = (t / F.tiles_w) * kTileH - 1, gj0 = (t % F.tiles_w) * kTileW - 1;
    // weights of this output block
    for (int e = threadIdx.x; e < CI * 9 * CO_BLK; e += kTileThreads) {
        const int c = e % CO_BLK, rest = e / CO_BLK;
        s_w[e] = wt[(long long)rest * CO + co0 + c];
    }
    // input tile with halo (zero outside the frame)
    for (int e = threadIdx.x; e < kNetHalo * CI; e += kTileThreads) {
        const int hp = e / CI, c = e % CI;
        const int gi = gi0 + hp / kNetHaloW, gj = gj0 + hp % kNetHaloW;
        float v = 0.0f;
        if (gi >= 0 && gi < F.h && gj >= 0 && gj < F.w) {
            const long long p = (long long)F.pix_base + gi * F.w + gj;
            if (MODE == kConvBackData) v = static_cast<const float*>(in)[p * CI + c];
            else v = bf16_bits_to_f(static_cast<const uint16_t*>(in)[p * CI + c]);
        }
        s_in[hp * (CI + 1) + c] = v;
    }
    __syncthreads();
    const int li = threadIdx.x / kTileW, lj = threadIdx.x % kTileW;
    const int gi = gi0 + 1 + li, gj = gj0 + 1 + lj;
    if (gi >= F.h || gj >= F.w) return;
    float acc[CO_BLK];
#pragma unroll
    for (int c = 0; c < CO_BLK; ++c) acc[c] = (MODE == kConvBackData) ? 0.0f : bias[co0 + c];
    for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = s_in[((li + k / 3) * kNetHaloW + lj + k % 3) * (CI + 1) + ci];
            const float* wk = s_w + (ci * 9 + k) * CO_BLK;
#pragma unroll
            for (int c = 0; c < CO_BLK; ++c) acc[c] = fmaf(v, wk[c], acc[c]);
        }
    }
    const long long p = (long long)F.pix_base + gi * F.w + gj;
    if (MODE == kConvHidden) {
        uint16_t* o = static_cast<uint16_t*>(out) + p * CO + co0;
#pragma unroll
        for (int c = 0; c < CO_BLK; ++c) o[c] = f_to_bf16_bits(fmaxf(acc[c], 0.0f));
    } else if (MODE == kConvOut) {
        float* o = static_cast<float*>(out) + p * CO + co0;
#pragma unroll
        for (int c = 0; c < CO_BLK; ++c) o[c] = acc[c];
    } else {
        float* o = static_cast<float*>(out) + p * CO + co0;
        const uint16_t* rr = ref + p * CO + co0;
#pragma unroll
        for (int c = 0; c < CO_BLK; ++c) o[c] = bf16_bits_to_f(rr[c]) > 0.0f ? acc[c] : 0.0f;
    }
}

// Weight and bias gradients of one layer: dW[co][ci][k] += sum_p dz[p][co]
// a[p + k][ci], db[co] += sum_p dz[p][co], over the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  One thread per (ci, k); each CTA adds its sums
// once (atomics into the FP32 gradient vector).
template <int CI, int CO>
__global__ void __launch_bounds__(((CI * 9 + 31) / 32) * 32)
k_net_wgrad(const Batch* __restrict__ Bp, const uint16_t* __restrict__ a, const float* __restrict__ dz,
            float* __restrict__ dW, float* __restrict__ db)
{
    const Batch& B = *Bp;
    extern __shared__ float net_smem[];
    float* s_a = net_smem;                                   // [halo px][CI + 1]
    float* s_dz = net_smem + kNetHalo * (CI + 1);            // [128][CO]
    const int item = threadIdx.x;                            // (ci, k)
    const bool active = item < CI * 9;
    const int ci = active ? item / 9 : 0, k = active ? item % 9 : 0;
    float acc[CO];
#pragma unroll
    for (int c = 0; c < CO; ++c) acc[c] = 0.0f;
    float bacc = 0.0f;
    for (int tile = blockIdx.x; tile < B.total_tiles; tile += gridDim.x) {
        const int fi = frame_of_tile(B, tile);
        const FrameDesc& F = B.f[fi];
        const int t = tile - F.tile_base;
        const int gi0 = (t / F.tiles_w) * kTileH - 1, gj0 = (t % F.tiles_w) * kTileW - 1;
        __syncthreads();
        for (int e = threadIdx.x; e < kNetHalo * CI; e += blockDim.x) {
            const int hp = e / CI, c = e % CI;
            const int gi = gi0 + hp / kNetHaloW, gj = gj0 + hp % kNetHaloW;
            float v = 0.0f;
            if (gi >= 0 && gi < F.h && gj >= 0 && gj < F.w)
                v = bf16_bits_to_f(a[((long long)F.pix_base + gi * F.w + gj) * CI + c]);
            s_a[hp * (CI + 1) + c] = v;
        }
        for (int e = threadIdx.x; e < kTileThreads * CO; e += blockDim.x) {
            const int px = e / CO, c = e % CO;
            const int gi = gi0 + 1 + px / kTileW, gj = gj0 + 1 + px % kTileW;
            float v = 0.0f;
            if (gi < F.h && gj < F.w) v = dz[((long long)F.pix_base + gi * F.w + gj) * CO + c];
            s_dz[px * CO + c] = v;
        }
        __syncthreads();
        if (active) {
            for (int px = 0; px < kTileThreads; ++px) {
                const int li = px / kTileW, lj = px % kTileW;
                const float av = s_a[((li + k / 3) * kNetHaloW + lj + k % 3) * (CI + 1) + ci];
                const float* dzp = s_dz + px * CO;
#pragma unroll
                for (int c = 0; c < CO; ++c) acc[c] = fmaf(av, dzp[c], acc[c]);
            }
        }
        if (threadIdx.x < CO)
            for (int px = 0; px < kTileThreads; ++px) bacc += s_dz[px * CO + threadIdx.x];
    }
    if (active)
#pragma unroll
        for (int c = 0; c < CO; ++c) atomicAdd(&dW[((long long)c * CI + ci) * 9 + k], acc[c]);
    if (threadIdx.x < CO) atomicAdd(&db[threadIdx.x], bacc);
}

// ------------------------------------------------------------------ loss

// y, target [n][2][h][w] planes (FP32) and mask -> dy [pix][2] = 2 m (y - t)
// (the 1 / sum m factor is applied in the optimiser step), acc[0] += sum m
// (y - t)^2, acc[1] += sum m.
__global__ void k_net_loss(long long npix, int n, const float* __restrict__ y, const float* __restrict__ target,
                           const uint8_t* __restrict__ mask, float* __restrict__ dy, float* __restrict__ acc)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float se = 0.0f, ms = 0.0f;
    if (idx < (long long)n * npix) {
        const long long im = idx / npix, p = idx % npix;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const long long q = (im * 2 + k) * npix + p;
            const float e = mask[q] ? y[q] - target[q] : 0.0f;
            dy[idx * 2 + k] = 2.0f * e;
            se += e * e;
            ms += mask[q] ? 1.0f : 0.0f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], se);
        atomicAdd(&acc[1], ms);
    }
}

// y [pix][2] (NHWC) -> planes [n][2][h][w]
__global__ void k_net_unpack_output(long long npix, int n, const float* __restrict__ yh, float* __restrict__ y)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * npix) return;
    const long long im = idx / npix, p = idx % npix;
    y[(im * 2) * npix + p] = yh[idx * 2];
    y[(im * 2 + 1) * npix + p] = yh[idx * 2 + 1];
}

// --------------------------------------------------------------- optimiser

// Per layer: the forward weights [ci][k][co] and the backward-data weights
// [co][8 - k][ci], both the bfloat16 rounding of the FP32 masters.
__global__ void k_net_prep_weights(const float* __restrict__ theta, float* __restrict__ wf, float* __restrict__ wb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNetWeights) return;
    int l = 0;
    while (l + 1 < kNetLayers && e >= net_wfoff(l + 1)) ++l;
    const int CI = net_cin(l), CO = net_cout(l);
    const long long q = e - net_wfoff(l);          // index in W[co][ci][k]
    const int co = (int)(q / (CI * 9)), ci = (int)((q / 9) % CI), k = (int)(q % 9);
    const float v = bf16_round(theta[net_woff(l) + q]);
    wf[net_wfoff(l) + ((long long)ci * 9 + k) * CO + co] = v;
    wb[net_wfoff(l) + ((long long)co * 9 + (8 - k)) * CI + ci] = v;
}

// AdamW (decoupled weight decay on convolution weights only); g = grad /
// max(1, acc[1]) (the masked mean's normaliser); clears the gradient.
__global__ void k_net_adamw(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ acc, float lr, float beta1,
                            float beta2, float eps, float wd, float c1, float c2)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNetParams) return;
    int l = 0;
    while (l + 1 < kNetLayers && q >= net_woff(l + 1)) ++l;
    const bool is_w = q < net_boff(l);
    const float g = grad[q] / fmaxf(acc[1], 1.0f);
    const float mq = beta1 * m[q] + (1.0f - beta1) * g;
    const float vq = beta2 * v[q] + (1.0f - beta2) * g * g;
    m[q] = mq;
    v[q] = vq;
    const float upd = (mq / c1) / (sqrtf(vq / c2) + eps);
    theta[q] -= lr * (upd + (is_w ? wd * theta[q] : 0.0f));
    grad[q] = 0.0f;
}

// gradient / max(1, acc[1]) (the masked mean's gradient) into out
__global__ void k_net_scale_grad(const float* __restrict__ grad, const float* __restrict__ acc, float* __restrict__ out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kNetParams) out[q] = grad[q] / fmaxf(acc[1], 1.0f);
}


// ======================================================================
// Forward convolution on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in tensor memory) as an implicit GEMM:
//   D[128 pixels][CO] = sum over the 9 taps of A_tap[128][CI] B_tap[CI][CO],
// one CTA per 128-pixel strip of an image row.  The strip's three input rows
// with a one-pixel margin (3 x 130 pixels) sit in shared memory in the
// no-swizzle K-major layout: 16-byte rows of 8 channels, chunk-major
// ([chunk][pixel][8]), so the operand of tap (ky, kx) is the same buffer
// started ky * 130 + kx pixels later (core matrices of 8 consecutive pixels
// 128 bytes apart, chunks one plane apart).  B (the rounded weights) is a
// prepared image [tap][k-step][chunk][out channel][8] in the same layout.
// ======================================================================

constexpr int kStrip = 128;
constexpr int kStripHaloW = kStrip + 2;
constexpr int kStripHalo = 3 * kStripHaloW;
__host__ __device__ constexpr int net_pad16(int c) { return c < 16 ? 16 : (c + 15) / 16 * 16; }
__host__ __device__ constexpr int net_tc_a_bytes(int ci) { return net_pad16(ci) / 8 * kStripHalo * 16; }
__host__ __device__ constexpr int net_tc_b_bytes(int ci, int co) { return 9 * net_pad16(ci) * net_pad16(co) * 2; }
__host__ __device__ constexpr long net_tcoff(int l)
{
    return l == 0 ? 0 : net_tcoff(l - 1) + net_tc_b_bytes(net_cin(l - 1), net_cout(l - 1)) / 2;
}
constexpr long kNetTcElems = net_tcoff(kNetLayers);   // bf16 elements of all B images

// B images of all layers: element (t, s, c2, n, e) = W[n][16 s + 8 c2 + e][t]
// rounded to bfloat16 (zero past the real channel counts).
__global__ void k_net_prep_tc(const float* __restrict__ theta, uint16_t* __restrict__ img)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNetTcElems) return;
    int l = 0;
    while (l + 1 < kNetLayers && q >= net_tcoff(l + 1)) ++l;
    const int CI = net_cin(l), CO = net_cout(l), CIp = net_pad16(CI), COp = net_pad16(CO);
    long long r = q - net_tcoff(l);
    const int e = (int)(r % 8);
    r /= 8;
    const int n = (int)(r % COp);
    r /= COp;
    const int c2 = (int)(r % 2);
    r /= 2;
    const int s = (int)(r % (CIp / 16));
    const int t = (int)(r / (CIp / 16));
    const int ci = 16 * s + 8 * c2 + e;
    float v = 0.0f;
    if (n < CO && ci < CI) v = theta[net_woff(l) + ((long long)n * CI + ci) * 9 + t];
    img[q] = f_to_bf16_bits(v);
}

__device__ __forceinline__ uint64_t tc_desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // no swizzle, K-major: LBO = byte distance of K-adjacent core matrices,
    // SBO = byte distance of M/N-adjacent (8-row) core matrices; version 1
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Hidden activations for the pipelined layers are stored chunk-planar per
// frame: element (row i, channel 8c + e, column j) at
//   (i * C/8 + c) * w + j) * 8 + e   from the frame's first element,
// so a halo box of one channel chunk is 130 contiguous 16-byte rows.
template <int CO>
__device__ __forceinline__ uint4* planar_chunk(uint16_t* out, const FrameDesc& F, int gi, int gj, int c)
{
    return reinterpret_cast<uint4*>(out + (long long)F.pix_base * CO +
                                    (((long long)gi * (CO / 8) + c) * F.w + gj) * 8);
}

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128)
k_net_conv_tc(const Batch* __restrict__ Bp, const uint16_t* __restrict__ in, const uint16_t* __restrict__ bimg,
              const float* __restrict__ bias, void* __restrict__ out, int* __restrict__ status)
{
    constexpr int CIp = net_pad16(CI), COp = net_pad16(CO), KS = CIp / 16;
    static_assert(CI % 8 == 0 || CI == 6, "input rows are read as 16-byte chunks or three words");
    constexpr int A_BYTES = net_tc_a_bytes(CI), B_BYTES = net_tc_b_bytes(CI, CO);
    constexpr int TM_COLS = COp <= 32 ? 32 : 64;
    constexpr uint32_t kChunkBytes = kStripHalo * 16;
    const Batch& B = *Bp;
    extern __shared__ __align__(128) unsigned char net_tc_smem[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;
    unsigned char* sa = net_tc_smem;
    unsigned char* sb = net_tc_smem + A_BYTES;
    const uint32_t a_addr = smem_u32(sa), b_addr = smem_u32(sb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < B_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sb)[i] = reinterpret_cast<const uint4*>(bimg)[i];
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COp >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    uint32_t phase = 0;
    for (int strip = blockIdx.x; strip < B.net_strips; strip += gridDim.x) {
        // strip -> frame, row, first column
        int lo = 0, hi = B.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.f[mid].net_strip_base <= strip) lo = mid; else hi = mid - 1;
        }
        const FrameDesc& F = B.f[lo];
        const int spr = (F.w + kStrip - 1) / kStrip;
        const int local = strip - F.net_strip_base;
        const int gi = local / spr, j0 = (local % spr) * kStrip;
        // the three input rows with margins, zero outside the frame: thread q
        // takes pixel q + 1 of each row (threads 0 and 1 also the two margin
        // pixels), every 16-byte chunk; all loads are issued before the stores
        {
            const int q = threadIdx.x;
#pragma unroll
            for (int extra = 0; extra < 2; ++extra) {
                // extra = 0: pixel q + 1 (q < 128); extra = 1: margin pixel 0 or 129 (q < 2)
                if (extra == 1 && q >= 2) break;
                const int p = extra == 0 ? q + 1 : (q == 0 ? 0 : kStripHaloW - 1);
                const int jj = j0 - 1 + p;
                const bool jin = jj >= 0 && jj < F.w;
                uint4 v[3][CIp / 8];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int ii = gi - 1 + r;
                    const bool in_f = jin && ii >= 0 && ii < F.h;
                    const long long px = (long long)F.pix_base + (long long)ii * F.w + jj;
#pragma unroll
                    for (int c = 0; c < CIp / 8; ++c) {
                        v[r][c] = make_uint4(0, 0, 0, 0);
                        if (in_f && 8 * c < CI) {
                            if constexpr (CI % 8 == 0) {
                                v[r][c] = *reinterpret_cast<const uint4*>(in + px * CI + 8 * c);
                            } else {
                                // 6 channels = three 32-bit words per pixel
                                const uint32_t* w32 = reinterpret_cast<const uint32_t*>(in + px * CI);
                                v[r][c] = make_uint4(w32[0], w32[1], w32[2], 0u);
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < CIp / 8; ++c)
                        *reinterpret_cast<uint4*>(sa + (size_t)c * kChunkBytes + (size_t)(r * kStripHaloW + p) * 16) =
                            v[r][c];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            // descriptors differ from the first one only in the start-address field
            const uint64_t da0 = tc_desc_plain(a_addr, kChunkBytes, 128);
            const uint64_t db0 = tc_desc_plain(b_addr, (uint32_t)(COp * 16), 128);
            uint32_t acc = 0;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
#pragma unroll
                for (int s = 0; s < KS; ++s) {
                    const uint64_t da = da0 + (uint64_t)(((uint32_t)(2 * s) * kChunkBytes +
                                                          (uint32_t)(ky * kStripHaloW + kx) * 16) >> 4);
                    const uint64_t db = db0 + (uint64_t)((uint32_t)((t * KS + s) * 2 * COp * 16) >> 4);
                    tc_mma(tmem, da, db, idesc, acc);
                    acc = 1;
                }
            }
            tc_commit(smem_u32(&bar));
        }
        // wait for the accumulator (bounded)
        {
            bool ok = mbar_try_wait(smem_u32(&bar), phase);
            if (!ok) {
                const unsigned long long t0 = global_ns();
                while (!(ok = mbar_try_wait_sleep(smem_u32(&bar), phase)))
                    if (global_ns() - t0 > kTcWaitNs) break;
            }
            if (!ok) s_abort = 1;
        }
        phase ^= 1u;
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        // epilogue: thread = pixel (its tensor-memory lane)
        const int m = warp * 32 + lane;
        float acc[COp];
#pragma unroll
        for (int c0 = 0; c0 < COp; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                "%12, %13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            tc_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[c0 + q] = __uint_as_float(v[q]);
        }
        const int gj = j0 + m;
        if (gj < F.w) {
            const long long px = (long long)F.pix_base + gi * F.w + gj;
            if (MODE == kConvHidden) {
                uint32_t pk[CO / 2];
#pragma unroll
                for (int c = 0; c < CO / 2; ++c)
                    pk[c] = (uint32_t)f_to_bf16_bits(fmaxf(acc[2 * c] + bias[2 * c], 0.0f)) |
                            ((uint32_t)f_to_bf16_bits(fmaxf(acc[2 * c + 1] + bias[2 * c + 1], 0.0f)) << 16);
                uint4* o = reinterpret_cast<uint4*>(static_cast<uint16_t*>(out) + px * CO);
#pragma unroll
                for (int c = 0; c < CO / 8; ++c) o[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
            } else {
                float* o = static_cast<float*>(out) + px * CO;
#pragma unroll
                for (int c = 0; c < CO; ++c) o[c] = acc[c] + bias[c];
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (s_abort && threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
    }
}

// ======================================================================
// The same convolution as k_net_conv_tc for chunk-planar inputs (CI a
// multiple of 8, see planar_chunk), pipelined.  A work item is a block of
// kPipeRows output rows of one 128-pixel column strip; consecutive strips of
// an item share two of their three input rows, so each input row is loaded
// once per item into a ring of kPipeRing row buffers ([chunk][pixel][8], 130
// pixels with the one-pixel margins) instead of three times.  Persistent CTAs
// (one per SM) walk the items with
//   warp 4      producer: each input row as 16-byte asynchronous copies
//               (CI/8 contiguous runs of 130 x 16 bytes spread over the
//               lanes; zero-size copies fill margin columns outside the
//               frame with zeros), completion counted on the row's barrier;
//   warp 5      MMA issuer (one thread), owns the tensor memory: per output
//               row the 9 x CI/16 MMAs into one of two accumulators, then
//               releases the input row it used for the last time;
//   warps 0..3  epilogue, one thread per pixel (its tensor-memory lane).
// The copies write through the generic proxy, so the MMA thread orders them
// before its MMAs with a proxy fence after its wait.  Rows outside the frame
// are a resident row of zeros.  The operand of tap
// (ky, kx) starts kx pixels into the ring slot of input row ky, with
// K-adjacent core matrices one chunk plane (130 x 16 bytes) apart.  The MMAs
// run in the order k_net_conv_tc issues them, so both kernels give the same
// sums.  Hidden outputs are written chunk-planar.  Every wait is bounded; on
// expiry the CTA raises the timeout status and the roles drain.
// ======================================================================

constexpr int kPipeThreads = 6 * 32;
constexpr int kPipeRows = 8;          // output rows per work item
constexpr int kPipeRing = 6;          // input rows held in shared memory

// 16-byte asynchronous copy; src_bytes = 0 writes 16 zero bytes
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"((unsigned long long)src),
                 "r"(src_bytes)
                 : "memory");
}

// The barrier's pending count drops by one when this thread's earlier
// asynchronous copies have completed.
__device__ __forceinline__ void cp_async_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// one input row in shared memory: CI/8 chunk planes of 130 x 16 bytes
__host__ __device__ constexpr int net_pipe_row_bytes(int ci) { return (net_pad16(ci) / 8 * kStripHaloW * 16 + 127) / 128 * 128; }

__host__ __device__ constexpr int net_pipe_smem(int ci, int co)
{
    return (kPipeRing + 1) * net_pipe_row_bytes(ci) + net_tc_b_bytes(ci, co);
}

// Work items of the batch: per frame, ceil(w / 128) column strips x
// ceil(h / kPipeRows) row blocks.  Item -> frame, first column, rows [g0, g1).
__device__ __forceinline__ int net_pipe_items(const Batch& B)
{
    int n = 0;
    for (int i = 0; i < B.n; ++i)
        n += ((B.f[i].w + kStrip - 1) / kStrip) * ((B.f[i].h + kPipeRows - 1) / kPipeRows);
    return n;
}

__device__ __forceinline__ void net_pipe_item(const Batch& B, int item, int& fi, int& j0, int& g0, int& g1)
{
    int base = 0;
    fi = B.n - 1;
    for (int i = 0; i < B.n; ++i) {
        const int spr = (B.f[i].w + kStrip - 1) / kStrip;
        const int cnt = spr * ((B.f[i].h + kPipeRows - 1) / kPipeRows);
        if (item < base + cnt) {
            fi = i;
            break;
        }
        base += cnt;
    }
    const FrameDesc& F = B.f[fi];
    const int spr = (F.w + kStrip - 1) / kStrip, local = item - base;
    j0 = (local % spr) * kStrip;
    g0 = (local / spr) * kPipeRows;
    g1 = min(g0 + kPipeRows, F.h);
}

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1)
k_net_conv_pipe(const Batch* __restrict__ Bp, const uint16_t* __restrict__ in, const uint16_t* __restrict__ bimg,
                const float* __restrict__ bias, void* __restrict__ out, int* __restrict__ status,
                const unsigned long long* __restrict__ wait_ns)
{
    // bound of every wait: read from device memory at run time (the launch
    // sits in a replayed graph); the default without one
    const unsigned long long wlim = wait_ns ? *wait_ns : kTcWaitNs;
    static_assert(CI % 8 == 0, "16-byte input rows");
    // NCS chunk planes per input row are stored, NC are read by the MMAs
    // (planes NCS..NC-1 stay zero: CI below 16)
    constexpr int CIp = net_pad16(CI), COp = net_pad16(CO), KS = CIp / 16, NC = CIp / 8, NCS = CI / 8;
    constexpr int ROW = net_pipe_row_bytes(CI), B_BYTES = net_tc_b_bytes(CI, CO);
    constexpr int R = kPipeRing;
    constexpr int TM_COLS = COp <= 32 ? 32 : 64;            // one accumulator
    constexpr uint32_t kPlane = kStripHaloW * 16;            // one chunk plane of one row
    const Batch& B = *Bp;
    extern __shared__ __align__(1024) unsigned char net_pipe_smem_buf[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bars[2 * R + 4];
    __shared__ int s_abort;
    __shared__ float s_bias[COp];
    unsigned char* srow = net_pipe_smem_buf;                 // ring of R input rows
    unsigned char* zrow = net_pipe_smem_buf + R * ROW;       // zeros: rows outside the frame
    unsigned char* sb = zrow + ROW;                          // weights
    const uint32_t row_addr = smem_u32(srow), zrow_addr = smem_u32(zrow), b_addr = smem_u32(sb);
    const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[R]);
    const uint32_t bar_accf = smem_u32(&bars[2 * R]), bar_acce = smem_u32(&bars[2 * R + 2]);
    volatile int* abort_flag = &s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < B_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sb)[i] = reinterpret_cast<const uint4*>(bimg)[i];
    for (int i = threadIdx.x; i < ROW / 16; i += blockDim.x) reinterpret_cast<uint4*>(zrow)[i] = make_uint4(0, 0, 0, 0);
    if constexpr (NCS < NC)
        for (int i = threadIdx.x; i < R * (NC - NCS) * (int)kPlane / 16; i += blockDim.x) {
            const int slot = i / ((NC - NCS) * (int)kPlane / 16), rem = i % ((NC - NCS) * (int)kPlane / 16);
            reinterpret_cast<uint4*>(srow + slot * ROW + NCS * kPlane)[rem] = make_uint4(0, 0, 0, 0);
        }
    for (int i = threadIdx.x; i < COp; i += blockDim.x) s_bias[i] = i < CO ? bias[i] : 0.0f;
    if (threadIdx.x == 0) {
        for (int i = 0; i < R; ++i) {
            mbar_init(bar_full + 8 * i, 32);
            mbar_init(bar_empty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar_accf + 8 * i, 1);
            mbar_init(bar_acce + 8 * i, 4);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(2 * TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights and zeros were written by the generic proxy and are read by the MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COp >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    const int n_items = net_pipe_items(B);

    if (warp == 4) {
        // ------------------------------------------------ producer (whole warp)
        uint32_t q = 0;                                      // rows loaded: ring position
        bool stop = false;
        for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
            int fi, j0, g0, g1;
            net_pipe_item(B, item, fi, j0, g0, g1);
            const FrameDesc& F = B.f[fi];
            // in-frame columns [c_lo, c_hi) of the row's j0 - 1 .. j0 + 128
            const int c_lo = max(j0 - 1, 0), c_hi = min(j0 + kStripHaloW - 1, F.w);
            const int p_lo = c_lo - (j0 - 1), npx = c_hi - c_lo;
            const uint16_t* fbase = in + (long long)F.pix_base * CI;
            for (int r = max(g0 - 1, 0); r <= min(g1, F.h - 1); ++r, ++q) {
                const uint32_t slot = q % R;
                if (!__all_sync(0xffffffffu, mbar_wait(bar_empty + 8 * slot, ((q / R) & 1u) ^ 1u, abort_flag, wlim))) {
                    stop = true;
                    break;
                }
                // (chunk, pixel slot) pairs spread over the lanes; slots outside
                // the frame's columns are filled with zeros
                const uint32_t dst0 = row_addr + slot * ROW;
                for (int idx = lane; idx < NCS * kStripHaloW; idx += 32) {
                    const int c = idx / kStripHaloW, p = idx - c * kStripHaloW;
                    const bool in_f = p >= p_lo && p < p_lo + npx;
                    const uint16_t* src = fbase + (((long long)r * NCS + c) * F.w + (in_f ? c_lo + p - p_lo : 0)) * 8;
                    cp_async16(dst0 + (uint32_t)(c * kPlane + p * 16), src, in_f ? 16u : 0u);
                }
                cp_async_arrive(bar_full + 8 * slot);
            }
        }
        // every copy has landed before the CTA leaves (matters after an abort)
        if (lane == 0)
            for (uint32_t x = q > (uint32_t)R ? q - R : 0u; x < q; ++x) mbar_drain(bar_full + 8 * (x % R), (x / R) & 1u);
    } else if (warp == 5) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint64_t db0 = tc_desc_plain(b_addr, (uint32_t)(COp * 16), 128);
            uint32_t q = 0, k = 0;
            bool stop = false;
            for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
                int fi, j0, g0, g1;
                net_pipe_item(B, item, fi, j0, g0, g1);
                const int H = B.f[fi].h;
                const int r_first = max(g0 - 1, 0), r_last = min(g1, H - 1);
                for (int g = g0; g < g1; ++g, ++k) {
                    const uint32_t a = k & 1u;
                    uint32_t rows3[3];
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky) {
                        const int r = g - 1 + ky;
                        rows3[ky] = zrow_addr;
                        if (r < 0 || r >= H) continue;
                        const uint32_t pos = q + (uint32_t)(r - r_first);
                        if (!mbar_wait(bar_full + 8 * (pos % R), (pos / R) & 1u, abort_flag, wlim)) stop = true;
                        rows3[ky] = row_addr + (pos % R) * ROW;
                    }
                    if (stop || !mbar_wait(bar_acce + 8 * a, ((k >> 1) & 1u) ^ 1u, abort_flag, wlim)) {
                        stop = true;
                        break;
                    }
                    // the rows were written by generic-proxy copies
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc_fence_after();
                    // descriptors differ from the row's or the weights' first one only
                    // in the 16-byte start-address field (shared addresses stay below 2^18)
                    const uint64_t da0[3] = {tc_desc_plain(rows3[0], kPlane, 128), tc_desc_plain(rows3[1], kPlane, 128),
                                             tc_desc_plain(rows3[2], kPlane, 128)};
                    uint32_t acc = 0;
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const int ky = t / 3, kx = t % 3;
#pragma unroll
                        for (int s2 = 0; s2 < KS; ++s2) {
                            const uint64_t da = da0[ky] + (uint64_t)(((uint32_t)(2 * s2) * kPlane + (uint32_t)kx * 16) >> 4);
                            const uint64_t db = db0 + (uint64_t)((uint32_t)((t * KS + s2) * 2 * COp * 16) >> 4);
                            tc_mma(tmem + a * TM_COLS, da, db, idesc, acc);
                            acc = 1;
                        }
                    }
                    tc_commit(bar_accf + 8 * a);
                    // input row g - 1 is not read again
                    if (g - 1 >= 0) tc_commit(bar_empty + 8 * ((q + (uint32_t)(g - 1 - r_first)) % R));
                }
                if (stop) break;
                // nor are the item's last two input rows
                for (int r = g1 - 1; r <= g1; ++r)
                    if (r >= r_first && r <= r_last) tc_commit(bar_empty + 8 * ((q + (uint32_t)(r - r_first)) % R));
                q += (uint32_t)(r_last - r_first + 1);
            }
            // every MMA has finished before the tensor memory is freed (matters after an abort)
            if (k > 0) mbar_drain(bar_accf + 8 * ((k - 1) & 1u), ((k - 1) >> 1) & 1u);
        }
    } else {
        // ------------------------------------------------ epilogue: thread = pixel
        const int m = warp * 32 + lane;
        uint32_t k = 0;
        bool stop = false;
        for (int item = blockIdx.x; item < n_items && !stop; item += gridDim.x) {
            int fi, j0, g0, g1;
            net_pipe_item(B, item, fi, j0, g0, g1);
            const FrameDesc& F = B.f[fi];
            for (int gi = g0; gi < g1; ++gi, ++k) {
                const uint32_t a = k & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(bar_accf + 8 * a, (k >> 1) & 1u, abort_flag, wlim))) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                float acc[COp];
#pragma unroll
                for (int c0 = 0; c0 < COp; c0 += 16) {
                    uint32_t v[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(tmem + ((uint32_t)(warp * 32) << 16) + a * TM_COLS + (uint32_t)c0));
#pragma unroll
                    for (int q2 = 0; q2 < 16; ++q2) acc[c0 + q2] = __uint_as_float(v[q2]);
                }
                tc_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acce + 8 * a);
                const int gj = j0 + m;
                if (gj < F.w) {
                    if (MODE == kConvHidden) {
                        uint32_t pk[CO / 2];
#pragma unroll
                        for (int c = 0; c < CO / 2; ++c)
                            pk[c] = (uint32_t)f_to_bf16_bits(fmaxf(acc[2 * c] + s_bias[2 * c], 0.0f)) |
                                    ((uint32_t)f_to_bf16_bits(fmaxf(acc[2 * c + 1] + s_bias[2 * c + 1], 0.0f)) << 16);
#pragma unroll
                        for (int c = 0; c < CO / 8; ++c)
                            *planar_chunk<CO>(static_cast<uint16_t*>(out), F, gi, gj, c) =
                                make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
                    } else {
                        float* o = static_cast<float*>(out) + ((long long)F.pix_base + gi * F.w + gj) * CO;
#pragma unroll
                        for (int c = 0; c < CO; ++c) o[c] = acc[c] + s_bias[c];
                    }
                }
            }
        }
    }

    // ---- teardown: every role has left its loop (all waits are bounded)
    if (*abort_flag && threadIdx.x == 0 && status) atomicOr(status, kStatusTimeout);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TM_COLS)
                     : "memory");
    }
}

}  // namespace rt3d
