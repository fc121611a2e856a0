// rt3d_device.cuh -- types and device helpers shared by the rt3d kernels.
//
// What a kernel needs about a call lives in one device-resident CallRecord:
// KParams (the method's constants, the normalised IRF, the quantised log-IRF
// and the background filter taps) and Batch (one descriptor per frame),
// uploaded once per call.  Launches then carry only a pointer to it and the
// small Work descriptor, so the launch sequence of a call shape is fixed and
// can be replayed as a CUDA graph.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "rt3d.h"

namespace rt3d {

constexpr int kMaxK = RT3D_MAX_K;
constexpr int kMaxIrf = RT3D_MAX_IRF;
constexpr int kMaxIrfs = RT3D_MAX_IRFS;
constexpr int kMaxBatch = RT3D_MAX_BATCH;
constexpr int kMaxWinR = RT3D_MAX_WIN_R;
constexpr int kMaxBkgR = RT3D_MAX_BKG_R;
constexpr int kIrfPad = 3;          // zero samples on each side of the padded IRF

// device status bits (or-ed into Work::status)
constexpr int kStatusCapacity = 1;
constexpr int kStatusRange = 2;
constexpr int kStatusTimeout = 4;

// tensor-core matched filter: the block offsets a 64-position output tile
// reads (its window of bins spans at most this many 64-bin blocks)
constexpr int kTcMaxOff = 5;

struct KParams {
    int n_iter, k;
    float t_step, r_step, b_step, dt_max, eps_r, eps_b, b_floor, lam_floor;
    float pitch, apss_h, int_h, r_min, merge_dist;
    int win_r, apss_min_nb;
    int depth_den, int_den, bkg_mode, bkg_rad;
    int apss_fp64;                  // APSS solve (and the learned form's fallback) in FP64
    int up;                         // super-resolution factor u of the mapping f (1 = off)
    int irf_len, irf_origin;        // response 0 (the tensor-core init's)
    float irf_sum;                  // sum of the float IRF samples (H in the interior)
    // instrument responses a pixel picks from (FrameDesc::irf_index): samples
    // of response i at irf[irf_offs[i]], lmf taps at lmf[irf_offs[i]]
    int n_irf;
    int irf_lens[kMaxIrfs], irf_origins[kMaxIrfs], irf_offs[kMaxIrfs];
    float irf_sums[kMaxIrfs];
    int peak_sep, peak_min_photons;
    int lmf_kmax;                   // largest quantised log-IRF value
    // tensor-core matched filter (dense frames, lmf_precision BF16 / FP16)
    int tc_mode;                    // 0 off, 1 BF16 operands, 2 FP16 operands
    int tc_dlo, tc_nd;              // bin blocks j + tc_dlo .. j + tc_dlo + tc_nd - 1 feed output tile j
    int tc_ksmask[kTcMaxOff];       // per block offset: which 16-bin K-steps carry nonzero taps
    int tc_stages;                  // shared-memory stages of histogram blocks
    int tc_count_limit;             // counts >= this are not exact as raw operand bits
    int tc_wmin_bits;               // float bits of peak_min_photons in accumulator units
    float tc_unit_inv;              // accumulator value * tc_unit_inv = exact integer
    float net_scale, net_fallback;  // learned depth denoiser: feature/output scale, APSS fallback threshold
    unsigned long long wait_ns;     // bound of every device-side wait of the tensor-core kernels
    float irf[kMaxIrf];             // normalised IRF samples (all responses, concatenated)
    int lmf[kMaxIrf];               // quantised log-IRF K_s (same offsets)
    float bkg_ker[2 * kMaxBkgR + 1];
};

struct FrameDesc {
    int h, w, nt, npix;             // point-cloud (world) grid; nt = histogram bins
    int lh, lw, lnpix;              // lidar pixels (= h, w, npix without super-resolution)
    int tiles_w, tile_base;         // tile grid of the loop kernels
    int pix_base;                   // first world pixel of this frame in the batch workspace
    int lpix_base;                  // first lidar pixel (sparse segments, backgrounds)
    int use_csr;                    // loop reads the caller's sparse list
    const uint16_t* dense;
    const uint32_t* csr_off;
    const uint32_t* ent;            // entries the loop reads (caller's or workspace)
    const float* gain;
    const uint8_t* irf_index;       // [h][w] response of each pixel, or null (response 0)
    int tc;                         // cold start of this frame runs in the tensor-core init
    int tc_tile_base;               // its first 128-pixel tile there
    int net_strip_base;             // first 128-pixel row strip of the frame (learned denoiser)
    float* t;                       // [k][h][w] primary state (the result buffers)
    float* r;
    uint8_t* alive;
    float* b;                       // [h][w]
    int32_t* n_points;
};

struct Batch {
    int n, total_tiles, total_pix, max_t;
    int total_lpix;                 // lidar pixels of all frames
    int tc_tiles;                   // 128-pixel tiles of the tensor-core init
    long long tc_entries;           // entries reserved for its frames (pixels x bins)
    long long ent_base_int;         // the CUDA-core init allocates entries from here on
    int net_strips;                 // 128-pixel row strips of all frames (learned denoiser)
    FrameDesc f[kMaxBatch];
};

struct CallRecord {
    KParams P;
    Batch B;
    CUtensorMap maps[kMaxBatch];    // TMA descriptors of the dense histograms (tensor-core init)
};

struct Work {
    uint2* seg;                     // [stride] (start, count) per pixel
    uint32_t* ent;                  // nonzero-bin entries built from dense histograms
    unsigned long long* ent_count;  // allocation cursor into ent
    long long ent_cap;
    float* t_half;                  // [K][stride]
    float* r_half;                  // [K][stride]
    float* b_half;                  // [stride]
    uint8_t* alive_b;               // [K][stride] pruning output (ping-pong with alive)
    int32_t* y_out;                 // matched-filter dump (rt3d_lmf) or null
    const float* net_y;             // learned depth denoiser output [pix][2] (dt / scale) or null
    int stride;
    int* status;
};

constexpr int kTileH = 8, kTileW = 16, kTileThreads = kTileH * kTileW;

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ int frame_of_tile(const Batch& B, int tile)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.f[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int frame_of_tc_tile(const Batch& B, int tile)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.f[mid].tc_tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int frame_of_pixel(const Batch& B, int pix)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.f[mid].pix_base <= pix) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int frame_of_lpixel(const Batch& B, int lpix)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.f[mid].lpix_base <= lpix) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// A pixel's instrument response h_{i,j} (the likelihood's response is per
// pixel): its length, origin and sample sum, and where its padded samples and
// its interval coefficients start in the kernels' shared tables (each
// response padded by kIrfPad zeros on both sides; L + 5 coefficient entries).
struct IrfRef {
    int pad_off, coef_off, len, origin;
    float sum;
};

__device__ __forceinline__ IrfRef irf_ref(const KParams& P, int which)
{
    IrfRef r;
    r.len = P.irf_lens[which];
    r.origin = P.irf_origins[which];
    r.sum = P.irf_sums[which];
    r.pad_off = P.irf_offs[which] + 2 * kIrfPad * which;
    r.coef_off = P.irf_offs[which] + 5 * which;
    return r;
}

// Response index of local pixel lp (an index past the last response reads as
// the last).
__device__ __forceinline__ int pixel_irf(const KParams& P, const FrameDesc& F, int lp)
{
    return F.irf_index ? min((int)F.irf_index[lp], P.n_irf - 1) : 0;
}

// Catmull-Rom (Keys a = -1/2) interpolation of the IRF samples and its
// derivative at offset x from a point's depth.  `pad` holds the samples with
// kIrfPad zeros on each side, so pad[k + kIrfPad] = h_k for k in [-3, L+2].
__device__ __forceinline__ void irf_eval(const float* pad, int L, int origin, float x,
                                         float& h, float& dh)
{
    const float y = x + (float)origin;
    if (!(y > -2.0f && y < (float)L + 1.0f)) {
        h = 0.0f;
        dh = 0.0f;
        return;
    }
    const float kf = floorf(y);
    const int k = (int)kf + kIrfPad;
    const float u = y - kf;
    const float pm = pad[k - 1], p0 = pad[k], p1 = pad[k + 1], p2 = pad[k + 2];
    const float c1 = p1 - pm;
    const float c2 = 2.0f * pm - 5.0f * p0 + 4.0f * p1 - p2;
    const float c3 = -pm + 3.0f * p0 - 3.0f * p1 + p2;
    h = 0.5f * (2.0f * p0 + u * (c1 + u * (c2 + u * c3)));
    dh = 0.5f * (c1 + u * (2.0f * c2 + 3.0f * c3 * u));
}

// H = sum_{t in [0,T)} h(t - tn) and H' = sum h'(t - tn) for the response R
// (its padded samples at pad + R.pad_off).  In the interior the Catmull-Rom
// interpolant reproduces constants: H = sum of samples, H' = 0; near the
// histogram ends the sums are taken explicitly.
__device__ __forceinline__ void support_sums(const float* pad, const IrfRef& R, int T, float tn, float& H,
                                             float& dH)
{
    const int base = (int)floorf(tn) - R.origin;
    int lo = base - 3, hi = base + R.len + 2;
    if (lo >= 0 && hi <= T - 1) {
        H = R.sum;
        dH = 0.0f;
        return;
    }
    if (lo < 0) lo = 0;
    if (hi > T - 1) hi = T - 1;
    float sh = 0.0f, sdh = 0.0f;
    for (int tb = lo; tb <= hi; ++tb) {
        float hv, dv;
        irf_eval(pad + R.pad_off, R.len, R.origin, (float)tb - tn, hv, dv);
        sh += hv;
        sdh += dv;
    }
    H = sh;
    dH = sdh;
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi)
{
    return fminf(fmaxf(v, lo), hi);
}

}  // namespace rt3d
