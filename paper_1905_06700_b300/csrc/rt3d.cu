// rt3d.cu -- host implementation of the C ABI declared in include/rt3d.h.
//
// The context owns one device workspace sized at creation; every call builds
// the by-value kernel parameters (KParams: constants and tables derived from
// the IRF; Batch: one descriptor per frame) and enqueues the kernels on the
// caller's stream.  Nothing here computes any part of the method on the host
// beyond the per-call tables (normalised IRF, quantised log-IRF, background
// filter taps), which are O(IRF length) and identical for every pixel.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "rt3d.h"
#include "rt3d_device.cuh"
#include "k_synth.cuh"
#include "k_init.cuh"
#include "k_init_tc.cuh"
#include "k_net.cuh"
#include "k_loop.cuh"
#include "k_sr.cuh"
#include "k_compact.cuh"

using namespace rt3d;

namespace {

constexpr int kNumKernelClasses = 9;
enum KernelClass {
    kcInit = 0, kcA = 1, kcB = 2, kcC = 3, kcFinal = 4, kcSynth = 5, kcCompact = 6, kcNet = 7,
    kcInitTc = 8
};

struct PendingTiming {
    int cls;
    cudaEvent_t a, b;
};

// One captured launch sequence of a call geometry (same grids, same smem,
// same iteration count) replayed as a CUDA graph; its kernels read the call
// record, so replays differ only in what was uploaded into it.
struct GraphKey {
    int total_pix, total_tiles, n_iter, warm, init_warps, profiled;
    size_t init_smem;
    int tc_tiles, tc_stages, tc_nd, any_int, learned, fused, split_tiles, den_variant, up, init_var;
    bool operator<(const GraphKey& o) const
    {
        return std::tie(total_pix, total_tiles, n_iter, warm, init_warps, profiled, init_smem, tc_tiles,
                        tc_stages, tc_nd, any_int, learned, fused, split_tiles, den_variant, up, init_var) <
               std::tie(o.total_pix, o.total_tiles, o.n_iter, o.warm, o.init_warps, o.profiled,
                        o.init_smem, o.tc_tiles, o.tc_stages, o.tc_nd, o.any_int, o.learned, o.fused,
                        o.split_tiles, o.den_variant, o.up, o.init_var);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<PendingTiming> timing;   // event pairs recorded by the graph itself
    int kernels = 0;
};

}  // namespace

// The learned depth denoiser: FP32 master parameters with AdamW state, the
// rounded weight layouts the convolutions read, and a training workspace.
struct rt3d_net {
    int device = 0, max_images = 0, max_h = 0, max_w = 0;
    long long max_pix = 0;
    float* theta = nullptr;         // [kNetParams]
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* wf = nullptr;            // [kNetWeights] forward layout
    float* wb = nullptr;            // [kNetWeights] backward-data layout
    uint16_t* wtc = nullptr;        // [kNetTcElems] tensor-core operand images of the rounded weights
    int* status = nullptr;          // device status of the network's own calls
    float* acc = nullptr;           // [2] loss sums
    uint16_t* a[4] = {nullptr, nullptr, nullptr, nullptr};   // layer inputs, NHWC bf16
    float* yh = nullptr;            // [pix][2]
    float* g0 = nullptr;            // [pix][48] gradient ping-pong
    float* g1 = nullptr;
    Batch* d_batch = nullptr;
    Batch h_batch{};
    int step = 0;
};

struct rt3d_ctx {
    rt3d_config cfg{};
    // instrument responses, each normalised in double in index order; frames
    // pick one per pixel (response 0 without an index)
    int n_irf = 1;
    std::vector<double> irf_norm[kMaxIrfs];
    int irf_len[kMaxIrfs] = {0}, irf_origin[kMaxIrfs] = {0};
    Work W{};
    long long stride = 0;           // workspace pixels = max_batch * max_h * max_w
    int* d_status = nullptr;
    unsigned long long* d_count = nullptr;
    CallRecord* d_rec = nullptr;    // per-call tables and frame descriptors (device)
    CallRecord h_rec;               // host copy, uploaded once per call
    uint32_t* d_tmp = nullptr;      // [stride + 1] scratch of rt3d_compact
    // tensor-core matched filter: band operands (device) and the host image last uploaded
    uint8_t* d_band = nullptr;
    std::vector<uint8_t> band_img, band_last;
    int n_sms = 0;
    unsigned long long wait_ns = kTcWaitNs;   // bound of the tensor-core kernels' waits
    // learned depth denoiser: the attached network and the loop's inference buffers
    rt3d_net* net = nullptr;
    uint16_t* net_a0 = nullptr;     // [stride][8] (6 features, 2 zero)
    uint16_t* net_a1 = nullptr;     // [stride][48]
    uint16_t* net_a2 = nullptr;     // [stride][48]
    float* net_y = nullptr;         // [stride][2]
    long long launches = 0;
    bool profiling = false;
    std::vector<PendingTiming> pending;
    std::map<GraphKey, GraphEntry> graphs;
    GraphEntry* capturing = nullptr;        // set while a launch sequence is being captured
    std::vector<GraphEntry*> pending_graphs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;    // second branch of a split capture
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> event_pool;
    double ms[kNumKernelClasses] = {0};
    long long counts[kNumKernelClasses] = {0};
    // staging of rt3d_reconstruct_host (allocated on first use)
    uint16_t* s_dense = nullptr;
    uint32_t* s_off = nullptr;
    uint32_t* s_ent = nullptr;
    long long s_ent_cap = 0;
    float* s_gain = nullptr;
    uint8_t* s_idx = nullptr;
    float* s_t = nullptr;
    float* s_r = nullptr;
    float* s_b = nullptr;
    uint8_t* s_alive = nullptr;
    int32_t* s_np = nullptr;
    // staging of rt3d_reconstruct_batch_host (grown on demand)
    unsigned char* s_batch = nullptr;
    size_t s_batch_cap = 0;
    // its copy stream and group events (large dense frames: copies of the next
    // group overlap the reconstruction of the current one)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copy[5] = {};
};

namespace {

rt3d_status cuda_fail(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? RT3D_E_NOMEM : RT3D_E_CUDA;
}

#define RT3D_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_);      \
    } while (0)

cudaEvent_t take_event(rt3d_ctx* c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch bookkeeping: counts every launch; with profiling on, brackets it with
// events on the launch stream.
struct LaunchScope {
    rt3d_ctx* c;
    cudaStream_t s;
    int cls;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchScope(rt3d_ctx* c_, cudaStream_t s_, int cls_) : c(c_), s(s_), cls(cls_)
    {
        if (c->capturing) ++c->capturing->kernels;
        else ++c->launches;
        if (c->profiling) {
            a = take_event(c);
            b = take_event(c);
            record(a);
        }
    }
    // inside a capture only an "external" record becomes a node that the
    // replayed graph records
    void record(cudaEvent_t e)
    {
        if (c->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    ~LaunchScope()
    {
        if (a) {
            record(b);
            if (c->capturing) c->capturing->timing.push_back({cls, a, b});
            else c->pending.push_back({cls, a, b});
        }
    }
};

bool frame_ok(const rt3d_config* cfg, const rt3d_frame* f)
{
    if (!f) return false;
    if (f->h < 1 || f->w < 1 || f->t < 1) return false;
    if (f->h > cfg->max_h || f->w > cfg->max_w || f->t > cfg->max_t) return false;
    if (f->t > RT3D_MAX_T) return false;
    const bool has_dense = f->dense != nullptr;
    const bool has_csr = f->csr_off != nullptr && f->csr_ent != nullptr;
    if (!has_dense && !has_csr) return false;
    if ((f->csr_off == nullptr) != (f->csr_ent == nullptr)) return false;
    return true;
}

bool params_ok(const rt3d_config* cfg, const rt3d_params* p)
{
    if (!p) return false;
    if (p->n_iter < 0 || p->n_iter > 100000) return false;
    if (p->k_max < 1 || p->k_max > cfg->k_max || p->k_max > RT3D_MAX_K) return false;
    const float pos[] = {p->t_step, p->r_step, p->b_step, p->dt_max, p->pixel_pitch,
                         p->apss_radius, p->int_radius, p->r_min, p->lam_floor};
    for (float v : pos)
        if (!(v > 0.0f) || !std::isfinite(v)) return false;
    const float nonneg[] = {p->eps_r, p->eps_b, p->b_floor, p->lmf_delta_rel, p->merge_dist};
    for (float v : nonneg)
        if (!(v >= 0.0f) || !std::isfinite(v)) return false;
    if (!(p->lmf_delta_rel > 0.0f)) return false;
    if (p->win_r < 0 || p->win_r > RT3D_MAX_WIN_R) return false;
    if (p->apss_min_nb < 0) return false;
    if (p->depth_denoiser < 0 || p->depth_denoiser > RT3D_DEPTH_BILATERAL) return false;
    if (p->apss_fp64 < 0 || p->apss_fp64 > 1) return false;
    if (p->upsample < 1 || p->upsample > RT3D_MAX_UPSAMPLE) return false;
    if (p->intensity_denoiser < 0 || p->intensity_denoiser > 1) return false;
    if (p->bkg_mode < 0 || p->bkg_mode > 1) return false;
    if (p->bkg_mode == RT3D_BKG_LOWPASS && !(p->bkg_sigma > 0.0f)) return false;
    if (p->bkg_radius < 0 || p->bkg_radius > RT3D_MAX_BKG_R) return false;
    if (p->lmf_frac_bits < 0 || p->lmf_frac_bits > 12) return false;
    if (p->peak_min_photons < 0 || p->peak_min_photons > 255) return false;
    if (p->peak_sep < 0 || p->peak_sep > 4096) return false;
    if (p->lmf_precision < 0 || p->lmf_precision > 2) return false;
    if (p->warm_start < 0 || p->warm_start > 1) return false;
    if (!(p->net_scale > 0.0f) || !std::isfinite(p->net_scale) || !std::isfinite(p->net_fallback)) return false;
    return true;
}

bool config_ok(const rt3d_config* cfg)
{
    if (!cfg) return false;
    if (cfg->max_h < 1 || cfg->max_w < 1 || cfg->max_t < 1 || cfg->max_t > RT3D_MAX_T) return false;
    if (cfg->k_max < 1 || cfg->k_max > RT3D_MAX_K) return false;
    if (cfg->max_batch < 1 || cfg->max_batch > RT3D_MAX_BATCH) return false;
    if (cfg->max_entries < 0 || cfg->mem_budget < 0) return false;
    const long long pix = (long long)cfg->max_batch * cfg->max_h * cfg->max_w;
    if (pix > (1ll << 30)) return false;
    return cfg->device >= 0;
}

rt3d_status build_tc_params(const rt3d_params* p, KParams* K);

// The instrument responses' per-call tables: float samples (concatenated),
// their sums, the quantised log-IRF taps
//   K_s = round(2^f log1p(h_s / (delta_rel max h)))
// of each response (max h of that response), and response 0's fields for the
// tensor-core init.  norms[i] holds lens[i] samples normalised in double.
rt3d_status fill_irf_tables(KParams* K, int n, const double* const* norms, const int* lens,
                            const int* origins, const rt3d_params* p)
{
    K->n_irf = n;
    int off = 0, kmax = 0;
    const double scale = std::ldexp(1.0, p->lmf_frac_bits);
    for (int i = 0; i < n; ++i) {
        K->irf_offs[i] = off;
        K->irf_lens[i] = lens[i];
        K->irf_origins[i] = origins[i];
        float fsum = 0.0f;
        double hmax = 0.0;
        for (int s = 0; s < lens[i]; ++s) {
            K->irf[off + s] = (float)norms[i][s];
            fsum += K->irf[off + s];
            if (norms[i][s] > hmax) hmax = norms[i][s];
        }
        K->irf_sums[i] = fsum;
        const double delta = (double)p->lmf_delta_rel * hmax;
        for (int s = 0; s < lens[i]; ++s) {
            const double v = std::nearbyint(scale * std::log1p(norms[i][s] / delta));
            if (v > 1e9) return RT3D_E_INVALID;
            K->lmf[off + s] = (int)v;
            if (K->lmf[off + s] > kmax) kmax = K->lmf[off + s];
        }
        off += lens[i];
    }
    K->irf_len = lens[0];
    K->irf_origin = origins[0];
    K->irf_sum = K->irf_sums[0];
    K->lmf_kmax = kmax;
    if (p->lmf_precision == RT3D_LMF_BF16 && kmax > 256) return RT3D_E_INVALID;
    if (p->lmf_precision == RT3D_LMF_FP16 && kmax > 2048) return RT3D_E_INVALID;
    return RT3D_OK;
}

// Per-call tables derived from the IRF and the parameters.
rt3d_status build_kparams(const rt3d_ctx* c, const rt3d_params* p, KParams* K)
{
    std::memset(K, 0, sizeof(KParams));
    K->n_iter = p->n_iter;
    K->k = p->k_max;
    K->t_step = p->t_step;
    K->r_step = p->r_step;
    K->b_step = p->b_step;
    K->dt_max = p->dt_max;
    K->eps_r = p->eps_r;
    K->eps_b = p->eps_b;
    K->b_floor = p->b_floor;
    K->lam_floor = p->lam_floor;
    K->pitch = p->pixel_pitch;
    K->apss_h = p->apss_radius;
    K->int_h = p->int_radius;
    K->r_min = p->r_min;
    K->merge_dist = p->merge_dist;
    K->win_r = p->win_r;
    K->apss_min_nb = p->apss_min_nb;
    K->depth_den = p->depth_denoiser;
    K->apss_fp64 = p->apss_fp64;
    K->up = p->upsample;
    K->int_den = p->intensity_denoiser;
    K->bkg_mode = p->bkg_mode;
    K->bkg_rad = p->bkg_radius;
    K->peak_sep = p->peak_sep;
    K->peak_min_photons = p->peak_min_photons;
    K->net_scale = p->net_scale;
    K->net_fallback = p->net_fallback;
    K->wait_ns = c->wait_ns;
    const double* norms[kMaxIrfs];
    for (int i = 0; i < c->n_irf; ++i) norms[i] = c->irf_norm[i].data();
    const rt3d_status st = fill_irf_tables(K, c->n_irf, norms, c->irf_len, c->irf_origin, p);
    if (st != RT3D_OK) return st;
    if (p->bkg_mode == RT3D_BKG_LOWPASS) {
        const double sg = (double)p->bkg_sigma;
        double ks = 0.0;
        double tap[2 * kMaxBkgR + 1];
        for (int d = -p->bkg_radius; d <= p->bkg_radius; ++d) {
            tap[d + p->bkg_radius] = std::exp(-(double)d * d / (2.0 * sg * sg));
            ks += tap[d + p->bkg_radius];
        }
        for (int d = 0; d <= 2 * p->bkg_radius; ++d) K->bkg_ker[d] = (float)(tap[d] / ks);
    }
    return build_tc_params(p, K);
}

// ---- tensor-core matched filter: operand tables and TMA descriptors

// FP16 bits of a non-negative integer below 2^11 and BF16 bits of v 2^100 for
// v below 2^8: both exact (the float's low mantissa bits are zero).
uint16_t fp16_bits_of_int(int v)
{
    if (v == 0) return 0;
    uint32_t fb;
    const float f = (float)v;
    std::memcpy(&fb, &f, 4);
    const int e = (int)((fb >> 23) & 0xff) - 127;
    return (uint16_t)(((e + 15) << 10) | ((fb >> 13) & 0x3ff));
}

uint16_t bf16_bits_scaled(int v)
{
    if (v == 0) return 0;
    uint32_t fb;
    const float f = std::ldexp((float)v, 100);
    std::memcpy(&fb, &f, 4);
    return (uint16_t)(fb >> 16);
}

// Tensor-core parameters of the log-matched filter (precision modes BF16 and
// FP16): the block offsets an output tile reads, the nonzero K-steps of each
// band, the stage count that fits shared memory and the exactness limits.
rt3d_status build_tc_params(const rt3d_params* p, KParams* K)
{
    K->tc_mode = 0;
    if (p->lmf_precision == RT3D_LMF_INT) return RT3D_OK;
    const int L = K->irf_len, O = K->irf_origin;
    if (p->peak_sep < 1 || p->peak_sep > kTcMaxSep) return RT3D_E_INVALID;
    const int dlo = -((O + kTcBlk - 1) / kTcBlk);
    const int dhi = (kTcBlk - 1 - O + L - 1) / kTcBlk;
    const int nd = dhi - dlo + 1;
    if (nd > kTcMaxOff) return RT3D_E_INVALID;
    const int avail = kTcSmemLimit - tc_smem_bytes(nd, 0);
    const int stages = std::min(kTcMaxStages, avail / kTcStageBytes);
    if (stages < nd + 1) return RT3D_E_INVALID;
    K->tc_mode = p->lmf_precision == RT3D_LMF_BF16 ? 1 : 2;
    K->tc_dlo = dlo;
    K->tc_nd = nd;
    K->tc_stages = stages;
    for (int di = 0; di < kTcMaxOff; ++di) {
        int mask = 0;
        for (int ks = 0; ks < 4 && di < nd; ++ks) {
            // taps s = 64 d + i - n + origin for i in the K-step, n in [0, 64)
            const int smin = kTcBlk * (dlo + di) + 16 * ks - 63 + O;
            const int smax = kTcBlk * (dlo + di) + 16 * ks + 15 + O;
            if (smax >= 0 && smin <= L - 1) mask |= 1 << ks;
        }
        K->tc_ksmask[di] = mask;
    }
    const bool bf16 = K->tc_mode == 1;
    K->tc_count_limit = bf16 ? 128 : 1024;
    const int unit_exp = bf16 ? -33 : -24;
    const float wmin = std::ldexp((float)p->peak_min_photons, unit_exp);
    std::memcpy(&K->tc_wmin_bits, &wmin, 4);
    K->tc_unit_inv = std::ldexp(1.0f, -unit_exp);
    return RT3D_OK;
}

// The nd band operands, 128 x 64 each, in the 128-byte-swizzled K-major
// layout the MMA reads (row n at 128 n bytes, 16-byte chunk c at c ^ (n & 7)).
void build_band_image(const KParams& K, std::vector<uint8_t>& img)
{
    img.assign((size_t)K.tc_nd * kTcBBytes, 0);
    const bool bf16 = K.tc_mode == 1;
    const uint16_t one = bf16 ? bf16_bits_scaled(1) : fp16_bits_of_int(1);
    for (int di = 0; di < K.tc_nd; ++di) {
        uint8_t* blk = img.data() + (size_t)di * kTcBBytes;
        for (int n = 0; n < kTcN; ++n)
            for (int i = 0; i < kTcBlk; ++i) {
                const int col = n % kTcBlk;
                const int sidx = kTcBlk * (K.tc_dlo + di) + i - col + K.irf_origin;
                if (sidx < 0 || sidx >= K.irf_len) continue;
                uint16_t v;
                if (n < kTcBlk) v = bf16 ? bf16_bits_scaled(K.lmf[sidx]) : fp16_bits_of_int(K.lmf[sidx]);
                else v = one;
                const size_t off = (size_t)n * 128 + (size_t)((((i >> 3) ^ (n & 7)) << 4)) + (size_t)(i & 7) * 2;
                std::memcpy(blk + off, &v, 2);
            }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA descriptor of a dense histogram [npix][T] uint16: boxes of 64 bins x
// 128 pixels, 128-byte swizzle, zero fill outside the histogram.
rt3d_status encode_histogram_map(const rt3d_frame* f, CUtensorMap* map)
{
    auto enc = tensor_map_encoder();
    if (!enc) return RT3D_E_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)f->t, (cuuint64_t)f->h * (cuuint64_t)f->w};
    cuuint64_t strides[1] = {(cuuint64_t)f->t * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBlk, (cuuint32_t)kTcRows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)f->dense, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? RT3D_OK : RT3D_E_INVALID;
}

// Batch descriptors for n frames whose results go to out[i].
rt3d_status build_batch(const rt3d_ctx* c, int n, const rt3d_frame* f, const rt3d_result* out,
                        Batch* B, CallRecord* rec = nullptr, bool tc_init = false, int up = 1)
{
    std::memset(B, 0, sizeof(Batch));
    B->n = n;
    int tiles = 0, pix = 0, lpix = 0, tmax = 0;
    int tc_tiles = 0, strips = 0;
    long long tc_ent = 0;
    for (int i = 0; i < n; ++i) {
        FrameDesc& d = B->f[i];
        // the point cloud's grid: up times finer than the pixels with super-resolution
        d.h = f[i].h * up;
        d.w = f[i].w * up;
        d.nt = f[i].t;
        d.npix = d.h * d.w;
        d.lh = f[i].h;
        d.lw = f[i].w;
        d.lnpix = f[i].h * f[i].w;
        d.tiles_w = (d.w + kTileW - 1) / kTileW;
        d.tile_base = tiles;
        d.pix_base = pix;
        d.lpix_base = lpix;
        tiles += d.tiles_w * ((d.h + kTileH - 1) / kTileH);
        pix += d.npix;
        lpix += d.lnpix;
        tmax = f[i].t > tmax ? f[i].t : tmax;
        d.dense = f[i].dense;
        d.csr_off = f[i].csr_off;
        d.use_csr = f[i].csr_off != nullptr;
        d.ent = d.use_csr ? f[i].csr_ent : c->W.ent;
        d.gain = f[i].gain;
        d.irf_index = f[i].irf_index;
        d.tc_tile_base = tc_tiles;
        d.net_strip_base = strips;
        strips += d.h * ((d.w + kStrip - 1) / kStrip);
        // tensor-core init of a dense frame whose rows TMA can address (16-byte
        // aligned start and row stride) and whose pixels share response 0;
        // other frames take the CUDA-core path, which computes the identical
        // integer filter
        if (tc_init && up == 1 && !d.use_csr && !f[i].irf_index && f[i].t % 8 == 0 &&
            ((uintptr_t)f[i].dense & 15) == 0) {
            // each pixel's entries at a fixed offset (pixel x bins) of the
            // frame's region, so no allocation order is needed
            const long long cells = (long long)d.npix * f[i].t;
            if (cells > 0xffffffffll || tc_ent + cells > c->W.ent_cap) return RT3D_E_INVALID;
            d.tc = 1;
            d.ent = c->W.ent + tc_ent;
            tc_ent += cells;
            tc_tiles += (d.npix + kTcRows - 1) / kTcRows;
            if (rec) {
                const rt3d_status st = encode_histogram_map(&f[i], &rec->maps[i]);
                if (st != RT3D_OK) return st;
            }
        }
        if (out) {
            d.t = out[i].t;
            d.r = out[i].r;
            d.alive = out[i].alive;
            d.b = out[i].b;
            d.n_points = out[i].n_points;
        }
    }
    if (pix > c->stride) return RT3D_E_INVALID;
    B->tc_tiles = tc_tiles;
    B->tc_entries = tc_ent;
    B->ent_base_int = tc_ent;
    B->net_strips = strips;
    B->total_tiles = tiles;
    B->total_pix = pix;
    B->total_lpix = lpix;
    B->max_t = tmax;
    return RT3D_OK;
}

// The init kernel's variant: per-pixel responses in the batch, super-resolution.
int init_variant(const KParams& K, const Batch& B)
{
    bool any_idx = false;
    for (int i = 0; i < B.n; ++i) any_idx |= B.f[i].irf_index != nullptr;
    return (any_idx ? kInitIdx : 0) | (K.up > 1 ? kInitUp : 0);
}

int init_warps(int sep)
{
    int w = kInitSmemBudget / init_warp_bytes(sep);
    return w < 1 ? 1 : (w > kInitWarps ? kInitWarps : w);
}

size_t init_smem(const KParams& K, int sep)
{
    const int n_taps = K.irf_offs[K.n_irf - 1] + K.irf_lens[K.n_irf - 1];
    return (size_t)((n_taps * 4 + 15) & ~15) + (size_t)init_warps(sep) * init_warp_bytes(sep);
}

// One upload per call of the tables and frame descriptors the kernels read.
// The host copy is pageable, so the runtime stages it before returning and
// it may be rewritten by the next call at once.
rt3d_status upload_record(rt3d_ctx* c, cudaStream_t s)
{
    size_t bytes = c->h_rec.B.tc_tiles > 0 ? offsetof(CallRecord, maps) + sizeof(CUtensorMap) * c->h_rec.B.n
                                           : offsetof(CallRecord, maps);

    RT3D_CUDA(cudaMemcpyAsync(c->d_rec, &c->h_rec, bytes, cudaMemcpyHostToDevice, s));
    // band operands of the tensor-core filter, re-uploaded only when they change
    if (c->h_rec.P.tc_mode && c->h_rec.B.tc_tiles > 0) {
        build_band_image(c->h_rec.P, c->band_img);
        if (c->band_img != c->band_last) {
            if (!c->d_band) RT3D_CUDA(cudaMalloc((void**)&c->d_band, (size_t)kTcMaxOff * kTcBBytes));
            RT3D_CUDA(cudaMemcpyAsync(c->d_band, c->band_img.data(), c->band_img.size(), cudaMemcpyHostToDevice, s));
            c->band_last = c->band_img;
        }
    }
    return RT3D_OK;
}

// some frame initialised by the CUDA-core kernel
bool batch_has_int(const Batch& B)
{
    for (int i = 0; i < B.n; ++i)
        if (!B.f[i].tc) return true;
    return false;
}

// pix0 / pix_end: the batch pixels this launch covers, tc0 / tc1 the
// tensor-core init's 128-pixel tiles of the same frames (negative: all)
rt3d_status launch_init(rt3d_ctx* c, const KParams& K, const Batch& B, Work W, cudaStream_t s,
                        bool dump, bool compact_only, int pix0 = 0, int pix_end = -1, int tc0 = 0, int tc1 = -1)
{
    if (pix_end < 0) pix_end = B.total_lpix;    // the init runs per lidar pixel
    if (tc1 < 0) tc1 = B.tc_tiles;
    // the tensor-core kernel takes the dense frames of a cold start; the
    // CUDA-core kernel the rest (it skips those frames)
    const bool tc = K.tc_mode != 0 && !compact_only && tc1 > tc0;
    // every pixel's sparse segment starts empty: a tensor-core init that gives
    // up at its wait bound leaves the pixels it did not reach with no entries
    // (the loop then reads nothing for them)
    if (tc && pix_end > pix0)
        RT3D_CUDA(cudaMemsetAsync(W.seg + pix0, 0, sizeof(uint2) * (size_t)(pix_end - pix0), s));
    if (!tc || compact_only || batch_has_int(B) || B.tc_tiles == 0) {
        const size_t smem = init_smem(K, K.peak_sep);
        const int warps = init_warps(K.peak_sep);
        const int grid = (pix_end - pix0 + warps - 1) / warps;
        if (grid > 0) {
            const int var = init_variant(K, B);
            const bool any_idx = (var & kInitIdx) != 0;
            auto fn = dump ? (any_idx ? k_init<true, false, kInitIdx> : k_init<true, false, 0>)
                           : compact_only ? k_init<false, true, 0>
                           : var == 0 ? k_init<false, false, 0>
                           : var == kInitIdx ? k_init<false, false, kInitIdx>
                           : var == kInitUp ? k_init<false, false, kInitUp>
                           : k_init<false, false, kInitIdx | kInitUp>;
            RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            {
                LaunchScope ls(c, s, kcInit);
                fn<<<grid, warps * 32, smem, s>>>(c->d_rec, W, pix0, pix_end);
            }
            RT3D_CUDA(cudaGetLastError());
        }
    }
    if (tc) {
        if (!c->n_sms) RT3D_CUDA(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->cfg.device));
        const int smem = tc_smem_bytes(K.tc_nd, K.tc_stages);
        const int grid = std::min(c->n_sms, tc1 - tc0);
        auto fn = dump ? k_init_tc<true> : k_init_tc<false>;
        RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        {
            LaunchScope ls(c, s, kcInitTc);
            fn<<<grid, kTcThreads, smem, s>>>(c->d_rec, W, c->d_band, tc0, tc1);
        }
        RT3D_CUDA(cudaGetLastError());
    }
    return RT3D_OK;
}

template <int CI, int CO, int CO_BLK, int MODE>
rt3d_status launch_conv(rt3d_ctx* c, int tiles, const Batch* B, const void* in, const float* wt,
                        const float* bias, void* out, const uint16_t* ref, cudaStream_t s)
{
    auto fn = k_net_conv<CI, CO, CO_BLK, MODE>;
    const int smem = net_conv_smem(CI, CO_BLK);
    RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    LaunchScope ls(c, s, kcNet);
    fn<<<dim3(tiles, CO / CO_BLK), kTileThreads, smem, s>>>(B, in, wt, bias, out, ref);
    return RT3D_OK;
}

template <int CI, int CO, int MODE>
rt3d_status launch_conv_tc(rt3d_ctx* c, int strips, const Batch* B, const uint16_t* in, const uint16_t* img,
                           const float* bias, void* out, int* status, cudaStream_t s)
{
    if (strips <= 0) return RT3D_OK;
    auto fn = k_net_conv_tc<CI, CO, MODE>;
    const int smem = net_tc_a_bytes(CI) + net_tc_b_bytes(CI, CO);
    RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, sms = 148;
    RT3D_CUDA(cudaGetDevice(&dev));
    RT3D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(strips, 2 * sms);
    LaunchScope ls(c, s, kcNet);
    fn<<<grid, 128, smem, s>>>(B, in, img, bias, out, status);
    return RT3D_OK;
}

template <int CI, int CO, int MODE>
rt3d_status launch_conv_pipe(rt3d_ctx* c, int strips, const Batch* B, const uint16_t* in, const uint16_t* img,
                             const float* bias, void* out, int* status, const unsigned long long* wait_ns,
                             cudaStream_t s)
{
    if (strips <= 0) return RT3D_OK;
    auto fn = k_net_conv_pipe<CI, CO, MODE>;
    const int smem = net_pipe_smem(CI, CO);
    RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, sms = 148;
    RT3D_CUDA(cudaGetDevice(&dev));
    RT3D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LaunchScope ls(c, s, kcNet);
    fn<<<sms, kPipeThreads, smem, s>>>(B, in, img, bias, out, status, wait_ns);
    return RT3D_OK;
}

// Forward pass of the network over a batch's 128-pixel row strips on the
// tensor cores: a0 -> a1 -> a2 -> a3 -> y.  pipelined: the 48-channel layers
// run on the pipelined kernel with chunk-planar hidden activations (the
// reconstruction loop); otherwise every layer uses the register-staged
// kernel with NHWC activations (the network's own training calls).
rt3d_status net_forward_tiles(rt3d_ctx* c, const rt3d_net* net, int strips, const Batch* B, const uint16_t* a0,
                              uint16_t* a1, uint16_t* a2, uint16_t* a3, float* y, int* status, cudaStream_t s,
                              bool pipelined = false, const unsigned long long* wait_ns = nullptr)
{
    if (pipelined) {
        // a0 holds 8 channels per pixel (the last two zero); the weights of
        // channels 6 and 7 are zero in the operand image
        rt3d_status st = launch_conv_pipe<8, 48, kConvHidden>(c, strips, B, a0, net->wtc + net_tcoff(0),
                                                              net->theta + net_boff(0), a1, status, wait_ns, s);
        if (st == RT3D_OK)
            st = launch_conv_pipe<48, 48, kConvHidden>(c, strips, B, a1, net->wtc + net_tcoff(1),
                                                       net->theta + net_boff(1), a2, status, wait_ns, s);
        if (st == RT3D_OK)
            st = launch_conv_pipe<48, 48, kConvHidden>(c, strips, B, a2, net->wtc + net_tcoff(2),
                                                       net->theta + net_boff(2), a3, status, wait_ns, s);
        if (st == RT3D_OK)
            st = launch_conv_pipe<48, 2, kConvOut>(c, strips, B, a3, net->wtc + net_tcoff(3),
                                                   net->theta + net_boff(3), y, status, wait_ns, s);
        return st;
    }
    rt3d_status st = launch_conv_tc<6, 48, kConvHidden>(c, strips, B, a0, net->wtc + net_tcoff(0),
                                                        net->theta + net_boff(0), a1, status, s);
    if (st == RT3D_OK)
        st = launch_conv_tc<48, 48, kConvHidden>(c, strips, B, a1, net->wtc + net_tcoff(1),
                                                 net->theta + net_boff(1), a2, status, s);
    if (st == RT3D_OK)
        st = launch_conv_tc<48, 48, kConvHidden>(c, strips, B, a2, net->wtc + net_tcoff(2),
                                                 net->theta + net_boff(2), a3, status, s);
    if (st == RT3D_OK)
        st = launch_conv_tc<48, 2, kConvOut>(c, strips, B, a3, net->wtc + net_tcoff(3), net->theta + net_boff(3),
                                             y, status, s);
    return st;
}

// One PALM phase kernel (0: A, 1: B, 2: C), instantiated for the slot count
// (and phase B for its depth-denoiser variant, den_variant).
// flag: phase A -- first iteration; phase B -- alive flags still in alive_b;
// phase C -- run the next iteration's depth step too.
// (tiles [tile0, tile0 + tiles) of the batch)
int den_variant(const KParams& P)
{
    if (P.depth_den == RT3D_DEPTH_PLANE) return kDenPlane;
    if (P.depth_den == RT3D_DEPTH_BILATERAL) return kDenBilateral;
    return P.apss_fp64 ? kDenApss64 : kDenApss;
}

template <int K>
void launch_phase_k(int phase, int flag, int variant, int tiles, cudaStream_t s, const CallRecord* rec,
                    const Work& W, int tile0)
{
    if (phase == 0) {
        k_phase_a<K><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0);
    } else if (phase == 1) {
        switch (variant) {
        case kDenApss64: k_phase_b<K, kDenApss64><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0); break;
        case kDenPlane: k_phase_b<K, kDenPlane><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0); break;
        case kDenBilateral:
            k_phase_b<K, kDenBilateral><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0);
            break;
        default: k_phase_b<K, kDenApss><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0); break;
        }
    } else {
        k_phase_c<K><<<tiles, kTileThreads, 0, s>>>(rec, W, flag, tile0);
    }
}

void launch_phase(const KParams& P, int phase, int flag, int tiles, cudaStream_t s, const CallRecord* rec,
                  const Work& W, int tile0 = 0)
{
    static_assert(kMaxK == 4, "one instantiation per slot count");
    if (tiles <= 0) return;
    const int v = den_variant(P);
    switch (P.k) {
    case 1: launch_phase_k<1>(phase, flag, v, tiles, s, rec, W, tile0); break;
    case 2: launch_phase_k<2>(phase, flag, v, tiles, s, rec, W, tile0); break;
    case 3: launch_phase_k<3>(phase, flag, v, tiles, s, rec, W, tile0); break;
    default: launch_phase_k<4>(phase, flag, v, tiles, s, rec, W, tile0); break;
    }
}

// With the identity background denoiser the depth step needs only its own
// pixel's state, so it rides on the previous iteration's phase C (two
// launches per iteration instead of three; the learned form's features and
// network then run between that phase C and phase B).
bool fused_depth_step(const KParams& P)
{
    return P.bkg_mode != RT3D_BKG_LOWPASS;
}

rt3d_status launch_loop(rt3d_ctx* c, const Batch& B, cudaStream_t s, int n_iter, int tile0 = 0, int tiles = -1)
{
    if (tiles < 0) tiles = B.total_tiles;
    const bool learned = c->h_rec.P.depth_den == RT3D_DEPTH_LEARNED;
    const bool fused = fused_depth_step(c->h_rec.P);
    for (int it = 0; it < n_iter; ++it) {
        if (it == 0 || !fused) {
            LaunchScope ls(c, s, kcA);
            launch_phase(c->h_rec.P, 0, it == 0 ? 1 : 0, tiles, s, c->d_rec, c->W, tile0);
        }
        if (learned) {
            {
                LaunchScope ls(c, s, kcNet);
                k_net_features_loop<<<B.total_tiles, kTileThreads, 0, s>>>(c->d_rec, c->W, c->net_a0,
                                                                           c->h_rec.P.net_scale,
                                                                           fused && it > 0 ? 1 : 0);
            }
            const rt3d_status st = net_forward_tiles(
                c, c->net, B.net_strips, &c->d_rec->B, c->net_a0, c->net_a1, c->net_a2, c->net_a1, c->net_y,
                c->W.status, s, true, &c->d_rec->P.wait_ns);
            if (st != RT3D_OK) return st;
        }
        {
            LaunchScope ls(c, s, kcB);
            launch_phase(c->h_rec.P, 1, fused && it > 0 ? 1 : 0, tiles, s, c->d_rec, c->W, tile0);
        }
        {
            LaunchScope ls(c, s, kcC);
            launch_phase(c->h_rec.P, 2, fused && it + 1 < n_iter ? 1 : 0, tiles, s, c->d_rec, c->W, tile0);
        }
    }
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

// The super-resolved iteration (upsample u > 1): the gradient steps per lidar
// pixel (k_sr_step), the denoisers on the world grid (phases B and C, which
// skip their per-pixel steps then):
//   depth step -> APSS -> intensity step -> intensity low-pass, pruning,
//   merge -> background step; the background denoiser runs at the head of the
//   next depth step (and in the finaliser).
template <int K>
void launch_sr_step(int mode, int first, int lpix, cudaStream_t s, const CallRecord* rec, const Work& W)
{
    const int grid = (lpix + kSrWarps - 1) / kSrWarps;
    if (mode == 0)
        k_sr_step<K, 0><<<grid, kSrWarps * 32, 0, s>>>(rec, W, first, 0, lpix);
    else if (mode == 1)
        k_sr_step<K, 1><<<grid, kSrWarps * 32, 0, s>>>(rec, W, first, 0, lpix);
    else
        k_sr_step<K, 2><<<grid, kSrWarps * 32, 0, s>>>(rec, W, first, 0, lpix);
}

rt3d_status launch_loop_sr(rt3d_ctx* c, const Batch& B, cudaStream_t s, int n_iter)
{
    const KParams& P = c->h_rec.P;
    auto step = [&](int mode, int first) {
        LaunchScope ls(c, s, mode == 0 ? kcA : (mode == 1 ? kcB : kcC));
        switch (P.k) {
        case 1: launch_sr_step<1>(mode, first, B.total_lpix, s, c->d_rec, c->W); break;
        case 2: launch_sr_step<2>(mode, first, B.total_lpix, s, c->d_rec, c->W); break;
        case 3: launch_sr_step<3>(mode, first, B.total_lpix, s, c->d_rec, c->W); break;
        default: launch_sr_step<4>(mode, first, B.total_lpix, s, c->d_rec, c->W); break;
        }
    };
    for (int it = 0; it < n_iter; ++it) {
        step(0, it == 0 ? 1 : 0);
        {
            LaunchScope ls(c, s, kcB);
            launch_phase(P, 1, 0, B.total_tiles, s, c->d_rec, c->W);
        }
        step(1, 0);
        {
            LaunchScope ls(c, s, kcC);
            launch_phase(P, 2, 0, B.total_tiles, s, c->d_rec, c->W);
        }
        step(2, 0);
    }
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status launch_final(rt3d_ctx* c, const Batch& B, cudaStream_t s, int ran, int tile0 = 0, int tiles = -1)
{
    if (tiles < 0) tiles = B.total_tiles;
    if (tiles <= 0) return RT3D_OK;
    {
        LaunchScope ls(c, s, kcFinal);
        k_final<<<tiles, kTileThreads, 0, s>>>(c->d_rec, c->W, ran, tile0);
    }
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status check_common(rt3d_ctx* c, int n, const rt3d_frame* f, const rt3d_params* p,
                         const rt3d_result* out)
{
    if (!c || !f || !p || n < 1 || n > c->cfg.max_batch) return RT3D_E_INVALID;
    if (!params_ok(&c->cfg, p)) return RT3D_E_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!frame_ok(&c->cfg, &f[i])) return RT3D_E_INVALID;
        if (out && (!out[i].t || !out[i].r || !out[i].alive || !out[i].b)) return RT3D_E_INVALID;
    }
    if (p->depth_denoiser == RT3D_DEPTH_LEARNED && !c->net) return RT3D_E_INVALID;
    if (p->upsample > 1) {
        // the world grid's pixels share the workspace with the batch's pixels
        long long world = 0;
        for (int i = 0; i < n; ++i) world += (long long)f[i].h * f[i].w * p->upsample * p->upsample;
        if (world > c->stride) return RT3D_E_INVALID;
        if (p->depth_denoiser == RT3D_DEPTH_LEARNED) return RT3D_E_UNIMPL;
    }
    return RT3D_OK;
}

rt3d_status run_batch(rt3d_ctx* c, int n, const rt3d_frame* f, const rt3d_params* p,
                      rt3d_result* out, cudaStream_t s)
{
    rt3d_status st = check_common(c, n, f, p, out);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    KParams& K = c->h_rec.P;
    st = build_kparams(c, p, &K);
    if (st != RT3D_OK) return st;
    Batch& B = c->h_rec.B;
    st = build_batch(c, n, f, out, &B, &c->h_rec, K.tc_mode != 0 && !p->warm_start, p->upsample);
    if (st != RT3D_OK) return st;
    st = upload_record(c, s);
    if (st != RT3D_OK) return st;
    // Two chains of frames (init, loop, finaliser each) captured as parallel
    // branches: each chain's launches fill the other's partly empty last wave.
    // Frames are independent, so the results are those of one chain.  Kept as
    // one chain for the learned form (its network kernels cover the whole
    // batch) and while kernel times are recorded (so each kernel's duration is
    // its own).
    int n0 = 0, split_tiles = 0, split_pix = 0, split_tc = 0;
    if (n >= 2 && K.depth_den != RT3D_DEPTH_LEARNED && !c->profiling && K.up == 1) {
        // first chain: the frames whose tiles end by half the batch's tiles (at least one)
        auto tiles_end = [&](int i) { return i + 1 < n ? B.f[i + 1].tile_base : B.total_tiles; };
        while (n0 < n - 1 && 2 * tiles_end(n0) <= B.total_tiles) ++n0;
        if (n0 == 0) n0 = 1;
        split_tiles = B.f[n0].tile_base;
        split_pix = B.f[n0].lpix_base;
        split_tc = B.f[n0].tc_tile_base;
    }
    const GraphKey key{B.total_pix, B.total_tiles, p->n_iter, p->warm_start != 0,
                       init_warps(K.peak_sep), c->profiling ? 1 : 0, init_smem(K, K.peak_sep),
                       B.tc_tiles, K.tc_stages, K.tc_nd, batch_has_int(B) ? 1 : 0,
                       K.depth_den == RT3D_DEPTH_LEARNED ? 1 : 0, fused_depth_step(K) ? 1 : 0, split_tiles,
                       den_variant(K), K.up, init_variant(K, B)};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        // capture the launch sequence of this geometry once, on a private stream
        if (!c->cap_stream) RT3D_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (split_tiles && !c->cap_stream2) {
            RT3D_CUDA(cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking));
            RT3D_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
            RT3D_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        }
        GraphEntry entry;
        c->capturing = &entry;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        rt3d_status cst = RT3D_OK;
        if (e == cudaSuccess) {
            e = cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), c->cap_stream);
            const int ran = p->n_iter > 0 ? 1 : 0;
            const bool warm = p->warm_start != 0;
            if (split_tiles == 0) {
                if (e == cudaSuccess) cst = launch_init(c, K, B, c->W, c->cap_stream, false, warm);
                if (e == cudaSuccess && cst == RT3D_OK)
                    cst = K.up > 1 ? launch_loop_sr(c, B, c->cap_stream, p->n_iter)
                                   : launch_loop(c, B, c->cap_stream, p->n_iter);
                if (e == cudaSuccess && cst == RT3D_OK) cst = launch_final(c, B, c->cap_stream, ran);
            } else {
                // the tensor-core init holds most of an SM's shared memory, so it
                // runs once over the batch before the fork (a split one would
                // lock the other chain's loop kernels out of the SMs)
                const bool tc_init = B.tc_tiles > 0;
                if (e == cudaSuccess && tc_init) cst = launch_init(c, K, B, c->W, c->cap_stream, false, warm);
                // fork: frames [n0, n) on the second capture stream
                if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, c->cap_stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap_stream2, c->ev_fork, 0);
                const int t1 = B.total_tiles - split_tiles;
                if (e == cudaSuccess && cst == RT3D_OK && !tc_init)
                    cst = launch_init(c, K, B, c->W, c->cap_stream, false, warm, 0, split_pix, 0, split_tc);
                if (e == cudaSuccess && cst == RT3D_OK && !tc_init)
                    cst = launch_init(c, K, B, c->W, c->cap_stream2, false, warm, split_pix, B.total_lpix, split_tc,
                                      B.tc_tiles);
                if (e == cudaSuccess && cst == RT3D_OK) cst = launch_loop(c, B, c->cap_stream, p->n_iter, 0, split_tiles);
                if (e == cudaSuccess && cst == RT3D_OK)
                    cst = launch_loop(c, B, c->cap_stream2, p->n_iter, split_tiles, t1);
                if (e == cudaSuccess && cst == RT3D_OK) cst = launch_final(c, B, c->cap_stream, ran, 0, split_tiles);
                if (e == cudaSuccess && cst == RT3D_OK) cst = launch_final(c, B, c->cap_stream2, ran, split_tiles, t1);
                // join
                if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->cap_stream2);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap_stream, c->ev_join, 0);
            }
            const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
            if (e == cudaSuccess) e = e2;
        }
        c->capturing = nullptr;
        if (e == cudaSuccess && cst == RT3D_OK) e = cudaGraphInstantiate(&entry.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || cst != RT3D_OK) {
            for (auto& pt : entry.timing) {
                cudaEventDestroy(pt.a);
                cudaEventDestroy(pt.b);
            }
            cudaGetLastError();
            return cst != RT3D_OK ? cst : cuda_fail(e);
        }
        it = c->graphs.emplace(key, std::move(entry)).first;
    }
    RT3D_CUDA(cudaGraphLaunch(it->second.exec, s));
    c->launches += it->second.kernels;
    if (c->profiling) {
        bool seen = false;
        for (GraphEntry* g : c->pending_graphs) seen |= g == &it->second;
        if (!seen) c->pending_graphs.push_back(&it->second);
    }
    return RT3D_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char* rt3d_status_str(int status)
{
    switch (status) {
        case RT3D_OK: return "ok";
        case RT3D_E_INVALID: return "invalid argument";
        case RT3D_E_NOMEM: return "out of device memory";
        case RT3D_E_CUDA: return "CUDA error";
        case RT3D_E_TIMEOUT: return "timeout";
        case RT3D_E_UNIMPL: return "not implemented";
        case RT3D_E_CAPACITY: return "sparse-entry capacity exceeded";
        case RT3D_E_RANGE: return "counts exceed exact-arithmetic range";
        default: return "unknown status";
    }
}

int rt3d_version(void) { return RT3D_VERSION; }

rt3d_status rt3d_default_params(rt3d_params* p)
{
    if (!p) return RT3D_E_INVALID;
    std::memset(p, 0, sizeof(*p));
    p->n_iter = 20;
    p->k_max = 2;
    p->t_step = 8.0f;
    p->r_step = 0.5f;
    p->b_step = 0.5f;
    p->dt_max = 4.0f;
    p->eps_r = 1e-3f;
    p->eps_b = 1e-6f;
    p->b_floor = 1e-7f;
    p->lam_floor = 1e-9f;
    p->pixel_pitch = 16.0f;
    p->apss_radius = 56.0f;
    p->win_r = 3;
    p->apss_min_nb = 6;
    p->int_radius = 56.0f;
    p->r_min = 0.5f;
    p->merge_dist = 8.0f;
    p->depth_denoiser = RT3D_DEPTH_APSS;
    p->intensity_denoiser = 1;
    p->bkg_mode = RT3D_BKG_IDENTITY;
    p->bkg_sigma = 1.0f;
    p->bkg_radius = 3;
    p->lmf_delta_rel = 1e-3f;
    p->lmf_frac_bits = 5;
    p->peak_min_photons = 2;
    p->peak_sep = 8;
    p->lmf_precision = RT3D_LMF_INT;
    p->warm_start = 0;
    p->net_scale = 3.0f;
    p->net_fallback = 6.0f;
    p->apss_fp64 = 0;
    p->upsample = 1;
    return RT3D_OK;
}

rt3d_status rt3d_validate(const rt3d_config* cfg, const rt3d_frame* f, const rt3d_params* p)
{
    if (!config_ok(cfg)) return RT3D_E_INVALID;
    if (f && !frame_ok(cfg, f)) return RT3D_E_INVALID;
    if (p && !params_ok(cfg, p)) return RT3D_E_INVALID;
    return RT3D_OK;
}

rt3d_status rt3d_workspace_bytes(const rt3d_config* cfg, int64_t* bytes, int64_t* entries)
{
    if (!config_ok(cfg) || !bytes) return RT3D_E_INVALID;
    const long long stride = (long long)cfg->max_batch * cfg->max_h * cfg->max_w;
    const int K = cfg->k_max;
    // seg 8, t_half and r_half 4 K each, b_half 4, alive_b K, scan buffer 4 (+ 4 once)
    const long long fixed = (long long)stride * (16 + 9 * K) + 4 + sizeof(unsigned long long) + sizeof(int) +
                            sizeof(CallRecord);
    long long cap = cfg->max_entries;
    if (cap == 0) {
        cap = stride * cfg->max_t;
        if (cfg->mem_budget > 0) {
            const long long room = (cfg->mem_budget - fixed) / 4;
            if (room < 1) return RT3D_E_NOMEM;
            if (room < cap) cap = room;
        }
    }
    const long long total = fixed + 4 * cap;
    if (cfg->mem_budget > 0 && total > cfg->mem_budget) return RT3D_E_NOMEM;
    *bytes = total;
    if (entries) *entries = cap;
    return RT3D_OK;
}

rt3d_status rt3d_create(const rt3d_config* cfg, const rt3d_irf* irf, rt3d_ctx_t** out)
{
    if (!out) return RT3D_E_INVALID;
    *out = nullptr;
    if (!config_ok(cfg) || !irf || !irf->samples) return RT3D_E_INVALID;
    if (irf->len < 1 || irf->len > RT3D_MAX_IRF || irf->origin < 0 || irf->origin >= irf->len)
        return RT3D_E_INVALID;
    double sum = 0.0;
    for (int s = 0; s < irf->len; ++s) {
        if (!(irf->samples[s] >= 0.0) || !std::isfinite(irf->samples[s])) return RT3D_E_INVALID;
        sum += irf->samples[s];
    }
    if (!(sum > 0.0)) return RT3D_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device >= ndev) return RT3D_E_CUDA;
    RT3D_CUDA(cudaSetDevice(cfg->device));

    rt3d_ctx* c = new (std::nothrow) rt3d_ctx();
    if (!c) return RT3D_E_NOMEM;
    c->cfg = *cfg;
    c->n_irf = 1;
    c->irf_len[0] = irf->len;
    c->irf_origin[0] = irf->origin;
    c->irf_norm[0].resize(irf->len);
    for (int s = 0; s < irf->len; ++s) c->irf_norm[0][s] = irf->samples[s] / sum;
    c->stride = (long long)cfg->max_batch * cfg->max_h * cfg->max_w;
    int64_t ws_bytes = 0, cap = 0;
    {
        const rt3d_status wst = rt3d_workspace_bytes(cfg, &ws_bytes, &cap);
        if (wst != RT3D_OK) {
            rt3d_destroy(c);
            return wst;
        }
    }
    const int K = cfg->k_max;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes ? bytes : 16);
    };
    alloc((void**)&c->W.seg, sizeof(uint2) * c->stride);
    alloc((void**)&c->W.ent, sizeof(uint32_t) * cap);
    alloc((void**)&c->d_count, sizeof(unsigned long long));
    alloc((void**)&c->W.t_half, sizeof(float) * K * c->stride);
    alloc((void**)&c->W.r_half, sizeof(float) * K * c->stride);
    alloc((void**)&c->W.b_half, sizeof(float) * c->stride);
    alloc((void**)&c->W.alive_b, (size_t)K * c->stride);
    alloc((void**)&c->d_status, sizeof(int));
    alloc((void**)&c->d_tmp, sizeof(uint32_t) * (c->stride + 1));
    alloc((void**)&c->d_rec, sizeof(CallRecord));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->W.alive_b, 0, (size_t)K * c->stride);
    if (e != cudaSuccess) {
        rt3d_destroy(c);
        return cuda_fail(e);
    }
    c->W.ent_count = c->d_count;
    c->W.ent_cap = cap;
    c->W.stride = (int)c->stride;
    c->W.status = c->d_status;
    c->W.y_out = nullptr;
    *out = c;
    return RT3D_OK;
}

rt3d_status rt3d_set_irfs(rt3d_ctx_t* c, int n, const rt3d_irf* irfs)
{
    if (!c || !irfs || n < 1 || n > RT3D_MAX_IRFS) return RT3D_E_INVALID;
    int room = 0;
    for (int i = 0; i < n; ++i) {
        const rt3d_irf& r = irfs[i];
        if (!r.samples || r.len < 1 || r.len > RT3D_MAX_IRF || r.origin < 0 || r.origin >= r.len)
            return RT3D_E_INVALID;
        double sum = 0.0;
        for (int s = 0; s < r.len; ++s) {
            if (!(r.samples[s] >= 0.0) || !std::isfinite(r.samples[s])) return RT3D_E_INVALID;
            sum += r.samples[s];
        }
        if (!(sum > 0.0)) return RT3D_E_INVALID;
        room += r.len + 2 * kIrfPad;
    }
    if (room > RT3D_MAX_IRF + 2 * kIrfPad) return RT3D_E_INVALID;
    c->n_irf = n;
    for (int i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int s = 0; s < irfs[i].len; ++s) sum += irfs[i].samples[s];
        c->irf_len[i] = irfs[i].len;
        c->irf_origin[i] = irfs[i].origin;
        c->irf_norm[i].resize(irfs[i].len);
        for (int s = 0; s < irfs[i].len; ++s) c->irf_norm[i][s] = irfs[i].samples[s] / sum;
    }
    return RT3D_OK;
}

void rt3d_destroy(rt3d_ctx_t* c)
{
    if (!c) return;
    cudaSetDevice(c->cfg.device);
    void* ptrs[] = {c->W.seg, c->W.ent, c->d_count, c->W.t_half, c->W.r_half, c->W.b_half,
                    c->W.alive_b, c->d_status, c->d_tmp, c->d_rec, c->s_dense, c->s_off, c->s_ent,
                    c->s_gain, c->s_idx, c->s_t, c->s_r, c->s_b, c->s_alive, c->s_np, c->s_batch, c->d_band,
                    c->net_a0, c->net_a1, c->net_a2, c->net_y};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& pt : c->pending) {
        cudaEventDestroy(pt.a);
        cudaEventDestroy(pt.b);
    }
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto& pt : kv.second.timing) {
            cudaEventDestroy(pt.a);
            cudaEventDestroy(pt.b);
        }
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (auto ev : c->ev_copy)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : c->event_pool) cudaEventDestroy(ev);
    delete c;
}

rt3d_status rt3d_synthesize(rt3d_ctx_t* c, const rt3d_scene* sc, uint64_t seed, uint16_t* dense,
                            void* stream)
{
    if (!c || !sc || !dense) return RT3D_E_INVALID;
    if (sc->h < 1 || sc->w < 1 || sc->t < 1 || sc->t > RT3D_MAX_T) return RT3D_E_INVALID;
    if (sc->n_comp < 0 || sc->n_comp > RT3D_MAX_SYNTH_COMP) return RT3D_E_INVALID;
    if (sc->irf_len < 1 || sc->irf_len > RT3D_MAX_IRF) return RT3D_E_INVALID;
    if (sc->irf_origin < 0 || sc->irf_origin >= sc->irf_len) return RT3D_E_INVALID;
    if (!sc->n_parts || !sc->p0 || !sc->mu || (sc->irf_len > 1 && !sc->irf_cdf)) return RT3D_E_INVALID;
    if (sc->n_comp > 0 && (!sc->depth_int || !sc->depth_split)) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    SynthArgs a;
    a.h = sc->h;
    a.w = sc->w;
    a.t = sc->t;
    a.n_comp = sc->n_comp;
    a.depth_int = sc->depth_int;
    a.depth_split = sc->depth_split;
    a.n_parts = sc->n_parts;
    a.p0 = sc->p0;
    a.mu = sc->mu;
    a.irf_cdf = sc->irf_cdf;
    a.irf_len = sc->irf_len;
    a.irf_origin = sc->irf_origin;
    a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    a.out = dense;
    const long long npix = (long long)sc->h * sc->w;
    const size_t smem = sizeof(uint32_t) * (((sc->irf_len - 1) + 3) & ~3) +
                        sizeof(uint32_t) * kSynthWarps * ((sc->t + 3) & ~3);
    RT3D_CUDA(cudaFuncSetAttribute(k_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        LaunchScope ls(c, s, kcSynth);
        k_synth<<<(unsigned)((npix + kSynthWarps - 1) / kSynthWarps), kSynthWarps * 32, smem, s>>>(a);
    }
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status rt3d_compact(rt3d_ctx_t* c, const rt3d_frame* f, uint32_t* csr_off, uint32_t* csr_ent,
                         int64_t capacity, int64_t* nnz_host, void* stream)
{
    if (!c || !f || !f->dense || !csr_off || capacity < 0 || !nnz_host) return RT3D_E_INVALID;
    if (!frame_ok(&c->cfg, f)) return RT3D_E_INVALID;
    if (capacity > 0 && !csr_ent) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const int npix = f->h * f->w;
    const int grid = (npix + kCompactWarps - 1) / kCompactWarps;
    {
        LaunchScope ls(c, s, kcCompact);
        k_count_nnz<<<grid, kCompactWarps * 32, 0, s>>>(f->dense, npix, f->t, c->d_tmp);
    }
    {
        LaunchScope ls(c, s, kcCompact);
        k_exclusive_scan<<<1, 1024, 0, s>>>(c->d_tmp, npix, csr_off);
    }
    RT3D_CUDA(cudaGetLastError());
    uint32_t total = 0;
    RT3D_CUDA(cudaMemcpyAsync(&total, csr_off + npix, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaStreamSynchronize(s));
    *nnz_host = total;
    if ((int64_t)total > capacity) return RT3D_E_CAPACITY;
    {
        LaunchScope ls(c, s, kcCompact);
        k_emit<<<grid, kCompactWarps * 32, 0, s>>>(f->dense, npix, f->t, csr_off, csr_ent);
    }
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status rt3d_lmf(rt3d_ctx_t* c, const rt3d_frame* f, const rt3d_params* p, int32_t* y,
                     void* stream)
{
    if (!y) return RT3D_E_INVALID;
    rt3d_status st = check_common(c, 1, f, p, nullptr);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    KParams& K = c->h_rec.P;
    st = build_kparams(c, p, &K);
    if (st != RT3D_OK) return st;
    Batch& B = c->h_rec.B;
    st = build_batch(c, 1, f, nullptr, &B, &c->h_rec, K.tc_mode != 0);
    if (st != RT3D_OK) return st;
    st = upload_record(c, s);
    if (st != RT3D_OK) return st;
    Work W = c->W;
    W.y_out = y;
    RT3D_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), s));
    return launch_init(c, K, B, W, s, true, false);
}

rt3d_status rt3d_init(rt3d_ctx_t* c, const rt3d_frame* f, const rt3d_params* p, rt3d_result* out,
                      void* stream)
{
    if (!out) return RT3D_E_INVALID;
    rt3d_status st = check_common(c, 1, f, p, out);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    KParams& K = c->h_rec.P;
    st = build_kparams(c, p, &K);
    if (st != RT3D_OK) return st;
    Batch& B = c->h_rec.B;
    st = build_batch(c, 1, f, out, &B, &c->h_rec, K.tc_mode != 0, p->upsample);
    if (st != RT3D_OK) return st;
    st = upload_record(c, s);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), s));
    st = launch_init(c, K, B, c->W, s, false, false);
    if (st != RT3D_OK) return st;
    return launch_final(c, B, s, 0);
}

rt3d_status rt3d_reconstruct(rt3d_ctx_t* c, const rt3d_frame* f, const rt3d_params* p,
                             rt3d_result* out, void* stream)
{
    if (!out) return RT3D_E_INVALID;
    return run_batch(c, 1, f, p, out, (cudaStream_t)stream);
}

rt3d_status rt3d_reconstruct_batch(rt3d_ctx_t* c, int n, const rt3d_frame* f,
                                   const rt3d_params* p, rt3d_result* out, void* stream)
{
    if (!out) return RT3D_E_INVALID;
    return run_batch(c, n, f, p, out, (cudaStream_t)stream);
}

rt3d_status rt3d_reconstruct_host(rt3d_ctx_t* c, const rt3d_frame* f, const rt3d_params* p,
                                  rt3d_result* out, void* stream)
{
    if (!c || !f || !p || !out) return RT3D_E_INVALID;
    rt3d_status st = check_common(c, 1, f, p, out);
    if (st != RT3D_OK) return st;
    if (p->upsample > 1) return RT3D_E_UNIMPL;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long mpix = (long long)c->cfg.max_h * c->cfg.max_w;
    const int K = c->cfg.k_max;
    if (!c->s_t) {
        RT3D_CUDA(cudaMalloc((void**)&c->s_dense, sizeof(uint16_t) * mpix * c->cfg.max_t));
        RT3D_CUDA(cudaMalloc((void**)&c->s_off, sizeof(uint32_t) * (mpix + 1)));
        RT3D_CUDA(cudaMalloc((void**)&c->s_gain, sizeof(float) * mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_idx, (size_t)mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_t, sizeof(float) * K * mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_r, sizeof(float) * K * mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_b, sizeof(float) * mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_alive, (size_t)K * mpix));
        RT3D_CUDA(cudaMalloc((void**)&c->s_np, sizeof(int32_t)));
    }
    const long long npix = (long long)f->h * f->w;
    rt3d_frame df = *f;
    if (f->dense) {
        RT3D_CUDA(cudaMemcpyAsync(c->s_dense, f->dense, sizeof(uint16_t) * npix * f->t,
                                  cudaMemcpyHostToDevice, s));
        df.dense = c->s_dense;
    }
    if (f->csr_off) {
        const long long nent = f->csr_off[npix];
        if (nent > c->s_ent_cap) {
            if (c->s_ent) cudaFree(c->s_ent);
            c->s_ent = nullptr;
            c->s_ent_cap = 0;
            RT3D_CUDA(cudaMalloc((void**)&c->s_ent, sizeof(uint32_t) * (nent > 0 ? nent : 1)));
            c->s_ent_cap = nent;
        }
        RT3D_CUDA(cudaMemcpyAsync(c->s_off, f->csr_off, sizeof(uint32_t) * (npix + 1),
                                  cudaMemcpyHostToDevice, s));
        if (nent > 0)
            RT3D_CUDA(cudaMemcpyAsync(c->s_ent, f->csr_ent, sizeof(uint32_t) * nent,
                                      cudaMemcpyHostToDevice, s));
        df.csr_off = c->s_off;
        df.csr_ent = c->s_ent;
    }
    if (f->gain) {
        RT3D_CUDA(cudaMemcpyAsync(c->s_gain, f->gain, sizeof(float) * npix, cudaMemcpyHostToDevice, s));
        df.gain = c->s_gain;
    }
    if (f->irf_index) {
        RT3D_CUDA(cudaMemcpyAsync(c->s_idx, f->irf_index, (size_t)npix, cudaMemcpyHostToDevice, s));
        df.irf_index = c->s_idx;
    }
    rt3d_result dr{c->s_t, c->s_r, c->s_alive, c->s_b, c->s_np};
    const int Kp = p->k_max;
    if (p->warm_start) {
        RT3D_CUDA(cudaMemcpyAsync(c->s_t, out->t, sizeof(float) * Kp * npix, cudaMemcpyHostToDevice, s));
        RT3D_CUDA(cudaMemcpyAsync(c->s_r, out->r, sizeof(float) * Kp * npix, cudaMemcpyHostToDevice, s));
        RT3D_CUDA(cudaMemcpyAsync(c->s_alive, out->alive, (size_t)Kp * npix, cudaMemcpyHostToDevice, s));
        RT3D_CUDA(cudaMemcpyAsync(c->s_b, out->b, sizeof(float) * npix, cudaMemcpyHostToDevice, s));
    }
    st = run_batch(c, 1, &df, p, &dr, s);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaMemcpyAsync(out->t, c->s_t, sizeof(float) * Kp * npix, cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaMemcpyAsync(out->r, c->s_r, sizeof(float) * Kp * npix, cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaMemcpyAsync(out->alive, c->s_alive, (size_t)Kp * npix, cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaMemcpyAsync(out->b, c->s_b, sizeof(float) * npix, cudaMemcpyDeviceToHost, s));
    if (out->n_points)
        RT3D_CUDA(cudaMemcpyAsync(out->n_points, c->s_np, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaStreamSynchronize(s));
    return RT3D_OK;
}

// host batches: frames of at least this many dense bytes are copied in groups
// that overlap the reconstruction (a 64 MB copy takes ~1.2 ms on the host link,
// more than one frame's reconstruction)
constexpr size_t kHostGroupMinBytes = 64ull << 20;
constexpr int kHostMaxGroups = 4;

rt3d_status rt3d_reconstruct_batch_host(rt3d_ctx_t* c, int n, const rt3d_frame* f, const rt3d_params* p,
                                        rt3d_result* out, void* stream)
{
    if (!c || !f || !p || !out || n < 1) return RT3D_E_INVALID;
    rt3d_status st = check_common(c, n, f, p, out);
    if (st != RT3D_OK) return st;
    if (p->upsample > 1) return RT3D_E_UNIMPL;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const int Kp = p->k_max;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // one staging area: every frame's inputs, then every frame's results
    struct Span { size_t dense, off, ent, gain, idx, t, r, a, b, np; long long npix, nent; };
    std::vector<Span> sp(n);
    size_t bytes = 0;
    for (int i = 0; i < n; ++i) {
        Span& x = sp[i];
        x.npix = (long long)f[i].h * f[i].w;
        x.nent = f[i].csr_off ? (long long)f[i].csr_off[x.npix] : 0;
        x.dense = bytes;
        if (f[i].dense) bytes += al(sizeof(uint16_t) * x.npix * f[i].t);
        x.off = bytes;
        if (f[i].csr_off) bytes += al(sizeof(uint32_t) * (x.npix + 1));
        x.ent = bytes;
        if (f[i].csr_off) bytes += al(sizeof(uint32_t) * (x.nent > 0 ? x.nent : 1));
        x.gain = bytes;
        if (f[i].gain) bytes += al(sizeof(float) * x.npix);
        x.idx = bytes;
        if (f[i].irf_index) bytes += al((size_t)x.npix);
        x.t = bytes;
        bytes += al(sizeof(float) * Kp * x.npix);
        x.r = bytes;
        bytes += al(sizeof(float) * Kp * x.npix);
        x.a = bytes;
        bytes += al((size_t)Kp * x.npix);
        x.b = bytes;
        bytes += al(sizeof(float) * x.npix);
        x.np = bytes;
        bytes += al(sizeof(int32_t));
    }
    if (bytes > c->s_batch_cap) {
        // the previous staging may still be read by work queued on `s` (or
        // written by a copy group of a call that stopped on an error)
        RT3D_CUDA(cudaStreamSynchronize(s));
        if (c->copy_stream) RT3D_CUDA(cudaStreamSynchronize(c->copy_stream));
        if (c->s_batch) cudaFree(c->s_batch);
        c->s_batch = nullptr;
        c->s_batch_cap = 0;
        RT3D_CUDA(cudaMalloc((void**)&c->s_batch, bytes));
        c->s_batch_cap = bytes;
    }
    unsigned char* base = c->s_batch;
    std::vector<rt3d_frame> df(f, f + n);
    std::vector<rt3d_result> dr(n);
    // Large dense frames are link-bound: the batch runs in up to four groups
    // of frames whose copies, on a copy stream, run ahead of the groups'
    // reconstructions (each group one batched call; results are per frame, so
    // they equal the single call's).  Otherwise one group on `s`.
    bool big_dense = n >= 2;
    for (int i = 0; i < n && big_dense; ++i)
        big_dense = f[i].dense && sizeof(uint16_t) * (size_t)sp[i].npix * f[i].t >= kHostGroupMinBytes;
    const int G = big_dense ? std::min(n, kHostMaxGroups) : 1;
    cudaStream_t cs = s;
    if (G > 1) {
        if (!c->copy_stream) RT3D_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int g = 0; g <= G; ++g)
            if (!c->ev_copy[g]) RT3D_CUDA(cudaEventCreateWithFlags(&c->ev_copy[g], cudaEventDisableTiming));
        cs = c->copy_stream;
        // the copies follow the work already queued on `s`
        RT3D_CUDA(cudaEventRecord(c->ev_copy[G], s));
        RT3D_CUDA(cudaStreamWaitEvent(cs, c->ev_copy[G], 0));
    }
    auto copy_in = [&](int i) -> rt3d_status {
        const Span& x = sp[i];
        if (f[i].dense) {
            df[i].dense = reinterpret_cast<const uint16_t*>(base + x.dense);
            RT3D_CUDA(cudaMemcpyAsync(base + x.dense, f[i].dense, sizeof(uint16_t) * x.npix * f[i].t,
                                      cudaMemcpyHostToDevice, cs));
        }
        if (f[i].csr_off) {
            df[i].csr_off = reinterpret_cast<const uint32_t*>(base + x.off);
            df[i].csr_ent = reinterpret_cast<const uint32_t*>(base + x.ent);
            RT3D_CUDA(cudaMemcpyAsync(base + x.off, f[i].csr_off, sizeof(uint32_t) * (x.npix + 1),
                                      cudaMemcpyHostToDevice, cs));
            if (x.nent > 0)
                RT3D_CUDA(cudaMemcpyAsync(base + x.ent, f[i].csr_ent, sizeof(uint32_t) * x.nent,
                                          cudaMemcpyHostToDevice, cs));
        }
        if (f[i].gain) {
            df[i].gain = reinterpret_cast<const float*>(base + x.gain);
            RT3D_CUDA(cudaMemcpyAsync(base + x.gain, f[i].gain, sizeof(float) * x.npix, cudaMemcpyHostToDevice, cs));
        }
        if (f[i].irf_index) {
            df[i].irf_index = base + x.idx;
            RT3D_CUDA(cudaMemcpyAsync(base + x.idx, f[i].irf_index, (size_t)x.npix, cudaMemcpyHostToDevice, cs));
        }
        dr[i] = rt3d_result{reinterpret_cast<float*>(base + x.t), reinterpret_cast<float*>(base + x.r),
                            base + x.a, reinterpret_cast<float*>(base + x.b),
                            reinterpret_cast<int32_t*>(base + x.np)};
        if (p->warm_start) {
            RT3D_CUDA(cudaMemcpyAsync(dr[i].t, out[i].t, sizeof(float) * Kp * x.npix, cudaMemcpyHostToDevice, cs));
            RT3D_CUDA(cudaMemcpyAsync(dr[i].r, out[i].r, sizeof(float) * Kp * x.npix, cudaMemcpyHostToDevice, cs));
            RT3D_CUDA(cudaMemcpyAsync(dr[i].alive, out[i].alive, (size_t)Kp * x.npix, cudaMemcpyHostToDevice, cs));
            RT3D_CUDA(cudaMemcpyAsync(dr[i].b, out[i].b, sizeof(float) * x.npix, cudaMemcpyHostToDevice, cs));
        }
        return RT3D_OK;
    };
    // every group's copies are queued first (the copy stream runs ahead)
    for (int g = 0; g < G; ++g) {
        for (int i = g * n / G; i < (g + 1) * n / G; ++i) {
            st = copy_in(i);
            if (st != RT3D_OK) return st;
        }
        if (G > 1) RT3D_CUDA(cudaEventRecord(c->ev_copy[g], cs));
    }
    for (int g = 0; g < G; ++g) {
        const int i0 = g * n / G, i1 = (g + 1) * n / G;
        if (G > 1) RT3D_CUDA(cudaStreamWaitEvent(s, c->ev_copy[g], 0));
        st = run_batch(c, i1 - i0, df.data() + i0, p, dr.data() + i0, s);
        if (st != RT3D_OK) {
            if (G > 1) cudaStreamSynchronize(cs);   // no copy still writes the staging on return
            return st;
        }
        for (int i = i0; i < i1; ++i) {
            const long long npix = sp[i].npix;
            RT3D_CUDA(cudaMemcpyAsync(out[i].t, dr[i].t, sizeof(float) * Kp * npix, cudaMemcpyDeviceToHost, s));
            RT3D_CUDA(cudaMemcpyAsync(out[i].r, dr[i].r, sizeof(float) * Kp * npix, cudaMemcpyDeviceToHost, s));
            RT3D_CUDA(cudaMemcpyAsync(out[i].alive, dr[i].alive, (size_t)Kp * npix, cudaMemcpyDeviceToHost, s));
            RT3D_CUDA(cudaMemcpyAsync(out[i].b, dr[i].b, sizeof(float) * npix, cudaMemcpyDeviceToHost, s));
            if (out[i].n_points)
                RT3D_CUDA(cudaMemcpyAsync(out[i].n_points, dr[i].n_points, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                          s));
        }
    }
    RT3D_CUDA(cudaStreamSynchronize(s));
    return RT3D_OK;
}

rt3d_status rt3d_phase(rt3d_ctx_t* c, int phase, int first, const rt3d_frame* f,
                       const rt3d_params* p, rt3d_result* state, void* stream)
{
    if (!state || phase < 0 || phase > 2) return RT3D_E_INVALID;
    rt3d_status st = check_common(c, 1, f, p, state);
    if (st != RT3D_OK) return st;
    if (!f->csr_off) return RT3D_E_INVALID;
    if (p->upsample > 1) return RT3D_E_UNIMPL;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    KParams& K = c->h_rec.P;
    st = build_kparams(c, p, &K);
    if (st != RT3D_OK) return st;
    Batch& B = c->h_rec.B;
    st = build_batch(c, 1, f, state, &B);
    if (st != RT3D_OK) return st;
    st = upload_record(c, s);
    if (st != RT3D_OK) return st;
    // sparse segments of the caller's list
    st = launch_init(c, K, B, c->W, s, false, true);
    if (st != RT3D_OK) return st;
    const long long np = (long long)f->h * f->w;
    const long long S = c->stride;
    const int Kp = p->k_max;
    for (int k = 0; k < Kp; ++k) {
        if (phase == 0)
            RT3D_CUDA(cudaMemcpyAsync(c->W.alive_b + k * S, state->alive + k * np, np,
                                      cudaMemcpyDeviceToDevice, s));
        if (phase == 1)
            RT3D_CUDA(cudaMemcpyAsync(c->W.t_half + k * S, state->t + k * np, sizeof(float) * np,
                                      cudaMemcpyDeviceToDevice, s));
        if (phase == 2)
            RT3D_CUDA(cudaMemcpyAsync(c->W.r_half + k * S, state->r + k * np, sizeof(float) * np,
                                      cudaMemcpyDeviceToDevice, s));
    }
    if (phase == 0)
        RT3D_CUDA(cudaMemcpyAsync(c->W.b_half, state->b, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
    {
        LaunchScope ls(c, s, phase == 0 ? kcA : (phase == 1 ? kcB : kcC));
        launch_phase(K, phase, phase == 0 ? first : 0, B.total_tiles, s, c->d_rec, c->W);
    }
    RT3D_CUDA(cudaGetLastError());
    for (int k = 0; k < Kp; ++k) {
        if (phase == 0)
            RT3D_CUDA(cudaMemcpyAsync(state->t + k * np, c->W.t_half + k * S, sizeof(float) * np,
                                      cudaMemcpyDeviceToDevice, s));
        if (phase == 1)
            RT3D_CUDA(cudaMemcpyAsync(state->r + k * np, c->W.r_half + k * S, sizeof(float) * np,
                                      cudaMemcpyDeviceToDevice, s));
        if (phase == 2)
            RT3D_CUDA(cudaMemcpyAsync(state->alive + k * np, c->W.alive_b + k * S, np,
                                      cudaMemcpyDeviceToDevice, s));
    }
    if (phase == 2)
        RT3D_CUDA(cudaMemcpyAsync(state->b, c->W.b_half, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
    return RT3D_OK;
}

rt3d_status rt3d_device_status(rt3d_ctx_t* c, void* stream)
{
    if (!c) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    RT3D_CUDA(cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    RT3D_CUDA(cudaStreamSynchronize(s));
    if (h & kStatusTimeout) return RT3D_E_TIMEOUT;
    if (h & kStatusCapacity) return RT3D_E_CAPACITY;
    if (h & kStatusRange) return RT3D_E_RANGE;
    return RT3D_OK;
}

int64_t rt3d_launch_count(rt3d_ctx_t* c) { return c ? c->launches : -1; }

rt3d_status rt3d_set_wait_limit(rt3d_ctx_t* c, int64_t ns)
{
    if (!c || ns < 0) return RT3D_E_INVALID;
    c->wait_ns = (unsigned long long)ns;
    return RT3D_OK;
}

rt3d_status rt3d_set_profiling(rt3d_ctx_t* c, int on)
{
    if (!c) return RT3D_E_INVALID;
    c->profiling = on != 0;
    return RT3D_OK;
}

rt3d_status rt3d_kernel_times(rt3d_ctx_t* c, double* ms, int64_t* launches, int n, int reset)
{
    if (!c || n < 0) return RT3D_E_INVALID;
    for (auto& pt : c->pending) {
        if (cudaEventSynchronize(pt.b) != cudaSuccess) return RT3D_E_CUDA;
        float v = 0.0f;
        cudaEventElapsedTime(&v, pt.a, pt.b);
        c->ms[pt.cls] += v;
        c->counts[pt.cls] += 1;
        c->event_pool.push_back(pt.a);
        c->event_pool.push_back(pt.b);
    }
    c->pending.clear();
    // a replayed graph re-records the same events: its kernels are timed once,
    // from its most recent launch
    for (GraphEntry* g : c->pending_graphs)
        for (auto& pt : g->timing) {
            if (cudaEventSynchronize(pt.b) != cudaSuccess) return RT3D_E_CUDA;
            float v = 0.0f;
            cudaEventElapsedTime(&v, pt.a, pt.b);
            c->ms[pt.cls] += v;
            c->counts[pt.cls] += 1;
        }
    c->pending_graphs.clear();
    for (int i = 0; i < n && i < kNumKernelClasses; ++i) {
        if (ms) ms[i] = c->ms[i];
        if (launches) launches[i] = c->counts[i];
    }
    if (reset)
        for (int i = 0; i < kNumKernelClasses; ++i) {
            c->ms[i] = 0.0;
            c->counts[i] = 0;
        }
    return RT3D_OK;
}

rt3d_status rt3d_get_sparse(rt3d_ctx_t* c, uint32_t* seg_host, int64_t n_pix, uint32_t* ent_host,
                            int64_t n_ent, int64_t* n_ent_used, void* stream)
{
    if (!c || n_pix < 0 || n_pix > c->stride || n_ent < 0 || n_ent > c->W.ent_cap) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long used = 0;
    RT3D_CUDA(cudaMemcpyAsync(&used, c->d_count, sizeof(used), cudaMemcpyDeviceToHost, s));
    if (seg_host && n_pix)
        RT3D_CUDA(cudaMemcpyAsync(seg_host, c->W.seg, sizeof(uint2) * n_pix, cudaMemcpyDeviceToHost, s));
    if (ent_host && n_ent)
        RT3D_CUDA(cudaMemcpyAsync(ent_host, c->W.ent, sizeof(uint32_t) * n_ent, cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaStreamSynchronize(s));
    if (n_ent_used) *n_ent_used = (int64_t)used;
    return RT3D_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- learned depth denoiser

namespace {

// n images of h x w as a batch of the loop kernels' tiles
rt3d_status net_batch(rt3d_net* net, int n, int h, int w, cudaStream_t s)
{
    if (n < 1 || n > net->max_images || h < 1 || w < 1 || h > net->max_h || w > net->max_w) return RT3D_E_INVALID;
    Batch& B = net->h_batch;
    std::memset(&B, 0, sizeof(Batch));
    B.n = n;
    const int tw = (w + kTileW - 1) / kTileW, th = (h + kTileH - 1) / kTileH;
    for (int i = 0; i < n; ++i) {
        FrameDesc& d = B.f[i];
        d.h = h;
        d.w = w;
        d.npix = h * w;
        d.tiles_w = tw;
        d.tile_base = i * tw * th;
        d.pix_base = i * h * w;
        d.lh = h;
        d.lw = w;
        d.lnpix = h * w;
        d.lpix_base = d.pix_base;
        d.net_strip_base = i * h * ((w + kStrip - 1) / kStrip);
    }
    B.net_strips = n * h * ((w + kStrip - 1) / kStrip);
    B.total_tiles = n * tw * th;
    B.total_pix = n * h * w;
    B.total_lpix = B.total_pix;
    RT3D_CUDA(cudaMemcpyAsync(net->d_batch, &B, sizeof(Batch), cudaMemcpyHostToDevice, s));
    return RT3D_OK;
}

template <int CI, int CO>
rt3d_status launch_wgrad(const rt3d_net* net, int l, const uint16_t* a, const float* dz, cudaStream_t s)
{
    auto fn = k_net_wgrad<CI, CO>;
    const int threads = ((CI * 9 + 31) / 32) * 32;
    const int smem = (kNetHalo * (CI + 1) + kTileThreads * CO) * 4;
    RT3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = std::min(net->h_batch.total_tiles, 296);
    fn<<<grid, threads, smem, s>>>(net->d_batch, a, dz, net->grad + net_woff(l), net->grad + net_boff(l));
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

// forward, loss and backward of n images into net->grad (unnormalised) and net->acc
rt3d_status net_fwd_bwd(rt3d_net* net, int n, int h, int w, const float* x, const float* target,
                        const uint8_t* mask, cudaStream_t s)
{
    rt3d_status st = net_batch(net, n, h, w, s);
    if (st != RT3D_OK) return st;
    const long long npix = (long long)h * w;
    const long long cnt = npix * n;
    const int blocks = (int)((cnt + 255) / 256);
    k_net_pack_input<<<blocks, 256, 0, s>>>(npix, n, x, net->a[0]);
    // a throwaway context object carries only the launch bookkeeping
    rt3d_ctx tmp;
    st = net_forward_tiles(&tmp, net, net->h_batch.net_strips, net->d_batch, net->a[0], net->a[1], net->a[2],
                           net->a[3], net->yh, net->status, s);
    if (st != RT3D_OK) return st;
    float* yplanes = net->g1;   // [n][2][h][w] scratch before the backward pass needs g1
    k_net_unpack_output<<<blocks, 256, 0, s>>>(npix, n, net->yh, yplanes);
    RT3D_CUDA(cudaMemsetAsync(net->acc, 0, 2 * sizeof(float), s));
    k_net_loss<<<blocks, 256, 0, s>>>(npix, n, yplanes, target, mask, net->g0, net->acc);
    const int T = net->h_batch.total_tiles;
    const Batch* Bd = net->d_batch;
    // layer 3: dy (g0, 2 channels) -> dz2 (g1)
    st = launch_wgrad<48, 2>(net, 3, net->a[3], net->g0, s);
    if (st == RT3D_OK)
        st = launch_conv<2, 48, 48, kConvBackData>(&tmp, T, Bd, net->g0, net->wb + net_wfoff(3), nullptr, net->g1,
                                                   net->a[3], s);
    // layer 2: dz2 (g1) -> dz1 (g0)
    if (st == RT3D_OK) st = launch_wgrad<48, 48>(net, 2, net->a[2], net->g1, s);
    if (st == RT3D_OK)
        st = launch_conv<48, 48, 24, kConvBackData>(&tmp, T, Bd, net->g1, net->wb + net_wfoff(2), nullptr, net->g0,
                                                    net->a[2], s);
    // layer 1: dz1 (g0) -> dz0 (g1)
    if (st == RT3D_OK) st = launch_wgrad<48, 48>(net, 1, net->a[1], net->g0, s);
    if (st == RT3D_OK)
        st = launch_conv<48, 48, 24, kConvBackData>(&tmp, T, Bd, net->g0, net->wb + net_wfoff(1), nullptr, net->g1,
                                                    net->a[1], s);
    // layer 0
    if (st == RT3D_OK) st = launch_wgrad<6, 48>(net, 0, net->a[0], net->g1, s);
    RT3D_CUDA(cudaGetLastError());
    return st;
}

rt3d_status net_prep(rt3d_net* net, cudaStream_t s)
{
    k_net_prep_weights<<<(int)((kNetWeights + 255) / 256), 256, 0, s>>>(net->theta, net->wf, net->wb);
    k_net_prep_tc<<<(int)((kNetTcElems + 255) / 256), 256, 0, s>>>(net->theta, net->wtc);
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

}  // namespace

extern "C" {

rt3d_status rt3d_net_create(int device, int max_images, int max_h, int max_w, rt3d_net_t** out)
{
    if (!out) return RT3D_E_INVALID;
    *out = nullptr;
    if (max_images < 1 || max_images > RT3D_MAX_BATCH || max_h < 1 || max_w < 1) return RT3D_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RT3D_E_CUDA;
    RT3D_CUDA(cudaSetDevice(device));
    rt3d_net* net = new (std::nothrow) rt3d_net();
    if (!net) return RT3D_E_NOMEM;
    net->device = device;
    net->max_images = max_images;
    net->max_h = max_h;
    net->max_w = max_w;
    net->max_pix = (long long)max_images * max_h * max_w;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    const size_t P = sizeof(float) * kNetParams;
    alloc((void**)&net->theta, P);
    alloc((void**)&net->grad, P);
    alloc((void**)&net->m, P);
    alloc((void**)&net->v, P);
    alloc((void**)&net->wf, sizeof(float) * kNetWeights);
    alloc((void**)&net->wb, sizeof(float) * kNetWeights);
    alloc((void**)&net->wtc, sizeof(uint16_t) * kNetTcElems);
    alloc((void**)&net->status, sizeof(int));
    alloc((void**)&net->acc, 2 * sizeof(float));
    alloc((void**)&net->a[0], sizeof(uint16_t) * 6 * net->max_pix);
    for (int l = 1; l < 4; ++l) alloc((void**)&net->a[l], sizeof(uint16_t) * kNetCh * net->max_pix);
    alloc((void**)&net->yh, sizeof(float) * 2 * net->max_pix);
    alloc((void**)&net->g0, sizeof(float) * kNetCh * net->max_pix);
    alloc((void**)&net->g1, sizeof(float) * kNetCh * net->max_pix);
    alloc((void**)&net->d_batch, sizeof(Batch));
    if (e == cudaSuccess) e = cudaMemset(net->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(net->theta, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->grad, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, P);
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, P);
    if (e == cudaSuccess && net_prep(net, nullptr) != RT3D_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rt3d_net_destroy(net);
        return cuda_fail(e);
    }
    *out = net;
    return RT3D_OK;
}

void rt3d_net_destroy(rt3d_net_t* net)
{
    if (!net) return;
    cudaSetDevice(net->device);
    void* ptrs[] = {net->theta, net->grad, net->m, net->v, net->wf, net->wb, net->wtc, net->status, net->acc,
                    net->a[0], net->a[1], net->a[2], net->a[3], net->yh, net->g0, net->g1, net->d_batch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete net;
}

rt3d_status rt3d_net_set_params(rt3d_net_t* net, const float* theta)
{
    if (!net || !theta) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    const size_t P = sizeof(float) * kNetParams;
    RT3D_CUDA(cudaMemcpy(net->theta, theta, P, cudaMemcpyHostToDevice));
    RT3D_CUDA(cudaMemset(net->grad, 0, P));
    RT3D_CUDA(cudaMemset(net->m, 0, P));
    RT3D_CUDA(cudaMemset(net->v, 0, P));
    net->step = 0;
    rt3d_status st = net_prep(net, nullptr);
    if (st != RT3D_OK) return st;
    RT3D_CUDA(cudaDeviceSynchronize());
    return RT3D_OK;
}

rt3d_status rt3d_net_get_params(rt3d_net_t* net, float* theta)
{
    if (!net || !theta) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    RT3D_CUDA(cudaDeviceSynchronize());
    RT3D_CUDA(cudaMemcpy(theta, net->theta, sizeof(float) * kNetParams, cudaMemcpyDeviceToHost));
    return RT3D_OK;
}

rt3d_status rt3d_net_features(rt3d_net_t* net, int n, int k, int h, int w, const float* t, const float* r,
                              const uint8_t* alive, float scale, float* x, void* stream)
{
    if (!net || !t || !r || !alive || !x || n < 1 || k < 1 || k > RT3D_MAX_K || h < 1 || w < 1) return RT3D_E_INVALID;
    if (!(scale > 0.0f)) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    const long long cnt = (long long)n * h * w;
    k_net_features_images<<<(int)((cnt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, k, h, w, t, r, alive,
                                                                                      scale, x);
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status rt3d_net_forward(rt3d_net_t* net, int n, int h, int w, const float* x, float* y, void* stream)
{
    if (!net || !x || !y) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    cudaStream_t s = (cudaStream_t)stream;
    rt3d_status st = net_batch(net, n, h, w, s);
    if (st != RT3D_OK) return st;
    const long long npix = (long long)h * w;
    const int blocks = (int)((npix * n + 255) / 256);
    k_net_pack_input<<<blocks, 256, 0, s>>>(npix, n, x, net->a[0]);
    rt3d_ctx tmp;
    st = net_forward_tiles(&tmp, net, net->h_batch.net_strips, net->d_batch, net->a[0], net->a[1], net->a[2],
                           net->a[3], net->yh, net->status, s);
    if (st != RT3D_OK) return st;
    k_net_unpack_output<<<blocks, 256, 0, s>>>(npix, n, net->yh, y);
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status rt3d_net_gradient(rt3d_net_t* net, int n, int h, int w, const float* x, const float* target,
                              const uint8_t* mask, float* grad, float* loss, void* stream)
{
    if (!net || !x || !target || !mask || !grad) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    cudaStream_t s = (cudaStream_t)stream;
    RT3D_CUDA(cudaMemsetAsync(net->grad, 0, sizeof(float) * kNetParams, s));
    rt3d_status st = net_fwd_bwd(net, n, h, w, x, target, mask, s);
    if (st != RT3D_OK) return st;
    k_net_scale_grad<<<(int)((kNetParams + 255) / 256), 256, 0, s>>>(net->grad, net->acc, grad);
    RT3D_CUDA(cudaGetLastError());
    if (loss) k_net_scale_grad<<<1, 1, 0, s>>>(net->acc, net->acc, loss);   // acc[0] / max(1, acc[1])
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

rt3d_status rt3d_net_train_step(rt3d_net_t* net, int n, int h, int w, const float* x, const float* target,
                                const uint8_t* mask, const rt3d_adamw* opt, float* loss, void* stream)
{
    if (!net || !x || !target || !mask || !opt) return RT3D_E_INVALID;
    if (!(opt->lr >= 0.0f) || !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
        !(opt->eps > 0.0f) || !(opt->weight_decay >= 0.0f))
        return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(net->device));
    cudaStream_t s = (cudaStream_t)stream;
    rt3d_status st = net_fwd_bwd(net, n, h, w, x, target, mask, s);
    if (st != RT3D_OK) return st;
    if (loss) k_net_scale_grad<<<1, 1, 0, s>>>(net->acc, net->acc, loss);
    net->step += 1;
    const float c1 = 1.0f - (float)std::pow((double)opt->beta1, net->step);
    const float c2 = 1.0f - (float)std::pow((double)opt->beta2, net->step);
    k_net_adamw<<<(int)((kNetParams + 255) / 256), 256, 0, s>>>(net->theta, net->grad, net->m, net->v, net->acc,
                                                               opt->lr, opt->beta1, opt->beta2, opt->eps,
                                                               opt->weight_decay, c1, c2);
    RT3D_CUDA(cudaGetLastError());
    return net_prep(net, s);
}

rt3d_status rt3d_set_depth_net(rt3d_ctx_t* c, rt3d_net_t* net)
{
    if (!c) return RT3D_E_INVALID;
    if (net && net->device != c->cfg.device) return RT3D_E_INVALID;
    RT3D_CUDA(cudaSetDevice(c->cfg.device));
    if (net && !c->net_a0) {
        cudaError_t e = cudaSuccess;
        auto alloc = [&](void** ptr, size_t bytes) {
            if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
        };
        alloc((void**)&c->net_a0, sizeof(uint16_t) * 8 * c->stride);
        alloc((void**)&c->net_a1, sizeof(uint16_t) * kNetCh * c->stride);
        alloc((void**)&c->net_a2, sizeof(uint16_t) * kNetCh * c->stride);
        alloc((void**)&c->net_y, sizeof(float) * 2 * c->stride);
        if (e != cudaSuccess) return cuda_fail(e);
        c->W.net_y = c->net_y;
    }
    if (net != c->net) {
        // captured graphs hold the launch arguments of the network they were
        // captured with (its weights and scratch) and the Work descriptor
        // from before the network buffers existed; a launch of one may still
        // run on a caller's stream, so the device finishes its work first
        if (!c->graphs.empty()) RT3D_CUDA(cudaDeviceSynchronize());
        for (auto& kv : c->graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            for (auto& pt : kv.second.timing) {
                cudaEventDestroy(pt.a);
                cudaEventDestroy(pt.b);
            }
        }
        c->graphs.clear();
        c->pending_graphs.clear();
    }
    c->net = net;
    return RT3D_OK;
}

}  // extern "C"

// ============================================================================
// Reconstruction without any allocation (rt3d_reconstruct_noalloc).
//
// Callers that must not allocate device memory after start-up get the whole
// method with its scratch in one file-scope device array, held by every GPU
// that has loaded the library's module until the process exits.  Under CUDA's
// lazy module loading (the default) the module -- and with it the array -- is
// loaded on a device at the first use there (the first call's address
// look-up), and each kernel's code at its first launch.  Its size bounds the
// frames this entry point accepts:
//   pixels h*w <= kStaticMaxPixels, and for a dense histogram h*w*t <=
//   kStaticMaxEntries (so that even a histogram with every bin nonzero fits
//   the sparse-entry area; a caller's own sparse list needs no entry area).
namespace {

constexpr long long kStaticMaxPixels = 16384;            // e.g. 128 x 128
constexpr long long kStaticMaxEntries = 1ll << 21;       // 8 MiB of entries
constexpr long long kStaticEntBytes = 4 * kStaticMaxEntries;
constexpr long long kStaticSegBytes = 8 * kStaticMaxPixels;
constexpr long long kStaticHalfBytes = 4ll * RT3D_MAX_K * kStaticMaxPixels;   // t_half or r_half
constexpr long long kStaticBBytes = 4 * kStaticMaxPixels;
constexpr long long kStaticAliveBytes = (long long)RT3D_MAX_K * kStaticMaxPixels;
constexpr long long kStaticOffSeg = kStaticEntBytes;
constexpr long long kStaticOffT = kStaticOffSeg + kStaticSegBytes;
constexpr long long kStaticOffR = kStaticOffT + kStaticHalfBytes;
constexpr long long kStaticOffB = kStaticOffR + kStaticHalfBytes;
constexpr long long kStaticOffA = kStaticOffB + kStaticBBytes;
constexpr long long kStaticOffCount = (kStaticOffA + kStaticAliveBytes + 255) & ~255ll;
constexpr long long kStaticOffStatus = kStaticOffCount + 256;
constexpr long long kStaticOffRec = kStaticOffStatus + 256;
constexpr long long kStaticBytes = kStaticOffRec + (((long long)sizeof(CallRecord) + 255) & ~255ll);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
unsigned char* g_static_ptr[kStaticMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (host code sees
// only a host-side stand-in for the symbol, never usable as a device pointer).
rt3d_status static_scratch(int device, unsigned char** out)
{
    if (device < 0 || device >= kStaticMaxDevices) return RT3D_E_INVALID;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) return RT3D_E_CUDA;
        g_static_ptr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[device];
    return RT3D_OK;
}

// The per-call tables of build_kparams, from a caller's IRF instead of a
// context (normalised in double, summing in index order, on the stack).
rt3d_status static_kparams(const rt3d_irf* irf, const rt3d_params* p, KParams* K)
{
    double hn[RT3D_MAX_IRF];
    double sum = 0.0;
    for (int s = 0; s < irf->len; ++s) {
        if (!(irf->samples[s] >= 0.0) || !std::isfinite(irf->samples[s])) return RT3D_E_INVALID;
        sum += irf->samples[s];
    }
    if (!(sum > 0.0)) return RT3D_E_INVALID;
    for (int s = 0; s < irf->len; ++s) hn[s] = irf->samples[s] / sum;
    std::memset(K, 0, sizeof(KParams));
    K->n_iter = p->n_iter;
    K->k = p->k_max;
    K->t_step = p->t_step;
    K->r_step = p->r_step;
    K->b_step = p->b_step;
    K->dt_max = p->dt_max;
    K->eps_r = p->eps_r;
    K->eps_b = p->eps_b;
    K->b_floor = p->b_floor;
    K->lam_floor = p->lam_floor;
    K->pitch = p->pixel_pitch;
    K->apss_h = p->apss_radius;
    K->int_h = p->int_radius;
    K->r_min = p->r_min;
    K->merge_dist = p->merge_dist;
    K->win_r = p->win_r;
    K->apss_min_nb = p->apss_min_nb;
    K->depth_den = p->depth_denoiser;
    K->apss_fp64 = p->apss_fp64;
    K->up = 1;
    K->int_den = p->intensity_denoiser;
    K->bkg_mode = p->bkg_mode;
    K->bkg_rad = p->bkg_radius;
    K->peak_sep = p->peak_sep;
    K->peak_min_photons = p->peak_min_photons;
    K->net_scale = p->net_scale;
    K->net_fallback = p->net_fallback;
    K->wait_ns = kTcWaitNs;
    const double* norms[1] = {hn};
    const rt3d_status st = fill_irf_tables(K, 1, norms, &irf->len, &irf->origin, p);
    if (st != RT3D_OK) return st;
    if (p->bkg_mode == RT3D_BKG_LOWPASS) {
        const double sg = (double)p->bkg_sigma;
        double ks = 0.0;
        double tap[2 * kMaxBkgR + 1];
        for (int d = -p->bkg_radius; d <= p->bkg_radius; ++d) {
            tap[d + p->bkg_radius] = std::exp(-(double)d * d / (2.0 * sg * sg));
            ks += tap[d + p->bkg_radius];
        }
        for (int d = 0; d <= 2 * p->bkg_radius; ++d) K->bkg_ker[d] = (float)(tap[d] / ks);
    }
    return RT3D_OK;
}

}  // namespace

extern "C" rt3d_status rt3d_reconstruct_noalloc(const rt3d_irf* irf, const rt3d_frame* f,
                                                const rt3d_params* p, rt3d_result* out,
                                                void* stream)
{
    if (!irf || !irf->samples || !f || !p || !out) return RT3D_E_INVALID;
    if (!out->t || !out->r || !out->alive || !out->b) return RT3D_E_INVALID;
    if (irf->len < 1 || irf->len > RT3D_MAX_IRF || irf->origin < 0 || irf->origin >= irf->len)
        return RT3D_E_INVALID;
    // limits of the static scratch, checked before anything is launched
    const long long npix = (long long)f->h * f->w;
    if (f->h < 1 || f->w < 1 || f->t < 1 || f->t > RT3D_MAX_T) return RT3D_E_INVALID;
    if (npix > kStaticMaxPixels) return RT3D_E_INVALID;
    const bool has_csr = f->csr_off != nullptr && f->csr_ent != nullptr;
    if ((f->csr_off == nullptr) != (f->csr_ent == nullptr)) return RT3D_E_INVALID;
    if (!has_csr && (!f->dense || npix * f->t > kStaticMaxEntries)) return RT3D_E_INVALID;
    rt3d_config cfg{};
    cfg.max_h = f->h;
    cfg.max_w = f->w;
    cfg.max_t = f->t;
    cfg.k_max = RT3D_MAX_K;
    cfg.max_batch = 1;
    if (!params_ok(&cfg, p)) return RT3D_E_INVALID;
    if (p->depth_denoiser == RT3D_DEPTH_LEARNED) return RT3D_E_UNIMPL;
    if (f->irf_index) return RT3D_E_UNIMPL;      // one response: `irf`
    if (p->upsample > 1) return RT3D_E_UNIMPL;

    // the call record goes up from a pageable stack copy, which a stream
    // capture would record by address: not while `stream` is being captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    RT3D_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return RT3D_E_INVALID;

    int device = 0;
    RT3D_CUDA(cudaGetDevice(&device));
    unsigned char* base = nullptr;
    rt3d_status st = static_scratch(device, &base);
    if (st != RT3D_OK) return st;
    CallRecord rec;                      // host copy, uploaded into the static array
    KParams& K = rec.P;
    st = static_kparams(irf, p, &K);
    if (st != RT3D_OK) return st;

    Work W{};
    W.ent = reinterpret_cast<uint32_t*>(base);
    W.seg = reinterpret_cast<uint2*>(base + kStaticOffSeg);
    W.t_half = reinterpret_cast<float*>(base + kStaticOffT);
    W.r_half = reinterpret_cast<float*>(base + kStaticOffR);
    W.b_half = reinterpret_cast<float*>(base + kStaticOffB);
    W.alive_b = base + kStaticOffA;
    W.ent_count = reinterpret_cast<unsigned long long*>(base + kStaticOffCount);
    W.ent_cap = kStaticMaxEntries;
    W.stride = (int)kStaticMaxPixels;
    W.status = reinterpret_cast<int*>(base + kStaticOffStatus);
    W.y_out = nullptr;

    Batch& B = rec.B;
    std::memset(&B, 0, sizeof(Batch));
    B.n = 1;
    FrameDesc& d = B.f[0];
    d.h = f->h;
    d.w = f->w;
    d.nt = f->t;
    d.npix = (int)npix;
    d.tiles_w = (f->w + kTileW - 1) / kTileW;
    d.tile_base = 0;
    d.pix_base = 0;
    d.lh = f->h;
    d.lw = f->w;
    d.lnpix = (int)npix;
    d.lpix_base = 0;
    d.dense = f->dense;
    d.csr_off = f->csr_off;
    d.use_csr = has_csr;
    d.ent = has_csr ? f->csr_ent : W.ent;
    d.gain = f->gain;
    d.t = out->t;
    d.r = out->r;
    d.alive = out->alive;
    d.b = out->b;
    d.n_points = out->n_points;
    B.total_tiles = d.tiles_w * ((f->h + kTileH - 1) / kTileH);
    B.total_pix = (int)npix;
    B.total_lpix = (int)npix;
    B.max_t = f->t;

    cudaStream_t s = (cudaStream_t)stream;
    const CallRecord* d_rec = reinterpret_cast<const CallRecord*>(base + kStaticOffRec);
    // pageable source: staged by the runtime before the call returns
    RT3D_CUDA(cudaMemcpyAsync((void*)d_rec, &rec, sizeof(CallRecord), cudaMemcpyHostToDevice, s));
    // the allocation cursor and the device status word start at zero every call
    RT3D_CUDA(cudaMemsetAsync(W.ent_count, 0, sizeof(unsigned long long), s));
    RT3D_CUDA(cudaMemsetAsync(W.status, 0, sizeof(int), s));

    const size_t smem = init_smem(K, K.peak_sep);
    const int warps = init_warps(K.peak_sep);
    auto init_fn = p->warm_start ? k_init<false, true> : k_init<false, false>;
    RT3D_CUDA(cudaFuncSetAttribute(init_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    init_fn<<<(B.total_pix + warps - 1) / warps, warps * 32, smem, s>>>(d_rec, W, 0, B.total_pix);
    for (int it = 0; it < p->n_iter; ++it) {
        const bool fused = fused_depth_step(K);
        if (it == 0 || !fused) launch_phase(K, 0, it == 0 ? 1 : 0, B.total_tiles, s, d_rec, W);
        launch_phase(K, 1, fused && it > 0 ? 1 : 0, B.total_tiles, s, d_rec, W);
        launch_phase(K, 2, fused && it + 1 < p->n_iter ? 1 : 0, B.total_tiles, s, d_rec, W);
    }
    k_final<<<B.total_tiles, kTileThreads, 0, s>>>(d_rec, W, p->n_iter > 0 ? 1 : 0, 0);
    RT3D_CUDA(cudaGetLastError());
    return RT3D_OK;
}

extern "C" rt3d_status rt3d_noalloc_status(void* stream)
{
    int device = 0;
    RT3D_CUDA(cudaGetDevice(&device));
    unsigned char* base = nullptr;
    const rt3d_status st = static_scratch(device, &base);
    if (st != RT3D_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    RT3D_CUDA(cudaMemcpyAsync(&h, base + kStaticOffStatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT3D_CUDA(cudaMemsetAsync(base + kStaticOffStatus, 0, sizeof(int), s));
    RT3D_CUDA(cudaStreamSynchronize(s));
    if (h & kStatusTimeout) return RT3D_E_TIMEOUT;
    if (h & kStatusCapacity) return RT3D_E_CAPACITY;
    if (h & kStatusRange) return RT3D_E_RANGE;
    return RT3D_OK;
}
