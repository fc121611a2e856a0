/*
 * rt3d.h -- C ABI of the B300 (sm_103a) reconstruction library for
 * time-correlated single-photon (TCSPC) lidar histograms.
 *
 * The library implements the method of Tachella et al., "Real-time 3D
 * reconstruction from single-photon lidar data using plug-and-play point cloud
 * denoisers" (Nature Communications 2019):
 *   - the Poisson observation model and its negative log-likelihood
 *     (Results, "Observation model", the likelihood equation and g(t, r, b));
 *   - a per-pixel initialisation (Methods, "3D Reconstruction algorithm"):
 *     log-matched filter and peak picking into up to K points per pixel;
 *   - the PALM loop over depth, intensity and background (Results,
 *     "Reconstruction algorithm", Fig. 2): a gradient step on each block
 *     followed by a plug-and-play denoiser -- APSS sphere fitting for depth,
 *     a manifold low-pass plus pruning for intensity, identity or an
 *     FFT-equivalent low-pass for the background.
 *
 * Conventions, for every entry point below:
 *   - All frame and result pointers are DEVICE pointers owned by the caller,
 *     unless the function says otherwise.  The library never frees them.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  A return of RT3D_OK means the work was
 *     validated and launched.  Errors detected on the device (capacity,
 *     arithmetic range) are reported by rt3d_device_status().
 *   - Arguments are validated on the host before anything is launched; an
 *     invalid argument returns RT3D_E_INVALID and launches nothing.
 *   - No exception crosses the ABI.  A context may be used from one host
 *     thread at a time; calls that share a context are ordered on their
 *     streams by the caller.
 *   - Layouts: histograms [h][w][t] (bin-contiguous uint16); point slots
 *     [k][h][w]; images [h][w].  Depths t are in bins (real-valued, bin b
 *     covers [b, b+1)), intensities r in expected signal photons at gain 1,
 *     backgrounds b in photons per bin.
 */
#ifndef RT3D_H
#define RT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT3D_VERSION 1
#define RT3D_MAX_K 4          /* point slots per pixel */
#define RT3D_MAX_IRF 256      /* samples of the instrument response */
#define RT3D_MAX_IRFS 4       /* instrument responses a context holds (rt3d_set_irfs) */
#define RT3D_MAX_UPSAMPLE 4   /* super-resolution factor of rt3d_params.upsample */
#define RT3D_MAX_BATCH 64     /* frames per batched call */
#define RT3D_MAX_T 16384      /* histogram bins */
#define RT3D_MAX_WIN_R 4      /* neighbourhood half-width of the denoisers, pixels */
#define RT3D_MAX_BKG_R 15     /* background filter half-width, pixels */
#define RT3D_MAX_SYNTH_COMP 64 /* surfaces per pixel in rt3d_synthesize */

/* Opaque context: owns the device workspace of one CUDA device. */
typedef struct rt3d_ctx rt3d_ctx_t;

typedef enum {
    RT3D_OK = 0,
    RT3D_E_INVALID = -1,   /* bad argument; nothing was launched */
    RT3D_E_NOMEM = -2,     /* device memory for the workspace is not available */
    RT3D_E_CUDA = -3,      /* a CUDA runtime call failed */
    RT3D_E_TIMEOUT = -4,   /* a bounded wait gave up */
    RT3D_E_UNIMPL = -5,    /* option not built */
    RT3D_E_CAPACITY = -6,  /* device: more nonzero bins than the sparse buffer holds */
    RT3D_E_RANGE = -7      /* device: counts exceed the exact-arithmetic range */
} rt3d_status;

/* Matched-filter arithmetic (all exact for counts within range). */
enum { RT3D_LMF_INT = 0, RT3D_LMF_BF16 = 1, RT3D_LMF_FP16 = 2 };
/* Depth denoiser: none, APSS (the paper's), learned conv net (if loaded), and
 * two other plug-in point cloud denoisers (the Discussion's quality / speed
 * trade-off) over the APSS neighbourhood, weights and radius:
 *   RT3D_DEPTH_PLANE      weighted least-squares plane u0 + u1 x + u2 y + z = 0
 *                         in the point's local coordinates, point moved along
 *                         the line of sight onto it (APSS without the sphere
 *                         term: planes are kept, spheres flattened);
 *   RT3D_DEPTH_BILATERAL  the weight-averaged depth of the neighbours (itself
 *                         included): a bilateral depth filter.
 * Both leave a point unchanged with fewer than apss_min_nb weighted
 * neighbours; the plane fit also with collinear neighbour pixels. */
enum { RT3D_DEPTH_NONE = 0, RT3D_DEPTH_APSS = 1, RT3D_DEPTH_LEARNED = 2, RT3D_DEPTH_PLANE = 3,
       RT3D_DEPTH_BILATERAL = 4 };
/* Background denoiser: identity (bistatic) or periodic Gaussian (= FFT low-pass). */
enum { RT3D_BKG_IDENTITY = 0, RT3D_BKG_LOWPASS = 1 };

/* Sizes the context's device workspace (allocated once, in rt3d_create). */
typedef struct {
    int32_t max_h, max_w, max_t;   /* largest frame */
    int32_t k_max;                 /* point slots per pixel, 1..RT3D_MAX_K */
    int32_t max_batch;             /* frames per batched call, 1..RT3D_MAX_BATCH */
    int64_t max_entries;           /* nonzero-bin capacity per call; 0 = max_batch*max_h*max_w*max_t,
                                      or with mem_budget > 0 the largest the budget leaves */
    int32_t device;                /* CUDA device ordinal */
    int64_t mem_budget;            /* bytes of device memory the workspace may take (0 = no limit):
                                      rt3d_create returns RT3D_E_NOMEM if the per-pixel state and the
                                      entry capacity do not fit it (see rt3d_workspace_bytes) */
} rt3d_config;

/* Instrument response h_{i,j}(.) of the likelihood equation, shared by all
 * pixels: HOST pointer to len samples at unit bin spacing; sample `origin`
 * sits at depth offset 0 (a depth names the position of that sample).  The
 * library normalises the samples to unit sum (in double precision, summing in
 * index order) and interpolates them with the Catmull-Rom cubic.  Copied at
 * rt3d_create; the caller keeps ownership. */
typedef struct {
    const double* samples;
    int32_t len;                   /* 1..RT3D_MAX_IRF */
    int32_t origin;                /* 0..len-1 */
} rt3d_irf;

/* One lidar frame, DEVICE pointers.  Give `dense`, or the sparse list
 * (csr_off, csr_ent), or both (then the sparse list is used by the loop and
 * the dense histogram by the initialisation).
 *   dense     [h][w][t] uint16 photon counts
 *   csr_off   [h*w + 1] offsets into csr_ent (pixel p owns off[p]..off[p+1])
 *   csr_ent   packed (bin << 16) | count, count >= 1, bins increasing per pixel;
 *             a photon list with repeated bins is NOT accepted -- merge first
 *   gain      [h][w] detector gain g_{i,j} (0 = dead pixel) or NULL for 1
 *   irf_index [h][w] the instrument response h_{i,j} of each pixel: an index
 *             into the context's responses (rt3d_set_irfs; an index past the
 *             last reads as the last), or NULL for response 0.  A frame with
 *             an index is initialised by the CUDA-core matched filter (its
 *             lmf_precision is not used). */
typedef struct {
    int32_t h, w, t;
    const uint16_t* dense;
    const uint32_t* csr_off;
    const uint32_t* csr_ent;
    const float* gain;
    const uint8_t* irf_index;
} rt3d_frame;

/* Every constant of the method.  Step sizes of the gradient steps (the paper's
 * are in its supplement; these are the library's reading):
 *   depth      beta_t = t_step / (g r + eps_r), step clamped to +-dt_max,
 *              t clamped to [0, T-1]; t_step = eta / I_h with I_h the IRF's
 *              location Fisher information sum h'^2/h is a scaled Fisher step
 *   intensity  r <- max(0, r - r_step (r + eps_r)(H - sum z h / lambda))
 *              (r_step = 1, eps_r = 0: the EM update r <- r sum z h/lambda / H)
 *   background b <- max(b_floor, b - b_step (b + eps_b)(1 - sum z / lambda / T))
 * with lambda floored at lam_floor. */
typedef struct {
    int32_t n_iter;                /* PALM iterations, >= 0 */
    int32_t k_max;                 /* slots used, 1..config.k_max */
    float t_step, r_step, b_step, dt_max, eps_r, eps_b, b_floor, lam_floor;
    float pixel_pitch;             /* world units (bins) per pixel, orthographic f */
    float apss_radius;             /* APSS kernel radius h (bins, world units) */
    int32_t win_r;                 /* denoiser pixel window half-width, 0..RT3D_MAX_WIN_R */
    int32_t apss_min_nb;           /* fewer weighted neighbours: depth left unchanged */
    float int_radius;              /* intensity low-pass radius (bins, world units) */
    float r_min;                   /* pruning threshold on intensity, > 0 */
    float merge_dist;              /* same-pixel points closer than this (bins) merge, >= 0 */
    int32_t depth_denoiser;        /* RT3D_DEPTH_* */
    int32_t intensity_denoiser;    /* 0 = off (pruning still applies), 1 = low-pass */
    int32_t bkg_mode;              /* RT3D_BKG_* */
    float bkg_sigma;               /* background Gaussian sigma, pixels */
    int32_t bkg_radius;            /* background kernel half-width, 0..RT3D_MAX_BKG_R */
    float lmf_delta_rel;           /* matched-filter floor delta / max h */
    int32_t lmf_frac_bits;         /* matched-filter fixed-point fraction bits, 0..12 */
    int32_t peak_min_photons;      /* counts required in a peak's IRF window, 0..255 */
    int32_t peak_sep;              /* local-maximum half-width, bins, >= 0 */
    int32_t lmf_precision;         /* RT3D_LMF_* */
    int32_t warm_start;            /* 1: start from the points already in the result */
    float net_scale;               /* learned depth denoiser: depth scale of its features and output (bins), > 0 */
    float net_fallback;            /* learned depth denoiser: a point whose proposed move exceeds this (bins)
                                      takes the APSS update instead */
    int32_t apss_fp64;             /* 1: the APSS fit's normal equations (centring, Cholesky, projection)
                                      are solved in FP64 from the FP32 neighbourhood moments, for APSS
                                      and the learned form's APSS fallback; 0: in FP32 */
    int32_t upsample;              /* super-resolution factor u of the point-to-cube mapping f (Results,
                                      "Observation model"; "3D Dynamic scenes"), 1..RT3D_MAX_UPSAMPLE:
                                      the point cloud lives on a world grid u times finer than the
                                      pixels, lidar pixel (i, j) observing the points of world pixels
                                      (u i + a, u j + c), 0 <= a, c < u.  The result's t, r, alive are
                                      then [k_max][u h][u w] (b stays [h][w]); pixel_pitch and the
                                      denoisers' radii are in world pixels; the initialisation gives
                                      each world pixel its lidar pixel's peaks with 1/u^2 of the
                                      intensity.  1 = off.  With u > 1: rt3d_reconstruct,
                                      rt3d_reconstruct_batch and rt3d_init only (the other entry points
                                      return RT3D_E_UNIMPL), not with the learned denoiser
                                      (RT3D_E_UNIMPL), the matched filter on CUDA cores whatever
                                      lmf_precision says, and the frames' world pixels must fit the
                                      context's max_batch x max_h x max_w (else RT3D_E_INVALID). */
} rt3d_params;

/* Output (and, with warm_start, input) point cloud: DEVICE buffers owned by
 * the caller.  t, r, alive: [params.k_max][h][w] ([k_max][u h][u w] with
 * params.upsample = u); b: [h][w]; n_points: one int32 (number of alive
 * points) or NULL. */
typedef struct {
    float* t;
    float* r;
    uint8_t* alive;
    float* b;
    int32_t* n_points;
} rt3d_result;

/* Synthetic scene for rt3d_synthesize (test and benchmark input).  DEVICE
 * pointers; S = n_comp surfaces, P = h*w:
 *   depth_int [S][P] int32, depth_split [S][P] uint32 (photon lands one bin
 *   later when a uniform word is below it), n_parts/p0/mu [S+1][P] (the last
 *   plane is the background; fixed-point Poisson parameters, see below),
 *   irf_cdf [irf_len-1] uint32 offset thresholds. */
typedef struct {
    int32_t h, w, t, n_comp;
    const int32_t* depth_int;
    const uint32_t* depth_split;
    const uint32_t* n_parts;
    const uint64_t* p0;
    const uint64_t* mu;
    const uint32_t* irf_cdf;
    int32_t irf_len, irf_origin;
} rt3d_scene;

/* Human-readable name of a status code (static string). */
const char* rt3d_status_str(int status);
int rt3d_version(void);

/* Fill `p` with the library defaults (n_iter 20, K 2, 7x7 window, ...). */
rt3d_status rt3d_default_params(rt3d_params* p);

/* Host-only validation of a frame and parameters against a configuration.
 * Touches no device; frame pointers are only checked for NULL-ness. */
rt3d_status rt3d_validate(const rt3d_config* cfg, const rt3d_frame* f, const rt3d_params* p);

/* Device bytes the workspace of rt3d_create(cfg) takes: per pixel of the
 * batch 16 + 9 k_max bytes (sparse segments, half-step state, pruning flags,
 * a scan buffer), 4 bytes per sparse entry, and the call record.  With
 * max_entries = 0 and mem_budget > 0, the entry capacity is the largest that
 * keeps this within the budget; *entries (may be NULL) receives it.  Host
 * only.  RT3D_E_INVALID for a bad configuration, RT3D_E_NOMEM if the budget
 * does not hold the per-pixel state (or the given max_entries). */
rt3d_status rt3d_workspace_bytes(const rt3d_config* cfg, int64_t* bytes, int64_t* entries);

/* Create a context on cfg->device: copies the IRF, allocates the workspace
 * (sparse-entry buffer, half-step state, counters).  *out is NULL on error. */
rt3d_status rt3d_create(const rt3d_config* cfg, const rt3d_irf* irf, rt3d_ctx_t** out);
void rt3d_destroy(rt3d_ctx_t* ctx);

/* Per-pixel instrument responses (Results, "Observation model": the response
 * h_{i,j} of the likelihood is per pixel).  Replaces the context's responses
 * with n of them (HOST array, copied; 1..RT3D_MAX_IRFS); frames pick one per
 * pixel with rt3d_frame.irf_index, and response 0 serves frames without an
 * index (rt3d_create's IRF is the single response 0 until this is called).
 * Each response is normalised as in rt3d_create.  Their samples must fit the
 * kernels' tables: sum over responses of (len + 6) <= RT3D_MAX_IRF + 6.
 * Takes effect from the next call.  RT3D_E_INVALID for a bad count, length,
 * origin or sample (nothing changes then). */
rt3d_status rt3d_set_irfs(rt3d_ctx_t* ctx, int n, const rt3d_irf* irfs);

/* Photon synthesis (test/benchmark input, not the method): Poisson counts of
 * the observation model drawn with Philox4x32-10 (Salmon et al., SC'11),
 * key = seed, counters (pixel, component, part, 1) for a count and
 * (pixel, component, photon, 2) for a photon; background is component 255.
 * Counts: each of n_parts parts by fixed-point inversion from p0 = exp(-mu)
 * 2^62 and mu 2^32.  Writes dense [h][w][t] (device).  Integer-only on the
 * device, so the result is bit-reproducible on any implementation. */
rt3d_status rt3d_synthesize(rt3d_ctx_t* ctx, const rt3d_scene* scene, uint64_t seed,
                            uint16_t* dense, void* stream);

/* Dense histogram -> sparse list (nonzero bins per pixel, increasing), the
 * representation whose cost is linear in active bins (Methods, Fig. 5).
 * csr_off [h*w+1] and csr_ent [capacity] are device outputs; *nnz_host gets
 * the total (the call synchronises on `stream` to return it).  Returns
 * RT3D_E_CAPACITY (and writes nothing past `capacity`) if it does not fit. */
rt3d_status rt3d_compact(rt3d_ctx_t* ctx, const rt3d_frame* f, uint32_t* csr_off,
                         uint32_t* csr_ent, int64_t capacity, int64_t* nnz_host,
                         void* stream);

/* Log-matched filter output of the initialisation kernel, for inspection:
 * y[h][w][t] int32 = sum_s z(tau + s - origin) K_s with the quantised
 * log-IRF K_s = round(2^f log1p(h_s / (delta_rel max h))).  Needs `dense`. */
rt3d_status rt3d_lmf(rt3d_ctx_t* ctx, const rt3d_frame* f, const rt3d_params* p,
                     int32_t* y, void* stream);

/* Initialisation only (matched filter, peaks, initial t, r, alive, b). */
rt3d_status rt3d_init(rt3d_ctx_t* ctx, const rt3d_frame* f, const rt3d_params* p,
                      rt3d_result* out, void* stream);

/* The whole method on one frame: initialisation (or warm start) then
 * params.n_iter PALM iterations.  Results land in `out`.  The launch sequence
 * of each call geometry (frame sizes, iteration count) is captured once as a
 * CUDA graph on a private stream and replayed on `stream`. */
rt3d_status rt3d_reconstruct(rt3d_ctx_t* ctx, const rt3d_frame* f, const rt3d_params* p,
                             rt3d_result* out, void* stream);

/* n frames (any mix of sizes within the configuration) in one set of
 * launches; frame i's results land in out[i].  Each frame's result is
 * bitwise identical to reconstructing it alone. */
rt3d_status rt3d_reconstruct_batch(rt3d_ctx_t* ctx, int n, const rt3d_frame* f,
                                   const rt3d_params* p, rt3d_result* out, void* stream);

/* End-to-end form with HOST buffers: copies the frame's arrays (HOST
 * pointers in `f`) to the device, reconstructs, and copies the results back
 * into HOST buffers `out` (n_points may be NULL).  Synchronous: returns after
 * the results are on the host.  Uses the context's staging buffers. */
rt3d_status rt3d_reconstruct_host(rt3d_ctx_t* ctx, const rt3d_frame* f, const rt3d_params* p,
                                  rt3d_result* out, void* stream);

/* Batched end-to-end form: n frames in HOST buffers (f[i]: HOST pointers;
 * dense and/or csr_off/csr_ent, optional gain), results into HOST buffers
 * out[i].  One copy per input array into a context staging area (grown to the
 * call's size on first use, freed by rt3d_destroy), one batched
 * reconstruction (as rt3d_reconstruct_batch), one copy back per result array;
 * with params.warm_start, out[i] is also the starting state.  When every
 * frame is dense and holds at least 64 MiB of histogram, the frames run in up
 * to four groups: their copies go on a stream of the context (after the work
 * already queued on `stream`) and each group's reconstruction starts as soon
 * as its own frames have arrived, overlapping the next groups' copies (the
 * results are per frame, so they equal the single batch's).  Synchronous:
 * returns after the results are on the host.  Page-locked host buffers give
 * full link bandwidth.  Errors: RT3D_E_INVALID for a NULL argument, n < 1 or
 * anything rt3d_reconstruct_batch rejects; RT3D_E_NOMEM if the staging cannot
 * be allocated. */
rt3d_status rt3d_reconstruct_batch_host(rt3d_ctx_t* ctx, int n, const rt3d_frame* f,
                                        const rt3d_params* p, rt3d_result* out, void* stream);

/* One fused phase of iteration k, for testing the loop kernels in isolation.
 * state holds t, r, alive, b (device, as rt3d_result); the frame's sparse list
 * (csr_off/csr_ent) is required.  phase:
 *   0 (A): [b <- background denoiser(b), unless `first`] then the depth
 *          gradient step: t <- t - beta_t dg/dt
 *   1 (B): APSS on t, then the intensity gradient step with the new t
 *   2 (C): intensity low-pass + pruning, then the background gradient step
 *          (b receives the step's output, before its denoiser)
 * All three update `state` in place. */
rt3d_status rt3d_phase(rt3d_ctx_t* ctx, int phase, int first, const rt3d_frame* f,
                       const rt3d_params* p, rt3d_result* state, void* stream);

/* Synchronise `stream`, then return and clear the device-side status word
 * (RT3D_OK, RT3D_E_TIMEOUT, RT3D_E_CAPACITY or RT3D_E_RANGE, in that order of
 * precedence). */
rt3d_status rt3d_device_status(rt3d_ctx_t* ctx, void* stream);

/* Kernel launches made by this context since creation (all entry points). */
int64_t rt3d_launch_count(rt3d_ctx_t* ctx);

/* Bound, in nanoseconds, of every device-side wait of this context's
 * tensor-core kernels (the BF16/FP16 matched filter and the learned
 * denoiser's pipelined convolution); default 1e9.  It takes effect from the
 * next call (it travels in the call record).  A kernel whose wait reaches the
 * bound stops, awaits its copies and matrix operations in flight, frees its
 * tensor memory and raises RT3D_E_TIMEOUT in rt3d_device_status(); that
 * call's results are not valid, the context stays usable.  0 gives up at the
 * first wait that has not already completed (a test of that path).
 * RT3D_E_INVALID for ns < 0. */
rt3d_status rt3d_set_wait_limit(rt3d_ctx_t* ctx, int64_t ns);

/* Per-kernel timing with CUDA events recorded around each launch (off by
 * default).  rt3d_kernel_times synchronises and returns, for kernel class i
 * (0 init, 1 phase A, 2 phase B, 3 phase C, 4 final, 5 synthesize, 6 compact),
 * the accumulated milliseconds and launch count since the last reset.  The
 * reconstruction entry points replay a CUDA graph per call geometry (captured
 * on first use); a graph re-records the same events, so its kernels count once,
 * from its latest replay -- averages per launch are exact, totals are one
 * replay's. */
rt3d_status rt3d_set_profiling(rt3d_ctx_t* ctx, int on);
rt3d_status rt3d_kernel_times(rt3d_ctx_t* ctx, double* ms, int64_t* launches, int n, int reset);

/* The whole method (as rt3d_reconstruct) without any allocation and without a
 * context.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory when they run -- processing loops that
 * reserve all memory at start-up for a fixed footprint, plugins whose host
 * framework owns the device memory, processes under a strict memory quota.
 * The kernels' scratch (sparse entries, half-step state, counters) lives in
 * one static device array of about 8.8 MiB, held by every GPU on which the
 * library's module has been loaded, until the process exits.  Under CUDA's
 * lazy module loading (the default since CUDA 12.2) the module -- and the
 * array -- is loaded on a device at the first call there, and each kernel's
 * code at its first launch: a caller that then reserves the rest of the
 * device's memory should first make one call of every form it will use
 * (cold and warm start; dense or sparse input) on each device, or load
 * modules eagerly (CUDA_MODULE_LOADING=EAGER).  Limits, checked on the host
 * before anything is launched (RT3D_E_INVALID otherwise): h*w <= 16384
 * pixels; with a dense histogram also h*w*t <= 2^21 bins; k_max <=
 * RT3D_MAX_K.  `irf` is a HOST pointer (normalised per call); frame and
 * result pointers are DEVICE pointers owned by the caller; the work is
 * enqueued on `stream` on the current CUDA device.  The matched filter runs
 * on CUDA cores whatever params.lmf_precision says (its integers are the same).
 * The learned depth denoiser, a per-pixel irf_index and upsample > 1 return
 * RT3D_E_UNIMPL.  The first call on a device looks the array's device address
 * up once (cudaGetSymbolAddress), so make that first call before any stream
 * capture; no call may be made while `stream` is being captured (the call
 * record goes up from a pageable host copy; RT3D_E_INVALID then).  Every call
 * shares the one array and reuses it from the previous call (the counters
 * and the device status word are cleared each call): calls whose work
 * overlaps on the GPU -- on different streams, or from several threads --
 * race on it and must be ordered by the caller.  Errors found on the device
 * (capacity, exact-arithmetic range) are read with rt3d_noalloc_status.  No
 * cudaMalloc, cudaFree or other allocating routine is called. */
rt3d_status rt3d_reconstruct_noalloc(const rt3d_irf* irf, const rt3d_frame* f,
                                     const rt3d_params* p, rt3d_result* out, void* stream);

/* The device status word of the last rt3d_reconstruct_noalloc call on the
 * current device (no counterpart in the paper; allocation-free like that
 * entry point): synchronises `stream`, returns RT3D_OK, RT3D_E_CAPACITY or
 * RT3D_E_RANGE (pixels whose counts exceed the exact-arithmetic range keep no
 * points) and clears the word. */
rt3d_status rt3d_noalloc_status(void* stream);

/* Copy the sparse representation built by the last initialisation out to
 * HOST buffers, for inspection: seg[p] = (start, count) per pixel of the
 * batch (in frame order) and ent[0..n_ent).  Synchronises `stream`. */
rt3d_status rt3d_get_sparse(rt3d_ctx_t* ctx, uint32_t* seg_host, int64_t n_pix,
                            uint32_t* ent_host, int64_t n_ent, int64_t* n_ent_used,
                            void* stream);

/* ---------------------------------------------------------------------------
 * Learned depth denoiser.  Not in the paper: an extension that stands in for
 * the APSS depth step (Results, "Depth update") with a small convolutional
 * network trained on pairs the plain method generates; APSS stays as the
 * per-point fallback (params.net_fallback) and as the reference for its error.
 *
 * Network: four 3x3 convolutions 6 -> 48 -> 48 -> 48 -> 2, zero padding,
 * bias, ReLU after the first three; RT3D_NET_PARAMS FP32 parameters, for each
 * layer W[co][ci][ky][kx] then b[co].  The convolutions use the bfloat16
 * rounding of the weights and of every layer input, with FP32 sums.
 * Features per pixel, first two slots k, from the n alive points of any slot
 * in the 8 neighbouring pixels within 4 scale in depth of t_k (its surface):
 * (t_k - their mean depth) / scale clamped to +-4 (0 if n = 0), log(1 + r_k),
 * (1 + n) / 9 for alive points (0 for dead or absent ones), channels
 * (t0, r0, a0, t1, r1, a1).  Output
 * y = (dt_0, dt_1) / scale.  Loss: masked mean of (y - target)^2.  Optimiser:
 * AdamW, decay on weights only.
 * --------------------------------------------------------------------------- */
#define RT3D_NET_PARAMS 45074

typedef struct rt3d_net rt3d_net_t;

typedef struct {
    float lr, beta1, beta2, eps, weight_decay;
} rt3d_adamw;

/* A network with device parameters, AdamW state and a workspace for batches
 * of up to max_images images of up to max_h x max_w pixels.  Parameters
 * start at zero (set them with rt3d_net_set_params). */
rt3d_status rt3d_net_create(int device, int max_images, int max_h, int max_w, rt3d_net_t** out);
void rt3d_net_destroy(rt3d_net_t* net);

/* HOST FP32 [RT3D_NET_PARAMS] in / out.  Setting resets the AdamW state. */
rt3d_status rt3d_net_set_params(rt3d_net_t* net, const float* theta);
rt3d_status rt3d_net_get_params(rt3d_net_t* net, float* theta);

/* Features of n point clouds (DEVICE): t, r [n][k][h][w] float, alive
 * [n][k][h][w] uint8 -> x [n][6][h][w] float holding bfloat16 values. */
rt3d_status rt3d_net_features(rt3d_net_t* net, int n, int k, int h, int w, const float* t, const float* r,
                              const uint8_t* alive, float scale, float* x, void* stream);

/* Forward pass (DEVICE): x [n][6][h][w] -> y [n][2][h][w]. */
rt3d_status rt3d_net_forward(rt3d_net_t* net, int n, int h, int w, const float* x, float* y, void* stream);

/* Forward, loss and backward (DEVICE): target [n][2][h][w] float, mask
 * [n][2][h][w] uint8 -> grad [RT3D_NET_PARAMS] (gradient of the masked mean
 * loss), loss [1]. */
rt3d_status rt3d_net_gradient(rt3d_net_t* net, int n, int h, int w, const float* x, const float* target,
                              const uint8_t* mask, float* grad, float* loss, void* stream);

/* One training step: gradient as above, then AdamW on the parameters.
 * loss [1] (DEVICE) receives the step's loss; may be NULL. */
rt3d_status rt3d_net_train_step(rt3d_net_t* net, int n, int h, int w, const float* x, const float* target,
                                const uint8_t* mask, const rt3d_adamw* opt, float* loss, void* stream);

/* The network a context's loop uses when params.depth_denoiser is
 * RT3D_DEPTH_LEARNED (NULL detaches).  The network must outlive its use; the
 * context allocates its inference buffers here.  Attaching a different
 * network waits for the device to finish its work and drops the context's
 * captured call graphs (they hold the previous network's buffers), so the
 * next call of each shape captures again; new
 * parameters set on the attached network (rt3d_net_set_params, training
 * steps) are seen by the next call without that. */
rt3d_status rt3d_set_depth_net(rt3d_ctx_t* ctx, rt3d_net_t* net);

#ifdef __cplusplus
}
#endif
#endif
