/*
 * rt3d_oracle.h -- plain, slow, FP64 CPU oracle of the reconstruction method of
 * Tachella et al., "Real-time 3D reconstruction from single-photon lidar data
 * using plug-and-play point cloud denoisers" (Nature Communications 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this code.  It shares nothing with the
 * CUDA library: no headers, no helpers, no tables.
 *
 * Paper passages followed (no numbered equations in the paper):
 *   - observation model: Results, "Observation model", the Poisson likelihood
 *     equation and the negative log-likelihood g(t, r, b) below it;
 *   - PALM block structure: Results, "Reconstruction algorithm" and Fig. 2;
 *   - depth / intensity / background updates: the three paragraphs of that
 *     section ("Depth update", "Intensity update", "Background update");
 *   - per-pixel initialisation and GPU mapping: Methods, "3D Reconstruction
 *     algorithm"; linear cost in active bins: Methods and Fig. 5.
 * Where the paper defers details to its supplementary notes (not available),
 * the reading used here is stated at the function; every such reading is
 * listed in the design notes of the repository.
 *
 * Parity status: every function below is pinned by a CPU test.  The paper has
 * no worked example of the full multi-iteration loop; or_palm and
 * or_reconstruct as a whole are pinned by properties the method has: noise-free
 * counts of two slanted planes are a fixed point of the whole iteration with
 * both denoisers and are recovered from a perturbed start, and the whole
 * reconstruction is equivariant under a shift of the time axis and under
 * transposing or mirroring the pixel grid.  The order of the steps within an
 * iteration is the paper's (Fig. 2) as written; no property separates it.
 */
#ifndef RT3D_ORACLE_H
#define RT3D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Instrument response: samples h[0..len), h[origin] sits at depth offset 0. */
typedef struct {
    int len;
    int origin;
    const double* h;          /* normalised so that sum h = 1 */
} or_irf;

/* Sparse histogram: per pixel p the nonzero bins bin[off[p]..off[p+1]) with
 * their counts (double so that expected counts can be fed as well).
 * irf_idx: the likelihood's instrument response is per pixel (h_{i,j}); every
 * function below that takes `irf` takes an array of responses, and pixel p
 * uses irf[irf_idx[p]] (irf_idx NULL: every pixel uses irf[0]). */
typedef struct {
    int h, w, t;
    const int64_t* off;       /* [h*w + 1] */
    const int32_t* bin;       /* [nnz] increasing within a pixel */
    const double* cnt;        /* [nnz] > 0 */
    const double* gain;       /* [h*w] */
    const uint8_t* irf_idx;   /* [h*w] or NULL */
} or_frame;

/* Point cloud in K slots per pixel plus the background image. */
typedef struct {
    int k;
    double* t;                /* [k][h][w] depth in bins */
    double* r;                /* [k][h][w] intensity (expected signal photons at gain 1) */
    uint8_t* alive;           /* [k][h][w] */
    double* b;                /* [h][w] background photons per bin */
} or_state;

typedef struct {
    int n_iter, k_max;
    double t_step, r_step, b_step, dt_max, eps_r, eps_b, b_floor, lam_floor;
    double pixel_pitch, apss_radius;
    int win_r, apss_min_nb;
    double int_radius, r_min, merge_dist;
    int depth_denoiser, intensity_denoiser, bkg_mode;
    double bkg_sigma;
    int bkg_radius;
    double lmf_delta_rel;
    int lmf_frac_bits, peak_min_photons, peak_sep;
    /* learned depth denoiser (depth_denoiser == 2): flat parameters, feature
     * and output depth scale (bins), per-point APSS fallback threshold (bins) */
    const double* net_theta;
    double net_scale, net_fallback;
    /* point-to-cube mapping f: super-resolution factor u (1 = off).  The
     * state's t, r, alive are then [K][u h][u w] on the world grid, whose
     * u x u blocks map to the h x w lidar pixels; b stays [h][w]. */
    int upsample;
} or_params;

/* ---- synthetic photons (input generation, not the method) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t or_poisson_fixed(uint32_t u, uint64_t p0, uint64_t mu);
void or_synthesize(int h, int w, int t, int n_comp,
                   const int32_t* depth_int, const uint32_t* depth_split,
                   const uint32_t* n_parts, const uint64_t* p0, const uint64_t* mu,
                   const uint32_t* irf_cdf, int irf_len, int irf_origin,
                   uint64_t seed, uint16_t* dense);

/* ---- observation model ---- */
void or_irf_eval(const or_irf* irf, double x, double* h, double* dh);
double or_nll_dense(int h, int w, int t, const double* z, const double* gain,
                    const or_state* s, const or_irf* irf, double lam_floor);
double or_nll_dense_idx(int h, int w, int t, const double* z, const double* gain, const uint8_t* irf_idx,
                        int up, const or_state* s, const or_irf* irf, double lam_floor);
void or_gradients(const or_frame* f, const or_state* s, const or_irf* irf,
                  const or_params* p, double* gt, double* gr, double* gb);

/* ---- initialisation ---- */
void or_lmf_kernel(const or_irf* irf, double delta_rel, int frac_bits, int32_t* kern);
void or_lmf(const uint16_t* z, int t, const int32_t* kern, int len, int origin,
            int64_t* y, int64_t* wcount);
int or_peaks(const int64_t* y, const int64_t* wcount, int t, int sep, int min_photons,
             int kmax, int32_t* taus);
void or_init(const uint16_t* dense, const double* gain, int h, int w, int t,
             const or_irf* irf, const or_params* p, or_state* s);
void or_init_idx(const uint16_t* dense, const double* gain, const uint8_t* irf_idx, int h, int w, int t,
                 const or_irf* irf, const or_params* p, or_state* s);

/* ---- one PALM iteration, step by step ---- */
void or_t_step(const or_frame* f, const or_irf* irf, const or_params* p, or_state* s);
void or_apss(int h, int w, int t, const or_params* p, or_state* s);
void or_plane(int h, int w, int t, const or_params* p, or_state* s);
void or_bilateral(int h, int w, int t, const or_params* p, or_state* s);
void or_r_step(const or_frame* f, const or_irf* irf, const or_params* p, or_state* s);
void or_int_lowpass(int h, int w, const or_params* p, or_state* s);
void or_b_step(const or_frame* f, const or_irf* irf, const or_params* p, or_state* s);
void or_bkg_lowpass(int h, int w, const or_params* p, double* b);

/* ---- learned depth denoiser (extension; net.c) ---- */
#define OR_NET_LAYERS 4
int or_net_cin(int layer);
int or_net_cout(int layer);
long or_net_offset(int layer, int bias);
long or_net_nparams(void);
double or_bf16(double x);
void or_bf16_round(double* x, long n);
void or_net_features(int h, int w, const or_state* s, double scale, double* x);
void or_net_forward(int n, int h, int w, const double* theta, const double* x, int bf16, double* acts,
                    double* y);
double or_net_loss(int n, int h, int w, const double* y, const double* target, const uint8_t* mask,
                   double* dy);
void or_net_backward(int n, int h, int w, const double* theta, const double* acts, const double* dy,
                     int bf16, double* dtheta, double* dx);
void or_adamw(double* theta, const double* g, double* m, double* v, int step, double lr, double beta1,
              double beta2, double eps, double wd);
void or_learned_depth(int h, int w, int t, const or_params* p, or_state* s);

/* ---- whole method ---- */
void or_depth_denoise(int h, int w, int t, const or_params* p, or_state* s);
void or_palm(const or_frame* f, const or_irf* irf, const or_params* p, or_state* s, int n_iter);
void or_reconstruct(const uint16_t* dense, const or_frame* f, const or_irf* irf,
                    const or_params* p, or_state* s);
int or_num_threads(void);
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
