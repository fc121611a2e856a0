/*
 * The reconstruction loop.  TEST INFRASTRUCTURE ONLY -- see rt3d_oracle.h.
 *
 * PALM (Bolte, Sabach & Teboulle 2014) over the blocks t, r, b as in Results,
 * "Reconstruction algorithm" and Fig. 2: each block takes a gradient step on
 * the negative log-likelihood and then a denoiser in the role of the proximal
 * operator, in the order depth, intensity, background.  A fixed number of
 * iterations is run (reading: the paper gives no stopping rule).
 */
#include "rt3d_oracle.h"

/* The depth block's denoiser, by p->depth_denoiser: 0 none, 1 APSS (the
 * paper's), 2 the learned network with its APSS fallback, 3 a local plane
 * fit, 4 a bilateral depth filter (the last two: denoise.c). */
void or_depth_denoise(int h, int w, int t, const or_params* p, or_state* s)
{
    if (p->depth_denoiser == 1) or_apss(h, w, t, p, s);
    if (p->depth_denoiser == 2) or_learned_depth(h, w, t, p, s);
    if (p->depth_denoiser == 3) or_plane(h, w, t, p, s);
    if (p->depth_denoiser == 4) or_bilateral(h, w, t, p, s);
}

void or_palm(const or_frame* f, const or_irf* irf, const or_params* p, or_state* s, int n_iter)
{
    /* the point cloud's denoisers run on the world grid (u times finer than
     * the pixels with super-resolution), the background's on the pixels */
    const int up = p->upsample > 1 ? p->upsample : 1;
    const int wh = f->h * up, ww = f->w * up;
    for (int it = 0; it < n_iter; ++it) {
        or_t_step(f, irf, p, s);                         /* depth: gradient step */
        or_depth_denoise(wh, ww, f->t, p, s);            /* depth: denoiser */
        or_r_step(f, irf, p, s);                         /* intensity: gradient step */
        or_int_lowpass(wh, ww, p, s);                    /* intensity: low-pass + pruning */
        or_b_step(f, irf, p, s);                         /* background: gradient step */
        or_bkg_lowpass(f->h, f->w, p, s->b);             /* background: denoiser */
    }
}

void or_reconstruct(const uint16_t* dense, const or_frame* f, const or_irf* irf,
                    const or_params* p, or_state* s)
{
    or_init_idx(dense, f->gain, f->irf_idx, f->h, f->w, f->t, irf, p, s);
    or_palm(f, irf, p, s, p->n_iter);
}
