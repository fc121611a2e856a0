/*
 * Observation model, negative log-likelihood, gradients and the three gradient
 * steps of the PALM iteration.  TEST INFRASTRUCTURE ONLY -- see rt3d_oracle.h.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include "rt3d_oracle.h"

#define IDX(k, p, npix) ((int64_t)(k) * (npix) + (p))

static double irf_sample(const or_irf* irf, int k)
{
    return (k < 0 || k >= irf->len) ? 0.0 : irf->h[k];
}

/* h(x) and h'(x): the continuous instrument response h_{i,j}(t - t_n) of the
 * likelihood equation (Results, "Observation model").  The paper samples it per
 * bin; a depth is real-valued, so the reading used here is the Catmull-Rom
 * cubic (Keys, a = -1/2) interpolant of the samples, which is C^1 and
 * reproduces constants (sum_t h(t - tau) = sum_k h_k when the support lies
 * inside the histogram). */
void or_irf_eval(const or_irf* irf, double x, double* h, double* dh)
{
    const double y = x + irf->origin;
    if (!(y > -2.0 && y < irf->len + 1.0)) {   /* outside the 4-tap support */
        *h = 0.0;
        *dh = 0.0;
        return;
    }
    const double kf = floor(y);
    const int k = (int)kf;
    const double u = y - kf;
    const double pm = irf_sample(irf, k - 1), p0 = irf_sample(irf, k);
    const double p1 = irf_sample(irf, k + 1), p2 = irf_sample(irf, k + 2);
    const double c1 = p1 - pm;
    const double c2 = 2.0 * pm - 5.0 * p0 + 4.0 * p1 - p2;
    const double c3 = -pm + 3.0 * p0 - 3.0 * p1 + p2;
    *h = 0.5 * (2.0 * p0 + c1 * u + c2 * u * u + c3 * u * u * u);
    *dh = 0.5 * (c1 + 2.0 * c2 * u + 3.0 * c3 * u * u);
}

/* The instrument response of pixel p: h_{i,j} of the likelihood equation is
 * per pixel; `irf` is the array of responses and idx[p] picks one (NULL:
 * every pixel uses irf[0]). */
static const or_irf* irf_at(const or_irf* irf, const uint8_t* idx, int64_t p)
{
    return idx ? irf + idx[p] : irf;
}

/* The point-to-cube mapping f(c_n) (Results, "Observation model"): with a
 * super-resolution factor u = p->upsample (1 = off), the point cloud lives on
 * a world grid u times finer than the pixels (Results, "3D Dynamic scenes":
 * a window of u x u world pixels maps to one lidar pixel), so the points N_ij
 * of lidar pixel (i, j) are those of world pixels (u i + a, u j + c),
 * 0 <= a, c < u.  The state's t, r, alive are [K][u h][u w]; b stays
 * [h][w].  block_points lists the world pixels of lidar pixel p. */
static int upsample_of(const or_params* prm)
{
    return prm && prm->upsample > 1 ? prm->upsample : 1;
}

static int block_points(int h, int w, int up, int64_t p, int64_t* q)
{
    const int64_t i = p / w, j = p % w, ww = (int64_t)w * up;
    int n = 0;
    for (int a = 0; a < up; ++a)
        for (int c = 0; c < up; ++c) q[n++] = (i * up + a) * ww + (j * up + c);
    (void)h;
    return n;
}

/* Mean count of lidar pixel p in bin t (likelihood equation):
 *   lambda = g (sum over the alive points n of N_ij of r_n h(t - t_n) + b),
 * floored at lam_floor so that the logarithm and 1/lambda exist.  q lists the
 * pixel's nq world pixels, wnpix is the world grid's pixel count. */
static double pixel_lambda(const or_state* s, const int64_t* q, int nq, int64_t wnpix, double b, double g,
                           const or_irf* irf, double tb, double lam_floor)
{
    double acc = b;
    for (int a = 0; a < nq; ++a)
        for (int k = 0; k < s->k; ++k) {
            const int64_t n = IDX(k, q[a], wnpix);
            if (!s->alive[n]) continue;
            double h, dh;
            or_irf_eval(irf, tb - s->t[n], &h, &dh);
            acc += s->r[n] * h;
        }
    const double lam = g * acc;
    return lam > lam_floor ? lam : lam_floor;
}

/* g(t, r, b) = sum_{i,j,t} (lambda - z log lambda), the negative log-likelihood
 * of Results, "Observation model", without the constant log z! term.  Dense
 * over every bin: the reference the sparse gradients are checked against.
 * h, w: the lidar grid; up: the super-resolution factor of the state. */
double or_nll_dense_idx(int h, int w, int t, const double* z, const double* gain, const uint8_t* irf_idx,
                        int up, const or_state* s, const or_irf* irf, double lam_floor)
{
    const int64_t npix = (int64_t)h * w, wnpix = npix * up * up;
    double total = 0.0;
    int64_t q[64];
    for (int64_t p = 0; p < npix; ++p) {
        const int nq = block_points(h, w, up, p, q);
        for (int tb = 0; tb < t; ++tb) {
            const double lam = pixel_lambda(s, q, nq, wnpix, s->b[p], gain[p], irf_at(irf, irf_idx, p),
                                            (double)tb, lam_floor);
            const double zz = z[p * t + tb];
            total += lam - (zz > 0.0 ? zz * log(lam) : 0.0);
        }
    }
    return total;
}

double or_nll_dense(int h, int w, int t, const double* z, const double* gain,
                    const or_state* s, const or_irf* irf, double lam_floor)
{
    return or_nll_dense_idx(h, w, t, z, gain, NULL, 1, s, irf, lam_floor);
}

/* H_n = sum_{t in [0,T)} h(t - t_n) and H'_n = sum_t h'(t - t_n): the part of the
 * gradient carried by the zero bins.  Summed over every bin where h can be
 * nonzero (explicitly, also in the interior where H = 1 and H' = 0). */
static void support_sums(const or_irf* irf, double tn, int t, double* H, double* dH)
{
    const int base = (int)floor(tn) - irf->origin;
    int lo = base - 3, hi = base + irf->len + 2;
    if (lo < 0) lo = 0;
    if (hi > t - 1) hi = t - 1;
    double sh = 0.0, sdh = 0.0;
    for (int tb = lo; tb <= hi; ++tb) {
        double hv, dv;
        or_irf_eval(irf, tb - tn, &hv, &dv);
        sh += hv;
        sdh += dv;
    }
    *H = sh;
    *dH = sdh;
}

/* Sums over the nonzero bins of lidar pixel p (the cost is linear in active
 * bins, Methods and Fig. 5), for the points of its world pixels q[0..nq)
 * (point (a, k) at index a K + k):
 *   sh[a K + k] = sum z h(t - t_n) / lambda,  sdh[...] = sum z h'(t - t_n) / lambda,
 *   *sz = sum z / lambda. */
static void pixel_sums(const or_frame* f, const or_state* s, const or_irf* irf_set, double lam_floor,
                       int64_t p, const int64_t* q, int nq, int64_t wnpix, double* sh, double* sdh, double* sz)
{
    const double g = f->gain[p];
    const or_irf* irf = irf_at(irf_set, f->irf_idx, p);
    for (int a = 0; a < nq * s->k; ++a) sh[a] = sdh[a] = 0.0;
    *sz = 0.0;
    for (int64_t e = f->off[p]; e < f->off[p + 1]; ++e) {
        const double tb = f->bin[e], zz = f->cnt[e];
        const double lam = pixel_lambda(s, q, nq, wnpix, s->b[p], g, irf, tb, lam_floor);
        *sz += zz / lam;
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) {
                const int64_t n = IDX(k, q[a], wnpix);
                if (!s->alive[n]) continue;
                double hv, dv;
                or_irf_eval(irf, tb - s->t[n], &hv, &dv);
                sh[a * s->k + k] += zz * hv / lam;
                sdh[a * s->k + k] += zz * dv / lam;
            }
    }
}

/* Gradient of g with respect to every t_n, r_n (alive points; 0 otherwise) and
 * b_ij.  Differentiating lambda - z log lambda:
 *   dg/dt_n = g r_n ( -H'_n + sum_{z>0} z h'(t - t_n) / lambda )
 *   dg/dr_n = g     (  H_n  - sum_{z>0} z h (t - t_n) / lambda )
 *   dg/db   = g     (  T    - sum_{z>0} z / lambda )
 * with lambda that of the lidar pixel whose block holds the point. */
void or_gradients(const or_frame* f, const or_state* s, const or_irf* irf,
                  const or_params* prm, double* gt, double* gr, double* gb)
{
    const int up = upsample_of(prm);
    const int64_t npix = (int64_t)f->h * f->w, wnpix = npix * up * up;
    for (int64_t p = 0; p < npix; ++p) {
        int64_t q[64];
        double sh[256], sdh[256], sz;
        const int nq = block_points(f->h, f->w, up, p, q);
        pixel_sums(f, s, irf, prm->lam_floor, p, q, nq, wnpix, sh, sdh, &sz);
        const double g = f->gain[p];
        gb[p] = g * (f->t - sz);
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) {
                const int64_t n = IDX(k, q[a], wnpix);
                if (!s->alive[n]) {
                    gt[n] = gr[n] = 0.0;
                    continue;
                }
                double H, dH;
                support_sums(irf_at(irf, f->irf_idx, p), s->t[n], f->t, &H, &dH);
                gt[n] = g * s->r[n] * (-dH + sdh[a * s->k + k]);
                gr[n] = g * (H - sh[a * s->k + k]);
            }
    }
}

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Depth update, gradient part (Results, "Reconstruction algorithm", depth
 * update).  All points of a lidar pixel move together from the same lambda.
 * Step (reading; the paper's step sizes are in its supplement): a scaled
 * Fisher-scoring step.  The expected information of a depth is about
 * g r_n I_h, I_h = sum h'^2/h the IRF's location information, so with
 * t_step = eta / I_h
 *   beta_t = t_step / (g r_n + eps_r),
 *   t_n <- clamp(t_n - clamp(beta_t dg/dt_n, +-dt_max), 0, T-1). */
void or_t_step(const or_frame* f, const or_irf* irf, const or_params* prm, or_state* s)
{
    const int up = upsample_of(prm);
    const int64_t npix = (int64_t)f->h * f->w, wnpix = npix * up * up;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        const double g = f->gain[p];
        if (!(g > 0.0)) continue;
        int64_t q[64];
        double sh[256], sdh[256], sz, newt[256];
        const int nq = block_points(f->h, f->w, up, p, q);
        pixel_sums(f, s, irf, prm->lam_floor, p, q, nq, wnpix, sh, sdh, &sz);
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) {
                const int64_t n = IDX(k, q[a], wnpix);
                double* nt = &newt[a * s->k + k];
                *nt = s->t[n];
                if (!s->alive[n]) continue;
                double H, dH;
                support_sums(irf_at(irf, f->irf_idx, p), s->t[n], f->t, &H, &dH);
                const double grad = g * s->r[n] * (-dH + sdh[a * s->k + k]);
                const double beta = prm->t_step / (g * s->r[n] + prm->eps_r);
                const double step = clampd(-beta * grad, -prm->dt_max, prm->dt_max);
                *nt = clampd(s->t[n] + step, 0.0, (double)(f->t - 1));
            }
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) s->t[IDX(k, q[a], wnpix)] = newt[a * s->k + k];
    }
}

/* Intensity update, gradient part.  Step (reading): beta_r = r_step (r_n + eps_r)/g,
 *   r_n <- max(0, r_n - r_step (r_n + eps_r)(H_n - sum z h / lambda));
 * with r_step = 1 and eps_r = 0 this is the EM (Richardson-Lucy) update
 * r <- r sum z h / lambda / H, so the step is a damped EM step. */
void or_r_step(const or_frame* f, const or_irf* irf, const or_params* prm, or_state* s)
{
    const int up = upsample_of(prm);
    const int64_t npix = (int64_t)f->h * f->w, wnpix = npix * up * up;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        const double g = f->gain[p];
        if (!(g > 0.0)) continue;
        int64_t q[64];
        double sh[256], sdh[256], sz, newr[256];
        const int nq = block_points(f->h, f->w, up, p, q);
        pixel_sums(f, s, irf, prm->lam_floor, p, q, nq, wnpix, sh, sdh, &sz);
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) {
                const int64_t n = IDX(k, q[a], wnpix);
                double* nr = &newr[a * s->k + k];
                *nr = s->r[n];
                if (!s->alive[n]) continue;
                double H, dH;
                support_sums(irf_at(irf, f->irf_idx, p), s->t[n], f->t, &H, &dH);
                const double v = s->r[n] - prm->r_step * (s->r[n] + prm->eps_r) * (H - sh[a * s->k + k]);
                *nr = v > 0.0 ? v : 0.0;
            }
        for (int a = 0; a < nq; ++a)
            for (int k = 0; k < s->k; ++k) s->r[IDX(k, q[a], wnpix)] = newr[a * s->k + k];
    }
}

/* Background update, gradient part.  Step (reading): beta_b = b_step (b + eps_b)/(g T),
 *   b <- max(b_floor, b - b_step (b + eps_b)(1 - sum z/lambda / T)),
 * likewise a damped EM step for the background (one per lidar pixel). */
void or_b_step(const or_frame* f, const or_irf* irf, const or_params* prm, or_state* s)
{
    const int up = upsample_of(prm);
    const int64_t npix = (int64_t)f->h * f->w, wnpix = npix * up * up;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        const double g = f->gain[p];
        if (!(g > 0.0)) continue;
        int64_t q[64];
        double sh[256], sdh[256], sz;
        const int nq = block_points(f->h, f->w, up, p, q);
        pixel_sums(f, s, irf, prm->lam_floor, p, q, nq, wnpix, sh, sdh, &sz);
        const double v = s->b[p] - prm->b_step * (s->b[p] + prm->eps_b) * (1.0 - sz / f->t);
        s->b[p] = v > prm->b_floor ? v : prm->b_floor;
    }
}

/* Threads of the OpenMP parallel loops (n >= 1); no effect without OpenMP. */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
