/*
 * Plug-and-play denoisers of the PALM iteration.  TEST INFRASTRUCTURE ONLY --
 * see rt3d_oracle.h.
 *
 *   or_apss          depth: algebraic point set surfaces (Results, "Depth
 *                    update"; Guennebaud & Gross 2007)
 *   or_int_lowpass   intensity: neighbourhood low-pass on the surface, then
 *                    pruning (Results, "Intensity update")
 *   or_bkg_lowpass   background: identity or FFT-equivalent low-pass
 *                    (Results, "Background update"; Methods)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "rt3d_oracle.h"

/* Solve the 4x4 system A u = rhs by Gaussian elimination with partial pivoting.
 * Returns 0 if a pivot vanishes. */
static int solve4(double A[4][4], double rhs[4], double u[4])
{
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 0;
        if (piv != c) {
            for (int q = 0; q < 4; ++q) {
                double tmp = A[c][q];
                A[c][q] = A[piv][q];
                A[piv][q] = tmp;
            }
            double tmp = rhs[c];
            rhs[c] = rhs[piv];
            rhs[piv] = tmp;
        }
        for (int r = c + 1; r < 4; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int q = c; q < 4; ++q) A[r][q] -= f * A[c][q];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = 3; c >= 0; --c) {
        double acc = rhs[c];
        for (int q = c + 1; q < 4; ++q) acc -= A[c][q] * u[q];
        u[c] = acc / A[c][c];
    }
    return 1;
}

/* APSS step for one point n at pixel (i, j), slot k (reading of the depth
 * denoiser; the fit variant is in the paper's supplement):
 *  - world coordinates c = (pitch j, pitch i, t) (orthographic f);
 *  - neighbours: alive points of all slots in the (2R+1)^2 pixel window,
 *    weight w = (1 - |c_m - c_n|^2 / h^2)^4 inside the radius h, else 0;
 *  - in local coordinates x = (c_m - c_n)/h, fit the algebraic sphere
 *    s(x) = u0 + u1 x + u2 y + z + u4 |x|^2 (gradient normalised to 1 along the
 *    line of sight) minimising sum w s(x_m)^2, i.e. the weighted least squares
 *    problem  [1 x y |x|^2] u = -z;
 *  - project the point along the line of sight onto s = 0: the root of
 *    u4 z^2 + z + u0 = 0 nearest 0, z* = -2 u0 / (1 + sqrt(max(0, 1 - 4 u0 u4))),
 *    clamped to [-1, 1]; t_n <- clamp(t_n + h z*, 0, T-1);
 *  - left unchanged when fewer than apss_min_nb neighbours carry weight or
 *    their pixel offsets are collinear (the fit is then undetermined).
 * The cut-off test |x|^2 < 1 is taken in single precision, like the kernel. */
static double apss_point(const double* tsrc, const uint8_t* alive, int h, int w, int t, int K,
                         int i, int j, int k, const or_params* prm)
{
    const int64_t npix = (int64_t)h * w;
    const double hr = prm->apss_radius, pitch = prm->pixel_pitch;
    const int R = prm->win_r;
    const double tn = tsrc[(int64_t)k * npix + (int64_t)i * w + j];
    double A[4][4] = {{0}}, rhs[4] = {0};
    int nw = 0;
    int64_t c0 = 0, ci = 0, cj = 0, cii = 0, cjj = 0, cij = 0;
    for (int di = -R; di <= R; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= h) continue;
        for (int dj = -R; dj <= R; ++dj) {
            const int jj = j + dj;
            if (jj < 0 || jj >= w) continue;
            for (int m = 0; m < K; ++m) {
                const int64_t q = (int64_t)m * npix + (int64_t)ii * w + jj;
                if (!alive[q]) continue;
                const double x = pitch * dj / hr, y = pitch * di / hr, z = (tsrc[q] - tn) / hr;
                const double d2 = x * x + y * y + z * z;
                if (!((float)d2 < 1.0f)) continue;
                const double om = 1.0 - d2;
                const double wt = om * om * om * om;
                const double bv[4] = {1.0, x, y, d2};
                for (int a = 0; a < 4; ++a) {
                    for (int c = 0; c < 4; ++c) A[a][c] += wt * bv[a] * bv[c];
                    rhs[a] -= wt * bv[a] * z;
                }
                ++nw;
                c0 += 1; ci += di; cj += dj;
                cii += (int64_t)di * di; cjj += (int64_t)dj * dj; cij += (int64_t)di * dj;
            }
        }
    }
    if (nw < prm->apss_min_nb) return tn;
    /* collinear pixel offsets <=> singular 2x2 covariance of (di, dj), in integers */
    const int64_t vii = c0 * cii - ci * ci, vjj = c0 * cjj - cj * cj, vij = c0 * cij - ci * cj;
    if (vii * vjj - vij * vij == 0) return tn;
    double u[4];
    if (!solve4(A, rhs, u)) return tn;
    const double disc = 1.0 - 4.0 * u[0] * u[3];
    double zs = -2.0 * u[0] / (1.0 + sqrt(disc > 0.0 ? disc : 0.0));
    if (zs > 1.0) zs = 1.0;
    if (zs < -1.0) zs = -1.0;
    double tn_new = tn + hr * zs;
    if (tn_new < 0.0) tn_new = 0.0;
    if (tn_new > t - 1) tn_new = t - 1;
    return tn_new;
}

/* All points are projected from the same input cloud (a Jacobi sweep). */
void or_apss(int h, int w, int t, const or_params* prm, or_state* s)
{
    const int64_t npix = (int64_t)h * w;
    const int K = s->k;
    double* src = (double*)malloc(sizeof(double) * K * npix);
    memcpy(src, s->t, sizeof(double) * K * npix);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        const int i = (int)(p / w), j = (int)(p % w);
        for (int k = 0; k < K; ++k) {
            const int64_t n = (int64_t)k * npix + p;
            if (s->alive[n]) s->t[n] = apss_point(src, s->alive, h, w, t, K, i, j, k, prm);
        }
    }
    free(src);
}

/* Other plug-in depth denoisers (the paper's Discussion: the framework takes
 * other point cloud denoisers, trading quality against speed; the variants
 * themselves are in its supplement, which is not available).  Both use the
 * APSS neighbourhood: the alive points of all slots in the (2R+1)^2 pixel
 * window, local coordinates x = (c_m - c_n)/h with h = apss_radius, weight
 * w = (1 - |x|^2)^4 inside the unit ball (the cut-off test in single
 * precision, as for APSS), and leave the point unchanged when fewer than
 * apss_min_nb neighbours carry weight.
 *
 * or_plane      local plane fit: the weighted least-squares plane
 *               u0 + u1 x + u2 y + z = 0 (3x3 normal equations of [1 x y]
 *               against -z, Gaussian elimination), the point moved along the
 *               line of sight onto it: z* = -u0, clamped to one radius; also
 *               unchanged when the neighbours' pixel offsets are collinear.
 *               Planes are fixed points; spheres are not (the sphere term of
 *               APSS is dropped).
 * or_bilateral  bilateral depth filter: the weight-averaged depth offset
 *               z* = sum w z / sum w over the same neighbours (the point
 *               itself included, z = 0, w = 1): a zero-order fit. */
static int solve_n(int n, double A[4][4], double rhs[4], double u[4])
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 0;
        if (piv != c) {
            for (int q = 0; q < n; ++q) {
                double tmp = A[c][q];
                A[c][q] = A[piv][q];
                A[piv][q] = tmp;
            }
            double tmp = rhs[c];
            rhs[c] = rhs[piv];
            rhs[piv] = tmp;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int q = c; q < n; ++q) A[r][q] -= f * A[c][q];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double acc = rhs[c];
        for (int q = c + 1; q < n; ++q) acc -= A[c][q] * u[q];
        u[c] = acc / A[c][c];
    }
    return 1;
}

/* mode 0: plane fit, 1: bilateral filter (see above). */
static double local_fit_point(const double* tsrc, const uint8_t* alive, int h, int w, int t, int K,
                              int i, int j, int k, const or_params* prm, int mode)
{
    const int64_t npix = (int64_t)h * w;
    const double hr = prm->apss_radius, pitch = prm->pixel_pitch;
    const int R = prm->win_r;
    const double tn = tsrc[(int64_t)k * npix + (int64_t)i * w + j];
    double A[4][4] = {{0}}, rhs[4] = {0};
    double sw = 0.0, swz = 0.0;
    int nw = 0;
    int64_t c0 = 0, ci = 0, cj = 0, cii = 0, cjj = 0, cij = 0;
    for (int di = -R; di <= R; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= h) continue;
        for (int dj = -R; dj <= R; ++dj) {
            const int jj = j + dj;
            if (jj < 0 || jj >= w) continue;
            for (int m = 0; m < K; ++m) {
                const int64_t q = (int64_t)m * npix + (int64_t)ii * w + jj;
                if (!alive[q]) continue;
                const double x = pitch * dj / hr, y = pitch * di / hr, z = (tsrc[q] - tn) / hr;
                const double d2 = x * x + y * y + z * z;
                if (!((float)d2 < 1.0f)) continue;
                const double om = 1.0 - d2;
                const double wt = om * om * om * om;
                const double bv[3] = {1.0, x, y};
                for (int a = 0; a < 3; ++a) {
                    for (int c = 0; c < 3; ++c) A[a][c] += wt * bv[a] * bv[c];
                    rhs[a] -= wt * bv[a] * z;
                }
                sw += wt;
                swz += wt * z;
                ++nw;
                c0 += 1; ci += di; cj += dj;
                cii += (int64_t)di * di; cjj += (int64_t)dj * dj; cij += (int64_t)di * dj;
            }
        }
    }
    if (nw < prm->apss_min_nb) return tn;
    double zs;
    if (mode == 0) {
        const int64_t vii = c0 * cii - ci * ci, vjj = c0 * cjj - cj * cj, vij = c0 * cij - ci * cj;
        if (vii * vjj - vij * vij == 0) return tn;
        double u[4];
        if (!solve_n(3, A, rhs, u)) return tn;
        zs = -u[0];
    } else {
        zs = swz / sw;
    }
    if (zs > 1.0) zs = 1.0;
    if (zs < -1.0) zs = -1.0;
    double tn_new = tn + hr * zs;
    if (tn_new < 0.0) tn_new = 0.0;
    if (tn_new > t - 1) tn_new = t - 1;
    return tn_new;
}

static void local_fit(int h, int w, int t, const or_params* prm, or_state* s, int mode)
{
    const int64_t npix = (int64_t)h * w;
    const int K = s->k;
    double* src = (double*)malloc(sizeof(double) * K * npix);
    memcpy(src, s->t, sizeof(double) * K * npix);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        const int i = (int)(p / w), j = (int)(p % w);
        for (int k = 0; k < K; ++k) {
            const int64_t n = (int64_t)k * npix + p;
            if (s->alive[n]) s->t[n] = local_fit_point(src, s->alive, h, w, t, K, i, j, k, prm, mode);
        }
    }
    free(src);
}

void or_plane(int h, int w, int t, const or_params* prm, or_state* s) { local_fit(h, w, t, prm, s, 0); }

void or_bilateral(int h, int w, int t, const or_params* prm, or_state* s) { local_fit(h, w, t, prm, s, 1); }

/* Intensity denoiser (reading): each alive point takes the weighted mean of the
 * intensities of the alive points of its (2R+1)^2 pixel window that lie on the
 * same surface patch, w = (1 - d^2/h_r^2)^4 for the world distance d < h_r
 * (itself included, w = 1) -- a nearest-neighbour low-pass in the manifold
 * metric.  Then points whose intensity is below r_min are removed (Results,
 * "Intensity update"); that decision is taken in single precision, like the
 * kernel.  Finally two surviving points of one pixel closer in depth than
 * merge_dist describe one surface: scanning slot pairs (a, c), a < c, in
 * order, the one with the smaller intensity (c on a tie) is removed and its
 * intensity added to the other (reading: keeps one point per surface and
 * pixel, which the likelihood alone cannot separate). */
void or_int_lowpass(int h, int w, const or_params* prm, or_state* s)
{
    const int64_t npix = (int64_t)h * w;
    const int K = s->k, R = prm->win_r;
    const double hr = prm->int_radius, pitch = prm->pixel_pitch;
    double* rsrc = (double*)malloc(sizeof(double) * K * npix);
    memcpy(rsrc, s->r, sizeof(double) * K * npix);
    uint8_t* asrc = (uint8_t*)malloc((size_t)K * npix);
    memcpy(asrc, s->alive, (size_t)K * npix);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        const int i = (int)(p / w), j = (int)(p % w);
        for (int k = 0; k < K; ++k) {
            const int64_t n = (int64_t)k * npix + p;
            if (!asrc[n]) continue;
            double rbar = rsrc[n];
            if (prm->intensity_denoiser) {
                double num = 0.0, den = 0.0;
                for (int di = -R; di <= R; ++di) {
                    const int ii = i + di;
                    if (ii < 0 || ii >= h) continue;
                    for (int dj = -R; dj <= R; ++dj) {
                        const int jj = j + dj;
                        if (jj < 0 || jj >= w) continue;
                        for (int m = 0; m < K; ++m) {
                            const int64_t q = (int64_t)m * npix + (int64_t)ii * w + jj;
                            if (!asrc[q]) continue;
                            const double x = pitch * dj / hr, y = pitch * di / hr;
                            const double z = (s->t[q] - s->t[n]) / hr;
                            const double d2 = x * x + y * y + z * z;
                            if (!(d2 < 1.0)) continue;
                            const double om = 1.0 - d2;
                            const double wt = om * om * om * om;
                            num += wt * rsrc[q];
                            den += wt;
                        }
                    }
                }
                rbar = num / den;
            }
            s->r[n] = rbar;
            s->alive[n] = ((float)rbar >= (float)prm->r_min) ? 1 : 0;
        }
        for (int a = 0; a < K; ++a)
            for (int c = a + 1; c < K; ++c) {
                const int64_t na = (int64_t)a * npix + p, nc = (int64_t)c * npix + p;
                if (!s->alive[na] || !s->alive[nc]) continue;
                if (!((float)fabs(s->t[na] - s->t[nc]) < (float)prm->merge_dist)) continue;
                const int64_t keep = s->r[nc] > s->r[na] ? nc : na;
                const int64_t drop = keep == na ? nc : na;
                s->r[keep] += s->r[drop];
                s->alive[drop] = 0;
            }
    }
    free(rsrc);
    free(asrc);
}

/* Background denoiser.  Mode 0 (bistatic systems): identity.  Mode 1 (monostatic
 * systems and arrays): the paper filters the background image with the FFT; the
 * reading here is the periodic convolution with the normalised separable
 * Gaussian k(d) ~ exp(-d^2 / (2 sigma^2)), |d| <= radius, which equals
 * multiplying the image's 2-D DFT by the DFT of that kernel. */
void or_bkg_lowpass(int h, int w, const or_params* prm, double* b)
{
    if (prm->bkg_mode != 1) return;
    const int rad = prm->bkg_radius;
    double* ker = (double*)malloc(sizeof(double) * (2 * rad + 1));
    double ksum = 0.0;
    for (int d = -rad; d <= rad; ++d) {
        ker[d + rad] = exp(-(double)d * d / (2.0 * prm->bkg_sigma * prm->bkg_sigma));
        ksum += ker[d + rad];
    }
    for (int d = 0; d <= 2 * rad; ++d) ker[d] /= ksum;
    const int64_t npix = (int64_t)h * w;
    double* src = (double*)malloc(sizeof(double) * npix);
    memcpy(src, b, sizeof(double) * npix);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npix; ++p) {
        const int i = (int)(p / w), j = (int)(p % w);
        double acc = 0.0;
        for (int di = -rad; di <= rad; ++di) {
            const int ii = (int)((((int64_t)i + di) % h + h) % h);
            for (int dj = -rad; dj <= rad; ++dj) {
                const int jj = (int)((((int64_t)j + dj) % w + w) % w);
                acc += ker[di + rad] * ker[dj + rad] * src[(int64_t)ii * w + jj];
            }
        }
        b[p] = acc;
    }
    free(src);
    free(ker);
}
