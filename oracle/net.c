/*
 * Learned depth denoiser -- TEST INFRASTRUCTURE ONLY, see rt3d_oracle.h.
 *
 * Not in the paper: an extension that stands in for the APSS depth step
 * (Results, "Depth update") with a small convolutional network, trained on
 * pairs the plain method generates.  The reading implemented here:
 *
 *  - features, per pixel and for the first two slots k (absent slots give 0):
 *    the point's same-surface neighbours are the alive points of any slot in
 *    the 8 neighbouring pixels whose depth is within 4 scale of t_k (the
 *    decision in single precision, like the kernel); with n of them and m
 *    their mean depth,
 *      f_t = clamp((t_k - m) / scale, -4, 4)  (0 when n = 0),
 *      f_r = log(1 + r_k),  f_a = (1 + n) / 9  (alive points only; dead give 0);
 *    channel order (f_t0, f_r0, f_a0, f_t1, f_r1, f_a1);
 *  - network: four 3x3 convolutions, 6 -> 48 -> 48 -> 48 -> 2 channels, zero
 *    padding, bias, ReLU after the first three; output y = (dt_0, dt_1) / scale;
 *  - precision (what the GPU computes): weights and every layer input rounded
 *    to bfloat16 (round to nearest even, through float), sums in FP32 on the
 *    GPU and FP64 here; the output is not rounded.  Gradients treat the
 *    rounding as identity;
 *  - loss: mean of m (y - target)^2 over the mask m (1 for alive points of
 *    slots 0 and 1), divided by max(1, sum m);
 *  - optimiser: AdamW (Loshchilov & Hutter), decoupled weight decay on the
 *    convolution weights only;
 *  - in the loop: a point moves by dt = y scale when |dt| <= fallback (in
 *    single precision, like the kernel), otherwise it takes the APSS update;
 *    slots beyond the second always take APSS.
 *
 * Parameters are one flat vector theta: for each layer its weights
 * W[co][ci][ky][kx] then its biases b[co].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "rt3d_oracle.h"

static const int cin_[OR_NET_LAYERS] = {6, 48, 48, 48};
static const int cout_[OR_NET_LAYERS] = {48, 48, 48, 2};

int or_net_cin(int l) { return cin_[l]; }
int or_net_cout(int l) { return cout_[l]; }

long or_net_offset(int l, int bias)
{
    long off = 0;
    for (int q = 0; q < l; ++q) off += (long)cout_[q] * cin_[q] * 9 + cout_[q];
    return bias ? off + (long)cout_[l] * cin_[l] * 9 : off;
}

long or_net_nparams(void) { return or_net_offset(OR_NET_LAYERS, 0); }

/* bfloat16 rounding: to float (nearest), then the top 16 bits (nearest, ties
 * to even).  Infinities and NaN do not occur here. */
double or_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

void or_bf16_round(double* x, long n)
{
    for (long q = 0; q < n; ++q) x[q] = or_bf16(x[q]);
}

void or_net_features(int h, int w, const or_state* s, double scale, double* x)
{
    const long npix = (long)h * w;
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < w; ++j) {
                const long p = (long)i * w + j;
                double ft = 0.0, fr = 0.0, fa = 0.0;
                if (k < s->k && s->alive[k * npix + p]) {
                    const double tk = s->t[k * npix + p];
                    double sum = 0.0;
                    int n = 0;
                    for (int di = -1; di <= 1; ++di)
                        for (int dj = -1; dj <= 1; ++dj) {
                            if (di == 0 && dj == 0) continue;
                            const int ii = i + di, jj = j + dj;
                            if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                            for (int kk = 0; kk < s->k; ++kk) {
                                const long q = kk * npix + (long)ii * w + jj;
                                if (!s->alive[q]) continue;
                                if (!(fabsf((float)(s->t[q] - tk)) <= (float)(4.0 * scale))) continue;
                                sum += s->t[q];
                                ++n;
                            }
                        }
                    if (n > 0) {
                        ft = (tk - sum / n) / scale;
                        if (ft > 4.0) ft = 4.0;
                        if (ft < -4.0) ft = -4.0;
                    }
                    const double rk = s->r[k * npix + p];
                    fr = log1p(rk > 0.0 ? rk : 0.0);
                    fa = (1.0 + n) / 9.0;
                }
                x[(3 * k + 0) * npix + p] = ft;
                x[(3 * k + 1) * npix + p] = fr;
                x[(3 * k + 2) * npix + p] = fa;
            }
}

/* One 3x3 convolution of one image: out[co] = b[co] + sum W[co][ci] * in[ci]
 * (zero padding); planes [c][h][w]. */
static void conv3x3(int h, int w, int ci_n, int co_n, const double* W, const double* b,
                    const double* in, double* out)
{
    const long npix = (long)h * w;
    /* output channels in parallel when the caller's image loop is not (one
     * image); each output keeps its own summation order */
#pragma omp parallel for schedule(static)
    for (int co = 0; co < co_n; ++co)
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < w; ++j) {
                double acc = b[co];
                for (int ci = 0; ci < ci_n; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const int ii = i + ky - 1, jj = j + kx - 1;
                            if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                            acc += W[((long)(co * ci_n + ci) * 3 + ky) * 3 + kx] *
                                   in[ci * npix + (long)ii * w + jj];
                        }
                out[co * npix + (long)i * w + j] = acc;
            }
}

static void round_vec(double* v, long n, int bf16)
{
    if (!bf16) return;
    for (long q = 0; q < n; ++q) v[q] = or_bf16(v[q]);
}

/* Forward pass of n images x [n][6][h][w]; acts holds each layer's input
 * a_0 .. a_3 (a_0 = x as used), as [n][c][h][w] blocks one after the other,
 * y [n][2][h][w].  bf16 = 1 applies the rounding described at the top. */
void or_net_forward(int n, int h, int w, const double* theta, const double* x, int bf16, double* acts,
                    double* y)
{
    const long npix = (long)h * w;
    const long np = or_net_nparams();
    double* th = (double*)malloc(sizeof(double) * np);
    memcpy(th, theta, sizeof(double) * np);
    for (int l = 0; l < OR_NET_LAYERS; ++l)
        round_vec(th + or_net_offset(l, 0), (long)cout_[l] * cin_[l] * 9, bf16);
    long aoff[OR_NET_LAYERS];
    long off = 0;
    for (int l = 0; l < OR_NET_LAYERS; ++l) {
        aoff[l] = off;
        off += (long)n * cin_[l] * npix;
    }
    memcpy(acts, x, sizeof(double) * n * cin_[0] * npix);
    round_vec(acts, (long)n * cin_[0] * npix, bf16);
#pragma omp parallel for if (n > 1)
    for (int im = 0; im < n; ++im) {
        for (int l = 0; l < OR_NET_LAYERS; ++l) {
            const double* in = acts + aoff[l] + (long)im * cin_[l] * npix;
            double* out = l + 1 < OR_NET_LAYERS ? acts + aoff[l + 1] + (long)im * cout_[l] * npix
                                                : y + (long)im * cout_[l] * npix;
            conv3x3(h, w, cin_[l], cout_[l], th + or_net_offset(l, 0), th + or_net_offset(l, 1), in, out);
            if (l + 1 < OR_NET_LAYERS) {
                const long cnt = (long)cout_[l] * npix;
                for (long q = 0; q < cnt; ++q) out[q] = out[q] > 0.0 ? out[q] : 0.0;
                round_vec(out, cnt, bf16);
            }
        }
    }
    free(th);
}

double or_net_loss(int n, int h, int w, const double* y, const double* target, const uint8_t* mask,
                   double* dy)
{
    const long cnt = (long)n * 2 * h * w;
    double msum = 0.0, sse = 0.0;
    for (long q = 0; q < cnt; ++q) msum += mask[q];
    const double inv = 1.0 / (msum > 1.0 ? msum : 1.0);
    for (long q = 0; q < cnt; ++q) {
        const double e = mask[q] ? y[q] - target[q] : 0.0;
        sse += e * e;
        if (dy) dy[q] = 2.0 * e * inv;
    }
    return sse * inv;
}

/* Gradient of the loss with respect to theta (and optionally x) given the
 * forward's activations and dL/dy.  The derivative of ReLU is 1 where the
 * stored activation is positive. */
void or_net_backward(int n, int h, int w, const double* theta, const double* acts, const double* dy,
                     int bf16, double* dtheta, double* dx)
{
    const long npix = (long)h * w;
    const long np = or_net_nparams();
    double* th = (double*)malloc(sizeof(double) * np);
    memcpy(th, theta, sizeof(double) * np);
    for (int l = 0; l < OR_NET_LAYERS; ++l)
        round_vec(th + or_net_offset(l, 0), (long)cout_[l] * cin_[l] * 9, bf16);
    long aoff[OR_NET_LAYERS];
    long off = 0;
    for (int l = 0; l < OR_NET_LAYERS; ++l) {
        aoff[l] = off;
        off += (long)n * cin_[l] * npix;
    }
    memset(dtheta, 0, sizeof(double) * np);
    const int cmax = 48;
    double* gz = (double*)malloc(sizeof(double) * cmax * npix);   /* dL/dz of the current layer */
    double* ga = (double*)malloc(sizeof(double) * cmax * npix);   /* dL/d(input) of the current layer */
    for (int im = 0; im < n; ++im) {
        memcpy(gz, dy + (long)im * 2 * npix, sizeof(double) * 2 * npix);
        for (int l = OR_NET_LAYERS - 1; l >= 0; --l) {
            const int ci_n = cin_[l], co_n = cout_[l];
            const double* W = th + or_net_offset(l, 0);
            double* dW = dtheta + or_net_offset(l, 0);
            double* db = dtheta + or_net_offset(l, 1);
            const double* a = acts + aoff[l] + (long)im * ci_n * npix;
            for (int co = 0; co < co_n; ++co)
                for (long p = 0; p < npix; ++p) db[co] += gz[co * npix + p];
            for (int co = 0; co < co_n; ++co)
                for (int ci = 0; ci < ci_n; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            double acc = 0.0;
                            for (int i = 0; i < h; ++i)
                                for (int j = 0; j < w; ++j) {
                                    const int ii = i + ky - 1, jj = j + kx - 1;
                                    if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                                    acc += gz[co * npix + (long)i * w + j] * a[ci * npix + (long)ii * w + jj];
                                }
                            dW[((long)(co * ci_n + ci) * 3 + ky) * 3 + kx] += acc;
                        }
            /* dL/d(input)[ci][q] = sum_co sum_k W[co][ci][k] gz[co][q - k + 1] */
            memset(ga, 0, sizeof(double) * ci_n * npix);
            for (int co = 0; co < co_n; ++co)
                for (int ci = 0; ci < ci_n; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const double wv = W[((long)(co * ci_n + ci) * 3 + ky) * 3 + kx];
                            for (int i = 0; i < h; ++i)
                                for (int j = 0; j < w; ++j) {
                                    const int ii = i + ky - 1, jj = j + kx - 1;
                                    if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                                    ga[ci * npix + (long)ii * w + jj] += wv * gz[co * npix + (long)i * w + j];
                                }
                        }
            if (l == 0) {
                if (dx) memcpy(dx + (long)im * ci_n * npix, ga, sizeof(double) * ci_n * npix);
            } else {
                for (long q = 0; q < (long)ci_n * npix; ++q) gz[q] = a[q] > 0.0 ? ga[q] : 0.0;
            }
        }
    }
    free(gz);
    free(ga);
    free(th);
}

void or_adamw(double* theta, const double* g, double* m, double* v, int step, double lr, double beta1,
              double beta2, double eps, double wd)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (int l = 0; l < OR_NET_LAYERS; ++l) {
        const long w0 = or_net_offset(l, 0), b0 = or_net_offset(l, 1), e = or_net_offset(l + 1, 0);
        for (long q = w0; q < e; ++q) {
            m[q] = beta1 * m[q] + (1.0 - beta1) * g[q];
            v[q] = beta2 * v[q] + (1.0 - beta2) * g[q] * g[q];
            const double upd = (m[q] / c1) / (sqrt(v[q] / c2) + eps);
            theta[q] -= lr * (upd + (q < b0 ? wd * theta[q] : 0.0));
        }
    }
}

/* The learned depth step of one PALM iteration (replaces or_apss). */
void or_learned_depth(int h, int w, int t, const or_params* p, or_state* s)
{
    const long npix = (long)h * w;
    double* x = (double*)malloc(sizeof(double) * 6 * npix);
    long na = 0;
    for (int l = 0; l < OR_NET_LAYERS; ++l) na += (long)cin_[l] * npix;
    double* acts = (double*)malloc(sizeof(double) * na);
    double* y = (double*)malloc(sizeof(double) * 2 * npix);
    or_net_features(h, w, s, p->net_scale, x);
    or_net_forward(1, h, w, p->net_theta, x, 1, acts, y);
    /* points the net does not take keep their APSS update (same Jacobi input) */
    or_state ap = *s;
    ap.t = (double*)malloc(sizeof(double) * s->k * npix);
    memcpy(ap.t, s->t, sizeof(double) * s->k * npix);
    or_apss(h, w, t, p, &ap);
    for (int k = 0; k < s->k; ++k)
        for (long q = 0; q < npix; ++q) {
            const long n = k * npix + q;
            if (!s->alive[n]) continue;
            double tn = ap.t[n];
            if (k < 2) {
                const double dt = y[k * npix + q] * p->net_scale;
                if (fabsf((float)dt) <= (float)p->net_fallback) {
                    tn = s->t[n] + dt;
                    if (tn < 0.0) tn = 0.0;
                    if (tn > t - 1) tn = t - 1;
                }
            }
            s->t[n] = tn;
        }
    free(ap.t);
    free(x);
    free(acts);
    free(y);
}
