/*
 * cnn_oracle.c -- FP64 CPU oracle of the learned candidate proposal network.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  Shares
 * no code with the CUDA path.  Plain direct loops in the definitions' order:
 *   conv 3x3 / stride 2 / pad 1 (+ bias, ReLU), NHWC, weights W[co][ky][kx][ci];
 *   fully connected y = W x + b; softmax cross-entropy (mean over the batch);
 *   backward by the chain rule; Adam (Kingma and Ba, 2015).
 * Flat parameter layout: per conv layer W then b; FC1 W[1024][1536], b;
 * FC2 W[64][1024], b.  Input [B][47][176][2].
 *
 * act_bf16 != 0: every stored activation (each convolution's and FC1's
 * output after the ReLU) is rounded to BF16 (round to nearest even of the
 * FP32 value), the storage format of the method's BF16 network; the
 * backward pass is the chain rule at those stored values (the rounding
 * passes gradients through unchanged), everything else stays FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NL 5
static const int CIN[NL] = {2, 32, 64, 64, 128}, COUT[NL] = {32, 64, 64, 128, 128};
#define IH 47
#define IW 176
#define F1I 1536
#define F1O 1024
#define F2O 64

/* BF16 round to nearest even of the FP32 value of x (the standard bit
 * construction: add 0x7FFF plus the lowest kept bit, truncate 16 bits). */
double orc_bf16_round(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) {
        u += 0x7FFFu + ((u >> 16) & 1u);
        u &= 0xFFFF0000u;
        memcpy(&f, &u, 4);
    }
    return (double)f;
}

typedef struct { int H, W, Ho, Wo; } dims;
static void layer_dims(dims *d)
{
    int H = IH, W = IW;
    for (int l = 0; l < NL; ++l) { d[l].H = H; d[l].W = W; d[l].Ho = (H - 1) / 2 + 1; d[l].Wo = (W - 1) / 2 + 1; H = d[l].Ho; W = d[l].Wo; }
}

int64_t orc_param_count(void)
{
    int64_t n = 0;
    for (int l = 0; l < NL; ++l) n += (int64_t)COUT[l] * 9 * CIN[l] + COUT[l];
    return n + (int64_t)F1O * F1I + F1O + (int64_t)F2O * F1O + F2O;
}

/* offsets of W and b of layer t (0..4 conv, 5 fc1, 6 fc2) in the flat vector */
static void offsets(int64_t *wo, int64_t *bo)
{
    int64_t o = 0;
    for (int l = 0; l < NL; ++l) { wo[l] = o; o += (int64_t)COUT[l] * 9 * CIN[l]; bo[l] = o; o += COUT[l]; }
    wo[5] = o; o += (int64_t)F1O * F1I; bo[5] = o; o += F1O;
    wo[6] = o; o += (int64_t)F2O * F1O; bo[6] = o;
}

static void conv_fwd(const double *x, int H, int W, int Ci, const double *w, const double *b, int Co, int Ho, int Wo, double *y)
{
    for (int oy = 0; oy < Ho; ++oy)
        for (int ox = 0; ox < Wo; ++ox)
            for (int co = 0; co < Co; ++co) {
                double s = b[co];
                for (int ky = 0; ky < 3; ++ky) {
                    int yy = 2 * oy - 1 + ky;
                    if (yy < 0 || yy >= H) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        int xx = 2 * ox - 1 + kx;
                        if (xx < 0 || xx >= W) continue;
                        const double *xi = x + ((int64_t)yy * W + xx) * Ci;
                        const double *wi = w + (((int64_t)co * 3 + ky) * 3 + kx) * Ci;
                        for (int ci = 0; ci < Ci; ++ci) s += wi[ci] * xi[ci];
                    }
                }
                y[((int64_t)oy * Wo + ox) * Co + co] = s > 0 ? s : 0;   /* ReLU */
            }
}

/* One 3x3 / stride 2 / pad 1 convolution + bias + ReLU of one NHWC image
 * (exported for the pins). */
void orc_conv3x3s2(const double *x, int H, int W, int Ci, const double *w, const double *b, int Co, double *y)
{
    conv_fwd(x, H, W, Ci, w, b, Co, (H - 1) / 2 + 1, (W - 1) / 2 + 1, y);
}

/* activations of one sample: a[0] = input, a[l+1] = conv l output, h1, logits */
typedef struct { double *a[NL + 1]; double *h1, *z; } acts;

static void round_all(double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) a[i] = orc_bf16_round(a[i]);
}

static void fwd_one(const double *p, const double *in, acts *A, int act_bf16)
{
    dims d[NL];
    int64_t wo[7], bo[7];
    layer_dims(d);
    offsets(wo, bo);
    memcpy(A->a[0], in, sizeof(double) * IH * IW * 2);
    for (int l = 0; l < NL; ++l) {
        conv_fwd(A->a[l], d[l].H, d[l].W, CIN[l], p + wo[l], p + bo[l], COUT[l], d[l].Ho, d[l].Wo, A->a[l + 1]);
        if (act_bf16) round_all(A->a[l + 1], (int64_t)d[l].Ho * d[l].Wo * COUT[l]);
    }
    const double *x5 = A->a[NL];
    for (int n = 0; n < F1O; ++n) {
        double s = p[bo[5] + n];
        for (int k = 0; k < F1I; ++k) s += p[wo[5] + (int64_t)n * F1I + k] * x5[k];
        A->h1[n] = s > 0 ? s : 0;
    }
    if (act_bf16) round_all(A->h1, F1O);
    for (int n = 0; n < F2O; ++n) {
        double s = p[bo[6] + n];
        for (int k = 0; k < F1O; ++k) s += p[wo[6] + (int64_t)n * F1O + k] * A->h1[k];
        A->z[n] = s;
    }
}

static acts alloc_acts(void)
{
    dims d[NL];
    layer_dims(d);
    acts A;
    A.a[0] = (double *)malloc(sizeof(double) * IH * IW * 2);
    for (int l = 0; l < NL; ++l) A.a[l + 1] = (double *)malloc(sizeof(double) * d[l].Ho * d[l].Wo * COUT[l]);
    A.h1 = (double *)malloc(sizeof(double) * F1O);
    A.z = (double *)malloc(sizeof(double) * F2O);
    return A;
}
static void free_acts(acts *A) { for (int l = 0; l <= NL; ++l) free(A->a[l]); free(A->h1); free(A->z); }

/* logits [B][64] */
void orc_forward_ex(const double *p, const double *in, int B, double *logits, int act_bf16)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        acts A = alloc_acts();
        fwd_one(p, in + (int64_t)b * IH * IW * 2, &A, act_bf16);
        memcpy(logits + (int64_t)b * F2O, A.z, sizeof(double) * F2O);
        free_acts(&A);
    }
}

void orc_forward(const double *p, const double *in, int B, double *logits)
{
    orc_forward_ex(p, in, B, logits, 0);
}

/* Mean softmax cross-entropy over the batch and its gradient w.r.t. every
 * parameter (grad, flat layout) and, optionally, the input (grad_in). */
double orc_loss_grad_ex(const double *p, const double *in, const int32_t *labels, int B, double *grad, double *grad_in,
                        int act_bf16)
{
    const int64_t np = orc_param_count();
    dims d[NL];
    int64_t wo[7], bo[7];
    layer_dims(d);
    offsets(wo, bo);
    memset(grad, 0, sizeof(double) * np);
    double loss = 0;
    for (int b = 0; b < B; ++b) {
        acts A = alloc_acts();
        fwd_one(p, in + (int64_t)b * IH * IW * 2, &A, act_bf16);
        /* softmax cross-entropy */
        double mx = A.z[0];
        for (int c = 1; c < F2O; ++c) if (A.z[c] > mx) mx = A.z[c];
        double se = 0;
        for (int c = 0; c < F2O; ++c) se += exp(A.z[c] - mx);
        loss += (log(se) + mx - A.z[labels[b]]) / B;
        double dz[F2O];
        for (int c = 0; c < F2O; ++c) dz[c] = (exp(A.z[c] - mx) / se - (c == labels[b])) / B;
        /* FC2 */
        double *dh = (double *)calloc(F1O, sizeof(double));
        for (int n = 0; n < F2O; ++n) {
            grad[bo[6] + n] += dz[n];
            for (int k = 0; k < F1O; ++k) {
                grad[wo[6] + (int64_t)n * F1O + k] += dz[n] * A.h1[k];
                dh[k] += dz[n] * p[wo[6] + (int64_t)n * F1O + k];
            }
        }
        for (int k = 0; k < F1O; ++k) if (!(A.h1[k] > 0)) dh[k] = 0;     /* ReLU */
        /* FC1 */
        double *dx = (double *)calloc(F1I, sizeof(double));
        for (int n = 0; n < F1O; ++n) {
            grad[bo[5] + n] += dh[n];
            for (int k = 0; k < F1I; ++k) {
                grad[wo[5] + (int64_t)n * F1I + k] += dh[n] * A.a[NL][k];
                dx[k] += dh[n] * p[wo[5] + (int64_t)n * F1I + k];
            }
        }
        free(dh);
        /* conv layers: dx is dL/d(output of layer l) */
        for (int l = NL - 1; l >= 0; --l) {
            const int Ho = d[l].Ho, Wo = d[l].Wo, H = d[l].H, W = d[l].W, Ci = CIN[l], Co = COUT[l];
            const double *x = A.a[l], *y = A.a[l + 1];
            double *dxi = (double *)calloc((size_t)H * W * Ci, sizeof(double));
            for (int oy = 0; oy < Ho; ++oy)
                for (int ox = 0; ox < Wo; ++ox)
                    for (int co = 0; co < Co; ++co) {
                        const int64_t o = ((int64_t)oy * Wo + ox) * Co + co;
                        if (!(y[o] > 0)) continue;                          /* ReLU */
                        const double g = dx[o];
                        grad[bo[l] + co] += g;
                        for (int ky = 0; ky < 3; ++ky) {
                            int yy = 2 * oy - 1 + ky;
                            if (yy < 0 || yy >= H) continue;
                            for (int kx = 0; kx < 3; ++kx) {
                                int xx = 2 * ox - 1 + kx;
                                if (xx < 0 || xx >= W) continue;
                                const int64_t wi = wo[l] + (((int64_t)co * 3 + ky) * 3 + kx) * Ci;
                                const int64_t xi = ((int64_t)yy * W + xx) * Ci;
                                for (int ci = 0; ci < Ci; ++ci) {
                                    grad[wi + ci] += g * x[xi + ci];
                                    dxi[xi + ci] += g * p[wi + ci];
                                }
                            }
                        }
                    }
            free(dx);
            dx = dxi;
        }
        if (grad_in) memcpy(grad_in + (int64_t)b * IH * IW * 2, dx, sizeof(double) * IH * IW * 2);
        free(dx);
        free_acts(&A);
    }
    return loss;
}

double orc_loss_grad(const double *p, const double *in, const int32_t *labels, int B, double *grad, double *grad_in)
{
    return orc_loss_grad_ex(p, in, labels, B, grad, grad_in, 0);
}

/* One Adam step (t = step number, 1-based) on n parameters. */
void orc_adam(double *w, double *m, double *v, const double *g, int64_t n, double lr, double b1, double b2,
              double eps, int t)
{
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1 - b1) * g[i];
        v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
        const double mh = m[i] / (1 - pow(b1, t)), vh = v[i] / (1 - pow(b2, t));
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Gray (mean of R, G, B) box average over f x f pixels of a planar [3][H][W]
 * image: out [H/f][W/f]. */
void orc_downsample_gray(const float *img, int H, int W, int f, double *out)
{
    const int Ho = H / f, Wo = W / f;
    const int64_t HW = (int64_t)H * W;
    for (int oy = 0; oy < Ho; ++oy)
        for (int ox = 0; ox < Wo; ++ox) {
            double s = 0;
            for (int y = oy * f; y < oy * f + f; ++y)
                for (int x = ox * f; x < ox * f + f; ++x) {
                    const int64_t q = (int64_t)y * W + x;
                    s += ((double)img[q] + img[HW + q] + img[2 * HW + q]) / 3.0;
                }
            out[(int64_t)oy * Wo + ox] = s / (f * f);
        }
}
