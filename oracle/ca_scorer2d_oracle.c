/*
 * ca_scorer2d_oracle.c -- TEST INFRASTRUCTURE ONLY (see ca_oracle.h).
 *
 * Plain restatement of the paper's own learned edge scorer (Sec. 2.2.4):
 * three 3x3 convolutions with 8, 16 and 32 output features, each followed by
 * a ReLU, then a 1x1 convolution to one feature and a sigmoid, giving an
 * edge probability per pixel.  The input has five features per pixel, RGB
 * and the pixel's coordinates (RGBXY), and the network runs on strips 7
 * rows high, the size of its receptive field, so that the three
 * convolutions, unpadded in the vertical direction, leave exactly the
 * strip's middle row (7 -> 5 -> 3 -> 1 rows).  Horizontally each
 * convolution is "same" with zero padding.  Training uses the soft binary
 * cross-entropy against an edge map blurred with a Gaussian of sigma 3
 * (here optionally weighted: column x counts 1 + (pos_weight - 1) t_x times,
 * pos_weight = 1 being the paper's unweighted loss).
 *
 * Two modes for the forward pass, as for the 1-D scorer:
 *   ORC_SC_EXACT  binary64 with no rounding (the exact network), whose
 *                 gradient the tests pin by finite differences;
 *   ORC_SC_MIXED  rounded where a tensor-core kernel stores a narrower
 *                 value: features, weights and activations in bfloat16, the
 *                 bias added in binary32, the head summed in binary32 in
 *                 channel order over bfloat16 head weights.  Each convolution
 *                 sum itself is taken in binary64 and rounded once to
 *                 binary32: a tensor core accumulates its products in its
 *                 own order and width, so this mode is the reference a
 *                 kernel meets within a tolerance, not its bit pattern.
 *
 * Readings where the paper is silent:
 *   - colour features are (v - 128) / 128 (the paper normalises by its
 *     dataset's mean and standard deviation, which do not exist here);
 *   - X = (x - (W - 1) / 2) / W and Y = (y - (H - 1) / 2) / H, in [-0.5, 0.5]
 *     with (0, 0) at the image centre, y the frame row of the pixel;
 *   - the 7 rows of a strip centred on row y are y - 3 .. y + 3, clamped into
 *     the frame (edge rows repeated);
 *   - the soft target of a pixel is exp(-d^2 / (2 sigma^2)), d its distance
 *     to the true circle (the blurred edge map scaled to 1 on the edge); 0
 *     when the frame has no circle.
 *
 * Convention: out[r][x] = sum_{dr, dx} W[dr][dx] in[r + dr][x + dx - 1],
 * dr, dx = 0..2, columns outside [0, W) zero.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ca_oracle.h"

#define CIN ORC_SC2_CIN
#define NL 3
static const int COUT[NL] = {8, 16, 32};
static const int CINL[NL] = {ORC_SC2_CIN, 8, 16};
static const int ROWS_IN[NL] = {7, 5, 3};

/* Offsets of W1[8][5][3][3], b1, W2[16][8][3][3], b2, W3[32][16][3][3], b3,
 * wh[32], bh in the flat parameter vector. */
void orc_sc2_offsets(int32_t out[8]) {
    int o = 0;
    for (int l = 0; l < NL; ++l) {
        out[2 * l] = o;
        o += COUT[l] * CINL[l] * 9;
        out[2 * l + 1] = o;
        o += COUT[l];
    }
    out[6] = o;
    out[7] = o + 32;
}

void orc_sc2_strip(const uint8_t *rgb, int H, int W, int64_t pitch, int y, uint8_t *rgb7,
                   int32_t rows[7]) {
    for (int k = 0; k < 7; ++k) {
        int r = y - 3 + k;
        if (r < 0) r = 0;
        if (r > H - 1) r = H - 1;
        rows[k] = r;
        memcpy(rgb7 + (size_t)k * W * 3, rgb + (int64_t)r * pitch, (size_t)W * 3);
    }
}

/* Features of the 7 x W pixels: feat[(k * W + x) * 5 + c]. */
void orc_sc2_features(const uint8_t *rgb7, const int32_t rows[7], int W, int H, double *feat) {
    for (int k = 0; k < 7; ++k)
        for (int x = 0; x < W; ++x) {
            const uint8_t *p = rgb7 + ((size_t)k * W + x) * 3;
            double *f = feat + ((size_t)k * W + x) * CIN;
            f[0] = (p[0] - 128) / 128.0;
            f[1] = (p[1] - 128) / 128.0;
            f[2] = (p[2] - 128) / 128.0;
            f[3] = ((double)x - 0.5 * (W - 1)) / W;
            f[4] = ((double)rows[k] - 0.5 * (H - 1)) / H;
        }
}

static float bf16_of(double v) { return orc_bf16((float)v); }

/* One 3x3 convolution + ReLU: in rows_in x W x cin -> (rows_in - 2) x W x cout;
 * pre (optional) receives the pre-activations; mixed: ORC_SC_MIXED roundings. */
static void conv3x3_mode(const double *in, int rows_in, int W, int cin, int cout, const float *w,
                         const float *b, int mixed, double *out, double *pre) {
    const int ro = rows_in - 2;
    for (int r = 0; r < ro; ++r)
        for (int x = 0; x < W; ++x)
            for (int co = 0; co < cout; ++co) {
                double s = 0.0;
                for (int ci = 0; ci < cin; ++ci)
                    for (int dr = 0; dr < 3; ++dr)
                        for (int dx = 0; dx < 3; ++dx) {
                            const int xx = x + dx - 1;
                            if (xx < 0 || xx >= W) continue;
                            const float wv = w[((co * cin + ci) * 3 + dr) * 3 + dx];
                            s += (mixed ? (double)orc_bf16(wv) : (double)wv) *
                                 in[((size_t)(r + dr) * W + xx) * cin + ci];
                        }
                const double z = mixed ? (double)((float)s + b[co]) : s + (double)b[co];
                if (pre) pre[((size_t)r * W + x) * cout + co] = z;
                const double a = z > 0.0 ? z : 0.0;
                out[((size_t)r * W + x) * cout + co] = mixed ? (double)bf16_of(a) : a;
            }
}

int orc_sc2_forward_mode(const uint8_t *rgb7, const int32_t rows[7], int W, int H,
                         const float *prm, int mode, double *logits) {
    if (W < 1 || !rgb7 || !prm || !logits || (mode != ORC_SC_EXACT && mode != ORC_SC_MIXED))
        return -1;
    const int mixed = mode == ORC_SC_MIXED;
    int32_t off[8];
    orc_sc2_offsets(off);
    double *a[NL + 1];
    a[0] = (double *)malloc(sizeof(double) * 7 * (size_t)W * CIN);
    for (int l = 0; l < NL; ++l)
        a[l + 1] = (double *)malloc(sizeof(double) * (size_t)(ROWS_IN[l] - 2) * W * COUT[l]);
    orc_sc2_features(rgb7, rows, W, H, a[0]);
    if (mixed)   /* the kernel's features: X and Y in binary32, then bfloat16 */
        for (int k = 0; k < 7; ++k)
            for (int x = 0; x < W; ++x) {
                double *f = a[0] + ((size_t)k * W + x) * CIN;
                const float xf = ((float)x - 0.5f * (float)(W - 1)) / (float)W;
                const float yf = ((float)rows[k] - 0.5f * (float)(H - 1)) / (float)H;
                f[3] = orc_bf16(xf);
                f[4] = orc_bf16(yf);
            }
    for (int l = 0; l < NL; ++l)
        conv3x3_mode(a[l], ROWS_IN[l], W, CINL[l], COUT[l], prm + off[2 * l],
                     prm + off[2 * l + 1], mixed, a[l + 1], NULL);
    for (int x = 0; x < W; ++x) {
        if (mixed) {
            float acc = 0.0f;
            for (int c = 0; c < 32; ++c)
                acc = acc + orc_bf16(prm[off[6] + c]) * (float)a[NL][(size_t)x * 32 + c];
            logits[x] = (double)(prm[off[7]] + acc);
        } else {
            double z = prm[off[7]];
            for (int c = 0; c < 32; ++c) z += (double)prm[off[6] + c] * a[NL][(size_t)x * 32 + c];
            logits[x] = z;
        }
    }
    for (int l = 0; l <= NL; ++l) free(a[l]);
    return 0;
}

int orc_sc2_forward(const uint8_t *rgb7, const int32_t rows[7], int W, int H, const float *prm,
                    double *logits) {
    return orc_sc2_forward_mode(rgb7, rows, W, H, prm, ORC_SC_EXACT, logits);
}

/* Soft binary cross-entropy of the W columns against targets t in [0, 1],
 * column x weighted by w_x = 1 + (pos_weight - 1) t_x, summed, and its
 * gradient added into grads (ORC_SC2_NPARAM doubles). */
double orc_sc2_loss_grad(const uint8_t *rgb7, const int32_t rows[7], int W, int H,
                         const double *targets, double pos_weight, const float *prm,
                         double *grads) {
    int32_t off[8];
    orc_sc2_offsets(off);
    double *a[NL + 1], *pre[NL];
    a[0] = (double *)malloc(sizeof(double) * 7 * (size_t)W * CIN);
    for (int l = 0; l < NL; ++l) {
        const size_t n = (size_t)(ROWS_IN[l] - 2) * W * COUT[l];
        a[l + 1] = (double *)malloc(sizeof(double) * n);
        pre[l] = (double *)malloc(sizeof(double) * n);
    }
    orc_sc2_features(rgb7, rows, W, H, a[0]);
    for (int l = 0; l < NL; ++l)
        conv3x3_mode(a[l], ROWS_IN[l], W, CINL[l], COUT[l], prm + off[2 * l],
                     prm + off[2 * l + 1], 0, a[l + 1], pre[l]);
    /* head, loss and dL/da3 */
    double loss = 0.0;
    double *g = (double *)calloc((size_t)W * 32, sizeof(double));   /* dL/d(layer output) */
    for (int x = 0; x < W; ++x) {
        double z = prm[off[7]];
        for (int c = 0; c < 32; ++c) z += (double)prm[off[6] + c] * a[NL][(size_t)x * 32 + c];
        const double t = targets[x];
        const double w = 1.0 + (pos_weight - 1.0) * t;
        /* -t log p - (1 - t) log(1 - p) = softplus(z) - t z, stably */
        const double sp = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
        loss += w * (sp - t * z);
        const double p = 1.0 / (1.0 + exp(-z));
        const double dz = w * (p - t);
        grads[off[7]] += dz;
        for (int c = 0; c < 32; ++c) {
            grads[off[6] + c] += dz * a[NL][(size_t)x * 32 + c];
            g[(size_t)x * 32 + c] = dz * prm[off[6] + c];
        }
    }
    /* layers 3, 2, 1: through the ReLU, weight / bias gradients, input gradient */
    for (int l = NL - 1; l >= 0; --l) {
        const int ro = ROWS_IN[l] - 2, cin = CINL[l], cout = COUT[l];
        const float *w = prm + off[2 * l];
        double *gw = grads + off[2 * l], *gb = grads + off[2 * l + 1];
        double *gin = l > 0 ? (double *)calloc((size_t)ROWS_IN[l] * W * cin, sizeof(double)) : NULL;
        for (int r = 0; r < ro; ++r)
            for (int x = 0; x < W; ++x)
                for (int co = 0; co < cout; ++co) {
                    const size_t i = ((size_t)r * W + x) * cout + co;
                    const double dz = pre[l][i] > 0.0 ? g[i] : 0.0;
                    if (dz == 0.0) continue;
                    gb[co] += dz;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dr = 0; dr < 3; ++dr)
                            for (int dx = 0; dx < 3; ++dx) {
                                const int xx = x + dx - 1;
                                if (xx < 0 || xx >= W) continue;
                                const size_t j = ((size_t)(r + dr) * W + xx) * cin + ci;
                                const int wi = ((co * cin + ci) * 3 + dr) * 3 + dx;
                                gw[wi] += dz * a[l][j];
                                if (gin) gin[j] += dz * (double)w[wi];
                            }
                }
        free(g);
        g = gin;
    }
    for (int l = 0; l <= NL; ++l) free(a[l]);
    for (int l = 0; l < NL; ++l) free(pre[l]);
    return loss;
}

void orc_sc2_targets(float cx, float cy, float r, int valid, int W, int y, double sigma,
                     double *t) {
    for (int x = 0; x < W; ++x) {
        if (!valid) {
            t[x] = 0.0;
            continue;
        }
        const double d = fabs(hypot((double)x - cx, (double)y - cy) - r);
        t[x] = exp(-d * d / (2.0 * sigma * sigma));
    }
}
