/*
 * ca_scorer_oracle.c -- TEST INFRASTRUCTURE ONLY (see ca_oracle.h).
 *
 * Plain restatement of the learned edge scorer: per strip column a feature
 * vector, three 1-D convolutions (kernel 7, 32 channels, "same" zero padding,
 * ReLU), a 1x1 head and a sigmoid giving the edge probability of each column
 * (the learned variant of Sec. 2.2.4, here over 1-D strip profiles), and the
 * weighted binary cross-entropy used to train it (Sec. 2.2.4 trains with a
 * cross-entropy against edge labels), with its gradient by the chain rule.
 *
 * Two modes:
 *   ORC_SC_EXACT  every quantity in binary64, no rounding: the plain network,
 *                 whose gradient the tests pin by finite differences;
 *   ORC_SC_MIXED  the same sums in binary64, rounded at the points where the
 *                 CUDA kernels store a narrower value: features, weights and
 *                 activations in bfloat16, convolution sums in binary32.
 * Convention: out[x] = sum_t W[t] in[x + t - 3], t = 0..6, inputs outside
 * [0, W) are zero.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ca_oracle.h"

#define CIN ORC_SC_CIN
#define CH ORC_SC_CH
#define KW ORC_SC_K
#define HALF (ORC_SC_K / 2)

/* bfloat16 round-to-nearest-even of a binary32 value (NaN not expected) */
static float to_bf16(float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

float orc_bf16(float v) { return to_bf16(v); }

static double rnd_bf16(double v, int mixed) { return mixed ? (double)to_bf16((float)v) : v; }
static double rnd_f32(double v, int mixed) { return mixed ? (double)(float)v : v; }

/* Parameter offsets in the flat vector (W1[co][ci][t], b1, W2, b2, W3, b3, wh, bh). */
static const int OFF_W[3] = {0, CH * CIN * KW + CH, CH * CIN * KW + CH + CH * CH * KW + CH};
static const int OFF_B[3] = {CH * CIN * KW, CH * CIN * KW + CH + CH * CH * KW,
                             CH * CIN * KW + 2 * CH + 2 * CH * CH * KW};
#define OFF_WH (CH * CIN * KW + 3 * CH + 2 * CH * CH * KW)
#define OFF_BH (OFF_WH + CH)

void orc_sc_offsets(int32_t out[8]) {
    out[0] = OFF_W[0]; out[1] = OFF_B[0]; out[2] = OFF_W[1]; out[3] = OFF_B[1];
    out[4] = OFF_W[2]; out[5] = OFF_B[2]; out[6] = OFF_WH; out[7] = OFF_BH;
}

/* Features of column x: for rows y-1, y, y+1 the luma and R, G, B, each
 * (v - 128) / 128, then x and y centred and divided by W and H. */
void orc_sc_features(const uint8_t *rgb3, int W, int y, int H, int mixed, double *feat) {
    for (int x = 0; x < W; ++x) {
        double *f = feat + (size_t)x * CIN;
        for (int r = 0; r < 3; ++r) {
            const uint8_t *p = rgb3 + ((size_t)r * W + x) * 3;
            int luma = orc_luma(p[0], p[1], p[2]);
            f[4 * r + 0] = (luma - 128) / 128.0;
            f[4 * r + 1] = (p[0] - 128) / 128.0;
            f[4 * r + 2] = (p[1] - 128) / 128.0;
            f[4 * r + 3] = (p[2] - 128) / 128.0;
        }
        if (mixed) {
            float xf = ((float)x - 0.5f * (float)(W - 1)) / (float)W;
            float yf = ((float)y - 0.5f * (float)(H - 1)) / (float)H;
            f[12] = to_bf16(xf);
            f[13] = to_bf16(yf);
        } else {
            f[12] = ((double)x - 0.5 * (W - 1)) / W;
            f[13] = ((double)y - 0.5 * (H - 1)) / H;
        }
    }
}

/* One convolution layer: z[x][co] = b[co] + sum_{ci,t} w[co][ci][t] in[x+t-3][ci]. */
static void conv(const double *in, int cin, int W, const float *w, const float *b, int mixed,
                 double *z) {
    for (int x = 0; x < W; ++x)
        for (int co = 0; co < CH; ++co) {
            double s = 0.0;
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < KW; ++t) {
                    int xx = x + t - HALF;
                    if (xx < 0 || xx >= W) continue;
                    s += rnd_bf16(w[(co * cin + ci) * KW + t], mixed) * in[(size_t)xx * cin + ci];
                }
            z[(size_t)x * CH + co] = mixed ? (double)((float)s + b[co]) : s + (double)b[co];
        }
}

static double sigmoid(double l) { return 1.0 / (1.0 + exp(-l)); }

/* Forward pass of one strip.  acts (optional): 4 arrays in one block --
 * features (W x 14), a1, a2, a3 (W x 32 each, after ReLU). */
int orc_sc_forward(const uint8_t *rgb3, int W, int y, int H, const float *prm, int mode,
                   double *logits, double *acts) {
    if (W < 1 || (mode != ORC_SC_EXACT && mode != ORC_SC_MIXED)) return -1;
    const int mixed = mode == ORC_SC_MIXED;
    double *feat = (double *)malloc(sizeof(double) * (size_t)W * CIN);
    double *a[3], *z = (double *)malloc(sizeof(double) * (size_t)W * CH);
    for (int l = 0; l < 3; ++l) a[l] = (double *)malloc(sizeof(double) * (size_t)W * CH);
    orc_sc_features(rgb3, W, y, H, mixed, feat);
    const double *in = feat;
    int cin = CIN;
    for (int l = 0; l < 3; ++l) {
        conv(in, cin, W, prm + OFF_W[l], prm + OFF_B[l], mixed, z);
        for (size_t i = 0; i < (size_t)W * CH; ++i) a[l][i] = rnd_bf16(z[i] > 0.0 ? z[i] : 0.0, mixed);
        in = a[l];
        cin = CH;
    }
    /* head: logit = bh + sum_c wh[c] a3[c]; the kernels add the 32 products
     * in channel order in binary32, and so does the mixed mode */
    for (int x = 0; x < W; ++x) {
        if (mixed) {
            float acc = 0.0f;
            for (int c = 0; c < CH; ++c)
                acc = acc + to_bf16(prm[OFF_WH + c]) * (float)a[2][(size_t)x * CH + c];
            logits[x] = (double)(prm[OFF_BH] + acc);
        } else {
            double acc = 0.0;
            for (int c = 0; c < CH; ++c) acc += (double)prm[OFF_WH + c] * a[2][(size_t)x * CH + c];
            logits[x] = (double)prm[OFF_BH] + acc;
        }
    }
    if (acts) {
        memcpy(acts, feat, sizeof(double) * (size_t)W * CIN);
        for (int l = 0; l < 3; ++l)
            memcpy(acts + (size_t)W * CIN + (size_t)l * W * CH, a[l], sizeof(double) * (size_t)W * CH);
    }
    free(feat);
    free(z);
    for (int l = 0; l < 3; ++l) free(a[l]);
    return 0;
}

/* Loss of one strip, sum over its columns of w_x [log(1 + e^l) - y l] with
 * w_x = pos_weight on edge columns (label 1) and 1 elsewhere, and its
 * gradient (added into grads, 17601 values) by the chain rule. */
double orc_sc_loss_grad(const uint8_t *rgb3, int W, int y, int H, const uint8_t *labels,
                        float pos_weight, const float *prm, int mode, double *grads) {
    const int mixed = mode == ORC_SC_MIXED;
    const size_t n_act = (size_t)W * CIN + 3 * (size_t)W * CH;
    double *acts = (double *)malloc(sizeof(double) * n_act);
    double *logit = (double *)malloc(sizeof(double) * (size_t)W);
    if (orc_sc_forward(rgb3, W, y, H, prm, mode, logit, acts) != 0) {
        free(acts);
        free(logit);
        return NAN;
    }
    const double *a_in[3] = {acts, acts + (size_t)W * CIN, acts + (size_t)W * CIN + (size_t)W * CH};
    const double *a3 = acts + (size_t)W * CIN + 2 * (size_t)W * CH;
    const int cin_of[3] = {CIN, CH, CH};
    double loss = 0.0;
    double *dl = (double *)malloc(sizeof(double) * (size_t)W);
    for (int x = 0; x < W; ++x) {
        double l = logit[x], t = labels[x] ? 1.0 : 0.0, w = labels[x] ? pos_weight : 1.0;
        /* log(1 + e^l) - t l, written to stay finite for large |l| */
        double sp = l > 0 ? l + log1p(exp(-l)) : log1p(exp(l));
        loss += w * (sp - t * l);
        dl[x] = rnd_f32(w * (sigmoid(l) - t), mixed);
    }
    /* head */
    double *dz = (double *)malloc(sizeof(double) * (size_t)W * CH);
    double *da = (double *)malloc(sizeof(double) * (size_t)W * CH);
    double gbh = 0.0;
    for (int x = 0; x < W; ++x) gbh += dl[x];
    grads[OFF_BH] += rnd_f32(gbh, mixed);
    for (int c = 0; c < CH; ++c) {
        double g = 0.0;
        for (int x = 0; x < W; ++x) g += dl[x] * a3[(size_t)x * CH + c];
        grads[OFF_WH + c] += rnd_f32(g, mixed);
    }
    for (int x = 0; x < W; ++x)
        for (int c = 0; c < CH; ++c) {
            double wh = rnd_bf16(prm[OFF_WH + c], mixed);
            dz[(size_t)x * CH + c] = a3[(size_t)x * CH + c] > 0.0 ? rnd_bf16(dl[x] * wh, mixed) : 0.0;
        }
    /* layers 3, 2, 1: dz holds the gradient at the layer's pre-activation */
    for (int l = 2; l >= 0; --l) {
        const int cin = cin_of[l];
        const double *in = a_in[l];
        const float *w = prm + OFF_W[l];
        for (int co = 0; co < CH; ++co) {
            double gb = 0.0;
            for (int x = 0; x < W; ++x) gb += dz[(size_t)x * CH + co];
            grads[OFF_B[l] + co] += rnd_f32(gb, mixed);
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < KW; ++t) {
                    double g = 0.0;
                    for (int x = 0; x < W; ++x) {
                        int xx = x + t - HALF;
                        if (xx < 0 || xx >= W) continue;
                        g += dz[(size_t)x * CH + co] * in[(size_t)xx * cin + ci];
                    }
                    grads[OFF_W[l] + (co * cin + ci) * KW + t] += rnd_f32(g, mixed);
                }
        }
        if (l == 0) break;
        /* gradient at the layer's input a_{l}: da[xx][ci] = sum_{co,t} dz[x][co] w[co][ci][t],
         * xx = x + t - 3; then through the ReLU of that layer */
        for (int xx = 0; xx < W; ++xx)
            for (int ci = 0; ci < cin; ++ci) {
                double s = 0.0;
                for (int co = 0; co < CH; ++co)
                    for (int t = 0; t < KW; ++t) {
                        int x = xx - t + HALF;
                        if (x < 0 || x >= W) continue;
                        s += dz[(size_t)x * CH + co] * rnd_bf16(w[(co * cin + ci) * KW + t], mixed);
                    }
                da[(size_t)xx * cin + ci] = rnd_f32(s, mixed);
            }
        for (size_t i = 0; i < (size_t)W * CH; ++i)
            dz[i] = in[i] > 0.0 ? rnd_bf16(da[i], mixed) : 0.0;
    }
    free(acts);
    free(logit);
    free(dl);
    free(dz);
    free(da);
    return loss;
}
