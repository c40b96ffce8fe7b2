/*
 * ca_oracle.c -- TEST INFRASTRUCTURE ONLY (see ca_oracle.h).
 *
 * Plain single-threaded restatement of the method of Budd et al. (arXiv
 * 2210.14771), step by step in the paper's order:
 *   Sec. 2.2.2, Eq. 1      strip rows h_i
 *   Sec. 2.2.3, Eq. 2-3    handcrafted features and soft-threshold scores
 *   Sec. 2.2.5             best point per half-strip, t_px / t_ps filter,
 *                          RANSAC over triples, inliers within t_ri,
 *                          least-squares refits (Coope 1993), score = sum of
 *                          inlier scores, r/d filters, best circle, t_cs
 *   Sec. 1.1, Fig. 1       content area = disc intersected with the sensor
 *                          rectangle; no clear circle -> whole rectangle
 *                          (Sec. 2.2.1, Sec. 2.2.5)
 *
 * No blocking, fusion or reordering: every loop runs over every pixel,
 * point and hypothesis in index order.  Build with -ffp-contract=off.
 *
 * Readings of points the paper leaves open (luma, Sobel normalisation, the
 * score quantisation, candidate ranks, the Philox draw, the refit schedule,
 * the circle-score normaliser) are the ones this project documents beside
 * the C API; the comments below restate each where it is used.
 */
#include "ca_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

void orc_params_default(orc_params *p) {
    memset(p, 0, sizeof(*p));
    p->n_strips = 16;        /* Appendix A */
    p->cands_per_strip = 2;  /* one per half-strip, Sec. 2.2.5 */
    p->n_hyps = 1024;
    p->refine_iters = 3;     /* Sec. 2.2.5 */
    p->alpha = 8.0f;         /* Appendix A */
    p->t_g = 20.0f;
    p->t_theta_deg = 30.0f;
    p->t_iota = 25.0f;
    p->t_ps = 0.03f;
    p->t_cs = 0.06f;
    p->t_px = 3.0f;
    p->t_ri = 3.0f;
    p->r_min = 0.1f;
    p->r_max = 0.8f;
    p->d_max = 0.2f;
    p->sup_px = 8;
    p->hyp_mode = ORC_HYP_RANDOM;
    p->score_norm = ORC_NORM_CIRCLE;
    p->sobel_norm = 1;
    p->seed = 0;
}

/* ---------------------------------------------------------------- Eq. 1 -- */
/* h_i = H / (1 + exp(-(alpha/N) (i - (N-1)/2))), floored, clamped to the rows
 * that have a row above and below (the 3x3 Sobel support). */
int orc_strip_rows(int H, int N, float alpha, int32_t *rows) {
    if (H < 3 || N < 1) return -1;
    for (int i = 0; i < N; ++i) {
        double t = (double)alpha / (double)N;
        double u = (double)i - (double)(N - 1) / 2.0;
        double e = exp(-(t * u));
        double h = (double)H / (1.0 + e);
        long v = (long)floor(h);
        if (v < 1) v = 1;
        if (v > H - 2) v = H - 2;
        rows[i] = (int32_t)v;
    }
    return 0;
}

/* ---------------------------------------------------------------- Eq. 2 -- */
static uint16_t q15(double v) { /* v in [0,1] -> round(32768 v) */
    double x = floor(32768.0 * v + 0.5);
    if (x < 0) x = 0;
    if (x > 32768) x = 32768;
    return (uint16_t)x;
}

/* s_g = tanh(|g| / t_g) sampled at |g| = q/4 (quarter-level steps of the raw
 * Sobel magnitude, divided by sobel_norm);
 * s_theta = 1 - tanh(theta / t_theta), theta in degrees, sampled at the
 * centre of bin q of the signed squared cosine u = cos|cos| (bin width
 * 1/4096, q = floor(4096 (u + 1)));
 * s_iota = 1 - tanh(iota / t_iota) for every 8-bit iota. */
void orc_build_luts(const orc_params *p, uint16_t *lut_g, uint16_t *lut_t, uint16_t *lut_i) {
    for (int q = 0; q < ORC_LUT_G; ++q) {
        double arg = ((double)q * 0.25) / ((double)p->sobel_norm * (double)p->t_g);
        lut_g[q] = q15(tanh(arg));
    }
    for (int q = 0; q < ORC_LUT_T; ++q) {
        double u = ((double)q + 0.5) / 4096.0 - 1.0;
        if (u > 1.0) u = 1.0;
        double c = u < 0.0 ? -sqrt(-u) : sqrt(u);
        double deg = acos(c) * (180.0 / 3.14159265358979323846);
        lut_t[q] = q15(1.0 - tanh(deg / (double)p->t_theta_deg));
    }
    for (int v = 0; v < ORC_LUT_I; ++v)
        lut_i[v] = q15(1.0 - tanh((double)v / (double)p->t_iota));
}

/* Intensity on the paper's 0-255 scale: integer BT.601 luma. */
int orc_luma(int r, int g, int b) { return (77 * r + 150 * g + 29 * b + 128) >> 8; }

static int64_t isqrt64(int64_t n) { /* floor(sqrt(n)), exact */
    int64_t r = (int64_t)sqrt((double)n);
    while (r > 0 && r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

/* Eq. 2-3 in double straight from the definitions (no tables): used only to
 * bound the quantisation error of the table-driven score. */
double orc_score_exact(int gx, int gy, int cx2, int cy2, int iota, const orc_params *p) {
    double ng = (double)gx * gx + (double)gy * gy;
    double nc = (double)cx2 * cx2 + (double)cy2 * cy2;
    if (ng == 0.0 || nc == 0.0) return 0.0;
    double mag = sqrt(ng) / (double)p->sobel_norm;
    double cs = ((double)gx * cx2 + (double)gy * cy2) / (sqrt(ng) * sqrt(nc));
    if (cs > 1.0) cs = 1.0;
    if (cs < -1.0) cs = -1.0;
    double deg = acos(cs) * (180.0 / 3.14159265358979323846);
    double sg = tanh(mag / p->t_g);
    double st = 1.0 - tanh(deg / p->t_theta_deg);
    double si = 1.0 - tanh((double)iota / p->t_iota);
    return sg * st * si;
}

/* Sec. 2.2.3 for the strip centred on `row`: Sobel gradient g on the middle
 * row (y down, g pointing dark -> bright, zero on the first and last column),
 * angle to the vector c from the pixel towards the centre (c2x0 / 2, c2y0 / 2)
 * -- the image centre ((W-1)/2, (H-1)/2) unless a prior centre is given --
 * as the doubled integer vector (c2x0 - 2x, c2y0 - 2 row), preceding maximum
 * iota of the middle row scanned from the outer image edge (exclusive of the
 * pixel), and the quantised product score s_q in Q15. */
static void strip_scores(const uint8_t *rgb, int H, int W, int64_t pitch, int row,
                         const uint16_t *lut_g, const uint16_t *lut_t, const uint16_t *lut_i,
                         int c2x0, int c2y0,
                         uint16_t *s_out, int32_t *gx_out, int32_t *gy_out, uint8_t *iota_out) {
    int32_t *Y = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)W);
    uint8_t *iota = (uint8_t *)malloc((size_t)W);
    for (int k = 0; k < 3; ++k) {
        const uint8_t *src = rgb + (int64_t)(row - 1 + k) * pitch;
        for (int x = 0; x < W; ++x)
            Y[k * W + x] = orc_luma(src[3 * x], src[3 * x + 1], src[3 * x + 2]);
    }
    const int32_t *Yu = Y, *Ym = Y + W, *Yd = Y + 2 * W;

    /* preceding maximum: left half scans x = 0 .. hw-1, right half
     * scans x = W-1 .. hw, each from the outer edge inwards */
    int hw = W / 2;
    int run = 0;
    for (int x = 0; x < hw; ++x) {
        iota[x] = (uint8_t)run;
        if (Ym[x] > run) run = Ym[x];
    }
    run = 0;
    for (int x = W - 1; x >= hw; --x) {
        iota[x] = (uint8_t)run;
        if (Ym[x] > run) run = Ym[x];
    }

    for (int x = 0; x < W; ++x) {
        int gx = 0, gy = 0;
        if (x > 0 && x < W - 1) {
            gx = (Yu[x + 1] + 2 * Ym[x + 1] + Yd[x + 1]) - (Yu[x - 1] + 2 * Ym[x - 1] + Yd[x - 1]);
            gy = (Yd[x - 1] + 2 * Yd[x] + Yd[x + 1]) - (Yu[x - 1] + 2 * Yu[x] + Yu[x + 1]);
        }
        int cx2 = c2x0 - 2 * x, cy2 = c2y0 - 2 * row;
        int64_t ng = (int64_t)gx * gx + (int64_t)gy * gy;
        int64_t nc = (int64_t)cx2 * cx2 + (int64_t)cy2 * cy2;
        uint32_t s = 0;
        if (ng != 0 && nc != 0) {
            int64_t qg = isqrt64(16 * ng);
            if (qg > ORC_LUT_G - 1) qg = ORC_LUT_G - 1;
            /* angle bin: q = floor(4096 (u + 1)), u = dot |dot| / (ng nc) the
             * signed squared cosine, as an exact integer quotient */
            int64_t dot = (int64_t)gx * cx2 + (int64_t)gy * cy2;
            int64_t P = ng * nc;
            int64_t d2 = dot * (dot < 0 ? -dot : dot);
            int64_t qt = (4096 * (d2 + P)) / P;
            if (qt > ORC_LUT_T - 1) qt = ORC_LUT_T - 1;
            uint32_t gt = ((uint32_t)lut_g[qg] * lut_t[qt] + 16384u) >> 15;
            s = (gt * lut_i[iota[x]] + 16384u) >> 15;
        }
        s_out[x] = (uint16_t)s;
        if (gx_out) gx_out[x] = gx;
        if (gy_out) gy_out[x] = gy;
        if (iota_out) iota_out[x] = iota[x];
    }
    free(Y); free(iota);
}

int orc_strip_scores(const uint8_t *rgb, int H, int W, int64_t pitch, int row,
                     const orc_params *p, uint16_t *s_out, int32_t *gx_out,
                     int32_t *gy_out, uint8_t *iota_out) {
    if (row < 1 || row > H - 2 || W < 3) return -1;
    uint16_t *lut_g = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_G);
    uint16_t *lut_t = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_T);
    uint16_t *lut_i = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_I);
    orc_build_luts(p, lut_g, lut_t, lut_i);
    strip_scores(rgb, H, W, pitch, row, lut_g, lut_t, lut_i, W - 1, H - 1, s_out, gx_out, gy_out,
                 iota_out);
    free(lut_g); free(lut_t); free(lut_i);
    return 0;
}

/* ------------------------------------------------ Sec. 2.2.5, candidates -- */
/* For each strip and each half: K/2 successive picks of the highest score,
 * each excluding pixels within sup_px of an earlier pick of that half; equal
 * scores go to the outermost pixel.  Then the paper's filter: drop points
 * closer than t_px to the image edge or scoring below t_ps. */
/* Best K/2 points of one half-strip [x0, x1) by the key (score, outer rank),
 * each at least sup_px + 1 away from the earlier ones (Sec. 2.2.5: the best
 * pixel of each half; K/2 > 1 is this project's extension).  Appends the
 * kept ones (t_px / t_ps filter) to xs/ys/ss; returns the first pick's score
 * (or -1 if the half is empty). */
static int pick_half(const uint16_t *s, int x0, int x1, int half, int y, int H, int W,
                     const orc_params *p, int cap, int16_t *xs, int16_t *ys, uint16_t *ss,
                     int *m, int32_t *picks) {
    uint32_t T_ps = (uint32_t)ceil((double)p->t_ps * 32768.0);
    int T_px = (int)ceil((double)p->t_px);
    int np = 0, first = -1;
    for (int r = 0; r < p->cands_per_strip / 2; ++r) {
        int best = -1;
        uint32_t bestkey = 0;
        for (int x = x0; x < x1; ++x) {
            int sup = 0;
            for (int j = 0; j < np; ++j)
                if (abs(x - picks[j]) <= p->sup_px) sup = 1;
            if (sup) continue;
            uint32_t rank = half ? (uint32_t)x : (uint32_t)(0xFFFF - x);
            uint32_t key = ((uint32_t)s[x] << 16) | rank;
            if (best < 0 || key > bestkey) { best = x; bestkey = key; }
        }
        if (best < 0) break;
        if (r == 0) first = s[best];
        picks[np++] = best;
        int keep = s[best] >= T_ps && best >= T_px && best <= W - 1 - T_px &&
                   y >= T_px && y <= H - 1 - T_px;
        if (keep) {
            if (*m < cap) { xs[*m] = (int16_t)best; ys[*m] = (int16_t)y; ss[*m] = s[best]; }
            ++*m;
        }
    }
    return first;
}

static int candidates_impl(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                           const uint16_t *learned, int fallback, int c2x0, int c2y0, int cap,
                           int16_t *xs, int16_t *ys, uint16_t *ss, int32_t *M) {
    int N = p->n_strips, K = p->cands_per_strip;
    if (N < 1 || K < 2 || (K & 1)) return -1;
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * N);
    uint16_t *s = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)W);
    int32_t *picks = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    uint16_t *lut_g = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_G);
    uint16_t *lut_t = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_T);
    uint16_t *lut_i = (uint16_t *)malloc(sizeof(uint16_t) * ORC_LUT_I);
    orc_build_luts(p, lut_g, lut_t, lut_i);
    orc_strip_rows(H, N, p->alpha, rows);
    int hw = W / 2, m = 0;
    for (int i = 0; i < N; ++i) {
        int y = rows[i];
        strip_scores(rgb, H, W, pitch, y, lut_g, lut_t, lut_i, c2x0, c2y0, s, NULL, NULL, NULL);
        for (int half = 0; half < 2; ++half) {
            int x0 = half ? hw : 0, x1 = half ? W : hw;
            if (learned) {
                /* learned scores; with the fallback, a half whose best
                 * learned score is below one half (16384 in Q15) takes the
                 * handcrafted points instead */
                int m0 = m;
                int first = pick_half(learned + (size_t)i * W, x0, x1, half, y, H, W, p, cap,
                                      xs, ys, ss, &m, picks);
                if (!fallback || first >= 16384) continue;
                m = m0;
            }
            pick_half(s, x0, x1, half, y, H, W, p, cap, xs, ys, ss, &m, picks);
        }
    }
    *M = m;
    free(rows); free(s); free(picks); free(lut_g); free(lut_t); free(lut_i);
    return 0;
}

int orc_candidates(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                   int cap, int16_t *xs, int16_t *ys, uint16_t *ss, int32_t *M) {
    return candidates_impl(rgb, H, W, pitch, p, NULL, 0, W - 1, H - 1, cap, xs, ys, ss, M);
}

/* Doubled centre (C2x, C2y) of the angle term for a prior circle centre
 * (cx, cy) in frame pixels: 2 cx and 2 cy (exact in binary32) rounded to the
 * nearest integer, ties to even, then clamped into [0, 2(W-1)] x [0, 2(H-1)]
 * (half-pixel resolution, inside the frame). */
void orc_prior_centre2(float cx, float cy, int H, int W, int32_t out[2]) {
    long vx = lrintf(2.0f * cx), vy = lrintf(2.0f * cy);
    if (vx < 0) vx = 0;
    if (vx > 2L * (W - 1)) vx = 2L * (W - 1);
    if (vy < 0) vy = 0;
    if (vy > 2L * (H - 1)) vy = 2L * (H - 1);
    out[0] = (int32_t)vx;
    out[1] = (int32_t)vy;
}

int orc_candidates_centre(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                          int32_t c2x0, int32_t c2y0, int cap, int16_t *xs, int16_t *ys,
                          uint16_t *ss, int32_t *M) {
    if (c2x0 < 0 || c2x0 > 2 * (W - 1) || c2y0 < 0 || c2y0 > 2 * (H - 1)) return -1;
    return candidates_impl(rgb, H, W, pitch, p, NULL, 0, c2x0, c2y0, cap, xs, ys, ss, M);
}

int orc_learned_candidates(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                           const uint16_t *learned, int fallback, int cap, int16_t *xs,
                           int16_t *ys, uint16_t *ss, int32_t *M) {
    if (!learned) return -1;
    return candidates_impl(rgb, H, W, pitch, p, learned, fallback, W - 1, H - 1, cap, xs, ys, ss,
                           M);
}

/* ------------------------------------------------------- Philox4x32-10 -- */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11: ten rounds of two 32x32->64 multiplies with the Weyl key schedule. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t mulhi_n(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

/* Uniform random triple (Sec. 2.2.5): counter (h, frame_key lo, hi, 0),
 * key = seed; three draws mapped to distinct indices by skipping the ones
 * already taken. */
void orc_triple(uint64_t seed, uint64_t frame_key, uint32_t h, int M, int32_t out[3]) {
    uint32_t ctr[4] = {h, (uint32_t)frame_key, (uint32_t)(frame_key >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4];
    orc_philox4x32_10(ctr, key, u);
    uint32_t i0 = mulhi_n(u[0], (uint32_t)M);
    uint32_t i1 = mulhi_n(u[1], (uint32_t)(M - 1));
    if (i1 >= i0) ++i1;
    uint32_t i2 = mulhi_n(u[2], (uint32_t)(M - 2));
    uint32_t a = i0 < i1 ? i0 : i1, b = i0 < i1 ? i1 : i0;
    if (i2 >= a) ++i2;
    if (i2 >= b) ++i2;
    out[0] = (int32_t)i0; out[1] = (int32_t)i1; out[2] = (int32_t)i2;
}

void orc_triple_exhaustive(int64_t h, int M, int32_t out[3]) {
    int64_t c = 0;
    for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j)
            for (int k = j + 1; k < M; ++k) {
                if (c == h) { out[0] = i; out[1] = j; out[2] = k; return; }
                ++c;
            }
    out[0] = out[1] = out[2] = -1;
}

/* --------------------------------------------------------- circle maths -- */
float orc_i128_to_f32(int64_t hi, uint64_t lo) {
    i128 v = (i128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
    return (float)v; /* correctly rounded (IEEE round-to-nearest-even) */
}

/* The binary32 value nearest to num / den (den != 0; ties to even; +0 for
 * num = 0), by integer steps: the quotient scaled by a power of two to 25 or
 * 26 significant bits, then rounded on the bits below 24 and the remainder.
 * Needs |num|, |den| < 2^38 (so that the scaled operand fits in 64 bits). */
float orc_rn_ratio(int64_t num, int64_t den) {
    if (num == 0) return 0.0f;
    const int neg = (num < 0) != (den < 0);
    const uint64_t a = num < 0 ? (uint64_t)0 - (uint64_t)num : (uint64_t)num;
    const uint64_t b = den < 0 ? (uint64_t)0 - (uint64_t)den : (uint64_t)den;
    int la = 63, lb = 63;
    while (!((a >> la) & 1u)) --la;
    while (!((b >> lb) & 1u)) --lb;
    const int s = 25 - (la - lb);   /* a 2^s / b lies in [2^24, 2^26) */
    uint64_t q, r;
    if (s >= 0) {
        q = (a << s) / b;
        r = (a << s) % b;
    } else {
        q = a / (b << -s);
        r = a % (b << -s);
    }
    int e = -s;                     /* num / den = (q + remainder) 2^e */
    int sticky = r != 0;
    if (q >= (1ull << 25)) {        /* keep 25 bits: 24 of mantissa and a round bit */
        sticky |= (int)(q & 1u);
        q >>= 1;
        e += 1;
    }
    uint64_t m = q >> 1;
    const int round_bit = (int)(q & 1u);
    if (round_bit && (sticky || (m & 1u))) m += 1;   /* may reach 2^24: still exact */
    const float v = ldexpf((float)m, e + 1);
    return neg ? -v : v;
}

/* Circle through a, b, c (Sec. 2.2.5, "analytically"): the circumcentre is
 * (Ux/D, Uy/D) with exact integer D, Ux, Uy, each coordinate the binary32
 * value nearest to that ratio; the radius is the binary32 distance to a. */
int orc_circumcircle(int ax, int ay, int bx, int by, int cx, int cy, float out[3]) {
    int64_t D = 2 * ((int64_t)ax * (by - cy) + (int64_t)bx * (cy - ay) + (int64_t)cx * (ay - by));
    if (D == 0) return 0;
    int64_t a2 = (int64_t)ax * ax + (int64_t)ay * ay;
    int64_t b2 = (int64_t)bx * bx + (int64_t)by * by;
    int64_t c2 = (int64_t)cx * cx + (int64_t)cy * cy;
    int64_t Ux = a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by);
    int64_t Uy = a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax);
    const float ox = orc_rn_ratio(Ux, D), oy = orc_rn_ratio(Uy, D);
    float dx = (float)ax - ox, dy = (float)ay - oy;
    out[0] = ox; out[1] = oy; out[2] = sqrtf(dx * dx + dy * dy);
    return 1;
}

/* Algebraic least-squares circle (Coope 1993; Kasa form): minimise
 * sum (x^2 + y^2 + D x + E y + F)^2.  In coordinates centred on the mean the
 * centre offset (a, b) solves
 *     [Suu Suv; Suv Svv] [a; b] = 1/2 [Suuu + Suvv; Svvv + Suuv]
 * and r^2 = a^2 + b^2 + (Suu + Svv)/n.  Every sum is formed exactly from
 * integer moments, scaled by powers of n; only the final quotients are
 * rounded to binary32. */
int orc_ls_fit(const int32_t *X, const int32_t *Y, int n, float out[3]) {
    if (n < 3) return 0;
    i128 Sx = 0, Sy = 0, Sxx = 0, Sxy = 0, Syy = 0, Sxxx = 0, Sxxy = 0, Sxyy = 0, Syyy = 0;
    for (int j = 0; j < n; ++j) {
        i128 x = X[j], y = Y[j];
        Sx += x; Sy += y;
        Sxx += x * x; Sxy += x * y; Syy += y * y;
        Sxxx += x * x * x; Sxxy += x * x * y; Sxyy += x * y * y; Syyy += y * y * y;
    }
    i128 N = n;
    i128 A = N * Sxx - Sx * Sx;          /* n   * Suu */
    i128 B = N * Sxy - Sx * Sy;          /* n   * Suv */
    i128 C = N * Syy - Sy * Sy;          /* n   * Svv */
    i128 P = N * N * Sxxx - 3 * N * Sx * Sxx + 2 * Sx * Sx * Sx     /* n^2 (Suuu + Suvv) */
           + N * N * Sxyy - 2 * N * Sy * Sxy - N * Sx * Syy + 2 * Sx * Sy * Sy;
    i128 Q = N * N * Syyy - 3 * N * Sy * Syy + 2 * Sy * Sy * Sy     /* n^2 (Svvv + Suuv) */
           + N * N * Sxxy - 2 * N * Sx * Sxy - N * Sy * Sxx + 2 * Sy * Sx * Sx;
    i128 det = A * C - B * B;
    if (det == 0) return 0;
    i128 a_num = C * P - B * Q;          /* a = a_num / den */
    i128 b_num = A * Q - B * P;
    i128 den = 2 * N * det;
    i128 cx_num = 2 * det * Sx + a_num;  /* cx = Sx/n + a */
    i128 cy_num = 2 * det * Sy + b_num;
    float fden = (float)den;
    float ocx = (float)cx_num / fden;
    float ocy = (float)cy_num / fden;
    float af = (float)a_num / fden;
    float bf = (float)b_num / fden;
    float t1 = (float)(A + C) / (float)(N * N);
    float r2 = (t1 + af * af) + bf * bf;
    out[0] = ocx; out[1] = ocy; out[2] = sqrtf(r2);
    return 1;
}

/* Inliers of a circle: points within t_ri of it, taken as
 * max(r - t_ri, 0)^2 <= |p - c|^2 <= (r + t_ri)^2 in binary32. */
static int inliers(const int32_t *X, const int32_t *Y, int M, const float c[3], float t_ri,
                   uint8_t *flag) {
    float lo = c[2] - t_ri;
    if (lo < 0.0f) lo = 0.0f;
    float hi = c[2] + t_ri;
    float lo2 = lo * lo, hi2 = hi * hi;
    int n = 0;
    for (int j = 0; j < M; ++j) {
        float dx = (float)X[j] - c[0], dy = (float)Y[j] - c[1];
        float d2 = dx * dx + dy * dy;
        flag[j] = (uint8_t)(d2 >= lo2 && d2 <= hi2);
        n += flag[j];
    }
    return n;
}

/* -------------------------------------------- Sec. 2.2.5, circle fitting -- */
int orc_estimate(const uint8_t *rgb, int H, int W, int64_t pitch, uint64_t frame_key,
                 const orc_params *p, orc_result *res, orc_debug *dbg) {
    memset(res, 0, sizeof(*res));
    int N = p->n_strips, K = p->cands_per_strip;
    if (W < 8 || H < 3 || N < 1 || K < 2 || (K & 1) || N * K > 256) return -1;
    int cap = N * K;
    int16_t *cx16 = (int16_t *)malloc(sizeof(int16_t) * cap);
    int16_t *cy16 = (int16_t *)malloc(sizeof(int16_t) * cap);
    uint16_t *cs = (uint16_t *)malloc(sizeof(uint16_t) * cap);
    int32_t M = 0;
    orc_candidates(rgb, H, W, pitch, p, cap, cx16, cy16, cs, &M);
    int rc = orc_fit(cx16, cy16, cs, M, H, W, frame_key, p, res, dbg);
    free(cx16);
    free(cy16);
    free(cs);
    return rc;
}

/* Sec. 2.2.5 from the candidate list on: RANSAC, refits, scores, filters,
 * best circle and the t_cs acceptance. */
int orc_fit(const int16_t *cx16, const int16_t *cy16, const uint16_t *cs, int32_t M, int H,
            int W, uint64_t frame_key, const orc_params *p, orc_result *res, orc_debug *dbg) {
    return orc_fit_prior(cx16, cy16, cs, M, H, W, frame_key, p, NULL, res, dbg);
}

/* The same with the previous frame's circle (pixel coordinates cx, cy, r) as
 * one more hypothesis after the random ones, the use of the previous
 * estimate that Sec. 4 suggests; prior == NULL: none. */
int orc_fit_prior(const int16_t *cx16, const int16_t *cy16, const uint16_t *cs, int32_t M,
                  int H, int W, uint64_t frame_key, const orc_params *p, const float *prior,
                  orc_result *res, orc_debug *dbg) {
    memset(res, 0, sizeof(*res));
    int N = p->n_strips, K = p->cands_per_strip;
    if (W < 8 || H < 3 || N < 1 || K < 2 || (K & 1) || N * K > 256 || M < 0 || M > N * K)
        return -1;
    int cap = N * K;
    if (dbg) {
        if (dbg->n_cands) *dbg->n_cands = M;
        for (int j = 0; j < M && j < dbg->cand_cap; ++j) {
            if (dbg->cand_x) dbg->cand_x[j] = cx16[j];
            if (dbg->cand_y) dbg->cand_y[j] = cy16[j];
            if (dbg->cand_s) dbg->cand_s[j] = cs[j];
        }
        if (dbg->best_h) *dbg->best_h = -1;
        if (dbg->n_hyps) *dbg->n_hyps = 0;
    }
    /* origin of the integer coordinates: (floor(W/2), floor(H/2)) */
    int ox = W / 2, oy = H / 2;
    int32_t *X = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *Y = (int32_t *)malloc(sizeof(int32_t) * cap);
    for (int j = 0; j < M; ++j) { X[j] = cx16[j] - ox; Y[j] = cy16[j] - oy; }

    int64_t NH = 0;
    if (M >= 3)
        NH = p->hyp_mode == ORC_HYP_EXHAUSTIVE ? (int64_t)M * (M - 1) * (M - 2) / 6 : p->n_hyps;
    int64_t NH_all = NH + ((prior && M >= 3) ? 1 : 0);
    if (dbg && dbg->n_hyps) *dbg->n_hyps = (int32_t)NH_all;

    uint8_t *flag = (uint8_t *)malloc((size_t)cap + 1);
    int32_t *IX = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *IY = (int32_t *)malloc(sizeof(int32_t) * cap);
    float Wf = (float)W;
    float rlo = p->r_min * Wf, rhi = p->r_max * Wf, dm = p->d_max * Wf;
    float ex = (W & 1) ? 0.0f : -0.5f; /* image centre ((W-1)/2, (H-1)/2) minus origin */
    float ey = (H & 1) ? 0.0f : -0.5f;

    int32_t ti = 0, tj = 1, tk = 2; /* lexicographic triple of the exhaustive mode */
    int64_t best = -1;
    uint32_t bestS = 0;
    float bestc[3] = {0, 0, 0};
    int32_t bestn = 0;
    for (int64_t h = 0; h < NH_all; ++h) {
        int32_t t[3];
        float c[3];
        int ok;
        if (h == NH) {
            /* the previous circle, in the origin-relative coordinates */
            t[0] = t[1] = t[2] = -1;
            c[0] = prior[0] - (float)ox;
            c[1] = prior[1] - (float)oy;
            c[2] = prior[2];
            ok = 1;
        } else {
        if (p->hyp_mode == ORC_HYP_EXHAUSTIVE) {
            t[0] = ti; t[1] = tj; t[2] = tk;
            if (++tk == M) { if (++tj == M - 1) { ++ti; tj = ti + 1; } tk = tj + 1; }
        } else {
            orc_triple(p->seed, frame_key, (uint32_t)h, M, t);
        }
        /* the circle of a triple depends only on the set: take the points in
         * increasing candidate order */
        int32_t s0 = t[0], s1 = t[1], s2 = t[2], tmp;
        if (s0 > s1) { tmp = s0; s0 = s1; s1 = tmp; }
        if (s1 > s2) { tmp = s1; s1 = s2; s2 = tmp; }
        if (s0 > s1) { tmp = s0; s0 = s1; s1 = tmp; }
        ok = orc_circumcircle(X[s0], Y[s0], X[s1], Y[s1], X[s2], Y[s2], c);
        }
        int32_t n_inl = 0;
        uint32_t S = 0;
        int pass = 0;
        if (ok) {
            for (int it = 0; it < p->refine_iters; ++it) {
                inliers(X, Y, M, c, p->t_ri, flag);
                int n = 0;
                for (int j = 0; j < M; ++j)
                    if (flag[j]) { IX[n] = X[j]; IY[n] = Y[j]; ++n; }
                float f[3];
                if (!orc_ls_fit(IX, IY, n, f)) break;
                c[0] = f[0]; c[1] = f[1]; c[2] = f[2];
            }
            n_inl = inliers(X, Y, M, c, p->t_ri, flag);
            for (int j = 0; j < M; ++j)
                if (flag[j]) S += cs[j];
            float dx = c[0] - ex, dy = c[1] - ey;
            pass = c[2] >= rlo && c[2] <= rhi && (dx * dx + dy * dy) <= dm * dm;
            if (pass && (best < 0 || S > bestS)) {
                best = h; bestS = S; bestn = n_inl;
                bestc[0] = c[0]; bestc[1] = c[1]; bestc[2] = c[2];
                if (dbg && dbg->best_inl)
                    for (int j = 0; j < M && j < dbg->cand_cap; ++j) dbg->best_inl[j] = flag[j];
            }
        } else {
            c[0] = c[1] = c[2] = 0.0f;
        }
        if (dbg && h < dbg->hyp_cap) {
            if (dbg->triple) { dbg->triple[3 * h] = t[0]; dbg->triple[3 * h + 1] = t[1]; dbg->triple[3 * h + 2] = t[2]; }
            if (dbg->hyp_n_inl) dbg->hyp_n_inl[h] = n_inl;
            if (dbg->hyp_score) dbg->hyp_score[h] = S;
            if (dbg->hyp_pass) dbg->hyp_pass[h] = pass;
            if (dbg->hyp_circle) { dbg->hyp_circle[3 * h] = c[0]; dbg->hyp_circle[3 * h + 1] = c[1]; dbg->hyp_circle[3 * h + 2] = c[2]; }
        }
    }
    if (dbg && dbg->best_h) *dbg->best_h = (int32_t)best;

    if (best >= 0) {
        res->cx = (float)ox + bestc[0];
        res->cy = (float)oy + bestc[1];
        res->r = bestc[2];
        /* divisor of the score compared with t_cs (Sec. 2.2.5): the paper's
         * candidate count 2N, the slot count N K, none, or the most inliers
         * the best circle can have, K per strip it crosses */
        double norm = p->score_norm == ORC_NORM_2N ? 2.0 * N
                    : p->score_norm == ORC_NORM_NK ? (double)N * K : 1.0;
        if (p->score_norm == ORC_NORM_CIRCLE) {
            int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
            orc_strip_rows(H, N, p->alpha, rows);
            norm = (double)K * orc_circle_strips(rows, N, res->cy, res->r, p->t_ri);
            free(rows);
        }
        uint32_t T_cs = (uint32_t)ceil((double)p->t_cs * 32768.0 * norm);
        res->score = norm > 0.0 ? (float)((double)bestS / (32768.0 * norm)) : 0.0f;
        res->n_inliers = bestn;
        res->valid = norm > 0.0 && bestS >= T_cs;
    }
    free(X); free(Y); free(flag); free(IX); free(IY);
    return 0;
}

int orc_circle_strips(const int32_t *rows, int N, float cy, float r, float t_ri) {
    const float reach = r + t_ri;
    int n = 0;
    for (int i = 0; i < N; ++i) {
        const float dy = (float)rows[i] - cy;
        if (fabsf(dy) <= reach) ++n;
    }
    return n;
}

/* ----------------------------------------------------- Sec. 1.1, Fig. 1 -- */
void orc_mask(const orc_result *res, int H, int W, uint8_t *out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t m = 1;
            if (res->valid) {
                float dx = (float)x - res->cx, dy = (float)y - res->cy;
                m = (uint8_t)((dx * dx + dy * dy) <= res->r * res->r);
            }
            out[(int64_t)y * W + x] = m;
        }
}

/* ------------------------------------------- temporal smoothing (Sec. 4) -- */
void orc_smooth(const orc_result *cur, int W, const orc_smooth_params *sp, float state[4],
                orc_result *out) {
    const float d = state[3] * sp->gamma;
    if (cur->valid) {
        const float J = sp->jump * (float)W;
        const int near = d > 0.0f && fabsf(cur->cx - state[0]) <= J &&
                         fabsf(cur->cy - state[1]) <= J && fabsf(cur->r - state[2]) <= J;
        *out = *cur;
        if (near) {
            const float w = d + cur->score;
            const float pcx = d * state[0], ccx = cur->score * cur->cx;
            const float pcy = d * state[1], ccy = cur->score * cur->cy;
            const float pr = d * state[2], cr = cur->score * cur->r;
            out->cx = (pcx + ccx) / w;
            out->cy = (pcy + ccy) / w;
            out->r = (pr + cr) / w;
            state[3] = w;
        } else {
            state[3] = cur->score;
        }
        state[0] = out->cx;
        state[1] = out->cy;
        state[2] = out->r;
    } else if (d > 0.0f && d >= sp->t_hold) {
        out->cx = state[0];
        out->cy = state[1];
        out->r = state[2];
        out->score = 0.0f;
        out->valid = 1;
        out->n_inliers = 0;
        state[3] = d;
    } else {
        *out = *cur;
        state[0] = state[1] = state[2] = state[3] = 0.0f;
    }
}
