/*
 * ca_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded CPU implementation of the lean content-area
 * pipeline of Budd et al., "Rapid and robust endoscopic content area
 * estimation" (arXiv 2210.14771): strip sampling (Sec. 2.2.2, Eq. 1),
 * handcrafted edge scoring (Sec. 2.2.3, Eq. 2-3), candidate selection and
 * RANSAC + least-squares circle fitting (Sec. 2.2.5) and the content-area
 * mask (Sec. 1.1, Fig. 1).
 *
 * It exists to check the CUDA library.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the library never does.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every floating-point step that decides an integer (a quantised score index,
 * an inlier flag, a filter) is taken in the precision the CUDA kernels use
 * (IEEE binary32, round-to-nearest, no fused multiply-add), so that both sides
 * take the same decisions; everything else is exact integer arithmetic.
 */
#ifndef CA_ORACLE_H
#define CA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_HYP_RANDOM = 0, ORC_HYP_EXHAUSTIVE = 1 };
enum { ORC_NORM_2N = 0, ORC_NORM_NK = 1, ORC_NORM_RAW = 2, ORC_NORM_CIRCLE = 3 };

/* Sizes of the quantised score tables (index ranges are 0..N-1). */
enum { ORC_LUT_G = 5772, ORC_LUT_T = 8193, ORC_LUT_I = 256 };

typedef struct {
    int32_t n_strips;        /* N, Eq. 1 (Appendix A: 16) */
    int32_t cands_per_strip; /* K, even; K/2 picks per half-strip (paper: 2) */
    int32_t n_hyps;          /* RANSAC attempts (random mode) */
    int32_t refine_iters;    /* least-squares refits (Sec. 2.2.5: 3) */
    float alpha;             /* Eq. 1 (8) */
    float t_g;               /* Eq. 2 (20) */
    float t_theta_deg;       /* Eq. 2 (30 degrees) */
    float t_iota;            /* Eq. 2 (25) */
    float t_ps;              /* point-score filter (0.03) */
    float t_cs;              /* circle-score acceptance (0.06) */
    float t_px;              /* edge-distance filter in pixels (3) */
    float t_ri;              /* RANSAC inlier distance in pixels (3) */
    float r_min, r_max;      /* radius limits, multiples of W (0.1, 0.8) */
    float d_max;             /* centre-offset limit, multiple of W (0.2) */
    int32_t sup_px;          /* suppression half-window between picks of a half */
    int32_t hyp_mode;        /* ORC_HYP_* */
    int32_t score_norm;      /* ORC_NORM_*: divisor of the circle score */
    int32_t sobel_norm;      /* 1 = raw 3x3 Sobel, 8 = Sobel / 8 */
    uint64_t seed;           /* Philox key */
} orc_params;

typedef struct {
    float cx, cy, r;   /* pixel-index coordinates (pixel centre = integer) */
    float score;       /* S_best / (32768 * norm) */
    int32_t valid;     /* 0: content area is the whole rectangle */
    int32_t n_inliers; /* final inlier count of the best circle */
} orc_result;

/* Optional dumps of one frame's intermediate values.  Every pointer may be
 * NULL; arrays are filled up to the stated capacity. */
typedef struct {
    int32_t cand_cap;     /* capacity of the candidate arrays */
    int32_t *n_cands;     /* out: M, candidates kept after filtering */
    int16_t *cand_x, *cand_y;
    uint16_t *cand_s;     /* Q15 score */
    int32_t hyp_cap;      /* capacity of the per-hypothesis arrays */
    int32_t *n_hyps;      /* out: hypotheses evaluated */
    int32_t *triple;      /* 3 per hypothesis: candidate indices */
    int32_t *hyp_n_inl;   /* final inlier count */
    uint32_t *hyp_score;  /* S_h, sum of Q15 scores of the final inliers */
    int32_t *hyp_pass;    /* 1 if the final circle passed the filters */
    float *hyp_circle;    /* 3 per hypothesis: final cx, cy, r (origin-relative) */
    int32_t *best_h;      /* out: index of the winning hypothesis or -1 */
    uint8_t *best_inl;    /* M flags: final inlier set of the winner */
} orc_debug;

void orc_params_default(orc_params *p);

/* Eq. 1 strip rows: floor, then clamp to [1, H-2]. Returns 0 on success. */
int orc_strip_rows(int H, int N, float alpha, int32_t *rows);

/* Quantised score tables (Eq. 2); sizes ORC_LUT_G, ORC_LUT_T, ORC_LUT_I. */
void orc_build_luts(const orc_params *p, uint16_t *lut_g, uint16_t *lut_t, uint16_t *lut_i);

/* BT.601 integer luma of one RGB pixel. */
int orc_luma(int r, int g, int b);

/* Per-pixel Q15 scores s_q of the strip centred on `row` (W outputs), plus
 * optional features (any may be NULL): gx, gy, iota. */
int orc_strip_scores(const uint8_t *rgb, int H, int W, int64_t pitch, int row,
                     const orc_params *p, uint16_t *s_out, int32_t *gx_out,
                     int32_t *gy_out, uint8_t *iota_out);

/* The same score in double precision straight from Eq. 2-3 (no tables). */
double orc_score_exact(int gx, int gy, int cx2, int cy2, int iota, const orc_params *p);

/* Candidates of a frame, in order (strip, left picks, right picks). */
int orc_candidates(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                   int cap, int16_t *xs, int16_t *ys, uint16_t *ss, int32_t *M);

/* Prior-guided scoring (the use of the previous estimate that Sec. 4
 * suggests): the angle term measures the direction of g against the vector
 * to a prior centre instead of the image centre.  orc_prior_centre2 gives
 * the doubled integer centre of a prior circle centre (cx, cy): round(2 cx),
 * round(2 cy), ties to even, clamped into [0, 2(W-1)] x [0, 2(H-1)];
 * orc_candidates_centre is orc_candidates with that doubled centre
 * ((W-1, H-1) is the image centre: the same as orc_candidates). */
void orc_prior_centre2(float cx, float cy, int H, int W, int32_t out[2]);
int orc_candidates_centre(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                          int32_t c2x0, int32_t c2y0, int cap, int16_t *xs, int16_t *ys,
                          uint16_t *ss, int32_t *M);

/* Candidates from learned per-pixel Q15 scores (learned: N x W, strip by
 * strip), picked by the same rule; with `fallback`, a half-strip whose best
 * learned score is below 16384 (probability one half) takes the handcrafted
 * points of that half instead. */
int orc_learned_candidates(const uint8_t *rgb, int H, int W, int64_t pitch, const orc_params *p,
                           const uint16_t *learned, int fallback, int cap, int16_t *xs,
                           int16_t *ys, uint16_t *ss, int32_t *M);

/* Philox4x32-10 (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Hypothesis h's distinct candidate triple, drawn with Philox. */
void orc_triple(uint64_t seed, uint64_t frame_key, uint32_t h, int M, int32_t out[3]);

/* h-th triple (i<j<k) in lexicographic order. */
void orc_triple_exhaustive(int64_t h, int M, int32_t out[3]);

/* Circle through three integer points; 0 if collinear. out = cx, cy, r. */
float orc_rn_ratio(int64_t num, int64_t den);
int orc_circumcircle(int ax, int ay, int bx, int by, int cx, int cy, float out[3]);

/* Algebraic least-squares circle (Coope 1993) of n integer points; 0 if the
 * fit is degenerate (n < 3 or zero determinant).  out = cx, cy, r. */
int orc_ls_fit(const int32_t *X, const int32_t *Y, int n, float out[3]);

/* Correctly rounded conversion of the 128-bit integer hi*2^64+lo. */
float orc_i128_to_f32(int64_t hi, uint64_t lo);

/* Whole pipeline for one frame (device-independent, single-threaded). */
int orc_estimate(const uint8_t *rgb, int H, int W, int64_t pitch, uint64_t frame_key,
                 const orc_params *p, orc_result *res, orc_debug *dbg);

/* The fitting part of the pipeline (Sec. 2.2.5) on a given candidate list
 * (pixel coordinates and Q15 scores, in order): same steps and outputs as
 * orc_estimate after its candidate stage. */
int orc_fit(const int16_t *xs, const int16_t *ys, const uint16_t *ss, int32_t M, int H, int W,
            uint64_t frame_key, const orc_params *p, orc_result *res, orc_debug *dbg);

/* ---- Learned edge scorer (1-D CNN over strip profiles; see
 * ca_scorer_oracle.c).  Parameters: one flat binary32 vector of
 * ORC_SC_NPARAM values, W1[32][14][7], b1[32], W2[32][32][7], b2[32],
 * W3[32][32][7], b3[32], wh[32], bh. */
enum { ORC_SC_CIN = 14, ORC_SC_CH = 32, ORC_SC_K = 7, ORC_SC_NPARAM = 17601 };
enum { ORC_SC_EXACT = 0, ORC_SC_MIXED = 1 };

/* bfloat16 round-to-nearest-even of a binary32 value. */
float orc_bf16(float v);

/* Offsets of W1, b1, W2, b2, W3, b3, wh, bh in the parameter vector. */
void orc_sc_offsets(int32_t out[8]);

/* Column features of a strip (rgb3: rows y-1, y, y+1, each W x 3 bytes). */
void orc_sc_features(const uint8_t *rgb3, int W, int y, int H, int mixed, double *feat);

/* Logits of the W columns; acts (optional) receives features (W x 14) and
 * the activations a1, a2, a3 (W x 32 each). */
int orc_sc_forward(const uint8_t *rgb3, int W, int y, int H, const float *prm, int mode,
                   double *logits, double *acts);

/* Weighted cross-entropy of the strip's columns against labels (0/1), and
 * its gradient, added into grads (ORC_SC_NPARAM doubles). */
double orc_sc_loss_grad(const uint8_t *rgb3, int W, int y, int H, const uint8_t *labels,
                        float pos_weight, const float *prm, int mode, double *grads);

/* ---- The paper's own learned edge scorer (Sec. 2.2.4; see
 * ca_scorer2d_oracle.c): 3x3 convolutions to 8, 16, 32 features with ReLU,
 * a 1x1 head and a sigmoid, on RGBXY strips 7 rows high.  Parameters: one
 * flat binary32 vector of ORC_SC2_NPARAM values, W1[8][5][3][3], b1[8],
 * W2[16][8][3][3], b2[16], W3[32][16][3][3], b3[32], wh[32], bh. */
enum { ORC_SC2_CIN = 5, ORC_SC2_NPARAM = 6209 };

void orc_sc2_offsets(int32_t out[8]);
/* The 7 rows y-3 .. y+3 of a frame (clamped into it) into rgb7 (7 x W x 3),
 * their frame rows into rows. */
void orc_sc2_strip(const uint8_t *rgb, int H, int W, int64_t pitch, int y, uint8_t *rgb7,
                   int32_t rows[7]);
/* RGBXY features of the 7 x W pixels, feat[(k W + x) 5 + c]. */
void orc_sc2_features(const uint8_t *rgb7, const int32_t rows[7], int W, int H, double *feat);
/* Logits of the strip's middle row (W values). */
int orc_sc2_forward(const uint8_t *rgb7, const int32_t rows[7], int W, int H, const float *prm,
                    double *logits);
/* The same with a mode: ORC_SC_EXACT (= orc_sc2_forward) or ORC_SC_MIXED
 * (the stored-value roundings of a bfloat16 tensor-core kernel, sums in
 * binary64: a tolerance reference, see the source). */
int orc_sc2_forward_mode(const uint8_t *rgb7, const int32_t rows[7], int W, int H,
                         const float *prm, int mode, double *logits);
/* Summed soft binary cross-entropy against targets in [0, 1], column x
 * weighted by 1 + (pos_weight - 1) t_x; gradient added into grads
 * (ORC_SC2_NPARAM doubles). */
double orc_sc2_loss_grad(const uint8_t *rgb7, const int32_t rows[7], int W, int H,
                         const double *targets, double pos_weight, const float *prm,
                         double *grads);
/* Soft targets of row y: exp(-d^2 / (2 sigma^2)), d the distance of the
 * pixel to the circle; 0 without a circle. */
void orc_sc2_targets(float cx, float cy, float r, int valid, int W, int y, double sigma,
                     double *t);

/* Strips whose row is within r + t_ri of the circle's centre row,
 * |rows[i] - cy| <= r + t_ri in binary32: the strips the circle (widened by
 * the inlier distance) crosses, each of which can give it at most K inliers
 * (the normaliser K n of ORC_NORM_CIRCLE). */
int orc_circle_strips(const int32_t *rows, int N, float cy, float r, float t_ri);

/* orc_fit with the previous frame's circle (cx, cy, r in pixel coordinates)
 * as one more hypothesis, index n_hyps (Sec. 4: using the previous
 * estimate); prior == NULL is orc_fit. */
int orc_fit_prior(const int16_t *xs, const int16_t *ys, const uint16_t *ss, int32_t M, int H,
                  int W, uint64_t frame_key, const orc_params *p, const float *prior,
                  orc_result *res, orc_debug *dbg);

/* Content-area mask of a result: disc intersected with the rectangle, or the
 * whole rectangle when the circle is not valid.  H*W bytes, 0/1. */
void orc_mask(const orc_result *res, int H, int W, uint8_t *out);

/* Temporal smoothing of one stream's results (an extension in the direction
 * Sec. 4 points to: the estimates of earlier frames inform the current one).
 * state = {cx, cy, r, conf} of the stream (conf 0: none), updated in place.
 * In binary32, each operation rounded on its own, in this order:
 *   d = conf * gamma                          (the decayed confidence)
 *   valid frame, d > 0 and |cx - cx'|, |cy - cy'|, |r - r'| <= jump * W:
 *     w = d + score;  c = (d * c' + score * c) / w for c in cx, cy, r;
 *     conf = w                                  (confidence-weighted mean)
 *   valid frame otherwise (first frame, or a jump: a new scene):
 *     the frame's circle, conf = score
 *   invalid frame with d > 0 and d >= t_hold:
 *     the previous circle held (valid, score 0, n_inliers 0), conf = d
 *   invalid frame otherwise: invalid, conf = 0 (state cleared).
 * A valid output keeps the frame's score and n_inliers. */
typedef struct {
    float gamma;    /* decay of the confidence per frame, [0, 1) */
    float jump;     /* scene-change distance, multiple of W */
    float t_hold;   /* least decayed confidence that holds a circle */
    int32_t pad;
} orc_smooth_params;
void orc_smooth(const orc_result *cur, int W, const orc_smooth_params *sp, float state[4],
                orc_result *out);

#ifdef __cplusplus
}
#endif
#endif
