/*
 * ca.h -- C ABI of libca, a single-GPU (sm_103a) implementation of the lean
 * content-area pipeline of Budd et al., "Rapid and robust endoscopic content
 * area estimation: a lean GPU-based pipeline and curated benchmark dataset"
 * (arXiv 2210.14771).
 *
 * What one call computes, per frame (paper sections in brackets):
 *   strip rows h_i of Eq. 1 [Sec. 2.2.2] -> per-pixel handcrafted score
 *   s = s_g s_theta s_iota of Eq. 2-3 [Sec. 2.2.3] -> best points of each
 *   half-strip, filtered by t_px and t_ps -> RANSAC over random triples, each
 *   refined by three least-squares refits, scored by the sum of its inlier
 *   scores, filtered by r_min/r_max/d_max -> best circle, accepted if its score
 *   reaches t_cs [Sec. 2.2.5] -> content-area mask = disc intersected with the
 *   sensor rectangle, or the whole rectangle when no circle is accepted
 *   [Sec. 1.1, Fig. 1; Sec. 2.2.1].
 *
 * Conventions for every function:
 *   - Pointers named *_dev are device pointers; everything else is host memory.
 *   - The caller owns frames, results and masks and keeps them alive until the
 *     work queued on the given stream has completed.  The handle owns its
 *     workspace, tables, graphs, scorer weights and serving state.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream only queue work on it and return.
 *   - Every call returns a ca_status and never aborts.  Argument errors are
 *     detected on the host before any work is queued (CA_ERR_INVALID_ARG);
 *     CUDA errors surface as CA_ERR_CUDA, by this call or the next one.
 *     ca_last_error() gives a one-line description of the last failure.
 *   - Results depend only on (frame bytes, params, frame_key), never on the
 *     batch size or position: the RANSAC draws are keyed on frame_key.
 *   - Limits: 8 <= W <= 4096, 3 <= H <= 4096, row pitch >= 3W bytes,
 *     N*K <= 256 candidate slots per frame.
 *
 * Not thread-safe: one handle serves one host thread at a time.
 */
#ifndef CA_H
#define CA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CA_OK = 0,
    CA_ERR_INVALID_ARG = 1, /* bad pointer, size, layout or parameter */
    CA_ERR_CUDA = 2,        /* a CUDA runtime call or a kernel failed */
    CA_ERR_OOM = 3,         /* device or pinned allocation failed */
    CA_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    CA_ERR_UNSUPPORTED = 5, /* feature not available (e.g. no scorer weights) */
    CA_ERR_ADMISSION = 6,   /* serving: request does not fit the memory budget */
    CA_ERR_STATE = 7        /* call not valid in the handle's current state */
} ca_status;

enum { CA_HYP_RANDOM = 0, CA_HYP_EXHAUSTIVE = 1 };
/* divisor of the circle score compared with t_cs (Sec. 2.2.5): the paper's
 * candidate count 2N, the slot count N*K, none, or (the default) the most
 * inliers the best circle can have, K per strip whose row lies within
 * r + t_ri of the circle's centre row (|h_i - cy| <= r + t_ri in binary32) */
enum { CA_NORM_2N = 0, CA_NORM_NK = 1, CA_NORM_RAW = 2, CA_NORM_CIRCLE = 3 };
/* edge scorer: handcrafted (Sec. 2.2.3); a learned 1-D CNN over 3-row strip
 * profiles, alone or with the handcrafted score taking over half-strips the
 * network is unsure about; the paper's own 2-D CNN over 7-row strips
 * (Sec. 2.2.4), alone or with the same fallback */
enum { CA_SCORER_HAND = 0, CA_SCORER_LEARNED = 1, CA_SCORER_LEARNED_FALLBACK = 2,
       CA_SCORER_2D = 3, CA_SCORER_2D_FALLBACK = 4 };
/* how a call is launched (results never depend on it): AUTO = the fastest
 * configuration ca_tune found for this shape of batch, else a size-based
 * choice; STAGED = three kernels (strips, fit, mask); FUSED = one persistent
 * kernel that runs all three phases, frames pipelined in waves */
enum { CA_BATCH_AUTO = 0, CA_BATCH_STAGED = 1, CA_BATCH_FUSED = 2 };

/* Parameters; ca_params_default() fills the values of the paper's Appendix A. */
typedef struct ca_params {
    int32_t n_strips;        /* N, number of strips (Eq. 1; default 16) */
    int32_t cands_per_strip; /* K, even: K/2 best points per half-strip (2) */
    int32_t n_hyps;          /* RANSAC attempts per frame (1024) */
    int32_t refine_iters;    /* least-squares refits per attempt (3) */
    float alpha;             /* strip weighting of Eq. 1 (8) */
    float t_g;               /* gradient-magnitude soft threshold (20) */
    float t_theta_deg;       /* gradient-direction soft threshold, degrees (30) */
    float t_iota;            /* preceding-maximum soft threshold (25) */
    float t_ps;              /* point-score filter (0.03) */
    float t_cs;              /* circle-score acceptance threshold (0.06) */
    float t_px;              /* drop points closer than this to the edge (3) */
    float t_ri;              /* inlier distance, pixels (3) */
    float r_min, r_max;      /* radius bounds, multiples of W (0.1, 0.8) */
    float d_max;             /* centre offset bound, multiple of W (0.2) */
    int32_t sup_px;          /* suppression half-window between picks (8) */
    int32_t hyp_mode;        /* CA_HYP_* */
    int32_t score_norm;      /* CA_NORM_* */
    int32_t sobel_norm;      /* 1: raw 3x3 Sobel; 8: Sobel divided by 8 */
    int32_t scorer_mode;     /* CA_SCORER_* */
    int32_t hyp_threads;     /* threads per RANSAC hypothesis: 0 = chosen per call
                                from the work size, or 1, 2, 4, 8; results do not
                                depend on it */
    int32_t batch_mode;      /* CA_BATCH_* (results do not depend on it) */
    int32_t wave_frames;     /* fused launch: frames per pipeline wave, 0 = chosen
                                per call (results do not depend on it) */
    int32_t prior_centre;    /* tracked calls (ca_estimate_tracked): 1 = for a frame
                                whose track has an accepted previous circle, the
                                direction term of the edge score (Eq. 2) measures
                                the angle between g and the vector to that
                                circle's centre instead of the image centre (the
                                use of the previous estimate Sec. 4 suggests); the
                                centre is taken as round(2 cx) / 2, round(2 cy) / 2
                                (ties to even) clamped into the frame.  0 = image
                                centre (default); other calls ignore it */
    int32_t reserved;        /* must be 0 */
    uint64_t seed;           /* key of the RANSAC random stream */
} ca_params;

/* One input frame: packed RGB, 8 bits per channel, rows `pitch` bytes apart
 * (device memory).  `mask_dev`, when not NULL, receives the H*W content-area
 * mask (one byte per pixel, 0 or 1, rows W bytes apart). */
typedef struct ca_frame {
    const uint8_t *rgb_dev;
    uint8_t *mask_dev;
    int32_t H, W;
    int64_t pitch;
    uint64_t frame_key;
} ca_frame;

/* One result (24 bytes): circle in pixel-index coordinates (pixel centres at
 * integer x, y; y down), score = best circle score / (32768 * normaliser),
 * valid = 0 when the content area is the whole rectangle. */
typedef struct ca_result {
    float cx, cy, r, score;
    int32_t valid, n_inliers;
} ca_result;

typedef struct ca_handle ca_handle;

/* Fills *p with the defaults above (Appendix A of the paper). */
void ca_params_default(ca_params *p);

/* Creates a handle bound to CUDA device `device`.  Allocates only small
 * tables; workspaces grow on first use.  *out is NULL on failure. */
ca_status ca_create(ca_handle **out, int device);

/* Synchronises the handle's streams and frees everything it owns. */
ca_status ca_destroy(ca_handle *h);

/* Estimates the content area of B frames (Sec. 2.2.1-2.2.5) and, for frames
 * whose mask_dev is set, writes the mask (Sec. 1.1).  frames: host array of B
 * descriptors pointing to device memory, any mix of resolutions.  out_dev:
 * device array of B ca_result.  Queued on `stream`; returns once queued. */
ca_status ca_estimate(ca_handle *h, const ca_frame *frames, int B, const ca_params *p,
                      ca_result *out_dev, void *stream);

/* Same for B frames of one resolution stored back to back:
 * frames_dev = B x H x W x 3 bytes; masks_dev = B x H x W bytes or NULL;
 * keys = host array of B frame keys, or NULL for keys 0..B-1. */
ca_status ca_estimate_uniform(ca_handle *h, const uint8_t *frames_dev, int B, int H, int W,
                              const uint64_t *keys, const ca_params *p, ca_result *out_dev,
                              uint8_t *masks_dev, void *stream);

/* Tracked estimate (video): the previous estimate of a frame's track is used
 * for the current one, as the paper's discussion suggests (Sec. 4): when the
 * track's previous result (state_dev[track[i]]) was accepted (valid), its
 * circle joins RANSAC as one more hypothesis, index n_hyps after the random
 * ones, refined and scored like them (ties still go to the lowest index).
 * After the call state_dev[track[i]] holds frame i's result.  state_dev:
 * device array of n_tracks results (zero = no previous circle); track: host
 * array of B indices in [0, n_tracks), or -1 for an untracked frame; a track
 * may appear once per call.  Otherwise as ca_estimate. */
ca_status ca_estimate_tracked(ca_handle *h, const ca_frame *frames, int B, const ca_params *p,
                              ca_result *state_dev, const int32_t *track, int n_tracks,
                              ca_result *out_dev, void *stream);

/* Allocation-free estimate, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a packaging variant of
 * ca_estimate_uniform (same arguments and results, bit for bit) with no handle.
 *
 * Who needs it: applications that reserve their whole device-memory budget up
 * front and forbid libraries from allocating on their own (a video appliance
 * that must not fail a cudaMalloc in the middle of a procedure, or a host
 * framework whose memory pool owns the device), and frame loops that cannot
 * absorb the stalls of cudaMalloc / cudaFree, which may synchronise the
 * device.  This call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * Instead it uses one fixed scratch array of CA_STATIC_SCRATCH_BYTES of device
 * memory, defined in the library, which every GPU that loads the library holds
 * until the process exits.  The caller still passes the inputs and outputs
 * (frames_dev, out_dev, masks_dev, keys as in ca_estimate_uniform).
 *   - Limits: B <= CA_STATIC_MAX_FRAMES, and at most CA_STATIC_MAX_HYPS
 *     hypotheses per frame (n_hyps, or C(N*K,3) in exhaustive mode); larger
 *     requests return CA_ERR_INVALID_ARG before any work is queued.  The other
 *     limits are those of ca_estimate_uniform.  No debug capture.
 *   - The first call on each device looks up the array's device address, with
 *     that device current.
 *   - Not for CUDA graphs: each call copies its tables and frame descriptors
 *     from the host call stack with ordinary copies, which a graph would
 *     replay from memory that no longer holds them.  A call made while
 *     `stream` is being captured returns CA_ERR_UNSUPPORTED before it queues
 *     anything.
 *   - Every call uses the same array, which keeps the last call's contents:
 *     the call clears what must start at zero, but calls whose work overlaps
 *     on the GPU (other streams, other host threads) race and corrupt each
 *     other.  Order them on one stream or wait between them.
 *   - The parameter tables (about 43 KB) are copied from host memory on each
 *     call with ordinary asynchronous copies; the call returns once queued.
 *   - Errors: a status only (there is no handle for ca_last_error). */
#define CA_STATIC_MAX_FRAMES 256
#define CA_STATIC_MAX_HYPS 4096
#define CA_STATIC_SCRATCH_BYTES 706560
ca_status ca_estimate_static(const uint8_t *frames_dev, int B, int H, int W, const uint64_t *keys,
                             const ca_params *p, ca_result *out_dev, uint8_t *masks_dev,
                             void *stream);

/* ---- Batching: autotuner and captured plans (no counterpart in the paper,
 * which runs one frame per launch, Sec. 2.2.6). */

/* Outcome of ca_tune.  Times are mean milliseconds per call on the tuning
 * batch, measured with CUDA events on the call's stream: 3 calls per
 * configuration in the sweep (host side included), then, for each of the 6
 * fastest (among them the fastest staged and the fastest fused one), 24
 * replays of a plan captured with it (as ca_plan_launch runs it); the lowest
 * mean of those is chosen. */
typedef struct ca_tuning {
    int32_t batch_mode;   /* chosen CA_BATCH_STAGED or CA_BATCH_FUSED */
    int32_t hyp_threads;  /* chosen threads per hypothesis */
    int32_t wave_frames;  /* chosen frames per wave (fused) */
    int32_t n_tried;      /* configurations timed */
    float ms;             /* chosen configuration (24 plan replays) */
    float ms_staged;      /* fastest staged configuration in the sweep */
    float ms_fused;       /* fastest fused configuration in the sweep */
    float ms_untuned;     /* the configuration CA_BATCH_AUTO used before tuning */
    int32_t fit_lag;      /* chosen (fused): the fit of a wave follows the strips of
                             the wave fit_lag waves later */
    int32_t mask_lag;     /* chosen (fused): its masks follow the strips of the wave
                             mask_lag waves later */
} ca_tuning;

/* Autotuner.  Runs the batch (arguments as in ca_estimate) under every launch
 * configuration that leaves the results unchanged -- staged or fused launch,
 * 1/2/4/8 threads per hypothesis, and for the fused launch the frames per
 * wave -- times each, and remembers the fastest for later CA_BATCH_AUTO calls
 * on batches of the same shape (B, the list of resolutions, N, K, hypotheses,
 * hypothesis mode, which frames have masks).  Synchronous; overwrites out_dev
 * and the masks; *out (may be NULL) receives the outcome.  The parameters
 * that do change results (N, K, hypotheses) are the caller's to choose. */
ca_status ca_tune(ca_handle *h, const ca_frame *frames, int B, const ca_params *p,
                  ca_result *out_dev, void *stream, ca_tuning *out);

/* A captured estimate: the launch(es) of one batch -- fixed frame buffers,
 * masks, keys, parameters and output -- recorded once in a CUDA graph with
 * the plan's own tables, descriptors and workspace, then replayed by
 * ca_plan_launch as a single graph launch.  New frame contents are picked up
 * by each launch; changing a pointer, key or parameter needs a new plan.
 * The plan records the handle's launch configuration (tuned or explicit) at
 * creation.  Launches of one plan must not overlap on the GPU (they share
 * the plan's workspace); different plans are independent.  The plan must be
 * destroyed before its handle. */
typedef struct ca_plan ca_plan;
ca_status ca_plan_create(ca_handle *h, const ca_frame *frames, int B, const ca_params *p,
                         ca_result *out_dev, ca_plan **out);
ca_status ca_plan_launch(ca_plan *plan, void *stream);
ca_status ca_plan_destroy(ca_plan *plan);

/* ---- Learned edge scorer (Sec. 2.2.4: a learned alternative to the
 * handcrafted edge score; here a 1-D network over strip profiles).
 *
 * Per strip column x (the strip's rows y-1, y, y+1), 14 features: luma, R, G,
 * B of each row as (v - 128) / 128, then (x - (W-1)/2) / W and (y - (H-1)/2)
 * / H.  Three convolutions of kernel 7 with 32 output channels and ReLU
 * ("same" zero padding; conv[x][co] = b[co] + sum_{ci,t} W[co][ci][t]
 * in[x + t - 3][ci]), a 1x1 head logit = bh + wh . a3 and p = sigmoid(logit).
 * Weights and activations are rounded to bfloat16, sums accumulate in f32 on
 * the tensor cores.  The edge score of a column is round(32768 p).
 *
 * Parameters: CA_SCORER_NPARAM binary32 values in the order W1[32][14][7],
 * b1[32], W2[32][32][7], b2[32], W3[32][32][7], b3[32], wh[32], bh.
 *
 * With scorer_mode LEARNED the candidates of every half-strip come from the
 * learned scores (same pick rule, K <= 16); with LEARNED_FALLBACK a half-strip
 * whose best learned score is below 16384 (p < 1/2) keeps its handcrafted
 * candidates.  Either mode needs parameters (init, set or load) first. */
#define CA_SCORER_NPARAM 17601

/* Training hyper-parameters: SGD with momentum on the weighted binary
 * cross-entropy of the columns, mean over the columns of the step:
 *     f = min(1, clip_norm / |g|)   (f = 1 when clip_norm is 0)
 *     v = momentum v + f g,   w = w - lr_t v
 * with g the mean gradient of the step and |g| its Euclidean norm over all
 * CA_SCORER_NPARAM parameters.  lr_t = lr, except in ca_scorer_train with
 * lr_schedule CA_LR_COSINE: over the T steps of the call, a linear warm-up
 * lr (t + 1) / U for the first U = clamp(T / 20, 1, 200) steps, then
 * lr (1 + cos(pi (t - U) / (T - U))) / 2.  Invalid values (non-finite,
 * momentum outside [0, 1), pos_weight <= 0, clip_norm < 0, unknown schedule)
 * return CA_ERR_INVALID_ARG. */
enum { CA_LR_CONSTANT = 0, CA_LR_COSINE = 1 };
typedef struct ca_train_params {
    float lr;            /* step size (peak step size with CA_LR_COSINE) */
    float momentum;      /* momentum of the SGD update */
    float pos_weight;    /* loss weight of edge columns (label 1); others weigh 1 */
    int32_t apply;       /* 0: compute the gradient only (no update) */
    float clip_norm;     /* > 0: clip the gradient norm of a step to this value */
    int32_t lr_schedule; /* CA_LR_CONSTANT or CA_LR_COSINE (ca_scorer_train only) */
} ca_train_params;

/* Random initial parameters (He-normal convolution weights, zero biases,
 * head bias -3), seeded; resets the momentum. */
ca_status ca_scorer_init(ca_handle *h, uint64_t seed);
/* Copies n = CA_SCORER_NPARAM parameters in / out (host memory); set resets
 * the momentum. */
ca_status ca_scorer_set_params(ca_handle *h, const float *params, size_t n);
ca_status ca_scorer_get_params(ca_handle *h, float *params, size_t n);
/* Checkpoint: parameters and momentum in a small binary file (magic "CASC",
 * version, count, then binary32 values). */
ca_status ca_scorer_save(ca_handle *h, const char *path);
ca_status ca_scorer_load(ca_handle *h, const char *path);

/* Network on n stand-alone strips: strips_dev = n x 3 x W x 3 bytes (rows
 * y-1, y, y+1 of each strip, packed RGB), ys_dev = n middle-row indices in
 * frames of height H.  Writes the n x W logits (f32) and/or Q15 scores (either
 * may be NULL).  Queued on `stream`. */
ca_status ca_scorer_forward(ca_handle *h, const uint8_t *strips_dev, const int32_t *ys_dev, int n,
                            int W, int H, float *logits_dev, uint16_t *scores_dev, void *stream);

/* One training step on the strips idx_dev[0..n-1] (or 0..n-1 when idx_dev is
 * NULL) of a strip set as in ca_scorer_forward, with labels_dev = per strip W
 * bytes (1 = edge column).  Runs the forward pass, the loss and its gradient
 * with the library's kernels and, if tp->apply, the SGD update.  Synchronous.
 * loss_host (may be NULL): the summed loss of the step; grads_host (may be
 * NULL): the summed gradient (CA_SCORER_NPARAM values, before the 1/columns
 * scaling of the update). */
ca_status ca_scorer_step(ca_handle *h, const uint8_t *strips_dev, const int32_t *ys_dev,
                         const uint8_t *labels_dev, const int32_t *idx_dev, int n, int W, int H,
                         const ca_train_params *tp, float *loss_host, float *grads_host);

/* Training loop: `epochs` passes over the n strips in minibatches of `batch`
 * strips, shuffled per epoch by `seed`.  epoch_loss_host (may be NULL)
 * receives the mean loss per column of each epoch.  Synchronous. */
ca_status ca_scorer_train(ca_handle *h, const uint8_t *strips_dev, const int32_t *ys_dev,
                          const uint8_t *labels_dev, int n, int W, int H, const ca_train_params *tp,
                          int epochs, int batch, uint64_t seed, float *epoch_loss_host);

/* Temporal smoothing of tracked results (an extension in the direction
 * Sec. 4 points to: the estimates of earlier frames inform the current one).
 * Per track a state {cx, cy, r, conf} (4 binary32 in state_dev, zero = none)
 * is updated in binary32, each operation rounded on its own, in this order:
 *   d = conf * gamma                            (the decayed confidence)
 *   valid result, d > 0 and |cx - cx'|, |cy - cy'|, |r - r'| <= jump * W:
 *     w = d + score;  c = (d * c' + score * c) / w for c in cx, cy, r;
 *     conf = w                                  (confidence-weighted mean)
 *   valid result otherwise (first frame, or a jump: a new scene): the
 *     result's circle, conf = score
 *   invalid result with d > 0 and d >= t_hold: the previous circle held
 *     (valid, score 0, n_inliers 0), conf = d
 *   invalid result otherwise: invalid, the state cleared.
 * A valid output keeps the frame's score and n_inliers. */
typedef struct ca_smooth_params {
    float gamma;      /* confidence decay per frame, [0, 1); 0 = no memory */
    float jump;       /* scene-change distance, multiple of W, >= 0 */
    float t_hold;     /* least decayed confidence that holds a circle, >= 0 */
    int32_t reserved; /* must be 0 */
} ca_smooth_params;

/* Smooths B results (res_dev, device) of frames of widths W[i] (host) on
 * tracks track[i] (host, in [0, n_tracks), each at most once per call, or -1:
 * passed through) into out_dev (device, may equal res_dev), updating
 * state_dev (device, 4 x n_tracks floats).  Masks of the smoothed circles:
 * ca_mask on out_dev.  Queued on `stream`. */
ca_status ca_smooth_tracked(ca_handle *h, const ca_result *res_dev, int B, const int32_t *W,
                            const int32_t *track, int n_tracks, const ca_smooth_params *sp,
                            float *state_dev, ca_result *out_dev, void *stream);

/* The paper's own learned edge scorer (Sec. 2.2.4): three 3x3 convolutions
 * to 8, 16 and 32 features with ReLU, a 1x1 head and a sigmoid, on RGBXY
 * strips 7 rows high (unpadded vertically: the logits are those of the
 * strip's middle row; zero-padded horizontally), run on the tensor cores
 * (bf16 weights and activations, f32 accumulation).  Features: R, G, B as
 * (v - 128) / 128, then (x - (W-1)/2) / W and (row - (H-1)/2) / H.  The 7
 * rows of a strip at row y are y-3 .. y+3 clamped into the frame.
 * Parameters: CA_SCORER2D_NPARAM binary32 values, W1[8][5][3][3], b1[8],
 * W2[16][8][3][3], b2[16], W3[32][16][3][3], b3[32], wh[32], bh, with
 * conv[r][x][co] = b[co] + sum_{ci,dr,dx} W[co][ci][dr][dx] in[r+dr][x+dx-1][ci].
 *
 * With scorer_mode CA_SCORER_2D the candidates of every half-strip come from
 * the network's scores round(32768 p) of the strip's middle row (same pick
 * rule, K <= 16); with CA_SCORER_2D_FALLBACK a half-strip whose best score is
 * below 16384 (p < 1/2) keeps its handcrafted candidates.  Either mode needs
 * 2-D parameters (init, set or load) first. */
#define CA_SCORER2D_NPARAM 6209

/* Seeded initial parameters (He-normal convolutions, head weights N(0, 1/32),
 * head bias -3); resets the momentum. */
ca_status ca_scorer2d_init(ca_handle *h, uint64_t seed);
/* Copies n = CA_SCORER2D_NPARAM parameters in / out (host memory); set resets
 * the momentum. */
ca_status ca_scorer2d_set_params(ca_handle *h, const float *params, size_t n);
ca_status ca_scorer2d_get_params(ca_handle *h, float *params, size_t n);
/* Parameters and momentum to / from a file (little-endian: magic "CAS2",
 * version, count, then binary32 values). */
ca_status ca_scorer2d_save(ca_handle *h, const char *path);
ca_status ca_scorer2d_load(ca_handle *h, const char *path);

/* Forward pass on n strips: strips7_dev = n x 7 x W x 3 bytes (the 7 rows of
 * each strip, packed RGB), rows_dev = n x 7 frame rows of those rows (device),
 * frames of height H.  params_dev: CA_SCORER2D_NPARAM binary32 values in
 * device memory, or NULL for the handle's parameters.  Writes the n x W
 * logits (f32) and/or the Q15 scores round(32768 p) (either may be NULL).
 * Queued on `stream`. */
ca_status ca_scorer2d_forward(ca_handle *h, const uint8_t *strips7_dev, const int32_t *rows_dev,
                              int n, int W, int H, const float *params_dev, float *logits_dev,
                              uint16_t *scores_dev, void *stream);

/* One training step on the strips idx_dev[0 .. n-1] (device indices, or NULL
 * for strips 0 .. n-1) of a strip set as in ca_scorer2d_forward, with
 * targets_dev = per strip W soft targets in [0, 1] (the paper blurs its edge
 * map with a Gaussian of sigma 3).  Loss: the soft binary cross-entropy of the
 * columns, each weighted by 1 + (pos_weight - 1) t (pos_weight = 1: the
 * paper's unweighted loss), mean over the columns of the step; update as
 * ca_scorer_step.  Synchronous.  loss_host (may be NULL): the summed loss;
 * grads_host (may be NULL): the summed gradient (CA_SCORER2D_NPARAM values,
 * before the 1/columns scaling of the update). */
ca_status ca_scorer2d_step(ca_handle *h, const uint8_t *strips7_dev, const int32_t *rows_dev,
                           const float *targets_dev, const int32_t *idx_dev, int n, int W, int H,
                           const ca_train_params *tp, float *loss_host, float *grads_host);

/* `epochs` passes of steps of `batch` strips over the n strips, shuffled per
 * epoch by `seed`, with tp->lr_schedule as ca_scorer_train.  epoch_loss_host
 * (may be NULL) receives the mean loss per column of each epoch.
 * Synchronous. */
ca_status ca_scorer2d_train(ca_handle *h, const uint8_t *strips7_dev, const int32_t *rows_dev,
                            const float *targets_dev, int n, int W, int H,
                            const ca_train_params *tp, int epochs, int batch, uint64_t seed,
                            float *epoch_loss_host);

/* ---- Serving (no counterpart in the paper, which estimates one frame at a
 * time): frames of many video streams under continuous batching.
 *
 * A request is one frame of one stream.  ca_server_submit admits it when its
 * device buffers (the frame, and its mask when masks are kept) fit the
 * server's memory budget -- else CA_ERR_ADMISSION, and the caller submits it
 * again once results have been polled -- and queues its copy to the device.
 * Every ca_server_poll launches the admitted frames (at most one per stream
 * and max_batch per launch, oldest first) as one tracked estimate without
 * waiting for more frames or for earlier launches to finish, and returns the
 * results that have completed.  Each stream's previous result stays on the
 * device and, with `track`, its circle joins the stream's next RANSAC
 * (ca_estimate_tracked).  A stream's frames are estimated in submission
 * order, so a frame's result is the same whether its stream is served alone
 * or among others.  Times are seconds of ca_server_now()'s clock. */
typedef struct ca_server ca_server;

typedef struct ca_server_config {
    ca_params params;    /* estimation parameters of every frame */
    size_t mem_budget;   /* device bytes for the buffers of admitted frames */
    int32_t max_streams; /* stream ids 0 .. max_streams-1 */
    int32_t max_batch;   /* frames per launch */
    int32_t track;       /* 1: previous circle of each stream as an extra hypothesis */
    int32_t want_masks;  /* 1: write each frame's mask (copied to the host buffer
                            given at submit, if any) */
    int32_t smooth;      /* 1 (with track): each stream's results are smoothed
                            over time by ca_smooth_tracked with smooth_params
                            before they and their masks are returned */
    ca_smooth_params smooth_params;
    int32_t zero_copy;   /* 1: frames are never copied to the device.  Every
                            submitted frame must be page-locked host memory
                            (cudaHostAlloc, cudaHostRegister, pinned torch
                            tensors); the kernels read the strip rows they need
                            straight from it over the host link, and a
                            page-locked mask_host receives its mask directly.
                            Admission then counts only device masks. */
    int32_t reserved;    /* 0 */
} ca_server_config;

typedef struct ca_server_result {
    uint64_t ticket;     /* from ca_server_submit */
    int32_t stream_id;
    int32_t status;      /* CA_OK, or the error of a launch whose work was
                            already queued when a later step of it failed
                            (result zero; the stream's previous circle and
                            smoothing state are cleared) */
    uint64_t frame_key;
    ca_result result;
    double t_arrival;    /* as given at submit */
    double t_submit;     /* admitted */
    double t_launch;     /* its launch was queued */
    double t_done;       /* seen complete by a poll */
} ca_server_result;

/* Monotonic clock of the server, in seconds. */
double ca_server_now(void);

/* Creates a server on the handle's device (made current by this call) with
 * its own streams, a device pool of cfg->mem_budget bytes and the per-stream
 * state.  The handle must outlive the server. */
ca_status ca_server_create(ca_handle *h, const ca_server_config *cfg, ca_server **out);

/* Admits frame (H x W x 3 bytes of host memory; pinned memory makes the copy
 * asynchronous) of stream `stream_id` with RANSAC key `frame_key` and arrival
 * time `t_arrival`.  The frame buffer (and mask_host, H x W bytes or NULL)
 * must stay valid and unchanged until the frame's result has been polled.
 * Returns CA_ERR_ADMISSION, with nothing queued, when the budget is full.
 * With cfg.zero_copy the frame is not copied (it must be page-locked, else
 * CA_ERR_INVALID_ARG). */
ca_status ca_server_submit(ca_server *s, int stream_id, const uint8_t *frame_host, int H, int W,
                           uint64_t frame_key, double t_arrival, uint8_t *mask_host,
                           uint64_t *ticket);

/* One request of ca_server_submit_batch (the arguments of ca_server_submit). */
typedef struct ca_server_request {
    const uint8_t *frame_host;   /* H x W x 3 bytes of host memory */
    uint8_t *mask_host;          /* H x W bytes, or NULL */
    uint64_t frame_key;
    double t_arrival;
    int32_t stream_id;
    int32_t H, W;
    int32_t reserved;            /* 0 */
} ca_server_request;

/* Admits reqs[0 .. n-1] in order, as n calls of ca_server_submit would, in
 * one call.  Every request is checked before any is admitted
 * (CA_ERR_INVALID_ARG, nothing admitted).  Admission stops at the first
 * request the budget refuses: *n_admitted (required) receives how many were
 * admitted, tickets (n entries, may be NULL) their tickets, and the call
 * returns CA_ERR_ADMISSION if fewer than n were admitted. */
ca_status ca_server_submit_batch(ca_server *s, const ca_server_request *reqs, int n,
                                 uint64_t *tickets, int *n_admitted);

/* Launches what is admitted and returns up to `max` finished results (in
 * completion order).  wait != 0: if nothing has finished, blocks until the
 * oldest launch completes.  If a launch fails before any of its work is
 * queued (the estimate call returns an error), its requests go back to the
 * front of the queue in their order, the error is returned, and a later poll
 * launches them again. */
ca_status ca_server_poll(ca_server *s, int wait, ca_server_result *out, int max, int *n_done);

/* Bytes of the pool in use, admitted frames not yet launched, launches queued. */
ca_status ca_server_stats(const ca_server *s, size_t *bytes_in_use, int32_t *pending,
                          int32_t *launches_in_flight);

/* Waits for the server's work and frees it. */
ca_status ca_server_destroy(ca_server *s);

/* The server's admission allocator on its own (host bookkeeping only, no
 * device memory): first-fit offsets in [0, bytes), aligned to `align`,
 * adjacent free blocks merged.  CA_ERR_ADMISSION when no block fits. */
typedef struct ca_pool ca_pool;
ca_status ca_pool_create(size_t bytes, size_t align, ca_pool **out);
ca_status ca_pool_alloc(ca_pool *p, size_t bytes, size_t *offset);
ca_status ca_pool_free(ca_pool *p, size_t offset);
ca_status ca_pool_stats(const ca_pool *p, size_t *used, size_t *largest_free);
ca_status ca_pool_destroy(ca_pool *p);

/* Writes the content-area masks of B results (Sec. 1.1, Fig. 1): pixel (x, y)
 * is 1 iff (x-cx)^2 + (y-cy)^2 <= r^2 in binary32 (each operation rounded, no
 * fused multiply-add), or 1 everywhere when valid == 0.  res_dev: device array
 * of B results; H, W: host arrays of B sizes; masks_dev: host array of B
 * device pointers, each to H[i]*W[i] bytes. */
ca_status ca_mask(ca_handle *h, const ca_result *res_dev, int B, const int32_t *H,
                  const int32_t *W, uint8_t *const *masks_dev, void *stream);

/* End-to-end call on HOST buffers: copies B frames (B x H x W x 3 bytes, host)
 * to the device, estimates, and copies the B results (host) and, when
 * masks_host is not NULL, the B x H x W masks back.  Synchronous.  Pinned host
 * memory gives the fastest copies.  keys as in ca_estimate_uniform. */
ca_status ca_run_host(ca_handle *h, const uint8_t *frames_host, int B, int H, int W,
                      const uint64_t *keys, const ca_params *p, ca_result *res_host,
                      uint8_t *masks_host);

/* End-to-end call on page-locked HOST buffers without copying the frames:
 * the kernels read the strip rows they need straight from host memory (on
 * Grace-Blackwell over NVLink-C2C) and write the masks straight into
 * masks_host; only the B results are copied.  frames_host and masks_host
 * (when not NULL) must be page-locked (cudaHostAlloc / cudaHostRegister);
 * otherwise CA_ERR_INVALID_ARG.  Results and masks equal ca_run_host's.
 * With batch_mode CA_BATCH_AUTO the call runs the fused launch in waves of 4
 * frames with 8 threads per hypothesis (unless p sets hyp_threads or
 * wave_frames), so that the mask writes over the link, which bound the call,
 * start with the first frames and overlap the strip reads of the later ones.
 * Synchronous. */
ca_status ca_run_host_zero_copy(ca_handle *h, const uint8_t *frames_host, int B, int H, int W,
                                const uint64_t *keys, const ca_params *p, ca_result *res_host,
                                uint8_t *masks_host);

/* Waits for `stream` and reports any asynchronous device error raised by the
 * handle's kernels: CA_ERR_CUDA, or CA_ERR_TIMEOUT when a bounded wait of the
 * fused kernel gave up (its results are then not valid; the handle re-arms
 * itself and stays usable). */
ca_status ca_sync(ca_handle *h, void *stream);

/* Debug capture of the intermediate values of subsequent calls: 0 = off,
 * 1 = candidates, 2 = candidates and per-hypothesis records.  Capturing costs
 * extra device memory and writes; results are unchanged.  Level 3 (level 2
 * plus a test of the failure path): the fused launch withholds the signals
 * that release its mask work, so those waits run out after the wait limit and
 * the call reports CA_ERR_TIMEOUT through ca_sync; its masks are not valid. */
ca_status ca_set_debug(ca_handle *h, int level);

/* Bound on each dependency wait of the fused launch (nanoseconds, 1 ms to
 * 60 s; default 2 s).  Waits normally last microseconds. */
ca_status ca_set_wait_limit(ca_handle *h, uint64_t ns);

/* Host-side failure injection, for testing callers' error paths without any
 * device fault: after `after_calls` more estimates have been queued through
 * the handle (by ca_estimate, ca_estimate_uniform, ca_estimate_tracked,
 * ca_run_host*, the trials of ca_tune, or the launches of a server on it),
 * the next one returns `status` (a ca_status other than CA_OK) before it
 * queues any work, once.  status CA_OK disarms. */
ca_status ca_inject_failure(ca_handle *h, int after_calls, int status);

enum {
    /* per frame: int32 M, int32 n_slots(=N*K), then n_slots records of
     * {int16 x, int16 y, uint16 score, uint16 kept}: candidate slots in the
     * order (strip, left ranks, right ranks), of which the kept ones are the
     * frame's candidates in order */
    CA_DUMP_CANDIDATES = 1,
    /* per frame: int32 n_hyps, then n_hyps records of {int32 i0, i1, i2,
     * int32 n_inliers, uint32 score_sum, int32 passed, float cx, cy, r}
     * (circle relative to the origin (floor(W/2), floor(H/2))) */
    CA_DUMP_HYPOTHESES = 2,
    /* library-built tables for the given params: uint16 s_g table (5772),
     * s_theta table (8193), s_iota table (256), then int32 strip rows for
     * H = frame (pass the frame height as `frame`); host computation only,
     * h may be NULL and no device is needed */
    CA_DUMP_TABLES = 3,
    /* per frame: N x W uint16 learned scores of the last call (learned
     * scorer modes only) */
    CA_DUMP_LEARNED = 4,
    /* the whole last call (`frame` is not used; needs ca_set_trace and a
     * fused launch): int32 n_items, int32 0, then n_items records of four
     * uint64 {t_grab, t_ready, t_end, tag}, see ca_set_trace; a buffer too
     * small for the records receives the 8-byte header alone */
    CA_DUMP_TRACE = 5
};

/* Copies debug data of frame `frame` of the last ca_estimate call (synchronises
 * the handle's last stream).  *written receives the byte count. */
ca_status ca_debug_dump(ca_handle *h, int what, int frame, const ca_params *p,
                        void *host_buf, size_t bytes, size_t *written);

/* Number of kernel launches the handle has queued since creation. */
uint64_t ca_launch_count(const ca_handle *h);

/* Timeline of the fused launch: when on, every later fused call through
 * ca_estimate, ca_estimate_uniform or ca_estimate_tracked (not plans) records
 * for each work item (one strip, one tile of hypotheses, or one band of mask
 * rows, in the order the CTAs take them) four uint64 words: t_grab, the
 * %globaltimer nanoseconds when a CTA took the item; t_ready, when its
 * dependency wait ended (t_grab for strips); t_end, when its work ended; and
 * tag = phase << 48 | SM id << 32 | CTA index (phase 0 strips, 1 fit,
 * 2 mask).  Read with ca_debug_dump(CA_DUMP_TRACE).  Costs one 32-byte store
 * per item; results are unchanged. */
ca_status ca_set_trace(ca_handle *h, int on);

/* Kernel timing: when on, every later ca_estimate / ca_mask call records CUDA
 * events on its stream around each kernel it launches. */
ca_status ca_set_timing(ca_handle *h, int on);

/* Sums of the recorded kernel durations in milliseconds since the last read:
 * ms[0] strip scoring, ms[1] circle fitting, ms[2] mask writing, ms[3] the
 * fused kernel (all three phases), ms[4] the learned scorer's network;
 * counts[i] = launches timed.  Waits for the recorded events, then clears
 * them. */
ca_status ca_kernel_times(ca_handle *h, double ms[5], int32_t counts[5]);

const char *ca_status_string(ca_status s);
const char *ca_last_error(const ca_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* CA_H */
