// ca_internal.h -- structures shared by the host API (ca_api.cu) and the
// kernels (ca_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ca.h"

namespace ca {

constexpr int kMaxSlots = 256;       // N*K candidate slots per frame
constexpr int kMaxDim = 4096;        // W, H limit: keeps every moment sum inside int64
constexpr int kLutG = 5772;          // s_g table: floor(4|g|), |g| <= sqrt(2)*1020
constexpr int kLutT = 8193;          // s_theta table: floor(4096 (cos + 1))
constexpr int kLutI = 256;           // s_iota table: 8-bit preceding maximum
constexpr int kBoundBins = 1024;     // s_g upper bounds over bins of 16 values of |g|^2
// Device copy of the tables, 16-byte aligned pieces (uint16 offsets):
// [s_theta (8200)][s_iota (256)][s_g bin bounds (1024)][s_g (5776)].
constexpr int kDevOffT = 0;
constexpr int kDevOffI = 8200;
constexpr int kDevOffB = kDevOffI + kLutI;
constexpr int kDevOffG = kDevOffB + kBoundBins;
constexpr int kDevTableU16 = kDevOffG + 5776;
constexpr int kHypTile = 256;        // hypotheses per fit CTA (one per thread)
constexpr int kMaxHyps = 65536;      // random-mode hypotheses per frame
constexpr int kStripThreads = 256;   // strip CTA: 128 threads per half-strip
constexpr int kMaskRowsPerUnit = 8;  // mask work unit: 8 rows of one frame (one warp)

// One frame as the kernels see it (64 bytes).
struct DevFrame {
    const uint8_t *rgb;
    uint8_t *mask;
    int64_t pitch;
    uint64_t key;
    int32_t H, W;
    int32_t rows_off;   // offset of this frame's strip rows in the rows table
    int32_t unit_off;   // prefix sum of mask units before this frame
    int16_t vec_ok;     // 1: rgb, pitch and 3W are multiples of 16 bytes
    int16_t mask_vec_ok;// 2: mask pointer and W multiples of 32 bytes, 1: of 16, 0: neither
    int32_t mitem_off;  // prefix sum of fused-kernel mask items before this frame
    int32_t sc_seg_off; // learned scorer: prefix sum of its segments before this frame
    int32_t sc_pix_off; // learned scorer: offset of this frame's N x W pixel scores
};
static_assert(sizeof(DevFrame) == 64, "DevFrame layout");

// Fused kernel (k_batch): work items of three phases, numbered in one order in
// which every item comes after the items it depends on.  The order is a list
// of segments, each the items of one phase for frames [f0, f1).
enum { kPhaseStrips = 0, kPhaseFit = 1, kPhaseMask = 2 };
struct BatchSeg {
    int32_t start;    // index of the segment's first item
    int32_t phase;    // kPhase*
    int32_t f0, f1;   // frames
};
// Mask item: kStripThreads / 32 units of 8 rows of one frame.
constexpr int kMaskUnitsPerItem = kStripThreads / 32;
__host__ __device__ inline int mask_items_of(int H) {
    const int units = (H + kMaskRowsPerUnit - 1) / kMaskRowsPerUnit;
    return (units + kMaskUnitsPerItem - 1) / kMaskUnitsPerItem;
}
// Strip items per frame: one strip (both halves) for K = 2, four strips for K > 2.
__host__ __device__ inline int strip_items_of(int N, int K) { return K == 2 ? N : (N + 3) / 4; }

// Synchronisation words of the fused kernel: [0] next item, [1] CTAs that
// have finished, [2] error flags, [3] unused, then per frame: result ready,
// mask items done.  Every word returns to 0 by the end of a call that
// completes without error.  (A fit item learns that the strips of its frame
// are done from their candidate slots themselves: kSlotFresh below.)
constexpr int kSyncGlobal = 4;
constexpr uint32_t kSyncErrTimeout = 1u;
__host__ __device__ inline uint32_t *sync_ready(uint32_t *s, int nf) { return s + kSyncGlobal; }
__host__ __device__ inline uint32_t *sync_maskdone(uint32_t *s, int nf) {
    return s + kSyncGlobal + nf;
}
__host__ __device__ inline size_t sync_words(int nf) { return kSyncGlobal + 2 * (size_t)nf; }

// Per-call constants, passed by value (kernel parameter space).
struct DevParams {
    int32_t N, K, NH, refine;
    int32_t T_px, sup_px, hyp_mode, debug;
    uint32_t T_ps, T_cs;   // T_cs: with norm_circle, computed per frame instead
    int32_t qg_sat;      // first index from which the s_g table stays at 32768
    int32_t n_tiles;     // fit CTAs per frame (each 256 / hyp_threads hypotheses)
    float t_ri, r_min, r_max, d_max;
    double score_den;    // 32768 * normaliser (fixed normalisers)
    double tcs_unit;     // t_cs * 32768 (circle normaliser: threshold = ceil(tcs_unit * K n))
    int32_t norm_circle; // 1: normaliser K n, n = strips the best circle crosses
    const int32_t *rows_tab;   // the call's strip-row table (DevFrame::rows_off)
    uint64_t seed;
    int32_t max_w;       // widest frame of the call (shared-memory sizing)
    int32_t hyp_threads; // threads per hypothesis in k_fit: 1, 2, 4 or 8
    int32_t io_cut;      // preceding maxima >= io_cut have s_iota < T_ps: never kept
    int32_t track;       // 1: tracked call (previous circles as extra hypotheses)
    int32_t prior_centre;  // tracked call: the angle term points at the previous centre
    int32_t theta_cut_on;  // 1: pixels whose angle bin has s_theta < T_ps are skipped
    float theta_u_cut;     // their signed squared cosines are below this (margin included)
    const int32_t *trk;          // tracked call: [B] track of each frame (-1: none)
    const ca_result *trk_state;  // tracked call: per-track previous result
};

// A candidate slot (8 bytes): x, y, Q15 score, flags.  Flag kSlotKept: the
// point is a candidate.  Flag kSlotFresh: written by the current call and not
// yet consumed; the fit tile that completes the frame clears it.  A slot is
// stored and loaded as one 64-bit word, so a reader that sees kSlotFresh sees
// the rest of that write too.
struct CandSlot {
    int16_t x, y;
    uint16_t s, kept;
};
constexpr uint16_t kSlotKept = 1u, kSlotFresh = 2u;

__device__ __forceinline__ unsigned long long slot_bits(CandSlot v) {
    return (unsigned long long)(uint16_t)v.x | ((unsigned long long)(uint16_t)v.y << 16) |
           ((unsigned long long)v.s << 32) | ((unsigned long long)v.kept << 48);
}
__device__ __forceinline__ CandSlot slot_of(unsigned long long b) {
    CandSlot v;
    v.x = (int16_t)(b & 0xFFFFu);
    v.y = (int16_t)((b >> 16) & 0xFFFFu);
    v.s = (uint16_t)((b >> 32) & 0xFFFFu);
    v.kept = (uint16_t)(b >> 48);
    return v;
}
// Writes slot *p of the current call (kSlotFresh set) in one store.
__device__ __forceinline__ void store_slot(CandSlot *p, CandSlot v) {
    v.kept = (uint16_t)(v.kept | kSlotFresh);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(slot_bits(v)) : "memory");
}
__device__ __forceinline__ unsigned long long load_slot_bits(const CandSlot *p) {
    unsigned long long b;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
    return b;
}

// Best circle of one fit CTA.
struct TileRec {
    float cx, cy, r;
    int32_t n_inl;
    uint32_t S;
    int32_t pad[3];
};

// Debug record of one hypothesis (matches CA_DUMP_HYPOTHESES).
struct HypRec {
    int32_t i0, i1, i2, n_inl;
    uint32_t S;
    int32_t pass;
    float cx, cy, r;
};

// Device workspace of one handle.
struct Workspace {
    CandSlot *slots = nullptr;       // [B][kMaxSlots]
    TileRec *tiles = nullptr;        // [B][n_tiles]
    unsigned long long *best = nullptr; // [B] packed best key, reset after use
    uint32_t *done = nullptr;        // [B] finished fit CTAs, reset after use
    HypRec *hyps = nullptr;          // [B][NH] when debug level 2
    int32_t *n_hyps = nullptr;       // [B]
    int32_t *n_cands = nullptr;      // [B]
    uint32_t *sync = nullptr;        // sync_words(sync_frames), fused kernel
    int32_t sync_frames = 0;
    const int32_t *track = nullptr;  // tracked call: [B] track of each frame (-1: none)
    ca_result *state = nullptr;      // tracked call: per-track previous result
    unsigned long long *trace = nullptr;   // fused kernel timeline: 4 words per item (or none)
    int32_t trace_cap = 0;                 // items the trace buffer holds
};

// ---- Learned edge scorer (ca_scorer.cu): 1-D CNN over strip profiles.
constexpr int kScCin = 14, kScCh = 32, kScTaps = 7;
constexpr int kScHalo = 9;                       // 3 layers x 3 columns of context
constexpr int kScInferTiles = 3, kScTrainTiles = 4;   // 128-column tiles per segment
constexpr int kScSegOutInfer = 128 * kScInferTiles - 2 * kScHalo;   // output columns per segment
constexpr int kScSegOutTrain = 128 * kScTrainTiles - 2 * kScHalo;
constexpr int kScNParam = 17601;                 // flat parameter count (see ca.h)
constexpr int kScMaxPicks = 8;                   // K/2 limit with the learned scorer
constexpr uint32_t kScErrTimeout = 2u;
// parameter offsets in the flat vector: W1[32][14][7], b1, W2[32][32][7], b2, W3, b3, wh, bh
constexpr int kScPW1 = 0, kScPB1 = 3136, kScPW2 = 3168, kScPB2 = 10336, kScPW3 = 10368,
              kScPB3 = 17536, kScPWh = 17568, kScPBh = 17600;
// packed device weight block (bytes): bf16 B operands of the forward convolutions
// ([tap x input chunk][32 out][8 in]), of the input-gradient convolutions of
// layers 2-3 ([tap x output chunk][32 in][8 out], taps reversed), then floats
constexpr int kScOffW1f = 0, kScOffW2f = 7168, kScOffW3f = 21504, kScOffW2b = 35840,
              kScOffW3b = 50176, kScOffVec = 64512;
constexpr int kScFwdBytes = 35840, kScVecBytes = 528, kScBlockBytes = 65040;
constexpr int kScPartialStride = 17664;          // per-CTA gradient partials (+ loss at kScNParam)
constexpr int kScSgdBlocks = 276;                // reduction blocks of 64 parameters (+ loss slot)

// Rows of the strips a scorer launch reads: either frames (rows from the
// strip-row table) or stand-alone strips (3 rows x W x 3 bytes each).
struct ScSource {
    const DevFrame *frames;   // frames mode
    int B;
    const int32_t *rows;
    int N;
    const uint8_t *strips;    // strips mode (frames == nullptr)
    const int32_t *ys;        // middle row of each strip in its frame
    const int32_t *idx;       // strips mode: optional index list of the strips to use
    int n, W, H;
};

cudaError_t sc_launch_pack(const float *params, unsigned char *block, cudaStream_t s);
size_t sc_infer_smem();
int sc_infer_blocks_per_sm();
cudaError_t sc_launch_infer(const ScSource &src, const unsigned char *block, uint16_t *scores,
                            float *logits, int total_segs, uint32_t *err, int grid, cudaStream_t s);
cudaError_t sc_launch_pick(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                           const uint16_t *scores, int fallback, CandSlot *slots, int grid,
                           cudaStream_t s);
size_t sc_train_smem();
cudaError_t sc_launch_train(const ScSource &src, const uint8_t *labels, float pos_weight,
                            const unsigned char *block, float *partial, int total_segs,
                            uint32_t *err, int grid, cudaStream_t s);
// One SGD step from the partials (two launches when clip > 0 and apply;
// gbuf: kScNParam floats, norm_part: kScSgdBlocks floats of scratch).  With
// apply, the updated weights are also written into `block`.
cudaError_t sc_launch_sgd(float *params, float *mom, float *partial, int n_partials, float scale,
                          float lr, float momentum, int apply, float clip, float *gbuf,
                          float *norm_part, float *grads_out, float *loss_out,
                          unsigned char *block, cudaStream_t s);

// ---- The paper's 2-D scorer (ca_scorer2d.cu, Sec. 2.2.4): 3x3 convolutions
// to 8, 16, 32 features over 7-row RGBXY strips, on tcgen05.
constexpr int kScorer2dNParam = 6209;
constexpr int kSc2Tiles = 3;                               // 128-column tiles per segment
constexpr int kSc2Halo = 3;                                // one column of context per layer
constexpr int kSc2SegOut = 128 * kSc2Tiles - 2 * kSc2Halo; // output columns per segment
// parameter offsets: W1[8][5][3][3], b1, W2[16][8][3][3], b2, W3[32][16][3][3], b3, wh, bh
constexpr int kSc2PW1 = 0, kSc2PB1 = 360, kSc2PW2 = 368, kSc2PB2 = 1520, kSc2PW3 = 1536,
              kSc2PB3 = 6144, kSc2PWh = 6176, kSc2PBh = 6208;
// packed device weight block (bytes): bf16 B operands of the forward
// convolutions (L1, L2: per row tap and column-tap pair [2 chunks][16 out][8 in];
// L3: per tap [2 chunks][32 out][8 in]), of the input-gradient convolutions
// (W3 transposed: per tap [4 chunks of 8 out][16 in][8]; W2 transposed: per
// tap [2 chunks][16 (8 real) in][8]), then floats
constexpr int kSc2OffW1 = 0, kSc2OffW2 = 3072, kSc2OffW3 = 6144, kSc2OffW3b = 15360,
              kSc2OffW2b = 24576, kSc2OffVec = 29184;
constexpr int kSc2FwdBytes = 15360, kSc2VecBytes = 384, kSc2BlockBytes = 29568;
constexpr int kSc2PartialStride = 6272;   // per-CTA gradient partials (+ loss at kScorer2dNParam)
constexpr int kSc2SgdBlocks = (kScorer2dNParam + 1 + 63) / 64;

// Strips the 2-D scorer reads: frames (the 7 rows around each strip row of the
// strip-row table, clamped into the frame) or stand-alone 7-row strips.
struct Sc2Source {
    const DevFrame *frames;   // frames mode (segments numbered by DevFrame::sc_seg_off)
    int B;
    const int32_t *rows;
    int N;
    const uint8_t *strips7;   // strips mode (frames == nullptr): n x 7 x W x 3 bytes
    const int32_t *rows7;     // n x 7 frame rows of the strips' rows
    const int32_t *idx;       // optional index list of the strips to use
    int n, W, H;
};

cudaError_t sc2_launch_pack(const float *params, unsigned char *block, cudaStream_t s);
size_t sc2_infer_smem();
int sc2_infer_blocks_per_sm();
cudaError_t sc2_launch_infer(const Sc2Source &src, const unsigned char *block, uint16_t *scores,
                             float *logits, int total_segs, uint32_t *err, int grid,
                             cudaStream_t s);
size_t sc2_train_smem();
cudaError_t sc2_launch_train(const Sc2Source &src, const float *targets, float pos_weight,
                             const unsigned char *block, float *partial, int total_segs,
                             uint32_t *err, int grid, cudaStream_t s);
// As sc_launch_sgd, for the 2-D scorer (gbuf: kScorer2dNParam floats,
// norm_part: kSc2SgdBlocks floats).
cudaError_t sc2_launch_sgd(float *params, float *mom, float *partial, int n_partials, float scale,
                           float lr, float momentum, int apply, float clip, float *gbuf,
                           float *norm_part, float *grads_out, float *loss_out,
                           unsigned char *block, cudaStream_t s);

// Kernel launchers (ca_kernels.cu).  Each returns the CUDA error of the launch.

// Temporal smoothing of B results (one thread per frame); w_trk: [B] pairs
// (W, track) on the device.
cudaError_t launch_smooth(const ca_result *res, int B, const int32_t *w_trk, float gamma,
                          float jump, float t_hold, float *state, ca_result *out, cudaStream_t s);

cudaError_t launch_strips(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                          const uint16_t *luts, CandSlot *slots, int grid, cudaStream_t s);
cudaError_t launch_fit(const DevFrame *frames, int B, const DevParams &P, CandSlot *slots,
                       const Workspace &ws, ca_result *out, cudaStream_t s);
cudaError_t launch_mask(const DevFrame *frames, int B, const ca_result *res, int total_units,
                        int grid, cudaStream_t s);
// Fused persistent kernel: every phase of B frames in one launch of `grid`
// CTAs (see ca_kernels.cu).  Waits give up after wait_ns nanoseconds.
cudaError_t launch_batch(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                         const uint16_t *luts, const Workspace &ws, ca_result *out,
                         const BatchSeg *segs, int n_segs, int total_items, int grid,
                         uint64_t wait_ns, cudaStream_t s);
size_t batch_smem_bytes(const DevParams &P);
int batch_blocks_per_sm(int hyp_threads, size_t smem);   // occupancy of k_batch
int mask_blocks_per_sm();   // resident k_mask CTAs per SM (occupancy), cached
int fit_threads_per_sm(int hyp_threads);   // resident k_fit threads per SM, cached
// Threads per hypothesis for B frames of NH hypotheses on `sms` SMs.
int choose_hyp_threads(int requested, long long B, long long NH, int sms);
size_t strips_smem_bytes(const DevParams &P);
cudaError_t strips_occupancy(int *blocks_per_sm, size_t smem);

// Host helpers (ca_api.cu).
int handle_device(const ca_handle *h);                            // the handle's CUDA device
void strip_rows(int H, int N, float alpha, int32_t *rows);        // Eq. 1 rows
void build_luts(const ca_params &p, uint16_t *out, int *qg_sat);  // Eq. 2 tables
ca_status check_params(ca_handle *h, const ca_params *p);         // h may be NULL
int iota_cut(const uint16_t *li, uint32_t T_ps);                  // see ca_api.cu
void angle_cut(const uint16_t *lt, uint32_t T_ps, DevParams &P);  // see ca_api.cu
// Device table block (kDevTableU16 entries) from build_luts' [s_g][s_theta][s_iota].
void pack_device_tables(const uint16_t *luts, int qg_sat, uint16_t *out);

}  // namespace ca
