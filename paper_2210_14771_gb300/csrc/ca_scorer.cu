// ca_scorer.cu -- learned edge scorer: a 1-D convolutional network over strip
// profiles (the learned variant of Sec. 2.2.4, here with 1-D convolutions over
// 3-row strips), run on the 5th-generation tensor cores (tcgen05) with bf16
// operands and f32 accumulators in tensor memory.
//
// Network, per strip column x (W columns, "same" zero padding):
//   features f[x] (14): luma, R, G, B of rows y-1, y, y+1 as (v - 128) / 128,
//                       then (x - (W-1)/2) / W and (y - (H-1)/2) / H
//   a1 = relu(conv7(f,  W1) + b1), a2 = relu(conv7(a1, W2) + b2),
//   a3 = relu(conv7(a2, W3) + b3)          (32 channels, kernel 7 each)
//   logit = bh + wh . a3,  p = sigmoid(logit)
// with conv7(in, W)[x][co] = sum_{ci,t} W[co][ci][t] in[x + t - 3][ci].
// Activations and weights are stored in bf16, every sum accumulates in f32.
//
// Layout.  A strip is processed in segments of 512 consecutive columns (4
// tiles of 128), of which the middle 494 are outputs: three layers of kernel
// 7 need 9 columns of context on each side.  Activations of a segment live in
// shared memory as "planes": plane c holds channels 8c..8c+7 of every column,
// one 16-byte row per column, with 8 zero guard rows at both ends.  A tile of
// 128 columns and 16 channels is then a K-major tcgen05 operand (core
// matrices of 8 columns x 8 channels = 128 contiguous bytes; SBO = 128 bytes
// between 8-column groups, LBO = one plane between channel groups), and the
// column shift t - 3 of a convolution tap is only a 16-byte offset of the
// operand's start address: the 7 taps need no im2col copy.  The same planes
// read as MN-major operands (channels contiguous, columns as K) give the
// weight gradients: dW[co][ci][t] = sum_x dz[x][co] a[x + t - 3][ci].
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "ca_internal.h"

namespace ca {

namespace {

constexpr int kCh = kScCh, kTaps = kScTaps;
constexpr int kTile = 128;
constexpr int kGuard = 8;

// Segment geometry: TILES tiles of 128 columns, of which all but 9 columns of
// context at each end are outputs.
template <int TILES>
struct SegGeom {
    static constexpr int kTiles = TILES;
    static constexpr int kRows = kTile * TILES;
    static constexpr int kPlane = (kRows + 2 * kGuard) * 16;   // bytes of one channel plane
    static constexpr int kOut = kRows - 2 * kScHalo;
};
using SegI = SegGeom<kScInferTiles>;   // inference
using SegT = SegGeom<kScTrainTiles>;   // training
static_assert(SegI::kOut == kScSegOutInfer && SegT::kOut == kScSegOutTrain, "segment sizes");

#include "ca_tc.cuh"

// Writes the 32 values of a row into 4 planes (bf16).
template <class G>
__device__ __forceinline__ void store_row32(unsigned char *planes, int row, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 q;
        q.x = pack_bf16(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_bf16(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_bf16(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_bf16(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(planes + c * G::kPlane + (kGuard + row) * 16) = q;
    }
}

template <class G>
__device__ __forceinline__ void load_row32(const unsigned char *planes, int row, float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint4 q = *reinterpret_cast<const uint4 *>(planes + c * G::kPlane + (kGuard + row) * 16);
        v[8 * c + 0] = bf16_lo(q.x); v[8 * c + 1] = bf16_hi(q.x);
        v[8 * c + 2] = bf16_lo(q.y); v[8 * c + 3] = bf16_hi(q.y);
        v[8 * c + 4] = bf16_lo(q.z); v[8 * c + 5] = bf16_hi(q.z);
        v[8 * c + 6] = bf16_lo(q.w); v[8 * c + 7] = bf16_hi(q.w);
    }
}

// Sum over the warp of each of 32 per-lane values: lane c receives channel c.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < o; ++k) {
            const float send = upper ? v[k] : v[k + o];
            const float keep = upper ? v[k + o] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__device__ __forceinline__ float luma_f(uint32_t r, uint32_t g, uint32_t b) {
    return (float)((int)((77u * r + 150u * g + 29u * b + 128u) >> 8) - 128) * (1.0f / 128.0f);
}

// Column features of a segment: rows r in [0, 512) <-> columns b0 + r; two
// planes (14 features + 2 zero channels), zero outside [0, W).  Pixel x of
// row k is read at row_k + 3 x - bias (bias 0 for the strip rows themselves,
// the staged block's start for a copy in shared memory).
template <class G>
__device__ __forceinline__ void build_features(unsigned char *x0, const uint8_t *row0,
                                               const uint8_t *row1, const uint8_t *row2, int W,
                                               int y, int H, int b0, int bias = 0) {
    const float yf = __fdiv_rn(__fsub_rn((float)y, __fmul_rn(0.5f, (float)(H - 1))), (float)H);
    const float xc = __fmul_rn(0.5f, (float)(W - 1));
    const float Wf = (float)W;
    for (int r = threadIdx.x; r < G::kRows; r += blockDim.x) {
        const int x = b0 + r;
        uint4 q0 = make_uint4(0, 0, 0, 0), q1 = make_uint4(0, 0, 0, 0);
        if (x >= 0 && x < W) {
            float f[16];
            const int o = 3 * x - bias;
            const uint8_t *p[3] = {row0 + o, row1 + o, row2 + o};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint32_t R = p[k][0], Gr = p[k][1], B = p[k][2];
                f[4 * k + 0] = luma_f(R, Gr, B);
                f[4 * k + 1] = (float)((int)R - 128) * (1.0f / 128.0f);
                f[4 * k + 2] = (float)((int)Gr - 128) * (1.0f / 128.0f);
                f[4 * k + 3] = (float)((int)B - 128) * (1.0f / 128.0f);
            }
            f[12] = __fdiv_rn(__fsub_rn((float)x, xc), Wf);
            f[13] = yf;
            f[14] = f[15] = 0.0f;
            q0 = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                            pack_bf16(f[6], f[7]));
            q1 = make_uint4(pack_bf16(f[8], f[9]), pack_bf16(f[10], f[11]), pack_bf16(f[12], f[13]),
                            pack_bf16(f[14], f[15]));
        }
        *reinterpret_cast<uint4 *>(x0 + (kGuard + r) * 16) = q0;
        *reinterpret_cast<uint4 *>(x0 + G::kPlane + (kGuard + r) * 16) = q1;
    }
}

// Issues one convolution of a segment (single thread): for each tile j and
// tap t, MMAs over channel pairs of planes; D of tile j = columns 32 j.
//   in: planes of the input (n_in_chunks = 2 or 4), w: weight chunks
//   [t * n_in_chunks + c][32 out][8 in] (512 bytes each).
template <class G, int NIN>
__device__ __forceinline__ void issue_conv(uint32_t tmem, const unsigned char *in,
                                           const unsigned char *w) {
    // base descriptors; an operand's start address is bits 0-13 (16-byte
    // units), so a byte offset d moves it by adding d >> 4
    constexpr uint32_t idesc = idesc_bf16(128, 32, false, false);
    const uint64_t da = sdesc(smem_u32(in) + (kGuard - 3) * 16, G::kPlane, 128);
    const uint64_t db = sdesc(smem_u32(w), 512, 128);
#pragma unroll
    for (int j = 0; j < G::kTiles; ++j)
#pragma unroll
        for (int t = 0; t < kTaps; ++t)
#pragma unroll
            for (int q = 0; q < NIN / 2; ++q) {
                const uint32_t ao = (2 * q * G::kPlane + (kTile * j + t) * 16) >> 4;
                const uint32_t bo = ((t * NIN + 2 * q) * 512) >> 4;
                mma_bf16(tmem + 32 * j, da + ao, db + bo, idesc, (t | q) != 0);
            }
}

struct ScVec {   // float part of the weight block
    float b[3][kCh];
    float whq[kCh];   // head weights rounded to bf16
    float bh;
    float pad[3];
};
static_assert(sizeof(ScVec) == kScVecBytes, "vector block size");

// Epilogue helper: the 32 accumulator channels of row r = 128 j + 32 q + lane,
// q = warp % 4 (a warp can only read its own quarter of the TMEM lanes).
__device__ __forceinline__ void acc_row(uint32_t tmem, int j, float (&v)[32]) {
    const int q = (threadIdx.x >> 5) & 3;
    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32 * j, v);
}

// Where segment g of a launch reads and writes.
struct SegInfo {
    const uint8_t *r0;   // row y-1 of the strip (rows y, y+1 follow at `pitch`)
    int64_t pitch;
    int W, H, y;
    int s0, s1;          // output columns [s0, s1)
    int64_t out;         // index of column 0 of the strip in the per-column outputs
    int strip;           // strips mode: index of the strip in the source
};

template <class G>
__device__ __forceinline__ SegInfo seg_info(const ScSource &src, int g) {
    SegInfo si;
    if (src.frames) {
        int lo = 0, hi = src.B - 1;   // frame of segment g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (src.frames[mid].sc_seg_off <= g) lo = mid;
            else hi = mid - 1;
        }
        const DevFrame &fr = src.frames[lo];
        const int nseg = (fr.W + G::kOut - 1) / G::kOut;
        const int local = g - fr.sc_seg_off;
        const int i = local / nseg, s = local - i * nseg;
        si.y = src.rows[fr.rows_off + i];
        si.W = fr.W;
        si.H = fr.H;
        si.pitch = fr.pitch;
        si.r0 = fr.rgb + (int64_t)(si.y - 1) * fr.pitch;
        si.s0 = s * G::kOut;
        si.out = (int64_t)fr.sc_pix_off + (int64_t)i * fr.W;
        si.strip = -1;
    } else {
        const int nseg = (src.W + G::kOut - 1) / G::kOut;
        const int j = g / nseg, s = g - j * nseg;
        const int id = src.idx ? src.idx[j] : j;
        si.y = src.ys[id];
        si.W = src.W;
        si.H = src.H;
        si.pitch = (int64_t)src.W * 3;
        si.r0 = src.strips + (int64_t)id * 3 * si.pitch;
        si.s0 = s * G::kOut;
        si.out = (int64_t)j * src.W;
        si.strip = id;
    }
    si.s1 = min(si.W, si.s0 + G::kOut);
    return si;
}

// L2 prefetch (TMA) of the strip rows a segment reads: the bytes of columns
// [b0, b0 + rows) of rows y-1, y, y+1, shrunk to whole 16-byte blocks inside
// each row (a hint: the loads of the segment read the same bytes).
template <class G>
__device__ __forceinline__ void prefetch_rows(const SegInfo &si) {
    const int c0 = max(si.s0 - kScHalo, 0), c1 = min(si.s0 - kScHalo + G::kRows, si.W);
    if (c1 <= c0) return;
    for (int r = 0; r < 3; ++r) {
        const uint8_t *row = si.r0 + r * si.pitch;
        const uintptr_t a = ((uintptr_t)(row + 3 * c0) + 15) & ~(uintptr_t)15;
        const uintptr_t b = (uintptr_t)(row + 3 * c1) & ~(uintptr_t)15;
        if (b > a)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                         : "memory");
    }
}

// Staging of a segment's strip bytes in shared memory by cp.async (16-byte
// asynchronous copies), issued one segment ahead.  Possible when the copies
// stay inside each row: rows start on 16-byte boundaries and 3 W is a
// multiple of 16 (then the 16-byte blocks around columns [c0, c1) lie in
// [row, row + 3 W)).  Row k of the segment lands at stage + k kStageRow.
constexpr int kStageRow = 1200;   // >= 3 x 384 columns + 30 bytes of alignment, 16 x 75

__device__ __forceinline__ bool stageable(const SegInfo &si) {
    return (((uintptr_t)si.r0 | (uintptr_t)si.pitch | (uintptr_t)(3 * si.W)) & 15) == 0;
}

// First byte (a multiple of 16, relative to the row) of the staged block.
template <class G>
__device__ __forceinline__ int stage_bias(const SegInfo &si) {
    return (3 * max(si.s0 - kScHalo, 0)) & ~15;
}

template <class G>
__device__ __forceinline__ void stage_rows(unsigned char *stage, const SegInfo &si) {
    static_assert(3 * G::kRows + 30 <= kStageRow, "a staged row fits its slot");
    const int c0 = max(si.s0 - kScHalo, 0), c1 = min(si.s0 - kScHalo + G::kRows, si.W);
    const int a = stage_bias<G>(si), b = (3 * c1 + 15) & ~15;
    const int nb = c1 > c0 ? (b - a) >> 4 : 0;   // 16-byte blocks per row
    for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) {
        const int k = i / nb, j = i - k * nb;
        const uint8_t *src = si.r0 + k * si.pitch + a + 16 * j;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         smem_u32(stage + k * kStageRow + 16 * j)),
                     "l"(src)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Zeroes the guard rows (8 above and 8 below the segment) of `n_planes`
// consecutive planes from `planes`.
template <class G>
__device__ __forceinline__ void zero_guards(unsigned char *planes, int n_planes) {
    for (int i = threadIdx.x; i < n_planes * kGuard * 2; i += blockDim.x) {
        const int plane = i / (2 * kGuard), g = i % (2 * kGuard);
        const int row = g < kGuard ? g : G::kRows + g;   // rows [0, 8) and [520, 528)
        *reinterpret_cast<uint4 *>(planes + plane * G::kPlane + row * 16) = make_uint4(0, 0, 0, 0);
    }
}

// Common prologue of the scorer kernels: zero guard rows of `n_planes`
// planes from `sm`, init the barriers, allocate TMEM, start the weight copy.
template <class G>
__device__ __forceinline__ uint32_t sc_prologue(unsigned char *sm, int n_planes, uint64_t *bar_w,
                                                uint64_t *bar_m, uint32_t *tslot, uint32_t ncols,
                                                unsigned char *wdst, const unsigned char *wsrc,
                                                uint32_t wbytes, void *vdst, const void *vsrc) {
    const int tid = threadIdx.x, warp = tid >> 5;
    zero_guards<G>(sm, n_planes);
    if (tid == 0) {
        bar_init(bar_w, 1);
        bar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, ncols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
        bar_expect_tx(bar_w, wbytes + kScVecBytes);
        bulk_g2s(wdst, wsrc, wbytes, bar_w);
        bulk_g2s(vdst, vsrc, kScVecBytes, bar_w);
    }
    return *tslot;
}

}  // namespace

// ============================================================ inference ==
// One CTA (4 warps) per 512-column segment at a time, 2 CTAs per SM.  Output:
// the Q15 score round(32768 p) of every output column, and the logit when
// `logits` is set.
constexpr int kInfThreads = 256;   // 8 warps: two per TMEM lane quarter
constexpr size_t kInfSmem = 6 * (size_t)SegI::kPlane + kScFwdBytes + kScVecBytes + 64;

__global__ void __launch_bounds__(kInfThreads, 3)
    k_sc_infer(ScSource src, const unsigned char *__restrict__ wblock, uint16_t *__restrict__ scores,
               float *__restrict__ logits, int total_segs, uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *X0 = sm;                       // 2 planes: features
    unsigned char *A = sm + 2 * SegI::kPlane;      // 4 planes: a1, then a2 (in place)
    unsigned char *Wf = A + 4 * SegI::kPlane;
    ScVec *vec = reinterpret_cast<ScVec *>(Wf + kScFwdBytes);
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(vec) + kScVecBytes);
    uint64_t *bar_m = bar_w + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t tmem = sc_prologue<SegI>(sm, 6, bar_w, bar_m, tslot, 128, Wf, wblock + kScOffW1f,
                                      kScFwdBytes, vec, wblock + kScOffVec);
    bool abort = __syncthreads_or(!bar_wait(bar_w, 0, err)) != 0;
    uint32_t phase = 0;
    // Staged strip bytes of the next segment: in the interior rows of the
    // first a1/a2 plane, free from the end of the last convolution of a
    // segment until the first epilogue of the next one.
    static_assert(3 * kStageRow <= SegI::kRows * 16, "staging fits the interior rows of a plane");
    unsigned char *stage = A + kGuard * 16;
    bool staged = false;   // this segment's bytes are in `stage`

    // where the current and the next segment of this CTA read and write: the
    // next one's (a search over the frames) is looked up while the current
    // segment's first convolution runs
    SegInfo si, sn;
    if ((int)blockIdx.x < total_segs) si = seg_info<SegI>(src, blockIdx.x);
    for (int g = blockIdx.x; g < total_segs && !abort; g += gridDim.x) {
        const int b0 = si.s0 - kScHalo;
        const bool has_next = g + (int)gridDim.x < total_segs;
        __syncthreads();   // the previous segment is done with A and X0
        if (staged) {
            stage_wait();
            __syncthreads();
            build_features<SegI>(X0, stage, stage + kStageRow, stage + 2 * kStageRow, si.W, si.y,
                                 si.H, b0, stage_bias<SegI>(si));
        } else {
            build_features<SegI>(X0, si.r0, si.r0 + si.pitch, si.r0 + 2 * si.pitch, si.W, si.y,
                                 si.H, b0);
        }
        staged = false;
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        for (int l = 0; l < 3; ++l) {
            if (tid == 0) {
                const int woff = l == 0 ? 0 : (l == 1 ? kScOffW2f : kScOffW3f) - kScOffW1f;
                if (l == 0) issue_conv<SegI, 2>(tmem, X0, Wf + woff);
                else issue_conv<SegI, 4>(tmem, A, Wf + woff);
                mma_commit(bar_m);
            }
            if (l == 0 && has_next) {   // this CTA's next segment
                sn = seg_info<SegI>(src, g + gridDim.x);
                if (tid == 0) prefetch_rows<SegI>(sn);
            }
            const bool ok = bar_wait(bar_m, phase, err);
            phase ^= 1u;
            tc_after_sync();
            if (__syncthreads_or(!ok)) { abort = true; break; }
            if (l == 2 && has_next) {   // the MMAs are done with A
                if (stageable(sn)) {
                    stage_rows<SegI>(stage, sn);
                    staged = true;
                }
            }
            for (int j = warp >> 2; j < SegI::kTiles; j += 2) {   // warp w: tiles w/4, w/4 + 2
                float v[32];
                acc_row(tmem, j, v);
                const int r = kTile * j + 32 * (warp & 3) + (tid & 31);
                const int x = b0 + r;
                const bool inside = x >= 0 && x < si.W;
                // relu(z + b) rounded to bf16, two channels per conversion;
                // zero outside the strip
                uint32_t w[16];
                const float *bl = vec->b[l];
                if (inside) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        w[c] = pack_relu_bf16(__fadd_rn(v[2 * c], bl[2 * c]),
                                              __fadd_rn(v[2 * c + 1], bl[2 * c + 1]));
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c) w[c] = 0u;
                }
                if (l < 2) {   // every MMA reading A has completed: overwrite in place
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        *reinterpret_cast<uint4 *>(A + c * SegI::kPlane + (kGuard + r) * 16) =
                            make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                } else if (x >= si.s0 && x < si.s1) {
                    // head: fused multiply-adds over the bf16 activations
                    float acc = 0.0f;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        acc = __fmaf_rn(vec->whq[2 * c], bf16_lo(w[c]), acc);
                        acc = __fmaf_rn(vec->whq[2 * c + 1], bf16_hi(w[c]), acc);
                    }
                    const float lg = __fadd_rn(vec->bh, acc);
                    const float p = 1.0f / (1.0f + expf(-lg));
                    const int q = min(32768, max(0, __float2int_rn(p * 32768.0f)));
                    if (scores) scores[si.out + x] = (uint16_t)q;
                    if (logits) logits[si.out + x] = lg;
                }
            }
            fence_async_smem();
            tc_before_sync();
            __syncthreads();
            tc_after_sync();
        }
        si = sn;
    }
    stage_wait();   // no copy outlives the CTA
    __syncthreads();
    if (abort && tid == 0) {   // let MMAs still in flight finish (bounded) before freeing TMEM
        mma_commit(bar_m);
        bar_wait(bar_m, phase, nullptr);
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 128);
}

size_t sc_infer_smem() { return kInfSmem; }

int sc_infer_blocks_per_sm() {
    // shared memory per SM (each CTA also reserves 1 KB), at most 4 CTAs for
    // the 512 TMEM columns (128 each)
    static int nb = [] {
        int dev = 0, smem_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess)
            return 1;
        const int v = smem_sm / (int)(kInfSmem + 1024);
        return v < 1 ? 1 : (v > 4 ? 4 : v);
    }();
    return nb;
}

cudaError_t sc_launch_infer(const ScSource &src, const unsigned char *block, uint16_t *scores,
                            float *logits, int total_segs, uint32_t *err, int grid, cudaStream_t s) {
    if (total_segs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sc_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kInfSmem);
    if (e != cudaSuccess) return e;
    k_sc_infer<<<grid, kInfThreads, kInfSmem, s>>>(src, block, scores, logits, total_segs, err);
    return cudaGetLastError();
}

// ============================================================= training ==
// One CTA (8 warps, one per SM) per segment, segments assigned statically
// (g = blockIdx.x + k gridDim.x) so that every run sums the same gradient
// terms in the same order.  Per segment: forward (features -> a1 -> a2 ->
// head), loss and its gradient at the logits, then for layers 3, 2, 1 the
// weight gradient and, for layers 3 and 2, the input gradient (a forward
// convolution of the gradient planes with the reversed, transposed
// weights).  The sums of the CTA go to its own slice of `partial`.
//
// Weight gradients: dW_t[co][ci] = sum_x dz[x][co] in[x + t - 3][ci] on
// tcgen05 (MN-major operands, N = input channels, K = 16 columns per MMA).
// tcgen05 has no M = 32, so one M = 64 MMA takes two taps: its rows 0-31 read
// the gradient planes dz and its rows 32-63 the next four planes, dz1, which
// hold dz one column later (dz1[x] = dz[x - 1]).  With `in` shifted by t, rows
// 32-63 sum dz[y] in[y + t - 2] over y = 0 .. 510: tap t + 1.  The term it
// leaves out, y = 511, is zero, as dz is zero on the 9 context columns at
// each end of the segment.  Taps (0, 1), (2, 3), (4, 5), (6, -): 4 x 32 MMAs
// per layer.  The weight gradients of consecutive layers go to two TMEM
// accumulator sets, so a layer's sums are added into `partial` while the next
// layer's MMAs run.
constexpr int kTrainThreads = 256;   // 8 warps: two per TMEM lane quarter
constexpr int kTrainPlanes = 18;   // D (4) | D1 (4) | A1 (4) | A2 (4) | X0 (2)
constexpr int kTapPairs = (kTaps + 1) / 2;
constexpr size_t kTrainStageBytes = (size_t)kTaps * 32 * 32 * sizeof(float);   // one layer's dW
static_assert(kTrainStageBytes <= 4 * (size_t)SegT::kPlane, "a layer's dW is staged in 4 planes");
constexpr size_t kTrainSmem = (size_t)kTrainPlanes * SegT::kPlane + (kScBlockBytes - kScVecBytes) +
                              kScVecBytes + 64 + 3 * 4 * 32 * sizeof(float);
constexpr int kDwCol = 128;   // TMEM columns of the weight-gradient sets: [128, 256), [256, 384)
constexpr int kDwSet = 32 * kTapPairs;
static_assert(kDwCol >= 32 * kScTrainTiles && kDwCol + 2 * kDwSet <= 512,
              "convolution and weight-gradient accumulators fit the 512 TMEM columns");
static_assert(kTrainSmem <= 227 * 1024, "training shared memory fits one CTA per SM");

namespace {

// Weight-gradient MMAs of one layer into the accumulator set at `tmem`:
// columns 32 p hold taps 2p (rows 0-31) and 2p + 1 (rows 32-63), summed over
// the 512 rows of the segment.  dz: the planes dz (4), then dz1 (4).
template <class G>
__device__ __forceinline__ void issue_dw(uint32_t tmem, const unsigned char *dz,
                                         const unsigned char *in, int n_in) {
    const uint32_t idesc = idesc_bf16(64, 8 * n_in, true, true);
    const uint64_t da = sdesc(smem_u32(dz) + kGuard * 16, 128, G::kPlane);
    const uint64_t db = sdesc(smem_u32(in) + (kGuard - 3) * 16, 128, G::kPlane);
    for (int p = 0; p < kTapPairs; ++p)
#pragma unroll 4
        for (int k = 0; k < G::kRows / 16; ++k)
            mma_bf16(tmem + 32 * p, da + (uint32_t)(16 * k), db + (uint32_t)(16 * k + 2 * p), idesc,
                     k != 0);
}

// Row r of the gradient planes dz and row r + 1 of dz1 (row 0 of dz1, the
// column before the segment, is zero).
template <class G>
__device__ __forceinline__ void store_dz(unsigned char *dz, int r, const float (&v)[32]) {
    store_row32<G>(dz, r, v);
    store_row32<G>(dz + 4 * G::kPlane, r + 1, v);
    if (r == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(dz + (4 + c) * G::kPlane + kGuard * 16) = make_uint4(0, 0, 0, 0);
    }
}

// Adds the weight gradient of a layer into the CTA's partial sums (layout
// [t][co][ci] per layer; written instead of added on the CTA's first
// segment).  An M = 64 accumulator keeps rows 16q .. 16q+15 in lanes 0-15 of
// TMEM lane quarter q, so quarter q of pair p holds output channels
// 16 (q & 1) .. +15 of tap 2p + (q >> 1).  Warps 0-3 read pairs 0 and 1,
// warps 4-7 pairs 2 and 3, into `stage`; then every thread adds its share
// with 16-byte loads and stores.
__device__ __forceinline__ void flush_dw(uint32_t tmem, float *stage, float *part, int off,
                                         int n_in_real, bool first) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
    for (int p = 2 * (warp >> 2); p < 2 * (warp >> 2) + 2; ++p) {
        const int t = 2 * p + (q >> 1);
        if (t >= kTaps) continue;   // rows 32-63 of the last pair: no tap 7
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32 * p, v);
        if (lane < 16) {
            float *row = stage + (t * 32 + 16 * (q & 1) + lane) * n_in_real;
#pragma unroll
            for (int ci = 0; ci < 32; ++ci)
                if (ci < n_in_real) row[ci] = v[ci];
        }
    }
    __syncthreads();
    const int n4 = kTaps * 32 * n_in_real / 4;
    float4 *dst = reinterpret_cast<float4 *>(part + off);
    const float4 *src = reinterpret_cast<const float4 *>(stage);
    for (int i = threadIdx.x; i < n4; i += 2 * kTrainThreads) {
        const int j = i + kTrainThreads;
        float4 a = src[i], b = j < n4 ? src[j] : make_float4(0, 0, 0, 0);
        if (!first) {
            const float4 pa = dst[i];
            const float4 pb = j < n4 ? dst[j] : make_float4(0, 0, 0, 0);
            a = make_float4(__fadd_rn(pa.x, a.x), __fadd_rn(pa.y, a.y), __fadd_rn(pa.z, a.z),
                            __fadd_rn(pa.w, a.w));
            b = make_float4(__fadd_rn(pb.x, b.x), __fadd_rn(pb.y, b.y), __fadd_rn(pb.z, b.z),
                            __fadd_rn(pb.w, b.w));
        }
        dst[i] = a;
        if (j < n4) dst[j] = b;
    }
    __syncthreads();
}

// Sums a per-thread 32-vector over the CTA (fixed order) into part[off + c].
__device__ __forceinline__ void flush_vec32(float (&v)[32], float *red, float *part, int off,
                                            bool first) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float w = warp_transpose_sum(v);
    red[warp * 32 + lane] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = 0.0f;
        for (int k = 0; k < kTrainThreads / 32; ++k) t = __fadd_rn(t, red[k * 32 + threadIdx.x]);
        part[off + threadIdx.x] = first ? t : __fadd_rn(part[off + threadIdx.x], t);
    }
    __syncthreads();
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

__global__ void __launch_bounds__(kTrainThreads, 1)
    k_sc_train(ScSource src, const uint8_t *__restrict__ labels, float pos_weight,
               const unsigned char *__restrict__ wblock, float *__restrict__ partial,
               int total_segs, uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *D = sm;                      // gradient planes dz, then dz1 (planes 4-7)
    unsigned char *A1 = sm + 8 * SegT::kPlane;
    unsigned char *A2 = sm + 12 * SegT::kPlane;   // also the dW stage once a2 is no longer read
    unsigned char *X0 = sm + 16 * SegT::kPlane;
    unsigned char *Wall = sm + kTrainPlanes * SegT::kPlane;
    ScVec *vec = reinterpret_cast<ScVec *>(Wall + (kScBlockBytes - kScVecBytes));
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(vec) + kScVecBytes);
    uint64_t *bar_m = bar_w + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 1);
    float *red = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(bar_w) + 64);
    float *stage = reinterpret_cast<float *>(A2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem = sc_prologue<SegT>(sm, kTrainPlanes, bar_w, bar_m, tslot, 512, Wall, wblock,
                                      kScBlockBytes - kScVecBytes, vec, wblock + kScOffVec);
    bool abort = __syncthreads_or(!bar_wait(bar_w, 0, err)) != 0;
    float *part = partial + (size_t)blockIdx.x * kScPartialStride;
    uint32_t phase = 0;
    const unsigned char *Wf1 = Wall + kScOffW1f, *Wf2 = Wall + kScOffW2f, *Wf3 = Wall + kScOffW3f;
    const unsigned char *Wb2 = Wall + kScOffW2b, *Wb3 = Wall + kScOffW3b;

    auto mma_sync_point = [&]() {   // st.shared visible to MMAs, TMEM reads done
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
    };
    // a wait that gave up ends the CTA's work (uniformly: the flag is reduced
    // over the CTA), so a fault shows as one ~2 s wait, not one per MMA batch
    auto wait_mma = [&]() {
        const bool ok = bar_wait(bar_m, phase, err);
        phase ^= 1u;
        tc_after_sync();
        if (__syncthreads_or(!ok)) abort = true;
        return !abort;
    };

    for (int g = blockIdx.x; g < total_segs && !abort; g += gridDim.x) {
        const SegInfo si = seg_info<SegT>(src, g);
        const int b0 = si.s0 - kScHalo;
        if (tid == 0 && g + (int)gridDim.x < total_segs)   // this CTA's next segment
            prefetch_rows<SegT>(seg_info<SegT>(src, g + gridDim.x));
        const uint8_t *lab = labels + (int64_t)si.strip * si.W;
        const bool first = g == (int)blockIdx.x;   // the CTA's first segment writes its partials
        __syncthreads();
        build_features<SegT>(X0, si.r0, si.r0 + si.pitch, si.r0 + 2 * si.pitch, si.W, si.y, si.H, b0);
        mma_sync_point();

        // ---- forward: layers 1 and 2
        for (int l = 0; l < 2; ++l) {
            if (tid == 0) {
                if (l == 0) issue_conv<SegT, 2>(tmem, X0, Wf1);
                else issue_conv<SegT, 4>(tmem, A1, Wf2);
                mma_commit(bar_m);
            }
            if (!wait_mma()) break;
            unsigned char *dst = l == 0 ? A1 : A2;
            for (int j = warp >> 2; j < SegT::kTiles; j += 2) {   // warp w: tiles w/4, w/4 + 2
                float v[32];
                acc_row(tmem, j, v);
                const int r = kTile * j + 32 * (warp & 3) + lane, x = b0 + r;
                const bool inside = x >= 0 && x < si.W;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float z = __fadd_rn(v[c], vec->b[l][c]);
                    v[c] = inside && z > 0.0f ? __bfloat162float(__float2bfloat16_rn(z)) : 0.0f;
                }
                store_row32<SegT>(dst, r, v);
            }
            mma_sync_point();
        }
        // ---- layer 3, head, loss; gradient at the logits and at z3
        if (abort) break;
        if (tid == 0) {
            issue_conv<SegT, 4>(tmem, A2, Wf3);
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        {
            float gwh[32], gb3[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) gwh[c] = gb3[c] = 0.0f;
            float gbh = 0.0f, loss = 0.0f;
            for (int j = warp >> 2; j < SegT::kTiles; j += 2) {   // warp w: tiles w/4, w/4 + 2
                float v[32];
                acc_row(tmem, j, v);
                const int r = kTile * j + 32 * (warp & 3) + lane, x = b0 + r;
                const bool inside = x >= 0 && x < si.W;
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float z = __fadd_rn(v[c], vec->b[2][c]);
                    v[c] = inside && z > 0.0f ? __bfloat162float(__float2bfloat16_rn(z)) : 0.0f;
                    acc = __fadd_rn(acc, __fmul_rn(vec->whq[c], v[c]));
                }
                float dl = 0.0f;
                if (x >= si.s0 && x < si.s1) {
                    const float lg = __fadd_rn(vec->bh, acc);
                    const float y = lab[x] ? 1.0f : 0.0f, w = lab[x] ? pos_weight : 1.0f;
                    const float p = 1.0f / (1.0f + expf(-lg));
                    dl = __fmul_rn(w, __fsub_rn(p, y));
                    const float sp = lg > 0.0f ? lg + log1pf(expf(-lg)) : log1pf(expf(lg));
                    loss = __fadd_rn(loss, __fmul_rn(w, __fsub_rn(sp, __fmul_rn(y, lg))));
                }
                gbh = __fadd_rn(gbh, dl);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    gwh[c] = __fadd_rn(gwh[c], __fmul_rn(dl, v[c]));
                    const float dz = v[c] > 0.0f
                                         ? __bfloat162float(__float2bfloat16_rn(__fmul_rn(dl, vec->whq[c])))
                                         : 0.0f;
                    gb3[c] = __fadd_rn(gb3[c], dz);
                    v[c] = dz;
                }
                store_dz<SegT>(D, r, v);
            }
            flush_vec32(gwh, red, part, kScPWh, first);
            flush_vec32(gb3, red + 128, part, kScPB3, first);
            gbh = warp_sum(gbh);
            loss = warp_sum(loss);
            if (lane == 0) { red[256 + 2 * warp] = gbh; red[256 + 2 * warp + 1] = loss; }
            __syncthreads();
            if (tid == 0) {
                float a = 0.0f, b = 0.0f;
                for (int k = 0; k < kTrainThreads / 32; ++k) {
                    a = __fadd_rn(a, red[256 + 2 * k]);
                    b = __fadd_rn(b, red[256 + 2 * k + 1]);
                }
                part[kScPBh] = first ? a : __fadd_rn(part[kScPBh], a);
                part[kScNParam] = first ? b : __fadd_rn(part[kScNParam], b);
            }
        }
        mma_sync_point();
        // ---- layers 3 and 2: weight gradient (sets 0, 1) and input gradient
        for (int l = 2; l >= 1; --l) {
            const unsigned char *in = l == 2 ? A2 : A1;
            if (tid == 0) {
                issue_conv<SegT, 4>(tmem, D, l == 2 ? Wb3 : Wb2);   // input gradient, columns [0, 128)
                issue_dw<SegT>(tmem + kDwCol + (l == 2 ? 0 : kDwSet), D, in, 4);
                mma_commit(bar_m);
            }
            if (l == 1)   // layer 3's weight gradient, while these MMAs run
                flush_dw(tmem + kDwCol, stage, part, kScPW3, kCh, first);
            if (!wait_mma()) break;
            float gb[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) gb[c] = 0.0f;
            for (int j = warp >> 2; j < SegT::kTiles; j += 2) {   // warp w: tiles w/4, w/4 + 2
                float v[32], a[32];
                acc_row(tmem, j, v);
                const int r = kTile * j + 32 * (warp & 3) + lane;
                load_row32<SegT>(in, r, a);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    v[c] = a[c] > 0.0f ? __bfloat162float(__float2bfloat16_rn(v[c])) : 0.0f;
                    gb[c] = __fadd_rn(gb[c], v[c]);
                }
                store_dz<SegT>(D, r, v);   // every MMA reading D has completed
            }
            __syncthreads();
            flush_vec32(gb, red, part, l == 2 ? kScPB2 : kScPB1, first);
            mma_sync_point();
        }
        // ---- layer 1: weight gradient only (set 0; layer 2's is added meanwhile)
        if (abort) break;
        if (tid == 0) {
            issue_dw<SegT>(tmem + kDwCol, D, X0, 2);
            mma_commit(bar_m);
        }
        flush_dw(tmem + kDwCol + kDwSet, stage, part, kScPW2, kCh, first);
        if (!wait_mma()) break;
        flush_dw(tmem + kDwCol, stage, part, kScPW1, kScCin, first);
        zero_guards<SegT>(A2, 4);   // the stage overwrote them; the next forward reads them
        tc_before_sync();
    }
    __syncthreads();
    if (abort && tid == 0) {   // let MMAs still in flight finish (bounded) before freeing TMEM
        mma_commit(bar_m);
        bar_wait(bar_m, phase, nullptr);
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 512);
}

size_t sc_train_smem() { return kTrainSmem; }

cudaError_t sc_launch_train(const ScSource &src, const uint8_t *labels, float pos_weight,
                            const unsigned char *block, float *partial, int total_segs,
                            uint32_t *err, int grid, cudaStream_t s) {
    if (total_segs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sc_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    k_sc_train<<<grid, kTrainThreads, kTrainSmem, s>>>(src, labels, pos_weight, block, partial,
                                                      total_segs, err);
    return cudaGetLastError();
}

// =============================================================== picks ==
// One warp per half-strip: K/2 best learned scores with the suppression
// window; a half whose best learned score is under 16384 (p < 1/2) keeps the
// handcrafted points already in its slots when `fallback` is set.
__global__ void __launch_bounds__(256)
    k_sc_pick(const DevFrame *__restrict__ frames, int B, const int32_t *__restrict__ rows,
              DevParams P, const uint16_t *__restrict__ scores, int fallback,
              CandSlot *__restrict__ slots) {
    const int lane = threadIdx.x & 31;
    const int items = B * P.N * 2;
    const int kk = P.K >> 1;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items;
         it += (gridDim.x * blockDim.x) >> 5) {
        const int f = it / (2 * P.N), j = it - f * 2 * P.N;
        const int i = j >> 1, half = j & 1;
        const DevFrame fr = frames[f];
        const int W = fr.W, H = fr.H, hw = W >> 1;
        const int x0 = half ? hw : 0, x1 = half ? W : hw;
        const int y = rows[fr.rows_off + i];
        const uint16_t *s = scores + fr.sc_pix_off + (int64_t)i * W;
        int picks[kScMaxPicks];
        for (int r = 0; r < kk; ++r) {
            uint32_t b = 0u;
            for (int x = x0 + lane; x < x1; x += 32) {
                bool sup = false;
                for (int q = 0; q < r; ++q) sup |= abs(x - picks[q]) <= P.sup_px;
                if (!sup) b = max(b, ((uint32_t)s[x] << 16) | (uint32_t)(half ? x : (0xFFFF - x)));
            }
            b = __reduce_max_sync(0xffffffffu, b);
            const int rank = (int)(b & 0xFFFFu);
            const int px = b == 0u ? -1000000 : (half ? rank : (0xFFFF - rank));
            const uint32_t scv = b >> 16;
            if (r == 0 && fallback && scv < 16384u) break;   // keep the handcrafted points
            picks[r] = px;
            if (lane == 0) {
                CandSlot out;
                out.x = (int16_t)(b == 0u ? -1 : px);
                out.y = (int16_t)y;
                out.s = (uint16_t)scv;
                out.kept = (uint16_t)(b != 0u && scv >= P.T_ps && px >= P.T_px &&
                                      px <= W - 1 - P.T_px && y >= P.T_px && y <= H - 1 - P.T_px);
                store_slot(slots + (int64_t)f * kMaxSlots + i * P.K + half * kk + r, out);
            }
        }
    }
}

cudaError_t sc_launch_pick(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                           const uint16_t *scores, int fallback, CandSlot *slots, int grid,
                           cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    k_sc_pick<<<grid, 256, 0, s>>>(frames, B, rows, P, scores, fallback, slots);
    return cudaGetLastError();
}

// ============================================================= weights ==
// Packs the f32 parameters into the device weight block: the bf16 B operands
// of the forward convolutions and of the input-gradient convolutions, the
// biases, the bf16-rounded head weights and the head bias.
// Writes parameter p (value w) into its places in the device weight block.
__device__ __forceinline__ void sc_pack_one(int p, float w, unsigned char *blk) {
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    ScVec *vec = reinterpret_cast<ScVec *>(blk + kScOffVec);
    auto put = [&](int off) { *reinterpret_cast<__nv_bfloat16 *>(blk + off) = wb; };
    if (p < kScPB1) {                           // W1[co][ci][t], 2 input chunks per tap
        const int co = p / (kScCin * kTaps), ci = (p / kTaps) % kScCin, t = p % kTaps;
        put(kScOffW1f + ((t * 2 + ci / 8) * 32 + co) * 16 + (ci % 8) * 2);
    } else if (p < kScPW2) {
        vec->b[0][p - kScPB1] = w;
    } else if (p < kScPB2 || (p >= kScPW3 && p < kScPB3)) {   // W2 / W3 [co][ci][t]
        const bool l3 = p >= kScPW3;
        const int q = p - (l3 ? kScPW3 : kScPW2);
        const int co = q / (kCh * kTaps), ci = (q / kTaps) % kCh, t = q % kTaps;
        put((l3 ? kScOffW3f : kScOffW2f) + ((t * 4 + ci / 8) * 32 + co) * 16 + (ci % 8) * 2);
        // input gradient: da[x][ci] = sum dz[x + t' - 3][co] W[co][ci][6 - t']
        put((l3 ? kScOffW3b : kScOffW2b) + (((kTaps - 1 - t) * 4 + co / 8) * 32 + ci) * 16 +
            (co % 8) * 2);
    } else if (p < kScPW3) {
        vec->b[1][p - kScPB2] = w;
    } else if (p < kScPWh) {
        vec->b[2][p - kScPB3] = w;
    } else if (p < kScPBh) {
        vec->whq[p - kScPWh] = __bfloat162float(wb);
    } else {
        vec->bh = w;
    }
}

__global__ void k_sc_pack(const float *__restrict__ prm, unsigned char *__restrict__ blk) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kScNParam) sc_pack_one(p, prm[p], blk);
}

cudaError_t sc_launch_pack(const float *params, unsigned char *block, cudaStream_t s) {
    k_sc_pack<<<(kScNParam + 255) / 256, 256, 0, s>>>(params, block);
    return cudaGetLastError();
}

// Sums the per-CTA gradient partials in a fixed order, then optionally takes
// an SGD step with momentum:  v = momentum v + scale g,  w = w - lr v, and
// writes w into the device weight block.  Weight blocks of the partials are
// laid out [t][co][ci]; the parameters are [co][ci][t].  A block reduces 64
// parameters with 16 threads each (partials c = q, q + 16, ...), combined in
// order.  With norm_part set (gradient clipping) it takes no step: it stores
// the summed gradient in gbuf and the block's sum of squares of the mean
// gradient in norm_part[block], and k_sc_clip_step takes the step once the
// whole norm is known.
constexpr int kSgdParams = 64;   // parameters per block
constexpr int kSgdQ = 16;        // threads per parameter, each summing every 16th partial
static_assert(kScSgdBlocks == (kScNParam + 1 + kSgdParams - 1) / kSgdParams, "sgd grid");

__device__ __forceinline__ int partial_index(int p) {
    auto tr = [](int q, int off, int cin) {
        const int co = q / (cin * kTaps), ci = (q / kTaps) % cin, t = q % kTaps;
        return off + (t * 32 + co) * cin + ci;
    };
    if (p < kScPB1) return tr(p - kScPW1, kScPW1, kScCin);
    if (p >= kScPW2 && p < kScPB2) return tr(p - kScPW2, kScPW2, kCh);
    if (p >= kScPW3 && p < kScPB3) return tr(p - kScPW3, kScPW3, kCh);
    return p;
}

__global__ void __launch_bounds__(kSgdQ * kSgdParams)
    k_sc_sgd(float *__restrict__ prm, float *__restrict__ mom, const float *__restrict__ part,
             int n_part, float scale, float lr, float momentum, int apply,
             float *__restrict__ grads_out, float *__restrict__ loss_out,
             float *__restrict__ gbuf, float *__restrict__ norm_part, unsigned char *__restrict__ blk) {
    __shared__ float red[kSgdQ][kSgdParams];
    const int pl = threadIdx.x % kSgdParams, q = threadIdx.x / kSgdParams;
    const int p = blockIdx.x * kSgdParams + pl;
    float g = 0.0f;
    if (p <= kScNParam) {
        const float *src = part + partial_index(p);
        int c = q;
        for (; c + 7 * kSgdQ < n_part; c += 8 * kSgdQ) {   // eight loads in flight, added in order
            float t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = __ldcg(src + (size_t)(c + kSgdQ * u) * kScPartialStride);
#pragma unroll
            for (int u = 0; u < 8; ++u) g = __fadd_rn(g, t[u]);
        }
        for (; c < n_part; c += kSgdQ) g = __fadd_rn(g, __ldcg(src + (size_t)c * kScPartialStride));
    }
    red[q][pl] = g;
    __syncthreads();
    g = red[0][pl];
#pragma unroll
    for (int k = 1; k < kSgdQ; ++k) g = __fadd_rn(g, red[k][pl]);
    if (norm_part) {   // clipping: squares of the mean gradient, summed in order by thread 0
        __syncthreads();
        if (q == 0) {
            const float m = __fmul_rn(scale, g);
            red[1][pl] = p < kScNParam ? __fmul_rn(m, m) : 0.0f;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int i = 0; i < kSgdParams; ++i) t = __fadd_rn(t, red[1][i]);
            norm_part[blockIdx.x] = t;
        }
    }
    if (q != 0 || p > kScNParam) return;
    if (p == kScNParam) {   // loss slot
        if (loss_out) *loss_out = g;
        return;
    }
    if (grads_out) grads_out[p] = g;
    if (norm_part) {
        gbuf[p] = g;
    } else if (apply) {
        const float v = __fadd_rn(__fmul_rn(momentum, mom[p]), __fmul_rn(scale, g));
        const float w = __fsub_rn(prm[p], __fmul_rn(lr, v));
        mom[p] = v;
        prm[p] = w;
        sc_pack_one(p, w, blk);
    }
}

// The clipped step: every block sums the kScSgdBlocks partial squares in the
// same order (strided per thread, then a fixed tree, so all blocks agree on
// the norm), f = min(1, clip / |scale g|), then
// v = momentum v + f (scale g),  w = w - lr v, and w into the weight block.
__global__ void __launch_bounds__(kSgdParams)
    k_sc_clip_step(float *__restrict__ prm, float *__restrict__ mom, const float *__restrict__ gbuf,
                   const float *__restrict__ norm_part, float scale, float lr, float momentum,
                   float clip, unsigned char *__restrict__ blk) {
    __shared__ float red[kSgdParams];
    __shared__ float f_s;
    float t = 0.0f;
    for (int i = threadIdx.x; i < kScSgdBlocks; i += kSgdParams)
        t = __fadd_rn(t, __ldcg(norm_part + i));
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = kSgdParams / 2; w > 0; w >>= 1) {   // fixed tree: every block sums alike
        if (threadIdx.x < w) red[threadIdx.x] = __fadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float n = sqrtf(red[0]);
        f_s = n > clip ? __fdiv_rn(clip, n) : 1.0f;
    }
    __syncthreads();
    const int p = blockIdx.x * kSgdParams + threadIdx.x;
    if (p >= kScNParam) return;
    const float m = __fmul_rn(f_s, __fmul_rn(scale, gbuf[p]));
    const float v = __fadd_rn(__fmul_rn(momentum, mom[p]), m);
    const float w = __fsub_rn(prm[p], __fmul_rn(lr, v));
    mom[p] = v;
    prm[p] = w;
    sc_pack_one(p, w, blk);
}

cudaError_t sc_launch_sgd(float *params, float *mom, float *partial, int n_partials, float scale,
                          float lr, float momentum, int apply, float clip, float *gbuf,
                          float *norm_part, float *grads_out, float *loss_out,
                          unsigned char *block, cudaStream_t s) {
    const bool clipped = apply && clip > 0.0f;
    k_sc_sgd<<<kScSgdBlocks, kSgdQ * kSgdParams, 0, s>>>(
        params, mom, partial, n_partials, scale, lr, momentum, apply, grads_out, loss_out,
        clipped ? gbuf : nullptr, clipped ? norm_part : nullptr, block);
    if (clipped)
        k_sc_clip_step<<<kScSgdBlocks, kSgdParams, 0, s>>>(params, mom, gbuf, norm_part, scale, lr,
                                                           momentum, clip, block);
    return cudaGetLastError();
}

}  // namespace ca
