// ca_scorer2d.cu -- the paper's own learned edge scorer (Sec. 2.2.4) on the
// 5th-generation tensor cores: three 3x3 convolutions to 8, 16 and 32
// features with ReLU, a 1x1 head and a sigmoid, on RGBXY strips 7 rows high
// (unpadded vertically, so 7 -> 5 -> 3 -> 1 rows: the strip's middle row;
// zero-padded horizontally).  bf16 operands, f32 accumulators in TMEM.
//
// Convention: out[r][x] = b + sum_{dr, dx, ci} W[co][ci][dr][dx] in[r + dr][x + dx - 1][ci].
//
// Layout.  A strip is processed in segments of 384 consecutive columns (3
// tiles of 128); three layers of 3x3 need one column of context each, so the
// middle 378 columns are outputs.  Every image row of a layer lives in shared
// memory as "planes" of 8 channels: one 16-byte row per column, 8 zero guard
// rows at both ends.  A tile of 128 columns of one plane is a K-major operand
// core-matrix column (SBO = 128 bytes between 8-column groups).  With the
// leading byte offset (the step between the two K halves of a K = 16 MMA) set
// to 16 bytes, the second half is the same plane one column further on: one
// MMA then covers two column taps of 8 channels, so the 5- and 8-channel
// inputs of layers 1 and 2 need 2 MMAs per row tap (taps -1/0, then +1 with a
// zero-weight fourth tap) and no zero padding of channels.  Layer 3 reads its
// 16-channel input as two planes (LBO = one plane), one MMA per tap.  Column
// taps are 16-byte offsets of the operand start: no im2col copy.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "ca_internal.h"

namespace ca {

namespace {

#include "ca_tc.cuh"

constexpr int kTile = 128;
constexpr int kCols = kTile * kSc2Tiles;     // columns of a segment
constexpr int kG = 8;                         // guard rows at each end of a plane
constexpr int kPlane = (kCols + 2 * kG) * 16; // bytes of one plane
static_assert(kCols - 2 * kSc2Halo == kSc2SegOut, "segment geometry");

struct Sc2Vec {   // float part of the weight block
    float b1[8], b2[16], b3[32];
    float whq[32];   // head weights rounded to bf16
    float bh;
    float pad[7];
};
static_assert(sizeof(Sc2Vec) == kSc2VecBytes, "vector block size");

// Where segment g of a launch reads and writes.
struct Seg2 {
    const uint8_t *base;   // frame (frames mode) or the strip's 7 rows (strips mode)
    int64_t pitch;         // bytes between rows of `base`
    int W, H, y;           // y: the strip's middle row
    int s0, s1;            // output columns [s0, s1)
    int64_t out;           // index of column 0 of the strip in the per-column outputs
    int strip;             // strips mode: index of the strip in the source
    const int32_t *rows7;  // strips mode: frame rows of the 7 rows
};

__device__ __forceinline__ Seg2 seg2_info(const Sc2Source &src, int g) {
    Seg2 si;
    if (src.frames) {
        int lo = 0, hi = src.B - 1;   // frame of segment g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (src.frames[mid].sc_seg_off <= g) lo = mid;
            else hi = mid - 1;
        }
        const DevFrame &fr = src.frames[lo];
        const int nseg = (fr.W + kSc2SegOut - 1) / kSc2SegOut;
        const int local = g - fr.sc_seg_off;
        const int i = local / nseg, s = local - i * nseg;
        si.base = fr.rgb;
        si.pitch = fr.pitch;
        si.W = fr.W;
        si.H = fr.H;
        si.y = src.rows[fr.rows_off + i];
        si.s0 = s * kSc2SegOut;
        si.out = (int64_t)fr.sc_pix_off + (int64_t)i * fr.W;
        si.strip = -1;
        si.rows7 = nullptr;
    } else {
        const int nseg = (src.W + kSc2SegOut - 1) / kSc2SegOut;
        const int j = g / nseg, s = g - j * nseg;
        const int id = src.idx ? src.idx[j] : j;
        si.W = src.W;
        si.H = src.H;
        si.pitch = (int64_t)src.W * 3;
        si.base = src.strips7 + (int64_t)id * 7 * si.pitch;
        si.rows7 = src.rows7 + (int64_t)id * 7;
        si.y = si.rows7[3];
        si.s0 = s * kSc2SegOut;
        si.out = (int64_t)j * src.W;
        si.strip = id;
    }
    si.s1 = min(si.W, si.s0 + kSc2SegOut);
    return si;
}

// Image row k (0..6) of the strip: its bytes and its frame row.
__device__ __forceinline__ const uint8_t *seg2_row(const Seg2 &si, int k, int *frame_row) {
    if (si.rows7) {
        *frame_row = si.rows7[k];
        return si.base + k * si.pitch;
    }
    const int r = min(max(si.y - 3 + k, 0), si.H - 1);
    *frame_row = r;
    return si.base + (int64_t)r * si.pitch;
}

// L2 prefetch (TMA) of the bytes a segment reads from its 7 rows, shrunk
// to whole 16-byte blocks inside each row (a hint: the loads read the same
// bytes).
__device__ __forceinline__ void prefetch7(const Seg2 &si) {
    const int b0 = si.s0 - kSc2Halo;
    const int c0 = max(b0, 0), c1 = min(b0 + kCols, si.W);
    if (c1 <= c0) return;
    for (int k = 0; k < 7; ++k) {
        int fr_row;
        const uint8_t *row = seg2_row(si, k, &fr_row);
        const uintptr_t a = ((uintptr_t)(row + 3 * c0) + 15) & ~(uintptr_t)15;
        const uintptr_t b = (uintptr_t)(row + 3 * c1) & ~(uintptr_t)15;
        if (b > a)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                         : "memory");
    }
}

// Staging of a segment's 7 rows in shared memory by cp.async (16-byte
// asynchronous copies), issued one segment ahead into the interior rows of
// the a1 planes (free from the end of the third layer until the next
// segment's first epilogue; the planes' zero guard rows are not touched).
// Possible when the copies stay inside each row: rows start on 16-byte
// boundaries and 3 W is a multiple of 16.  Row k lands at stage2_row(k).
constexpr int kStage2Row = 1200;   // >= 3 x 384 columns + 30 bytes of alignment, 16 x 75
static_assert(3 * kCols + 30 <= kStage2Row && 5 * kStage2Row <= kCols * 16, "staged rows fit");

__device__ __forceinline__ unsigned char *stage2_row(unsigned char *a1, int k) {
    return a1 + (k / 5) * kPlane + kG * 16 + (k % 5) * kStage2Row;
}

__device__ __forceinline__ bool stageable2(const Seg2 &si) {
    return (((uintptr_t)si.base | (uintptr_t)si.pitch | (uintptr_t)(3 * si.W)) & 15) == 0;
}

// First byte (a multiple of 16, relative to a row) of the staged block.
__device__ __forceinline__ int stage2_bias(const Seg2 &si) {
    return (3 * max(si.s0 - kSc2Halo, 0)) & ~15;
}

__device__ __forceinline__ void stage2_rows(unsigned char *a1, const Seg2 &si) {
    const int b0 = si.s0 - kSc2Halo;
    const int c0 = max(b0, 0), c1 = min(b0 + kCols, si.W);
    const int a = stage2_bias(si), b = (3 * c1 + 15) & ~15;
    const int nb = c1 > c0 ? (b - a) >> 4 : 0;   // 16-byte blocks per row
    for (int i = threadIdx.x; i < 7 * nb; i += blockDim.x) {
        const int k = i / nb, j = i - k * nb;
        int fr_row;
        const uint8_t *src = seg2_row(si, k, &fr_row) + a + 16 * j;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         smem_u32(stage2_row(a1, k) + 16 * j)),
                     "l"(src)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void stage2_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// RGBXY features of the 7 x 384 pixels of a segment (columns b0 ...) into 7
// planes: channels R, G, B as (v - 128) / 128, X = (x - (W-1)/2) / W and
// Y = (row - (H-1)/2) / H in binary32, all rounded to bf16; zero outside the
// frame's columns.
__device__ __forceinline__ void build_x(unsigned char *X, const Seg2 &si, int b0,
                                        unsigned char *staged_a1 = nullptr) {
    const float xc = __fmul_rn(0.5f, (float)(si.W - 1)), Wf = (float)si.W;
    const float yc = __fmul_rn(0.5f, (float)(si.H - 1)), Hf = (float)si.H;
    // a thread per column: X once per column, Y once per row; pixel x of row
    // k at rowp[k] + 3 x (the staged copy is offset by its first byte)
    const uint8_t *rowp[7];
    float Yf[7];
    const int bias = staged_a1 ? stage2_bias(si) : 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        int fr_row;
        rowp[k] = seg2_row(si, k, &fr_row);
        if (staged_a1) rowp[k] = stage2_row(staged_a1, k) - bias;
        Yf[k] = __fdiv_rn(__fsub_rn((float)fr_row, yc), Hf);
    }
    for (int c = threadIdx.x; c < kCols; c += blockDim.x) {
        const int x = b0 + c;
        const bool inside = x >= 0 && x < si.W;
        const float Xf = inside ? __fdiv_rn(__fsub_rn((float)x, xc), Wf) : 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (inside) {
                const uint8_t *p = rowp[k] + 3 * x;
                const float R = (float)((int)p[0] - 128) * (1.0f / 128.0f);
                const float G = (float)((int)p[1] - 128) * (1.0f / 128.0f);
                const float B = (float)((int)p[2] - 128) * (1.0f / 128.0f);
                q = make_uint4(pack_bf16(R, G), pack_bf16(B, Xf), pack_bf16(Yf[k], 0.0f), 0u);
            }
            *reinterpret_cast<uint4 *>(X + k * kPlane + (kG + c) * 16) = q;
        }
    }
}

// Zero guard rows of n planes from `p`.
__device__ __forceinline__ void zero_guards(unsigned char *p, int n) {
    for (int i = threadIdx.x; i < n * kG * 2; i += blockDim.x) {
        const int plane = i / (2 * kG), g = i % (2 * kG);
        const int row = g < kG ? g : kCols + g;
        *reinterpret_cast<uint4 *>(p + plane * kPlane + row * 16) = make_uint4(0, 0, 0, 0);
    }
}

// ---- forward MMAs (one thread issues them)

// Layers 1 and 2: 8-channel input planes `in` (rows r + dr), N = 16 outputs
// per row into TMEM columns tile * stride + 16 r.  Per row tap two MMAs:
// column taps (-1, 0), then (+1, +2) with the +2 weights zero.
__device__ __forceinline__ void issue_conv8(uint32_t tmem, const unsigned char *in,
                                            const unsigned char *w, int out_rows, int stride) {
    constexpr uint32_t idesc = idesc_bf16(128, 16, false, false);
    const uint64_t db = sdesc(smem_u32(w), 256, 128);
    for (int j = 0; j < kSc2Tiles; ++j)
        for (int r = 0; r < out_rows; ++r)
#pragma unroll
            for (int dr = 0; dr < 3; ++dr)
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const uint64_t da = sdesc(smem_u32(in + (r + dr) * kPlane) +
                                                  (kG + kTile * j + 2 * o - 1) * 16,
                                              16, 128);
                    mma_bf16(tmem + stride * j + 16 * r, da, db + (uint32_t)(((dr * 2 + o) * 512) >> 4),
                             idesc, (dr | o) != 0);
                }
}

// Layer 3: 16-channel input rows (two planes each, rows dr = 0..2), N = 32
// outputs into TMEM columns 32 tile; one MMA per tap.
__device__ __forceinline__ void issue_conv16(uint32_t tmem, const unsigned char *in,
                                             const unsigned char *w) {
    constexpr uint32_t idesc = idesc_bf16(128, 32, false, false);
    const uint64_t db = sdesc(smem_u32(w), 512, 128);
    for (int j = 0; j < kSc2Tiles; ++j)
#pragma unroll
        for (int dr = 0; dr < 3; ++dr)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint64_t da = sdesc(smem_u32(in + 2 * dr * kPlane) +
                                              (kG + kTile * j + dx - 1) * 16,
                                          kPlane, 128);
                mma_bf16(tmem + 32 * j, da, db + (uint32_t)(((dr * 3 + dx) * 1024) >> 4), idesc,
                         (dr | dx) != 0);
            }
}

// TMEM address of the calling warp's lane quarter at column `col`.
__device__ __forceinline__ uint32_t tq(uint32_t tmem, int col) {
    const int q = (threadIdx.x >> 5) & 3;
    return tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col;
}

// relu(v + b) of 8 values rounded to bf16 into one 16-byte plane row (zero
// when `inside` is false).
__device__ __forceinline__ uint4 relu_row8(const float *v, const float *b, bool inside) {
    if (!inside) return make_uint4(0u, 0u, 0u, 0u);
    return make_uint4(pack_relu_bf16(__fadd_rn(v[0], b[0]), __fadd_rn(v[1], b[1])),
                      pack_relu_bf16(__fadd_rn(v[2], b[2]), __fadd_rn(v[3], b[3])),
                      pack_relu_bf16(__fadd_rn(v[4], b[4]), __fadd_rn(v[5], b[5])),
                      pack_relu_bf16(__fadd_rn(v[6], b[6]), __fadd_rn(v[7], b[7])));
}

}  // namespace

// =============================================================== pack ==
// f32 parameters -> the device weight block (bf16 B operands, floats).
// Writes parameter p (value w) into its places in the block.
__device__ __forceinline__ void sc2_pack_one(int p, float w, unsigned char *blk) {
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    Sc2Vec *vec = reinterpret_cast<Sc2Vec *>(blk + kSc2OffVec);
    auto put = [&](int off) { *reinterpret_cast<__nv_bfloat16 *>(blk + off) = wb; };
    if (p < kSc2PB1) {                        // W1[co][ci][dr][dx]
        const int co = p / 45, ci = (p / 9) % 5, dr = (p / 3) % 3, dx = p % 3;
        const int o = dx >> 1, c = dx & 1;    // pair o: taps 2o, 2o + 1
        put(kSc2OffW1 + (dr * 2 + o) * 512 + (c * 16 + co) * 16 + ci * 2);
    } else if (p < kSc2PW2) {
        vec->b1[p - kSc2PB1] = w;
    } else if (p < kSc2PB2) {                 // W2[co][ci][dr][dx]
        const int q = p - kSc2PW2;
        const int co = q / 72, ci = (q / 9) % 8, dr = (q / 3) % 3, dx = q % 3;
        const int o = dx >> 1, c = dx & 1;
        put(kSc2OffW2 + (dr * 2 + o) * 512 + (c * 16 + co) * 16 + ci * 2);
        // input gradient of layer 2: B[n = ci][k = co] per tap, 2 chunks of 8 co
        put(kSc2OffW2b + (dr * 3 + dx) * 512 + ((co >> 3) * 16 + ci) * 16 + (co & 7) * 2);
    } else if (p < kSc2PW3) {
        vec->b2[p - kSc2PB2] = w;
    } else if (p < kSc2PB3) {                 // W3[co][ci][dr][dx]
        const int q = p - kSc2PW3;
        const int co = q / 144, ci = (q / 9) % 16, dr = (q / 3) % 3, dx = q % 3;
        put(kSc2OffW3 + (dr * 3 + dx) * 1024 + ((ci >> 3) * 32 + co) * 16 + (ci & 7) * 2);
        // input gradient of layer 3: B[n = ci][k = co] per tap, 4 chunks of 8 co
        put(kSc2OffW3b + (dr * 3 + dx) * 1024 + ((co >> 3) * 16 + ci) * 16 + (co & 7) * 2);
    } else if (p < kSc2PWh) {
        vec->b3[p - kSc2PB3] = w;
    } else if (p < kSc2PBh) {
        vec->whq[p - kSc2PWh] = __bfloat162float(wb);
    } else {
        vec->bh = w;
    }
}

__global__ void k_sc2_pack(const float *__restrict__ prm, unsigned char *__restrict__ blk) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kScorer2dNParam) sc2_pack_one(p, prm[p], blk);
}

cudaError_t sc2_launch_pack(const float *params, unsigned char *block, cudaStream_t s) {
    // padding (the zero weights of the fourth column tap and of the padded
    // channels) must be zero
    cudaError_t e = cudaMemsetAsync(block, 0, kSc2BlockBytes, s);
    if (e != cudaSuccess) return e;
    k_sc2_pack<<<(kScorer2dNParam + 255) / 256, 256, 0, s>>>(params, block);
    return cudaGetLastError();
}

// ========================================================== inference ==
// One CTA (8 warps, two per TMEM lane quarter) per segment at a time, 2 CTAs
// per SM.  Output per output column: the Q15 score round(32768 p) and/or the
// logit.
constexpr int kInf2Threads = 256;
constexpr int kInf2Cols = 256;                        // TMEM columns (layer 1: 3 x 80)
constexpr size_t kInf2Smem = 12 * (size_t)kPlane + kSc2FwdBytes + kSc2VecBytes + 64;

__global__ void __launch_bounds__(kInf2Threads, 2)
    k_sc2_infer(Sc2Source src, const unsigned char *__restrict__ wblock,
                uint16_t *__restrict__ scores, float *__restrict__ logits, int total_segs,
                uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *X = sm;                     // 7 planes: features; then a2 (3 rows x 2 planes)
    unsigned char *A1 = sm + 7 * kPlane;       // 5 planes: a1
    unsigned char *Wf = A1 + 5 * kPlane;
    Sc2Vec *vec = reinterpret_cast<Sc2Vec *>(Wf + kSc2FwdBytes);
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(vec) + kSc2VecBytes);
    uint64_t *bar_m = bar_w + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 1);
    unsigned char *A2 = X;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    zero_guards(sm, 12);
    if (tid == 0) {
        bar_init(bar_w, 1);
        bar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, kInf2Cols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        bar_expect_tx(bar_w, kSc2FwdBytes + kSc2VecBytes);
        bulk_g2s(Wf, wblock, kSc2FwdBytes, bar_w);
        bulk_g2s(vec, wblock + kSc2OffVec, kSc2VecBytes, bar_w);
    }
    bool abort = __syncthreads_or(!bar_wait(bar_w, 0, err)) != 0;
    uint32_t phase = 0;
    const int q = warp & 3, half = warp >> 2;   // lane quarter; two warps per quarter

    auto sync_point = [&]() {   // st.shared visible to the MMAs, TMEM reads done
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
    };
    // where the current and the next segment of this CTA read and write: the
    // next one's (a search over the frames) is looked up, and its rows are
    // prefetched into L2, while the current segment's first layer runs
    Seg2 si, sn;
    bool has_next = false;
    auto run = [&](int layer, int g) {   // issue one layer, wait for it
        if (tid == 0) {
            if (layer == 0) issue_conv8(tmem, X, Wf + kSc2OffW1, 5, 80);
            else if (layer == 1) issue_conv8(tmem, A1, Wf + kSc2OffW2, 3, 48);
            else issue_conv16(tmem, A2, Wf + kSc2OffW3);
            mma_commit(bar_m);
        }
        if (layer == 0 && has_next) {
            sn = seg2_info(src, g + gridDim.x);
            if (tid == 0) prefetch7(sn);
        }
        const bool ok = bar_wait(bar_m, phase, err);
        phase ^= 1u;
        tc_after_sync();
        if (__syncthreads_or(!ok)) abort = true;
        return !abort;
    };

    if ((int)blockIdx.x < total_segs) si = seg2_info(src, blockIdx.x);
    bool staged = false;   // this segment's rows are in A1's interior
    for (int g = blockIdx.x; g < total_segs && !abort; g += gridDim.x) {
        const int b0 = si.s0 - kSc2Halo;
        has_next = g + (int)gridDim.x < total_segs;
        __syncthreads();   // the previous segment is done with X / A1 / A2
        if (staged) {
            stage2_wait();
            __syncthreads();
            build_x(X, si, b0, A1);
        } else {
            build_x(X, si, b0);
        }
        staged = false;
        sync_point();
        // ---- layer 1: 5 rows of 8 channels
        if (!run(0, g)) break;
        for (int it = half; it < kSc2Tiles * 5; it += 2) {
            const int j = it / 5, r = it - 5 * j;
            float v[8];
            tmem_ld8(tq(tmem, 80 * j + 16 * r), v);
            const int row = kTile * j + 32 * q + lane, x = b0 + row;
            *reinterpret_cast<uint4 *>(A1 + r * kPlane + (kG + row) * 16) =
                relu_row8(v, vec->b1, x >= 0 && x < si.W);
        }
        sync_point();
        // ---- layer 2: 3 rows of 16 channels (two planes each), over the features
        if (!run(1, g)) break;
        for (int it = half; it < kSc2Tiles * 3; it += 2) {
            const int j = it / 3, r = it - 3 * j;
            float v[16];
            tmem_ld16(tq(tmem, 48 * j + 16 * r), v);
            const int row = kTile * j + 32 * q + lane, x = b0 + row;
            const bool inside = x >= 0 && x < si.W;
            *reinterpret_cast<uint4 *>(A2 + 2 * r * kPlane + (kG + row) * 16) =
                relu_row8(v, vec->b2, inside);
            *reinterpret_cast<uint4 *>(A2 + (2 * r + 1) * kPlane + (kG + row) * 16) =
                relu_row8(v + 8, vec->b2 + 8, inside);
        }
        sync_point();
        // ---- layer 3 and the head
        if (!run(2, g)) break;
        if (has_next && stageable2(sn)) {   // the MMAs are done with A1
            stage2_rows(A1, sn);
            staged = true;
        }
        for (int j = half; j < kSc2Tiles; j += 2) {
            float v[32];
            tmem_ld32(tq(tmem, 32 * j), v);
            const int row = kTile * j + 32 * q + lane, x = b0 + row;
            if (x >= si.s0 && x < si.s1) {
                // relu(z + b3) rounded to bf16; logit = bh + sum_c whq[c] a3[c]
                // in channel order, each product and sum rounded
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    const uint32_t a = pack_relu_bf16(__fadd_rn(v[c], vec->b3[c]),
                                                      __fadd_rn(v[c + 1], vec->b3[c + 1]));
                    acc = __fadd_rn(acc, __fmul_rn(vec->whq[c], bf16_lo(a)));
                    acc = __fadd_rn(acc, __fmul_rn(vec->whq[c + 1], bf16_hi(a)));
                }
                const float lg = __fadd_rn(vec->bh, acc);
                if (logits) logits[si.out + x] = lg;
                if (scores) {
                    const float p = 1.0f / (1.0f + expf(-lg));
                    scores[si.out + x] = (uint16_t)min(32768, max(0, __float2int_rn(p * 32768.0f)));
                }
            }
        }
        sync_point();
        si = sn;
    }
    stage2_wait();   // no copy outlives the CTA
    __syncthreads();
    if (abort && tid == 0) {   // let MMAs still in flight finish (bounded) before freeing TMEM
        mma_commit(bar_m);
        bar_wait(bar_m, phase, nullptr);
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, kInf2Cols);
}

size_t sc2_infer_smem() { return kInf2Smem; }

int sc2_infer_blocks_per_sm() {
    // shared memory per SM (each CTA also reserves 1 KB), at most 2 CTAs for
    // the 512 TMEM columns (256 each)
    static int nb = [] {
        int dev = 0, smem_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess)
            return 1;
        const int v = smem_sm / (int)(kInf2Smem + 1024);
        return v < 1 ? 1 : (v > 2 ? 2 : v);
    }();
    return nb;
}

cudaError_t sc2_launch_infer(const Sc2Source &src, const unsigned char *block, uint16_t *scores,
                             float *logits, int total_segs, uint32_t *err, int grid,
                             cudaStream_t s) {
    if (total_segs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sc2_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kInf2Smem);
    if (e != cudaSuccess) return e;
    k_sc2_infer<<<grid, kInf2Threads, kInf2Smem, s>>>(src, block, scores, logits, total_segs, err);
    return cudaGetLastError();
}

// ============================================================= training ==
// One CTA (8 warps, one CTA per SM) per segment, segments assigned statically
// (g = blockIdx.x + k gridDim.x) so that every run sums the same gradient
// terms in the same order.  Per segment: forward (features -> a1 -> a2 ->
// a3 -> head), soft cross-entropy and its gradient at the logits, then for
// layers 3, 2, 1 the weight gradient (tcgen05 with MN-major operands, M = 64
// rows, N = input channels, K = 16 columns per MMA) and, for layers 3 and 2,
// the input gradient (a forward convolution of the gradient planes with the
// transposed weights).  A weight-gradient MMA takes every gradient row of the
// layer in M (1 row of 32 channels, 3 of 16, 5 of 8: 32, 48 and 40 of the 64
// rows) and every input row in N (3 rows of 16 channels, 5 and 7 of 8), one
// accumulator per column tap: 3 x 24 MMAs per layer.  Gradient sums stay
// in shared memory across the CTA's segments; the CTA writes them to its own
// slice of `partial` at the end.
constexpr int kTrain2Threads = 256;
constexpr int kTrain2Planes = 24;   // D (6: dz3, then dz2, then dz1) | X (7) | A1 (5) | A2 (6)
constexpr int kTrain2Sum = 6272;    // floats of the CTA's gradient sums (+ loss)
constexpr size_t kTrain2Smem = (size_t)kTrain2Planes * kPlane + (kSc2BlockBytes - kSc2VecBytes) +
                               kSc2VecBytes + 64 + 4 * kTrain2Sum + 4 * 8 * 64;
constexpr int kDw = 256;            // TMEM column of the weight-gradient accumulators
static_assert(kTrain2Sum >= kScorer2dNParam + 1 && kTrain2Sum % 4 == 0, "sum slots");
static_assert(kTrain2Sum == kSc2PartialStride, "partial stride");
static_assert(kTrain2Smem <= 227 * 1024, "training shared memory fits one CTA per SM");
// weight-gradient accumulators: 3 column taps x (input planes x 8) columns
// (layer 1: 7 planes, layer 3: 6, layer 2: 5) above the convolutions' 240
static_assert(kDw >= 3 * 80 && kDw + 3 * 8 * 7 <= 512, "TMEM columns of the training kernel");

namespace {

// Weight-gradient MMAs of one layer, dW[co][ci][dr][dx] = sum over gradient
// rows r and columns x of dz[r][x][co] in[r + dr][x + dx - 1][ci], with every
// gradient row in M and every input row in N.  A = the 8 planes from `dz`
// (the layer's gradient rows: 1 of 32 channels, 3 of 16 or 5 of 8, row by
// row; planes after the last row unused), B = the n_in planes of all the
// layer's input rows (consecutive, row by row) shifted by the column tap dx.
// Accumulator dx, N = 8 n_in columns at kDw + N dx, holds in row (r, co),
// column 8 p + c (input plane p, channel c), the sum over x of dz[r][x][co]
// plane_p[x + dx - 1][c]: the term of gradient row r for the input row of
// plane p, i.e. of row tap dr = (that input row) - r.
__device__ __forceinline__ void issue_dw2(uint32_t tmem, const unsigned char *dz,
                                          const unsigned char *in, int n_in) {
    const int N = 8 * n_in;
    const uint32_t idesc = idesc_bf16(64, N, true, true);
    const uint64_t da = sdesc(smem_u32(dz) + kG * 16, 128, kPlane);
    for (int dx = 0; dx < 3; ++dx) {
        const uint64_t db = sdesc(smem_u32(in) + (kG + dx - 1) * 16, 128, kPlane);
#pragma unroll 4
        for (int k = 0; k < kCols / 16; ++k)
            mma_bf16(tmem + kDw + N * dx, da + (uint32_t)(16 * k), db + (uint32_t)(16 * k), idesc,
                     k != 0);
    }
}

// Adds layer 3's weight gradient (one gradient row of 32 channels, input
// rows of two planes) into the sums, layout [co][ci][dr][dx] at `off`.  Row
// co of an M = 64 accumulator is in lane co % 16 of TMEM lane quarter co / 16;
// the quarter's two warps share the 9 taps.
__device__ __forceinline__ void flush_dw2_l3(uint32_t tmem, float *sum, int off) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
    if (q >= 2) return;
    const int co = 16 * q + lane;
    for (int t = h; t < 9; t += 2) {
        const int dr = t / 3, dx = t - 3 * dr;
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + kDw + 48 * dx + 16 * dr, v);
        if (lane < 16) {
            for (int ci = 0; ci < 16; ++ci) {
                float &dst = sum[off + (co * 16 + ci) * 9 + t];
                dst = __fadd_rn(dst, v[ci]);
            }
        }
    }
}

// Adds the weight gradient of layer 2 or 1 (R gradient rows of n_out
// channels, R + 2 input rows of one plane of n_in real channels) into the
// sums, layout [co][ci][dr][dx] at `off`.  Row 8 g + c of an M = 64
// accumulator (plane g of dz, channel c) is in lane 8 (g % 2) + c of TMEM
// lane quarter g / 2.  Each lane copies the terms of its gradient row to
// stage[r][co][ci][dr][dx] (each written once: input row r + dr), then the R
// terms of every weight are summed in row order.
__device__ __forceinline__ void flush_dw2_stacked(uint32_t tmem, float *stage, float *sum, int off,
                                                  int R, int n_out, int n_in) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
    const int ppr = n_out / 8;                       // planes per gradient row
    const int g = 2 * q + ((lane >> 3) & 1);         // plane of this lane's row
    const int r = g / ppr, co = 8 * (g % ppr) + (lane & 7);
    const bool mine = lane < 16 && r < R;
    const int per_r = n_out * n_in * 9;
    const int N = 8 * (R + 2);
    if (2 * q < R * ppr) {   // the quarter holds gradient rows (uniform over the warp)
        // (input row rho, column tap dx), i = 3 rho + dx; the quarter's two warps share them
        for (int i = h; i < 3 * (R + 2); i += 2) {
            const int rho = i / 3, dx = i - 3 * rho, dr = rho - r;
            float v[8];
            tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + kDw + N * dx + 8 * rho, v);
            if (mine && dr >= 0 && dr <= 2) {
                float *dst = stage + r * per_r + co * n_in * 9 + 3 * dr + dx;
                for (int ci = 0; ci < n_in; ++ci) dst[9 * ci] = v[ci];
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < per_r; t += blockDim.x) {
        float a = stage[t];
        for (int rr = 1; rr < R; ++rr) a = __fadd_rn(a, stage[rr * per_r + t]);
        sum[off + t] = __fadd_rn(sum[off + t], a);
    }
    __syncthreads();
}

// Sums a per-thread vector of n values over the CTA (fixed order) into
// sum[off + c]; red: 8 x 64 floats of scratch.
template <int NV>
__device__ __forceinline__ void flush_vec(const float (&v)[NV], float *red, float *sum, int off) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        float w = v[c];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) w = __fadd_rn(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) red[warp * 64 + c] = w;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float t = 0.0f;
        for (int k = 0; k < kTrain2Threads / 32; ++k) t = __fadd_rn(t, red[k * 64 + threadIdx.x]);
        sum[off + threadIdx.x] = __fadd_rn(sum[off + threadIdx.x], t);
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(kTrain2Threads, 1)
    k_sc2_train(Sc2Source src, const float *__restrict__ targets, float pos_weight,
                const unsigned char *__restrict__ wblock, float *__restrict__ partial,
                int total_segs, uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *D = sm;                     // gradient planes (the planes after them pad M = 64)
    unsigned char *X = sm + 6 * kPlane;
    unsigned char *A1 = X + 7 * kPlane;
    unsigned char *A2 = A1 + 5 * kPlane;       // also the weight-gradient stage of layers 2 and 1
    float *stage = reinterpret_cast<float *>(A2);
    unsigned char *Wall = sm + kTrain2Planes * kPlane;
    Sc2Vec *vec = reinterpret_cast<Sc2Vec *>(Wall + (kSc2BlockBytes - kSc2VecBytes));
    uint64_t *bar_w = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(vec) + kSc2VecBytes);
    uint64_t *bar_m = bar_w + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 1);
    float *sum = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(bar_w) + 64);
    float *red = sum + kTrain2Sum;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, half = warp >> 2;
    zero_guards(sm, kTrain2Planes);
    for (int i = tid; i < kTrain2Sum; i += kTrain2Threads) sum[i] = 0.0f;
    if (tid == 0) {
        bar_init(bar_w, 1);
        bar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        bar_expect_tx(bar_w, kSc2BlockBytes);
        bulk_g2s(Wall, wblock, kSc2BlockBytes - kSc2VecBytes, bar_w);
        bulk_g2s(vec, wblock + kSc2OffVec, kSc2VecBytes, bar_w);
    }
    bool abort = __syncthreads_or(!bar_wait(bar_w, 0, err)) != 0;
    uint32_t phase = 0;
    const unsigned char *W3b = Wall + kSc2OffW3b, *W2b = Wall + kSc2OffW2b;

    auto sync_point = [&]() {
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
    };
    auto wait_mma = [&]() {
        const bool ok = bar_wait(bar_m, phase, err);
        phase ^= 1u;
        tc_after_sync();
        if (__syncthreads_or(!ok)) abort = true;
        return !abort;
    };

    for (int g = blockIdx.x; g < total_segs && !abort; g += gridDim.x) {
        const Seg2 si = seg2_info(src, g);
        const int b0 = si.s0 - kSc2Halo;
        const float *tgt = targets + (int64_t)si.strip * si.W;
        __syncthreads();
        build_x(X, si, b0);
        sync_point();
        // ---- forward: layer 1
        if (tid == 0) {
            issue_conv8(tmem, X, Wall + kSc2OffW1, 5, 80);
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        for (int it = half; it < kSc2Tiles * 5; it += 2) {
            const int j = it / 5, r = it - 5 * j;
            float v[8];
            tmem_ld8(tq(tmem, 80 * j + 16 * r), v);
            const int row = kTile * j + 32 * q + lane, x = b0 + row;
            *reinterpret_cast<uint4 *>(A1 + r * kPlane + (kG + row) * 16) =
                relu_row8(v, vec->b1, x >= 0 && x < si.W);
        }
        sync_point();
        // ---- layer 2
        if (tid == 0) {
            issue_conv8(tmem, A1, Wall + kSc2OffW2, 3, 48);
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        for (int it = half; it < kSc2Tiles * 3; it += 2) {
            const int j = it / 3, r = it - 3 * j;
            float v[16];
            tmem_ld16(tq(tmem, 48 * j + 16 * r), v);
            const int row = kTile * j + 32 * q + lane, x = b0 + row;
            const bool inside = x >= 0 && x < si.W;
            *reinterpret_cast<uint4 *>(A2 + 2 * r * kPlane + (kG + row) * 16) =
                relu_row8(v, vec->b2, inside);
            *reinterpret_cast<uint4 *>(A2 + (2 * r + 1) * kPlane + (kG + row) * 16) =
                relu_row8(v + 8, vec->b2 + 8, inside);
        }
        sync_point();
        // ---- layer 3, head, loss; gradient at the logits and at z3 (plane D, 4 planes)
        if (tid == 0) {
            issue_conv16(tmem, A2, Wall + kSc2OffW3);
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        {
            float gwh[32], gb3[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) gwh[c] = gb3[c] = 0.0f;
            float gbh = 0.0f, loss = 0.0f;
            for (int j = half; j < kSc2Tiles; j += 2) {
                float v[32];
                tmem_ld32(tq(tmem, 32 * j), v);
                const int row = kTile * j + 32 * q + lane, x = b0 + row;
                const bool out = x >= si.s0 && x < si.s1;
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    const uint32_t a = pack_relu_bf16(__fadd_rn(v[c], vec->b3[c]),
                                                      __fadd_rn(v[c + 1], vec->b3[c + 1]));
                    v[c] = out ? bf16_lo(a) : 0.0f;
                    v[c + 1] = out ? bf16_hi(a) : 0.0f;
                    acc = __fadd_rn(acc, __fmul_rn(vec->whq[c], v[c]));
                    acc = __fadd_rn(acc, __fmul_rn(vec->whq[c + 1], v[c + 1]));
                }
                float dl = 0.0f;
                if (out) {
                    const float lg = __fadd_rn(vec->bh, acc);
                    const float t = tgt[x];
                    const float w = __fadd_rn(1.0f, __fmul_rn(__fsub_rn(pos_weight, 1.0f), t));
                    const float p = 1.0f / (1.0f + expf(-lg));
                    dl = __fmul_rn(w, __fsub_rn(p, t));
                    const float sp = lg > 0.0f ? lg + log1pf(expf(-lg)) : log1pf(expf(lg));
                    loss = __fadd_rn(loss, __fmul_rn(w, __fsub_rn(sp, __fmul_rn(t, lg))));
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
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4)
                    *reinterpret_cast<uint4 *>(D + c4 * kPlane + (kG + row) * 16) = make_uint4(
                        pack_bf16(v[8 * c4], v[8 * c4 + 1]), pack_bf16(v[8 * c4 + 2], v[8 * c4 + 3]),
                        pack_bf16(v[8 * c4 + 4], v[8 * c4 + 5]), pack_bf16(v[8 * c4 + 6], v[8 * c4 + 7]));
            }
            // rows no warp wrote this segment are the tiles of the other half
            // of the warps: every row of D is written (half 0: tiles 0, 2;
            // half 1: tile 1)
            flush_vec<32>(gwh, red, sum, kSc2PWh);
            flush_vec<32>(gb3, red, sum, kSc2PB3);
            float tail[2] = {gbh, loss};
            flush_vec<2>(tail, red, sum, kSc2PBh);   // bh, then the loss slot after it
        }
        sync_point();
        // ---- layer 3: weight gradient (M: the 32 channels of dz3, N: the 3 a2
        // rows of 16) and the input gradient da2 (3 rows x 16 channels per tile)
        if (tid == 0) {
            issue_dw2(tmem, D, A2, 6);
            constexpr uint32_t idesc = idesc_bf16(128, 16, false, false);
            for (int j = 0; j < kSc2Tiles; ++j)
                for (int dr = 0; dr < 3; ++dr)
                    for (int dx = 0; dx < 3; ++dx)
                        for (int h2 = 0; h2 < 2; ++h2) {   // input channels 16 h2 .. 16 h2 + 15
                            const uint64_t da = sdesc(smem_u32(D + 2 * h2 * kPlane) +
                                                          (kG + kTile * j + 1 - dx) * 16,
                                                      kPlane, 128);
                            const uint64_t db = sdesc(smem_u32(W3b + (dr * 3 + dx) * 1024 + h2 * 512),
                                                      256, 128);
                            mma_bf16(tmem + 48 * j + 16 * dr, da, db, idesc, (dx | h2) != 0);
                        }
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        flush_dw2_l3(tmem, sum, kSc2PW3);
        {
            float gb[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) gb[c] = 0.0f;
            for (int it = half; it < kSc2Tiles * 3; it += 2) {
                const int j = it / 3, r = it - 3 * j;
                float v[16];
                tmem_ld16(tq(tmem, 48 * j + 16 * r), v);
                const int row = kTile * j + 32 * q + lane;
                const uint4 a0 = *reinterpret_cast<const uint4 *>(A2 + 2 * r * kPlane + (kG + row) * 16);
                const uint4 a1 = *reinterpret_cast<const uint4 *>(A2 + (2 * r + 1) * kPlane + (kG + row) * 16);
                const uint32_t aw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float a = (c & 1) ? bf16_hi(aw[c >> 1]) : bf16_lo(aw[c >> 1]);
                    v[c] = a > 0.0f ? __bfloat162float(__float2bfloat16_rn(v[c])) : 0.0f;
                    gb[c] = __fadd_rn(gb[c], v[c]);
                }
                // dz2 of row r: planes 2r, 2r + 1 of D (every MMA reading D is done)
                *reinterpret_cast<uint4 *>(D + 2 * r * kPlane + (kG + row) * 16) =
                    make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                               pack_bf16(v[6], v[7]));
                *reinterpret_cast<uint4 *>(D + (2 * r + 1) * kPlane + (kG + row) * 16) =
                    make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                               pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
            }
            flush_vec<16>(gb, red, sum, kSc2PB2);
        }
        sync_point();
        // ---- layer 2: weight gradient (M: the 3 dz2 rows of 16 channels, N: the
        // 5 a1 rows of 8) and the input gradient da1 (5 rows x 16 columns of which
        // 8 real per tile)
        if (tid == 0) {
            issue_dw2(tmem, D, A1, 5);
            constexpr uint32_t idesc = idesc_bf16(128, 16, false, false);
            for (int j = 0; j < kSc2Tiles; ++j)
                for (int r1 = 0; r1 < 5; ++r1) {
                    bool first = true;
                    for (int r = 0; r < 3; ++r) {
                        const int dr = r1 - r;
                        if (dr < 0 || dr > 2) continue;
                        for (int dx = 0; dx < 3; ++dx) {
                            const uint64_t da = sdesc(smem_u32(D + 2 * r * kPlane) +
                                                          (kG + kTile * j + 1 - dx) * 16,
                                                      kPlane, 128);
                            const uint64_t db = sdesc(smem_u32(W2b + (dr * 3 + dx) * 512), 256, 128);
                            mma_bf16(tmem + 80 * j + 16 * r1, da, db, idesc, first ? 0u : 1u);
                            first = false;
                        }
                    }
                }
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        flush_dw2_stacked(tmem, stage, sum, kSc2PW2, 3, 16, 8);   // a2 is no longer read
        {
            float gb[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) gb[c] = 0.0f;
            for (int it = half; it < kSc2Tiles * 5; it += 2) {
                const int j = it / 5, r = it - 5 * j;
                float v[8];
                tmem_ld8(tq(tmem, 80 * j + 16 * r), v);
                const int row = kTile * j + 32 * q + lane;
                const uint4 a0 = *reinterpret_cast<const uint4 *>(A1 + r * kPlane + (kG + row) * 16);
                const uint32_t aw[4] = {a0.x, a0.y, a0.z, a0.w};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float a = (c & 1) ? bf16_hi(aw[c >> 1]) : bf16_lo(aw[c >> 1]);
                    v[c] = a > 0.0f ? __bfloat162float(__float2bfloat16_rn(v[c])) : 0.0f;
                    gb[c] = __fadd_rn(gb[c], v[c]);
                }
                // dz1 of row r: plane r of D (every MMA reading D is done)
                *reinterpret_cast<uint4 *>(D + r * kPlane + (kG + row) * 16) =
                    make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                               pack_bf16(v[6], v[7]));
            }
            flush_vec<8>(gb, red, sum, kSc2PB1);
        }
        sync_point();
        // ---- layer 1: weight gradient only (M: the 5 dz1 rows of 8 channels,
        // N: the 7 feature rows of 8, of which 5 real)
        if (tid == 0) {
            issue_dw2(tmem, D, X, 7);
            mma_commit(bar_m);
        }
        if (!wait_mma()) break;
        flush_dw2_stacked(tmem, stage, sum, kSc2PW1, 5, 8, 5);
        zero_guards(A2, 6);   // the stage overwrote them; the next forward reads them
        tc_before_sync();
    }
    __syncthreads();
    // the CTA's sums to its slice of the partials (every CTA has a segment)
    float *part = partial + (size_t)blockIdx.x * kSc2PartialStride;
    for (int i = tid; i < kTrain2Sum; i += kTrain2Threads) part[i] = sum[i];
    if (abort && tid == 0) {   // let MMAs still in flight finish (bounded) before freeing TMEM
        mma_commit(bar_m);
        bar_wait(bar_m, phase, nullptr);
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 512);
}

size_t sc2_train_smem() { return kTrain2Smem; }

cudaError_t sc2_launch_train(const Sc2Source &src, const float *targets, float pos_weight,
                             const unsigned char *block, float *partial, int total_segs,
                             uint32_t *err, int grid, cudaStream_t s) {
    if (total_segs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sc2_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrain2Smem);
    if (e != cudaSuccess) return e;
    k_sc2_train<<<grid, kTrain2Threads, kTrain2Smem, s>>>(src, targets, pos_weight, block, partial,
                                                          total_segs, err);
    return cudaGetLastError();
}

// ================================================================ SGD ==
// Sums the per-CTA partials in a fixed order, then optionally a momentum SGD
// step (clipped by the global gradient norm when clip > 0), as the 1-D
// scorer's step: v = momentum v + f scale g, w = w - lr v, with w written
// into the device weight block.  64 parameters per block, 16 threads each
// (partials c = q, q + 16, ...), combined in order.
constexpr int kSgd2Params = 64;
constexpr int kSgd2Q = 16;

__global__ void __launch_bounds__(kSgd2Q * kSgd2Params)
    k_sc2_sgd(float *__restrict__ prm, float *__restrict__ mom, const float *__restrict__ part,
              int n_part, float scale, float lr, float momentum, int apply,
              float *__restrict__ grads_out, float *__restrict__ loss_out,
              float *__restrict__ gbuf, float *__restrict__ norm_part, unsigned char *__restrict__ blk) {
    __shared__ float red2[kSgd2Q][kSgd2Params];
    const int pl = threadIdx.x % kSgd2Params, qq = threadIdx.x / kSgd2Params;
    const int p = blockIdx.x * kSgd2Params + pl;
    float g = 0.0f;
    if (p <= kScorer2dNParam) {
        const float *src = part + p;
        int c = qq;
        for (; c + 7 * kSgd2Q < n_part; c += 8 * kSgd2Q) {   // eight loads in flight, added in order
            float t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = __ldcg(src + (size_t)(c + kSgd2Q * u) * kSc2PartialStride);
#pragma unroll
            for (int u = 0; u < 8; ++u) g = __fadd_rn(g, t[u]);
        }
        for (; c < n_part; c += kSgd2Q) g = __fadd_rn(g, __ldcg(src + (size_t)c * kSc2PartialStride));
    }
    red2[qq][pl] = g;
    __syncthreads();
    g = red2[0][pl];
#pragma unroll
    for (int k = 1; k < kSgd2Q; ++k) g = __fadd_rn(g, red2[k][pl]);
    if (norm_part) {
        __syncthreads();
        if (qq == 0) {
            const float m = __fmul_rn(scale, g);
            red2[1][pl] = p < kScorer2dNParam ? __fmul_rn(m, m) : 0.0f;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int i = 0; i < kSgd2Params; ++i) t = __fadd_rn(t, red2[1][i]);
            norm_part[blockIdx.x] = t;
        }
    }
    if (qq != 0 || p > kScorer2dNParam) return;
    if (p == kScorer2dNParam) {   // loss slot
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
        sc2_pack_one(p, w, blk);
    }
}

__global__ void __launch_bounds__(kSgd2Params)
    k_sc2_clip_step(float *__restrict__ prm, float *__restrict__ mom, const float *__restrict__ gbuf,
                    const float *__restrict__ norm_part, float scale, float lr, float momentum,
                    float clip, unsigned char *__restrict__ blk) {
    __shared__ float red2[kSgd2Params];
    __shared__ float f_s;
    float t = 0.0f;
    for (int i = threadIdx.x; i < kSc2SgdBlocks; i += kSgd2Params) t = __fadd_rn(t, __ldcg(norm_part + i));
    red2[threadIdx.x] = t;
    __syncthreads();
    for (int w = kSgd2Params / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red2[threadIdx.x] = __fadd_rn(red2[threadIdx.x], red2[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float n = sqrtf(red2[0]);
        f_s = n > clip ? __fdiv_rn(clip, n) : 1.0f;
    }
    __syncthreads();
    const int p = blockIdx.x * kSgd2Params + threadIdx.x;
    if (p >= kScorer2dNParam) return;
    const float m = __fmul_rn(f_s, __fmul_rn(scale, gbuf[p]));
    const float v = __fadd_rn(__fmul_rn(momentum, mom[p]), m);
    const float w = __fsub_rn(prm[p], __fmul_rn(lr, v));
    mom[p] = v;
    prm[p] = w;
    sc2_pack_one(p, w, blk);
}

cudaError_t sc2_launch_sgd(float *params, float *mom, float *partial, int n_partials, float scale,
                           float lr, float momentum, int apply, float clip, float *gbuf,
                           float *norm_part, float *grads_out, float *loss_out,
                           unsigned char *block, cudaStream_t s) {
    const bool clipped = apply && clip > 0.0f;
    k_sc2_sgd<<<kSc2SgdBlocks, kSgd2Q * kSgd2Params, 0, s>>>(
        params, mom, partial, n_partials, scale, lr, momentum, apply, grads_out, loss_out,
        clipped ? gbuf : nullptr, clipped ? norm_part : nullptr, block);
    if (clipped)
        k_sc2_clip_step<<<kSc2SgdBlocks, kSgd2Params, 0, s>>>(params, mom, gbuf, norm_part, scale,
                                                              lr, momentum, clip, block);
    return cudaGetLastError();
}

}  // namespace ca
