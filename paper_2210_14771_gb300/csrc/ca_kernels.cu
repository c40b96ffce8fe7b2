// ca_kernels.cu -- sm_103a kernels of the content-area pipeline.
//
//   k_strips  strip rows -> luma -> Sobel / angle / preceding-max features ->
//             Q15 score -> best points of each half-strip      (Sec. 2.2.2-2.2.3, 2.2.5)
//   k_fit     candidates -> RANSAC triples -> circumcircle -> inliers and
//             least-squares refits -> score, filters -> best circle  (Sec. 2.2.5)
//   k_mask    circle -> content-area mask (disc within the rectangle)  (Sec. 1.1, Fig. 1)
//
// Bit-exactness: every decision is taken either in exact integer arithmetic or
// in binary32/binary64 with explicitly rounded intrinsics (no contraction into
// fused multiply-adds), so the results are fully determined by the inputs and
// do not depend on launch shapes.
#include <cstdint>

#include "ca_internal.h"
#include "ca_fconv.h"

namespace ca {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// 16-byte streaming store.  No memory clobber: nothing in the issuing kernel
// reads the stored bytes, so the compiler may schedule around it freely.
__device__ __forceinline__ void st_cs_v4(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w));
}

// Integer BT.601 luma on the 0-255 scale.
__device__ __forceinline__ uint32_t luma(uint32_t r, uint32_t g, uint32_t b) {
    return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// 16 pixels (48 bytes of packed RGB) -> 16 luma bytes, with byte dot products:
// pixel 4m+t occupies bytes 12m+3t .. 12m+3t+2, so each pixel is one or two
// dp4a of its words against the weights (77, 150, 29) placed at its bytes.
__device__ __forceinline__ uint32_t luma4(uint32_t w0, uint32_t w1, uint32_t w2) {
    const uint32_t y0 = __dp4a(w0, 77u | (150u << 8) | (29u << 16), 128u) >> 8;
    const uint32_t y1 = __dp4a(w0, 77u << 24, __dp4a(w1, 150u | (29u << 8), 128u)) >> 8;
    const uint32_t y2 = __dp4a(w1, (77u << 16) | (150u << 24), __dp4a(w2, 29u, 128u)) >> 8;
    const uint32_t y3 = __dp4a(w2, (77u << 8) | (150u << 16) | (29u << 24), 128u) >> 8;
    return __byte_perm(__byte_perm(y0, y1, 0x3340), __byte_perm(y2, y3, 0x3340), 0x5410);
}

__device__ __forceinline__ uint4 luma16(uint4 a, uint4 b, uint4 c) {
    return make_uint4(luma4(a.x, a.y, a.z), luma4(a.w, b.x, b.y), luma4(b.z, b.w, c.x),
                      luma4(c.y, c.z, c.w));
}

// floor(sqrt(16 ng)) clamped to qsat (exact; the float estimate only seeds it).
__device__ __forceinline__ int qmag(int ng, int qsat) {
    const int n = ng << 4;
    if (n >= qsat * qsat) return qsat;
    const float fn = __int2float_rn(n);
    int r = __float2int_rz(__fmul_rn(fn, rsqrtf(fn)));
    r = max(r, 0);
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

// L2 load of a result (other CTAs may have written it during the kernel).  A
// result is 24 bytes with 4-byte alignment: loaded word by word.
__device__ __forceinline__ ca_result load_result(const ca_result *p) {
    ca_result r;
    r.cx = __ldcg(&p->cx);
    r.cy = __ldcg(&p->cy);
    r.r = __ldcg(&p->r);
    r.score = __ldcg(&p->score);
    r.valid = __ldcg(&p->valid);
    r.n_inliers = __ldcg(&p->n_inliers);
    return r;
}

}  // namespace

// ============================================================== k_strips ==
// One warp per half-strip: work items (frame, strip, half) are spread over all
// warps of the grid, and a warp never waits for another one.  The 8 warps of a
// CTA share the score tables in shared memory.  A warp keeps its half-strip
// plus one column of the other half as one 32-bit word per column: luma of
// rows h-1, h, h+1 in bytes 0, 1, 2.
constexpr int kStripWarps = kStripThreads / 32;

__host__ __device__ __forceinline__ int strip_lg_len(const DevParams &P) {
    return (P.qg_sat + 1 + 7) & ~7;
}

// Columns one warp may hold: half of the widest frame, the halo column and
// 16-pixel alignment at both ends.
__host__ __device__ __forceinline__ int strip_cols(const DevParams &P) {
    return ((P.max_w / 2 + 1 + 15) & ~15) + 32;
}

// Shared memory: part of the device table block -- s_iota, the s_g bounds of
// bins of 16 values of ng = |g|^2 (bin j holds ng in [16 j, 16 j + 15]; ng
// beyond the last bin is bounded by 32768) and s_g up to its saturation --
// then the column words of each warp and, for K > 2 only, the score of each
// pixel and the picks of each warp.  s_theta, needed only by the few pixels
// that get an exact score, is read through L1.
__host__ __device__ __forceinline__ size_t strip_tables_bytes(const DevParams &P) {
    return 2 * (size_t)(kDevOffG - kDevOffI + strip_lg_len(P));
}

// K = 2: each warp's queue of pixels awaiting their exact score (one round of
// 32 pushes on top of at most 31 waiting entries).
constexpr int kQueueCap = 64;
constexpr int kMaxBlocks = (kMaxDim / 2 + 31) / 32;   // 32-pixel blocks of a half-strip

// K = 2 (a CTA per strip): column words of the whole strip, then per half the
// block maxima and carries of the preceding maximum, the warps' queues and
// the two halves' best keys.
__host__ __device__ __forceinline__ int pair_words(const DevParams &P) {
    return ((P.max_w + 15) & ~15) + 16;
}

size_t strips_smem_bytes(const DevParams &P) {
    size_t b = strip_tables_bytes(P);
    if (P.K > 2)
        b += (size_t)kStripWarps * strip_cols(P) * 4 +
             (size_t)kStripWarps * (strip_cols(P) * 2 + 4 * (kMaxSlots / 2));
    else
        b += (size_t)pair_words(P) * 4 + 4 * 4 * kMaxBlocks +
             (size_t)kStripWarps * kQueueCap * sizeof(uint2) + 16;
    return b;
}

namespace {

// Luma of rows h-1, h, h+1 for 4 pixels (bytes of a, b, c) -> 4 column words.
__device__ __forceinline__ uint4 interleave4(uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t t01 = __byte_perm(a, b, 0x5140), t23 = __byte_perm(a, b, 0x7362);
    return make_uint4(__byte_perm(t01, c, 0x0410), __byte_perm(t01, c, 0x0532),
                      __byte_perm(t23, c, 0x0610), __byte_perm(t23, c, 0x0732));
}

// Float near a 64-bit integer of magnitude below 2^63 (relative error below
// 2^-22), from two 32-bit conversions.
__device__ __forceinline__ float approx_f32(long long v) {
    const uint64_t u = (uint64_t)(v < 0 ? -v : v);
    const float f = __fadd_rn(__fmul_rn(__uint2float_rn((uint32_t)(u >> 32)), 4294967296.0f),
                              __uint2float_rn((uint32_t)u));
    return v < 0 ? -f : f;
}

// Angle bin floor(4096 (u + 1)), u = dot |dot| / (ng nc) the signed squared
// cosine between g and c, as an exact integer quotient: a float estimate is
// corrected by one exact comparison (the estimate is within one bin).
__device__ __forceinline__ int qtheta(int dot, int ng, int nc) {
    const long long P = (long long)ng * nc;
    const long long d2 = (long long)dot * (dot < 0 ? -dot : dot);
    const long long num = (d2 + P) << 12;
    const float uf = __fdividef(approx_f32(d2), approx_f32(P));
    int q = __float2int_rz(__fmul_rn(__fadd_rn(uf, 1.0f), 4096.0f));
    q = min(max(q, 0), kLutT - 1);
    const long long t = (long long)q * P;
    if (t > num) --q;
    else if (t + P <= num) ++q;
    return min(max(q, 0), kLutT - 1);
}

struct StripCtx {
    int c2x, cy2;   // doubled centre x of the angle term; doubled vector y of the strip
    const uint16_t *lt, *lg, *li;
};

// Q15 score of Eq. 2-3 through the tables from a pixel's gradient.  Scores
// that cannot reach T_ps (bounded by the s_g s_iota product) count as 0: such
// pixels are never kept, and every kept pick is unchanged by it.
__device__ __forceinline__ uint32_t score_from_g(const StripCtx &c, int gx, int gy, int x,
                                                 int iota, const DevParams &P) {
    const int ng = gx * gx + gy * gy;
    const int cx2 = c.c2x - 2 * x;
    const int nc = cx2 * cx2 + c.cy2 * c.cy2;
    if (ng == 0 || nc == 0) return 0u;
    const uint32_t g = c.lg[qmag(ng, P.qg_sat)];
    const uint32_t ii = c.li[iota];
    if (((g * ii + 16384u) >> 15) < P.T_ps) return 0u;
    const uint32_t gt =
        (g * (uint32_t)__ldg(c.lt + qtheta(gx * cx2 + gy * c.cy2, ng, nc)) + 16384u) >> 15;
    return (gt * ii + 16384u) >> 15;
}

// Angle cut: false when the pixel's angle bin certainly has s_theta < T_ps, so
// that its score (at most s_theta) can never be kept.  The bins below the cut
// are those with u = dot |dot| / (ng nc) < u_cut; the host passes u_cut lowered
// by a margin far above the rounding error of this binary32 test, so the cut
// never drops a pixel whose bin reaches the threshold.
__device__ __forceinline__ bool angle_ok(const StripCtx &c, int gx, int gy, int x, int ng,
                                         const DevParams &P) {
    if (!P.theta_cut_on) return true;
    const int cx2 = c.c2x - 2 * x;
    const int dot = gx * cx2 + gy * c.cy2;
    const float fd = __int2float_rn(dot);
    const float fnc = __int2float_rn(cx2 * cx2 + c.cy2 * c.cy2);
    return __fmul_rn(fd, fabsf(fd)) >= __fmul_rn(P.theta_u_cut, __fmul_rn(__int2float_rn(ng), fnc));
}

}  // namespace

namespace {

// Shared-memory view of one strip CTA: the tables (copied once per CTA) and
// the per-warp buffers.
struct StripShared {
    const uint16_t *li, *lgb, *lg;   // s_iota, s_g bin bounds, s_g
    unsigned char *wmem;             // per-warp column words (+ scores, picks), or the
                                     // strip's words, block carries and queues (K = 2)
};

// Copies the table block from s_iota on into shared memory: every 16-byte
// load of a thread is issued before its stores (one L2 round trip per CTA).
__device__ __forceinline__ void strip_tables_load(const DevParams &P, const uint16_t *luts,
                                                  uint16_t *tab) {
    constexpr int kPer = ((kDevTableU16 - kDevOffI) / 8 + kStripThreads - 1) / kStripThreads;
    const int n16 = (int)(strip_tables_bytes(P) / 16);
    const uint4 *src = reinterpret_cast<const uint4 *>(luts + kDevOffI);
    uint4 *dst = reinterpret_cast<uint4 *>(tab);
    uint4 v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * kStripThreads;
        if (i < n16) v[k] = __ldg(src + i);
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * kStripThreads;
        if (i < n16) dst[i] = v[k];
    }
}

// Doubled centre of the angle term of frame f in a tracked call with
// prior-guided scoring: the previous accepted circle of its track, 2 cx and
// 2 cy rounded to the nearest integer (ties to even) and clamped into
// [0, 2(W-1)] x [0, 2(H-1)]; the image centre (W-1, H-1) otherwise.  Out of
// line: it runs once per half-strip and keeps the scan's registers free.
__device__ __noinline__ int2 prior_centre2(const int32_t *trk, const ca_result *state, int f,
                                           int W, int H) {
    int2 c2 = make_int2(W - 1, H - 1);
    const int t = trk[f];
    if (t >= 0) {
        const ca_result pr = load_result(state + t);
        if (pr.valid) {
            c2.x = min(max(__float2int_rn(__fmul_rn(2.0f, pr.cx)), 0), 2 * (W - 1));
            c2.y = min(max(__float2int_rn(__fmul_rn(2.0f, pr.cy)), 0), 2 * (H - 1));
        }
    }
    return c2;
}

// K > 2: half `half` of strip i of frame f by the calling warp alone: the
// exact score of every pixel, then K/2 picks, each excluding +-sup_px around
// the earlier ones.
__device__ __forceinline__ void strip_half(const DevFrame *__restrict__ frames,
                                           const int32_t *__restrict__ rows, const DevParams &P,
                                           const uint16_t *__restrict__ lt, const StripShared &ss,
                                           CandSlot *__restrict__ slots, int f, int i, int half) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cols = strip_cols(P);
    const uint16_t *li = ss.li, *lg = ss.lg;
    uint32_t *yy = reinterpret_cast<uint32_t *>(ss.wmem) + warp * cols;
    uint16_t *sc = reinterpret_cast<uint16_t *>(ss.wmem + (size_t)kStripWarps * cols * 4) + warp * cols;
    int *s_pick = reinterpret_cast<int *>(ss.wmem + (size_t)kStripWarps * cols * 6) + warp * (kMaxSlots / 2);
    const int kk = P.K >> 1;   // picks per half-strip
    const DevFrame fr = frames[f];
    const int W = fr.W, H = fr.H;
    const int y = rows[fr.rows_off + i];
    const int hw = W >> 1;
    const int c_lo = half ? hw - 1 : 0, c_hi = half ? W : hw + 1;   // columns of the half
    const int len = half ? (W - hw) : hw;
    // the half's scan positions [q0, q1) and the columns they need (one
    // neighbour on each side)
    const int q0 = 0, q1 = len;
    int col_lo = c_lo, col_hi = c_lo;
    if (q0 < q1) {
        const int xa = half ? W - q1 : q0, xb = half ? W - 1 - q0 : q1 - 1;
        col_lo = max(xa - 1, c_lo);
        col_hi = min(xb + 2, c_hi);
    }
    int base = col_lo;
    __syncwarp();   // the previous item is done with yy / sc

    // ---- rows y-1, y, y+1 -> column words (16-byte loads when aligned);
    // returns this lane's maximum of the middle row over columns [xa, xb]
    auto load_words = [&](int xa, int xb) -> int {
        int qm = 0;
        if (fr.vec_ok) {
            const int g0 = col_lo >> 4, g1 = (col_hi + 15) >> 4;
            base = g0 << 4;
            const uint8_t *r0 = fr.rgb + (int64_t)(y - 1) * fr.pitch;
            for (int g = g0 + lane; g < g1; g += 32) {
                const uint8_t *p0 = r0 + g * 48, *p1 = p0 + fr.pitch, *p2 = p1 + fr.pitch;
                const uint4 a0 = ld_nc_v4(p0), b0 = ld_nc_v4(p0 + 16), c0 = ld_nc_v4(p0 + 32);
                const uint4 a1 = ld_nc_v4(p1), b1 = ld_nc_v4(p1 + 16), c1 = ld_nc_v4(p1 + 32);
                const uint4 a2 = ld_nc_v4(p2), b2 = ld_nc_v4(p2 + 16), c2 = ld_nc_v4(p2 + 32);
                const uint4 L0 = luma16(a0, b0, c0), L1 = luma16(a1, b1, c1), L2 = luma16(a2, b2, c2);
                uint4 *dst = reinterpret_cast<uint4 *>(yy + (g - g0) * 16);
                dst[0] = interleave4(L0.x, L1.x, L2.x);
                dst[1] = interleave4(L0.y, L1.y, L2.y);
                dst[2] = interleave4(L0.z, L1.z, L2.z);
                dst[3] = interleave4(L0.w, L1.w, L2.w);
                // middle-row maximum over the group's pixels inside [xa, xb]
                const int x0 = 16 * g;
                uint32_t m;
                if (x0 >= xa && x0 + 15 <= xb) {
                    m = __vmaxu4(__vmaxu4(L1.x, L1.y), __vmaxu4(L1.z, L1.w));
                } else {
                    const uint32_t wv[4] = {L1.x, L1.y, L1.z, L1.w};
                    m = 0u;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int x = x0 + k;
                        if (x >= xa && x <= xb) m = max(m, (wv[k >> 2] >> (8 * (k & 3))) & 0xffu);
                    }
                }
                m = __vmaxu4(m, m >> 16);
                m = __vmaxu4(m, m >> 8);
                qm = max(qm, (int)(m & 0xffu));
            }
        } else {
            base = col_lo;
            for (int cc = col_lo + lane; cc < col_hi; cc += 32) {
                const uint8_t *p0 = fr.rgb + (int64_t)(y - 1) * fr.pitch + 3 * cc;
                const uint8_t *p1 = p0 + fr.pitch, *p2 = p1 + fr.pitch;
                const uint32_t m1 = luma(p1[0], p1[1], p1[2]);
                yy[cc - base] = luma(p0[0], p0[1], p0[2]) | (m1 << 8) | (luma(p2[0], p2[1], p2[2]) << 16);
                if (cc >= xa && cc <= xb) qm = max(qm, (int)m1);
            }
        }
        __syncwarp();
        return qm;
    };

    // the angle term's centre, doubled: the image centre, or in a tracked
    // call with prior-guided scoring the previous accepted circle's centre
    // (rounded to half pixels, ties to even, clamped into the frame)
    int2 c2 = make_int2(W - 1, H - 1);
    if (P.prior_centre) c2 = prior_centre2(P.trk, P.trk_state, f, W, H);
    const StripCtx ctx{c2.x, c2.y - 2 * y, lt, lg, li};
    const int dir = half ? -1 : 1;
    uint32_t best = 0u;

    load_words(0, -1);
    // ---- K > 2: exact score per pixel over this lane's chunk, with a
    // sliding window of the vertical Sobel sums
    const int cpl = (len + 31) >> 5;
    const int p0 = min(lane * cpl, len), p1 = min(p0 + cpl, len);
    const int xs = half ? (W - 1 - p0) : p0;
    int lm = 0;
    for (int p = p0, x = xs; p < p1; ++p, x += dir) lm = max(lm, (int)((yy[x - base] >> 8) & 0xff));
    int inc = lm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc = max(inc, t);
    }
    int run = __shfl_up_sync(kFull, inc, 1);
    if (lane == 0) run = 0;
    auto col = [&](int cc, int &S, int &T, int &M) {
        cc = min(max(cc, c_lo), c_hi - 1);
        const uint32_t w = yy[cc - base];
        const int u = w & 0xff, m = (w >> 8) & 0xff, d = (w >> 16) & 0xff;
        S = u + 2 * m + d;
        T = d - u;
        M = m;
    };
    int S0, T0, M0, S1, T1, M1;
    col(xs - dir, S0, T0, M0);
    col(xs, S1, T1, M1);
    // the preceding maximum never decreases along the scan: once it
    // reaches io_cut no later pixel of the half can be kept
    for (int p = p0, x = xs; p < p1; ++p, x += dir) {
        uint32_t sv = 0u;
        if (run < P.io_cut) {
            int S2, T2, M2;
            col(x + dir, S2, T2, M2);
            if (x != 0 && x != W - 1) {
                const int gx = dir * (S2 - S0), gy = T0 + 2 * T1 + T2;
                const int ng = gx * gx + gy * gy;
                if (ng != 0 && angle_ok(ctx, gx, gy, x, ng, P))
                    sv = score_from_g(ctx, gx, gy, x, run, P);
            }
            run = max(run, M1);
            S0 = S1; T0 = T1; S1 = S2; T1 = T2; M1 = M2;
        }
        sc[x - base] = (uint16_t)sv;
    }

    // ---- K/2 picks per half, each excluding +-sup_px around earlier picks
    for (int r = 0; r < kk; ++r) {
        {
            const int cpl = (len + 31) >> 5;
            const int p0 = min(lane * cpl, len), p1 = min(p0 + cpl, len);
            const int xs = half ? (W - 1 - p0) : p0;
            uint32_t b = 0u;
            for (int p = p0, x = xs; p < p1; ++p, x += dir) {
                bool sup = false;
                for (int j = 0; j < r; ++j) sup |= abs(x - s_pick[j]) <= P.sup_px;
                if (!sup)
                    b = max(b, ((uint32_t)sc[x - base] << 16) | (uint32_t)(half ? x : (0xFFFF - x)));
            }
            best = __reduce_max_sync(kFull, b);
        }
        int px = -1000000;
        CandSlot out;
        out.kept = 0;
        out.x = -1;
        out.y = (int16_t)y;
        out.s = 0;
        if (best != 0u) {
            const int rank = (int)(best & 0xFFFFu);
            px = half ? rank : (0xFFFF - rank);
            const uint32_t scv = best >> 16;
            out.x = (int16_t)px;
            out.s = (uint16_t)scv;
            out.kept = (uint16_t)(scv >= P.T_ps && px >= P.T_px && px <= W - 1 - P.T_px &&
                                  y >= P.T_px && y <= H - 1 - P.T_px);
        }
        if (lane == 0) {
            s_pick[r] = px;
            store_slot(slots + (int64_t)f * kMaxSlots + i * P.K + half * kk + r, out);
        }
        __syncwarp();   // this round's pick visible to the whole warp
    }
}

// K = 2: both halves of strip i of frame f by the whole CTA, the best point of
// each half into its candidate slot.  The preceding maximum iota of a pixel
// depends only on the middle row before it, so it is known for every block
// of 32 scan positions up front (the maximum of the earlier blocks, then a
// warp scan inside the block); the blocks whose carry has not reached io_cut
// -- the border region from each outer edge to the content -- are then
// independent and are shared out among the 8 warps.  A pixel's key is
// (Q15 score << 16) | outer rank exactly as the paper's argmax needs; the
// exact score is formed only for pixels that pass the angle cut and whose
// bound beats the best key so far, 32 at a time from each warp's queue.
__device__ __forceinline__ void strip_pair(const DevFrame *__restrict__ frames,
                                           const int32_t *__restrict__ rows, const DevParams &P,
                                           const uint16_t *__restrict__ lt, const StripShared &ss,
                                           CandSlot *__restrict__ slots, int f, int i) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *li = ss.li, *lgb = ss.lgb, *lg = ss.lg;
    uint32_t *yy = reinterpret_cast<uint32_t *>(ss.wmem);           // column words, x = 0 .. W-1
    int *bmax = reinterpret_cast<int *>(yy + pair_words(P));        // [2][kMaxBlocks]
    int *carry = bmax + 2 * kMaxBlocks;                              // [2][kMaxBlocks]
    uint2 *queue = reinterpret_cast<uint2 *>(carry + 2 * kMaxBlocks) + warp * kQueueCap;
    uint32_t *s_best = reinterpret_cast<uint32_t *>(queue - warp * kQueueCap + kStripWarps * kQueueCap);
    int *s_live = reinterpret_cast<int *>(s_best + 2);
    const DevFrame fr = frames[f];
    const int W = fr.W, H = fr.H;
    const int y = rows[fr.rows_off + i];
    const int hw = W >> 1;
    const int len[2] = {hw, W - hw};                  // scan positions of each half
    const int nb0 = (len[0] + 31) >> 5, nb1 = (len[1] + 31) >> 5;
    __syncthreads();   // the previous item is done with the words and queues

    // ---- rows y-1, y, y+1 of the whole strip -> column words.  With
    // 64-column alignment (W a multiple of 64) every block of 32 scan
    // positions of either half is one aligned group of 32 columns, so its
    // middle-row maximum comes from the two 16-column groups of a lane pair.
    const bool blocks_aligned = fr.vec_ok && (W & 63) == 0;
    if (fr.vec_ok) {
        const uint8_t *r0 = fr.rgb + (int64_t)(y - 1) * fr.pitch;
        for (int g = tid; g < (W >> 4); g += blockDim.x) {
            const uint8_t *p0 = r0 + g * 48, *p1 = p0 + fr.pitch, *p2 = p1 + fr.pitch;
            const uint4 a0 = ld_nc_v4(p0), b0 = ld_nc_v4(p0 + 16), c0 = ld_nc_v4(p0 + 32);
            const uint4 a1 = ld_nc_v4(p1), b1 = ld_nc_v4(p1 + 16), c1 = ld_nc_v4(p1 + 32);
            const uint4 a2 = ld_nc_v4(p2), b2 = ld_nc_v4(p2 + 16), c2 = ld_nc_v4(p2 + 32);
            const uint4 L0 = luma16(a0, b0, c0), L1 = luma16(a1, b1, c1), L2 = luma16(a2, b2, c2);
            uint4 *dst = reinterpret_cast<uint4 *>(yy + g * 16);
            dst[0] = interleave4(L0.x, L1.x, L2.x);
            dst[1] = interleave4(L0.y, L1.y, L2.y);
            dst[2] = interleave4(L0.z, L1.z, L2.z);
            dst[3] = interleave4(L0.w, L1.w, L2.w);
            if (blocks_aligned) {   // W / 16 is even: lanes g and g ^ 1 are both here
                uint32_t m = __vmaxu4(__vmaxu4(L1.x, L1.y), __vmaxu4(L1.z, L1.w));
                m = __vmaxu4(m, m >> 16);
                m = __vmaxu4(m, m >> 8);
                m &= 0xffu;
                m = max(m, __shfl_xor_sync(__activemask(), m, 1));
                const int G = g >> 1;   // columns [32 G, 32 G + 32)
                if ((g & 1) == 0) {
                    if (32 * G < hw) bmax[G] = (int)m;
                    else bmax[kMaxBlocks + (W >> 5) - 1 - G] = (int)m;
                }
            }
        }
    } else {
        for (int x = tid; x < W; x += blockDim.x) {
            const uint8_t *p0 = fr.rgb + (int64_t)(y - 1) * fr.pitch + 3 * x;
            const uint8_t *p1 = p0 + fr.pitch, *p2 = p1 + fr.pitch;
            yy[x] = luma(p0[0], p0[1], p0[2]) | (luma(p1[0], p1[1], p1[2]) << 8) |
                    (luma(p2[0], p2[1], p2[2]) << 16);
        }
    }
    __syncthreads();
    // ---- middle-row maximum of every block of 32 scan positions
    for (int k = warp; k < nb0 + nb1 && !blocks_aligned; k += kStripWarps) {
        const int h = k < nb0 ? 0 : 1, b = h ? k - nb0 : k;
        const int p = 32 * b + lane;
        int m = 0;
        if (p < len[h]) m = (int)((yy[h ? W - 1 - p : p] >> 8) & 0xffu);
        m = __reduce_max_sync(kFull, m);
        if (lane == 0) bmax[h * kMaxBlocks + b] = m;
    }
    __syncthreads();
    // ---- carry of each block (maximum of the earlier blocks of its half) and
    // the live blocks (carry below io_cut; the carry never decreases)
    if (warp < 2) {
        const int h = warp, nb = h ? nb1 : nb0;
        int run = 0, live = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            int inc = b < nb ? bmax[h * kMaxBlocks + b] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc = max(inc, t);
            }
            int excl = __shfl_up_sync(kFull, inc, 1);
            if (lane == 0) excl = 0;
            const int c = max(run, excl);
            if (b < nb) carry[h * kMaxBlocks + b] = c;
            live += __popc(__ballot_sync(kFull, b < nb && c < P.io_cut));
            run = max(run, __shfl_sync(kFull, inc, 31));
        }
        if (lane == 0) {
            s_live[h] = live;
            // every scanned pixel has at least the key of score 0, (0 << 16) |
            // rank; the largest is the half's first pixel (ranks fall along
            // the scan)
            const int x = h ? W - 1 : 0;
            s_best[h] = live > 0 ? (uint32_t)(h ? x : (0xFFFF - x)) : 0u;
        }
    }
    __syncthreads();

    // ---- the live blocks of both halves, shared out among the warps
    const int2 c2 = P.prior_centre ? prior_centre2(P.trk, P.trk_state, f, W, H)
                                   : make_int2(W - 1, H - 1);
    const StripCtx ctx{c2.x, c2.y - 2 * y, lt, lg, li};
    const int L0 = s_live[0], L1 = s_live[1];
    uint32_t best0 = s_best[0], best1 = s_best[1];   // this warp's best keys
    int qn = 0;
    auto flush = [&]() {
        __syncwarp();   // the pushes are visible
        for (int e0 = 0; e0 < qn; e0 += 32) {
            uint32_t k0 = 0u, k1 = 0u;
            if (e0 + lane < qn) {
                const uint2 e = queue[e0 + lane];
                const int x = (int)(e.x >> 16), iota = (int)(e.x & 0xffu), h = (int)((e.x >> 8) & 1u);
                const int gx = (int)(int16_t)(e.y & 0xffffu), gy = (int)(int16_t)(e.y >> 16);
                const uint32_t key = (score_from_g(ctx, gx, gy, x, iota, P) << 16) |
                                     (uint32_t)(h ? x : (0xFFFF - x));
                if (h) k1 = key; else k0 = key;
            }
            best0 = max(best0, __reduce_max_sync(kFull, k0));
            best1 = max(best1, __reduce_max_sync(kFull, k1));
        }
        qn = 0;
        __syncwarp();   // the entries are read before new pushes
    };
    // chunks of kPpl live blocks (32 kPpl scan positions), kPpl consecutive
    // positions per lane: a serial prefix maximum inside the lane, one warp
    // scan per chunk, and the Sobel terms from the lane's kPpl + 2 column words
    constexpr int kPpl = 2;
    const int C0 = (L0 + kPpl - 1) / kPpl, C1 = (L1 + kPpl - 1) / kPpl;
    for (int k = warp; k < C0 + C1; k += kStripWarps) {
        const int h = k < C0 ? 0 : 1, c = h ? k - C0 : k;
        const int cin = carry[h * kMaxBlocks + kPpl * c];
        const uint32_t bh = h ? best1 : best0;
        // no pixel of this chunk (its s_iota <= s_iota(cin)) can beat the best
        if (bh != 0u && (bh >> 16) >= (uint32_t)li[cin]) continue;
        const int p0 = 32 * kPpl * c + kPpl * lane, lh = len[h];
        // sw[i]: the column word of scan position p0 - 1 + i (clamped into the row)
        uint32_t sw[kPpl + 2];
#pragma unroll
        for (int i = 0; i < kPpl + 2; ++i) {
            const int xc = h ? W - p0 - i : p0 - 1 + i;
            sw[i] = yy[min(max(xc, 0), W - 1)];
        }
        int lp[kPpl];   // inclusive prefix maxima of the middle row along the lane
        int run = 0;
#pragma unroll
        for (int j = 0; j < kPpl; ++j) {
            if (p0 + j < lh) run = max(run, (int)((sw[j + 1] >> 8) & 0xffu));
            lp[j] = run;
        }
        int inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc = max(inc, t);
        }
        int excl = __shfl_up_sync(kFull, inc, 1);
        if (lane == 0) excl = 0;
        const int base = max(cin, excl);   // preceding maximum of the lane's first position
        // no pixel of this lane (s_iota <= s_iota(base)) can beat the best
        const bool lane_live = !(bh != 0u && (bh >> 16) >= (uint32_t)li[base]);
#pragma unroll
        for (int j = 0; j < kPpl; ++j) {
            const int p = p0 + j;
            const int x = h ? (W - 1 - p) : p;
            const int iota = j ? max(base, lp[j - 1]) : base;
            bool cand = false;
            uint2 ent = make_uint2(0u, 0u);
            if (lane_live && p < lh && iota < P.io_cut && x != 0 && x != W - 1) {
                // columns x - 1, x, x + 1 (the scan runs right to left in the right half)
                const uint32_t w0 = h ? sw[j + 2] : sw[j], w1 = sw[j + 1];
                const uint32_t w2 = h ? sw[j] : sw[j + 2];
                const int u0 = w0 & 0xff, m0 = (w0 >> 8) & 0xff, d0 = (w0 >> 16) & 0xff;
                const int u1 = w1 & 0xff, d1 = (w1 >> 16) & 0xff;
                const int u2 = w2 & 0xff, m2 = (w2 >> 8) & 0xff, d2 = (w2 >> 16) & 0xff;
                const int gx = (u2 + 2 * m2 + d2) - (u0 + 2 * m0 + d0);
                const int gy = (d0 + 2 * d1 + d2) - (u0 + 2 * u1 + u2);
                const int ng = gx * gx + gy * gy;
                if (ng != 0 && angle_ok(ctx, gx, gy, x, ng, P)) {
                    const uint32_t gub = (ng >> 4) < kBoundBins ? (uint32_t)lgb[ng >> 4] : 32768u;
                    const uint32_t bound = (gub * (uint32_t)li[iota] + 16384u) >> 15;
                    const uint32_t rank = (uint32_t)(h ? x : (0xFFFF - x));
                    cand = ((bound << 16) | rank) > bh;   // could beat the best so far
                    ent = make_uint2(((uint32_t)x << 16) | ((uint32_t)h << 8) | (uint32_t)iota,
                                     ((uint32_t)gx & 0xffffu) | ((uint32_t)gy << 16));
                }
            }
            const unsigned bal = __ballot_sync(kFull, cand);
            if (cand) queue[qn + __popc(bal & ((1u << lane) - 1u))] = ent;
            qn += __popc(bal);
            if (qn >= 32) flush();
        }
    }
    if (qn > 0) flush();
    if (lane == 0) {
        atomicMax(s_best, best0);
        atomicMax(s_best + 1, best1);
    }
    __syncthreads();
    // ---- the best point of each half into its slot
    if (tid < 2) {
        const int h = tid;
        const uint32_t best = s_best[h];
        CandSlot out;
        out.kept = 0;
        out.x = -1;
        out.y = (int16_t)y;
        out.s = 0;
        if (best != 0u) {
            const int rank = (int)(best & 0xFFFFu);
            const int px = h ? rank : (0xFFFF - rank);
            const uint32_t scv = best >> 16;
            out.x = (int16_t)px;
            out.s = (uint16_t)scv;
            out.kept = (uint16_t)(scv >= P.T_ps && px >= P.T_px && px <= W - 1 - P.T_px &&
                                  y >= P.T_px && y <= H - 1 - P.T_px);
        }
        store_slot(slots + (int64_t)f * kMaxSlots + i * P.K + h, out);
    }
}

}  // namespace

__global__ void __launch_bounds__(kStripThreads)
    k_strips(const DevFrame *__restrict__ frames, int B, const int32_t *__restrict__ rows,
             DevParams P, const uint16_t *__restrict__ luts, CandSlot *__restrict__ slots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);   // table block from s_iota on
    strip_tables_load(P, luts, tab);
    __syncthreads();
    const StripShared ss{tab, tab + (kDevOffB - kDevOffI), tab + (kDevOffG - kDevOffI),
                         smem_raw + strip_tables_bytes(P)};
    const uint16_t *lt = luts + kDevOffT;   // global, through L1

    // K = 2: the CTA takes a strip; K > 2: a warp takes a half-strip.  Items
    // are interleaved across frames (consecutive items belong to consecutive
    // frames), so every CTA and SM gets a mix of cheap and expensive strips.
    if (P.K == 2) {
        for (int it = blockIdx.x; it < B * P.N; it += gridDim.x) {
            const int i = it / B;
            strip_pair(frames, rows, P, lt, ss, slots, it - i * B, i);
        }
        return;
    }
    const int items = B * P.N * 2;
    for (int it = blockIdx.x * kStripWarps + warp; it < items; it += gridDim.x * kStripWarps) {
        const int j = it / B;
        const int f = it - j * B;
        strip_half(frames, rows, P, lt, ss, slots, f, j >> 1, j & 1);
    }
}

namespace {
// Largest dynamic shared memory k_strips can ask for (W = 4096, full s_g table).
cudaError_t strips_allow_max_smem() {
    static cudaError_t once = [] {
        DevParams P{};
        P.max_w = kMaxDim;
        P.K = 4;
        P.qg_sat = kLutG - 1;
        return cudaFuncSetAttribute(k_strips, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)strips_smem_bytes(P));
    }();
    return once;
}
}  // namespace

cudaError_t strips_occupancy(int *blocks_per_sm, size_t smem) {
    cudaError_t e = strips_allow_max_smem();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_strips, kStripThreads,
                                                         smem);
}

cudaError_t launch_strips(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                          const uint16_t *luts, CandSlot *slots, int grid, cudaStream_t s) {
    cudaError_t e = strips_allow_max_smem();
    if (e != cudaSuccess) return e;
    k_strips<<<grid, kStripThreads, strips_smem_bytes(P), s>>>(frames, B, rows, P, luts, slots);
    return cudaGetLastError();
}

// ================================================================= k_fit ==
namespace {

// Correctly rounded binary32 value of a 128-bit integer (integer arithmetic:
// ca_fconv.h).
__device__ __forceinline__ float i128_to_f32(__int128 v) {
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const float f = u128_to_f32((uint64_t)(u >> 64), (uint64_t)u);
    return neg ? -f : f;
}

struct Circle {
    float cx, cy, r;
};

// Circle through three points (origin-relative integers); false if collinear.
__device__ __forceinline__ bool circumcircle(int ax, int ay, int bx, int by, int cx, int cy,
                                             Circle &o) {
    const long long D = 2 * ((long long)ax * (by - cy) + (long long)bx * (cy - ay) +
                             (long long)cx * (ay - by));
    if (D == 0) return false;
    const long long a2 = (long long)ax * ax + (long long)ay * ay;
    const long long b2 = (long long)bx * bx + (long long)by * by;
    const long long c2 = (long long)cx * cx + (long long)cy * cy;
    const long long Ux = a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by);
    const long long Uy = a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax);
    // each coordinate the binary32 value nearest to the exact ratio
    // (integer steps: ca_fconv.h)
    o.cx = ratio_to_f32(Ux, D);
    o.cy = ratio_to_f32(Uy, D);
    const float dx = __fsub_rn(__int2float_rn(ax), o.cx);
    const float dy = __fsub_rn(__int2float_rn(ay), o.cy);
    o.r = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
    return true;
}

struct Moments {
    int n, Sx, Sy, Sxx, Sxy, Syy;
    long long Sxxx, Sxxy, Sxyy, Syyy;
    uint32_t S;
};

// Lanes of the T-thread group that contains this lane.  Groups of one warp
// take different branches (hypotheses past the end, early exits), so their
// shuffles name only their own lanes.
template <int T>
__device__ __forceinline__ unsigned group_mask() {
    return T >= 32 ? kFull : (((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1)));
}

// Sum of the moments held by the T threads of one hypothesis group.
template <int T>
__device__ __forceinline__ void group_sum(Moments &m, unsigned gm) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        m.n += __shfl_xor_sync(gm, m.n, o);
        m.Sx += __shfl_xor_sync(gm, m.Sx, o);
        m.Sy += __shfl_xor_sync(gm, m.Sy, o);
        m.Sxx += __shfl_xor_sync(gm, m.Sxx, o);
        m.Sxy += __shfl_xor_sync(gm, m.Sxy, o);
        m.Syy += __shfl_xor_sync(gm, m.Syy, o);
        m.Sxxx += __shfl_xor_sync(gm, m.Sxxx, o);
        m.Sxxy += __shfl_xor_sync(gm, m.Sxxy, o);
        m.Sxyy += __shfl_xor_sync(gm, m.Sxyy, o);
        m.Syyy += __shfl_xor_sync(gm, m.Syyy, o);
        m.S += __shfl_xor_sync(gm, m.S, o);
    }
}

// Algebraic least-squares circle (Coope 1993) from exact integer moments.
__device__ __forceinline__ bool ls_fit(const Moments &m, Circle &o) {
    if (m.n < 3) return false;
    const long long n = m.n;
    const long long Sx = m.Sx, Sy = m.Sy;
    const long long A = n * m.Sxx - Sx * Sx;
    const long long B = n * m.Sxy - Sx * Sy;
    const long long C = n * m.Syy - Sy * Sy;
    const long long P = n * n * m.Sxxx - 3 * n * Sx * m.Sxx + 2 * Sx * Sx * Sx + n * n * m.Sxyy -
                        2 * n * Sy * m.Sxy - n * Sx * m.Syy + 2 * Sx * Sy * Sy;
    const long long Q = n * n * m.Syyy - 3 * n * Sy * m.Syy + 2 * Sy * Sy * Sy + n * n * m.Sxxy -
                        2 * n * Sx * m.Sxy - n * Sy * m.Sxx + 2 * Sy * Sx * Sx;
    const __int128 det = (__int128)A * C - (__int128)B * B;
    if (det == 0) return false;
    const __int128 an = (__int128)C * P - (__int128)B * Q;
    const __int128 bn = (__int128)A * Q - (__int128)B * P;
    const __int128 den = 2 * (__int128)n * det;
    const __int128 cxn = 2 * det * (__int128)Sx + an;
    const __int128 cyn = 2 * det * (__int128)Sy + bn;
    const float fden = i128_to_f32(den);
    o.cx = __fdiv_rn(i128_to_f32(cxn), fden);
    o.cy = __fdiv_rn(i128_to_f32(cyn), fden);
    const float af = __fdiv_rn(i128_to_f32(an), fden);
    const float bf = __fdiv_rn(i128_to_f32(bn), fden);
    const float t1 = __fdiv_rn(i64_to_f32(A + C), i64_to_f32(n * n));
    const float r2 = __fadd_rn(__fadd_rn(t1, __fmul_rn(af, af)), __fmul_rn(bf, bf));
    o.r = __fsqrt_rn(r2);
    return true;
}

// One candidate point in shared memory (32 bytes: two 16-byte loads).
struct __align__(16) Pt {
    float fx, fy;
    int32_t X, Y;
    int32_t XX, XY, YY;
    uint32_t S;
};

struct FitSmem {
    Pt pt[kMaxSlots];
    Moments lsq[kHypTile];   // a refinement round's fit queue: moments in,
    Circle lsc[kHypTile];    // circles out (r < 0: no fit)
    int nls[2];              // queue lengths of alternate rounds
    int wcount[kHypTile / 32];
    unsigned long long wbest[kHypTile / 32];
    int last;
};

// Inliers of circle c among this thread's share of the candidates (points
// j = sub, sub + T, ...), as a bit set, with their moments (if `moments`) and
// score sum.  Returns true if this share of the set differs from `bits`.
template <int T>
__device__ __forceinline__ bool inlier_pass(const FitSmem &sm, int M, int sub, const Circle &c,
                                            float t_ri, bool moments, uint32_t (&bits)[8 / T],
                                            Moments &m) {
    float lo = __fsub_rn(c.r, t_ri);
    if (lo < 0.0f) lo = 0.0f;
    const float hi = __fadd_rn(c.r, t_ri);
    const float lo2 = __fmul_rn(lo, lo), hi2 = __fmul_rn(hi, hi);
    m = Moments{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0u};
    bool changed = false;
#pragma unroll
    for (int w = 0; w < 8 / T; ++w) {
        uint32_t word = 0u;
        const int j0 = sub + T * 32 * w;
        if (j0 < M) {
            const int nb = min(32, (M - j0 + T - 1) / T);
            for (int b = 0; b < nb; ++b) {
                const int j = j0 + T * b;
                const uint4 q0 = *reinterpret_cast<const uint4 *>(&sm.pt[j]);
                const float dx = __fsub_rn(__uint_as_float(q0.x), c.cx);
                const float dy = __fsub_rn(__uint_as_float(q0.y), c.cy);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (d2 >= lo2 && d2 <= hi2) {
                    const uint4 q1 = *reinterpret_cast<const uint4 *>(&sm.pt[j].XX);
                    word |= 1u << b;
                    m.n += 1;
                    m.S += q1.w;
                    if (moments) {
                        const int X = (int)q0.z, Y = (int)q0.w;
                        const int XX = (int)q1.x, XY = (int)q1.y, YY = (int)q1.z;
                        m.Sx += X;
                        m.Sy += Y;
                        m.Sxx += XX;
                        m.Sxy += XY;
                        m.Syy += YY;
                        m.Sxxx += (long long)X * XX;
                        m.Sxxy += (long long)XX * Y;
                        m.Sxyy += (long long)X * YY;
                        m.Syyy += (long long)Y * YY;
                    }
                }
            }
        }
        changed |= word != bits[w];
        bits[w] = word;
    }
    return changed;
}

// Lexicographic unranking of the h-th triple i < j < k of 0..M-1.
__device__ __forceinline__ void unrank_triple(long long h, int M, int &i, int &j, int &k) {
    long long rem = h;
    i = 0;
    for (; i < M - 2; ++i) {
        const long long n = M - 1 - i;
        const long long cnt = n * (n - 1) / 2;
        if (rem < cnt) break;
        rem -= cnt;
    }
    j = i + 1;
    for (; j < M - 1; ++j) {
        const long long cnt = M - 1 - j;
        if (rem < cnt) break;
        rem -= cnt;
    }
    k = j + 1 + (int)rem;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t (&o)[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

__device__ __forceinline__ uint64_t clock_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until slot *p carries kSlotFresh and returns it; after limit_ns sets
// kSyncErrTimeout in *err and returns an empty slot.
__device__ __noinline__ unsigned long long wait_slot(const CandSlot *p, uint32_t *err,
                                                     uint64_t limit_ns) {
    const uint64_t t0 = clock_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        const unsigned long long b = load_slot_bits(p);
        if ((b >> 48) & kSlotFresh) return b;
        __nanosleep(128);
        if ((it & 15u) == 15u && clock_ns() - t0 > limit_ns) break;
    }
    atomicOr(err, kSyncErrTimeout);
    return 0ull;
}

}  // namespace

// Tile `tile` of the hypotheses of frame f.  T threads share one hypothesis
// (points split among them, moments combined by shuffles); a CTA holds
// 256 / T hypotheses.  With `sync` (fused kernel) the strips of the frame may
// still be running: each thread waits for its slot to be written (kSlotFresh),
// bounded by limit_ns (error flag set, slot taken as empty).  The last tile of
// the frame to finish clears the slots' kSlotFresh and writes the frame's
// result; with `sync` it also publishes the result to the frame's mask items.
// t_ready (fused kernel traces, thread 0): when every slot had been read.
template <int T>
__device__ __forceinline__ void fit_tile(FitSmem &sm, const DevFrame *__restrict__ frames,
                                         const DevParams &P, CandSlot *slots,
                                         const Workspace &ws, ca_result *out, int f, int tile,
                                         uint32_t *sync, uint64_t limit_ns = 0,
                                         uint64_t *t_ready = nullptr) {
    constexpr int HPT = kHypTile / T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = tid & (T - 1);
    const DevFrame fr = frames[f];
    const int NK = P.N * P.K;
    const int ox = fr.W >> 1, oy = fr.H >> 1;

    // ---- kept candidate slots -> compact, in slot order
    CandSlot c;
    c.x = c.y = 0;
    c.s = c.kept = 0;
    if (tid < NK) {   // L2 load: in the fused kernel other CTAs write the slots
        const CandSlot *sp = slots + (int64_t)f * kMaxSlots + tid;
        unsigned long long b = load_slot_bits(sp);
        if (sync && !((b >> 48) & kSlotFresh)) b = wait_slot(sp, sync + 2, limit_ns);
        c = slot_of(b);
    }
    const bool kept = tid < NK && (c.kept & kSlotKept);
    const unsigned bal = __ballot_sync(kFull, kept);
    if (lane == 0) sm.wcount[warp] = __popc(bal);
    if (tid == 0) sm.nls[0] = 0;
    __syncthreads();
    if (t_ready && tid == 0) *t_ready = clock_ns();
    int off = 0, M = 0;
    for (int w = 0; w < kHypTile / 32; ++w) {
        off += (w < warp) ? sm.wcount[w] : 0;
        M += sm.wcount[w];
    }
    if (kept) {
        const int j = off + __popc(bal & ((1u << lane) - 1u));
        const int X = c.x - ox, Y = c.y - oy;
        Pt p;
        p.fx = __int2float_rn(X); p.fy = __int2float_rn(Y);
        p.X = X; p.Y = Y;
        p.XX = X * X; p.XY = X * Y; p.YY = Y * Y;
        p.S = c.s;
        sm.pt[j] = p;
    }
    __syncthreads();

    long long NH = 0;
    if (M >= 3) NH = P.hyp_mode == CA_HYP_EXHAUSTIVE ? (long long)M * (M - 1) * (M - 2) / 6 : P.NH;
    // tracked call: the previous circle of the frame's track, when it was
    // accepted, is one more hypothesis (index NH), refined and scored like
    // the others
    int trk = -1;
    ca_result prior;
    prior.valid = 0;
    if (P.track) {
        trk = ws.track[f];
        if (trk >= 0) prior = load_result(ws.state + trk);
    }
    const long long NH_all = NH + ((M >= 3 && prior.valid) ? 1 : 0);
    const long long h = (long long)tile * HPT + tid / T;
    if (P.debug >= 1 && tile == 0 && tid == 0) {
        ws.n_cands[f] = M;
        ws.n_hyps[f] = (int)NH_all;
    }

    unsigned long long key = 0ull;
    Circle c0{0.f, 0.f, 0.f};
    int n_fin = 0;
    uint32_t S_fin = 0u;
    int t0 = 0, t1 = 0, t2 = 0, pass = 0;
    bool active = false;   // the group refines a circle
    if (h < NH_all) {   // uniform across the T threads of a group
        bool have_circle;
        if (h == NH) {
            c0 = Circle{__fsub_rn(prior.cx, __int2float_rn(ox)), __fsub_rn(prior.cy, __int2float_rn(oy)),
                        prior.r};
            t0 = t1 = t2 = -1;
            have_circle = true;
        } else {
        if (P.hyp_mode == CA_HYP_EXHAUSTIVE) {
            unrank_triple(h, M, t0, t1, t2);
        } else {
            uint32_t u[4];
            philox4x32_10((uint32_t)h, (uint32_t)fr.key, (uint32_t)(fr.key >> 32), 0u,
                          (uint32_t)P.seed, (uint32_t)(P.seed >> 32), u);
            const uint32_t m = (uint32_t)M;
            uint32_t i0 = __umulhi(u[0], m);
            uint32_t i1 = __umulhi(u[1], m - 1u);
            if (i1 >= i0) ++i1;
            uint32_t i2 = __umulhi(u[2], m - 2u);
            const uint32_t a = min(i0, i1), b = max(i0, i1);
            if (i2 >= a) ++i2;
            if (i2 >= b) ++i2;
            t0 = (int)i0; t1 = (int)i1; t2 = (int)i2;
        }
        int s0 = t0, s1 = t1, s2 = t2, tmp;
        if (s0 > s1) { tmp = s0; s0 = s1; s1 = tmp; }
        if (s1 > s2) { tmp = s1; s1 = s2; s2 = tmp; }
        if (s0 > s1) { tmp = s0; s0 = s1; s1 = tmp; }
        have_circle = circumcircle(sm.pt[s0].X, sm.pt[s0].Y, sm.pt[s1].X, sm.pt[s1].Y,
                                   sm.pt[s2].X, sm.pt[s2].Y, c0);
        }
        active = have_circle;
        if (!have_circle) c0 = Circle{0.f, 0.f, 0.f};
    }

    // ---- refinement, in step across the CTA: each group's inlier pass, then
    // the least-squares fits the groups need, each computed once (by one of
    // the CTA's first threads, from the group's moments in shared memory)
    // rather than by all T threads of its group
    uint32_t bits[8 / T];
#pragma unroll
    for (int w = 0; w < 8 / T; ++w) bits[w] = 0u;
    Moments m = Moments{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0u};
    bool final_known = !active;   // the group's inlier set is final
    const unsigned gm = group_mask<T>();
    for (int it = 0; it < P.refine; ++it) {
        int q = -1;   // the group's entry in this round's fit queue
        if (!final_known) {   // uniform across the T threads of a group
            int changed = inlier_pass<T>(sm, M, sub, c0, P.t_ri, true, bits, m) ? 1 : 0;
            group_sum<T>(m, gm);
#pragma unroll
            for (int o = 1; o < T; o <<= 1) changed |= __shfl_xor_sync(gm, changed, o);
            if (it > 0 && !changed) {
                final_known = true;   // the fit would repeat
            } else {
                if (sub == 0) {
                    q = atomicAdd(&sm.nls[it & 1], 1);
                    sm.lsq[q] = m;
                }
                q = __shfl_sync(gm, q, lane & ~(T - 1));
            }
        }
        if (!__syncthreads_or(q >= 0)) break;   // every set is final
        if (tid == 0) sm.nls[(it + 1) & 1] = 0;   // the next round's queue
        if (tid < sm.nls[it & 1]) {
            Circle nc;
            if (!ls_fit(sm.lsq[tid], nc)) nc.r = -1.0f;   // no fit: circle unchanged
            sm.lsc[tid] = nc;
        }
        __syncthreads();
        if (q >= 0) {
            const Circle nc = sm.lsc[q];
            if (nc.r < 0.0f) final_known = true;
            else c0 = nc;
        }
    }
    if (active) {
        if (!final_known) {
            inlier_pass<T>(sm, M, sub, c0, P.t_ri, false, bits, m);
            group_sum<T>(m, gm);
        }
        n_fin = m.n;
        S_fin = m.S;
        const float Wf = __int2float_rn(fr.W);
        const float rlo = __fmul_rn(P.r_min, Wf), rhi = __fmul_rn(P.r_max, Wf);
        const float dm = __fmul_rn(P.d_max, Wf);
        const float ex = (fr.W & 1) ? 0.0f : -0.5f, ey = (fr.H & 1) ? 0.0f : -0.5f;
        const float dx = __fsub_rn(c0.cx, ex), dy = __fsub_rn(c0.cy, ey);
        pass = c0.r >= rlo && c0.r <= rhi &&
               __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= __fmul_rn(dm, dm);
        if (pass && sub == 0)
            key = ((unsigned long long)(S_fin + 1u) << 32) | (0xFFFFFFFFu - (uint32_t)h);
    }
    if (h < NH_all && P.debug >= 2 && sub == 0) {
        HypRec rec;
        rec.i0 = t0; rec.i1 = t1; rec.i2 = t2;
        rec.n_inl = n_fin; rec.S = S_fin; rec.pass = pass;
        rec.cx = c0.cx; rec.cy = c0.cy; rec.r = c0.r;
        ws.hyps[(int64_t)f * (P.NH + P.track) + h] = rec;
    }

    // ---- best of the CTA: highest score, lowest hypothesis index
    unsigned long long wk = key;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, wk, o);
        wk = t > wk ? t : wk;
    }
    if (lane == 0) sm.wbest[warp] = wk;
    __syncthreads();
    unsigned long long cb = 0ull;
    for (int w = 0; w < kHypTile / 32; ++w) cb = sm.wbest[w] > cb ? sm.wbest[w] : cb;
    if (key != 0ull && key == cb) {
        TileRec tr;
        tr.cx = c0.cx; tr.cy = c0.cy; tr.r = c0.r;
        tr.n_inl = n_fin; tr.S = S_fin;
        tr.pad[0] = tr.pad[1] = tr.pad[2] = 0;
        ws.tiles[(int64_t)f * P.n_tiles + tile] = tr;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        if (cb != 0ull) atomicMax(&ws.best[f], cb);
        __threadfence();
        const unsigned prev = atomicAdd(&ws.done[f], 1u);
        sm.last = prev == (unsigned)(P.n_tiles - 1);
    }
    __syncthreads();
    if (sm.last && tid < NK) {   // every tile of this frame has read the slots
        CandSlot *sp = slots + (int64_t)f * kMaxSlots + tid;
        const unsigned long long b = load_slot_bits(sp);
        *reinterpret_cast<unsigned long long *>(sp) = b & ~((unsigned long long)kSlotFresh << 48);
    }
    if (sm.last && tid == 0) {   // last CTA of this frame writes the result
        __threadfence();
        const unsigned long long k = atomicAdd(&ws.best[f], 0ull);
        ca_result res;
        res.cx = res.cy = res.r = res.score = 0.0f;
        res.valid = 0;
        res.n_inliers = 0;
        if (k != 0ull) {
            const uint32_t hb = 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
            const uint32_t S = (uint32_t)(k >> 32) - 1u;
            const volatile TileRec *tr = ws.tiles + (int64_t)f * P.n_tiles + hb / HPT;
            res.cx = __fadd_rn(__int2float_rn(ox), tr->cx);
            res.cy = __fadd_rn(__int2float_rn(oy), tr->cy);
            res.r = tr->r;
            res.n_inliers = tr->n_inl;
            double den = P.score_den;
            uint32_t Tcs = P.T_cs;
            if (P.norm_circle) {
                // the most inliers this circle can have: K per strip whose
                // row is within r + t_ri of the centre row
                const float reach = __fadd_rn(res.r, P.t_ri);
                int n = 0;
                for (int i = 0; i < P.N; ++i)
                    n += fabsf(__fsub_rn(__int2float_rn(P.rows_tab[fr.rows_off + i]), res.cy)) <= reach;
                const double norm = __dmul_rn((double)P.K, (double)n);
                den = __dmul_rn(32768.0, norm);
                Tcs = n > 0 ? (uint32_t)ceil(__dmul_rn(P.tcs_unit, norm)) : 0xFFFFFFFFu;
            }
            res.score = den > 0.0 ? __double2float_rn(__ddiv_rn((double)S, den)) : 0.0f;
            res.valid = den > 0.0 && S >= Tcs ? 1 : 0;
        }
        out[f] = res;
        if (trk >= 0) ws.state[trk] = res;   // every tile of the frame has read the prior
        ws.best[f] = 0ull;   // ready for the next call
        ws.done[f] = 0u;
        if (sync) {
            // publish the result to the mask items
            if (fr.mask && P.debug < 3) {   // debug level 3 withholds it (tests the bounded waits)
                __threadfence();
                atomicExch(sync_ready(sync, ws.sync_frames) + f, 1u);
            }
        }
    }
}

// T threads share one hypothesis; grid (frames, tiles).
template <int T>
__global__ void __launch_bounds__(kHypTile, 4)
    k_fit(const DevFrame *__restrict__ frames, int B, DevParams P,
          CandSlot *__restrict__ slots, Workspace ws, ca_result *__restrict__ out) {
    __shared__ FitSmem sm;
    fit_tile<T>(sm, frames, P, slots, ws, out, blockIdx.x, blockIdx.y, nullptr);
}

int fit_threads_per_sm(int T) {
    static int cache[9] = {0};
    if (T < 1 || T > 8) return 1024;
    if (cache[T] == 0) {
        int v = 0;
        cudaError_t e = cudaErrorInvalidValue;
        if (T == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_fit<1>, kHypTile, 0);
        if (T == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_fit<2>, kHypTile, 0);
        if (T == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_fit<4>, kHypTile, 0);
        if (T == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_fit<8>, kHypTile, 0);
        cache[T] = (e == cudaSuccess && v > 0 ? v : 2) * kHypTile;
    }
    return cache[T];
}

int choose_hyp_threads(int requested, long long B, long long NH, int sms) {
    if (requested == 1 || requested == 2 || requested == 4 || requested == 8) return requested;
    // the largest split whose threads still fit one wave of resident CTAs
    // (more threads per hypothesis shorten each thread's serial work)
    int T = 1;
    while (T < 8 && B * NH * (2 * T) <= (long long)sms * fit_threads_per_sm(2 * T)) T <<= 1;
    return T;
}

cudaError_t launch_fit(const DevFrame *frames, int B, const DevParams &P, CandSlot *slots,
                       const Workspace &ws, ca_result *out, cudaStream_t s) {
    dim3 grid((unsigned)B, (unsigned)P.n_tiles);
    switch (P.hyp_threads) {
        case 1: k_fit<1><<<grid, kHypTile, 0, s>>>(frames, B, P, slots, ws, out); break;
        case 2: k_fit<2><<<grid, kHypTile, 0, s>>>(frames, B, P, slots, ws, out); break;
        case 4: k_fit<4><<<grid, kHypTile, 0, s>>>(frames, B, P, slots, ws, out); break;
        case 8: k_fit<8><<<grid, kHypTile, 0, s>>>(frames, B, P, slots, ws, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ================================================================ k_mask ==
namespace {

struct RowSpan {
    int a, b, exact;
};

// Columns [a, b] of row y inside the disc, by the binary32 predicate
// ((x - cx)^2 + (y - cy)^2 <= r^2, each operation rounded).  The predicate is
// monotone in |x - cx|, so its solutions form one interval; a float estimate
// of the ends is corrected by a few exact predicate evaluations.
__device__ __forceinline__ bool in_disc(int x, float cx, float dy2, float rr) {
    const float dx = __fsub_rn(__int2float_rn(x), cx);
    return __fadd_rn(__fmul_rn(dx, dx), dy2) <= rr;
}

__device__ __forceinline__ RowSpan row_span(const ca_result &res, int W, int y) {
    RowSpan s{0, W - 1, 1};
    if (!res.valid) return s;
    const float cx = res.cx, rr = __fmul_rn(res.r, res.r);
    const float dy = __fsub_rn(__int2float_rn(y), res.cy);
    const float dy2 = __fmul_rn(dy, dy);
    s.a = W;
    s.b = -1;
    if (dy2 > rr) return s;                  // whole row outside (exact)
    const float half = sqrtf(fmaxf(__fsub_rn(rr, dy2), 0.0f));
    if (!(fabsf(cx) < 1.0e6f) || !(half < 1.0e7f)) { s.exact = 0; return s; }
    // the solutions contain floor(cx) or floor(cx) + 1 when there are any
    const int m0 = (int)floorf(cx), m1 = m0 + 1;
    const bool in0 = in_disc(m0, cx, dy2, rr), in1 = in_disc(m1, cx, dy2, rr);
    if (!in0 && !in1) return s;              // empty row
    const int pl = in0 ? m0 : m1, pr = in1 ? m1 : m0;
    int L = min((int)ceilf(cx - half), pl), R = max((int)floorf(cx + half), pr);
    int steps = 0;
    if (in_disc(L, cx, dy2, rr)) {
        while (steps < 64 && in_disc(L - 1, cx, dy2, rr)) { --L; ++steps; }
    } else {
        while (steps < 64 && !in_disc(L, cx, dy2, rr)) { ++L; ++steps; }   // stops at pl
    }
    if (in_disc(R, cx, dy2, rr)) {
        while (steps < 128 && in_disc(R + 1, cx, dy2, rr)) { ++R; ++steps; }
    } else {
        while (steps < 128 && !in_disc(R, cx, dy2, rr)) { --R; ++steps; }  // stops at pr
    }
    if (steps >= 64) { s.exact = 0; return s; }  // estimate far off: evaluate per pixel
    s.a = max(L, 0);
    s.b = min(R, W - 1);
    return s;
}

__device__ __forceinline__ uint32_t span_word(int x0, int a, int b) {
    uint32_t w = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) w |= (uint32_t)(x0 + j >= a && x0 + j <= b) << (8 * j);
    return w;
}

__device__ __forceinline__ uint32_t exact_word(int x0, float cx, float dy2, float rr) {
    uint32_t w = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) w |= (uint32_t)in_disc(x0 + j, cx, dy2, rr) << (8 * j);
    return w;
}

// Unit u (rows 8u .. 8u+7) of the mask of one frame, by one warp: lanes r
// and 8 + r compute the span of row r and the 16-byte vectors holding its
// left and right ends; then the warp stores each row with consecutive 16-byte
// vectors per lane, whole vectors from two comparisons, end vectors from the
// lanes that built them.
__device__ __forceinline__ void mask_unit(const DevFrame &fr, const ca_result &res, int u) {
    const int lane = threadIdx.x & 31;
    const int W = fr.W, H = fr.H;
    const int y0 = u * kMaskRowsPerUnit;
    const int nrows = min(kMaskRowsPerUnit, H - y0);
    const RowSpan sp = row_span(res, W, y0 + min(lane & 7, nrows - 1));
    const float rr = __fmul_rn(res.r, res.r);
    uint4 ev = make_uint4(0u, 0u, 0u, 0u);   // end vector: left (lanes 0-7) or right (8-15)
    if (fr.mask_vec_ok && sp.exact && sp.a <= sp.b) {
        const int x0 = ((lane & 8) ? sp.b : sp.a) & ~15;
        ev = make_uint4(span_word(x0, sp.a, sp.b), span_word(x0 + 4, sp.a, sp.b),
                        span_word(x0 + 8, sp.a, sp.b), span_word(x0 + 12, sp.a, sp.b));
    }
    for (int r = 0; r < nrows; ++r) {
        const int a = __shfl_sync(kFull, sp.a, r);
        const int b = __shfl_sync(kFull, sp.b, r);
        const int ex = __shfl_sync(kFull, sp.exact, r);
        const int y = y0 + r;
        uint8_t *row = fr.mask + (int64_t)y * W;
        if (fr.mask_vec_ok && ex) {
            uint4 la, ra;   // the row's end vectors
            la.x = __shfl_sync(kFull, ev.x, r);
            la.y = __shfl_sync(kFull, ev.y, r);
            la.z = __shfl_sync(kFull, ev.z, r);
            la.w = __shfl_sync(kFull, ev.w, r);
            ra.x = __shfl_sync(kFull, ev.x, r + 8);
            ra.y = __shfl_sync(kFull, ev.y, r + 8);
            ra.z = __shfl_sync(kFull, ev.z, r + 8);
            ra.w = __shfl_sync(kFull, ev.w, r + 8);
            // vectors wholly inside [a, b] are ones, wholly outside zeros; the
            // (at most two) that hold an end come from the end vectors (both
            // built from the whole span, so equal when the ends share one)
            const int VW = W >> 4;
            const int fa = (a + 15) >> 4, fb = ((b + 1) >> 4) - 1;   // whole vectors inside
            const int ea = a >> 4, eb = b >> 4;                      // vectors holding an end
            for (int v = lane; v < VW; v += 32) {
                const bool whole = v >= fa && v <= fb;
                const uint32_t w = whole ? 0x01010101u : 0u;
                uint4 val = make_uint4(w, w, w, w);
                if (!whole && a <= b) {
                    if (v == ea) val = la;
                    else if (v == eb) val = ra;
                }
                st_cs_v4(row + (v << 4), val);
            }
        } else if (fr.mask_vec_ok) {
            const float dy = __fsub_rn(__int2float_rn(y), res.cy);
            const float dy2 = __fmul_rn(dy, dy);
            const int VW = W >> 4;
            for (int v = lane; v < VW; v += 32) {
                const int x0 = v << 4;
                st_cs_v4(row + x0, make_uint4(exact_word(x0, res.cx, dy2, rr),
                                              exact_word(x0 + 4, res.cx, dy2, rr),
                                              exact_word(x0 + 8, res.cx, dy2, rr),
                                              exact_word(x0 + 12, res.cx, dy2, rr)));
            }
        } else {
            const float dy = __fsub_rn(__int2float_rn(y), res.cy);
            const float dy2 = __fmul_rn(dy, dy);
            for (int x = lane; x < W; x += 32) {
                uint8_t v;
                if (!res.valid) v = 1;
                else if (ex) v = (uint8_t)(x >= a && x <= b);
                else v = (uint8_t)in_disc(x, res.cx, dy2, rr);
                row[x] = v;
            }
        }
    }
}

}  // namespace

// One warp per unit of 8 rows; units of all frames are numbered consecutively
// (DevFrame::unit_off).
__global__ void __launch_bounds__(256)
    k_mask(const DevFrame *__restrict__ frames, int B, const ca_result *__restrict__ results,
           int total_units) {
    const int wpb = blockDim.x >> 5;
    const int nw = gridDim.x * wpb;
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < total_units; u += nw) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (frames[mid].unit_off <= u) lo = mid;
            else hi = mid - 1;
        }
        const DevFrame fr = frames[lo];
        if (fr.mask == nullptr) continue;
        mask_unit(fr, load_result(results + lo), u - fr.unit_off);
    }
}

int mask_blocks_per_sm() {
    static int nb = [] {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_mask, 256, 0) != cudaSuccess) v = 4;
        return v < 1 ? 1 : v;
    }();
    return nb;
}

cudaError_t launch_mask(const DevFrame *frames, int B, const ca_result *res, int total_units,
                        int grid, cudaStream_t s) {
    if (total_units <= 0) return cudaSuccess;
    k_mask<<<grid, 256, 0, s>>>(frames, B, res, total_units);
    return cudaGetLastError();
}

// ================================================================ k_batch ==
// The whole path of a batch in one persistent launch.  CTAs take work items
// from one atomic counter, in an order in which every item comes after the
// items it depends on (the strips of a frame before its fit tiles, its fit
// tiles before its mask items).  A CTA that takes an item whose inputs are not
// ready waits for them; those inputs belong to items that running CTAs have
// already taken and that wait only on earlier items, so every wait ends
// whatever the number of resident CTAs.  Each wait is still bounded in time:
// on expiry the CTA sets an error flag (read back by ca_sync) and goes on.
namespace {

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread-level wait until *p >= target; false after `limit_ns` (error flag set).
__device__ __noinline__ bool wait_at_least(const uint32_t *p, uint32_t target, uint32_t *err,
                                           uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (ld_acquire(p) >= target) return true;
        __nanosleep(128);
        if ((it & 15u) == 15u && globaltimer_ns() - t0 > limit_ns) break;
    }
    atomicOr(err, kSyncErrTimeout);
    return false;
}

}  // namespace

size_t batch_smem_bytes(const DevParams &P) {
    const size_t strip_part = strips_smem_bytes(P) - strip_tables_bytes(P);
    return strip_tables_bytes(P) + (strip_part > sizeof(FitSmem) ? strip_part : sizeof(FitSmem));
}

template <int T>
__global__ void __launch_bounds__(kStripThreads, 4)
    k_batch(const DevFrame *__restrict__ frames, const int32_t *__restrict__ rows, DevParams P,
            const uint16_t *__restrict__ luts, Workspace ws, ca_result *out,
            const BatchSeg *__restrict__ segs, int n_segs, int total_items, uint64_t wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    strip_tables_load(P, luts, tab);   // once per CTA; visible after the first barrier
    unsigned char *un = smem_raw + strip_tables_bytes(P);   // strip buffers or FitSmem
    const StripShared ss{tab, tab + (kDevOffB - kDevOffI), tab + (kDevOffG - kDevOffI), un};
    FitSmem &fs = *reinterpret_cast<FitSmem *>(un);
    const uint16_t *lt = luts + kDevOffT;
    uint32_t *sync = ws.sync;
    const int nf = ws.sync_frames;
    const int warp = threadIdx.x >> 5;
    const int spf = strip_items_of(P.N, P.K);
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (threadIdx.x == 0) s_item = (int)atomicAdd(sync + 0, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        uint64_t t_grab = 0, t_ready = 0;
        if (ws.trace && threadIdx.x == 0) t_grab = t_ready = globaltimer_ns();
        int lo = 0, hi = n_segs - 1;   // last segment starting at or before item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].start <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchSeg sg = segs[lo];
        const int local = item - sg.start;
        if (sg.phase == kPhaseStrips) {
            const int f = sg.f0 + local / spf, si = local % spf;
            if (P.K == 2) {
                strip_pair(frames, rows, P, lt, ss, ws.slots, f, si);
            } else {
                const int i = 4 * si + (warp >> 1);
                if (i < P.N) strip_half(frames, rows, P, lt, ss, ws.slots, f, i, warp & 1);
            }
            // the slots it wrote tell the fit items of f that it is done
        } else if (sg.phase == kPhaseFit) {
            const int f = sg.f0 + local / P.n_tiles, tile = local % P.n_tiles;
            fit_tile<T>(fs, frames, P, ws.slots, ws, out, f, tile, sync, wait_ns,
                        ws.trace ? &t_ready : nullptr);
        } else {
            const int g = frames[sg.f0].mitem_off + local;
            int a = sg.f0, b = sg.f1 - 1;   // frame of mask item g
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (frames[mid].mitem_off <= g) a = mid;
                else b = mid - 1;
            }
            const int f = a;
            const DevFrame fr = frames[f];
            if (threadIdx.x == 0) {
                wait_at_least(sync_ready(sync, nf) + f, 1u, sync + 2, wait_ns);
                __threadfence();
                if (ws.trace) t_ready = globaltimer_ns();
            }
            __syncthreads();
            const int u = (g - fr.mitem_off) * kMaskUnitsPerItem + warp;
            if (u * kMaskRowsPerUnit < fr.H) mask_unit(fr, load_result(out + f), u);
            __syncthreads();
            if (threadIdx.x == 0) {
                const uint32_t c = atomicAdd(sync_maskdone(sync, nf) + f, 1u);
                if (c + 1u == (uint32_t)mask_items_of(fr.H)) {   // every mask item of f has passed its wait
                    sync_maskdone(sync, nf)[f] = 0u;
                    sync_ready(sync, nf)[f] = 0u;
                }
            }
        }
        if (ws.trace && threadIdx.x == 0 && item < ws.trace_cap) {   // the item's timeline
            unsigned long long *tr = ws.trace + 4 * (size_t)item;
            uint32_t smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            tr[0] = t_grab;
            tr[1] = t_ready;
            tr[2] = globaltimer_ns();
            tr[3] = ((unsigned long long)sg.phase << 48) | ((unsigned long long)smid << 32) |
                    blockIdx.x;
        }
    }
    if (threadIdx.x == 0 && atomicAdd(sync + 1, 1u) + 1u == gridDim.x) {
        sync[0] = 0u;   // every CTA has taken its last item: re-arm the counter
        sync[1] = 0u;
    }
}

int batch_blocks_per_sm(int T, size_t smem) {
    int v = 0;
    cudaError_t e = cudaErrorInvalidValue;
    auto occ = [&](auto kern) {
        cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (a != cudaSuccess) return a;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kStripThreads, smem);
    };
    if (T == 1) e = occ(k_batch<1>);
    if (T == 2) e = occ(k_batch<2>);
    if (T == 4) e = occ(k_batch<4>);
    if (T == 8) e = occ(k_batch<8>);
    return e == cudaSuccess && v > 0 ? v : 1;
}

cudaError_t launch_batch(const DevFrame *frames, int B, const int32_t *rows, const DevParams &P,
                         const uint16_t *luts, const Workspace &ws, ca_result *out,
                         const BatchSeg *segs, int n_segs, int total_items, int grid,
                         uint64_t wait_ns, cudaStream_t s) {
    (void)B;
    if (total_items <= 0) return cudaSuccess;
    const size_t smem = batch_smem_bytes(P);
    auto go = [&](auto kern) {
        cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (a != cudaSuccess) return a;
        kern<<<grid, kStripThreads, smem, s>>>(frames, rows, P, luts, ws, out, segs, n_segs,
                                               total_items, wait_ns);
        return cudaGetLastError();
    };
    switch (P.hyp_threads) {
        case 1: return go(k_batch<1>);
        case 2: return go(k_batch<2>);
        case 4: return go(k_batch<4>);
        case 8: return go(k_batch<8>);
        default: return cudaErrorInvalidValue;
    }
}

// ============================================================= k_smooth ==
// Temporal smoothing of tracked results, one thread per frame (the tracks of
// a call are distinct, so no two threads share a state).  The order of the
// binary32 operations is the one ca.h states.
__global__ void k_smooth(const ca_result *res, int B, const int32_t *__restrict__ w_trk,
                         float gamma, float jump, float t_hold, float *__restrict__ state,
                         ca_result *out) {   // out may be res: thread i reads and writes row i
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const ca_result cur = res[i];
    const int W = w_trk[2 * i], t = w_trk[2 * i + 1];
    if (t < 0) {
        out[i] = cur;
        return;
    }
    float *st = state + 4 * (size_t)t;
    const float s0 = st[0], s1 = st[1], s2 = st[2];
    const float d = __fmul_rn(st[3], gamma);
    ca_result o = cur;
    if (cur.valid) {
        const float J = __fmul_rn(jump, __int2float_rn(W));
        const bool near = d > 0.0f && fabsf(__fsub_rn(cur.cx, s0)) <= J &&
                          fabsf(__fsub_rn(cur.cy, s1)) <= J && fabsf(__fsub_rn(cur.r, s2)) <= J;
        if (near) {
            const float w = __fadd_rn(d, cur.score);
            o.cx = __fdiv_rn(__fadd_rn(__fmul_rn(d, s0), __fmul_rn(cur.score, cur.cx)), w);
            o.cy = __fdiv_rn(__fadd_rn(__fmul_rn(d, s1), __fmul_rn(cur.score, cur.cy)), w);
            o.r = __fdiv_rn(__fadd_rn(__fmul_rn(d, s2), __fmul_rn(cur.score, cur.r)), w);
            st[3] = w;
        } else {
            st[3] = cur.score;
        }
        st[0] = o.cx;
        st[1] = o.cy;
        st[2] = o.r;
    } else if (d > 0.0f && d >= t_hold) {
        o.cx = s0;
        o.cy = s1;
        o.r = s2;
        o.score = 0.0f;
        o.valid = 1;
        o.n_inliers = 0;
        st[3] = d;
    } else {
        st[0] = st[1] = st[2] = st[3] = 0.0f;
    }
    out[i] = o;
}

cudaError_t launch_smooth(const ca_result *res, int B, const int32_t *w_trk, float gamma,
                          float jump, float t_hold, float *state, ca_result *out, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    k_smooth<<<(B + 127) / 128, 128, 0, s>>>(res, B, w_trk, gamma, jump, t_hold, state, out);
    return cudaGetLastError();
}

}  // namespace ca
