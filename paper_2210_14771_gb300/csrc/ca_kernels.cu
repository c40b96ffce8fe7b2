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
// fused multiply-adds), so the results are fully determined by the inputs.
#include <cstdint>

#include "ca_internal.h"

namespace ca {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_cs_v4(void *p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Integer BT.601 luma on the 0-255 scale.
__device__ __forceinline__ uint32_t luma(uint32_t r, uint32_t g, uint32_t b) {
    return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// 16 pixels (48 bytes of packed RGB) -> 16 luma bytes.
__device__ __forceinline__ uint4 luma16(uint4 a, uint4 b, uint4 c) {
    const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    uint32_t o[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int i0 = 3 * j, i1 = 3 * j + 1, i2 = 3 * j + 2;
        const uint32_t r = (w[i0 >> 2] >> ((i0 & 3) * 8)) & 0xffu;
        const uint32_t g = (w[i1 >> 2] >> ((i1 & 3) * 8)) & 0xffu;
        const uint32_t bl = (w[i2 >> 2] >> ((i2 & 3) * 8)) & 0xffu;
        o[j >> 2] |= luma(r, g, bl) << ((j & 3) * 8);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
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

}  // namespace

// ============================================================== k_strips ==
// One CTA per strip (grid-stride), 256 threads: threads 0-127 take the left
// half-strip, 128-255 the right one; each thread owns a contiguous chunk of
// its half in scan order (outer edge inwards).
struct StripSmem {
    uint16_t *lt, *lg, *li;
    uint8_t *Y;   // 3 rows of luma, row stride Wp
    uint32_t *keys;
    int Wp;
};

__device__ __forceinline__ StripSmem strip_smem(unsigned char *base, const DevParams &P) {
    StripSmem s;
    s.lt = reinterpret_cast<uint16_t *>(base);
    s.lg = s.lt + ((kLutT + 7) & ~7);
    s.li = s.lg + ((kLutG + 7) & ~7);
    s.Y = reinterpret_cast<uint8_t *>(s.li + kLutI);
    s.Wp = (P.max_w + 15) & ~15;
    s.keys = reinterpret_cast<uint32_t *>(s.Y + 3 * s.Wp);
    return s;
}

size_t strips_smem_bytes(const DevParams &P) {
    const size_t Wp = (size_t)((P.max_w + 15) & ~15);
    size_t b = 2 * (size_t)(((kLutT + 7) & ~7) + ((kLutG + 7) & ~7) + kLutI) + 3 * Wp;
    if (P.K > 2) b += 4 * Wp;
    return b;
}

// Q15 edge score of pixel x of the strip (Eq. 2-3 through the tables).  Scores
// that cannot reach T_ps (bounded by the s_g s_iota product) are returned as 0:
// such pixels are never kept, so the kept candidates are unchanged.
__device__ __forceinline__ uint32_t pixel_score(const StripSmem &sm, int x, int W, int cy2,
                                                int iota, const DevParams &P) {
    if (x <= 0 || x >= W - 1) return 0u;
    const uint8_t *Yu = sm.Y, *Ym = sm.Y + sm.Wp, *Yd = sm.Y + 2 * sm.Wp;
    const int gx = ((int)Yu[x + 1] + 2 * (int)Ym[x + 1] + (int)Yd[x + 1]) -
                   ((int)Yu[x - 1] + 2 * (int)Ym[x - 1] + (int)Yd[x - 1]);
    const int gy = ((int)Yd[x - 1] + 2 * (int)Yd[x] + (int)Yd[x + 1]) -
                   ((int)Yu[x - 1] + 2 * (int)Yu[x] + (int)Yu[x + 1]);
    const int ng = gx * gx + gy * gy;
    const int cx2 = W - 1 - 2 * x;
    const int nc = cx2 * cx2 + cy2 * cy2;
    if (ng == 0 || nc == 0) return 0u;
    const uint32_t g = sm.lg[qmag(ng, P.qg_sat)];
    const uint32_t ii = sm.li[iota];
    if (((g * ii + 16384u) >> 15) < P.T_ps) return 0u;
    const int dot = gx * cx2 + gy * cy2;
    const float den = __fsqrt_rn(__fmul_rn(__int2float_rn(ng), __int2float_rn(nc)));
    const float cs = __fdiv_rn(__int2float_rn(dot), den);
    int qt = __float2int_rz(__fmul_rn(__fadd_rn(cs, 1.0f), 4096.0f));
    qt = min(max(qt, 0), kLutT - 1);
    const uint32_t gt = (g * (uint32_t)sm.lt[qt] + 16384u) >> 15;
    return (gt * ii + 16384u) >> 15;
}

__global__ void __launch_bounds__(kStripThreads)
    k_strips(const DevFrame *__restrict__ frames, int B, const int32_t *__restrict__ rows,
             DevParams P, const uint16_t *__restrict__ luts, CandSlot *__restrict__ slots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const StripSmem sm = strip_smem(smem_raw, P);
    __shared__ uint32_t s_red[8];
    __shared__ int s_wmax[8];
    __shared__ int s_pick[2][kMaxSlots / 2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // tables: luts = [s_g (kLutG)][s_theta (kLutT)][s_iota (kLutI)]
    for (int i = tid; i <= P.qg_sat; i += blockDim.x) sm.lg[i] = luts[i];
    for (int i = tid; i < kLutT; i += blockDim.x) sm.lt[i] = luts[kLutG + i];
    for (int i = tid; i < kLutI; i += blockDim.x) sm.li[i] = luts[kLutG + kLutT + i];

    const int half = tid >> 7;          // 0 left, 1 right
    const int ht = tid & 127;           // thread index within the half
    const int kk = P.K >> 1;            // picks per half-strip
    const int total = B * P.N;

    for (int s = blockIdx.x; s < total; s += gridDim.x) {
        const int f = s / P.N, i = s - f * P.N;
        const DevFrame fr = frames[f];
        const int W = fr.W, H = fr.H;
        const int y = rows[fr.rows_off + i];
        __syncthreads();   // previous strip finished with Y / keys / picks; tables loaded

        // ---- rows y-1, y, y+1 -> luma (16-byte loads when aligned)
        if (fr.vec_ok) {
            const int G = W >> 4;
            for (int g = tid; g < 3 * G; g += blockDim.x) {
                const int k = g / G, grp = g - k * G;
                const uint8_t *src = fr.rgb + (int64_t)(y - 1 + k) * fr.pitch + grp * 48;
                const uint4 a = ld_nc_v4(src), b = ld_nc_v4(src + 16), c = ld_nc_v4(src + 32);
                *reinterpret_cast<uint4 *>(sm.Y + k * sm.Wp + grp * 16) = luma16(a, b, c);
            }
        } else {
            for (int idx = tid; idx < 3 * W; idx += blockDim.x) {
                const int k = idx / W, x = idx - k * W;
                const uint8_t *src = fr.rgb + (int64_t)(y - 1 + k) * fr.pitch + 3 * x;
                sm.Y[k * sm.Wp + x] = (uint8_t)luma(src[0], src[1], src[2]);
            }
        }
        __syncthreads();

        // ---- preceding maximum of the middle row, scanned from the outer edge
        const uint8_t *Ym = sm.Y + sm.Wp;
        const int hw = W >> 1;
        const int len = half ? (W - hw) : hw;
        const int c = (len + 127) >> 7;
        const int p0 = min(ht * c, len), p1 = min(p0 + c, len);
        int lm = 0;
        for (int p = p0; p < p1; ++p) lm = max(lm, (int)Ym[half ? (W - 1 - p) : p]);
        int inc = lm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc = max(inc, t);
        }
        int excl = __shfl_up_sync(kFull, inc, 1);
        if (lane == 0) excl = 0;
        if (lane == 31) s_wmax[warp] = inc;
        __syncthreads();
        for (int w = half * 4; w < warp; ++w) excl = max(excl, s_wmax[w]);

        // ---- scores and keys: (s << 16) | outwardness
        const int cy2 = H - 1 - 2 * y;
        uint32_t best = 0u;
        int run = excl;
        for (int p = p0; p < p1; ++p) {
            const int x = half ? (W - 1 - p) : p;
            const uint32_t sc = pixel_score(sm, x, W, cy2, run, P);
            const uint32_t key = (sc << 16) | (uint32_t)(half ? x : (0xFFFF - x));
            if (kk == 1) best = max(best, key);
            else sm.keys[x] = key;
            run = max(run, (int)Ym[x]);
        }

        // ---- K/2 picks per half, each excluding +-sup_px around earlier picks
        for (int r = 0; r < kk; ++r) {
            if (kk > 1) {
                if (r > 0) __syncthreads();   // s_pick of round r-1 visible
                best = 0u;
                for (int p = p0; p < p1; ++p) {
                    const int x = half ? (W - 1 - p) : p;
                    bool sup = false;
                    for (int j = 0; j < r; ++j) sup |= abs(x - s_pick[half][j]) <= P.sup_px;
                    if (!sup) best = max(best, sm.keys[x]);
                }
            }
            const uint32_t wbest = __reduce_max_sync(kFull, best);
            if (lane == 0) s_red[warp] = wbest;
            __syncthreads();
            if (ht == 0) {
                uint32_t hb = 0u;
                for (int w = half * 4; w < half * 4 + 4; ++w) hb = max(hb, s_red[w]);
                CandSlot out;
                out.kept = 0;
                out.x = -1;
                out.y = (int16_t)y;
                out.s = 0;
                int px = -1000000;
                if (hb != 0u) {
                    const int rank = (int)(hb & 0xFFFFu);
                    px = half ? rank : (0xFFFF - rank);
                    const uint32_t sc = hb >> 16;
                    out.x = (int16_t)px;
                    out.s = (uint16_t)sc;
                    out.kept = (uint16_t)(sc >= P.T_ps && px >= P.T_px && px <= W - 1 - P.T_px &&
                                          y >= P.T_px && y <= H - 1 - P.T_px);
                }
                s_pick[half][r] = px;
                slots[(int64_t)f * kMaxSlots + i * P.K + half * kk + r] = out;
            }
        }
    }
}

namespace {
// Largest dynamic shared memory k_strips can ask for (W = 4096, K > 2).
cudaError_t strips_allow_max_smem() {
    static cudaError_t once = [] {
        DevParams P{};
        P.max_w = kMaxDim;
        P.K = 4;
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

// Correctly rounded binary32 value of a 128-bit integer.
__device__ __forceinline__ float i128_to_f32(__int128 v) {
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    float f;
    if (hi == 0) {
        f = __ull2float_rn(lo);
    } else {
        const int lz = __clzll((long long)hi);
        const int sh = 64 - lz;   // bits dropped to fit 64
        uint64_t top, rest;
        if (lz == 0) { top = hi; rest = lo; }
        else { top = (hi << lz) | (lo >> sh); rest = lo << lz; }
        top |= (rest != 0) ? 1ull : 0ull;   // sticky bit, far below the rounding point
        f = __fmul_rn(__ull2float_rn(top), __int_as_float((127 + sh) << 23));
    }
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
    const long long aD = D < 0 ? -D : D;
    if (aD < 65536) {   // nearly collinear: binary64 quotient
        o.cx = __double2float_rn(__ddiv_rn(__ll2double_rn(Ux), __ll2double_rn(D)));
        o.cy = __double2float_rn(__ddiv_rn(__ll2double_rn(Uy), __ll2double_rn(D)));
    } else {
        const float fD = __ll2float_rn(D);
        o.cx = __fdiv_rn(__ll2float_rn(Ux), fD);
        o.cy = __fdiv_rn(__ll2float_rn(Uy), fD);
    }
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
    const float t1 = __fdiv_rn(__ll2float_rn(A + C), __ll2float_rn(n * n));
    const float r2 = __fadd_rn(__fadd_rn(t1, __fmul_rn(af, af)), __fmul_rn(bf, bf));
    o.r = __fsqrt_rn(r2);
    return true;
}

struct FitSmem {
    int32_t X[kMaxSlots], Y[kMaxSlots], XX[kMaxSlots], XY[kMaxSlots], YY[kMaxSlots];
    float fX[kMaxSlots], fY[kMaxSlots];
    uint32_t S[kMaxSlots];
    int wcount[kHypTile / 32];
    unsigned long long wbest[kHypTile / 32];
    int last;
};

// Inliers of circle c among the M candidates, as a bit set (8 words for up to
// 256 points), with their moments (if `moments`) and score sum.  Returns true
// if the set differs from `bits` on entry; `bits` receives the new set.
__device__ __forceinline__ bool inlier_pass(const FitSmem &sm, int M, const Circle &c, float t_ri,
                                            bool moments, uint32_t (&bits)[8], Moments &m) {
    float lo = __fsub_rn(c.r, t_ri);
    if (lo < 0.0f) lo = 0.0f;
    const float hi = __fadd_rn(c.r, t_ri);
    const float lo2 = __fmul_rn(lo, lo), hi2 = __fmul_rn(hi, hi);
    m = Moments{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0u};
    bool changed = false;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t word = 0u;
        if (w * 32 < M) {
            const int jend = min(32, M - w * 32);
            for (int b = 0; b < jend; ++b) {
                const int j = w * 32 + b;
                const float dx = __fsub_rn(sm.fX[j], c.cx);
                const float dy = __fsub_rn(sm.fY[j], c.cy);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (d2 >= lo2 && d2 <= hi2) {
                    word |= 1u << b;
                    m.n += 1;
                    m.S += sm.S[j];
                    if (moments) {
                        const int X = sm.X[j], Y = sm.Y[j];
                        const int XX = sm.XX[j], XY = sm.XY[j], YY = sm.YY[j];
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

}  // namespace

__global__ void __launch_bounds__(kHypTile)
    k_fit(const DevFrame *__restrict__ frames, int B, DevParams P,
          const CandSlot *__restrict__ slots, Workspace ws, ca_result *__restrict__ out) {
    __shared__ FitSmem sm;
    const int f = blockIdx.x, tile = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevFrame fr = frames[f];
    const int NK = P.N * P.K;
    const int ox = fr.W >> 1, oy = fr.H >> 1;

    // ---- kept candidate slots -> compact, in slot order
    CandSlot c;
    c.x = c.y = 0;
    c.s = c.kept = 0;
    if (tid < NK) c = slots[(int64_t)f * kMaxSlots + tid];
    const bool kept = tid < NK && c.kept;
    const unsigned bal = __ballot_sync(kFull, kept);
    if (lane == 0) sm.wcount[warp] = __popc(bal);
    __syncthreads();
    int off = 0, M = 0;
    for (int w = 0; w < kHypTile / 32; ++w) {
        off += (w < warp) ? sm.wcount[w] : 0;
        M += sm.wcount[w];
    }
    if (kept) {
        const int j = off + __popc(bal & ((1u << lane) - 1u));
        const int X = c.x - ox, Y = c.y - oy;
        sm.X[j] = X; sm.Y[j] = Y;
        sm.XX[j] = X * X; sm.XY[j] = X * Y; sm.YY[j] = Y * Y;
        sm.fX[j] = __int2float_rn(X); sm.fY[j] = __int2float_rn(Y);
        sm.S[j] = c.s;
    }
    __syncthreads();

    long long NH = 0;
    if (M >= 3) NH = P.hyp_mode == CA_HYP_EXHAUSTIVE ? (long long)M * (M - 1) * (M - 2) / 6 : P.NH;
    const long long h = (long long)tile * kHypTile + tid;
    if (P.debug >= 1 && tile == 0 && tid == 0) {
        ws.n_cands[f] = M;
        ws.n_hyps[f] = (int)NH;
    }

    unsigned long long key = 0ull;
    Circle c0{0.f, 0.f, 0.f};
    int n_fin = 0;
    uint32_t S_fin = 0u;
    int t0 = 0, t1 = 0, t2 = 0, pass = 0;
    if (h < NH) {
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
        if (circumcircle(sm.X[s0], sm.Y[s0], sm.X[s1], sm.Y[s1], sm.X[s2], sm.Y[s2], c0)) {
            uint32_t bits[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            Moments m;
            bool final_known = false;
            for (int it = 0; it < P.refine; ++it) {
                const bool changed = inlier_pass(sm, M, c0, P.t_ri, true, bits, m);
                if (it > 0 && !changed) { final_known = true; break; }   // fit would repeat
                Circle nc;
                if (!ls_fit(m, nc)) { final_known = true; break; }       // circle unchanged
                c0 = nc;
            }
            if (!final_known) inlier_pass(sm, M, c0, P.t_ri, false, bits, m);
            n_fin = m.n;
            S_fin = m.S;
            const float Wf = __int2float_rn(fr.W);
            const float rlo = __fmul_rn(P.r_min, Wf), rhi = __fmul_rn(P.r_max, Wf);
            const float dm = __fmul_rn(P.d_max, Wf);
            const float ex = (fr.W & 1) ? 0.0f : -0.5f, ey = (fr.H & 1) ? 0.0f : -0.5f;
            const float dx = __fsub_rn(c0.cx, ex), dy = __fsub_rn(c0.cy, ey);
            pass = c0.r >= rlo && c0.r <= rhi &&
                   __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= __fmul_rn(dm, dm);
            if (pass)
                key = ((unsigned long long)(S_fin + 1u) << 32) | (0xFFFFFFFFu - (uint32_t)h);
        } else {
            c0 = Circle{0.f, 0.f, 0.f};
        }
        if (P.debug >= 2) {
            HypRec rec;
            rec.i0 = t0; rec.i1 = t1; rec.i2 = t2;
            rec.n_inl = n_fin; rec.S = S_fin; rec.pass = pass;
            rec.cx = c0.cx; rec.cy = c0.cy; rec.r = c0.r;
            ws.hyps[(int64_t)f * P.NH + h] = rec;
        }
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
            const volatile TileRec *tr = ws.tiles + (int64_t)f * P.n_tiles + hb / kHypTile;
            res.cx = __fadd_rn(__int2float_rn(ox), tr->cx);
            res.cy = __fadd_rn(__int2float_rn(oy), tr->cy);
            res.r = tr->r;
            res.n_inliers = tr->n_inl;
            res.score = __double2float_rn(__ddiv_rn((double)S, P.score_den));
            res.valid = S >= P.T_cs ? 1 : 0;
        }
        out[f] = res;
        ws.best[f] = 0ull;   // ready for the next call
        ws.done[f] = 0u;
    }
}

cudaError_t launch_fit(const DevFrame *frames, int B, const DevParams &P, const CandSlot *slots,
                       const Workspace &ws, ca_result *out, cudaStream_t s) {
    dim3 grid((unsigned)B, (unsigned)P.n_tiles);
    k_fit<<<grid, kHypTile, 0, s>>>(frames, B, P, slots, ws, out);
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

__device__ __forceinline__ uint32_t exact_word(int x0, const ca_result &res, float dy2) {
    uint32_t w = 0u;
    const float rr = __fmul_rn(res.r, res.r);
#pragma unroll
    for (int j = 0; j < 4; ++j) w |= (uint32_t)in_disc(x0 + j, res.cx, dy2, rr) << (8 * j);
    return w;
}

}  // namespace

// One warp per 32-row unit of one frame; lanes stride over the unit's 16-byte
// vectors (row-major), so every lane stores on every iteration.
__global__ void __launch_bounds__(256)
    k_mask(const DevFrame *__restrict__ frames, int B, const ca_result *__restrict__ results,
           int total_units) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total_units; u += nw) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (frames[mid].unit_off <= u) lo = mid;
            else hi = mid - 1;
        }
        const DevFrame fr = frames[lo];
        if (fr.mask == nullptr) continue;
        const ca_result res = results[lo];
        const int W = fr.W, H = fr.H;
        const int y0 = (u - fr.unit_off) * kMaskRowsPerWarp;
        const int nrows = min(kMaskRowsPerWarp, H - y0);
        const RowSpan sp = row_span(res, W, y0 + min(lane, nrows - 1));
        if (fr.mask_vec_ok) {
            const int VW = W >> 4;
            const int nvec = nrows * VW;
            int row = lane / VW, col = lane - row * VW;
            for (int base = 0; base < nvec; base += 32) {
                const int src = min(row, 31);
                const int a = __shfl_sync(kFull, sp.a, src);
                const int b = __shfl_sync(kFull, sp.b, src);
                const int ex = __shfl_sync(kFull, sp.exact, src);
                if (base + lane < nvec) {
                    const int x0 = col << 4;
                    uint4 v;
                    if (ex && x0 >= a && x0 + 15 <= b) {
                        v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
                    } else if (ex && (x0 + 15 < a || x0 > b)) {
                        v = make_uint4(0u, 0u, 0u, 0u);
                    } else if (ex) {
                        v = make_uint4(span_word(x0, a, b), span_word(x0 + 4, a, b),
                                       span_word(x0 + 8, a, b), span_word(x0 + 12, a, b));
                    } else {
                        const float dy = __fsub_rn(__int2float_rn(y0 + row), res.cy);
                        const float dy2 = __fmul_rn(dy, dy);
                        v = make_uint4(exact_word(x0, res, dy2), exact_word(x0 + 4, res, dy2),
                                       exact_word(x0 + 8, res, dy2), exact_word(x0 + 12, res, dy2));
                    }
                    st_cs_v4(fr.mask + (int64_t)(y0 + row) * W + x0, v);
                }
                col += 32;
                while (col >= VW) { col -= VW; ++row; }
            }
        } else {
            for (int r = 0; r < nrows; ++r) {
                const int a = __shfl_sync(kFull, sp.a, r);
                const int b = __shfl_sync(kFull, sp.b, r);
                const int ex = __shfl_sync(kFull, sp.exact, r);
                const int y = y0 + r;
                const float dy = __fsub_rn(__int2float_rn(y), res.cy);
                const float dy2 = __fmul_rn(dy, dy);
                const float rr = __fmul_rn(res.r, res.r);
                for (int x = lane; x < W; x += 32) {
                    uint8_t v;
                    if (!res.valid) v = 1;
                    else if (ex) v = (uint8_t)(x >= a && x <= b);
                    else v = (uint8_t)in_disc(x, res.cx, dy2, rr);
                    fr.mask[(int64_t)y * W + x] = v;
                }
            }
        }
    }
}

cudaError_t launch_mask(const DevFrame *frames, int B, const ca_result *res, int total_units,
                        int grid, cudaStream_t s) {
    if (total_units <= 0) return cudaSuccess;
    k_mask<<<grid, 256, 0, s>>>(frames, B, res, total_units);
    return cudaGetLastError();
}

}  // namespace ca
