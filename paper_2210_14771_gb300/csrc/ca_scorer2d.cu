// ca_scorer2d.cu -- the paper's own learned edge scorer (Sec. 2.2.4): three
// 3x3 convolutions to 8, 16 and 32 features with ReLU, a 1x1 head, on RGBXY
// strips 7 rows high (unpadded vertically, so 7 -> 5 -> 3 -> 1 rows: the
// strip's middle row; zero-padded horizontally).  Forward pass in binary32
// on the CUDA cores: one CTA per 128 output columns of a strip, every layer
// of the tile kept in shared memory with the halo columns it needs.
#include "ca_internal.h"

namespace ca {
namespace {

constexpr int kT = 128;                        // output columns per CTA (one per thread)
constexpr int kInC = kT + 6, kA1C = kT + 4, kA2C = kT + 2;
constexpr int kWOff1 = 0, kBOff1 = 360, kWOff2 = 368, kBOff2 = 1520, kWOff3 = 1536,
              kBOff3 = 6144, kWhOff = 6176, kBhOff = 6208;
constexpr int kWFloats = 6212;                 // 6209 parameters, padded
constexpr int kInFloats = 7 * kInC * 5, kA1Floats = 5 * kA1C * 8, kA2Floats = 3 * kA2C * 16;
constexpr size_t kSmem = sizeof(float) * (kWFloats + kInFloats + kA1Floats + kA2Floats);
static_assert(kBhOff + 1 == kScorer2dNParam, "parameter layout");

__global__ void __launch_bounds__(kT)
    k_sc2_forward(const uint8_t *__restrict__ strips7, const int32_t *__restrict__ rows, int W,
                  int H, const float *__restrict__ prm, float *__restrict__ logits) {
    extern __shared__ float sm2[];
    float *w = sm2;
    float *in = w + kWFloats;       // 7 rows x columns x0-3 .. x0+130 x 5 features
    float *a1 = in + kInFloats;     // 5 rows x columns x0-2 .. x0+129 x 8
    float *a2 = a1 + kA1Floats;     // 3 rows x columns x0-1 .. x0+128 x 16
    const int tid = threadIdx.x;
    const int tiles = (W + kT - 1) / kT;
    const int s = blockIdx.x / tiles, x0 = (blockIdx.x % tiles) * kT;
    for (int i = tid; i < kScorer2dNParam; i += kT) w[i] = prm[i];
    const uint8_t *src = strips7 + (size_t)s * 7 * W * 3;
    const float xc = 0.5f * (float)(W - 1), yc = 0.5f * (float)(H - 1);
    for (int i = tid; i < 7 * kInC; i += kT) {
        const int k = i / kInC, c = i - k * kInC, x = x0 - 3 + c;
        float *f = in + i * 5;
        if (x >= 0 && x < W) {
            const uint8_t *p = src + ((size_t)k * W + x) * 3;
            f[0] = (float)((int)p[0] - 128) * (1.0f / 128.0f);
            f[1] = (float)((int)p[1] - 128) * (1.0f / 128.0f);
            f[2] = (float)((int)p[2] - 128) * (1.0f / 128.0f);
            f[3] = __fdiv_rn(__fsub_rn((float)x, xc), (float)W);
            f[4] = __fdiv_rn(__fsub_rn((float)rows[(size_t)s * 7 + k], yc), (float)H);
        } else {
            f[0] = f[1] = f[2] = f[3] = f[4] = 0.0f;
        }
    }
    __syncthreads();
    // layer 1: 5 output rows, columns x0-2 .. x0+129; zero outside the strip
    for (int i = tid; i < 5 * kA1C; i += kT) {
        const int r = i / kA1C, c = i - r * kA1C, x = x0 - 2 + c;
        float *o = a1 + i * 8;
        if (x < 0 || x >= W) {
            for (int co = 0; co < 8; ++co) o[co] = 0.0f;
            continue;
        }
        for (int co = 0; co < 8; ++co) {
            float z = w[kBOff1 + co];
            for (int ci = 0; ci < 5; ++ci)
                for (int dr = 0; dr < 3; ++dr)
                    for (int dx = 0; dx < 3; ++dx)
                        z = fmaf(w[kWOff1 + ((co * 5 + ci) * 3 + dr) * 3 + dx],
                                 in[((r + dr) * kInC + c + dx) * 5 + ci], z);
            o[co] = fmaxf(z, 0.0f);
        }
    }
    __syncthreads();
    // layer 2: 3 output rows, columns x0-1 .. x0+128
    for (int i = tid; i < 3 * kA2C; i += kT) {
        const int r = i / kA2C, c = i - r * kA2C, x = x0 - 1 + c;
        float *o = a2 + i * 16;
        if (x < 0 || x >= W) {
            for (int co = 0; co < 16; ++co) o[co] = 0.0f;
            continue;
        }
        for (int co = 0; co < 16; ++co) {
            float z = w[kBOff2 + co];
            for (int ci = 0; ci < 8; ++ci)
                for (int dr = 0; dr < 3; ++dr)
                    for (int dx = 0; dx < 3; ++dx)
                        z = fmaf(w[kWOff2 + ((co * 8 + ci) * 3 + dr) * 3 + dx],
                                 a1[((r + dr) * kA1C + c + dx) * 8 + ci], z);
            o[co] = fmaxf(z, 0.0f);
        }
    }
    __syncthreads();
    // layer 3 and the head: this thread's column x0 + tid
    const int x = x0 + tid;
    if (x >= W) return;
    float lg = w[kBhOff];
    for (int co = 0; co < 32; ++co) {
        float z = w[kBOff3 + co];
        for (int ci = 0; ci < 16; ++ci)
            for (int dr = 0; dr < 3; ++dr)
                for (int dx = 0; dx < 3; ++dx)
                    z = fmaf(w[kWOff3 + ((co * 16 + ci) * 3 + dr) * 3 + dx],
                             a2[(dr * kA2C + tid + dx) * 16 + ci], z);
        lg = fmaf(w[kWhOff + co], fmaxf(z, 0.0f), lg);
    }
    logits[(size_t)s * W + x] = lg;
}

}  // namespace

cudaError_t sc2_launch_forward(const uint8_t *strips7, const int32_t *rows, int n, int W, int H,
                               const float *params, float *logits, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(k_sc2_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)n * ((W + kT - 1) / kT);
    if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    k_sc2_forward<<<(unsigned)blocks, kT, kSmem, s>>>(strips7, rows, W, H, params, logits);
    return cudaGetLastError();
}

}  // namespace ca
