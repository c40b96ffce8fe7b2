// ca_static.cu -- ca_estimate_static: the estimate call for callers that must
// not allocate device memory.
//
// Everything the three kernels need beyond the caller's inputs and outputs
// (score tables, strip rows, frame descriptors, candidate slots, per-tile best
// circles, per-frame counters) lives in one fixed array of device memory,
// g_ca_static_scratch, defined below.  Every GPU that loads this library holds
// that array until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ca_internal.h"

using namespace ca;

namespace {

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

constexpr int kTilesStatic = CA_STATIC_MAX_HYPS / kHypTile;
constexpr size_t kLutBytes = sizeof(uint16_t) * kDevTableU16;
constexpr size_t kOffLuts = 0;
constexpr size_t kOffRows = align256(kOffLuts + kLutBytes);
constexpr size_t kOffFrames = align256(kOffRows + sizeof(int32_t) * kMaxSlots);
constexpr size_t kOffSlots = align256(kOffFrames + sizeof(DevFrame) * CA_STATIC_MAX_FRAMES);
constexpr size_t kOffTiles =
    align256(kOffSlots + sizeof(CandSlot) * kMaxSlots * (size_t)CA_STATIC_MAX_FRAMES);
constexpr size_t kOffBest =
    align256(kOffTiles + sizeof(TileRec) * kTilesStatic * (size_t)CA_STATIC_MAX_FRAMES);
constexpr size_t kOffDone = align256(kOffBest + sizeof(unsigned long long) * CA_STATIC_MAX_FRAMES);
constexpr size_t kStaticBytes = align256(kOffDone + sizeof(uint32_t) * CA_STATIC_MAX_FRAMES);
static_assert(kStaticBytes == CA_STATIC_SCRATCH_BYTES, "scratch size stated in ca.h");

}  // namespace

// The shared scratch.  Its name in host code is only a handle for the CUDA
// runtime, not a device address: host code must use the address returned by
// cudaGetSymbolAddress (see static_scratch below).
static __device__ __align__(256) unsigned char g_ca_static_scratch[kStaticBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device `dev`, looked up once
// per device (with that device current) and cached.
ca_status static_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return CA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ca_static_scratch);
        if (e != cudaSuccess || p == nullptr) return CA_ERR_CUDA;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return CA_OK;
}

// Host-side copy of what the kernels read: staged on the host stack and copied
// with ordinary (pageable) asynchronous copies, which allocate nothing.
struct HostTables {
    uint16_t luts[kLutG + kLutT + kLutI];
    uint16_t dev[kDevTableU16];
    int32_t rows[kMaxSlots];
};

}  // namespace

extern "C" ca_status ca_estimate_static(const uint8_t *frames_dev, int B, int H, int W,
                                        const uint64_t *keys, const ca_params *p,
                                        ca_result *out_dev, uint8_t *masks_dev, void *stream) {
    ca_status st = check_params(nullptr, p);
    if (st != CA_OK) return st;
    if (B < 0 || B > CA_STATIC_MAX_FRAMES) return CA_ERR_INVALID_ARG;
    if (B == 0) return CA_OK;
    if (!frames_dev || !out_dev) return CA_ERR_INVALID_ARG;
    if (W < 8 || W > kMaxDim || H < 3 || H > kMaxDim) return CA_ERR_INVALID_ARG;
    long long nh = p->n_hyps;
    if (p->hyp_mode == CA_HYP_EXHAUSTIVE) {
        const long long nk = (long long)p->n_strips * p->cands_per_strip;
        nh = std::max(1LL, nk * (nk - 1) * (nk - 2) / 6);
    }
    if (nh > CA_STATIC_MAX_HYPS) return CA_ERR_INVALID_ARG;

    // the host-stack copies below cannot be recorded into a graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return CA_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return CA_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CA_ERR_CUDA;
    unsigned char *scratch = nullptr;
    if ((st = static_scratch(dev, &scratch)) != CA_OK) return st;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;

    // parameters, as ca_estimate_uniform derives them
    HostTables ht;
    int qg_sat = kLutG - 1;
    build_luts(*p, ht.luts, &qg_sat);
    pack_device_tables(ht.luts, qg_sat, ht.dev);
    strip_rows(H, p->n_strips, p->alpha, ht.rows);
    DevParams P;
    std::memset(&P, 0, sizeof(P));
    P.N = p->n_strips;
    P.K = p->cands_per_strip;
    P.refine = p->refine_iters;
    P.T_px = (int)std::ceil((double)p->t_px);
    P.sup_px = p->sup_px;
    P.hyp_mode = p->hyp_mode;
    P.debug = 0;
    P.T_ps = (uint32_t)std::ceil((double)p->t_ps * 32768.0);
    const double norm = p->score_norm == CA_NORM_2N ? 2.0 * p->n_strips
                      : p->score_norm == CA_NORM_NK ? (double)p->n_strips * p->cands_per_strip
                                                    : 1.0;
    P.T_cs = (uint32_t)std::ceil((double)p->t_cs * 32768.0 * norm);
    P.score_den = 32768.0 * norm;
    P.tcs_unit = (double)p->t_cs * 32768.0;
    P.norm_circle = p->score_norm == CA_NORM_CIRCLE ? 1 : 0;
    P.qg_sat = qg_sat;
    P.io_cut = iota_cut(ht.luts + kLutG + kLutT, P.T_ps);
    angle_cut(ht.luts + kLutG, P.T_ps, P);
    P.NH = (int)nh;
    P.hyp_threads = choose_hyp_threads(p->hyp_threads, B, nh, sms);
    P.n_tiles = (int)((nh + kHypTile / P.hyp_threads - 1) / (kHypTile / P.hyp_threads));
    // the tile records of all frames must fit the scratch's tile region
    while (P.hyp_threads > 1 && (long long)B * P.n_tiles > (long long)kTilesStatic * CA_STATIC_MAX_FRAMES) {
        P.hyp_threads >>= 1;
        P.n_tiles = (int)((nh + kHypTile / P.hyp_threads - 1) / (kHypTile / P.hyp_threads));
    }
    P.t_ri = p->t_ri;
    P.r_min = p->r_min;
    P.r_max = p->r_max;
    P.d_max = p->d_max;
    P.seed = p->seed;
    P.max_w = W;

    // frame descriptors (uniform batch stored back to back)
    DevFrame frames[CA_STATIC_MAX_FRAMES];
    const size_t fbytes = (size_t)H * W * 3, mbytes = (size_t)H * W;
    const int units_per_frame = (H + kMaskRowsPerUnit - 1) / kMaskRowsPerUnit;
    for (int i = 0; i < B; ++i) {
        DevFrame &d = frames[i];
        std::memset(&d, 0, sizeof(d));
        d.rgb = frames_dev + fbytes * i;
        d.mask = masks_dev ? masks_dev + mbytes * i : nullptr;
        d.pitch = (int64_t)W * 3;
        d.key = keys ? keys[i] : (uint64_t)i;
        d.H = H;
        d.W = W;
        d.rows_off = 0;
        d.unit_off = masks_dev ? units_per_frame * i : 0;
        d.vec_ok = ((uintptr_t)d.rgb % 16 == 0) && (W % 16 == 0);
        d.mask_vec_ok = !masks_dev ? 0
                      : ((uintptr_t)d.mask % 32 == 0 && W % 32 == 0) ? 2
                      : ((uintptr_t)d.mask % 16 == 0 && W % 16 == 0) ? 1 : 0;
    }

    DevFrame *d_frames = reinterpret_cast<DevFrame *>(scratch + kOffFrames);
    int32_t *d_rows = reinterpret_cast<int32_t *>(scratch + kOffRows);
    uint16_t *d_luts = reinterpret_cast<uint16_t *>(scratch + kOffLuts);
    Workspace ws;
    ws.slots = reinterpret_cast<CandSlot *>(scratch + kOffSlots);
    ws.tiles = reinterpret_cast<TileRec *>(scratch + kOffTiles);
    ws.best = reinterpret_cast<unsigned long long *>(scratch + kOffBest);
    ws.done = reinterpret_cast<uint32_t *>(scratch + kOffDone);
    P.rows_tab = d_rows;

    if (cudaMemcpyAsync(d_luts, ht.dev, kLutBytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_rows, ht.rows, sizeof(int32_t) * P.N, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_frames, frames, sizeof(DevFrame) * B, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return CA_ERR_CUDA;
    // per-frame best keys and finished-CTA counters must start at zero
    if (cudaMemsetAsync(ws.best, 0, sizeof(unsigned long long) * B, s) != cudaSuccess ||
        cudaMemsetAsync(ws.done, 0, sizeof(uint32_t) * B, s) != cudaSuccess)
        return CA_ERR_CUDA;

    int nb = 0;
    if (strips_occupancy(&nb, strips_smem_bytes(P)) != cudaSuccess) return CA_ERR_CUDA;
    const int sgrid = P.K == 2 ? B * P.N : (2 * B * P.N + 7) / 8;
    (void)nb;
    if (launch_strips(d_frames, B, d_rows, P, d_luts, ws.slots, sgrid, s) != cudaSuccess ||
        launch_fit(d_frames, B, P, ws.slots, ws, out_dev, s) != cudaSuccess)
        return CA_ERR_CUDA;
    if (masks_dev) {
        const int units = units_per_frame * B;
        const int mgrid = std::max(1, std::min((units + 7) / 8, sms * mask_blocks_per_sm()));
        if (launch_mask(d_frames, B, out_dev, units, mgrid, s) != cudaSuccess) return CA_ERR_CUDA;
    }
    return CA_OK;
}
