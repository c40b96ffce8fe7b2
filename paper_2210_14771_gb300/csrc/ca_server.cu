// ca_server.cu -- serving: frames of many video streams estimated with
// continuous batching under a device-memory budget.
//
// A request (one frame of one stream) is admitted when its device buffers
// (frame, and mask when asked for) fit the server's memory pool; its frame is
// copied to the device on the copy stream at once.  Every poll launches the
// admitted requests whose copies are queued -- at most one frame per stream
// per launch, up to max_batch -- as one tracked estimate on the compute
// stream, without waiting for a batch to fill or for earlier launches to end:
// the GPU works through the launches back to back while new frames are copied
// in and finished results are copied out.  Each stream's previous circle
// stays on the device and joins the RANSAC of its next frame (tracked
// estimate, Sec. 4's use of the previous estimate).  Frames of one stream are
// estimated in submission order, so every result equals the one the frame
// gets when its stream is served alone.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "ca_internal.h"

namespace {

// First-fit offset allocator over [0, size) with coalescing (host bookkeeping
// of the server's device pool).
struct Pool {
    size_t size = 0, align = 256, used = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> taken;   // offset -> length

    void init(size_t bytes, size_t al) {
        size = bytes;
        align = std::max<size_t>(al, 1);
        used = 0;
        free_.clear();
        taken.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t *off) {
        const size_t need = (std::max<size_t>(bytes, 1) + align - 1) / align * align;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t o = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[o + need] = len - need;
            taken[o] = need;
            used += need;
            *off = o;
            return true;
        }
        return false;
    }
    bool release(size_t off) {
        auto t = taken.find(off);
        if (t == taken.end()) return false;
        size_t o = off, len = t->second;
        taken.erase(t);
        used -= len;
        auto nx = free_.lower_bound(o);
        if (nx != free_.end() && nx->first == o + len) {   // merge with the next block
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                         // merge with the previous block
            auto pv = std::prev(nx);
            if (pv->first + pv->second == o) {
                o = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = len;
        return true;
    }
    size_t largest_free() const {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    int sid;
    uint64_t key;
    int H, W;
    size_t frame_off, mask_off;
    bool has_mask;
    uint8_t *mask_host;
    double t_arrival, t_submit, t_launch;
};

struct Batch {
    std::vector<Request> reqs;
    cudaEvent_t done = nullptr;
    ca_result *res_dev = nullptr;    // max_batch results
    ca_result *raw_dev = nullptr;    // max_batch results before smoothing (smooth only)
    ca_result *res_host = nullptr;   // pinned
    bool busy = false;
};

}  // namespace

struct ca_pool {
    Pool p;
};

struct ca_server {
    ca_handle *h = nullptr;
    int device = 0;
    ca_server_config cfg{};
    Pool pool;
    unsigned char *arena = nullptr;   // the device pool
    ca_result *state = nullptr;       // per stream: previous result
    float *smooth_state = nullptr;    // per stream: smoothing state {cx, cy, r, conf}
    cudaStream_t copy = nullptr, compute = nullptr;
    cudaEvent_t copied = nullptr;     // last frame copy queued
    std::deque<Request> pending;      // admitted, not yet launched
    std::vector<Batch> batches;       // ring of launch slots
    std::deque<int> in_flight;        // batch indices, oldest first
    std::vector<int> stream_busy;     // frames of each stream admitted and not yet done
    uint64_t next_ticket = 1;
    std::vector<ca_server_result> done;   // finished, not yet returned
};

namespace {

constexpr int kServerBatches = 4;   // launches that may be queued on the GPU at once

ca_status server_cuda(cudaError_t e) {
    return e == cudaSuccess ? CA_OK : (e == cudaErrorMemoryAllocation ? CA_ERR_OOM : CA_ERR_CUDA);
}

#define SV_CUDA(call)                               \
    do {                                            \
        ca_status s_ = server_cuda(call);           \
        if (s_ != CA_OK) return s_;                 \
    } while (0)

// Moves finished launches to the done list (blocking on the oldest if `wait`).
ca_status collect(ca_server *s, bool wait) {
    while (!s->in_flight.empty()) {
        Batch &b = s->batches[s->in_flight.front()];
        cudaError_t q = wait ? cudaEventSynchronize(b.done) : cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) break;
        SV_CUDA(q);
        const double t = now_s();
        for (size_t i = 0; i < b.reqs.size(); ++i) {
            const Request &r = b.reqs[i];
            ca_server_result o;
            std::memset(&o, 0, sizeof(o));
            o.ticket = r.ticket;
            o.stream_id = r.sid;
            o.frame_key = r.key;
            o.result = b.res_host[i];
            o.t_arrival = r.t_arrival;
            o.t_submit = r.t_submit;
            o.t_launch = r.t_launch;
            o.t_done = t;
            s->done.push_back(o);
            s->pool.release(r.frame_off);
            if (r.has_mask) s->pool.release(r.mask_off);
            s->stream_busy[r.sid] -= 1;
        }
        b.reqs.clear();
        b.busy = false;
        s->in_flight.pop_front();
        wait = false;   // block at most once
    }
    return CA_OK;
}

// Launches admitted requests, one frame per stream per launch, oldest first.
ca_status launch(ca_server *s) {
    while (!s->pending.empty()) {
        int slot = -1;
        for (int i = 0; i < (int)s->batches.size(); ++i)
            if (!s->batches[i].busy) { slot = i; break; }
        if (slot < 0) return CA_OK;   // every launch slot is queued on the GPU
        Batch &b = s->batches[slot];
        std::vector<char> taken(s->cfg.max_streams, 0);
        std::deque<Request> keep;
        while (!s->pending.empty()) {
            Request r = s->pending.front();
            s->pending.pop_front();
            if ((int)b.reqs.size() < s->cfg.max_batch && !taken[r.sid]) {
                taken[r.sid] = 1;
                b.reqs.push_back(r);
            } else {
                keep.push_back(r);
            }
        }
        s->pending.swap(keep);
        const int B = (int)b.reqs.size();
        std::vector<ca_frame> fr(B);
        std::vector<int32_t> track(B);
        const double t = now_s();
        for (int i = 0; i < B; ++i) {
            Request &r = b.reqs[i];
            r.t_launch = t;
            fr[i].rgb_dev = s->arena + r.frame_off;
            fr[i].mask_dev = r.has_mask ? s->arena + r.mask_off : nullptr;
            fr[i].H = r.H;
            fr[i].W = r.W;
            fr[i].pitch = (int64_t)r.W * 3;
            fr[i].frame_key = r.key;
            track[i] = s->cfg.track ? r.sid : -1;
        }
        SV_CUDA(cudaStreamWaitEvent(s->compute, s->copied, 0));
        const bool smooth = s->smooth_state != nullptr;
        if (smooth)   // masks follow the smoothed circles
            for (int i = 0; i < B; ++i) fr[i].mask_dev = nullptr;
        ca_status st = ca_estimate_tracked(s->h, fr.data(), B, &s->cfg.params, s->state,
                                           track.data(), s->cfg.max_streams,
                                           smooth ? b.raw_dev : b.res_dev, s->compute);
        if (st != CA_OK) return st;
        if (smooth) {
            std::vector<int32_t> Hs(B), Ws(B);
            std::vector<uint8_t *> ms(B);
            bool all_masks = true;
            for (int i = 0; i < B; ++i) {
                Hs[i] = b.reqs[i].H;
                Ws[i] = b.reqs[i].W;
                ms[i] = b.reqs[i].has_mask ? s->arena + b.reqs[i].mask_off : nullptr;
                all_masks = all_masks && b.reqs[i].has_mask;
            }
            st = ca_smooth_tracked(s->h, b.raw_dev, B, Ws.data(), track.data(), s->cfg.max_streams,
                                   &s->cfg.smooth_params, s->smooth_state, b.res_dev, s->compute);
            if (st == CA_OK && all_masks)
                st = ca_mask(s->h, b.res_dev, B, Hs.data(), Ws.data(), ms.data(), s->compute);
            if (st != CA_OK) return st;
        }
        SV_CUDA(cudaMemcpyAsync(b.res_host, b.res_dev, sizeof(ca_result) * B,
                                cudaMemcpyDeviceToHost, s->compute));
        for (int i = 0; i < B; ++i)
            if (b.reqs[i].has_mask && b.reqs[i].mask_host)
                SV_CUDA(cudaMemcpyAsync(b.reqs[i].mask_host, s->arena + b.reqs[i].mask_off,
                                        (size_t)b.reqs[i].H * b.reqs[i].W, cudaMemcpyDeviceToHost,
                                        s->compute));
        SV_CUDA(cudaEventRecord(b.done, s->compute));
        b.busy = true;
        s->in_flight.push_back(slot);
    }
    return CA_OK;
}

void server_free(ca_server *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto &b : s->batches) {
        if (b.done) cudaEventDestroy(b.done);
        cudaFree(b.res_dev);
        cudaFree(b.raw_dev);
        if (b.res_host) cudaFreeHost(b.res_host);
    }
    if (s->copied) cudaEventDestroy(s->copied);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->compute) cudaStreamDestroy(s->compute);
    cudaFree(s->arena);
    cudaFree(s->state);
    cudaFree(s->smooth_state);
    delete s;
}

}  // namespace

extern "C" {

double ca_server_now(void) { return now_s(); }

ca_status ca_server_create(ca_handle *h, const ca_server_config *cfg, ca_server **out) {
    if (!h || !cfg || !out) return CA_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_streams < 1 || cfg->max_streams > (1 << 20) || cfg->max_batch < 1 ||
        cfg->max_batch > 4096 || cfg->mem_budget < 4096)
        return CA_ERR_INVALID_ARG;
    if (cfg->smooth != 0 && cfg->smooth != 1) return CA_ERR_INVALID_ARG;
    if (cfg->smooth) {
        const ca_smooth_params &sp = cfg->smooth_params;
        if (!cfg->track || !std::isfinite(sp.gamma) || !std::isfinite(sp.jump) ||
            !std::isfinite(sp.t_hold) || sp.gamma < 0.0f || sp.gamma >= 1.0f || sp.jump < 0.0f ||
            sp.t_hold < 0.0f || sp.reserved != 0)
            return CA_ERR_INVALID_ARG;
    }
    ca_status st = ca::check_params(h, &cfg->params);
    if (st != CA_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CA_ERR_CUDA;
    ca_server *s = new ca_server();
    s->h = h;
    s->device = dev;
    s->cfg = *cfg;
    s->pool.init(cfg->mem_budget, 256);
    s->stream_busy.assign(cfg->max_streams, 0);
    auto bail = [&](cudaError_t e) {
        server_free(s);
        return server_cuda(e);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&s->arena, cfg->mem_budget)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->state, sizeof(ca_result) * cfg->max_streams)) != cudaSuccess) return bail(e);
    if ((e = cudaMemset(s->state, 0, sizeof(ca_result) * cfg->max_streams)) != cudaSuccess) return bail(e);
    if (cfg->smooth) {
        if ((e = cudaMalloc(&s->smooth_state, sizeof(float) * 4 * cfg->max_streams)) != cudaSuccess)
            return bail(e);
        if ((e = cudaMemset(s->smooth_state, 0, sizeof(float) * 4 * cfg->max_streams)) != cudaSuccess)
            return bail(e);
    }
    if ((e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    if ((e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    if ((e = cudaEventCreateWithFlags(&s->copied, cudaEventDisableTiming)) != cudaSuccess) return bail(e);
    if ((e = cudaEventRecord(s->copied, s->copy)) != cudaSuccess) return bail(e);
    s->batches.resize(kServerBatches);
    for (auto &b : s->batches) {
        if ((e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming)) != cudaSuccess) return bail(e);
        if ((e = cudaMalloc(&b.res_dev, sizeof(ca_result) * cfg->max_batch)) != cudaSuccess) return bail(e);
        if (cfg->smooth &&
            (e = cudaMalloc(&b.raw_dev, sizeof(ca_result) * cfg->max_batch)) != cudaSuccess)
            return bail(e);
        if ((e = cudaMallocHost(&b.res_host, sizeof(ca_result) * cfg->max_batch)) != cudaSuccess)
            return bail(e);
    }
    *out = s;
    return CA_OK;
}

ca_status ca_server_submit(ca_server *s, int stream_id, const uint8_t *frame_host, int H, int W,
                           uint64_t frame_key, double t_arrival, uint8_t *mask_host,
                           uint64_t *ticket) {
    if (!s || !frame_host) return CA_ERR_INVALID_ARG;
    if (stream_id < 0 || stream_id >= s->cfg.max_streams) return CA_ERR_INVALID_ARG;
    if (W < 8 || W > 4096 || H < 3 || H > 4096) return CA_ERR_INVALID_ARG;
    const size_t fb = (size_t)H * W * 3, mb = (size_t)H * W;
    const bool want_mask = s->cfg.want_masks != 0;
    size_t foff = 0, moff = 0;
    if (!s->pool.alloc(fb, &foff)) return CA_ERR_ADMISSION;
    if (want_mask && !s->pool.alloc(mb, &moff)) {
        s->pool.release(foff);
        return CA_ERR_ADMISSION;
    }
    cudaSetDevice(s->device);
    cudaError_t e = cudaMemcpyAsync(s->arena + foff, frame_host, fb, cudaMemcpyHostToDevice, s->copy);
    if (e == cudaSuccess) e = cudaEventRecord(s->copied, s->copy);
    if (e != cudaSuccess) {
        s->pool.release(foff);
        if (want_mask) s->pool.release(moff);
        return server_cuda(e);
    }
    Request r;
    r.ticket = s->next_ticket++;
    r.sid = stream_id;
    r.key = frame_key;
    r.H = H;
    r.W = W;
    r.frame_off = foff;
    r.mask_off = moff;
    r.has_mask = want_mask;
    r.mask_host = mask_host;
    r.t_arrival = t_arrival;
    r.t_submit = now_s();
    r.t_launch = 0.0;
    s->pending.push_back(r);
    s->stream_busy[stream_id] += 1;
    if (ticket) *ticket = r.ticket;
    return CA_OK;
}

ca_status ca_server_poll(ca_server *s, int wait, ca_server_result *out, int max, int *n_done) {
    if (!s || !n_done || (max > 0 && !out)) return CA_ERR_INVALID_ARG;
    *n_done = 0;
    cudaSetDevice(s->device);
    ca_status st = collect(s, false);
    if (st == CA_OK) st = launch(s);
    if (st == CA_OK && wait && s->done.empty() && !s->in_flight.empty()) {
        st = collect(s, true);
        if (st == CA_OK) st = launch(s);
    }
    if (st != CA_OK) return st;
    const int n = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < n; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_done = n;
    return CA_OK;
}

ca_status ca_server_stats(const ca_server *s, size_t *bytes_in_use, int32_t *pending,
                          int32_t *launches_in_flight) {
    if (!s) return CA_ERR_INVALID_ARG;
    if (bytes_in_use) *bytes_in_use = s->pool.used;
    if (pending) *pending = (int32_t)s->pending.size();
    if (launches_in_flight) *launches_in_flight = (int32_t)s->in_flight.size();
    return CA_OK;
}

ca_status ca_server_destroy(ca_server *s) {
    if (!s) return CA_ERR_INVALID_ARG;
    server_free(s);
    return CA_OK;
}

// ---- the admission allocator on its own (host only)
ca_status ca_pool_create(size_t bytes, size_t align, ca_pool **out) {
    if (!out || bytes == 0) return CA_ERR_INVALID_ARG;
    *out = new ca_pool();
    (*out)->p.init(bytes, align);
    return CA_OK;
}

ca_status ca_pool_alloc(ca_pool *p, size_t bytes, size_t *offset) {
    if (!p || !offset) return CA_ERR_INVALID_ARG;
    return p->p.alloc(bytes, offset) ? CA_OK : CA_ERR_ADMISSION;
}

ca_status ca_pool_free(ca_pool *p, size_t offset) {
    if (!p) return CA_ERR_INVALID_ARG;
    return p->p.release(offset) ? CA_OK : CA_ERR_INVALID_ARG;
}

ca_status ca_pool_stats(const ca_pool *p, size_t *used, size_t *largest_free) {
    if (!p) return CA_ERR_INVALID_ARG;
    if (used) *used = p->p.used;
    if (largest_free) *largest_free = p->p.largest_free();
    return CA_OK;
}

ca_status ca_pool_destroy(ca_pool *p) {
    if (!p) return CA_ERR_INVALID_ARG;
    delete p;
    return CA_OK;
}

}  // extern "C"
