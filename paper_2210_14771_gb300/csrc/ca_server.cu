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
//
// Zero-copy serving (cfg.zero_copy): frames stay in the caller's page-locked
// host memory and are never copied; the strip kernels read the 3 rows of each
// strip (9 N W bytes of a W-wide frame) over the host link, and masks go to
// page-locked mask buffers directly.  Only device-resident masks then count
// against the budget.
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
    const uint8_t *frame_dev;   // frame as the kernels address it (pool or mapped host memory)
    uint8_t *mask_dev;          // mask as the kernels address it, or NULL
    size_t frame_off, mask_off;
    bool frame_in_pool, mask_in_pool;
    uint8_t *mask_copy_to;      // host buffer the pool mask is copied to, or NULL
    double t_arrival, t_submit, t_launch;
};

struct Batch {
    std::vector<Request> reqs;
    cudaEvent_t done = nullptr;
    ca_result *res_dev = nullptr;    // max_batch results
    ca_result *raw_dev = nullptr;    // max_batch results before smoothing (smooth only)
    ca_result *res_host = nullptr;   // pinned
    bool busy = false;
    ca_status status = CA_OK;        // a step after the estimate failed
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

// Completes the requests of batch b (results from its pinned copy, or zero
// with the batch's error) and frees their pool blocks.
void finish_batch(ca_server *s, Batch &b) {
    const double t = now_s();
    for (size_t i = 0; i < b.reqs.size(); ++i) {
        const Request &r = b.reqs[i];
        ca_server_result o;
        std::memset(&o, 0, sizeof(o));
        o.ticket = r.ticket;
        o.stream_id = r.sid;
        o.status = b.status;
        o.frame_key = r.key;
        if (b.status == CA_OK) o.result = b.res_host[i];
        o.t_arrival = r.t_arrival;
        o.t_submit = r.t_submit;
        o.t_launch = r.t_launch;
        o.t_done = t;
        s->done.push_back(o);
        if (r.frame_in_pool) s->pool.release(r.frame_off);
        if (r.mask_in_pool) s->pool.release(r.mask_off);
        s->stream_busy[r.sid] -= 1;
    }
    b.reqs.clear();
    b.busy = false;
    b.status = CA_OK;
}

// Moves finished launches to the done list (blocking on the oldest if `wait`).
ca_status collect(ca_server *s, bool wait) {
    while (!s->in_flight.empty()) {
        Batch &b = s->batches[s->in_flight.front()];
        cudaError_t q = wait ? cudaEventSynchronize(b.done) : cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) break;
        SV_CUDA(q);
        finish_batch(s, b);
        s->in_flight.pop_front();
        wait = false;   // block at most once
    }
    return CA_OK;
}

// The steps of a launch after its estimate (smoothing, masks, copies back,
// completion event).  A failure here leaves part of the launch queued.
ca_status finish_launch(ca_server *s, Batch &b, const std::vector<int32_t> &track) {
    const int B = (int)b.reqs.size();
    if (s->smooth_state) {
        std::vector<int32_t> Hs(B), Ws(B);
        std::vector<uint8_t *> ms(B);
        bool all_masks = true;
        for (int i = 0; i < B; ++i) {
            Hs[i] = b.reqs[i].H;
            Ws[i] = b.reqs[i].W;
            ms[i] = b.reqs[i].mask_dev;
            all_masks = all_masks && ms[i] != nullptr;
        }
        ca_status st = ca_smooth_tracked(s->h, b.raw_dev, B, Ws.data(), track.data(),
                                         s->cfg.max_streams, &s->cfg.smooth_params,
                                         s->smooth_state, b.res_dev, s->compute);
        if (st == CA_OK && all_masks)
            st = ca_mask(s->h, b.res_dev, B, Hs.data(), Ws.data(), ms.data(), s->compute);
        if (st != CA_OK) return st;
    }
    SV_CUDA(cudaMemcpyAsync(b.res_host, b.res_dev, sizeof(ca_result) * B, cudaMemcpyDeviceToHost,
                            s->compute));
    for (int i = 0; i < B; ++i)
        if (b.reqs[i].mask_copy_to)
            SV_CUDA(cudaMemcpyAsync(b.reqs[i].mask_copy_to, b.reqs[i].mask_dev,
                                    (size_t)b.reqs[i].H * b.reqs[i].W, cudaMemcpyDeviceToHost,
                                    s->compute));
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
            fr[i].rgb_dev = r.frame_dev;
            fr[i].mask_dev = r.mask_dev;
            fr[i].H = r.H;
            fr[i].W = r.W;
            fr[i].pitch = (int64_t)r.W * 3;
            fr[i].frame_key = r.key;
            track[i] = s->cfg.track ? r.sid : -1;
        }
        if (!s->cfg.zero_copy) SV_CUDA(cudaStreamWaitEvent(s->compute, s->copied, 0));
        const bool smooth = s->smooth_state != nullptr;
        if (smooth)   // masks follow the smoothed circles
            for (int i = 0; i < B; ++i) fr[i].mask_dev = nullptr;
        ca_status st = ca_estimate_tracked(s->h, fr.data(), B, &s->cfg.params, s->state,
                                           track.data(), s->cfg.max_streams,
                                           smooth ? b.raw_dev : b.res_dev, s->compute);
        if (st != CA_OK) {
            // nothing of this launch is queued: its requests go back to the
            // front of the queue, in order, and a later poll retries them
            for (int i = B - 1; i >= 0; --i) s->pending.push_front(b.reqs[i]);
            b.reqs.clear();
            return st;
        }
        st = finish_launch(s, b, track);
        if (st != CA_OK) {
            // the estimate is queued (and has advanced the streams' state):
            // the frames complete with the error and their streams start afresh
            b.status = st;
            for (int i = 0; i < B; ++i) {
                if (track[i] < 0) continue;
                cudaMemsetAsync(s->state + track[i], 0, sizeof(ca_result), s->compute);
                if (s->smooth_state)
                    cudaMemsetAsync(s->smooth_state + 4 * (size_t)track[i], 0, 4 * sizeof(float),
                                    s->compute);
            }
        }
        if (cudaEventRecord(b.done, s->compute) != cudaSuccess) {
            if (b.status == CA_OK) b.status = CA_ERR_CUDA;
            finish_batch(s, b);   // nothing to wait for
            return b.status;
        }
        b.busy = true;
        s->in_flight.push_back(slot);
        if (st != CA_OK) return st;
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
    if (cfg->zero_copy != 0 && cfg->zero_copy != 1) return CA_ERR_INVALID_ARG;
    if (cfg->reserved != 0) return CA_ERR_INVALID_ARG;
    ca_status st = ca::check_params(h, &cfg->params);
    if (st != CA_OK) return st;
    // everything the server allocates lives on the handle's device, where its
    // estimates run
    const int dev = ca::handle_device(h);
    if (cudaSetDevice(dev) != cudaSuccess) return CA_ERR_CUDA;
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

}  // extern "C"

namespace {

// Device-visible address of page-locked host memory, or NULL.
const void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // pageable memory is not an error of the server
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

ca_status check_request(const ca_server *s, const ca_server_request &q) {
    if (!q.frame_host || q.reserved != 0) return CA_ERR_INVALID_ARG;
    if (q.stream_id < 0 || q.stream_id >= s->cfg.max_streams) return CA_ERR_INVALID_ARG;
    if (q.W < 8 || q.W > 4096 || q.H < 3 || q.H > 4096) return CA_ERR_INVALID_ARG;
    return CA_OK;
}

// Admits one checked request: device buffers from the pool (the frame unless
// zero-copy, the mask when kept on the device), the frame copy queued.
ca_status admit(ca_server *s, const ca_server_request &q, uint64_t *ticket) {
    const size_t fb = (size_t)q.H * q.W * 3, mb = (size_t)q.H * q.W;
    Request r;
    std::memset(&r, 0, sizeof(r));
    r.sid = q.stream_id;
    r.key = q.frame_key;
    r.H = q.H;
    r.W = q.W;
    const bool zc = s->cfg.zero_copy != 0;
    if (zc) {
        r.frame_dev = static_cast<const uint8_t *>(mapped_host(q.frame_host));
        if (!r.frame_dev) return CA_ERR_INVALID_ARG;   // not page-locked
    }
    const void *mask_mapped =
        zc && q.mask_host && s->cfg.want_masks ? mapped_host(q.mask_host) : nullptr;
    if (!zc) {
        if (!s->pool.alloc(fb, &r.frame_off)) return CA_ERR_ADMISSION;
        r.frame_in_pool = true;
    }
    if (s->cfg.want_masks) {
        if (mask_mapped) {   // written straight into the caller's page-locked buffer
            r.mask_dev = static_cast<uint8_t *>(const_cast<void *>(mask_mapped));
        } else {
            if (!s->pool.alloc(mb, &r.mask_off)) {
                if (r.frame_in_pool) s->pool.release(r.frame_off);
                return CA_ERR_ADMISSION;
            }
            r.mask_in_pool = true;
            r.mask_dev = s->arena + r.mask_off;
            r.mask_copy_to = q.mask_host;
        }
    }
    if (!zc) {
        r.frame_dev = s->arena + r.frame_off;
        cudaError_t e = cudaMemcpyAsync(s->arena + r.frame_off, q.frame_host, fb,
                                        cudaMemcpyHostToDevice, s->copy);
        if (e == cudaSuccess) e = cudaEventRecord(s->copied, s->copy);
        if (e != cudaSuccess) {
            s->pool.release(r.frame_off);
            if (r.mask_in_pool) s->pool.release(r.mask_off);
            return server_cuda(e);
        }
    }
    r.ticket = s->next_ticket++;
    r.t_arrival = q.t_arrival;
    r.t_submit = now_s();
    r.t_launch = 0.0;
    s->pending.push_back(r);
    s->stream_busy[q.stream_id] += 1;
    if (ticket) *ticket = r.ticket;
    return CA_OK;
}

}  // namespace

extern "C" {

ca_status ca_server_submit(ca_server *s, int stream_id, const uint8_t *frame_host, int H, int W,
                           uint64_t frame_key, double t_arrival, uint8_t *mask_host,
                           uint64_t *ticket) {
    if (!s) return CA_ERR_INVALID_ARG;
    ca_server_request q;
    std::memset(&q, 0, sizeof(q));
    q.frame_host = frame_host;
    q.mask_host = mask_host;
    q.frame_key = frame_key;
    q.t_arrival = t_arrival;
    q.stream_id = stream_id;
    q.H = H;
    q.W = W;
    ca_status st = check_request(s, q);
    if (st != CA_OK) return st;
    if (cudaSetDevice(s->device) != cudaSuccess) return CA_ERR_CUDA;
    return admit(s, q, ticket);
}

ca_status ca_server_submit_batch(ca_server *s, const ca_server_request *reqs, int n,
                                 uint64_t *tickets, int *n_admitted) {
    if (!s || !n_admitted || n < 0 || (n > 0 && !reqs)) return CA_ERR_INVALID_ARG;
    *n_admitted = 0;
    for (int i = 0; i < n; ++i) {
        ca_status st = check_request(s, reqs[i]);
        if (st != CA_OK) return st;
        if (s->cfg.zero_copy && !mapped_host(reqs[i].frame_host)) return CA_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(s->device) != cudaSuccess) return CA_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        ca_status st = admit(s, reqs[i], tickets ? tickets + i : nullptr);
        if (st != CA_OK) return st;
        *n_admitted = i + 1;
    }
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
