// gs_server.cu -- continuous-batching request loop over device-resident scenes.
//
// Requests (scene, camera of any supported size, options, host output buffer) are queued by
// gs_server_submit.  A worker thread keeps up to `slots` batches in flight, each on its own
// stream with its own frame (pair buffers, records, scratch) and device output pool:
//   1. when a slot is free and requests are waiting, it takes the oldest ones (at most
//      max_batch, at most max_gaussians Gaussians in total) as candidates;
//   2. admission by pair-buffer memory: one count pass over the candidates (geometry and exact
//      pair counts, the first kernel of the pipeline) gives every request's pair count; the
//      oldest requests whose cumulative pairs fit the slot's pair capacity are admitted, the
//      rest go back to the head of the queue (a request that alone exceeds the capacity fails
//      with GS_ERR_PAIR_OVERFLOW);
//   3. the admitted batch runs every stage once over all its requests (per-request tile
//      ranges, gs_render_batch), then each image is copied to its host buffer and a host
//      callback marks the batch complete.
// Batches on different slots overlap on the device, and a request arriving while others run is
// admitted as soon as a slot frees -- continuous batching rather than a queue alone.  Streams are
// prioritised by batch age (the oldest batch in flight runs at the highest priority), and a lone
// request runs without the admission round trip.  Each
// request's image is bit-identical to rendering it alone.  `plain` mode is the baseline: one
// request at a time, synchronously, no count pass.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_internal.cuh"

gs_status frame_batch_count(gs_frame *f, int n, const gs_scene *const *scenes, const gs_camera *cams,
                            const gs_render_opts *opts, unsigned long long *req_pairs_dev, gs_stream stream);
int context_device(const gs_context *ctx);
gs_status frame_counters_async(gs_frame *f, void *host_dst, gs_stream stream);
gs_status frame_batch_finish(gs_frame *f, float *const *rgb, float *const *T, uint32_t *const *last,
                             gs_stream stream);
namespace gs {
void set_error_message(const char *msg);
}

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

gs_status err(gs_status code, const char *msg) {
    gs::set_error_message(msg);
    return code;
}

struct Request {
    uint64_t ticket = 0;
    const gs_scene *scene = nullptr;
    gs_camera cam{};
    gs_render_opts opts{};
    float *rgb_host = nullptr;
    double arrival = 0, admit = 0, done = 0;
    long long pairs = 0;
    int batch_size = 0;
    gs_status status = GS_OK;
    bool finished = false;
};

constexpr int kPrioLevels = 3;
constexpr long long kBacklog = 1;        // default: pending requests that justify overlapping batches
constexpr int kFifoLoadPct = 30;         // default: below this load, one request at a time
constexpr int kArrivalRing = 64;         // recent arrivals kept for the rate estimate
constexpr double kRateWindow = 0.25;     // seconds of arrivals that count
constexpr long long kBurst = 4;          // waiting requests that count as load whatever the estimate

struct Slot {
    cudaStream_t stream = nullptr;              // the stream of the batch in flight
    cudaStream_t streams[kPrioLevels] = {};     // by priority, highest first
    bool single = false;                        // the batch in flight is one unadmitted request
    gs_frame *frame = nullptr;
    float *out = nullptr;                       // max_batch images of max_width x max_height
    unsigned long long *pairs_dev = nullptr;    // per-request pair counts of the count pass
    unsigned long long *pairs_host = nullptr;   // pinned mirror
    gs::FrameCounters *ctr_host = nullptr;      // pinned copy of the frame's counters after the batch
    std::vector<uint64_t> inflight;
    bool busy = false;
    bool done = false;
    double done_time = 0;
    struct gs_server *server = nullptr;
};

}  // namespace

struct gs_server {
    gs_context *ctx = nullptr;
    int device = 0;
    gs_server_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    bool hold = false;
    uint64_t next_ticket = 1;
    long long completed = 0, batches = 0, batched_requests = 0;
    gs_status fatal = GS_OK;
    // load estimate: recent arrival times and the mean service time (admission to completion)
    double arrivals[kArrivalRing] = {};
    long long n_arrivals = 0;
    double svc_ema = 0;
};

namespace {

void CUDART_CB on_batch_done(void *p) {
    Slot *s = (Slot *)p;
    gs_server *sv = s->server;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        s->done = true;
        s->done_time = now_s();
    }
    sv->cv.notify_all();
}

// Marks the requests of finished slots complete.  Called with the lock held.
void reap(gs_server *sv) {
    for (Slot &s : sv->slots) {
        if (!s.busy || !s.done) continue;
        // device-side failures of the batch (pairs over the capacity, a wait past its limit)
        const unsigned dev = s.ctr_host ? s.ctr_host->status : 0u;
        const gs_status dev_st = (dev & gs::kStTimeout) ? GS_ERR_DEVICE_TIMEOUT
                                 : (dev & gs::kStPairOverflow) ? GS_ERR_PAIR_OVERFLOW
                                                               : GS_OK;
        for (uint64_t t : s.inflight) {
            auto it = sv->reqs.find(t);
            if (it == sv->reqs.end()) continue;
            if (dev_st != GS_OK && it->second.status == GS_OK) it->second.status = dev_st;
            // a lone request (or the plain loop's) ran without the admission pass: its count
            // arrived with the frame's counters
            if (sv->cfg.plain || s.single) it->second.pairs = (long long)s.ctr_host->n_pairs;
            it->second.done = s.done_time;
            it->second.finished = true;
            ++sv->completed;
            const double svc = s.done_time - it->second.admit;
            if (svc > 0) sv->svc_ema = sv->svc_ema > 0 ? 0.9 * sv->svc_ema + 0.1 * svc : svc;
        }
        s.inflight.clear();
        s.busy = false;
        s.done = false;
    }
}

size_t image_floats(const gs_server_cfg &c) { return (size_t)3 * c.max_width * c.max_height; }

// Launches one batch on slot `s`; returns the tickets that were not admitted (to requeue).
std::vector<uint64_t> launch_batch(gs_server *sv, Slot &s, std::vector<uint64_t> cand) {
    std::vector<uint64_t> back;
    const gs_server_cfg &cfg = sv->cfg;
    std::vector<const gs_scene *> scenes;
    std::vector<gs_camera> cams;
    std::vector<gs_render_opts> opts;
    std::vector<Request *> rq;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (uint64_t t : cand) {
            Request &r = sv->reqs[t];
            rq.push_back(&r);
            scenes.push_back(r.scene);
            cams.push_back(r.cam);
            opts.push_back(r.opts);
        }
    }
    const double t_admit = now_s();
    int n = (int)cand.size();
    std::vector<long long> req_pairs(n, 0);
    std::vector<float *> rgb(n);
    for (int i = 0; i < n; ++i) rgb[i] = s.out + (size_t)i * image_floats(cfg);
    gs_status st = GS_OK;
    // Priority by age: a batch launched while k others are in flight runs at the k-th highest
    // stream priority, so the oldest batch keeps the SMs it needs (its latency stays that of a
    // lone render) and younger ones fill what it leaves idle.
    int level = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (const Slot &o : sv->slots) level += (&o != &s && o.busy) ? 1 : 0;
    }
    s.stream = s.streams[level < kPrioLevels ? level : kPrioLevels - 1];
    s.single = !cfg.plain && n == 1;
    if (s.single) {
        // One request: nothing to admit or defer, so it renders without the admission round trip;
        // its pair count (and an overflow, if it alone exceeds the capacity) comes back with the
        // frame's counters when it completes.
        st = gs_render_batch(s.frame, 1, scenes.data(), cams.data(), opts.data(), rgb.data(), nullptr, nullptr,
                             s.stream);
    } else if (!cfg.plain) {
        // admission: exact pair counts of the candidates
        st = frame_batch_count(s.frame, n, scenes.data(), cams.data(), opts.data(), s.pairs_dev, s.stream);
        if (!st) {
            cudaMemcpyAsync(s.pairs_host, s.pairs_dev, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s.stream);
            cudaStreamSynchronize(s.stream);
        }
        int admit = 0;
        long long cum = 0;
        if (!st) {
            for (int i = 0; i < n; ++i) {
                const long long p = (long long)s.pairs_host[i];
                if (cum + p > cfg.pair_capacity) break;
                cum += p;
                req_pairs[i] = p;
                ++admit;
            }
            if (admit == 0) {
                // the oldest request alone does not fit: it fails, the others wait
                std::lock_guard<std::mutex> lk(sv->mu);
                rq[0]->status = GS_ERR_PAIR_OVERFLOW;
                rq[0]->pairs = (long long)s.pairs_host[0];
                rq[0]->admit = t_admit;
                rq[0]->done = now_s();
                rq[0]->finished = true;
                ++sv->completed;
                for (int i = 1; i < n; ++i) back.push_back(cand[i]);
                sv->cv.notify_all();
                return back;
            }
        }
        if (!st && admit < n) {
            for (int i = admit; i < n; ++i) back.push_back(cand[i]);
            n = admit;
            cand.resize(n);
            st = frame_batch_count(s.frame, n, scenes.data(), cams.data(), opts.data(), s.pairs_dev, s.stream);
        }
        if (!st) st = frame_batch_finish(s.frame, rgb.data(), nullptr, nullptr, s.stream);
    } else {
        st = gs_render_batch(s.frame, n, scenes.data(), cams.data(), opts.data(), rgb.data(), nullptr, nullptr,
                             s.stream);
    }
    if (!st) st = frame_counters_async(s.frame, s.ctr_host, (gs_stream)s.stream);
    if (!st) {
        for (int i = 0; i < n; ++i) {
            const size_t bytes = sizeof(float) * 3 * (size_t)cams[i].width * cams[i].height;
            if (cudaMemcpyAsync(rq[i]->rgb_host, rgb[i], bytes, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
                st = GS_ERR_CUDA;
        }
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    for (int i = 0; i < n; ++i) {
        rq[i]->admit = t_admit;
        rq[i]->batch_size = n;
        rq[i]->pairs = req_pairs[i];
    }
    if (st) {
        for (int i = 0; i < n; ++i) {
            rq[i]->status = st;
            rq[i]->done = now_s();
            rq[i]->finished = true;
            ++sv->completed;
        }
        sv->cv.notify_all();
        return back;
    }
    s.inflight = cand;
    s.busy = true;
    s.done = false;
    ++sv->batches;
    sv->batched_requests += n;
    lk.unlock();
    cudaLaunchHostFunc(s.stream, on_batch_done, &s);
    // one request at a time (plain), or a lone request on an idle device: the worker waits for it
    // itself, which returns the result sooner than the completion callback's thread hand-offs
    if (cfg.plain || (s.single && level == 0)) cudaStreamSynchronize(s.stream);
    return back;
}

// Estimated load: the arrival rate over the last kRateWindow seconds (at most kArrivalRing
// arrivals) times the mean service time.  Called with the lock held.
double estimate_load(const gs_server *sv, double now) {
    const long long n = sv->n_arrivals < kArrivalRing ? sv->n_arrivals : kArrivalRing;
    if (n < 2 || sv->svc_ema <= 0) return 0.0;
    const double newest = sv->arrivals[(sv->n_arrivals - 1) % kArrivalRing];
    if (now - newest > kRateWindow) return 0.0;
    long long k = 1;
    double oldest = newest;
    for (; k < n; ++k) {
        const double t = sv->arrivals[(sv->n_arrivals - 1 - k) % kArrivalRing];
        if (now - t > kRateWindow) break;
        oldest = t;
    }
    const double span = now - oldest;
    return span > 0 ? (double)k / span * sv->svc_ema : 0.0;
}

void worker_main(gs_server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        reap(sv);
        Slot *free_slot = nullptr;
        int busy = 0;
        for (Slot &s : sv->slots) {
            if (!s.busy && !free_slot) free_slot = &s;
            busy += s.busy ? 1 : 0;
        }
        // At light load one request at a time in arrival order is the fastest for every request:
        // a batch makes its first request wait for the others' work, and an overlapping batch
        // slows the older one (younger kernels, persistent and cooperative ones in particular,
        // hold SMs it needs).  Under load (estimated from arrivals and service times, or a queue
        // of kBurst), requests are batched, and a batch starts beside running ones once
        // overlap_pending requests wait.
        const int fifo_pct = sv->cfg.fifo_load_pct ? sv->cfg.fifo_load_pct : kFifoLoadPct;
        const bool fifo = !sv->cfg.plain && fifo_pct > 0 && (long long)sv->pending.size() < kBurst &&
                          estimate_load(sv, now_s()) * 100.0 < fifo_pct;
        const long long need = sv->cfg.overlap_pending > 0 ? sv->cfg.overlap_pending : kBacklog;
        const bool backlog = !fifo && (long long)sv->pending.size() >= need;
        if (!free_slot || sv->pending.empty() || sv->hold || (busy > 0 && !backlog)) {
            sv->cv.notify_all();
            sv->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        // candidates: oldest requests, bounded by max_batch and the frame's Gaussian capacity
        std::vector<uint64_t> cand;
        long long g = 0, px = 0;
        const int maxb = sv->cfg.plain || fifo ? 1 : sv->cfg.max_batch;
        const long long max_px = sv->cfg.batch_pixels > 0 ? sv->cfg.batch_pixels : 2ll * 1920 * 1080;
        while (!sv->pending.empty() && (int)cand.size() < maxb) {
            const uint64_t t = sv->pending.front();
            const Request &r = sv->reqs[t];
            const long long P = gs_scene_size(r.scene);
            const long long npx = (long long)r.cam.width * r.cam.height;
            if (!cand.empty() && (g + P > sv->cfg.max_gaussians || px + npx > max_px)) break;
            g += P;
            px += npx;
            cand.push_back(t);
            sv->pending.pop_front();
        }
        lk.unlock();
        std::vector<uint64_t> back = launch_batch(sv, *free_slot, cand);
        lk.lock();
        for (auto it = back.rbegin(); it != back.rend(); ++it) sv->pending.push_front(*it);
        sv->cv.notify_all();
    }
}

}  // namespace

extern "C" {

double gs_clock_s(void) { return now_s(); }

gs_status gs_default_server_cfg(gs_server_cfg *c) {
    if (!c) return err(GS_ERR_INVALID_ARG, "cfg is NULL");
    memset(c, 0, sizeof(*c));
    c->slots = 3;
    c->max_batch = 8;
    c->pair_capacity = 1ll << 26;
    c->max_gaussians = 1ll << 26;
    c->max_width = 3840;
    c->max_height = 2160;
    c->sort_mode = -1;
    c->blend_variant = -1;
    c->plain = 0;
    c->batch_pixels = 2 * 1920 * 1080;
    return GS_OK;
}

gs_status gs_server_create(gs_context *ctx, const gs_server_cfg *cfg, gs_server **out) {
    if (!ctx || !cfg || !out) return err(GS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    gs_server_cfg c = *cfg;
    if (c.plain) {
        c.slots = 1;
        c.max_batch = 1;
    }
    if (c.slots < 1 || c.slots > 8 || c.max_batch < 1 || c.max_batch > gs::kMaxBatch || c.pair_capacity <= 0 ||
        c.pair_capacity >= (1ll << 30) || c.max_gaussians <= 0 || c.max_width <= 0 || c.max_height <= 0 ||
        c.batch_pixels < 0 || c.overlap_pending < 0 || c.fifo_load_pct < -1)
        return err(GS_ERR_INVALID_ARG, "server configuration out of range");
    gs_server *sv = new (std::nothrow) gs_server();
    if (!sv) return err(GS_ERR_OOM, "host allocation failed");
    sv->ctx = ctx;
    sv->device = context_device(ctx);
    sv->cfg = c;
    sv->slots.resize(c.slots);
    const int tile_rows = (c.max_height + gs::kTile - 1) / gs::kTile;
    for (Slot &s : sv->slots) {
        s.server = sv;
        gs_status st = gs_frame_create(ctx, c.max_gaussians, c.pair_capacity, c.max_width,
                                       tile_rows * gs::kTile * c.max_batch, &s.frame);
        if (!st && (c.sort_mode >= 0 || c.blend_variant >= 0)) {
            gs_tuning t;
            gs_frame_get_tuning(s.frame, &t);
            if (c.sort_mode >= 0) t.sort_mode = c.sort_mode;
            if (c.blend_variant >= 0) t.blend_variant = c.blend_variant;
            st = gs_frame_set_tuning(s.frame, &t);
        }
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        for (int k = 0; k < kPrioLevels && !st; ++k) {
            const int prio = greatest + k < least ? greatest + k : least;
            if (cudaStreamCreateWithPriority(&s.streams[k], cudaStreamNonBlocking, prio) != cudaSuccess)
                st = GS_ERR_CUDA;
        }
        s.stream = s.streams[0];
        if (!st && cudaMalloc(&s.out, sizeof(float) * image_floats(c) * c.max_batch) != cudaSuccess) st = GS_ERR_OOM;
        if (!st && cudaMalloc(&s.pairs_dev, sizeof(unsigned long long) * gs::kMaxBatch) != cudaSuccess) st = GS_ERR_OOM;
        if (!st && cudaMallocHost(&s.ctr_host, sizeof(gs::FrameCounters)) != cudaSuccess) st = GS_ERR_OOM;
        if (!st) memset(s.ctr_host, 0, sizeof(gs::FrameCounters));
        if (!st && cudaMallocHost(&s.pairs_host, sizeof(unsigned long long) * gs::kMaxBatch) != cudaSuccess)
            st = GS_ERR_OOM;
        if (st) {
            gs_server_destroy(sv);
            return err(st, "server slot allocation failed");
        }
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return GS_OK;
}

gs_status gs_server_destroy(gs_server *sv) {
    if (!sv) return GS_OK;
    cudaSetDevice(sv->device);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &s : sv->slots) {
        for (cudaStream_t q : s.streams)
            if (q) cudaStreamSynchronize(q);
        if (s.frame) gs_frame_destroy(s.frame);
        for (cudaStream_t q : s.streams)
            if (q) cudaStreamDestroy(q);
        cudaFree(s.out);
        cudaFree(s.pairs_dev);
        cudaFreeHost(s.pairs_host);
        cudaFreeHost(s.ctr_host);
    }
    cudaGetLastError();
    delete sv;
    return GS_OK;
}

gs_status gs_server_submit(gs_server *sv, const gs_scene *scene, const gs_camera *cam, const gs_render_opts *opts,
                           float *rgb_host, double arrival_s, uint64_t *ticket) {
    if (!sv || !scene || !cam || !rgb_host || !ticket) return err(GS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > sv->cfg.max_width || cam->height > sv->cfg.max_height)
        return err(GS_ERR_INVALID_ARG, "image size outside the server's maximum");
    if (gs_scene_size(scene) > sv->cfg.max_gaussians) return err(GS_ERR_CAPACITY, "scene larger than a batch");
    Request r;
    r.scene = scene;
    r.cam = *cam;
    if (opts)
        r.opts = *opts;
    else
        gs_default_opts(&r.opts);
    r.rgb_host = rgb_host;
    r.arrival = arrival_s > 0 ? arrival_s : now_s();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->fatal) return err(sv->fatal, "server stopped after an error");
        r.ticket = sv->next_ticket++;
        *ticket = r.ticket;
        sv->reqs.emplace(r.ticket, r);
        sv->pending.push_back(r.ticket);
        sv->arrivals[sv->n_arrivals % kArrivalRing] = now_s();
        ++sv->n_arrivals;
    }
    sv->cv.notify_all();
    return GS_OK;
}

gs_status gs_server_wait(gs_server *sv, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out) {
    if (!sv) return err(GS_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return err(GS_ERR_INVALID_ARG, "unknown ticket");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (true) {
        reap(sv);
        it = sv->reqs.find(ticket);
        if (it->second.finished) break;
        if (timeout_ms >= 0 && std::chrono::steady_clock::now() >= deadline)
            return err(GS_ERR_DEVICE_TIMEOUT, "request not finished before the time limit");
        sv->cv.wait_for(lk, std::chrono::microseconds(200));
    }
    const Request r = it->second;
    sv->reqs.erase(it);
    if (out) {
        out->status = r.status;
        out->batch_size = r.batch_size;
        out->arrival_s = r.arrival;
        out->admit_s = r.admit;
        out->done_s = r.done;
        out->pairs = r.pairs;
    }
    return r.status;
}

gs_status gs_server_hold(gs_server *sv, int32_t hold) {
    if (!sv) return err(GS_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->hold = hold != 0;
    sv->cv.notify_all();
    if (sv->hold) {
        // the worker admits nothing more; wait for the batches in flight to be reaped
        auto idle = [&] {
            for (const Slot &s : sv->slots)
                if (s.busy) return false;
            return true;
        };
        while (!idle() && !sv->stop) sv->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    return GS_OK;
}

gs_status gs_server_get_stats(gs_server *sv, gs_server_stats *out) {
    if (!sv || !out) return err(GS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->completed = sv->completed;
    out->batches = sv->batches;
    out->batched_requests = sv->batched_requests;
    out->pending = (int64_t)sv->pending.size();
    return GS_OK;
}

}  // extern "C"
