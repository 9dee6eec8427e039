// gs_router.cu -- requests routed across replicas (one gs_server per GPU).
//
// Frames and requests are independent, so several GPUs serve them as replicas with no exchange
// between them; what is left to decide is where each request goes.  A request may only go to a
// replica that holds its scene; among those it goes to the one with the fewest image pixels
// outstanding (submitted through the router and not yet waited for), a proxy for the work queued
// there that needs no device query.  The router is host code only: submit and wait reach the
// replicas through a backend (gs_server objects, or caller-supplied functions, which is how the
// policy is tested without GPUs).
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "gs.h"

namespace gs {
void set_error_message(const char *msg);
}

namespace {

constexpr int kMaxReplicas = 64;
constexpr int kMaxScenes = 4096;

gs_status fail(gs_status code, const char *msg) {
    gs::set_error_message(msg);
    return code;
}

struct Routed {
    int32_t replica;
    uint64_t ticket;
    int64_t pixels;
};

}  // namespace

struct gs_router {
    int replicas = 0;
    gs_router_backend backend{};
    std::vector<gs_server *> servers;                        // server backend only
    std::vector<std::vector<const gs_scene *>> handles;      // [scene][replica]
    std::vector<uint64_t> placed;                            // [scene] bit mask of replicas
    std::vector<int64_t> out_requests, out_pixels;           // [replica]
    std::unordered_map<uint64_t, Routed> routed;
    uint64_t next_ticket = 1;
    std::mutex mu;
};

namespace {

gs_status server_submit(void *user, int32_t replica, int32_t scene, const gs_camera *cam, const gs_render_opts *opts,
                        float *rgb_host, double arrival_s, uint64_t *ticket) {
    gs_router *r = (gs_router *)user;
    const gs_scene *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(r->mu);
        s = r->handles[scene][replica];
    }
    if (!s) return fail(GS_ERR_INVALID_ARG, "no scene handle placed on this replica");
    return gs_server_submit(r->servers[replica], s, cam, opts, rgb_host, arrival_s, ticket);
}

gs_status server_wait(void *user, int32_t replica, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out) {
    gs_router *r = (gs_router *)user;
    return gs_server_wait(r->servers[replica], ticket, timeout_ms, out);
}

gs_status make(int32_t replicas, gs_router **out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (replicas < 1 || replicas > kMaxReplicas) return fail(GS_ERR_INVALID_ARG, "replicas out of range (1..64)");
    gs_router *r = new (std::nothrow) gs_router();
    if (!r) return fail(GS_ERR_OOM, "host allocation failed");
    r->replicas = replicas;
    r->out_requests.assign(replicas, 0);
    r->out_pixels.assign(replicas, 0);
    *out = r;
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_router_create(int32_t replicas, const gs_router_backend *backend, gs_router **out) {
    if (!backend || !backend->submit || !backend->wait) return fail(GS_ERR_INVALID_ARG, "backend incomplete");
    gs_status st = make(replicas, out);
    if (st) return st;
    (*out)->backend = *backend;
    return GS_OK;
}

gs_status gs_router_create_on_servers(int32_t replicas, gs_server *const *servers, gs_router **out) {
    if (!servers) return fail(GS_ERR_INVALID_ARG, "servers is NULL");
    for (int i = 0; i < replicas && i < kMaxReplicas; ++i)
        if (!servers[i]) return fail(GS_ERR_INVALID_ARG, "a server is NULL");
    gs_status st = make(replicas, out);
    if (st) return st;
    gs_router *r = *out;
    r->servers.assign(servers, servers + replicas);
    r->backend.submit = server_submit;
    r->backend.wait = server_wait;
    r->backend.user = r;
    return GS_OK;
}

gs_status gs_router_destroy(gs_router *r) {
    delete r;
    return GS_OK;
}

gs_status gs_router_place_scene(gs_router *r, int32_t scene, int32_t replica, const gs_scene *handle) {
    if (!r) return fail(GS_ERR_INVALID_ARG, "router is NULL");
    if (scene < 0 || scene >= kMaxScenes || replica < 0 || replica >= r->replicas)
        return fail(GS_ERR_INVALID_ARG, "scene or replica out of range");
    if (!r->servers.empty() && !handle) return fail(GS_ERR_INVALID_ARG, "the server backend needs a scene handle");
    std::lock_guard<std::mutex> lk(r->mu);
    if ((int)r->placed.size() <= scene) {
        r->placed.resize(scene + 1, 0);
        r->handles.resize(scene + 1, std::vector<const gs_scene *>(r->replicas, nullptr));
    }
    r->placed[scene] |= 1ull << replica;
    r->handles[scene][replica] = handle;
    return GS_OK;
}

gs_status gs_router_submit(gs_router *r, int32_t scene, const gs_camera *cam, const gs_render_opts *opts,
                           float *rgb_host, double arrival_s, uint64_t *ticket) {
    if (!r || !cam || !ticket) return fail(GS_ERR_INVALID_ARG, "NULL router, camera or ticket");
    const int64_t px = (int64_t)cam->width * cam->height;
    int best = -1;
    {
        std::lock_guard<std::mutex> lk(r->mu);
        const uint64_t mask = (scene >= 0 && scene < (int)r->placed.size()) ? r->placed[scene] : 0;
        for (int i = 0; i < r->replicas; ++i)
            if (((mask >> i) & 1ull) && (best < 0 || r->out_pixels[i] < r->out_pixels[best])) best = i;
        if (best < 0) return fail(GS_ERR_INVALID_ARG, "scene is placed on no replica");
        r->out_pixels[best] += px;      // reserve before submitting, so concurrent submits spread
        r->out_requests[best] += 1;
    }
    uint64_t inner = 0;
    gs_status st = r->backend.submit(r->backend.user, best, scene, cam, opts, rgb_host, arrival_s, &inner);
    std::lock_guard<std::mutex> lk(r->mu);
    if (st) {
        r->out_pixels[best] -= px;
        r->out_requests[best] -= 1;
        return st;
    }
    *ticket = r->next_ticket++;
    r->routed[*ticket] = Routed{best, inner, px};
    return GS_OK;
}

gs_status gs_router_wait(gs_router *r, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out,
                         int32_t *replica) {
    if (!r) return fail(GS_ERR_INVALID_ARG, "router is NULL");
    Routed rt;
    {
        std::lock_guard<std::mutex> lk(r->mu);
        auto it = r->routed.find(ticket);
        if (it == r->routed.end()) return fail(GS_ERR_INVALID_ARG, "unknown ticket");
        rt = it->second;
    }
    if (replica) *replica = rt.replica;
    gs_request_stats local;
    gs_request_stats *o = out ? out : &local;
    memset(o, 0, sizeof(*o));
    gs_status st = r->backend.wait(r->backend.user, rt.replica, rt.ticket, timeout_ms, o);
    // a wait that ran out leaves the request outstanding (no completion time): the ticket stays
    // valid; a request that completed with a device timeout has one
    if (st == GS_ERR_DEVICE_TIMEOUT && o->done_s == 0.0) return st;
    std::lock_guard<std::mutex> lk(r->mu);
    r->routed.erase(ticket);
    r->out_pixels[rt.replica] -= rt.pixels;
    r->out_requests[rt.replica] -= 1;
    return st;
}

gs_status gs_router_outstanding(gs_router *r, int32_t replica, int64_t *requests, int64_t *pixels) {
    if (!r || replica < 0 || replica >= r->replicas) return fail(GS_ERR_INVALID_ARG, "router or replica invalid");
    std::lock_guard<std::mutex> lk(r->mu);
    if (requests) *requests = r->out_requests[replica];
    if (pixels) *pixels = r->out_pixels[replica];
    return GS_OK;
}

}  // extern "C"
