// gs_api.cu -- the C ABI (include/gs.h): contexts, device-resident scenes, per-frame state
// allocated once (Section 5.3.1 "we reduce the dynamic memory allocation"), the four stages and
// their CUDA-graph replay, statistics and debug copies.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <algorithm>
#include <atomic>

#include "gs_internal.cuh"

using namespace gs;

namespace {

thread_local std::string g_err;
std::atomic<unsigned> g_wait_limit{0};   // 0: kSpinLimit

}  // namespace

namespace gs {
void set_error_message(const char *msg) { g_err = msg ? msg : ""; }
unsigned wait_limit() {
    const unsigned v = g_wait_limit.load(std::memory_order_relaxed);
    return v ? v : kSpinLimit;
}
}  // namespace gs

namespace {

gs_status fail(gs_status code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
gs_status fail(gs_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

gs_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GS_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves aligned slices out of one device allocation.
constexpr size_t kHistBytes = 8 * 256 * sizeof(unsigned);   // the sort's [8][256] digit histograms
// The blend takes its tiles longest list first up to this many tiles (a 1080p frame has 8160);
// beyond, each SM works through so many tiles that the last ones no longer set the makespan,
// and the one-CTA ordering kernel would cost more than it saves (4K: 32400 tiles).
constexpr int kOrderMaxTiles = 16384;

struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        size_t o = align_up(off, 256);
        off = o + count * sizeof(T);
        return o;
    }
};

int ceil_log2(long long x) {
    int b = 0;
    while ((1ll << b) < x) ++b;
    return b;
}

Opts make_opts(const gs_render_opts *o) {
    gs_render_opts d;
    gs_default_opts(&d);
    if (!o) o = &d;
    Opts r;
    for (int i = 0; i < 3; ++i) r.bg[i] = o->bg[i];
    r.tau = o->tau;
    r.alpha_max = o->alpha_max;
    r.T_min = o->T_min;
    r.dilation = o->dilation;
    r.cap_3sigma = o->cap_3sigma;
    r.clamp_fov = o->clamp_fov;
    r.intersect = o->intersect;
    return r;
}

}  // namespace

struct gs_context {
    int device = 0;
    int sm_count = 0;
    FrameCounters *ctr = nullptr;     // counters of the stand-alone sort
    SortScratch sort{};
    void *sort_mem = nullptr;
};

int context_device(const gs_context *ctx);

struct gs_scene {
    gs_context *ctx = nullptr;
    int device = 0;                  // kept here so that destruction never reads the context
    long long P = 0;
    int sh_degree = 3;
    int activated = 1;
    int sh_half = 0;                 // SH stored as binary16 (fixed at creation)
    void *mem = nullptr;
    float4 *pos_opa = nullptr, *rs = nullptr;
    void *sh = nullptr;
};

struct gs_frame {
    gs_context *ctx = nullptr;
    int device = 0;                  // kept here so that destruction never reads the context
    long long max_g = 0, max_pairs = 0;
    int max_w = 0, max_h = 0;
    long long max_tiles = 0, max_chunks = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    Rec *recs = nullptr;
    unsigned long long *keys[2] = {nullptr, nullptr};
    unsigned *vals[2] = {nullptr, nullptr};
    unsigned *starts = nullptr;
    unsigned *torder = nullptr;      // blend order of the tiles
    unsigned long long *chunk_base = nullptr, *vis_base = nullptr, *chunk_base2 = nullptr;
    unsigned *chunk_hits = nullptr, *chunk_vis = nullptr, *chunk_hits2 = nullptr, *counts = nullptr;
    unsigned *dkey[2] = {nullptr, nullptr}, *dval[2] = {nullptr, nullptr};
    uint4 *big = nullptr, *mid = nullptr;
    int mode_used = 0;
    float4 *geo0 = nullptr, *geo1 = nullptr;
    int4 *geo2 = nullptr;
    SortScratch sort{};
    FrameCounters *ctr = nullptr;
    // state of the last call
    int W = 0, H = 0, tiles_x = 0, tiles_y = 0;
    int sorted_buf = 0, passes = 0;
    // graph replay
    int use_graph = 0;
    cudaGraphExec_t exec = nullptr;
    // stage timing
    int timing = 0, timed = 0, bwd_timed = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t evb[3] = {nullptr, nullptr, nullptr};   // backward: start, between the kernels, end
    // frame-owned outputs for gs_render_host (allocated on first use)
    void *out_mem = nullptr;
    gs_tuning tuning{1, 1, 0, {0, 0, 0, 0, 0}};
    int counting = 0;
    // camera and options of the last preprocess (used by the backward)
    Cam cam{};
    Opts opt{};
    const gs_scene *scene_used = nullptr;
    float *grad2d = nullptr;         // allocated on the first backward
    BatchDesc batch{};               // requests of the last preprocess
};

int context_device(const gs_context *ctx) { return ctx ? ctx->device : 0; }

extern "C" {

const char *gs_last_error(void) { return g_err.c_str(); }

int32_t gs_version(void) { return 100; }

gs_status gs_default_opts(gs_render_opts *o) {
    if (!o) return fail(GS_ERR_INVALID_ARG, "opts is NULL");
    o->bg[0] = o->bg[1] = o->bg[2] = 0.0f;
    o->tau = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->T_min = 1e-4f;
    o->dilation = 0.3f;
    o->cap_3sigma = 0;
    o->clamp_fov = 1;
    o->intersect = 0;
    return GS_OK;
}

gs_status gs_context_create(int32_t device, gs_context **out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return fail(GS_ERR_NO_DEVICE, "no CUDA device");
    }
    if (device < 0 || device >= n) return fail(GS_ERR_INVALID_ARG, "device %d out of range [0,%d)", device, n);
    GS_CUDA(cudaSetDevice(device));
    gs_context *c = new (std::nothrow) gs_context();
    if (!c) return fail(GS_ERR_OOM, "host allocation failed");
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->ctr, sizeof(FrameCounters));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaMalloc(counters)");
    }
    cudaMemset(c->ctr, 0, sizeof(FrameCounters));
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(c->ctr);
        delete c;
        return cuda_fail(e, "context init");
    }
    *out = c;
    return GS_OK;
}

gs_status gs_context_destroy(gs_context *c) {
    if (!c) return GS_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->ctr);
    cudaFree(c->sort_mem);
    cudaGetLastError();
    delete c;
    return GS_OK;
}

// ------------------------------------------------------------------------------------------ scenes
static gs_status check_gaussians(const gs_gaussians *g) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->P <= 0 || g->P >= (1ll << 31)) return fail(GS_ERR_INVALID_ARG, "P = %lld out of range", (long long)g->P);
    if (!g->means || !g->scales || !g->quats || !g->opacity || !g->sh)
        return fail(GS_ERR_INVALID_ARG, "a Gaussian array pointer is NULL");
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(GS_ERR_INVALID_ARG, "sh_degree %d not in 0..3", g->sh_degree);
    if (g->sh_half != 0 && g->sh_half != 1) return fail(GS_ERR_INVALID_ARG, "sh_half %d not 0 or 1", g->sh_half);
    return GS_OK;
}

gs_status gs_scene_create(gs_context *ctx, const gs_gaussians *g, gs_stream stream, gs_scene **out) {
    if (!ctx || !out) return fail(GS_ERR_INVALID_ARG, "NULL context or out");
    *out = nullptr;
    gs_status st = check_gaussians(g);
    if (st) return st;
    GS_CUDA(cudaSetDevice(ctx->device));
    gs_scene *s = new (std::nothrow) gs_scene();
    if (!s) return fail(GS_ERR_OOM, "host allocation failed");
    s->ctx = ctx;
    s->device = ctx->device;
    s->P = g->P;
    s->sh_half = g->sh_half;
    // SH blocks first (256-byte aligned by cudaMalloc, so every 192-byte block starts on a
    // 64-byte boundary, every 96-byte binary16 block on a 32-byte one), then scale/rotation, then
    // positions
    const size_t sh_f4 = (size_t)(g->sh_half ? kShPlanes / 2 : kShPlanes) * (size_t)g->P;   // in float4 units
    cudaError_t e = cudaMalloc(&s->mem, (sh_f4 + 3 * (size_t)g->P) * sizeof(float4));
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaMalloc(scene)");
    }
    float4 *base = (float4 *)s->mem;
    s->sh = base;
    s->rs = base + sh_f4;
    s->pos_opa = base + sh_f4 + 2 * (size_t)g->P;
    st = gs_scene_update(s, g, stream);
    if (st) {
        cudaFree(s->mem);
        delete s;
        return st;
    }
    *out = s;
    return GS_OK;
}

gs_status gs_scene_update(gs_scene *s, const gs_gaussians *g, gs_stream stream) {
    if (!s) return fail(GS_ERR_INVALID_ARG, "scene is NULL");
    gs_status st = check_gaussians(g);
    if (st) return st;
    if (g->P != s->P) return fail(GS_ERR_INVALID_ARG, "P changed (%lld != %lld)", (long long)g->P, s->P);
    if (g->sh_half != s->sh_half) return fail(GS_ERR_INVALID_ARG, "sh_half differs from the scene's creation");
    s->sh_degree = g->sh_degree;
    s->activated = g->activated ? 1 : 0;
    launch_pack_scene(*g, s->pos_opa, s->rs, s->sh, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status gs_scene_destroy(gs_scene *s) {
    if (!s) return GS_OK;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    cudaFree(s->mem);
    cudaGetLastError();   // leave no error behind for unrelated later calls
    delete s;
    return GS_OK;
}

int64_t gs_scene_size(const gs_scene *s) { return s ? s->P : 0; }

// ------------------------------------------------------------------------------------------ frames
gs_status gs_frame_create(gs_context *ctx, int64_t max_g, int64_t max_pairs, int32_t max_w, int32_t max_h,
                          gs_frame **out) {
    if (!ctx || !out) return fail(GS_ERR_INVALID_ARG, "NULL context or out");
    *out = nullptr;
    if (max_g <= 0 || max_g >= (1ll << 31)) return fail(GS_ERR_INVALID_ARG, "max_gaussians out of range");
    if (max_pairs <= 0 || max_pairs >= (1ll << 30)) return fail(GS_ERR_INVALID_ARG, "max_pairs must be in (0, 2^30)");
    if (max_w <= 0 || max_h <= 0 || max_w > 65536 || max_h > 65536) return fail(GS_ERR_INVALID_ARG, "bad image size");
    long long tiles = (long long)((max_w + kTile - 1) / kTile) * ((max_h + kTile - 1) / kTile);
    if (tiles >= (1ll << 31)) return fail(GS_ERR_INVALID_ARG, "too many tiles");
    GS_CUDA(cudaSetDevice(ctx->device));
    gs_frame *f = new (std::nothrow) gs_frame();
    if (!f) return fail(GS_ERR_OOM, "host allocation failed");
    f->ctx = ctx;
    f->device = ctx->device;
    f->max_g = max_g;
    f->max_pairs = max_pairs;
    f->max_w = max_w;
    f->max_h = max_h;
    f->max_tiles = tiles;
    f->max_chunks = (max_g + preprocess_chunk() - 1) / preprocess_chunk();
    f->sort.max_tiles = sort_max_tiles_for(max_pairs > max_g ? max_pairs : max_g);
    Carver cv;
    size_t o_recs = cv.take<Rec>(max_g);
    size_t o_k0 = cv.take<unsigned long long>(max_pairs), o_k1 = cv.take<unsigned long long>(max_pairs);
    size_t o_v0 = cv.take<unsigned>(max_pairs), o_v1 = cv.take<unsigned>(max_pairs);
    size_t o_starts = cv.take<unsigned>(tiles + 1);
    size_t o_torder = cv.take<unsigned>(tiles);
    size_t o_cbase = cv.take<unsigned long long>(f->max_chunks);
    size_t o_chits = cv.take<unsigned>(f->max_chunks);
    size_t o_vbase = cv.take<unsigned long long>(f->max_chunks), o_cbase2 = cv.take<unsigned long long>(f->max_chunks);
    size_t o_cvis = cv.take<unsigned>(f->max_chunks), o_chits2 = cv.take<unsigned>(f->max_chunks);
    size_t o_counts = cv.take<unsigned>(max_g);
    size_t o_dk0 = cv.take<unsigned>(max_g), o_dk1 = cv.take<unsigned>(max_g);
    size_t o_dv0 = cv.take<unsigned>(max_g), o_dv1 = cv.take<unsigned>(max_g);
    size_t o_big = cv.take<uint4>(max_g), o_mid = cv.take<uint4>(max_g);
    size_t o_geo0 = cv.take<float4>(max_g), o_geo1 = cv.take<float4>(max_g), o_geo2 = cv.take<int4>(max_g);
    size_t o_offs = cv.take<unsigned>(8 * 256);
    size_t o_desc = cv.take<unsigned long long>(sort_desc_words(f->sort.max_tiles));
    size_t o_rts = cv.take<unsigned>(rts_stride(f->sort.max_tiles) * 256);
    // the digit histograms sit right before the counters: one memset clears both every frame
    size_t o_hist = cv.take<unsigned char>(kHistBytes);
    size_t o_ctr = cv.take<FrameCounters>(1);
    static_assert(kHistBytes % 256 == 0, "the counters follow the histograms with no alignment gap");
    f->bytes = align_up(cv.off, 256);
    cudaError_t e = cudaMalloc(&f->mem, f->bytes);
    if (e != cudaSuccess) {
        delete f;
        cudaGetLastError();
        return fail(GS_ERR_OOM, "cudaMalloc(frame, %zu bytes): %s", f->bytes, cudaGetErrorString(e));
    }
    char *b = (char *)f->mem;
    f->recs = (Rec *)(b + o_recs);
    f->keys[0] = (unsigned long long *)(b + o_k0);
    f->keys[1] = (unsigned long long *)(b + o_k1);
    f->vals[0] = (unsigned *)(b + o_v0);
    f->vals[1] = (unsigned *)(b + o_v1);
    f->starts = (unsigned *)(b + o_starts);
    f->torder = (unsigned *)(b + o_torder);
    f->chunk_base = (unsigned long long *)(b + o_cbase);
    f->chunk_hits = (unsigned *)(b + o_chits);
    f->vis_base = (unsigned long long *)(b + o_vbase);
    f->chunk_base2 = (unsigned long long *)(b + o_cbase2);
    f->chunk_vis = (unsigned *)(b + o_cvis);
    f->chunk_hits2 = (unsigned *)(b + o_chits2);
    f->counts = (unsigned *)(b + o_counts);
    f->dkey[0] = (unsigned *)(b + o_dk0);
    f->dkey[1] = (unsigned *)(b + o_dk1);
    f->dval[0] = (unsigned *)(b + o_dv0);
    f->dval[1] = (unsigned *)(b + o_dv1);
    f->big = (uint4 *)(b + o_big);
    f->mid = (uint4 *)(b + o_mid);
    f->geo0 = (float4 *)(b + o_geo0);
    f->geo1 = (float4 *)(b + o_geo1);
    f->geo2 = (int4 *)(b + o_geo2);
    f->sort.hist = (unsigned *)(b + o_hist);
    f->sort.offs = (unsigned *)(b + o_offs);
    f->sort.desc = (unsigned long long *)(b + o_desc);
    f->sort.counts = (unsigned *)(b + o_rts);
    f->ctr = (FrameCounters *)(b + o_ctr);
    // zero scratch that must start cleared (histograms, descriptors, counters, tile starts)
    cudaMemset(b + o_starts, 0, f->bytes - o_starts);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(f->mem);
        delete f;
        return cuda_fail(e, "frame init");
    }
    *out = f;
    return GS_OK;
}

gs_status gs_frame_destroy(gs_frame *f) {
    if (!f) return GS_OK;
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    if (f->exec) cudaGraphExecDestroy(f->exec);
    for (int i = 0; i < 5; ++i)
        if (f->ev[i]) cudaEventDestroy(f->ev[i]);
    for (int i = 0; i < 3; ++i)
        if (f->evb[i]) cudaEventDestroy(f->evb[i]);
    cudaFree(f->out_mem);
    cudaFree(f->grad2d);
    cudaFree(f->mem);
    cudaGetLastError();
    delete f;
    return GS_OK;
}

int64_t gs_frame_bytes(const gs_frame *f) { return f ? (int64_t)f->bytes : 0; }

gs_status gs_frame_use_graph(gs_frame *f, int32_t enable) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    f->use_graph = enable ? 1 : 0;
    return GS_OK;
}

gs_status gs_frame_set_tuning(gs_frame *f, const gs_tuning *t) {
    if (!f || !t) return fail(GS_ERR_INVALID_ARG, "NULL frame or tuning");
    if (t->blend_variant < 0 || t->blend_variant >= blend_variant_count())
        return fail(GS_ERR_INVALID_ARG, "blend_variant %d out of range", t->blend_variant);
    if (t->sort_mode < 0 || t->sort_mode > 1) return fail(GS_ERR_INVALID_ARG, "sort_mode %d not 0 or 1", t->sort_mode);
    if (t->sort_algo < 0 || t->sort_algo > 2) return fail(GS_ERR_INVALID_ARG, "sort_algo %d not 0, 1 or 2", t->sort_algo);
    if ((t->blend_variant != f->tuning.blend_variant || t->sort_mode != f->tuning.sort_mode ||
         t->sort_algo != f->tuning.sort_algo) &&
        f->exec) {
        cudaGraphExecDestroy(f->exec);
        f->exec = nullptr;
    }
    f->tuning = *t;
    f->sort.algo = t->sort_algo;
    return GS_OK;
}

gs_status gs_frame_set_counting(gs_frame *f, int32_t enable) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    if (f->counting != (enable ? 1 : 0) && f->exec) {
        cudaGraphExecDestroy(f->exec);
        f->exec = nullptr;
    }
    f->counting = enable ? 1 : 0;
    return GS_OK;
}

gs_status gs_frame_get_tuning(const gs_frame *f, gs_tuning *t) {
    if (!f || !t) return fail(GS_ERR_INVALID_ARG, "NULL frame or tuning");
    *t = f->tuning;
    return GS_OK;
}

gs_status gs_frame_enable_timing(gs_frame *f, int32_t enable) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    if (enable && !f->ev[0]) {
        GS_CUDA(cudaSetDevice(f->device));
        for (int i = 0; i < 5; ++i) GS_CUDA(cudaEventCreate(&f->ev[i]));
        for (int i = 0; i < 3; ++i) GS_CUDA(cudaEventCreate(&f->evb[i]));
    }
    if (f->timing != (enable ? 1 : 0) && f->exec) {   // topology changes: re-instantiate the graph
        cudaGraphExecDestroy(f->exec);
        f->exec = nullptr;
    }
    f->timing = enable ? 1 : 0;
    f->timed = 0;
    f->bwd_timed = 0;
    return GS_OK;
}

gs_status gs_frame_backward_ms(gs_frame *f, float ms[2]) {
    if (!f || !ms) return fail(GS_ERR_INVALID_ARG, "NULL frame or ms");
    if (!f->timing || !f->bwd_timed) return fail(GS_ERR_INVALID_ARG, "no timed backward on this frame");
    GS_CUDA(cudaEventSynchronize(f->evb[2]));
    for (int i = 0; i < 2; ++i) GS_CUDA(cudaEventElapsedTime(&ms[i], f->evb[i], f->evb[i + 1]));
    return GS_OK;
}

gs_status gs_frame_stage_ms(gs_frame *f, float ms[4]) {
    if (!f || !ms) return fail(GS_ERR_INVALID_ARG, "NULL frame or ms");
    if (!f->timing || !f->timed) return fail(GS_ERR_INVALID_ARG, "no timed render on this frame");
    GS_CUDA(cudaEventSynchronize(f->ev[4]));
    for (int i = 0; i < 4; ++i) GS_CUDA(cudaEventElapsedTime(&ms[i], f->ev[i], f->ev[i + 1]));
    return GS_OK;
}

// ------------------------------------------------------------------------------------------ stages
}  // extern "C"

// ------------------------------------------------------------------------------------------ batches
static gs_status make_cam(const gs_camera *cam, Cam &c) {
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 || cam->height > 65535)
        return fail(GS_ERR_INVALID_ARG, "bad image size %dx%d", cam->width, cam->height);
    if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f)) return fail(GS_ERR_INVALID_ARG, "focal lengths must be positive");
    for (int i = 0; i < 9; ++i) c.R[i] = cam->R[i];
    for (int i = 0; i < 3; ++i) c.t[i] = cam->t[i];
    c.fx = cam->fx;
    c.fy = cam->fy;
    c.cx = cam->cx;
    c.cy = cam->cy;
    c.near_z = cam->near_z;
    c.W = cam->width;
    c.H = cam->height;
    c.tiles_x = (cam->width + kTile - 1) / kTile;
    c.tiles_y = (cam->height + kTile - 1) / kTile;
    // clamp bounds, binary32 as in the Jacobian definition: 1.3 * ((W/2) / fx)
    volatile float hw = 0.5f * (float)cam->width, hh = 0.5f * (float)cam->height;
    volatile float qx = hw / cam->fx, qy = hh / cam->fy;
    c.limx = 1.3f * qx;
    c.limy = 1.3f * qy;
    for (int i = 0; i < 3; ++i)
        c.campos[i] = -(cam->R[i] * cam->t[0] + cam->R[3 + i] * cam->t[1] + cam->R[6 + i] * cam->t[2]);
    return GS_OK;
}

static SceneView view_of(const gs_scene *s) {
    SceneView v;
    v.pos_opa = s->pos_opa;
    v.rs = s->rs;
    v.sh = s->sh;
    v.P = s->P;
    v.sh_degree = s->sh_degree;
    v.activated = s->activated;
    v.sh_half = s->sh_half;
    return v;
}

// Builds the descriptor of n requests into f->batch after checking the frame's capacities.
static gs_status make_batch(gs_frame *f, int n, const gs_scene *const *scenes, const gs_camera *cams,
                            const gs_render_opts *opts) {
    if (n < 1 || n > kMaxBatch) return fail(GS_ERR_INVALID_ARG, "batch of %d requests (1..%d)", n, kMaxBatch);
    BatchDesc &B = f->batch;
    B.n = n;
    long long chunks = 0, recs = 0;
    long long tiles = 0;
    for (int r = 0; r < n; ++r) {
        if (!scenes[r]) return fail(GS_ERR_INVALID_ARG, "scene %d is NULL", r);
        ReqDesc &R = B.r[r];
        gs_status st = make_cam(&cams[r], R.cam);
        if (st) return st;
        R.opt = make_opts(opts ? &opts[r] : nullptr);
        R.scene = view_of(scenes[r]);
        R.chunk0 = chunks;
        R.rec0 = recs;
        R.tile0 = (int)tiles;
        R.rgb = nullptr;
        R.T = nullptr;
        R.last = nullptr;
        chunks += (scenes[r]->P + preprocess_chunk() - 1) / preprocess_chunk();
        recs += scenes[r]->P;
        tiles += (long long)R.cam.tiles_x * R.cam.tiles_y;
    }
    if (recs > f->max_g)
        return fail(GS_ERR_CAPACITY, "batch has %lld Gaussians, the frame holds %lld", recs, f->max_g);
    if (tiles > f->max_tiles) return fail(GS_ERR_CAPACITY, "batch has %lld tiles, the frame holds %lld", tiles, f->max_tiles);
    B.total_chunks = chunks;
    B.total_recs = recs;
    B.total_tiles = (int)tiles;
    return GS_OK;
}

static PreprocessArgs pre_args(gs_frame *f) {
    PreprocessArgs a;
    a.B = f->batch;
    a.recs = f->recs;
    a.keys = f->keys[0];
    a.vals = f->vals[0];
    a.geo0 = f->geo0;
    a.geo1 = f->geo1;
    a.geo2 = f->geo2;
    a.chunk_hits = f->chunk_hits;
    a.chunk_base = f->chunk_base;
    a.counts = f->counts;
    a.tkeys = (unsigned *)f->keys[0];
    a.chunk_vis = f->chunk_vis;
    a.vis_base = f->vis_base;
    a.dkey = f->dkey[0];
    a.dval = f->dval[0];
    a.dkey_tmp = f->dkey[1];
    a.dval_tmp = f->dval[1];
    a.dsorted = f->dval[0];
    a.chunk_hits2 = f->chunk_hits2;
    a.chunk_base2 = f->chunk_base2;
    a.big = f->big;
    a.mid = f->mid;
    // the sort's second key buffer is free until the sort: the count pass keeps its masks there
    a.masks = (unsigned char *)f->keys[1];
    a.mask_cap = std::min<long long>(8ll * f->max_pairs, 0xfffffffell);
    a.ctr = f->ctr;
    a.pair_cap = f->max_pairs;
    a.n_chunks = f->batch.total_chunks;
    return a;
}

// First half of the preprocess of f->batch: geometry and exact pair counts (k_pre_count).
// Clears the per-frame counters and the digit histograms (adjacent in the frame); the sort epoch
// and what follows it persist across frames.
static gs_status clear_frame_counters(gs_frame *f, cudaStream_t st) {
    GS_CUDA(cudaMemsetAsync(f->sort.hist, 0, kHistBytes + offsetof(FrameCounters, sort_epoch), st));
    return GS_OK;
}

static gs_status batch_count(gs_frame *f, cudaStream_t st) {
    if (gs_status r = clear_frame_counters(f, st)) return r;
    launch_pre_count(pre_args(f), st);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

// Second half: scan, (depth order,) and emission.  `counted`: batch_count already ran.
static gs_status batch_emit(gs_frame *f, cudaStream_t st, bool counted) {
    if (!counted)
        if (gs_status r = clear_frame_counters(f, st)) return r;
    f->mode_used = f->tuning.sort_mode;
    const PreprocessArgs a = pre_args(f);
    if (f->mode_used == 1)
        launch_preprocess_depth(a, f->sort, st, counted);
    else
        launch_preprocess(a, st, counted);
    GS_CUDA(cudaGetLastError());
    const ReqDesc &R0 = f->batch.r[0];
    f->W = R0.cam.W;
    f->H = R0.cam.H;
    f->tiles_x = R0.cam.tiles_x;
    f->tiles_y = R0.cam.tiles_y;
    f->sorted_buf = 0;
    f->cam = R0.cam;
    f->opt = R0.opt;
    return GS_OK;
}

gs_status frame_batch_count(gs_frame *f, int n, const gs_scene *const *scenes, const gs_camera *cams,
                            const gs_render_opts *opts, unsigned long long *req_pairs_dev, gs_stream stream) {
    gs_status st = make_batch(f, n, scenes, cams, opts);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    if ((st = batch_count(f, cs))) return st;
    launch_req_pairs(pre_args(f), req_pairs_dev, cs);
    GS_CUDA(cudaGetLastError());
    f->scene_used = n == 1 ? scenes[0] : nullptr;
    return GS_OK;
}

extern "C" {

gs_status gs_preprocess(gs_frame *f, const gs_scene *s, const gs_camera *cam, const gs_render_opts *opts,
                        gs_stream stream) {
    if (!f || !s || !cam) return fail(GS_ERR_INVALID_ARG, "NULL frame, scene or camera");
    if (s->P > f->max_g) return fail(GS_ERR_INVALID_ARG, "scene has %lld Gaussians, frame holds %lld", s->P, f->max_g);
    if (cam->width <= 0 || cam->height <= 0 || cam->width > f->max_w || cam->height > f->max_h)
        return fail(GS_ERR_INVALID_ARG, "image %dx%d outside the frame's %dx%d", cam->width, cam->height, f->max_w,
                    f->max_h);
    gs_status st = make_batch(f, 1, &s, cam, opts);
    if (st) return st == GS_ERR_CAPACITY ? GS_ERR_INVALID_ARG : st;
    if ((st = batch_emit(f, (cudaStream_t)stream, false))) return st;
    f->scene_used = s;
    return GS_OK;
}

gs_status gs_sort(gs_frame *f, gs_stream stream) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    if (f->W <= 0) return fail(GS_ERR_INVALID_ARG, "gs_sort before gs_preprocess");
    const int tile_bits = ceil_log2((long long)f->batch.total_tiles);
    if (f->mode_used == 1) {
        f->passes = launch_sort32((unsigned *)f->keys[0], f->vals[0], (unsigned *)f->keys[1], f->vals[1],
                                  &f->ctr->n_pairs, f->max_pairs, tile_bits > 0 ? tile_bits : 1, f->sort, f->ctr,
                                  (cudaStream_t)stream);
    } else {
        f->passes = launch_sort(f->keys[0], f->vals[0], f->keys[1], f->vals[1], &f->ctr->n_pairs, 0, f->max_pairs,
                                32 + tile_bits, f->sort, f->ctr, (cudaStream_t)stream);
    }
    GS_CUDA(cudaGetLastError());
    f->sorted_buf = f->passes & 1;
    return GS_OK;
}

gs_status gs_ranges(gs_frame *f, gs_stream stream) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    if (f->W <= 0) return fail(GS_ERR_INVALID_ARG, "gs_ranges before gs_preprocess");
    if (f->mode_used == 1)
        launch_ranges32((const unsigned *)f->keys[f->sorted_buf], &f->ctr->n_pairs, f->max_pairs,
                        f->batch.total_tiles, f->starts, f->ctr, (cudaStream_t)stream);
    else
        launch_ranges(f->keys[f->sorted_buf], &f->ctr->n_pairs, f->max_pairs, f->batch.total_tiles, f->starts,
                      f->ctr, (cudaStream_t)stream);
    if (f->batch.total_tiles <= kOrderMaxTiles)
        launch_tile_order(f->starts, f->batch.total_tiles, f->torder, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

static gs_status blend_batch(gs_frame *f, float *const *rgb, float *const *T, uint32_t *const *last,
                             const gs_render_opts *opts_override, gs_stream stream) {
    BlendArgs a;
    a.B = f->batch;
    a.ctr = f->ctr;
    for (int r = 0; r < a.B.n; ++r) {
        if (!rgb[r]) return fail(GS_ERR_INVALID_ARG, "rgb output %d is NULL", r);
        a.B.r[r].rgb = rgb[r];
        a.B.r[r].T = T ? T[r] : nullptr;
        a.B.r[r].last = last ? (unsigned *)last[r] : nullptr;
        if (opts_override) a.B.r[r].opt = make_opts(opts_override);
    }
    a.recs = f->recs;
    a.vals = f->vals[f->sorted_buf];
    a.starts = f->starts;
    a.order = f->batch.total_tiles <= kOrderMaxTiles ? f->torder : nullptr;
    a.n_dev = &f->ctr->n_pairs;
    a.cap = f->max_pairs;
    a.evals = f->ctr->evals;
    a.variant = f->tuning.blend_variant;
    a.count = f->counting;
    if (f->counting) GS_CUDA(cudaMemsetAsync(f->ctr->evals, 0, sizeof(f->ctr->evals), (cudaStream_t)stream));
    launch_blend(a, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status gs_blend(gs_frame *f, const gs_render_opts *opts, float *rgb, float *T, uint32_t *last,
                   gs_stream stream) {
    if (!f || !rgb) return fail(GS_ERR_INVALID_ARG, "NULL frame or rgb");
    if (f->W <= 0) return fail(GS_ERR_INVALID_ARG, "gs_blend before gs_preprocess");
    if (f->batch.n != 1) return fail(GS_ERR_INVALID_ARG, "the frame holds a batch: use gs_render_batch");
    gs_render_opts o;
    if (!opts) gs_default_opts(&o);
    return blend_batch(f, &rgb, &T, &last, opts ? opts : &o, stream);
}

// Records stage event i; inside a stream capture the record must become an event node of the
// graph (cudaEventRecordExternal), otherwise the event is only a capture dependency.
static gs_status record_stage(gs_frame *f, int i, cudaStream_t cs) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GS_CUDA(cudaStreamIsCapturing(cs, &cap));
    if (cap == cudaStreamCaptureStatusActive)
        GS_CUDA(cudaEventRecordWithFlags(f->ev[i], cs, cudaEventRecordExternal));
    else
        GS_CUDA(cudaEventRecord(f->ev[i], cs));
    return GS_OK;
}

static gs_status enqueue_all(gs_frame *f, const gs_scene *s, const gs_camera *cam, const gs_render_opts *opts,
                             float *rgb, float *T, uint32_t *last, gs_stream stream) {
    cudaStream_t cs = (cudaStream_t)stream;
    const bool tm = f->timing != 0;
    gs_status st;
    if (tm && (st = record_stage(f, 0, cs))) return st;
    if ((st = gs_preprocess(f, s, cam, opts, stream))) return st;
    if (tm && (st = record_stage(f, 1, cs))) return st;
    if ((st = gs_sort(f, stream))) return st;
    if (tm && (st = record_stage(f, 2, cs))) return st;
    if ((st = gs_ranges(f, stream))) return st;
    if (tm && (st = record_stage(f, 3, cs))) return st;
    if ((st = gs_blend(f, opts, rgb, T, last, stream))) return st;
    if (tm) {
        if ((st = record_stage(f, 4, cs))) return st;
        f->timed = 1;
    }
    return GS_OK;
}

gs_status gs_render(gs_frame *f, const gs_scene *s, const gs_camera *cam, const gs_render_opts *opts, float *rgb,
                    float *T, uint32_t *last, gs_stream stream) {
    if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
    if (!f->use_graph) return enqueue_all(f, s, cam, opts, rgb, T, last, stream);
    if (!stream) return fail(GS_ERR_INVALID_ARG, "graph replay needs a non-default stream");
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gs_status r = enqueue_all(f, s, cam, opts, rgb, T, last, stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if (f->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(f->exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(f->exec);
            f->exec = nullptr;
        }
    }
    if (!f->exec) {
        e = cudaGraphInstantiate(&f->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            f->exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(g);
    GS_CUDA(cudaGraphLaunch(f->exec, st));
    return GS_OK;
}

gs_status gs_frame_get_stats(gs_frame *f, gs_frame_stats *out, gs_stream stream) {
    if (!f || !out) return fail(GS_ERR_INVALID_ARG, "NULL frame or out");
    GS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    FrameCounters c;
    GS_CUDA(cudaMemcpy(&c, f->ctr, sizeof(c), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->pairs = (int64_t)c.n_pairs;
    out->visible = c.n_visible;
    out->pair_capacity = f->max_pairs;
    out->status = (c.status & kStTimeout) ? GS_ERR_DEVICE_TIMEOUT
                  : (c.status & kStPairOverflow) ? GS_ERR_PAIR_OVERFLOW
                                                 : GS_OK;
    out->width = f->W;
    out->height = f->H;
    out->tiles_x = f->tiles_x;
    out->tiles_y = f->tiles_y;
    out->sort_passes = f->passes;
    out->culled_in = c.n_culled_in;
    out->evaluations = (int64_t)c.evals[0];
    out->contributions = (int64_t)c.evals[1];
    // count + scan + emit, sort, ranges, blend; the depth-ordered mode adds the visible-list
    // compaction, the 4-pass depth sort, the rank-chunk sums and scan and the medium- and
    // large-Gaussian emission.  A sort runs histogram + offsets + one scatter per pass (onesweep),
    // count + scan + scatter per pass (reduce-then-scan) or one fused launch (two passes or more).
    const int algo = f->tuning.sort_algo;
    const int sort_k = algo == 1 ? 3 * f->passes : algo == 2 && f->passes >= 2 ? 1 : 2 + f->passes;
    const int depth_k = 1;   // the depth sort always runs fused
    const int ranges_k = f->batch.total_tiles <= kOrderMaxTiles ? 2 : 1;   // starts (+ blend order)
    out->kernels = f->mode_used == 1 ? 3 + 5 + depth_k + sort_k + ranges_k + 1 : 3 + sort_k + ranges_k + 1;
    return GS_OK;
}

gs_status gs_render_host(gs_frame *f, const gs_scene *s, const gs_camera *cam, const gs_render_opts *opts,
                         float *rgb_host, float *T_host, uint32_t *last_host, gs_stream stream) {
    if (!f || !cam || !rgb_host) return fail(GS_ERR_INVALID_ARG, "NULL frame, camera or rgb_host");
    const size_t npx = (size_t)f->max_w * (size_t)f->max_h;
    if (!f->out_mem) {
        GS_CUDA(cudaSetDevice(f->device));
        GS_CUDA(cudaMalloc(&f->out_mem, npx * 5 * sizeof(float)));
    }
    float *rgb = (float *)f->out_mem;
    float *T = rgb + 3 * npx;
    uint32_t *last = (uint32_t *)(T + npx);
    gs_status st = gs_render(f, s, cam, opts, rgb, T_host ? T : nullptr, last_host ? last : nullptr, stream);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t n = (size_t)cam->width * (size_t)cam->height;
    GS_CUDA(cudaMemcpyAsync(rgb_host, rgb, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, cs));
    if (T_host) GS_CUDA(cudaMemcpyAsync(T_host, T, n * sizeof(float), cudaMemcpyDeviceToHost, cs));
    if (last_host) GS_CUDA(cudaMemcpyAsync(last_host, last, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, cs));
    return GS_OK;
}

gs_status gs_frame_pairs(gs_frame *f, int32_t which, uint64_t *keys, uint32_t *vals, int64_t cap, int64_t *n_out,
                         gs_stream stream) {
    if (!f || !n_out) return fail(GS_ERR_INVALID_ARG, "NULL frame or n_out");
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA(cudaStreamSynchronize(st));
    unsigned long long n = 0;
    GS_CUDA(cudaMemcpy(&n, &f->ctr->n_pairs, sizeof(n), cudaMemcpyDeviceToHost));
    long long m = (long long)n;
    if (m > f->max_pairs) m = f->max_pairs;
    if (m > cap) m = cap;
    const int b = which ? f->sorted_buf : 0;
    if (m > 0) {
        if (keys) {
            if (f->mode_used == 1)   // rebuild (tile << 32 | depth bits) from the 32-bit tile keys
                launch_make_keys((const unsigned *)f->keys[b], f->vals[b], f->geo1, m, (unsigned long long *)keys,
                                 f->ctr, st);
            else
                GS_CUDA(cudaMemcpyAsync(keys, f->keys[b], (size_t)m * 8, cudaMemcpyDeviceToDevice, st));
            GS_CUDA(cudaGetLastError());
        }
        if (vals) GS_CUDA(cudaMemcpyAsync(vals, f->vals[b], (size_t)m * 4, cudaMemcpyDeviceToDevice, st));
    }
    GS_CUDA(cudaStreamSynchronize(st));
    *n_out = m;
    return GS_OK;
}

gs_status gs_frame_ranges(gs_frame *f, uint32_t *starts, int64_t cap, gs_stream stream) {
    if (!f || !starts) return fail(GS_ERR_INVALID_ARG, "NULL frame or starts");
    const long long n = (long long)f->tiles_x * f->tiles_y + 1;
    if (cap < n) return fail(GS_ERR_CAPACITY, "need %lld entries", n);
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA(cudaMemcpyAsync(starts, f->starts, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_sort_pairs(gs_context *ctx, uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                        int64_t n, int32_t end_bit, int32_t *in_tmp, gs_stream stream) {
    if (!ctx || !in_tmp) return fail(GS_ERR_INVALID_ARG, "NULL context or in_tmp");
    if (n < 0 || n >= (1ll << 30)) return fail(GS_ERR_INVALID_ARG, "n = %lld out of range", (long long)n);
    if (end_bit < 1 || end_bit > 64) return fail(GS_ERR_INVALID_ARG, "end_bit %d not in 1..64", end_bit);
    if (n > 0 && (!keys || !vals || !keys_tmp || !vals_tmp)) return fail(GS_ERR_INVALID_ARG, "NULL buffer");
    GS_CUDA(cudaSetDevice(ctx->device));
    const long long tiles = sort_max_tiles_for(n > 0 ? n : 1);
    if (tiles > ctx->sort.max_tiles) {
        GS_CUDA(cudaDeviceSynchronize());
        cudaFree(ctx->sort_mem);
        ctx->sort_mem = nullptr;
        ctx->sort.max_tiles = 0;
        Carver cv;
        size_t oh = cv.take<unsigned>(8 * 256), oo = cv.take<unsigned>(8 * 256);
        size_t od = cv.take<unsigned long long>(sort_desc_words(tiles));
        GS_CUDA(cudaMalloc(&ctx->sort_mem, cv.off));
        GS_CUDA(cudaMemset(ctx->sort_mem, 0, cv.off));
        char *b = (char *)ctx->sort_mem;
        ctx->sort.hist = (unsigned *)(b + oh);
        ctx->sort.offs = (unsigned *)(b + oo);
        ctx->sort.desc = (unsigned long long *)(b + od);
        ctx->sort.max_tiles = tiles;
    }
    // a timeout reported by an earlier sort on this context must not stop this one
    GS_CUDA(cudaMemsetAsync(&ctx->ctr->status, 0, sizeof(unsigned), (cudaStream_t)stream));
    const int passes = launch_sort((unsigned long long *)keys, vals, (unsigned long long *)keys_tmp, vals_tmp, nullptr,
                                   n, n, end_bit, ctx->sort, ctx->ctr, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    *in_tmp = passes & 1;
    return GS_OK;
}

gs_status gs_sort_pairs_status(gs_context *ctx, gs_stream stream) {
    if (!ctx) return fail(GS_ERR_INVALID_ARG, "context is NULL");
    GS_CUDA(cudaSetDevice(ctx->device));
    GS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned status = 0;
    GS_CUDA(cudaMemcpy(&status, &ctx->ctr->status, sizeof(status), cudaMemcpyDeviceToHost));
    if (status & kStTimeout)
        return fail(GS_ERR_DEVICE_TIMEOUT, "a bounded wait of the last gs_sort_pairs gave up: its output is invalid");
    return GS_OK;
}

gs_status gs_set_wait_limit(uint32_t polls) {
    g_wait_limit.store(polls, std::memory_order_relaxed);
    return GS_OK;
}

uint32_t gs_get_wait_limit(void) { return wait_limit(); }

}  // extern "C"

// ------------------------------------------------------------------------------------------ batch API
extern "C" gs_status gs_render_batch(gs_frame *f, int32_t n, const gs_scene *const *scenes, const gs_camera *cams,
                                     const gs_render_opts *opts, float *const *rgb, float *const *T,
                                     uint32_t *const *last, gs_stream stream) {
    if (!f || !scenes || !cams || !rgb) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status st = make_batch(f, n, scenes, cams, opts);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    if ((st = batch_emit(f, cs, false))) return st;
    f->scene_used = n == 1 ? scenes[0] : nullptr;
    if ((st = gs_sort(f, stream))) return st;
    if ((st = gs_ranges(f, stream))) return st;
    return blend_batch(f, rgb, T, last, nullptr, stream);
}

// Server path: finish a batch whose counts are already on the device (frame_batch_count).
// Enqueues a copy of the frame's device counters (status word, pair count) to page-locked host
// memory, so that a completion callback can judge the batch without a synchronising read.
gs_status frame_counters_async(gs_frame *f, void *host_dst, gs_stream stream) {
    GS_CUDA(cudaMemcpyAsync(host_dst, f->ctr, sizeof(FrameCounters), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    return GS_OK;
}

gs_status frame_batch_finish(gs_frame *f, float *const *rgb, float *const *T, uint32_t *const *last,
                             gs_stream stream) {
    gs_status st = batch_emit(f, (cudaStream_t)stream, true);
    if (st) return st;
    if ((st = gs_sort(f, stream))) return st;
    if ((st = gs_ranges(f, stream))) return st;
    return blend_batch(f, rgb, T, last, nullptr, stream);
}

// ------------------------------------------------------------------------------------------ autotune
static gs_status frame_outputs(gs_frame *f, float **rgb, float **T, uint32_t **last) {
    const size_t npx = (size_t)f->max_w * (size_t)f->max_h;
    if (!f->out_mem) {
        GS_CUDA(cudaSetDevice(f->device));
        GS_CUDA(cudaMalloc(&f->out_mem, npx * 5 * sizeof(float)));
    }
    *rgb = (float *)f->out_mem;
    *T = *rgb + 3 * npx;
    *last = (uint32_t *)(*T + npx);
    return GS_OK;
}

extern "C" gs_status gs_autotune(gs_frame *f, const gs_scene *s, const gs_camera *cams, int32_t ncams,
                                 const gs_render_opts *opts, const char *cache_path, gs_tuning *out,
                                 gs_stream stream) {
    if (!f || !s || !cams || ncams <= 0) return fail(GS_ERR_INVALID_ARG, "NULL frame/scene/cameras or ncams <= 0");
    cudaDeviceProp prop;
    GS_CUDA(cudaGetDeviceProperties(&prop, f->device));
    std::string dev = prop.name;
    for (char &ch : dev)
        if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    char key[256];
    snprintf(key, sizeof(key), "gs-autotune-v2 %s %lld %d %d", dev.c_str(), s->P, cams[0].width, cams[0].height);
    if (cache_path) {
        FILE *fp = fopen(cache_path, "r");
        if (fp) {
            char line[512];
            int found_v = -1, found_m = -1, found_a = -1;
            const size_t kl = strlen(key);
            while (fgets(line, sizeof(line), fp))
                if (strncmp(line, key, kl) == 0 && line[kl] == ' ')
                    sscanf(line + kl + 1, "%d %d %d", &found_v, &found_m, &found_a);
            fclose(fp);
            if (found_v >= 0 && found_v < blend_variant_count() && (found_m == 0 || found_m == 1) &&
                found_a >= 0 && found_a <= 2) {
                gs_tuning t = f->tuning;
                t.blend_variant = found_v;
                t.sort_mode = found_m;
                t.sort_algo = found_a;
                gs_status st = gs_frame_set_tuning(f, &t);
                if (st) return st;
                if (out) *out = f->tuning;
                return GS_OK;
            }
        }
    }
    float *rgb, *T;
    uint32_t *last;
    gs_status st = frame_outputs(f, &rgb, &T, &last);
    if (st) return st;
    const int timing_before = f->timing;
    if ((st = gs_frame_enable_timing(f, 1))) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    // time `ncams` renders with the current tuning; returns the summed stage times
    auto timed = [&](float stage_ms[4]) -> gs_status {
        gs_status r = gs_render(f, s, &cams[0], opts, rgb, T, last, stream);   // warm-up
        if (r) return r;
        for (int i = 0; i < 4; ++i) stage_ms[i] = 0.0f;
        for (int c = 0; c < ncams; ++c) {
            if ((r = gs_render(f, s, &cams[c], opts, rgb, T, last, stream))) return r;
            float ms[4];
            if ((r = gs_frame_stage_ms(f, ms))) return r;
            for (int i = 0; i < 4; ++i) stage_ms[i] += ms[i];
        }
        return GS_OK;
    };
    // 1) ordering: preprocess + sort + ranges time of each sort mode and sort algorithm
    int best_mode = f->tuning.sort_mode, best_algo = f->tuning.sort_algo;
    float best_ms = 1e30f;
    for (int m = 0; m <= 1; ++m)
        for (int a = 0; a <= 2; ++a) {
            gs_tuning t = f->tuning;
            t.sort_mode = m;
            t.sort_algo = a;
            if ((st = gs_frame_set_tuning(f, &t))) return st;
            float ms[4];
            if ((st = timed(ms))) return st;
            if (ms[0] + ms[1] + ms[2] < best_ms) {
                best_ms = ms[0] + ms[1] + ms[2];
                best_mode = m;
                best_algo = a;
            }
        }
    // 2) blend launch shape
    int best = f->tuning.blend_variant;
    best_ms = 1e30f;
    for (int v = 0; v < blend_variant_count(); ++v) {
        gs_tuning t = f->tuning;
        t.sort_mode = best_mode;
        t.sort_algo = best_algo;
        t.blend_variant = v;
        if ((st = gs_frame_set_tuning(f, &t))) return st;
        float ms[4];
        if ((st = timed(ms))) return st;
        if (ms[3] < best_ms) {
            best_ms = ms[3];
            best = v;
        }
    }
    GS_CUDA(cudaStreamSynchronize(cs));
    gs_tuning t = f->tuning;
    t.blend_variant = best;
    t.sort_mode = best_mode;
    t.sort_algo = best_algo;
    if ((st = gs_frame_set_tuning(f, &t))) return st;
    if ((st = gs_frame_enable_timing(f, timing_before))) return st;
    if (cache_path) {
        FILE *fp = fopen(cache_path, "a");
        if (fp) {
            fprintf(fp, "%s %d %d %d\n", key, best, best_mode, best_algo);
            fclose(fp);
        }
    }
    if (out) *out = f->tuning;
    return GS_OK;
}

// ------------------------------------------------------------------------------------------ backward
extern "C" gs_status gs_render_backward(gs_frame *f, const gs_scene *s, const float *dL_drgb, const float *T,
                                        const uint32_t *last, const gs_gaussian_grads *g, int32_t accumulate,
                                        gs_stream stream) {
    if (!f || !s || !dL_drgb || !T || !last || !g) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (!g->means || !g->scales || !g->quats || !g->opacity || !g->sh)
        return fail(GS_ERR_INVALID_ARG, "a gradient array is NULL");
    if (f->W <= 0 || f->scene_used != s || f->batch.n != 1)
        return fail(GS_ERR_INVALID_ARG, "no single render of this scene on the frame");
    cudaStream_t st = (cudaStream_t)stream;
    if (!f->grad2d) {
        GS_CUDA(cudaSetDevice(f->device));
        GS_CUDA(cudaMalloc(&f->grad2d, sizeof(float) * (size_t)grad2d_floats() * (size_t)f->max_g));
    }
    GS_CUDA(cudaMemsetAsync(f->grad2d, 0, sizeof(float) * (size_t)grad2d_floats() * (size_t)s->P, st));
    BwdArgs a;
    a.ctr = f->ctr;
    a.recs = f->recs;
    a.vals = f->vals[f->sorted_buf];
    a.starts = f->starts;
    a.n_dev = &f->ctr->n_pairs;
    a.cap = f->max_pairs;
    a.opt = f->opt;
    a.cam = f->cam;
    a.scene.pos_opa = s->pos_opa;
    a.scene.rs = s->rs;
    a.scene.sh = s->sh;
    a.scene.P = s->P;
    a.scene.sh_degree = s->sh_degree;
    a.scene.activated = s->activated;
    a.scene.sh_half = s->sh_half;
    a.W = f->W;
    a.H = f->H;
    a.tiles_x = f->tiles_x;
    a.tiles_y = f->tiles_y;
    a.dL_drgb = dL_drgb;
    a.T_final = T;
    a.last = last;
    a.grad2d = f->grad2d;
    a.g_means = g->means;
    a.g_scales = g->scales;
    a.g_quats = g->quats;
    a.g_opacity = g->opacity;
    a.g_sh = g->sh;
    a.accumulate = accumulate ? 1 : 0;
    a.vec16 = (((uintptr_t)g->quats | (uintptr_t)g->sh) & 15u) == 0 ? 1 : 0;
    if (f->timing) GS_CUDA(cudaEventRecord(f->evb[0], st));
    launch_backward(a, st, f->timing ? f->evb[1] : nullptr);
    if (f->timing) {
        GS_CUDA(cudaEventRecord(f->evb[2], st));
        f->bwd_timed = 1;
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}
