/*
 * gs.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting forward rasterizer with
 * FlashGS's opacity-aware exact intersection (arXiv 2408.07967).
 *
 * Pipeline (Section 2.2 and Fig. "FlashGS Overview"; Algorithm 4):
 *   gs_preprocess  per-Gaussian cull, projection, EWA conic, Eq. 3 threshold, tight box,
 *                  exact ellipse/tile test (Algorithm 3, Eq. 9) and (tile, depth) key
 *                  emission, SH colour, all in one kernel;
 *   gs_sort        stable radix sort of the 64-bit (tile, depth) keys with Gaussian ids;
 *   gs_ranges      [start, end) of every tile in the sorted list;
 *   gs_blend       per-16x16-tile front-to-back alpha blending with early stop.
 *   gs_render      the four stages in order (replayed from a CUDA graph when enabled).
 *
 * Conventions used by every call:
 *   - Pointers named *_dev are device pointers; others are host pointers.  The caller owns
 *     every buffer it passes in; the library owns contexts, scenes and frames and the device
 *     memory inside them, which it allocates once at creation (Section 5.3.1: no per-frame
 *     allocation) and frees at destruction.
 *   - Calls taking a gs_stream (a cudaStream_t; NULL is the legacy default stream) only
 *     enqueue work on it and return without synchronising, unless documented otherwise.
 *   - Errors are returned as negative gs_status codes; gs_last_error() gives a message for
 *     the calling thread.  No call aborts the process.  Errors found on the device (pair
 *     buffer overflow, a bounded wait that gave up) are recorded in the frame and reported by
 *     gs_frame_get_stats().
 *   - Cameras are pinholes: x_cam = R x_world + t (R row-major), the camera looks down +z with
 *     x right and y down; pixel (i, j) covers [i, i+1) x [j, j+1) and is sampled at its centre;
 *     u = fx x/z + cx, v = fy y/z + cy.
 *   - Gaussians are given as canonical arrays of float32: means [P,3], scales [P,3] (or
 *     log-scales), quaternions [P,4] as (w, x, y, z) (normalised internally), opacities [P]
 *     (or logits), SH coefficients [P,16,3] (coefficient-major, RGB-minor; degree <= 3).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gs_status;
#define GS_OK 0
#define GS_ERR_INVALID_ARG (-1)
#define GS_ERR_OOM (-2)
#define GS_ERR_PAIR_OVERFLOW (-3)
#define GS_ERR_CUDA (-4)
#define GS_ERR_DEVICE_TIMEOUT (-5)
#define GS_ERR_BUSY (-6)
#define GS_ERR_CAPACITY (-7)
#define GS_ERR_NO_DEVICE (-8)

typedef struct gs_context gs_context;
typedef struct gs_scene gs_scene;
typedef struct gs_frame gs_frame;
typedef void *gs_stream; /* cudaStream_t */

typedef struct {
    float R[9];      /* world -> camera rotation, row-major */
    float t[3];      /* world -> camera translation */
    float fx, fy;    /* focal lengths in pixels */
    float cx, cy;    /* principal point in pixel-area coordinates */
    int32_t width, height;
    float near_z;    /* near plane; Algorithm 4 culls z <= 0.2 */
} gs_camera;

typedef struct {
    const float *means;    /* [P,3] device */
    const float *scales;   /* [P,3] device: scales, or log-scales when activated == 0 */
    const float *quats;    /* [P,4] device: (w,x,y,z) */
    const float *opacity;  /* [P] device: opacity, or logits when activated == 0 */
    const float *sh;       /* [P,16,3] device */
    int64_t P;
    int32_t sh_degree;     /* 0..3 */
    int32_t activated;     /* 1: scales/opacities as given; 0: exp / sigmoid applied on device */
    int32_t sh_half;       /* 1: opt-in reduced precision -- the scene keeps the SH coefficients as
                              IEEE binary16 (round to nearest even), 96 instead of 192 bytes per
                              Gaussian; colours then follow the rounded coefficients (the paper
                              quantises nothing; pairs and keys do not depend on SH).  0: binary32.
                              Fixed at gs_scene_create: gs_scene_update must pass the same value. */
    int32_t reserved;      /* 0 */
} gs_gaussians;

typedef struct {
    float bg[3];        /* background colour added with the final transmittance */
    float tau;          /* alpha threshold, 1/255 (Section 4.1) */
    float alpha_max;    /* alpha clamp, 0.99 */
    float T_min;        /* early-stop transmittance, 1e-4 */
    float dilation;     /* low-pass added to the 2D covariance diagonal, 0.3 px^2 */
    int32_t cap_3sigma; /* 0: t = 2 ln(alpha0/tau) (Eq. 3); 1: t = min(9, Eq. 3) (Section 4.1) */
    int32_t clamp_fov;  /* 1: clamp x/z, y/z to 1.3 tan(half fov) in the EWA Jacobian */
    int32_t intersect;  /* 0: exact tile pairs (Alg. 3, the default); 1: the 3DGS pairs the paper
                           compares against -- every tile of the square of radius
                           ceil(3 sqrt(max eigenvalue of Sigma')) about the mean (Eq. 1, Alg. 1-2).
                           Same blend; under cap_3sigma both give the same image. */
} gs_render_opts;

typedef struct {
    int64_t pairs;          /* Gaussian/tile pairs emitted by gs_preprocess (may exceed capacity) */
    int64_t visible;        /* Gaussians with at least one pair */
    int64_t pair_capacity;  /* pairs the frame can hold */
    int32_t status;         /* GS_OK, GS_ERR_PAIR_OVERFLOW or GS_ERR_DEVICE_TIMEOUT */
    int32_t width, height;
    int32_t tiles_x, tiles_y;
    int32_t sort_passes;    /* 8-bit digit passes of the last sort */
    int64_t culled_in;      /* Gaussians passing the near-plane and opacity cull */
    int64_t evaluations;    /* counting mode: (pixel, list entry) pairs walked by the last gs_blend */
    int64_t contributions;  /* counting mode: of those, entries with q <= t (alpha >= tau) */
    int32_t kernels;        /* kernels one gs_render launches */
    int32_t pad;
} gs_frame_stats;

/* Message for the last error returned on the calling thread ("" if none). */
const char *gs_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t gs_version(void);

/* Fills *opts with the defaults above (bg 0, tau 1/255, alpha_max 0.99, T_min 1e-4,
   dilation 0.3, cap_3sigma 0, clamp_fov 1).  GS_ERR_INVALID_ARG if opts is NULL. */
gs_status gs_default_opts(gs_render_opts *opts);

/* Creates a context bound to CUDA device `device` (made current on the calling thread).
   Errors: GS_ERR_NO_DEVICE, GS_ERR_CUDA, GS_ERR_OOM. */
gs_status gs_context_create(int32_t device, gs_context **out);
gs_status gs_context_destroy(gs_context *ctx);

/* Device-resident scene: copies the canonical arrays in `g` into the library's internal
   layout (240 bytes per Gaussian: a plane of position+opacity, read by the cull of every
   Gaussian; a plane of scale and quaternion, read for Gaussians that pass the cull; and each
   Gaussian's 48 SH floats as one contiguous 192-byte block, read only for paired Gaussians),
   enqueued on `stream`.  The input arrays may be freed
   once the stream has passed this call.  Section 5.3.1 (per-scene work done once).
   Errors: GS_ERR_INVALID_ARG (NULL pointers, P <= 0, P >= 2^31, bad degree), GS_ERR_OOM. */
gs_status gs_scene_create(gs_context *ctx, const gs_gaussians *g, gs_stream stream, gs_scene **out);
/* Re-packs new parameter values of the same P into an existing scene (training steps). */
gs_status gs_scene_update(gs_scene *scene, const gs_gaussians *g, gs_stream stream);
gs_status gs_scene_destroy(gs_scene *scene);
int64_t gs_scene_size(const gs_scene *scene);

/* Per-frame state (Table 2 / Section 5.3.1: allocated once, reused every frame): render
   records for up to max_gaussians, two ping-pong pair buffers of max_pairs (u64 key, u32
   value), tile ranges for up to max_width x max_height, and the scratch of the scan and the
   sort.  Errors: GS_ERR_INVALID_ARG, GS_ERR_OOM (nothing is left allocated). */
gs_status gs_frame_create(gs_context *ctx, int64_t max_gaussians, int64_t max_pairs,
                          int32_t max_width, int32_t max_height, gs_frame **out);
gs_status gs_frame_destroy(gs_frame *frame);
/* Bytes of device memory held by the frame. */
int64_t gs_frame_bytes(const gs_frame *frame);

/* Stage a (Algorithm 4; Algorithm 3; Eq. 2-3, 9): per Gaussian, cull z <= near_z and
   alpha0 <= tau, project, build the EWA conic, compute t = 2 ln(alpha0/tau), test every tile
   of the tight bounding box exactly, and write one (key, Gaussian id) pair per intersecting
   tile, key = (tile_id << 32) | float_bits(z), tile_id = ty * tiles_x + tx.  Pairs are written
   in (Gaussian id, tile row-major) order.  Also writes each paired Gaussian's render record
   (centre, conic, threshold, colour).  Errors: GS_ERR_INVALID_ARG (scene larger than the frame,
   image larger than the frame, camera with non-positive focal length). */
gs_status gs_preprocess(gs_frame *frame, const gs_scene *scene, const gs_camera *cam,
                        const gs_render_opts *opts, gs_stream stream);

/* Stage b (Section 2.2 sort): stable LSD radix sort of the frame's pairs by key in 8-bit digits
   (one histogram pass, then one chained-scan scatter pass per digit): over bits
   [0, 32 + ceil(log2(tiles))) of the 64-bit keys in sort_mode 0, over the tile bits of the 32-bit
   keys in sort_mode 1 (where gs_preprocess already ordered the pairs by depth).  The pair count is
   read on the device. */
gs_status gs_sort(gs_frame *frame, gs_stream stream);

/* Stage c: start of every tile's run in the sorted keys -- one pass over the keys when the tiles
   hold between 1 and 512 pairs on average, else a binary search per tile. */
gs_status gs_ranges(gs_frame *frame, gs_stream stream);

/* Stage d (Section 2.2 render; Section 5.2): per 16x16 tile, walk the tile's sorted list
   front to back; per pixel alpha = min(alpha_max, alpha0 exp(-q/2)), skip when
   alpha < tau, stop before a Gaussian that would take T below T_min, C += rgb alpha T.
   Writes rgb_dev [3,H,W] = C + T bg, T_dev [H,W] (nullable) and last_dev [H,W] (nullable:
   1-based position in the tile list of the last contributor, 0 if none). */
gs_status gs_blend(gs_frame *frame, const gs_render_opts *opts, float *rgb_dev, float *T_dev,
                   uint32_t *last_dev, gs_stream stream);

/* Stages a-d in order.  When graphs are enabled on the frame (gs_frame_use_graph) the
   sequence is captured once per (scene, image size) and replayed with updated camera and
   options.  Errors: as the stages. */
gs_status gs_render(gs_frame *frame, const gs_scene *scene, const gs_camera *cam,
                    const gs_render_opts *opts, float *rgb_dev, float *T_dev, uint32_t *last_dev,
                    gs_stream stream);

/* Gradients w.r.t. the parameters as given to gs_scene_create / gs_scene_update (log-scales
   and logits when the scene is not activated).  Device arrays owned by the caller. */
typedef struct {
    float *means;    /* [P,3] */
    float *scales;   /* [P,3] */
    float *quats;    /* [P,4] (w.r.t. the unnormalised quaternion) */
    float *opacity;  /* [P]   */
    float *sh;       /* [P,16,3] */
} gs_gaussian_grads;

/* Backward of the last gs_render on this frame (the paper claims a differentiable rasterizer,
   abstract; no backward is described, so this is the exact derivative of the forward with its
   decisions held fixed: contributing entries, early stop, alpha / colour / Jacobian clamps).
   dL_drgb_dev [3,H,W] is the loss gradient of the rendered image; T_dev and last_dev are the
   transmittance and last-contributor outputs of that render (required).  The scene must be the
   one rendered, unchanged since.  Per tile, pixels walk their lists back to front recovering T
   by division; per-Gaussian sums are warp-reduced, accumulated per CTA in shared memory and
   added to a frame-owned buffer; a per-Gaussian kernel then applies the chain rule through the
   projection, covariance, quaternion, activations and SH.  accumulate = 0 overwrites `grads`,
   1 adds to them.  Errors: GS_ERR_INVALID_ARG (no render on the frame, NULL pointers, scene
   size mismatch). */
gs_status gs_render_backward(gs_frame *frame, const gs_scene *scene, const float *dL_drgb_dev,
                             const float *T_dev, const uint32_t *last_dev, const gs_gaussian_grads *grads,
                             int32_t accumulate, gs_stream stream);

/* Renders n (1..16) requests in one pass of every stage: each request r has its own scene
   (any of the device-resident scenes), camera, image size and options (opts: array of n, or
   NULL for defaults) and writes rgb[r] [3,H_r,W_r] (device), T[r] and last[r] (arrays of n
   device pointers, or NULL).  Request r's Gaussians occupy records rec0_r + id, its tiles the
   global tile ids tile0_r .. in the (tile, depth) keys, so the preprocess, the sort, the ranges
   and the blend each run once over the whole batch with per-request tile ranges.  Each request's
   result is bit-identical to rendering it alone.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CAPACITY
   (more Gaussians or tiles than the frame holds). */
gs_status gs_render_batch(gs_frame *frame, int32_t n, const gs_scene *const *scenes, const gs_camera *cams,
                          const gs_render_opts *opts, float *const *rgb_dev, float *const *T_dev,
                          uint32_t *const *last_dev, gs_stream stream);

/* Enables (1) or disables (0) CUDA-graph replay of gs_render on this frame. */
gs_status gs_frame_use_graph(gs_frame *frame, int32_t enable);

/* Launch-shape and ordering choices of a frame (picked by gs_autotune).
   blend_variant 0..5 = (pixels per thread, records per staged batch) of (1, 256), (2, 128),
   (4, 128), (2, 256), (4, 64), (4, 256); 256 / pixels-per-thread threads per 16x16 tile.
   sort_mode 0: pairs emitted in (Gaussian id, tile) order with 64-bit (tile << 32 | depth bits)
   keys and sorted over 32 + ceil(log2 tiles) bits; sort_mode 1 (two-level): the paired
   Gaussians are sorted once by depth (32-bit keys), pairs are emitted in that order with the
   tile id alone as a 32-bit key, and a stable sort over ceil(log2 tiles) bits finishes -- the
   same (tile, depth, id) order with far fewer bytes moved.  sort_algo picks how the radix passes
   of the pair sort are carried out (below; the depth sort of sort_mode 1 always runs fused).
   Results are bit-identical across all choices.  GS_ERR_INVALID_ARG for out-of-range values. */
typedef struct {
    int32_t blend_variant;
    int32_t sort_mode;
    int32_t sort_algo;     /* 0: onesweep passes (decoupled look-back between tiles); 1: reduce-then-
                              scan passes (per-tile digit counts, a scan across tiles, then the
                              scatter: keys read twice, no tile waits on another); 2: the onesweep
                              passes of a sort fused into one cooperative launch (histograms, then
                              the passes, separated by grid-wide barriers; sorts of one pass, and
                              any sort whose cooperative launch the device refuses, run as 0) */
    int32_t reserved[5];
} gs_tuning;
gs_status gs_frame_set_tuning(gs_frame *frame, const gs_tuning *tuning);
gs_status gs_frame_get_tuning(const gs_frame *frame, gs_tuning *tuning);

/* Autotuner: picks the frame's gs_tuning for rendering `scene` at the size of cams[0].  With
   cache_path non-NULL, a line "gs-autotune-v2 <device> <P> <W> <H> <blend_variant> <sort_mode>
   <sort_algo>" matching this device, scene size and image size is reused when present; otherwise
   every (sort_mode, sort_algo) is timed (preprocess + sort + ranges) and then every blend_variant
   (blend), each over the
   ncams cameras after one warm-up render with CUDA-event stage times, and the fastest choices are
   kept and appended to the cache file.  The frame
   is left with the chosen tuning, which is also written to *out (nullable).  Synchronises
   `stream`; renders into frame-owned buffers.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA; an
   unreadable or unwritable cache file is ignored. */
gs_status gs_autotune(gs_frame *frame, const gs_scene *scene, const gs_camera *cams, int32_t ncams,
                      const gs_render_opts *opts, const char *cache_path, gs_tuning *out, gs_stream stream);

/* Measured arithmetic throughput of a device, the denominator of the blend stage's roofline (the
   blend is bound by FP32 and special-function work, and neither rate is a published measured
   figure).  Two probe kernels run on every SM at full occupancy: one issues independent chains of
   FP32 fused multiply-adds (one lane-operation each), the other independent chains of ex2.approx.
   Each runs about `target_ms` milliseconds (<= 0: 200 ms) after a warm-up, timed with CUDA events
   on a private stream; the result is lane-operations per second / 1e12 and the elapsed time of each
   probe.  The paper has no counterpart (it reports no roofline).  Synchronous; allocates a 4 KiB
   buffer for the probes' sinks.  Errors: GS_ERR_INVALID_ARG (NULL out), GS_ERR_NO_DEVICE,
   GS_ERR_CUDA. */
typedef struct {
    double fma_tops;     /* FP32 FMA lane-operations per second / 1e12 */
    double ex2_tops;     /* ex2.approx.ftz.f32 results per second / 1e12 */
    double fma_ms;       /* duration of the timed FMA probe */
    double ex2_ms;       /* duration of the timed ex2 probe */
    int32_t sm_count;
    int32_t pad;
} gs_alu_peaks;
gs_status gs_measure_alu_peaks(int32_t device, double target_ms, gs_alu_peaks *out);

/* Evaluates, over n binary32 inputs x_dev[i] (device), the device routines whose bits decide the
   pair set, exactly as the preprocess kernel runs them, into y_dev[i] (device):
     fn 0: t = 2 ln(x / param), the opacity-aware threshold of Eq. 3 (x = alpha0, param = tau,
           Section 4.1);
     fn 1: e^x, the activation of a log-scale (Section 2.2's 3D covariance from scales);
     fn 2: 1 / (1 + e^-x), the activation of an opacity logit.
   ln and exp are the library's own binary32 routines (argument reduction, a fixed polynomial,
   every operation explicitly rounded), so that a host program implementing the same published
   method reproduces them bit for bit; this call exists to test that over whole input domains.
   Enqueued on `stream`, no synchronisation.  The caller owns both arrays.  Errors:
   GS_ERR_INVALID_ARG (fn out of range, n < 0, NULL array with n > 0), GS_ERR_CUDA. */
gs_status gs_eval_decision_math(int32_t fn, const float *x_dev, float *y_dev, int64_t n, float param,
                                gs_stream stream);

/* Enables (1) or disables (0) the instrumented blend that counts, per frame, the (pixel, entry)
   pairs walked before early stop and those passing q <= t (gs_frame_stats.evaluations /
   .contributions).  Same outputs; slower; meant for measurement, not for timed runs. */
gs_status gs_frame_set_counting(gs_frame *frame, int32_t enable);

/* Enables (1) or disables (0) CUDA events around the four stages of gs_render (recorded inside
   the graph when graphs are enabled). */
gs_status gs_frame_enable_timing(gs_frame *frame, int32_t enable);

/* Waits for the last gs_render_backward run with timing enabled and writes the device time of its
   two kernels in milliseconds: ms[0] the reverse blend (per tile, back to front, per-Gaussian 2D
   gradients), ms[1] the per-Gaussian chain rule to the 3D parameters.  GS_ERR_INVALID_ARG when
   timing is off or no backward was timed.  The paper describes no backward (abstract only). */
gs_status gs_frame_backward_ms(gs_frame *frame, float ms[2]);

/* Waits for the last timed gs_render and writes the device time of its stages in milliseconds:
   ms[0] preprocess, ms[1] sort, ms[2] ranges, ms[3] blend.  GS_ERR_INVALID_ARG when timing is
   off or nothing was timed yet. */
gs_status gs_frame_stage_ms(gs_frame *frame, float ms[4]);

/* gs_render into buffers owned by the frame, then copies the result to HOST memory: rgb_host
   [3,H,W] float, T_host [H,W] float (nullable), last_host [H,W] uint32 (nullable); `cam` and
   `opts` are host structs passed by value to the kernels.  The copies are enqueued on `stream`
   (asynchronous when the host buffers are page-locked); the call returns without waiting --
   synchronise `stream` before reading the host buffers.  Errors: as gs_render. */
gs_status gs_render_host(gs_frame *frame, const gs_scene *scene, const gs_camera *cam,
                         const gs_render_opts *opts, float *rgb_host, float *T_host, uint32_t *last_host,
                         gs_stream stream);

/* Synchronises `stream` and reads the frame's counters.  status carries device-side errors:
   GS_ERR_PAIR_OVERFLOW when more pairs were found than max_pairs (outputs are then invalid;
   pairs holds the number needed), GS_ERR_DEVICE_TIMEOUT when a bounded wait gave up. */
gs_status gs_frame_get_stats(gs_frame *frame, gs_frame_stats *out, gs_stream stream);

/* Copies min(pairs, capacity, cap) pairs to caller buffers keys_dev / vals_dev (device):
   which = 0 the emission-order list written by gs_preprocess (valid before gs_sort),
   which = 1 the sorted list (valid after gs_sort).  *n_out (host) receives the count copied.
   Synchronises `stream`. */
gs_status gs_frame_pairs(gs_frame *frame, int32_t which, uint64_t *keys_dev, uint32_t *vals_dev,
                         int64_t cap, int64_t *n_out, gs_stream stream);

/* Copies the tile starts (tiles + 1 entries of uint32) to starts_dev.  Synchronises. */
gs_status gs_frame_ranges(gs_frame *frame, uint32_t *starts_dev, int64_t cap, gs_stream stream);

/* Stand-alone stable radix sort of n (u64 key, u32 value) pairs by key bits [0, end_bit)
   (end_bit <= 64), the primitive behind gs_sort.  keys_dev/vals_dev hold the input; tmp
   buffers of the same sizes are caller-provided ping-pong storage.  *in_tmp (host) is set to 1
   when the result ended in the tmp buffers (odd number of passes), else 0.  Scratch for the
   histograms and the chained scan comes from the context (grown on demand, never freed before
   gs_context_destroy).  The call only enqueues work; a device-side failure (a bounded wait that
   gave up, which leaves the output invalid) is reported by gs_sort_pairs_status.  Errors:
   GS_ERR_INVALID_ARG (n < 0, n >= 2^30, end_bit out of range). */
gs_status gs_sort_pairs(gs_context *ctx, uint64_t *keys_dev, uint32_t *vals_dev, uint64_t *keys_tmp_dev,
                        uint32_t *vals_tmp_dev, int64_t n, int32_t end_bit, int32_t *in_tmp,
                        gs_stream stream);

/* Synchronises `stream` and reports the device-side outcome of the last gs_sort_pairs on `ctx`:
   GS_OK, or GS_ERR_DEVICE_TIMEOUT when one of its bounded waits gave up (its output is then not
   a sorted permutation and must be discarded; the next gs_sort_pairs starts clean).  Errors:
   GS_ERR_INVALID_ARG (NULL context), GS_ERR_CUDA. */
gs_status gs_sort_pairs_status(gs_context *ctx, gs_stream stream);

/* Bounded waits.  Kernels that wait on other thread blocks (the sort's look-back between tiles,
   the grid barriers of the fused sort) give up after a number of polls, set a device status
   (reported as GS_ERR_DEVICE_TIMEOUT by gs_frame_get_stats, gs_sort_pairs_status and
   gs_sort_pairs_noalloc_status) and return; kernels launched after such a failure that would read
   its output write nothing.  gs_set_wait_limit sets that number of polls for every launch that
   follows, process-wide (0 restores the default, 2^22 polls of at least 20 ns each); a small value
   makes correct runs fail and exists to test the failure path.  Waits of a thread block on its own
   bulk copies always keep the default, so that no block leaves while a copy into its shared memory
   is in flight.  gs_get_wait_limit returns the limit in force.  The paper has no counterpart. */
gs_status gs_set_wait_limit(uint32_t polls);
uint32_t gs_get_wait_limit(void);

/* ------------------------------------------------------------------------------------------
   Serving: a continuous-batching request loop over device-resident scenes (a worker thread
   inside the library).  Requests -- a scene, a camera of any size up to the configured maximum,
   options and a HOST output buffer -- are queued by gs_server_submit.  Up to `slots` batches are
   in flight at once, each on its own stream with its own frame and output pool, so batches
   overlap on the device; a batch starts beside a running one only once two or more requests
   are waiting (overlap costs the older batch latency, so it is spent only on a backlog).  When a slot is free the oldest waiting requests (at most max_batch,
   at most max_gaussians Gaussians together) are admitted by pair-buffer memory: one count pass
   (geometry + exact pair counts) gives each request's pairs, and the oldest requests whose
   pairs fit pair_capacity run as one batch through gs_render_batch's single pass per stage with
   per-request tile ranges; the rest wait for the next free slot (at light load, see fifo_load_pct,
   requests instead run one at a time in arrival order).  A lone request skips the
   admission round trip (it has nothing to defer; if it alone exceeds pair_capacity it completes
   with GS_ERR_PAIR_OVERFLOW).  Batches run on streams prioritised by age: a batch launched while
   k others are in flight gets the k-th highest stream priority, so the oldest batch keeps the
   SMs it needs and younger ones fill the rest.  Images are copied to the callers' host buffers
   (asynchronous when page-locked).  Every request's image is
   bit-identical to rendering it alone.  plain = 1 is the baseline loop: one request at a time,
   synchronously, no count pass.  The paper describes single frames only; batching requests is
   this library's extension (Section 5.3.1's static allocation carries over: all buffers are
   allocated at creation). */
typedef struct gs_server gs_server;
typedef struct {
    int32_t slots;            /* batches in flight at once, 1..8 (plain: 1) */
    int32_t max_batch;        /* requests per batch, 1..16 (plain: 1) */
    int64_t pair_capacity;    /* pairs per batch (pair buffers of each slot), < 2^30 */
    int64_t max_gaussians;    /* Gaussians per batch, summed over its requests */
    int32_t max_width, max_height;   /* largest request image */
    int32_t sort_mode;        /* gs_tuning.sort_mode of the slots' frames, -1 for the default */
    int32_t blend_variant;    /* gs_tuning.blend_variant, -1 for the default */
    int32_t plain;            /* 1: one request at a time (the baseline loop) */
    int32_t batch_pixels;     /* image pixels per batch, summed over its requests (0: 2 x 1920 x 1080);
                                 a larger request runs alone -- batching amortises launches and
                                 small kernels, while a request that fills the GPU by itself only
                                 waits longer in a batch */
    int32_t overlap_pending;  /* under load, a batch starts beside batches in flight when at least this
                                 many requests are waiting (0: the default, 1) */
    int32_t fifo_load_pct;    /* while the estimated load -- the recent arrival rate times the mean
                                 service time of recent requests -- is below this percentage, requests
                                 run one at a time in arrival order with nothing beside them, as in the
                                 plain loop (at light load a batch or an overlap only makes its first
                                 request wait for the others' work); above it they are batched and
                                 overlapped.  0: the default, 30; -1: always batch. */
} gs_server_cfg;
typedef struct {
    int32_t status;           /* GS_OK, GS_ERR_PAIR_OVERFLOW (alone over the pair capacity), ... */
    int32_t batch_size;       /* requests in the batch it ran in */
    double arrival_s;         /* gs_clock_s() time of arrival (as submitted) */
    double admit_s;           /* time the batch was formed */
    double done_s;            /* time its image was in the host buffer */
    int64_t pairs;            /* its Gaussian/tile pairs */
} gs_request_stats;
typedef struct {
    int64_t completed, batches, batched_requests, pending;
} gs_server_stats;

/* Monotonic clock of the server, seconds (for arrival times). */
double gs_clock_s(void);
/* Defaults: 3 slots, batches of up to 8, 2^26 pairs and 2^26 Gaussians per batch, 3840x2160. */
gs_status gs_default_server_cfg(gs_server_cfg *cfg);
/* Allocates every slot's frame, stream and output pool and starts the worker.  Errors:
   GS_ERR_INVALID_ARG, GS_ERR_OOM. */
gs_status gs_server_create(gs_context *ctx, const gs_server_cfg *cfg, gs_server **out);
/* Stops the worker after the batches in flight; unfinished queued requests are dropped. */
gs_status gs_server_destroy(gs_server *server);
/* Queues a request; rgb_host receives [3,H,W] floats and must stay valid until the request is
   waited for.  arrival_s <= 0 means now.  The scene must stay alive and unchanged until then.
   Returns at once with *ticket.  Errors: GS_ERR_INVALID_ARG (image larger than the maximum),
   GS_ERR_CAPACITY (scene larger than a batch). */
gs_status gs_server_submit(gs_server *server, const gs_scene *scene, const gs_camera *cam,
                           const gs_render_opts *opts, float *rgb_host, double arrival_s, uint64_t *ticket);
/* Waits for a request (timeout_ms < 0: no limit) and returns its status; GS_ERR_DEVICE_TIMEOUT
   when the limit passes first (the request stays queued).  *out (nullable) gets its times. */
gs_status gs_server_wait(gs_server *server, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out);
gs_status gs_server_get_stats(gs_server *server, gs_server_stats *out);
/* hold = 1: stop admitting requests (they keep queueing) and wait until no batch is in flight,
   e.g. before gs_scene_update of a scene the server renders, or to let a burst queue up and run
   in full batches; hold = 0: resume.  Errors: GS_ERR_INVALID_ARG (NULL server). */
gs_status gs_server_hold(gs_server *server, int32_t hold);

/* ------------------------------------------------------------------------------------------
   Routing across replicas: frames and requests are independent units, so a machine with several
   GPUs serves them with one gs_server per GPU, each holding its own copy of the scenes it serves.
   The router sends each request to the replica that holds its scene and has the fewest image
   pixels outstanding (submitted, not yet waited for; ties to the lower index), and keeps the
   (replica, ticket) behind each router ticket.  Replicas are reached through a backend: either
   gs_router_create_on_servers (gs_server objects, scenes placed with gs_router_place_scene) or any
   caller-supplied pair of submit/wait functions (gs_router_create).  The paper renders on one GPU
   and has no counterpart.  Thread-safe; submit never blocks on a device. */
typedef struct gs_router gs_router;
typedef struct {
    /* submit a request for scene `scene` to replica `replica`; *ticket identifies it there */
    gs_status (*submit)(void *user, int32_t replica, int32_t scene, const gs_camera *cam,
                        const gs_render_opts *opts, float *rgb_host, double arrival_s, uint64_t *ticket);
    /* wait for it (timeout_ms < 0: no limit); fills *out as gs_server_wait does */
    gs_status (*wait)(void *user, int32_t replica, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out);
    void *user;
} gs_router_backend;
/* replicas 1..64.  Errors: GS_ERR_INVALID_ARG, GS_ERR_OOM. */
gs_status gs_router_create(int32_t replicas, const gs_router_backend *backend, gs_router **out);
/* Backend over gs_server objects (servers[i] = replica i, not owned by the router). */
gs_status gs_router_create_on_servers(int32_t replicas, gs_server *const *servers, gs_router **out);
gs_status gs_router_destroy(gs_router *router);
/* Declares that replica `replica` holds scene id `scene` (0 <= scene < 4096); `handle` is that
   replica's gs_scene for the server backend (ignored, may be NULL, for a custom backend). */
gs_status gs_router_place_scene(gs_router *router, int32_t scene, int32_t replica, const gs_scene *handle);
/* Routes one request.  Errors: GS_ERR_INVALID_ARG (scene placed nowhere), or the backend's. */
gs_status gs_router_submit(gs_router *router, int32_t scene, const gs_camera *cam, const gs_render_opts *opts,
                           float *rgb_host, double arrival_s, uint64_t *ticket);
/* Waits for a routed request; *replica (nullable) receives where it ran.  Returns its status. */
gs_status gs_router_wait(gs_router *router, uint64_t ticket, int32_t timeout_ms, gs_request_stats *out,
                         int32_t *replica);
/* Requests and image pixels outstanding on one replica. */
gs_status gs_router_outstanding(gs_router *router, int32_t replica, int64_t *requests, int64_t *pixels);

/* gs_sort_pairs without any allocation.  The paper has no counterpart: this entry point exists
   for callers that must not allocate device memory -- code handed its buffers by a host
   application that owns the device-memory budget (an embedded renderer, a plugin, a real-time
   loop), where cudaMalloc/cudaFree could synchronise the device or fail because the host
   application has reserved all memory for its own pool.
   Same sort and arguments as gs_sort_pairs (the caller passes the key/value buffers and the
   ping-pong buffers), but the histograms, digit offsets, look-back descriptors and tickets live
   in one fixed array inside the library's device image (about 2 MiB, held by every GPU that loads
   the library until the process exits).  n may be at most 2,097,152 pairs; larger n returns
   GS_ERR_CAPACITY with a message in gs_last_error().  The first call on a device looks up the
   array's device address with that device current; make that first call before any stream
   capture.  Every call on a device shares the array and it keeps the last call's contents (the
   call clears what must start at zero), so calls whose work overlaps on the GPU -- e.g. on two
   streams without an ordering between them -- race and must not be issued.  Calls no cudaMalloc,
   cudaFree or allocating library routine.  The device address looked up by the first call is kept
   for the life of the process: after cudaDeviceReset on that device the array's old address is
   stale, so do not use this entry point again in that process.  Like gs_sort_pairs it only
   enqueues work; gs_sort_pairs_noalloc_status reports a device-side failure of the last call. */
gs_status gs_sort_pairs_noalloc(uint64_t *keys_dev, uint32_t *vals_dev, uint64_t *keys_tmp_dev,
                                uint32_t *vals_tmp_dev, int64_t n, int32_t end_bit, int32_t *in_tmp,
                                gs_stream stream);

/* Synchronises `stream` (on which the last gs_sort_pairs_noalloc of the current device was issued)
   and reads that call's device status from the fixed array: GS_OK, or GS_ERR_DEVICE_TIMEOUT when
   one of its bounded waits gave up (the output is then invalid; the next call clears the status).
   Allocates nothing.  Errors: GS_ERR_INVALID_ARG (no allocation-free sort has run on the current
   device), GS_ERR_CUDA. */
gs_status gs_sort_pairs_noalloc_status(gs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
