/*
 * gsr.h -- C ABI of the GB300 low-resolution 3D Gaussian Splatting render core
 * (the render that feeds the super-sampling and frame-interpolation networks of
 * 3DGS^3, arXiv 2605.11489).
 *
 * What it computes (paper Sec. 3, "Preliminaries"):
 *   - Gaussians G(x) = exp(-1/2 (x - xc)^T Sigma^-1 (x - xc))              (Eq. 1)
 *     with Sigma = R S S^T R^T (R from a quaternion, S = diag(exp(log_scale)))
 *   - EWA splatting to screen-space conics, plus a 0.3 px^2 low-pass
 *   - view-dependent colour c_i from SH coefficients (degree 0..3, +0.5, >= 0)
 *   - depth sort: instances keyed by (tile id, fp32 depth), radix sorted
 *   - front-to-back alpha blending I = sum_i c_i a_i T_i                   (Eq. 2)
 *     a_i = min(0.99, opacity * G), skipped below 1/255, stop before T < 1e-4
 *   - in the same pass, the analytic screen-space image gradients           (Eq. 3)
 *     dI/dx = sum_i c_i (dT_i/dx a_i + T_i da_i/dx) with                    (Eq. 4)
 *     dT_i/dx = -da_{i-1}/dx T_{i-1} + (1 - a_{i-1}) dT_{i-1}/dx (same in y),
 *     plus depth = sum_i z_i a_i T_i and alpha = 1 - T_final.
 *
 * Conventions shared by every call:
 *   - Device memory: every float pointer in gs_scene, gs_outputs and
 *     gs_scene_grads is a CUDA device pointer owned by the caller. Planes are
 *     fp32, attribute-planar (structure of arrays) with row stride n_pad
 *     (n_pad % 4 == 0, n_pad >= n) and every base pointer 16-byte aligned.
 *   - Image planes are planar fp32: rgb/dcdx/dcdy are [3][H][W], depth/alpha
 *     [H][W], row-major, pixel (i, j) sampled at (i + 0.5, j + 0.5).
 *   - Camera: OpenCV axes (x right, y down, z forward); viewmat is the
 *     world->camera transform as a row-major 3x4 [R | t].
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream) unless stated otherwise.
 *   - Every call returns a gs_status and never aborts. On error the contents
 *     of the output buffers are unspecified; gs_last_error() returns a
 *     thread-local message describing the last failure on the calling thread.
 *   - A context is used by one host thread, and its calls go to one stream
 *     (or the caller orders the streams it uses). The server is thread safe.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_NOT_READY = 1,          /* gs_server_poll: request still in flight */
    GS_ERR_INVALID_ARG = -1,   /* bad pointer, size, alignment or option */
    GS_ERR_OOM = -2,           /* device or host allocation failed */
    GS_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    GS_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    GS_ERR_CAPACITY = -5,      /* instance list exceeded a fixed capacity */
    GS_ERR_CANCELLED = -6,     /* request cancelled or server shut down */
    GS_ERR_INTERNAL = -7       /* an internal failure: the server's scheduler stopped, or (in
                                  a GSR_DEBUG build) a device index check fired; see
                                  gs_last_error */
} gs_status;

typedef struct gs_context gs_context;
typedef struct gs_fwd_state gs_fwd_state;
typedef struct gs_graph gs_graph;
typedef struct gs_server gs_server;
typedef void *gs_stream; /* cudaStream_t */

/* Gaussians (Sec. 3: mean, rotation + scale, opacity, SH coefficients). */
typedef struct {
    int64_t n;                    /* number of Gaussians (>= 0) */
    int64_t n_pad;                /* plane stride, multiple of 4, >= n */
    int32_t sh_degree;            /* 0..3; (sh_degree+1)^2 coefficients per channel */
    int32_t _reserved;
    const float *means;           /* [3][n_pad]  x, y, z */
    const float *log_scales;      /* [3][n_pad]  log of per-axis scale */
    const float *quats;           /* [4][n_pad]  w, x, y, z, any nonzero norm */
    const float *opacity_logits;  /* [n_pad]     opacity = sigmoid(logit) */
    const float *sh;              /* [(deg+1)^2][3][n_pad], l-major, m = -l..l */
} gs_scene;

/* Pinhole camera and output resolution. */
typedef struct {
    float viewmat[12];            /* world -> camera, row-major 3x4 [R | t] */
    float fx, fy, cx, cy;         /* focal lengths and principal point, pixels */
    float near_plane;             /* Gaussians with camera z <= near are culled */
    int32_t width, height;        /* 1..65535 */
} gs_camera;

enum {
    GS_EMIT_BWD_STATE = 1u,       /* keep what gs_render_backward needs */
    GS_TIME_STAGES = 2u,          /* record CUDA events at every stage boundary (see gs_frame_stats) */
    GS_COUNT_PAIRS = 4u,          /* diagnostic: count evaluated and blended (pixel, Gaussian) pairs
                                     (plain forward only; adds a synchronisation; see gs_frame_stats) */
    GS_TIME_COMPOSITE = 8u        /* record CUDA events around the compositing stage only (stage_ms[7]):
                                     two events per frame instead of nine (ignored with GS_TIME_STAGES) */
};

typedef struct {
    int32_t tile;                 /* tile side: 8, 16 or 32; 0 = autotuned/default */
    int32_t batch;                /* Gaussians per shared-memory batch: 32/64/128/256; 0 = default */
    float bg[3];                  /* background colour */
    uint32_t flags;               /* GS_EMIT_* */
    int32_t chunk;                /* least records per chunk of a long tile list. A list longer than
                                     `head` is composited by G warps per 8x4 pixel block (8 at tile
                                     8 while lists average at most 1,024 records, else 16), one per
                                     depth-contiguous chunk of ceil(len / g) records, g = min(G,
                                     ceil(len / chunk)), merged exactly (the product rule of Eq. 2-4,
                                     the stop rule re-applied in the chunk where it falls).
                                     16..2^24, 0 = autotuned/default 512 */
    int32_t head;                 /* a list longer than this is long, >= chunk; 0 = 4 * chunk */
} gs_render_opts;

/* Caller-owned device outputs; a NULL plane is not written (and, for dcdx and
 * dcdy both NULL, the gradient recursion is not evaluated).
 * normal / nv: the normal channel the paper renders with RaDe-GS (Sec. 5.1) and the
 * normal-view inner product map its super-sampling takes (Sec. 4.1). Each Gaussian's
 * normal is its shortest axis (the smallest of the fp32 log-scales, the first of equal
 * ones), turned to face the camera (n . (mean - camera centre) < 0), in camera
 * coordinates; normal = sum n_i a_i T_i, nv = -normal . (unit ray of the pixel centre).
 * depth_isect: RaDe-GS's ray-Gaussian intersection depth (Sec. 5.1). In the EWA ray space
 * (u, v, z) of the projection (the same clamped Jacobian J), the densest point of Gaussian i
 * along the ray of pixel p is the mean of z given (u, v) = p, affine in p:
 *   z_i(p) = z_i + Sigma_{z,uv} (J W Sigma W^T J^T + 0.3 I)^-1 (p - mu2D_i),
 * Sigma_{z,uv} the covariance of camera z with (u, v); depth_isect = sum z_i(p) a_i T_i.
 * Only gs_render_forward renders these three, one warp per pixel block on every list;
 * graphs, the server, host outputs and GS_EMIT_BWD_STATE / GS_COUNT_PAIRS reject them. */
typedef struct {
    float *rgb;    /* [3][H][W] */
    float *dcdx;   /* [3][H][W]  dI/dx, Eq. 3 */
    float *dcdy;   /* [3][H][W]  dI/dy */
    float *depth;  /* [H][W]     sum z_i a_i T_i */
    float *alpha;  /* [H][W]     1 - T_final */
    float *normal; /* [3][H][W]  sum n_i a_i T_i, camera coordinates */
    float *nv;     /* [H][W]     -normal . ray */
    float *depth_isect; /* [H][W] sum z_i(p) a_i T_i, the intersection depth (above) */
} gs_outputs;

/* Per-parameter gradients, same layout and stride as gs_scene (caller-owned,
 * accumulated with +=, so the caller zeroes them). NULL planes are skipped. */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
} gs_scene_grads;

/* Read-only view of a forward state's device buffers (inspection and tests). */
typedef struct {
    int64_t n_instances;          /* K: (Gaussian, tile) pairs */
    int64_t n_visible;            /* Gaussians that survived culling */
    int32_t n_tiles, tiles_x, tiles_y, tile;
    const uint64_t *keys;         /* [K] sorted (tile << 32) | fp32 bits of depth */
    const uint32_t *vals;         /* [K] Gaussian index of each sorted key */
    const uint32_t *ranges;       /* [n_tiles][2] [start, end) into keys */
    const uint32_t *ntiles;       /* [n] tiles touched by each Gaussian (0 = culled) */
    const float *records;         /* [n][12] u', v', conic a, b, c, opacity, depth, r, g, b, rect_lo, rect_hi:
                                     rect_lo/hi = x | y << 16 (inclusive pixel rectangle, as bits);
                                     (u', v') = projected centre minus the centre (x0 + 0.5, y0 + 0.5)
                                     of the rectangle's first pixel */
    const float *final_T;         /* [H][W] (with GS_EMIT_BWD_STATE) */
    const uint32_t *n_contrib;    /* [H][W] list positions walked up to the last blended one */
} gs_state_view;

/* Counters of the frames rendered since the last reset, and (with
 * GS_TIME_STAGES) the mean per-frame device time of each stage, from CUDA
 * events recorded on the launch stream at the stage boundaries (see stage_ms). */
typedef struct {
    int64_t frames;               /* frames since the last reset */
    int64_t instances_total;      /* sum over those frames of K, the (Gaussian, tile) instances */
    int64_t visible_total;        /* sum of Gaussians that survived culling */
    int64_t instances_max;        /* largest K */
    double stage_ms[8];           /* mean device ms per frame of: projection (+ colour), block scan,
                                     visible compaction, depth sort, tile-key duplication, tile sort,
                                     tile ranges (+ work plan), compositing (all of its launches) */
    int64_t timed_frames;         /* frames that carried stage events */
    int64_t pairs_evaluated;      /* GS_COUNT_PAIRS: pixel inside a Gaussian's support rectangle, before the stop */
    int64_t pairs_blended;        /* GS_COUNT_PAIRS: of those, alpha >= 1/255 and blended */
} gs_frame_stats;

/* ---------------------------------------------------------------- context */

/* Create a render context on CUDA device `device`. The context owns its
 * workspace (per-Gaussian records, instance keys, sort buffers), grown on
 * demand with cudaMalloc and freed by gs_context_destroy. */
gs_status gs_context_create(int device, gs_context **ctx);
gs_status gs_context_destroy(gs_context *ctx);

/* Forward render (Eq. 1-4). Enqueues projection + SH colour, tile-key
 * duplication, the (tile, depth) radix sort, tile ranges and the
 * compositing+gradient pass on `stream`. It synchronises `stream` once,
 * after the instance count is known, to size the sort buffers.
 * If `state` is non-NULL a gs_fwd_state is returned that owns the buffers the
 * backward pass needs (free with gs_state_free); GS_EMIT_BWD_STATE must be set.
 * Errors: GS_ERR_INVALID_ARG (NULL scene/camera/opts/outputs, misaligned or
 * negative sizes, unsupported tile/batch/degree), GS_ERR_OOM, GS_ERR_CUDA,
 * GS_ERR_TIMEOUT (a bounded device wait gave up: the sort's lookback or a
 * compositing batch wait). The sort and compositing run after the call's one
 * synchronisation, so their device errors are kept in the context and
 * reported by the next call that synchronises: the next gs_render_forward
 * (which then renders nothing and returns the error) or gs_context_check. The
 * outputs of a frame whose wait gave up are unspecified; nothing is read or
 * written out of bounds, and the context stays usable. */
gs_status gs_render_forward(gs_context *ctx, const gs_scene *scene, const gs_camera *cam,
                            const gs_render_opts *opts, const gs_outputs *out, gs_fwd_state **state,
                            gs_stream stream);

/* Same as gs_render_forward, but the outputs are HOST buffers (pinned memory
 * recommended): the call renders into context-owned device planes, copies
 * them to the host and synchronises `stream` before returning. */
gs_status gs_render_forward_to_host(gs_context *ctx, const gs_scene *scene, const gs_camera *cam,
                                    const gs_render_opts *opts, const gs_outputs *host_out,
                                    gs_stream stream);

/* Backward of gs_render_forward: the reverse walk of Eq. 2-4 with the upstream
 * gradients of rgb, dcdx, dcdy, depth and alpha (`grad_in` planes, device,
 * same layout as the outputs; NULL = zero), then the chain rule to means,
 * log-scales, quaternions, opacity logits and SH coefficients. Adds into
 * `grads` (caller zeroes). `scene` must be the one given to the forward.
 * Errors: GS_ERR_INVALID_ARG (state without GS_EMIT_BWD_STATE, NULL args),
 * GS_ERR_CUDA. */
gs_status gs_render_backward(gs_context *ctx, const gs_fwd_state *state, const gs_scene *scene,
                             const gs_outputs *grad_in, const gs_scene_grads *grads, gs_stream stream);

gs_status gs_state_view_get(const gs_fwd_state *state, gs_state_view *view);
/* Synchronises `stream` and returns the device error status of the plain
 * forward frames rendered on the context since the last report (GS_OK, or
 * GS_ERR_TIMEOUT when a bounded wait gave up), then clears it. */
gs_status gs_context_check(gs_context *ctx, gs_stream stream);
/* Diagnostic for testing the failure path without a stuck GPU: with
 * give_up = 1, every bounded device wait of the context's later plain forwards
 * gives up at once instead of after its ~4M polls (each radix-sort and
 * duplication lookback before its first look, each warp's first compositing
 * batch wait before its first poll; a warp that gave up still waits, with the
 * normal bound, for the copies it has in flight). A sort that gave up leaves
 * nothing planned, so compositing then waits on nothing; give_up = 2 makes only
 * the compositing batch waits give up, which are polled in the frames that
 * stage batches by TMA bulk copies (those with the normal channels; the others
 * gather with cp.async and have no poll). Those frames report GS_ERR_TIMEOUT
 * through gs_context_check; 0 restores the normal bound. Other values:
 * GS_ERR_INVALID_ARG. */
gs_status gs_context_debug_waits(gs_context *ctx, int32_t give_up);
/* Synchronises `stream` and returns the context's frame statistics (plain
 * forward calls); `reset` != 0 clears them afterwards. */
gs_status gs_context_stats(gs_context *ctx, gs_stream stream, int reset, gs_frame_stats *stats);
gs_status gs_state_free(gs_fwd_state *state);

/* ---------------------------------------------------------------- CUDA graphs
 * A graph replays the whole forward (same scene, resolution, options and
 * output buffers) with a new camera per frame and no host synchronisation.
 * The instance buffers have a fixed `capacity` (0 = 4 * n); a frame whose
 * instance count exceeds it renders incompletely and is reported by
 * gs_graph_check as GS_ERR_CAPACITY. */
gs_status gs_graph_create(gs_context *ctx, const gs_scene *scene, const gs_camera *cam,
                          const gs_render_opts *opts, const gs_outputs *out, int64_t capacity,
                          gs_stream stream, gs_graph **graph);
/* Replay with camera `cam` (same width/height as at creation). Asynchronous. */
gs_status gs_graph_render(gs_graph *graph, const gs_camera *cam, gs_stream stream);
/* Synchronises `stream`; GS_ERR_CAPACITY if any replay since the last check
 * overflowed; `max_instances` (nullable) receives the largest count seen. */
gs_status gs_graph_check(gs_graph *graph, gs_stream stream, int64_t *max_instances);
/* Synchronises `stream` and returns the statistics of the replays since the
 * last reset (stage times if the graph was created with GS_TIME_STAGES);
 * returns the replays' error status like gs_graph_check. */
gs_status gs_graph_stats(gs_graph *graph, gs_stream stream, int reset, gs_frame_stats *stats);
gs_status gs_graph_destroy(gs_graph *graph);

/* ---------------------------------------------------------------- frames in flight
 * A frame stream renders a camera sequence with `slots` frames in flight: one captured
 * graph (as gs_graph_create) and one high-priority stream per slot. Frame f (numbered
 * from 0 in submission order) goes to slot f % slots and renders into that slot's device
 * planes. Consecutive frames are independent, so one frame's compositing runs beside
 * the next frames' projection and sorts.
 *
 * outs: `slots` caller-owned device output sets (W x H of cam0, fp32, the layouts of
 *   gs_outputs; each non-NULL plane is rendered, and every set names the same planes;
 *   the RaDe-GS channels are not rendered here). They must outlive the stream.
 * opts, capacity: as gs_graph_create (capacity 0 = 4 N); timing flags apply to every slot.
 *
 * submit: enqueues the frame with camera `cam` (the resolution of cam0) and returns its
 *   number in *frame. If `host` is not NULL, each of its non-NULL planes receives a copy
 *   of the same device plane (cudaMemcpyAsync on the slot's stream, after the render;
 *   pinned host memory lets it overlap, pageable memory makes it synchronous). Slot k
 *   renders again only after its previous frame's copies and any release (below). The
 *   call does not wait for the GPU.
 * join: makes stream `consumer` wait until frame f has rendered (and its host copies are done).
 * release: frame f's slot renders its next frame only after the work enqueued on
 *   `consumer` so far (the consumer's reads of the frame's planes). Without a release, the
 *   slot is rewritten `slots` frames later, stream-ordered after its own earlier work.
 * wait: the host waits for frame f (its render and copies).
 * For join, release and wait, f must be among the last `slots` submitted frames
 * (GS_ERR_INVALID_ARG otherwise).
 * synchronize: waits for every submitted frame; returns the first error any slot's frames
 *   raised since the last call (GS_ERR_CAPACITY for instances beyond capacity,
 *   GS_ERR_TIMEOUT for a bounded wait that gave up), like gs_graph_check.
 * stats: gs_graph_stats of slot `slot`.
 * destroy: waits for every frame, then frees the graphs, streams and events (not outs). */
typedef struct gs_frame_stream gs_frame_stream;
gs_status gs_frame_stream_create(gs_context *ctx, const gs_scene *scene, const gs_camera *cam0,
                                 const gs_render_opts *opts, const gs_outputs *outs, int32_t slots,
                                 int64_t capacity, gs_frame_stream **fs);
gs_status gs_frame_stream_submit(gs_frame_stream *fs, const gs_camera *cam, const gs_outputs *host,
                                 int64_t *frame);
gs_status gs_frame_stream_join(gs_frame_stream *fs, int64_t frame, gs_stream consumer);
gs_status gs_frame_stream_release(gs_frame_stream *fs, int64_t frame, gs_stream consumer);
gs_status gs_frame_stream_wait(gs_frame_stream *fs, int64_t frame);
gs_status gs_frame_stream_synchronize(gs_frame_stream *fs);
gs_status gs_frame_stream_stats(gs_frame_stream *fs, int32_t slot, int reset, gs_frame_stats *stats);
gs_status gs_frame_stream_destroy(gs_frame_stream *fs);

/* ---------------------------------------------------------------- autotuner
 * Times the render for every tile in {8, 16, 32}, batch in {32, 64, 128, 256}
 * (pairs whose per-warp staging rings fit shared memory) and chunk in
 * {256, 512, 1024}: one plain forward gives the configuration's instance count,
 * which sizes a graph (as gs_graph_create), whose replays of `cam` are timed
 * (CUDA events, `iters` frames one at a time, after one warm-up). It
 * records the fastest in the context's cache, keyed by (W, H, N bucket, SH
 * degree); later calls with tile / batch / chunk = 0 use it. Synchronous.
 * Any output pointer may be NULL. */
gs_status gs_autotune(gs_context *ctx, const gs_scene *scene, const gs_camera *cam,
                      const gs_outputs *out, int iters, gs_stream stream, int32_t *best_tile,
                      int32_t *best_batch, int32_t *best_chunk, float *best_ms);

/* ---------------------------------------------------------------- serving
 * Continuous batching over resident scenes: requests (scene, camera, options,
 * caller-owned device outputs) are queued by gs_server_submit; a scheduler
 * thread admits them as in-flight slots and sort-buffer memory free up,
 * projects and sorts each on its own stream, and composites every ready
 * request's tiles in one persistent launch driven by a (request, tile) work
 * list, so new requests' preparation overlaps other requests' compositing. */
gs_status gs_server_create(int device, size_t sort_budget_bytes, int max_inflight, gs_server **srv);
/* Copies the scene (device pointers) into server-owned memory. */
gs_status gs_server_load_scene(gs_server *srv, const gs_scene *scene, int32_t *scene_id);
gs_status gs_server_submit(gs_server *srv, int32_t scene_id, const gs_camera *cam,
                           const gs_render_opts *opts, const gs_outputs *out, uint64_t *req_id);
/* GS_OK (done, latency in ms since submit), GS_NOT_READY, or the request's
 * error. A finished request is forgotten after the first GS_OK/error poll. */
gs_status gs_server_poll(gs_server *srv, uint64_t req_id, double *latency_ms);
gs_status gs_server_cancel(gs_server *srv, uint64_t req_id);
/* Blocks until every submitted request has finished. */
gs_status gs_server_drain(gs_server *srv);
gs_status gs_server_destroy(gs_server *srv);

/* ---------------------------------------------------------------- sorting without allocation
 * No counterpart in the paper: an entry point for callers that cannot call
 * cudaMalloc -- a host framework whose caching allocator owns all of the
 * device's memory, or a real-time loop that must not allocate after start-up
 * (cudaMalloc can synchronise the device and take milliseconds).
 * Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of the
 * key -- the same onesweep kernels that sort the render's (tile, depth) keys.
 * keys_in/vals_in (device, read only) are sorted into keys_out/vals_out
 * (device, caller-owned; may alias the inputs). Keys 8-byte and values 4-byte
 * aligned. Asynchronous on `stream`.
 * Scratch comes from one static device array of about 14 MB that the library
 * image holds on every GPU it is loaded on, until the process exits; n is at
 * most 1,048,576 (GS_ERR_INVALID_ARG beyond). It allocates nothing: the first
 * call on a device looks up the array's device address once, so make that
 * first call before any stream capture. Every call reuses the same array:
 * calls whose work overlaps on the GPU race and must be ordered by the caller.
 * status (nullable, device, 4-byte aligned): receives, in stream order, the
 * call's device error bits -- 0, or nonzero when a bounded lookback wait gave
 * up and the output is not sorted (the sort never waits without bound). */
gs_status gs_sort_pairs_static(const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out,
                               uint32_t *vals_out, int64_t n, int32_t bits, uint32_t *status, gs_stream stream);

/* ---------------------------------------------------------------- frame-interpolation warp
 * The geometric half of the paper's frame interpolation (Sec. 4.2, "Forward-
 * Backward Warping"), applied to one rendered source frame toward one target
 * camera (the forward-backward scheme calls it twice: frame 0 and frame 1,
 * each toward the intermediate pose):
 *   motion  V[x] = Proj(UnProj(x, D[x], P_src), P_dst) - x               (Sec. 4.2)
 *   warp    w(F, V): every moving source pixel lands on the target pixel that
 *           contains x + V[x]; among several, the one nearest the target camera
 *           wins (target-camera z, ties to the smaller source index j*W+i); a
 *           target pixel nobody reaches is a hole (index -1, planes 0)
 *   warped gradient  G_dst = w(G_src, V) . (I + dV/dx)^-1                (Sec. 4.2)
 *           (the row vector of source image gradients times the inverse of
 *           the landing map's Jacobian, taken by central differences over the
 *           source pixel grid, one-sided where a neighbour does not move, the
 *           identity where neither does; 0 where the determinant is <= 0)
 * UnProj lifts pixel centre (i + 0.5, j + 0.5) to source-camera z = D, where
 * D = depth / alpha (the render's depth channel is alpha-weighted) and a pixel
 * moves only where alpha > alpha_min and its target-camera z exceeds the target
 * camera's near_plane. With alpha == NULL, depth is a point depth and a pixel
 * moves where it is > 0. The landing position, the depth test and the motion
 * map follow one fixed fp32 round-to-nearest operation sequence (exactly
 * reproducible); the Jacobian and the gradient product are fp32 with
 * compensated 2x2 determinants. Depth must be finite.
 * Layouts: source planes [c][H][W], target planes [c][Ht][Wt], fp32, device,
 * caller-owned, 4-byte aligned; (W, H) and (Wt, Ht) are the cameras' sizes. */
typedef struct {
    const float *depth;           /* [H][W] alpha-weighted depth (or point depth when alpha is NULL) */
    const float *alpha;           /* [H][W] nullable */
    float alpha_min;              /* a pixel moves only where alpha > alpha_min */
    int32_t channels;             /* planes carried by the warp (colour, depth, normals ...), 0..64 */
    const float *planes;          /* [channels][H][W] */
    int32_t grad_channels;        /* image-gradient channels, 0..64 */
    const float *dcdx, *dcdy;     /* [grad_channels][H][W] dI/dx, dI/dy of the source frame */
} gs_warp_input;

typedef struct {                  /* every plane nullable (NULL = not written) */
    float *motion;                /* [2][H][W]   V (x then y), NaN where the pixel does not move */
    int32_t *index;               /* [Ht][Wt]    winning source pixel j*W+i, -1 for a hole */
    float *z;                     /* [Ht][Wt]    the winner's target-camera z, 0 for a hole */
    float *planes;                /* [channels][Ht][Wt] */
    float *dcdx, *dcdy;           /* [grad_channels][Ht][Wt] warped gradient */
} gs_warp_output;

/* Motion vectors, depth-tested forward warp and warped gradient of one source
 * frame (above). Two kernel launches on `stream`, asynchronous. The context
 * owns the scratch (a 64-bit depth-test slot per target pixel, kept all ones
 * between calls, and a landing position per source pixel), grown with
 * cudaMalloc on demand; calls on one context must be ordered on the GPU.
 * Errors: GS_ERR_INVALID_ARG (NULL context/cameras/input/output/depth, camera
 * sizes outside 1..65535, negative target near_plane, channel counts outside
 * 0..64, gradients asked for without both input and output planes, misaligned
 * planes), GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_warp(gs_context *ctx, const gs_camera *src, const gs_camera *dst, const gs_warp_input *in,
                  const gs_warp_output *out, gs_stream stream);

/* ---------------------------------------------------------------- gradient-aware interpolation
 * The interpolation step of the paper's super-sampling (Sec. 4.1, "Gradient-Aware
 * Interpolation", Eq. 5-8), applied to the render's outputs: each low-resolution pixel's
 * S x S high-resolution block is a linear map of its 3x3 neighbourhood's colour and
 * analytic gradients (Eq. 7),
 *   Vec(I_SxS) = M [Vec(I_3x3); Vec(dI/dx_3x3); Vec(dI/dy_3x3)] + b.
 * Vec is column-wise: input 9 q + 3 (i + 1) + (j + 1) is plane q (0 colour, 1 dI/dx,
 * 2 dI/dy) at node (x0 + i, y0 + j), and output u S + v is the high-resolution pixel
 * (S x0 + u, S y0 + v). Nodes outside the image read 0.
 * The weights come as the paper's two layers (Eq. 8): a 3x3 convolution to `features`
 * channels (wc, bc) and an SxS stride-S transposed convolution (wt, bt). The call folds
 * them, in double, into M = wt wc and b = wt bc + bt, and evaluates M x + b in fp32. The
 * same weights serve every colour channel. The paper's refinement network (GTRR) is not
 * part of this call. */
typedef struct {
    int32_t scale;                /* S: 2, 3 or 4 */
    int32_t features;             /* C, the feature channels between the layers: 1..1024 */
    const float *wc;              /* [C][27] host, row-major (convolution weights) */
    const float *bc;              /* [C] host, nullable = 0 */
    const float *wt;              /* [S*S][C] host, row-major (transposed-convolution weights) */
    const float *bt;              /* [S*S] host, nullable = 0 */
} gs_gai_weights;

/* Super-samples `channels` planes of W x H (rgb, dcdx, dcdy: device, [channels][H][W]
 * fp32, caller-owned, 4-byte aligned) into out ([channels][S H][S W] fp32, device,
 * caller-owned, 16-byte aligned). One kernel launch on `stream` (current CUDA device),
 * asynchronous; the weights are read on the host during the call. Allocates nothing.
 * Errors: GS_ERR_INVALID_ARG (NULL weights or planes, scale not 2..4, features not
 * 1..1024, channels not 1..64, sizes outside 1..65535, misaligned planes), GS_ERR_CUDA. */
gs_status gs_gai_upsample(const gs_gai_weights *w, const float *rgb, const float *dcdx, const float *dcdy,
                          int32_t channels, int32_t width, int32_t height, float *out, gs_stream stream);

/* ---------------------------------------------------------------- misc */
const char *gs_last_error(void);
const char *gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
