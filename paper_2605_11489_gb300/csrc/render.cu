// Render core: workspace management, the forward launch sequence, the
// backward, CUDA-graph replay, the autotuner, and the C ABI entry points of
// include/gsr.h (except serving, in server.cu).
//
// Forward launch sequence on one stream (paper Sec. 3: project, depth-sort,
// alpha-blend; plus the Eq. 3-4 gradient channels):
//   K1 project+SH  ->  K2 scan of per-block tile counts  ->  [read K]  ->
//   K3 duplicate (tile, depth) keys  ->  K4 radix sort  ->  K5 tile ranges  ->
//   K6 composite + gradients + depth + alpha
// The plain path reads the instance count K back once (one stream sync) to size
// the sort buffers. The graph path keeps K on the device, with buffers of a
// fixed capacity and an overflow bit, so a whole frame replays with no sync.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gsr_internal.cuh"

namespace gsr {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

gs_status fail(gs_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

gs_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

const void *project_kernel_ptr(int deg, int which);  // project.cu: 0 projection, 1 colour

namespace {

constexpr int64_t kMaxInstances = (1ll << 30) - 1;  // sort status words hold 30-bit counts

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    ~Buf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes && p) return cudaSuccess;
        release();
        size_t sz = std::max<size_t>(want + want / 4, 256);
        cudaError_t e = cudaMalloc(&p, sz);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = sz;
        return cudaSuccess;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// A second stream and its fork / join events: the long tiles are composited on it,
// beside the short ones on the launch stream (also inside a graph capture, where
// the events make the fork and join edges).
struct ForkJoin {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ForkJoin() = default;
    ForkJoin(const ForkJoin &) = delete;
    ForkJoin &operator=(const ForkJoin &) = delete;
    ~ForkJoin()
    {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
    }
    cudaError_t ensure()
    {
        cudaError_t e = cudaSuccess;
        if (!s && (e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if (!fork && (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if (!join && (e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) != cudaSuccess) return e;
        return e;
    }
};

// All per-frame device buffers. Owned by a context (pooled), a state or a graph.
struct Frame {
    Buf rec, bin, ntiles, bsums, boffs;
    Buf keys[2], vals[2], sort_scr, rec_sorted;     // tile keys (u32) and Gaussian indices, per instance
    Buf dkeys[2], dvals[2], vsums, voffs, dlook;  // depth order of the visible Gaussians
    Buf keys64;                                     // (tile << 32 | depth bits) per instance, for a state view
    Buf ranges, order;
    Buf plan;             // (n_long, long-tile work counter, n_short): launch_plan
    int chunk = 512;      // least records per chunk of a long tile list
    int head = 4 * 512;   // a list longer than this is a long tile
    int64_t max_long = 0; // long tiles the frame's capacity allows (0: none composited apart)
    int long_bpc = 2;     // pixel blocks per long-tile CTA (composite.cu)
    ForkJoin fork;        // the long tiles' stream beside the launch stream
    Buf fT, fTx, fTy, ncontrib;
    Buf nrm, nrm_sorted;      // the normal channel: per Gaussian, then in sorted (instance) order
    Buf plane, plane_sorted;  // the intersection depth's slopes, likewise
    bool want_nrm = false;
    Buf counters;
    int64_t n = 0, K = 0, key_cap = 0;
    int sorted = 0;
    int W = 0, H = 0, tile = 16, batch = 64, tiles_x = 0, tiles_y = 0, n_tiles = 0, bits = 32;
    int deg = 0;
    float bg[3] = {0, 0, 0};
    CamParams cam{};
    bool has_state = false;
    bool count_pairs = false;
    // device word the sort and compositing kernels raise their error bits in: the
    // context's sticky word for plain frames, the frame's counters for graphs
    uint32_t *err_word = nullptr;
    bool give_up = false;            // diagnostic: the sorts' and duplication's lookbacks give up at once
    bool give_up_composite = false;  // diagnostic: compositing's first batch wait gives up at once
};

// Per-stage CUDA-event timer: a ring of event sets, one set of kBounds events
// per frame, recorded at the stage boundaries on the launch stream (plain
// path) or retargeted into a graph's event-record nodes before each replay.
struct StageTimer {
    static constexpr int kBounds = 9;  // before K1 | K1 | K2 | K3a | K4a | K3b | K4b | K5+plan | K6
    static constexpr uint32_t kAll = (1u << kBounds) - 1u;
    static constexpr uint32_t kCompositeOnly = (1u << 7) | (1u << 8);  // around K6 only: two events
    static constexpr int kRing = 512;
    std::vector<cudaEvent_t> ev;
    std::vector<uint32_t> slot_mask;  // which bounds each slot's frame recorded
    int head = 0;
    int64_t in_ring = 0;  // recorded slots not yet folded
    double sum_ms[kBounds - 1] = {};
    int64_t folded = 0;
    ~StageTimer()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    cudaError_t init()
    {
        if (!ev.empty()) return cudaSuccess;
        ev.resize((size_t)kRing * kBounds, nullptr);
        slot_mask.assign(kRing, 0u);
        for (auto &e : ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    void fold(int slot)
    {
        cudaEvent_t *e = &ev[(size_t)slot * kBounds];
        const uint32_t m = slot_mask[slot];
        if (!m) return;
        cudaEventSynchronize(e[31 - __builtin_clz(m)]);
        bool ok = true;
        float ms[kBounds - 1] = {};
        for (int k = 0; k < kBounds - 1 && ok; ++k)
            if ((m >> k & 1u) && (m >> (k + 1) & 1u)) ok = cudaEventElapsedTime(&ms[k], e[k], e[k + 1]) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();  // do not leave the failure for the next launch check
            return;
        }
        for (int k = 0; k < kBounds - 1; ++k) sum_ms[k] += ms[k];
        ++folded;
    }
    // events of the next frame slot, recording the bounds in `mask` (the
    // slot's previous frame is folded first)
    cudaEvent_t *next(uint32_t mask = kAll)
    {
        if (in_ring == kRing) {
            fold(head);
            --in_ring;
        }
        cudaEvent_t *e = &ev[(size_t)head * kBounds];
        slot_mask[head] = mask;
        head = (head + 1) % kRing;
        ++in_ring;
        return e;
    }
    void collect(double *ms, int64_t *frames)
    {
        int slot = (head - (int)in_ring + kRing) % kRing;
        for (int64_t k = 0; k < in_ring; ++k, slot = (slot + 1) % kRing) fold(slot);
        in_ring = 0;
        for (int k = 0; k < kBounds - 1; ++k) ms[k] = folded ? sum_ms[k] / folded : 0.0;
        *frames = folded;
    }
    void reset()
    {
        in_ring = 0;
        folded = 0;
        for (double &v : sum_ms) v = 0;
    }
};

// Stage-boundary events of one frame: `ev` (nullptr = untimed), the bounds
// recorded, and whether the stream is being captured (external event nodes).
struct Marks {
    cudaEvent_t *ev = nullptr;
    uint32_t mask = 0;
    bool capture = false;
};

uint32_t timing_mask(uint32_t flags)
{
    if (flags & GS_TIME_STAGES) return StageTimer::kAll;
    if (flags & GS_TIME_COMPOSITE) return StageTimer::kCompositeOnly;
    return 0u;
}

}  // namespace

int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

CamParams make_cam(const gs_camera &c, int tile)
{
    CamParams p{};
    for (int k = 0; k < 12; ++k) p.vm[k] = c.viewmat[k];
    p.fx = c.fx;
    p.fy = c.fy;
    p.cx = c.cx;
    p.cy = c.cy;
    p.near_plane = c.near_plane;
    for (int k = 0; k < 3; ++k) {
        // camera centre -R^T t, in double then rounded
        const double v = -((double)c.viewmat[k] * c.viewmat[3] + (double)c.viewmat[4 + k] * c.viewmat[7] +
                           (double)c.viewmat[8 + k] * c.viewmat[11]);
        p.campos[k] = (float)v;
    }
    p.width = c.width;
    p.height = c.height;
    // the Jacobian guard, 1.3 x the half field of view in x/z and y/z, by the discrete spec's
    // fp32 sequence (products and quotients only, so no contraction can change it)
    const volatile float hw = 0.5f * (float)c.width, hh = 0.5f * (float)c.height;
    const volatile float qx = hw / c.fx, qy = hh / c.fy;
    p.limx = 1.29999995f * qx;
    p.limy = 1.29999995f * qy;
    p.tile_shift = ilog2(tile);
    p.tiles_x = (c.width + tile - 1) / tile;
    p.tiles_y = (c.height + tile - 1) / tile;
    return p;
}

gs_status check_scene(const gs_scene *s)
{
    if (!s) return fail(GS_ERR_INVALID_ARG, "scene is NULL");
    if (s->n < 0 || s->n_pad < s->n || (s->n_pad & 3)) return fail(GS_ERR_INVALID_ARG, "need 0 <= n <= n_pad, n_pad % 4 == 0");
    if (s->n > 0xFFFFFFFFll) return fail(GS_ERR_INVALID_ARG, "n exceeds 2^32 - 1");
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (s->n == 0) return GS_OK;
    const void *ps[5] = {s->means, s->log_scales, s->quats, s->opacity_logits, s->sh};
    for (const void *p : ps) {
        if (!p) return fail(GS_ERR_INVALID_ARG, "scene plane pointer is NULL");
        if (reinterpret_cast<uintptr_t>(p) & 15) return fail(GS_ERR_INVALID_ARG, "scene planes must be 16-byte aligned");
    }
    return GS_OK;
}

gs_status check_cam(const gs_camera *c)
{
    if (!c) return fail(GS_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 65535 || c->height > 65535)
        return fail(GS_ERR_INVALID_ARG, "width/height must be in 1..65535");
    if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(GS_ERR_INVALID_ARG, "fx, fy must be > 0");
    return GS_OK;
}

struct TuneKey {
    int W, H, nb, deg;
    bool operator<(const TuneKey &o) const { return std::tie(W, H, nb, deg) < std::tie(o.W, o.H, o.nb, o.deg); }
};

}  // namespace gsr

using namespace gsr;

struct gs_context {
    int device = 0;
    std::vector<Frame *> pool;
    uint32_t *h_counters = nullptr;  // pinned: kCntSlots words, then the sticky error word's copy
    Buf err;                         // device: error bits of plain frames, kept until reported
    int give_up = 0;                 // gs_context_debug_waits: 0, 1 (every wait) or 2 (compositing's)
    Buf g2d;
    Buf host_planes;
    Buf warp_pos, warp_best;    // frame-interpolation warp: landing positions, depth-test slots
    bool warp_best_clean = false;  // warp_best holds all ones (every slot empty)
    struct Tuned {
        int tile, batch, chunk;
    };
    std::map<TuneKey, Tuned> tune;
    StageTimer timer;
    int64_t st_frames = 0, st_sum_k = 0, st_sum_v = 0, st_max_k = 0, st_pairs_eval = 0, st_pairs_blend = 0;
    ~gs_context()
    {
        for (Frame *f : pool) delete f;
        if (h_counters) cudaFreeHost(h_counters);
    }
    Frame *acquire()
    {
        if (pool.empty()) return new Frame();
        Frame *f = pool.back();
        pool.pop_back();
        return f;
    }
    void give_back(Frame *f) { pool.push_back(f); }
};

struct gs_fwd_state {
    gs_context *ctx = nullptr;
    Frame *f = nullptr;
    int64_t n = 0, n_pad = 0;
};

struct gs_graph {
    gs_context *ctx = nullptr;
    Frame *f = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t proj_node = nullptr, colour_node = nullptr;  // the camera-dependent kernels
    ProjectArgs proj_args{};
    int64_t capacity = 0;
    int tile = 16;
    cudaStream_t cap_stream = nullptr;
    bool timed = false;
    StageTimer timer;
    cudaGraphNode_t ev_node[StageTimer::kBounds] = {};
    uint32_t mark_mask = 0;  // stage bounds the graph records
};

namespace gsr {
namespace {

constexpr int kDefaultTile = 16, kDefaultBatch = 32, kDefaultChunk = 512;
// average records per tile (capacity / tiles) up to which a tile-8 long-tile CTA takes the
// whole tile
constexpr int64_t kLongBpcAvgMax = 1024;

// tile / batch / chunk: explicit options win, then the autotuner's cache for
// (W, H, N bucket, SH degree), then the defaults.
void pick_config(gs_context *ctx, const gs_scene *s, const gs_camera *c, const gs_render_opts *o, int *tile,
                 int *batch, int *chunk)
{
    int t = o->tile, b = o->batch, k = o->chunk;
    if (t == 0 || b == 0 || k == 0) {
        const int nb = s->n > 0 ? (int)std::log2((double)s->n) : 0;
        auto it = ctx->tune.find(TuneKey{c->width, c->height, nb, s->sh_degree});
        if (it != ctx->tune.end()) {
            if (t == 0) t = it->second.tile;
            if (b == 0) b = it->second.batch;
            if (k == 0) k = it->second.chunk;
        }
    }
    *tile = t ? t : kDefaultTile;
    *batch = b ? b : kDefaultBatch;
    *chunk = k ? k : kDefaultChunk;
}

// Per-Gaussian and per-pixel buffers + geometry of a frame.
gs_status frame_setup(Frame *f, const gs_scene *s, const gs_camera *c, const gs_render_opts *o, int tile, int batch,
                      int chunk, bool state)
{
    f->n = s->n;
    f->W = c->width;
    f->H = c->height;
    f->tile = tile;
    f->batch = batch;
    if (chunk < 16 || chunk > (1 << 24)) return fail(GS_ERR_INVALID_ARG, "chunk must be 0 or 16..2^24");
    const int64_t head = o->head ? (int64_t)o->head : (int64_t)kHeadChunks * chunk;
    if (head < chunk || head > (1ll << 30)) return fail(GS_ERR_INVALID_ARG, "head must be 0 or chunk..2^30");
    f->chunk = chunk;
    f->head = (int)head;
    f->want_nrm = false;
    f->deg = s->sh_degree;
    for (int k = 0; k < 3; ++k) f->bg[k] = o->bg[k];
    f->cam = make_cam(*c, tile);
    f->tiles_x = f->cam.tiles_x;
    f->tiles_y = f->cam.tiles_y;
    f->n_tiles = f->tiles_x * f->tiles_y;
    f->bits = 32 + ilog2(std::max(f->n_tiles, 1));
    const int64_t n4 = (s->n + 3) / 4 * 4;
    const int nb = project_blocks(s->n);
    GSR_CUDA(f->rec.ensure(sizeof(GaussRec) * (size_t)std::max<int64_t>(s->n, 1)));
    GSR_CUDA(f->bin.ensure(sizeof(uint4) * (size_t)std::max<int64_t>(s->n, 1)));
    GSR_CUDA(f->ntiles.ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(n4, 4)));
    GSR_CUDA(f->bsums.ensure(sizeof(uint32_t) * (size_t)std::max(nb, 1)));
    GSR_CUDA(f->boffs.ensure(sizeof(uint32_t) * (size_t)std::max(nb, 1)));
    for (int k = 0; k < 2; ++k) {
        GSR_CUDA(f->dkeys[k].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(s->n, 1)));
        GSR_CUDA(f->dvals[k].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(s->n, 1)));
    }
    GSR_CUDA(f->vsums.ensure(sizeof(uint32_t) * (size_t)std::max(nb, 1)));
    GSR_CUDA(f->voffs.ensure(sizeof(uint32_t) * (size_t)std::max(nb, 1)));
    GSR_CUDA(f->dlook.ensure(duplicate_look_bytes(std::max<int64_t>(s->n, 1))));
    GSR_CUDA(f->ranges.ensure(sizeof(uint2) * (size_t)f->n_tiles));
    GSR_CUDA(f->order.ensure(sizeof(uint32_t) * (size_t)f->n_tiles));
    GSR_CUDA(f->counters.ensure(sizeof(uint32_t) * kCntSlots));
    const size_t hw = (size_t)f->W * f->H;
    if (state) {
        GSR_CUDA(f->fT.ensure(sizeof(float) * hw));
        GSR_CUDA(f->fTx.ensure(sizeof(float) * hw));
        GSR_CUDA(f->fTy.ensure(sizeof(float) * hw));
        GSR_CUDA(f->ncontrib.ensure(sizeof(uint32_t) * hw));
    }
    f->has_state = state;
    return GS_OK;
}

gs_status frame_keys(Frame *f, int64_t cap)
{
    GSR_CUDA(f->keys[0].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(cap, 1)));
    GSR_CUDA(f->keys[1].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(cap, 1)));
    GSR_CUDA(f->vals[0].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(cap, 1)));
    GSR_CUDA(f->vals[1].ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(cap, 1)));
    f->key_cap = cap;
    return GS_OK;
}

// Plan and sort buffers for up to `cap` instances. At most cap / (head + 1) tiles
// have lists longer than head.
gs_status frame_plan(Frame *f, int64_t cap)
{
    f->max_long = f->head >= (1 << 30) ? 0 : std::min<int64_t>(f->n_tiles, cap / ((int64_t)f->head + 1) + 1);
    // a long-tile CTA takes a whole 8x8 tile (8 chunk warps per block) while lists hold a few
    // hundred records on average; with longer lists, and at larger tiles, one block (16)
    f->long_bpc = (f->tile == 8 && cap <= kLongBpcAvgMax * (int64_t)f->n_tiles) ? 2 : 1;
    GSR_CUDA(f->plan.ensure(sizeof(uint32_t) * 3));
    if (f->max_long > 0) GSR_CUDA(f->fork.ensure());
    if (f->has_state) GSR_CUDA(f->keys64.ensure(sizeof(uint64_t) * (size_t)std::max<int64_t>(cap, 1)));
    // one scratch serves both sorts (they run one after the other): sized for
    // the larger of the instance capacity and the Gaussian count
    GSR_CUDA(f->sort_scr.ensure(sort_scratch_bytes(std::max<int64_t>(std::max<int64_t>(cap, f->n), 1))));
    return GS_OK;
}

ProjectArgs proj_args(Frame *f, const gs_scene *s)
{
    ProjectArgs a{};
    a.means = s->means;
    a.log_scales = s->log_scales;
    a.quats = s->quats;
    a.logits = s->opacity_logits;
    a.sh = s->sh;
    a.n = s->n;
    a.n_pad = s->n_pad;
    a.deg = s->sh_degree;
    a.cam = f->cam;
    a.rec = f->rec.as<GaussRec>();
    a.bin = f->bin.as<uint4>();
    a.ntiles = f->ntiles.as<uint32_t>();
    a.block_sums = f->bsums.as<uint32_t>();
    a.block_vis = f->vsums.as<uint32_t>();
    a.counters = f->counters.as<uint32_t>();
    if (f->want_nrm) {
        a.nrm = f->nrm.as<float4>();
        a.plane = f->plane.as<float2>();
    }
    return a;
}

// A frame without the normal channels composites from the records by Gaussian index, each
// warp gathering its batches through the sorted indices, so K5 does not copy the records
// into instance order (the backward reads them by index too). The normal channels' K5 pass
// gathers the sorted normals and slopes, and the records with them.
bool gather_records(const Frame *f) { return !f->want_nrm; }

CompositeArgs comp_args(Frame *f, const gs_outputs *out)
{
    CompositeArgs c{};
    c.vals = f->vals[f->sorted].as<uint32_t>();
    if (gather_records(f)) {
        c.rec_index = f->rec.as<GaussRec>();
        c.n_gauss = (uint32_t)std::max<int64_t>(f->n, 1);
    } else {
        c.rec = f->rec_sorted.as<GaussRec>();
    }
    c.ranges = f->ranges.as<uint2>();
    c.width = f->W;
    c.height = f->H;
    c.tiles_x = f->tiles_x;
    c.tiles_y = f->tiles_y;
    for (int k = 0; k < 3; ++k) c.bg[k] = f->bg[k];
    c.rgb = out->rgb;
    c.dcdx = out->dcdx;
    c.dcdy = out->dcdy;
    c.depth = out->depth;
    c.alpha = out->alpha;
    if (f->has_state) {
        c.final_T = f->fT.as<float>();
        c.final_Tx = f->fTx.as<float>();
        c.final_Ty = f->fTy.as<float>();
        c.n_contrib = f->ncontrib.as<uint32_t>();
    }
    c.err_word = f->err_word ? f->err_word : f->counters.as<uint32_t>() + kCntErr;
    c.give_up = f->give_up_composite ? 1u : 0u;
    c.tile_order = f->order.as<uint32_t>();
    c.plan = f->plan.as<uint32_t>();
    c.long_counter = f->plan.as<uint32_t>() + 1;
    c.long_bpc = f->long_bpc;
    c.chunk = f->chunk;
    if (f->count_pairs) c.pair_counts = reinterpret_cast<unsigned long long *>(f->counters.as<uint32_t>() + kCntPairs);
    if (f->want_nrm) {
        c.nrm_sorted = f->nrm_sorted.as<float4>();
        c.plane_sorted = f->plane_sorted.as<float2>();
        c.normal = out->normal;
        c.nv = out->nv;
        c.depth_isect = out->depth_isect;
        c.fx = f->cam.fx;
        c.fy = f->cam.fy;
        c.cx = f->cam.cx;
        c.cy = f->cam.cy;
    }
    return c;
}

// K3..K6 given capacity `cap` (graph path) or the exact count (plain path).
// Boundary event k, if timed and in the mask; graph capture records external nodes.
cudaError_t mark(const Marks &m, int k, cudaStream_t st)
{
    if (!m.ev || !(m.mask >> k & 1u)) return cudaSuccess;
    return m.capture ? cudaEventRecordWithFlags(m.ev[k], st, cudaEventRecordExternal) : cudaEventRecord(m.ev[k], st);
}

gs_status enqueue_after_scan(Frame *f, const gs_outputs *out, int64_t max_k, cudaStream_t st, const Marks &mk = Marks{})
{
    uint32_t *cnt = f->counters.as<uint32_t>();
    uint32_t *err = f->err_word ? f->err_word : cnt + kCntErr;
    SortScratch scr;
    sort_scratch_carve(f->sort_scr.p, std::max<int64_t>(f->key_cap, f->n), &scr);
    // K3a, K4a: the visible Gaussians in depth order
    NvtxStages nvtx_stage("gsr.depth_sort");
    GSR_CUDA(launch_compact(f->ntiles.as<uint32_t>(), f->bin.as<uint4>(), f->voffs.as<uint32_t>(), f->n,
                            f->dkeys[0].as<uint32_t>(), f->dvals[0].as<uint32_t>(), scr.hist, st));
    GSR_CUDA(mark(mk, 3, st));
    uint32_t *dk[2] = {f->dkeys[0].as<uint32_t>(), f->dkeys[1].as<uint32_t>()};
    uint32_t *dv[2] = {f->dvals[0].as<uint32_t>(), f->dvals[1].as<uint32_t>()};
    int dres = 0;
    GSR_CUDA(launch_sort32(dk, dv, cnt + kCntVisible, err, f->n, 32, scr, &dres, st, true, f->give_up, true));
    GSR_CUDA(mark(mk, 4, st));
    nvtx_stage.next("gsr.tile_keys_sort");
    // K3b, K4b: tile keys in depth order, then stable by tile
    const int tbits = f->bits - 32;
    GSR_CUDA(launch_duplicate(dv[dres], cnt + kCntVisible, f->n, f->ntiles.as<uint32_t>(), f->bin.as<uint4>(),
                              f->dlook.as<unsigned long long>(), f->cam.tile_shift, f->tiles_x,
                              f->keys[0].as<uint32_t>(), f->vals[0].as<uint32_t>(), f->key_cap, cnt, scr.hist,
                              sort_passes(tbits), st, err, f->give_up));
    GSR_CUDA(mark(mk, 5, st));
    uint32_t *kk[2] = {f->keys[0].as<uint32_t>(), f->keys[1].as<uint32_t>()};
    uint32_t *vv[2] = {f->vals[0].as<uint32_t>(), f->vals[1].as<uint32_t>()};
    int res = 0;
    GSR_CUDA(launch_sort32(kk, vv, cnt + kCntEff, err, max_k, tbits, scr, &res, st, true, f->give_up));
    f->sorted = res;
    GSR_CUDA(mark(mk, 6, st));
    nvtx_stage.next("gsr.ranges_plan");
    GSR_CUDA(launch_ranges(kk[res], vv[res], cnt, max_k, f->n, f->rec.as<GaussRec>(),
                           gather_records(f) ? nullptr : f->rec_sorted.as<GaussRec>(),
                           f->ranges.as<uint2>(), f->n_tiles, f->bin.as<uint4>(),
                           f->has_state ? f->keys64.as<uint64_t>() : nullptr, st,
                           f->want_nrm ? f->nrm.as<float4>() : nullptr,
                           f->want_nrm ? f->nrm_sorted.as<float4>() : nullptr,
                           f->want_nrm ? f->plane.as<float2>() : nullptr,
                           f->want_nrm ? f->plane_sorted.as<float2>() : nullptr, err));
    GSR_CUDA(launch_plan(f->ranges.as<uint2>(), f->n_tiles, f->head, f->order.as<uint32_t>(),
                         f->plan.as<uint32_t>(), err, st));
    GSR_CUDA(mark(mk, 7, st));
    nvtx_stage.next("gsr.composite");
    const CompositeArgs ca = comp_args(f, out);
    if (f->max_long > 0) {  // long tiles on the second stream, beside the short ones
        GSR_CUDA(cudaEventRecord(f->fork.fork, st));
        GSR_CUDA(cudaStreamWaitEvent(f->fork.s, f->fork.fork, 0));
        GSR_CUDA(launch_composite_long(ca, f->tile, f->max_long, f->fork.s));
        GSR_CUDA(cudaEventRecord(f->fork.join, f->fork.s));
    }
    GSR_CUDA(launch_composite(ca, f->tile, f->batch, st));
    if (f->max_long > 0) GSR_CUDA(cudaStreamWaitEvent(st, f->fork.join, 0));
    GSR_CUDA(mark(mk, 8, st));
    return GS_OK;
}

}  // namespace

gs_status err_status(uint32_t err)
{
    if (err & kErrSortTimeout) return fail(GS_ERR_TIMEOUT, "radix sort lookback wait gave up");
    if (err & kErrTmaTimeout) return fail(GS_ERR_TIMEOUT, "compositing batch wait gave up");
    if (err & kErrCapacity) return fail(GS_ERR_CAPACITY, "instance count exceeded capacity");
    if (err & kErrBounds) return fail(GS_ERR_INTERNAL, "a device index check fired (GSR_DEBUG build)");
    return GS_OK;
}

namespace {

gs_status forward_plain(gs_context *ctx, const gs_scene *s, const gs_camera *c, const gs_render_opts *o,
                        const gs_outputs *out, Frame *f, cudaStream_t st)
{
    int tile, batch, chunk;
    pick_config(ctx, s, c, o, &tile, &batch, &chunk);
    if (!composite_supported(tile, batch))
        return fail(GS_ERR_INVALID_ARG, "tile must be 8/16/32 and batch 32/64/128/256 with the warps' staging rings "
                                        "fitting shared memory");
    const bool state = (o->flags & GS_EMIT_BWD_STATE) != 0;
    // the RaDe-GS channels (normal, nv, intersection depth) composite every list with one
    // warp per block (the long tiles' partial states keep neither), so no list counts as
    // long (head 2^30 records)
    const bool nrm = out->normal || out->nv || out->depth_isect;
    if (nrm && (o->flags & (GS_EMIT_BWD_STATE | GS_COUNT_PAIRS)))
        return fail(GS_ERR_INVALID_ARG,
                    "normal, nv and depth_isect are rendered without GS_EMIT_BWD_STATE and GS_COUNT_PAIRS");
    gs_render_opts on = *o;
    if (nrm) {
        chunk = 1 << 24;
        on.head = 1 << 30;
    }
    // the pair census counts the sequential pass: every list takes one warp per block
    if (o->flags & GS_COUNT_PAIRS) on.head = 1 << 30;
    gs_status r = frame_setup(f, s, c, &on, tile, batch, chunk, state);
    f->count_pairs = (o->flags & GS_COUNT_PAIRS) != 0;
    if (r != GS_OK) return r;
    f->err_word = ctx->err.as<uint32_t>();
    f->give_up = ctx->give_up == 1;
    f->give_up_composite = ctx->give_up != 0;
    f->want_nrm = nrm;
    if (nrm) {
        GSR_CUDA(f->nrm.ensure(sizeof(float4) * (size_t)std::max<int64_t>(s->n, 1)));
        GSR_CUDA(f->plane.ensure(sizeof(float2) * (size_t)std::max<int64_t>(s->n, 1)));
    }
    uint32_t *cnt = f->counters.as<uint32_t>();
    Marks mk;
    mk.mask = timing_mask(o->flags);
    if (mk.mask) {
        GSR_CUDA(ctx->timer.init());
        mk.ev = ctx->timer.next(mk.mask);
    }
    GSR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCntSlots, st));
    GSR_CUDA(mark(mk, 0, st));
    const ProjectArgs pa = proj_args(f, s);
    {
        NvtxRange nvtx_("gsr.project_scan");
        GSR_CUDA(launch_project(pa, st));
    }
    GSR_CUDA(mark(mk, 1, st));
    GSR_CUDA(launch_scan_blocks(pa.block_sums, pa.block_vis, project_blocks(s->n), f->boffs.as<uint32_t>(),
                                f->voffs.as<uint32_t>(), cnt, kMaxInstances, st));
    GSR_CUDA(mark(mk, 2, st));
    GSR_CUDA(cudaMemcpyAsync(ctx->h_counters, cnt, sizeof(uint32_t) * kCntSlots, cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaMemcpyAsync(ctx->h_counters + kCntSlots, f->err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    if (ctx->h_counters[kCntSlots]) {  // a wait of an earlier frame on this context gave up
        const uint32_t bits = ctx->h_counters[kCntSlots];
        GSR_CUDA(cudaMemsetAsync(f->err_word, 0, sizeof(uint32_t), st));
        return err_status(bits);
    }
    const uint64_t K = (uint64_t)ctx->h_counters[kCntTotal] | ((uint64_t)ctx->h_counters[kCntTotalHi] << 32);
    if ((int64_t)K > kMaxInstances) return fail(GS_ERR_CAPACITY, "more than 2^30 - 1 (Gaussian, tile) instances");
    f->K = (int64_t)K;
    ctx->st_frames += 1;
    ctx->st_sum_k += (int64_t)K;
    ctx->st_sum_v += ctx->h_counters[kCntVisible];
    ctx->st_max_k = std::max<int64_t>(ctx->st_max_k, (int64_t)K);
    if (f->key_cap < f->K || f->key_cap == 0) {
        r = frame_keys(f, f->K);
        if (r != GS_OK) return r;
    }
    // the sorted record copy, for the frames whose K5 makes one (the normal channels)
    if (!gather_records(f))
        GSR_CUDA(f->rec_sorted.ensure(sizeof(GaussRec) * (size_t)std::max<int64_t>(f->key_cap, 1)));
    if ((r = frame_plan(f, f->K)) != GS_OK) return r;
    if (nrm) {
        GSR_CUDA(f->nrm_sorted.ensure(sizeof(float4) * (size_t)std::max<int64_t>(f->K, 1)));
        GSR_CUDA(f->plane_sorted.ensure(sizeof(float2) * (size_t)std::max<int64_t>(f->K, 1)));
    }
    // counters[kCntEff] was clamped to kMaxInstances; K fits, so it equals K.
    r = enqueue_after_scan(f, out, f->K, st, mk);
    if (r != GS_OK || !f->count_pairs) return r;
    GSR_CUDA(cudaMemcpyAsync(ctx->h_counters, cnt, sizeof(uint32_t) * kCntSlots, cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    const uint32_t *h = ctx->h_counters;
    ctx->st_pairs_eval += (int64_t)((uint64_t)h[kCntPairs] | ((uint64_t)h[kCntPairs + 1] << 32));
    ctx->st_pairs_blend += (int64_t)((uint64_t)h[kCntPairs + 2] | ((uint64_t)h[kCntPairs + 3] << 32));
    return GS_OK;
}

}  // namespace
}  // namespace gsr

namespace gsr {

int context_device(const gs_context *ctx) { return ctx->device; }

gs_status context_warp_scratch(gs_context *ctx, size_t n_src, size_t n_dst, cudaStream_t st, float2 **pos,
                               unsigned long long **best)
{
    GSR_CUDA(ctx->warp_pos.ensure(sizeof(float2) * std::max<size_t>(n_src, 1)));
    // a reallocation always grows the capacity (it may return the freed address again,
    // so the pointer alone does not show it)
    const size_t old_bytes = ctx->warp_best.bytes;
    GSR_CUDA(ctx->warp_best.ensure(sizeof(unsigned long long) * std::max<size_t>(n_dst, 1)));
    if (ctx->warp_best.bytes != old_bytes || !ctx->warp_best_clean) {
        // every slot starts empty; the gather kernel leaves it so after each call
        GSR_CUDA(cudaMemsetAsync(ctx->warp_best.p, 0xFF, ctx->warp_best.bytes, st));
        ctx->warp_best_clean = true;
    }
    *pos = ctx->warp_pos.as<float2>();
    *best = ctx->warp_best.as<unsigned long long>();
    return GS_OK;
}

void warp_scratch_dirty(gs_context *ctx) { ctx->warp_best_clean = false; }

}  // namespace gsr

// ============================================================================ C ABI

extern "C" {

gs_status gs_context_create(int device, gs_context **ctx)
{
    if (!ctx) return fail(GS_ERR_INVALID_ARG, "ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    GSR_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GS_ERR_INVALID_ARG, "no such CUDA device");
    GSR_CUDA(cudaSetDevice(device));
    gs_context *c = new gs_context();
    c->device = device;
    cudaError_t e = cudaMallocHost(&c->h_counters, sizeof(uint32_t) * (kCntSlots + 1));
    if (e == cudaSuccess) e = c->err.ensure(sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->err.p, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "gs_context_create");
    }
    *ctx = c;
    return GS_OK;
}

gs_status gs_context_check(gs_context *ctx, gs_stream stream)
{
    if (!ctx) return fail(GS_ERR_INVALID_ARG, "ctx is NULL");
    GSR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    GSR_CUDA(cudaMemcpyAsync(ctx->h_counters + kCntSlots, ctx->err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    const uint32_t bits = ctx->h_counters[kCntSlots];
    if (!bits) return GS_OK;
    GSR_CUDA(cudaMemsetAsync(ctx->err.p, 0, sizeof(uint32_t), st));
    GSR_CUDA(cudaStreamSynchronize(st));
    return err_status(bits);
}

gs_status gs_context_debug_waits(gs_context *ctx, int32_t give_up)
{
    if (!ctx) return fail(GS_ERR_INVALID_ARG, "ctx is NULL");
    if (give_up < 0 || give_up > 2) return fail(GS_ERR_INVALID_ARG, "give_up must be 0, 1 or 2");
    ctx->give_up = give_up;
    return GS_OK;
}

gs_status gs_context_destroy(gs_context *ctx)
{
    if (!ctx) return GS_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    delete ctx;
    return GS_OK;
}

gs_status gs_render_forward(gs_context *ctx, const gs_scene *scene, const gs_camera *cam, const gs_render_opts *opts,
                            const gs_outputs *out, gs_fwd_state **state, gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.forward");
    if (state) *state = nullptr;
    if (!ctx || !opts || !out) return fail(GS_ERR_INVALID_ARG, "ctx, opts and out must be non-NULL");
    gs_status r = check_scene(scene);
    if (r != GS_OK) return r;
    if ((r = check_cam(cam)) != GS_OK) return r;
    if (state && !(opts->flags & GS_EMIT_BWD_STATE))
        return fail(GS_ERR_INVALID_ARG, "a backward state needs GS_EMIT_BWD_STATE");
    GSR_CUDA(cudaSetDevice(ctx->device));
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    Frame *f = ctx->acquire();
    r = forward_plain(ctx, scene, cam, opts, out, f, (cudaStream_t)stream);
    if (r != GS_OK) {
        ctx->give_back(f);
        return r;
    }
    // errors raised by this frame's earlier kernels are visible at the next sync; report those seen so far
    r = err_status(ctx->h_counters[kCntErr]);
    if (r != GS_OK) {
        ctx->give_back(f);
        return r;
    }
    if (state) {
        gs_fwd_state *sst = new gs_fwd_state();
        sst->ctx = ctx;
        sst->f = f;
        sst->n = scene->n;
        sst->n_pad = scene->n_pad;
        *state = sst;
    } else {
        ctx->give_back(f);
    }
    return GS_OK;
}

gs_status gs_render_forward_to_host(gs_context *ctx, const gs_scene *scene, const gs_camera *cam,
                                    const gs_render_opts *opts, const gs_outputs *host_out, gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.forward_to_host");
    if (!ctx || !host_out || !cam || !opts) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (host_out->normal || host_out->nv || host_out->depth_isect)
        return fail(GS_ERR_INVALID_ARG, "host outputs carry no RaDe-GS channel (render it with gs_render_forward)");
    gs_status r = check_cam(cam);
    if (r != GS_OK) return r;
    GSR_CUDA(cudaSetDevice(ctx->device));
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    const size_t hw = (size_t)cam->width * cam->height;
    GSR_CUDA(ctx->host_planes.ensure(sizeof(float) * hw * 11));
    float *d = ctx->host_planes.as<float>();
    gs_outputs dev{};
    dev.rgb = host_out->rgb ? d : nullptr;
    dev.dcdx = host_out->dcdx ? d + 3 * hw : nullptr;
    dev.dcdy = host_out->dcdy ? d + 6 * hw : nullptr;
    dev.depth = host_out->depth ? d + 9 * hw : nullptr;
    dev.alpha = host_out->alpha ? d + 10 * hw : nullptr;
    gs_render_opts o = *opts;
    o.flags &= ~GS_EMIT_BWD_STATE;
    r = gs_render_forward(ctx, scene, cam, &o, &dev, nullptr, stream);
    if (r != GS_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const float *src[5] = {dev.rgb, dev.dcdx, dev.dcdy, dev.depth, dev.alpha};
    float *dst[5] = {host_out->rgb, host_out->dcdx, host_out->dcdy, host_out->depth, host_out->alpha};
    const size_t sz[5] = {3 * hw, 3 * hw, 3 * hw, hw, hw};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) GSR_CUDA(cudaMemcpyAsync(dst[k], src[k], sizeof(float) * sz[k], cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_render_backward(gs_context *ctx, const gs_fwd_state *state, const gs_scene *scene,
                             const gs_outputs *grad_in, const gs_scene_grads *grads, gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.backward");
    if (!ctx || !state || !grad_in || !grads) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_scene(scene);
    if (r != GS_OK) return r;
    const Frame *f = state->f;
    if (!f->has_state) return fail(GS_ERR_INVALID_ARG, "forward state was made without GS_EMIT_BWD_STATE");
    if (scene->n != state->n || scene->n_pad != state->n_pad || scene->sh_degree != f->deg)
        return fail(GS_ERR_INVALID_ARG, "scene does not match the forward state");
    GSR_CUDA(cudaSetDevice(ctx->device));
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    cudaStream_t st = (cudaStream_t)stream;
    if (f->n == 0) return GS_OK;
    GSR_CUDA(ctx->g2d.ensure(sizeof(float) * 10 * (size_t)f->n));
    GSR_CUDA(cudaMemsetAsync(ctx->g2d.p, 0, sizeof(float) * 10 * (size_t)f->n, st));
    BackwardArgs b{};
    b.rec = f->rec.as<GaussRec>();
    b.vals = f->vals[f->sorted].as<uint32_t>();
    b.ranges = f->ranges.as<uint2>();
    b.width = f->W;
    b.height = f->H;
    b.tiles_x = f->tiles_x;
    b.tiles_y = f->tiles_y;
    b.tile = f->tile;
    for (int k = 0; k < 3; ++k) b.bg[k] = f->bg[k];
    b.final_T = f->fT.as<float>();
    b.final_Tx = f->fTx.as<float>();
    b.final_Ty = f->fTy.as<float>();
    b.n_contrib = f->ncontrib.as<uint32_t>();
    b.g_rgb = grad_in->rgb;
    b.g_dcdx = grad_in->dcdx;
    b.g_dcdy = grad_in->dcdy;
    b.g_depth = grad_in->depth;
    b.g_alpha = grad_in->alpha;
    b.g2d = ctx->g2d.as<float>();
    b.n = (uint32_t)f->n;
    GSR_CUDA(launch_composite_backward(b, st));
    ProjectBwdArgs p{};
    p.means = scene->means;
    p.log_scales = scene->log_scales;
    p.quats = scene->quats;
    p.logits = scene->opacity_logits;
    p.sh = scene->sh;
    p.n = scene->n;
    p.n_pad = scene->n_pad;
    p.deg = scene->sh_degree;
    p.cam = f->cam;
    p.ntiles = f->ntiles.as<uint32_t>();
    p.g2d = ctx->g2d.as<float>();
    p.d_means = grads->means;
    p.d_log_scales = grads->log_scales;
    p.d_quats = grads->quats;
    p.d_logits = grads->opacity_logits;
    p.d_sh = grads->sh;
    GSR_CUDA(launch_project_backward(p, st));
    return GS_OK;
}

gs_status gs_state_view_get(const gs_fwd_state *state, gs_state_view *v)
{
    if (!state || !v) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    const Frame *f = state->f;
    std::memset(v, 0, sizeof(*v));
    v->n_instances = f->K;
    v->n_tiles = f->n_tiles;
    v->tiles_x = f->tiles_x;
    v->tiles_y = f->tiles_y;
    v->tile = f->tile;
    v->keys = f->has_state ? f->keys64.as<uint64_t>() : nullptr;
    v->vals = f->vals[f->sorted].as<uint32_t>();
    v->ranges = f->ranges.as<uint32_t>();
    v->ntiles = f->ntiles.as<uint32_t>();
    v->records = f->rec.as<float>();
    v->final_T = f->has_state ? f->fT.as<float>() : nullptr;
    v->n_contrib = f->has_state ? f->ncontrib.as<uint32_t>() : nullptr;
    v->n_visible = -1;
    return GS_OK;
}

gs_status gs_state_free(gs_fwd_state *state)
{
    if (!state) return GS_OK;
    state->ctx->give_back(state->f);
    delete state;
    return GS_OK;
}

// ---------------------------------------------------------------------------- graphs

gs_status gs_graph_create(gs_context *ctx, const gs_scene *scene, const gs_camera *cam, const gs_render_opts *opts,
                          const gs_outputs *out, int64_t capacity, gs_stream stream, gs_graph **graph)
{
    if (!graph) return fail(GS_ERR_INVALID_ARG, "graph is NULL");
    *graph = nullptr;
    if (!ctx || !opts || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (out->normal || out->nv || out->depth_isect)
        return fail(GS_ERR_INVALID_ARG, "graphs do not render the RaDe-GS channels");
    gs_status r = check_scene(scene);
    if (r != GS_OK) return r;
    if ((r = check_cam(cam)) != GS_OK) return r;
    if (opts->flags & GS_EMIT_BWD_STATE) return fail(GS_ERR_INVALID_ARG, "graphs do not keep backward state");
    GSR_CUDA(cudaSetDevice(ctx->device));
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    int tile, batch, chunk;
    pick_config(ctx, scene, cam, opts, &tile, &batch, &chunk);
    if (!composite_supported(tile, batch)) return fail(GS_ERR_INVALID_ARG, "unsupported tile/batch");
    if (capacity <= 0) capacity = std::max<int64_t>(4 * scene->n, 1024);
    if (capacity > kMaxInstances) return fail(GS_ERR_INVALID_ARG, "capacity above 2^30 - 1");
    // capture on a private stream (the legacy default stream cannot be captured)
    GSR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    cudaStream_t st = nullptr;
    GSR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    gs_graph *g = new gs_graph();
    g->cap_stream = st;
    g->ctx = ctx;
    g->f = new Frame();
    g->capacity = capacity;
    g->tile = tile;
    Frame *f = g->f;
    r = frame_setup(f, scene, cam, opts, tile, batch, chunk, false);
    if (r == GS_OK) r = frame_keys(f, capacity);
    if (r == GS_OK) r = frame_plan(f, capacity);
    if (r == GS_OK) {
        cudaError_t e = cudaMemsetAsync(f->counters.p, 0, sizeof(uint32_t) * kCntSlots, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "graph setup");
    }
    // warm-up (sets kernel attributes outside capture), then capture
    if (r == GS_OK) {
        uint32_t *cnt = f->counters.as<uint32_t>();
        g->mark_mask = timing_mask(opts->flags);
        g->timed = g->mark_mask != 0u;
        cudaEvent_t *cap_ev = nullptr;
        if (g->timed) {
            cudaError_t e = g->timer.init();
            if (e != cudaSuccess) r = cuda_fail(e, "stage timer");
            else cap_ev = g->timer.next(g->mark_mask);
        }
        auto enqueue = [&](cudaStream_t s2, bool capture) -> gs_status {
            Marks evs;
            evs.ev = capture ? cap_ev : nullptr;
            evs.mask = g->mark_mask;
            evs.capture = capture;
            GSR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCntPerFrame, s2));
            GSR_CUDA(mark(evs, 0, s2));
            g->proj_args = proj_args(f, scene);
            NvtxRange nvtx_("gsr.project_scan");
            GSR_CUDA(launch_project(g->proj_args, s2));
            GSR_CUDA(mark(evs, 1, s2));
            GSR_CUDA(launch_scan_blocks(g->proj_args.block_sums, g->proj_args.block_vis, project_blocks(scene->n),
                                        f->boffs.as<uint32_t>(), f->voffs.as<uint32_t>(), cnt, capacity, s2));
            GSR_CUDA(mark(evs, 2, s2));
            return enqueue_after_scan(f, out, capacity, s2, evs);
        };
        if (r == GS_OK) r = enqueue(st, false);
        if (r == GS_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCntSlots, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) r = cuda_fail(e, "graph warm-up");
        }
        if (r == GS_OK) {
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamBeginCapture");
            else {
                gs_status r2 = enqueue(st, true);
                cudaGraph_t gr = nullptr;
                e = cudaStreamEndCapture(st, &gr);
                if (r2 != GS_OK) r = r2;
                else if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamEndCapture");
                g->graph = gr;
            }
        }
        if (r == GS_OK) {
            cudaError_t e = cudaGraphInstantiate(&g->exec, g->graph, 0);
            if (e != cudaSuccess) r = cuda_fail(e, "cudaGraphInstantiate");
        }
        if (r == GS_OK) {
            size_t nn = 0;
            cudaGraphGetNodes(g->graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(g->graph, nodes.data(), &nn);
            const void *fp = project_kernel_ptr(scene->sh_degree, 0), *fc = project_kernel_ptr(scene->sh_degree, 1);
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                cudaGraphNodeGetType(nd, &ty);
                if (ty != cudaGraphNodeTypeKernel) continue;
                cudaKernelNodeParams kp;
                if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
                if (kp.func == fp) g->proj_node = nd;
                if (kp.func == fc) g->colour_node = nd;
            }
            if (!g->proj_node || !g->colour_node) r = fail(GS_ERR_CUDA, "projection node not found in captured graph");
            if (g->timed) {
                for (auto nd : nodes) {
                    cudaGraphNodeType ty;
                    cudaGraphNodeGetType(nd, &ty);
                    if (ty != cudaGraphNodeTypeEventRecord) continue;
                    cudaEvent_t e = nullptr;
                    cudaGraphEventRecordNodeGetEvent(nd, &e);
                    for (int k = 0; k < StageTimer::kBounds; ++k)
                        if ((g->mark_mask >> k & 1u) && cap_ev[k] == e) g->ev_node[k] = nd;
                }
                for (int k = 0; k < StageTimer::kBounds; ++k)
                    if ((g->mark_mask >> k & 1u) && !g->ev_node[k])
                        r = fail(GS_ERR_CUDA, "stage event node not found in captured graph");
                g->timer.reset();  // the capture-time event set was never recorded
            }
        }
    }
    if (r != GS_OK) {
        gs_graph_destroy(g);
        return r;
    }
    *graph = g;
    return GS_OK;
}

gs_status gs_graph_render(gs_graph *g, const gs_camera *cam, gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.graph_render");
    if (!g || !cam) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (cam->width != g->f->W || cam->height != g->f->H) return fail(GS_ERR_INVALID_ARG, "resolution differs from the graph's");
    gs_status r = check_cam(cam);
    if (r != GS_OK) return r;
    g->proj_args.cam = make_cam(*cam, g->tile);
    for (cudaGraphNode_t nd : {g->proj_node, g->colour_node}) {
        cudaKernelNodeParams kp;
        GSR_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
        void *args[1] = {&g->proj_args};
        kp.kernelParams = args;
        kp.extra = nullptr;
        GSR_CUDA(cudaGraphExecKernelNodeSetParams(g->exec, nd, &kp));
    }
    if (g->timed) {
        cudaEvent_t *ev = g->timer.next(g->mark_mask);
        for (int k = 0; k < StageTimer::kBounds; ++k)
            if (g->mark_mask >> k & 1u) GSR_CUDA(cudaGraphExecEventRecordNodeSetEvent(g->exec, g->ev_node[k], ev[k]));
    }
    GSR_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_graph_check(gs_graph *g, gs_stream stream, int64_t *max_instances)
{
    if (!g) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t h[kCntSlots];
    GSR_CUDA(cudaMemcpyAsync(h, g->f->counters.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    if (max_instances) *max_instances = (int64_t)h[kCntMaxTotal];
    GSR_CUDA(cudaMemsetAsync(g->f->counters.as<uint32_t>() + kCntErr, 0, sizeof(uint32_t) * 2, st));
    GSR_CUDA(cudaStreamSynchronize(st));
    return err_status(h[kCntErr]);
}

gs_status gs_graph_destroy(gs_graph *g)
{
    if (!g) return GS_OK;
    if (g->cap_stream) cudaStreamSynchronize(g->cap_stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g->f;
    delete g;
    return GS_OK;
}

static void fill_stats(gs_frame_stats *o, int64_t frames, int64_t sk, int64_t sv, int64_t mk, StageTimer &t)
{
    std::memset(o, 0, sizeof(*o));
    o->frames = frames;
    o->instances_total = sk;
    o->visible_total = sv;
    o->instances_max = mk;
    int64_t tf = 0;
    if (!t.ev.empty()) t.collect(o->stage_ms, &tf);
    o->timed_frames = tf;
}

gs_status gs_graph_stats(gs_graph *g, gs_stream stream, int reset, gs_frame_stats *stats)
{
    if (!g || !stats) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t h[kCntSlots];
    GSR_CUDA(cudaStreamSynchronize(st));
    GSR_CUDA(cudaMemcpy(h, g->f->counters.p, sizeof(h), cudaMemcpyDeviceToHost));
    auto u64 = [&](int k) { return (int64_t)((uint64_t)h[k] | ((uint64_t)h[k + 1] << 32)); };
    fill_stats(stats, h[kCntFrames], u64(kCntSumK), u64(kCntSumV), h[kCntMaxTotal], g->timer);
    if (reset) {
        GSR_CUDA(cudaMemset(g->f->counters.as<uint32_t>() + kCntMaxTotal, 0, sizeof(uint32_t) * (kCntSlots - kCntMaxTotal)));
        g->timer.reset();
    }
    return err_status(h[kCntErr]);
}

gs_status gs_context_stats(gs_context *ctx, gs_stream stream, int reset, gs_frame_stats *stats)
{
    if (!ctx || !stats) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    GSR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    fill_stats(stats, ctx->st_frames, ctx->st_sum_k, ctx->st_sum_v, ctx->st_max_k, ctx->timer);
    stats->pairs_evaluated = ctx->st_pairs_eval;
    stats->pairs_blended = ctx->st_pairs_blend;
    if (reset) {
        ctx->st_frames = ctx->st_sum_k = ctx->st_sum_v = ctx->st_max_k = 0;
        ctx->st_pairs_eval = ctx->st_pairs_blend = 0;
        ctx->timer.reset();
    }
    return GS_OK;
}

// ---------------------------------------------------------------------------- autotuner

gs_status gs_autotune(gs_context *ctx, const gs_scene *scene, const gs_camera *cam, const gs_outputs *out, int iters,
                      gs_stream stream, int32_t *best_tile, int32_t *best_batch, int32_t *best_chunk, float *best_ms)
{
    if (!ctx || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_scene(scene);
    if (r != GS_OK) return r;
    if ((r = check_cam(cam)) != GS_OK) return r;
    if (iters < 1) iters = 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    GSR_CUDA(cudaEventCreate(&e0));
    GSR_CUDA(cudaEventCreate(&e1));
    const int tiles[3] = {8, 16, 32}, batches[4] = {32, 64, 128, 256}, chunks[3] = {256, 512, 1024};
    gs_outputs planes = *out;  // timed on the standard planes (graphs render no RaDe-GS channel)
    planes.normal = planes.nv = planes.depth_isect = nullptr;
    out = &planes;
    float best = 1e30f;
    int bt = kDefaultTile, bb = kDefaultBatch, bc = kDefaultChunk;
    for (int t : tiles)
        for (int b : batches)
            for (int c : chunks) {
                if (!composite_supported(t, b)) continue;  // the warps' staging rings must fit shared memory
                gs_render_opts o{};
                o.tile = t;
                o.batch = b;
                o.chunk = c;
                // one plain forward gives this configuration's instance count, which sizes a
                // graph; the graph's replays are timed, as frames are rendered in streams
                r = gs_render_forward(ctx, scene, cam, &o, out, nullptr, stream);
                if (r != GS_OK) break;
                const int64_t K =
                    (int64_t)ctx->h_counters[kCntTotal] | ((int64_t)ctx->h_counters[kCntTotalHi] << 32);
                gs_graph *g = nullptr;
                r = gs_graph_create(ctx, scene, cam, &o, out, std::min<int64_t>(K + K / 4 + 4096, kMaxInstances),
                                    stream, &g);
                if (r != GS_OK) break;
                r = gs_graph_render(g, cam, stream);  // warm-up
                cudaEventRecord(e0, st);
                for (int it = 0; it < iters && r == GS_OK; ++it) r = gs_graph_render(g, cam, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                if (r == GS_OK) r = gs_graph_check(g, stream, nullptr);
                gs_graph_destroy(g);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= iters;
                if (r == GS_OK && ms < best) {
                    best = ms;
                    bt = t;
                    bb = b;
                    bc = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GS_OK) return r;
    const int nb = scene->n > 0 ? (int)std::log2((double)scene->n) : 0;
    ctx->tune[TuneKey{cam->width, cam->height, nb, scene->sh_degree}] = {bt, bb, bc};
    if (best_tile) *best_tile = bt;
    if (best_batch) *best_batch = bb;
    if (best_chunk) *best_chunk = bc;
    if (best_ms) *best_ms = best;
    return GS_OK;
}

const char *gs_last_error(void) { return gsr::g_last_error.c_str(); }

const char *gs_version(void) { return "gsr 0.1 (sm_103a)"; }

}  // extern "C"
