// Serving: continuous batching of render requests over resident scenes.
//
// Requests from many viewers (scene, camera, resolution, caller-owned output
// planes) are queued by gs_server_submit. One scheduler thread moves each
// through three stages:
//   1. admit   - a free in-flight slot takes it; projection + scan (K1, K2) run
//                on the slot's own stream and the instance count K is copied back.
//   2. sort    - once K is known the request's sort buffers (tile keys and
//                values, both ping-pong halves, sort scratch: about 18 B per
//                instance; compositing gathers the records by index) are
//                taken from a fixed byte budget; if the budget is short the
//                request waits, in arrival order. K3-K5 run on the slot stream.
//   3. compose - whenever the compositing stream is idle, every sorted request
//                is put into one persistent compositing launch whose CTAs pull
//                (request, tile) items from a flat work list: each request's short
//                tile lists, in its plan's order. Its long lists (longer than
//                4 x kServeChunk records) go to k_composite_long on its own slot
//                stream, beside that launch.
// So requests that arrive while others are on the GPU are admitted as slots and
// memory free up, and their projection and sorting overlap the compositing of
// the others. Completion frees the slot and the sort memory and stamps the
// latency, measured from submit. Nothing on the device waits on anything.
//
// Host-side fault injection for tests: GSR_FAULT=alloc:<k> makes the k-th sort
// allocation fail (that request finishes with GS_ERR_OOM, others proceed);
// GSR_FAULT=enqueue:<k> makes the k-th admission's first launch fail;
// GSR_FAULT=wait:<k> runs the k-th admitted request's kernels with waits that give
// up at once (its sort and duplication lookbacks), so that request
// finishes with GS_ERR_TIMEOUT through its device error word, others proceed;
// GSR_FAULT=thread:<k> makes the scheduler thread throw (a host exception) before its
// k-th admission. The thread catches whatever escapes its loop: it waits for the GPU work
// it has enqueued (so no kernel still writes a caller's planes), finishes every request
// not yet done with GS_ERR_INTERNAL, and stops; later submits fail with GS_ERR_INTERNAL.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

using Clock = std::chrono::steady_clock;
// Served requests are composited at tile 8 with staging batches of 32 records (the persistent
// kernel's); measured on the mixed serving stream against tile 16: 983 against 788 Mpix/s, and a
// Poisson-load p99 of 10 against 146 ms.
constexpr int kServeTile = 8;
constexpr int kServeBatch = 32;
// long tile lists (longer than kHeadChunks * kServeChunk records) are composited per request by
// k_composite_long, beside the batch's persistent kernel
constexpr int kServeChunk = 512;
constexpr int kMaxSlots = 256;

// First-fit allocator over one device allocation (the sort-buffer budget).
class Arena {
  public:
    cudaError_t init(size_t bytes)
    {
        bytes_ = (bytes + 255) & ~size_t(255);
        if (bytes_ == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&base_, bytes_);
        if (e != cudaSuccess) {
            base_ = nullptr;
            bytes_ = 0;
            return e;
        }
        free_[0] = bytes_;
        return cudaSuccess;
    }
    ~Arena()
    {
        if (base_) cudaFree(base_);
    }
    size_t capacity() const { return bytes_; }
    void *alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_[off] = bytes;
                return static_cast<char *>(base_) + off;
            }
        }
        return nullptr;
    }
    void release(void *p)
    {
        if (!p) return;
        const size_t off = static_cast<size_t>(static_cast<char *>(p) - static_cast<char *>(base_));
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t len = u->second;
        used_.erase(u);
        size_t start = off;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first == off + len) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }

  private:
    void *base_ = nullptr;
    size_t bytes_ = 0;
    std::map<size_t, size_t> free_, used_;
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (p && want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 256));
        if (e == cudaSuccess) bytes = std::max<size_t>(want, 256);
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct SceneRes {
    gs_scene view{};
    void *mem = nullptr;
};

enum class Stage { Queued, Scan, Sorted, Composing, Done };

struct Request {
    uint64_t id = 0;
    int scene = 0;
    gs_camera cam{};
    gs_render_opts opts{};
    gs_outputs out{};
    Clock::time_point t_submit, t_done;
    Stage stage = Stage::Queued;
    gs_status status = GS_OK;
    bool cancelled = false;
    int slot = -1;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_scan = nullptr, ev_sorted = nullptr;
    cudaEvent_t ev_done = nullptr;  // the request's long tiles and error word, after its batch
    DevBuf rec, bin, ntiles, bsums, boffs, ranges, order, counters, plan;
    DevBuf vsums, voffs, dlook, dkeys[2], dvals[2], dscr;  // depth order (per Gaussian)
    uint32_t n_gauss = 1;            // the scene's Gaussians (bounds the gathered indices)
    uint32_t *h_counters = nullptr;  // pinned
    void *sort_mem = nullptr;        // from the arena
    Request *req = nullptr;
    CamParams cam{};
    int n_tiles = 0, bits = 32;
    int64_t K = 0;
    int sorted = 0;
    bool give_up = false;  // GSR_FAULT=wait: this request's waits give up at once
    uint32_t *keys[2] = {nullptr, nullptr};  // tile keys, in the sort memory
    uint32_t *vals[2] = {nullptr, nullptr};
    // every device buffer the slot owns (the sort memory belongs to the arena)
    void release_buffers()
    {
        DevBuf *all[] = {&rec, &bin, &ntiles, &bsums, &boffs, &ranges, &order, &counters, &plan, &vsums, &voffs,
                         &dlook, &dkeys[0], &dkeys[1], &dvals[0], &dvals[1], &dscr};
        for (DevBuf *b : all) b->release();
    }
};

int fault_at(const char *kind)
{
    const char *f = std::getenv("GSR_FAULT");
    if (!f) return -1;
    const size_t n = std::strlen(kind);
    if (std::strncmp(f, kind, n) != 0 || f[n] != ':') return -1;
    return std::atoi(f + n + 1);
}

}  // namespace
}  // namespace gsr

using namespace gsr;

struct gs_server {
    int device = 0;
    int max_inflight = 8;
    Arena arena;
    std::vector<SceneRes> scenes;
    std::vector<Slot> slots;
    std::deque<Request *> queue;     // submitted, not admitted
    std::deque<Request *> sort_wait; // scanned, waiting for sort memory (arrival order)
    std::map<uint64_t, Request *> all;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::thread thr;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t pending = 0;  // submitted and not finished
    // compositing
    cudaStream_t comp_stream = nullptr;
    cudaEvent_t comp_done = nullptr;
    bool comp_busy = false;
    std::vector<int> comp_slots;
    ServeItem *h_items = nullptr;  // pinned
    ServeItem *d_items = nullptr;
    uint32_t *d_work = nullptr;
    int comp_grid = 0;
    int alloc_count = 0, enqueue_count = 0, admit_count = 0;
    int fault_alloc = -1, fault_enqueue = -1, fault_wait = -1, fault_thread = -1;
    bool dead = false;       // the scheduler stopped on a failure (thread_msg)
    std::string thread_msg;
};

namespace gsr {
namespace {

void finish(gs_server *S, Request *r, gs_status st)
{
    r->status = r->cancelled && st == GS_OK ? GS_ERR_CANCELLED : st;
    r->stage = Stage::Done;
    r->t_done = Clock::now();
    if (--S->pending == 0) S->cv_done.notify_all();
}

void slot_free(gs_server *S, Slot &sl)
{
    if (sl.sort_mem) S->arena.release(sl.sort_mem);
    sl.sort_mem = nullptr;
    sl.req = nullptr;
}

size_t sort_bytes(int64_t K)
{
    const int64_t k = std::max<int64_t>(K, 1);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    return 4 * up(sizeof(uint32_t) * k) + up(sort_scratch_bytes(k));
}

// The slot's per-Gaussian and per-tile buffers for n Gaussians and n_tiles tiles.
// Growing one frees and allocates device memory, and cudaFree waits for the whole
// device; gs_server_load_scene therefore sizes every slot for the largest scene
// before requests arrive, so that admission never reallocates while others render.
cudaError_t slot_reserve(Slot &sl, int64_t n, int n_tiles)
{
    const int64_t n1 = std::max<int64_t>(n, 1), n4 = (n + 3) / 4 * 4;
    const int nb = std::max(project_blocks(n), 1);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    ok(sl.rec.ensure(sizeof(GaussRec) * (size_t)n1));
    ok(sl.bin.ensure(sizeof(uint4) * (size_t)n1));
    ok(sl.ntiles.ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(n4, 4)));
    DevBuf *per_block[] = {&sl.bsums, &sl.boffs, &sl.vsums, &sl.voffs};
    for (DevBuf *b : per_block) ok(b->ensure(sizeof(uint32_t) * (size_t)nb));
    ok(sl.dlook.ensure(duplicate_look_bytes(n1)));
    for (int k = 0; k < 2; ++k) {
        ok(sl.dkeys[k].ensure(sizeof(uint32_t) * (size_t)n1));
        ok(sl.dvals[k].ensure(sizeof(uint32_t) * (size_t)n1));
    }
    ok(sl.dscr.ensure(sort_scratch_bytes(n1)));
    ok(sl.ranges.ensure(sizeof(uint2) * (size_t)std::max(n_tiles, 1)));
    ok(sl.order.ensure(sizeof(uint32_t) * (size_t)std::max(n_tiles, 1)));
    ok(sl.counters.ensure(sizeof(uint32_t) * kCntSlots));
    ok(sl.plan.ensure(sizeof(uint32_t) * 3));
    return e;
}

// Stage 1: projection + scan on the slot's stream; K copied back.
gs_status admit(gs_server *S, int si, Request *r)
{
    Slot &sl = S->slots[si];
    const SceneRes &sc = S->scenes[r->scene];
    const gs_scene &s = sc.view;
    if (S->fault_enqueue >= 0 && S->enqueue_count++ == S->fault_enqueue)
        return fail(GS_ERR_CUDA, "injected enqueue failure");
    sl.give_up = S->fault_wait >= 0 && S->admit_count == S->fault_wait;
    ++S->admit_count;
    sl.cam = make_cam(r->cam, kServeTile);
    sl.n_tiles = sl.cam.tiles_x * sl.cam.tiles_y;
    sl.bits = 32 + ilog2(std::max(sl.n_tiles, 1));
    const int nb = project_blocks(s.n);
    GSR_CUDA(slot_reserve(sl, s.n, sl.n_tiles));
    uint32_t *cnt = static_cast<uint32_t *>(sl.counters.p);
    GSR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCntSlots, sl.stream));
    ProjectArgs a{};
    a.means = s.means;
    a.log_scales = s.log_scales;
    a.quats = s.quats;
    a.logits = s.opacity_logits;
    a.sh = s.sh;
    a.n = s.n;
    a.n_pad = s.n_pad;
    a.deg = s.sh_degree;
    a.cam = sl.cam;
    a.rec = static_cast<GaussRec *>(sl.rec.p);
    a.bin = static_cast<uint4 *>(sl.bin.p);
    a.ntiles = static_cast<uint32_t *>(sl.ntiles.p);
    a.block_sums = static_cast<uint32_t *>(sl.bsums.p);
    a.block_vis = static_cast<uint32_t *>(sl.vsums.p);
    a.counters = cnt;
    GSR_CUDA(launch_project(a, sl.stream));
    GSR_CUDA(launch_scan_blocks(a.block_sums, a.block_vis, nb, static_cast<uint32_t *>(sl.boffs.p),
                                static_cast<uint32_t *>(sl.voffs.p), cnt, (1ll << 30) - 1, sl.stream));
    GSR_CUDA(cudaMemcpyAsync(sl.h_counters, cnt, sizeof(uint32_t) * kCntSlots, cudaMemcpyDeviceToHost, sl.stream));
    GSR_CUDA(cudaEventRecord(sl.ev_scan, sl.stream));
    sl.req = r;
    r->slot = si;
    r->stage = Stage::Scan;
    return GS_OK;
}

// Stage 2: with K known and memory granted, duplicate, sort and range.
gs_status enqueue_sort(gs_server *S, Slot &sl)
{
    Request *r = sl.req;
    const gs_scene &s = S->scenes[r->scene].view;
    uint32_t *cnt = static_cast<uint32_t *>(sl.counters.p);
    const int64_t K = sl.K;
    const int64_t k1 = std::max<int64_t>(K, 1);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(sl.sort_mem);
    sl.keys[0] = reinterpret_cast<uint32_t *>(p);
    p += up(sizeof(uint32_t) * k1);
    sl.keys[1] = reinterpret_cast<uint32_t *>(p);
    p += up(sizeof(uint32_t) * k1);
    sl.vals[0] = reinterpret_cast<uint32_t *>(p);
    p += up(sizeof(uint32_t) * k1);
    sl.vals[1] = reinterpret_cast<uint32_t *>(p);
    p += up(sizeof(uint32_t) * k1);
    sl.n_gauss = (uint32_t)std::max<int64_t>(s.n, 1);
    SortScratch scr, dscr;
    sort_scratch_carve(p, k1, &scr);
    sort_scratch_carve(sl.dscr.p, std::max<int64_t>(s.n, 1), &dscr);
    // the visible Gaussians in depth order, then their tile keys in that order, stable by tile
    uint32_t *dk[2] = {static_cast<uint32_t *>(sl.dkeys[0].p), static_cast<uint32_t *>(sl.dkeys[1].p)};
    uint32_t *dv[2] = {static_cast<uint32_t *>(sl.dvals[0].p), static_cast<uint32_t *>(sl.dvals[1].p)};
    GSR_CUDA(launch_compact(static_cast<uint32_t *>(sl.ntiles.p), static_cast<uint4 *>(sl.bin.p),
                            static_cast<uint32_t *>(sl.voffs.p), s.n, dk[0], dv[0], dscr.hist, sl.stream));
    int dres = 0;
    GSR_CUDA(launch_sort32(dk, dv, cnt + kCntVisible, cnt + kCntErr, s.n, 32, dscr, &dres, sl.stream, true,
                           sl.give_up, true));
    const int tbits = sl.bits - 32;
    GSR_CUDA(launch_duplicate(dv[dres], cnt + kCntVisible, s.n, static_cast<uint32_t *>(sl.ntiles.p),
                              static_cast<uint4 *>(sl.bin.p), static_cast<unsigned long long *>(sl.dlook.p),
                              sl.cam.tile_shift, sl.cam.tiles_x, sl.keys[0], sl.vals[0], K, cnt, scr.hist,
                              sort_passes(tbits), sl.stream, nullptr, sl.give_up));
    int res = 0;
    GSR_CUDA(launch_sort32(sl.keys, sl.vals, cnt + kCntEff, cnt + kCntErr, K, tbits, scr, &res, sl.stream, true,
                           sl.give_up));
    sl.sorted = res;
    GSR_CUDA(launch_ranges(sl.keys[res], sl.vals[res], cnt, K, s.n, static_cast<const GaussRec *>(sl.rec.p), nullptr,
                           static_cast<uint2 *>(sl.ranges.p), sl.n_tiles, static_cast<const uint4 *>(sl.bin.p),
                           nullptr, sl.stream));
    GSR_CUDA(launch_plan(static_cast<const uint2 *>(sl.ranges.p), sl.n_tiles, (int64_t)kHeadChunks * kServeChunk,
                         static_cast<uint32_t *>(sl.order.p), static_cast<uint32_t *>(sl.plan.p), cnt + kCntErr,
                         sl.stream));
    GSR_CUDA(cudaEventRecord(sl.ev_sorted, sl.stream));
    r->stage = Stage::Sorted;
    return GS_OK;
}

CompositeArgs slot_comp_args(Slot &sl)
{
    Request *r = sl.req;
    CompositeArgs c{};
    c.rec_index = static_cast<const GaussRec *>(sl.rec.p);  // gathered by index through vals
    c.n_gauss = sl.n_gauss;
    c.vals = sl.vals[sl.sorted];
    c.tile_order = static_cast<const uint32_t *>(sl.order.p);
    c.ranges = static_cast<const uint2 *>(sl.ranges.p);
    c.width = r->cam.width;
    c.height = r->cam.height;
    c.tiles_x = sl.cam.tiles_x;
    c.tiles_y = sl.cam.tiles_y;
    for (int k = 0; k < 3; ++k) c.bg[k] = r->opts.bg[k];
    c.rgb = r->out.rgb;
    c.dcdx = r->out.dcdx;
    c.dcdy = r->out.dcdy;
    c.depth = r->out.depth;
    c.alpha = r->out.alpha;
    c.err_word = static_cast<uint32_t *>(sl.counters.p) + kCntErr;
    c.give_up = sl.give_up ? 1u : 0u;
    c.plan = static_cast<const uint32_t *>(sl.plan.p);
    c.long_counter = static_cast<uint32_t *>(sl.plan.p) + 1;
    c.chunk = kServeChunk;
    c.long_bpc = (kServeTile == 8 && sl.K <= 1024 * (int64_t)sl.n_tiles) ? 2 : 1;
    return c;
}

void scheduler_loop(gs_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        // 3a. retire a finished compositing batch: its persistent kernel and every request's
        // long tiles and error word (ev_done)
        bool batch_done = S->comp_busy && cudaEventQuery(S->comp_done) == cudaSuccess;
        for (int si : S->comp_slots) batch_done = batch_done && cudaEventQuery(S->slots[si].ev_done) == cudaSuccess;
        if (batch_done) {
            for (int si : S->comp_slots) {
                Slot &sl = S->slots[si];
                // the slot's device error bits, copied after its compositing (sort lookback,
                // batch waits); a request whose kernels gave up finishes with that error
                const uint32_t err = sl.h_counters[kCntErr];
                Request *r = sl.req;
                slot_free(S, sl);
                finish(S, r, err ? err_status(err) : GS_OK);
            }
            S->comp_slots.clear();
            S->comp_busy = false;
            progressed = true;
        }
        // 1. admit queued requests into free slots
        NvtxStages nvtx_stage("gsr.serve.admit");
        for (int si = 0; si < (int)S->slots.size() && !S->queue.empty(); ++si) {
            if (S->slots[si].req) continue;
            if (S->fault_thread >= 0 && S->admit_count == S->fault_thread)
                throw std::runtime_error("injected scheduler failure (GSR_FAULT=thread)");
            Request *r = S->queue.front();
            S->queue.pop_front();
            gs_status st = admit(S, si, r);
            if (st != GS_OK) {
                slot_free(S, S->slots[si]);
                finish(S, r, st);
            }
            progressed = true;
        }
        // 2. requests whose scan finished: read K, ask for sort memory in arrival order
        nvtx_stage.next("gsr.serve.sort");
        for (Slot &sl : S->slots) {
            if (!sl.req || sl.req->stage != Stage::Scan) continue;
            if (cudaEventQuery(sl.ev_scan) != cudaSuccess) continue;
            sl.K = (int64_t)sl.h_counters[kCntTotal] | ((int64_t)sl.h_counters[kCntTotalHi] << 32);
            sl.req->stage = Stage::Sorted;  // placeholder: waiting for memory
            S->sort_wait.push_back(sl.req);
            progressed = true;
        }
        while (!S->sort_wait.empty()) {
            Request *r = S->sort_wait.front();
            Slot &sl = S->slots[r->slot];
            const size_t need = sort_bytes(sl.K);
            if (sl.K >= (1ll << 30) || need > S->arena.capacity()) {
                S->sort_wait.pop_front();
                slot_free(S, sl);
                finish(S, r, fail(GS_ERR_OOM, "request's sort buffers exceed the server's budget"));
                progressed = true;
                continue;
            }
            void *mem = nullptr;
            const bool inject = S->fault_alloc >= 0 && S->alloc_count == S->fault_alloc;
            ++S->alloc_count;
            if (!inject) mem = S->arena.alloc(need);
            if (inject) {
                S->sort_wait.pop_front();
                slot_free(S, sl);
                finish(S, r, fail(GS_ERR_OOM, "injected sort allocation failure"));
                progressed = true;
                continue;
            }
            if (!mem) break;  // wait for memory, keep arrival order
            S->sort_wait.pop_front();
            sl.sort_mem = mem;
            gs_status st = enqueue_sort(S, sl);
            if (st != GS_OK) {
                slot_free(S, sl);
                finish(S, r, st);
            }
            progressed = true;
        }
        // 3b. launch one compositing batch over every sorted request
        nvtx_stage.next("gsr.serve.composite");
        if (!S->comp_busy) {
            int n = 0;
            uint32_t total = 0;
            for (int si = 0; si < (int)S->slots.size(); ++si) {
                Slot &sl = S->slots[si];
                if (!sl.req || sl.req->stage != Stage::Sorted || !sl.sort_mem) continue;
                if (cudaEventQuery(sl.ev_sorted) != cudaSuccess) continue;
                ServeItem &it = S->h_items[n];
                it.args = slot_comp_args(sl);
                it.first_item = total;
                it.n_items = (uint32_t)sl.n_tiles;
                total += (uint32_t)sl.n_tiles;
                sl.req->stage = Stage::Composing;
                S->comp_slots.push_back(si);
                ++n;
            }
            if (n > 0) {
                cudaError_t e = cudaMemcpyAsync(S->d_items, S->h_items, sizeof(ServeItem) * n, cudaMemcpyHostToDevice,
                                                S->comp_stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(S->d_work, 0, sizeof(uint32_t), S->comp_stream);
                if (e == cudaSuccess)
                    e = launch_composite_persistent(S->d_items, n, total, kServeTile, kServeBatch, S->d_work,
                                                    S->comp_grid, S->comp_stream);
                if (e == cudaSuccess) e = cudaEventRecord(S->comp_done, S->comp_stream);
                // each request's long tiles on its own stream, beside the batch's kernel; then its
                // error bits, once both are done
                for (size_t k = 0; k < S->comp_slots.size() && e == cudaSuccess; ++k) {
                    Slot &sl = S->slots[S->comp_slots[k]];
                    const int64_t head = (int64_t)kHeadChunks * kServeChunk;
                    const int64_t max_long = std::min<int64_t>(sl.n_tiles, sl.K / (head + 1) + 1);
                    e = launch_composite_long(S->h_items[k].args, kServeTile, max_long, sl.stream);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.stream, S->comp_done, 0);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(sl.h_counters + kCntErr, static_cast<uint32_t *>(sl.counters.p) + kCntErr,
                                            sizeof(uint32_t), cudaMemcpyDeviceToHost, sl.stream);
                    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_done, sl.stream);
                }
                if (e != cudaSuccess) {
                    // nothing of the batch may still write a caller's planes when its requests end
                    cudaStreamSynchronize(S->comp_stream);
                    for (int si : S->comp_slots) cudaStreamSynchronize(S->slots[si].stream);
                    for (int si : S->comp_slots) {
                        Request *r = S->slots[si].req;
                        slot_free(S, S->slots[si]);
                        finish(S, r, cuda_fail(e, "serving composite launch"));
                    }
                    S->comp_slots.clear();
                } else {
                    S->comp_busy = true;
                }
                progressed = true;
            }
        }
        bool inflight = S->comp_busy || !S->queue.empty() || !S->sort_wait.empty();
        for (const Slot &sl : S->slots) inflight |= sl.req != nullptr;
        if (S->stop && !inflight) break;
        if (!progressed) {
            if (inflight) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            }
        }
    }
}

// The scheduler stopped on a failure: wait for the GPU work it enqueued, then finish every
// request that is not done with GS_ERR_INTERNAL and free what they held. Later submits fail.
void scheduler_failed(gs_server *S, const char *what)
{
    std::lock_guard<std::mutex> g(S->mu);
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (S->comp_stream) cudaStreamSynchronize(S->comp_stream);
    S->dead = true;
    S->thread_msg = what;
    const std::string msg = std::string("the server's scheduler stopped: ") + what;
    for (Slot &sl : S->slots) {
        if (!sl.req) continue;
        Request *r = sl.req;
        slot_free(S, sl);
        finish(S, r, fail(GS_ERR_INTERNAL, msg));
    }
    for (Request *r : S->queue) finish(S, r, fail(GS_ERR_INTERNAL, msg));
    S->queue.clear();
    S->sort_wait.clear();  // their slots were freed above
    S->comp_slots.clear();
    S->comp_busy = false;
    S->cv_done.notify_all();
}

void scheduler(gs_server *S)
{
    try {
        scheduler_loop(S);
    } catch (const std::exception &e) {
        scheduler_failed(S, e.what());
    } catch (...) {
        scheduler_failed(S, "unknown exception");
    }
}

}  // namespace
}  // namespace gsr

extern "C" {

gs_status gs_server_create(int device, size_t sort_budget_bytes, int max_inflight, gs_server **srv)
{
    if (!srv) return fail(GS_ERR_INVALID_ARG, "srv is NULL");
    *srv = nullptr;
    if (max_inflight < 1 || max_inflight > kMaxSlots) return fail(GS_ERR_INVALID_ARG, "max_inflight must be 1..256");
    int ndev = 0;
    GSR_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GS_ERR_INVALID_ARG, "no such CUDA device");
    GSR_CUDA(cudaSetDevice(device));
    gs_server *S = new gs_server();
    S->device = device;
    S->max_inflight = max_inflight;
    S->fault_alloc = fault_at("alloc");
    S->fault_enqueue = fault_at("enqueue");
    S->fault_wait = fault_at("wait");
    S->fault_thread = fault_at("thread");
    cudaError_t e = S->arena.init(sort_budget_bytes);
    S->slots.resize(max_inflight);
    for (Slot &sl : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_scan, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_sorted, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_counters, sizeof(uint32_t) * kCntSlots);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->comp_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->comp_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_items, sizeof(ServeItem) * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_items, sizeof(ServeItem) * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_work, sizeof(uint32_t));
    if (e != cudaSuccess) {
        gs_server_destroy(S);
        return cuda_fail(e, "gs_server_create");
    }
    S->comp_grid = composite_persistent_grid(kServeTile, kServeBatch);
    S->thr = std::thread(scheduler, S);
    *srv = S;
    return GS_OK;
}

gs_status gs_server_load_scene(gs_server *S, const gs_scene *scene, int32_t *scene_id)
{
    if (!S || !scene_id) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_scene(scene);
    if (r != GS_OK) return r;
    GSR_CUDA(cudaSetDevice(S->device));
    const size_t plane = sizeof(float) * (size_t)scene->n_pad;
    const int nk = (scene->sh_degree + 1) * (scene->sh_degree + 1);
    const size_t rows = 3 + 3 + 4 + 1 + (size_t)nk * 3;
    SceneRes res;
    res.view = *scene;
    if (scene->n > 0) {
        GSR_CUDA(cudaMalloc(&res.mem, plane * rows));
        float *b = static_cast<float *>(res.mem);
        const float *src[5] = {scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh};
        const size_t nr[5] = {3, 3, 4, 1, (size_t)nk * 3};
        const float **dst[5] = {&res.view.means, &res.view.log_scales, &res.view.quats, &res.view.opacity_logits,
                                &res.view.sh};
        size_t off = 0;
        for (int k = 0; k < 5; ++k) {
            cudaError_t e = cudaMemcpy(b + off, src[k], plane * nr[k], cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) {
                cudaFree(res.mem);
                return cuda_fail(e, "scene copy");
            }
            *dst[k] = b + off;
            off += (size_t)scene->n_pad * nr[k];
        }
    }
    std::lock_guard<std::mutex> g(S->mu);
    // every slot sized for the largest scene and a 1920x1080 frame at the serving tile
    // (larger frames still grow a slot on first use)
    const int tiles_1080p = ((1920 + kServeTile - 1) / kServeTile) * ((1080 + kServeTile - 1) / kServeTile);
    for (Slot &sl : S->slots) {
        if (sl.req) continue;  // busy: it grows on its next admission if it has to
        cudaError_t e = slot_reserve(sl, scene->n, tiles_1080p);
        if (e != cudaSuccess) {
            if (res.mem) cudaFree(res.mem);
            return cuda_fail(e, "serving slot buffers");
        }
    }
    S->scenes.push_back(res);
    *scene_id = (int32_t)S->scenes.size() - 1;
    return GS_OK;
}

gs_status gs_server_submit(gs_server *S, int32_t scene_id, const gs_camera *cam, const gs_render_opts *opts,
                           const gs_outputs *out, uint64_t *req_id)
{
    if (!S || !cam || !opts || !out || !req_id) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_cam(cam);
    if (r != GS_OK) return r;
    if (opts->flags & GS_EMIT_BWD_STATE) return fail(GS_ERR_INVALID_ARG, "serving does not keep backward state");
    if (out->normal || out->nv || out->depth_isect)
        return fail(GS_ERR_INVALID_ARG, "serving does not render the RaDe-GS channels");
    if ((opts->tile && opts->tile != kServeTile) || (opts->batch && opts->batch != kServeBatch))
        return fail(GS_ERR_INVALID_ARG, "serving renders with tile " + std::to_string(kServeTile) + ", batch " +
                                            std::to_string(kServeBatch));
    Request *q = new Request();
    q->cam = *cam;
    q->opts = *opts;
    q->out = *out;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (scene_id < 0 || scene_id >= (int32_t)S->scenes.size()) {
            delete q;
            return fail(GS_ERR_INVALID_ARG, "unknown scene id");
        }
        if (S->stop) {
            delete q;
            return fail(GS_ERR_CANCELLED, "server is shutting down");
        }
        if (S->dead) {
            delete q;
            return fail(GS_ERR_INTERNAL, "the server's scheduler stopped: " + S->thread_msg);
        }
        q->scene = scene_id;
        q->id = S->next_id++;
        S->all[q->id] = q;
        S->queue.push_back(q);
        ++S->pending;
        *req_id = q->id;
    }
    S->cv.notify_one();
    return GS_OK;
}

gs_status gs_server_poll(gs_server *S, uint64_t req_id, double *latency_ms)
{
    if (!S) return fail(GS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(req_id);
    if (it == S->all.end()) return fail(GS_ERR_INVALID_ARG, "unknown request id");
    Request *q = it->second;
    if (q->stage != Stage::Done) return GS_NOT_READY;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    const gs_status st = q->status;
    S->all.erase(it);
    delete q;
    if (st != GS_OK) set_error("request failed");
    return st;
}

gs_status gs_server_cancel(gs_server *S, uint64_t req_id)
{
    if (!S) return fail(GS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(req_id);
    if (it == S->all.end()) return fail(GS_ERR_INVALID_ARG, "unknown request id");
    Request *q = it->second;
    q->cancelled = true;
    auto qi = std::find(S->queue.begin(), S->queue.end(), q);
    if (qi != S->queue.end()) {
        S->queue.erase(qi);
        finish(S, q, GS_ERR_CANCELLED);
    }
    return GS_OK;
}

gs_status gs_server_drain(gs_server *S)
{
    if (!S) return fail(GS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->pending == 0; });
    if (S->dead) return fail(GS_ERR_INTERNAL, "the server's scheduler stopped: " + S->thread_msg);
    return GS_OK;
}

gs_status gs_server_destroy(gs_server *S)
{
    if (!S) return GS_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->thr.joinable()) S->thr.join();
    cudaSetDevice(S->device);
    cudaDeviceSynchronize();
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.ev_scan) cudaEventDestroy(sl.ev_scan);
        if (sl.ev_sorted) cudaEventDestroy(sl.ev_sorted);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        if (sl.h_counters) cudaFreeHost(sl.h_counters);
        sl.release_buffers();
    }
    for (SceneRes &s : S->scenes)
        if (s.mem) cudaFree(s.mem);
    for (auto &kv : S->all) delete kv.second;
    if (S->comp_stream) cudaStreamDestroy(S->comp_stream);
    if (S->comp_done) cudaEventDestroy(S->comp_done);
    if (S->h_items) cudaFreeHost(S->h_items);
    if (S->d_items) cudaFree(S->d_items);
    if (S->d_work) cudaFree(S->d_work);
    delete S;
    return GS_OK;
}

}  // extern "C"
