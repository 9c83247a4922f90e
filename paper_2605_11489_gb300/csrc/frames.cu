// Frames in flight behind the C ABI (gs_frame_stream_*): a camera sequence rendered by
// graph replay with `slots` frames at once, each slot a captured whole-frame graph
// (gs_graph) on its own high-priority stream, rendering into caller-owned device
// planes, optionally followed by device-to-host copies of the frame on the same stream.
//
// Ordering, all by stream order and events (the host never waits in submit):
//   - slot k's frames, and their copies, follow one another on slot k's stream;
//   - a release records an event on the consumer's stream that slot k's next render
//     waits for;
//   - done[k] marks the end of slot k's latest frame (render and copies); join and
//     wait use it.
#include <cuda_runtime.h>

#include <vector>

#include "gsr_internal.cuh"

struct gs_frame_stream {
    int slots = 0;
    int W = 0, H = 0;
    std::vector<gs_outputs> outs;
    std::vector<gs_graph *> graphs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done, released;
    std::vector<char> pending_release;
    int64_t next = 0;  // frames submitted so far
};

namespace {

using gsr::fail;

constexpr int kMaxSlots = 64;

// The planes a frame stream renders and copies: (pointer member, channels).
struct PlaneDesc {
    float *gs_outputs::*p;
    int channels;
};
constexpr PlaneDesc kPlanes[] = {{&gs_outputs::rgb, 3},
                                 {&gs_outputs::dcdx, 3},
                                 {&gs_outputs::dcdy, 3},
                                 {&gs_outputs::depth, 1},
                                 {&gs_outputs::alpha, 1}};

bool has_rade(const gs_outputs &o) { return o.normal || o.nv || o.depth_isect; }

void destroy_parts(gs_frame_stream *fs)
{
    for (cudaStream_t s : fs->streams)
        if (s) cudaStreamSynchronize(s);
    for (gs_graph *g : fs->graphs)
        if (g) gs_graph_destroy(g);
    for (cudaEvent_t e : fs->done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : fs->released)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : fs->streams)
        if (s) cudaStreamDestroy(s);
    delete fs;
}

// frame f is one of the last `slots` submitted: its slot still holds it
gs_status check_frame(const gs_frame_stream *fs, int64_t frame)
{
    if (frame < 0 || frame >= fs->next || frame < fs->next - fs->slots)
        return fail(GS_ERR_INVALID_ARG, "frame is not among the stream's last `slots` submitted frames");
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_frame_stream_create(gs_context *ctx, const gs_scene *scene, const gs_camera *cam0,
                                 const gs_render_opts *opts, const gs_outputs *outs, int32_t slots,
                                 int64_t capacity, gs_frame_stream **fs_out)
{
    if (!fs_out) return fail(GS_ERR_INVALID_ARG, "fs is NULL");
    *fs_out = nullptr;
    if (!ctx || !scene || !cam0 || !opts || !outs) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (slots < 1 || slots > kMaxSlots) return fail(GS_ERR_INVALID_ARG, "slots must be 1..64");
    int n_planes = 0;
    for (const PlaneDesc &d : kPlanes) n_planes += outs[0].*d.p != nullptr;
    if (n_planes == 0) return fail(GS_ERR_INVALID_ARG, "the output sets name no plane");
    for (int k = 0; k < slots; ++k) {
        if (has_rade(outs[k])) return fail(GS_ERR_INVALID_ARG, "frame streams do not render the RaDe-GS channels");
        for (const PlaneDesc &d : kPlanes)
            if ((outs[k].*d.p == nullptr) != (outs[0].*d.p == nullptr))
                return fail(GS_ERR_INVALID_ARG, "every slot's output set must name the same planes");
    }
    gs_frame_stream *fs = new gs_frame_stream();
    fs->slots = slots;
    fs->W = cam0->width;
    fs->H = cam0->height;
    fs->outs.assign(outs, outs + slots);
    fs->graphs.assign(slots, nullptr);
    fs->streams.assign(slots, nullptr);
    fs->done.assign(slots, nullptr);
    fs->released.assign(slots, nullptr);
    fs->pending_release.assign(slots, 0);
    for (int k = 0; k < slots; ++k) {
        // the graph's creation selects the context's device for what follows
        gs_status r = gs_graph_create(ctx, scene, cam0, opts, &fs->outs[k], capacity, nullptr, &fs->graphs[k]);
        if (r != GS_OK) {
            destroy_parts(fs);
            return r;
        }
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&fs->streams[k], cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fs->done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fs->released[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            destroy_parts(fs);
            return gsr::cuda_fail(e, "frame stream setup");
        }
    }
    *fs_out = fs;
    return GS_OK;
}

gs_status gs_frame_stream_submit(gs_frame_stream *fs, const gs_camera *cam, const gs_outputs *host, int64_t *frame)
{
    gsr::NvtxRange nvtx_("gsr.frame_stream_submit");
    if (!fs || !cam) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    const int k = (int)(fs->next % fs->slots);
    const gs_outputs &dev = fs->outs[k];
    if (host) {
        if (has_rade(*host)) return fail(GS_ERR_INVALID_ARG, "frame streams do not render the RaDe-GS channels");
        for (const PlaneDesc &d : kPlanes)
            if (host->*d.p && !(dev.*d.p)) return fail(GS_ERR_INVALID_ARG, "a host plane the stream does not render");
    }
    cudaStream_t st = fs->streams[k];
    if (fs->pending_release[k]) {
        GSR_CUDA(cudaStreamWaitEvent(st, fs->released[k], 0));
        fs->pending_release[k] = 0;
    }
    gs_status r = gs_graph_render(fs->graphs[k], cam, st);
    if (r != GS_OK) return r;
    if (host) {
        const size_t hw = (size_t)fs->W * fs->H;
        for (const PlaneDesc &d : kPlanes)
            if (host->*d.p)
                GSR_CUDA(cudaMemcpyAsync(host->*d.p, dev.*d.p, sizeof(float) * d.channels * hw,
                                         cudaMemcpyDeviceToHost, st));
    }
    GSR_CUDA(cudaEventRecord(fs->done[k], st));
    if (frame) *frame = fs->next;
    ++fs->next;
    return GS_OK;
}

gs_status gs_frame_stream_join(gs_frame_stream *fs, int64_t frame, gs_stream consumer)
{
    if (!fs) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_frame(fs, frame);
    if (r != GS_OK) return r;
    GSR_CUDA(cudaStreamWaitEvent((cudaStream_t)consumer, fs->done[frame % fs->slots], 0));
    return GS_OK;
}

gs_status gs_frame_stream_release(gs_frame_stream *fs, int64_t frame, gs_stream consumer)
{
    if (!fs) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_frame(fs, frame);
    if (r != GS_OK) return r;
    const int k = (int)(frame % fs->slots);
    GSR_CUDA(cudaEventRecord(fs->released[k], (cudaStream_t)consumer));
    fs->pending_release[k] = 1;
    return GS_OK;
}

gs_status gs_frame_stream_wait(gs_frame_stream *fs, int64_t frame)
{
    if (!fs) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_frame(fs, frame);
    if (r != GS_OK) return r;
    GSR_CUDA(cudaEventSynchronize(fs->done[frame % fs->slots]));
    return GS_OK;
}

gs_status gs_frame_stream_synchronize(gs_frame_stream *fs)
{
    if (!fs) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    for (cudaStream_t s : fs->streams) GSR_CUDA(cudaStreamSynchronize(s));
    gs_status first = GS_OK;
    for (int k = 0; k < fs->slots; ++k) {
        const gs_status r = gs_graph_check(fs->graphs[k], fs->streams[k], nullptr);
        if (first == GS_OK) first = r;
    }
    return first;
}

gs_status gs_frame_stream_stats(gs_frame_stream *fs, int32_t slot, int reset, gs_frame_stats *stats)
{
    if (!fs || !stats) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (slot < 0 || slot >= fs->slots) return fail(GS_ERR_INVALID_ARG, "no such slot");
    return gs_graph_stats(fs->graphs[slot], fs->streams[slot], reset, stats);
}

gs_status gs_frame_stream_destroy(gs_frame_stream *fs)
{
    if (!fs) return GS_OK;
    destroy_parts(fs);
    return GS_OK;
}

}  // extern "C"
