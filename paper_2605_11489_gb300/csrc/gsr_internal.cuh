// Internal declarations shared by the render core's translation units.
// Nothing here is part of the C ABI (include/gsr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gsr.h"

namespace gsr {

// ---------------------------------------------------------------- constants
// Rasterizer conventions (3DGS, which the paper builds on; Sec. 3 and Eq. 2):
constexpr float kAlphaCap = 0.99f;          // a_i = min(0.99, o G)
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip a_i < 1/255
constexpr float kTMin = 1e-4f;              // stop before T would fall below 1e-4
constexpr int kProjThreads = 256;           // projection block: 256 threads x 4 Gaussians
constexpr int kProjPerBlock = kProjThreads * 4;

// NVTX range over a host scope (the entry points and the stages of a frame's enqueue), so
// that a profiler shows which stage launched which kernels. NVTX3 is header-only: without a
// profiler attached a range is two calls that return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// Consecutive stages in one scope: next() ends the current range and starts the next.
struct NvtxStages {
    explicit NvtxStages(const char *first) { nvtxRangePushA(first); }
    void next(const char *name)
    {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~NvtxStages() { nvtxRangePop(); }
    NvtxStages(const NvtxStages &) = delete;
    NvtxStages &operator=(const NvtxStages &) = delete;
};

// Error bits written by kernels into a device status word.
enum : uint32_t {
    kErrSortTimeout = 1u,       // a radix-sort or duplication lookback gave up waiting
    kErrTmaTimeout = 2u,        // compositing waited too long for a staged batch
    kErrCapacity = 4u,          // instance list exceeded the buffers' capacity
    kErrBounds = 8u,            // a GSR_DEBUG index check fired (the access was skipped)
};

// Index guards. In every build the guarded access is skipped when i >= n. A GSR_DEBUG build
// also raises kErrBounds in the kernel's error word, so that a guard that fires is seen (the
// build's stand-in for a memory checker; nothing traps).
#ifdef GSR_DEBUG
__device__ __forceinline__ bool gsr_in_bounds(uint64_t i, uint64_t n, uint32_t *err)
{
    if (i < n) return true;
    if (err) atomicOr(err, kErrBounds);
    return false;
}
#define GSR_IN_BOUNDS(i, n, err) ::gsr::gsr_in_bounds((uint64_t)(i), (uint64_t)(n), (err))
#else
#define GSR_IN_BOUNDS(i, n, err) ((uint64_t)(i) < (uint64_t)(n))
#endif

// ---------------------------------------------------------------- device-side camera
struct CamParams {
    float vm[12];      // world -> camera [R | t], row-major
    float fx, fy, cx, cy;
    float near_plane;
    float limx, limy;  // guard of the EWA Jacobian: x/z and y/z clamped to 1.3x the half field of view
    float campos[3];   // camera centre in world space, -R^T t
    int32_t width, height;
    int32_t tile_shift;  // log2(tile)
    int32_t tiles_x, tiles_y;
};

// Per-Gaussian compositing record, 48 bytes (3 x float4), written by the
// projection kernel for visible Gaussians and gathered by compositing:
//   r0 = (u', v', conic_a, conic_b)     projected centre, conic (Sigma2D^-1)
//   r1 = (conic_c, opacity, depth, red)
//   r2 = (green, blue, rect_lo, rect_hi)   rect as bits: x | y << 16 (inclusive)
// (u', v') is the centre relative to the centre of the rectangle's first pixel (x0, y0):
// u' = u - (x0 + 0.5), computed in float-float and rounded once. A pixel's offset
// d = (px + 0.5) - u is then (px - x0) - u', where px - x0 is an exact small integer, so d
// carries the rounding of u' (~1e-7 of the footprint) instead of that of the absolute
// coordinate u (up to ~1e-4 px at 1,000 px). The record, and so the arithmetic of every
// pixel, is the same whatever the tile size: the image does not depend on it, bit for bit.
struct __align__(16) GaussRec {
    float4 r0, r1, r2;
};
static_assert(sizeof(GaussRec) == 48, "record must be 48 bytes");

// Per-Gaussian binning entry: (depth bits, rect_lo, rect_hi, 0).
// Counters block (device, u32 words):
enum CounterSlot : int {
    kCntTotal = 0,      // K (instances) reported by the scan, before clamping
    kCntTotalHi = 1,
    kCntEff = 2,        // min(K, capacity): what sort/ranges/compositing use
    kCntVisible = 3,    // visible Gaussians
    kCntErr = 4,        // error bits
    kCntMaxTotal = 5,   // largest K seen (graph replays)
    kCntSumK = 6,       // u64 (slots 6-7): sum of K over frames since reset
    kCntSumV = 8,       // u64 (slots 8-9): sum of visible Gaussians over frames since reset
    kCntFrames = 10,    // frames since reset
    kCntPairs = 12,     // u64 x2 (slots 12-15): evaluated and blended pairs (GS_COUNT_PAIRS)
    kCntSlots = 16,
    kCntPerFrame = 4,   // slots 0..3 are cleared at the start of every frame
};

// ---------------------------------------------------------------- status plumbing
void set_error(const std::string &msg);
gs_status fail(gs_status st, const std::string &msg);
gs_status cuda_fail(cudaError_t e, const char *what);

#define GSR_CUDA(call)                                     \
    do {                                                   \
        cudaError_t e__ = (call);                          \
        if (e__ != cudaSuccess) return ::gsr::cuda_fail(e__, #call); \
    } while (0)

// ---------------------------------------------------------------- shared host helpers (render.cu)
CamParams make_cam(const gs_camera &c, int tile);
gs_status check_scene(const gs_scene *s);
gs_status check_cam(const gs_camera *c);
int ilog2(int v);
// device error bits (counters[kCntErr]) -> the status they stand for (GS_OK for none)
gs_status err_status(uint32_t err);

// ---------------------------------------------------------------- launchers
struct ProjectArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n, n_pad;
    int deg;
    CamParams cam;
    GaussRec *rec;
    uint4 *bin;
    uint32_t *ntiles;
    uint32_t *block_sums;  // per block of 1,024 Gaussians: tiles touched
    uint32_t *block_vis;   // per block of 1,024 Gaussians: visible Gaussians
    uint32_t *counters;    // visible count accumulates into kCntVisible / kCntSumV
    float4 *nrm;           // per Gaussian: camera-space normal (x, y, z, 0) of the visible ones (nullable)
    float2 *plane;         // per Gaussian, with nrm: the intersection depth's slope (dz/du, dz/dv) per pixel
};
int project_blocks(int64_t n);
// geometry (records without colour, bin, tile counts, block sums), then the SH
// colour of the visible Gaussians; launch_project runs both on one stream
cudaError_t launch_project_geometry(const ProjectArgs &a, cudaStream_t s);
cudaError_t launch_colour(const ProjectArgs &a, cudaStream_t s);
cudaError_t launch_project(const ProjectArgs &a, cudaStream_t s);

// K2: scans of the projection's per-block tile counts (-> K in counters) and,
// when vis_sums is given, of its per-block visible counts
cudaError_t launch_scan_blocks(const uint32_t *block_sums, const uint32_t *vis_sums, int nblocks,
                               uint32_t *block_offsets, uint32_t *vis_offsets, uint32_t *counters, int64_t capacity,
                               cudaStream_t s);
// K3a: depth keys + indices of the visible Gaussians, compacted; `hist`
// ([8][256], cleared here) gets the depth sort's 4 digit histograms
cudaError_t launch_compact(const uint32_t *ntiles, const uint4 *bin, const uint32_t *vis_offsets, int64_t n,
                           uint32_t *dkeys, uint32_t *dvals, uint32_t *hist, cudaStream_t s);
// K3b: tile keys (u32) + indices of the depth-sorted Gaussians dvals[0, *vcount),
// in that order; `hist` (cleared here) gets the tile sort's `passes` (<= 2)
// digit histograms. look: duplicate_look_bytes(max_v) bytes of lookback words (cleared
// here). give_up: the lookback gives up at once (diagnostic; sets kErrSortTimeout).
cudaError_t launch_duplicate(const uint32_t *dvals, const uint32_t *vcount, int64_t max_v, const uint32_t *ntiles,
                             const uint4 *bin, unsigned long long *look, int tile_shift, int tiles_x, uint32_t *keys,
                             uint32_t *vals, int64_t capacity, uint32_t *counters, uint32_t *hist, int passes,
                             cudaStream_t s, uint32_t *err = nullptr, bool give_up = false);
size_t duplicate_look_bytes(int64_t max_v);
// K5: per-tile [start, end) from the sorted tile keys, the records gathered into
// sorted order, and (keys64 != NULL) each instance's (tile << 32 | depth bits)
cudaError_t launch_ranges(const uint32_t *keys, const uint32_t *vals, uint32_t *counters, int64_t max_k,
                          int64_t n, const GaussRec *rec, GaussRec *rec_sorted, uint2 *ranges, int n_tiles,
                          const uint4 *bin, uint64_t *keys64, cudaStream_t s, const float4 *nrm = nullptr,
                          float4 *nrm_sorted = nullptr, const float2 *plane = nullptr,
                          float2 *plane_sorted = nullptr, uint32_t *err = nullptr);
// (launch_duplicate, launch_ranges: `err` is the error word for kErrCapacity and kErrBounds,
// by default counters + kCntErr)

// onesweep LSD radix sort of (keys, vals) on the low `bits` bits, K from counters[kCntEff]
struct SortScratch {
    uint32_t *hist;      // [8][256]
    uint32_t *status;    // [passes][max_parts][256]
    uint32_t *part_ctr;  // [8]
    int64_t max_parts;
};
size_t sort_scratch_bytes(int64_t capacity);
void sort_scratch_carve(void *base, int64_t capacity, SortScratch *s);
int sort_passes(int bits);
// Sorts keys[0]/vals[0] into the buffer pair returned in *result (0 or 1).
// hist_ready: scr.hist already holds the digit histograms of the keys (built
// by launch_duplicate), so the histogram pass is skipped. give_up: every
// lookback gives up at once (diagnostic; sets kErrSortTimeout, output unsorted).
// wide: partitions of 512 threads with 8 keys each instead of 256 with 16 (the faster
// shape for the depth sort of the visible Gaussians; the narrow one for the tile keys).
cudaError_t launch_sort(uint64_t *keys[2], uint32_t *vals[2], const uint32_t *counters, uint32_t *err_word,
                        int64_t max_k, int bits, const SortScratch &scr, int *result, cudaStream_t s,
                        bool hist_ready = false, bool give_up = false, bool wide = false);
// The same over 32-bit keys; the element count is the device word *count.
cudaError_t launch_sort32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *count, uint32_t *err_word,
                          int64_t max_k, int bits, const SortScratch &scr, int *result, cudaStream_t s,
                          bool hist_ready, bool give_up = false, bool wide = false);

struct CompositeArgs {
    const GaussRec *rec;  // records in sorted (instance) order: tile t's list is rec[ranges[t].x, ranges[t].y)
    const uint32_t *vals;  // the Gaussian index of each instance, sorted like rec
    // gather mode (rec_index set, rec unused): the records by Gaussian index, each batch
    // gathered through vals; indices >= n_gauss (possible only after a sort gave up) read
    // record 0
    const GaussRec *rec_index;
    uint32_t n_gauss;
    const uint2 *ranges;
    int32_t width, height, tiles_x, tiles_y;
    float bg[3];
    float *rgb, *dcdx, *dcdy, *depth, *alpha;
    float *final_T, *final_Tx, *final_Ty;  // backward state (nullable)
    uint32_t *n_contrib;
    uint32_t *err_word;
    // compositing plan (launch_plan): tile_order lists the long tiles (list > head records)
    // first, then the others, each part longest first; plan = (n_long, long-tile work
    // counter, n_short)
    const uint32_t *tile_order;
    const uint32_t *plan;
    uint32_t *long_counter;        // plan + 1, handed out by k_composite_long's CTAs
    int32_t chunk;                 // least records per chunk of a long tile
    int32_t long_bpc;              // pixel blocks per k_composite_long CTA: 2 (8 chunk warps each) or 1 (16)
    unsigned long long *pair_counts;  // (evaluated, blended) pairs: the GS_COUNT_PAIRS census (nullable)
    // normal channel (nullable: the normal variant runs only when nrm_sorted is set, whole tiles only)
    const float4 *nrm_sorted;      // normals in sorted (instance) order, like rec
    const float2 *plane_sorted;    // intersection-depth slopes in sorted order (with nrm_sorted)
    float *normal, *nv, *depth_isect;
    float fx, fy, cx, cy;          // intrinsics: nv's pixel rays
    uint32_t give_up;              // diagnostic: each warp's first batch wait gives up without polling
                                   // (kErrTmaTimeout), then waits for its copies in flight
};
// Long tile lists. A list longer than `head` records (default kHeadChunks * chunk)
// is composited by k_composite_long: G warps per 8x4 pixel block (8 when a CTA takes
// two blocks, 16 when it takes one), each taking one of g = min(G, ceil(len / chunk))
// depth-contiguous chunks, merged exactly in shared memory. Shorter lists take one
// warp per block (k_composite).
constexpr int kHeadChunks = 4;
// Plan of a frame's compositing: tile_order = the long tiles, then the others, each
// part bucketed by floor(log2(length)), longest first; plan = (n_long, 0, n_short).
// After a sort timeout (kErrSortTimeout in *err) nothing is planned (n_long = n_short
// = 0): the ranges need not partition anything, and the frame reports the error.
cudaError_t launch_plan(const uint2 *ranges, int n_tiles, int64_t head, uint32_t *order, uint32_t *plan,
                        const uint32_t *err, cudaStream_t s);
// order tiles by decreasing list length (power-of-two buckets), for the serving kernel
cudaError_t launch_tile_order(const uint2 *ranges, int n_tiles, uint32_t *order, cudaStream_t s);
bool composite_supported(int tile, int batch);
// The short tiles of a plan: one CTA per tile (grid n_tiles, CTAs past n_short exit).
cudaError_t launch_composite(const CompositeArgs &a, int tile, int batch, cudaStream_t s);
// The long tiles of a plan, up to max_long of them: a persistent grid of CTAs that take
// (tile, pixel-block group) items from the plan's work counter (a.long_bpc blocks a group:
// 2 only at tile 8).
cudaError_t launch_composite_long(const CompositeArgs &a, int tile, int64_t max_long, cudaStream_t s);

// serving: tiles of several requests from one (request, tile) work list
struct ServeItem {  // one request's compositing description (device copy)
    CompositeArgs args;
    uint32_t first_item;  // prefix of tiles over the batch's requests
    uint32_t n_items;
};
cudaError_t launch_composite_persistent(const ServeItem *reqs, int n_reqs, uint32_t total_items, int tile,
                                        int batch, uint32_t *work_counter, int grid, cudaStream_t s);
int composite_persistent_grid(int tile, int batch);

// backward
struct BackwardArgs {
    // compositing side
    const GaussRec *rec;  // the records by Gaussian index, read through vals as the forward gathered them
    const uint32_t *vals;
    const uint2 *ranges;
    int32_t width, height, tiles_x, tiles_y, tile;
    float bg[3];
    const float *final_T, *final_Tx, *final_Ty;
    const uint32_t *n_contrib;
    const float *g_rgb, *g_dcdx, *g_dcdy, *g_depth, *g_alpha;
    float *g2d;  // [n][10] per-Gaussian 2D adjoints: u, v, ca, cb, cc, o, z, r, g, b
    uint32_t n;  // Gaussians: a sorted index >= n (an unsorted list after a sort gave up) is skipped
};
cudaError_t launch_composite_backward(const BackwardArgs &a, cudaStream_t s);

struct ProjectBwdArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n, n_pad;
    int deg;
    CamParams cam;
    const uint32_t *ntiles;
    const float *g2d;
    float *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh;
};
cudaError_t launch_project_backward(const ProjectBwdArgs &a, cudaStream_t s);

// frame-interpolation warp (warp.cu): scatter + gather launches, and the
// context-owned scratch it runs on (render.cu)
gs_status check_warp_args(const gs_camera *src, const gs_camera *dst, const gs_warp_input *in,
                          const gs_warp_output *out);
bool warp_needs_positions(const gs_warp_input &in, const gs_warp_output &out);
cudaError_t launch_warp(const gs_camera &src, const gs_camera &dst, const gs_warp_input &in, const gs_warp_output &out,
                        float2 *pos, unsigned long long *best, cudaStream_t s);
// Device of the context, and its warp scratch for n_src source and n_dst target
// pixels; `best` is all ones on return (filled on (re)allocation or after a
// failed call). A call that fails after launching must call warp_scratch_dirty.
int context_device(const gs_context *ctx);
gs_status context_warp_scratch(gs_context *ctx, size_t n_src, size_t n_dst, cudaStream_t st, float2 **pos,
                               unsigned long long **best);
void warp_scratch_dirty(gs_context *ctx);

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase. Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t max_tries)
{
    for (uint32_t t = 0; t < max_tries; ++t)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// TMA bulk copy (non-tensor) global -> this CTA's shared memory, completing
// `bytes` transactions on `bar`. Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void tma_bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Alpha of a Gaussian record at pixel centre (pxc, pyc), with every operation
// spelled out so that the forward and backward kernels make identical
// skip/cap decisions. ex, ey = conic * d (the pixel-derivative factors).
struct AlphaEval {
    float dx, dy, ex, ey, al;
    float g;  // exp(-Q/2), the Gaussian's falloff before the opacity scales it
    bool capped;
};
// Compositing evaluates a record at the pixels of one 8x4 block of the absolute pixel grid
// (a warp's block in the forward; the block of the pixel in the backward), with the centre
// taken relative to the block's middle, (bx0 + 4, by0 + 2):
//   c = u' + ((x0 - bx0) - 4, (y0 - by0) - 2)   (block_centre; u' of GaussRec, (x0, y0) its
//                                                rectangle's first pixel)
//   d = ((px - bx0) - 4, (py - by0) - 2) - c    (both small: c's rounding is ~1e-7 of it)
// Blocks are the same for every tile size, so the image does not depend on it, bit for bit.
__device__ __forceinline__ float2 block_centre(const float4 &r0, const float4 &r2, int bx0, int by0)
{
    const uint32_t lo = __float_as_uint(r2.z);
    return make_float2(__fadd_rn(r0.x, (float)((int)(lo & 0xFFFFu) - bx0 - 4)),
                       __fadd_rn(r0.y, (float)((int)(lo >> 16) - by0 - 2)));
}
// The pixel's place in its block, relative to the block's middle: exact small floats.
__device__ __forceinline__ float block_px(int px) { return (float)((px & 7) - 4); }
__device__ __forceinline__ float block_py(int py) { return (float)((py & 3) - 2); }
// r0.x, r0.y: the block-relative centre (block_centre); (lx, ly) = (block_px, block_py).
__device__ __forceinline__ AlphaEval eval_alpha(const float4 &r0, const float4 &r1, float lx, float ly)
{
    AlphaEval e;
    e.dx = __fsub_rn(lx, r0.x);
    e.dy = __fsub_rn(ly, r0.y);
    e.ex = __fmaf_rn(r0.z, e.dx, __fmul_rn(r0.w, e.dy));
    e.ey = __fmaf_rn(r0.w, e.dx, __fmul_rn(r1.x, e.dy));
    const float Q = __fmaf_rn(e.dx, e.ex, __fmul_rn(e.dy, e.ey));
    e.g = ex2_approx(__fmul_rn(Q, -0.72134752044448170f));
    const float al = __fmul_rn(r1.y, e.g);
    e.capped = al > kAlphaCap;
    e.al = e.capped ? kAlphaCap : al;
    return e;
}

__device__ __forceinline__ bool rect_contains(const float4 &r2, uint32_t px, uint32_t py)
{
    const uint32_t lo = __float_as_uint(r2.z), hi = __float_as_uint(r2.w);
    return px >= (lo & 0xFFFFu) && px <= (hi & 0xFFFFu) && py >= (lo >> 16) && py <= (hi >> 16);
}

}  // namespace gsr
