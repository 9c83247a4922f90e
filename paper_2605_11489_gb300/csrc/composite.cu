// K6: front-to-back compositing with the analytic image gradients (paper
// Sec. 3, Eq. 2-4), plus depth and alpha, in one pass.
//
// Per pixel, over its tile's depth-sorted Gaussians:
//   a_i  = min(0.99, o_i exp(-Q/2)),  Q = d^T conic d, d = p - mu2D; skip a_i < 1/255
//   stop before a Gaussian with T (1 - a_i) < 1e-4
//   I   += c_i a_i T_i                                   (Eq. 2)
//   I_x += c_i (T_x,i a_i + T_i a_x,i), a_x = -a (conic d)_x, 0 when capped (Eq. 3)
//   T_x,i+1 = -a_x,i T_i + (1 - a_i) T_x,i               (Eq. 4), same in y
//   D   += z_i a_i T_i; at the end rgb = I + T bg, dC/dx = I_x + bg T_x, alpha = 1 - T.
// A Gaussian is evaluated only at pixels inside its support rectangle, which
// both skips most of a tile's pairs and makes the image independent of the
// tile size.
//
// GB300 layout: one CTA per TILE x TILE tile, one pixel per thread. The tile's
// records (48 B each, already gathered into sorted order, so a tile's list is
// contiguous) are staged into shared memory in batches of BATCH by one TMA
// bulk copy per batch (cp.async.bulk, completion counted on an mbarrier), in a
// ring of NSTAGE buffers so that NSTAGE-1 batches are in flight while one is
// blended. Every lane of a warp reads the same record (shared-memory
// broadcast). Per landed batch each warp builds, with one ballot per 32
// records, the mask of records whose rectangle reaches its pixel rows, and
// visits only those, in order. Warps whose pixels are all saturated skip
// (warp ballot); the CTA stops loading once every pixel is done. Tiles are
// dispatched heaviest first. Waits on the mbarriers are bounded.
#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr uint32_t kWaitTries = 1u << 22;
constexpr int kStages = 3;

template <int TILE, int BATCH>
struct TileSmem {
    GaussRec rec[kStages][BATCH];
    uint64_t bar[kStages];
};

struct PixelAcc {
    float T, Tx, Ty, D;
    float C[3], Cx[3], Cy[3];
    uint32_t last;
    bool done;
};

// Composites one tile. `phase` carries the mbarriers' parities across tiles
// (persistent use). Returns false if a bounded wait gave up.
template <int TILE, int BATCH, bool GRAD, bool STATE>
__device__ __forceinline__ bool composite_tile(const CompositeArgs &a, int tile_x, int tile_y,
                                               TileSmem<TILE, BATCH> &sm, uint32_t (&phase)[kStages])
{
    // each warp owns an 8 x 4 pixel block of the tile, so a small Gaussian's
    // support covers a large share of the warp's lanes and misses most warps
    constexpr int WX = 8, WY = 4, WPR = TILE / WX;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bx0 = tile_x * TILE + (warp % WPR) * WX, by0 = tile_y * TILE + (warp / WPR) * WY;
    const int px = bx0 + (lane % WX), py = by0 + (lane / WX);
    const bool inside = px < a.width && py < a.height;
    const uint2 range = a.ranges[tile_y * a.tiles_x + tile_x];
    const uint32_t total = range.y > range.x ? range.y - range.x : 0u;
    const int nbatches = (int)((total + BATCH - 1) / BATCH);

    // batch b -> buffer b % kStages; one bulk copy of the batch's contiguous records
    auto issue = [&](int b) {
        if (tid == 0) {
            const int buf = b % kStages;
            const uint32_t start = range.x + (uint32_t)b * BATCH;
            const uint32_t cnt = min((uint32_t)BATCH, range.y - start);
            const uint32_t bytes = cnt * (uint32_t)sizeof(GaussRec);
            mbar_arrive_expect_tx(&sm.bar[buf], bytes);
            tma_bulk_g2s(&sm.rec[buf][0], a.rec + start, bytes, &sm.bar[buf]);
        }
    };

    PixelAcc s;
    s.T = 1.0f;
    s.Tx = s.Ty = s.D = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) s.C[c] = s.Cx[c] = s.Cy[c] = 0.0f;
    s.last = 0;
    s.done = !inside;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint32_t upx = (uint32_t)px, upy = (uint32_t)py;
    const uint32_t wx0 = (uint32_t)bx0, wx1 = (uint32_t)(bx0 + WX - 1);
    const uint32_t wy0 = (uint32_t)by0, wy1 = (uint32_t)(by0 + WY - 1);
    bool ok = true;

    for (int b = 0; b < kStages - 1 && b < nbatches; ++b) issue(b);
    int b = 0;
    for (; b < nbatches; ++b) {
        const int buf = b % kStages;
        if (b + kStages - 1 < nbatches) issue(b + kStages - 1);
        if (!mbar_wait_bounded(&sm.bar[buf], phase[buf], kWaitTries)) ok = false;
        phase[buf] ^= 1u;
        const uint32_t cnt = min((uint32_t)BATCH, range.y - (range.x + (uint32_t)b * BATCH));
        const bool warp_idle = __all_sync(0xffffffffu, s.done || !ok);
        if (ok && !warp_idle) {
            const GaussRec *recs = sm.rec[buf];
            // which of the batch's records reach this warp's pixel block (one ballot per 32 records)
            uint32_t rows_mask[BATCH / 32];
#pragma unroll
            for (int w = 0; w < BATCH / 32; ++w) {
                const uint32_t k = (uint32_t)w * 32u + (uint32_t)lane;
                bool hit = false;
                if (k < cnt) {
                    const uint32_t lo = __float_as_uint(recs[k].r2.z), hi = __float_as_uint(recs[k].r2.w);
                    hit = (hi >> 16) >= wy0 && (lo >> 16) <= wy1 && (hi & 0xFFFFu) >= wx0 && (lo & 0xFFFFu) <= wx1;
                }
                rows_mask[w] = __ballot_sync(0xffffffffu, hit);
            }
#pragma unroll
            for (int w = 0; w < BATCH / 32; ++w) {
                uint32_t m = s.done ? 0u : rows_mask[w];
                while (m) {
                    const uint32_t k = (uint32_t)w * 32u + (uint32_t)(__ffs(m) - 1);
                    m &= m - 1u;
                    const float4 r2 = recs[k].r2;
                    if (!rect_contains(r2, upx, upy)) continue;
                    const float4 r0 = recs[k].r0;
                    const float4 r1 = recs[k].r1;
                    const AlphaEval e = eval_alpha(r0, r1, pxc, pyc);
                    const float al = e.al;
                    if (al < kAlphaMin) continue;
                    const float om = __fsub_rn(1.0f, al);
                    const float nT = __fmul_rn(s.T, om);
                    if (nT < kTMin) {
                        s.done = true;
                        break;
                    }
                    const float wgt = __fmul_rn(al, s.T);
                    const float col[3] = {r1.w, r2.x, r2.y};
#pragma unroll
                    for (int c = 0; c < 3; ++c) s.C[c] = __fmaf_rn(col[c], wgt, s.C[c]);
                    s.D = __fmaf_rn(r1.z, wgt, s.D);
                    if (GRAD) {
                        const float ax = e.capped ? 0.0f : -__fmul_rn(al, e.ex);
                        const float ay = e.capped ? 0.0f : -__fmul_rn(al, e.ey);
                        const float wx = __fmaf_rn(s.Tx, al, __fmul_rn(s.T, ax));
                        const float wy = __fmaf_rn(s.Ty, al, __fmul_rn(s.T, ay));
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            s.Cx[c] = __fmaf_rn(col[c], wx, s.Cx[c]);
                            s.Cy[c] = __fmaf_rn(col[c], wy, s.Cy[c]);
                        }
                        s.Tx = __fmaf_rn(-ax, s.T, __fmul_rn(om, s.Tx));
                        s.Ty = __fmaf_rn(-ay, s.T, __fmul_rn(om, s.Ty));
                    }
                    s.T = nT;
                    if (STATE) s.last = (uint32_t)b * BATCH + k + 1u;
                }
            }
        }
        if (!ok) s.done = true;
        if (__syncthreads_and(s.done)) {
            ++b;
            break;
        }
    }
    // batches issued ahead of an early exit must land before their buffers are reused or the CTA exits
    for (int q = b; q < nbatches && q < b + kStages - 1; ++q) {
        if (!mbar_wait_bounded(&sm.bar[q % kStages], phase[q % kStages], kWaitTries)) ok = false;
        phase[q % kStages] ^= 1u;
    }
    if (inside) {
        const int64_t HW = (int64_t)a.width * a.height;
        const int64_t p = (int64_t)py * a.width + px;
        if (a.rgb)
#pragma unroll
            for (int c = 0; c < 3; ++c) a.rgb[c * HW + p] = __fmaf_rn(s.T, a.bg[c], s.C[c]);
        if (GRAD) {
            if (a.dcdx)
#pragma unroll
                for (int c = 0; c < 3; ++c) a.dcdx[c * HW + p] = __fmaf_rn(a.bg[c], s.Tx, s.Cx[c]);
            if (a.dcdy)
#pragma unroll
                for (int c = 0; c < 3; ++c) a.dcdy[c * HW + p] = __fmaf_rn(a.bg[c], s.Ty, s.Cy[c]);
        }
        if (a.depth) a.depth[p] = s.D;
        if (a.alpha) a.alpha[p] = __fsub_rn(1.0f, s.T);
        if (STATE) {
            a.final_T[p] = s.T;
            a.final_Tx[p] = s.Tx;
            a.final_Ty[p] = s.Ty;
            a.n_contrib[p] = s.last;
        }
    }
    return ok;
}

template <int TILE, int BATCH>
__device__ __forceinline__ void init_barriers(TileSmem<TILE, BATCH> &sm)
{
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

template <int TILE, int BATCH, bool GRAD, bool STATE>
__global__ void __launch_bounds__(TILE *TILE) k_composite(const CompositeArgs a)
{
    __shared__ TileSmem<TILE, BATCH> sm;
    init_barriers(sm);
    uint32_t phase[kStages] = {};
    // heaviest tiles first: CTAs are dispatched roughly in blockIdx order
    const uint32_t t = a.tile_order ? a.tile_order[blockIdx.x] : blockIdx.x;
    const int tx = (int)(t % (uint32_t)a.tiles_x), ty = (int)(t / (uint32_t)a.tiles_x);
    const bool ok = composite_tile<TILE, BATCH, GRAD, STATE>(a, tx, ty, sm, phase);
    if (!ok && threadIdx.x == 0) atomicOr(a.err_word, kErrTmaTimeout);
}

// Serving: a persistent grid pulls (request, tile) items from a flat work list
// described by per-request prefixes; every request's outputs and buffers are
// its own. Items are handed out by an atomic counter (no waiting on anything).
constexpr int kMaxServeReqs = 256;

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE *TILE) k_composite_persistent(const ServeItem *__restrict__ reqs, int n_reqs,
                                                                     uint32_t total_items, uint32_t *work_counter)
{
    __shared__ TileSmem<TILE, BATCH> sm;
    __shared__ uint32_t s_first[kMaxServeReqs + 1];
    __shared__ uint32_t s_item;
    for (int r = threadIdx.x; r < n_reqs; r += blockDim.x) s_first[r] = reqs[r].first_item;
    if (threadIdx.x == 0) s_first[n_reqs] = total_items;
    init_barriers(sm);
    uint32_t phase[kStages] = {};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work_counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total_items) break;
        int lo = 0, hi = n_reqs - 1;  // last request with first_item <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const CompositeArgs &a = reqs[lo].args;
        uint32_t t = item - s_first[lo];
        if (a.tile_order) t = a.tile_order[t];
        const int tx = (int)(t % (uint32_t)a.tiles_x), ty = (int)(t / (uint32_t)a.tiles_x);
        bool ok;
        if (a.dcdx || a.dcdy) ok = composite_tile<TILE, BATCH, true, false>(a, tx, ty, sm, phase);
        else ok = composite_tile<TILE, BATCH, false, false>(a, tx, ty, sm, phase);
        if (!ok && threadIdx.x == 0) atomicOr(a.err_word, kErrTmaTimeout);
        __syncthreads();
    }
}

template <int TILE, int BATCH>
cudaError_t launch_tb(const CompositeArgs &a, cudaStream_t s)
{
    const dim3 grid(a.tiles_x * a.tiles_y);
    const bool grad = a.dcdx || a.dcdy;
    const bool state = a.final_T != nullptr;
    if (grad && state) k_composite<TILE, BATCH, true, true><<<grid, TILE * TILE, 0, s>>>(a);
    else if (grad) k_composite<TILE, BATCH, true, false><<<grid, TILE * TILE, 0, s>>>(a);
    else if (state) k_composite<TILE, BATCH, false, true><<<grid, TILE * TILE, 0, s>>>(a);
    else k_composite<TILE, BATCH, false, false><<<grid, TILE * TILE, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TILE>
cudaError_t launch_t(const CompositeArgs &a, int batch, cudaStream_t s)
{
    switch (batch) {
    case 32: return launch_tb<TILE, 32>(a, s);
    case 64: return launch_tb<TILE, 64>(a, s);
    case 128: return launch_tb<TILE, 128>(a, s);
    default: return launch_tb<TILE, 256>(a, s);
    }
}

template <int TILE, int BATCH>
int persistent_grid()
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite_persistent<TILE, BATCH>, TILE * TILE, 0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
}

}  // namespace

bool composite_supported(int tile, int batch)
{
    return (tile == 8 || tile == 16 || tile == 32) && (batch == 32 || batch == 64 || batch == 128 || batch == 256);
}

cudaError_t launch_composite(const CompositeArgs &a, int tile, int batch, cudaStream_t s)
{
    if (a.tiles_x == 0 || a.tiles_y == 0) return cudaSuccess;
    switch (tile) {
    case 8: return launch_t<8>(a, batch, s);
    case 16: return launch_t<16>(a, batch, s);
    default: return launch_t<32>(a, batch, s);
    }
}

int composite_persistent_grid(int tile, int batch)
{
    (void)batch;
    if (tile == 8) return persistent_grid<8, 128>();
    if (tile == 32) return persistent_grid<32, 128>();
    return persistent_grid<16, 128>();
}

cudaError_t launch_composite_persistent(const ServeItem *reqs, int n_reqs, uint32_t total_items, int tile, int batch,
                                        uint32_t *work_counter, int grid, cudaStream_t s)
{
    (void)batch;
    if (n_reqs <= 0 || total_items == 0) return cudaSuccess;
    if (n_reqs > kMaxServeReqs) return cudaErrorInvalidValue;
    if (tile == 8) k_composite_persistent<8, 128><<<grid, 64, 0, s>>>(reqs, n_reqs, total_items, work_counter);
    else if (tile == 32) k_composite_persistent<32, 128><<<grid, 1024, 0, s>>>(reqs, n_reqs, total_items, work_counter);
    else k_composite_persistent<16, 128><<<grid, 256, 0, s>>>(reqs, n_reqs, total_items, work_counter);
    return cudaGetLastError();
}

}  // namespace gsr
