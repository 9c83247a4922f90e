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
// GB300 layout: one CTA per work item (a tile, or a chunk of a long tile
// list), one pixel per thread, and every warp an independent 8x4 pixel block
// with its own shared-memory ring of kStages batches of BATCH records and its
// own mbarriers. The next batches are staged while the warp blends the current
// one: from the tile's contiguous sorted records (the frames that keep that copy:
// the normal channels), lane 0 issues one TMA bulk copy per batch (cp.async.bulk,
// completion counted on the warp's mbarrier); in every other frame each lane
// gathers its batch positions' records by Gaussian index (cp.async, one group
// per batch), so no sorted copy is made. Per
// group of 32 records, each lane forms the mask of block pixels inside one
// record's rectangle, and a warp-wide bit transpose of those masks gives each
// lane the records whose rectangle holds its own pixel; it blends only these,
// in order. While forming the masks each lane also rewrites its record's centre
// in the warp's ring copy relative to the warp's block (block_centre), so a
// pixel's offset from it is one subtraction of small numbers. No barrier
// spans warps: a warp whose pixels are all saturated stops on its own. The
// tile's list is read once per warp from L2 (DRAM once). Waits are bounded.
//
// Load balance. The plan (launch_plan) orders the tiles longest first and
// separates the long ones (list longer than `head` records). k_composite takes
// the short tiles, one CTA each. k_composite_long runs beside it on a second
// stream: a persistent grid whose 16-warp CTAs take (long tile, group of 8x4 pixel
// blocks) items from a counter, with G warps per block (8 for a two-block group,
// 16 for a one-block group). Warp j of a block takes the j-th of g depth-contiguous
// chunks of the list (g = min(G, ceil(len / chunk))) and composites it from the
// identity state into a per-pixel partial state (C, C_x, C_y, D, T, T_x, T_y) in
// shared memory. Two segments a, b compose exactly as
//   C = Ca + Ta Cb,  C_x = Cxa + Txa Cb + Ta Cxb,  D = Da + Ta Db,
//   T = Ta Tb,       T_x = Txa Tb + Ta Txb                     (product rule)
// which equals the sequential result as long as no Gaussian of the tile was
// cut off by the T < 1e-4 stop. T only decreases, so a pixel's stop falls in
// chunk c exactly when c stopped locally or (prefix T) * (chunk T) < 1e-4.
// After one barrier, every warp follows that product chain for its pixels:
//   - the warp of the chunk holding a pixel's stop folds the chunks in front
//     of it into the exact prefix state and walks on from the chunk's start
//     until the pixel stops (chunk 0 needs no walk: its state is exact);
//   - the last chunk's warp writes the pixels that stop in no chunk, folding
//     all chunks front to back;
// so every pixel is written exactly once, by one warp, in one launch.
#include "gsr_internal.cuh"
#include <algorithm>

namespace gsr {
namespace {

constexpr uint32_t kWaitTries = 1u << 22;
constexpr int kStages = 3;
constexpr int kPartialVals = 15;  // floats per pixel in a partial state
constexpr int kMaxSmem = 227 * 1024;

template <int BATCH>
struct WarpRing {
    GaussRec rec[kStages][BATCH];
    uint64_t bar[kStages];
};

template <int TILE, int BATCH>
constexpr size_t smem_bytes()
{
    return sizeof(WarpRing<BATCH>) * (size_t)(TILE * TILE / 32);
}

struct PixelAcc {
    float T, Tx, Ty, D;
    float C[3], Cx[3], Cy[3];
    float N[3];  // normal channel (the NRM instantiations only)
    float Di;    // intersection depth (the NRM instantiations only)
    uint32_t last;
    uint32_t n_eval, n_blend;  // pairs counted in the GS_COUNT_PAIRS instantiation only
    bool done, stopped;
};

__device__ __forceinline__ void acc_init(PixelAcc &s, bool inside)
{
    s.T = 1.0f;
    s.Tx = s.Ty = s.D = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) s.C[c] = s.Cx[c] = s.Cy[c] = s.N[c] = 0.0f;
    s.Di = 0.0f;
    s.last = 0;
    s.done = !inside;
    s.stopped = false;
    s.n_eval = s.n_blend = 0;
}

// Pixel of thread `tid`: warps own 8x4 blocks, row-major over the tile.
template <int TILE>
__device__ __forceinline__ void tile_pixel(int tid, int tile_x, int tile_y, int &px, int &py, int &bx0, int &by0)
{
    constexpr int WX = 8, WY = 4, WPR = TILE / WX;
    const int warp = tid >> 5, lane = tid & 31;
    bx0 = tile_x * TILE + (warp % WPR) * WX;
    by0 = tile_y * TILE + (warp / WPR) * WY;
    px = bx0 + (lane % WX);
    py = by0 + (lane / WX);
}

// One Gaussian record at one pixel (Eq. 2-4). Returns true when the pixel
// stops (the record would take T below 1e-4; it is not blended).
template <bool GRAD, bool STATE, bool COUNT = false, bool NRM = false>
__device__ __forceinline__ bool blend(PixelAcc &s, const float4 &r0, const float4 &r1, const float4 &r2, float lx,
                                      float ly, uint32_t pos, const float4 *nrm = nullptr,
                                      const float2 *plane = nullptr)
{
    if (COUNT) ++s.n_eval;
    const AlphaEval e = eval_alpha(r0, r1, lx, ly);  // r0's centre relative to the block (block_centre)
    const float al = e.al;
    if (al < kAlphaMin) return false;
    const float om = __fsub_rn(1.0f, al);
    const float nT = __fmul_rn(s.T, om);
    if (nT < kTMin) return true;
    const float wgt = __fmul_rn(al, s.T);
    const float col[3] = {r1.w, r2.x, r2.y};
#pragma unroll
    for (int c = 0; c < 3; ++c) s.C[c] = __fmaf_rn(col[c], wgt, s.C[c]);
    s.D = __fmaf_rn(r1.z, wgt, s.D);
    if (NRM) {  // the record's normal, blended like the colour
        const float4 n = __ldg(nrm);
        s.N[0] = __fmaf_rn(n.x, wgt, s.N[0]);
        s.N[1] = __fmaf_rn(n.y, wgt, s.N[1]);
        s.N[2] = __fmaf_rn(n.z, wgt, s.N[2]);
        // the intersection depth at this pixel, z + (dz/du, dz/dv) . (p - mu2D), blended
        // like the colour
        const float2 pl = __ldg(plane);
        s.Di = __fmaf_rn(__fmaf_rn(pl.x, e.dx, __fmaf_rn(pl.y, e.dy, r1.z)), wgt, s.Di);
    }
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
    if (STATE) s.last = pos;
    if (COUNT) ++s.n_blend;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// gather mode: one 16-byte piece global -> shared (through L2), per-lane groups
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 32x32 bit-matrix transpose across a warp: lane j holds row j (bit L = column
// L); returns column `lane` (bit j = row j's bit `lane`). Five butterfly stages,
// each swapping the off-diagonal blocks of the next-smaller block size.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
    const uint32_t keep[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sh = 16 >> k;
        const uint32_t m = keep[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y >> sh) & m)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

template <int BATCH>
__device__ __forceinline__ void ring_init(WarpRing<BATCH> &ring)
{
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&ring.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// Warp-level: composites records [s0, s1) of the sorted list onto this lane's
// pixel state. (px, py) is the lane's pixel, (bx0, by0) the warp's 8x4 block,
// pos0 the list position of s0 within its tile. The warp's ring carries its
// mbarrier parities in `phase`. Returns false if a bounded wait gave up.
template <int BATCH, bool GRAD, bool STATE, bool COUNT = false, bool NRM = false>
__device__ __forceinline__ bool warp_span(const CompositeArgs &a, int px, int py, int bx0, int by0, uint32_t s0,
                                          uint32_t s1, uint32_t pos0, WarpRing<BATCH> &ring,
                                          uint32_t (&phase)[kStages], PixelAcc &s)
{
    const int lane = threadIdx.x & 31;
    const uint32_t total = s1 > s0 ? s1 - s0 : 0u;
    const int nbatches = (int)((total + BATCH - 1) / BATCH);
    if (__all_sync(0xffffffffu, s.done) || nbatches == 0) return true;

    // batch b -> ring slot b % kStages. Sorted records: lane 0 issues one bulk copy per batch,
    // counted on the slot's mbarrier. Gather mode: each lane copies the records of its batch
    // positions (lane, lane + 32, ...) by index, three 16-byte pieces each, as one cp.async
    // group per batch; every lane commits exactly one group per batch slot (empty past the
    // list), so waiting for all but the newest kStages - 1 groups waits for batch b.
    // The indices of the next batch to gather are loaded when the current one is issued, so
    // they arrive while the warp blends.
    const bool gather = a.rec_index != nullptr;
    uint32_t next_idx[BATCH / 32];
    auto load_idx = [&](int b) {
        const uint32_t start = s0 + (uint32_t)b * BATCH;
        const uint32_t cnt = b < nbatches ? min((uint32_t)BATCH, s1 - start) : 0u;
#pragma unroll
        for (int w = 0; w < BATCH / 32; ++w) {
            const uint32_t j = (uint32_t)(w * 32 + lane);
            next_idx[w] = j < cnt ? __ldg(a.vals + start + j) : 0u;
        }
    };
    if (gather) load_idx(0);
    auto issue = [&](int b) {
        if (gather) {
            const int buf = b % kStages;
            const uint32_t start = s0 + (uint32_t)b * BATCH;
            const uint32_t cnt = min((uint32_t)BATCH, s1 - start);
#pragma unroll
            for (int w = 0; w < BATCH / 32; ++w) {
                const uint32_t j = (uint32_t)(w * 32 + lane);
                if (j >= cnt) break;
                uint32_t g = next_idx[w];
                if (!GSR_IN_BOUNDS(g, a.n_gauss, a.err_word)) g = 0u;
                const float4 *src = reinterpret_cast<const float4 *>(a.rec_index + g);
                float4 *dst = reinterpret_cast<float4 *>(&ring.rec[buf][j]);
                cp_async16(dst, src);
                cp_async16(dst + 1, src + 1);
                cp_async16(dst + 2, src + 2);
            }
            cp_async_commit();
            load_idx(b + 1);
        } else if (lane == 0) {
            const int buf = b % kStages;
            const uint32_t start = s0 + (uint32_t)b * BATCH;
            const uint32_t cnt = min((uint32_t)BATCH, s1 - start);
            const uint32_t bytes = cnt * (uint32_t)sizeof(GaussRec);
            fence_proxy_async_smem();  // this warp's earlier reads of the slot precede the async write
            mbar_arrive_expect_tx(&ring.bar[buf], bytes);
            tma_bulk_g2s(&ring.rec[buf][0], a.rec + start, bytes, &ring.bar[buf]);
        }
    };

    const float lx = block_px(px), ly = block_py(py);
    bool ok = true;

    for (int b = 0; b < kStages - 1; ++b) {
        if (b < nbatches) issue(b);
        else if (gather) cp_async_commit();
    }
    int b = 0;
    const uint32_t first_tries = a.give_up ? 0u : kWaitTries;
    for (; b < nbatches; ++b) {
        const int buf = b % kStages;
        __syncwarp();  // the lanes' reads and writes of block centres in the slot precede its refill
        if (b + kStages - 1 < nbatches) issue(b + kStages - 1);
        else if (gather) cp_async_commit();
        if (gather) {
            cp_async_wait<kStages - 1>();  // this lane's copies of batch b have landed
            __syncwarp();                  // and every other lane's
        } else {
            if (!mbar_wait_bounded(&ring.bar[buf], phase[buf], first_tries)) ok = false;
            if (!__all_sync(0xffffffffu, ok)) {  // batch b is still in flight: drained below
                ok = false;                      // (the same on every lane, so the drain is too)
                break;
            }
            phase[buf] ^= 1u;
        }
        const uint32_t cnt = min((uint32_t)BATCH, s1 - (s0 + (uint32_t)b * BATCH));
        GaussRec *recs = ring.rec[buf];  // this warp's own staged copy
        const uint32_t pos_b = pos0 + (uint32_t)b * BATCH + 1u;
#pragma unroll
        for (int w = 0; w < BATCH / 32; ++w) {
            // Each lane takes record w*32 + lane of the batch and forms the mask of
            // the warp's 8x4 block pixels (bit 8*row + column = the lane owning that
            // pixel) inside its support rectangle; a transpose of these 32 masks
            // across the warp gives every lane its own list: the records of the
            // group whose rectangle holds its pixel, in list order. Each lane then
            // blends only these, at its own pace.
            const uint32_t kk = (uint32_t)w * 32u + (uint32_t)lane;
            uint32_t cover = 0u;
            if (kk < cnt) {
                const uint32_t lo = __float_as_uint(recs[kk].r2.z), hi = __float_as_uint(recs[kk].r2.w);
                const int x0 = max((int)(lo & 0xFFFFu) - bx0, 0), x1 = min((int)(hi & 0xFFFFu) - bx0, 7);
                const int y0 = max((int)(lo >> 16) - by0, 0), y1 = min((int)(hi >> 16) - by0, 3);
                if (x0 <= x1 && y0 <= y1) {
                    const uint32_t xm = (0xFFu >> (7 - x1)) & (0xFFu << x0);
                    const uint32_t rows = (0xFu >> (3 - y1)) & (0xFu << y0);
                    cover = xm * ((rows & 1u) | ((rows & 2u) << 7) | ((rows & 4u) << 14) | ((rows & 8u) << 21));
                    // the record's centre relative to this warp's block, once per record
                    const float2 cb = block_centre(recs[kk].r0, recs[kk].r2, bx0, by0);
                    recs[kk].r0.x = cb.x;
                    recs[kk].r0.y = cb.y;
                }
            }
            if (!__any_sync(0xffffffffu, cover != 0u)) continue;
            __syncwarp();  // the block-relative centres are written before other lanes read them
            uint32_t mine = warp_transpose32(cover, lane);
            if (s.done) mine = 0u;
            if (mine) {  // the next record's loads are issued before the current one is blended
                uint32_t k = (uint32_t)w * 32u + (uint32_t)(__ffs(mine) - 1);
                mine &= mine - 1u;
                float4 a0 = recs[k].r0, a1 = recs[k].r1, a2 = recs[k].r2;
                for (;;) {
                    const bool more = mine != 0u;
                    const uint32_t kn = more ? (uint32_t)w * 32u + (uint32_t)(__ffs(mine) - 1) : k;
                    mine &= mine - 1u;
                    const float4 b0 = recs[kn].r0, b1 = recs[kn].r1, b2 = recs[kn].r2;
                    if (blend<GRAD, STATE, COUNT, NRM>(
                            s, a0, a1, a2, lx, ly, pos_b + k,
                            NRM ? a.nrm_sorted + (s0 + (uint32_t)b * BATCH + k) : nullptr,
                            NRM ? a.plane_sorted + (s0 + (uint32_t)b * BATCH + k) : nullptr)) {
                        s.done = true;
                        s.stopped = true;
                        break;
                    }
                    if (!more) break;
                    k = kn;
                    a0 = b0;
                    a1 = b1;
                    a2 = b2;
                }
            }
        }
        if (__all_sync(0xffffffffu, s.done)) {
            ++b;
            break;
        }
    }
    // Batches issued ahead of an early exit must land before their slots are reused or the
    // CTA exits: after a warp finishes batch b - 1 early, batches b .. b + kStages - 2 are in
    // flight; after a wait on batch b gives up, batches b .. b + kStages - 1 are (b's own copy
    // included). Each is waited for with the full bound.
    if (gather) {
        cp_async_wait<0>();  // the copies issued ahead of an early exit, before the slots are reused
        __syncwarp();
        return ok;
    }
    const int in_flight_end = ok ? b + kStages - 1 : b + kStages;
    for (int q = b; q < nbatches && q < in_flight_end; ++q) {
        if (!mbar_wait_bounded(&ring.bar[q % kStages], phase[q % kStages], kWaitTries)) ok = false;
        phase[q % kStages] ^= 1u;
    }
    __syncwarp();
    return ok;
}

template <bool GRAD, bool STATE, bool NRM = false>
__device__ __forceinline__ void write_final(const CompositeArgs &a, int px, int py, const PixelAcc &s)
{
    const int64_t HW = (int64_t)a.width * a.height;
    const int64_t p = (int64_t)py * a.width + px;
    if (!GSR_IN_BOUNDS(p, HW, a.err_word)) return;
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
    if (NRM) {
        if (a.normal)
#pragma unroll
            for (int c = 0; c < 3; ++c) a.normal[c * HW + p] = s.N[c];
        if (a.nv) {  // -normal . (unit ray of the pixel centre)
            const float rx = ((float)px + 0.5f - a.cx) / a.fx, ry = ((float)py + 0.5f - a.cy) / a.fy;
            const float inv = rsqrtf(rx * rx + ry * ry + 1.0f);
            a.nv[p] = -(s.N[0] * rx + s.N[1] * ry + s.N[2]) * inv;
        }
        if (a.depth_isect) a.depth_isect[p] = s.Di;
    }
    if (STATE) {
        a.final_T[p] = s.T;
        a.final_Tx[p] = s.Tx;
        a.final_Ty[p] = s.Ty;
        a.n_contrib[p] = s.last;
    }
}

// Partial state of one pixel over one chunk, in k_composite_long's shared memory:
// planar [value][NT] per chunk (NT pixels of the tile), so a warp's 32 pixels
// fall in 32 banks. Values: C[3], C_x[3], C_y[3], D, T, T_x, T_y, last, stopped.
template <int NT>
__device__ __forceinline__ void write_partial(float *part, int pix, const PixelAcc &s)
{
    const float v[kPartialVals] = {s.C[0],  s.C[1], s.C[2], s.Cx[0], s.Cx[1], s.Cx[2], s.Cy[0],
                                   s.Cy[1], s.Cy[2], s.D,   s.T,     s.Tx,    s.Ty,    __uint_as_float(s.last),
                                   s.stopped ? 1.0f : 0.0f};
#pragma unroll
    for (int k = 0; k < kPartialVals; ++k) part[k * NT + pix] = v[k];
}

template <int NT>
__device__ __forceinline__ void read_partial(const float *part, int pix, PixelAcc &q)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        q.C[c] = part[c * NT + pix];
        q.Cx[c] = part[(3 + c) * NT + pix];
        q.Cy[c] = part[(6 + c) * NT + pix];
    }
    q.D = part[9 * NT + pix];
    q.T = part[10 * NT + pix];
    q.Tx = part[11 * NT + pix];
    q.Ty = part[12 * NT + pix];
    q.last = __float_as_uint(part[13 * NT + pix]);
    q.stopped = part[14 * NT + pix] != 0.0f;
}

// P <- P then Q (composition of two consecutive segments, product rule)
template <bool GRAD, bool STATE>
__device__ __forceinline__ void compose(PixelAcc &P, const PixelAcc &Q)
{
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        if (GRAD) {
            P.Cx[ch] = __fmaf_rn(P.T, Q.Cx[ch], __fmaf_rn(P.Tx, Q.C[ch], P.Cx[ch]));
            P.Cy[ch] = __fmaf_rn(P.T, Q.Cy[ch], __fmaf_rn(P.Ty, Q.C[ch], P.Cy[ch]));
        }
        P.C[ch] = __fmaf_rn(P.T, Q.C[ch], P.C[ch]);
    }
    P.D = __fmaf_rn(P.T, Q.D, P.D);
    if (GRAD) {
        const float tx2 = __fmaf_rn(P.Tx, Q.T, __fmul_rn(P.T, Q.Tx));
        const float ty2 = __fmaf_rn(P.Ty, Q.T, __fmul_rn(P.T, Q.Ty));
        P.Tx = tx2;
        P.Ty = ty2;
    }
    P.T = __fmul_rn(P.T, Q.T);
    if (STATE && Q.last) P.last = Q.last;
}

// The short tiles of the plan: CTA i composites tile_order[n_long + i], one warp
// per 8x4 pixel block over the whole list.
template <int TILE, int BATCH, bool GRAD, bool STATE, bool COUNT = false, bool NRM = false>
__global__ void __launch_bounds__(TILE *TILE) k_composite(const CompositeArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (blockIdx.x >= a.plan[2]) return;
    const uint32_t tile = a.tile_order[a.plan[0] + blockIdx.x];
    if (!GSR_IN_BOUNDS(tile, (uint32_t)(a.tiles_x * a.tiles_y), a.err_word)) return;
    const uint2 r = a.ranges[tile];
    const uint32_t s0 = r.x, s1 = r.y > r.x ? r.y : r.x;
    WarpRing<BATCH> &ring = reinterpret_cast<WarpRing<BATCH> *>(smem_raw)[threadIdx.x >> 5];
    ring_init(ring);
    uint32_t phase[kStages] = {};
    const int tx = (int)(tile % (uint32_t)a.tiles_x), ty = (int)(tile / (uint32_t)a.tiles_x);
    int px, py, bx0, by0;
    tile_pixel<TILE>(threadIdx.x, tx, ty, px, py, bx0, by0);
    const bool inside = px < a.width && py < a.height;
    PixelAcc s;
    acc_init(s, inside);
    const bool ok = warp_span<BATCH, GRAD, STATE, COUNT, NRM>(a, px, py, bx0, by0, s0, s1, 0u, ring, phase, s);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(a.err_word, kErrTmaTimeout);
    if (COUNT) {  // evaluated (inside a support rectangle) and blended pairs of this warp
        unsigned long long ne = s.n_eval, nb = s.n_blend;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ne += __shfl_xor_sync(0xffffffffu, ne, o);
            nb += __shfl_xor_sync(0xffffffffu, nb, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.pair_counts, ne);
            atomicAdd(a.pair_counts + 1, nb);
        }
    }
    if (inside) write_final<GRAD, STATE, NRM>(a, px, py, s);
}

// The long tiles of the plan (the load-balance note at the top): a persistent grid
// whose CTAs of kLongWarps warps take (long tile, group of BPC pixel blocks) items from the
// plan's counter. Warp w owns pixel block w % BPC of the group and chunk j = w / BPC of the
// tile's list; a list of `len` records has g = min(G, ceil(len / chunk)) chunks of
// ceil(len / g) records, G = kLongWarps / BPC. BPC = 2 (a whole 8x8 tile, 8 chunk warps per
// block) measured best on lists of a few hundred records on average; BPC = 1 (16 chunk warps
// per block) serves longer lists and the larger tiles.
constexpr int kLongBatch = 32;
constexpr int kLongWarps = 16;
__host__ __device__ constexpr size_t long_smem_bytes()
{
    return sizeof(WarpRing<kLongBatch>) * (size_t)kLongWarps + sizeof(float) * kPartialVals * 32 * kLongWarps;
}

template <int TILE, int BPC, bool GRAD, bool STATE>
__global__ void __launch_bounds__(kLongWarps * 32) k_composite_long(const CompositeArgs a)
{
    constexpr int NB = TILE * TILE / 32, G = kLongWarps / BPC, NP = BPC * 32, GROUPS = NB / BPC;
    static_assert(NB % BPC == 0 && kLongWarps % BPC == 0, "blocks per CTA must divide the tile and the CTA");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t j = (uint32_t)(warp / BPC);
    const int q = (warp % BPC) * 32 + lane;  // the pixel's index within the group's NP pixels
    WarpRing<kLongBatch> &ring = reinterpret_cast<WarpRing<kLongBatch> *>(smem_raw)[warp];
    // per chunk, planar [value][NP pixels]
    float *const part = reinterpret_cast<float *>(smem_raw + sizeof(WarpRing<kLongBatch>) * kLongWarps);
    ring_init(ring);
    uint32_t phase[kStages] = {};
    bool ok = true;
    const uint32_t n_items = a.plan[0] * (uint32_t)GROUPS;
    const uint32_t chunk = (uint32_t)max(a.chunk, 1);
    for (;;) {
        __syncthreads();  // every warp is done with the previous item's partial states
        if (threadIdx.x == 0) s_item = atomicAdd(a.long_counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) break;
        const uint32_t tile = a.tile_order[item / GROUPS];
        const int pix = (int)(item % GROUPS) * NP + q;  // the pixel's index in the tile, as in k_composite
        const uint2 r = a.ranges[tile];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        const uint32_t g = max(1u, min((uint32_t)G, (len + chunk - 1) / chunk));
        const uint32_t cl = (len + g - 1) / g;
        const int tx = (int)(tile % (uint32_t)a.tiles_x), ty = (int)(tile / (uint32_t)a.tiles_x);
        int px, py, bx0, by0;
        tile_pixel<TILE>(pix, tx, ty, px, py, bx0, by0);
        const bool inside = px < a.width && py < a.height;
        // phase 1: chunk j from the identity state
        const uint32_t c0 = min(len, j * cl), c1 = min(len, c0 + cl);
        PixelAcc s;
        acc_init(s, inside && j < g);
        if (j < g) ok &= warp_span<kLongBatch, GRAD, STATE>(a, px, py, bx0, by0, r.x + c0, r.x + c1, c0, ring, phase, s);
        write_partial<NP>(part + (size_t)j * kPartialVals * NP, q, s);
        __syncthreads();
        if (j >= g) continue;
        // phase 2: the chunk holding the pixel's stop, from the product chain of the
        // chunks' T (the same chain in every warp): -1 before j, 0 in j, 1 not up to j
        int rel = 1;
        float T = 1.0f;
        for (uint32_t i = 0; i <= j; ++i) {
            const float *pi = part + (size_t)i * kPartialVals * NP;
            const float Ti = pi[10 * NP + q];
            if (pi[14 * NP + q] != 0.0f || __fmul_rn(T, Ti) < kTMin) {
                rel = i < j ? -1 : 0;
                break;
            }
            T = __fmul_rn(T, Ti);
        }
        if (inside && rel == 0 && j == 0) write_final<GRAD, STATE>(a, px, py, s);  // exact: from the identity
        if (inside && rel == 1 && j == g - 1) {  // stops in no chunk: all chunks, front to back
            PixelAcc P;
            acc_init(P, true);
            for (uint32_t i = 0; i < j; ++i) {
                PixelAcc Q;
                read_partial<NP>(part + (size_t)i * kPartialVals * NP, q, Q);
                compose<GRAD, STATE>(P, Q);
            }
            compose<GRAD, STATE>(P, s);
            write_final<GRAD, STATE>(a, px, py, P);
        }
        // the stop falls in chunk j > 0: the exact prefix state, then a walk from the
        // chunk's start until the pixel stops (on into later chunks if rounding has it
        // stop later, which continues the sequential pass exactly)
        const bool walk = inside && rel == 0 && j > 0;
        if (__any_sync(0xffffffffu, walk)) {
            PixelAcc P;
            acc_init(P, walk);
            if (walk)
                for (uint32_t i = 0; i < j; ++i) {
                    PixelAcc Q;
                    read_partial<NP>(part + (size_t)i * kPartialVals * NP, q, Q);
                    compose<GRAD, STATE>(P, Q);
                }
            ok &= warp_span<kLongBatch, GRAD, STATE>(a, px, py, bx0, by0, r.x + c0, r.y, c0, ring, phase, P);
            if (walk) write_final<GRAD, STATE>(a, px, py, P);
        }
    }
    if (!ok && lane == 0) atomicOr(a.err_word, kErrTmaTimeout);
}
// Serving: a persistent grid pulls (request, tile) items from a flat work list
// described by per-request prefixes; every request's outputs and buffers are
// its own. Items are handed out by an atomic counter (no waiting on anything).
// A request with a plan (launch_plan) gives this kernel its short tiles only; its
// long tiles go to k_composite_long on the request's own stream.
constexpr int kMaxServeReqs = 256;
constexpr int kServeBatch = 32;

template <int TILE>
__global__ void __launch_bounds__(TILE *TILE) k_composite_persistent(const ServeItem *__restrict__ reqs, int n_reqs,
                                                                     uint32_t total_items, uint32_t *work_counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_first[kMaxServeReqs + 1];
    __shared__ uint32_t s_item;
    for (int r = threadIdx.x; r < n_reqs; r += blockDim.x) s_first[r] = reqs[r].first_item;
    if (threadIdx.x == 0) s_first[n_reqs] = total_items;
    WarpRing<kServeBatch> &ring = reinterpret_cast<WarpRing<kServeBatch> *>(smem_raw)[threadIdx.x >> 5];
    ring_init(ring);
    uint32_t phase[kStages] = {};
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(work_counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= total_items) break;
        int lo = 0, hi = n_reqs - 1;  // last request with first_item <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const CompositeArgs &a = reqs[lo].args;
        uint32_t t = item - s_first[lo];
        if (a.plan) {  // the request's long tiles are composited apart: its short ones, in plan order
            if (t >= a.plan[2]) continue;
            t = a.tile_order[a.plan[0] + t];
        } else if (a.tile_order) {
            t = a.tile_order[t];
        }
        const int tx = (int)(t % (uint32_t)a.tiles_x), ty = (int)(t / (uint32_t)a.tiles_x);
        int px, py, bx0, by0;
        tile_pixel<TILE>(threadIdx.x, tx, ty, px, py, bx0, by0);
        const bool inside = px < a.width && py < a.height;
        const uint2 rg = a.ranges[t];
        PixelAcc s;
        acc_init(s, inside);
        bool ok;
        const bool grad = a.dcdx || a.dcdy;
        const uint32_t e = rg.y > rg.x ? rg.y : rg.x;
        if (grad) ok = warp_span<kServeBatch, true, false>(a, px, py, bx0, by0, rg.x, e, 0, ring, phase, s);
        else ok = warp_span<kServeBatch, false, false>(a, px, py, bx0, by0, rg.x, e, 0, ring, phase, s);
        if (!ok && (threadIdx.x & 31) == 0) atomicOr(a.err_word, kErrTmaTimeout);
        if (inside) {
            if (grad) write_final<true, false>(a, px, py, s);
            else write_final<false, false>(a, px, py, s);
        }
    }
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel and device;
// done on the first (never captured) launch. `done` is the kernel's own flags.
template <class F>
cudaError_t opt_in_smem(F *kernel, size_t bytes, bool (&done)[64])
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <int TILE, int BATCH, bool GRAD, bool STATE, bool COUNT = false, bool NRM = false>
cudaError_t launch_one(const CompositeArgs &a, unsigned nb, cudaStream_t s)
{
    constexpr size_t smem = smem_bytes<TILE, BATCH>();
    static bool done[64];
    cudaError_t e = opt_in_smem(k_composite<TILE, BATCH, GRAD, STATE, COUNT, NRM>, smem, done);
    if (e != cudaSuccess) return e;
    k_composite<TILE, BATCH, GRAD, STATE, COUNT, NRM><<<nb, TILE * TILE, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TILE, int BATCH>
cudaError_t launch_tb(const CompositeArgs &a, cudaStream_t s)
{
    if constexpr (smem_bytes<TILE, BATCH>() > (size_t)kMaxSmem) {
        return cudaErrorInvalidValue;
    } else {
        const unsigned nb = (unsigned)(a.tiles_x * a.tiles_y);
        if (nb == 0) return cudaSuccess;
        const bool grad = a.dcdx || a.dcdy;
        const bool state = a.final_T != nullptr;
        if (a.nrm_sorted) {  // the normal channel: no backward state, no census, whole tiles
            if (state || a.pair_counts) return cudaErrorInvalidValue;
            return grad ? launch_one<TILE, BATCH, true, false, false, true>(a, nb, s)
                        : launch_one<TILE, BATCH, false, false, false, true>(a, nb, s);
        }
        if (a.pair_counts && !state)  // diagnostic pair census (GS_COUNT_PAIRS)
            return grad ? launch_one<TILE, BATCH, true, false, true>(a, nb, s)
                        : launch_one<TILE, BATCH, false, false, true>(a, nb, s);
        if (grad && state) return launch_one<TILE, BATCH, true, true>(a, nb, s);
        if (grad) return launch_one<TILE, BATCH, true, false>(a, nb, s);
        if (state) return launch_one<TILE, BATCH, false, true>(a, nb, s);
        return launch_one<TILE, BATCH, false, false>(a, nb, s);
    }
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

// CTAs of k_composite_long per SM (two of its 16-warp CTAs leave room for the short tiles' CTAs)
constexpr int kLongCtasPerSm = 2;

template <int TILE, int BPC, bool GRAD, bool STATE>
cudaError_t launch_long_one(const CompositeArgs &a, int64_t max_long, cudaStream_t s)
{
    constexpr size_t smem = long_smem_bytes();
    static bool done[64];
    cudaError_t e = opt_in_smem(k_composite_long<TILE, BPC, GRAD, STATE>, smem, done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t items = max_long * (TILE * TILE / 32 / BPC);
    const int64_t grid = std::min<int64_t>(items, (int64_t)std::max(sms, 1) * kLongCtasPerSm);
    if (grid <= 0) return cudaSuccess;
    k_composite_long<TILE, BPC, GRAD, STATE><<<(unsigned)grid, kLongWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TILE, int BPC>
cudaError_t launch_long_tb(const CompositeArgs &a, int64_t max_long, cudaStream_t s)
{
    const bool grad = a.dcdx || a.dcdy;
    const bool state = a.final_T != nullptr;
    if (grad && state) return launch_long_one<TILE, BPC, true, true>(a, max_long, s);
    if (grad) return launch_long_one<TILE, BPC, true, false>(a, max_long, s);
    if (state) return launch_long_one<TILE, BPC, false, true>(a, max_long, s);
    return launch_long_one<TILE, BPC, false, false>(a, max_long, s);
}

static_assert(long_smem_bytes() <= (size_t)kMaxSmem, "k_composite_long must fit shared memory");

template <int TILE>
int persistent_grid()
{
    constexpr size_t smem = smem_bytes<TILE, kServeBatch>();
    static bool done[64];
    opt_in_smem(k_composite_persistent<TILE>, smem, done);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite_persistent<TILE>, TILE * TILE, smem);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
}

}  // namespace

bool composite_supported(int tile, int batch)
{
    if (!(tile == 8 || tile == 16 || tile == 32) || !(batch == 32 || batch == 64 || batch == 128 || batch == 256))
        return false;
    // each warp holds kStages batches of 48-byte records
    const size_t bytes = (size_t)(tile * tile / 32) * ((size_t)kStages * batch * sizeof(GaussRec) + 8 * kStages);
    return bytes <= (size_t)kMaxSmem;
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

cudaError_t launch_composite_long(const CompositeArgs &a, int tile, int64_t max_long, cudaStream_t s)
{
    if (a.tiles_x == 0 || a.tiles_y == 0 || max_long <= 0) return cudaSuccess;
    if (a.nrm_sorted || a.pair_counts) return cudaErrorInvalidValue;  // those frames have no long tiles
    switch (tile) {
    case 8: return a.long_bpc == 2 ? launch_long_tb<8, 2>(a, max_long, s) : launch_long_tb<8, 1>(a, max_long, s);
    case 16: return launch_long_tb<16, 1>(a, max_long, s);
    default: return launch_long_tb<32, 1>(a, max_long, s);
    }
}

int composite_persistent_grid(int tile, int batch)
{
    (void)batch;
    if (tile == 8) return persistent_grid<8>();
    if (tile == 32) return persistent_grid<32>();
    return persistent_grid<16>();
}

cudaError_t launch_composite_persistent(const ServeItem *reqs, int n_reqs, uint32_t total_items, int tile, int batch,
                                        uint32_t *work_counter, int grid, cudaStream_t s)
{
    (void)batch;
    if (n_reqs <= 0 || total_items == 0) return cudaSuccess;
    if (n_reqs > kMaxServeReqs) return cudaErrorInvalidValue;
    if (tile == 8)
        k_composite_persistent<8><<<grid, 64, smem_bytes<8, kServeBatch>(), s>>>(reqs, n_reqs, total_items, work_counter);
    else if (tile == 32)
        k_composite_persistent<32><<<grid, 1024, smem_bytes<32, kServeBatch>(), s>>>(reqs, n_reqs, total_items,
                                                                                     work_counter);
    else
        k_composite_persistent<16><<<grid, 256, smem_bytes<16, kServeBatch>(), s>>>(reqs, n_reqs, total_items,
                                                                                   work_counter);
    return cudaGetLastError();
}

}  // namespace gsr
