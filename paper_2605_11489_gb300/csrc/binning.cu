// Tile binning and the depth order (paper Sec. 3: the projected Gaussians are
// depth-sorted; binning by tile lets compositing walk only the Gaussians whose
// support reaches each tile). The order wanted is (tile, depth, index), the
// order of a stable sort of (tile << 32 | fp32 depth bits) keys. It is built
// depth first, which moves far fewer bytes than sorting the 12-byte
// (key, value) pairs of every instance on all 45 bits:
//   K2  scan of the projection's per-block tile and visible counts: K, and the
//       compacted position of each block's visible Gaussians;
//   K3a the visible Gaussians' 32-bit depth keys and indices, compacted in
//       index order, with the depth sort's digit histograms;
//   K4a stable radix sort of those V pairs by depth (sort.cu, 4 passes);
//   K3b per 1,024 depth-sorted Gaussians the sum of their tile counts, a scan
//       of those sums, then every Gaussian's tile keys (32-bit tile id) and
//       index, emitted in depth order, with the tile sort's digit histograms;
//   K4b stable radix sort of the K instances by tile id (1 or 2 passes);
//   K5  per-tile ranges, with the records gathered into sorted order.
// Equal (tile, depth) keep index order because K3a emits in index order and
// both sorts are stable.
#include <algorithm>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kScanThreads = 1024;

// Exclusive scan over 1,024 threads of per-block counts `sums[0, nb)` into
// `offs`; returns the total in every thread.
__device__ unsigned long long block_scan_counts(const uint32_t *__restrict__ sums, int nb, uint32_t *__restrict__ offs,
                                                unsigned long long *s_warp)
{
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per;
    unsigned long long local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) local += sums[b0 + k];
    unsigned long long v = local;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();  // s_warp may still be read by an earlier call
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    unsigned long long run = v - local + (warp > 0 ? s_warp[warp - 1] : 0ull);
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) {
            offs[b0 + k] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
            run += sums[b0 + k];
        }
    return s_warp[31];
}

// K2: exclusive scans of the per-block tile counts (-> K, the capacity-clamped
// K used downstream, with an overflow bit if clamped) and of the per-block
// visible counts (-> where each block's visible Gaussians go when compacted).
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const uint32_t *__restrict__ sums,
                                                              const uint32_t *__restrict__ vis_sums, int nb,
                                                              uint32_t *__restrict__ offs,
                                                              uint32_t *__restrict__ vis_offs, uint32_t *counters,
                                                              unsigned long long capacity)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const unsigned long long total = block_scan_counts(sums, nb, offs, s_warp);
    if (vis_sums) block_scan_counts(vis_sums, nb, vis_offs, s_warp);
    if (threadIdx.x == kScanThreads - 1) {
        counters[kCntTotal] = (uint32_t)(total & 0xffffffffull);
        counters[kCntTotalHi] = (uint32_t)(total >> 32);
        const unsigned long long eff = total < capacity ? total : capacity;
        counters[kCntEff] = (uint32_t)eff;
        if (total > capacity) atomicOr(&counters[kCntErr], kErrCapacity);
        atomicMax(&counters[kCntMaxTotal], (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull));
        atomicAdd(reinterpret_cast<unsigned long long *>(counters + kCntSumK), total);
        atomicAdd(&counters[kCntFrames], 1u);
    }
}

// Block-wide exclusive prefix of one value per thread (256 threads) and the
// block total.
__device__ __forceinline__ uint32_t block_excl(uint32_t mine, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    uint32_t before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kProjThreads / 32; ++w) {
        const uint32_t x = s_warp[w];
        if (w < warp) before += x;
        total += x;
    }
    return before + v - mine;
}

// Adds a block's digit histograms (shared, `n` bins) into the global ones.
// floor(a / b) for a < 2^16 and 1 <= b < 2^16 (a key's position in its Gaussian's tile
// rectangle and the rectangle's width; at most 65,536 tiles): a single-precision estimate,
// with exact operands and a relative error under 2^-22, is within 1/64 of a / b, so at most
// one off; the remainder corrects it.
__device__ __forceinline__ uint32_t div_small(uint32_t a, uint32_t b)
{
    uint32_t q = (uint32_t)__fmul_rz((float)a, __frcp_rn((float)b));
    const int r = (int)a - (int)(q * b);
    if (r < 0) --q;
    else if (r >= (int)b) ++q;
    return q;
}

__device__ __forceinline__ void flush_hist(const uint32_t *s_hist, uint32_t *hist, int n)
{
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kProjThreads)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// K3a: one thread per quad of Gaussians (the projection's partition). Writes
// the visible ones' depth keys (fp32 bits) and indices at their compacted
// positions, in index order, and counts the 4 depth digits.
__global__ void __launch_bounds__(kProjThreads) k_compact(const uint32_t *__restrict__ ntiles,
                                                          const uint4 *__restrict__ bin,
                                                          const uint32_t *__restrict__ vis_offs, int64_t n,
                                                          uint32_t *__restrict__ dkeys, uint32_t *__restrict__ dvals,
                                                          uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_warp[kProjThreads / 32];
    __shared__ uint32_t s_hist[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += kProjThreads) s_hist[i] = 0;
    const int64_t i0 = ((int64_t)blockIdx.x * kProjThreads + threadIdx.x) * 4;
    uint4 nt = make_uint4(0, 0, 0, 0);
    if (i0 < n) nt = *reinterpret_cast<const uint4 *>(ntiles + i0);
    const uint32_t vis[4] = {nt.x != 0u, nt.y != 0u, nt.z != 0u, nt.w != 0u};
    // the visible Gaussians' depth keys are loaded before the block scan's barrier
    uint32_t zk[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) zk[g] = vis[g] ? bin[i0 + g].x : 0u;
    uint32_t total;
    uint32_t off = vis_offs[blockIdx.x] + block_excl(vis[0] + vis[1] + vis[2] + vis[3], s_warp, total);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (!vis[g]) continue;
        const uint32_t z = zk[g];
        dkeys[off] = z;
        dvals[off] = (uint32_t)(i0 + g);
        ++off;
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p * 256 + ((z >> (8 * p)) & 0xFFu)], 1u);
    }
    flush_hist(s_hist, hist, 4 * 256);
}

// K3b's lookback words: word 0 the partition ticket, then per partition of 1,024 sorted
// Gaussians its tile count (flag kDupAgg) or the inclusive prefix of the counts (kDupPre).
constexpr unsigned long long kDupAgg = 1ull << 62;
constexpr unsigned long long kDupPre = 2ull << 62;
constexpr unsigned long long kDupFlags = 3ull << 62;
constexpr unsigned long long kDupVal = kDupAgg - 1ull;
constexpr uint32_t kDupMaxSpins = 1u << 22;

__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void st_vol64(unsigned long long *p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

// Decoupled lookback of partition `part` (called by one whole warp): publishes the
// partition's count, reads up to 32 predecessors' words per round trip and sums them, newest
// first, up to the nearest inclusive prefix, then publishes its own inclusive prefix. Returns
// the exclusive prefix on every lane. A partition only waits for partitions that drew earlier
// tickets, which are running or done; each wait is still bounded: after max_spins polls it
// sets kErrSortTimeout and takes the sum so far (the keys then land at wrong offsets, in
// bounds). max_spins = 0 gives up before the first look (a diagnostic setting).
__device__ unsigned long long dup_lookback(unsigned long long *st, uint32_t part, uint32_t count,
                                           uint32_t max_spins, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    if (part == 0) {
        if (lane == 0) st_vol64(st, kDupPre | count);
        return 0ull;
    }
    if (lane == 0) st_vol64(st + part, kDupAgg | count);
    unsigned long long excl = 0ull;
    int p = (int)part - 1;  // the newest predecessor not yet summed
    uint32_t spins = 0;
    bool gave_up = max_spins == 0u;
    while (!gave_up) {
        const int q = p - lane;
        const unsigned long long w = q >= 0 ? ld_vol64(st + q) : kDupPre;  // before partition 0: 0
        const uint32_t ready = __ballot_sync(0xffffffffu, (w & kDupFlags) != 0ull);
        const uint32_t pre = __ballot_sync(0xffffffffu, (w & kDupFlags) == kDupPre);
        const int lim = pre ? __ffs(pre) - 1 : 31;  // lanes 0..lim are summed
        const uint32_t need = lim == 31 ? 0xffffffffu : (2u << lim) - 1u;
        if ((ready & need) != need) {
            if (++spins > max_spins) {
                gave_up = true;
                break;
            }
            __nanosleep(32);
            continue;
        }
        unsigned long long v = lane <= lim ? (w & kDupVal) : 0ull;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pre) break;
        p -= 32;
    }
    if (gave_up && lane == 0) atomicOr(err, kErrSortTimeout);
    if (lane == 0) st_vol64(st + part, kDupPre | ((excl + count) & kDupVal));
    return excl;
}

// K3b: every depth-sorted Gaussian's keys, key = tile id (32-bit) and value = Gaussian
// index, for every tile of its support rectangle (rows, then columns), in depth order; counts
// the tile digits. Keys past `capacity` are not written (the overflow bit is set). One pass:
// each block takes a partition of 1,024 sorted Gaussians by ticket, sums their tile counts and
// finds the partition's offset by decoupled lookback (`look`). Each warp owns 128 consecutive
// sorted Gaussians and deals their keys out to consecutive lanes, so that the stores are
// coalesced: lane l emits the warp's keys l, l + 32, ..., finding each key's Gaussian by a
// search over the warp's prefix of tile counts.
// An index >= n (only possible when the depth sort gave up and left its output unsorted,
// holes included) counts as a Gaussian with no tiles.
__global__ void __launch_bounds__(kProjThreads) k_duplicate(const uint32_t *__restrict__ dvals,
                                                            const uint32_t *__restrict__ vcount,
                                                            const uint32_t *__restrict__ ntiles,
                                                            const uint4 *__restrict__ bin,
                                                            unsigned long long *__restrict__ look, int tile_shift,
                                                            int tiles_x, uint32_t *__restrict__ keys,
                                                            uint32_t *__restrict__ vals, unsigned long long capacity,
                                                            uint32_t *err, uint32_t *__restrict__ hist, int passes,
                                                            uint32_t n, uint32_t max_spins)
{
    constexpr int kWarps = kProjThreads / 32, kPerWarp = 128;
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_hist[2 * 256];
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_pre[kWarps][kPerWarp + 1];  // exclusive prefix of tile counts, then the warp's total
    __shared__ uint32_t s_idx[kWarps][kPerWarp];      // Gaussian index
    __shared__ uint32_t s_org[kWarps][kPerWarp];      // first tile of its rectangle: tx | ty << 16
    __shared__ uint32_t s_wid[kWarps][kPerWarp];      // width of its rectangle in tiles
    for (int i = threadIdx.x; i < 2 * 256; i += kProjThreads) s_hist[i] = 0;
    if (threadIdx.x == 0) s_part = (uint32_t)atomicAdd(look, 1ull);
    __syncthreads();
    const uint32_t part = s_part;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t V = *vcount;
    // a partition past the visible Gaussians has no keys, nor has any later ticket's: none
    // of them is waited for
    if ((unsigned long long)part * kProjPerBlock >= V) return;
    const uint32_t i0 = (part * kProjThreads + threadIdx.x) * 4;
    uint32_t cnt[4], mine = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint32_t idx = i0 + g < V ? dvals[i0 + g] : 0u;
        if (!GSR_IN_BOUNDS(idx, n, err)) idx = 0u;  // (an unsorted depth order): no tiles
        cnt[g] = i0 + g < V && dvals[i0 + g] < n ? ntiles[idx] : 0u;
        uint32_t org = 0, wid = 1;
        if (cnt[g]) {
            const uint4 b = bin[idx];
            const uint32_t x0 = (b.y & 0xFFFFu) >> tile_shift, y0 = (b.y >> 16) >> tile_shift;
            const uint32_t x1 = (b.z & 0xFFFFu) >> tile_shift;
            org = x0 | (y0 << 16);
            wid = x1 - x0 + 1;
        }
        s_idx[warp][lane * 4 + g] = idx;
        s_org[warp][lane * 4 + g] = org;
        s_wid[warp][lane * 4 + g] = wid;
        mine += cnt[g];
    }
    uint32_t total;
    const uint32_t excl = block_excl(mine, s_warp, total);  // (block-wide; includes a barrier)
    if (warp == 0) {
        const unsigned long long b = dup_lookback(look + 1, part, total, max_spins, err);
        if (lane == 0) s_base = b;
    }
    // the warp's offsets: prefix within the warp, the warp's first key's global offset
    const uint32_t warp_first = __shfl_sync(0xffffffffu, excl, 0);
    uint32_t run = excl - warp_first;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        s_pre[warp][lane * 4 + g] = run;
        run += cnt[g];
    }
    if (lane == 31) s_pre[warp][kPerWarp] = run;
    __syncwarp();
    __syncthreads();  // s_base
    const uint32_t T = s_pre[warp][kPerWarp];
    const unsigned long long base = s_base + warp_first;
    bool overflow = false;
    for (uint32_t e = (uint32_t)lane; e < T; e += 32) {
        // the last j with s_pre[j] <= e (it has a nonzero count, as s_pre[kPerWarp] = T > e):
        // seven fixed halving steps, s_pre[0] = 0 <= e throughout
        int j = 0;
#pragma unroll
        for (int step = kPerWarp / 2; step >= 1; step >>= 1)
            if (s_pre[warp][j + step] <= e) j += step;
        const uint32_t li = e - s_pre[warp][j], w = s_wid[warp][j], org = s_org[warp][j];
        const uint32_t q = div_small(li, w);
        const uint32_t tile = ((org >> 16) + q) * (uint32_t)tiles_x + (org & 0xFFFFu) + (li - q * w);
        const unsigned long long off = base + e;
        if (off < capacity) {
            keys[off] = tile;
            vals[off] = s_idx[warp][j];
            for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p * 256 + ((tile >> (8 * p)) & 0xFFu)], 1u);
        } else {
            overflow = true;
        }
    }
    if (overflow) atomicOr(err, kErrCapacity);
    flush_hist(s_hist, hist, passes * 256);
}

// K5: per-tile [start, end) of the sorted tile keys and, in the same pass, the
// records gathered into sorted (instance) order, so compositing stages each
// batch of a tile's list with one contiguous bulk copy. With `keys64` it also
// writes each instance's (tile << 32) | depth-bits key (the state view's).
// The sorted records are gathered one 16-byte piece per thread: piece e of the
// output is piece e % 3 of record vals[e / 3], so three consecutive lanes read
// one record's 48 contiguous bytes and a warp's stores are 512 contiguous bytes
// (with a thread per record, every lane's load and store touched its own line
// and the L1 request path bound the kernel). Each thread takes four pieces, a
// block apart, so their loads are in flight together. The pieces with e % 3 == 0
// also write the tile ranges, (keys64 != NULL) the 64-bit keys and (nrm_sorted, plane_sorted !=
// NULL) the instance's normal and intersection-depth slope. With rec_sorted NULL (compositing
// then gathers each batch's records by index) a thread takes whole instances instead.
constexpr int kRangeThreads = 256, kRangePer = 4;

__global__ void __launch_bounds__(kRangeThreads)
    k_ranges(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
             const uint32_t *__restrict__ counters, uint32_t *err, const GaussRec *__restrict__ rec,
             GaussRec *__restrict__ rec_sorted, uint2 *ranges, const uint4 *__restrict__ bin,
             uint64_t *__restrict__ keys64, const float4 *__restrict__ nrm, float4 *__restrict__ nrm_sorted,
             const float2 *__restrict__ plane, float2 *__restrict__ plane_sorted,
             uint32_t n, uint32_t n_tiles)
{
    // Indices and tile ids are checked against n and n_tiles: after a sort that gave up
    // (kErrSortTimeout) the keys are not sorted and may hold stale words, and the frame is
    // reported as failed, but nothing is read or written out of bounds.
    const uint32_t K = counters[kCntEff];
    // work units: three 16-byte pieces per instance when the records are gathered, else the
    // instances themselves
    const uint32_t per = rec_sorted ? 3u : 1u;
    const uint32_t P = per * K;  // (K < 2^30)
    const uint32_t e0 = blockIdx.x * (kRangeThreads * kRangePer) + threadIdx.x;
    const float4 *src = reinterpret_cast<const float4 *>(rec);
    float4 *dst = reinterpret_cast<float4 *>(rec_sorted);
    float4 v[kRangePer];
    uint32_t g[kRangePer];
    // the Gaussian index is read only for what needs it (the record copy, the 64-bit keys,
    // the normals): a plain forward's ranges read the keys alone
    const bool need_g = rec_sorted || keys64 || nrm_sorted || plane_sorted;
#pragma unroll
    for (int k = 0; k < kRangePer; ++k) {
        const uint32_t e = e0 + (uint32_t)k * kRangeThreads;
        g[k] = e < P && need_g ? vals[e / per] : 0u;
        if (!GSR_IN_BOUNDS(g[k], n, err)) g[k] = 0u;
    }
    if (rec_sorted) {
#pragma unroll
        for (int k = 0; k < kRangePer; ++k) {
            const uint32_t e = e0 + (uint32_t)k * kRangeThreads;
            if (e < P) v[k] = __ldg(src + 3ull * g[k] + e % 3u);
        }
#pragma unroll
        for (int k = 0; k < kRangePer; ++k) {
            const uint32_t e = e0 + (uint32_t)k * kRangeThreads;
            if (e < P) dst[e] = v[k];
        }
    }
#pragma unroll
    for (int k = 0; k < kRangePer; ++k) {
        const uint32_t e = e0 + (uint32_t)k * kRangeThreads;
        if (e >= P || e % per != 0u) continue;
        const uint32_t i = e / per;
        const uint32_t t = keys[i];
        if (GSR_IN_BOUNDS(t, n_tiles, err)) {
            if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
            if (i == K - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
        }
        if (keys64) keys64[i] = ((uint64_t)t << 32) | (uint64_t)bin[g[k]].x;
        if (nrm_sorted) nrm_sorted[i] = __ldg(nrm + g[k]);
        if (plane_sorted) plane_sorted[i] = __ldg(plane + g[k]);
    }
}

// Tiles ordered by decreasing list length, bucketed by floor(log2(length)), so
// compositing dispatches the heaviest tiles first and the light ones fill in.
__global__ void __launch_bounds__(1024) k_tile_order(const uint2 *__restrict__ ranges, int n_tiles,
                                                     uint32_t *__restrict__ order)
{
    __shared__ uint32_t s_cnt[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [&](int t) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        return len == 0 ? 32 : __clz(len);  // longer lists -> smaller bucket index
    };
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&s_cnt[bucket(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < 33; ++b) {
            const uint32_t c = s_cnt[b];
            s_cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) order[atomicAdd(&s_cnt[bucket(t)], 1u)] = (uint32_t)t;
}

// Compositing plan (one CTA). Every tile gets a bucket: the long tiles (list longer
// than `head`) floor(log2(length)) in [0, 32), the others 32 + that (empty lists
// last), so tile_order lists the long tiles first, each part longest first:
// k_composite_long's CTAs take the long ones from the front, k_composite's the
// others. plan = (n_long, 0 = the long tiles' work counter, n_short). Range loads
// are issued four tiles per thread at a time; the bucket counts and cursors are
// shared-memory atomics, one per bucket and warp (__match_any_sync). The order
// within a bucket depends on the warps' timing, which no result depends on.
constexpr int kPlanBuckets = 65;
constexpr int kPlanUnroll = 4;

__device__ __forceinline__ uint32_t plan_bucket(uint2 r, uint32_t head)
{
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    const uint32_t lg = len == 0 ? 32u : (uint32_t)__clz(len);  // longer -> smaller
    return len > head ? lg : 32u + lg;
}

__global__ void __launch_bounds__(1024) k_plan(const uint2 *__restrict__ ranges, int n_tiles, uint32_t head,
                                               uint32_t *__restrict__ order, uint32_t *__restrict__ plan,
                                               const uint32_t *err)
{
    __shared__ uint32_t s_cnt[kPlanBuckets + 1];  // counts, then cursors; the last one is "no tile"
    __shared__ bool s_skip;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_skip = (*reinterpret_cast<const volatile uint32_t *>(err) & kErrSortTimeout) != 0u;
    if (threadIdx.x <= kPlanBuckets) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    if (s_skip) {
        if (threadIdx.x < 3) plan[threadIdx.x] = 0u;
        return;
    }
    constexpr int kStride = 1024 * kPlanUnroll;
    for (int base = threadIdx.x; base - (int)threadIdx.x < n_tiles; base += kStride) {
        uint32_t bk[kPlanUnroll];
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {
            const int t = base + u * 1024;
            bk[u] = t < n_tiles ? plan_bucket(ranges[t], head) : (uint32_t)kPlanBuckets;
        }
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {
            const uint32_t peers = __match_any_sync(0xffffffffu, bk[u]);
            if (bk[u] < (uint32_t)kPlanBuckets && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[bk[u]], __popc(peers));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0, n_long = 0;
        for (int q = 0; q < kPlanBuckets; ++q) {
            const uint32_t c = s_cnt[q];
            s_cnt[q] = run;
            run += c;
            if (q == 31) n_long = run;
        }
        plan[0] = n_long;
        plan[1] = 0u;
        plan[2] = (uint32_t)n_tiles - n_long;
    }
    __syncthreads();
    for (int base = threadIdx.x; base - (int)threadIdx.x < n_tiles; base += kStride) {
        uint32_t bk[kPlanUnroll];
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {
            const int t = base + u * 1024;
            bk[u] = t < n_tiles ? plan_bucket(ranges[t], head) : (uint32_t)kPlanBuckets;
        }
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {
            const uint32_t peers = __match_any_sync(0xffffffffu, bk[u]);
            const int leader = __ffs(peers) - 1;
            uint32_t first = 0u;
            if (bk[u] < (uint32_t)kPlanBuckets && lane == leader) first = atomicAdd(&s_cnt[bk[u]], __popc(peers));
            first = __shfl_sync(0xffffffffu, first, leader);
            if (bk[u] < (uint32_t)kPlanBuckets) order[first + __popc(peers & lt)] = (uint32_t)(base + u * 1024);
        }
    }
}

}  // namespace

// a split tile has > head >= chunk records and at most 2 + (len - head) / chunk slots
cudaError_t launch_plan(const uint2 *ranges, int n_tiles, int64_t head, uint32_t *order, uint32_t *plan,
                        const uint32_t *err, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaMemsetAsync(plan, 0, sizeof(uint32_t) * 3, s);
    k_plan<<<1, 1024, 0, s>>>(ranges, n_tiles, (uint32_t)std::min<int64_t>(head, 0xFFFFFFFFll), order, plan, err);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const uint2 *ranges, int n_tiles, uint32_t *order, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_tile_order<<<1, 1024, 0, s>>>(ranges, n_tiles, order);
    return cudaGetLastError();
}

cudaError_t launch_scan_blocks(const uint32_t *block_sums, const uint32_t *vis_sums, int nblocks,
                               uint32_t *block_offsets, uint32_t *vis_offsets, uint32_t *counters, int64_t capacity,
                               cudaStream_t s)
{
    k_scan_blocks<<<1, kScanThreads, 0, s>>>(block_sums, vis_sums, nblocks, block_offsets, vis_offsets, counters,
                                              (unsigned long long)capacity);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t *ntiles, const uint4 *bin, const uint32_t *vis_offsets, int64_t n,
                           uint32_t *dkeys, uint32_t *dvals, uint32_t *hist, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 8 * 256, s);
    if (e != cudaSuccess) return e;
    const int nb = project_blocks(n);
    if (nb == 0) return cudaSuccess;
    k_compact<<<nb, kProjThreads, 0, s>>>(ntiles, bin, vis_offsets, n, dkeys, dvals, hist);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const uint32_t *dvals, const uint32_t *vcount, int64_t max_v, const uint32_t *ntiles,
                             const uint4 *bin, unsigned long long *look, int tile_shift, int tiles_x, uint32_t *keys,
                             uint32_t *vals, int64_t capacity, uint32_t *counters, uint32_t *hist, int passes,
                             cudaStream_t s, uint32_t *err, bool give_up)
{
    if (!err) err = counters + kCntErr;
    if (passes < 0 || passes > 2) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 8 * 256, s);
    if (e != cudaSuccess) return e;
    const int nb = project_blocks(max_v);
    if (nb == 0) return cudaSuccess;
    e = cudaMemsetAsync(look, 0, duplicate_look_bytes(max_v), s);
    if (e != cudaSuccess) return e;
    k_duplicate<<<nb, kProjThreads, 0, s>>>(dvals, vcount, ntiles, bin, look, tile_shift, tiles_x, keys, vals,
                                            (unsigned long long)capacity, err, hist, passes, (uint32_t)max_v,
                                            give_up ? 0u : kDupMaxSpins);
    return cudaGetLastError();
}

size_t duplicate_look_bytes(int64_t max_v) { return sizeof(unsigned long long) * ((size_t)project_blocks(max_v) + 1); }

cudaError_t launch_ranges(const uint32_t *keys, const uint32_t *vals, uint32_t *counters, int64_t max_k,
                          int64_t n, const GaussRec *rec, GaussRec *rec_sorted, uint2 *ranges, int n_tiles,
                          const uint4 *bin, uint64_t *keys64, cudaStream_t s, const float4 *nrm, float4 *nrm_sorted,
                          const float2 *plane, float2 *plane_sorted, uint32_t *err)
{
    if (!err) err = counters + kCntErr;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
    if (e != cudaSuccess) return e;
    if (max_k <= 0) return cudaSuccess;
    const int64_t per_block = (int64_t)kRangeThreads * kRangePer;
    const int64_t nb = ((rec_sorted ? 3 : 1) * max_k + per_block - 1) / per_block;
    k_ranges<<<(unsigned)nb, kRangeThreads, 0, s>>>(keys, vals, counters, err, rec, rec_sorted, ranges, bin, keys64,
                                                    nrm, nrm_sorted, plane, plane_sorted, (uint32_t)std::max<int64_t>(n, 1),
                                                    (uint32_t)n_tiles);
    return cudaGetLastError();
}

}  // namespace gsr
