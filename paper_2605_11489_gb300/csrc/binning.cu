// Tile binning: instance offsets (K2), (tile, depth) key duplication (K3) and
// per-tile ranges of the sorted keys (K5). The depth sort itself (paper Sec. 3:
// "the resulting 2D Gaussians are depth-sorted") is a radix sort over these
// keys (sort.cu); binning by tile lets compositing walk only the Gaussians
// whose support reaches each tile.
//
// The scan is split to avoid a separate pass over the per-Gaussian counts: the
// projection kernel already reduced tiles-touched per block of 1024 Gaussians;
// K2 scans those block sums in one CTA; K3 re-reads the counts it needs anyway
// and finishes the scan inside each block.
#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kScanThreads = 1024;

// Exclusive scan of per-block tile counts; writes offsets, K = total, and the
// capacity-clamped K used downstream (with an overflow bit if clamped).
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const uint32_t *__restrict__ sums, int nb,
                                                              uint32_t *__restrict__ offs, uint32_t *counters,
                                                              unsigned long long capacity)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per;
    unsigned long long local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) local += sums[b0 + k];
    // inclusive warp scan
    unsigned long long v = local;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
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
    if (threadIdx.x == kScanThreads - 1) {
        const unsigned long long total = run;
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

// One thread per quad of Gaussians (same partition as the projection); emits
// key = (tile id << 32) | fp32 bits of depth, val = Gaussian index, for every
// tile of each Gaussian's support rectangle, in index order. With `hist`, it
// also builds the radix sort's per-pass digit histograms of exactly the keys
// it writes (8-bit digits, `passes` of them): the four depth digits are shared
// by all of a Gaussian's keys and counted once per Gaussian, the tile digits
// once per key; block counts are merged into `hist` with one atomic per bin.
__global__ void __launch_bounds__(kProjThreads) k_duplicate(const uint32_t *__restrict__ ntiles,
                                                            const uint4 *__restrict__ bin,
                                                            const uint32_t *__restrict__ block_offs, int64_t n,
                                                            int tile_shift, int tiles_x, uint64_t *__restrict__ keys,
                                                            uint32_t *__restrict__ vals, unsigned long long capacity,
                                                            uint32_t *counters, uint32_t *__restrict__ hist,
                                                            int passes)
{
    __shared__ uint32_t s_warp[kProjThreads / 32];
    __shared__ uint32_t s_hist[8 * 256];
    if (hist)
        for (int i = threadIdx.x; i < passes * 256; i += kProjThreads) s_hist[i] = 0;
    const int64_t i0 = ((int64_t)blockIdx.x * kProjThreads + threadIdx.x) * 4;
    uint4 nt = make_uint4(0, 0, 0, 0);
    if (i0 < n) nt = *reinterpret_cast<const uint4 *>(ntiles + i0);
    const uint32_t mine = nt.x + nt.y + nt.z + nt.w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    unsigned long long off = (unsigned long long)block_offs[blockIdx.x] + before + (v - mine);
    const uint32_t cnt[4] = {nt.x, nt.y, nt.z, nt.w};
    bool overflow = false;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (cnt[g] == 0) continue;
        const uint4 b = bin[i0 + g];
        const int x0 = (b.y & 0xFFFFu) >> tile_shift, y0 = (b.y >> 16) >> tile_shift;
        const int x1 = (b.z & 0xFFFFu) >> tile_shift, y1 = (b.z >> 16) >> tile_shift;
        const uint32_t idx = (uint32_t)(i0 + g);
        if (hist) {  // depth digits: every written key of this Gaussian shares them
            const uint32_t written =
                off >= capacity ? 0u : (uint32_t)min((unsigned long long)cnt[g], capacity - off);
            for (int p = 0; p < passes && p < 4; ++p)
                if (written) atomicAdd(&s_hist[p * 256 + ((b.x >> (8 * p)) & 0xFFu)], written);
        }
        for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) {
                const uint32_t tile = (uint32_t)(ty * tiles_x + tx);
                if (off < capacity) {
                    keys[off] = ((uint64_t)tile << 32) | (uint64_t)b.x;
                    vals[off] = idx;
                    if (hist)
                        for (int p = 4; p < passes; ++p) atomicAdd(&s_hist[p * 256 + ((tile >> (8 * (p - 4))) & 0xFFu)], 1u);
                } else {
                    overflow = true;
                }
                ++off;
            }
    }
    if (overflow) atomicOr(&counters[kCntErr], kErrCapacity);
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < passes * 256; i += kProjThreads)
            if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
    }
}

// Per-tile [start, end) of the sorted keys and, in the same pass, the records
// gathered into sorted (instance) order, so compositing stages each batch of a
// tile's list with one contiguous bulk copy.
__global__ void k_ranges(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                         const uint32_t *__restrict__ counters, const GaussRec *__restrict__ rec,
                         GaussRec *__restrict__ rec_sorted, uint2 *ranges)
{
    const uint32_t K = counters[kCntEff];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = i;
    if (i == K - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = i + 1;
    if (rec_sorted) {
        const GaussRec *src = rec + vals[i];
        GaussRec r;
        r.r0 = __ldg(&src->r0);
        r.r1 = __ldg(&src->r1);
        r.r2 = __ldg(&src->r2);
        rec_sorted[i] = r;
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

// Compositing work plan. A tile whose list is longer than `head` is split into
// depth-contiguous chunks: the first of `head` records, the others of `chunk`
// (chunk_of / chunk_start / chunk_count); each chunk is a work item whose
// per-pixel partial state goes to its own slot (a split tile's slots are
// consecutive), and the split tile is finished front to back afterwards.
// Items come in two waves, composited by two launches:
//   wave A, items [0, n_tiles): the first chunk of every split tile (in split
//     order), then the whole tiles, longest lists first;
//   wave B, items [n_tiles, n_items): the later chunks, in slot order. They
//     run after wave A, so they can leave out the pixels that already stopped
//     in their tile's first chunk.
//   items[i]       = (tile, start, end, slot | kWholeTile)
//   split_tiles[s] = tile id of the s-th split tile, split_slot0[s] = its first slot
//   slot_split[k]  = the split tile (index s) that slot k belongs to
//   counts         = (n_items, n_split, n_slots, n_tiles = size of wave A)
// One CTA; each warp takes 32 consecutive tiles at a time. A split tile gets
// its split index and its slots from one packed counter, (splits << 32) +
// slots, so that both come in the same order and the later chunks before a
// tile's own number slot - split index. Whole tiles are bucketed by
// floor(log2(length)), with one atomic per bucket and warp.
__global__ void __launch_bounds__(1024) k_plan(const uint2 *__restrict__ ranges, int n_tiles, uint32_t chunk,
                                               uint32_t head, uint4 *__restrict__ items,
                                               uint32_t *__restrict__ split_tiles,
                                               uint32_t *__restrict__ split_slot0, uint32_t *__restrict__ slot_split,
                                               uint32_t *__restrict__ counts)
{
    __shared__ unsigned long long s_alloc;  // (split tiles << 32) | slots handed out so far
    __shared__ uint32_t s_bucket[33];       // whole tiles per bucket, then next free item per bucket
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_alloc = 0ull;
    if (threadIdx.x < 33) s_bucket[threadIdx.x] = 0u;
    __syncthreads();
    auto bucket_of = [](uint32_t len) { return len == 0 ? 32u : (uint32_t)__clz(len); };  // longer -> smaller

    // pass 1: split tiles are placed; whole tiles are counted per bucket
    for (int base = warp * 32; base < n_tiles; base += 1024) {
        const int t = base + lane;
        uint2 r = make_uint2(0u, 0u);
        if (t < n_tiles) r = ranges[t];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        const uint32_t c = t < n_tiles ? chunk_count(len, head, chunk) : 0u;
        const bool split = c > 1, whole = c == 1;
        // split: exclusive prefix of slot counts over the warp's split lanes
        const uint32_t smask = __ballot_sync(0xffffffffu, split);
        uint32_t inc = split ? c : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        unsigned long long got = 0ull;
        if (lane == 0 && smask)
            got = atomicAdd(&s_alloc, ((unsigned long long)__popc(smask) << 32) | (unsigned long long)total);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (split) {
            const uint32_t sp = (uint32_t)(got >> 32) + (uint32_t)__popc(smask & lt);
            const uint32_t slot = (uint32_t)(got & 0xffffffffull) + inc - c;
            split_tiles[sp] = (uint32_t)t;
            split_slot0[sp] = slot;
            items[sp] = make_uint4((uint32_t)t, r.x, r.x + head, slot);  // wave A: first chunk
            const uint32_t later = (uint32_t)n_tiles + (slot - sp);      // wave B: later chunks before ours
            for (uint32_t k = 0; k < c; ++k) {
                slot_split[slot + k] = sp;
                if (k == 0) continue;
                const uint32_t s0 = r.x + chunk_start(k, head, chunk);
                items[later + k - 1] = make_uint4((uint32_t)t, s0, min(r.y, s0 + chunk), slot + k);
            }
        }
        const uint32_t b = whole ? bucket_of(len) : 64u;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (whole && lane == __ffs(peers) - 1) atomicAdd(&s_bucket[b], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t n_split = (uint32_t)(s_alloc >> 32), n_slots = (uint32_t)(s_alloc & 0xffffffffull);
        uint32_t run = n_split;  // whole tiles follow the first chunks
        for (int q = 0; q < 33; ++q) {
            const uint32_t cnt = s_bucket[q];
            s_bucket[q] = run;
            run += cnt;
        }
        counts[0] = (uint32_t)n_tiles + n_slots - n_split;
        counts[1] = n_split;
        counts[2] = n_slots;
        counts[3] = (uint32_t)n_tiles;
    }
    __syncthreads();
    // pass 2: whole tiles into their buckets
    for (int base = warp * 32; base < n_tiles; base += 1024) {
        const int t = base + lane;
        uint2 r = make_uint2(0u, 0u);
        if (t < n_tiles) r = ranges[t];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        const bool whole = t < n_tiles && chunk_count(len, head, chunk) == 1;
        const uint32_t b = whole ? bucket_of(len) : 64u;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t pos = 0;
        if (whole && lane == leader) pos = atomicAdd(&s_bucket[b], (uint32_t)__popc(peers));
        pos = __shfl_sync(0xffffffffu, pos, leader) + (uint32_t)__popc(peers & lt);
        if (whole) items[pos] = make_uint4((uint32_t)t, r.x, r.x + len, kWholeTile);
    }
}

}  // namespace

// a split tile has > head >= chunk records and at most 2 + (len - head) / chunk slots
int64_t plan_max_slots(int64_t max_k, int chunk) { return 3 * (max_k / chunk) + 2; }
int64_t plan_max_items(int n_tiles, int64_t max_k, int chunk) { return n_tiles + plan_max_slots(max_k, chunk); }

cudaError_t launch_plan(const uint2 *ranges, int n_tiles, int chunk, int head, uint4 *items, uint32_t *split_tiles,
                        uint32_t *split_slot0, uint32_t *slot_split, uint32_t *counts, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 4, s);
    k_plan<<<1, 1024, 0, s>>>(ranges, n_tiles, (uint32_t)chunk, (uint32_t)head, items, split_tiles, split_slot0,
                              slot_split, counts);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const uint2 *ranges, int n_tiles, uint32_t *order, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_tile_order<<<1, 1024, 0, s>>>(ranges, n_tiles, order);
    return cudaGetLastError();
}

cudaError_t launch_scan_blocks(const uint32_t *block_sums, int nblocks, uint32_t *block_offsets, uint32_t *counters,
                               int64_t capacity, cudaStream_t s)
{
    k_scan_blocks<<<1, kScanThreads, 0, s>>>(block_sums, nblocks, block_offsets, counters,
                                              (unsigned long long)capacity);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const uint32_t *ntiles, const uint4 *bin, const uint32_t *block_offsets, int64_t n,
                             int tile_shift, int tiles_x, uint64_t *keys, uint32_t *vals, int64_t capacity,
                             uint32_t *counters, uint32_t *hist, int passes, cudaStream_t s)
{
    if (hist) {
        if (passes < 1 || passes > 8) return cudaErrorInvalidValue;
        const cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 8 * 256, s);
        if (e != cudaSuccess) return e;
    }
    const int nb = project_blocks(n);
    if (nb == 0) return cudaSuccess;
    k_duplicate<<<nb, kProjThreads, 0, s>>>(ntiles, bin, block_offsets, n, tile_shift, tiles_x, keys, vals,
                                            (unsigned long long)capacity, counters, hist, passes);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint64_t *keys, const uint32_t *vals, const uint32_t *counters, int64_t max_k,
                          const GaussRec *rec, GaussRec *rec_sorted, uint2 *ranges, int n_tiles, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
    if (e != cudaSuccess) return e;
    if (max_k <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t nb = (max_k + threads - 1) / threads;
    k_ranges<<<(unsigned)nb, threads, 0, s>>>(keys, vals, counters, rec, rec_sorted, ranges);
    return cudaGetLastError();
}

}  // namespace gsr
