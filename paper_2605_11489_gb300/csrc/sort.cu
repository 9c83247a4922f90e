// K4: stable LSD radix sort of keys (32- or 64-bit) with 32-bit values,
// "onesweep" style (Adinets & Merrill, 2022): every digit's global histogram
// is known before the first pass (built by the kernel that wrote the keys, or
// by one pass over them), then each 8-bit digit is sorted in a single pass
// over the data, with partitions publishing their per-digit counts and
// resolving their global offsets by decoupled lookback.
//
// The render sorts twice: the visible Gaussians by their 32-bit depth key
// (fp32 depth is positive, so its bit pattern orders like the value), then,
// after the keys are duplicated per tile in that order, the instances by tile
// id alone. Both are stable, so the result is ordered by (tile, depth, index),
// the order of a stable sort of (tile << 32 | depth) keys. Only the low `bits`
// bits are sorted.
//
// Partition ids are taken from an atomic ticket, so a partition only ever waits
// for partitions that are already running. Every wait is still bounded: a
// partition that gives up sets kErrSortTimeout and publishes what it has.
#include <algorithm>
#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kThreads = 256;  // the histogram kernel
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;
// A sort pass takes partitions of 4,096 keys, as 256 threads of 16 keys or 512 threads of 8
// (the caller's choice, kept for the whole sort). In the 512-thread shape the first 256
// threads also own one digit each for the per-digit steps (offsets, lookback, bases). Both
// shapes hold 32 warps per SM for 32-bit keys; 512 threads halve each warp's serial
// ranking, load and scatter work, 256 threads keep twice the partitions in flight.
// Measured on the 1M and 6M scenes: 512 threads sort the visible Gaussians by depth 7-25 %
// faster; 256 threads sort the 8M tile keys of the 6M scene 6 % faster.
constexpr int kPart = 4096;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kMaxSpins = 1u << 22;
constexpr int kLook = 8;  // predecessors read per lookback round trip
template <typename KeyT, int kT>
constexpr size_t pass_smem()
{
    return (size_t)kPart * sizeof(KeyT) + (size_t)kPart * 4 + (size_t)(kT / 32) * kRadix * 4;
}

__device__ __forceinline__ uint32_t ld_vol(const uint32_t *p) { return *reinterpret_cast<const volatile uint32_t *>(p); }

// The lanes of the warp holding the same 8-bit digit as this lane: the AND, over the
// digit's 8 bits, of the ballot of lanes with that bit set (or its complement). A fixed
// 9 ballots, where __match_any_sync takes time growing with the number of distinct digits
// in the warp. Measured on the depth sort's passes: ranking over the random low bytes took
// 7.5 us with __match_any_sync and 3.9 us with ballots; over the few distinct top bytes,
// 1.9 us and 3.8 us. So every pass but the most significant one ranks with ballots.
// Lanes without a key match each other and no valid lane.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, bool valid)
{
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    uint32_t peers = valid ? vmask : ~vmask;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = ((d >> b) & 1u) != 0u;
        const uint32_t bal = __ballot_sync(0xffffffffu, valid && bit);
        if (valid) peers &= bit ? bal : ~bal;
    }
    return peers;
}
__device__ __forceinline__ void st_vol(uint32_t *p, uint32_t v) { *reinterpret_cast<volatile uint32_t *>(p) = v; }

template <typename KeyT>
__global__ void __launch_bounds__(kThreads) k_sort_hist(const KeyT *__restrict__ keys,
                                                        const uint32_t *__restrict__ count, int passes,
                                                        uint32_t *__restrict__ hist)
{
    __shared__ uint32_t sh[8 * kRadix];
    for (int i = threadIdx.x; i < 8 * kRadix; i += kThreads) sh[i] = 0;
    __syncthreads();
    const uint32_t K = *count;
    const int lane = threadIdx.x & 31;
    const uint32_t warp_global = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    for (uint32_t base = warp_global * 32; base < K; base += nwarps * 32) {
        const uint32_t idx = base + lane;
        const bool valid = idx < K;
        const uint64_t key = valid ? (uint64_t)keys[idx] : 0ull;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (uint32_t)(key >> (8 * p)) & 0xFFu : 0x100u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&sh[p * kRadix + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of two per-thread values over the kW warps of the block (s_tmp: 2 x kW).
template <int kW>
__device__ __forceinline__ void block_excl_scan2(uint32_t a, uint32_t b, uint32_t &ea, uint32_t &eb, uint32_t *s_tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ta;
            ib += tb;
        }
    }
    if (lane == 31) {
        s_tmp[warp] = ia;
        s_tmp[kW + warp] = ib;
    }
    __syncthreads();
    uint32_t pa = 0, pb = 0;
    for (int w = 0; w < warp; ++w) {
        pa += s_tmp[w];
        pb += s_tmp[kW + w];
    }
    ea = pa + ia - a;
    eb = pb + ib - b;
}

// Partitions resident per SM, by the launch bound: 32-bit keys four of 256 threads or two of
// 512; 64-bit keys (80 registers, the largest carveout) three of 256 or one of 512.
// max_spins: polls of a predecessor's word before the lookback gives up; 0 gives up before
// the first look (a diagnostic setting that exercises the give-up path deterministically).
// A partition that gave up publishes its own count as its prefix: the output is then not
// sorted, but every element is still written inside [0, K). The scatter also keeps inside
// [0, K) when the input itself is the unsorted output of a pass that gave up (whose digit
// counts no longer match the histogram).
template <typename KeyT, bool kBallot, int kT>
__global__ void __launch_bounds__(kT, kT == 512 ? (sizeof(KeyT) == 8 ? 1 : 2) : (sizeof(KeyT) == 8 ? 3 : 4))
    k_sort_pass(const KeyT *__restrict__ kin, const uint32_t *__restrict__ vin, KeyT *__restrict__ kout,
                uint32_t *__restrict__ vout, const uint32_t *__restrict__ count, int shift,
                const uint32_t *__restrict__ hist, uint32_t *status, uint32_t *part_ctr, uint32_t *err,
                uint32_t max_spins)
{
    constexpr int kW = kT / 32, kItems = kPart / kT;
    extern __shared__ __align__(16) unsigned char smem[];
    KeyT *s_keys = reinterpret_cast<KeyT *>(smem);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(smem + (size_t)kPart * sizeof(KeyT));
    uint32_t *s_whist = reinterpret_cast<uint32_t *>(smem + (size_t)kPart * (sizeof(KeyT) + 4));
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_start[kRadix];
    __shared__ uint32_t s_tmp[2 * kW];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t K = *count;
    const uint32_t nparts = (K + kPart - 1) / kPart;
    if (tid == 0) s_part = atomicAdd(part_ctr, 1u);
    for (int i = tid; i < kW * kRadix; i += kT) s_whist[i] = 0;
    __syncthreads();
    const uint32_t part = s_part;
    if (part >= nparts) return;
    const uint32_t base = part * kPart;
    const bool digit = kT == kRadix || tid < kRadix;  // this thread owns digit tid in the per-digit steps
    const uint32_t hist_d = digit ? hist[tid] : 0u;  // the digit's global count, loaded early

    KeyT k[kItems];
    uint32_t v[kItems], rk[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = base + warp * (kItems * 32) + j * 32 + lane;
        if (idx < K) {
            k[j] = kin[idx];
            v[j] = vin[idx];
        } else {
            k[j] = ~KeyT(0);
            v[j] = 0u;
        }
    }
    // warp-level stable ranking: items are ordered (warp, j, lane)
    uint32_t *wh = s_whist + warp * kRadix;
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = base + warp * (kItems * 32) + j * 32 + lane;
        const bool valid = idx < K;
        const uint32_t d = valid ? (uint32_t)(k[j] >> shift) & 0xFFu : 0x100u;
        const uint32_t peers = kBallot ? match_digit(d, valid) : __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t prev = 0;
        if (lane == leader && valid) {
            prev = wh[d];
            wh[d] = prev + (uint32_t)__popc(peers);
        }
        prev = __shfl_sync(0xffffffffu, prev, leader);
        rk[j] = prev + (uint32_t)__popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets across warps and the partition's count
    uint32_t cnt = 0;
    if (digit) {
#pragma unroll
        for (int w = 0; w < kW; ++w) {
            const uint32_t c = s_whist[w * kRadix + tid];
            s_whist[w * kRadix + tid] = cnt;
            cnt += c;
        }
    }
    uint32_t cexcl, hexcl;
    block_excl_scan2<kW>(cnt, hist_d, cexcl, hexcl, s_tmp);  // every thread: it synchronises the block
    // decoupled lookback for this digit, kLook predecessors per round trip:
    // their words are loaded together and summed newest first until an
    // inclusive prefix is met; a word not yet published is re-read on its own.
    if (digit) {
        uint32_t *st = status + (size_t)part * kRadix + tid;
        uint32_t excl = 0;
        if (part == 0) {
            st_vol(st, kFlagPre | cnt);
        } else {
            st_vol(st, kFlagAgg | cnt);
            int p = (int)part - 1;
            uint32_t spins = 0;
            bool done = false;
            if (max_spins == 0u) {  // diagnostic: give up before the first look
                atomicOr(err, kErrSortTimeout);
                done = true;
            }
            while (!done && p >= 0) {
                uint32_t w[kLook];
#pragma unroll
                for (int u = 0; u < kLook; ++u)
                    w[u] = p - u >= 0 ? ld_vol(status + (size_t)(p - u) * kRadix + tid) : 0u;
#pragma unroll
                for (int u = 0; u < kLook; ++u) {
                    if (done || p < 0) break;
                    uint32_t s = w[u];
                    while ((s & kFlagMask) == 0u) {
                        if (++spins > max_spins) {
                            atomicOr(err, kErrSortTimeout);
                            break;
                        }
                        __nanosleep(32);
                        s = ld_vol(status + (size_t)p * kRadix + tid);
                    }
                    if ((s & kFlagMask) == 0u) {  // gave up
                        done = true;
                        break;
                    }
                    excl += s & kValMask;
                    if ((s & kFlagMask) == kFlagPre) done = true;
                    --p;
                }
            }
            st_vol(st, kFlagPre | ((excl + cnt) & kValMask));
        }
        s_base[tid] = hexcl + excl;
        s_start[tid] = cexcl;
    }
    __syncthreads();
    // stable local scatter into shared memory, then coalesced global writes
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = base + warp * (kItems * 32) + j * 32 + lane;
        if (idx < K) {
            const uint32_t d = (uint32_t)(k[j] >> shift) & 0xFFu;
            const uint32_t pos = s_start[d] + s_whist[warp * kRadix + d] + rk[j];
            s_keys[pos] = k[j];
            s_vals[pos] = v[j];
        }
    }
    __syncthreads();
    const uint32_t nval = min((uint32_t)kPart, K - base);
    for (uint32_t i = tid; i < nval; i += kT) {
        const KeyT key = s_keys[i];
        const uint32_t d = (uint32_t)(key >> shift) & 0xFFu;
        const uint32_t g = s_base[d] + (i - s_start[d]);
        if (GSR_IN_BOUNDS(g, K, err)) {
            kout[g] = key;
            vout[g] = s_vals[i];
        }
    }
}

}  // namespace

int sort_passes(int bits) { return (bits + 7) / 8; }

static int64_t parts_for(int64_t k) { return (k + kPart - 1) / kPart; }

size_t sort_scratch_bytes(int64_t capacity)
{
    const int64_t parts = parts_for(capacity) + 1;
    return sizeof(uint32_t) * (8 * kRadix + 8 + (size_t)8 * parts * kRadix) + 256;
}

void sort_scratch_carve(void *base, int64_t capacity, SortScratch *s)
{
    uint32_t *p = reinterpret_cast<uint32_t *>(base);
    s->hist = p;
    s->part_ctr = p + 8 * kRadix;
    s->status = p + 8 * kRadix + 8;
    s->max_parts = parts_for(capacity) + 1;
}

namespace {

template <typename KeyT>
cudaError_t sort_impl(KeyT *keys[2], uint32_t *vals[2], const uint32_t *count, uint32_t *err_word, int64_t max_k,
                      int bits, const SortScratch &scr, int *result, cudaStream_t s, bool hist_ready, bool give_up,
                      bool wide)
{
    const int passes = sort_passes(bits);
    *result = passes & 1;
    if (max_k <= 0) return cudaSuccess;
    const int64_t parts = parts_for(max_k);
    if (parts > scr.max_parts || passes > (int)sizeof(KeyT)) return cudaErrorInvalidValue;
    // once per device, outside any stream capture (the first sort on a device is never
    // captured); serialised, because the server's scheduler thread sorts too
    static bool attr_set[64] = {};
    static std::mutex attr_mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(attr_mu);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        const void *fns[4] = {reinterpret_cast<const void *>(k_sort_pass<KeyT, false, 256>),
                              reinterpret_cast<const void *>(k_sort_pass<KeyT, true, 256>),
                              reinterpret_cast<const void *>(k_sort_pass<KeyT, false, 512>),
                              reinterpret_cast<const void *>(k_sort_pass<KeyT, true, 512>)};
        const size_t fn_smem[4] = {pass_smem<KeyT, 256>(), pass_smem<KeyT, 256>(), pass_smem<KeyT, 512>(),
                                   pass_smem<KeyT, 512>()};
        for (int f = 0; f < 4; ++f) {
            const void *fn = fns[f];
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fn_smem[f]);
            if (e != cudaSuccess) return e;
            // several partitions per SM need the largest shared-memory carveout
            e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
        }
        attr_set[dev] = true;
    }
    // histograms (unless ready) and partition tickets, then the lookback words
    e = hist_ready ? cudaMemsetAsync(scr.part_ctr, 0, sizeof(uint32_t) * 8, s)
                   : cudaMemsetAsync(scr.hist, 0, sizeof(uint32_t) * (8 * kRadix + 8), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(scr.status, 0, sizeof(uint32_t) * (size_t)passes * parts * kRadix, s);
    if (e != cudaSuccess) return e;
    if (!hist_ready) {
        const int64_t hist_blocks = std::min<int64_t>((max_k + kThreads * 8 - 1) / (kThreads * 8), 152 * 8);
        k_sort_hist<KeyT><<<(unsigned)hist_blocks, kThreads, 0, s>>>(keys[0], count, passes, scr.hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int p = 0; p < passes; ++p) {
        const int src = p & 1, dst = src ^ 1;
        // ballot ranking on the lower digits, __match_any_sync on the most significant (few distinct values)
        const bool ballot = p + 1 < passes;
        auto kern = wide ? (ballot ? k_sort_pass<KeyT, true, 512> : k_sort_pass<KeyT, false, 512>)
                         : (ballot ? k_sort_pass<KeyT, true, 256> : k_sort_pass<KeyT, false, 256>);
        const int threads = wide ? 512 : 256;
        const size_t smem = wide ? pass_smem<KeyT, 512>() : pass_smem<KeyT, 256>();
        kern<<<(unsigned)parts, threads, smem, s>>>(keys[src], vals[src], keys[dst], vals[dst], count, 8 * p,
                                                    scr.hist + p * kRadix, scr.status + (size_t)p * parts * kRadix,
                                                    scr.part_ctr + p, err_word, give_up ? 0u : kMaxSpins);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_sort(uint64_t *keys[2], uint32_t *vals[2], const uint32_t *counters, uint32_t *err_word,
                        int64_t max_k, int bits, const SortScratch &scr, int *result, cudaStream_t s, bool hist_ready,
                        bool give_up, bool wide)
{
    return sort_impl<uint64_t>(keys, vals, counters + kCntEff, err_word, max_k, bits, scr, result, s, hist_ready,
                               give_up, wide);
}

cudaError_t launch_sort32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *count, uint32_t *err_word,
                          int64_t max_k, int bits, const SortScratch &scr, int *result, cudaStream_t s, bool hist_ready,
                          bool give_up, bool wide)
{
    return sort_impl<uint32_t>(keys, vals, count, err_word, max_k, bits, scr, result, s, hist_ready, give_up, wide);
}

}  // namespace gsr
