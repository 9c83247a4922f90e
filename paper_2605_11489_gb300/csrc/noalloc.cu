// gs_sort_pairs_static: the render's stable LSD radix sort of (key, value)
// pairs, for callers that may not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted after start-up -- under a host framework whose caching allocator owns
// the whole device, or in a real-time loop that must not allocate (cudaMalloc
// can synchronise the device and take milliseconds) -- still needs to sort
// keys. This entry point takes its scratch (digit histograms, decoupled-lookback
// status words, partition tickets and the ping-pong buffer of the passes) from
// one file-scope __device__ array of fixed size instead of allocating it.
//
// The array is part of the library image: every GPU that loads the library
// holds it (about 14 MB) until the process exits. Every call shares it and it
// keeps the previous call's contents, so the sort clears what must start at
// zero itself, and calls whose work overlaps on the GPU (different streams
// without ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int64_t kStaticMaxPairs = 1 << 20;  // largest n accepted
constexpr int kStaticMaxPasses = 8;
constexpr int64_t kStaticParts = kStaticMaxPairs / 4096 + 1;  // 4096 keys per onesweep partition

// layout of the scratch array (256-byte aligned pieces)
constexpr size_t kOffCounters = 0;                                   // u32[kCntSlots]
constexpr size_t kOffHist = 256;                                     // u32[8][256] + u32[8] tickets
constexpr size_t kOffStatus = kOffHist + (8 * 256 + 8) * 4 + 224;    // u32[passes][parts][256]
constexpr size_t kStatusBytes = (size_t)kStaticMaxPasses * kStaticParts * 256 * 4;
constexpr size_t kOffKeys = (kOffStatus + kStatusBytes + 255) / 256 * 256;   // u64[max]
constexpr size_t kOffVals = kOffKeys + (size_t)kStaticMaxPairs * 8;          // u32[max]
constexpr size_t kStaticBytes = kOffVals + (size_t)kStaticMaxPairs * 4;
static_assert(kOffHist % 16 == 0 && kOffStatus % 16 == 0, "scratch pieces must be aligned");

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

__global__ void k_set_count(uint32_t *counters, uint32_t n)
{
    counters[kCntEff] = n;
    counters[kCntErr] = 0u;
}

// copies the sort's error bits (0, or kErrSortTimeout) to the caller's word
__global__ void k_report(const uint32_t *counters, uint32_t *status) { *status = counters[kCntErr]; }

// Device address of the scratch array for the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
// The library's own threads (the server's scheduler) may sort at the same time
// as a caller's thread, so the lookup is serialised.
cudaError_t scratch_address(unsigned char **out)
{
    static unsigned char *addr[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" gs_status gs_sort_pairs_static(const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out,
                                          uint32_t *vals_out, int64_t n, int32_t bits, uint32_t *status,
                                          gs_stream stream)
{
    if (n < 0 || n > kStaticMaxPairs)
        return fail(GS_ERR_INVALID_ARG, "gs_sort_pairs_static: n must be 0..1048576 (the static scratch's capacity)");
    if (bits < 1 || bits > 64) return fail(GS_ERR_INVALID_ARG, "gs_sort_pairs_static: bits must be 1..64");
    if (reinterpret_cast<uintptr_t>(status) & 3)
        return fail(GS_ERR_INVALID_ARG, "gs_sort_pairs_static: the status word must be 4-byte aligned");
    if (n == 0) {
        if (status) GSR_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), (cudaStream_t)stream));
        return GS_OK;
    }
    if (!keys_in || !vals_in || !keys_out || !vals_out)
        return fail(GS_ERR_INVALID_ARG, "gs_sort_pairs_static: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(keys_in) | reinterpret_cast<uintptr_t>(keys_out)) & 7 ||
        (reinterpret_cast<uintptr_t>(vals_in) | reinterpret_cast<uintptr_t>(vals_out)) & 3)
        return fail(GS_ERR_INVALID_ARG, "gs_sort_pairs_static: keys must be 8-byte and values 4-byte aligned");
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    unsigned char *base = nullptr;
    GSR_CUDA(scratch_address(&base));
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + kOffCounters);
    uint64_t *ping_k = reinterpret_cast<uint64_t *>(base + kOffKeys);
    uint32_t *ping_v = reinterpret_cast<uint32_t *>(base + kOffVals);
    SortScratch scr;
    scr.hist = reinterpret_cast<uint32_t *>(base + kOffHist);
    scr.part_ctr = scr.hist + 8 * 256;
    scr.status = reinterpret_cast<uint32_t *>(base + kOffStatus);
    scr.max_parts = kStaticParts;
    // Passes alternate between two buffers; the one the input is copied into is
    // chosen so that the last pass writes the caller's output.
    const int passes = sort_passes(bits);
    uint64_t *k[2];
    uint32_t *v[2];
    if (passes % 2 == 0) {
        k[0] = keys_out, v[0] = vals_out, k[1] = ping_k, v[1] = ping_v;
    } else {
        k[0] = ping_k, v[0] = ping_v, k[1] = keys_out, v[1] = vals_out;
    }
    if (k[0] != keys_in) GSR_CUDA(cudaMemcpyAsync(k[0], keys_in, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (v[0] != vals_in) GSR_CUDA(cudaMemcpyAsync(v[0], vals_in, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    k_set_count<<<1, 1, 0, st>>>(counters, (uint32_t)n);
    GSR_CUDA(cudaGetLastError());
    int result = 0;
    GSR_CUDA(launch_sort(k, v, counters, counters + kCntErr, n, bits, scr, &result, st));
    if (status) {
        k_report<<<1, 1, 0, st>>>(counters, status);
        GSR_CUDA(cudaGetLastError());
    }
    return GS_OK;
}
