// Gradient-aware interpolation (paper Sec. 4.1, Eq. 5-8): super-sampling of the
// low-resolution render by S from its colour and its analytic gradients.
//
// For every low-resolution pixel (x0, y0) and colour channel, the 27 inputs of
// Eq. 7 are Vec(I_3x3), Vec(dI/dx_3x3) and Vec(dI/dy_3x3).
// - Vec is column-wise: input 9 q + 3 (i + 1) + (j + 1) is plane q (0 = I, 1 = dI/dx,
//   2 = dI/dy) at node (x0 + i, y0 + j).
// - Nodes outside the image read 0.
// Each output block is Vec(I_SxS) = M x + b, and output u S + v is the high-resolution pixel
// (S x0 + u, S y0 + v).
//
// The paper realises M as a 3x3 convolution to C feature channels followed by an SxS
// stride-S transposed convolution (Eq. 8). Nothing nonlinear sits between the two, so the
// host folds them, in double, into
//     M = Wt Wc   (S*S x 27)   and   b = Wt bc + bt,
// rounded once to fp32. That is Eq. 7 itself. Per pixel and channel it costs 27 S^2 FMAs
// (432 at S = 4) instead of 27 C + C S^2 (1,376 at C = 32), which puts the FP32 pipe on
// a par with the 192 bytes per pixel of the high-resolution write.
//
// Kernel: one CTA of 128 threads per 32x8 low-resolution pixels. Per colour channel:
// - the three input planes and their one-pixel halo are staged in shared memory (zero
//   outside the image);
// - each thread evaluates M x + b for two pixels 16 apart, one row of their S x S blocks at
//   a time. The two pixels' inputs and sums sit in register pairs, and each weight of M is
//   stored twice in the kernel-parameter constant bank, so one 64-bit constant load and one
//   packed FMA (fma.rn.f32x2, two IEEE fmas, the same results as two scalar ones) serve both
//   pixels;
// - each block row is written as S contiguous floats (one 16-byte store at S = 4).
#include <cuda_runtime.h>

#include <vector>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kGaiTX = 32, kGaiTY = 8;
constexpr int kGaiPx = 2;                              // pixels per thread, kGaiTX / 2 apart in x
constexpr int kGaiThreads = kGaiTX * kGaiTY / kGaiPx;  // 128
constexpr int kHaloX = kGaiTX + 2, kHaloY = kGaiTY + 2;

// M and b with every entry duplicated ({m, m}): the operand of a packed FMA over two pixels
template <int S>
struct GaiParams {
    float2 M[S * S][27];
    float2 b[S * S];
};

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
// two fmas, lane by lane: (a.x * b.x + c.x, a.y * b.y + c.y), each rounded once
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <int S>
__global__ void __launch_bounds__(kGaiThreads, 6) k_gai(const GaiParams<S> w, const float *__restrict__ rgb,
                                                     const float *__restrict__ dcdx, const float *__restrict__ dcdy,
                                                     int W, int H, int channels, float *__restrict__ out)
{
    __shared__ float tile[3][kHaloY][kHaloX];
    constexpr int kHalf = kGaiTX / kGaiPx;
    const int x0 = blockIdx.x * kGaiTX, y0 = blockIdx.y * kGaiTY;
    const int tx = threadIdx.x % kHalf, ty = threadIdx.x / kHalf;
    const int y = y0 + ty;
    const size_t HW = (size_t)W * H;
    const size_t Wo = (size_t)S * W, HWo = Wo * (size_t)S * H;
    for (int c = 0; c < channels; ++c) {
        for (int k = threadIdx.x; k < kHaloY * kHaloX; k += kGaiThreads) {
            const int ly = k / kHaloX, lx = k % kHaloX;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const size_t g = c * HW + (size_t)gy * W + gx;
            tile[0][ly][lx] = ok ? rgb[g] : 0.f;
            tile[1][ly][lx] = ok ? dcdx[g] : 0.f;
            tile[2][ly][lx] = ok ? dcdy[g] : 0.f;
        }
        __syncthreads();
        static_assert(kGaiPx == 2, "the packed FMA takes the thread's two pixels");
        unsigned long long in[27];  // {pixel 0, pixel 1}
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    in[9 * q + 3 * i + j] = pack2(tile[q][ty + j][tx + i], tile[q][ty + j][tx + kHalf + i]);
        // one row v of the S x S blocks at a time: every weight is fetched once for both pixels
#pragma unroll
        for (int v = 0; v < S; ++v) {
            float acc[kGaiPx][S];
#pragma unroll
            for (int u = 0; u < S; ++u) {
                const int s = u * S + v;
                unsigned long long a2 = pack2(w.b[s].x, w.b[s].y);
#pragma unroll
                for (int k = 0; k < 27; ++k) a2 = fma2(pack2(w.M[s][k].x, w.M[s][k].y), in[k], a2);
                const float2 r = unpack2(a2);
                acc[0][u] = r.x;
                acc[1][u] = r.y;
            }
#pragma unroll
            for (int p = 0; p < kGaiPx; ++p) {
                const int x = x0 + tx + p * kHalf;
                if (x >= W || y >= H) continue;
                float *row = out + c * HWo + ((size_t)S * y + v) * Wo + (size_t)S * x;
                if constexpr (S == 4) {
                    *reinterpret_cast<float4 *>(row) = make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
                } else if constexpr (S == 2) {
                    *reinterpret_cast<float2 *>(row) = make_float2(acc[p][0], acc[p][1]);
                } else {
#pragma unroll
                    for (int u = 0; u < S; ++u) row[u] = acc[p][u];
                }
            }
        }
        __syncthreads();
    }
}

template <int S>
cudaError_t launch_gai_s(const std::vector<double> &M, const std::vector<double> &b, const float *rgb,
                         const float *dcdx, const float *dcdy, int W, int H, int channels, float *out,
                         cudaStream_t st)
{
    GaiParams<S> p;
    for (int s = 0; s < S * S; ++s) {
        for (int k = 0; k < 27; ++k) {
            const float m = (float)M[(size_t)s * 27 + k];
            p.M[s][k] = make_float2(m, m);
        }
        p.b[s] = make_float2((float)b[s], (float)b[s]);
    }
    const dim3 grid((W + kGaiTX - 1) / kGaiTX, (H + kGaiTY - 1) / kGaiTY);  // kGaiThreads threads each
    k_gai<S><<<grid, kGaiThreads, 0, st>>>(p, rgb, dcdx, dcdy, W, H, channels, out);
    return cudaGetLastError();
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace gsr

// ============================================================================ C ABI

extern "C" gs_status gs_gai_upsample(const gs_gai_weights *w, const float *rgb, const float *dcdx,
                                     const float *dcdy, int32_t channels, int32_t width, int32_t height, float *out,
                                     gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.gai_upsample");
    using namespace gsr;
    if (!w || !w->wc || !w->wt) return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: weights are NULL");
    const int S = w->scale, C = w->features;
    if (S < 2 || S > 4) return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: scale must be 2, 3 or 4");
    if (C < 1 || C > 1024) return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: features must be 1..1024");
    if (channels < 1 || channels > 64) return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: channels must be 1..64");
    if (width < 1 || height < 1 || width > 65535 || height > 65535)
        return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: width/height must be in 1..65535");
    if (!rgb || !dcdx || !dcdy || !out) return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: NULL plane");
    if (!aligned(rgb, 4) || !aligned(dcdx, 4) || !aligned(dcdy, 4) || !aligned(out, 16))
        return fail(GS_ERR_INVALID_ARG, "gs_gai_upsample: planes must be 4-byte and the output 16-byte aligned");
    // M = Wt Wc and b = Wt bc + bt in double (Eq. 7 from the two layers of Eq. 8)
    std::vector<double> M((size_t)S * S * 27, 0.0), b((size_t)S * S, 0.0);
    for (int s = 0; s < S * S; ++s) {
        double bs = w->bt ? (double)w->bt[s] : 0.0;
        for (int f = 0; f < C; ++f) {
            const double t = (double)w->wt[(size_t)s * C + f];
            if (t == 0.0) continue;
            for (int k = 0; k < 27; ++k) M[(size_t)s * 27 + k] += t * (double)w->wc[(size_t)f * 27 + k];
            if (w->bc) bs += t * (double)w->bc[f];
        }
        b[s] = bs;
    }
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launch
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = S == 2 ? launch_gai_s<2>(M, b, rgb, dcdx, dcdy, width, height, channels, out, st)
                  : S == 3 ? launch_gai_s<3>(M, b, rgb, dcdx, dcdy, width, height, channels, out, st)
                           : launch_gai_s<4>(M, b, rgb, dcdx, dcdy, width, height, channels, out, st);
    if (e != cudaSuccess) return cuda_fail(e, "gs_gai_upsample launch");
    return GS_OK;
}
