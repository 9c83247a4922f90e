// Frame-interpolation geometry (paper Sec. 4.2, "Forward-Backward Warping"):
// camera motion vectors, the depth-tested forward warp w(., V) and the warped
// image gradient, for one source frame toward one target camera.
//
//   V[x]   = Proj(UnProj(x, D[x], P_src), P_dst) - x                       (Sec. 4.2)
//   w(F,V) : each moving source pixel lands on the target pixel that contains
//            x + V[x]; of several landing on one target pixel the nearest to the
//            target camera wins (target-camera z, then the smaller source index);
//            a target pixel nobody reaches is a hole (index -1, zeros)
//   G_dst  = w(G_src, V) . (dy/dx)^-1, dy/dx = I + dV/dx taken by differences
//            of the landing positions over the source pixel grid (the chain
//            rule behind the paper's "nabla V . w(G_1, V)")
//
// Readings where the paper is silent: D is the render's depth channel divided
// by its alpha (a pixel moves only where alpha > alpha_min; with no alpha plane
// the depth is a point depth and moves where it is > 0); UnProj lifts the pixel
// centre (i + 0.5, j + 0.5) to camera z = D; central differences, one-sided
// where a neighbour does not move, identity where neither does; a non-positive
// determinant (a fold) gives a zero warped gradient.
//
// Two launches:
//   k_warp_scatter (one thread per source column over 4 rows): the landing
//     position, fixed to one fp32 round-to-nearest operation sequence (no
//     contraction), written to a position scratch (only when the warped
//     gradient is asked for) and as the motion map; an atomicMin of the 64-bit
//     key (z bits << 32 | source index) into the target pixel's slot. z > near
//     >= 0, so the bit pattern of z orders like its value.
//   k_warp_gather (four target pixels per thread, a block apart): reads and
//     resets the slots (so the slot array is all ones again for the next
//     call), copies the winners' planes with every load of four channels in
//     flight at once, and forms the warped gradient from each winner's
//     neighbours' positions.
#include <cuda_runtime.h>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kWarpThreadsX = 128;

struct WarpCams {
    float sv[12], tv[12];          // source and target world -> camera [R | t]
    float sfx, sfy, scx, scy;      // source intrinsics
    float tfx, tfy, tcx, tcy, tnear;
    int32_t W, H, Wt, Ht;
};

// Normalised ray offset of pixel-centre coordinate k for focal f and principal
// point c: ((k + 0.5) - c) / f, rounded to nearest at each step.
__device__ __forceinline__ float ray_offset(int k, float cpp, float f)
{
    return __fdiv_rn(__fsub_rn(__fadd_rn((float)k, 0.5f), cpp), f);
}

// Landing position (u, v) and target-camera z of the source pixel whose ray
// offsets are (xn, yn), at lifted depth d: every operation rounded to nearest,
// in this order.
__device__ __forceinline__ bool land(const WarpCams &c, float xn, float yn, float d, float &u, float &v, float &z)
{
    const float a0 = __fsub_rn(__fmul_rn(xn, d), c.sv[3]);
    const float a1 = __fsub_rn(__fmul_rn(yn, d), c.sv[7]);
    const float a2 = __fsub_rn(d, c.sv[11]);
    // world = R^T (camera - t)
    const float xw = __fadd_rn(__fadd_rn(__fmul_rn(c.sv[0], a0), __fmul_rn(c.sv[4], a1)), __fmul_rn(c.sv[8], a2));
    const float yw = __fadd_rn(__fadd_rn(__fmul_rn(c.sv[1], a0), __fmul_rn(c.sv[5], a1)), __fmul_rn(c.sv[9], a2));
    const float zw = __fadd_rn(__fadd_rn(__fmul_rn(c.sv[2], a0), __fmul_rn(c.sv[6], a1)), __fmul_rn(c.sv[10], a2));
    const float X = __fadd_rn(
        __fadd_rn(__fadd_rn(__fmul_rn(c.tv[0], xw), __fmul_rn(c.tv[1], yw)), __fmul_rn(c.tv[2], zw)), c.tv[3]);
    const float Y = __fadd_rn(
        __fadd_rn(__fadd_rn(__fmul_rn(c.tv[4], xw), __fmul_rn(c.tv[5], yw)), __fmul_rn(c.tv[6], zw)), c.tv[7]);
    const float Z = __fadd_rn(
        __fadd_rn(__fadd_rn(__fmul_rn(c.tv[8], xw), __fmul_rn(c.tv[9], yw)), __fmul_rn(c.tv[10], zw)), c.tv[11]);
    if (!(Z > c.tnear)) return false;
    u = __fadd_rn(__fdiv_rn(__fmul_rn(c.tfx, X), Z), c.tcx);
    v = __fadd_rn(__fdiv_rn(__fmul_rn(c.tfy, Y), Z), c.tcy);
    z = Z;
    return true;
}

// One thread per source column over kScatterRows rows: the column's ray offset
// is computed once and the rows' offsets once per block (the same values a
// per-pixel evaluation gives).
constexpr int kScatterRows = 4;

template <bool kAlpha>
__global__ void __launch_bounds__(kWarpThreadsX) k_warp_scatter(WarpCams c, const float *__restrict__ depth,
                                                                const float *__restrict__ alpha, float alpha_min,
                                                                float2 *__restrict__ pos, float *__restrict__ motion,
                                                                unsigned long long *__restrict__ best)
{
    __shared__ float s_yn[kScatterRows];
    const int i = blockIdx.x * kWarpThreadsX + threadIdx.x, j0 = blockIdx.y * kScatterRows;
    if (threadIdx.x < kScatterRows) s_yn[threadIdx.x] = ray_offset(j0 + (int)threadIdx.x, c.scy, c.sfy);
    __syncthreads();
    if (i >= c.W) return;
    const float xn = ray_offset(i, c.scx, c.sfx);
    const size_t n = (size_t)c.W * c.H;
    const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int r = 0; r < kScatterRows; ++r) {
        const int j = j0 + r;
        if (j >= c.H) break;
        const size_t p = (size_t)j * c.W + i;
        float d;
        bool moves;
        if (kAlpha) {
            const float a = alpha[p];
            moves = a > alpha_min;
            d = moves ? __fdiv_rn(depth[p], a) : 0.f;
        } else {
            d = depth[p];
            moves = d > 0.f;
        }
        float u = qnan, v = qnan, z = 0.f;
        if (moves) moves = land(c, xn, s_yn[r], d, u, v, z);
        if (!moves) u = v = qnan;
        if (pos) pos[p] = make_float2(u, v);  // only the warped gradient needs the neighbours' positions
        if (motion) {
            motion[p] = moves ? __fsub_rn(u, __fadd_rn((float)i, 0.5f)) : u;
            motion[n + p] = moves ? __fsub_rn(v, __fadd_rn((float)j, 0.5f)) : v;
        }
        if (moves && u >= 0.f && u < (float)c.Wt && v >= 0.f && v < (float)c.Ht) {
            const size_t q = (size_t)floorf(v) * c.Wt + (size_t)floorf(u);
            atomicMin(best + q, ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)p);
        }
    }
}

// a * b - c * d with one rounding error in each product compensated (Kahan's
// 2x2 determinant): relative error within a few ulps even under cancellation.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d)
{
    const float w = c * d;
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return f + e;
}

__device__ __forceinline__ bool moving(const float2 &q) { return q.x == q.x; }

constexpr int kGatherThreads = 128;
constexpr int kGatherPx = 4;  // target pixels per thread, kGatherThreads apart (every access coalesced)

// Warped gradient of one winner p (source pixel (i, j)): J from its neighbours'
// landing positions, then (g0, g1) . J^-1 for every gradient channel.
__device__ __forceinline__ void warped_gradient(const WarpCams &c, const float2 *__restrict__ pos, uint32_t p,
                                               bool hit, size_t q, size_t n, size_t nt, int gch,
                                               const float *__restrict__ dcdx, const float *__restrict__ dcdy,
                                               float *__restrict__ odx, float *__restrict__ ody)
{
    const float qnan = __int_as_float(0x7fc00000);
    float J0 = 1.f, J1 = 0.f, J2 = 0.f, J3 = 1.f;
    if (hit) {
        // J = [[du/dx, du/dy], [dv/dx, dv/dy]] from the neighbours' landing positions
        const int i = (int)(p % (uint32_t)c.W), j = (int)(p / (uint32_t)c.W);
        const float2 m = pos[p];
        const float2 l = i > 0 ? pos[p - 1] : make_float2(qnan, 0.f);
        const float2 r = i < c.W - 1 ? pos[p + 1] : make_float2(qnan, 0.f);
        const float2 t = j > 0 ? pos[p - c.W] : make_float2(qnan, 0.f);
        const float2 b = j < c.H - 1 ? pos[p + c.W] : make_float2(qnan, 0.f);
        const bool L = moving(l), R = moving(r), U = moving(t), D = moving(b);
        if (L && R) {
            J0 = (r.x - l.x) * 0.5f;
            J2 = (r.y - l.y) * 0.5f;
        } else if (R) {
            J0 = r.x - m.x;
            J2 = r.y - m.y;
        } else if (L) {
            J0 = m.x - l.x;
            J2 = m.y - l.y;
        }
        if (U && D) {
            J1 = (b.x - t.x) * 0.5f;
            J3 = (b.y - t.y) * 0.5f;
        } else if (D) {
            J1 = b.x - m.x;
            J3 = b.y - m.y;
        } else if (U) {
            J1 = m.x - t.x;
            J3 = m.y - t.y;
        }
    }
    const float det = diff_of_products(J0, J3, J1, J2);
    const bool ok = hit && det > 0.f;
    for (int ch = 0; ch < gch; ++ch) {
        float gx = 0.f, gy = 0.f;
        if (ok) {
            const float g0 = __ldg(dcdx + ch * n + p), g1 = __ldg(dcdy + ch * n + p);
            // (g0, g1) . J^-1, J^-1 = [[J3, -J1], [-J2, J0]] / det
            gx = __fdiv_rn(diff_of_products(g0, J3, g1, J2), det);
            gy = __fdiv_rn(diff_of_products(g1, J0, g0, J1), det);
        }
        odx[ch * nt + q] = gx;
        ody[ch * nt + q] = gy;
    }
}

template <bool kGrad>
__global__ void __launch_bounds__(kGatherThreads)
    k_warp_gather(WarpCams c, const float2 *__restrict__ pos, unsigned long long *__restrict__ best, int channels,
                  const float *__restrict__ planes, int gch, const float *__restrict__ dcdx,
                  const float *__restrict__ dcdy, int32_t *__restrict__ index, float *__restrict__ zout,
                  float *__restrict__ out, float *__restrict__ odx, float *__restrict__ ody)
{
    const size_t nt = (size_t)c.Wt * c.Ht, n = (size_t)c.W * c.H;
    const size_t q0 = (size_t)blockIdx.x * (kGatherThreads * kGatherPx) + threadIdx.x;
    size_t q[kGatherPx];
    unsigned long long key[kGatherPx];
#pragma unroll
    for (int k = 0; k < kGatherPx; ++k) {
        q[k] = q0 + (size_t)k * kGatherThreads;
        key[k] = q[k] < nt ? best[q[k]] : kEmpty;
    }
    uint32_t p[kGatherPx];
    bool hit[kGatherPx];
#pragma unroll
    for (int k = 0; k < kGatherPx; ++k) {
        p[k] = 0u;
        hit[k] = false;
        if (q[k] >= nt) continue;
        best[q[k]] = kEmpty;  // leave the slot array all ones for the next call
        p[k] = (uint32_t)key[k];
        // a slot that names no source pixel of this call (only possible if calls on
        // one context overlapped on the GPU) reads as a hole rather than out of bounds
        hit[k] = key[k] != kEmpty && (size_t)p[k] < n;
        if (!hit[k]) p[k] = 0u;
        if (index) index[q[k]] = hit[k] ? (int32_t)p[k] : -1;
        if (zout) zout[q[k]] = hit[k] ? __uint_as_float((uint32_t)(key[k] >> 32)) : 0.f;
    }
    if (out) {
        // four channels at a time: 4 x kGatherPx independent loads in flight
        int ch = 0;
        for (; ch + 4 <= channels; ch += 4) {
            float v[4][kGatherPx];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                for (int k = 0; k < kGatherPx; ++k)
                    v[cc][k] = (q[k] < nt && hit[k]) ? __ldg(planes + (size_t)(ch + cc) * n + p[k]) : 0.f;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                for (int k = 0; k < kGatherPx; ++k)
                    if (q[k] < nt) out[(size_t)(ch + cc) * nt + q[k]] = v[cc][k];
        }
        for (; ch < channels; ++ch) {
            float v[kGatherPx];
#pragma unroll
            for (int k = 0; k < kGatherPx; ++k)
                v[k] = (q[k] < nt && hit[k]) ? __ldg(planes + (size_t)ch * n + p[k]) : 0.f;
#pragma unroll
            for (int k = 0; k < kGatherPx; ++k)
                if (q[k] < nt) out[(size_t)ch * nt + q[k]] = v[k];
        }
    }
    if constexpr (kGrad) {
#pragma unroll
        for (int k = 0; k < kGatherPx; ++k)
            if (q[k] < nt) warped_gradient(c, pos, p[k], hit[k], q[k], n, nt, gch, dcdx, dcdy, odx, ody);
    }
}

WarpCams warp_cams(const gs_camera &s, const gs_camera &t)
{
    WarpCams c{};
    for (int k = 0; k < 12; ++k) {
        c.sv[k] = s.viewmat[k];
        c.tv[k] = t.viewmat[k];
    }
    c.sfx = s.fx;
    c.sfy = s.fy;
    c.scx = s.cx;
    c.scy = s.cy;
    c.tfx = t.fx;
    c.tfy = t.fy;
    c.tcx = t.cx;
    c.tcy = t.cy;
    c.tnear = t.near_plane;
    c.W = s.width;
    c.H = s.height;
    c.Wt = t.width;
    c.Ht = t.height;
    return c;
}

bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace

bool warp_needs_positions(const gs_warp_input &in, const gs_warp_output &out)
{
    return in.grad_channels > 0 && out.dcdx && out.dcdy;
}

cudaError_t launch_warp(const gs_camera &src, const gs_camera &dst, const gs_warp_input &in, const gs_warp_output &out,
                        float2 *pos, unsigned long long *best, cudaStream_t s)
{
    const WarpCams c = warp_cams(src, dst);
    if (!warp_needs_positions(in, out)) pos = nullptr;
    const dim3 blk(kWarpThreadsX);
    const dim3 gs((src.width + kWarpThreadsX - 1) / kWarpThreadsX, (src.height + kScatterRows - 1) / kScatterRows);
    const size_t nt = (size_t)dst.width * dst.height;
    const unsigned gt = (unsigned)((nt + kGatherThreads * kGatherPx - 1) / (kGatherThreads * kGatherPx));
    if (in.alpha)
        k_warp_scatter<true><<<gs, blk, 0, s>>>(c, in.depth, in.alpha, in.alpha_min, pos, out.motion, best);
    else
        k_warp_scatter<false><<<gs, blk, 0, s>>>(c, in.depth, nullptr, in.alpha_min, pos, out.motion, best);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (warp_needs_positions(in, out))
        k_warp_gather<true><<<gt, kGatherThreads, 0, s>>>(c, pos, best, in.channels, in.planes, in.grad_channels,
                                                          in.dcdx, in.dcdy, out.index, out.z, out.planes, out.dcdx,
                                                          out.dcdy);
    else
        k_warp_gather<false><<<gt, kGatherThreads, 0, s>>>(c, nullptr, best, in.channels, in.planes, 0, nullptr,
                                                           nullptr, out.index, out.z, out.planes, nullptr, nullptr);
    return cudaGetLastError();
}

gs_status check_warp_args(const gs_camera *src, const gs_camera *dst, const gs_warp_input *in,
                          const gs_warp_output *out)
{
    gs_status r;
    if (!in || !out) return fail(GS_ERR_INVALID_ARG, "warp input and output must be non-NULL");
    if ((r = check_cam(src)) != GS_OK) return r;
    if ((r = check_cam(dst)) != GS_OK) return r;
    if (!(dst->near_plane >= 0.f)) return fail(GS_ERR_INVALID_ARG, "the target camera's near_plane must be >= 0");
    if (!in->depth) return fail(GS_ERR_INVALID_ARG, "warp depth plane is NULL");
    if (in->channels < 0 || in->grad_channels < 0 || in->channels > 64 || in->grad_channels > 64)
        return fail(GS_ERR_INVALID_ARG, "channels and grad_channels must be in 0..64");
    if (in->channels > 0 && out->planes && !in->planes)
        return fail(GS_ERR_INVALID_ARG, "output planes requested without input planes");
    const bool grads = in->grad_channels > 0 && (out->dcdx || out->dcdy);
    if (grads && (!in->dcdx || !in->dcdy || !out->dcdx || !out->dcdy))
        return fail(GS_ERR_INVALID_ARG, "warped gradients need dcdx and dcdy on both sides");
    const void *ps[] = {in->depth, in->alpha, in->planes, in->dcdx, in->dcdy, out->motion, out->index,
                        out->z, out->planes, out->dcdx, out->dcdy};
    for (const void *p : ps)
        if (p && !aligned4(p)) return fail(GS_ERR_INVALID_ARG, "warp planes must be 4-byte aligned");
    return GS_OK;
}

}  // namespace gsr

// ============================================================================ C ABI

extern "C" gs_status gs_warp(gs_context *ctx, const gs_camera *src, const gs_camera *dst, const gs_warp_input *in,
                             const gs_warp_output *out, gs_stream stream)
{
    gsr::NvtxRange nvtx_("gsr.warp");
    using namespace gsr;
    if (!ctx) return fail(GS_ERR_INVALID_ARG, "ctx is NULL");
    gs_status r = check_warp_args(src, dst, in, out);
    if (r != GS_OK) return r;
    GSR_CUDA(cudaSetDevice(context_device(ctx)));
    cudaGetLastError();  // a stale non-sticky error must not be charged to this call's launches
    cudaStream_t st = (cudaStream_t)stream;
    float2 *pos = nullptr;
    unsigned long long *best = nullptr;
    const size_t n_pos = warp_needs_positions(*in, *out) ? (size_t)src->width * src->height : 0;
    r = context_warp_scratch(ctx, n_pos, (size_t)dst->width * dst->height, st, &pos, &best);
    if (r != GS_OK) return r;
    const cudaError_t e = launch_warp(*src, *dst, *in, *out, pos, best, st);
    if (e != cudaSuccess) {
        warp_scratch_dirty(ctx);
        return cuda_fail(e, "gs_warp launch");
    }
    return GS_OK;
}
