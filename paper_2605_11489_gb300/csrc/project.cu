// K1: projection, culling and SH colour of 3D Gaussians (paper Sec. 3).
//
// Per Gaussian: activations (scale = exp(log_scale), unit quaternion, opacity =
// sigmoid(logit)), Sigma = R S S^T R^T, camera transform, EWA local-affine
// projection Sigma2D = J W Sigma W^T J^T plus a 0.3 px^2 low-pass, the conic
// Sigma2D^-1, the support rectangle (exact bounding box of the ellipse where
// opacity * G >= 1/255), the number of tiles it touches, and the view-dependent
// colour from real SH (Condon-Shortley phase, degree 0..3, +0.5, clamped at 0).
//
// The depth key and the support rectangle decide culling, tiling and sort
// order, so they are computed by a fixed sequence of IEEE fp32 round-to-nearest
// operations (explicit __f*_rn intrinsics, never contracted), including a
// Cody-Waite exp and an atanh-series log written from their published methods.
// Any other fp32 implementation of the same sequence reproduces them bit for
// bit.
//
// Layout: in k_project one thread owns one Gaussian, so a warp reads 128
// contiguous bytes of every geometry plane; it writes whole records with the
// colour left at 0. k_colour then streams the SH
// planes (192 B per Gaussian at degree 3) for the visible Gaussians only, one
// thread each, and fills in the colour.
#include "gsr_internal.cuh"
#include <algorithm>

namespace gsr {
namespace {

__device__ __forceinline__ float A(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float S(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float M(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float D(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float F(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// e^x: n = rint(x log2 e), r = x - n ln2 (ln2 as 0.693359375 + lo, two FMAs),
// e^r by its degree-7 Taylor polynomial (Horner, FMA), times 2^n built exactly.
__device__ float rn_exp(float x)
{
    if (x != x) return x;
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    const float n = rintf(M(x, 1.44269502e+00f));
    float r = F(-n, 0.693359375f, x);
    r = F(-n, -2.12194442e-04f, r);
    float p = 1.98412701e-04f;
    p = F(p, r, 1.38888892e-03f);
    p = F(p, r, 8.33333377e-03f);
    p = F(p, r, 4.16666679e-02f);
    p = F(p, r, 1.66666672e-01f);
    p = F(p, r, 0.5f);
    p = F(p, r, 1.0f);
    p = F(p, r, 1.0f);
    return M(p, __int_as_float(((int)n + 127) << 23));
}

// ln x for normal x > 0: x = m 2^e, m in [sqrt(1/2), sqrt(2)]; ln m = 2 atanh(s)
// with s = (m - 1)/(m + 1) by the odd series through s^11.
__device__ float rn_log(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421354e+00f) {
        m = M(m, 0.5f);
        e += 1;
    }
    const float s = D(S(m, 1.0f), A(m, 1.0f));
    const float w = M(s, s);
    float p = 9.09090936e-02f;
    p = F(p, w, 1.11111112e-01f);
    p = F(p, w, 1.42857149e-01f);
    p = F(p, w, 2.00000003e-01f);
    p = F(p, w, 3.33333343e-01f);
    const float t = M(2.0f, s);
    const float lm = F(M(t, w), p, t);
    const float ef = (float)e;
    return F(ef, 0.693359375f, F(ef, -2.12194442e-04f, lm));
}

struct Proj {
    bool vis;
    float u, v, ca, cb, cc, o, z;  // u, v: the centre relative to the rectangle's first pixel centre
    uint32_t rlo, rhi, nt;
    float n[3];  // camera-space normal (with NRM only)
    float pl[2]; // intersection-depth slope per pixel, (dz/du, dz/dv) (with NRM only)
};

// Error-free transformations (Dekker, Knuth): a * b = p + e and a + b = s + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = M(a, b);
    e = F(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = A(a, b);
    const float bb = S(s, a);
    e = A(S(a, S(s, bb)), S(b, bb));
}
// w . m + t as an unevaluated sum hi + lo (about 44 significant bits)
__device__ __forceinline__ void ff_affine(const float *w, float m0, float m1, float m2, float t, float &hi, float &lo)
{
    float p0, e0, p1, e1, p2, e2, s, q1, q2, q3;
    two_prod(w[0], m0, p0, e0);
    two_prod(w[1], m1, p1, e1);
    two_prod(w[2], m2, p2, e2);
    two_sum(p0, p1, s, q1);
    two_sum(s, p2, s, q2);
    two_sum(s, t, hi, q3);
    lo = A(A(A(e0, e1), A(e2, q1)), A(q2, q3));
}
// f * (x / z) + c - origin, with x, z float-float and rz ~ 1/z: the projected centre
// relative to an integer pixel origin, rounded once at the end
__device__ __forceinline__ float ff_centre(float xh, float xl, float zh, float zl, float rz, float f, float c,
                                           float origin)
{
    const float qh = M(xh, rz);
    float p, pe;
    two_prod(qh, zh, p, pe);
    const float r = A(S(S(xh, p), pe), F(-qh, zl, xl));  // x - qh z
    const float ql = M(r, rz);
    float fp, fe, s, se;
    two_prod(f, qh, fp, fe);
    two_sum(fp, c, s, se);
    return A(S(s, origin), A(se, F(f, ql, fe)));
}

// Projection of one Gaussian (Sec. 3: Sigma = R S S^T R^T, EWA Sigma2D = J W Sigma W^T J^T + 0.3 I).
// The depth key and the support rectangle follow the fixed fp32 round-to-nearest sequence below
// (the same as the oracle's discrete spec, step by step). The centre and the conic, which only
// scale the compositing arithmetic, are computed for accuracy instead: the centre in float-float,
// relative to the rectangle's first pixel, so that its error is ~1e-7 of the distance to a pixel
// rather than of the absolute pixel coordinate; the determinant of Sigma2D = N N^T + 0.3 I as
// |N0 x N1|^2 + 0.3 (|N0|^2 + |N1|^2) + 0.09 (Binet-Cauchy), a sum of positive terms that
// does not cancel for elongated footprints.
template <bool NRM = false>
__device__ __forceinline__ void project_one(const CamParams &c, float mx, float my, float mz, float ls0, float ls1,
                                            float ls2, float qw, float qx, float qy, float qz, float logit,
                                            Proj &P)
{
    P.vis = false;
    P.nt = 0;
    const float *vm = c.vm;
    // D1, D2: camera-space position
    const float tz = A(A(A(M(vm[8], mx), M(vm[9], my)), M(vm[10], mz)), vm[11]);
    if (!(tz > c.near_plane)) return;
    const float tx = A(A(A(M(vm[0], mx), M(vm[1], my)), M(vm[2], mz)), vm[3]);
    const float ty = A(A(A(M(vm[4], mx), M(vm[5], my)), M(vm[6], mz)), vm[7]);
    // D3: scales; D4, D5: R(q / |q|) from the unnormalised quaternion with f = 2 / |q|^2
    const float s0 = rn_exp(ls0), s1 = rn_exp(ls1), s2 = rn_exp(ls2);
    const float n2 = A(A(A(M(qw, qw), M(qx, qx)), M(qy, qy)), M(qz, qz));
    if (!(n2 > 0.0f)) return;
    const float f = D(2.0f, n2);
    float R[9];
    R[0] = S(1.0f, M(f, A(M(qy, qy), M(qz, qz))));
    R[1] = M(f, S(M(qx, qy), M(qw, qz)));
    R[2] = M(f, A(M(qx, qz), M(qw, qy)));
    R[3] = M(f, A(M(qx, qy), M(qw, qz)));
    R[4] = S(1.0f, M(f, A(M(qx, qx), M(qz, qz))));
    R[5] = M(f, S(M(qy, qz), M(qw, qx)));
    R[6] = M(f, S(M(qx, qz), M(qw, qy)));
    R[7] = M(f, A(M(qy, qz), M(qw, qx)));
    R[8] = S(1.0f, M(f, A(M(qx, qx), M(qy, qy))));
    // D6: M = R diag(s); D7: V = W M
    const float sc[3] = {s0, s1, s2};
    float V[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            V[3 * r + k] = A(A(M(vm[4 * r], M(R[k], sc[k])), M(vm[4 * r + 1], M(R[3 + k], sc[k]))),
                             M(vm[4 * r + 2], M(R[6 + k], sc[k])));
    // D8: one reciprocal of the depth; the guard-clamped x/z, y/z for the Jacobian
    const float rz = D(1.0f, tz);
    const float xz = M(tx, rz), yz = M(ty, rz);
    const float xc = fminf(c.limx, fmaxf(-c.limx, xz)), yc = fminf(c.limy, fmaxf(-c.limy, yz));
    // D9: N = J V, row by row: N0 = (fx/z)(V0 - x' V2), N1 = (fy/z)(V1 - y' V2)
    const float ax = M(c.fx, rz), ay = M(c.fy, rz);
    float N[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        N[k] = M(ax, S(V[k], M(xc, V[6 + k])));
        N[3 + k] = M(ay, S(V[3 + k], M(yc, V[6 + k])));
    }
    // D10: diagonal of Sigma2D
    const float A0 = A(A(M(N[0], N[0]), M(N[1], N[1])), M(N[2], N[2]));
    const float C0 = A(A(M(N[3], N[3]), M(N[4], N[4])), M(N[5], N[5]));
    const float Aa = A(A0, 3.00000012e-01f), Cc = A(C0, 3.00000012e-01f);
    // D13: opacity, the alpha-cut level; D14: half-extents; D15: centre; D16: rectangle
    const float o = D(1.0f, A(1.0f, rn_exp(-logit)));
    if (!(M(255.0f, o) >= 1.0f)) return;
    const float kk = M(2.0f, rn_log(M(255.0f, o)));
    const float ex = __fsqrt_rn(M(kk, Aa)), ey = __fsqrt_rn(M(kk, Cc));
    const float u = A(M(c.fx, xz), c.cx);
    const float v = A(M(c.fy, yz), c.cy);
    const float xlo = S(S(u, ex), 0.5f), xhi = S(A(u, ex), 0.5f);
    const float ylo = S(S(v, ey), 0.5f), yhi = S(A(v, ey), 0.5f);
    const float wm1 = (float)(c.width - 1), hm1 = (float)(c.height - 1);
    if (!(xhi >= 0.0f) || !(xlo <= wm1) || !(yhi >= 0.0f) || !(ylo <= hm1)) return;
    const int x0 = (int)fmaxf(0.0f, ceilf(xlo)), x1 = (int)fminf(wm1, floorf(xhi));
    const int y0 = (int)fmaxf(0.0f, ceilf(ylo)), y1 = (int)fminf(hm1, floorf(yhi));
    if (x0 > x1 || y0 > y1) return;
    P.vis = true;
    // continuous part: the centre relative to pixel (x0, y0)'s centre, in float-float
    float Xh, Xl, Yh, Yl, Zh, Zl;
    ff_affine(vm + 0, mx, my, mz, vm[3], Xh, Xl);
    ff_affine(vm + 4, mx, my, mz, vm[7], Yh, Yl);
    ff_affine(vm + 8, mx, my, mz, vm[11], Zh, Zl);
    const float rzh = D(1.0f, Zh);
    P.u = ff_centre(Xh, Xl, Zh, Zl, rzh, c.fx, c.cx, A((float)x0, 0.5f));
    P.v = ff_centre(Yh, Yl, Zh, Zl, rzh, c.fy, c.cy, A((float)y0, 0.5f));
    // the conic Sigma2D^-1 with the non-cancelling determinant
    const float B = F(N[0], N[3], F(N[1], N[4], M(N[2], N[5])));
    const float cr0 = F(N[1], N[5], -M(N[2], N[4]));
    const float cr1 = F(N[2], N[3], -M(N[0], N[5]));
    const float cr2 = F(N[0], N[4], -M(N[1], N[3]));
    const float det = A(F(0.3f, A(A0, C0), F(cr0, cr0, F(cr1, cr1, M(cr2, cr2)))), 0.09f);
    const float inv = __frcp_rn(det);
    P.ca = M(Cc, inv);
    P.cb = -M(B, inv);
    P.cc = M(Aa, inv);
    P.o = o;
    P.z = tz;
    P.rlo = (uint32_t)x0 | ((uint32_t)y0 << 16);
    P.rhi = (uint32_t)x1 | ((uint32_t)y1 << 16);
    const int sh = c.tile_shift;
    P.nt = (uint32_t)(((x1 >> sh) - (x0 >> sh) + 1) * ((y1 >> sh) - (y0 >> sh) + 1));
    if (NRM) {
        // normal (RaDe-GS, Sec. 5.1): the axis of the smallest scale (the first of equal
        // log-scales), turned to face the camera, in camera coordinates
        const int k = ls1 < ls0 ? (ls2 < ls1 ? 2 : 1) : (ls2 < ls0 ? 2 : 0);
        float nw0 = k == 0 ? R[0] : (k == 1 ? R[1] : R[2]);
        float nw1 = k == 0 ? R[3] : (k == 1 ? R[4] : R[5]);
        float nw2 = k == 0 ? R[6] : (k == 1 ? R[7] : R[8]);
        const float facing = (mx - c.campos[0]) * nw0 + (my - c.campos[1]) * nw1 + (mz - c.campos[2]) * nw2;
        if (facing > 0.0f) {
            nw0 = -nw0;
            nw1 = -nw1;
            nw2 = -nw2;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) P.n[r] = vm[4 * r] * nw0 + vm[4 * r + 1] * nw1 + vm[4 * r + 2] * nw2;
        // RaDe-GS intersection depth: in the EWA ray space (u, v, z) the Gaussian's densest
        // point along the pixel's ray is the mean of z given (u, v), affine in the pixel:
        //   z(p) = z + Sigma_{z,uv} (Sigma2D + 0.3 I)^-1 (p - mu2D),
        // Sigma_{z,uv} = (V2 . N0, V2 . N1) with V2 the camera-z row of W R S (the same
        // clamped Jacobian as Sigma2D), and (Sigma2D + 0.3 I)^-1 the conic.
        const float szu = F(V[6], N[0], F(V[7], N[1], M(V[8], N[2])));
        const float szv = F(V[6], N[3], F(V[7], N[4], M(V[8], N[5])));
        P.pl[0] = F(szu, P.ca, M(szv, P.cb));
        P.pl[1] = F(szu, P.cb, M(szv, P.cc));
    }
}


// Real SH basis value k (l-major, m = -l..l, Condon-Shortley phase) at unit (x, y, z).
template <int K>
__device__ __forceinline__ float sh_basis(float x, float y, float z)
{
    constexpr float c0 = 0.28209479177387814f;   // sqrt(1/(4 pi))
    constexpr float c1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
    constexpr float c2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
    constexpr float c2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
    constexpr float c2c = 0.54627421529603959f;  // sqrt(15/(16 pi))
    constexpr float c3a = 0.59004358992664352f;  // sqrt(35/(32 pi))
    constexpr float c3b = 2.8906114426405538f;   // sqrt(105/(4 pi))
    constexpr float c3c = 0.45704579946446572f;  // sqrt(21/(32 pi))
    constexpr float c3d = 0.37317633259011540f;  // sqrt(7/(16 pi))
    constexpr float c3e = 1.4453057213202769f;   // sqrt(105/(16 pi))
    if (K == 0) return c0;
    if (K == 1) return -c1 * y;
    if (K == 2) return c1 * z;
    if (K == 3) return -c1 * x;
    if (K == 4) return c2a * x * y;
    if (K == 5) return -c2a * y * z;
    if (K == 6) return c2b * (2.f * z * z - x * x - y * y);
    if (K == 7) return -c2a * x * z;
    if (K == 8) return c2c * (x * x - y * y);
    if (K == 9) return -c3a * y * (3.f * x * x - y * y);
    if (K == 10) return c3b * x * y * z;
    if (K == 11) return -c3c * y * (4.f * z * z - x * x - y * y);
    if (K == 12) return c3d * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
    if (K == 13) return -c3c * x * (4.f * z * z - x * x - y * y);
    if (K == 14) return c3e * z * (x * x - y * y);
    return -c3a * x * (x * x - 3.f * y * y);
}

template <int K, int NK>
struct ShAccum {
    __device__ __forceinline__ static void run(const float *__restrict__ sh, int64_t n_pad, int64_t i, float x,
                                               float y, float z, float (&col)[3])
    {
        const float yk = sh_basis<K>(x, y, z);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(yk, __ldg(sh + (int64_t)(K * 3 + ch) * n_pad + i), col[ch]);
        ShAccum<K + 1, NK>::run(sh, n_pad, i, x, y, z, col);
    }
};
template <int NK>
struct ShAccum<NK, NK> {
    __device__ __forceinline__ static void run(const float *, int64_t, int64_t, float, float, float, float (&)[3]) {}
};

// Colour of the visible Gaussians (one thread each, so a warp reads 128
// contiguous bytes of every SH plane): direction from the camera centre, the
// SH sum, +0.5, clamped at 0, into the colour fields of the record k_project
// wrote. Kept apart from the projection so that this stream of SH bytes, the
// bulk of the step's traffic at degree 3, runs with few registers and many
// warps in flight (measured faster than 4 Gaussians per thread with 16-byte
// loads).
template <int DEG>
__global__ void __launch_bounds__(256) k_colour(ProjectArgs a)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= a.n || a.ntiles[i] == 0) return;
    const int64_t np = a.n_pad;
    const float ex = __ldg(a.means + i) - a.cam.campos[0];
    const float ey = __ldg(a.means + np + i) - a.cam.campos[1];
    const float ez = __ldg(a.means + 2 * np + i) - a.cam.campos[2];
    const float rn = rsqrtf(ex * ex + ey * ey + ez * ez);
    float col[3] = {0.0f, 0.0f, 0.0f};
    ShAccum<0, NK>::run(a.sh, np, i, ex * rn, ey * rn, ez * rn, col);
    float *r = reinterpret_cast<float *>(a.rec + i);
    r[7] = fmaxf(col[0] + 0.5f, 0.0f);  // r1.w
    r[8] = fmaxf(col[1] + 0.5f, 0.0f);  // r2.x
    r[9] = fmaxf(col[2] + 0.5f, 0.0f);  // r2.y
}

// Two Gaussians per thread, 512 apart (each warp reads 128 contiguous bytes of every plane),
// kProjPerBlock (1,024) per block -- the unit of the per-block tile and visibility sums the
// scan reads. Both Gaussians' parameters are loaded before either is projected, so the
// second one's loads are in flight during the first one's arithmetic; two 512-thread blocks
// share an SM. (One Gaussian per thread in 1,024-thread blocks, one block per SM at 54
// registers, stalled on those loads; four Gaussians per thread with 16-byte loads needed
// 80 registers and left the SMs at ~36 % warp occupancy.)
constexpr int kGeomPer = 2;
constexpr int kGeomThreads = kProjPerBlock / kGeomPer;

struct GaussIn {
    float mx, my, mz, ls0, ls1, ls2, qw, qx, qy, qz, logit;
};

template <bool NRM>
__device__ __forceinline__ void project_store(const ProjectArgs &a, int64_t i, const GaussIn &g, uint32_t &tiles,
                                              uint32_t &vis)
{
    const int64_t n4 = (a.n + 3) & ~(int64_t)3;  // ntiles is read 4 at a time: its padding is written 0
    tiles = vis = 0u;
    if (i >= n4) return;
    Proj Q;
    Q.vis = false;
    Q.nt = 0;
    if (i < a.n)
        project_one<NRM>(a.cam, g.mx, g.my, g.mz, g.ls0, g.ls1, g.ls2, g.qw, g.qx, g.qy, g.qz, g.logit, Q);
    if (Q.vis) {  // colour left 0 for k_colour
        GaussRec r;
        r.r0 = make_float4(Q.u, Q.v, Q.ca, Q.cb);
        r.r1 = make_float4(Q.cc, Q.o, Q.z, 0.0f);
        r.r2 = make_float4(0.0f, 0.0f, __uint_as_float(Q.rlo), __uint_as_float(Q.rhi));
        a.rec[i] = r;
        a.bin[i] = make_uint4(__float_as_uint(Q.z), Q.rlo, Q.rhi, 0u);
        if (NRM) {
            a.nrm[i] = make_float4(Q.n[0], Q.n[1], Q.n[2], 0.0f);
            a.plane[i] = make_float2(Q.pl[0], Q.pl[1]);
        }
    }
    a.ntiles[i] = Q.nt;
    tiles = Q.nt;
    vis = Q.vis ? 1u : 0u;
}

template <bool NRM>
__global__ void __launch_bounds__(kGeomThreads, 2) k_project(ProjectArgs a)
{
    const int64_t i0 = (int64_t)blockIdx.x * kProjPerBlock + threadIdx.x;
    const int64_t np = a.n_pad;
    GaussIn g[kGeomPer];
#pragma unroll
    for (int k = 0; k < kGeomPer; ++k) {
        const int64_t i = i0 + (int64_t)k * kGeomThreads;
        const bool in = i < a.n;
        auto ld = [&](const float *base, int row) { return in ? __ldg(base + (int64_t)row * np + i) : 0.0f; };
        g[k] = GaussIn{ld(a.means, 0),  ld(a.means, 1), ld(a.means, 2), ld(a.log_scales, 0), ld(a.log_scales, 1),
                       ld(a.log_scales, 2), ld(a.quats, 0), ld(a.quats, 1), ld(a.quats, 2), ld(a.quats, 3),
                       ld(a.logits, 0)};
    }
    uint32_t my_tiles = 0, my_vis = 0;
#pragma unroll
    for (int k = 0; k < kGeomPer; ++k) {
        uint32_t t, v;
        project_store<NRM>(a, i0 + (int64_t)k * kGeomThreads, g[k], t, v);
        my_tiles += t;
        my_vis += v;
    }
    // block sum of tiles touched -> per-block sums for the instance-offset scan
    __shared__ uint32_t s_warp[2][kGeomThreads / 32];
    uint32_t v = my_tiles, c = my_vis;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_warp[0][threadIdx.x >> 5] = v;
        s_warp[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0, cv = 0;
#pragma unroll
        for (int w = 0; w < kGeomThreads / 32; ++w) {
            t += s_warp[0][w];
            cv += s_warp[1][w];
        }
        a.block_sums[blockIdx.x] = t;
        if (a.block_vis) a.block_vis[blockIdx.x] = cv;
        if (cv) {
            atomicAdd(&a.counters[kCntVisible], cv);
            atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + kCntSumV), (unsigned long long)cv);
        }
    }
}

}  // namespace

int project_blocks(int64_t n) { return (int)((n + kProjPerBlock - 1) / kProjPerBlock); }

// The entries of the two kernels that take the camera, to find their nodes
// in a captured graph: 0 = projection, 1 = colour.
const void *project_kernel_ptr(int deg, int which)
{
    if (which == 1) {
        switch (deg) {
        case 0: return reinterpret_cast<const void *>(k_colour<0>);
        case 1: return reinterpret_cast<const void *>(k_colour<1>);
        case 2: return reinterpret_cast<const void *>(k_colour<2>);
        default: return reinterpret_cast<const void *>(k_colour<3>);
        }
    }
    return reinterpret_cast<const void *>(k_project<false>);
}

cudaError_t launch_project_geometry(const ProjectArgs &a, cudaStream_t s)
{
    const int nb = project_blocks(a.n);
    if (nb == 0) return cudaSuccess;
    if (a.nrm)
        k_project<true><<<nb, kGeomThreads, 0, s>>>(a);
    else
        k_project<false><<<nb, kGeomThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_colour(const ProjectArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const unsigned nc = (unsigned)((a.n + 255) / 256);
    switch (a.deg) {
    case 0: k_colour<0><<<nc, 256, 0, s>>>(a); break;
    case 1: k_colour<1><<<nc, 256, 0, s>>>(a); break;
    case 2: k_colour<2><<<nc, 256, 0, s>>>(a); break;
    default: k_colour<3><<<nc, 256, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_project(const ProjectArgs &a, cudaStream_t s)
{
    cudaError_t e = launch_project_geometry(a, s);
    return e != cudaSuccess ? e : launch_colour(a, s);
}

}  // namespace gsr
