// Backward of the render: K7 walks each pixel's blended Gaussians in reverse
// and forms the per-Gaussian adjoints of the 2D quantities; K8 chains them to
// the 3D parameters. Together they are the exact reverse mode of Eq. 1-4
// (Sec. 3), including the image-gradient channels dI/dx, dI/dy, whose
// adjoints need the second-order terms through a_x = -a (conic d)_x.
//
// K7 state recovery, per pixel, from the forward's final T, T_x, T_y and the
// number of list entries walked: going back over a blended Gaussian,
//   T_i = T_{i+1} / (1 - a_i)
//   r_i = r_{i+1} + a_x,i / (1 - a_i),    r = T_x / T = d(log T)/dx
// and T_x,i = T_i r_i (same in y). Eq. 4 is equivalent to r_{i+1} = r_i -
// a_x,i / (1 - a_i): the reverse recursion is additive and does not amplify
// rounding the way undoing Eq. 4 directly (dividing T_x by 1 - a) would.
//
// Adjoints kept while walking back: Tb = dL/dT, Txb = dL/dT_x, Tyb = dL/dT_y
// of the state after the Gaussian. Per blended Gaussian (colour c, depth z):
//   dL/dc   += g_rgb a T + g_dx (T_x a + T a_x) + g_dy (T_y a + T a_y)
//   dL/dz   += g_d a T
//   dL/da    = G_c T + G_x T_x + G_y T_y + g_d z T - Tb T - Txb T_x - Tyb T_y
//   dL/da_x  = (G_x - Txb) T,   dL/da_y = (G_y - Tyb) T
//   Tb'  = G_c a + G_x a_x + G_y a_y + g_d z a + Tb (1 - a) - Txb a_x - Tyb a_y
//   Txb' = G_x a + Txb (1 - a),  Tyb' = G_y a + Tyb (1 - a)
// with G_c = <g_rgb, c>, G_x = <g_dx, c>, G_y = <g_dy, c>. Through a = o exp(-Q/2)
// and a_x = -a e_x, a_y = -a e_y (e = conic d), unless a was capped at 0.99.
// The 10 adjoints (u, v, conic a/b/c, opacity, depth, rgb) of a Gaussian are
// summed over the warp's pixels by a reduce-scatter; ten lanes add the totals
// atomically.
#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kBwdBatch = 64;

// Sums 10 per-lane values over the warp with 16 shuffles instead of 50: at each step
// (offsets 16, 8, 4, 2) a lane keeps half of its values, sends the other half to its
// partner and adds the partner's copy of the half it kept; a last butterfly step
// (offset 1) completes the sum. Returns, in v[0], the warp total of value
// ((lane>>4)&1)*8 + ((lane>>3)&1)*4 + ((lane>>2)&1)*2 + ((lane>>1)&1) (values 10..15
// are zeros), and that index.
__device__ __forceinline__ int warp_reduce_scatter10(float (&v)[10], int lane)
{
    float w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = i < 10 ? v[i] : 0.0f;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {  // offset 2h: keep w[0, h) or w[h, 2h)
        const bool hi = (lane & (2 * h)) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = hi ? w[i] : w[h + i];
            const float keep = hi ? w[h + i] : w[i];
            w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    v[0] = w[0] + __shfl_xor_sync(0xffffffffu, w[0], 1);
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// K7: one warp per CTA, walking 32 pixels of a tile (32 / TILE rows, or part of a
// row). The warps of a tile stage their own copies of its records (L2 hits after
// the first) and each walks back only from its own pixels' last blended entry,
// with no barrier between them.
template <int TILE>
__global__ void __launch_bounds__(32) k_composite_bwd(const BackwardArgs a)
{
    constexpr int WPT = TILE * TILE / 32;  // warps per tile
    __shared__ GaussRec s_rec[kBwdBatch];
    __shared__ uint32_t s_idx[kBwdBatch];
    const int lane = threadIdx.x;
    const int tx = blockIdx.x / WPT, l = (blockIdx.x % WPT) * 32 + lane;
    const int px = tx * TILE + l % TILE, py = blockIdx.y * TILE + l / TILE;
    const bool inside = px < a.width && py < a.height;
    const uint2 range = a.ranges[blockIdx.y * a.tiles_x + tx];
    const int64_t HW = (int64_t)a.width * a.height;
    const int64_t p = (int64_t)py * a.width + px;

    float T = 1.0f, rx = 0.0f, ry = 0.0f, Tb = 0.0f, Txb = 0.0f, Tyb = 0.0f;
    float gr[3] = {0, 0, 0}, gx[3] = {0, 0, 0}, gy[3] = {0, 0, 0}, gd = 0.0f;
    uint32_t last = 0;
    if (inside) {
        T = a.final_T[p];
        rx = a.final_Tx[p] / T;
        ry = a.final_Ty[p] / T;
        last = a.n_contrib[p];
        // never past the tile's list (a frame whose waits gave up leaves n_contrib unspecified)
        last = min(last, range.y > range.x ? range.y - range.x : 0u);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (a.g_rgb) gr[c] = a.g_rgb[c * HW + p];
            if (a.g_dcdx) gx[c] = a.g_dcdx[c * HW + p];
            if (a.g_dcdy) gy[c] = a.g_dcdy[c * HW + p];
            Tb += gr[c] * a.bg[c];
            Txb += gx[c] * a.bg[c];
            Tyb += gy[c] * a.bg[c];
        }
        if (a.g_depth) gd = a.g_depth[p];
        if (a.g_alpha) Tb -= a.g_alpha[p];
    }
    const uint32_t n_walk = __reduce_max_sync(0xffffffffu, last);
    const float pxb = block_px(px), pyb = block_py(py);
    const int bx0 = px & ~7, by0 = py & ~3;  // the pixel's 8x4 block, as in the forward

    for (int64_t end = (int64_t)n_walk; end > 0; end -= kBwdBatch) {
        const int64_t beg = end - kBwdBatch > 0 ? end - kBwdBatch : 0;
        const int cnt = (int)(end - beg);
        __syncwarp();
        for (int t = lane; t < cnt; t += 32) {  // the tile's records, gathered by index like the forward's
            const uint32_t idx = a.vals[range.x + beg + t];
            s_idx[t] = idx;
            GaussRec r = a.rec[idx < a.n ? idx : 0u];
            if (idx >= a.n) r.r2.z = r.r2.w = __uint_as_float(0xFFFFFFFFu);  // no pixel: never blended
            s_rec[t] = r;
        }
        __syncwarp();
        for (int k = cnt - 1; k >= 0; --k) {
            const uint32_t pos = (uint32_t)(beg + k);
            float g10[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            bool contrib = false;
            if (pos < last) {
                const float4 r0 = s_rec[k].r0, r1 = s_rec[k].r1, r2 = s_rec[k].r2;
                if (rect_contains(r2, (uint32_t)px, (uint32_t)py)) {
                    const float2 cb = block_centre(r0, r2, bx0, by0);  // the forward's exact arithmetic
                    const AlphaEval e = eval_alpha(make_float4(cb.x, cb.y, r0.z, r0.w), r1, pxb, pyb);
                    if (e.al >= kAlphaMin) {
                        contrib = true;
                        const float al = e.al, om = 1.0f - al;
                        const float ax = e.capped ? 0.0f : -al * e.ex;
                        const float ay = e.capped ? 0.0f : -al * e.ey;
                        const float inv = __frcp_rn(om);  // one reciprocal for the three quotients
                        const float Ti = T * inv;
                        const float rxi = rx + ax * inv, ryi = ry + ay * inv;
                        const float Txi = Ti * rxi, Tyi = Ti * ryi;
                        const float col[3] = {r1.w, r2.x, r2.y};
                        float Gc = 0.f, Gx = 0.f, Gy = 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            g10[7 + c] = gr[c] * al * Ti + gx[c] * (Txi * al + Ti * ax) + gy[c] * (Tyi * al + Ti * ay);
                            Gc += gr[c] * col[c];
                            Gx += gx[c] * col[c];
                            Gy += gy[c] * col[c];
                        }
                        const float z = r1.z;
                        g10[6] = gd * al * Ti;
                        const float dA = Gc * Ti + Gx * Txi + Gy * Tyi + gd * z * Ti - Tb * Ti - Txb * Txi - Tyb * Tyi;
                        const float dAx = (Gx - Txb) * Ti;
                        const float dAy = (Gy - Tyb) * Ti;
                        const float nTb = Gc * al + Gx * ax + Gy * ay + gd * z * al + Tb * om - Txb * ax - Tyb * ay;
                        const float nTxb = Gx * al + Txb * om;
                        const float nTyb = Gy * al + Tyb * om;
                        if (!e.capped) {
                            const float dx = e.dx, dy = e.dy, ex = e.ex, ey = e.ey;
                            const float Abar = dA - dAx * ex - dAy * ey;
                            g10[5] = Abar * e.g;  // d a / d o = a / o
                            const float gQ = -0.5f * al * Abar;
                            const float gex = -al * dAx, gey = -al * dAy;
                            g10[2] = gQ * dx * dx + gex * dx;
                            g10[3] = 2.0f * gQ * dx * dy + gex * dy + gey * dx;
                            g10[4] = gQ * dy * dy + gey * dy;
                            g10[0] = -(2.0f * gQ * ex + gex * r0.z + gey * r0.w);
                            g10[1] = -(2.0f * gQ * ey + gex * r0.w + gey * r1.x);
                        }
                        T = Ti;
                        rx = rxi;
                        ry = ryi;
                        Tb = nTb;
                        Txb = nTxb;
                        Tyb = nTyb;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                // warp sums of the 10 adjoints by reduce-scatter: lane l ends with the
                // total of value ((l>>4)&1)*8 + ((l>>3)&1)*4 + ((l>>2)&1)*2 + ((l>>1)&1),
                // so up to 10 lanes add their totals in one atomic instruction
                const int j = warp_reduce_scatter10(g10, lane);
                if ((lane & 1) == 0 && j < 10 && g10[0] != 0.0f)
                    atomicAdd(a.g2d + (size_t)s_idx[k] * 10 + j, g10[0]);
            }
        }
    }
}

// d/d(dir) of the real SH basis (Condon-Shortley phase), k < (deg+1)^2.
__device__ __forceinline__ void sh_eval_grad(int deg, float x, float y, float z, float *Y, float *gX, float *gY, float *gZ)
{
    const float c0 = 0.28209479177387814f, c1 = 0.48860251190291992f;
    const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.54627421529603959f;
    const float c3a = 0.59004358992664352f, c3b = 2.8906114426405538f, c3c = 0.45704579946446572f;
    const float c3d = 0.37317633259011540f, c3e = 1.4453057213202769f;
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = gX[k] = gY[k] = gZ[k] = 0.0f;
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = -c1 * y; gY[1] = -c1;
    Y[2] = c1 * z;  gZ[2] = c1;
    Y[3] = -c1 * x; gX[3] = -c1;
    if (deg < 2) return;
    Y[4] = c2a * x * y;  gX[4] = c2a * y; gY[4] = c2a * x;
    Y[5] = -c2a * y * z; gY[5] = -c2a * z; gZ[5] = -c2a * y;
    Y[6] = c2b * (2.f * z * z - x * x - y * y); gX[6] = -2.f * c2b * x; gY[6] = -2.f * c2b * y; gZ[6] = 4.f * c2b * z;
    Y[7] = -c2a * x * z; gX[7] = -c2a * z; gZ[7] = -c2a * x;
    Y[8] = c2c * (x * x - y * y); gX[8] = 2.f * c2c * x; gY[8] = -2.f * c2c * y;
    if (deg < 3) return;
    Y[9] = -c3a * y * (3.f * x * x - y * y);
    gX[9] = -6.f * c3a * x * y; gY[9] = -c3a * (3.f * x * x - 3.f * y * y);
    Y[10] = c3b * x * y * z;
    gX[10] = c3b * y * z; gY[10] = c3b * x * z; gZ[10] = c3b * x * y;
    Y[11] = -c3c * y * (4.f * z * z - x * x - y * y);
    gX[11] = 2.f * c3c * x * y; gY[11] = -c3c * (4.f * z * z - x * x - 3.f * y * y); gZ[11] = -8.f * c3c * y * z;
    Y[12] = c3d * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
    gX[12] = -6.f * c3d * x * z; gY[12] = -6.f * c3d * y * z; gZ[12] = c3d * (6.f * z * z - 3.f * x * x - 3.f * y * y);
    Y[13] = -c3c * x * (4.f * z * z - x * x - y * y);
    gX[13] = -c3c * (4.f * z * z - 3.f * x * x - y * y); gY[13] = 2.f * c3c * x * y; gZ[13] = -8.f * c3c * x * z;
    Y[14] = c3e * z * (x * x - y * y);
    gX[14] = 2.f * c3e * x * z; gY[14] = -2.f * c3e * y * z; gZ[14] = c3e * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.f * y * y);
    gX[15] = -c3a * (3.f * x * x - 3.f * y * y); gY[15] = 6.f * c3a * x * y;
}

// K8: one thread per Gaussian; recompute the forward quantities and chain the
// (u, v, conic, opacity, depth) adjoints to the 3D parameters. The colour's
// adjoint goes through SH in k_colour_bwd, launched after it.
__global__ void __launch_bounds__(256, 3) k_project_bwd(const ProjectBwdArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n || a.ntiles[i] == 0) return;
    const int64_t S = a.n_pad;
    // the gradients this thread adds to, read up front so that their loads overlap
    // the arithmetic (the colour kernel adds to d_means only after this one)
    float acc_ls[3] = {0.f, 0.f, 0.f}, acc_q[4] = {0.f, 0.f, 0.f, 0.f}, acc_lg = 0.f, acc_m[3] = {0.f, 0.f, 0.f};
    if (a.d_log_scales)
        for (int k = 0; k < 3; ++k) acc_ls[k] = a.d_log_scales[k * S + i];
    if (a.d_quats)
        for (int k = 0; k < 4; ++k) acc_q[k] = a.d_quats[k * S + i];
    if (a.d_logits) acc_lg = a.d_logits[i];
    if (a.d_means)
        for (int k = 0; k < 3; ++k) acc_m[k] = a.d_means[k * S + i];
    const float *g2 = a.g2d + 10 * i;
    float gu = g2[0], gv = g2[1], gca = g2[2], gcb = g2[3], gcc = g2[4], go = g2[5], gz = g2[6];
    const CamParams &c = a.cam;
    const float *W = c.vm;
    const float m[3] = {a.means[i], a.means[S + i], a.means[2 * S + i]};
    float s[3];
    for (int k = 0; k < 3; ++k) s[k] = __expf(a.log_scales[k * S + i]);
    const float q0 = a.quats[i], q1 = a.quats[S + i], q2 = a.quats[2 * S + i], q3 = a.quats[3 * S + i];
    const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 / qn, x = q1 / qn, y = q2 / qn, z = q3 / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float Mx[9], Sig[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Mx[3 * r + k] = R[3 * r + k] * s[k];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Sig[3 * r + k] = Mx[3 * r] * Mx[3 * k] + Mx[3 * r + 1] * Mx[3 * k + 1] + Mx[3 * r + 2] * Mx[3 * k + 2];
    float t[3];
    for (int r = 0; r < 3; ++r) t[r] = W[4 * r] * m[0] + W[4 * r + 1] * m[1] + W[4 * r + 2] * m[2] + W[4 * r + 3];
    const float tx = t[0], ty = t[1], tz = t[2];
    const float limx = 1.3f * (0.5f * c.width / c.fx), limy = 1.3f * (0.5f * c.height / c.fy);
    const float txtz = tx / tz, tytz = ty / tz;
    const bool clx = txtz > limx || txtz < -limx, cly = tytz > limy || tytz < -limy;
    const float cxs = fminf(limx, fmaxf(-limx, txtz)), cys = fminf(limy, fmaxf(-limy, tytz));
    const float J[6] = {c.fx / tz, 0.f, -c.fx * cxs / tz, 0.f, c.fy / tz, -c.fy * cys / tz};
    float T3[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) T3[3 * r + k] = J[3 * r] * W[k] + J[3 * r + 1] * W[4 + k] + J[3 * r + 2] * W[8 + k];
    // conic K = inverse(Sigma2D): recompute Sigma2D to get K exactly as the forward did (up to rounding)
    float S2[4];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) {
            float acc = 0.f;
            for (int aa = 0; aa < 3; ++aa)
                for (int bb = 0; bb < 3; ++bb) acc += T3[3 * r + aa] * Sig[3 * aa + bb] * T3[3 * q + bb];
            S2[2 * r + q] = acc;
        }
    const float A2 = S2[0] + 0.3f, B2 = 0.5f * (S2[1] + S2[2]), C2 = S2[3] + 0.3f;
    const float det = A2 * C2 - B2 * B2;
    const float K[4] = {C2 / det, -B2 / det, -B2 / det, A2 / det};
    float tb[3] = {0.f, 0.f, 0.f}, mb[3] = {0.f, 0.f, 0.f};
    const float o = 1.0f / (1.0f + __expf(-a.logits[i]));
    // opacity
    const float d_logit = go * o * (1.0f - o);
    // centre and depth
    tb[0] += gu * c.fx / tz;
    tb[1] += gv * c.fy / tz;
    tb[2] += -gu * c.fx * tx / (tz * tz) - gv * c.fy * ty / (tz * tz) + gz;
    // Sbar = -K Gbar K, Gbar = [[ga, gb/2], [gb/2, gc]]
    const float Gb[4] = {gca, 0.5f * gcb, 0.5f * gcb, gcc};
    float KG[4], Sb[4];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) KG[2 * r + q] = K[2 * r] * Gb[q] + K[2 * r + 1] * Gb[2 + q];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) Sb[2 * r + q] = -(KG[2 * r] * K[q] + KG[2 * r + 1] * K[2 + q]);
    // Sigmabar = T3^T Sb T3;  T3bar = 2 Sb T3 Sigma
    float Sigb[9], T3b[6];
    for (int aa = 0; aa < 3; ++aa)
        for (int bb = 0; bb < 3; ++bb) {
            float acc = 0.f;
            for (int r = 0; r < 2; ++r)
                for (int q = 0; q < 2; ++q) acc += T3[3 * r + aa] * Sb[2 * r + q] * T3[3 * q + bb];
            Sigb[3 * aa + bb] = acc;
        }
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            float acc = 0.f;
            for (int q = 0; q < 2; ++q)
                for (int j = 0; j < 3; ++j) acc += Sb[2 * r + q] * T3[3 * q + j] * Sig[3 * j + k];
            T3b[3 * r + k] = 2.f * acc;
        }
    float Jb[6];
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) Jb[3 * r + j] = T3b[3 * r] * W[4 * j] + T3b[3 * r + 1] * W[4 * j + 1] + T3b[3 * r + 2] * W[4 * j + 2];
    const float tz2 = tz * tz;
    tb[2] += Jb[0] * (-c.fx / tz2) + Jb[4] * (-c.fy / tz2);
    if (!clx) {
        tb[0] += Jb[2] * (-c.fx / tz2);
        tb[2] += Jb[2] * (2.f * c.fx * tx / (tz2 * tz));
    } else {
        tb[2] += Jb[2] * (c.fx * cxs / tz2);
    }
    if (!cly) {
        tb[1] += Jb[5] * (-c.fy / tz2);
        tb[2] += Jb[5] * (2.f * c.fy * ty / (tz2 * tz));
    } else {
        tb[2] += Jb[5] * (c.fy * cys / tz2);
    }
    for (int k = 0; k < 3; ++k) mb[k] += W[k] * tb[0] + W[4 + k] * tb[1] + W[8 + k] * tb[2];
    // Sigma = M M^T: Mbar = (Sigmabar + Sigmabar^T) M
    float Rb[9], sb[3] = {0.f, 0.f, 0.f};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            float acc = 0.f;
            for (int k = 0; k < 3; ++k) acc += (Sigb[3 * r + k] + Sigb[3 * k + r]) * Mx[3 * k + q];
            sb[q] += acc * R[3 * r + q];
            Rb[3 * r + q] = acc * s[q];
        }
    if (a.d_log_scales)
        for (int k = 0; k < 3; ++k) a.d_log_scales[k * S + i] = acc_ls[k] + sb[k] * s[k];
    float qb[4];
    qb[0] = 2.f * (-z * Rb[1] + y * Rb[2] + z * Rb[3] - x * Rb[5] - y * Rb[6] + x * Rb[7]);
    qb[1] = 2.f * (y * Rb[1] + z * Rb[2] + y * Rb[3] - 2.f * x * Rb[4] - w * Rb[5] + z * Rb[6] + w * Rb[7] - 2.f * x * Rb[8]);
    qb[2] = 2.f * (-2.f * y * Rb[0] + x * Rb[1] + w * Rb[2] + x * Rb[3] + z * Rb[5] - w * Rb[6] + z * Rb[7] - 2.f * y * Rb[8]);
    qb[3] = 2.f * (-2.f * z * Rb[0] - w * Rb[1] + x * Rb[2] + w * Rb[3] - 2.f * z * Rb[4] + y * Rb[5] + x * Rb[6] + y * Rb[7]);
    const float qh[4] = {w, x, y, z};
    const float dot = w * qb[0] + x * qb[1] + y * qb[2] + z * qb[3];
    if (a.d_quats)
        for (int k = 0; k < 4; ++k) a.d_quats[k * S + i] = acc_q[k] + (qb[k] - qh[k] * dot) / qn;
    if (a.d_logits) a.d_logits[i] = acc_lg + d_logit;
    if (a.d_means)
        for (int k = 0; k < 3; ++k) a.d_means[k * S + i] = acc_m[k] + mb[k];
}

// K8, colour part: the rgb adjoint through SH and the view direction, one thread
// per Gaussian, added to the SH coefficients' and the mean's gradients. Like the
// forward's colour kernel it streams the SH planes with few registers: one pass
// forms the raw colour (whose sign says whether the clamp at 0 let the gradient
// through) and reads d_sh, a second re-reads the coefficients (L2-resident by
// then) to update d_sh and the direction's adjoint. The SH degree is a template argument, so the
// basis and its gradient are registers.
template <int DEG>
__global__ void __launch_bounds__(256, 2) k_colour_bwd(const ProjectBwdArgs a)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n || a.ntiles[i] == 0) return;
    const int64_t S = a.n_pad;
    const float *__restrict__ sh = a.sh + i;
    float *__restrict__ dsh = a.d_sh ? a.d_sh + i : nullptr;
    const float *g2 = a.g2d + 10 * i;
    const float grgb[3] = {g2[7], g2[8], g2[9]};
    const CamParams &c = a.cam;
    const float m[3] = {__ldg(a.means + i), __ldg(a.means + S + i), __ldg(a.means + 2 * S + i)};
    const float dir[3] = {m[0] - c.campos[0], m[1] - c.campos[1], m[2] - c.campos[2]};
    const float dn = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    const float d[3] = {dir[0] / dn, dir[1] / dn, dir[2] / dn};
    float Y[16], gX[16], gY[16], gZ[16];
    sh_eval_grad(DEG, d[0], d[1], d[2], Y, gX, gY, gZ);
    // the gradient planes are read in the first pass too, so that one wait covers
    // both streams
    float raw[3] = {0.5f, 0.5f, 0.5f}, acc[NK * 3];
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            raw[ch] += Y[k] * __ldg(sh + (int64_t)(k * 3 + ch) * S);
            acc[k * 3 + ch] = dsh ? dsh[(int64_t)(k * 3 + ch) * S] : 0.0f;
        }
    float db[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (raw[ch] < 0.0f) continue;  // the colour was clamped to 0: no gradient
            const float gc = grgb[ch], shv = __ldg(sh + (int64_t)(k * 3 + ch) * S);
            if (dsh) dsh[(int64_t)(k * 3 + ch) * S] = acc[k * 3 + ch] + gc * Y[k];
            db[0] += gc * shv * gX[k];
            db[1] += gc * shv * gY[k];
            db[2] += gc * shv * gZ[k];
        }
    const float dd = db[0] * d[0] + db[1] * d[1] + db[2] * d[2];
    if (a.d_means)
#pragma unroll
        for (int k = 0; k < 3; ++k) a.d_means[k * S + i] += (db[k] - d[k] * dd) / dn;
}

}  // namespace

cudaError_t launch_composite_backward(const BackwardArgs &a, cudaStream_t s)
{
    if (a.tiles_x == 0 || a.tiles_y == 0) return cudaSuccess;
    const unsigned wpt = (unsigned)(a.tile * a.tile / 32);  // one warp-sized CTA per 32 pixels of a tile
    const dim3 grid((unsigned)a.tiles_x * wpt, (unsigned)a.tiles_y);
    switch (a.tile) {
    case 8: k_composite_bwd<8><<<grid, 32, 0, s>>>(a); break;
    case 32: k_composite_bwd<32><<<grid, 32, 0, s>>>(a); break;
    default: k_composite_bwd<16><<<grid, 32, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_project_backward(const ProjectBwdArgs &a, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    const int64_t nb = (a.n + 255) / 256;
    k_project_bwd<<<(unsigned)nb, 256, 0, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nc = (a.n + 255) / 256;
    switch (a.deg) {
    case 0: k_colour_bwd<0><<<(unsigned)nc, 256, 0, s>>>(a); break;
    case 1: k_colour_bwd<1><<<(unsigned)nc, 256, 0, s>>>(a); break;
    case 2: k_colour_bwd<2><<<(unsigned)nc, 256, 0, s>>>(a); break;
    default: k_colour_bwd<3><<<(unsigned)nc, 256, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace gsr
