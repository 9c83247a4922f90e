/*
 * oracle.c -- plain, slow CPU reference of the 3DGS^3 low-resolution render.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file; only the tests, the package smoke check and the bench's CPU
 * baseline do. It shares no code with the CUDA path.
 *
 * What it computes (the paper's preliminaries, Sec. 3):
 *   - Gaussian primitive G(x) = exp(-1/2 (x - xc)^T Sigma^-1 (x - xc))      (Eq. 1)
 *   - Sigma = R S S^T R^T, R from a unit quaternion, S = diag(scale)      (Sec. 3)
 *   - EWA splatting: local affine (Jacobian) projection of Sigma to 2D     (Sec. 3)
 *     plus a 0.3 px^2 low-pass on both diagonal entries
 *   - depth sort, then front-to-back alpha blending I = sum c_i a_i T_i   (Eq. 2)
 *     with a_i = opacity * G (capped at 0.99), c_i from SH coefficients
 *   - the analytic image gradients dI/dx, dI/dy                           (Eq. 3)
 *     with the transmittance-gradient recursion                           (Eq. 4)
 *   - depth = sum z_i a_i T_i and alpha = 1 - T_final
 *   - the RaDe-GS channels the paper renders depth and normals with (Sec. 5.1):
 *     normals (shortest axis) and the ray-Gaussian intersection depth, the
 *     conditional mean of camera z given the pixel in the EWA ray space
 *     (cont_project, or_cont.rd)
 *   - the reverse-mode adjoint of all of the above (backward)
 *
 * Precision: FP64 for every continuous quantity. The discrete decisions (the
 * depth sort key and the per-Gaussian pixel support rectangle, which also
 * decides culling) follow a fixed fp32 round-to-nearest operation sequence,
 * written out below ("discrete spec"), so that an fp32 GPU implementation can
 * reproduce them bit for bit. Compile with -ffp-contract=off (no implicit FMA).
 *
 * Readings where the paper is silent (3DGS conventions, which the paper builds
 * on): alpha cap 0.99, alpha cut 1/255, stop before a Gaussian that would take T
 * below 1e-4, pixel (i, j) sampled at (i + 0.5, j + 0.5), near plane cull,
 * Jacobian guard clamp of x/z, y/z at 1.3x the half field of view, support
 * rectangle = exact bounding box of the ellipse where o*G >= 1/255, ties in depth
 * broken by input index, real SH with the Condon-Shortley phase (+0.5 offset,
 * clamped at 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;       /* number of Gaussians */
    int64_t stride;  /* row stride of every plane (>= n) */
    int32_t deg;     /* SH degree 0..3 */
    int32_t _pad;
    const double *means;       /* [3][stride] */
    const double *log_scales;  /* [3][stride] */
    const double *quats;       /* [4][stride] w, x, y, z (not normalised) */
    const double *logits;      /* [stride] */
    const double *sh;          /* [(deg+1)^2][3][stride] */
} or_scene;

typedef struct {
    double viewmat[12];  /* world -> camera, row-major 3x4 [R | t] */
    double fx, fy, cx, cy;
    double near_plane;
    int32_t width, height;
    double bg[3];
} or_camera;

#define OR_ALPHA_CAP 0.99
#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_T_MIN 1e-4
#define OR_LOWPASS 0.3

/* ===================================================================== discrete spec
 * fp32 round-to-nearest sequence for the sort key and the support rectangle.
 * Every arithmetic operation below is a single IEEE fp32 operation (the source
 * is compiled without FP contraction); fmaf is the correctly rounded fused
 * multiply-add.
 */

/* Spec exp: Cody-Waite argument reduction (Cody & Waite, "Software Manual for
 * the Elementary Functions", 1980) with ln 2 split as 0.693359375 + ln2_lo, then
 * the degree-7 Taylor polynomial of e^r (|r| <= ln2/2) by Horner with fused
 * multiply-adds, then exact scaling by 2^n. Input clamped to [-87, 88]. */
float or_spec_exp(float x)
{
    if (x != x) return x;
    if (x > 88.0f) x = 88.0f;
    if (x < -87.0f) x = -87.0f;
    float n = rintf(x * 1.44269502e+00f);
    float r = fmaf(-n, 0.693359375f, x);
    r = fmaf(-n, -2.12194442e-04f, r);
    float p = 1.98412701e-04f;          /* 1/7! */
    p = fmaf(p, r, 1.38888892e-03f);    /* 1/6! */
    p = fmaf(p, r, 8.33333377e-03f);    /* 1/5! */
    p = fmaf(p, r, 4.16666679e-02f);    /* 1/4! */
    p = fmaf(p, r, 1.66666672e-01f);    /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int32_t ni = (int32_t)n;
    uint32_t sb = (uint32_t)(ni + 127) << 23;
    float scale;
    memcpy(&scale, &sb, 4);
    return p * scale;
}

/* Spec log for normal x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)],
 * log m = 2 atanh(s), s = (m - 1)/(m + 1), atanh by its odd series to s^11,
 * then e ln 2 added in two parts. */
float or_spec_log(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    int32_t e = (int32_t)((b >> 23) & 0xFFu) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 1.41421354e+00f) {
        m = m * 0.5f;
        e += 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float w = s * s;
    float p = 9.09090936e-02f;          /* 1/11 */
    p = fmaf(p, w, 1.11111112e-01f);    /* 1/9 */
    p = fmaf(p, w, 1.42857149e-01f);    /* 1/7 */
    p = fmaf(p, w, 2.00000003e-01f);    /* 1/5 */
    p = fmaf(p, w, 3.33333343e-01f);    /* 1/3 */
    float t = 2.0f * s;
    float lm = fmaf(t * w, p, t);
    float ef = (float)e;
    return fmaf(ef, 0.693359375f, fmaf(ef, -2.12194442e-04f, lm));
}

typedef struct {
    int32_t visible;
    float z32;
    int32_t rect[4]; /* xmin, ymin, xmax, ymax (inclusive pixel indices) */
} or_disc;

static void disc_project(const or_scene *sc, const or_camera *cam, int64_t i, or_disc *d)
{
    const int64_t S = sc->stride;
    d->visible = 0;
    d->z32 = 0.0f;
    d->rect[0] = d->rect[1] = d->rect[2] = d->rect[3] = 0;
    float vm[12];
    for (int k = 0; k < 12; ++k) vm[k] = (float)cam->viewmat[k];
    const float mx = (float)sc->means[i], my = (float)sc->means[S + i], mz = (float)sc->means[2 * S + i];
    const float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    const float near = (float)cam->near_plane;
    /* D1: camera-space depth, fixed left-to-right order */
    float tz = ((vm[8] * mx + vm[9] * my) + vm[10] * mz) + vm[11];
    if (!(tz > near)) return;
    /* D2 */
    float tx = ((vm[0] * mx + vm[1] * my) + vm[2] * mz) + vm[3];
    float ty = ((vm[4] * mx + vm[5] * my) + vm[6] * mz) + vm[7];
    /* D3: scales */
    float s[3];
    for (int k = 0; k < 3; ++k) s[k] = or_spec_exp((float)sc->log_scales[k * S + i]);
    /* D4: the quaternion's squared norm and f = 2 / |q|^2, so that R(q / |q|) is formed
     * from the unnormalised components with one division */
    float qw = (float)sc->quats[i], qx = (float)sc->quats[S + i], qy = (float)sc->quats[2 * S + i],
          qz = (float)sc->quats[3 * S + i];
    float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    if (!(n2 > 0.0f)) return;
    float f = 2.0f / n2;
    /* D5: rotation matrix R(q / |q|) = I + f [...] */
    float R[9];
    R[0] = 1.0f - f * (qy * qy + qz * qz);
    R[1] = f * (qx * qy - qw * qz);
    R[2] = f * (qx * qz + qw * qy);
    R[3] = f * (qx * qy + qw * qz);
    R[4] = 1.0f - f * (qx * qx + qz * qz);
    R[5] = f * (qy * qz - qw * qx);
    R[6] = f * (qx * qz - qw * qy);
    R[7] = f * (qy * qz + qw * qx);
    R[8] = 1.0f - f * (qx * qx + qy * qy);
    /* D6: M = R diag(s), so Sigma = M M^T */
    float M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * s[c];
    /* D7: V = W M (the camera rotation applied to M's columns) */
    float V[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[3 * r + c] = (vm[4 * r] * M[c] + vm[4 * r + 1] * M[3 + c]) + vm[4 * r + 2] * M[6 + c];
    /* D8: one reciprocal of the depth; x/z, y/z, clamped to the guard for the Jacobian */
    float rz = 1.0f / tz;
    float xz = tx * rz, yz = ty * rz;
    float limx = 1.29999995f * ((0.5f * (float)cam->width) / fx);
    float limy = 1.29999995f * ((0.5f * (float)cam->height) / fy);
    float xc = fminf(limx, fmaxf(-limx, xz)), yc = fminf(limy, fmaxf(-limy, yz));
    /* D9: N = J V with J = [[fx/z, 0, -fx x'/z], [0, fy/z, -fy y'/z]] (x', y' the clamped x/z,
     * y/z), row by row: N0 = (fx/z) (V0 - x' V2), N1 = (fy/z) (V1 - y' V2) */
    float ax = fx * rz, ay = fy * rz;
    float N[6];
    for (int k = 0; k < 3; ++k) {
        N[k] = ax * (V[k] - xc * V[6 + k]);
        N[3 + k] = ay * (V[3 + k] - yc * V[6 + k]);
    }
    /* D10: the diagonal of Sigma2D = N N^T + 0.3 I */
    float A = ((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]) + 3.00000012e-01f;
    float C = ((N[3] * N[3] + N[4] * N[4]) + N[5] * N[5]) + 3.00000012e-01f;
    /* D11: (Sigma2D's determinant is |N0 x N1|^2 + 0.3 (|N0|^2 + |N1|^2) + 0.09 > 0: no cull) */
    /* D13: opacity and the alpha-cut level */
    float o = 1.0f / (1.0f + or_spec_exp(-(float)sc->logits[i]));
    if (!(255.0f * o >= 1.0f)) return;
    float kk = 2.0f * or_spec_log(255.0f * o);
    /* D14: half-extents of the ellipse's bounding box */
    float ex = sqrtf(kk * A), ey = sqrtf(kk * C);
    /* D15: projected centre */
    float u = fx * xz + cx;
    float v = fy * yz + cy;
    /* D16: pixel rectangle */
    float xlo = (u - ex) - 0.5f, xhi = (u + ex) - 0.5f;
    float ylo = (v - ey) - 0.5f, yhi = (v + ey) - 0.5f;
    float wm1 = (float)(cam->width - 1), hm1 = (float)(cam->height - 1);
    if (!(xhi >= 0.0f) || !(xlo <= wm1) || !(yhi >= 0.0f) || !(ylo <= hm1)) return;
    int xmin = (int)fmaxf(0.0f, ceilf(xlo)), xmax = (int)fminf(wm1, floorf(xhi));
    int ymin = (int)fmaxf(0.0f, ceilf(ylo)), ymax = (int)fminf(hm1, floorf(yhi));
    if (xmin > xmax || ymin > ymax) return;
    d->visible = 1;
    d->z32 = tz;
    d->rect[0] = xmin;
    d->rect[1] = ymin;
    d->rect[2] = xmax;
    d->rect[3] = ymax;
}

/* ===================================================================== SH (Sec. 3)
 * Real spherical harmonics with the Condon-Shortley phase, l-major, m = -l..l:
 * Y_lm = sqrt2 Re Y_l^m (m > 0), Y_l^0, sqrt2 Im Y_l^|m| (m < 0), written as
 * homogeneous polynomials of the unit direction (x, y, z). */
#define PI_ 3.14159265358979323846

void or_sh_basis(int deg, const double *d, double *Y, double *dY /* [16][3] or NULL */)
{
    const double x = d[0], y = d[1], z = d[2];
    const double c0 = sqrt(1.0 / (4.0 * PI_));
    const double c1 = sqrt(3.0 / (4.0 * PI_));
    const double c2a = sqrt(15.0 / (4.0 * PI_)), c2b = sqrt(5.0 / (16.0 * PI_)), c2c = sqrt(15.0 / (16.0 * PI_));
    const double c3a = sqrt(35.0 / (32.0 * PI_)), c3b = sqrt(105.0 / (4.0 * PI_)), c3c = sqrt(21.0 / (32.0 * PI_));
    const double c3d = sqrt(7.0 / (16.0 * PI_)), c3e = sqrt(105.0 / (16.0 * PI_));
    double v[16], g[16][3];
    memset(g, 0, sizeof g);
    v[0] = c0;
    v[1] = -c1 * y;             g[1][1] = -c1;
    v[2] = c1 * z;              g[2][2] = c1;
    v[3] = -c1 * x;             g[3][0] = -c1;
    v[4] = c2a * x * y;         g[4][0] = c2a * y; g[4][1] = c2a * x;
    v[5] = -c2a * y * z;        g[5][1] = -c2a * z; g[5][2] = -c2a * y;
    v[6] = c2b * (2 * z * z - x * x - y * y);
    g[6][0] = -2 * c2b * x; g[6][1] = -2 * c2b * y; g[6][2] = 4 * c2b * z;
    v[7] = -c2a * x * z;        g[7][0] = -c2a * z; g[7][2] = -c2a * x;
    v[8] = c2c * (x * x - y * y); g[8][0] = 2 * c2c * x; g[8][1] = -2 * c2c * y;
    v[9] = -c3a * y * (3 * x * x - y * y);
    g[9][0] = -6 * c3a * x * y; g[9][1] = -c3a * (3 * x * x - 3 * y * y);
    v[10] = c3b * x * y * z;
    g[10][0] = c3b * y * z; g[10][1] = c3b * x * z; g[10][2] = c3b * x * y;
    v[11] = -c3c * y * (4 * z * z - x * x - y * y);
    g[11][0] = 2 * c3c * x * y; g[11][1] = -c3c * (4 * z * z - x * x - 3 * y * y); g[11][2] = -8 * c3c * y * z;
    v[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    g[12][0] = -6 * c3d * x * z; g[12][1] = -6 * c3d * y * z; g[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
    v[13] = -c3c * x * (4 * z * z - x * x - y * y);
    g[13][0] = -c3c * (4 * z * z - 3 * x * x - y * y); g[13][1] = 2 * c3c * x * y; g[13][2] = -8 * c3c * x * z;
    v[14] = c3e * z * (x * x - y * y);
    g[14][0] = 2 * c3e * x * z; g[14][1] = -2 * c3e * y * z; g[14][2] = c3e * (x * x - y * y);
    v[15] = -c3a * x * (x * x - 3 * y * y);
    g[15][0] = -c3a * (3 * x * x - 3 * y * y); g[15][1] = 6 * c3a * x * y;
    const int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < K; ++k) {
        Y[k] = v[k];
        if (dY) for (int a = 0; a < 3; ++a) dY[3 * k + a] = g[k][a];
    }
}

/* ===================================================================== continuous FP64 projection */
typedef struct {
    double s[3], qn, q[4], R[9], M[9], Sig[9];
    double t[3];
    int clamp_x, clamp_y;
    double cxs, cys;  /* clamp factor (tx/tz after clamping) */
    double J[6], T3[6];
    double A, B, C, det;
    double ca, cb, cc;  /* conic */
    double u, v, o, z;
    double dir[3], dn, d[3];
    double rgb[3];
    int rgb_clamped[3];
    double nrm[3];  /* camera-space normal: the shortest axis, facing the camera (RaDe-GS, Sec. 5.1) */
    double rd[2];   /* intersection depth's slope (dz/du, dz/dv) per pixel (RaDe-GS, Sec. 5.1) */
    int nrm_amb;    /* the axis is within 1e-5 of perpendicular to the view direction: orientation open */
} or_cont;

/* Sigma = R S S^T R^T (Sec. 3) for scale s and quaternion q (w, x, y, z), any norm. */
void or_cov3d(const double *s, const double *q, double *Sig, double *Rout)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * s[k] * s[k] * R[3 * c + k];
            Sig[3 * r + c] = acc;
        }
    if (Rout) memcpy(Rout, R, sizeof R);
}

static void cont_project(const or_scene *sc, const or_camera *cam, int64_t i, or_cont *P)
{
    const int64_t S = sc->stride;
    const double *W = cam->viewmat;
    double m[3] = {sc->means[i], sc->means[S + i], sc->means[2 * S + i]};
    for (int k = 0; k < 3; ++k) P->s[k] = exp(sc->log_scales[k * S + i]);
    double q[4] = {sc->quats[i], sc->quats[S + i], sc->quats[2 * S + i], sc->quats[3 * S + i]};
    P->qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) P->q[k] = q[k] / P->qn;
    or_cov3d(P->s, q, P->Sig, P->R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P->M[3 * r + c] = P->R[3 * r + c] * P->s[c];
    for (int r = 0; r < 3; ++r) P->t[r] = W[4 * r] * m[0] + W[4 * r + 1] * m[1] + W[4 * r + 2] * m[2] + W[4 * r + 3];
    const double tx = P->t[0], ty = P->t[1], tz = P->t[2];
    const double fx = cam->fx, fy = cam->fy;
    const double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
    double txtz = tx / tz, tytz = ty / tz;
    P->clamp_x = (txtz > limx || txtz < -limx);
    P->clamp_y = (tytz > limy || tytz < -limy);
    P->cxs = txtz > limx ? limx : (txtz < -limx ? -limx : txtz);
    P->cys = tytz > limy ? limy : (tytz < -limy ? -limy : tytz);
    /* J = [[fx/tz, 0, -fx x'/tz^2], [0, fy/tz, -fy y'/tz^2]], x' = clamp(tx/tz) tz */
    P->J[0] = fx / tz; P->J[1] = 0; P->J[2] = -fx * P->cxs / tz;
    P->J[3] = 0; P->J[4] = fy / tz; P->J[5] = -fy * P->cys / tz;
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += P->J[3 * r + j] * W[4 * j + k];
            P->T3[3 * r + k] = acc;
        }
    double S2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += P->T3[3 * r + a] * P->Sig[3 * a + b] * P->T3[3 * c + b];
            S2[2 * r + c] = acc;
        }
    P->A = S2[0] + OR_LOWPASS;
    P->B = 0.5 * (S2[1] + S2[2]);
    P->C = S2[3] + OR_LOWPASS;
    P->det = P->A * P->C - P->B * P->B;
    P->ca = P->C / P->det;
    P->cb = -P->B / P->det;
    P->cc = P->A / P->det;
    /* Intersection depth (RaDe-GS, which the paper renders depth with, Sec. 5.1). In the
     * EWA ray space (u, v, z) -- image coordinates through the same clamped J, and camera
     * z -- the Gaussian is N((u, v, z), [[J W Sig W^T J^T + 0.3 I, S_zuv^T], [S_zuv, .]]),
     * S_zuv = (W Sig W^T J^T)_{z,:} the covariance of camera z with (u, v). Its densest
     * point along the ray of image point p is the conditional mean of z given (u, v) = p:
     *   z(p) = z + S_zuv (J W Sig W^T J^T + 0.3 I)^-1 (p - (u, v)),
     * affine in p, with the slope rd = S_zuv . conic. */
    double szuv[2];
    for (int r = 0; r < 2; ++r) {
        double acc = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) acc += W[8 + a] * P->Sig[3 * a + b] * P->T3[3 * r + b];
        szuv[r] = acc;
    }
    P->rd[0] = szuv[0] * P->ca + szuv[1] * P->cb;
    P->rd[1] = szuv[0] * P->cb + szuv[1] * P->cc;
    P->u = fx * tx / tz + cam->cx;
    P->v = fy * ty / tz + cam->cy;
    P->o = 1.0 / (1.0 + exp(-sc->logits[i]));
    P->z = tz;
    /* view direction from the camera centre C = -R^T t */
    double cpos[3];
    for (int k = 0; k < 3; ++k) cpos[k] = -(W[k] * W[3] + W[4 + k] * W[7] + W[8 + k] * W[11]);
    for (int k = 0; k < 3; ++k) P->dir[k] = m[k] - cpos[k];
    P->dn = sqrt(P->dir[0] * P->dir[0] + P->dir[1] * P->dir[1] + P->dir[2] * P->dir[2]);
    for (int k = 0; k < 3; ++k) P->d[k] = P->dir[k] / P->dn;
    /* Normal (the normal channel of RaDe-GS, which the paper renders with, Sec. 5.1): the axis
     * of the smallest scale -- chosen on the fp32 log-scale inputs, the first of equal ones --
     * turned to face the camera (n . (mu - C) < 0), in camera coordinates. */
    int kmin = 0;
    for (int k = 1; k < 3; ++k)
        if ((float)sc->log_scales[k * S + i] < (float)sc->log_scales[kmin * S + i]) kmin = k;
    double nw[3] = {P->R[kmin], P->R[3 + kmin], P->R[6 + kmin]};
    const double facing = nw[0] * P->dir[0] + nw[1] * P->dir[1] + nw[2] * P->dir[2];
    P->nrm_amb = fabs(facing) <= 1e-5 * P->dn;
    if (facing > 0.0)
        for (int k = 0; k < 3; ++k) nw[k] = -nw[k];
    for (int r = 0; r < 3; ++r) P->nrm[r] = W[4 * r] * nw[0] + W[4 * r + 1] * nw[1] + W[4 * r + 2] * nw[2];
    double Y[16];
    or_sh_basis(sc->deg, P->d, Y, NULL);
    const int K = (sc->deg + 1) * (sc->deg + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += Y[k] * sc->sh[(int64_t)(k * 3 + c) * S + i];
        acc += 0.5;
        P->rgb_clamped[c] = acc < 0.0;
        P->rgb[c] = acc < 0.0 ? 0.0 : acc;
    }
}

/* ===================================================================== per-Gaussian export */
int or_project(const or_scene *sc, const or_camera *cam, int32_t tile, int32_t *visible, float *z32,
               int32_t *rect4, int32_t *ntiles, double *uv, double *conic, double *opacity, double *rgb,
               double *depth, double *cov2d)
{
    const int64_t n = sc->n;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        or_disc d;
        disc_project(sc, cam, i, &d);
        if (visible) visible[i] = d.visible;
        if (z32) z32[i] = d.z32;
        if (rect4) for (int k = 0; k < 4; ++k) rect4[4 * i + k] = d.rect[k];
        if (ntiles) {
            ntiles[i] = 0;
            if (d.visible && tile > 0)
                ntiles[i] = (d.rect[2] / tile - d.rect[0] / tile + 1) * (d.rect[3] / tile - d.rect[1] / tile + 1);
        }
        if (uv || conic || opacity || rgb || depth || cov2d) {
            or_cont P;
            cont_project(sc, cam, i, &P);
            if (uv) { uv[2 * i] = P.u; uv[2 * i + 1] = P.v; }
            if (conic) { conic[3 * i] = P.ca; conic[3 * i + 1] = P.cb; conic[3 * i + 2] = P.cc; }
            if (opacity) opacity[i] = P.o;
            if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * i + c] = P.rgb[c];
            if (depth) depth[i] = P.z;
            if (cov2d) { cov2d[3 * i] = P.A; cov2d[3 * i + 1] = P.B; cov2d[3 * i + 2] = P.C; }
        }
    }
    return 0;
}

/* ===================================================================== per-pixel compositing */
typedef struct {
    int64_t idx;
    float z32;
} or_cand;

static int cand_cmp(const void *a, const void *b)
{
    const or_cand *x = (const or_cand *)a, *y = (const or_cand *)b;
    if (x->z32 < y->z32) return -1;
    if (x->z32 > y->z32) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* one blended step, kept for the reverse pass */
typedef struct {
    int64_t g;
    double a, ax, ay, T, Tx, Ty, dx, dy;
    int capped;
} or_step;

typedef struct {
    double rgb[3], gx[3], gy[3], depth, alpha, T, Tx, Ty;
    double normal[3];  /* sum of n_i a_i T_i (camera space) */
    double depth_isect; /* sum of z_i(p) a_i T_i, the intersection depth (or_cont.rd) */
    int32_t nrm_amb;   /* a blended Gaussian's normal orientation is open (or_cont.nrm_amb) */
    double gx_abs[3], gy_abs[3]; /* the scale of an fp32 evaluation's error of dI/dx, dI/dy (below) */
    int32_t n_blended;
    uint32_t sig;
    int32_t amb; /* a discrete decision (cap, cut, stop) lies within its band (below) of its threshold */
} or_pix;

/* The band around a threshold inside which a decision counts as open (amb): 1e-5
 * relative, plus, per Gaussian, u * kappa with u = 2^-24 and kappa = max|conic| * |d|^2.
 * kappa bounds how much a one-ulp perturbation of the footprint's shape or direction
 * moves Q at this pixel, relative to u: about Q for a round footprint, far more for a
 * long thin one seen far along its long axis, whose alpha an fp32 evaluation from the
 * same fp32 inputs can only get to ~1e-4 of itself there. */
#define OR_AMB_REL 3e-5
#define OR_U32 5.9604644775390625e-08

/* Eq. 2-4 for one pixel over the depth-ordered candidate list. */
static void composite_pixel(const or_cand *list, int64_t len, const or_cont *P, int px, int py,
                            const double *bg, or_pix *out, or_step *trace, int64_t *n_trace)
{
    const double X = px + 0.5, Yp = py + 0.5;
    double T = 1.0, Tx = 0.0, Ty = 0.0, D = 0.0;
    double C[3] = {0, 0, 0}, Cx[3] = {0, 0, 0}, Cy[3] = {0, 0, 0}, Ax[3] = {0, 0, 0}, Ay[3] = {0, 0, 0};
    double N[3] = {0, 0, 0}, Di = 0.0;
    int32_t nb = 0, amb = 0, namb = 0;
    uint32_t sig = 2166136261u;
    int64_t nt = 0;
    for (int64_t k = 0; k < len; ++k) {
        const or_cont *g = &P[list[k].idx];
        double dx = X - g->u, dy = Yp - g->v;
        double Q = g->ca * dx * dx + 2.0 * g->cb * dx * dy + g->cc * dy * dy;
        double a = g->o * exp(-0.5 * Q);
        const double cmax = fmax(fabs(g->ca), fmax(fabs(g->cb), fabs(g->cc)));
        const double band = OR_AMB_REL + OR_U32 * cmax * (dx * dx + dy * dy);
        if (fabs(a - OR_ALPHA_CAP) <= band * OR_ALPHA_CAP || fabs(a - OR_ALPHA_MIN) <= band * OR_ALPHA_MIN)
            amb = 1;
        int capped = 0;
        if (a > OR_ALPHA_CAP) { a = OR_ALPHA_CAP; capped = 1; }
        if (a < OR_ALPHA_MIN) continue;
        if (fabs(T * (1.0 - a) - OR_T_MIN) <= band * OR_T_MIN) amb = 1;
        if (T * (1.0 - a) < OR_T_MIN) { sig = (sig ^ 0xA5A5A5A5u) * 16777619u; break; }
        double ax = capped ? 0.0 : -a * (g->ca * dx + g->cb * dy);
        double ay = capped ? 0.0 : -a * (g->cb * dx + g->cc * dy);
        if (trace) {
            or_step *s = &trace[nt];
            s->g = list[k].idx; s->a = a; s->ax = ax; s->ay = ay; s->T = T; s->Tx = Tx; s->Ty = Ty;
            s->dx = dx; s->dy = dy; s->capped = capped;
        }
        ++nt;
        /* Error scale of the x and y terms (a tolerance, not part of the render): the
         * magnitudes of their operands -- c T_x a and c T a (|a' dx| + |b' dy|), the
         * products inside (conic d) included -- each weighted by 1 + u kappa / 2e-4,
         * the conditioning of alpha at this pixel (kappa as in the decision band). */
        const double wk = 1.0 + OR_U32 * cmax * (dx * dx + dy * dy) / 2e-4;
        const double mx = capped ? 0.0 : a * (fabs(g->ca * dx) + fabs(g->cb * dy));
        const double my = capped ? 0.0 : a * (fabs(g->cb * dx) + fabs(g->cc * dy));
        for (int c = 0; c < 3; ++c) {
            C[c] += g->rgb[c] * a * T;                 /* Eq. 2 */
            Cx[c] += g->rgb[c] * (Tx * a + T * ax);    /* Eq. 3 */
            Cy[c] += g->rgb[c] * (Ty * a + T * ay);
            Ax[c] += fabs(g->rgb[c]) * (fabs(Tx) * a + T * mx) * wk;
            Ay[c] += fabs(g->rgb[c]) * (fabs(Ty) * a + T * my) * wk;
        }
        D += g->z * a * T;
        for (int c = 0; c < 3; ++c) N[c] += g->nrm[c] * a * T;  /* blended like the colour */
        Di += (g->z + g->rd[0] * dx + g->rd[1] * dy) * a * T;
        namb |= g->nrm_amb;
        Tx = -ax * T + (1.0 - a) * Tx;                 /* Eq. 4 */
        Ty = -ay * T + (1.0 - a) * Ty;
        T = T * (1.0 - a);
        ++nb;
        sig = (sig ^ (uint32_t)(list[k].idx * 2 + capped)) * 16777619u;
    }
    for (int c = 0; c < 3; ++c) {
        out->rgb[c] = C[c] + T * bg[c];
        out->gx[c] = Cx[c] + bg[c] * Tx;
        out->gy[c] = Cy[c] + bg[c] * Ty;
        out->gx_abs[c] = Ax[c] + fabs(bg[c] * Tx);
        out->gy_abs[c] = Ay[c] + fabs(bg[c] * Ty);
    }
    out->depth = D;
    out->alpha = 1.0 - T;
    for (int c = 0; c < 3; ++c) out->normal[c] = N[c];
    out->depth_isect = Di;
    out->nrm_amb = namb;
    out->T = T; out->Tx = Tx; out->Ty = Ty;
    out->n_blended = nb;
    out->sig = sig;
    out->amb = amb;
    if (n_trace) *n_trace = nt;
}

/* Projection of all Gaussians (discrete + continuous). */
typedef struct {
    or_disc *D;
    or_cont *P;
    int64_t *vis;   /* indices of visible Gaussians */
    int64_t nvis;
} or_frame;

static int frame_build(const or_scene *sc, const or_camera *cam, or_frame *F)
{
    const int64_t n = sc->n;
    F->D = (or_disc *)malloc(sizeof(or_disc) * (size_t)(n > 0 ? n : 1));
    F->P = (or_cont *)malloc(sizeof(or_cont) * (size_t)(n > 0 ? n : 1));
    F->vis = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!F->D || !F->P || !F->vis) return -2;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        disc_project(sc, cam, i, &F->D[i]);
        if (F->D[i].visible) cont_project(sc, cam, i, &F->P[i]);
    }
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (F->D[i].visible) F->vis[c++] = i;
    F->nvis = c;
    return 0;
}

static void frame_free(or_frame *F)
{
    free(F->D);
    free(F->P);
    free(F->vis);
}

static inline int rect_has(const or_disc *d, int px, int py)
{
    return px >= d->rect[0] && px <= d->rect[2] && py >= d->rect[1] && py <= d->rect[3];
}

/* Candidate list of one pixel, brute force: every visible Gaussian whose support
 * rectangle contains the pixel, ordered by (fp32 depth, index). */
static int64_t pixel_list_brute(const or_frame *F, int px, int py, or_cand *buf)
{
    int64_t len = 0;
    for (int64_t k = 0; k < F->nvis; ++k) {
        int64_t i = F->vis[k];
        if (rect_has(&F->D[i], px, py)) {
            buf[len].idx = i;
            buf[len].z32 = F->D[i].z32;
            ++len;
        }
    }
    qsort(buf, (size_t)len, sizeof(or_cand), cand_cmp);
    return len;
}

/* Binned lists: every visible Gaussian is entered into the 16x16-pixel buckets
 * its rectangle touches; each bucket is sorted once by (fp32 depth, index); a
 * pixel's list is its bucket's list filtered by rectangle containment, which is
 * the brute-force list in the same order. */
#define OR_BUCKET 16
typedef struct {
    int nbx, nby;
    int64_t *start;   /* [nb + 1] */
    or_cand *items;
} or_buckets;

static int buckets_build(const or_frame *F, int W, int H, or_buckets *B)
{
    B->nbx = (W + OR_BUCKET - 1) / OR_BUCKET;
    B->nby = (H + OR_BUCKET - 1) / OR_BUCKET;
    const int64_t nb = (int64_t)B->nbx * B->nby;
    B->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    if (!B->start) return -2;
    for (int64_t k = 0; k < F->nvis; ++k) {
        const or_disc *d = &F->D[F->vis[k]];
        for (int by = d->rect[1] / OR_BUCKET; by <= d->rect[3] / OR_BUCKET; ++by)
            for (int bx = d->rect[0] / OR_BUCKET; bx <= d->rect[2] / OR_BUCKET; ++bx)
                B->start[(int64_t)by * B->nbx + bx + 1]++;
    }
    for (int64_t b = 0; b < nb; ++b) B->start[b + 1] += B->start[b];
    B->items = (or_cand *)malloc(sizeof(or_cand) * (size_t)(B->start[nb] > 0 ? B->start[nb] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    if (!B->items || !fill) return -2;
    memcpy(fill, B->start, sizeof(int64_t) * (size_t)nb);
    for (int64_t k = 0; k < F->nvis; ++k) {
        int64_t i = F->vis[k];
        const or_disc *d = &F->D[i];
        for (int by = d->rect[1] / OR_BUCKET; by <= d->rect[3] / OR_BUCKET; ++by)
            for (int bx = d->rect[0] / OR_BUCKET; bx <= d->rect[2] / OR_BUCKET; ++bx) {
                or_cand *c = &B->items[fill[(int64_t)by * B->nbx + bx]++];
                c->idx = i;
                c->z32 = d->z32;
            }
    }
    free(fill);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nb; ++b)
        qsort(B->items + B->start[b], (size_t)(B->start[b + 1] - B->start[b]), sizeof(or_cand), cand_cmp);
    return 0;
}

static void buckets_free(or_buckets *B)
{
    free(B->start);
    free(B->items);
}

static int64_t pixel_list_binned(const or_frame *F, const or_buckets *B, int px, int py, or_cand *buf)
{
    const int64_t b = (int64_t)(py / OR_BUCKET) * B->nbx + px / OR_BUCKET;
    int64_t len = 0;
    for (int64_t k = B->start[b]; k < B->start[b + 1]; ++k)
        if (rect_has(&F->D[B->items[k].idx], px, py)) buf[len++] = B->items[k];
    return len;
}

static int64_t max_bucket(const or_buckets *B)
{
    int64_t m = 0;
    for (int64_t b = 0; b < (int64_t)B->nbx * B->nby; ++b)
        if (B->start[b + 1] - B->start[b] > m) m = B->start[b + 1] - B->start[b];
    return m;
}

/* Full-frame render. mode 0 = brute force, 1 = binned. Planar outputs:
 * rgb/dcdx/dcdy [3][H][W], depth/alpha/final_T [H][W]; any may be NULL. */
static int render_rows(const or_scene *sc, const or_camera *cam, int mode, int y0, int y1, double *rgb,
                       double *dcdx, double *dcdy, double *depth, double *alpha, double *final_T,
                       int32_t *n_blended, uint32_t *sig, int32_t *amb, double *gabs, double *normal, double *nv,
                       int32_t *nrm_amb, double *depth_isect);

int or_render(const or_scene *sc, const or_camera *cam, int mode, double *rgb, double *dcdx, double *dcdy,
              double *depth, double *alpha, double *final_T, int32_t *n_blended, uint32_t *sig, int32_t *amb, double *gabs)
{
    return render_rows(sc, cam, mode, 0, cam->height, rgb, dcdx, dcdy, depth, alpha, final_T, n_blended, sig, amb, gabs,
                       NULL, NULL, NULL, NULL);
}

/* Rows [y0, y1) of the frame (binned mode), written into full-size planes. */
int or_render_band(const or_scene *sc, const or_camera *cam, int y0, int y1, double *rgb, double *dcdx,
                   double *dcdy, double *depth, double *alpha)
{
    if (y0 < 0) y0 = 0;
    if (y1 > cam->height) y1 = cam->height;
    return render_rows(sc, cam, 1, y0, y1, rgb, dcdx, dcdy, depth, alpha, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                       NULL, NULL);
}

/* The RaDe-GS channels (binned mode) with the colour's weights: the normal channel, the
 * normal-view map and the intersection depth, plus alpha and the orientation-ambiguity
 * flag per pixel. */
int or_render_normals(const or_scene *sc, const or_camera *cam, double *normal, double *nv, double *alpha,
                      int32_t *nrm_amb, int32_t *amb, double *depth_isect)
{
    return render_rows(sc, cam, 1, 0, cam->height, NULL, NULL, NULL, NULL, alpha, NULL, NULL, NULL, amb, NULL, normal,
                       nv, nrm_amb, depth_isect);
}

static int render_rows(const or_scene *sc, const or_camera *cam, int mode, int y0, int y1, double *rgb,
                       double *dcdx, double *dcdy, double *depth, double *alpha, double *final_T,
                       int32_t *n_blended, uint32_t *sig, int32_t *amb, double *gabs, double *normal, double *nv,
                       int32_t *nrm_amb, double *depth_isect)
{
    const int W = cam->width, H = cam->height;
    const int64_t HW = (int64_t)W * H;
    or_frame F;
    if (frame_build(sc, cam, &F)) return -2;
    or_buckets B = {0, 0, NULL, NULL};
    int64_t cap = F.nvis;
    if (mode == 1) {
        if (buckets_build(&F, W, H, &B)) return -2;
        cap = max_bucket(&B);
    }
    int rc = 0;
#pragma omp parallel
    {
        or_cand *buf = (or_cand *)malloc(sizeof(or_cand) * (size_t)(cap > 0 ? cap : 1));
        if (!buf) rc = -2;
#pragma omp for schedule(dynamic, 1)
        for (int py = y0; py < y1; ++py) {
            if (!buf) continue;
            for (int px = 0; px < W; ++px) {
                int64_t len = mode == 1 ? pixel_list_binned(&F, &B, px, py, buf) : pixel_list_brute(&F, px, py, buf);
                or_pix o;
                composite_pixel(buf, len, F.P, px, py, cam->bg, &o, NULL, NULL);
                const int64_t p = (int64_t)py * W + px;
                for (int c = 0; c < 3; ++c) {
                    if (rgb) rgb[c * HW + p] = o.rgb[c];
                    if (dcdx) dcdx[c * HW + p] = o.gx[c];
                    if (dcdy) dcdy[c * HW + p] = o.gy[c];
                }
                if (depth) depth[p] = o.depth;
                if (alpha) alpha[p] = o.alpha;
                if (final_T) final_T[p] = o.T;
                if (n_blended) n_blended[p] = o.n_blended;
                if (sig) sig[p] = o.sig;
                if (amb) amb[p] = o.amb;
                if (gabs)
                    for (int c = 0; c < 3; ++c) {
                        gabs[c * HW + p] = o.gx_abs[c];
                        gabs[(3 + c) * HW + p] = o.gy_abs[c];
                    }
                if (normal)
                    for (int c = 0; c < 3; ++c) normal[c * HW + p] = o.normal[c];
                if (nv) {
                    /* Nv = -N . (unit ray of the pixel centre): 1 x alpha for a surface facing the camera */
                    const double r[3] = {(px + 0.5 - cam->cx) / cam->fx, (py + 0.5 - cam->cy) / cam->fy, 1.0};
                    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                    nv[p] = -(o.normal[0] * r[0] + o.normal[1] * r[1] + o.normal[2] * r[2]) / rn;
                }
                if (nrm_amb) nrm_amb[p] = o.nrm_amb;
                if (depth_isect) depth_isect[p] = o.depth_isect;
            }
        }
        free(buf);
    }
    if (mode == 1) buckets_free(&B);
    frame_free(&F);
    return rc;
}

/* A sample of pixels (brute force per pixel). out: [npix][11] =
 * rgb(3), dcdx(3), dcdy(3), depth, alpha. */
int or_render_pixels(const or_scene *sc, const or_camera *cam, int64_t npix, const int32_t *px,
                     const int32_t *py, double *out, int32_t *n_blended, int32_t *amb, double *gabs)
{
    or_frame F;
    if (frame_build(sc, cam, &F)) return -2;
    int rc = 0;
#pragma omp parallel
    {
        or_cand *buf = (or_cand *)malloc(sizeof(or_cand) * (size_t)(F.nvis > 0 ? F.nvis : 1));
        if (!buf) rc = -2;
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < npix; ++k) {
            if (!buf) continue;
            int64_t len = pixel_list_brute(&F, px[k], py[k], buf);
            or_pix o;
            composite_pixel(buf, len, F.P, px[k], py[k], cam->bg, &o, NULL, NULL);
            double *r = out + 11 * k;
            for (int c = 0; c < 3; ++c) { r[c] = o.rgb[c]; r[3 + c] = o.gx[c]; r[6 + c] = o.gy[c]; }
            r[9] = o.depth;
            r[10] = o.alpha;
            if (n_blended) n_blended[k] = o.n_blended;
            if (amb) amb[k] = o.amb;
            if (gabs)
                for (int c = 0; c < 3; ++c) {
                    gabs[6 * k + c] = o.gx_abs[c];
                    gabs[6 * k + 3 + c] = o.gy_abs[c];
                }
        }
        free(buf);
    }
    frame_free(&F);
    return rc;
}

/* ===================================================================== tile keys (depth sort, Sec. 3)
 * Instances: one per (visible Gaussian, tile its rectangle touches), key =
 * (tile id << 32) | fp32 bits of the depth, value = Gaussian index; sorted by
 * (key, value), i.e. a stable sort of the index-ordered instance list. */
typedef struct {
    uint64_t key;
    uint32_t val;
} or_kv;

static int kv_cmp(const void *a, const void *b)
{
    const or_kv *x = (const or_kv *)a, *y = (const or_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->val > y->val) - (x->val < y->val);
}

int64_t or_count_instances(const or_scene *sc, const or_camera *cam, int32_t tile)
{
    int64_t tot = 0;
#pragma omp parallel for reduction(+ : tot)
    for (int64_t i = 0; i < sc->n; ++i) {
        or_disc d;
        disc_project(sc, cam, i, &d);
        if (d.visible) tot += (int64_t)(d.rect[2] / tile - d.rect[0] / tile + 1) * (d.rect[3] / tile - d.rect[1] / tile + 1);
    }
    return tot;
}

int or_keys(const or_scene *sc, const or_camera *cam, int32_t tile, int64_t cap, uint64_t *keys, uint32_t *vals,
            uint32_t *ranges /* [n_tiles][2] */)
{
    const int W = cam->width, H = cam->height;
    const int tw = (W + tile - 1) / tile, th = (H + tile - 1) / tile;
    or_disc *D = (or_disc *)malloc(sizeof(or_disc) * (size_t)(sc->n > 0 ? sc->n : 1));
    if (!D) return -2;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < sc->n; ++i) disc_project(sc, cam, i, &D[i]);
    int64_t K = 0;
    for (int64_t i = 0; i < sc->n; ++i)
        if (D[i].visible) K += (int64_t)(D[i].rect[2] / tile - D[i].rect[0] / tile + 1) * (D[i].rect[3] / tile - D[i].rect[1] / tile + 1);
    if (K > cap) { free(D); return -5; }
    or_kv *kv = (or_kv *)malloc(sizeof(or_kv) * (size_t)(K > 0 ? K : 1));
    if (!kv) { free(D); return -2; }
    int64_t o = 0;
    for (int64_t i = 0; i < sc->n; ++i) {
        if (!D[i].visible) continue;
        uint32_t zb;
        memcpy(&zb, &D[i].z32, 4);
        for (int ty = D[i].rect[1] / tile; ty <= D[i].rect[3] / tile; ++ty)
            for (int tx = D[i].rect[0] / tile; tx <= D[i].rect[2] / tile; ++tx) {
                kv[o].key = ((uint64_t)(ty * tw + tx) << 32) | zb;
                kv[o].val = (uint32_t)i;
                ++o;
            }
    }
    qsort(kv, (size_t)K, sizeof(or_kv), kv_cmp);
    for (int64_t k = 0; k < K; ++k) { keys[k] = kv[k].key; vals[k] = kv[k].val; }
    if (ranges) {
        memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)tw * th);
        for (int64_t k = 0; k < K; ++k) {
            uint32_t t = (uint32_t)(kv[k].key >> 32);
            if (k == 0 || (uint32_t)(kv[k - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)k;
            if (k == K - 1 || (uint32_t)(kv[k + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
        }
    }
    free(kv);
    free(D);
    return 0;
}

/* ===================================================================== backward (adjoint) */
typedef struct {
    double u, v, a, b, c, o, z, rgb[3];
} or_g2;

/* Reverse pass of Eq. 2-4 for one pixel from its forward trace; accumulates the
 * per-Gaussian adjoints of (u, v, conic a/b/c, opacity, depth, colour). */
static void pixel_backward(const or_step *tr, int64_t nt, const or_cont *P, const or_pix *fw, const double *bg,
                           const double *gr, const double *gx, const double *gy, double gd, double ga, or_g2 *G)
{
    double Tb = -ga, Txb = 0.0, Tyb = 0.0;
    for (int c = 0; c < 3; ++c) {
        Tb += gr[c] * bg[c];
        Txb += gx[c] * bg[c];
        Tyb += gy[c] * bg[c];
    }
    (void)fw;
    for (int64_t s = nt - 1; s >= 0; --s) {
        const or_step *st = &tr[s];
        const or_cont *g = &P[st->g];
        or_g2 *o = &G[st->g];
        const double a = st->a, ax = st->ax, ay = st->ay, T = st->T, Tx = st->Tx, Ty = st->Ty;
        double Gc = 0, Gx = 0, Gy = 0;
        for (int c = 0; c < 3; ++c) {
            o->rgb[c] += gr[c] * a * T + gx[c] * (Tx * a + T * ax) + gy[c] * (Ty * a + T * ay);
            Gc += gr[c] * g->rgb[c];
            Gx += gx[c] * g->rgb[c];
            Gy += gy[c] * g->rgb[c];
        }
        o->z += gd * a * T;
        const double dA = Gc * T + Gx * Tx + Gy * Ty + gd * g->z * T - Tb * T - Txb * Tx - Tyb * Ty;
        const double dAx = Gx * T - Txb * T;
        const double dAy = Gy * T - Tyb * T;
        const double Tb_prev = Gc * a + Gx * ax + Gy * ay + gd * g->z * a + Tb * (1.0 - a) - Txb * ax - Tyb * ay;
        const double Txb_prev = Gx * a + Txb * (1.0 - a);
        const double Tyb_prev = Gy * a + Tyb * (1.0 - a);
        if (!st->capped) {
            const double dx = st->dx, dy = st->dy;
            const double ex = g->ca * dx + g->cb * dy, ey = g->cb * dx + g->cc * dy;
            const double Abar = dA - dAx * ex - dAy * ey;
            o->o += Abar * (a / g->o);
            const double gQ = -0.5 * a * Abar;
            const double gex = -a * dAx, gey = -a * dAy;
            o->a += gQ * dx * dx + gex * dx;
            o->b += gQ * 2.0 * dx * dy + gex * dy + gey * dx;
            o->c += gQ * dy * dy + gey * dy;
            const double gdx = gQ * 2.0 * ex + gex * g->ca + gey * g->cb;
            const double gdy = gQ * 2.0 * ey + gex * g->cb + gey * g->cc;
            o->u -= gdx;
            o->v -= gdy;
        }
        Tb = Tb_prev;
        Txb = Txb_prev;
        Tyb = Tyb_prev;
    }
}

/* Chain rule from the 2D adjoints of Gaussian i to its 3D parameters. */
static void gaussian_backward(const or_scene *sc, const or_camera *cam, int64_t i, const or_cont *P,
                              const or_g2 *g2, double *d_means, double *d_ls, double *d_q, double *d_lg,
                              double *d_sh)
{
    const int64_t S = sc->stride;
    const double *W = cam->viewmat;
    const double tx = P->t[0], ty = P->t[1], tz = P->t[2];
    const double fx = cam->fx, fy = cam->fy;
    double tb[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
    /* opacity */
    d_lg[i] += g2->o * P->o * (1.0 - P->o);
    /* centre u = fx tx/tz + cx, v = fy ty/tz + cy; depth z = tz */
    tb[0] += g2->u * fx / tz;
    tb[1] += g2->v * fy / tz;
    tb[2] += -g2->u * fx * tx / (tz * tz) - g2->v * fy * ty / (tz * tz) + g2->z;
    /* conic = inverse(Sigma2D): Sbar = -K Gbar K with Gbar = [[a, b/2], [b/2, c]] */
    const double K[4] = {P->ca, P->cb, P->cb, P->cc};
    const double Gb[4] = {g2->a, 0.5 * g2->b, 0.5 * g2->b, g2->c};
    double KG[4], Sb[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) KG[2 * r + c] = K[2 * r] * Gb[c] + K[2 * r + 1] * Gb[2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) Sb[2 * r + c] = -(KG[2 * r] * K[c] + KG[2 * r + 1] * K[2 + c]);
    /* Sigma2D = T3 Sigma T3^T + 0.3 I: Sigmabar = T3^T Sb T3, T3bar = 2 Sb T3 Sigma */
    double Sigb[9], T3b[6];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) acc += P->T3[3 * r + a] * Sb[2 * r + c] * P->T3[3 * c + b];
            Sigb[3 * a + b] = acc;
        }
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int c = 0; c < 2; ++c)
                for (int j = 0; j < 3; ++j) acc += Sb[2 * r + c] * P->T3[3 * c + j] * P->Sig[3 * j + k];
            T3b[3 * r + k] = 2.0 * acc;
        }
    /* T3 = J W: Jbar = T3bar W^T (W = rotation part of viewmat) */
    double Jb[6];
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += T3b[3 * r + k] * W[4 * j + k];
            Jb[3 * r + j] = acc;
        }
    /* J00 = fx/tz, J11 = fy/tz, J02 = -fx x'/tz^2, J12 = -fy y'/tz^2 with x' = tx
     * unless clamped, in which case x' = c tz and J02 = -fx c / tz. */
    tb[2] += Jb[0] * (-fx / (tz * tz)) + Jb[4] * (-fy / (tz * tz));
    if (!P->clamp_x) {
        tb[0] += Jb[2] * (-fx / (tz * tz));
        tb[2] += Jb[2] * (2.0 * fx * tx / (tz * tz * tz));
    } else {
        tb[2] += Jb[2] * (fx * P->cxs / (tz * tz));
    }
    if (!P->clamp_y) {
        tb[1] += Jb[5] * (-fy / (tz * tz));
        tb[2] += Jb[5] * (2.0 * fy * ty / (tz * tz * tz));
    } else {
        tb[2] += Jb[5] * (fy * P->cys / (tz * tz));
    }
    /* t = W m + t0 */
    for (int k = 0; k < 3; ++k) mb[k] += W[k] * tb[0] + W[4 + k] * tb[1] + W[8 + k] * tb[2];
    /* Sigma = M M^T, M = R diag(s): Mbar = 2 Sigmabar M */
    double Mb[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += (Sigb[3 * r + k] + Sigb[3 * k + r]) * P->M[3 * k + c];
            Mb[3 * r + c] = acc;
        }
    double Rb[9];
    for (int c = 0; c < 3; ++c) {
        double sb = 0;
        for (int r = 0; r < 3; ++r) {
            sb += Mb[3 * r + c] * P->R[3 * r + c];
            Rb[3 * r + c] = Mb[3 * r + c] * P->s[c];
        }
        d_ls[c * S + i] += sb * P->s[c];
    }
    /* R(q^) -> q^bar */
    const double w = P->q[0], x = P->q[1], y = P->q[2], z = P->q[3];
    double qb[4];
    qb[0] = 2 * (-z * Rb[1] + y * Rb[2] + z * Rb[3] - x * Rb[5] - y * Rb[6] + x * Rb[7]);
    qb[1] = 2 * (y * Rb[1] + z * Rb[2] + y * Rb[3] - 2 * x * Rb[4] - w * Rb[5] + z * Rb[6] + w * Rb[7] - 2 * x * Rb[8]);
    qb[2] = 2 * (-2 * y * Rb[0] + x * Rb[1] + w * Rb[2] + x * Rb[3] + z * Rb[5] - w * Rb[6] + z * Rb[7] - 2 * y * Rb[8]);
    qb[3] = 2 * (-2 * z * Rb[0] - w * Rb[1] + x * Rb[2] + w * Rb[3] - 2 * z * Rb[4] + y * Rb[5] + x * Rb[6] + y * Rb[7]);
    /* q^ = q / |q| */
    const double dot = w * qb[0] + x * qb[1] + y * qb[2] + z * qb[3];
    for (int k = 0; k < 4; ++k) d_q[k * S + i] += (qb[k] - P->q[k] * dot) / P->qn;
    /* colour: c = max(0, sum_k Y_k(d) sh_k + 0.5), d = (m - C)/|m - C| */
    double Y[16], dY[48], db[3] = {0, 0, 0};
    or_sh_basis(sc->deg, P->d, Y, dY);
    const int Kc = (sc->deg + 1) * (sc->deg + 1);
    for (int c = 0; c < 3; ++c) {
        if (P->rgb_clamped[c]) continue;
        const double gc = g2->rgb[c];
        for (int k = 0; k < Kc; ++k) {
            d_sh[(int64_t)(k * 3 + c) * S + i] += gc * Y[k];
            const double shv = sc->sh[(int64_t)(k * 3 + c) * S + i];
            for (int a = 0; a < 3; ++a) db[a] += gc * shv * dY[3 * k + a];
        }
    }
    const double dd = db[0] * P->d[0] + db[1] * P->d[1] + db[2] * P->d[2];
    for (int a = 0; a < 3; ++a) mb[a] += (db[a] - P->d[a] * dd) / P->dn;
    for (int a = 0; a < 3; ++a) d_means[a * S + i] += mb[a];
}

/* Adjoint of L = sum over pixels of <g_rgb, rgb> + <g_dcdx, dcdx> + <g_dcdy, dcdy>
 * + g_depth depth + g_alpha alpha (upstream planes, any may be NULL = 0).
 * Outputs are accumulated (+=) into planar grads with the scene's stride; the
 * 2D adjoints (u, v, conic a, b, c, opacity, depth, rgb) go to g2d [n][10] if
 * non-NULL. */
int or_backward(const or_scene *sc, const or_camera *cam, const double *g_rgb, const double *g_dcdx,
                const double *g_dcdy, const double *g_depth, const double *g_alpha, double *d_means,
                double *d_ls, double *d_q, double *d_lg, double *d_sh, double *g2d)
{
    const int W = cam->width, H = cam->height;
    const int64_t HW = (int64_t)W * H, n = sc->n;
    or_frame F;
    if (frame_build(sc, cam, &F)) return -2;
    or_buckets B;
    if (buckets_build(&F, W, H, &B)) return -2;
    const int64_t cap = max_bucket(&B);
    or_g2 *G = (or_g2 *)calloc((size_t)(n > 0 ? n : 1), sizeof(or_g2));
    if (!G) return -2;
    int rc = 0;
#pragma omp parallel
    {
        or_cand *buf = (or_cand *)malloc(sizeof(or_cand) * (size_t)(cap > 0 ? cap : 1));
        or_step *tr = (or_step *)malloc(sizeof(or_step) * (size_t)(cap > 0 ? cap : 1));
        or_g2 *Gl = (or_g2 *)calloc((size_t)(n > 0 ? n : 1), sizeof(or_g2));
        if (!buf || !tr || !Gl) rc = -2;
#pragma omp for schedule(dynamic, 1)
        for (int py = 0; py < H; ++py) {
            if (!buf || !tr || !Gl) continue;
            for (int px = 0; px < W; ++px) {
                const int64_t p = (int64_t)py * W + px;
                int64_t len = pixel_list_binned(&F, &B, px, py, buf), nt = 0;
                or_pix fw;
                composite_pixel(buf, len, F.P, px, py, cam->bg, &fw, tr, &nt);
                double gr[3] = {0, 0, 0}, gxv[3] = {0, 0, 0}, gyv[3] = {0, 0, 0};
                for (int c = 0; c < 3; ++c) {
                    if (g_rgb) gr[c] = g_rgb[c * HW + p];
                    if (g_dcdx) gxv[c] = g_dcdx[c * HW + p];
                    if (g_dcdy) gyv[c] = g_dcdy[c * HW + p];
                }
                pixel_backward(tr, nt, F.P, &fw, cam->bg, gr, gxv, gyv, g_depth ? g_depth[p] : 0.0,
                               g_alpha ? g_alpha[p] : 0.0, Gl);
            }
        }
#pragma omp critical
        {
            if (Gl)
                for (int64_t i = 0; i < n; ++i) {
                    double *dst = (double *)&G[i];
                    const double *src = (const double *)&Gl[i];
                    for (int k = 0; k < 10; ++k) dst[k] += src[k];
                }
        }
        free(buf);
        free(tr);
        free(Gl);
    }
    if (rc == 0) {
        for (int64_t k = 0; k < F.nvis; ++k) {
            const int64_t i = F.vis[k];
            gaussian_backward(sc, cam, i, &F.P[i], &G[i], d_means, d_ls, d_q, d_lg, d_sh);
        }
        if (g2d)
            for (int64_t i = 0; i < n; ++i) {
                const or_g2 *g = &G[i];
                double *r = g2d + 10 * i;
                r[0] = g->u; r[1] = g->v; r[2] = g->a; r[3] = g->b; r[4] = g->c; r[5] = g->o; r[6] = g->z;
                r[7] = g->rgb[0]; r[8] = g->rgb[1]; r[9] = g->rgb[2];
            }
    }
    free(G);
    buckets_free(&B);
    frame_free(&F);
    return rc;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ===================================================================== frame-interpolation geometry
 * The geometric half of the paper's frame interpolation (Sec. 4.2, "Forward-Backward
 * Warping"): camera motion vectors, the warp operator w(., V) and the warped gradient.
 *
 *   V[x]        = Proj(UnProj(x, D[x], P_src), P_dst) - x
 *   w(F, V)     : forward warp. Every source pixel that moves lands on the target pixel
 *                 containing x + V[x]; of the pixels landing on one target pixel, the one
 *                 nearest to the target camera wins (target-camera z, then the smaller
 *                 source index); a target pixel nobody lands on is a hole (0, index -1).
 *   G_dst       = w(G_src, V) . dx/dy : the gradient of a warped image by the chain rule,
 *                 dx/dy = (dy/dx)^-1 with dy/dx = I + dV/dx the spatial derivative of the
 *                 motion map, taken by central differences over the source pixel grid.
 *
 * Readings (the paper is silent on them): D is the render's depth channel normalised by
 * its alpha (a convex combination of the blended Gaussians' camera z) and a pixel moves
 * only where alpha > alpha_min; UnProj lifts pixel centre (i + 0.5, j + 0.5) to camera z
 * = D; the warp is nearest-pixel with a depth test; a one-sided difference replaces the
 * central one where a neighbour does not move, the identity where neither does; a
 * non-positive Jacobian determinant (a fold) gives a zero warped gradient.
 *
 * The discrete decisions (which target pixel, which source wins) follow the fp32
 * round-to-nearest sequence of warp_pos32 so that an fp32 implementation can reproduce
 * them bit for bit; motion vectors are reported from the same sequence. The determinant,
 * inverse and gradient products are FP64. warp_pos64 evaluates the same map in FP64
 * (pins compare it with closed forms and bound the fp32 sequence's rounding).
 */

/* fp32 spec: target position (u, v) and target-camera z of source pixel (i, j).
 * Returns 1 when the pixel moves: alpha > alpha_min (or depth > 0 without alpha) and
 * the lifted point lies beyond the target camera's near plane. */
static int warp_pos32(const or_camera *s, const or_camera *t, const double *depth, const double *alpha,
                      double alpha_min, int W, int i, int j, float *u, float *v, float *z)
{
    const int64_t p = (int64_t)j * W + i;
    float d;
    if (alpha) {
        const float a = (float)alpha[p];
        if (!(a > (float)alpha_min)) return 0;
        d = (float)depth[p] / a;
    } else {
        d = (float)depth[p];
        if (!(d > 0.0f)) return 0;
    }
    /* UnProj: camera-space point of the pixel centre at camera z = d, then world. */
    const float xn = (((float)i + 0.5f) - (float)s->cx) / (float)s->fx;
    const float yn = (((float)j + 0.5f) - (float)s->cy) / (float)s->fy;
    const float xc = xn * d, yc = yn * d, zc = d;
    float R[12], Q[12];
    for (int k = 0; k < 12; ++k) {
        R[k] = (float)s->viewmat[k];
        Q[k] = (float)t->viewmat[k];
    }
    const float a0 = xc - R[3], a1 = yc - R[7], a2 = zc - R[11];
    /* world = R^T (camera - t) */
    const float xw = (R[0] * a0 + R[4] * a1) + R[8] * a2;
    const float yw = (R[1] * a0 + R[5] * a1) + R[9] * a2;
    const float zw = (R[2] * a0 + R[6] * a1) + R[10] * a2;
    /* Proj into the target camera. */
    const float X = ((Q[0] * xw + Q[1] * yw) + Q[2] * zw) + Q[3];
    const float Y = ((Q[4] * xw + Q[5] * yw) + Q[6] * zw) + Q[7];
    const float Z = ((Q[8] * xw + Q[9] * yw) + Q[10] * zw) + Q[11];
    if (!(Z > (float)t->near_plane)) return 0;
    *u = ((float)t->fx * X) / Z + (float)t->cx;
    *v = ((float)t->fy * Y) / Z + (float)t->cy;
    *z = Z;
    return 1;
}

/* The same map in FP64 (same moving-pixel rule, decided in fp32 as above). */
static int warp_pos64(const or_camera *s, const or_camera *t, const double *depth, const double *alpha,
                      double alpha_min, int W, int i, int j, double *u, double *v, double *z)
{
    const int64_t p = (int64_t)j * W + i;
    double d;
    if (alpha) {
        if (!((float)alpha[p] > (float)alpha_min)) return 0;
        d = depth[p] / alpha[p];
    } else {
        if (!((float)depth[p] > 0.0f)) return 0;
        d = depth[p];
    }
    const double *R = s->viewmat, *Q = t->viewmat;
    const double cam[3] = {(i + 0.5 - s->cx) / s->fx * d, (j + 0.5 - s->cy) / s->fy * d, d};
    double w[3];
    for (int r = 0; r < 3; ++r)
        w[r] = R[0 * 4 + r] * (cam[0] - R[3]) + R[1 * 4 + r] * (cam[1] - R[7]) + R[2 * 4 + r] * (cam[2] - R[11]);
    double c[3];
    for (int r = 0; r < 3; ++r) c[r] = Q[r * 4 + 0] * w[0] + Q[r * 4 + 1] * w[1] + Q[r * 4 + 2] * w[2] + Q[r * 4 + 3];
    if (!(c[2] > t->near_plane)) return 0;
    *u = t->fx * c[0] / c[2] + t->cx;
    *v = t->fy * c[1] / c[2] + t->cy;
    *z = c[2];
    return 1;
}

/* Motion vectors, forward warp and warped gradients of one source frame.
 *   depth, alpha      [H][W] (alpha may be NULL: depth is then a point depth)
 *   planes            [channels][H][W], carried to the target by the warp
 *   dcdx, dcdy        [gch][H][W] source image gradients (NULL when gch == 0)
 * Outputs (any may be NULL):
 *   motion            [2][H][W] fp32 spec V, NaN where the pixel does not move
 *   motion64          [2][H][W] FP64 V, NaN where the pixel does not move
 *   index             [Ht][Wt]  winning source pixel j*W+i, -1 for a hole
 *   zdst              [Ht][Wt]  the winner's target-camera z (fp32 spec), 0 for a hole
 *   out               [channels][Ht][Wt]
 *   out_dcdx/out_dcdy [gch][Ht][Wt]
 *   jac               [4][Ht][Wt]  the Jacobian J used at each target pixel (J00, J01, J10, J11;
 *                                  the identity at holes), computed whether or not gch > 0 */
int or_warp(const or_camera *src, const or_camera *dst, const double *depth, const double *alpha,
            double alpha_min, int32_t channels, const double *planes, int32_t gch, const double *dcdx,
            const double *dcdy, float *motion, double *motion64, int32_t *index, float *zdst, double *out,
            double *out_dcdx, double *out_dcdy, double *jac)
{
    const int W = src->width, H = src->height, Wt = dst->width, Ht = dst->height;
    const int64_t n = (int64_t)W * H, nt = (int64_t)Wt * Ht;
    float *pu = malloc(sizeof(float) * (size_t)(n ? n : 1));
    float *pv = malloc(sizeof(float) * (size_t)(n ? n : 1));
    float *pz = malloc(sizeof(float) * (size_t)(n ? n : 1));
    unsigned char *mv = malloc((size_t)(n ? n : 1));
    uint64_t *best = malloc(sizeof(uint64_t) * (size_t)(nt ? nt : 1));
    if (!pu || !pv || !pz || !mv || !best) {
        free(pu); free(pv); free(pz); free(mv); free(best);
        return -1;
    }
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            const int64_t p = (int64_t)j * W + i;
            mv[p] = (unsigned char)warp_pos32(src, dst, depth, alpha, alpha_min, W, i, j, &pu[p], &pv[p], &pz[p]);
            if (motion) {
                motion[p] = mv[p] ? pu[p] - ((float)i + 0.5f) : NAN;
                motion[n + p] = mv[p] ? pv[p] - ((float)j + 0.5f) : NAN;
            }
            if (motion64) {
                double u, v, z;
                if (warp_pos64(src, dst, depth, alpha, alpha_min, W, i, j, &u, &v, &z)) {
                    motion64[p] = u - (i + 0.5);
                    motion64[n + p] = v - (j + 0.5);
                } else {
                    motion64[p] = motion64[n + p] = NAN;
                }
            }
        }
    /* The depth test: scatter every moving pixel into its target pixel. */
    for (int64_t q = 0; q < nt; ++q) best[q] = UINT64_MAX;
    for (int64_t p = 0; p < n; ++p) {
        if (!mv[p]) continue;
        if (!(pu[p] >= 0.0f && pu[p] < (float)Wt && pv[p] >= 0.0f && pv[p] < (float)Ht)) continue;
        const int64_t q = (int64_t)floorf(pv[p]) * Wt + (int64_t)floorf(pu[p]);
        uint32_t zb;
        memcpy(&zb, &pz[p], 4);
        const uint64_t key = ((uint64_t)zb << 32) | (uint64_t)p;
        if (key < best[q]) best[q] = key;
    }
    for (int64_t q = 0; q < nt; ++q) {
        const int hole = best[q] == UINT64_MAX;
        const int64_t p = hole ? -1 : (int64_t)(best[q] & 0xFFFFFFFFu);
        if (index) index[q] = (int32_t)p;
        if (zdst) zdst[q] = hole ? 0.0f : pz[p];
        if (out)
            for (int c = 0; c < channels; ++c) out[c * nt + q] = hole ? 0.0 : planes[c * n + p];
        if ((gch <= 0 || !out_dcdx || !out_dcdy) && !jac) continue;
        double J[4] = {1.0, 0.0, 0.0, 1.0}, det = 1.0;  /* J = [[du/dx, du/dy], [dv/dx, dv/dy]] */
        if (!hole) {
            const int i = (int)(p % W), j = (int)(p / W);
            /* d(position)/dx: neighbours left/right in the source row */
            const int L = i > 0 && mv[p - 1], Rn = i < W - 1 && mv[p + 1];
            if (L && Rn) {
                J[0] = ((double)pu[p + 1] - (double)pu[p - 1]) * 0.5;
                J[2] = ((double)pv[p + 1] - (double)pv[p - 1]) * 0.5;
            } else if (Rn) {
                J[0] = (double)pu[p + 1] - (double)pu[p];
                J[2] = (double)pv[p + 1] - (double)pv[p];
            } else if (L) {
                J[0] = (double)pu[p] - (double)pu[p - 1];
                J[2] = (double)pv[p] - (double)pv[p - 1];
            }
            /* d(position)/dy: neighbours above/below */
            const int U = j > 0 && mv[p - W], D = j < H - 1 && mv[p + W];
            if (U && D) {
                J[1] = ((double)pu[p + W] - (double)pu[p - W]) * 0.5;
                J[3] = ((double)pv[p + W] - (double)pv[p - W]) * 0.5;
            } else if (D) {
                J[1] = (double)pu[p + W] - (double)pu[p];
                J[3] = (double)pv[p + W] - (double)pv[p];
            } else if (U) {
                J[1] = (double)pu[p] - (double)pu[p - W];
                J[3] = (double)pv[p] - (double)pv[p - W];
            }
            det = J[0] * J[3] - J[1] * J[2];
        }
        if (jac)
            for (int k = 0; k < 4; ++k) jac[k * nt + q] = J[k];
        if (gch <= 0 || !out_dcdx || !out_dcdy) continue;
        for (int c = 0; c < gch; ++c) {
            double gx = 0.0, gy = 0.0;
            if (!hole && det > 0.0) {
                const double g0 = dcdx[c * n + p], g1 = dcdy[c * n + p];
                /* (g0, g1) . J^-1, J^-1 = [[J3, -J1], [-J2, J0]] / det */
                gx = (g0 * J[3] - g1 * J[2]) / det;
                gy = (g1 * J[0] - g0 * J[1]) / det;
            }
            out_dcdx[c * nt + q] = gx;
            out_dcdy[c * nt + q] = gy;
        }
    }
    free(pu); free(pv); free(pz); free(mv); free(best);
    return 0;
}
