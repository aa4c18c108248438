/*
 * orc_gaussians.c -- oracle: Gaussian projection, culling and rasterisation
 * into the sweeping planes.
 * TEST INFRASTRUCTURE ONLY (see lf_oracle.h).
 *
 * Sec. 4.4 (G2LF): primitives inside the reference frustum, their reference
 * depth, one chunk per primitive by centre depth, per-chunk alpha blending.
 * The per-Gaussian projection is the EWA splatting of 3DGS [kerbl20233d],
 * which the paper uses unchanged except for the dilation f' of
 * Eq. (gs_prefilter_fix).
 */
#include "lf_oracle.h"

#include <math.h>
#include <string.h>
#include <stdlib.h>

/* Reference depth in FP64 with a fixed fma order:
 *   z = fma(R20, x, fma(R21, y, fma(R22, z_w, t2))) - D_forward.
 * Shared as a definition (not as code) with the CUDA library, which must
 * produce the same bits because chunk membership depends on them. */
static double ref_depth(const orc_ref* r, const float* m)
{
    const double* R = r->cam.R;
    const double zc = fma(R[6], (double)m[0], fma(R[7], (double)m[1], fma(R[8], (double)m[2], r->cam.t[2])));
    return zc - r->D_forward;
}

/* Footprint rectangle of one Gaussian, decided in FP32 (the kernel's
 * precision) with a fixed operation order. The region is the 3-sigma square
 * of 3DGS, r = ceil(3 sqrt(lambda_max)), clipped to the plane.
 * Reading: a Gaussian touches exactly the plane pixels inside this
 * rectangle (not whole tiles), so results do not depend on tile shape.
 * Returns 1 and fills rect if culled in. */
static int gauss_rect_f32(const orc_ref* r, const float* m, const float* s, const float* q,
                          double z64, int32_t* rect)
{
    const double* Rd = r->cam.R;
    float R[9];
    for (int i = 0; i < 9; ++i) R[i] = (float)Rd[i];
    const float t0 = (float)r->cam.t[0];
    const float t1 = (float)r->cam.t[1];
    const float fxf = (float)r->fx, fyf = (float)r->fy;
    const float cxf = (float)r->cx, cyf = (float)r->cy;
    const float fpf = (float)r->f_prime;

    const float xc = fmaf(R[0], m[0], fmaf(R[1], m[1], fmaf(R[2], m[2], t0)));
    const float yc = fmaf(R[3], m[0], fmaf(R[4], m[1], fmaf(R[5], m[2], t1)));
    const float zc = (float)z64;

    /* unit quaternion (w, x, y, z) */
    const float n2 = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3])));
    const float inv = 1.0f / sqrtf(n2);
    const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z;
    const float wx = w * x, wy = w * y, wz = w * z;
    float Q[9];
    Q[0] = 1.0f - 2.0f * (yy + zz);
    Q[1] = 2.0f * (xy - wz);
    Q[2] = 2.0f * (xz + wy);
    Q[3] = 2.0f * (xy + wz);
    Q[4] = 1.0f - 2.0f * (xx + zz);
    Q[5] = 2.0f * (yz - wx);
    Q[6] = 2.0f * (xz - wy);
    Q[7] = 2.0f * (yz + wx);
    Q[8] = 1.0f - 2.0f * (xx + yy);

    /* M = Q diag(s), V = R_cam M (camera-frame square root of Sigma_3) */
    float M[9], V[9];
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) M[3 * i + l] = Q[3 * i + l] * s[l];
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l)
            V[3 * i + l] = fmaf(R[3 * i + 0], M[l], fmaf(R[3 * i + 1], M[3 + l], R[3 * i + 2] * M[6 + l]));

    /* U = J V with the EWA Jacobian J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
    const float iz = 1.0f / zc;
    const float xn = xc * iz, yn = yc * iz;
    const float ax = fxf * iz, ay = fyf * iz;
    float U0[3], U1[3];
    for (int l = 0; l < 3; ++l) {
        U0[l] = ax * fmaf(-xn, V[6 + l], V[0 + l]);
        U1[l] = ay * fmaf(-yn, V[6 + l], V[3 + l]);
    }
    const float S00 = fmaf(U0[0], U0[0], fmaf(U0[1], U0[1], U0[2] * U0[2])) + fpf;
    const float S01 = fmaf(U0[0], U1[0], fmaf(U0[1], U1[1], U0[2] * U1[2]));
    const float S11 = fmaf(U1[0], U1[0], fmaf(U1[1], U1[1], U1[2] * U1[2])) + fpf;
    const float det = fmaf(S00, S11, -(S01 * S01));
    if (!(det > 0.0f)) return 0;
    const float mid = 0.5f * (S00 + S11);
    const float lam = mid + sqrtf(fmaxf(fmaf(mid, mid, -det), 0.0f));
    const float rad = ceilf(3.0f * sqrtf(lam));
    const float px = fmaf(fxf, xn, cxf);
    const float py = fmaf(fyf, yn, cyf);

    const float fx0 = ceilf(px - rad), fx1 = floorf(px + rad);
    const float fy0 = ceilf(py - rad), fy1 = floorf(py + rad);
    const float wmax = (float)(r->W - 1), hmax = (float)(r->H - 1);
    if (!(fx0 <= wmax && fx1 >= 0.0f && fy0 <= hmax && fy1 >= 0.0f)) return 0;
    rect[0] = (int32_t)fmaxf(fx0, 0.0f);
    rect[1] = (int32_t)fmaxf(fy0, 0.0f);
    rect[2] = (int32_t)fminf(fx1, wmax);
    rect[3] = (int32_t)fminf(fy1, hmax);
    return 1;
}

void orc_gauss_decide(const orc_ref* r, int64_t n, const float* means, const float* scales,
                      const float* quats, double* z, uint8_t* valid, int32_t* rect)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        const double zg = ref_depth(r, means + 3 * g);
        z[g] = zg;
        valid[g] = 0;
        rect[4 * g + 0] = rect[4 * g + 1] = 0;
        rect[4 * g + 2] = rect[4 * g + 3] = -1;
        /* culled when not in front of the near plane */
        if (!(zg > r->disp.z_near)) continue;
        valid[g] = (uint8_t)gauss_rect_f32(r, means + 3 * g, scales + 3 * g, quats + 4 * g, zg,
                                           rect + 4 * g);
        if (!valid[g]) {
            rect[4 * g + 0] = rect[4 * g + 1] = 0;
            rect[4 * g + 2] = rect[4 * g + 3] = -1;
        }
    }
}

/* EWA projection in FP64 (values): Sigma_3 = Q S^2 Q^T in the world frame,
 * Sigma_cam = R Sigma_3 R^T, Sigma_2 = J Sigma_cam J^T + f' I, 2D mean
 * (fx x/z + cx, fy y/z + cy); conic = Sigma_2^{-1}. */
void orc_gauss_values(const orc_ref* r, int64_t n, const double* means, const double* scales,
                      const double* quats, double* mean2d, double* conic, double* cov2d)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        const double* m = means + 3 * g;
        const double* R = r->cam.R;
        const double* t = r->cam.t;
        double pc[3];
        for (int i = 0; i < 3; ++i)
            pc[i] = R[3 * i] * m[0] + R[3 * i + 1] * m[1] + R[3 * i + 2] * m[2] + t[i];
        pc[2] -= r->D_forward;

        const double* qf = quats + 4 * g;
        double qn = sqrt(qf[0] * qf[0] + qf[1] * qf[1] + qf[2] * qf[2] + qf[3] * qf[3]);
        const double w = qf[0] / qn, x = qf[1] / qn, y = qf[2] / qn, z = qf[3] / qn;
        const double Q[3][3] = {
            {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        const double s2[3] = {scales[3 * g] * scales[3 * g], scales[3 * g + 1] * scales[3 * g + 1],
                              scales[3 * g + 2] * scales[3 * g + 2]};
        double S3[3][3], Sc[3][3], tmp[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += Q[i][l] * s2[l] * Q[j][l];
                S3[i][j] = acc;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += R[3 * i + l] * S3[l][j];
                tmp[i][j] = acc;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += tmp[i][l] * R[3 * j + l];
                Sc[i][j] = acc;
            }
        const double zz = pc[2];
        const double J[2][3] = {{r->fx / zz, 0.0, -r->fx * pc[0] / (zz * zz)},
                                {0.0, r->fy / zz, -r->fy * pc[1] / (zz * zz)}};
        double S2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) acc += J[a][i] * Sc[i][j] * J[b][j];
                S2[a][b] = acc;
            }
        S2[0][0] += r->f_prime;
        S2[1][1] += r->f_prime;
        const double det = S2[0][0] * S2[1][1] - S2[0][1] * S2[1][0];
        mean2d[2 * g + 0] = r->fx * pc[0] / zz + r->cx;
        mean2d[2 * g + 1] = r->fy * pc[1] / zz + r->cy;
        conic[3 * g + 0] = S2[1][1] / det;
        conic[3 * g + 1] = -S2[0][1] / det;
        conic[3 * g + 2] = S2[0][0] / det;
        if (cov2d) {
            cov2d[3 * g + 0] = S2[0][0];
            cov2d[3 * g + 1] = S2[0][1];
            cov2d[3 * g + 2] = S2[1][1];
        }
    }
}

/* Sec. 4.4 / the per-chunk rendering step of Algorithm 1: each chunk is rendered alone
 * into its plane, front to back in (depth, index) order:
 *   alpha = min(0.99, o exp(-q/2)),  q = d^T Sigma_2^{-1} d,  d = p - mean2d,
 *   C += T alpha rgb,  T *= (1 - alpha);  texel = (C, 1 - T).
 * Reading: no alpha < 1/255 skip and no early stop (exact mode). Visiting the
 * members in order and updating every pixel of each member's rectangle gives
 * each pixel exactly its ordered sequence of contributions. */
void orc_splat_gaussians(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                         const int32_t* rect, const double* mean2d, const double* conic,
                         const double* opacity, const double* rgb, int32_t N, double* planes)
{
    const int64_t W = r->W, H = r->H;
    const int64_t plane_sz = W * H * 4;
    memset(planes, 0, sizeof(double) * (size_t)(plane_sz * N));

    /* member range of every chunk in the sorted order */
    int64_t start[N + 1];
    {
        int64_t k = 0;
        start[0] = 0;
        for (int64_t i = 0; i < M; ++i) {
            while (k < chunk[order[i]]) start[++k] = i;
        }
        while (k < N) start[++k] = M;
    }

#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t k = 0; k < N; ++k) {
        double* P = planes + plane_sz * k;
        /* P[.][3] holds T during accumulation */
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0;
        for (int64_t i = start[k]; i < start[k + 1]; ++i) {
            const int64_t g = order[i];
            const int32_t* rc = rect + 4 * g;
            const double mx = mean2d[2 * g], my = mean2d[2 * g + 1];
            const double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
            const double o = opacity[g];
            for (int32_t y = rc[1]; y <= rc[3]; ++y) {
                for (int32_t x = rc[0]; x <= rc[2]; ++x) {
                    const double dx = (double)x - mx, dy = (double)y - my;
                    const double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
                    double al = o * exp(-0.5 * q);
                    if (al > 0.99) al = 0.99;
                    double* px = P + 4 * (y * W + x);
                    const double T = px[3];
                    px[0] += T * al * rgb[3 * g + 0];
                    px[1] += T * al * rgb[3 * g + 1];
                    px[2] += T * al * rgb[3 * g + 2];
                    px[3] = T * (1.0 - al);
                }
            }
        }
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0 - P[4 * p + 3];
    }
}

/* The 3DGS cut-offs on top of the splat above (same member order, same
 * alpha): skip a member with alpha < 1/255; when T (1 - alpha) would fall
 * below 1e-4, the pixel is finished and blends nothing more. */
void orc_splat_gaussians_3dgs(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                              const int32_t* rect, const double* mean2d, const double* conic,
                              const double* opacity, const double* rgb, int32_t N, double* planes,
                              uint8_t* near)
{
    const double a_min = 1.0 / 255.0, t_min = 1e-4, window = 1e-6;
    const int64_t W = r->W, H = r->H;
    const int64_t plane_sz = W * H * 4;
    memset(planes, 0, sizeof(double) * (size_t)(plane_sz * N));
    if (near) memset(near, 0, (size_t)(W * H * N));

    int64_t start[N + 1];
    {
        int64_t k = 0;
        start[0] = 0;
        for (int64_t i = 0; i < M; ++i) {
            while (k < chunk[order[i]]) start[++k] = i;
        }
        while (k < N) start[++k] = M;
    }

#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t k = 0; k < N; ++k) {
        double* P = planes + plane_sz * k;
        uint8_t* done = (uint8_t*)calloc((size_t)(W * H), 1);
        uint8_t* nr = near ? near + W * H * k : NULL;
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0;
        for (int64_t i = start[k]; i < start[k + 1]; ++i) {
            const int64_t g = order[i];
            const int32_t* rc = rect + 4 * g;
            const double mx = mean2d[2 * g], my = mean2d[2 * g + 1];
            const double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
            const double o = opacity[g];
            for (int32_t y = rc[1]; y <= rc[3]; ++y) {
                for (int32_t x = rc[0]; x <= rc[2]; ++x) {
                    const int64_t p = (int64_t)y * W + x;
                    if (done[p]) continue;
                    const double dx = (double)x - mx, dy = (double)y - my;
                    const double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
                    double al = o * exp(-0.5 * q);
                    if (al > 0.99) al = 0.99;
                    if (nr && fabs(al - a_min) <= window) nr[p] = 1;
                    if (al < a_min) continue;
                    double* px = P + 4 * p;
                    const double T = px[3];
                    const double Tn = T * (1.0 - al);
                    if (nr && fabs(Tn - t_min) <= window) nr[p] = 1;
                    if (Tn < t_min) {
                        done[p] = 1;
                        continue;
                    }
                    px[0] += T * al * rgb[3 * g + 0];
                    px[1] += T * al * rgb[3 * g + 1];
                    px[2] += T * al * rgb[3 * g + 2];
                    px[3] = Tn;
                }
            }
        }
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0 - P[4 * p + 3];
        free(done);
    }
}
