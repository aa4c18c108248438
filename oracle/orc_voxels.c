/*
 * orc_voxels.c -- oracle: sparse-voxel projection, culling and rasterisation
 * into the sweeping planes (V2LF).
 * TEST INFRASTRUCTURE ONLY (see lf_oracle.h).
 *
 * Sec. 4.5: sparse voxels are primitives chunked like Gaussians (Sec. 4.4);
 * each voxel is rendered by the volume-rendering integral of its trilinear
 * density along the plane pixel's reference ray (the SVR model
 * [sun2024sparse], which the paper reuses unchanged).
 */
#include "lf_oracle.h"

#include <math.h>
#include <string.h>

static void voxel_box(const int32_t* ijk, uint8_t level, const double* origin, double base_size,
                      double* lo, double* side)
{
    const double s = ldexp(base_size, -(int)level);
    *side = s;
    for (int a = 0; a < 3; ++a) lo[a] = origin[a] + (double)ijk[a] * s;
}

void orc_voxel_decide(const orc_ref* r, int64_t n, const int32_t* ijk, const uint8_t* level,
                      const double* origin, double base_size,
                      double* z, uint8_t* valid, int32_t* rect)
{
    const double* R = r->cam.R;
    const double rho = fabs(R[6]) + fabs(R[7]) + fabs(R[8]);
    float Rf[9];
    for (int i = 0; i < 9; ++i) Rf[i] = (float)R[i];
    const float t0 = (float)r->cam.t[0], t1 = (float)r->cam.t[1];
    const float t2r = (float)(r->cam.t[2] - r->D_forward);
    const float fxf = (float)r->fx, fyf = (float)r->fy;
    const float cxf = (float)r->cx, cyf = (float)r->cy;
    const float wmax = (float)(r->W - 1), hmax = (float)(r->H - 1);

#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        double lo[3], s;
        voxel_box(ijk + 3 * v, level[v], origin, base_size, lo, &s);
        const double c[3] = {lo[0] + 0.5 * s, lo[1] + 0.5 * s, lo[2] + 0.5 * s};
        /* centre depth: same fixed fma order as for Gaussians */
        const double zv = fma(R[6], c[0], fma(R[7], c[1], fma(R[8], c[2], r->cam.t[2]))) - r->D_forward;
        z[v] = zv;
        valid[v] = 0;
        rect[4 * v + 0] = rect[4 * v + 1] = 0;
        rect[4 * v + 2] = rect[4 * v + 3] = -1;
        /* nearest corner depth; culled unless the whole cube is past z_near */
        const double zmin = zv - (0.5 * s) * rho;
        if (!(zmin > r->disp.z_near)) continue;

        /* FP32 footprint: bounding box of the 8 projected corners; the pixels
         * whose centres fall inside it are the only ones whose ray can meet
         * the cube. */
        float mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
        for (int cidx = 0; cidx < 8; ++cidx) {
            const float X = (float)(lo[0] + (double)(cidx & 1) * s);
            const float Y = (float)(lo[1] + (double)((cidx >> 1) & 1) * s);
            const float Z = (float)(lo[2] + (double)((cidx >> 2) & 1) * s);
            const float xc = fmaf(Rf[0], X, fmaf(Rf[1], Y, fmaf(Rf[2], Z, t0)));
            const float yc = fmaf(Rf[3], X, fmaf(Rf[4], Y, fmaf(Rf[5], Z, t1)));
            const float zc = fmaf(Rf[6], X, fmaf(Rf[7], Y, fmaf(Rf[8], Z, t2r)));
            const float iz = 1.0f / zc;
            const float px = fmaf(fxf, xc * iz, cxf);
            const float py = fmaf(fyf, yc * iz, cyf);
            mnx = fminf(mnx, px);
            mxx = fmaxf(mxx, px);
            mny = fminf(mny, py);
            mxy = fmaxf(mxy, py);
        }
        const float fx0 = ceilf(mnx), fx1 = floorf(mxx);
        const float fy0 = ceilf(mny), fy1 = floorf(mxy);
        if (!(fx0 <= fx1 && fy0 <= fy1)) continue;
        if (!(fx0 <= wmax && fx1 >= 0.0f && fy0 <= hmax && fy1 >= 0.0f)) continue;
        rect[4 * v + 0] = (int32_t)fmaxf(fx0, 0.0f);
        rect[4 * v + 1] = (int32_t)fmaxf(fy0, 0.0f);
        rect[4 * v + 2] = (int32_t)fminf(fx1, wmax);
        rect[4 * v + 3] = (int32_t)fminf(fy1, hmax);
        valid[v] = 1;
    }
}

/* Trilinear density inside the cube at local coordinates f in [0,1]^3.
 * Corner c = i + 2 j + 4 k holds the density at offset (i, j, k). */
static double trilinear(const double* rho8, const double* f)
{
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        const double wx = (c & 1) ? f[0] : 1.0 - f[0];
        const double wy = ((c >> 1) & 1) ? f[1] : 1.0 - f[1];
        const double wz = ((c >> 2) & 1) ? f[2] : 1.0 - f[2];
        acc += wx * wy * wz * rho8[c];
    }
    return acc;
}

static void local_coords(const double* lo, double side, const double* o, const double* dir,
                         double t, double* f)
{
    for (int a = 0; a < 3; ++a) {
        double v = (o[a] + t * dir[a] - lo[a]) / side;
        f[a] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
}

/* alpha = 1 - exp(-integral of sigma over the ray segment inside the cube).
 * Along a line the trilinear density is a cubic polynomial in t, so
 * Simpson's rule over the segment is exact. */
double orc_voxel_alpha(const double* lo, double side, const double* density8,
                       const double* o, const double* dir, double* seg_len)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const double hi = lo[a] + side;
        if (dir[a] != 0.0) {
            double ta = (lo[a] - o[a]) / dir[a];
            double tb = (hi - o[a]) / dir[a];
            if (ta > tb) { const double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        } else if (o[a] < lo[a] || o[a] > hi) {
            if (seg_len) *seg_len = 0.0;
            return 0.0;
        }
    }
    if (t0 < 0.0) t0 = 0.0;
    if (!(t1 > t0)) {
        if (seg_len) *seg_len = 0.0;
        return 0.0;
    }
    double f0[3], fm[3], f1[3];
    local_coords(lo, side, o, dir, t0, f0);
    local_coords(lo, side, o, dir, 0.5 * (t0 + t1), fm);
    local_coords(lo, side, o, dir, t1, f1);
    const double len = t1 - t0;
    const double integral = len / 6.0 * (trilinear(density8, f0) + 4.0 * trilinear(density8, fm) +
                                         trilinear(density8, f1));
    if (seg_len) *seg_len = len;
    return 1.0 - exp(-integral);
}

void orc_splat_voxels(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                      const int32_t* rect, const int32_t* ijk, const uint8_t* level,
                      const double* origin, double base_size, const double* density8,
                      const double* rgb, int32_t N, double* planes)
{
    const int64_t W = r->W, H = r->H;
    const int64_t plane_sz = W * H * 4;
    memset(planes, 0, sizeof(double) * (size_t)(plane_sz * N));
    const double* R = r->cam.R;
    const double* t = r->cam.t;
    /* reference camera centre in world coordinates: R o + t - D_forward e_z = 0 */
    double o[3];
    {
        const double b[3] = {-t[0], -t[1], r->D_forward - t[2]};
        for (int i = 0; i < 3; ++i) o[i] = R[i] * b[0] + R[3 + i] * b[1] + R[6 + i] * b[2];
    }

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
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0;
        for (int64_t i = start[k]; i < start[k + 1]; ++i) {
            const int64_t v = order[i];
            const int32_t* rc = rect + 4 * v;
            double lo[3], s;
            voxel_box(ijk + 3 * v, level[v], origin, base_size, lo, &s);
            for (int32_t y = rc[1]; y <= rc[3]; ++y) {
                for (int32_t x = rc[0]; x <= rc[2]; ++x) {
                    /* reference ray through the plane pixel centre */
                    const double dc[3] = {((double)x - r->cx) / r->fx, ((double)y - r->cy) / r->fy, 1.0};
                    double dw[3];
                    for (int a = 0; a < 3; ++a) dw[a] = R[a] * dc[0] + R[3 + a] * dc[1] + R[6 + a] * dc[2];
                    const double nrm = sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
                    for (int a = 0; a < 3; ++a) dw[a] /= nrm;
                    const double al = orc_voxel_alpha(lo, s, density8 + 8 * v, o, dw, NULL);
                    double* px = P + 4 * (y * W + x);
                    const double T = px[3];
                    px[0] += T * al * rgb[3 * v + 0];
                    px[1] += T * al * rgb[3 * v + 1];
                    px[2] += T * al * rgb[3 * v + 2];
                    px[3] = T * (1.0 - al);
                }
            }
        }
        for (int64_t p = 0; p < W * H; ++p) P[4 * p + 3] = 1.0 - P[4 * p + 3];
    }
}
