/*
 * orc_composite.c -- oracle: depth binning into chunks and swizzle blending.
 * TEST INFRASTRUCTURE ONLY (see lf_oracle.h).
 *
 * Sec. 4.4 (quantile binning, median plane distance), the culling, depth-sort
 * and chunking steps of Algorithm 1;
 * Sec. 4.3 swizzle blending, Eq. (u_prime), Eq. (alpha_blend),
 * the compositing steps of Algorithm 1.
 */
#include "lf_oracle.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double z;
    int64_t idx;
} zkey;

static int cmp_zkey(const void* a, const void* b)
{
    const zkey* x = (const zkey*)a;
    const zkey* y = (const zkey*)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Binning.
 * Quantile (Sec. 4.4): sort culled-in primitives by reference depth (ties by
 * index -- reading), split the sorted list into N chunks of nearly equal size
 * (rank r goes to chunk floor(r N / M)), plane distance d_k = median depth of
 * chunk k (mean of the two middle values for an even count -- reading).
 * Disparity (reading for the uniform-in-disparity configuration): N equal
 * bins in 1/z between the nearest and farthest culled-in depth,
 * chunk = min(N-1, floor(N (1/z_min - 1/z) / (1/z_min - 1/z_max))), d_k at
 * the bin's disparity midpoint.
 * d_k is returned in the BASE camera frame (reference depth + D_forward),
 * the frame Eq. (u_prime) measures d_k in. Empty chunks get d_k = 0. */
int64_t orc_bin(const orc_ref* r, int64_t n, const double* z, const uint8_t* valid,
                int32_t N, int32_t mode, int64_t* order, int32_t* chunk, double* d,
                int64_t* count)
{
    zkey* keys = (zkey*)malloc(sizeof(zkey) * (size_t)(n > 0 ? n : 1));
    int64_t M = 0;
    for (int64_t g = 0; g < n; ++g) {
        chunk[g] = -1;
        if (valid[g]) {
            keys[M].z = z[g];
            keys[M].idx = g;
            ++M;
        }
    }
    qsort(keys, (size_t)M, sizeof(zkey), cmp_zkey);
    for (int64_t i = 0; i < M; ++i) order[i] = keys[i].idx;
    for (int32_t k = 0; k < N; ++k) {
        d[k] = 0.0;
        count[k] = 0;
    }
    if (M == 0) {
        free(keys);
        return 0;
    }

    if (mode == 0) {
        for (int64_t i = 0; i < M; ++i) {
            const int32_t k = (int32_t)((i * (int64_t)N) / M);
            chunk[keys[i].idx] = k;
            count[k] += 1;
        }
        int64_t lo = 0;
        for (int32_t k = 0; k < N; ++k) {
            const int64_t c = count[k];
            if (c > 0) {
                double med;
                if (c & 1)
                    med = keys[lo + c / 2].z;
                else
                    med = (keys[lo + c / 2 - 1].z + keys[lo + c / 2].z) * 0.5;
                d[k] = med + r->D_forward;
            }
            lo += c;
        }
    } else {
        const double zmin = keys[0].z, zmax = keys[M - 1].z;
        const double izmin = 1.0 / zmin, izmax = 1.0 / zmax;
        const double span = izmin - izmax;
        for (int64_t i = 0; i < M; ++i) {
            int32_t k = 0;
            if (span > 0.0) {
                const double f = floor((double)N * (izmin - 1.0 / keys[i].z) / span);
                k = f >= (double)(N - 1) ? N - 1 : (int32_t)f;
            }
            chunk[keys[i].idx] = k;
            count[k] += 1;
        }
        for (int32_t k = 0; k < N; ++k) {
            /* disparity at the middle of bin k */
            const double disp = izmin - ((double)k + 0.5) / (double)N * span;
            d[k] = 1.0 / disp + r->D_forward;
        }
    }
    free(keys);
    return M;
}

/* One plane sample for the bilinear case: taps outside the plane are
 * transparent zeros (reading: zero padding). */
static void sample_bilinear(const double* P, int32_t W, int32_t H, double X, double Y, double* out)
{
    const double x0f = floor(X), y0f = floor(Y);
    const double wx = X - x0f, wy = Y - y0f;
    const int64_t x0 = (int64_t)x0f, y0 = (int64_t)y0f;
    for (int c = 0; c < 4; ++c) out[c] = 0.0;
    for (int dy = 0; dy < 2; ++dy) {
        for (int dx = 0; dx < 2; ++dx) {
            const int64_t xx = x0 + dx, yy = y0 + dy;
            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
            const double w = (dx ? wx : 1.0 - wx) * (dy ? wy : 1.0 - wy);
            const double* t = P + 4 * (yy * W + xx);
            for (int c = 0; c < 4; ++c) out[c] += w * t[c];
        }
    }
}

/* Swizzle blending (the compositing steps of Algorithm 1): for every quilt view (i, j)
 * and pixel (x, y), walk the planes front to back, sample each at its
 * Eq. (u_prime) location and composite
 *   Q <- Q + T c_k,  T <- T (1 - A_k)      (Eq. (alpha_blend), c_k premultiplied).
 * Nearest sampling takes its index from the FP32 decision form of
 * Eq. (u_prime) (orc_axis_coeffs), the precision the kernel decides in;
 * bilinear sampling uses the FP64 coordinate straight from Eq. (u_prime).
 * Empty chunks are skipped. Output (Q + T bg, 1 - T). */
void orc_composite(const orc_ref* r, int32_t N, const double* planes, const double* d,
                   const int64_t* count, int32_t Vx, int32_t Vy, int32_t bilinear,
                   const double* bg, double* views)
{
    const int32_t Nx = r->cam.Nx, Ny = r->cam.Ny, W = r->W, H = r->H;
    const int64_t plane_sz = (int64_t)W * H * 4;
    double* dx = (double*)malloc(sizeof(double) * (size_t)Vx);
    double* dy = (double*)malloc(sizeof(double) * (size_t)Vy);
    orc_view_offsets(r, Vx, Vy, dx, dy);

    /* Quilt2PlaneCoordinate(H, d_k) per view column / row and plane (the
     * map depends on (j, k) horizontally and (i, k) vertically only). */
    float* gmx = (float*)calloc((size_t)Vx * (size_t)N, sizeof(float));
    float* hnx = (float*)calloc((size_t)Vx * (size_t)N, sizeof(float));
    float* gmy = (float*)calloc((size_t)Vy * (size_t)N, sizeof(float));
    float* hny = (float*)calloc((size_t)Vy * (size_t)N, sizeof(float));
    for (int32_t k = 0; k < N; ++k) {
        if (count[k] == 0) continue;
        float hb;
        for (int32_t j = 0; j < Vx; ++j)
            orc_axis_coeffs(r, 0, dx[j], d[k], &gmx[j * N + k], &hnx[j * N + k], &hb);
        for (int32_t i = 0; i < Vy; ++i)
            orc_axis_coeffs(r, 1, dy[i], d[k], &gmy[i * N + k], &hny[i * N + k], &hb);
    }

#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int32_t v = 0; v < Vx * Vy; ++v) {
        for (int32_t y = 0; y < Ny; ++y) {
            const int32_t i = v / Vx, j = v % Vx;
            for (int32_t x = 0; x < Nx; ++x) {
                double Q[3] = {0.0, 0.0, 0.0};
                double T = 1.0;
                for (int32_t k = 0; k < N; ++k) {
                    if (count[k] == 0) continue;
                    const double* P = planes + plane_sz * k;
                    double c[4] = {0.0, 0.0, 0.0, 0.0};
                    if (bilinear) {
                        const double X = orc_plane_pixel(r, 0, dx[j], d[k], x);
                        const double Y = orc_plane_pixel(r, 1, dy[i], d[k], y);
                        sample_bilinear(P, W, H, X, Y, c);
                    } else {
                        const int32_t ix = orc_nearest_index(r, gmx[j * N + k], hnx[j * N + k], x);
                        const int32_t iy = orc_nearest_index(r, gmy[i * N + k], hny[i * N + k], y);
                        if (ix >= 0 && ix < W && iy >= 0 && iy < H) {
                            const double* t = P + 4 * ((int64_t)iy * W + ix);
                            for (int cc = 0; cc < 4; ++cc) c[cc] = t[cc];
                        }
                    }
                    Q[0] += T * c[0];
                    Q[1] += T * c[1];
                    Q[2] += T * c[2];
                    T *= 1.0 - c[3];
                }
                double* o = views + 4 * (((int64_t)v * Ny + y) * Nx + x);
                o[0] = Q[0] + T * bg[0];
                o[1] = Q[1] + T * bg[1];
                o[2] = Q[2] + T * bg[2];
                o[3] = 1.0 - T;
            }
        }
    }
    free(gmx);
    free(hnx);
    free(gmy);
    free(hny);
    free(dx);
    free(dy);
}

void orc_set_num_threads(int n)
{
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
}

int orc_num_threads(void)
{
    return omp_get_max_threads();
}
