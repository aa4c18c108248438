/*
 * orc_filter.c -- oracle: the low-pass plane filter of V2LF.
 * TEST INFRASTRUCTURE ONLY (see lf_oracle.h).
 *
 * Sec. 4.5: SVR's supersampling is replaced by a low-pass Gaussian filter
 * applied to the sweeping planes. The paper gives neither the width nor the
 * support; reading: a separable, normalised discrete Gaussian with standard
 * deviation sigma (plane pixels) and support [-radius, radius], applied to
 * every RGBA channel of every plane (rows first, then columns), with
 * transparent zero padding outside the plane.
 */
#include "lf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void orc_filter_weights(double sigma, int32_t radius, double* w)
{
    double sum = 0.0;
    for (int32_t i = -radius; i <= radius; ++i) {
        w[i + radius] = exp(-0.5 * (double)i * (double)i / (sigma * sigma));
        sum += w[i + radius];
    }
    for (int32_t i = 0; i <= 2 * radius; ++i) w[i] /= sum;
}

void orc_filter_planes(double* planes, int32_t N, int32_t H, int32_t W, double sigma, int32_t radius)
{
    double* w = (double*)malloc(sizeof(double) * (size_t)(2 * radius + 1));
    orc_filter_weights(sigma, radius, w);
    const int64_t plane = (int64_t)H * W * 4;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)plane);
    for (int32_t k = 0; k < N; ++k) {
        double* P = planes + plane * k;
        /* rows */
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x)
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int32_t i = -radius; i <= radius; ++i) {
                        const int32_t xx = x + i;
                        if (xx < 0 || xx >= W) continue;
                        acc += w[i + radius] * P[((int64_t)y * W + xx) * 4 + c];
                    }
                    tmp[((int64_t)y * W + x) * 4 + c] = acc;
                }
        /* columns */
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x)
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int32_t i = -radius; i <= radius; ++i) {
                        const int32_t yy = y + i;
                        if (yy < 0 || yy >= H) continue;
                        acc += w[i + radius] * tmp[((int64_t)yy * W + x) * 4 + c];
                    }
                    P[((int64_t)y * W + x) * 4 + c] = acc;
                }
    }
    free(tmp);
    free(w);
}
