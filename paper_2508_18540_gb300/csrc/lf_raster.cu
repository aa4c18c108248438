// lf_raster.cu -- 3D-tiled rasterisation of every chunk into its sweeping
// plane (Algorithm 1 lines 4-5, "Parallel for all k: Rasterize(H, P'_k)").
//
// One CTA per (16x16 tile, chunk). It walks the (32x32 super-tile, chunk)
// list holding its tile (ranks in depth order) in batches, keeps the entries
// whose footprint meets its tile (order-preserving compaction), stages those
// primitives (rank-ordered copies) in shared memory, and every thread blends
// its pixels front to back:
//   Gaussians (Sec. 4.4, 3DGS model): alpha = min(0.99, o exp(-q/2)),
//     q = d^T Sigma_2^{-1} d inside the primitive's footprint rectangle;
//   voxels (Sec. 4.5, SVR model): alpha = 1 - exp(-integral of the trilinear
//     density along the pixel's reference ray inside the cube), by Simpson's
//     rule, exact for the cubic the trilinear density becomes along a line;
//   C += T alpha rgb, T *= 1 - alpha. No early stop, no small-alpha skip.
// The texel (C, 1 - T) is stored as FP32, FP16 or BF16 (FP32 accumulation).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lf_internal.cuh"

namespace lf {

namespace {

template <int DT>
__device__ __forceinline__ void store_texel(void* planes, size_t idx, float r, float g, float b, float a)
{
    if (DT == LF_F32) {
        reinterpret_cast<float4*>(planes)[idx] = make_float4(r, g, b, a);
    } else if (DT == LF_F16) {
        const __half2 lo = __floats2half2_rn(r, g), hi = __floats2half2_rn(b, a);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        reinterpret_cast<uint2*>(planes)[idx] = u;
    } else {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(r, g), hi = __floats2bfloat162_rn(b, a);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        reinterpret_cast<uint2*>(planes)[idx] = u;
    }
}

// Order-preserving compaction of a batch: returns this thread's slot among
// the batch's hits (valid if hit) and the hit count. s_wc: [NT / 32] ints.
template <int NT>
__device__ __forceinline__ int compact_slot(bool hit, int* s_wc, int* count)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) s_wc[warp] = __popc(bal);
    __syncthreads();
    int off = 0, cnt = 0;
#pragma unroll
    for (int q = 0; q < NT / 32; ++q) {
        const int v = s_wc[q];
        off += q < warp ? v : 0;
        cnt += v;
    }
    *count = cnt;
    return off + __popc(bal & ((1u << lane) - 1u));
}

__device__ __forceinline__ bool meets_tile(int4 r, int x0, int y0)
{
    return r.x <= x0 + kTile - 1 && r.z >= x0 && r.y <= y0 + kTile - 1 && r.w >= y0;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Gaussians: 256 / PPT threads; thread t shades the PPT pixels of column
// t % 16 in rows PPT (t / 16) ... PPT (t / 16) + PPT - 1, so warp w owns the
// 2 PPT x 16 strip of rows 2 PPT w ... Each batch of list entries is staged
// as three 16-byte words {mean x, mean y, A, B}, {C, o, x0 | y0 << 16,
// (x1 - x0) | (y1 - y0) << 16}, {r, g, b, -}, with the conic pre-scaled so
// that alpha = min(0.99, o 2^(A dx^2 + B dx dy + C dy^2)),
// A = -log2(e)/2 a, B = -log2(e) b, C = -log2(e)/2 c. Every warp ballots which
// entries touch its strip and visits only those, in list order, so the
// blending order of every pixel is unchanged.
template <int DT, int PPT>
__global__ void __launch_bounds__(kTilePix / PPT) k_raster_gauss(BuildWs w, RasterParams p,
                                                                 const uint32_t* __restrict__ ranks, void* planes)
{
    constexpr int NT = kTilePix / PPT;
    constexpr float kL2E = 1.4426950408889634f;
    __shared__ float4 s_e0[NT];
    __shared__ float4 s_e1[NT];
    __shared__ float4 s_rgb[NT];
    __shared__ int s_wc[NT / 32];
    const int t = blockIdx.x, k = blockIdx.y;
    const int tx = t % p.tiles_x, ty = t / p.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py0 = ty * kTile + (threadIdx.x / kTile) * PPT;
    const int sx0 = tx * kTile, sx1 = sx0 + kTile - 1;                // warp strip bounds
    const int sy0 = ty * kTile + 2 * PPT * warp, sy1 = sy0 + 2 * PPT - 1;
    const int st = (ty / kTilesPerSuper) * p.supers_x + tx / kTilesPerSuper;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int L = sg.y - sg.x;
    const float fpx = (float)px;
    float C[PPT][3], T[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) C[r][0] = C[r][1] = C[r][2] = 0.f, T[r] = 1.f;
    for (int base = 0; base < L; base += NT) {
        const int i = base + threadIdx.x;
        uint32_t rk = 0;
        int4 r = make_int4(0, 0, -1, -1);
        if (i < L) {
            rk = ranks[sg.x + i];
            r = w.r_rect[rk];
        }
        const bool hit = i < L && meets_tile(r, sx0, ty * kTile);
        int cnt;
        const int slot = compact_slot<NT>(hit, s_wc, &cnt);
        if (hit) {
            const float4 geo = w.r_geo[rk];
            const float4 c = w.r_con[rk];
            s_e0[slot] = make_float4(geo.x, geo.y, -0.5f * kL2E * c.x, -kL2E * c.y);
            s_e1[slot] = make_float4(-0.5f * kL2E * c.z, c.w, __int_as_float((r.x & 0xffff) | (r.y << 16)),
                                     __int_as_float(((r.z - r.x) & 0xffff) | ((r.w - r.y) << 16)));
            s_rgb[slot] = w.r_rgb[rk];
        }
        __syncthreads();
        for (int m0 = 0; m0 < cnt; m0 += 32) {
            const int jl = m0 + lane;
            bool hit = false;
            if (jl < cnt) {
                const float4 e1 = s_e1[jl];
                const int xy = __float_as_int(e1.z), wh = __float_as_int(e1.w);
                const int rx0 = xy & 0xffff, ry0 = xy >> 16;
                hit = rx0 <= sx1 && rx0 + (wh & 0xffff) >= sx0 && ry0 <= sy1 && ry0 + (wh >> 16) >= sy0;
            }
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            while (mask) {
                const int j = m0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 e1 = s_e1[j];
                const int xy = __float_as_int(e1.z), wh = __float_as_int(e1.w);
                if ((uint32_t)(px - (xy & 0xffff)) > (uint32_t)(wh & 0xffff)) continue;
                const float4 e0 = s_e0[j];
                const float4 col = s_rgb[j];
                const float dx = fpx - e0.x;
                const float adx = e0.z * dx;
                const int ry0 = xy >> 16, rh = wh >> 16;
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    if ((uint32_t)(py0 + r - ry0) <= (uint32_t)rh) {
                        const float dy = (float)(py0 + r) - e0.y;
                        const float pw = fmaf(dx, fmaf(e0.w, dy, adx), e1.x * dy * dy);
                        const float al = fminf(0.99f, e1.y * ex2_approx(pw));
                        const float ta = T[r] * al;
                        C[r][0] = fmaf(ta, col.x, C[r][0]);
                        C[r][1] = fmaf(ta, col.y, C[r][1]);
                        C[r][2] = fmaf(ta, col.z, C[r][2]);
                        T[r] = fmaf(-T[r], al, T[r]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (px < p.W) {
#pragma unroll
        for (int r = 0; r < PPT; ++r)
            if (py0 + r < p.H)
                store_texel<DT>(planes, ((size_t)k * p.H + py0 + r) * p.W + px, C[r][0], C[r][1], C[r][2],
                                1.0f - T[r]);
    }
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

__device__ __forceinline__ float trilinear(const float* rho, float fx, float fy, float fz)
{
    const float c00 = lerpf(rho[0], rho[1], fx), c10 = lerpf(rho[2], rho[3], fx);
    const float c01 = lerpf(rho[4], rho[5], fx), c11 = lerpf(rho[6], rho[7], fx);
    return lerpf(lerpf(c00, c10, fy), lerpf(c01, c11, fy), fz);
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

// Voxels: one thread per pixel (256 threads); cube corner relative to the
// reference centre and side from the projection pass, densities and colour
// in rank order.
template <int DT>
__global__ void __launch_bounds__(kTilePix) k_raster_voxel(BuildWs w, RasterParams p,
                                                           const uint32_t* __restrict__ ranks, void* planes)
{
    constexpr int NT = kTilePix;
    __shared__ float4 s_box[NT];
    __shared__ float s_den[NT * 8];
    __shared__ float4 s_rgb[NT];
    __shared__ int4 s_rect[NT];
    __shared__ int s_wc[NT / 32];
    const int t = blockIdx.x, k = blockIdx.y;
    const int tx = t % p.tiles_x, ty = t / p.tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x / kTile);
    const int st = (ty / kTilesPerSuper) * p.supers_x + tx / kTilesPerSuper;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int L = sg.y - sg.x;

    // world-frame direction of the reference ray through this pixel centre
    const float dcx = ((float)px - p.cx) / p.fx, dcy = ((float)py - p.cy) / p.fy;
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = fmaf(p.Rt[3 * a], dcx, fmaf(p.Rt[3 * a + 1], dcy, p.Rt[3 * a + 2]));
    const float nrm = rsqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
    float inv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] *= nrm;
        inv[a] = 1.0f / d[a];
    }

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    for (int base = 0; base < L; base += NT) {
        const int i = base + threadIdx.x;
        uint32_t rk = 0;
        int4 r = make_int4(0, 0, -1, -1);
        if (i < L) {
            rk = ranks[sg.x + i];
            r = w.r_rect[rk];
        }
        const bool hit = i < L && meets_tile(r, tx * kTile, ty * kTile);
        int cnt;
        const int slot = compact_slot<NT>(hit, s_wc, &cnt);
        if (hit) {
            s_box[slot] = w.r_geo[rk];
            const float4 da = w.r_den[2 * (size_t)rk], db = w.r_den[2 * (size_t)rk + 1];
            float* sd = s_den + 8 * slot;
            sd[0] = da.x; sd[1] = da.y; sd[2] = da.z; sd[3] = da.w;
            sd[4] = db.x; sd[5] = db.y; sd[6] = db.z; sd[7] = db.w;
            s_rgb[slot] = w.r_rgb[rk];
            s_rect[slot] = r;
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const int4 rc = s_rect[j];
            if (!(px >= rc.x && px <= rc.z && py >= rc.y && py <= rc.w)) continue;
            const float4 b = s_box[j];  // cube low corner relative to the ray origin, side
            const float lo[3] = {b.x, b.y, b.z};
            float t0 = -__int_as_float(0x7f800000), t1 = __int_as_float(0x7f800000);
            bool miss = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float hi = lo[a] + b.w;
                if (d[a] != 0.0f) {
                    float ta = lo[a] * inv[a], tb = hi * inv[a];
                    if (ta > tb) {
                        const float tmp = ta;
                        ta = tb;
                        tb = tmp;
                    }
                    t0 = fmaxf(t0, ta);
                    t1 = fminf(t1, tb);
                } else if (0.0f < lo[a] || 0.0f > hi) {
                    miss = true;
                }
            }
            t0 = fmaxf(t0, 0.0f);
            if (miss || !(t1 > t0)) continue;
            const float tm = 0.5f * (t0 + t1);
            const float is = 1.0f / b.w;
            const float* rho = s_den + 8 * j;
            const float s0 = trilinear(rho, clamp01((t0 * d[0] - lo[0]) * is), clamp01((t0 * d[1] - lo[1]) * is),
                                       clamp01((t0 * d[2] - lo[2]) * is));
            const float sm = trilinear(rho, clamp01((tm * d[0] - lo[0]) * is), clamp01((tm * d[1] - lo[1]) * is),
                                       clamp01((tm * d[2] - lo[2]) * is));
            const float s1 = trilinear(rho, clamp01((t1 * d[0] - lo[0]) * is), clamp01((t1 * d[1] - lo[1]) * is),
                                       clamp01((t1 * d[2] - lo[2]) * is));
            const float integral = (t1 - t0) * (1.0f / 6.0f) * (s0 + 4.0f * sm + s1);
            const float al = 1.0f - __expf(-integral);
            const float4 col = s_rgb[j];
            const float ta = T * al;
            C0 = fmaf(ta, col.x, C0);
            C1 = fmaf(ta, col.y, C1);
            C2 = fmaf(ta, col.z, C2);
            T = T * (1.0f - al);
        }
        __syncthreads();
    }
    if (px < p.W && py < p.H) store_texel<DT>(planes, ((size_t)k * p.H + py) * p.W + px, C0, C1, C2, 1.0f - T);
}

}  // namespace

void launch_raster_gaussians(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                             cudaStream_t s)
{
    const dim3 grid((unsigned)(p.tiles_x * p.tiles_y), (unsigned)p.N);
    constexpr int kPPT = 2;   // pixels per thread
    constexpr int kThreads = kTilePix / kPPT;
    switch (p.dtype) {
    case LF_F32: k_raster_gauss<LF_F32, kPPT><<<grid, kThreads, 0, s>>>(ws, p, ranks, planes); break;
    case LF_F16: k_raster_gauss<LF_F16, kPPT><<<grid, kThreads, 0, s>>>(ws, p, ranks, planes); break;
    default: k_raster_gauss<LF_BF16, kPPT><<<grid, kThreads, 0, s>>>(ws, p, ranks, planes); break;
    }
    note_launches(1);
}

void launch_raster_voxels(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                          cudaStream_t s)
{
    const dim3 grid((unsigned)(p.tiles_x * p.tiles_y), (unsigned)p.N);
    switch (p.dtype) {
    case LF_F32: k_raster_voxel<LF_F32><<<grid, kTilePix, 0, s>>>(ws, p, ranks, planes); break;
    case LF_F16: k_raster_voxel<LF_F16><<<grid, kTilePix, 0, s>>>(ws, p, ranks, planes); break;
    default: k_raster_voxel<LF_BF16><<<grid, kTilePix, 0, s>>>(ws, p, ranks, planes); break;
    }
    note_launches(1);
}

}  // namespace lf
