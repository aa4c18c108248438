// lf_raster.cu -- 3D-tiled rasterisation of every chunk into its sweeping
// plane (the per-chunk rendering step of Algorithm 1, all chunks in parallel).
//
// Every (32x32 super-tile, chunk) list holds the ranks, in depth order, of
// the primitives whose footprint meets the super-tile. Gaussians: one CTA
// per list (long lists cut into parts, composed with the "over" operator;
// see below). Voxels: one CTA per (16x16 tile, chunk), keeping the entries of
// its super-tile's list that meet its tile (order-preserving compaction).
// The CTA stages the primitives (rank-ordered copies) in shared memory in
// batches, and every thread blends its pixels front to back:
//   Gaussians (Sec. 4.4, 3DGS model): alpha = min(0.99, o exp(-q/2)),
//     q = d^T Sigma_2^{-1} d inside the primitive's footprint rectangle;
//   voxels (Sec. 4.5, SVR model): alpha = 1 - exp(-integral of the trilinear
//     density along the pixel's reference ray inside the cube), by Simpson's
//     rule, exact for the cubic the trilinear density becomes along a line
//     (computed pair-parallel into shared memory first: voxel footprints
//     cover only a few pixels);
//   C += T alpha rgb, T *= 1 - alpha. No early stop and no small-alpha skip,
//   unless the Gaussian build asks for the 3DGS cut-offs.
// The texel (C, 1 - T) is stored as FP32, FP16, BF16 or RGBA8 (FP32
// accumulation).
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
    } else if (DT == LF_U8) {
        // RGBA8 unorm: round(255 clamp(v, 0, 1)) per channel
        reinterpret_cast<uint32_t*>(planes)[idx] = u8_pack(r, g, b, a);
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

// Gaussians. A CTA rasterises one (32 x 32 super-tile, chunk) list, or one
// part of a long one, with 8 warps. Warp w owns the 8-column x 16-row strip
// at column group w % 4 and row group w / 4 of the super-tile; lane l shades
// column l % 8 in rows l / 8 + 4 s, s = 0 .. 3, so the lanes' s-th pixels
// form the 8 x 4 sub-block s of the strip, and a footprint that misses a
// sub-block costs the warp nothing there (sub-blocks of 32 pixels fit the
// footprint sizes better than wide strips). Each batch of list entries is
// staged as three 16-byte words {mean x, mean y, A, B}, {C, log2 o, cm, rm},
// {r, g, b, wm}, with the conic pre-scaled so that
//   alpha = min(0.99, 2^(A dx^2 + B dx dy + C dy^2 + log2 o)),
// A = -log2(e)/2 a, B = -log2(e) b, C = -log2(e)/2 c, and the footprint
// rectangle as bit masks over the super-tile: bit c of cm for column c, bit r
// of rm for row r, bit w of wm for the warps whose strips it meets (computed
// once per entry and CTA, so a warp's visit tests bits instead of bounds).
// Per visited entry a lane forms g1 = B dx and g0 = A dx^2 + log2 o for its
// column once; each of its rows inside the footprint then costs the Horner
// form (C dy + g1) dy + g0, one ex2 and the blend. Every warp ballots which
// entries touch its strip and visits only those, in list order, so each
// pixel blends its members front to back. Two staging buffers alternate: one
// CTA barrier per batch.
//
// Load balance. The work of a list grows with its length, and dense regions
// of the scene make a few lists far longer than the rest. k_raster_plan cuts
// every list longer than r_seg entries into parts of r_seg entries, and
// k_raster_gauss_parts rasterises the parts: each blends its entries into a
// partial (C, T) started from (0, 1) and stores it in its slot, and the CTA
// that finishes a list's last part composes the partials in part order,
// C += T C_q, T *= T_q (the "over" operator is associative), and writes the
// texels. k_raster_gauss rasterises the other lists, one CTA each, and is
// launched right behind the parts kernel with programmatic dependent launch,
// so the long lists' parts start first and the short lists fill the machine
// around them. The 3DGS cut-offs are not associative (the stop depends on
// the running transmittance), so that mode splits no list.
constexpr int kPlanThreads = 256;
constexpr int kGaussNS = 4;                       // pixels per thread
constexpr int kGaussThreads = 32 * 4 * (8 / kGaussNS);

struct GaussSmem {
    float4 e0[2][kGaussThreads];
    float4 e1[2][kGaussThreads];
    float4 rgb[2][kGaussThreads];
};

// Split parts of one raster (one thread per (super-tile, chunk) list): a list
// of L > r_seg entries takes P = ceil(L / r_seg) consecutive partial slots;
// its parts become items [0, r_heavy) of the form {list, part, P, slot}.
__global__ void __launch_bounds__(kPlanThreads) k_raster_plan(BuildWs w, int lists, int split)
{
    pdl_wait();
    pdl_trigger();
    const long long total = (long long)w.hdr->tile_n;
    int S = 0x7fffffff;
    if (split) {
        long long need = (2 * total + w.r_nslots - 1) / w.r_nslots;   // keeps the parts within the slots
        need = (need + 255) / 256 * 256;
        S = (int)(need > kRasterSegMin ? need : kRasterSegMin);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) w.hdr->r_seg = S;
    for (int id = blockIdx.x * kPlanThreads + threadIdx.x; id < lists; id += gridDim.x * kPlanThreads) {
        const int2 sg = w.seg[id];
        const int L = sg.y - sg.x;
        if (L <= S) continue;
        const int P = (int)(((long long)L + S - 1) / S);
        const unsigned int pos = atomicAdd(&w.hdr->r_heavy, (unsigned int)P);
        w.r_arrive[id] = 0;
        for (int q = 0; q < P; ++q)   // pos + P <= r_nslots, by the choice of S
            w.r_items[pos + q] = make_int4(id, q, P, (int)(pos + q));
    }
}

// List (st, k): the whole list (SPLIT false), or part `part` of P with
// partial slot `slot`, S entries per part (SPLIT true). Every thread of the
// CTA calls it. G3 adds the two cut-offs of the 3DGS rasteriser: a member
// with alpha < 1/255 is skipped, and a pixel whose next blend would take
// T (1 - alpha) below 1e-4 stops blending (bit s of `stopped`).
template <int DT, bool G3, bool SPLIT>
__device__ __forceinline__ void raster_gauss_list(const BuildWs& w, const RasterParams& p,
                                                  const uint32_t* __restrict__ ranks, void* planes, int st, int k,
                                                  GaussSmem& sm, int part, int P, int slot, int S, int* s_last)
{
    constexpr int NS = kGaussNS;
    constexpr int NT = kGaussThreads;
    constexpr float kL2E = 1.4426950408889634f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int SX = (st % p.supers_x) * kSuper, SY = (st / p.supers_x) * kSuper;
    const int sx0 = SX + 8 * (warp & 3);                                  // warp strip origin
    const int sy0 = SY + 4 * NS * (warp >> 2);
    const int px = sx0 + (lane & 7);
    const int py0 = sy0 + (lane >> 3);                                    // slot s: row py0 + 4 s
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int beg = SPLIT ? sg.x + part * S : sg.x;
    const int L = SPLIT ? min(sg.y - beg, S) : sg.y - sg.x;
    const float fpx = (float)px;
    // bit of this lane's column in cm, of its slot-0 row in rm
    const int csh = px - SX, rsh = py0 - SY;
    float C[NS][3], T[NS];
    uint32_t stopped = 0u;
#pragma unroll
    for (int s = 0; s < NS; ++s) C[s][0] = C[s][1] = C[s][2] = 0.f, T[s] = 1.f;
    int buf = 0;
    for (int base = 0; base < L; base += NT, buf ^= 1) {
        const int i = base + threadIdx.x;
        if (i < L) {
            const uint32_t rk = ranks[beg + i];
            const int4 r = w.r_rect[rk];
            const float4 geo = w.r_geo[rk];
            const float4 c = w.r_con[rk];
            sm.e0[buf][threadIdx.x] = make_float4(geo.x, geo.y, -0.5f * kL2E * c.x, -kL2E * c.y);
            // footprint columns / rows of the super-tile as bit masks, and
            // the warps whose 8 x 16 strips it meets
            const int cl = max(r.x - SX, 0), ch = min(r.z - SX, kSuper - 1);
            const int rl = max(r.y - SY, 0), rh = min(r.w - SY, kSuper - 1);
            const uint32_t cm = cl <= ch ? (0xffffffffu >> (31 - ch)) & (0xffffffffu << cl) : 0u;
            const uint32_t rm = rl <= rh ? (0xffffffffu >> (31 - rh)) & (0xffffffffu << rl) : 0u;
            uint32_t wm = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                wm |= ((cm >> (8 * (q & 3))) & 0xffu) && ((rm >> (16 * (q >> 2))) & 0xffffu) ? 1u << q : 0u;
            sm.e1[buf][threadIdx.x] =
                make_float4(-0.5f * kL2E * c.z, __log2f(c.w), __uint_as_float(cm), __uint_as_float(rm));
            const float4 rgb = w.r_rgb[rk];
            sm.rgb[buf][threadIdx.x] = make_float4(rgb.x, rgb.y, rgb.z, __uint_as_float(wm));
        }
        // orders this batch's staging before its walk, and every warp's walk
        // of the batch before last before this staging overwrote its buffer
        __syncthreads();
        const int cnt = min(NT, L - base);
        const float4* s_e0 = sm.e0[buf];
        const float4* s_e1 = sm.e1[buf];
        const float4* s_rgb = sm.rgb[buf];
        for (int m0 = 0; m0 < cnt; m0 += 32) {
            const int jl = m0 + lane;
            const bool hit = jl < cnt && ((__float_as_uint(s_rgb[jl].w) >> warp) & 1u);
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            while (mask) {
                const int j = m0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 e0 = s_e0[j];
                const float4 e1 = s_e1[j];
                const float4 col = s_rgb[j];
                // slot s of this lane lies in the footprint iff bit 4 s of m is set
                const uint32_t m = (__float_as_uint(e1.z) >> csh) & 1u ? __float_as_uint(e1.w) >> rsh : 0u;
                const float dx = fpx - e0.x;
                const float g1 = e0.w * dx;
                const float g0 = fmaf(e0.z * dx, dx, e1.y);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    if (m & (1u << (4 * s))) {
                        const float dy = (float)(py0 + 4 * s) - e0.y;
                        const float pw = fmaf(fmaf(e1.x, dy, g1), dy, g0);
                        const float al = fminf(0.99f, ex2_approx(pw));
                        const float tn = fmaf(-T[s], al, T[s]);
                        if (G3) {
                            if ((stopped >> s) & 1u) continue;
                            if (al < 1.0f / 255.0f) continue;
                            if (tn < 1e-4f) {
                                stopped |= 1u << s;
                                continue;
                            }
                        }
                        const float ta = T[s] * al;
                        C[s][0] = fmaf(ta, col.x, C[s][0]);
                        C[s][1] = fmaf(ta, col.y, C[s][1]);
                        C[s][2] = fmaf(ta, col.z, C[s][2]);
                        T[s] = tn;
                    }
                }
            }
        }
    }
    if (SPLIT) {
        // publish the partial; the last part of the list to finish composes
        // all of them, this one included, read back through L2 in order
        const int slot0 = slot - part;
        float4* mine = w.r_part + (size_t)slot * (kSuper * kSuper);
#pragma unroll
        for (int s = 0; s < NS; ++s)
            __stcg(mine + (warp * NS + s) * 32 + lane, make_float4(C[s][0], C[s][1], C[s][2], T[s]));
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) *s_last = atomicAdd(&w.r_arrive[st * p.N + k], 1) == P - 1;
        __syncthreads();
        if (!*s_last) return;
        __threadfence();
#pragma unroll
        for (int s = 0; s < NS; ++s) C[s][0] = C[s][1] = C[s][2] = 0.f, T[s] = 1.f;
        for (int q = 0; q < P; ++q) {
            const float4* src = w.r_part + (size_t)(slot0 + q) * (kSuper * kSuper);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float4 v = __ldcg(src + (warp * NS + s) * 32 + lane);
                C[s][0] = fmaf(T[s], v.x, C[s][0]);
                C[s][1] = fmaf(T[s], v.y, C[s][1]);
                C[s][2] = fmaf(T[s], v.z, C[s][2]);
                T[s] *= v.w;
            }
        }
    }
    if (px < p.W) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (py0 + 4 * s < p.H)
                store_texel<DT>(planes, ((size_t)k * p.H + py0 + 4 * s) * p.W + px, C[s][0], C[s][1], C[s][2],
                                1.0f - T[s]);
    }
}

// Lists no longer than r_seg entries: one CTA per (super-tile x, chunk y).
// The FP32 form takes 48 registers: five CTAs (40 warps) per SM. (A
// minimum-blocks bound of five, same register count, measured 8 % slower;
// only the 3DGS form, 58 registers unbounded, gains from it.)
// Launched behind the parts kernel, it does not wait for it to start;
// CTA (0, 0) waits for it to finish before exiting, so this grid completes
// after every part's texels are written and work ordered after it sees them.
template <int DT, bool G3>
__global__ void __launch_bounds__(kGaussThreads, G3 ? 5 : 0) k_raster_gauss(BuildWs w, RasterParams p,
                                                               const uint32_t* __restrict__ ranks, void* planes)
{
    __shared__ GaussSmem sm;
    const int st = blockIdx.x, k = blockIdx.y;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    if (sg.y - sg.x <= w.hdr->r_seg)   // longer lists: k_raster_gauss_parts
        raster_gauss_list<DT, G3, false>(w, p, ranks, planes, st, k, sm, 0, 1, -1, 0, nullptr);
    if (st == 0 && k == 0) pdl_wait();
}

// The parts of the split lists: CTA b takes item b (CTAs past r_heavy exit).
// Bounded to 64 registers (four CTAs per SM; 66 unbounded, three): parts
// dominate at few chunks (N = 16: 0.436 -> 0.398 ms).
// It lets the list kernel launch at once: that kernel reads nothing the
// parts write.
template <int DT>
__global__ void __launch_bounds__(kGaussThreads, 4) k_raster_gauss_parts(BuildWs w, RasterParams p,
                                                                     const uint32_t* __restrict__ ranks, void* planes)
{
    __shared__ GaussSmem sm;
    __shared__ int s_last;
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x >= w.hdr->r_heavy) return;
    const int4 it = w.r_items[blockIdx.x];
    const int st = it.x / p.N;
    raster_gauss_list<DT, false, true>(w, p, ranks, planes, st, it.x - st * p.N, sm, it.y, it.z, it.w,
                                       w.hdr->r_seg, &s_last);
}

// Several scenes in one grid: CTA b < parts_total takes a split part (scene s
// from pbase), the others a list (scene s from lbase), in scene-table order.
template <int DT>
__global__ void __launch_bounds__(kGaussThreads) k_raster_gauss_batched(const RasterScene* __restrict__ sc, int n_sc,
                                                                       long long parts_total)
{
    __shared__ GaussSmem sm;
    __shared__ int s_last;
    const long long b = blockIdx.x;
    const bool part = b < parts_total;
    int lo = 0, hi = n_sc - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((part ? sc[mid].pbase : sc[mid].lbase) <= b) lo = mid; else hi = mid - 1;
    }
    const RasterScene& S = sc[lo];
    if (part) {
        const long long q = b - S.pbase;
        if (q >= (long long)S.w.hdr->r_heavy) return;
        const int4 it = S.w.r_items[q];
        const int st = it.x / S.p.N;
        raster_gauss_list<DT, false, true>(S.w, S.p, S.ranks, S.planes, st, it.x - st * S.p.N, sm, it.y, it.z, it.w,
                                           S.w.hdr->r_seg, &s_last);
    } else {
        const int supers = S.p.supers_x * S.p.supers_y;
        const int li = (int)(b - S.lbase);
        const int k = li / supers, st = li - k * supers;
        const int2 sg = S.w.seg[(size_t)st * S.p.N + k];
        if (sg.y - sg.x > S.w.hdr->r_seg) return;
        raster_gauss_list<DT, false, false>(S.w, S.p, S.ranks, S.planes, st, k, sm, 0, 1, -1, 0, nullptr);
    }
}

// clamp to [0, 1] (NaN -> 0) in one saturating operation
__device__ __forceinline__ float clamp01(float v) { return __saturatef(v); }

// The trilinear density of corner values r[x + 2y + 4z] in polynomial form:
// rho(f) = c0 + c1 fx + c2 fy + c3 fz + c4 fx fy + c5 fx fz + c6 fy fz
// + c7 fx fy fz; coefficients computed once per voxel, 7 FMAs per sample.
__device__ __forceinline__ void trilinear_coeffs(const float* r, float* c)
{
    c[0] = r[0];
    c[1] = r[1] - r[0];
    c[2] = r[2] - r[0];
    c[3] = r[4] - r[0];
    c[4] = (r[3] - r[2]) - (r[1] - r[0]);
    c[5] = (r[5] - r[4]) - (r[1] - r[0]);
    c[6] = (r[6] - r[4]) - (r[2] - r[0]);
    c[7] = ((r[7] - r[6]) - (r[5] - r[4])) - ((r[3] - r[2]) - (r[1] - r[0]));
}

__device__ __forceinline__ float trilinear_poly(const float* c, float fx, float fy, float fz)
{
    const float b = fmaf(fy, fmaf(fz, c[7], c[4]), fmaf(fz, c[5], c[1]));
    const float e = fmaf(fz, c[6], c[2]);
    return fmaf(fx, b, fmaf(fy, e, fmaf(fz, c[3], c[0])));
}

// Opacity of one voxel for one pixel's reference ray (unit direction d,
// inv = 1 / d): the ray's parameter interval inside the cube (slab test),
// then Simpson's rule on the trilinear density, exact for the cubic it
// becomes along a line; 0 when the ray misses the cube.
__device__ __forceinline__ float voxel_alpha(const float4 b, const float is, const float* cf, const float d[3],
                                             const float inv[3])
{
    const float lo[3] = {b.x, b.y, b.z};   // cube low corner relative to the ray origin; b.w = side
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
    if (miss || !(t1 > t0)) return 0.0f;
    const float tm = 0.5f * (t0 + t1);
    const float s0 = trilinear_poly(cf, clamp01((t0 * d[0] - lo[0]) * is), clamp01((t0 * d[1] - lo[1]) * is),
                                    clamp01((t0 * d[2] - lo[2]) * is));
    const float sm = trilinear_poly(cf, clamp01((tm * d[0] - lo[0]) * is), clamp01((tm * d[1] - lo[1]) * is),
                                    clamp01((tm * d[2] - lo[2]) * is));
    const float s1 = trilinear_poly(cf, clamp01((t1 * d[0] - lo[0]) * is), clamp01((t1 * d[1] - lo[1]) * is),
                                    clamp01((t1 * d[2] - lo[2]) * is));
    const float integral = (t1 - t0) * (1.0f / 6.0f) * (s0 + 4.0f * sm + s1);
    return 1.0f - __expf(-integral);
}

// Exclusive prefix sum of one value per thread over a 256-thread block (in
// thread order); s_ws: [8] ints; *total receives the block sum.
__device__ __forceinline__ int block_exscan_256(int v, int* s_ws, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_ws[warp] = x;
    __syncthreads();
    int before = 0, sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int s = s_ws[q];
        before += q < warp ? s : 0;
        sum += s;
    }
    *total = sum;
    return before + x - v;
}

constexpr int kVoxPairs = 2048;   // (voxel, pixel) opacities held in shared memory per pass

// Voxels: one CTA of 256 threads per (16x16 tile, chunk), thread t owning
// tile pixel (t % 16, t / 16). A voxel's footprint covers only a few pixels,
// so each batch of staged voxels is processed pair-parallel: the footprints
// clipped to the tile are numbered (voxel order, then rows, then columns),
// every thread computes the opacities of pairs t, t + 256, ... into shared
// memory, and then every pixel blends its pairs front to back in list order
// (each warp visits only the voxels that touch its two rows). A pair whose
// ray misses the cube has opacity 0, which leaves C and T unchanged exactly.
// Cube corner relative to the reference centre and side come from the
// projection pass; densities and colour in rank order.
template <int DT>
__global__ void __launch_bounds__(kTilePix, 5) k_raster_voxel(BuildWs w, RasterParams p,
                                                           const uint32_t* __restrict__ ranks, void* planes)
{
    constexpr int NT = kTilePix;
    __shared__ float4 s_box[NT];
    __shared__ float s_inv_side[NT];   // 1 / side, once per staged voxel
    __shared__ float s_den[NT * 8];    // trilinear polynomial coefficients per voxel
    __shared__ float4 s_rgb[NT];
    __shared__ int4 s_rect[NT];        // footprint clipped to the tile, tile-local (x0, y0, x1, y1)
    __shared__ int s_off[NT];          // number of the voxel's first pair
    __shared__ float4 s_dir[NT];       // per pixel: unit reference-ray direction
    __shared__ float4 s_inv[NT];       // per pixel: its reciprocal
    __shared__ uint16_t s_pair[kVoxPairs];   // voxel slot | x << 8 | y << 12 (tile-local pixel)
    __shared__ float s_alpha[kVoxPairs];
    __shared__ int s_wc[NT / 32];
    __shared__ int s_ws[NT / 32];
    const int t = blockIdx.x, k = blockIdx.y;
    const int tx = t % p.tiles_x, ty = t / p.tiles_x;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const int wy0 = 2 * (threadIdx.x >> 5), wy1 = wy0 + 1;   // this warp's two tile rows
    const int st = (ty / kTilesPerSuper) * p.supers_x + tx / kTilesPerSuper;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int L = sg.y - sg.x;

    {
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
        s_dir[threadIdx.x] = make_float4(d[0], d[1], d[2], 0.f);
        s_inv[threadIdx.x] = make_float4(inv[0], inv[1], inv[2], 0.f);
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
        int4 cr = make_int4(0, 0, -1, -1);
        if (hit) {
            cr = make_int4(max(r.x - tx * kTile, 0), max(r.y - ty * kTile, 0), min(r.z - tx * kTile, kTile - 1),
                           min(r.w - ty * kTile, kTile - 1));
            const float4 box = w.r_geo[rk];
            s_box[slot] = box;
            s_inv_side[slot] = 1.0f / box.w;
            const float4 da = w.r_den[2 * (size_t)rk], db = w.r_den[2 * (size_t)rk + 1];
            const float rho8[8] = {da.x, da.y, da.z, da.w, db.x, db.y, db.z, db.w};
            trilinear_coeffs(rho8, s_den + 8 * slot);   // polynomial coefficients, not corners
            s_rgb[slot] = w.r_rgb[rk];
            s_rect[slot] = cr;
        }
        // pairs are numbered in slot order, which is thread order among the hits
        int P;
        const int off = block_exscan_256(hit ? (cr.z - cr.x + 1) * (cr.w - cr.y + 1) : 0, s_ws, &P);
        if (hit) s_off[slot] = off;
        __syncthreads();
        for (int c0 = 0; c0 < P; c0 += kVoxPairs) {
            const int c1 = min(P, c0 + kVoxPairs);
            if (hit && off < c1) {
                int q = off;
                for (int yy = cr.y; yy <= cr.w && q < c1; ++yy)
                    for (int xx = cr.x; xx <= cr.z && q < c1; ++xx, ++q)
                        if (q >= c0) s_pair[q - c0] = (uint16_t)(slot | (xx << 8) | (yy << 12));
            }
            __syncthreads();
            for (int q = threadIdx.x; q < c1 - c0; q += NT) {
                const uint32_t e = s_pair[q];
                const int j = e & 0xff, pix = (int)((e >> 12) << 4) + (int)((e >> 8) & 15);
                const float4 dd = s_dir[pix], iv = s_inv[pix];
                const float d[3] = {dd.x, dd.y, dd.z}, inv[3] = {iv.x, iv.y, iv.z};
                s_alpha[q] = voxel_alpha(s_box[j], s_inv_side[j], s_den + 8 * j, d, inv);
            }
            __syncthreads();
            // every warp ballots which staged voxels touch its rows and
            // visits only those, in list order; each pixel takes its pair
            // if it lies in this pass
            for (int m0 = 0; m0 < cnt; m0 += 32) {
                const int jl = m0 + (threadIdx.x & 31);
                bool touches = false;
                if (jl < cnt) {
                    const int4 rl = s_rect[jl];
                    touches = rl.y <= wy1 && rl.w >= wy0;
                }
                uint32_t vmask = __ballot_sync(0xffffffffu, touches);
                while (vmask) {
                    const int j = m0 + __ffs(vmask) - 1;
                    vmask &= vmask - 1;
                    const int4 rc = s_rect[j];
                    if (lx < rc.x || lx > rc.z || ly < rc.y || ly > rc.w) continue;
                    const int q = s_off[j] + (ly - rc.y) * (rc.z - rc.x + 1) + (lx - rc.x);
                    if (q < c0 || q >= c1) continue;
                    const float al = s_alpha[q - c0];
                    const float4 col = s_rgb[j];
                    const float ta = T * al;
                    C0 = fmaf(ta, col.x, C0);
                    C1 = fmaf(ta, col.y, C1);
                    C2 = fmaf(ta, col.z, C2);
                    T = T * (1.0f - al);
                }
            }
            // another pass of this batch overwrites s_pair and s_alpha; the
            // next batch writes them only after its staging barrier
            if (c1 < P) __syncthreads();
        }
    }
    if (px < p.W && py < p.H) store_texel<DT>(planes, ((size_t)k * p.H + py) * p.W + px, C0, C1, C2, 1.0f - T);
}

// ---------------------------------------------------------------------------
// Adjoints of the per-chunk blending (the splat half of the backward pass).
//
// Per plane pixel the forward computes C = sum_i T_i a_i c_i and A = 1 - T_end
// with T_{i+1} = T_i (1 - a_i). With upstream gradients dC (3) and dA, and
// w_i = c_i . dC + dA (because 1 - T_end = sum_i T_i a_i):
//   dL/dc_i = T_i a_i dC,   dL/da_i = T_i (w_i - S_i),
//   S_i = sum_{j>i} (T_j / T_{i+1}) a_j w_j,  S_{i-1} = a_i w_i + (1 - a_i) S_i.
// Both kernels walk each list front to back in the forward's arithmetic and
// form the term behind entry i from the pixel's end values (below), so no
// transmittance is divided back and nothing per entry is stored.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gaussians, front to back. For the pixel's entries i of a list, with
// w_i = c_i . dC + dA and R_i the part of C . dC + A dA = sum_j T_j a_j w_j
// behind entry i,
//   R_i = sum_{j>i} T_j a_j w_j = K - C_{i+1} . dC + T_{i+1} dA,
//   K = C_end . dC - T_end dA,
//   dL/dc_i = T_i a_i dC,   dL/da_i = T_i w_i - R_i / (1 - a_i),
// (the T_j, j > i, carry the factor 1 - a_i) where C_{i+1}, T_{i+1} are the
// running colour and transmittance behind entry i: one walk in the forward's
// order and arithmetic gives every term, with no division chain and no
// rescaling (1 - a_i >= 0.01). K comes from the forward's texel (FP32 planes:
// C_end exact, T_end = 1 - A within 2^-24), from the split list's partials
// (composed as the forward composed them), or, for the other plane types,
// from a first walk that recomputes (C_end, T_end).
// CTA layout, staging and list walk as k_raster_gauss (one (super-tile,
// chunk) list, or one part of a split list, per CTA; 8 warps of 8 x 16
// pixel strips, lane rows l / 8 + 4 s). A part starts from the composition
// of the partials in front of it. Per entry each warp adds its pixels'
// terms: Su = sum u, Sv = sum v (u = dq dx, v = dq dy, dq = -a_i dL/da_i / 2),
// Saa = sum u dx, Sbb = sum u dy, Scc = sum v dy, So = sum dL/da_i G, and the
// colour terms; eight of them are reduced by a butterfly that halves the
// values each step (9 shuffles), and
//   d mean = -2 (a Su + b Sv, b Su + c Sv), d(a, b, c) = (Saa, 2 Sbb, Scc)
// (q = a dx^2 + 2 b dx dy + c dy^2, alpha = min(0.99, o exp(-q/2)); a clamped
// alpha passes no gradient to o or q). Accumulator of rank r:
// g2d[3 r .. 3 r + 2] = {d mean x, d mean y, d a, d b}, {d c, d o, d r,
// d g}, {d b(lue), 0, 0, 0}.
constexpr int kGaussBwdThreads = kGaussThreads;

struct GaussBwdSmem {
    float4 e0[2][kGaussBwdThreads];
    float4 e1[2][kGaussBwdThreads];
    float4 rgb[2][kGaussBwdThreads];   // {r, g, b, 1 / o}
    uint32_t rank[2][kGaussBwdThreads];
    uint32_t wm[2][kGaussBwdThreads];  // warps whose strips the footprint meets
};

// v[0..7] summed over the warp; lane l ends with the sum of v[(l >> 2) & 7]
__device__ __forceinline__ float warp_reduce_scatter8(float (&v)[8], int lane)
{
    float h[4];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4], keep = b4 ? v[i + 4] : v[i];
        h[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float q[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? h[i] : h[i + 2], keep = b3 ? h[i + 2] : h[i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const float send = b2 ? q[0] : q[1], keep = b2 ? q[1] : q[0];
    float r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// One list (SPLIT false) or one part of a split list (SPLIT true).
template <int DT, bool SPLIT>
__device__ __forceinline__ void raster_gauss_bwd_list(const BuildWs& w, const RasterParams& p,
                                                      const uint32_t* __restrict__ ranks,
                                                      const void* __restrict__ planes,
                                                      const float4* __restrict__ dplanes, float4* __restrict__ g2d,
                                                      int st, int k, GaussBwdSmem& sm, int part, int P, int slot,
                                                      int S)
{
    constexpr int NS = kGaussNS;
    constexpr int NT = kGaussBwdThreads;
    constexpr float kL2E = 1.4426950408889634f;
    // K from a first walk: unsplit lists whose planes are not FP32
    constexpr bool WALK1 = !SPLIT && DT != LF_F32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int SX = (st % p.supers_x) * kSuper, SY = (st / p.supers_x) * kSuper;
    const int px = SX + 8 * (warp & 3) + (lane & 7);
    const int py0 = SY + 4 * NS * (warp >> 2) + (lane >> 3);
    // bit of this lane's column in cm, of its slot-0 row in rm
    const int csh = px - SX, rsh = py0 - SY;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int beg = SPLIT ? sg.x + part * S : sg.x;
    const int L = SPLIT ? min(sg.y - beg, S) : sg.y - sg.x;
    const float fpx = (float)px;

    float C[NS][3], T[NS], dC[NS][3], dA[NS], K[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int py = py0 + 4 * s;
        const bool in = px < p.W && py < p.H;
        const size_t idx = ((size_t)k * p.H + py) * p.W + px;
        const float4 g = in ? __ldg(dplanes + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        dC[s][0] = g.x, dC[s][1] = g.y, dC[s][2] = g.z, dA[s] = g.w;
        C[s][0] = C[s][1] = C[s][2] = 0.f, T[s] = 1.f;
        K[s] = 0.f;
        if (SPLIT) {
            // (C, T) in front of this part and at the list's end: the
            // partials composed in part order, as the forward composed them
            float ce0 = 0.f, ce1 = 0.f, ce2 = 0.f, te = 1.f;
            const int slot0 = slot - part;
            for (int q = 0; q < P; ++q) {
                if (q == part) C[s][0] = ce0, C[s][1] = ce1, C[s][2] = ce2, T[s] = te;
                const float4 v = __ldcg(w.r_part + (size_t)(slot0 + q) * (kSuper * kSuper) + (warp * NS + s) * 32 + lane);
                ce0 = fmaf(te, v.x, ce0);
                ce1 = fmaf(te, v.y, ce1);
                ce2 = fmaf(te, v.z, ce2);
                te *= v.w;
            }
            K[s] = fmaf(ce0, dC[s][0], fmaf(ce1, dC[s][1], fmaf(ce2, dC[s][2], -te * dA[s])));
        } else if (DT == LF_F32) {
            const float4 t = in ? __ldg(reinterpret_cast<const float4*>(planes) + idx) : make_float4(0.f, 0.f, 0.f, 1.f);
            K[s] = fmaf(t.x, dC[s][0], fmaf(t.y, dC[s][1], fmaf(t.z, dC[s][2], -(1.0f - t.w) * dA[s])));
        }
    }

    // stages batch `base` of the list into buffer buf
    auto stage = [&](int base, int buf) {
        const int i = base + threadIdx.x;
        if (i < L) {
            const uint32_t rk = ranks[beg + i];
            const int4 r = w.r_rect[rk];
            const float4 geo = w.r_geo[rk];
            const float4 c = w.r_con[rk];
            const float4 rgb = w.r_rgb[rk];
            sm.e0[buf][threadIdx.x] = make_float4(geo.x, geo.y, -0.5f * kL2E * c.x, -kL2E * c.y);
            // the footprint as bit masks over the super-tile, as in the forward
            const int cl = max(r.x - SX, 0), ch = min(r.z - SX, kSuper - 1);
            const int rl = max(r.y - SY, 0), rh = min(r.w - SY, kSuper - 1);
            const uint32_t cm = cl <= ch ? (0xffffffffu >> (31 - ch)) & (0xffffffffu << cl) : 0u;
            const uint32_t rm = rl <= rh ? (0xffffffffu >> (31 - rh)) & (0xffffffffu << rl) : 0u;
            uint32_t wm = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                wm |= ((cm >> (8 * (q & 3))) & 0xffu) && ((rm >> (16 * (q >> 2))) & 0xffffu) ? 1u << q : 0u;
            sm.e1[buf][threadIdx.x] =
                make_float4(-0.5f * kL2E * c.z, __log2f(c.w), __uint_as_float(cm), __uint_as_float(rm));
            sm.rgb[buf][threadIdx.x] = make_float4(rgb.x, rgb.y, rgb.z, 1.0f / c.w);
            sm.rank[buf][threadIdx.x] = rk;
            sm.wm[buf][threadIdx.x] = wm;
        }
    };
    auto strip_mask = [&](const uint32_t* s_wm, int m0, int cnt) -> uint32_t {
        const int jl = m0 + lane;
        return __ballot_sync(0xffffffffu, jl < cnt && ((s_wm[jl] >> warp) & 1u));
    };

    if (WALK1) {
        // (C_end, T_end) in the forward's arithmetic
        int buf = 0;
        for (int base = 0; base < L; base += NT, buf ^= 1) {
            stage(base, buf);
            __syncthreads();
            const int cnt = min(NT, L - base);
            const float4* s_e0 = sm.e0[buf];
            const float4* s_e1 = sm.e1[buf];
            const float4* s_rgb = sm.rgb[buf];
            for (int m0 = 0; m0 < cnt; m0 += 32) {
                uint32_t mask = strip_mask(sm.wm[buf], m0, cnt);
                while (mask) {
                    const int j = m0 + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float4 e0 = s_e0[j];
                    const float4 e1 = s_e1[j];
                    const float4 col = s_rgb[j];
                    const uint32_t m = (__float_as_uint(e1.z) >> csh) & 1u ? __float_as_uint(e1.w) >> rsh : 0u;
                    const float dx = fpx - e0.x;
                    const float g1 = e0.w * dx;
                    const float g0 = fmaf(e0.z * dx, dx, e1.y);
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        if (m & (1u << (4 * s))) {
                            const float dy = (float)(py0 + 4 * s) - e0.y;
                            const float pw = fmaf(fmaf(e1.x, dy, g1), dy, g0);
                            const float al = fminf(0.99f, ex2_approx(pw));
                            const float ta = T[s] * al;
                            C[s][0] = fmaf(ta, col.x, C[s][0]);
                            C[s][1] = fmaf(ta, col.y, C[s][1]);
                            C[s][2] = fmaf(ta, col.z, C[s][2]);
                            T[s] = fmaf(-T[s], al, T[s]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            K[s] = fmaf(C[s][0], dC[s][0], fmaf(C[s][1], dC[s][1], fmaf(C[s][2], dC[s][2], -T[s] * dA[s])));
            C[s][0] = C[s][1] = C[s][2] = 0.f, T[s] = 1.f;
        }
        __syncthreads();   // the walk's last reads before the buffers are staged again
    }

    int buf = 0;
    for (int base = 0; base < L; base += NT, buf ^= 1) {
        stage(base, buf);
        // orders this batch's staging before its walk, and every warp's walk
        // of the batch before last before this staging overwrote its buffer
        __syncthreads();
        const int cnt = min(NT, L - base);
        const float4* s_e0 = sm.e0[buf];
        const float4* s_e1 = sm.e1[buf];
        const float4* s_rgb = sm.rgb[buf];
        const uint32_t* s_rank = sm.rank[buf];
        for (int m0 = 0; m0 < cnt; m0 += 32) {
            uint32_t mask = strip_mask(sm.wm[buf], m0, cnt);
            while (mask) {
                const int j = m0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 e0 = s_e0[j];
                const float4 e1 = s_e1[j];
                const float4 col = s_rgb[j];
                // slot s of this lane lies in the footprint iff bit 4 s of m is set
                const uint32_t m = (__float_as_uint(e1.z) >> csh) & 1u ? __float_as_uint(e1.w) >> rsh : 0u;
                const float dx = fpx - e0.x;
                const float g1 = e0.w * dx;
                const float g0 = fmaf(e0.z * dx, dx, e1.y);
                // v: Su, Sv, Saa, Sbb, Scc, So, Sr, Sg; sbl: blue
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float sbl = 0.f;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    if (m & (1u << (4 * s))) {
                        const float dy = (float)(py0 + 4 * s) - e0.y;
                        const float pw = fmaf(fmaf(e1.x, dy, g1), dy, g0);
                        const float araw = ex2_approx(pw);
                        const float al = fminf(0.99f, araw);
                        const float Ti = T[s];
                        const float ta = Ti * al;
                        const float wv = fmaf(col.x, dC[s][0], fmaf(col.y, dC[s][1], fmaf(col.z, dC[s][2], dA[s])));
                        C[s][0] = fmaf(ta, col.x, C[s][0]);
                        C[s][1] = fmaf(ta, col.y, C[s][1]);
                        C[s][2] = fmaf(ta, col.z, C[s][2]);
                        T[s] = fmaf(-Ti, al, Ti);
                        v[6] = fmaf(ta, dC[s][0], v[6]);
                        v[7] = fmaf(ta, dC[s][1], v[7]);
                        sbl = fmaf(ta, dC[s][2], sbl);
                        if (araw < 0.99f) {
                            const float R = fmaf(T[s], dA[s],
                                                 K[s] - fmaf(C[s][0], dC[s][0],
                                                             fmaf(C[s][1], dC[s][1], C[s][2] * dC[s][2])));
                            const float dal = fmaf(Ti, wv, -__fdividef(R, 1.0f - al));
                            v[5] = fmaf(dal, araw * col.w, v[5]);     // G = alpha / o
                            const float dq = -0.5f * dal * al;
                            const float u = dq * dx, vv = dq * dy;
                            v[0] += u;
                            v[1] += vv;
                            v[2] = fmaf(u, dx, v[2]);
                            v[3] = fmaf(u, dy, v[3]);
                            v[4] = fmaf(vv, dy, v[4]);
                        }
                    }
                }
                const float r = warp_reduce_scatter8(v, lane);
                sbl = warp_sum(sbl);
                // lane 0: Su .. Sbb; lane 16: Scc, So, Sr, Sg
                const float r1 = __shfl_down_sync(0xffffffffu, r, 4);
                const float r2 = __shfl_down_sync(0xffffffffu, r, 8);
                const float r3 = __shfl_down_sync(0xffffffffu, r, 12);
                if ((lane & 15) == 0) {
                    float4* acc = g2d + 3 * (size_t)s_rank[j];
                    if (lane == 0) {
                        // raw conic from the staged (A, B, C) = -log2(e) (a/2, b, c/2)
                        const float ca = e0.z * (-2.0f / kL2E), cb = e0.w * (-1.0f / kL2E),
                                    cc = e1.x * (-2.0f / kL2E);
                        atomicAdd(acc, make_float4(-2.0f * fmaf(ca, r, cb * r1), -2.0f * fmaf(cb, r, cc * r1), r2,
                                                   2.0f * r3));
                        atomicAdd(&acc[2].x, sbl);
                    } else {
                        atomicAdd(acc + 1, make_float4(r, r1, r2, r3));
                    }
                }
            }
        }
    }
}

// Lists no longer than r_seg and the parts of the longer ones, one grid:
// CTA b < r_nslots takes part item b (CTAs past r_heavy exit), the others
// the list (b - r_nslots) of (super-tile, chunk) order, longer lists exiting.
template <int DT>
// three CTAs per SM (80 registers): 18 % faster than two at 87
__global__ void __launch_bounds__(kGaussBwdThreads, 3) k_raster_gauss_bwd(BuildWs w, RasterParams p,
                                                                      const uint32_t* __restrict__ ranks,
                                                                      const void* __restrict__ planes,
                                                                      const float4* __restrict__ dplanes,
                                                                      float4* __restrict__ g2d)
{
    __shared__ GaussBwdSmem sm;
    if (w.hdr->overflow) return;
    const long long b = blockIdx.x;
    if (b < w.r_nslots) {
        if (b >= (long long)w.hdr->r_heavy) return;
        const int4 it = w.r_items[b];
        const int st = it.x / p.N;
        raster_gauss_bwd_list<DT, true>(w, p, ranks, planes, dplanes, g2d, st, it.x - st * p.N, sm, it.y, it.z, it.w,
                                        w.hdr->r_seg);
    } else {
        const int supers = p.supers_x * p.supers_y;
        const int li = (int)(b - w.r_nslots);
        const int st = li % supers, k = li / supers;
        const int2 sg = w.seg[(size_t)st * p.N + k];
        if (sg.y - sg.x > w.hdr->r_seg || sg.y == sg.x) return;
        raster_gauss_bwd_list<DT, false>(w, p, ranks, planes, dplanes, g2d, st, k, sm, 0, 1, -1, 0);
    }
}

// Voxels, front to back and pair-parallel, in the forward's layout (one CTA
// of 256 threads per (16 x 16 tile, chunk), thread t owning tile pixel
// (t % 16, t / 16), the footprints of each batch of staged voxels clipped to
// the tile and numbered as pairs). With alpha_i = 1 - e^{-I_i},
//   dL/dI_i = (1 - alpha_i) dL/dalpha_i = T_{i+1} w_i - R_i
// (w_i, R_i and K as for Gaussians), with no division: an opacity that
// rounds to 1 needs no care. I_i = (t1 - t0)/6 (s(t0) + 4 s(tm) + s(t1)),
// s = sum_c W_c(f) rho_c (trilinear weights), so dI_i/drho_c is the
// Simpson-weighted sum of the three samples' weights. Per batch, and per
// pass of at most kVoxBwdPairs pairs:
//   0) pair-parallel: every pair's opacity, the forward's arithmetic;
//   A) per pixel, its pairs in list order (each warp visits the voxels that
//      touch its two rows): T_i alpha_i and dL/dI_i of the pair into shared
//      memory, C and T carried exactly as the forward carries them;
//   B) pair-parallel: the pair's weights, dL/drho_c += dL/dI_i dI_i/drho_c
//      and dL/dc += T_i alpha_i dC, summed per voxel in shared memory;
// then one thread per staged voxel adds the sums to the voxel's accumulator
// (rank order): g2d[3 r .. 3 r + 2] = {d rho_0..3}, {d rho_4..7},
// {d r, d g, d b, 0}. K: from the forward's texel with FP32 planes; other
// plane types first walk the list once (phases 0 and A, C and T only).
constexpr int kVoxBwdPairs = 1024;

struct VoxBwdSmem {
    float4 box[kTilePix];
    float inv_side[kTilePix];
    float den[kTilePix * 8];      // trilinear polynomial coefficients (the forward's)
    float4 rgb[kTilePix];
    int4 rect[kTilePix];          // footprint clipped to the tile, tile-local
    int off[kTilePix];            // number of the voxel's first pair
    uint32_t rank[kTilePix];
    float4 dir[kTilePix];         // per pixel: unit reference-ray direction
    float4 inv[kTilePix];         // per pixel: its reciprocal
    float4 grad[kTilePix];        // per pixel: (dC, dA)
    float acc[kTilePix][12];      // per staged voxel: d rho (8), d rgb (3)
    uint16_t pair[kVoxBwdPairs];  // voxel slot | x << 8 | y << 12
    float alpha[kVoxBwdPairs];
    float dI[kVoxBwdPairs];
    float ta[kVoxBwdPairs];
    int wc[kTilePix / 32];
    int ws[kTilePix / 32];
};

__device__ __forceinline__ void tri_weights(float fx, float fy, float fz, float s, float* Wc)
{
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    Wc[0] = fmaf(s, gx * gy * gz, Wc[0]);
    Wc[1] = fmaf(s, fx * gy * gz, Wc[1]);
    Wc[2] = fmaf(s, gx * fy * gz, Wc[2]);
    Wc[3] = fmaf(s, fx * fy * gz, Wc[3]);
    Wc[4] = fmaf(s, gx * gy * fz, Wc[4]);
    Wc[5] = fmaf(s, fx * gy * fz, Wc[5]);
    Wc[6] = fmaf(s, gx * fy * fz, Wc[6]);
    Wc[7] = fmaf(s, fx * fy * fz, Wc[7]);
}

// dI/drho_c of one voxel for one reference ray (the geometry of
// voxel_alpha): false when the ray misses the cube (I = 0, no gradient)
__device__ __forceinline__ bool voxel_weights(const float4 b, const float is, const float d[3], const float inv[3],
                                              float Wc[8])
{
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
    if (miss || !(t1 > t0)) return false;
    const float tm = 0.5f * (t0 + t1);
    const float len6 = (t1 - t0) * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 8; ++c) Wc[c] = 0.f;
    tri_weights(clamp01((t0 * d[0] - lo[0]) * is), clamp01((t0 * d[1] - lo[1]) * is),
                clamp01((t0 * d[2] - lo[2]) * is), len6, Wc);
    tri_weights(clamp01((tm * d[0] - lo[0]) * is), clamp01((tm * d[1] - lo[1]) * is),
                clamp01((tm * d[2] - lo[2]) * is), 4.0f * len6, Wc);
    tri_weights(clamp01((t1 * d[0] - lo[0]) * is), clamp01((t1 * d[1] - lo[1]) * is),
                clamp01((t1 * d[2] - lo[2]) * is), len6, Wc);
    return true;
}

template <int DT>
__global__ void __launch_bounds__(kTilePix) k_raster_voxel_bwd(BuildWs w, RasterParams p,
                                                               const uint32_t* __restrict__ ranks,
                                                               const void* __restrict__ planes,
                                                               const float4* __restrict__ dplanes,
                                                               float4* __restrict__ g2d)
{
    constexpr int NT = kTilePix;
    extern __shared__ __align__(16) unsigned char vox_smem[];
    VoxBwdSmem& sm = *reinterpret_cast<VoxBwdSmem*>(vox_smem);
    if (w.hdr->overflow) return;
    const int t = blockIdx.x, k = blockIdx.y;
    const int tx = t % p.tiles_x, ty = t / p.tiles_x;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const int wy0 = 2 * (threadIdx.x >> 5), wy1 = wy0 + 1;   // this warp's two tile rows
    const int st = (ty / kTilesPerSuper) * p.supers_x + tx / kTilesPerSuper;
    const int2 sg = w.seg[(size_t)st * p.N + k];
    const int L = sg.y - sg.x;
    if (L == 0) return;

    const bool in = px < p.W && py < p.H;
    const size_t idx = ((size_t)k * p.H + py) * p.W + px;
    const float4 g = in ? __ldg(dplanes + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
    {
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
        sm.dir[threadIdx.x] = make_float4(d[0], d[1], d[2], 0.f);
        sm.inv[threadIdx.x] = make_float4(inv[0], inv[1], inv[2], 0.f);
        sm.grad[threadIdx.x] = g;
    }
    float K = 0.f;
    if (DT == LF_F32) {
        const float4 tt = in ? __ldg(reinterpret_cast<const float4*>(planes) + idx) : make_float4(0.f, 0.f, 0.f, 1.f);
        K = fmaf(tt.x, g.x, fmaf(tt.y, g.y, fmaf(tt.z, g.z, -(1.0f - tt.w) * g.w)));
    }
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;

    // one walk over the list; GRAD false: C and T only
    auto walk = [&](const bool grad) {
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
            const int slot = compact_slot<NT>(hit, sm.wc, &cnt);
            int4 cr = make_int4(0, 0, -1, -1);
            if (hit) {
                cr = make_int4(max(r.x - tx * kTile, 0), max(r.y - ty * kTile, 0), min(r.z - tx * kTile, kTile - 1),
                               min(r.w - ty * kTile, kTile - 1));
                const float4 box = w.r_geo[rk];
                sm.box[slot] = box;
                sm.inv_side[slot] = 1.0f / box.w;
                const float4 da = w.r_den[2 * (size_t)rk], db = w.r_den[2 * (size_t)rk + 1];
                const float rho8[8] = {da.x, da.y, da.z, da.w, db.x, db.y, db.z, db.w};
                trilinear_coeffs(rho8, sm.den + 8 * slot);
                sm.rgb[slot] = w.r_rgb[rk];
                sm.rect[slot] = cr;
                sm.rank[slot] = rk;
#pragma unroll
                for (int c = 0; c < 12; ++c) sm.acc[slot][c] = 0.f;
            }
            int P;
            const int off = block_exscan_256(hit ? (cr.z - cr.x + 1) * (cr.w - cr.y + 1) : 0, sm.ws, &P);
            if (hit) sm.off[slot] = off;
            __syncthreads();
            for (int c0 = 0; c0 < P; c0 += kVoxBwdPairs) {
                const int c1 = min(P, c0 + kVoxBwdPairs);
                if (hit && off < c1) {
                    int q = off;
                    for (int yy = cr.y; yy <= cr.w && q < c1; ++yy)
                        for (int xx = cr.x; xx <= cr.z && q < c1; ++xx, ++q)
                            if (q >= c0) sm.pair[q - c0] = (uint16_t)(slot | (xx << 8) | (yy << 12));
                }
                __syncthreads();
                // 0) opacities
                for (int q = threadIdx.x; q < c1 - c0; q += NT) {
                    const uint32_t e = sm.pair[q];
                    const int j = e & 0xff, pix = (int)((e >> 12) << 4) + (int)((e >> 8) & 15);
                    const float4 dd = sm.dir[pix], iv = sm.inv[pix];
                    const float d[3] = {dd.x, dd.y, dd.z}, inv[3] = {iv.x, iv.y, iv.z};
                    sm.alpha[q] = voxel_alpha(sm.box[j], sm.inv_side[j], sm.den + 8 * j, d, inv);
                }
                __syncthreads();
                // A) per pixel, in list order
                for (int m0 = 0; m0 < cnt; m0 += 32) {
                    const int jl = m0 + (threadIdx.x & 31);
                    bool touches = false;
                    if (jl < cnt) {
                        const int4 rl = sm.rect[jl];
                        touches = rl.y <= wy1 && rl.w >= wy0;
                    }
                    uint32_t vmask = __ballot_sync(0xffffffffu, touches);
                    while (vmask) {
                        const int j = m0 + __ffs(vmask) - 1;
                        vmask &= vmask - 1;
                        const int4 rc = sm.rect[j];
                        if (lx < rc.x || lx > rc.z || ly < rc.y || ly > rc.w) continue;
                        const int q = sm.off[j] + (ly - rc.y) * (rc.z - rc.x + 1) + (lx - rc.x);
                        if (q < c0 || q >= c1) continue;
                        const float al = sm.alpha[q - c0];
                        const float4 col = sm.rgb[j];
                        const float ta = T * al;
                        C0 = fmaf(ta, col.x, C0);
                        C1 = fmaf(ta, col.y, C1);
                        C2 = fmaf(ta, col.z, C2);
                        T = T * (1.0f - al);
                        if (grad) {
                            const float wv = fmaf(col.x, g.x, fmaf(col.y, g.y, fmaf(col.z, g.z, g.w)));
                            const float R = fmaf(T, g.w, K - fmaf(C0, g.x, fmaf(C1, g.y, C2 * g.z)));
                            sm.dI[q - c0] = fmaf(T, wv, -R);
                            sm.ta[q - c0] = ta;
                        }
                    }
                }
                if (grad) {
                    __syncthreads();
                    // B) weights and per-voxel sums
                    for (int q = threadIdx.x; q < c1 - c0; q += NT) {
                        const uint32_t e = sm.pair[q];
                        const int j = e & 0xff, pix = (int)((e >> 12) << 4) + (int)((e >> 8) & 15);
                        const float4 dd = sm.dir[pix], iv = sm.inv[pix];
                        const float d[3] = {dd.x, dd.y, dd.z}, inv[3] = {iv.x, iv.y, iv.z};
                        float Wc[8];
                        if (!voxel_weights(sm.box[j], sm.inv_side[j], d, inv, Wc)) continue;
                        const float dI = sm.dI[q], ta = sm.ta[q];
                        const float4 gp = sm.grad[pix];
                        float* acc = sm.acc[j];
#pragma unroll
                        for (int c = 0; c < 8; ++c) atomicAdd(acc + c, dI * Wc[c]);
                        atomicAdd(acc + 8, ta * gp.x);
                        atomicAdd(acc + 9, ta * gp.y);
                        atomicAdd(acc + 10, ta * gp.z);
                    }
                }
                // the next pass overwrites the pairs; the next batch restages
                __syncthreads();
            }
            if (grad && threadIdx.x < cnt) {
                const float* a = sm.acc[threadIdx.x];
                float4* dst = g2d + 3 * (size_t)sm.rank[threadIdx.x];
                atomicAdd(dst, make_float4(a[0], a[1], a[2], a[3]));
                atomicAdd(dst + 1, make_float4(a[4], a[5], a[6], a[7]));
                atomicAdd(dst + 2, make_float4(a[8], a[9], a[10], 0.f));
            }
            __syncthreads();
        }
    };

    if (DT != LF_F32) {
        walk(false);
        K = fmaf(C0, g.x, fmaf(C1, g.y, fmaf(C2, g.z, -T * g.w)));
        C0 = C1 = C2 = 0.f, T = 1.f;
    }
    walk(true);
}

}  // namespace

void launch_raster_gaussians_bwd(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks,
                                 const void* planes, const float* dplanes, cudaStream_t s)
{
    const long long ctas = ws.r_nslots + (long long)p.supers_x * p.supers_y * p.N;
    const dim3 grid((unsigned)ctas);
    const float4* dp = reinterpret_cast<const float4*>(dplanes);
    float4* g = reinterpret_cast<float4*>(ws.g2d);
    switch (p.dtype) {
    case LF_F32: k_raster_gauss_bwd<LF_F32><<<grid, kGaussBwdThreads, 0, s>>>(ws, p, ranks, planes, dp, g); break;
    case LF_F16: k_raster_gauss_bwd<LF_F16><<<grid, kGaussBwdThreads, 0, s>>>(ws, p, ranks, planes, dp, g); break;
    case LF_U8: k_raster_gauss_bwd<LF_U8><<<grid, kGaussBwdThreads, 0, s>>>(ws, p, ranks, planes, dp, g); break;
    default: k_raster_gauss_bwd<LF_BF16><<<grid, kGaussBwdThreads, 0, s>>>(ws, p, ranks, planes, dp, g); break;
    }
    note_launches(1);
}

void launch_raster_voxels_bwd(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, const void* planes,
                              const float* dplanes, cudaStream_t s)
{
    const dim3 grid((unsigned)(p.tiles_x * p.tiles_y), (unsigned)p.N);
    const size_t smem = sizeof(VoxBwdSmem);
    const float4* dp = reinterpret_cast<const float4*>(dplanes);
    float4* g = reinterpret_cast<float4*>(ws.g2d);
    switch (p.dtype) {
    case LF_F32:
        cudaFuncSetAttribute(k_raster_voxel_bwd<LF_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_raster_voxel_bwd<LF_F32><<<grid, kTilePix, smem, s>>>(ws, p, ranks, planes, dp, g);
        break;
    case LF_F16:
        cudaFuncSetAttribute(k_raster_voxel_bwd<LF_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_raster_voxel_bwd<LF_F16><<<grid, kTilePix, smem, s>>>(ws, p, ranks, planes, dp, g);
        break;
    case LF_U8:
        cudaFuncSetAttribute(k_raster_voxel_bwd<LF_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_raster_voxel_bwd<LF_U8><<<grid, kTilePix, smem, s>>>(ws, p, ranks, planes, dp, g);
        break;
    default:
        cudaFuncSetAttribute(k_raster_voxel_bwd<LF_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_raster_voxel_bwd<LF_BF16><<<grid, kTilePix, smem, s>>>(ws, p, ranks, planes, dp, g);
        break;
    }
    note_launches(1);
}

long long raster_part_ctas(const BuildWs& ws) { return ws.r_nslots; }

void launch_raster_plan(const BuildWs& ws, const RasterParams& p, bool blend3dgs, cudaStream_t s)
{
    const int lists = p.supers_x * p.supers_y * p.N;
    int blocks = (lists + kPlanThreads - 1) / kPlanThreads;
    blocks = blocks < 1 ? 1 : blocks > 1024 ? 1024 : blocks;
    launch_pdl(k_raster_plan, dim3(blocks), dim3(kPlanThreads), 0, s, ws, lists, blend3dgs ? 0 : 1);
    note_launches(1);
}

template <int DT, bool G3>
static void launch_raster_gauss_dt(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                                   cudaStream_t s)
{
    const dim3 grid((unsigned)(p.supers_x * p.supers_y), (unsigned)p.N);
    if (!G3) {
        launch_overlapped(k_raster_gauss_parts<DT>, dim3((unsigned)raster_part_ctas(ws)), dim3(kGaussThreads), 0, s,
                          ws, p, ranks, planes);
        launch_overlapped(k_raster_gauss<DT, G3>, grid, dim3(kGaussThreads), 0, s, ws, p, ranks, planes);
        note_launches(2);
    } else {
        launch_pdl(k_raster_gauss<DT, G3>, grid, dim3(kGaussThreads), 0, s, ws, p, ranks, planes);
        note_launches(1);
    }
}

void launch_raster_gaussians(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                             bool blend3dgs, cudaStream_t s)
{
    launch_raster_plan(ws, p, blend3dgs, s);
    switch (p.dtype) {
    case LF_F32: blend3dgs ? launch_raster_gauss_dt<LF_F32, true>(ws, p, ranks, planes, s)
                           : launch_raster_gauss_dt<LF_F32, false>(ws, p, ranks, planes, s); break;
    case LF_F16: blend3dgs ? launch_raster_gauss_dt<LF_F16, true>(ws, p, ranks, planes, s)
                           : launch_raster_gauss_dt<LF_F16, false>(ws, p, ranks, planes, s); break;
    case LF_U8: blend3dgs ? launch_raster_gauss_dt<LF_U8, true>(ws, p, ranks, planes, s)
                          : launch_raster_gauss_dt<LF_U8, false>(ws, p, ranks, planes, s); break;
    default: blend3dgs ? launch_raster_gauss_dt<LF_BF16, true>(ws, p, ranks, planes, s)
                       : launch_raster_gauss_dt<LF_BF16, false>(ws, p, ranks, planes, s); break;
    }
}

void launch_raster_gauss_batched(const RasterScene* scenes_dev, int n_sc, int dtype, long long parts_total,
                                 long long total, cudaStream_t s)
{
    if (n_sc <= 0 || total <= 0) return;
    const unsigned g = (unsigned)total;
    switch (dtype) {
    case LF_F32: k_raster_gauss_batched<LF_F32><<<g, kGaussThreads, 0, s>>>(scenes_dev, n_sc, parts_total); break;
    case LF_F16: k_raster_gauss_batched<LF_F16><<<g, kGaussThreads, 0, s>>>(scenes_dev, n_sc, parts_total); break;
    case LF_U8: k_raster_gauss_batched<LF_U8><<<g, kGaussThreads, 0, s>>>(scenes_dev, n_sc, parts_total); break;
    default: k_raster_gauss_batched<LF_BF16><<<g, kGaussThreads, 0, s>>>(scenes_dev, n_sc, parts_total); break;
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
    case LF_U8: k_raster_voxel<LF_U8><<<grid, kTilePix, 0, s>>>(ws, p, ranks, planes); break;
    default: k_raster_voxel<LF_BF16><<<grid, kTilePix, 0, s>>>(ws, p, ranks, planes); break;
    }
    note_launches(1);
}

}  // namespace lf
