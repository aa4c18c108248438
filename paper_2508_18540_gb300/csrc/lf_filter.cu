// lf_filter.cu -- the V2LF low-pass plane filter (Sec. 4.5), in place.
//
// SVR's supersampling is replaced by a Gaussian low-pass filter on the
// sweeping planes, done in place with no extra memory. Separable: a normalised
// discrete Gaussian w[-r..r] (standard deviation sigma, in plane pixels) over
// the rows, then over the columns, every RGBA channel, transparent zero
// padding outside the plane, FP32 arithmetic, result stored in the plane type.
//  k_filter_rows  one CTA per (plane, row): the row is walked in segments;
//                 each segment and its right halo are read into shared
//                 memory, the left halo is the previous segment's tail of
//                 original texels carried in shared memory, so writing the
//                 segment back never destroys an input still needed.
//  k_filter_cols  one CTA per (plane, strip of 32 columns), 8 threads per
//                 column: walks down the strip in bands of 32 rows; each
//                 band and the r rows below it are read into shared memory
//                 (the r rows above are the previous band's tail of original
//                 texels, carried with the look-ahead), so writing the band
//                 back never destroys an input still needed. Every texel is
//                 read once and written once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kRowThreads = 256;
constexpr int kSeg = 1024;          // texels per row segment
constexpr int kColStrip = 32;   // columns per CTA of the column pass
constexpr int kColLanes = 8;    // threads per column
constexpr int kColBand = 32;    // output rows per step (>= 2 * kFilterMaxRadius: the carry never overlaps)
static_assert(kColBand >= 2 * kFilterMaxRadius, "column carry would overlap");

template <int DT>
__device__ __forceinline__ float4 ld(const void* p, size_t i)
{
    if (DT == LF_F32) return reinterpret_cast<const float4*>(p)[i];
    if (DT == LF_U8) return u8_unpack(reinterpret_cast<const uint32_t*>(p)[i]);
    const uint2 u = reinterpret_cast<const uint2*>(p)[i];
    if (DT == LF_F16) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

template <int DT>
__device__ __forceinline__ void st(void* p, size_t i, float4 v)
{
    if (DT == LF_F32) {
        reinterpret_cast<float4*>(p)[i] = v;
    } else if (DT == LF_U8) {
        reinterpret_cast<uint32_t*>(p)[i] = u8_pack(v.x, v.y, v.z, v.w);
    } else if (DT == LF_F16) {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        reinterpret_cast<uint2*>(p)[i] = u;
    } else {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&lo);
        u.y = *reinterpret_cast<const uint32_t*>(&hi);
        reinterpret_cast<uint2*>(p)[i] = u;
    }
}

__device__ __forceinline__ void fma4(float4& a, float w, float4 v)
{
    a.x = fmaf(w, v.x, a.x);
    a.y = fmaf(w, v.y, a.y);
    a.z = fmaf(w, v.z, a.z);
    a.w = fmaf(w, v.w, a.w);
}

template <int DT>
__global__ void __launch_bounds__(kRowThreads) k_filter_rows(void* planes, int W, int H, FilterParams f)
{
    extern __shared__ float4 buf[];   // [r + kSeg + r]: left halo, segment, right halo
    const int r = f.radius;
    const size_t row = (size_t)blockIdx.x;          // plane * H + y
    const size_t base = row * (size_t)W;
    for (int i = threadIdx.x; i < r; i += kRowThreads) buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int x0 = 0; x0 < W; x0 += kSeg) {
        const int n = min(kSeg, W - x0);
        for (int i = threadIdx.x; i < n + r; i += kRowThreads) {
            const int x = x0 + i;
            buf[r + i] = x < W ? ld<DT>(planes, base + x) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        float4 out[kSeg / kRowThreads];
#pragma unroll
        for (int q = 0; q < kSeg / kRowThreads; ++q) {
            const int i = threadIdx.x + q * kRowThreads;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n)
                for (int t = -r; t <= r; ++t) fma4(a, f.w[t + r], buf[r + i + t]);
            out[q] = a;
        }
        __syncthreads();
        // carry the segment's last r original texels as the next left halo
        if (n == kSeg)
            for (int i = threadIdx.x; i < r; i += kRowThreads) buf[i] = buf[kSeg + i];
#pragma unroll
        for (int q = 0; q < kSeg / kRowThreads; ++q) {
            const int i = threadIdx.x + q * kRowThreads;
            if (i < n) st<DT>(planes, base + x0 + i, out[q]);
        }
        __syncthreads();
    }
}

template <int DT>
__global__ void __launch_bounds__(kColStrip* kColLanes) k_filter_cols(void* planes, int W, int H, FilterParams f)
{
    extern __shared__ float4 cbuf[];   // rows [r + kColBand + r][kColStrip]: top halo, band, look-ahead
    const int r = f.radius;
    const int tx = threadIdx.x % kColStrip, ty = threadIdx.x / kColStrip;
    const int x = blockIdx.x * kColStrip + tx;
    const bool col = x < W;
    const size_t plane = (size_t)blockIdx.y * (size_t)W * H;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // rows -r .. r - 1 of the first band: zero padding above, then originals
    for (int i = ty; i < 2 * r; i += kColLanes) {
        const int y = i - r;
        cbuf[i * kColStrip + tx] = (col && y >= 0 && y < H) ? ld<DT>(planes, plane + (size_t)y * W + x) : zero;
    }
    for (int y0 = 0; y0 < H; y0 += kColBand) {
        const int n = min(kColBand, H - y0);
        // rows y0 + r .. y0 + n + r - 1 (originals; zero below the plane);
        // rows y0 - r .. y0 + r - 1 are already in place
        for (int i = 2 * r + ty; i < n + 2 * r; i += kColLanes) {
            const int y = y0 + i - r;
            cbuf[i * kColStrip + tx] = (col && y < H) ? ld<DT>(planes, plane + (size_t)y * W + x) : zero;
        }
        __syncthreads();
        float4 out[kColBand / kColLanes];
#pragma unroll
        for (int q = 0; q < kColBand / kColLanes; ++q) {
            const int i = ty + q * kColLanes;
            float4 a = zero;
            if (i < n)
                for (int t = -r; t <= r; ++t) fma4(a, f.w[t + r], cbuf[(r + i + t) * kColStrip + tx]);
            out[q] = a;
        }
        __syncthreads();
        // the band's last r rows and the look-ahead become the next band's
        // top halo and first rows (originals: nothing below y0 + n is written yet)
        if (n == kColBand)
            for (int i = threadIdx.x; i < 2 * r * kColStrip; i += blockDim.x) cbuf[i] = cbuf[kColBand * kColStrip + i];
#pragma unroll
        for (int q = 0; q < kColBand / kColLanes; ++q) {
            const int i = ty + q * kColLanes;
            if (col && i < n) st<DT>(planes, plane + (size_t)(y0 + i) * W + x, out[q]);
        }
        __syncthreads();
    }
}

template <int DT>
void launch_filter_t(void* planes, int N, int W, int H, const FilterParams& f, cudaStream_t s)
{
    k_filter_rows<DT><<<(unsigned)((size_t)N * H), kRowThreads, sizeof(float4) * (kSeg + 2 * f.radius), s>>>(
        planes, W, H, f);
    const dim3 grid((unsigned)((W + kColStrip - 1) / kColStrip), (unsigned)N);
    k_filter_cols<DT><<<grid, kColStrip * kColLanes, sizeof(float4) * (kColBand + 2 * f.radius) * kColStrip, s>>>(
        planes, W, H, f);
    note_launches(2);
}

}  // namespace

void launch_filter_planes(void* planes, int dtype, int N, int W, int H, const FilterParams& f, cudaStream_t s)
{
    switch (dtype) {
    case LF_F32: launch_filter_t<LF_F32>(planes, N, W, H, f, s); break;
    case LF_F16: launch_filter_t<LF_F16>(planes, N, W, H, f, s); break;
    case LF_U8: launch_filter_t<LF_U8>(planes, N, W, H, f, s); break;
    default: launch_filter_t<LF_BF16>(planes, N, W, H, f, s); break;
    }
}

}  // namespace lf
