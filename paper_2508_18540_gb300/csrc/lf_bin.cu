// lf_bin.cu -- depth binning (the chunking step of Algorithm 1; Sec. 4.4).
//
//  k_bin      rank r of the (depth, index) order -> chunk:
//               quantile:  floor(r N / M)   (equal-count chunks)
//               disparity: min(N-1, floor(N (1/z_min - 1/z) / (1/z_min - 1/z_max)))
//             records the first rank of every chunk (chunks are monotone in
//             rank) and copies the primitive's footprint, colour and
//             projection into rank order for the tile-list and raster kernels.
//  k_medians  d_k = median member depth + D_forward (quantile; mean of the two
//             middle depths for an even count) or the bin's disparity midpoint.
// All FP64 operations use explicit round-to-nearest intrinsics in the order
// of the definitions above. The depth of rank r is the FP64 whose IEEE bits
// are the depth key of primitive valA[r] (keyA, by primitive).
#include "lf_internal.cuh"

namespace lf {

namespace {

__device__ __forceinline__ double rank_depth(const BuildWs& w, long long r)
{
    return __longlong_as_double((long long)w.keyA[w.valA[r]]);
}

__device__ __forceinline__ int chunk_of_rank(const BuildWs& w, const BinParams& p, long long r, long long M)
{
    if (p.binning == LF_BIN_QUANTILE) return (int)((r * (long long)p.N) / M);
    const double zmin = rank_depth(w, 0), zmax = rank_depth(w, M - 1);
    const double izmin = __ddiv_rn(1.0, zmin), izmax = __ddiv_rn(1.0, zmax);
    const double span = __dsub_rn(izmin, izmax);
    if (!(span > 0.0)) return 0;
    const double z = rank_depth(w, r);
    const double f = floor(__ddiv_rn(__dmul_rn((double)p.N, __dsub_rn(izmin, __ddiv_rn(1.0, z))), span));
    return f >= (double)(p.N - 1) ? p.N - 1 : (int)f;
}

__global__ void __launch_bounds__(256) k_bin(BuildWs w, BinParams p, int32_t* chunk_out, const int4* __restrict__ rect,
                                             const float* __restrict__ rgb, const float* __restrict__ dens8, int kind)
{
    pdl_wait();
    pdl_trigger();
    const long long M = (long long)w.hdr->M;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (M == 0) {
        if (r == 0)
            for (int k = 0; k <= p.N; ++k) w.chunk_start[k] = 0;
        return;
    }
    if (r >= M) return;
    const int c = chunk_of_rank(w, p, r, M);
    const uint32_t g = w.valA[r];
    chunk_out[g] = c;
    const int cp = r == 0 ? -1 : chunk_of_rank(w, p, r - 1, M);
    for (int k = cp + 1; k <= c; ++k) w.chunk_start[k] = (int32_t)r;
    if (r == M - 1)
        for (int k = c + 1; k <= p.N; ++k) w.chunk_start[k] = (int32_t)M;
    // rank-ordered copies
    w.r_chunk[r] = c;
    w.r_rect[r] = rect[g];
    w.r_rgb[r] = make_float4(rgb[3 * (size_t)g], rgb[3 * (size_t)g + 1], rgb[3 * (size_t)g + 2], 0.f);
    if (kind == 0) {
        const float2 m = w.mean2d[g];
        w.r_geo[r] = make_float4(m.x, m.y, 0.f, 0.f);
        w.r_con[r] = w.conic_o[g];
    } else {
        w.r_geo[r] = w.conic_o[g];
        const float4* d4 = reinterpret_cast<const float4*>(dens8 + 8 * (size_t)g);
        w.r_den[2 * r] = d4[0];
        w.r_den[2 * r + 1] = d4[1];
    }
}

__global__ void k_medians(BuildWs w, BinParams p, double* d_out, int32_t* count_out)
{
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.N) return;
    const long long M = (long long)w.hdr->M;
    const int lo = w.chunk_start[k], hi = w.chunk_start[k + 1];
    const int c = hi - lo;
    count_out[k] = c;
    double d = 0.0;
    if (p.binning == LF_BIN_QUANTILE) {
        if (c > 0) {
            double med;
            if (c & 1)
                med = rank_depth(w, lo + c / 2);
            else
                med = __dmul_rn(__dadd_rn(rank_depth(w, lo + c / 2 - 1), rank_depth(w, lo + c / 2)),
                                0.5);
            d = __dadd_rn(med, p.D_forward);
        }
    } else if (M > 0) {
        const double izmin = __ddiv_rn(1.0, rank_depth(w, 0));
        const double izmax = __ddiv_rn(1.0, rank_depth(w, M - 1));
        const double span = __dsub_rn(izmin, izmax);
        const double disp = __dsub_rn(izmin, __dmul_rn(__ddiv_rn(__dadd_rn((double)k, 0.5), (double)p.N), span));
        d = __dadd_rn(__ddiv_rn(1.0, disp), p.D_forward);
    }
    d_out[k] = d;
}

}  // namespace

void launch_bin(const BuildWs& ws, const BinParams& p, long long n, int32_t* chunk, double* d, int32_t* count,
                const int32_t* rect, const float* rgb, const float* dens8, int kind, cudaStream_t s)
{
    const unsigned blocks = (unsigned)(((n > 0 ? n : 1) + 255) / 256);
    launch_pdl(k_bin, dim3(blocks), dim3(256), 0, s, ws, p, chunk, reinterpret_cast<const int4*>(rect), rgb, dens8, kind);
    note_launches(1);
    launch_pdl(k_medians, dim3((p.N + 127) / 128), dim3(128), 0, s, ws, p, d, count);
    note_launches(1);
}

}  // namespace lf
