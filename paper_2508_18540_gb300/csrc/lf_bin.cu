// lf_bin.cu -- depth binning and 3D tiling (Algorithm 1 lines 2-3; Sec. 4.4).
//
//  k_bin      rank r of the (depth, index) order -> chunk:
//               quantile:  floor(r N / M)   (equal-count chunks, FindQuantile)
//               disparity: min(N-1, floor(N (1/z_min - 1/z) / (1/z_min - 1/z_max)))
//             and the first rank of every chunk (chunks are monotone in rank).
//  k_medians  d_k = median member depth + D_forward (quantile; mean of the two
//             middle depths for an even count) or the bin's disparity midpoint.
//  k_dup_*    one (tile, primitive) pair per 16x16 tile the footprint touches,
//             emitted in rank order (count, scan, emit).
//  k_ranges   after the stable tile sort: [start, end) of every (tile, chunk).
// All FP64 operations use explicit round-to-nearest intrinsics in the order
// of the definitions above.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kDupThreads = 256;
constexpr int kDupPer = 4;
constexpr int kDupBlock = kDupThreads * kDupPer;

__device__ __forceinline__ double key_depth(unsigned long long k) { return __longlong_as_double((long long)k); }

__device__ __forceinline__ int chunk_of_rank(const BuildWs& w, const BinParams& p, long long r, long long M)
{
    if (p.binning == LF_BIN_QUANTILE) return (int)((r * (long long)p.N) / M);
    const double zmin = key_depth(w.keyA[0]), zmax = key_depth(w.keyA[M - 1]);
    const double izmin = __ddiv_rn(1.0, zmin), izmax = __ddiv_rn(1.0, zmax);
    const double span = __dsub_rn(izmin, izmax);
    if (!(span > 0.0)) return 0;
    const double z = key_depth(w.keyA[r]);
    const double f = floor(__ddiv_rn(__dmul_rn((double)p.N, __dsub_rn(izmin, __ddiv_rn(1.0, z))), span));
    return f >= (double)(p.N - 1) ? p.N - 1 : (int)f;
}

__global__ void __launch_bounds__(256) k_bin(BuildWs w, BinParams p, int32_t* chunk_out)
{
    const long long M = (long long)w.hdr->M;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (M == 0) {
        if (r == 0)
            for (int k = 0; k <= p.N; ++k) w.chunk_start[k] = 0;
        return;
    }
    if (r >= M) return;
    const int c = chunk_of_rank(w, p, r, M);
    chunk_out[w.valA[r]] = c;
    const int cp = r == 0 ? -1 : chunk_of_rank(w, p, r - 1, M);
    for (int k = cp + 1; k <= c; ++k) w.chunk_start[k] = (int32_t)r;
    if (r == M - 1)
        for (int k = c + 1; k <= p.N; ++k) w.chunk_start[k] = (int32_t)M;
}

__global__ void k_medians(BuildWs w, BinParams p, double* d_out, int32_t* count_out)
{
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
                med = key_depth(w.keyA[lo + c / 2]);
            else
                med = __dmul_rn(__dadd_rn(key_depth(w.keyA[lo + c / 2 - 1]), key_depth(w.keyA[lo + c / 2])), 0.5);
            d = __dadd_rn(med, p.D_forward);
        }
    } else if (M > 0) {
        const double izmin = __ddiv_rn(1.0, key_depth(w.keyA[0]));
        const double izmax = __ddiv_rn(1.0, key_depth(w.keyA[M - 1]));
        const double span = __dsub_rn(izmin, izmax);
        const double disp = __dsub_rn(izmin, __dmul_rn(__ddiv_rn(__dadd_rn((double)k, 0.5), (double)p.N), span));
        d = __dadd_rn(__ddiv_rn(1.0, disp), p.D_forward);
    }
    d_out[k] = d;
}

__device__ __forceinline__ uint32_t tile_count(int4 rc)
{
    if (rc.z < rc.x || rc.w < rc.y) return 0u;
    const int tx0 = rc.x / kTile, tx1 = rc.z / kTile, ty0 = rc.y / kTile, ty1 = rc.w / kTile;
    return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t wsum[kDupThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kDupThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        if (lane < kDupThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t before = warp ? wsum[warp - 1] : 0u;
    if (total) *total = wsum[kDupThreads / 32 - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(kDupThreads) k_dup_count(BuildWs w, const int4* __restrict__ rect)
{
    const long long M = (long long)w.hdr->M;
    const long long r0 = (long long)blockIdx.x * kDupBlock + (long long)threadIdx.x * kDupPer;
    uint32_t sum = 0;
    for (int j = 0; j < kDupPer; ++j) {
        const long long r = r0 + j;
        if (r < M) sum += tile_count(rect[w.valA[r]]);
    }
    uint32_t total;
    block_exclusive_scan(sum, &total);
    if (threadIdx.x == 0) w.bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_dup_scan(BuildWs w, int nb)
{
    __shared__ unsigned long long warp_tot[32];
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b = t * per, e = min(nb, b + per);
    unsigned long long sum = 0;
    for (int i = b; i < e; ++i) sum += w.bsum[i];
    unsigned long long v = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if ((t & 31) >= o) v += u;
    }
    if ((t & 31) == 31) warp_tot[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        unsigned long long x = warp_tot[t];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (t >= o) x += u;
        }
        warp_tot[t] = x;
    }
    __syncthreads();
    unsigned long long run = v - sum + ((t >> 5) ? warp_tot[(t >> 5) - 1] : 0ull);
    for (int i = b; i < e; ++i) {
        const uint32_t x = w.bsum[i];
        w.bsum[i] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
        run += x;
    }
    if (t == 1023) {
        const unsigned long long total = warp_tot[31];
        w.hdr->total_dups = total;
        const int over = total > (unsigned long long)w.hdr->dup_capacity;
        w.hdr->overflow = over;
        w.hdr->tile_n = over ? 0ull : total;
    }
}

__global__ void __launch_bounds__(kDupThreads) k_dup_emit(BuildWs w, const int4* __restrict__ rect, int tiles_x)
{
    if (w.hdr->overflow) return;
    const long long M = (long long)w.hdr->M;
    const long long r0 = (long long)blockIdx.x * kDupBlock + (long long)threadIdx.x * kDupPer;
    uint32_t sum = 0;
    for (int j = 0; j < kDupPer; ++j) {
        const long long r = r0 + j;
        if (r < M) sum += tile_count(rect[w.valA[r]]);
    }
    uint32_t off = w.bsum[blockIdx.x] + block_exclusive_scan(sum, nullptr);
    for (int j = 0; j < kDupPer; ++j) {
        const long long r = r0 + j;
        if (r >= M) break;
        const uint32_t g = w.valA[r];
        const int4 rc = rect[g];
        if (rc.z < rc.x || rc.w < rc.y) continue;
        const int tx0 = rc.x / kTile, tx1 = rc.z / kTile, ty0 = rc.y / kTile, ty1 = rc.w / kTile;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                w.dkeyA[off] = (uint32_t)(ty * tiles_x + tx);
                w.dvalA[off] = g;
                ++off;
            }
    }
}

__device__ __forceinline__ void range_one(const BuildWs& w, const uint32_t* __restrict__ keys,
                                          const uint32_t* __restrict__ vals, const int32_t* __restrict__ chunk,
                                          int N, long long n, long long i);

__global__ void __launch_bounds__(256) k_ranges(BuildWs w, const uint32_t* __restrict__ keys,
                                                const uint32_t* __restrict__ vals, const int32_t* __restrict__ chunk,
                                                int N)
{
    const long long n = (long long)w.hdr->tile_n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        range_one(w, keys, vals, chunk, N, n, i);
}

__device__ __forceinline__ void range_one(const BuildWs& w, const uint32_t* __restrict__ keys,
                                          const uint32_t* __restrict__ vals, const int32_t* __restrict__ chunk,
                                          int N, long long n, long long i)
{
    const uint32_t t = keys[i];
    const int c = chunk[vals[i]];
    const long long sidx = (long long)t * N + c;
    bool first = i == 0, last = i == n - 1;
    if (!first) first = keys[i - 1] != t || chunk[vals[i - 1]] != c;
    if (!last) last = keys[i + 1] != t || chunk[vals[i + 1]] != c;
    if (first) w.seg[sidx].x = (int)i;
    if (last) w.seg[sidx].y = (int)(i + 1);
}

}  // namespace

void launch_bin(const BuildWs& ws, const BinParams& p, long long n, int32_t* chunk, double* d, int32_t* count,
                cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n > 0 ? n : 1) + 255) / 256;
    k_bin<<<blocks, 256, 0, s>>>(ws, p, chunk);
    note_launches(1);
    k_medians<<<(p.N + 127) / 128, 128, 0, s>>>(ws, p, d, count);
    note_launches(1);
}

void launch_duplicate(const BuildWs& ws, long long n, const int32_t* rect, int tiles_x, cudaStream_t s)
{
    const int nb = (int)(((n > 0 ? n : 1) + kDupBlock - 1) / kDupBlock);
    const int4* r4 = reinterpret_cast<const int4*>(rect);
    k_dup_count<<<nb, kDupThreads, 0, s>>>(ws, r4);
    note_launches(1);
    k_dup_scan<<<1, 1024, 0, s>>>(ws, nb);
    note_launches(1);
    k_dup_emit<<<nb, kDupThreads, 0, s>>>(ws, r4, tiles_x);
    note_launches(1);
}

void launch_ranges(const BuildWs& ws, long long cap, const uint32_t* tkeys, const uint32_t* tvals, const int32_t* chunk,
                   int N, cudaStream_t s)
{
    if (cap <= 0) return;
    // grid-stride over the device-side pair count
    const long long want = (cap + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    k_ranges<<<blocks, 256, 0, s>>>(ws, tkeys, tvals, chunk, N);
    note_launches(1);
}

}  // namespace lf
