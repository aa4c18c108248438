// lf_tiles.cu -- 3D tiling (Sec. 4.4), two levels: lists are built per
// (32x32 super-tile, chunk) and every raster CTA (16x16 tile, chunk) filters
// its super-tile's list down to the primitives whose footprint meets its
// tile, keeping the order.
//
//  k_dup_count / k_dup_scan / k_dup_emit
//      one (super-tile id, rank) pair per super-tile a primitive's footprint
//      touches, written in rank (depth) order: per-block totals, one scan,
//      then every block writes its pairs at its offset;
//  sort_tile_keys (lf_sort.cu)
//      stable radix sort of the pairs by super-tile id: every list stays in
//      depth order, and chunks (monotone in rank) form contiguous runs;
//  k_ranges
//      [start, end) of every (super-tile, chunk) run.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kT = 256;
constexpr int kPer = kDupBlock / kT;   // consecutive ranks per thread

__device__ __forceinline__ uint32_t tile_count(int4 rc)
{
    if (rc.z < rc.x || rc.w < rc.y) return 0u;
    return (uint32_t)((rc.z / kSuper - rc.x / kSuper + 1) * (rc.w / kSuper - rc.y / kSuper + 1));
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) {
        const uint32_t t = wsum[w];
        before += w < warp ? t : 0u;
        tot += t;
    }
    if (total) *total = tot;
    return before + x - v;
}

__global__ void __launch_bounds__(kT) k_dup_count(BuildWs w)
{
    pdl_wait();
    pdl_trigger();
    const long long M = (long long)w.hdr->M;
    const long long r0 = (long long)blockIdx.x * kDupBlock + (long long)threadIdx.x * kPer;
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j)
        if (r0 + j < M) sum += tile_count(w.r_rect[r0 + j]);
    uint32_t total;
    block_exscan256(sum, &total);
    if (threadIdx.x == 0) w.bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_dup_scan(BuildWs w, int nb)
{
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long wt[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (nb + 1023) / 1024;
    const int b = t * per, e = min(nb, b + per);
    unsigned long long sum = 0;
    for (int i = b; i < e; ++i) sum += w.bsum[i];
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        wt[lane] = s;
    }
    __syncthreads();
    unsigned long long run = (warp ? wt[warp - 1] : 0ull) + x - sum;
    for (int i = b; i < e; ++i) {
        const uint32_t v = w.bsum[i];
        w.bsum[i] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
        run += v;
    }
    if (t == 1023) {
        const unsigned long long total = wt[31];
        w.hdr->total_dups = total;
        const int over = total > (unsigned long long)w.hdr->dup_capacity;
        w.hdr->overflow = over;
        w.hdr->tile_n = over ? 0ull : total;
    }
}

// The block's pairs are written to shared memory at their block-local
// offsets and copied out contiguously (coalesced); a block with more pairs
// than the staging area writes them directly.
constexpr int kEmitStage = 4096;

__global__ void __launch_bounds__(kT) k_dup_emit(BuildWs w, int supers_x)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_key[kEmitStage];
    __shared__ uint32_t s_rank[kEmitStage];
    if (w.hdr->overflow) return;
    const long long M = (long long)w.hdr->M;
    const long long r0 = (long long)blockIdx.x * kDupBlock + (long long)threadIdx.x * kPer;
    int4 rc[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        rc[j] = r0 + j < M ? w.r_rect[r0 + j] : make_int4(0, 0, -1, -1);
        sum += tile_count(rc[j]);
    }
    uint32_t total;
    const uint32_t local = block_exscan256(sum, &total);
    const uint32_t base = w.bsum[blockIdx.x];
    const bool staged = total <= (uint32_t)kEmitStage;
    uint32_t off = local;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (rc[j].z < rc[j].x || rc[j].w < rc[j].y) continue;
        const int sx0 = rc[j].x / kSuper, sx1 = rc[j].z / kSuper, sy0 = rc[j].y / kSuper, sy1 = rc[j].w / kSuper;
        for (int sy = sy0; sy <= sy1; ++sy)
            for (int sx = sx0; sx <= sx1; ++sx) {
                const uint32_t key = (uint32_t)(sy * supers_x + sx), rank = (uint32_t)(r0 + j);
                if (staged) {
                    s_key[off] = key;
                    s_rank[off] = rank;
                } else {
                    w.tkeyA[base + off] = key;
                    w.entA[base + off] = rank;
                }
                ++off;
            }
    }
    if (!staged) return;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < total; i += kT) {
        w.tkeyA[base + i] = s_key[i];
        w.entA[base + i] = s_rank[i];
    }
}

// Entry i starts a (super-tile, chunk) list when its super-tile or chunk
// differs from entry i - 1's; it then also ends the list of entry i - 1. A
// warp takes 32 consecutive entries: the chunk of an entry's rank comes from
// the rank-ordered chunk array, the previous entry's from the lane below.
__global__ void __launch_bounds__(256) k_ranges(BuildWs w, const uint32_t* __restrict__ keys,
                                                const uint32_t* __restrict__ ranks, int N)
{
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)w.hdr->tile_n;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x - lane); i0 < n; i0 += stride) {
        const long long i = i0 + lane;
        const bool in = i < n;
        const uint32_t t = in ? keys[i] : 0u;
        const int c = in ? w.r_chunk[ranks[i]] : 0;
        uint32_t tp = __shfl_up_sync(0xffffffffu, t, 1);
        int cp = __shfl_up_sync(0xffffffffu, c, 1);
        if (lane == 0 && in && i > 0) {
            tp = keys[i - 1];
            cp = w.r_chunk[ranks[i - 1]];
        }
        if (!in) continue;
        const bool first = i == 0 || tp != t || cp != c;
        if (first) {
            w.seg[(long long)t * N + c].x = (int)i;
            if (i > 0) w.seg[(long long)tp * N + cp].y = (int)i;
        }
        if (i == n - 1) w.seg[(long long)t * N + c].y = (int)n;
    }
}

}  // namespace

int tile_bits_for(long long tiles)
{
    int b = 1;
    while ((1ll << b) < tiles) ++b;
    return b;
}

const uint32_t* launch_tile_lists(const BuildWs& ws, long long n, long long cap, int N, int supers_x, int n_supers,
                                  cudaStream_t s)
{
    cudaMemsetAsync(ws.seg, 0, sizeof(int2) * (size_t)n_supers * N, s);
    const int nb = (int)(((n > 0 ? n : 1) + kDupBlock - 1) / kDupBlock);
    launch_pdl(k_dup_count, dim3(nb), dim3(kT), 0, s, ws);
    launch_pdl(k_dup_scan, dim3(1), dim3(1024), 0, s, ws, nb);
    launch_pdl(k_dup_emit, dim3(nb), dim3(kT), 0, s, ws, supers_x);
    note_launches(3);
    uint32_t* keys = nullptr;
    uint32_t* ranks = nullptr;
    sort_tile_keys(ws, cap, tile_bits_for(n_supers), s, &keys, &ranks);
    if (cap > 0) {
        const long long want = (cap + 255) / 256;
        const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
        launch_pdl(k_ranges, dim3(blocks), dim3(256), 0, s, ws, keys, ranks, N);
        note_launches(1);
    }
    return ranks;
}

}  // namespace lf
