// lf_tiles.cu -- 3D tiling (Sec. 4.4): the list of every (16x16 tile, chunk)
// pair, holding the ranks of the chunk's primitives whose footprint meets
// the tile.
//
//  k_seg_count  one counter per (tile, chunk), bumped for every tile a
//               primitive's footprint rectangle touches;
//  k_seg_scan_* exclusive scan of the counters -> [start, end) of every list,
//               total pair count (overflow check against the capacity) and the
//               lists longer than kSegSortCap;
//  k_seg_emit   writes every rank into its list through a countdown cursor
//               (list order arbitrary at this point);
//  k_sort_big   sorts the long lists by rank (ranks in a list are distinct
//               and lie inside their chunk's rank range: a shared-memory
//               bitmap over that range, compacted in order). Lists up to
//               kSegSortCap are sorted by the raster CTA that consumes them.
// Rank order is depth order, so every list ends in front-to-back order.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kT = 256;
constexpr int kBigWords = 8192;   // 32 KB bitmap: 262144 ranks per window

__device__ __forceinline__ void tile_span(int4 rc, int& tx0, int& tx1, int& ty0, int& ty1)
{
    tx0 = rc.x / kTile;
    tx1 = rc.z / kTile;
    ty0 = rc.y / kTile;
    ty1 = rc.w / kTile;
}

__global__ void __launch_bounds__(kT) k_seg_count(BuildWs w, int N, int tiles_x)
{
    const long long M = (long long)w.hdr->M;
    const long long r = (long long)blockIdx.x * kT + threadIdx.x;
    if (r >= M) return;
    const int4 rc = w.r_rect[r];
    const int c = w.r_chunk[r];
    int tx0, tx1, ty0, ty1;
    tile_span(rc, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&w.segcnt[((size_t)ty * tiles_x + tx) * N + c], 1u);
}

__device__ __forceinline__ uint32_t block_sum_1024(uint32_t v, uint32_t* wtmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wtmp[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    if (warp == 0) {
        t = wtmp[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in warp 0
}

// exclusive scan of one value per thread over a 1024-thread block
__device__ __forceinline__ uint32_t block_exscan_1024(uint32_t v, uint32_t* wtmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) wtmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = wtmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        wtmp[lane] = s;
    }
    __syncthreads();
    return (warp ? wtmp[warp - 1] : 0u) + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_seg_scan_a(BuildWs w, long long S)
{
    __shared__ uint32_t wtmp[32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t v = i < S ? w.segcnt[i] : 0u;
    const uint32_t t = block_sum_1024(v, wtmp);
    if (threadIdx.x == 0) w.bsum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_seg_scan_b(BuildWs w, int nbs)
{
    __shared__ unsigned long long wt[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (nbs + 1023) / 1024;
    const int b = t * per, e = min(nbs, b + per);
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
        w.hdr->overflow = total > (unsigned long long)w.hdr->dup_capacity;
    }
}

__global__ void __launch_bounds__(kScanBlock) k_seg_scan_c(BuildWs w, long long S)
{
    __shared__ uint32_t wtmp[32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t v = i < S ? w.segcnt[i] : 0u;
    const uint32_t start = w.bsum[blockIdx.x] + block_exscan_1024(v, wtmp);
    if (i >= S) return;
    if (w.hdr->overflow) {
        w.seg[i] = make_int2(0, 0);
        return;
    }
    w.seg[i] = make_int2((int)start, (int)(start + v));
    if (v > (uint32_t)kSegSortCap) w.biglist[atomicAdd(&w.hdr->n_big, 1ull)] = (uint32_t)i;
}

__global__ void __launch_bounds__(kT) k_seg_emit(BuildWs w, int N, int tiles_x)
{
    if (w.hdr->overflow) return;
    const long long M = (long long)w.hdr->M;
    const long long r = (long long)blockIdx.x * kT + threadIdx.x;
    if (r >= M) return;
    const int4 rc = w.r_rect[r];
    const int c = w.r_chunk[r];
    int tx0, tx1, ty0, ty1;
    tile_span(rc, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const size_t s = ((size_t)ty * tiles_x + tx) * N + c;
            const uint32_t left = atomicSub(&w.segcnt[s], 1u);
            w.entA[(size_t)w.seg[s].x + left - 1u] = (uint32_t)r;
        }
}

__global__ void __launch_bounds__(kT) k_sort_big(BuildWs w, int N)
{
    __shared__ uint32_t bm[kBigWords];
    __shared__ uint32_t wtmp[kT / 32];
    const unsigned long long nbig = w.hdr->n_big;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int P = kBigWords / kT;
    for (unsigned long long bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const uint32_t s = w.biglist[bi];
        const int c = (int)(s % (uint32_t)N);
        const int2 sg = w.seg[s];
        const uint32_t lo = (uint32_t)w.chunk_start[c], hi = (uint32_t)w.chunk_start[c + 1];
        uint32_t out = (uint32_t)sg.x;
        for (uint32_t w0 = lo; w0 < hi; w0 += 32u * kBigWords) {
            for (int i = threadIdx.x; i < kBigWords; i += kT) bm[i] = 0u;
            __syncthreads();
            for (int i = sg.x + threadIdx.x; i < sg.y; i += kT) {
                const uint32_t rk = w.entA[i];
                if (rk >= w0 && rk - w0 < 32u * kBigWords) atomicOr(&bm[(rk - w0) >> 5], 1u << ((rk - w0) & 31u));
            }
            __syncthreads();
            uint32_t cnt = 0;
#pragma unroll 4
            for (int q = 0; q < P; ++q) cnt += __popc(bm[threadIdx.x * P + q]);
            // block exclusive scan of cnt
            uint32_t x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            if (lane == 31) wtmp[warp] = x;
            __syncthreads();
            uint32_t before = 0, total = 0;
#pragma unroll
            for (int q = 0; q < kT / 32; ++q) {
                before += q < warp ? wtmp[q] : 0u;
                total += wtmp[q];
            }
            uint32_t o = out + before + x - cnt;
            for (int q = 0; q < P; ++q) {
                const int word = threadIdx.x * P + q;
                uint32_t bits = bm[word];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    w.entB[o++] = w0 + 32u * (uint32_t)word + (uint32_t)b;
                }
            }
            out += total;
            __syncthreads();
        }
        for (int i = sg.x + threadIdx.x; i < sg.y; i += kT) w.entA[i] = w.entB[i];
        __syncthreads();
    }
}

}  // namespace

void launch_tile_lists(const BuildWs& ws, long long n, long long cap, int N, int tiles_x, int n_tiles, cudaStream_t s)
{
    (void)cap;
    const long long S = (long long)n_tiles * N;
    cudaMemsetAsync(ws.segcnt, 0, sizeof(uint32_t) * (size_t)S, s);
    const unsigned rb = (unsigned)(((n > 0 ? n : 1) + kT - 1) / kT);
    k_seg_count<<<rb, kT, 0, s>>>(ws, N, tiles_x);
    const int nbs = (int)((S + kScanBlock - 1) / kScanBlock);
    k_seg_scan_a<<<nbs, kScanBlock, 0, s>>>(ws, S);
    k_seg_scan_b<<<1, 1024, 0, s>>>(ws, nbs);
    k_seg_scan_c<<<nbs, kScanBlock, 0, s>>>(ws, S);
    k_seg_emit<<<rb, kT, 0, s>>>(ws, N, tiles_x);
    k_sort_big<<<2 * 152, kT, 0, s>>>(ws, N);
    note_launches(6);
}

}  // namespace lf
