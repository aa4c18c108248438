// lf_sort.cu -- stable LSD radix sort of (key, primitive id) pairs.
//
// Used twice per build: the depth sort of Algorithm 1 line 3
// ("Sort_and_Chunk": primitives ordered by (FP64 reference depth, index),
// 64-bit keys, culled primitives dropped in the first pass), and the stable
// regrouping of (tile, primitive) pairs by tile id, which keeps every tile's
// list in depth order (the per-tile sort of the 3D-tiled rasteriser, Sec. 4.4).
//
// Each pass is reduce-then-scan: per-block digit histograms (upsweep), one
// exclusive scan over (digit, block), and a stable scatter (downsweep) that
// ranks equal digits within a block with warp match + per-warp counters.
// Item counts may live on the device (culled-in count, pair count), so the
// grids are sized for the capacity and blocks past the count only write
// zero histograms. A pass whose digit is the same for every key (known from
// the key range) degenerates to a copy.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kWarps = kSortThreads / 32;

struct PassArgs {
    long long n_static;                    // upper bound / fixed count
    const unsigned long long* n_dev;       // device count (or null)
    const unsigned long long* kmin;        // key range (or null): uniform-digit test
    const unsigned long long* kmax;
    int shift;
    int drop_invalid;                      // first depth pass: skip kInvalidKey
    int nb;                                // number of blocks (histogram stride)
};

__device__ __forceinline__ long long pass_count(const PassArgs& a)
{
    return a.n_dev ? (long long)*a.n_dev : a.n_static;
}

__device__ __forceinline__ bool pass_uniform(const PassArgs& a)
{
    if (!a.kmin || a.drop_invalid) return false;
    const unsigned long long lo = *a.kmin, hi = *a.kmax;
    if (lo > hi) return true;  // no valid keys at all
    return ((lo ^ hi) >> a.shift) == 0ull;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift)
{
    return (uint32_t)(k >> shift) & (uint32_t)(kRadix - 1);
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_upsweep(const K* __restrict__ keys, PassArgs a, uint32_t* hist)
{
    __shared__ uint32_t h[kRadix];
    if (pass_uniform(a)) return;
    const long long n = pass_count(a);
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    // warp-aggregated counting: one shared atomic per distinct digit per warp
    // (depth keys of nearby primitives share their high digits)
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long idx = base + (long long)it * kSortThreads + threadIdx.x;
        uint32_t d = (uint32_t)kRadix;
        if (idx < n) {
            const K k = keys[idx];
            if (!(a.drop_invalid && (unsigned long long)k == kInvalidKey)) d = digit_of(k, a.shift);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < (uint32_t)kRadix && (__ffs(peers) - 1) == lane) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) hist[(size_t)i * a.nb + blockIdx.x] = h[i];
}

// Exclusive scan of every digit's row of per-block counts (row d holds
// hist[d * nb + b] for blocks b), in place, one CTA per digit; the row total
// goes to tot[d]. The downsweep adds the prefix of the digit totals.
__global__ void __launch_bounds__(kSortThreads) k_rowscan(uint32_t* hist, uint32_t* tot, PassArgs a)
{
    if (pass_uniform(a)) return;
    __shared__ uint32_t warp_tot[kWarps];
    uint32_t* row = hist + (size_t)blockIdx.x * a.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < a.nb; base += kSortThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < a.nb ? row[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = warp_tot[w];
            before += w < warp ? t : 0u;
            total += t;
        }
        if (i < a.nb) row[i] = carry + before + x - v;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_downsweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                            K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            PassArgs a, const uint32_t* __restrict__ hist,
                                                            const uint32_t* __restrict__ tot)
{
    __shared__ uint32_t base_off[kRadix];
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    const long long n = pass_count(a);
    const long long base = (long long)blockIdx.x * kSortTile;
    if (pass_uniform(a)) {
        // every key has the same digit: the stable permutation is the identity
        for (int it = 0; it < kSortItems; ++it) {
            const long long idx = base + (long long)it * kSortThreads + threadIdx.x;
            if (idx < n) {
                kout[idx] = kin[idx];
                vout[idx] = vin[idx];
            }
        }
        return;
    }
    if (base >= n) return;
    // digit bases: exclusive scan of the digit totals (kRadix == kSortThreads)
    {
        const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
        const uint32_t v = tot[d];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) wcnt[0][warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wcnt[0][w];
        base_off[d] = before + x - v + hist[(size_t)d * a.nb + blockIdx.x];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) {
        run[i] = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][i] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int it = 0; it < kSortItems; ++it) {
        const long long idx = base + (long long)it * kSortThreads + threadIdx.x;
        bool valid = idx < n;
        K k = 0;
        uint32_t v = 0;
        if (valid) {
            k = kin[idx];
            v = vin[idx];
            if (a.drop_invalid && (unsigned long long)k == kInvalidKey) valid = false;
        }
        const uint32_t d = valid ? digit_of(k, a.shift) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
            const uint32_t pos = base_off[d] + run[d] + pre + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kRadix; i += kSortThreads) {
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                tot += wcnt[w][i];
                wcnt[w][i] = 0;
            }
            run[i] += tot;
        }
        __syncthreads();
    }
}

static_assert(kRadix == kSortThreads, "digit-base scan assumes one digit per thread");

template <typename K>
void radix_pass(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, const PassArgs& a, uint32_t* hist,
                uint32_t* tot, cudaStream_t s)
{
    k_upsweep<K><<<a.nb, kSortThreads, 0, s>>>(kin, a, hist);
    note_launches(1);
    k_rowscan<<<kRadix, kSortThreads, 0, s>>>(hist, tot, a);
    note_launches(1);
    k_downsweep<K><<<a.nb, kSortThreads, 0, s>>>(kin, vin, kout, vout, a, hist, tot);
    note_launches(1);
}

}  // namespace

void sort_depth_keys(const BuildWs& ws, long long n, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    unsigned long long* kb[2] = {ws.keyA, ws.keyB};
    uint32_t* vb[2] = {ws.valA, ws.valB};
    int cur = 0;
    for (int pass = 0; pass < 64 / kRadixBits; ++pass) {
        PassArgs a;
        a.n_static = n;
        a.n_dev = pass == 0 ? nullptr : &ws.hdr->M;
        a.kmin = &ws.hdr->kmin;
        a.kmax = &ws.hdr->kmax;
        a.shift = pass * kRadixBits;
        a.drop_invalid = pass == 0;
        a.nb = nb;
        radix_pass<unsigned long long>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist, ws.dtot, s);
        cur ^= 1;
    }
    // 64 / 8 = 8 passes: the result is back in (keyA, valA)
}

void sort_tile_keys(const BuildWs& ws, long long cap, int tile_bits, cudaStream_t s, uint32_t** keys_out,
                    uint32_t** vals_out)
{
    uint32_t* kb[2] = {ws.dkeyA, ws.dkeyB};
    uint32_t* vb[2] = {ws.dvalA, ws.dvalB};
    int cur = 0;
    if (cap > 0) {
        const int nb = (int)((cap + kSortTile - 1) / kSortTile);
        const int passes = (tile_bits + kRadixBits - 1) / kRadixBits;
        for (int pass = 0; pass < passes; ++pass) {
            PassArgs a;
            a.n_static = cap;
            a.n_dev = &ws.hdr->tile_n;
            a.kmin = nullptr;
            a.kmax = nullptr;
            a.shift = pass * kRadixBits;
            a.drop_invalid = 0;
            a.nb = nb;
            radix_pass<uint32_t>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist, ws.dtot, s);
            cur ^= 1;
        }
    }
    *keys_out = kb[cur];
    *vals_out = vb[cur];
}

}  // namespace lf
