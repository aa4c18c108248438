// lf_sort.cu -- stable LSD radix sort (8-bit digits) of (key, value) pairs.
//
// Used twice per build:
//  - the depth sort of Algorithm 1 line 3 ("Sort_and_Chunk"): 64-bit keys =
//    IEEE bits of the positive FP64 reference depth (they order like the
//    depths), values = primitive index. The first pass drops culled
//    primitives (key kInvalidKey) and makes every key relative to the
//    smallest valid key, so passes above the varying bits are plain copies.
//    Values start in index order and every pass is stable, so equal depths
//    stay in index order.
//  - the 3D tiling (Sec. 4.4): 32-bit keys = tile id of every (tile, rank)
//    pair emitted in rank order; the stable sort groups the pairs by tile and
//    keeps each tile's pairs in depth order.
//
// Each pass is reduce-then-scan over blocks of 4096 keys:
//   k_upsweep   per-block digit histogram (warp-aggregated shared atomics);
//   k_rowscan   one CTA per digit scans that digit's per-block counts;
//   k_downsweep ranks the block's keys stably (ballot-based digit matching,
//               per-warp counters, warps own contiguous key ranges), exchanges
//               them through shared memory into digit order and writes every
//               digit run contiguously.
// Item counts may live on the device (culled-in count, pair count), so grids
// are sized for the capacity and blocks past the count write zero histograms.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBits = 8;
constexpr int kDigits = 1 << kBits;             // 256 = one digit per thread
constexpr int kKPT = kRadixBlockKeys / kThreads; // 16 keys per thread
static_assert(kDigits == kThreads, "one digit per thread in the digit scans");

struct PassArgs {
    long long n_static;                    // upper bound / fixed count
    const unsigned long long* n_dev;       // device count (or null)
    const unsigned long long* kmin;        // valid key range (depth keys) or null
    const unsigned long long* kmax;
    int shift;
    int first;                             // depth keys: drop invalid, make relative
    int nb;                                // number of blocks (histogram stride)
};

__device__ __forceinline__ long long pass_count(const PassArgs& a)
{
    return a.n_dev ? (long long)*a.n_dev : a.n_static;
}

// every (relative) key has the same digit at this shift: identity pass
__device__ __forceinline__ bool pass_uniform(const PassArgs& a)
{
    if (a.first || !a.kmin) return false;
    const unsigned long long lo = *a.kmin, hi = *a.kmax;
    if (lo > hi) return true;   // no valid keys
    return ((hi - lo) >> a.shift) == 0ull;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift)
{
    return (uint32_t)(k >> shift) & (uint32_t)(kDigits - 1);
}

// the key as sorted; false if absent (past the count, or culled)
template <typename K>
__device__ __forceinline__ bool load_key(const K* keys, long long idx, long long n, const PassArgs& a,
                                         unsigned long long kmin, K& k)
{
    if (idx >= n) return false;
    k = keys[idx];
    if (a.first) {
        if ((unsigned long long)k == kInvalidKey) return false;
        k = (K)((unsigned long long)k - kmin);
    }
    return true;
}

// lanes holding the same digit (ballot per digit bit); valid lanes only
__device__ __forceinline__ uint32_t match_digit(uint32_t d, bool ok)
{
    uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < kBits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_upsweep(const K* __restrict__ keys, PassArgs a, uint32_t* hist)
{
    __shared__ uint32_t h[kDigits];
    if (pass_uniform(a)) return;
    const long long n = pass_count(a);
    const unsigned long long kmin = a.kmin ? *a.kmin : 0ull;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kRadixBlockKeys + warp * (32 * kKPT);
    K kk[kKPT];
    uint32_t okm = 0;
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        K k = 0;
        okm |= load_key(keys, base + r * 32 + lane, n, a, kmin, k) ? (1u << r) : 0u;
        kk[r] = k;
    }
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        const bool ok = (okm >> r) & 1u;
        const uint32_t d = ok ? digit_of(kk[r], a.shift) : 0u;
        const uint32_t peers = match_digit(d, ok);
        if (ok && (__ffs(peers) - 1) == lane) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * a.nb + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of digit row d (hist[d * nb + b] over blocks b), in place;
// the row total goes to tot[d].
__global__ void __launch_bounds__(kThreads) k_rowscan(uint32_t* hist, uint32_t* tot, PassArgs a)
{
    if (pass_uniform(a)) return;
    __shared__ uint32_t warp_tot[kWarps];
    uint32_t* row = hist + (size_t)blockIdx.x * a.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < a.nb; base += kThreads) {
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

// exclusive scan of one value per thread over the block; returns the total
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t* warp_tmp, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    __syncthreads();
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t t = warp_tmp[w];
        before += w < warp ? t : 0u;
        tot += t;
    }
    *total = tot;
    return before + x - v;
}

template <typename K>
struct DownSmem {
    uint32_t wcnt[kWarps][kDigits];       // per-warp digit counts, then per-warp offsets
    uint32_t blk_start[kDigits];          // block-local start of every digit run
    uint32_t glob_base[kDigits];          // global destination of every digit run
    K xkey[kRadixBlockKeys];              // exchange buffer in block-local digit order
    uint32_t xval[kRadixBlockKeys];
    uint32_t warp_tmp[kWarps];
};

template <typename K>
__global__ void __launch_bounds__(kThreads) k_downsweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                        K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                        PassArgs a, const uint32_t* __restrict__ hist,
                                                        const uint32_t* __restrict__ tot)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    DownSmem<K>& S = *reinterpret_cast<DownSmem<K>*>(dsm_raw);
    const long long n = pass_count(a);
    const long long blk = (long long)blockIdx.x * kRadixBlockKeys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (pass_uniform(a)) {
        // every key has the same digit: the stable permutation is the identity
        for (int i = threadIdx.x; i < kRadixBlockKeys; i += kThreads) {
            const long long idx = blk + i;
            if (idx < n) {
                kout[idx] = kin[idx];
                vout[idx] = vin[idx];
            }
        }
        return;
    }
    if (blk >= n) return;
    const unsigned long long kmin = a.kmin ? *a.kmin : 0ull;
    const int d0 = threadIdx.x;   // the digit this thread scans

#pragma unroll
    for (int w = 0; w < kWarps; ++w) S.wcnt[w][d0] = 0;
    {
        uint32_t total;
        S.glob_base[d0] = block_exscan(tot[d0], S.warp_tmp, &total) + hist[(size_t)d0 * a.nb + blockIdx.x];
    }
    __syncthreads();

    // rank: warp w owns keys [512 w, 512 w + 512) of the block, visited in
    // order round by round, so equal digits keep their order
    K key[kKPT];
    uint32_t val[kKPT], dig[kKPT], pos[kKPT];
    const long long wbase = blk + warp * (32 * kKPT);
    const uint32_t lt = (1u << lane) - 1u;
    // all loads first (the ranking rounds below synchronise the warp)
    uint32_t okm = 0;
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        const long long idx = wbase + r * 32 + lane;
        K k = 0;
        const bool ok = load_key(kin, idx, n, a, kmin, k);
        key[r] = k;
        val[r] = ok ? vin[idx] : 0u;
        okm |= ok ? (1u << r) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        const bool ok = (okm >> r) & 1u;
        const K k = key[r];
        const uint32_t d = ok ? digit_of(k, a.shift) : 0u;
        dig[r] = ok ? d : (uint32_t)kDigits;
        const uint32_t peers = match_digit(d, ok);
        const uint32_t before = ok ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        pos[r] = before + __popc(peers & lt);
        if (ok && (__ffs(peers) - 1) == lane) S.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets over warps and the block-local digit total
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = S.wcnt[w][d0];
        S.wcnt[w][d0] = run;
        run += c;
    }
    uint32_t placed;
    S.blk_start[d0] = block_exscan(run, S.warp_tmp, &placed);
    __syncthreads();
    // exchange into block-local digit order
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        if (dig[r] >= (uint32_t)kDigits) continue;
        const uint32_t l = S.blk_start[dig[r]] + S.wcnt[warp][dig[r]] + pos[r];
        S.xkey[l] = key[r];
        S.xval[l] = val[r];
    }
    __syncthreads();
    // coalesced write-out: item l of digit d goes to glob_base[d] + (l - blk_start[d])
    for (uint32_t l = threadIdx.x; l < placed; l += kThreads) {
        const K k = S.xkey[l];
        const uint32_t d = digit_of(k, a.shift);
        const uint32_t dst = S.glob_base[d] + (l - S.blk_start[d]);
        kout[dst] = k;
        vout[dst] = S.xval[l];
    }
}

template <typename K>
void radix_pass(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, const PassArgs& a, uint32_t* hist,
                uint32_t* tot, cudaStream_t s)
{
    cudaFuncSetAttribute(k_downsweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem<K>));
    k_upsweep<K><<<a.nb, kThreads, 0, s>>>(kin, a, hist);
    k_rowscan<<<kDigits, kThreads, 0, s>>>(hist, tot, a);
    k_downsweep<K><<<a.nb, kThreads, sizeof(DownSmem<K>), s>>>(kin, vin, kout, vout, a, hist, tot);
    note_launches(3);
}

}  // namespace

void sort_depth_keys(const BuildWs& ws, long long n, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = (int)((n + kRadixBlockKeys - 1) / kRadixBlockKeys);
    unsigned long long* kb[2] = {ws.keyA, ws.keyB};
    uint32_t* vb[2] = {ws.valA, ws.valB};
    int cur = 0;
    for (int pass = 0; pass < 64 / kBits; ++pass) {
        PassArgs a;
        a.n_static = n;
        a.n_dev = pass == 0 ? nullptr : &ws.hdr->M;
        a.kmin = &ws.hdr->kmin;
        a.kmax = &ws.hdr->kmax;
        a.shift = pass * kBits;
        a.first = pass == 0;
        a.nb = nb;
        radix_pass<unsigned long long>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist, ws.dtot, s);
        cur ^= 1;
    }
    // 8 passes: the result is back in (keyA, valA)
}

int tile_sort_passes(int tile_bits) { return (tile_bits + kBits - 1) / kBits; }

void sort_tile_keys(const BuildWs& ws, long long cap, int tile_bits, cudaStream_t s, uint32_t** keys_out,
                    uint32_t** vals_out)
{
    uint32_t* kb[2] = {ws.tkeyA, ws.tkeyB};
    uint32_t* vb[2] = {ws.entA, ws.entB};
    int cur = 0;
    if (cap > 0) {
        const int nb = (int)((cap + kRadixBlockKeys - 1) / kRadixBlockKeys);
        for (int pass = 0; pass < tile_sort_passes(tile_bits); ++pass) {
            PassArgs a;
            a.n_static = cap;
            a.n_dev = &ws.hdr->tile_n;
            a.kmin = nullptr;
            a.kmax = nullptr;
            a.shift = pass * kBits;
            a.first = 0;
            a.nb = nb;
            radix_pass<uint32_t>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist, ws.dtot, s);
            cur ^= 1;
        }
    }
    *keys_out = kb[cur];
    *vals_out = vb[cur];
}

}  // namespace lf
