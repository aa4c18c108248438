// lf_sort.cu -- stable LSD radix sort (8-bit digits) of (key, value) pairs,
// and the depth order built on it.
//
// Used twice per build:
//  - the depth sort of Algorithm 1 (its sort-and-chunk step): the order of
//    the culled-in primitives by (FP64 depth, index). The IEEE bits of a
//    positive FP64 depth order like the depth; relative to the smallest valid
//    key they span up to ~55 bits. The sort takes their top 24 varying bits
//    (an order-preserving truncation) as a 32-bit key, drops culled
//    primitives in the first pass and sorts stably in three passes (the
//    first pass takes each key's index as its value, so equal keys stay in
//    index order). Keys that share the truncated value form runs that are
//    then put in (full key, index) order: runs of up to 32 by one thread
//    (insertion), longer runs by one CTA each (Batcher's odd-even merge
//    network, in shared memory up to 2048 keys, in global memory beyond).
//    The run pass keeps the order exact for any input; 24 bits trade a
//    fourth pass for short runs (1M Gaussians over depths 1.5..10: runs of at
//    most 5 keys, 12k pairs to reorder; grid-aligned voxels: runs of equal
//    full keys, already in order).
//  - the 3D tiling (Sec. 4.4): 32-bit keys = tile id of every (tile, rank)
//    pair emitted in rank order; the stable sort groups the pairs by tile and
//    keeps each tile's pairs in depth order.
//
// Each pass is reduce-then-scan over blocks of 2048 keys:
//   k_upsweep   per-block digit histogram (warp-aggregated shared atomics);
//   k_rowscan   one CTA per digit scans that digit's per-block counts;
//   k_downsweep ranks the block's keys stably (ballot-based digit matching,
//               per-warp counters, warps own contiguous key ranges), exchanges
//               them through shared memory into digit order and writes every
//               digit run contiguously.
// Item counts may live on the device (culled-in count, pair count), so grids
// are sized for the capacity and blocks past the count exit early.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBits = 8;
constexpr int kDigits = 1 << kBits;             // 256 = one digit per thread
constexpr int kKPT = kRadixBlockKeys / kThreads; // 8 keys per thread
constexpr int kDepthKeyBits = 24;                // truncated depth key width
constexpr int kDepthPasses = (kDepthKeyBits + kBits - 1) / kBits;
static_assert(kDigits == kThreads, "one digit per thread in the digit scans");

struct PassArgs {
    long long n_static;                    // upper bound / fixed count
    const unsigned long long* n_dev;       // device count (or null)
    const unsigned long long* kmin;        // valid depth-key range (depth sort) or null
    const unsigned long long* kmax;
    int shift;
    int first;                             // depth sort: drop the invalid key (all ones); value = index
    int nb;                                // number of blocks (histogram stride)
};

__device__ __forceinline__ long long pass_count(const PassArgs& a)
{
    return a.n_dev ? (long long)*a.n_dev : a.n_static;
}

// Right shift that keeps the top kDepthKeyBits varying bits of a depth key
// relative to the smallest valid key (0 if the range already fits).
__device__ __forceinline__ int depth_shift(unsigned long long lo, unsigned long long hi)
{
    if (lo > hi) return 0;
    const int bits = 64 - __clzll((long long)(hi - lo));
    return bits > kDepthKeyBits ? bits - kDepthKeyBits : 0;
}

// every valid truncated depth key has the same digit at this shift: identity pass
__device__ __forceinline__ bool pass_uniform(const PassArgs& a)
{
    if (a.first || !a.kmin) return false;
    const unsigned long long lo = *a.kmin, hi = *a.kmax;
    if (lo > hi) return true;   // no valid keys
    return (((hi - lo) >> depth_shift(lo, hi)) >> a.shift) == 0ull;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift)
{
    return (uint32_t)(k >> shift) & (uint32_t)(kDigits - 1);
}

// the key as sorted; false if absent (past the count, or culled)
template <typename K>
__device__ __forceinline__ bool load_key(const K* keys, long long idx, long long n, const PassArgs& a, K& k)
{
    if (idx >= n) return false;
    k = keys[idx];
    return !(a.first && k == (K)~(K)0);
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
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t h[kDigits];
    if (pass_uniform(a)) return;
    const long long n = pass_count(a);
    if ((long long)blockIdx.x * kRadixBlockKeys >= n) {   // past the device count: empty histogram
        hist[(size_t)threadIdx.x * a.nb + blockIdx.x] = 0u;
        return;
    }
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kRadixBlockKeys + warp * (32 * kKPT);
    K kk[kKPT];
    uint32_t okm = 0;
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        K k = 0;
        okm |= load_key(keys, base + r * 32 + lane, n, a, k) ? (1u << r) : 0u;
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
    pdl_wait();
    pdl_trigger();
    if (pass_uniform(a)) return;
    __shared__ uint32_t warp_tot[kWarps];
    uint32_t* row = hist + (size_t)blockIdx.x * a.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // blocks past the device count hold no keys (their downsweep exits)
    const long long n = pass_count(a);
    const int nb = (int)min((long long)a.nb, (n + kRadixBlockKeys - 1) / kRadixBlockKeys);
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += kThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? row[i] : 0u;
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
        if (i < nb) row[i] = carry + before + x - v;
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
    pdl_wait();
    pdl_trigger();
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
        const bool ok = load_key(kin, idx, n, a, k);
        key[r] = k;
        val[r] = ok ? (a.first ? (uint32_t)idx : vin[idx]) : 0u;
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

// ---- depth order ---------------------------------------------------------

// truncated 32-bit depth key of every primitive (all ones if culled)
__global__ void __launch_bounds__(256) k_depth_key32(const unsigned long long* __restrict__ key64,
                                                     uint32_t* __restrict__ k32, long long n,
                                                     const WsHeader* __restrict__ hdr)
{
    pdl_wait();
    pdl_trigger();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long lo = hdr->kmin, hi = hdr->kmax;
    const unsigned long long k = key64[i];
    k32[i] = k == kInvalidKey ? 0xffffffffu : (uint32_t)((k - lo) >> depth_shift(lo, hi));
}

// (full key, index) order of two ranks' primitives
__device__ __forceinline__ bool depth_less(unsigned long long ka, uint32_t va, unsigned long long kb, uint32_t vb)
{
    return ka < kb || (ka == kb && va < vb);
}

constexpr int kShortRun = 32;
constexpr int kLongRunCtas = 304;
constexpr int kLongRunThreads = 1024;
constexpr int kSmemRun = 2048;

// Within a run of equal truncated keys the ranks are in index order (the
// sort is stable), so the run is already in (full key, index) order unless
// some neighbour pair has a larger full key first. One flag per rank marks
// such pairs (bytes over keyB, free at this point).
__global__ void __launch_bounds__(256) k_depth_bad(BuildWs w)
{
    pdl_wait();
    pdl_trigger();
    const long long M = (long long)w.hdr->M;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    uint8_t b = 0;
    if (r > 0 && w.tkeyA[r] == w.tkeyA[r - 1]) b = w.keyA[w.valA[r - 1]] > w.keyA[w.valA[r]] ? 1 : 0;
    reinterpret_cast<uint8_t*>(w.keyB)[r] = b;
}

// Runs of equal truncated keys that hold an out-of-order pair. Work starts
// at flagged ranks only: a flagged rank walks back to its run's start and
// leaves if it meets an earlier flag (that one owns the run), so every run
// is owned once and walked once. The owner finds the run's end, sorts a run
// of up to kShortRun keys itself and lists longer ones (start, length) in
// tkeyB. Runs with no flag (equal keys, e.g. primitives on one grid layer)
// cost nothing.
__global__ void __launch_bounds__(256) k_depth_runs(BuildWs w)
{
    pdl_wait();
    pdl_trigger();
    const long long M = (long long)w.hdr->M;
    const long long r0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint8_t* bad = reinterpret_cast<const uint8_t*>(w.keyB);
    if (r0 >= M || !bad[r0]) return;
    const uint32_t* k = w.tkeyA;
    const uint32_t kr = k[r0];
    long long r = r0 - 1;                         // candidate run start
    while (r > 0 && k[r - 1] == kr) {
        if (bad[r]) return;                       // an earlier flag owns this run
        --r;
    }
    long long e = r0 + 1;
    while (e < M && k[e] == kr) ++e;
    const int L = (int)min(e - r, (long long)0x7fffffff);
    if (L > kShortRun) {
        const unsigned long long q = atomicAdd(&w.hdr->long_runs, 1ull);
        w.tkeyB[2 * q] = (uint32_t)r;
        w.tkeyB[2 * q + 1] = (uint32_t)L;
        return;
    }
    unsigned long long kk[kShortRun];
    uint32_t vv[kShortRun];
    for (int i = 0; i < L; ++i) {
        const uint32_t v = w.valA[r + i];
        const unsigned long long key = w.keyA[v];
        int j = i;
        while (j > 0 && depth_less(key, v, kk[j - 1], vv[j - 1])) {
            kk[j] = kk[j - 1];
            vv[j] = vv[j - 1];
            --j;
        }
        kk[j] = key;
        vv[j] = v;
    }
    for (int i = 0; i < L; ++i) w.valA[r + i] = vv[i];
}

// Batcher's odd-even merge network over P = 2^m slots: every comparator puts
// the smaller element at the lower slot, so slots past the run length L act
// as +infinity and are never touched. Stage (p, k) compares slot a with
// a + k when a >= k mod p, (a - k mod p) mod 2k < k and a, a + k lie in the
// same block of 2p slots.
__device__ __forceinline__ bool oem_pair(long long a, long long p, long long k)
{
    const long long j0 = k % p;
    return a >= j0 && ((a - j0) % (2 * k)) < k && (a / (2 * p)) == ((a + k) / (2 * p));
}

// Runs longer than kShortRun: one CTA per run (grid-stride over the list).
__global__ void __launch_bounds__(kLongRunThreads) k_depth_long_runs(BuildWs w)
{
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long sk[kSmemRun];
    __shared__ uint32_t sv[kSmemRun];
    const unsigned long long nr = w.hdr->long_runs;
    for (unsigned long long q = blockIdx.x; q < nr; q += gridDim.x) {
        const long long r = w.tkeyB[2 * q];
        const long long L = w.tkeyB[2 * q + 1];
        long long P = 1;
        while (P < L) P <<= 1;
        if (P <= kSmemRun) {
            for (long long i = threadIdx.x; i < L; i += blockDim.x) {
                const uint32_t v = w.valA[r + i];
                sv[i] = v;
                sk[i] = w.keyA[v];
            }
            __syncthreads();
            for (long long p = 1; p < P; p <<= 1)
                for (long long k = p; k >= 1; k >>= 1) {
                    for (long long a = threadIdx.x; a + k < L; a += blockDim.x) {
                        if (!oem_pair(a, p, k)) continue;
                        const long long b = a + k;
                        if (depth_less(sk[b], sv[b], sk[a], sv[a])) {
                            const unsigned long long tk = sk[a];
                            const uint32_t tv = sv[a];
                            sk[a] = sk[b], sv[a] = sv[b];
                            sk[b] = tk, sv[b] = tv;
                        }
                    }
                    __syncthreads();
                }
            for (long long i = threadIdx.x; i < L; i += blockDim.x) w.valA[r + i] = sv[i];
            __syncthreads();
        } else {
            unsigned long long* gk = w.keyB + r;
            uint32_t* gv = w.valA + r;
            for (long long i = threadIdx.x; i < L; i += blockDim.x) gk[i] = w.keyA[gv[i]];
            __syncthreads();
            for (long long p = 1; p < P; p <<= 1)
                for (long long k = p; k >= 1; k >>= 1) {
                    for (long long a = threadIdx.x; a + k < L; a += blockDim.x) {
                        if (!oem_pair(a, p, k)) continue;
                        const long long b = a + k;
                        if (depth_less(gk[b], gv[b], gk[a], gv[a])) {
                            const unsigned long long tk = gk[a];
                            const uint32_t tv = gv[a];
                            gk[a] = gk[b], gv[a] = gv[b];
                            gk[b] = tk, gv[b] = tv;
                        }
                    }
                    __syncthreads();
                }
        }
    }
}

template <typename K>
void radix_pass(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, const PassArgs& a, uint32_t* hist,
                uint32_t* tot, cudaStream_t s)
{
    cudaFuncSetAttribute(k_downsweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem<K>));
    launch_pdl(k_upsweep<K>, dim3(a.nb), dim3(kThreads), 0, s, kin, a, hist);
    launch_pdl(k_rowscan, dim3(kDigits), dim3(kThreads), 0, s, hist, tot, a);
    launch_pdl(k_downsweep<K>, dim3(a.nb), dim3(kThreads), sizeof(DownSmem<K>), s, kin, vin, kout, vout, a, hist, tot);
    note_launches(3);
}

}  // namespace

void sort_depth_keys(const BuildWs& ws, long long n, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = (int)((n + kRadixBlockKeys - 1) / kRadixBlockKeys);
    uint32_t* kb[2] = {ws.tkeyA, ws.tkeyB};
    uint32_t* vb[2] = {ws.valA, ws.valB};
    // start in the buffer that makes the last pass end in tkeyA / valA
    int cur = kDepthPasses & 1;
    launch_pdl(k_depth_key32, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, ws.keyA, kb[cur], n, ws.hdr);
    for (int pass = 0; pass < kDepthPasses; ++pass) {
        PassArgs a;
        a.n_static = n;
        a.n_dev = pass == 0 ? nullptr : &ws.hdr->M;
        a.kmin = &ws.hdr->kmin;
        a.kmax = &ws.hdr->kmax;
        a.shift = pass * kBits;
        a.first = pass == 0;
        a.nb = nb;
        radix_pass<uint32_t>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist, ws.dtot, s);
        cur ^= 1;
    }
    // truncated keys in tkeyA, ranks in valA; now the runs
    launch_pdl(k_depth_bad, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, ws);
    launch_pdl(k_depth_runs, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, ws);
    launch_pdl(k_depth_long_runs, dim3(kLongRunCtas), dim3(kLongRunThreads), 0, s, ws);
    note_launches(4);
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
