// lf_sort.cu -- stable LSD radix sort of the culled-in primitives by
// (FP64 reference depth, index): Algorithm 1 line 3, "Sort_and_Chunk".
//
// Keys are the IEEE bits of the positive FP64 reference depth, which order
// like the depths. The first pass drops culled primitives (key kInvalidKey)
// and rewrites every key relative to the smallest valid key, so only the
// bits that vary across the scene are sorted; a later pass whose digit is
// the same for every key (known from the key range) is a plain copy. Values
// start in index order and every pass is stable, so equal depths stay in
// index order.
//
// Each pass is reduce-then-scan over blocks of 2048 keys with 11-bit digits:
//   k_upsweep   per-block digit histogram (warp-aggregated shared atomics);
//   k_rowscan   one CTA per digit scans that digit's per-block counts;
//   k_downsweep ranks the block's keys stably (warp match + per-warp
//               counters; warps own contiguous key ranges), exchanges them
//               through shared memory into digit order and writes every digit
//               run contiguously.
// Item counts may live on the device (the culled-in count), so grids are
// sized for the capacity and blocks past the count write zero histograms.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kKPT = kSortBlockKeys / kThreads;  // 8 keys per thread
constexpr int kDigits = kSortDigits;             // 2048
constexpr int kBits = 11;
static_assert((1 << kBits) == kDigits, "digit width");
static_assert(kKPT * 32 <= 65535, "per-warp counters are 16-bit");

struct PassArgs {
    long long n_static;                    // upper bound / fixed count
    const unsigned long long* n_dev;       // device count (or null)
    const unsigned long long* kmin;        // absolute range of the valid keys
    const unsigned long long* kmax;
    int shift;
    int first;                             // drop invalid keys, make keys relative
    int nb;                                // number of blocks (histogram stride)
};

__device__ __forceinline__ long long pass_count(const PassArgs& a)
{
    return a.n_dev ? (long long)*a.n_dev : a.n_static;
}

// every relative key has the same digit at this shift: identity pass
__device__ __forceinline__ bool pass_uniform(const PassArgs& a)
{
    if (a.first) return false;
    const unsigned long long lo = *a.kmin, hi = *a.kmax;
    if (lo > hi) return true;   // no valid keys
    return ((hi - lo) >> a.shift) == 0ull;
}

__device__ __forceinline__ uint32_t digit_of(unsigned long long k, int shift)
{
    return (uint32_t)(k >> shift) & (uint32_t)(kDigits - 1);
}

// the key as sorted (relative to the smallest valid key); false if absent
__device__ __forceinline__ bool load_key(const unsigned long long* keys, long long idx, long long n,
                                         const PassArgs& a, unsigned long long kmin, unsigned long long& k)
{
    if (idx >= n) return false;
    k = keys[idx];
    if (a.first) {
        if (k == kInvalidKey) return false;
        k -= kmin;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads) k_upsweep(const unsigned long long* __restrict__ keys, PassArgs a,
                                                      uint32_t* hist)
{
    __shared__ uint32_t h[kDigits];
    if (pass_uniform(a)) return;
    const long long n = pass_count(a);
    const unsigned long long kmin = *a.kmin;
    for (int i = threadIdx.x; i < kDigits; i += kThreads) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kSortBlockKeys + warp * (32 * kKPT);
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        unsigned long long k = 0;
        const bool ok = load_key(keys, base + r * 32 + lane, n, a, kmin, k);
        const uint32_t d = ok ? digit_of(k, a.shift) : (uint32_t)kDigits;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (ok && (__ffs(peers) - 1) == lane) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kDigits; i += kThreads) hist[(size_t)i * a.nb + blockIdx.x] = h[i];
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

// In-place exclusive scan of kDigits values (thread t owns kDigits/kThreads
// consecutive digits); returns the total. Ends with a CTA barrier.
__device__ __forceinline__ uint32_t scan_digits(uint32_t* vals, uint32_t* warp_tmp)
{
    constexpr int P = kDigits / kThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < P; ++i) s += vals[threadIdx.x * P + i];
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t t = warp_tmp[w];
        before += w < warp ? t : 0u;
        total += t;
    }
    uint32_t run = before + x - s;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const uint32_t v = vals[threadIdx.x * P + i];
        vals[threadIdx.x * P + i] = run;
        run += v;
    }
    __syncthreads();
    return total;
}

struct DownSmem {
    uint16_t wcnt[kWarps][kDigits];           // per-warp digit counts, then per-warp offsets
    uint32_t blk_start[kDigits];              // block-local start of every digit run
    uint32_t glob_base[kDigits];              // global destination of every digit run
    unsigned long long xkey[kSortBlockKeys];  // exchange buffer in block-local digit order
    uint32_t xval[kSortBlockKeys];
    uint32_t warp_tmp[kWarps];
};

__global__ void __launch_bounds__(kThreads) k_downsweep(const unsigned long long* __restrict__ kin,
                                                        const uint32_t* __restrict__ vin,
                                                        unsigned long long* __restrict__ kout,
                                                        uint32_t* __restrict__ vout, PassArgs a,
                                                        const uint32_t* __restrict__ hist,
                                                        const uint32_t* __restrict__ tot)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    DownSmem& S = *reinterpret_cast<DownSmem*>(dsm_raw);
    const long long n = pass_count(a);
    const long long blk = (long long)blockIdx.x * kSortBlockKeys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (pass_uniform(a)) {
        // every key has the same digit: the stable permutation is the identity
        for (int i = threadIdx.x; i < kSortBlockKeys; i += kThreads) {
            const long long idx = blk + i;
            if (idx < n) {
                kout[idx] = kin[idx];
                vout[idx] = vin[idx];
            }
        }
        return;
    }
    if (blk >= n) return;
    const unsigned long long kmin = *a.kmin;

    for (int i = threadIdx.x; i < kWarps * kDigits; i += kThreads) (&S.wcnt[0][0])[i] = 0;
    // global digit bases (exclusive scan of the digit totals) plus this
    // block's exclusive offset within each digit row
    for (int d = threadIdx.x; d < kDigits; d += kThreads) S.glob_base[d] = tot[d];
    scan_digits(S.glob_base, S.warp_tmp);
    for (int d = threadIdx.x; d < kDigits; d += kThreads) S.glob_base[d] += hist[(size_t)d * a.nb + blockIdx.x];

    // rank: warp w owns keys [256 w, 256 w + 256) of the block, visited in
    // order round by round, so equal digits keep their order
    unsigned long long key[kKPT];
    uint32_t val[kKPT], dig[kKPT], pos[kKPT];
    const long long wbase = blk + warp * (32 * kKPT);
#pragma unroll
    for (int r = 0; r < kKPT; ++r) {
        const long long idx = wbase + r * 32 + lane;
        unsigned long long k = 0;
        const bool ok = load_key(kin, idx, n, a, kmin, k);
        key[r] = k;
        val[r] = ok ? vin[idx] : 0u;
        dig[r] = ok ? digit_of(k, a.shift) : (uint32_t)kDigits;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        const uint32_t before = ok ? (uint32_t)S.wcnt[warp][dig[r]] : 0u;
        __syncwarp();
        pos[r] = before + __popc(peers & ((1u << lane) - 1u));
        if (ok && (__ffs(peers) - 1) == lane) S.wcnt[warp][dig[r]] = (uint16_t)(before + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets over warps and the block-local digit total
    for (int d = threadIdx.x; d < kDigits; d += kThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = S.wcnt[w][d];
            S.wcnt[w][d] = (uint16_t)run;
            run += c;
        }
        S.blk_start[d] = run;
    }
    const uint32_t placed = scan_digits(S.blk_start, S.warp_tmp);
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
        const unsigned long long k = S.xkey[l];
        const uint32_t d = digit_of(k, a.shift);
        const uint32_t dst = S.glob_base[d] + (l - S.blk_start[d]);
        kout[dst] = k;
        vout[dst] = S.xval[l];
    }
}

}  // namespace

void sort_depth_keys(const BuildWs& ws, long long n, cudaStream_t s)
{
    if (n <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem));
        attr_set = true;
    }
    const int nb = (int)((n + kSortBlockKeys - 1) / kSortBlockKeys);
    unsigned long long* kb[2] = {ws.keyA, ws.keyB};
    uint32_t* vb[2] = {ws.valA, ws.valB};
    int cur = 0;
    constexpr int kPasses = (64 + kBits - 1) / kBits;   // 6: the result returns to (keyA, valA)
    static_assert(kPasses % 2 == 0, "even pass count keeps the result in the A buffers");
    for (int pass = 0; pass < kPasses; ++pass) {
        PassArgs a;
        a.n_static = n;
        a.n_dev = pass == 0 ? nullptr : &ws.hdr->M;
        a.kmin = &ws.hdr->kmin;
        a.kmax = &ws.hdr->kmax;
        a.shift = pass * kBits;
        a.first = pass == 0;
        a.nb = nb;
        k_upsweep<<<nb, kThreads, 0, s>>>(kb[cur], a, ws.hist);
        note_launches(1);
        k_rowscan<<<kDigits, kThreads, 0, s>>>(ws.hist, ws.dtot, a);
        note_launches(1);
        k_downsweep<<<nb, kThreads, sizeof(DownSmem), s>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], a, ws.hist,
                                                           ws.dtot);
        note_launches(1);
        cur ^= 1;
    }
}

}  // namespace lf
