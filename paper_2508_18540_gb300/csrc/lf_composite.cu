// lf_composite.cu -- swizzle blending of the sweeping planes into the quilt
// views (Sec. 4.3; the compositing steps of Algorithm 1).
//
// k_comp_coeffs evaluates, per (view column j, plane k) and (view row i,
// plane k), the affine form of Eq. (u_prime) in plane pixels,
//   X(x) = P_s x + (gm x + hb),  X(x) + 1/2 = P_s x + (gm x + hn),
// from the FP64 display set-up (Delta x_j = 2 D_focal s_j tan(phi_x/2),
// den = (d_k - D_forward) tan(theta'/2), a = d_k tan(theta/2),
// g = W a / (Nx den), h = (W/2)((Delta (D_focal - d_k)/D_focal + a (1-Nx)/Nx)/den + 1) - 1/2,
// gm = g - P_s), rounded once to FP32.
// The composite kernels walk the planes front to back for every view pixel:
// nearest texel index P_s x + floor(fma(gm, x, hn)) (FP32 decision), or
// bilinear taps around X with zero padding; Q += T c_k, T *= 1 - A_k
// (Eq. (alpha_blend)); empty planes skipped; output (Q + T bg, 1 - T).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lf_internal.cuh"

namespace lf {

namespace {

// |fma(gm, x, h)| below this bound for every x of a row lets the staged
// kernel skip its clamps (and keeps the exact floor below valid).
constexpr float kNarrow = 1048576.0f;    // 2^20
constexpr float kClamp = 2097152.0f;     // 2^21

__device__ __forceinline__ double view_offset(int j, int V, double Df, double tphi)
{
    const double s = V <= 1 ? 0.0 : __dsub_rn(__ddiv_rn((double)j, (double)(V - 1)), 0.5);
    return __dmul_rn(__dmul_rn(__dmul_rn(2.0, Df), s), tphi);
}

__device__ __forceinline__ void axis_coeffs(double delta, double dk, double Df, double Dfwd, double tth, double tthp,
                                            int n, int Wp, int P_s, float* out)
{
    const double den = __dmul_rn(__dsub_rn(dk, Dfwd), tthp);
    const double a = __dmul_rn(dk, tth);
    const double g = __ddiv_rn(__dmul_rn((double)Wp, a), __dmul_rn((double)n, den));
    const double A = __ddiv_rn(__dmul_rn(delta, __dsub_rn(Df, dk)), Df);
    const double c0 = __ddiv_rn(__dmul_rn(a, (double)(1 - n)), (double)n);
    const double hw = __dmul_rn(0.5, (double)Wp);
    const double hn = __dmul_rn(hw, __dadd_rn(__ddiv_rn(__dadd_rn(A, c0), den), 1.0));
    out[0] = __double2float_rn(__dsub_rn(g, (double)P_s));
    out[1] = __double2float_rn(hn);
    out[2] = __double2float_rn(__dsub_rn(hn, 0.5));
}

__global__ void k_comp_coeffs(CompParams p, const double* __restrict__ d, const int32_t* __restrict__ count, CompWs w)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = p.Vx * p.N, ny = p.Vy * p.N;
    if (e >= nx + ny) return;
    const bool along_x = e < nx;
    const int idx = along_x ? e : e - nx;
    const int v = idx / p.N, k = idx % p.N;
    float* out = (along_x ? w.cx : w.cy) + 3 * (size_t)idx;
    if (count[k] == 0) {
        out[0] = out[1] = out[2] = 0.0f;
        return;
    }
    int n;
    if (along_x) {
        axis_coeffs(view_offset(v, p.Vx, p.D_focal, p.tphi_x), d[k], p.D_focal, p.D_forward, p.tth_x, p.tthp_x, p.Nx,
                    p.W, p.P_s, out);
        n = p.Nx;
    } else {
        axis_coeffs(view_offset(v, p.Vy, p.D_focal, p.tphi_y), d[k], p.D_focal, p.D_forward, p.tth_y, p.tthp_y, p.Ny,
                    p.H, p.P_s, out);
        n = p.Ny;
    }
    // the row's range of gm x + h (affine in x): flag planes that may leave it
    const double lo = fmin((double)out[2], (double)out[1]);
    const double hi = fmax((double)out[2], (double)out[1]);
    const double span = fabs((double)out[0]) * (double)(n - 1);
    if (!(fmax(fabs(lo), fabs(hi)) + span + 2.0 < (double)kNarrow)) atomicOr(&w.wide[k], 1);
}

// Four BF16 channels -> FP32, exactly: the mixed-precision add of each BF16
// operand and -0.0 (x + -0 = x, signed zeros included). It widens on the
// floating-point pipe; the shift-and-mask widening takes integer-pipe slots
// that the composite's index arithmetic needs (BF16 composite 0.425 ->
// 0.411 ms on the display frame, views bit for bit the same).
__device__ __forceinline__ float4 bf16x4_to_f32(uint2 u)
{
    float4 r;
    asm("{\n\t.reg .b16 a, b, c, d;\n\tmov.b32 {a, b}, %4;\n\tmov.b32 {c, d}, %5;\n\t"
        "add.rn.f32.bf16 %0, a, 0f80000000;\n\tadd.rn.f32.bf16 %1, b, 0f80000000;\n\t"
        "add.rn.f32.bf16 %2, c, 0f80000000;\n\tadd.rn.f32.bf16 %3, d, 0f80000000;\n\t}"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(u.x), "r"(u.y));
    return r;
}

template <int DT>
__device__ __forceinline__ float4 load_texel(const void* planes, size_t idx)
{
    if (DT == LF_F32) {
        return __ldg(reinterpret_cast<const float4*>(planes) + idx);
    } else if (DT == LF_U8) {
        return u8_unpack(__ldg(reinterpret_cast<const uint32_t*>(planes) + idx));
    } else {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(planes) + idx);
        if (DT == LF_F16) {
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            return bf16x4_to_f32(u);
        }
    }
}

// index of view v's pixel (x, y) in the output: separate views, or the
// quilt atlas (tile row v / c, tile column v % c)
__device__ __forceinline__ size_t view_pixel(const CompParams& p, int v, int x, int y)
{
    if (p.atlas_cols <= 0) return ((size_t)v * p.Ny + y) * p.Nx + x;
    const int c = p.atlas_cols;
    return ((size_t)(v / c) * p.Ny + y) * ((size_t)c * p.Nx) + (size_t)(v % c) * p.Nx + x;
}

// plane index of the nearest texel, or -1 when the FP32 result is far outside
__device__ __forceinline__ int nearest_index(int P_s, int x, float gm, float hn)
{
    const float f = floorf(__fmaf_rn(gm, (float)x, hn));
    if (!(f >= -1.0e6f && f <= 1.0e6f)) return -1;
    return P_s * x + (int)f;
}

// Transmittance carried as m 2^-e (e a multiple of 64) so that no product of
// many (1 - A) underflows: when m falls below 2^-64 it is scaled up by 2^64.
constexpr float kUpB = 18446744073709551616.0f;       // 2^64
constexpr float kDownB = 5.42101086242752217e-20f;    // 2^-64
constexpr float kBigB = 4294967296.0f;                // 2^32
__device__ __forceinline__ float scaled_t(float m, int e) { return e == 0 ? m : (e == 64 ? m * kDownB : 0.0f); }

// plain forms: T below this is taken as 0 at every fourth non-empty plane
constexpr float kTFlush = 5.9604644775390625e-8f;   // 2^-24
// saving forms: a walk stops once T would fall below this (taken as 0), the
// plain forms' flush threshold
constexpr float kTStop = kTFlush;
constexpr int kCompBX = 32, kCompBY = 8;

// Unstaged fallback (planes read through L1/L2), used when the staged kernel's
// shared-memory layout does not fit or rows are not 16-byte aligned.
// SAVE: T carried as m 2^-e and the adjoint's starting state written, as in
// the staged kernel's saving form.
template <int DT, bool BILINEAR, bool SAVE = false>
__global__ void __launch_bounds__(kCompBX* kCompBY) k_composite(CompParams p, const void* __restrict__ planes,
                                                               const int32_t* __restrict__ count, CompWs w,
                                                               float* __restrict__ out, float4* __restrict__ state)
{
    extern __shared__ float s_coef[];  // [N][6]: x (gm, hn, hb), y (gm, hn, hb); count in [N] ints after
    int* s_cnt = reinterpret_cast<int*>(s_coef + 6 * p.N);
    const int v = blockIdx.x;   // fastest: the views of one pixel tile share plane rows in L2
    const int i = v / p.Vx, j = v % p.Vx;
    const int tid = threadIdx.y * kCompBX + threadIdx.x;
    for (int k = tid; k < p.N; k += kCompBX * kCompBY) {
        const float* cx = w.cx + 3 * ((size_t)j * p.N + k);
        const float* cy = w.cy + 3 * ((size_t)i * p.N + k);
        s_coef[6 * k + 0] = cx[0];
        s_coef[6 * k + 1] = cx[1];
        s_coef[6 * k + 2] = cx[2];
        s_coef[6 * k + 3] = cy[0];
        s_coef[6 * k + 4] = cy[1];
        s_coef[6 * k + 5] = cy[2];
        s_cnt[k] = count[k];
    }
    __syncthreads();
    const int x = blockIdx.y * kCompBX + threadIdx.x;
    const int y = blockIdx.z * kCompBY + threadIdx.y;
    if (x >= p.Nx || y >= p.Ny) return;
    const size_t plane_sz = (size_t)p.W * p.H;
    float Q0 = 0.f, Q1 = 0.f, Q2 = 0.f, T = 1.f;
    int kq = -1;   // saving form: the plane the walk stopped at (blend_texel)
    int q = 0;     // non-empty planes so far
    for (int k = 0; k < p.N; ++k) {
        if (s_cnt[k] == 0) continue;
        // plain form: the staged kernels' flush of T below 2^-24 (flush_tiny),
        // at the same list positions
        if (!SAVE && (q & 3) == 0 && q > 0 && T < kTFlush) {
            T = 0.0f;
            break;
        }
        ++q;
        const float* c = s_coef + 6 * k;
        float4 tx = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!BILINEAR) {
            const int ix = nearest_index(p.P_s, x, c[0], c[1]);
            const int iy = nearest_index(p.P_s, y, c[3], c[4]);
            if (ix >= 0 && ix < p.W && iy >= 0 && iy < p.H)
                tx = load_texel<DT>(planes, (size_t)k * plane_sz + (size_t)iy * p.W + ix);
        } else {
            const float Dx = __fmaf_rn(c[0], (float)x, c[2]);
            const float Dy = __fmaf_rn(c[3], (float)y, c[5]);
            if (Dx >= -1.0e6f && Dx <= 1.0e6f && Dy >= -1.0e6f && Dy <= 1.0e6f) {
                const float flx = floorf(Dx), fly = floorf(Dy);
                const float wx = Dx - flx, wy = Dy - fly;
                const int x0 = p.P_s * x + (int)flx, y0 = p.P_s * y + (int)fly;
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int yy = y0 + dy;
                    if (yy < 0 || yy >= p.H) continue;
                    const float wyy = dy ? wy : 1.0f - wy;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int xx = x0 + dx;
                        if (xx < 0 || xx >= p.W) continue;
                        const float ww = wyy * (dx ? wx : 1.0f - wx);
                        const float4 t = load_texel<DT>(planes, (size_t)k * plane_sz + (size_t)yy * p.W + xx);
                        tx.x = fmaf(ww, t.x, tx.x);
                        tx.y = fmaf(ww, t.y, tx.y);
                        tx.z = fmaf(ww, t.z, tx.z);
                        tx.w = fmaf(ww, t.w, tx.w);
                    }
                }
            }
        }
        if (!SAVE) {
            Q0 = fmaf(T, tx.x, Q0);
            Q1 = fmaf(T, tx.y, Q1);
            Q2 = fmaf(T, tx.z, Q2);
            T = T * (1.0f - tx.w);
        } else {
            // the staged saving form's stop rule: T_k frozen at the stop plane
            Q0 = fmaf(T, tx.x, Q0);
            Q1 = fmaf(T, tx.y, Q1);
            Q2 = fmaf(T, tx.z, Q2);
            const float nt = T * (1.0f - tx.w);
            if (nt < kTStop) {
                kq = k;
                break;
            }
            T = nt;
        }
    }
    const float Tn = SAVE && kq >= 0 ? 0.0f : T;
    reinterpret_cast<float4*>(out)[view_pixel(p, v, x, y)] =
        make_float4(fmaf(Tn, p.bg[0], Q0), fmaf(Tn, p.bg[1], Q1), fmaf(Tn, p.bg[2], Q2), 1.0f - Tn);
    if (SAVE)
        state[((size_t)v * p.Ny + y) * p.Nx + x] = make_float4(T, __int_as_float(kq < 0 ? p.N : kq), 0.0f, 0.0f);
}

// ---------------------------------------------------------------------------
// Staged composite. All views of one view row i sample plane k on the same
// plane rows (their vertical map depends on (i, k) only), and neighbouring
// views read horizontally shifted copies of those rows. A CTA therefore owns
// BY output rows x TX output columns for a group of VG views of one view row;
// for every non-empty plane one producer thread copies the BY plane rows the
// CTA needs (2 BY for bilinear) into shared memory with bulk asynchronous
// copies (cp.async.bulk, completion counted on a "full" mbarrier), and every
// thread composites its pixel for the VG views from shared memory. Warps
// release a stage through an "empty" mbarrier, so no CTA-wide barrier sits in
// the nearest plane loop. Bilinear (single-scene kernel): the vertical tap
// pair depends on (i, k, y) only, so the threads of an output row first blend
// the two staged rows into an FP32 row in shared memory (double buffered by
// plane parity, one CTA barrier per plane, the stage released right after),
// and each view then takes its two horizontal taps from that row: 2 instead
// of 4 texel reads per view and plane. Every staged row carries zero texels
// on both sides: an out-of-plane index is clamped onto one and reads a
// transparent zero.
// The floor of the FP32 index uses the exact round-toward-minus-infinity add
// of 1.5 * 2^23 (valid for |value| < 2^22) instead of a conversion unit op.
// All waits are bounded; a wait that gives up sets the error word.
// ---------------------------------------------------------------------------

constexpr int kStagedWarps = kStagedThreads / 32;     // consumer warps
constexpr int kStagedBlock = kStagedThreads + 32;     // + one producer warp
constexpr int kBwdWarps = kBwdStagedThreads / 32;     // the adjoint's
constexpr int kBwdBlock = kBwdStagedThreads + 32;
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// explicit shared-space loads (32-bit shared addresses, LDS)
__device__ __forceinline__ float4 lds_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ uint2 lds_u2(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

template <int DT>
struct Texel;
template <>
struct Texel<LF_F32> {
    static constexpr int kBytes = 16;
    static __device__ __forceinline__ float4 load(uint32_t row, uint32_t i) { return lds_f4(row + i * 16u); }
};
template <>
struct Texel<LF_F16> {
    static constexpr int kBytes = 8;
    static __device__ __forceinline__ float4 load(uint32_t row, uint32_t i)
    {
        const uint2 u = lds_u2(row + i * 8u);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <>
struct Texel<LF_U8> {
    static constexpr int kBytes = 4;
    static __device__ __forceinline__ float4 load(uint32_t row, uint32_t i) { return u8_unpack(lds_u32(row + i * 4u)); }
};
template <>
struct Texel<LF_BF16> {
    static constexpr int kBytes = 8;
    static __device__ __forceinline__ float4 load(uint32_t row, uint32_t i)
    {
        const uint2 u = lds_u2(row + i * 8u);
        return bf16x4_to_f32(u);
    }
};


// floor(fma(g, x, h)) as the bit pattern of (value + 1.5 * 2^23) rounded
// toward minus infinity; callers add base - kMagicBits to get an index.
template <bool CLAMP>
__device__ __forceinline__ float floor_magic(float g, float x, float h)
{
    float f = __fmaf_rn(g, x, h);
    if (CLAMP) f = fminf(fmaxf(f, -kClamp), kClamp);
    return __fadd_rd(f, kMagic);
}

// plane row sampled by output row y (nearest) or its upper bilinear row
__device__ __forceinline__ int plane_row(int P_s, int y, float gm, float h)
{
    return P_s * y + (__float_as_int(floor_magic<true>(gm, (float)y, h)) - kMagicBits);
}

// Coefficient block of one plane (16-byte aligned, read with broadcast
// 16-byte loads): [gm_x, gm_y, h_y, wide] then h_x of the VG views.
template <int VG>
struct CoefBlock {
    static constexpr int kFloats = 4 + 4 * ((VG + 3) / 4);
};

inline size_t round16(size_t v) { return (v + 15) / 16 * 16; }

}  // namespace

// Staged layout of one composite: TX columns x BY rows per CTA (TX a
// multiple of 32 not above tx_max or the consumer threads, BY = threads /
// TX), VG views per thread.
StagedGeom staged_geom(const CompParams& p, int texel_bytes, bool bilinear, int VG, int tx_max, int threads)
{
    StagedGeom G;
    const int nx32 = (p.Nx + 31) / 32 * 32;
    G.TX = nx32 < tx_max ? nx32 : tx_max;
    if (G.TX > threads) G.TX = threads;
    G.BY = threads / G.TX;
    G.VG = VG;
    G.rows_per_y = bilinear ? 2 : 1;
    G.padl = 16 / texel_bytes;
    G.row_texels = (int)(round16((size_t)(G.padl + p.W + 1) * texel_bytes) / texel_bytes);
    G.row_bytes = (size_t)G.row_texels * texel_bytes;
    G.stage_bytes = G.row_bytes * G.BY * G.rows_per_y;
    G.groups_x = (p.Vx + VG - 1) / VG;
    G.blend_bytes = bilinear ? (size_t)2 * G.BY * G.row_texels * 16 : 0;
    const size_t fixed = G.blend_bytes + 2 * kStages * 8 + sizeof(float) * (size_t)p.N * (4 + 4 * ((VG + 3) / 4)) +
                         sizeof(int) * (size_t)p.N;
    // a bilinear stage is released once its rows are blended, so a shallower
    // ring suffices: keep the CTAs per SM the launch bounds aim at (256
    // threads: two for view groups wider than kTwoCtaViews, four below; 512:
    // one and two) where they fit
    G.stages = kStages;
    const size_t budget = threads == 256 ? (VG > kTwoCtaViews ? kTwoCtaSmem : kTwoCtaSmem / 2)
                                         : (VG > kTwoCtaViews ? (size_t)200 * 1024 : kTwoCtaSmem);
    while (bilinear && G.stages > 3 && G.stages * G.stage_bytes + fixed > budget) --G.stages;
    G.smem_bytes = G.stages * G.stage_bytes + fixed;
    return G;
}

namespace {

// Per-thread constants of one staged item, computed once per item.
struct ThreadGeom {
    float xf, yf;          // output pixel
    int psy;               // P_s y
    int base_x;            // P_s x + left pad - magic bits
    int H;                 // plane rows
    uint32_t row0;         // offset of the thread's (first) staged row in a stage
    uint32_t row_bytes;    // staged row pitch
    uint32_t maxi;         // first right-pad texel
};

__device__ __forceinline__ ThreadGeom thread_geom(const CompParams& p, const StagedGeom& G, int x, int y, int ty)
{
    ThreadGeom t;
    t.xf = (float)x;
    t.yf = (float)y;
    t.psy = p.P_s * y;
    t.base_x = p.P_s * x + G.padl - kMagicBits;
    t.H = p.H;
    t.row0 = (uint32_t)(ty * G.rows_per_y) * (uint32_t)G.row_bytes;
    t.row_bytes = (uint32_t)G.row_bytes;
    t.maxi = (uint32_t)(G.padl + p.W);
    return t;
}

// Stores q to view J's stop slot when on ([stop_a + immediate]: no address
// register per view, no branch).
template <int J>
__device__ __forceinline__ void st_stop(uint32_t stop_a, int q, bool on)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.shared.u32 [%0+%3], %1;\n\t}"
                 ::"r"(stop_a), "r"(q), "r"((uint32_t)on), "n"(4 * J));
}

// One view's blend of one texel t at plane list entry q (view jj of the
// thread's group). Plain form: Q += T c, T <- T - T A. Saving form: the
// view's walk stops at the first list entry q behind which T would fall
// below kTStop (0 behind a plane with A = 1): plane q still blends with its
// T_q, q goes to the view's stop slot in shared memory (stop_a + 4 jj, the
// thread's VG slots), and a[3] = -T_q marks the view as stopped (T_q >=
// kTStop > 0; T = 0 from there on, the colour the plain form would still
// add being below 2^-24 per plane). The kernel stores the state at the end
// of its walk.
template <bool SAVE>
__device__ __forceinline__ void blend_texel(float (&a)[4], float4 t, uint32_t stop_a, int jj, int q)
{
    if (!SAVE) {
        const float T = a[3];
        a[0] = fmaf(T, t.x, a[0]);
        a[1] = fmaf(T, t.y, a[1]);
        a[2] = fmaf(T, t.z, a[2]);
        a[3] = fmaf(-T, t.w, T);
    } else {
        const float T = fmaxf(a[3], 0.0f);
        a[0] = fmaf(T, t.x, a[0]);
        a[1] = fmaf(T, t.y, a[1]);
        a[2] = fmaf(T, t.z, a[2]);
        const float nt = fmaf(-T, t.w, T);
        const bool stop = a[3] > 0.0f && nt < kTStop;   // branch-free: a predicated store
        switch (jj) {   // jj is a constant in every (unrolled) caller
        case 0: st_stop<0>(stop_a, q, stop); break;
        case 1: st_stop<1>(stop_a, q, stop); break;
        case 2: st_stop<2>(stop_a, q, stop); break;
        case 3: st_stop<3>(stop_a, q, stop); break;
        case 4: st_stop<4>(stop_a, q, stop); break;
        case 5: st_stop<5>(stop_a, q, stop); break;
        case 6: st_stop<6>(stop_a, q, stop); break;
        case 7: st_stop<7>(stop_a, q, stop); break;
        case 8: st_stop<8>(stop_a, q, stop); break;
        case 9: st_stop<9>(stop_a, q, stop); break;
        case 10: st_stop<10>(stop_a, q, stop); break;
        case 11: st_stop<11>(stop_a, q, stop); break;
        case 12: st_stop<12>(stop_a, q, stop); break;
        case 13: st_stop<13>(stop_a, q, stop); break;
        default: st_stop<14>(stop_a, q, stop); break;
        }
        a[3] = stop ? -T : (a[3] > 0.0f ? nt : a[3]);
    }
}

// hdr: (gm_x, gm_y, h_y, -); ca: shared address of the plane's coefficient
// block; sb: shared address of the stage holding the plane's rows
template <int DT, bool BILINEAR, int VG, bool CLAMP, bool SAVE = false>
__device__ __forceinline__ void blend_plane(float (&acc)[VG][4], float4 hdr, uint32_t ca, uint32_t sb,
                                            const ThreadGeom& tg, uint32_t stop_a, int q)
{
    using TX_ = Texel<DT>;
    const uint32_t maxi = tg.maxi;
    float c[3 + 4 * ((VG + 3) / 4)];
    c[0] = hdr.x;
    c[1] = hdr.y;
    c[2] = hdr.z;
#pragma unroll
    for (int e = 0; e < (VG + 3) / 4; ++e) {
        const float4 v = lds_f4(ca + 16u * (1 + e));
        c[3 + 4 * e + 0] = v.x;
        c[3 + 4 * e + 1] = v.y;
        c[3 + 4 * e + 2] = v.z;
        c[3 + 4 * e + 3] = v.w;
    }
    const float gmx = c[0];
    const float xf = tg.xf;
    const int base_x = tg.base_x;
    if (!BILINEAR) {
        const int iy = tg.psy + (__float_as_int(floor_magic<true>(c[1], tg.yf, c[2])) - kMagicBits);
        if (iy < 0 || iy >= tg.H) return;
        const uint32_t row = sb + tg.row0;
#pragma unroll
        for (int jj = 0; jj < VG; ++jj) {
            const int ix = __float_as_int(floor_magic<CLAMP>(gmx, xf, c[3 + jj])) + base_x;
            const float T = acc[jj][3];
            if constexpr (DT == LF_U8 && !SAVE) {
                // colour bytes scale by 1/255 through T (one multiply per
                // texel instead of three); alpha keeps A = byte / 255
                constexpr float s = 1.0f / 255.0f;
                const uint32_t u = lds_u32(row + min((uint32_t)ix, maxi) * 4u);
                const float Ts = T * s;
                acc[jj][0] = fmaf(Ts, u8_byte<0>(u), acc[jj][0]);
                acc[jj][1] = fmaf(Ts, u8_byte<1>(u), acc[jj][1]);
                acc[jj][2] = fmaf(Ts, u8_byte<2>(u), acc[jj][2]);
                acc[jj][3] = fmaf(-T, u8_byte<3>(u) * s, T);
            } else {
                const float4 t = TX_::load(row, min((uint32_t)ix, maxi));
                blend_texel<SAVE>(acc[jj], t, stop_a, jj, q);
            }
        }
    } else {
        float fy = __fmaf_rn(c[1], tg.yf, c[2]);
        fy = fminf(fmaxf(fy, -kClamp), kClamp);
        const float ty_m = __fadd_rd(fy, kMagic);
        const float wy = fy - (ty_m - kMagic);
        const int y0 = tg.psy + (__float_as_int(ty_m) - kMagicBits);
        const bool v0 = y0 >= 0 && y0 < tg.H, v1 = y0 + 1 >= 0 && y0 + 1 < tg.H;
        if (!v0 && !v1) return;
        const float w0 = v0 ? 1.0f - wy : 0.0f, w1 = v1 ? wy : 0.0f;
        const uint32_t r0 = sb + tg.row0;
        const uint32_t r1 = r0 + tg.row_bytes;
#pragma unroll
        for (int jj = 0; jj < VG; ++jj) {
            float fx = __fmaf_rn(gmx, xf, c[3 + jj]);
            if (CLAMP) fx = fminf(fmaxf(fx, -kClamp), kClamp);
            const float tm = __fadd_rd(fx, kMagic);
            const float wx = fx - (tm - kMagic), wa = 1.0f - wx;
            const int i0 = __float_as_int(tm) + base_x;
            const uint32_t a0 = min((uint32_t)i0, maxi), a1 = min((uint32_t)(i0 + 1), maxi);
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v0) {
                const float4 ta = TX_::load(r0, a0), tb = TX_::load(r0, a1);
                t.x = w0 * fmaf(wa, ta.x, wx * tb.x);
                t.y = w0 * fmaf(wa, ta.y, wx * tb.y);
                t.z = w0 * fmaf(wa, ta.z, wx * tb.z);
                t.w = w0 * fmaf(wa, ta.w, wx * tb.w);
            }
            if (v1) {
                const float4 ta = TX_::load(r1, a0), tb = TX_::load(r1, a1);
                t.x = fmaf(w1, fmaf(wa, ta.x, wx * tb.x), t.x);
                t.y = fmaf(w1, fmaf(wa, ta.y, wx * tb.y), t.y);
                t.z = fmaf(w1, fmaf(wa, ta.z, wx * tb.z), t.z);
                t.w = fmaf(w1, fmaf(wa, ta.w, wx * tb.w), t.w);
            }
            blend_texel<SAVE>(acc[jj], t, stop_a, jj, q);
        }
    }
}

// Bilinear horizontal taps from a vertically pre-blended FP32 row (shared
// address ba, same texel layout as a staged row).
template <int VG, bool CLAMP, bool SAVE = false>
__device__ __forceinline__ void blend_blended_row(float (&acc)[VG][4], float4 hdr, uint32_t ca, uint32_t ba,
                                                  const ThreadGeom& tg, uint32_t stop_a, int q)
{
    float c[4 * ((VG + 3) / 4)];
#pragma unroll
    for (int e = 0; e < (VG + 3) / 4; ++e) {
        const float4 v = lds_f4(ca + 16u * (1 + e));
        c[4 * e + 0] = v.x;
        c[4 * e + 1] = v.y;
        c[4 * e + 2] = v.z;
        c[4 * e + 3] = v.w;
    }
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) {
        float fx = __fmaf_rn(hdr.x, tg.xf, c[jj]);
        if (CLAMP) fx = fminf(fmaxf(fx, -kClamp), kClamp);
        const float tm = __fadd_rd(fx, kMagic);
        const float wx = fx - (tm - kMagic), wa = 1.0f - wx;
        const int i0 = __float_as_int(tm) + tg.base_x;
        const uint32_t a0 = min((uint32_t)i0, tg.maxi), a1 = min((uint32_t)(i0 + 1), tg.maxi);
        const float4 ta = lds_f4(ba + a0 * 16u), tb = lds_f4(ba + a1 * 16u);
        const float4 t = make_float4(fmaf(wa, ta.x, wx * tb.x), fmaf(wa, ta.y, wx * tb.y), fmaf(wa, ta.z, wx * tb.z),
                                     fmaf(wa, ta.w, wx * tb.w));
        blend_texel<SAVE>(acc[jj], t, stop_a, jj, q);
    }
}

// Plain form, before every fourth non-empty plane of the list: a view whose
// transmittance has fallen below kTFlush = 2^-24 (the FP32 spacing at 1)
// takes T = 0, so the planes behind it add nothing; what they would still
// add is below 2^-24 of a colour's range per channel, and the output's
// 1 - T moves by less than 2^-24. The decision depends on the view pixel's
// own walk and the list position only, so every layout of the work
// (views per thread, tiles, batch plans) gives the same bits.
template <int VG>
__device__ __forceinline__ void flush_tiny(float (&acc)[VG][4])
{
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) acc[jj][3] = acc[jj][3] < kTFlush ? 0.0f : acc[jj][3];
}

// Every view of this thread has T == 0 exactly (or the thread is idle).
// T never leaves 0 (T <- T - T A), and behind it a plane adds T c = 0 to Q
// and leaves T = 0, so skipping such planes changes no bit of the output.
// (Saving form: every view has stopped, a[3] < 0.)
template <int VG, bool SAVE = false>
__device__ __forceinline__ bool saturated(const float (&acc)[VG][4], bool live)
{
    bool s = true;
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) s = s && (SAVE ? acc[jj][3] < 0.0f : acc[jj][3] == 0.0f);
    return s || !live;
}

// Stages the plane rows that list entry q (plane k = plist[q], coefficient
// block c) needs for output rows Y0 .. Y0 + BY - 1 into stage sb, with their
// byte count announced on mbarrier bar (one producer thread).
template <int DT>
__device__ __forceinline__ void produce_rows(const CompParams& p, const StagedGeom& G, const char* __restrict__ planes,
                                             int k, const float* c, int Y0, unsigned char* sb, uint32_t bar)
{
    constexpr int TB = Texel<DT>::kBytes;
    const size_t plane_bytes = (size_t)p.W * p.H * TB;
    const uint32_t row_copy = (uint32_t)((size_t)p.W * TB);   // a multiple of 16 (checked at launch)
    uint32_t bytes = 0;
    for (int r = 0; r < G.BY; ++r) {
        const int yy = Y0 + r;
        if (yy >= p.Ny) continue;
        const int base = plane_row(p.P_s, yy, c[1], c[2]);
        for (int t = 0; t < G.rows_per_y; ++t)
            if (base + t >= 0 && base + t < p.H) bytes += row_copy;
    }
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, bytes);
    for (int r = 0; r < G.BY; ++r) {
        const int yy = Y0 + r;
        if (yy >= p.Ny) continue;
        const int base = plane_row(p.P_s, yy, c[1], c[2]);
        for (int t = 0; t < G.rows_per_y; ++t) {
            const int iy = base + t;
            if (iy < 0 || iy >= p.H) continue;
            const char* src = planes + (size_t)k * plane_bytes + (size_t)iy * row_copy;
            unsigned char* dst = sb + (size_t)(r * G.rows_per_y + t) * G.row_bytes + (size_t)G.padl * TB;
            bulk_copy_g2s(smem_addr(dst), src, row_copy, bar);
        }
    }
}

// Non-empty planes in order into plist (warp 0 only); returns their count.
__device__ __forceinline__ int plane_list(const CompParams& p, const int32_t* __restrict__ count, int* plist)
{
    const int lane = threadIdx.x & 31;
    int n = 0;
    for (int b = 0; b < p.N; b += 32) {
        const int k = b + lane;
        const bool ne = k < p.N && count[k] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, ne);
        if (ne) plist[n + __popc(m & ((1u << lane) - 1u))] = k;
        n += __popc(m);
    }
    return n;
}

// Coefficient blocks of views j0 .. j0 + VG - 1 (view row vi), list order.
template <bool BILINEAR, int VG>
__device__ __forceinline__ void load_coefs(const CompParams& p, const CompWs& w, const int* plist, int P, int vi,
                                           int j0, float* coef)
{
    constexpr int CW = CoefBlock<VG>::kFloats;
    for (int e = threadIdx.x; e < P * VG; e += blockDim.x) {
        const int q = e / VG, jj = e % VG;
        const int k = plist[q];
        const int j = min(j0 + jj, p.Vx - 1);
        const float* cx = w.cx + 3 * ((size_t)j * p.N + k);
        coef[q * CW + 4 + jj] = BILINEAR ? cx[2] : cx[1];
        if (jj == 0) {
            const float* cy = w.cy + 3 * ((size_t)vi * p.N + k);
            coef[q * CW + 0] = cx[0];
            coef[q * CW + 1] = cy[0];
            coef[q * CW + 2] = BILINEAR ? cy[2] : cy[1];
            coef[q * CW + 3] = __int_as_float(w.wide[k]);
        }
    }
}

// Zero left and right pads of every staged row (the bulk copies never write them).
template <int DT>
__device__ __forceinline__ void zero_pads(const CompParams& p, const StagedGeom& G, unsigned char* stage_base,
                                          size_t stage_stride, int nstages)
{
    constexpr int TB = Texel<DT>::kBytes;
    const int nrows = G.BY * G.rows_per_y;
    // 16-byte chunks: left pad [0, padl TB), right pad [(padl + W) TB, row_bytes)
    const int lc = G.padl * TB / 16, rc = (int)((G.row_bytes - (size_t)(G.padl + p.W) * TB) / 16);
    const int per_row = lc + rc;
    for (int e = threadIdx.x; e < nstages * nrows * per_row; e += blockDim.x) {
        const int r = e / per_row, c = e % per_row;
        unsigned char* row = stage_base + (size_t)(r / nrows) * stage_stride + (size_t)(r % nrows) * G.row_bytes;
        const size_t off = c < lc ? (size_t)c * 16 : (size_t)(G.padl + p.W) * TB + (size_t)(c - lc) * 16;
        *reinterpret_cast<uint4*>(row + off) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// SAVE: also writes, per view pixel, the state the adjoint's back-to-front
// walk starts from, state[(v Ny + y) Nx + x] = {T_k, bits of k, 0, 0}: k the
// plane behind which T falls below 2^-24 (and is taken as 0), T_k the
// transmittance in front of it; or k = N and the transmittance behind the
// last plane (see blend_texel).
// NT consumer threads (256: two CTAs per SM at up to 15 views per thread,
// four below; 512 where two CTAs of 256 would not fit their shared memory on
// an SM: one CTA of 16 consumer warps then, two below).
template <int DT, bool BILINEAR, int VG, bool SAVE = false, int NT = kStagedThreads>
__global__ void __launch_bounds__(NT + 32, NT == 256 ? (VG > kTwoCtaViews ? 2 : 4) : (VG > kTwoCtaViews ? 1 : 2))
    k_composite_staged(CompParams p, StagedGeom G,
                                                                        const char* __restrict__ planes,
                                                                        const int32_t* __restrict__ count, CompWs w,
                                                                        float* __restrict__ out,
                                                                        float4* __restrict__ state)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // [stages][rows][row_bytes] | bilinear: [2][BY][row_texels] float4 |
    // full[kStages] | empty[kStages] | coef [N][CW] | plist [N] | saving
    // form: stop slots [NT][VG]
    constexpr int CW = CoefBlock<VG>::kFloats;
    unsigned char* stage_base = smem;
    // bilinear: the two staged rows of an output row are blended vertically
    // once per plane into an FP32 row (double buffered by plane parity)
    const int NS = BILINEAR ? G.stages : kStages;   // nearest keeps a compile-time ring depth
    unsigned char* blend_base = smem + NS * G.stage_bytes;
    // nearest has no blend rows; spelling its barrier base out as the ring's
    // end gives measurably faster per-plane barrier addressing
    uint64_t* full = reinterpret_cast<uint64_t*>(BILINEAR ? blend_base + G.blend_bytes : smem + kStages * G.stage_bytes);
    uint64_t* empty = full + kStages;
    float* coef = reinterpret_cast<float*>(empty + kStages);   // 16-byte aligned (stage_bytes, 2 kStages * 8)
    int* plist = reinterpret_cast<int*>(coef + (size_t)p.N * CW);
    __shared__ int s_nplanes;

    const int tid = threadIdx.x, lane = tid & 31;
    // fastest: the view groups, then the column tiles of one row band, so
    // that the CTAs reading the same plane rows run together (rows read from
    // DRAM once, then from L2)
    const int nvg = G.groups_x * p.Vy;
    const int vgroup = blockIdx.x % nvg;
    const int vi = vgroup / G.groups_x;            // view row
    const int j0 = (vgroup % G.groups_x) * VG;     // first view column of the group
    // row bands from both edges inward: the bands whose views rarely reach
    // T = 0 (the scene's borders) start first, the cheap centre ones last
    const int by = (int)blockIdx.y;
    const int band = (by & 1) ? (int)gridDim.y - 1 - (by >> 1) : (by >> 1);
    const int Y0 = band * G.BY;
    const int X0 = (blockIdx.x / nvg) * G.TX;
    const int tx = tid % G.TX, ty = tid / G.TX;
    const int x = X0 + tx, y = Y0 + ty;

    // list of non-empty planes in order (warp 0, ballot compaction)
    if (tid < 32) {
        const int n = plane_list(p, count, plist);
        if (tid == 0) s_nplanes = n;
    }
    __syncthreads();
    load_coefs<BILINEAR, VG>(p, w, plist, s_nplanes, vi, j0, coef);
    zero_pads<DT>(p, G, stage_base, G.stage_bytes, NS);
    if constexpr (BILINEAR) {
        // pads of the blended rows: zero once (the blend writes interiors only)
        float4* bb = reinterpret_cast<float4*>(blend_base);
        const int pads = G.row_texels - p.W;
        for (int e = tid; e < 2 * G.BY * pads; e += blockDim.x) {
            const int r = e / pads, t = e % pads;
            bb[(size_t)r * G.row_texels + (t < G.padl ? t : t + p.W)] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), (NT / 32));
        }
        fence_proxy_async();
    }
    __syncthreads();
    const int P = s_nplanes;

    // producer: stage the plane rows of list entry q into stage q % NS
    auto produce = [&](int q) {
        produce_rows<DT>(p, G, planes, plist[q], coef + (size_t)q * CW, Y0,
                         stage_base + (size_t)(q % NS) * G.stage_bytes, smem_addr(&full[q % NS]));
    };

    if (tid >= NT) {
        // producer warp: one lane streams the planes through the stage ring,
        // refilling a stage as soon as every consumer warp has released it
        if (tid == NT) {
            for (int q = 0; q < P; ++q) {
                const int s = q % NS;
                if (q >= NS && !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)(((q / NS) - 1) & 1))) {
                    atomicExch(w.err, 1);
                    break;
                }
                produce(q);
            }
        }
        return;
    }

    float acc[VG][4];
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) acc[jj][0] = acc[jj][1] = acc[jj][2] = 0.f, acc[jj][3] = 1.f;
    // saving form: the stop slots [NT][VG] follow plist
    const uint32_t stop_a = smem_addr(plist + p.N) + 4u * (uint32_t)(tid * VG);
    const uint32_t stage_a = smem_addr(stage_base), coef_a = smem_addr(coef);
    const bool live = ty < G.BY && x < p.Nx && y < p.Ny;   // threads past BY rows idle
    const ThreadGeom tg = thread_geom(p, G, x, y, ty);
    bool ok = true;
    bool warp_sat = false;   // every view of every lane of this warp has T == 0

    for (int q = 0; q < P; ++q) {
        const int s = q % NS;
        const uint32_t parity = (uint32_t)((q / NS) & 1);
        if ((!BILINEAR || ok) && !mbar_wait_bounded(smem_addr(&full[s]), parity)) {
            atomicExch(w.err, 1);
            ok = false;
            // bilinear: keep meeting the per-plane CTA barrier (results discarded)
            if (!BILINEAR) break;
        }
        if ((q & 3) == 0 && q > 0 && !warp_sat) {
            if (!SAVE) flush_tiny<VG>(acc);
            warp_sat = __all_sync(0xffffffffu, saturated<VG, SAVE>(acc, live));
        }
        if constexpr (BILINEAR) {
            // the threads of an output row blend interior texels tx, tx + TX,
            // ... of its two staged rows into the FP32 row buffer
            const uint32_t ca = coef_a + 4u * (uint32_t)(q * CW);
            const float4 hdr = lds_f4(ca);
            float4* brow = reinterpret_cast<float4*>(blend_base) + ((size_t)(q & 1) * G.BY + ty) * G.row_texels;
            if (ty < G.BY) {
                float fy = __fmaf_rn(hdr.y, tg.yf, hdr.z);
                fy = fminf(fmaxf(fy, -kClamp), kClamp);
                const float ty_m = __fadd_rd(fy, kMagic);
                const float wy = fy - (ty_m - kMagic);
                const int y0 = tg.psy + (__float_as_int(ty_m) - kMagicBits);
                const bool v0 = y0 >= 0 && y0 < tg.H, v1 = y0 + 1 >= 0 && y0 + 1 < tg.H;
                const float w0 = v0 ? 1.0f - wy : 0.0f, w1 = v1 ? wy : 0.0f;
                const uint32_t r0 = stage_a + (uint32_t)(s * G.stage_bytes) + tg.row0;
                const uint32_t r1 = r0 + tg.row_bytes;
                for (int i = G.padl + tx; i < G.padl + p.W; i += G.TX) {
                    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (v0) {
                        const float4 a = Texel<DT>::load(r0, (uint32_t)i);
                        t = make_float4(w0 * a.x, w0 * a.y, w0 * a.z, w0 * a.w);
                    }
                    if (v1) {
                        const float4 b = Texel<DT>::load(r1, (uint32_t)i);
                        t = make_float4(fmaf(w1, b.x, t.x), fmaf(w1, b.y, t.y), fmaf(w1, b.z, t.z), fmaf(w1, b.w, t.w));
                    }
                    brow[i] = t;
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
            // the staged rows are no longer needed: release the stage now
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
            if (live && !warp_sat) {
                const uint32_t ba = smem_addr(brow);
                if (__float_as_int(hdr.w))
                    blend_blended_row<VG, true, SAVE>(acc, hdr, ca, ba, tg, stop_a, q);
                else
                    blend_blended_row<VG, false, SAVE>(acc, hdr, ca, ba, tg, stop_a, q);
            }
        } else {
            if (live && !warp_sat) {
                const uint32_t ca = coef_a + 4u * (uint32_t)(q * CW);
                const uint32_t sb = stage_a + (uint32_t)(s * G.stage_bytes);
                const float4 hdr = lds_f4(ca);
                if (__float_as_int(hdr.w))
                    blend_plane<DT, BILINEAR, VG, true, SAVE>(acc, hdr, ca, sb, tg, stop_a, q);
                else
                    blend_plane<DT, BILINEAR, VG, false, SAVE>(acc, hdr, ca, sb, tg, stop_a, q);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
        }
    }
    if (!ok || !live) return;
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) {
        const int j = j0 + jj;
        if (j >= p.Vx) break;
        const int v = vi * p.Vx + j;
        const float T = SAVE ? fmaxf(acc[jj][3], 0.0f) : acc[jj][3];
        reinterpret_cast<float4*>(out)[view_pixel(p, v, x, y)] = make_float4(
            fmaf(T, p.bg[0], acc[jj][0]), fmaf(T, p.bg[1], acc[jj][1]), fmaf(T, p.bg[2], acc[jj][2]), 1.0f - T);
        if (SAVE) {
            // stopped: {T_k, k} of the stop plane; else {T behind the last plane, N}
            const bool stopped = acc[jj][3] < 0.0f;
            const int k = stopped ? plist[lds_u32(stop_a + 4u * (uint32_t)jj)] : p.N;
            state[((size_t)v * p.Ny + y) * p.Nx + x] =
                make_float4(fabsf(acc[jj][3]), __int_as_float(k), 0.0f, 0.0f);
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent staged composite over the items of several scenes (same plane
// type, sampling and views per thread). Each CTA takes (scene, view group,
// row band, column tile) items from a global counter until none are left;
// shared memory is laid out once for the largest stage and N of the batch.
// The plane-row ring and its mbarriers run on across items: the producer and
// the consumers count every plane they pass through the ring (Q), so stage
// Q % kStages and phase (Q / kStages) & 1 stay consistent from one item to
// the next. Between items the CTA synchronises, rebuilds the plane list and
// coefficient blocks, and re-zeroes row pads when the scene (row layout)
// changes. A wait that gives up sets the scene's error word and the CTA
// stops taking items.
// ---------------------------------------------------------------------------
template <int DT, bool BILINEAR, int VG>
__global__ void __launch_bounds__(kStagedBlock, VG > kTwoCtaViews ? 2 : 4) k_composite_batched(const CompScene* __restrict__ scs, int n_sc,
                                                                         long long total,
                                                                         unsigned long long* __restrict__ counter,
                                                                         size_t max_stage_bytes, int maxN)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CW = CoefBlock<VG>::kFloats;
    unsigned char* stage_base = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * max_stage_bytes);
    uint64_t* empty = full + kStages;
    float* coef = reinterpret_cast<float*>(empty + kStages);
    int* plist = reinterpret_cast<int*>(coef + (size_t)maxN * CW);
    __shared__ int s_nplanes, s_abort;
    __shared__ long long s_item;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(smem_addr(&full[st]), 1);
            mbar_init(smem_addr(&empty[st]), kStagedWarps);
        }
        fence_proxy_async();
        s_abort = 0;
    }
    const uint32_t stage_a = smem_addr(stage_base), coef_a = smem_addr(coef);
    // ring position of the next plane: stage st0, phase ph0 (flips every
    // kStages planes), and whether the ring has been round once (from then
    // on the producer waits for the consumers to release a stage)
    int st0 = 0;
    uint32_t ph0 = 0;
    bool wrapped = false;
    int prev = -1;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= total || s_abort) break;
        int si = 0;
        while (si + 1 < n_sc && it >= scs[si + 1].base) ++si;
        const CompParams p = scs[si].p;
        const StagedGeom G = scs[si].G;
        const CompWs w = scs[si].w;
        const char* planes = scs[si].planes;
        const long long li0 = it - scs[si].base;
        const int cgs = scs[si].groups;
        const int cg = (int)(li0 % cgs);              // chunk group
        const long long li = li0 / cgs;
        const int ng = G.groups_x * p.Vy;
        const int vgroup = (int)(li % ng);
        const long long rest = li / ng;
        const int vi = vgroup / G.groups_x, j0 = (vgroup % G.groups_x) * VG;
        // column tiles before row bands: the items reading the same plane
        // rows are taken together
        const int ntx = scs[si].nbz;
        const int X0 = (int)(rest % ntx) * G.TX, Y0 = (int)(rest / ntx) * G.BY;

        if (tid < 32) {
            const int n = plane_list(p, scs[si].count, plist);
            if (tid == 0) s_nplanes = n;
        }
        if (si != prev) zero_pads<DT>(p, G, stage_base, max_stage_bytes, kStages);
        __syncthreads();
        // chunk group cg takes the non-empty planes [q0, q1) of the list
        const int q0 = (int)((long long)s_nplanes * cg / cgs), q1 = (int)((long long)s_nplanes * (cg + 1) / cgs);
        load_coefs<BILINEAR, VG>(p, w, plist + q0, q1 - q0, vi, j0, coef);
        __syncthreads();
        const int P = q1 - q0;

        if (tid >= kStagedThreads) {
            if (tid == kStagedThreads) {
                int st = st0;
                uint32_t ph = ph0;
                bool wr = wrapped;
                for (int q = 0; q < P; ++q) {
                    if (wr && !mbar_wait_bounded(smem_addr(&empty[st]), ph ^ 1u)) {
                        atomicExch(w.err, 1);
                        s_abort = 1;
                        break;
                    }
                    produce_rows<DT>(p, G, planes, plist[q0 + q], coef + (size_t)q * CW, Y0,
                                     stage_base + (size_t)st * max_stage_bytes, smem_addr(&full[st]));
                    if (++st == kStages) st = 0, ph ^= 1u, wr = true;
                }
            }
        } else {
            const int tx = tid % G.TX, ty = tid / G.TX;
            const int x = X0 + tx, y = Y0 + ty;
            const bool live = ty < G.BY && x < p.Nx && y < p.Ny;
            const ThreadGeom tg = thread_geom(p, G, x, y, ty);
            float acc[VG][4];
            const uint32_t stop_a = 0;   // unused: the batch blends in the plain form
#pragma unroll
            for (int jj = 0; jj < VG; ++jj) acc[jj][0] = acc[jj][1] = acc[jj][2] = 0.f, acc[jj][3] = 1.f;
            bool ok = true;
            bool warp_sat = false;
            int st = st0;
            uint32_t ph = ph0;
            const uint32_t stage_stride = (uint32_t)max_stage_bytes;
            for (int q = 0; q < P; ++q) {
                if (!mbar_wait_bounded(smem_addr(&full[st]), ph)) {
                    atomicExch(w.err, 1);
                    s_abort = 1;
                    ok = false;
                    break;
                }
                if ((q & 3) == 0 && q > 0 && !warp_sat) {
                    flush_tiny<VG>(acc);
                    warp_sat = __all_sync(0xffffffffu, saturated<VG>(acc, live));
                }
                if (live && !warp_sat) {
                    const uint32_t ca = coef_a + 4u * (uint32_t)(q * CW);
                    const uint32_t sb = stage_a + (uint32_t)st * stage_stride;
                    const float4 hdr = lds_f4(ca);
                    if (__float_as_int(hdr.w))
                        blend_plane<DT, BILINEAR, VG, true>(acc, hdr, ca, sb, tg, stop_a, q);
                    else
                        blend_plane<DT, BILINEAR, VG, false>(acc, hdr, ca, sb, tg, stop_a, q);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
                if (++st == kStages) st = 0, ph ^= 1u;
            }
            if (ok && live) {
                float* out = scs[si].out;
#pragma unroll
                for (int jj = 0; jj < VG; ++jj) {
                    const int j = j0 + jj;
                    if (j >= p.Vx) break;
                    const int v = vi * p.Vx + j;
                    const float T = acc[jj][3];
                    if (cgs == 1) {
                        reinterpret_cast<float4*>(out)[view_pixel(p, v, x, y)] =
                            make_float4(fmaf(T, p.bg[0], acc[jj][0]), fmaf(T, p.bg[1], acc[jj][1]),
                                        fmaf(T, p.bg[2], acc[jj][2]), 1.0f - T);
                    } else {
                        // partial (Q, T) of this chunk group: group 0 in the
                        // view buffer, group c > 0 in partial buffer c - 1
                        const float4 qt = make_float4(acc[jj][0], acc[jj][1], acc[jj][2], T);
                        if (cg == 0)
                            reinterpret_cast<float4*>(out)[view_pixel(p, v, x, y)] = qt;
                        else
                            scs[si].part[(((size_t)(cg - 1) * p.Vx * p.Vy + v) * p.Ny + y) * p.Nx + x] = qt;
                    }
                }
            }
        }
        // every thread advances the ring position by the P planes of the item
        const int adv = st0 + P % kStages;
        ph0 ^= (uint32_t)((P / kStages + (adv >= kStages ? 1 : 0)) & 1);
        wrapped = wrapped || (st0 + P >= kStages);
        st0 = adv >= kStages ? adv - kStages : adv;
        prev = si;
        __syncthreads();
    }
}

template <int DT, bool BILINEAR, int VG, bool SAVE, int NT>
bool launch_staged_nt(const CompParams& p, const StagedGeom& G, const void* planes, const int32_t* count,
                      const CompWs& ws, float* out, cudaStream_t s, float4* state)
{
    auto kern = k_composite_staged<DT, BILINEAR, VG, SAVE, NT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.smem_bytes) != cudaSuccess)
        return false;
    const dim3 grid((unsigned)(G.groups_x * p.Vy * ((p.Nx + G.TX - 1) / G.TX)), (unsigned)((p.Ny + G.BY - 1) / G.BY));
    kern<<<grid, NT + 32, G.smem_bytes, s>>>(p, G, static_cast<const char*>(planes), count, ws, out, state);
    note_launches(1);
    return true;
}

// 256 consumer threads where two such CTAs fit an SM's shared memory, else
// 512 (one CTA of 16 consumer warps keeps the SM as busy as two of 8)
template <int DT, bool BILINEAR, int VG, bool SAVE = false>
bool launch_staged_vg(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                      cudaStream_t s, float4* state = nullptr)
{
    constexpr int TB = Texel<DT>::kBytes;
    // bulk copies need 16-byte aligned rows: plane base and row pitch
    if (((uintptr_t)planes) % 16 != 0 || ((size_t)p.W * TB) % 16 != 0) return false;
    StagedGeom G = staged_geom(p, TB, BILINEAR, VG, 512, 256);
    if (SAVE) G.smem_bytes += sizeof(int) * (size_t)VG * 256;   // stop slots
    if (2 * (G.smem_bytes + 1024) <= (size_t)228 * 1024)
        return launch_staged_nt<DT, BILINEAR, VG, SAVE, 256>(p, G, planes, count, ws, out, s, state);
    G = staged_geom(p, TB, BILINEAR, VG, 512, 512);
    if (SAVE) G.smem_bytes += sizeof(int) * (size_t)VG * 512;
    if (G.smem_bytes > 200 * 1024) return false;
    return launch_staged_nt<DT, BILINEAR, VG, SAVE, 512>(p, G, planes, count, ws, out, s, state);
}

// Views per thread of the staged composite, from {15, 9, 5, 3} (at most Vx,
// or 3): the one with the least padded work, ceil(Vx / VG) (VG + 3) -- a view
// group's fixed cost (plane list, coefficient block, staging every plane's
// rows) measured worth about three views. Groups of 15 run two CTAs of 256
// consumer threads per SM; 9 at four spills a little, and bilinear FP32
// (four-channel FP32 taps) spills more, so it skips 9. Measured on 45 views
// of 512^2, N 64 (one CTA of 512 threads per SM then): 15 beat 9 by 4 %
// (FP32) to 8 % (FP16) nearest and 7-15 % bilinear.
inline int staged_views_per_thread(int Vx, bool no9)
{
    int best = 3;
    long long best_cost = -1;
    for (int vg : {15, 9, 5, 3}) {
        if ((vg > Vx && vg != 3) || (no9 && vg == 9)) continue;
        const long long cost = (long long)((Vx + vg - 1) / vg) * (vg + 3);
        if (best_cost < 0 || cost < best_cost) best_cost = cost, best = vg;
    }
    return best;
}

template <int DT, bool BILINEAR, bool SAVE>
bool launch_staged(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                   cudaStream_t s, float4* state)
{
    switch (staged_views_per_thread(p.Vx, BILINEAR && DT == LF_F32)) {
    case 15: return launch_staged_vg<DT, BILINEAR, 15, SAVE>(p, planes, count, ws, out, s, state);
    case 9: return launch_staged_vg<DT, BILINEAR, 9, SAVE>(p, planes, count, ws, out, s, state);
    case 5: return launch_staged_vg<DT, BILINEAR, 5, SAVE>(p, planes, count, ws, out, s, state);
    default: return launch_staged_vg<DT, BILINEAR, 3, SAVE>(p, planes, count, ws, out, s, state);
    }
}

template <int DT, bool BILINEAR, bool SAVE>
void launch_unstaged(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                     cudaStream_t s, float4* state)
{
    const dim3 block(kCompBX, kCompBY);
    const dim3 grid((unsigned)(p.Vx * p.Vy), (unsigned)((p.Nx + kCompBX - 1) / kCompBX),
                    (unsigned)((p.Ny + kCompBY - 1) / kCompBY));
    const size_t smem = sizeof(float) * 6 * p.N + sizeof(int) * p.N;
    auto kern = k_composite<DT, BILINEAR, SAVE>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, s>>>(p, planes, count, ws, out, state);
    note_launches(1);
}

template <int DT, bool SAVE>
void launch_composite_t(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                        cudaStream_t s, float4* state)
{
    if (p.N <= 4096) {
        const bool ok = p.bilinear ? launch_staged<DT, true, SAVE>(p, planes, count, ws, out, s, state)
                                   : launch_staged<DT, false, SAVE>(p, planes, count, ws, out, s, state);
        if (ok) return;
    }
    if (p.bilinear)
        launch_unstaged<DT, true, SAVE>(p, planes, count, ws, out, s, state);
    else
        launch_unstaged<DT, false, SAVE>(p, planes, count, ws, out, s, state);
}

// ---------------------------------------------------------------------------
// Adjoint of the swizzle blending. For one view pixel the forward computes
// Q = sum_k T_k C_k, T_{k+1} = T_k (1 - A_k), output (Q + T_N bg, 1 - T_N).
// With upstream gradient g = (g_rgb, g_a):
//   dL/dC_k = T_k g_rgb,   dL/dA_k = -T_k B_k,
//   B_k = sum_{j>k} (prod_{k<l<j} (1 - A_l)) C_j . g_rgb + (prod_{l>k} (1 - A_l)) (g_rgb . bg - g_a),
//   B_{k-1} = C_k . g_rgb + (1 - A_k) B_k.
// B needs no transmittance; T_k is recovered back to front as
// T_{k+1} / (1 - A_k), carried as m 2^-e against underflow. A stored A_k
// can be exactly 1 (T_{k+1} = 0); the forward walk keeps T before the first
// such plane, and every plane behind it gets T = 0. The texel gradients are
// scattered with FP32 vector atomics into dplanes (nearest: the sampled
// texel; bilinear: the in-plane taps with their weights). The adjoint either
// recomputes the far-end transmittance with a front-to-back walk of its own,
// or starts from the 16 bytes per view pixel (m, e, first opaque plane) that
// the saving forward composite wrote, and walks the planes once.
// ---------------------------------------------------------------------------

// Views per thread of the staged adjoint, both forms. Started from the saved
// state, 9 views at one CTA per SM (no spills) measured 7 % slower than 3 at
// two (45 views of 512^2, N 64, FP32); 5 spills at the two-CTA cap.
constexpr int kBwdViews = 3;

// FS: the front-to-back walk is skipped and the pixel's transmittance taken
// from the state the saving forward wrote (as the staged adjoint's FS form).
template <int DT, bool BILINEAR, bool FS = false>
__global__ void __launch_bounds__(kCompBX* kCompBY) k_composite_bwd(CompParams p, const void* __restrict__ planes,
                                                                   const int32_t* __restrict__ count, CompWs w,
                                                                   const float4* __restrict__ dviews,
                                                                   float4* __restrict__ dplanes,
                                                                   const float4* __restrict__ state)
{
    extern __shared__ float s_coef[];  // as k_composite
    int* s_cnt = reinterpret_cast<int*>(s_coef + 6 * p.N);
    const int v = blockIdx.x;   // fastest: the views of one pixel tile share plane rows in L2
    const int i = v / p.Vx, j = v % p.Vx;
    const int tid = threadIdx.y * kCompBX + threadIdx.x;
    for (int k = tid; k < p.N; k += kCompBX * kCompBY) {
        const float* cx = w.cx + 3 * ((size_t)j * p.N + k);
        const float* cy = w.cy + 3 * ((size_t)i * p.N + k);
        s_coef[6 * k + 0] = cx[0];
        s_coef[6 * k + 1] = cx[1];
        s_coef[6 * k + 2] = cx[2];
        s_coef[6 * k + 3] = cy[0];
        s_coef[6 * k + 4] = cy[1];
        s_coef[6 * k + 5] = cy[2];
        s_cnt[k] = count[k];
    }
    __syncthreads();
    const int x = blockIdx.y * kCompBX + threadIdx.x;
    const int y = blockIdx.z * kCompBY + threadIdx.y;
    if (x >= p.Nx || y >= p.Ny) return;
    const size_t plane_sz = (size_t)p.W * p.H;

    // taps of plane k for this pixel: up to 4 (plane offset, weight)
    int tap[4];
    float wt[4];
    auto taps = [&](int k) -> int {
        const float* c = s_coef + 6 * k;
        int n = 0;
        if (!BILINEAR) {
            const int ix = nearest_index(p.P_s, x, c[0], c[1]);
            const int iy = nearest_index(p.P_s, y, c[3], c[4]);
            if (ix >= 0 && ix < p.W && iy >= 0 && iy < p.H) {
                tap[0] = iy * p.W + ix;
                wt[0] = 1.0f;
                n = 1;
            }
        } else {
            const float Dx = __fmaf_rn(c[0], (float)x, c[2]);
            const float Dy = __fmaf_rn(c[3], (float)y, c[5]);
            if (Dx >= -1.0e6f && Dx <= 1.0e6f && Dy >= -1.0e6f && Dy <= 1.0e6f) {
                const float flx = floorf(Dx), fly = floorf(Dy);
                const float wx = Dx - flx, wy = Dy - fly;
                const int x0 = p.P_s * x + (int)flx, y0 = p.P_s * y + (int)fly;
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int yy = y0 + dy;
                    if (yy < 0 || yy >= p.H) continue;
                    const float wyy = dy ? wy : 1.0f - wy;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int xx = x0 + dx;
                        if (xx < 0 || xx >= p.W) continue;
                        tap[n] = yy * p.W + xx;
                        wt[n] = wyy * (dx ? wx : 1.0f - wx);
                        ++n;
                    }
                }
            }
        }
        return n;
    };
    auto sample = [&](int k, int n) -> float4 {
        float4 tx = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < n; ++q) {
            const float4 t = load_texel<DT>(planes, (size_t)k * plane_sz + tap[q]);
            tx.x = fmaf(wt[q], t.x, tx.x);
            tx.y = fmaf(wt[q], t.y, tx.y);
            tx.z = fmaf(wt[q], t.z, tx.z);
            tx.w = fmaf(wt[q], t.w, tx.w);
        }
        return tx;
    };

    float Tm = 1.f, oTm = 0.f;
    int Te = 0, oTe = 0, ok = -1;
    if (FS) {
        // state {T_k, k}: T in front of plane k, 0 behind it; k = N: T
        // behind the last plane
        const float4 sv = state[((size_t)v * p.Ny + y) * p.Nx + x];
        const int kq = __float_as_int(sv.y);
        if (kq < p.N)
            Tm = 0.f, oTm = sv.x, ok = kq;
        else
            Tm = sv.x;
    }
    int nq = 0;   // non-empty planes so far (the forward's flush positions)
    for (int k = 0; k < (FS ? 0 : p.N); ++k) {
        if (s_cnt[k] == 0) continue;
        if ((nq & 3) == 0 && nq > 0 && ok < 0 && (Te == 0 ? Tm : ldexpf(Tm, -Te)) < kTFlush) {
            // the plain composite's flush: T is 0 from this plane on
            oTm = Tm;
            oTe = Te;
            ok = k;
            Tm = 0.0f;
        }
        ++nq;
        const float4 tx = sample(k, taps(k));
        const float oma = 1.0f - tx.w;
        if (!(oma > 0.0f) && Tm > 0.0f && ok < 0) {
            oTm = Tm;
            oTe = Te;
            ok = k;
        }
        Tm = Tm * oma;
        if (Tm < kDownB && Tm > 0.0f) {
            Tm *= kUpB;
            Te += 64;
        }
    }
    const float4 g = dviews[((size_t)v * p.Ny + y) * p.Nx + x];
    float B = fmaf(g.x, p.bg[0], fmaf(g.y, p.bg[1], fmaf(g.z, p.bg[2], -g.w)));
    for (int k = p.N - 1; k >= 0; --k) {
        if (s_cnt[k] == 0) continue;
        const int n = taps(k);
        const float4 tx = sample(k, n);
        const float oma = 1.0f - tx.w;
        if (k == ok) {
            Tm = oTm;
            Te = oTe;
        } else if (oma > 0.0f) {
            Tm = __fdiv_rn(Tm, oma);
            if (Te > 0 && Tm > kBigB) {
                Tm *= kDownB;
                Te -= 64;
            }
        }
        const float Tk = Te == 0 ? Tm : ldexpf(Tm, -Te);
        if (Tk > 0.0f) {
            const float4 gt = make_float4(Tk * g.x, Tk * g.y, Tk * g.z, -Tk * B);
            for (int q = 0; q < n; ++q)
                atomicAdd(dplanes + (size_t)k * plane_sz + tap[q],
                          make_float4(wt[q] * gt.x, wt[q] * gt.y, wt[q] * gt.z, wt[q] * gt.w));
        }
        B = fmaf(tx.x, g.x, fmaf(tx.y, g.y, fmaf(tx.z, g.z, oma * B)));
    }
}

// ---------------------------------------------------------------------------
// Staged adjoint: the forward staged layout (a CTA owns BY output rows x TX
// columns for VG views of one view row; one producer lane streams the plane
// rows those pixels sample into the shared-memory ring) run twice: the list
// of non-empty planes front to back to carry every view's transmittance to
// the far end (alpha only; T before its first opaque plane is noted), then
// back to front for the B recurrence, the T recovery by division and the
// texel gradients (FP32 vector atomics into dplanes, as the unstaged
// kernel). The row geometry of a plane is computed once per thread, the
// views' horizontal taps per view. The ring counts 2P planes; every wait is
// bounded, and a wait that gives up sets the error word and ends the walk.
// ---------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ float texel_alpha(uint32_t row, uint32_t i);
template <>
__device__ __forceinline__ float texel_alpha<LF_F32>(uint32_t row, uint32_t i)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(row + i * 16u + 12u));
    return v;
}
template <>
__device__ __forceinline__ float texel_alpha<LF_F16>(uint32_t row, uint32_t i)
{
    unsigned short h;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(row + i * 8u + 6u));
    return __half2float(__ushort_as_half(h));
}
template <>
__device__ __forceinline__ float texel_alpha<LF_BF16>(uint32_t row, uint32_t i)
{
    unsigned short h;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(row + i * 8u + 6u));
    return __uint_as_float((uint32_t)h << 16);
}
template <>
__device__ __forceinline__ float texel_alpha<LF_U8>(uint32_t row, uint32_t i)
{
    return u8_byte<3>(lds_u32(row + i * 4u)) * (1.0f / 255.0f);
}

// T = m 2^-e (e a multiple of 64): m, m 2^-64, or below 2^-96 (taken as 0)

// FS (from state): the front-to-back walk is skipped; each view pixel's
// transmittance behind the last plane, or in front of the first opaque one,
// comes from the state the saving forward composite wrote, and the ring
// carries only the back-to-front planes.
template <int DT, bool BILINEAR, int VG, bool FS = false>
__global__ void __launch_bounds__(kBwdBlock, VG > 5 ? 1 : 2) k_composite_bwd_staged(CompParams p, StagedGeom G,
                                                                            const char* __restrict__ planes,
                                                                            const int32_t* __restrict__ count,
                                                                            CompWs w,
                                                                            const float4* __restrict__ dviews,
                                                                            float4* __restrict__ dplanes,
                                                                            const float4* __restrict__ state)
{
    extern __shared__ __align__(128) unsigned char smem[];
    // [kStages][rows][row_bytes] | full[kStages] | empty[kStages] | coef [N][CW] | plist [N]
    constexpr int CW = CoefBlock<VG>::kFloats;
    constexpr int NC = 4 * ((VG + 3) / 4);
    using TX_ = Texel<DT>;
    unsigned char* stage_base = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * G.stage_bytes);
    uint64_t* empty = full + kStages;
    float* coef = reinterpret_cast<float*>(empty + kStages);
    int* plist = reinterpret_cast<int*>(coef + (size_t)p.N * CW);
    __shared__ int s_nplanes;

    const int tid = threadIdx.x, lane = tid & 31;
    const int nvg = G.groups_x * p.Vy;   // view groups, then column tiles (as the forward)
    const int vgroup = blockIdx.x % nvg;
    const int vi = vgroup / G.groups_x;
    const int j0 = (vgroup % G.groups_x) * VG;
    const int Y0 = blockIdx.y * G.BY;
    const int X0 = (blockIdx.x / nvg) * G.TX;
    const int tx = tid % G.TX, ty = tid / G.TX;
    const int x = X0 + tx, y = Y0 + ty;

    if (tid < 32) {
        const int n = plane_list(p, count, plist);
        if (tid == 0) s_nplanes = n;
    }
    __syncthreads();
    load_coefs<BILINEAR, VG>(p, w, plist, s_nplanes, vi, j0, coef);
    zero_pads<DT>(p, G, stage_base, G.stage_bytes, kStages);
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(smem_addr(&full[st]), 1);
            mbar_init(smem_addr(&empty[st]), kBwdWarps);
        }
        fence_proxy_async();
    }
    __syncthreads();
    const int P = s_nplanes;
    // walk step q < P visits list entry q, step q >= P list entry 2P - 1 - q;
    // step q uses ring position r = q - q0 (q0 = P when the first walk is
    // skipped)
    auto entry = [&](int q) { return q < P ? q : 2 * P - 1 - q; };
    const int q0 = FS ? P : 0;

    if (tid >= kBwdStagedThreads) {
        if (tid == kBwdStagedThreads) {
            for (int q = q0; q < 2 * P; ++q) {
                const int r = q - q0;
                const int st = r % kStages;
                if (r >= kStages &&
                    !mbar_wait_bounded(smem_addr(&empty[st]), (uint32_t)(((r / kStages) - 1) & 1))) {
                    atomicExch(w.err, 1);
                    break;
                }
                const int e = entry(q);
                produce_rows<DT>(p, G, planes, plist[e], coef + (size_t)e * CW, Y0,
                                 stage_base + (size_t)st * G.stage_bytes, smem_addr(&full[st]));
            }
        }
        return;
    }

    const bool live = ty < G.BY && x < p.Nx && y < p.Ny;
    const ThreadGeom tg = thread_geom(p, G, x, y, ty);
    const uint32_t stage_a = smem_addr(stage_base), coef_a = smem_addr(coef);
    const size_t plane_sz = (size_t)p.W * p.H;
    const uint32_t Wu = (uint32_t)p.W, padl = (uint32_t)G.padl;

    // per plane: the view offsets c[] and the vertical sample (nearest row
    // iy, or rows y0, y0 + 1 with weights w0, w1; a weight is 0 off the plane)
    auto load_c = [&](int e, float (&c)[NC]) {
#pragma unroll
        for (int m = 0; m < NC / 4; ++m) {
            const float4 v = lds_f4(coef_a + 4u * (uint32_t)(e * CW + 4 + 4 * m));
            c[4 * m + 0] = v.x;
            c[4 * m + 1] = v.y;
            c[4 * m + 2] = v.z;
            c[4 * m + 3] = v.w;
        }
    };
    // padded horizontal index (bits of the magic floor + base) and, for
    // bilinear, the fractional weight
    auto hindex = [&](float4 hdr, float cj, float& wx) -> int {
        float fx = __fmaf_rn(hdr.x, tg.xf, cj);
        if (__float_as_int(hdr.w)) fx = fminf(fmaxf(fx, -kClamp), kClamp);
        const float tm = __fadd_rd(fx, kMagic);
        wx = fx - (tm - kMagic);
        return __float_as_int(tm) + tg.base_x;
    };

    float Tm[VG], oTm[VG];
    int Te[VG], oTe[VG], okq[VG];
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) Tm[jj] = 1.f, oTm[jj] = 0.f, Te[jj] = 0, oTe[jj] = 0, okq[jj] = -1;
    if (FS && live) {
        // state {T_k, k}: T in front of plane k, 0 behind it (the saving
        // forward stopped there); k = N: T behind the last plane
#pragma unroll
        for (int jj = 0; jj < VG; ++jj) {
            if (j0 + jj >= p.Vx) break;
            const float4 sv = state[((size_t)(vi * p.Vx + j0 + jj) * p.Ny + y) * p.Nx + x];
            const int kq = __float_as_int(sv.y);
            if (kq < p.N)
                Tm[jj] = 0.f, oTm[jj] = sv.x, okq[jj] = kq;
            else
                Tm[jj] = sv.x;
        }
    }
    int q = q0;
    bool walk_done = false;   // two walks: every view of the warp has stopped (warp-uniform)
    // front to back: transmittance at the far end, and T before the first
    // opaque plane (alpha only). The plain composite's flush (flush_tiny) is
    // followed too: at the same list positions a view whose T has fallen
    // below 2^-24 stops there, as before an opaque plane, and a warp whose
    // views have all stopped walks no further
    for (; q < P; ++q) {
        const int st = q % kStages;   // q0 == 0 here
        if (!mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)((q / kStages) & 1))) {
            atomicExch(w.err, 1);
            return;
        }
        if ((q & 3) == 0 && q > 0 && !walk_done) {
            bool all = true;
#pragma unroll
            for (int jj = 0; jj < VG; ++jj) {
                if (okq[jj] < 0 && scaled_t(Tm[jj], Te[jj]) < kTFlush) {
                    oTm[jj] = Tm[jj];
                    oTe[jj] = Te[jj];
                    okq[jj] = q;
                    Tm[jj] = 0.0f;
                }
                all = all && (okq[jj] >= 0 || j0 + jj >= p.Vx);
            }
            walk_done = __all_sync(0xffffffffu, all || !live);
        }
        if (live && !walk_done) {
            const uint32_t sb = stage_a + (uint32_t)(st * G.stage_bytes) + tg.row0;
            const float4 hdr = lds_f4(coef_a + 4u * (uint32_t)(q * CW));
            float c[NC];
            load_c(q, c);
            float w0 = 0.f, w1 = 0.f;
            bool rv = false;
            if (!BILINEAR) {
                const int iy = tg.psy + (__float_as_int(floor_magic<true>(hdr.y, tg.yf, hdr.z)) - kMagicBits);
                rv = iy >= 0 && iy < tg.H;
            } else {
                float fy = fminf(fmaxf(__fmaf_rn(hdr.y, tg.yf, hdr.z), -kClamp), kClamp);
                const float ty_m = __fadd_rd(fy, kMagic);
                const float wy = fy - (ty_m - kMagic);
                const int y0 = tg.psy + (__float_as_int(ty_m) - kMagicBits);
                w0 = (y0 >= 0 && y0 < tg.H) ? 1.0f - wy : 0.0f;
                w1 = (y0 + 1 >= 0 && y0 + 1 < tg.H) ? wy : 0.0f;
            }
#pragma unroll
            for (int jj = 0; jj < VG; ++jj) {
                float wx;
                const int ip = hindex(hdr, c[jj], wx);
                float a = 0.0f;
                if (!BILINEAR) {
                    if (rv && (uint32_t)ip - padl < Wu) a = texel_alpha<DT>(sb, (uint32_t)ip);
                } else {
                    // vertical pair first, then the horizontal pair: the
                    // forward's rounding order (its blended rows)
                    const bool c0 = (uint32_t)ip - padl < Wu, c1 = (uint32_t)ip + 1u - padl < Wu;
                    const float wa = 1.0f - wx;
                    float u0 = 0.f, u1 = 0.f;
                    if (w0 != 0.0f) {
                        u0 = w0 * (c0 ? texel_alpha<DT>(sb, (uint32_t)ip) : 0.f);
                        u1 = w0 * (c1 ? texel_alpha<DT>(sb, (uint32_t)ip + 1u) : 0.f);
                    }
                    if (w1 != 0.0f) {
                        const uint32_t r1 = sb + tg.row_bytes;
                        u0 = fmaf(w1, c0 ? texel_alpha<DT>(r1, (uint32_t)ip) : 0.f, u0);
                        u1 = fmaf(w1, c1 ? texel_alpha<DT>(r1, (uint32_t)ip + 1u) : 0.f, u1);
                    }
                    a = fmaf(wa, u0, wx * u1);
                }
                const float oma = 1.0f - a;
                if (!(oma > 0.0f) && Tm[jj] > 0.0f && okq[jj] < 0) {
                    oTm[jj] = Tm[jj];
                    oTe[jj] = Te[jj];
                    okq[jj] = q;
                }
                Tm[jj] = Tm[jj] * oma;
                if (Tm[jj] < kDownB && Tm[jj] > 0.0f) {
                    Tm[jj] *= kUpB;
                    Te[jj] += 64;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
    }
    float4 g[VG];
    float B[VG];
#pragma unroll
    for (int jj = 0; jj < VG; ++jj) {
        const bool vv = live && j0 + jj < p.Vx;   // padding views of a ragged group get no gradient
        g[jj] = vv ? dviews[view_pixel(p, vi * p.Vx + j0 + jj, x, y)] : make_float4(0.f, 0.f, 0.f, 0.f);
        B[jj] = fmaf(g[jj].x, p.bg[0], fmaf(g[jj].y, p.bg[1], fmaf(g[jj].z, p.bg[2], -g[jj].w)));
    }
    // from the state: the planes behind the last stop plane of the warp's
    // views carry T = 0 for all of them, and their share of B is scaled by a
    // transmittance below the stop threshold; the warp walks from there
    // (two walks: the same for the list entries behind the last stop)
    int km = -1;
#pragma unroll
    for (int jj = 0; jj < VG; ++jj)
        if (live && j0 + jj < p.Vx) km = max(km, okq[jj] >= 0 ? okq[jj] : (FS ? p.N : P));
    const int kmax = __reduce_max_sync(0xffffffffu, km);
    // back to front: T recovered by division, texel gradients, B recurrence
    for (; q < 2 * P; ++q) {
        const int r = q - q0;
        const int st = r % kStages;
        if (!mbar_wait_bounded(smem_addr(&full[st]), (uint32_t)((r / kStages) & 1))) {
            atomicExch(w.err, 1);
            return;
        }
        if (live && (FS ? plist[entry(q)] : entry(q)) <= kmax) {
            const int e = entry(q);
            const uint32_t sb = stage_a + (uint32_t)(st * G.stage_bytes) + tg.row0;
            const float4 hdr = lds_f4(coef_a + 4u * (uint32_t)(e * CW));
            float c[NC];
            load_c(e, c);
            float4* dk = dplanes + (size_t)plist[e] * plane_sz;
            float w0 = 0.f, w1 = 0.f, wy = 0.f;
            bool rv = false;
            int yrow = 0;
            if (!BILINEAR) {
                yrow = tg.psy + (__float_as_int(floor_magic<true>(hdr.y, tg.yf, hdr.z)) - kMagicBits);
                rv = yrow >= 0 && yrow < tg.H;
            } else {
                float fy = fminf(fmaxf(__fmaf_rn(hdr.y, tg.yf, hdr.z), -kClamp), kClamp);
                const float ty_m = __fadd_rd(fy, kMagic);
                wy = fy - (ty_m - kMagic);
                yrow = tg.psy + (__float_as_int(ty_m) - kMagicBits);
                w0 = (yrow >= 0 && yrow < tg.H) ? 1.0f - wy : 0.0f;
                w1 = (yrow + 1 >= 0 && yrow + 1 < tg.H) ? wy : 0.0f;
            }
            float4* drow = dk + ((long long)yrow * p.W - (long long)padl);   // indexed by padded column
#pragma unroll
            for (int jj = 0; jj < VG; ++jj) {
                float wx;
                const int ip = hindex(hdr, c[jj], wx);
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                const bool c0 = (uint32_t)ip - padl < Wu;
                const bool c1 = BILINEAR && (uint32_t)ip + 1u - padl < Wu;
                const float wa = 1.0f - wx;
                if (!BILINEAR) {
                    if (rv && c0) t = TX_::load(sb, (uint32_t)ip);
                } else {
                    // vertical pairs first (u0 at column ip, u1 at ip + 1),
                    // then the horizontal pair: the forward's rounding order
                    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 u0 = z, u1 = z;
                    if (w0 != 0.0f) {
                        const float4 t0 = c0 ? TX_::load(sb, (uint32_t)ip) : z;
                        const float4 t1 = c1 ? TX_::load(sb, (uint32_t)ip + 1u) : z;
                        u0 = make_float4(w0 * t0.x, w0 * t0.y, w0 * t0.z, w0 * t0.w);
                        u1 = make_float4(w0 * t1.x, w0 * t1.y, w0 * t1.z, w0 * t1.w);
                    }
                    if (w1 != 0.0f) {
                        const uint32_t r1 = sb + tg.row_bytes;
                        const float4 t0 = c0 ? TX_::load(r1, (uint32_t)ip) : z;
                        const float4 t1 = c1 ? TX_::load(r1, (uint32_t)ip + 1u) : z;
                        u0 = make_float4(fmaf(w1, t0.x, u0.x), fmaf(w1, t0.y, u0.y), fmaf(w1, t0.z, u0.z),
                                         fmaf(w1, t0.w, u0.w));
                        u1 = make_float4(fmaf(w1, t1.x, u1.x), fmaf(w1, t1.y, u1.y), fmaf(w1, t1.z, u1.z),
                                         fmaf(w1, t1.w, u1.w));
                    }
                    t = make_float4(fmaf(wa, u0.x, wx * u1.x), fmaf(wa, u0.y, wx * u1.y), fmaf(wa, u0.z, wx * u1.z),
                                    fmaf(wa, u0.w, wx * u1.w));
                }
                const float oma = 1.0f - t.w;
                if constexpr (FS) {
                    // T in [2^-24, 1] from the stop plane on, 0 behind it: no scaling
                    if (plist[e] == okq[jj])
                        Tm[jj] = oTm[jj];
                    else if (oma > 0.0f)
                        Tm[jj] = __fdividef(Tm[jj], oma);
                } else {
                    if (e == okq[jj]) {
                        Tm[jj] = oTm[jj];
                        Te[jj] = oTe[jj];
                    } else if (oma > 0.0f) {
                        Tm[jj] = __fdividef(Tm[jj], oma);
                        if (Te[jj] > 0 && Tm[jj] > kBigB) {
                            Tm[jj] *= kDownB;
                            Te[jj] -= 64;
                        }
                    }
                }
                const float Tk = FS ? Tm[jj] : scaled_t(Tm[jj], Te[jj]);
                if (Tk > 0.0f) {
                    const float4 gt = make_float4(Tk * g[jj].x, Tk * g[jj].y, Tk * g[jj].z, -Tk * B[jj]);
                    if (!BILINEAR) {
                        if (rv && c0) atomicAdd(drow + ip, gt);
                    } else {
                        const float ww[4] = {w0 * wa, w0 * wx, w1 * wa, w1 * wx};
                        const bool ok4[4] = {w0 != 0.0f && c0, w0 != 0.0f && c1, w1 != 0.0f && c0, w1 != 0.0f && c1};
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            if (ok4[m])
                                atomicAdd(drow + (m >> 1) * p.W + ip + (m & 1),
                                          make_float4(ww[m] * gt.x, ww[m] * gt.y, ww[m] * gt.z, ww[m] * gt.w));
                    }
                }
                B[jj] = fmaf(t.x, g[jj].x, fmaf(t.y, g[jj].y, fmaf(t.z, g[jj].z, oma * B[jj])));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
    }
}

template <int DT, bool BILINEAR, int VG, bool FS = false>
bool launch_bwd_staged_vg(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                          const float4* dviews, float4* dplanes, cudaStream_t s, const float4* state = nullptr)
{
    constexpr int TB = Texel<DT>::kBytes;
    StagedGeom G = staged_geom(p, TB, BILINEAR, VG, 512, kBwdStagedThreads);
    // no blended rows here: the full ring
    G.blend_bytes = 0;
    G.stages = kStages;
    G.smem_bytes = kStages * G.stage_bytes + 2 * kStages * 8 + sizeof(float) * (size_t)p.N * CoefBlock<VG>::kFloats +
                   sizeof(int) * (size_t)p.N;
    if (G.smem_bytes > 200 * 1024) return false;
    if (((uintptr_t)planes) % 16 != 0 || ((size_t)p.W * TB) % 16 != 0) return false;
    auto kern = k_composite_bwd_staged<DT, BILINEAR, VG, FS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.smem_bytes) != cudaSuccess)
        return false;
    const dim3 grid((unsigned)(G.groups_x * p.Vy * ((p.Nx + G.TX - 1) / G.TX)), (unsigned)((p.Ny + G.BY - 1) / G.BY));
    kern<<<grid, kBwdBlock, G.smem_bytes, s>>>(p, G, static_cast<const char*>(planes), count, ws, dviews, dplanes,
                                                  state);
    note_launches(1);
    return true;
}

// Failure-detection self-test: one thread waits on an mbarrier of expected
// count 1 that nothing arrives on, with the wait limit given; the bounded
// wait gives up and the kernel records how (1: gave up, 2: the phase
// completed, which cannot happen) and exits normally.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* result)
{
    __shared__ uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);
    fence_proxy_async();
    *result = mbar_wait_for(b, 0u, limit_ns) ? 2 : 1;
}

template <int DT, bool FS>
void launch_composite_bwd_t(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                            const float* dviews, float* dplanes, cudaStream_t s, const float4* state)
{
    const dim3 block(kCompBX, kCompBY);
    const dim3 grid((unsigned)(p.Vx * p.Vy), (unsigned)((p.Nx + kCompBX - 1) / kCompBX),
                    (unsigned)((p.Ny + kCompBY - 1) / kCompBY));
    const size_t smem = sizeof(float) * 6 * p.N + sizeof(int) * p.N;
    const float4* dv = reinterpret_cast<const float4*>(dviews);
    float4* dp = reinterpret_cast<float4*>(dplanes);
    if (p.N <= 4096) {
        const bool ok = p.bilinear
                            ? launch_bwd_staged_vg<DT, true, kBwdViews, FS>(p, planes, count, ws, dv, dp, s, state)
                            : launch_bwd_staged_vg<DT, false, kBwdViews, FS>(p, planes, count, ws, dv, dp, s, state);
        if (ok) return;
    }
    auto kern = p.bilinear ? k_composite_bwd<DT, true, FS> : k_composite_bwd<DT, false, FS>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, s>>>(p, planes, count, ws, dv, dp, state);
    note_launches(1);
}

template <int DT, bool BILINEAR, int VG>
void launch_batched_t(const CompScene* scs, int n_sc, long long total, size_t max_stage_bytes, int maxN,
                      unsigned long long* counter, int n_ctas, size_t smem, cudaStream_t s)
{
    auto kern = k_composite_batched<DT, BILINEAR, VG>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<n_ctas, kStagedBlock, smem, s>>>(scs, n_sc, total, counter, max_stage_bytes, maxN);
}

template <int DT, bool BILINEAR>
void launch_batched_vg(int VG, const CompScene* scs, int n_sc, long long total, size_t mx, int maxN,
                       unsigned long long* counter, int n_ctas, size_t smem, cudaStream_t s)
{
    if (VG == 15)
        launch_batched_t<DT, BILINEAR, 15>(scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
    else if (VG == 9)
        launch_batched_t<DT, BILINEAR, 9>(scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
    else if (VG == 5)
        launch_batched_t<DT, BILINEAR, 5>(scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
    else
        launch_batched_t<DT, BILINEAR, 3>(scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
}

template <int DT>
void launch_batched_dt(bool bilinear, int VG, const CompScene* scs, int n_sc, long long total, size_t mx, int maxN,
                       unsigned long long* counter, int n_ctas, size_t smem, cudaStream_t s)
{
    if (bilinear)
        launch_batched_vg<DT, true>(VG, scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
    else
        launch_batched_vg<DT, false>(VG, scs, n_sc, total, mx, maxN, counter, n_ctas, smem, s);
}

}  // namespace

size_t composite_batched_smem(size_t max_stage_bytes, int maxN, int VG)
{
    return kStages * max_stage_bytes + 2 * kStages * 8 + sizeof(float) * (size_t)maxN * (4 + 4 * ((VG + 3) / 4)) +
           sizeof(int) * (size_t)maxN;
}

bool launch_composite_batched(const CompScene* scenes_dev, int n_sc, long long total, int dtype, bool bilinear,
                              int VG, size_t max_stage_bytes, int maxN, unsigned long long* counter, int n_ctas,
                              cudaStream_t s)
{
    if (total <= 0) return true;
    const size_t smem = composite_batched_smem(max_stage_bytes, maxN, VG);
    if (smem > 200 * 1024) return false;
    if (dtype == LF_U8)
        launch_batched_dt<LF_U8>(bilinear, VG, scenes_dev, n_sc, total, max_stage_bytes, maxN, counter, n_ctas, smem, s);
    else if (dtype == LF_F32)
        launch_batched_dt<LF_F32>(bilinear, VG, scenes_dev, n_sc, total, max_stage_bytes, maxN, counter, n_ctas, smem, s);
    else if (dtype == LF_F16)
        launch_batched_dt<LF_F16>(bilinear, VG, scenes_dev, n_sc, total, max_stage_bytes, maxN, counter, n_ctas, smem, s);
    else
        launch_batched_dt<LF_BF16>(bilinear, VG, scenes_dev, n_sc, total, max_stage_bytes, maxN, counter, n_ctas, smem,
                                   s);
    note_launches(1);
    return true;
}

namespace {

// Composition of a batch scene's chunk groups, front to back (the "over"
// operator is associative): Q = Q_0 + T_0 Q_1 + T_0 T_1 Q_2 ..., T = T_0 T_1
// ...; then the views (Q + T bg, 1 - T).
__global__ void k_merge_chunk_groups(CompParams p, int groups, const float4* __restrict__ part, float* out)
{
    const long long per = (long long)p.Nx * p.Ny;
    const long long total = per * p.Vx * p.Vy;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(e / per);
        const long long pix = e - (long long)v * per;
        const int y = (int)(pix / p.Nx), x = (int)(pix - (long long)y * p.Nx);
        float4* dst = reinterpret_cast<float4*>(out) + view_pixel(p, v, x, y);
        float4 a = *dst;
        for (int c = 1; c < groups; ++c) {
            const float4 b = __ldcs(part + ((size_t)(c - 1) * p.Vx * p.Vy * per + e));
            a.x = fmaf(a.w, b.x, a.x);
            a.y = fmaf(a.w, b.y, a.y);
            a.z = fmaf(a.w, b.z, a.z);
            a.w *= b.w;
        }
        *dst = make_float4(fmaf(a.w, p.bg[0], a.x), fmaf(a.w, p.bg[1], a.y), fmaf(a.w, p.bg[2], a.z), 1.0f - a.w);
    }
}

}  // namespace

void launch_merge_chunk_groups(const CompParams& p, int groups, const float4* part, float* out, cudaStream_t s)
{
    const long long total = (long long)p.Nx * p.Ny * p.Vx * p.Vy;
    const long long want = (total + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 32 ? want : 152 * 32);
    k_merge_chunk_groups<<<blocks, 256, 0, s>>>(p, groups, part, out);
    note_launches(1);
}

void launch_wait_selftest(unsigned long long limit_ns, int* result, cudaStream_t s)
{
    k_wait_selftest<<<1, 1, 0, s>>>(limit_ns, result);
    note_launches(1);
}

template <bool FS>
void launch_composite_bwd_dt(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                             const float* dviews, float* dplanes, const float4* state, cudaStream_t s)
{
    switch (p.dtype) {
    case LF_F32: launch_composite_bwd_t<LF_F32, FS>(p, planes, count, ws, dviews, dplanes, s, state); break;
    case LF_F16: launch_composite_bwd_t<LF_F16, FS>(p, planes, count, ws, dviews, dplanes, s, state); break;
    case LF_U8: launch_composite_bwd_t<LF_U8, FS>(p, planes, count, ws, dviews, dplanes, s, state); break;
    default: launch_composite_bwd_t<LF_BF16, FS>(p, planes, count, ws, dviews, dplanes, s, state); break;
    }
}

void launch_composite_bwd(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                          const float* dviews, float* dplanes, cudaStream_t s, const float4* state)
{
    if (state)
        launch_composite_bwd_dt<true>(p, planes, count, ws, dviews, dplanes, state, s);
    else
        launch_composite_bwd_dt<false>(p, planes, count, ws, dviews, dplanes, nullptr, s);
}

void launch_comp_coeffs(const CompParams& p, const double* d, const int32_t* count, const CompWs& ws, cudaStream_t s)
{
    const int n = (p.Vx + p.Vy) * p.N;
    k_comp_coeffs<<<(n + 127) / 128, 128, 0, s>>>(p, d, count, ws);
    note_launches(1);
}

template <bool SAVE>
void launch_composite_dt(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                         float4* state, cudaStream_t s)
{
    switch (p.dtype) {
    case LF_F32: launch_composite_t<LF_F32, SAVE>(p, planes, count, ws, out, s, state); break;
    case LF_F16: launch_composite_t<LF_F16, SAVE>(p, planes, count, ws, out, s, state); break;
    case LF_U8: launch_composite_t<LF_U8, SAVE>(p, planes, count, ws, out, s, state); break;
    default: launch_composite_t<LF_BF16, SAVE>(p, planes, count, ws, out, s, state); break;
    }
}

void launch_composite(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                      cudaStream_t s, float4* state)
{
    if (state)
        launch_composite_dt<true>(p, planes, count, ws, out, state, s);
    else
        launch_composite_dt<false>(p, planes, count, ws, out, nullptr, s);
}

}  // namespace lf
