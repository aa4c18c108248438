// lf_composite.cu -- swizzle blending of the sweeping planes into the quilt
// views (Sec. 4.3; Algorithm 1 lines 6-11).
//
// k_comp_coeffs evaluates, per (view column j, plane k) and (view row i,
// plane k), the affine form of Eq. (u_prime) in plane pixels,
//   X(x) = P_s x + (gm x + hb),  X(x) + 1/2 = P_s x + (gm x + hn),
// from the FP64 display set-up (Delta x_j = 2 D_focal s_j tan(phi_x/2),
// den = (d_k - D_forward) tan(theta'/2), a = d_k tan(theta/2),
// g = W a / (Nx den), h = (W/2)((Delta (D_focal - d_k)/D_focal + a (1-Nx)/Nx)/den + 1) - 1/2,
// gm = g - P_s), rounded once to FP32.
// k_composite walks the planes front to back for every view pixel:
// nearest texel index P_s x + floor(fma(gm, x, hn)) (FP32 decision), or
// bilinear taps around X with zero padding; Q += T c_k, T *= 1 - A_k
// (Eq. (alpha_blend)); empty planes skipped; output (Q + T bg, 1 - T).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lf_internal.cuh"

namespace lf {

namespace {

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
    if (along_x)
        axis_coeffs(view_offset(v, p.Vx, p.D_focal, p.tphi_x), d[k], p.D_focal, p.D_forward, p.tth_x, p.tthp_x, p.Nx,
                    p.W, p.P_s, out);
    else
        axis_coeffs(view_offset(v, p.Vy, p.D_focal, p.tphi_y), d[k], p.D_focal, p.D_forward, p.tth_y, p.tthp_y, p.Ny,
                    p.H, p.P_s, out);
}

template <int DT>
__device__ __forceinline__ float4 load_texel(const void* planes, size_t idx)
{
    if (DT == LF_F32) {
        return __ldg(reinterpret_cast<const float4*>(planes) + idx);
    } else {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(planes) + idx);
        if (DT == LF_F16) {
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
            return make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// plane index of the nearest texel, or -1 when the FP32 result is far outside
__device__ __forceinline__ int nearest_index(int P_s, int x, float gm, float hn)
{
    const float f = floorf(__fmaf_rn(gm, (float)x, hn));
    if (!(f >= -1.0e6f && f <= 1.0e6f)) return -1;
    return P_s * x + (int)f;
}

constexpr int kCompBX = 32, kCompBY = 8;

template <int DT, bool BILINEAR>
__global__ void __launch_bounds__(kCompBX* kCompBY) k_composite(CompParams p, const void* __restrict__ planes,
                                                               const int32_t* __restrict__ count, CompWs w,
                                                               float* __restrict__ out)
{
    extern __shared__ float s_coef[];  // [N][6]: x (gm, hn, hb), y (gm, hn, hb); count in [N] ints after
    int* s_cnt = reinterpret_cast<int*>(s_coef + 6 * p.N);
    const int v = blockIdx.z;
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
    const int x = blockIdx.x * kCompBX + threadIdx.x;
    const int y = blockIdx.y * kCompBY + threadIdx.y;
    if (x >= p.Nx || y >= p.Ny) return;
    const size_t plane_sz = (size_t)p.W * p.H;
    float Q0 = 0.f, Q1 = 0.f, Q2 = 0.f, T = 1.f;
    for (int k = 0; k < p.N; ++k) {
        if (s_cnt[k] == 0) continue;
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
        Q0 = fmaf(T, tx.x, Q0);
        Q1 = fmaf(T, tx.y, Q1);
        Q2 = fmaf(T, tx.z, Q2);
        T = T * (1.0f - tx.w);
    }
    reinterpret_cast<float4*>(out)[((size_t)v * p.Ny + y) * p.Nx + x] =
        make_float4(fmaf(T, p.bg[0], Q0), fmaf(T, p.bg[1], Q1), fmaf(T, p.bg[2], Q2), 1.0f - T);
}

template <int DT>
void launch_composite_t(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                        cudaStream_t s)
{
    const dim3 block(kCompBX, kCompBY);
    const dim3 grid((unsigned)((p.Nx + kCompBX - 1) / kCompBX), (unsigned)((p.Ny + kCompBY - 1) / kCompBY),
                    (unsigned)(p.Vx * p.Vy));
    const size_t smem = sizeof(float) * 6 * p.N + sizeof(int) * p.N;
    if (p.bilinear) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_composite<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_composite<DT, true><<<grid, block, smem, s>>>(p, planes, count, ws, out);
        note_launches(1);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_composite<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_composite<DT, false><<<grid, block, smem, s>>>(p, planes, count, ws, out);
        note_launches(1);
    }
}

}  // namespace

void launch_comp_coeffs(const CompParams& p, const double* d, const int32_t* count, const CompWs& ws, cudaStream_t s)
{
    const int n = (p.Vx + p.Vy) * p.N;
    k_comp_coeffs<<<(n + 127) / 128, 128, 0, s>>>(p, d, count, ws);
    note_launches(1);
}

void launch_composite(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws, float* out,
                      cudaStream_t s)
{
    switch (p.dtype) {
    case LF_F32: launch_composite_t<LF_F32>(p, planes, count, ws, out, s); break;
    case LF_F16: launch_composite_t<LF_F16>(p, planes, count, ws, out, s); break;
    default: launch_composite_t<LF_BF16>(p, planes, count, ws, out, s); break;
    }
}

}  // namespace lf
