// lf_project.cu -- per-primitive projection and culling (Algorithm 1 line 1,
// "CulledDepth"), for 3D Gaussians (Sec. 4.4) and sparse voxels (Sec. 4.5).
//
// Decisions that fix integers are taken in a prescribed precision and
// operation order, with explicit round-to-nearest intrinsics so that the
// compiler cannot contract or reorder them:
//  - reference depth z: FP64, fma(R20, x, fma(R21, y, fma(R22, z, t2))) - D_forward;
//  - Gaussian footprint: FP32, the 3-sigma square r = ceil(3 sqrt(lambda_max))
//    of the EWA 2D covariance J W Sigma_3 W^T J^T + f' I (3DGS projection with
//    the dilation f' of Eq. (gs_prefilter_fix)), clipped to the plane;
//  - voxel footprint: FP32 bounding box of the 8 projected corners.
#include "lf_internal.cuh"

namespace lf {

__global__ void k_init_header(WsHeader h, WsHeader* d) { *d = h; }

void launch_init_header(const WsHeader& h, WsHeader* d, cudaStream_t s)
{
    k_init_header<<<1, 1, 0, s>>>(h, d);
    note_launches(1);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Publishes the depth key range and culled-in count of one warp.
__device__ __forceinline__ void publish_key(WsHeader* hdr, unsigned long long key)
{
    const bool valid = key != kInvalidKey;
    const unsigned ballot = __ballot_sync(0xffffffffu, valid);
    const unsigned long long mn = warp_min_u64(valid ? key : ~0ull);
    const unsigned long long mx = warp_max_u64(valid ? key : 0ull);
    if ((threadIdx.x & 31) == 0 && ballot) {
        atomicAdd(&hdr->M, (unsigned long long)__popc(ballot));
        atomicMin(&hdr->kmin, mn);
        atomicMax(&hdr->kmax, mx);
    }
}

__device__ __forceinline__ double ref_depth(const ProjParams& p, double x, double y, double z)
{
    return __dsub_rn(__fma_rn(p.R[6], x, __fma_rn(p.R[7], y, __fma_rn(p.R[8], z, p.t[2]))), p.D_forward);
}

// FP32 footprint of one Gaussian (operation order fixed; see file header).
// Returns false if culled. Also returns the FP32 2D mean and conic.
__device__ __forceinline__ bool gauss_footprint(const ProjParams& p, float m0, float m1, float m2, float s0, float s1,
                                                float s2, float4 q, double z64, int4& rect, float2& mean,
                                                float4& conic)
{
    const float* R = p.Rf;
    const float xc = __fmaf_rn(R[0], m0, __fmaf_rn(R[1], m1, __fmaf_rn(R[2], m2, p.t0f)));
    const float yc = __fmaf_rn(R[3], m0, __fmaf_rn(R[4], m1, __fmaf_rn(R[5], m2, p.t1f)));
    const float zc = __double2float_rn(z64);

    const float n2 = __fmaf_rn(q.x, q.x, __fmaf_rn(q.y, q.y, __fmaf_rn(q.z, q.z, __fmul_rn(q.w, q.w))));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    const float w = __fmul_rn(q.x, inv), x = __fmul_rn(q.y, inv), y = __fmul_rn(q.z, inv), z = __fmul_rn(q.w, inv);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float Q[9];
    Q[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    Q[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    Q[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    Q[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    Q[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    Q[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    Q[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    Q[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    Q[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
    const float s[3] = {s0, s1, s2};
    float M[9], V[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) M[3 * i + l] = __fmul_rn(Q[3 * i + l], s[l]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            V[3 * i + l] = __fmaf_rn(R[3 * i + 0], M[l],
                                     __fmaf_rn(R[3 * i + 1], M[3 + l], __fmul_rn(R[3 * i + 2], M[6 + l])));

    const float iz = __fdiv_rn(1.0f, zc);
    const float xn = __fmul_rn(xc, iz), yn = __fmul_rn(yc, iz);
    const float ax = __fmul_rn(p.fxf, iz), ay = __fmul_rn(p.fyf, iz);
    float U0[3], U1[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        U0[l] = __fmul_rn(ax, __fmaf_rn(-xn, V[6 + l], V[0 + l]));
        U1[l] = __fmul_rn(ay, __fmaf_rn(-yn, V[6 + l], V[3 + l]));
    }
    const float S00 = __fadd_rn(__fmaf_rn(U0[0], U0[0], __fmaf_rn(U0[1], U0[1], __fmul_rn(U0[2], U0[2]))), p.fpf);
    const float S01 = __fmaf_rn(U0[0], U1[0], __fmaf_rn(U0[1], U1[1], __fmul_rn(U0[2], U1[2])));
    const float S11 = __fadd_rn(__fmaf_rn(U1[0], U1[0], __fmaf_rn(U1[1], U1[1], __fmul_rn(U1[2], U1[2]))), p.fpf);
    const float det = __fmaf_rn(S00, S11, -__fmul_rn(S01, S01));
    if (!(det > 0.0f)) return false;
    const float mid = __fmul_rn(0.5f, __fadd_rn(S00, S11));
    const float lam = __fadd_rn(mid, __fsqrt_rn(fmaxf(__fmaf_rn(mid, mid, -det), 0.0f)));
    const float rad = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
    const float px = __fmaf_rn(p.fxf, xn, p.cxf);
    const float py = __fmaf_rn(p.fyf, yn, p.cyf);
    const float fx0 = ceilf(__fsub_rn(px, rad)), fx1 = floorf(__fadd_rn(px, rad));
    const float fy0 = ceilf(__fsub_rn(py, rad)), fy1 = floorf(__fadd_rn(py, rad));
    if (!(fx0 <= p.wmax && fx1 >= 0.0f && fy0 <= p.hmax && fy1 >= 0.0f)) return false;
    rect.x = (int)fmaxf(fx0, 0.0f);
    rect.y = (int)fmaxf(fy0, 0.0f);
    rect.z = (int)fminf(fx1, p.wmax);
    rect.w = (int)fminf(fy1, p.hmax);
    mean = make_float2(px, py);
    const float idet = 1.0f / det;
    conic = make_float4(S11 * idet, -S01 * idet, S00 * idet, 0.0f);
    return true;
}

__global__ void __launch_bounds__(256) k_project_gaussians(lf_gaussians g, ProjParams p, BuildWs w, int4* rect_out,
                                                           int32_t* chunk_out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kInvalidKey;
    if (i < p.n) {
        const float m0 = g.means[3 * i + 0], m1 = g.means[3 * i + 1], m2 = g.means[3 * i + 2];
        const double z = ref_depth(p, (double)m0, (double)m1, (double)m2);
        int4 rect = make_int4(0, 0, -1, -1);
        chunk_out[i] = -1;
        if (z > p.z_near) {
            const float4 q = *reinterpret_cast<const float4*>(g.quats + 4 * i);
            float2 mean;
            float4 conic;
            if (gauss_footprint(p, m0, m1, m2, g.scales[3 * i + 0], g.scales[3 * i + 1], g.scales[3 * i + 2], q, z,
                                rect, mean, conic)) {
                key = (unsigned long long)__double_as_longlong(z);
                conic.w = g.opacity[i];
                w.mean2d[i] = mean;
                w.conic_o[i] = conic;
            } else {
                rect = make_int4(0, 0, -1, -1);
            }
        }
        rect_out[i] = rect;
        w.keyA[i] = key;
        w.valA[i] = (uint32_t)i;
    }
    publish_key(w.hdr, key);
}

// Voxel v: cube of side s = base_size 2^-level with low corner origin + ijk s.
// Depth = centre depth; culled unless the nearest corner lies past z_near;
// footprint = bounding box of the 8 projected corners (pixel centres inside).
__global__ void __launch_bounds__(256) k_project_voxels(lf_voxels v, ProjParams p, BuildWs w, int4* rect_out,
                                                        int32_t* chunk_out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kInvalidKey;
    if (i < p.n) {
        double s = p.base_size;
        for (int l = 0; l < (int)v.level[i]; ++l) s = __dmul_rn(s, 0.5);
        double lo[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = __dadd_rn(p.origin[a], __dmul_rn((double)v.ijk[3 * i + a], s));
        const double hs = __dmul_rn(0.5, s);
        const double z = ref_depth(p, __dadd_rn(lo[0], hs), __dadd_rn(lo[1], hs), __dadd_rn(lo[2], hs));
        const double zmin = __dsub_rn(z, __dmul_rn(hs, p.rho));
        int4 rect = make_int4(0, 0, -1, -1);
        chunk_out[i] = -1;
        if (zmin > p.z_near) {
            const float* R = p.Rf;
            float mnx = __int_as_float(0x7f800000), mny = mnx;
            float mxx = -mnx, mxy = -mnx;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float X = __double2float_rn(__dadd_rn(lo[0], __dmul_rn((double)(c & 1), s)));
                const float Y = __double2float_rn(__dadd_rn(lo[1], __dmul_rn((double)((c >> 1) & 1), s)));
                const float Z = __double2float_rn(__dadd_rn(lo[2], __dmul_rn((double)((c >> 2) & 1), s)));
                const float xc = __fmaf_rn(R[0], X, __fmaf_rn(R[1], Y, __fmaf_rn(R[2], Z, p.t0f)));
                const float yc = __fmaf_rn(R[3], X, __fmaf_rn(R[4], Y, __fmaf_rn(R[5], Z, p.t1f)));
                const float zc = __fmaf_rn(R[6], X, __fmaf_rn(R[7], Y, __fmaf_rn(R[8], Z, p.t2rf)));
                const float iz = __fdiv_rn(1.0f, zc);
                const float px = __fmaf_rn(p.fxf, __fmul_rn(xc, iz), p.cxf);
                const float py = __fmaf_rn(p.fyf, __fmul_rn(yc, iz), p.cyf);
                mnx = fminf(mnx, px);
                mxx = fmaxf(mxx, px);
                mny = fminf(mny, py);
                mxy = fmaxf(mxy, py);
            }
            const float fx0 = ceilf(mnx), fx1 = floorf(mxx);
            const float fy0 = ceilf(mny), fy1 = floorf(mxy);
            if ((fx0 <= fx1 && fy0 <= fy1) && (fx0 <= p.wmax && fx1 >= 0.0f && fy0 <= p.hmax && fy1 >= 0.0f)) {
                rect.x = (int)fmaxf(fx0, 0.0f);
                rect.y = (int)fmaxf(fy0, 0.0f);
                rect.z = (int)fminf(fx1, p.wmax);
                rect.w = (int)fminf(fy1, p.hmax);
                key = (unsigned long long)__double_as_longlong(z);
                // cube relative to the reference centre, for the ray integrals
                w.conic_o[i] = make_float4(__double2float_rn(__dsub_rn(lo[0], p.cam_o[0])),
                                           __double2float_rn(__dsub_rn(lo[1], p.cam_o[1])),
                                           __double2float_rn(__dsub_rn(lo[2], p.cam_o[2])), __double2float_rn(s));
            }
        }
        rect_out[i] = rect;
        w.keyA[i] = key;
        w.valA[i] = (uint32_t)i;
    }
    publish_key(w.hdr, key);
}

void launch_project_gaussians(const lf_gaussians& g, const ProjParams& p, const BuildWs& ws, int32_t* rect,
                              int32_t* chunk, cudaStream_t s)
{
    if (p.n <= 0) return;
    const unsigned blocks = (unsigned)((p.n + 255) / 256);
    k_project_gaussians<<<blocks, 256, 0, s>>>(g, p, ws, reinterpret_cast<int4*>(rect), chunk);
    note_launches(1);
}

void launch_project_voxels(const lf_voxels& v, const ProjParams& p, const BuildWs& ws, int32_t* rect, int32_t* chunk,
                           cudaStream_t s)
{
    if (p.n <= 0) return;
    const unsigned blocks = (unsigned)((p.n + 255) / 256);
    k_project_voxels<<<blocks, 256, 0, s>>>(v, p, ws, reinterpret_cast<int4*>(rect), chunk);
    note_launches(1);
}

}  // namespace lf
