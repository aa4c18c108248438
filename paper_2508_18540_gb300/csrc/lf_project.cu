// lf_project.cu -- per-primitive projection and culling (the first step of
// Algorithm 1), for 3D Gaussians (Sec. 4.4) and sparse voxels (Sec. 4.5).
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

__global__ void k_init_header(WsHeader h, WsHeader* d)
{
    pdl_wait();
    pdl_trigger();
    *d = h;
}

void launch_init_header(const WsHeader& h, WsHeader* d, cudaStream_t s)
{
    launch_pdl(k_init_header, dim3(1), dim3(1), 0, s, h, d);
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

constexpr int kProjThreads = 256;
constexpr int kProjItems = 4;   // primitives per thread (block-strided)

// Culled-in count and depth key range of the primitives one thread projected.
struct KeyStats {
    unsigned long long n = 0, mn = ~0ull, mx = 0ull;
    __device__ __forceinline__ void add(unsigned long long key)
    {
        if (key == kInvalidKey) return;
        ++n;
        mn = key < mn ? key : mn;
        mx = key > mx ? key : mx;
    }
};

// Publishes the statistics of one CTA with one atomic of each kind (the
// header words are shared by the whole grid, so per-warp atomics serialise).
__device__ __forceinline__ void publish_keys(WsHeader* hdr, KeyStats s)
{
    __shared__ unsigned long long sh[3][kProjThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s.n += __shfl_xor_sync(0xffffffffu, s.n, o);
    s.mn = warp_min_u64(s.mn);
    s.mx = warp_max_u64(s.mx);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[0][wid] = s.n, sh[1][wid] = s.mn, sh[2][wid] = s.mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kProjThreads / 32; ++k) {
            s.n += sh[0][k];
            s.mn = sh[1][k] < s.mn ? sh[1][k] : s.mn;
            s.mx = sh[2][k] > s.mx ? sh[2][k] : s.mx;
        }
        if (s.n) {
            atomicAdd(&hdr->M, s.n);
            atomicMin(&hdr->kmin, s.mn);
            atomicMax(&hdr->kmax, s.mx);
        }
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

__global__ void __launch_bounds__(kProjThreads) k_project_gaussians(lf_gaussians g, ProjParams p, BuildWs w,
                                                                    int4* rect_out, int32_t* chunk_out)
{
    pdl_wait();
    pdl_trigger();
    KeyStats st;
    for (int it = 0; it < kProjItems; ++it) {
        const long long i = ((long long)blockIdx.x * kProjItems + it) * kProjThreads + threadIdx.x;
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
        st.add(key);
    }
    publish_keys(w.hdr, st);
}

// Voxel v: cube of side s = base_size 2^-level with low corner origin + ijk s.
// Depth = centre depth; culled unless the nearest corner lies past z_near;
// footprint = bounding box of the 8 projected corners (pixel centres inside).
__global__ void __launch_bounds__(kProjThreads) k_project_voxels(lf_voxels v, ProjParams p, BuildWs w,
                                                                 int4* rect_out, int32_t* chunk_out)
{
    pdl_wait();
    pdl_trigger();
    KeyStats st;
    for (int it = 0; it < kProjItems; ++it) {
        const long long i = ((long long)blockIdx.x * kProjItems + it) * kProjThreads + threadIdx.x;
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
                // coordinate a of corner c is FP32(lo[a] + bit * s) with bit 0 or 1,
                // i.e. FP32(lo[a]) or FP32(lo[a] + s): two values per axis
                float cw[3][2];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cw[a][0] = __double2float_rn(lo[a]);
                    cw[a][1] = __double2float_rn(__dadd_rn(lo[a], s));
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float X = cw[0][c & 1];
                    const float Y = cw[1][(c >> 1) & 1];
                    const float Z = cw[2][(c >> 2) & 1];
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
        st.add(key);
    }
    publish_keys(w.hdr, st);
}

// ---------------------------------------------------------------------------
// Backward of the per-Gaussian projection (chain rule of the EWA splatting
// model, 3DGS, with the dilation f' of Eq. (gs_prefilter_fix)). Input per
// rank: gradients of the 2D mean (px, py), of the conic scalars (a, b, c)
// with q = a dx^2 + 2 b dx dy + c dy^2, of the opacity and of the colour,
// accumulated by the raster backward. Output per Gaussian index: gradients
// of means, scales, raw quaternions (through the normalisation), opacity and
// colour. Forward (FP32, as in the projection above):
//   (x, y, z) = R m + t - D_forward e_z, q^ = q / |q|, Q = rot(q^),
//   V = R Q diag(s), U0 = (fx/z) (V_0 - (x/z) V_2), U1 = (fy/z) (V_1 - (y/z) V_2),
//   S00 = U0.U0 + f', S01 = U0.U1, S11 = U1.U1 + f', det = S00 S11 - S01^2,
//   (a, b, c) = (S11, -S01, S00) / det,  px = fx x/z + cx, py = fy y/z + cy.
// The conic adjoint is G_S = -K G_K K with K the conic matrix and G_K =
// [[ga, gb/2], [gb/2, gc]] (b sits twice in the symmetric matrix).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gauss_chain(lf_gaussians g, ProjParams p, BuildWs w, lf_gaussians_grad out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w.hdr->overflow || r >= (long long)w.hdr->M) return;
    const uint32_t i = w.valA[r];
    const float4 a0 = reinterpret_cast<const float4*>(w.g2d)[3 * r];
    const float4 a1 = reinterpret_cast<const float4*>(w.g2d)[3 * r + 1];
    const float4 a2 = reinterpret_cast<const float4*>(w.g2d)[3 * r + 2];
    const float gpx = a0.x, gpy = a0.y, ga = a0.z, gb = a0.w, gc = a1.x;
    out.dopacity[i] = a1.y;
    out.drgb[3 * (size_t)i + 0] = a1.z;
    out.drgb[3 * (size_t)i + 1] = a1.w;
    out.drgb[3 * (size_t)i + 2] = a2.x;

    const float* R = p.Rf;
    const float m0 = g.means[3 * (size_t)i], m1 = g.means[3 * (size_t)i + 1], m2 = g.means[3 * (size_t)i + 2];
    const float xc = fmaf(R[0], m0, fmaf(R[1], m1, fmaf(R[2], m2, p.t0f)));
    const float yc = fmaf(R[3], m0, fmaf(R[4], m1, fmaf(R[5], m2, p.t1f)));
    const float zc = __double2float_rn(ref_depth(p, (double)m0, (double)m1, (double)m2));
    const float q[4] = {g.quats[4 * (size_t)i], g.quats[4 * (size_t)i + 1], g.quats[4 * (size_t)i + 2],
                        g.quats[4 * (size_t)i + 3]};
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float iqn = 1.0f / qn;
    const float qw = q[0] * iqn, qx = q[1] * iqn, qy = q[2] * iqn, qz = q[3] * iqn;
    float Q[9];
    Q[0] = 1.f - 2.f * (qy * qy + qz * qz);
    Q[1] = 2.f * (qx * qy - qw * qz);
    Q[2] = 2.f * (qx * qz + qw * qy);
    Q[3] = 2.f * (qx * qy + qw * qz);
    Q[4] = 1.f - 2.f * (qx * qx + qz * qz);
    Q[5] = 2.f * (qy * qz - qw * qx);
    Q[6] = 2.f * (qx * qz - qw * qy);
    Q[7] = 2.f * (qy * qz + qw * qx);
    Q[8] = 1.f - 2.f * (qx * qx + qy * qy);
    const float sc[3] = {g.scales[3 * (size_t)i], g.scales[3 * (size_t)i + 1], g.scales[3 * (size_t)i + 2]};
    float M[9], V[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int l = 0; l < 3; ++l) M[3 * a + l] = Q[3 * a + l] * sc[l];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int l = 0; l < 3; ++l) V[3 * a + l] = R[3 * a] * M[l] + R[3 * a + 1] * M[3 + l] + R[3 * a + 2] * M[6 + l];
    const float iz = 1.0f / zc;
    const float xn = xc * iz, yn = yc * iz, ax = p.fxf * iz, ay = p.fyf * iz;
    float U0[3], U1[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        U0[l] = ax * (V[l] - xn * V[6 + l]);
        U1[l] = ay * (V[3 + l] - yn * V[6 + l]);
    }
    const float S00 = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2] + p.fpf;
    const float S01 = U0[0] * U1[0] + U0[1] * U1[1] + U0[2] * U1[2];
    const float S11 = U1[0] * U1[0] + U1[1] * U1[1] + U1[2] * U1[2] + p.fpf;
    const float idet = 1.0f / (S00 * S11 - S01 * S01);
    const float Ka = S11 * idet, Kb = -S01 * idet, Kc = S00 * idet;
    // G_S = -K G_K K
    const float P00 = ga * Ka + 0.5f * gb * Kb, P01 = ga * Kb + 0.5f * gb * Kc;
    const float P10 = 0.5f * gb * Ka + gc * Kb, P11 = 0.5f * gb * Kb + gc * Kc;
    const float gS00 = -(Ka * P00 + Kb * P10);
    const float gS11 = -(Kb * P01 + Kc * P11);
    const float gS01 = -2.0f * (Ka * P01 + Kb * P11);
    // S = U U^T + f' I
    float gU0[3], gU1[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        gU0[l] = 2.0f * gS00 * U0[l] + gS01 * U1[l];
        gU1[l] = 2.0f * gS11 * U1[l] + gS01 * U0[l];
    }
    // U0 = ax (V_0 - xn V_2), U1 = ay (V_1 - yn V_2)
    float gV[9];
    float g_ax = 0.f, g_ay = 0.f, g_xn = p.fxf * gpx, g_yn = p.fyf * gpy;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        gV[l] = ax * gU0[l];
        gV[3 + l] = ay * gU1[l];
        gV[6 + l] = -ax * xn * gU0[l] - ay * yn * gU1[l];
        g_ax += gU0[l] * (V[l] - xn * V[6 + l]);
        g_ay += gU1[l] * (V[3 + l] - yn * V[6 + l]);
        g_xn -= ax * V[6 + l] * gU0[l];
        g_yn -= ay * V[6 + l] * gU1[l];
    }
    const float g_xc = g_xn * iz, g_yc = g_yn * iz;
    const float g_iz = g_xn * xc + g_yn * yc + g_ax * p.fxf + g_ay * p.fyf;
    const float g_zc = -g_iz * iz * iz;
    // m: camera point = R m + t
#pragma unroll
    for (int a = 0; a < 3; ++a)
        out.dmeans[3 * (size_t)i + a] = R[a] * g_xc + R[3 + a] * g_yc + R[6 + a] * g_zc;
    // V = R M -> gM = R^T gV; M = Q diag(s)
    float gQ[9];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        float gs = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float gM = R[a] * gV[l] + R[3 + a] * gV[3 + l] + R[6 + a] * gV[6 + l];
            gs += gM * Q[3 * a + l];
            gQ[3 * a + l] = gM * sc[l];
        }
        out.dscales[3 * (size_t)i + l] = gs;
    }
    // rotation matrix of the unit quaternion (w, x, y, z)
    const float gw = 2.f * (-qz * gQ[1] + qy * gQ[2] + qz * gQ[3] - qx * gQ[5] - qy * gQ[6] + qx * gQ[7]);
    const float gx = 2.f * (qy * gQ[1] + qz * gQ[2] + qy * gQ[3] - 2.f * qx * gQ[4] - qw * gQ[5] + qz * gQ[6] +
                            qw * gQ[7] - 2.f * qx * gQ[8]);
    const float gy = 2.f * (-2.f * qy * gQ[0] + qx * gQ[1] + qw * gQ[2] + qx * gQ[3] + qz * gQ[5] - qw * gQ[6] +
                            qz * gQ[7] - 2.f * qy * gQ[8]);
    const float gz = 2.f * (-2.f * qz * gQ[0] - qw * gQ[1] + qx * gQ[2] + qw * gQ[3] - 2.f * qz * gQ[4] +
                            qy * gQ[5] + qx * gQ[6] + qy * gQ[7]);
    // through q^ = q / |q|
    const float dot = gw * qw + gx * qx + gy * qy + gz * qz;
    out.dquats[4 * (size_t)i + 0] = (gw - qw * dot) * iqn;
    out.dquats[4 * (size_t)i + 1] = (gx - qx * dot) * iqn;
    out.dquats[4 * (size_t)i + 2] = (gy - qy * dot) * iqn;
    out.dquats[4 * (size_t)i + 3] = (gz - qz * dot) * iqn;
}

// Voxels: the accumulators are already the parameter gradients; scatter
// them from rank order to primitive order.
__global__ void __launch_bounds__(256) k_voxel_scatter(BuildWs w, lf_voxels_grad out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w.hdr->overflow || r >= (long long)w.hdr->M) return;
    const uint32_t i = w.valA[r];
    const float4* a = reinterpret_cast<const float4*>(w.g2d) + 3 * r;
    const float4 a0 = a[0], a1 = a[1], a2 = a[2];
    float* dd = out.ddensity8 + 8 * (size_t)i;
    dd[0] = a0.x; dd[1] = a0.y; dd[2] = a0.z; dd[3] = a0.w;
    dd[4] = a1.x; dd[5] = a1.y; dd[6] = a1.z; dd[7] = a1.w;
    out.drgb[3 * (size_t)i + 0] = a2.x;
    out.drgb[3 * (size_t)i + 1] = a2.y;
    out.drgb[3 * (size_t)i + 2] = a2.z;
}

void launch_gauss_chain(const lf_gaussians& g, const ProjParams& p, const BuildWs& ws, const lf_gaussians_grad& out,
                        cudaStream_t s)
{
    if (p.n <= 0) return;
    k_gauss_chain<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(g, p, ws, out);
    note_launches(1);
}

void launch_voxel_scatter(const BuildWs& ws, long long n, const lf_voxels_grad& out, cudaStream_t s)
{
    if (n <= 0) return;
    k_voxel_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ws, out);
    note_launches(1);
}

void launch_project_gaussians(const lf_gaussians& g, const ProjParams& p, const BuildWs& ws, int32_t* rect,
                              int32_t* chunk, cudaStream_t s)
{
    if (p.n <= 0) return;
    const long long per = (long long)kProjThreads * kProjItems;
    const unsigned blocks = (unsigned)((p.n + per - 1) / per);
    launch_pdl(k_project_gaussians, dim3(blocks), dim3(kProjThreads), 0, s, g, p, ws, reinterpret_cast<int4*>(rect), chunk);
    note_launches(1);
}

void launch_project_voxels(const lf_voxels& v, const ProjParams& p, const BuildWs& ws, int32_t* rect, int32_t* chunk,
                           cudaStream_t s)
{
    if (p.n <= 0) return;
    const long long per = (long long)kProjThreads * kProjItems;
    const unsigned blocks = (unsigned)((p.n + per - 1) / per);
    launch_pdl(k_project_voxels, dim3(blocks), dim3(kProjThreads), 0, s, v, p, ws, reinterpret_cast<int4*>(rect), chunk);
    note_launches(1);
}

}  // namespace lf
