/*
 * lf_oracle.h -- FP64 CPU oracle for the G2LF / V2LF hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path. Only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
 * may load it. It shares no code, header, table or constant with the CUDA
 * library under paper_2508_18540_gb300/.
 *
 * Paper: "Real-time 3D Visualization of Radiance Fields on Light Field
 * Displays" (arXiv 2508.18540), Sec. 4.
 *
 * Conventions (readings of the paper, all restated where used):
 *  - Camera frame: +x right, +y down, +z forward. The base camera maps world
 *    points p to R p + t. The reference camera is the base camera moved by
 *    D_forward along its +z axis (Sec. 4.2), so reference depth = base depth
 *    - D_forward.
 *  - Reference image W x H = (P_s Nx) x (P_s Ny) (Sec. 4.2). Pixel i has its
 *    centre at plane coordinate i, normalised coordinate (2i+1)/W - 1.
 *  - Planes are stored RGBA: premultiplied colour C and A = 1 - T.
 *  - Everything is FP64 except the few integer decisions that the kernel
 *    takes in FP32 (footprint rectangles, nearest-texel indices); those are
 *    written here in FP32 in a fixed operation order so that both sides take
 *    the same decision.
 */
#ifndef LF_ORACLE_H
#define LF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double R[9];      /* world -> base camera rotation, row-major */
    double t[3];      /* world -> base camera translation */
    double theta_x;   /* base camera horizontal field of view (radians) */
    double theta_y;   /* base camera vertical field of view (radians) */
    int32_t Nx, Ny;   /* per-view resolution of the quilt */
} orc_camera;

typedef struct {
    double D_focal;   /* camera-to-focal-plane distance */
    double phi_x;     /* display viewing angle, horizontal (radians) */
    double phi_y;     /* display viewing angle, vertical (radians) */
    double D_shift;   /* backward shift of the reference camera */
    int32_t P_s;      /* plane resolution scale (positive integer) */
    double f_aa;      /* 3DGS screen-space dilation f (0.3 px^2) */
    double z_near;    /* near clip in reference depth */
} orc_display;

typedef struct {
    orc_camera cam;
    orc_display disp;
    double tth_x, tth_y;     /* tan(theta/2) */
    double tphi_x, tphi_y;   /* tan(phi/2) */
    double D_forward0;       /* Eq. (1) before the near-field shift */
    double D_forward;        /* D_forward0 - D_shift */
    double tthp_x, tthp_y;   /* tan(theta'/2), Eq. (2) */
    double theta_px, theta_py;
    double fx, fy, cx, cy;   /* reference intrinsics in plane pixels */
    double f_prime;          /* adaptive dilation, Eq. (gs_prefilter_fix) */
    int32_t W, H;            /* plane resolution */
} orc_ref;

/* Sec. 4.2: reference camera. Returns 0, or -1 for invalid input. */
int orc_make_ref(const orc_camera* cam, const orc_display* disp, orc_ref* out);

/* Sec. 4.3: lateral offsets Delta x_j (Vx values) and Delta y_i (Vy values). */
void orc_view_offsets(const orc_ref* r, int32_t Vx, int32_t Vy, double* dx, double* dy);

/* Sec. 4.3, Eq. (u_prime): plane coordinate u' (axis 0) or v' (axis 1). */
double orc_plane_coord(const orc_ref* r, int32_t axis, double delta, double d_k, double u);

/* Plane-pixel coordinate X = ((u'+1) W - 1)/2 straight from Eq. (u_prime). */
double orc_plane_pixel(const orc_ref* r, int32_t axis, double delta, double d_k, int32_t x);

/* FP32 decision form of the same map: X = P_s x + (gm x + hb) and
 * X + 1/2 = P_s x + (gm x + hn), coefficients computed in FP64 in a fixed
 * order and rounded once to FP32. */
void orc_axis_coeffs(const orc_ref* r, int32_t axis, double delta, double d_k,
                     float* gm, float* hn, float* hb);

/* Nearest plane index for output pixel x: P_s x + floor(fmaf(gm, x, hn)). */
int32_t orc_nearest_index(const orc_ref* r, float gm, float hn, int32_t x);

/* Per-Gaussian decision data (FP64 depth, FP32 rectangle).
 * z[n]: reference depth (FP64, fixed fma order), valid[n]: 1 if culled in,
 * rect[n][4] = {x0, y0, x1, y1} inclusive plane-pixel bounds. */
void orc_gauss_decide(const orc_ref* r, int64_t n, const float* means, const float* scales,
                      const float* quats, double* z, uint8_t* valid, int32_t* rect);

/* Per-Gaussian FP64 values: mean2d[n][2] (plane pixels), conic[n][3] =
 * inverse 2D covariance {a, b, c}. Uses the EWA splatting projection.
 * Parameters are FP64 (finite differences perturb them below FP32 spacing). */
void orc_gauss_values(const orc_ref* r, int64_t n, const double* means, const double* scales,
                      const double* quats, double* mean2d, double* conic, double* cov2d);

/* Per-voxel decision data. Voxel v is the axis-aligned cube with low corner
 * origin + ijk * s and side s = base_size * 2^-level. */
void orc_voxel_decide(const orc_ref* r, int64_t n, const int32_t* ijk, const uint8_t* level,
                      const double* origin, double base_size,
                      double* z, uint8_t* valid, int32_t* rect);

/* Sec. 4.4 binning. mode 0 = quantile, 1 = uniform in disparity.
 * order[0..M) = culled-in primitive indices sorted by (z, index);
 * chunk[n] = chunk of each primitive (-1 if culled);
 * d[N] = plane distance in the BASE camera frame; count[N] = members.
 * Returns M. */
int64_t orc_bin(const orc_ref* r, int64_t n, const double* z, const uint8_t* valid,
                int32_t N, int32_t mode, int64_t* order, int32_t* chunk, double* d,
                int64_t* count);

/* Sec. 4.4: rasterise every chunk into its plane. planes[N][H][W][4] FP64. */
void orc_splat_gaussians(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                         const int32_t* rect, const double* mean2d, const double* conic,
                         const double* opacity, const double* rgb, int32_t N, double* planes);

/* Sec. 4.4 with the two cut-offs of the 3DGS rasteriser the chunks are
 * rendered with: a member whose alpha is below 1/255 is skipped, and a pixel
 * stops before the member whose blend would take T (1 - alpha) below 1e-4
 * (that member and all later ones are left out). near[N][H][W] (may be NULL)
 * is set to 1 where the pixel's trace, up to its stop, meets an alpha within
 * 1e-6 of 1/255 or a T (1 - alpha) within 1e-6 of 1e-4: a decision another
 * precision may take the other way. */
void orc_splat_gaussians_3dgs(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                              const int32_t* rect, const double* mean2d, const double* conic,
                              const double* opacity, const double* rgb, int32_t N, double* planes,
                              uint8_t* near);

/* Sec. 4.5: rasterise voxels (ray-segment integral of trilinear density). */
void orc_splat_voxels(const orc_ref* r, int64_t M, const int64_t* order, const int32_t* chunk,
                      const int32_t* rect, const int32_t* ijk, const uint8_t* level,
                      const double* origin, double base_size, const double* density8,
                      const double* rgb, int32_t N, double* planes);

/* Opacity of one voxel along one reference ray (exposed for pins):
 * ray origin o[3] and unit direction dir[3] in world coordinates. */
double orc_voxel_alpha(const double* lo, double side, const double* density8,
                       const double* o, const double* dir, double* seg_len);

/* Sec. 4.5 low-pass plane filter (V2LF): normalised discrete Gaussian
 * weights w[2 radius + 1] for offsets -radius..radius. */
void orc_filter_weights(double sigma, int32_t radius, double* w);

/* Separable filter of every RGBA channel of planes[N][H][W][4] (rows, then
 * columns), zero padding outside the plane; in place. */
void orc_filter_planes(double* planes, int32_t N, int32_t H, int32_t W, double sigma, int32_t radius);

/* Sec. 4.3 swizzle blending, Algorithm 1 second loop.
 * views[Vy*Vx][Ny][Nx][4] = (Q + T bg, 1 - T); view index i*Vx + j. */
void orc_composite(const orc_ref* r, int32_t N, const double* planes, const double* d,
                   const int64_t* count, int32_t Vx, int32_t Vy, int32_t bilinear,
                   const double* bg, double* views);

/* Threads the oracle's OpenMP loops run on (omp_get_max_threads). */
int orc_num_threads(void);

/* Sets that thread count (n <= 0: one per processor). */
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif

#endif
