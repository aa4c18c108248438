/*
 * lf.h -- C ABI of the GB300 (sm_103a) G2LF / V2LF library (liblf.so).
 *
 * Implements the hot path of "Real-time 3D Visualization of Radiance Fields
 * on Light Field Displays" (arXiv 2508.18540): a radiance field (3D Gaussians
 * with DC colour, or sparse voxels) is splatted once into N_chunk
 * depth-binned RGBA sweeping planes seen from a reference camera
 * (Sec. 4.2, 4.4, 4.5; the plane-building steps of Algorithm 1), and the planes are composited
 * into every light-field view in one pass ("swizzle blending", Sec. 4.3,
 * Eq. (u_prime), Eq. (alpha_blend); the compositing steps of Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Camera frame: +x right, +y down, +z forward. The base camera maps a world
 *    point p to R p + t. The reference camera is the base camera moved
 *    D_forward along +z (Sec. 4.2).
 *  - Planes are W x H = (P_s Nx) x (P_s Ny) (Sec. 4.2); texel (x, y) has its
 *    centre at normalised coordinate ((2x+1)/W - 1, (2y+1)/H - 1).
 *  - Every texel and view pixel is RGBA: premultiplied colour, A = 1 - T.
 *  - Memory: every pointer documented "device" is caller-owned device memory
 *    on the current CUDA device; "host" pointers are caller-owned host memory.
 *    The library allocates nothing: scratch lives in a caller-provided
 *    workspace whose size is returned by the matching *_workspace_size call.
 *  - Streams: compute entry points enqueue work on the given stream and return
 *    without synchronising. Their argument checks happen on the host before
 *    anything is enqueued. Data-dependent failures (tile-list overflow) are
 *    recorded in the workspace and read back with lf_mpi_status().
 *  - Errors: every call returns an lf_status; lf_last_error() gives a
 *    thread-local message for the last failing call on this thread.
 */
#ifndef LF_H
#define LF_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LF_OK = 0,
    LF_ERR_INVALID_ARG = 1,   /* bad pointer, size, layout or parameter */
    LF_ERR_WORKSPACE = 2,     /* workspace missing or too small */
    LF_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has it) */
    LF_ERR_OVERFLOW = 4,      /* tile list larger than the workspace capacity */
    LF_ERR_UNSUPPORTED = 5,   /* valid request the library does not implement */
    LF_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} lf_status;

/* Plane storage types. LF_U8 is RGBA8 unorm: every channel (premultiplied
 * colour, A) clamped to [0, 1] and stored as round(255 v), read back as
 * byte / 255 (the paper's default plane format). Accumulation is FP32. */
typedef enum { LF_F32 = 0, LF_F16 = 1, LF_BF16 = 2, LF_U8 = 3 } lf_dtype;

typedef enum {
    LF_BIN_QUANTILE = 0,      /* Sec. 4.4: equal-count chunks, d_k = median depth */
    LF_BIN_DISPARITY = 1      /* N equal bins in 1/z between nearest and farthest */
} lf_binning;

/* Blending flag, OR'd into the binning argument of lf_build_mpi_gaussians.
 * Without it ("exact" mode, the default) every chunk member whose footprint
 * rectangle holds the pixel is blended. LF_BLEND_3DGS adds the two cut-offs
 * of the 3DGS rasteriser that Sec. 4.4 renders each chunk with: a member
 * whose alpha is below 1/255 is skipped, and a pixel stops before the member
 * that would take its transmittance T (1 - alpha) below 1e-4 (that member
 * and every later one are left out). Gaussians only: the voxel build and the
 * batch reject it (LF_ERR_UNSUPPORTED), and the adjoint differentiates exact
 * mode. */
enum { LF_BLEND_3DGS = 0x100 };

/* Base camera (Sec. 4.2): world -> camera R (row-major), t; full fields of
 * view theta_x, theta_y in radians; per-view resolution Nx x Ny. */
typedef struct {
    double R[9];
    double t[3];
    double theta_x, theta_y;
    int32_t Nx, Ny;
} lf_camera;

/* Display set-up (Sec. 4.2, 4.3): focal distance D_focal, viewing angles
 * phi_x, phi_y (radians), backward shift D_shift, plane resolution scale P_s
 * (positive integer), 3DGS dilation f (f_aa, 0.3 px^2 in 3DGS), near clip
 * z_near (> 0) on reference depth. */
typedef struct {
    double D_focal, phi_x, phi_y, D_shift;
    int32_t P_s;
    double f_aa, z_near;
} lf_display;

/* Reference camera, filled by lf_make_ref_camera (all FP64):
 *  tth = tan(theta/2), tphi = tan(phi/2);
 *  D_forward0 = Eq. (1); D_forward = D_forward0 - D_shift;
 *  tthp = tan(theta'/2) from Eq. (2) with D_forward0; theta_p = theta';
 *  fx = W / (2 tthp_x), cx = (W - 1)/2 (plane pixels), same for y;
 *  f_prime = Eq. (gs_prefilter_fix) with the shifted D_forward. */
typedef struct {
    lf_camera base;
    lf_display disp;
    double tth_x, tth_y, tphi_x, tphi_y;
    double D_forward0, D_forward;
    double tthp_x, tthp_y, theta_px, theta_py;
    double fx, fy, cx, cy;
    double f_prime;
    int32_t W, H;
} lf_ref_camera;

/* 3D Gaussians, structure of arrays, device, FP32, activated values:
 * means [n][3], scales [n][3] (standard deviations), quats [n][4] (w, x, y, z;
 * normalised inside), opacity [n] in (0, 1), rgb [n][3] (DC colour). */
typedef struct {
    int64_t n;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacity;
    const float* rgb;
} lf_gaussians;

/* Sparse voxels (Sec. 4.5): voxel v is the axis-aligned cube with low corner
 * origin + ijk[v] * s_v and side s_v = base_size * 2^-level[v].
 * ijk [n][3] int32, level [n] uint8, density8 [n][8] FP32 (activated,
 * corner c = i + 2j + 4k at offset (i, j, k)), rgb [n][3] FP32; device. */
typedef struct {
    int64_t n;
    const int32_t* ijk;
    const uint8_t* level;
    double origin[3];
    double base_size;
    const float* density8;
    const float* rgb;
} lf_voxels;

/* Gradients with respect to the Gaussian parameters (device FP32, caller
 * allocated, layouts of lf_gaussians): dmeans [n][3], dscales [n][3],
 * dquats [n][4] (raw quaternion, through the normalisation), dopacity [n],
 * drgb [n][3]. */
typedef struct {
    float* dmeans;
    float* dscales;
    float* dquats;
    float* dopacity;
    float* drgb;
} lf_gaussians_grad;

/* Gradients with respect to the voxel parameters (device FP32, caller
 * allocated): ddensity8 [n][8], drgb [n][3]. */
typedef struct {
    float* ddensity8;
    float* drgb;
} lf_voxels_grad;

/* Sweeping planes (Sec. 4.2 C and T), caller-allocated device memory:
 *  rgba  [N][H][W][4] of dtype (premultiplied RGB, A = 1 - T);
 *  d     [N] FP64 plane distances in the base camera frame (0 if empty);
 *  count [N] int32 members per chunk;
 *  chunk [n] int32 chunk of every primitive (-1 = culled);
 *  rect  [n][4] int32 inclusive footprint {x0, y0, x1, y1} ({0,0,-1,-1} if culled).
 * N, H, W, dtype describe rgba; H, W must equal the reference camera's. */
typedef struct {
    int32_t N, H, W;
    int32_t dtype;
    void* rgba;
    double* d;
    int32_t* count;
    int32_t* chunk;
    int32_t* rect;
} lf_planes;

/* Quilt views (Sec. 4.3): Vx x Vy views, view index i * Vx + j; nearest
 * (bilinear = 0, the paper's default) or bilinear sampling; background
 * colour bg under the remaining transmittance (0 in the paper).
 * Output layout: atlas_cols = 0 gives separate views [V][Ny][Nx][4];
 * atlas_cols = c > 0 gives one quilt atlas image [ceil(V/c) Ny][c Nx][4]
 * with view v in tile (row v / c, column v % c), rows from the top (tiles
 * past V are left untouched). The adjoint takes separate views only. */
typedef struct {
    int32_t Vx, Vy;
    int32_t bilinear;
    float bg[3];
    int32_t atlas_cols;
} lf_view_set;

/* ---- set-up ------------------------------------------------------------ */

/* Sec. 4.2 Eqs. (1)-(2), the D_shift update and Eq. (gs_prefilter_fix).
 * cam, disp, out: host. Fails with LF_ERR_INVALID_ARG for non-positive sizes,
 * fields of view outside (0, pi), D_focal or z_near <= 0, P_s < 1, or a
 * shift that leaves D_forward >= D_focal. */
lf_status lf_make_ref_camera(const lf_camera* cam, const lf_display* disp, lf_ref_camera* out);

/* ---- splat: radiance field -> sweeping planes (Algorithm 1, plane building) --- */

/* Workspace bytes for lf_build_mpi_* on n primitives into N planes of the
 * reference camera ref, with room for dup_capacity (primitive, 32x32
 * super-tile) pairs (0 = 8 n + 2^20). */
size_t lf_build_mpi_workspace_size(const lf_ref_camera* ref, int64_t n, int32_t N, int64_t dup_capacity);

/* Sec. 4.4 (G2LF). Culls Gaussians to the reference frustum (reference depth
 * > z_near, non-empty footprint), sorts them by (FP64 depth, index), bins
 * them (quantile: chunk = floor(rank N / M), d_k = median depth; disparity:
 * equal bins in 1/z), and rasterises each chunk into its plane with the EWA
 * projection of 3DGS plus the dilation f' (alpha = min(0.99, o e^{-q/2}),
 * front to back, no early stop unless binning carries LF_BLEND_3DGS). All
 * planes are written (empty ones with 0).
 * g: host struct of device pointers; ref, out: host structs; ws: device
 * workspace of ws_bytes; stream: the CUDA stream to enqueue on.
 * Errors: LF_ERR_INVALID_ARG (null pointer, N < 1 or > 65535, plane size not
 * the reference camera's, unknown dtype, binning or flag), LF_ERR_WORKSPACE,
 * LF_ERR_CUDA (launch failure). Tile-list overflow is reported by
 * lf_mpi_status after the stream has run. */
lf_status lf_build_mpi_gaussians(const lf_gaussians* g, const lf_ref_camera* ref, int32_t N, int32_t binning,
                                 void* ws, size_t ws_bytes, lf_planes* out, cudaStream_t stream);

/* Sec. 4.5 (V2LF). Same pipeline for sparse voxels: depth = cube centre,
 * culled unless the whole cube lies past z_near; footprint = bounding box of
 * the 8 projected corners; alpha = 1 - exp(-integral of the trilinear
 * density over the pixel's reference-ray segment in the cube) (exact
 * Simpson rule). Arguments and errors as lf_build_mpi_gaussians, except that
 * a binning carrying LF_BLEND_3DGS fails with LF_ERR_UNSUPPORTED. */
lf_status lf_build_mpi_voxels(const lf_voxels* v, const lf_ref_camera* ref, int32_t N, int32_t binning,
                              void* ws, size_t ws_bytes, lf_planes* out, cudaStream_t stream);

/* Synchronises with the stream the last build on ws was enqueued on and
 * returns LF_ERR_OVERFLOW if its tile list exceeded the capacity (the planes
 * are then all zero); *needed (host, may be NULL) receives the pair count
 * and *culled_in (host, may be NULL) the number M of primitives kept. */
lf_status lf_mpi_status(const void* ws, int64_t* needed, int64_t* culled_in);

/* Copies the build's depth order and its 16x16 tile lists out of ws
 * (synchronous; for tests and inspection). order [n] int32 (host): primitive
 * index of ranks 0..M-1. tile_prims [cap] int32 (host): for every tile
 * (row-major over ceil(W/16) x ceil(H/16)) and chunk, the primitives of that
 * chunk whose footprint meets the tile, in depth order; seg [tiles * N][2]
 * int32 (host): [start, end) of list (tile, chunk) at index tile * N + chunk;
 * *n_pairs (host): total entries. Any output may be NULL. Fails with
 * LF_ERR_INVALID_ARG if cap is smaller than the entry count, LF_ERR_OVERFLOW
 * after an overflowed build. */
lf_status lf_mpi_tile_lists(const void* ws, int32_t* order, int64_t n, int32_t* tile_prims, int64_t cap,
                            int32_t* seg, int64_t* n_pairs);

/* Sec. 4.5 low-pass plane filter of V2LF (it replaces SVR's supersampling):
 * every RGBA channel of every plane is filtered in place with a separable,
 * normalised discrete Gaussian of standard deviation sigma (plane pixels)
 * over offsets -radius..radius (radius <= 0: ceil(3 sigma)), rows then
 * columns, transparent zero padding outside the plane, FP32 arithmetic.
 * Allocates nothing. Weights are computed on the host in FP64 and rounded
 * to FP32. Errors: LF_ERR_INVALID_ARG (sigma <= 0, radius > 16, bad planes). */
lf_status lf_filter_planes(const lf_planes* planes, double sigma, int32_t radius, cudaStream_t stream);

/* ---- composite: planes -> quilt views (Algorithm 1, compositing) --------- */

/* Workspace bytes for lf_composite / lf_composite_backward. */
size_t lf_composite_workspace_size(int32_t N, const lf_view_set* views);

/* Sec. 4.3 swizzle blending. For every view (i, j) and pixel (x, y), planes
 * are visited front to back; plane k is sampled at the Eq. (u_prime)
 * position X = ((u'+1) W - 1)/2 (nearest: floor(X + 1/2); bilinear with
 * transparent zero padding), and composited Q += T c_k, T *= 1 - A_k
 * (Eq. (alpha_blend)); empty planes (count 0) are skipped. Output
 * views [Vy*Vx][Ny][Nx][4] FP32 device = (Q + T bg, 1 - T).
 * The nearest index is decided in FP32 from per-(view, plane) coefficients
 * computed in FP64 (same decision as the CPU reference).
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_WORKSPACE, LF_ERR_CUDA. */
lf_status lf_composite(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views, float* out,
                       void* ws, size_t ws_bytes, cudaStream_t stream);

/* Synchronises stream and reads the error word that lf_composite /
 * lf_composite_backward keep in the composite workspace cws (laid out for N
 * and views): LF_ERR_TIMEOUT if a bounded wait of the last such call on cws
 * gave up (its views or dplanes are then not valid), else LF_OK. */
lf_status lf_composite_status(int32_t N, const lf_view_set* views, const void* cws, cudaStream_t stream);

/* Allocation-free form of lf_composite (the paper has no counterpart): the
 * same kernels and the same result, with the composite scratch (coefficient
 * tables and the error word) in a static device array of
 * lf_composite_noalloc_max_bytes() bytes (1 MiB) inside the library instead
 * of a caller workspace. It is for callers that cannot hand the library device
 * memory, for example a display runtime's per-frame present callback, which
 * runs where calling a device allocator is not allowed (it may synchronise
 * the device or stall the frame). Every GPU that loads the library holds the
 * array until the process exits. Each call looks up the array's device
 * address on the calling thread's current device (cudaGetSymbolAddress, no
 * allocation); the first call on a device may load the library's device code
 * there, so make it before any stream capture. Requests whose scratch
 * (lf_composite_workspace_size) exceeds the limit fail with LF_ERR_WORKSPACE
 * and a message, before any device work. Every call shares the one array and
 * it keeps the last call's contents (the error word is cleared by each
 * call): calls that overlap on the GPU race, so the caller must serialise
 * them. A bounded device wait that gives up is reported by
 * lf_composite_noalloc_status, not by this call. Other arguments and
 * argument errors as lf_composite. */
lf_status lf_composite_noalloc(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                               float* out, cudaStream_t stream);

/* Size in bytes of lf_composite_noalloc's static scratch. */
size_t lf_composite_noalloc_max_bytes(void);

/* Status of the last lf_composite_noalloc for N planes and views, read from
 * the static scratch after synchronising stream (the paper has no
 * counterpart): LF_ERR_TIMEOUT if one of its bounded device waits gave up
 * (its views are then not valid), else LF_OK. LF_ERR_INVALID_ARG for a
 * request lf_composite_noalloc would refuse. */
lf_status lf_composite_noalloc_status(int32_t N, const lf_view_set* views, cudaStream_t stream);

/* ---- differentiation ------------------------------------------------------ */
/*
 * Reverse-mode adjoints of the two stages, for fitting a scene against
 * target light-field views. The integer structure of the forward pass
 * (culling, chunk membership, plane depths d_k, footprint rectangles, tile
 * lists, nearest indices) is held fixed: it is piecewise constant in the
 * parameters and receives no gradient. The composite adjoint either
 * recomputes each view pixel's transmittance with a front-to-back walk of
 * its own (lf_composite_backward), or starts from 16 bytes per view pixel
 * that the saving forward (lf_composite_save) wrote and walks the planes
 * once (lf_composite_backward_saved). The clamp
 * alpha = min(0.99, .) passes no gradient where it is active. Gradients are
 * accumulated in FP32 with atomics, so their last bits depend on scheduling.
 */

/* Adjoint of lf_composite: given dviews = dL/d(views) [Vy*Vx][Ny][Nx][4]
 * FP32 device, writes dplanes = dL/d(planes.rgba) [N][H][W][4] FP32 device
 * (overwritten, whatever the plane dtype). planes, ref, views are those of
 * the forward call; planes->rgba must still hold the forward's planes.
 * ws: a composite workspace (lf_composite_workspace_size). Errors as
 * lf_composite. */
lf_status lf_composite_backward(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                                const float* dviews, float* dplanes, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Bytes of the saved composite state for these views of ref's output
 * resolution (ref->base.Nx x ref->base.Ny): 16 per view pixel,
 * Vy*Vx*Ny*Nx*16 (0 for a NULL argument or an empty view set). */
size_t lf_composite_state_size(const lf_ref_camera* ref, const lf_view_set* views);

/* lf_composite (Sec. 4.3, Eq. alpha_blend) in its saving form: each view
 * pixel's walk stops at the first plane k behind which T would fall below
 * 2^-24 (to 0 behind a plane with A = 1); plane k still blends, the colour
 * of the planes behind it (below 2^-24 each) is dropped and the output's
 * T is 0. Otherwise the same views as lf_composite. Per view pixel it also
 * writes the state the adjoint starts from to state [Vy*Vx][Ny][Nx] of four
 * 32-bit words (device, 16-byte aligned, state_bytes >=
 * lf_composite_state_size(ref, views); separate-views order, also when out
 * is an atlas): T_k (FP32) and k (int32), the transmittance in front of the
 * stop plane k; or, when the walk never stops, T behind the last plane and
 * k = N; then two zero words. The state is owned by the caller and stays
 * valid while planes, ref and views are unchanged. Errors as lf_composite,
 * and LF_ERR_INVALID_ARG for a NULL, misaligned or short state. */
lf_status lf_composite_save(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views, float* out,
                            float* state, size_t state_bytes, void* ws, size_t ws_bytes, cudaStream_t stream);

/* lf_composite_backward from the state lf_composite_save wrote for the same
 * planes, ref and views: one back-to-front walk over the planes instead of
 * two. The planes behind a pixel's stop plane get no gradient from it (their
 * T, below 2^-24, is taken as 0); otherwise the same gradients up to FP32
 * rounding. Same contract and errors as lf_composite_backward, and
 * LF_ERR_INVALID_ARG for a NULL, misaligned or short state. */
lf_status lf_composite_backward_saved(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                                      const float* dviews, const float* state, size_t state_bytes, float* dplanes,
                                      void* ws, size_t ws_bytes, cudaStream_t stream);

/* Adjoint of lf_build_mpi_gaussians: given dplanes = dL/d(planes.rgba)
 * [N][H][W][4] FP32 device, writes the parameter gradients into grad (every
 * array overwritten; culled Gaussians get 0). g, ref and planes must be those
 * of the forward call and ws (ws_bytes) the workspace that call used,
 * unchanged since: the adjoint reads the forward's depth order, rank-ordered
 * records and tile lists from it. After an overflowed build the gradients are
 * all 0 (lf_mpi_status reports the overflow). The adjoint is that of exact
 * blending; after a forward with LF_BLEND_3DGS it returns the exact-blending
 * gradient of the same structure. With FP32 planes it reads the forward's
 * texels (planes->rgba, 16-byte aligned). Errors: LF_ERR_INVALID_ARG,
 * LF_ERR_WORKSPACE, LF_ERR_CUDA. */
lf_status lf_build_mpi_backward_gaussians(const lf_gaussians* g, const lf_ref_camera* ref, const lf_planes* planes,
                                          const float* dplanes, lf_gaussians_grad* grad, void* ws, size_t ws_bytes,
                                          cudaStream_t stream);

/* Adjoint of lf_build_mpi_voxels (Sec. 4.5): gradients of the corner
 * densities and colours; same contract as lf_build_mpi_backward_gaussians. */
lf_status lf_build_mpi_backward_voxels(const lf_voxels* v, const lf_ref_camera* ref, const lf_planes* planes,
                                       const float* dplanes, lf_voxels_grad* grad, void* ws, size_t ws_bytes,
                                       cudaStream_t stream);

/* ---- batching ------------------------------------------------------------ */
/*
 * Several G2LF scenes of uneven sizes, view counts, resolutions and N
 * rendered together: each scene's build runs up to its tile lists, then ONE
 * persistent raster launch covers the (tile, chunk) items of every scene and
 * ONE persistent staged-composite launch covers the (chunk group, view
 * group, row band, column tile) items of every scene, CTAs pulling items
 * from a global counter; or (schedule 2) every scene's single-scene pipeline
 * runs on a stream of its own, all in parallel. With chunk groups G > 1 a
 * scene's non-empty planes are cut into G contiguous shares composited
 * separately into partial (Q, T) per view pixel and then composed front to
 * back, Q = Q_f + T_f Q_b, T = T_f T_b (the over operator of Eq.
 * alpha_blend is associative). The whole batch can be captured once into a
 * CUDA graph and relaunched per frame. An autotuner times candidate plans
 * (views per thread, composite tile shape, chunk groups, scene schedule) on
 * the batch itself. Integer results (chunks, rectangles, lists) are
 * identical for every plan, and so are the views for G = 1; G > 1 changes
 * only the rounding order of the composite.
 */

/* One scene of a batch. Every pointer is device memory the caller owns and
 * keeps alive (and unmoved) for the life of the batch; the fields mean what
 * they mean for lf_build_mpi_gaussians (ws: its build workspace) and
 * lf_composite (cws: its composite workspace, out: its views). All scenes of
 * a batch share planes.dtype and views.bilinear. Batches blend in exact
 * mode: lf_batch_create rejects a binning carrying LF_BLEND_3DGS
 * (LF_ERR_UNSUPPORTED). */
typedef struct {
    lf_gaussians g;
    lf_ref_camera ref;
    int32_t N, binning;
    lf_planes planes;
    lf_view_set views;
    float* out;
    void* ws;
    size_t ws_bytes;
    void* cws;
    size_t cws_bytes;
} lf_batch_scene;

/* Launch plan of a batch:
 *  views_per_thread  composite views per thread: 3, 5, 9 or 15 (15: one
 *                    CTA per SM, the others two);
 *  tile_x            composite CTA tile width (columns): 128, 256 or 512
 *                    (the tile is tile_x x 512/tile_x pixels);
 *  chunk_groups      1, 2 or 4: the contiguous shares of every scene's
 *                    non-empty planes that are composited as separate items
 *                    and composed in order (partial buffers in the batch
 *                    workspace: lf_batch_plan_workspace_size);
 *  schedule          0: items in scene order; 1: largest scenes first;
 *                    2: no persistent launches -- every scene's own
 *                    lf_build_mpi_gaussians + lf_composite on a stream of its
 *                    own, forked from and joined back into the caller's
 *                    stream (the other fields are then unused). */
typedef struct {
    int32_t views_per_thread;
    int32_t tile_x;
    int32_t chunk_groups;
    int32_t schedule;
} lf_batch_plan;

typedef struct lf_batch lf_batch;   /* opaque host-side batch object */

/* Validates the scenes and copies their descriptions (host) into a new batch
 * object. Errors: LF_ERR_INVALID_ARG (bad scene, mixed dtype or sampling),
 * LF_ERR_UNSUPPORTED (a plane row that is not a multiple of 16 bytes). */
lf_status lf_batch_create(const lf_batch_scene* scenes, int32_t n_scenes, lf_batch** out);

/* Device bytes of the batch workspace for plans with one chunk group (scene
 * tables and work counters). */
size_t lf_batch_workspace_size(const lf_batch* b);

/* Device bytes of the batch workspace for plan (NULL = default): the tables
 * plus, for chunk_groups G > 1, G - 1 partial buffers of every scene's
 * views (16 bytes per view pixel each). 0 for an invalid plan. */
size_t lf_batch_plan_workspace_size(const lf_batch* b, const lf_batch_plan* plan);

/* Sets the plan (NULL = default {9, 512, 1, 1}) and uploads the scene tables
 * into ws (device, ws_bytes >= lf_batch_plan_workspace_size, 256-byte
 * aligned) on stream. Must be called before lf_batch_render and again after
 * a plan change; not during capture. */
lf_status lf_batch_prepare(lf_batch* b, const lf_batch_plan* plan, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Enqueues one frame of the whole batch on stream (builds, persistent
 * raster, coefficient tables, persistent composite). No host
 * synchronisation; may be captured. */
lf_status lf_batch_render(lf_batch* b, cudaStream_t stream);

/* Captures lf_batch_render on stream (which must not be the legacy default
 * stream) into a CUDA graph kept by b, replacing any earlier one. */
lf_status lf_batch_capture(lf_batch* b, cudaStream_t stream);

/* Launches the captured graph on stream (LF_ERR_INVALID_ARG if none). */
lf_status lf_batch_launch(lf_batch* b, cudaStream_t stream);

/* Times every candidate plan (coordinate search: composite views per thread
 * {3, 5, 9, 15} x tile width, then chunk groups x schedules 0 and 1 -- the group counts
 * whose partial buffers fit in ws_bytes -- then schedule 2), reps frames each
 * after one warm-up frame, with CUDA events on stream; leaves b prepared with
 * the fastest plan and returns it in *best (host) and its mean frame time in
 * *best_ms (host, may be NULL). Synchronises the stream. */
lf_status lf_batch_autotune(lf_batch* b, void* ws, size_t ws_bytes, int32_t reps, cudaStream_t stream,
                            lf_batch_plan* best, float* best_ms);

/* Synchronises stream and returns LF_ERR_OVERFLOW if a scene's tile list
 * overflowed its capacity, LF_ERR_TIMEOUT if a bounded wait of the
 * composite gave up, else LF_OK. */
lf_status lf_batch_status(lf_batch* b, cudaStream_t stream);

/* Frees the batch object and its graph (device memory stays the caller's). */
lf_status lf_batch_destroy(lf_batch* b);

/* ---- tracing -------------------------------------------------------------- */

/* Number of kernels the library has launched in this process so far. */
int64_t lf_launch_count(void);

/* Turns stage tracing on or off for calls made from this thread: while on,
 * every pipeline stage of lf_build_mpi_* and lf_composite (project,
 * depth_sort, bin, duplicate, tile_sort, ranges, raster_*, comp_coeffs,
 * composite) is bracketed by a CUDA event pair recorded on the call's stream.
 * Always returns LF_OK. */
lf_status lf_trace_enable(int32_t on);

/* Waits for the recorded events, then returns the number of distinct stages
 * (at most max_stages) and for each, in first-seen order: its name in
 * names[32*k .. 32*k+31] (host, NUL-terminated), total milliseconds
 * total_ms[k] and number of traced calls launches[k] (host); any output may
 * be NULL. Clears the record. */
int32_t lf_trace_collect(char* names, double* total_ms, int64_t* launches, int32_t max_stages);

/* ---- failure detection ----------------------------------------------------- */

/* Every device-side wait of the library (the staged composite's mbarrier
 * waits) is bounded: after 2 s of wall time it gives up, the kernel sets the
 * call's error word and returns, and lf_composite_status / lf_batch_status
 * report LF_ERR_TIMEOUT;
 * the CUDA context stays usable. This self-test exercises that path without
 * a fault: one thread waits, with a limit of limit_ms (1..10000)
 * milliseconds, on a shared-memory mbarrier that nothing arrives on.
 * Synchronises the stream; returns LF_ERR_TIMEOUT when the wait gave up as
 * designed, LF_ERR_CUDA if the launch failed, LF_ERR_INVALID_ARG for a limit
 * out of range. Allocates nothing (the result word is a static device
 * variable). */
lf_status lf_selftest_bounded_wait(int32_t limit_ms, cudaStream_t stream);

/* ---- misc --------------------------------------------------------------- */

/* Thread-local description of the last error on this thread ("" if none). */
const char* lf_last_error(void);

/* Library version string. */
const char* lf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LF_H */
