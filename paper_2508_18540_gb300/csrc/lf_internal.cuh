// lf_internal.cuh -- shared declarations of the liblf implementation units.
//
// Not part of the public ABI (include/lf.h is). Holds the workspace layout,
// the per-launch parameter blocks derived on the host, error plumbing and
// the launchers each translation unit exports to lf_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <string>

#include "lf.h"

namespace lf {

constexpr int kTile = 16;                 // raster tile edge (pixels): one CTA per (tile, chunk)
constexpr int kTilePix = kTile * kTile;
constexpr int kSuper = 32;                // list super-tile edge (pixels): lists per (super-tile, chunk)
constexpr int kTilesPerSuper = kSuper / kTile;
constexpr int kRadixBlockKeys = 2048;     // keys per radix-sort block
constexpr int kSortDigits = 256;          // 8-bit radix digits
constexpr int kDupBlock = 1024;           // ranks per block of the tile-pair emission
constexpr uint64_t kInvalidKey = ~0ull;

// bytes of one RGBA texel of a plane type
inline int texel_bytes(int dtype) { return dtype == LF_F32 ? 16 : dtype == LF_U8 ? 4 : 8; }

// ---- programmatic dependent launch (the build's chain of short kernels) ----
// A kernel launched with launch_pdl outside a graph capture may be scheduled
// while its predecessor in the stream is still draining; it must call pdl_wait() before touching any
// memory the predecessor writes or reads (griddepcontrol.wait returns once
// the predecessor grid has completed and its writes are visible; it is a
// no-op for an ordinary launch). pdl_trigger() lets the successor launch as
// soon as every CTA of this grid has started.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl_attr(bool programmatic, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args)
{
    // a CUDA graph already hides the launch gaps (measured: programmatic
    // edges only add a few microseconds per frame there), so a launch that is
    // being captured is an ordinary one
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool pdl = cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    launch_pdl_attr(pdl, kern, grid, block, smem, s, static_cast<Args&&>(args)...);
}

// The same with a programmatic edge in a captured graph as well: for a
// kernel that must run alongside its predecessor, not after it.
template <typename... KArgs, typename... Args>
inline void launch_overlapped(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    launch_pdl_attr(true, kern, grid, block, smem, s, static_cast<Args&&>(args)...);
}
#endif

// ---- mbarriers with bounded waits (shared by the staged kernels) ---------
// Every device-side wait of the library gives up after about kWaitLimitNs of
// wall time or kSpinLimit tries; its caller then records an error word.
constexpr long long kSpinLimit = 1ll << 26;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s: a wait that long has failed
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity; gives up (false) after about
// limit_ns of wall time (the clock is read every 4096 failed tries, from the
// first such read on) or kSpinLimit tries, whichever comes first. One plain
// loop: the common case (first try succeeds) costs what an unbounded wait does.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    unsigned long long t0 = 0;
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 4095) == 4095) {
            const unsigned long long t = global_ns();
            if (t0 == 0)
                t0 = t;
            else if (t - t0 > limit_ns)
                return false;
        }
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    return mbar_wait_for(bar, parity, kWaitLimitNs);
}

#endif

// ---- RGBA8 unorm codec (exact, no conversion-unit instructions) -------------
// decode: byte k of u placed under the exponent of 2^23 reads 2^23 + byte;
//         subtracting 2^23 leaves the byte as an exact FP32 integer.
// encode: round(255 clamp(v, 0, 1)) to nearest even is the low byte of the
//         FP32 sum fl(255 clamp(v)) + 2^23, whose ulp there is 1.
#ifdef __CUDACC__
template <int K>
__device__ __forceinline__ float u8_byte(uint32_t u)
{
    return __int_as_float((int)__byte_perm(u, 0x4B000000u, 0x7440u | (uint32_t)K)) - 8388608.0f;
}

__device__ __forceinline__ float4 u8_unpack(uint32_t u)
{
    constexpr float s = 1.0f / 255.0f;
    return make_float4(u8_byte<0>(u) * s, u8_byte<1>(u) * s, u8_byte<2>(u) * s, u8_byte<3>(u) * s);
}

__device__ __forceinline__ uint32_t u8_code(float v)
{
    return __float_as_uint(__fadd_rn(__fmul_rn(__saturatef(v), 255.0f), 8388608.0f));   // code in the low byte
}

__device__ __forceinline__ uint32_t u8_pack(float r, float g, float b, float a)
{
    const uint32_t lo = __byte_perm(u8_code(r), u8_code(g), 0x0040u);   // [r, g, r, r]
    const uint32_t hi = __byte_perm(u8_code(b), u8_code(a), 0x0040u);   // [b, a, b, b]
    return __byte_perm(lo, hi, 0x5410u);                                // [r, g, b, a]
}
#endif

// ---- launch counting and stage tracing ------------------------------------
// Every kernel launch of the library bumps a process-wide counter; when
// tracing is on, each pipeline stage is bracketed by a CUDA event pair on the
// stream it runs on (see lf_trace_* in lf.h).
void note_launches(int k);
void trace_begin(const char* stage, cudaStream_t s);
void trace_end(cudaStream_t s);
bool trace_swap(bool on);   // sets this thread's tracing flag, returns the old one

// ---- error plumbing ------------------------------------------------------
void set_error(const std::string& msg);
lf_status fail(lf_status st, const std::string& msg);
lf_status check_launch(const char* what);

// ---- device-side state kept at the front of a build workspace -----------
struct WsHeader {
    unsigned long long kmin;      // smallest / largest valid depth key
    unsigned long long kmax;
    unsigned long long M;         // culled-in primitives
    unsigned long long total_dups;
    unsigned long long tile_n;    // pairs to sort (0 after an overflow)
    unsigned long long long_runs; // depth-sort runs longer than 32 keys, sorted by k_depth_long_runs
    int overflow;                 // 1 if total_dups > dup_capacity
    int kind;                     // 0 gaussians, 1 voxels
    long long n;
    long long dup_capacity;
    int N, W, H, tiles_x, tiles_y, supers_x, supers_y;
    int binning;
    // Gaussian raster (k_raster_plan): lists longer than r_seg entries are
    // split into parts
    unsigned int r_heavy;         // parts of split lists
    int r_seg;                    // entries per part (0x7fffffff: no list is split)
};

// Split lists of the Gaussian raster: a list of L > r_seg entries is cut into
// ceil(L / r_seg) parts, each with a partial (C, T) slot of one super-tile
// (kSuper^2 texels); r_seg is at least kRasterSegMin and large enough that
// the parts of a frame never need more than the workspace's slots.
constexpr int kRasterSegMin = 1024;
constexpr long long kRasterSlotsMax = 4096;

// Carved build workspace (all device pointers).
struct BuildWs {
    WsHeader* hdr;
    unsigned long long* keyA;     // [n] depth keys by primitive (IEEE bits of the FP64 depth, or invalid)
    unsigned long long* keyB;     // [n] scratch of the depth sort
    uint32_t* valA;               // [n] primitive ids (rank order after sorting)
    uint32_t* valB;
    float2* mean2d;               // [n] per primitive (Gaussians)
    float4* conic_o;              // [n] per primitive: (a, b, c, opacity) / voxel (lo_rel xyz, side)
    // copies in rank order, made while binning
    float4* r_geo;                // [n] (mean x, mean y, -) or voxel (lo_rel xyz, side)
    float4* r_con;                // [n] Gaussian (a, b, c, opacity)
    int4* r_rect;                 // [n] footprint
    float4* r_rgb;                // [n] colour
    float4* r_den;                // [2 n] voxel corner densities
    int32_t* r_chunk;             // [n]
    uint32_t* hist;               // [kSortDigits * nb] radix histograms
    uint32_t* dtot;               // [kSortDigits] per-digit totals of a radix pass
    uint32_t* bsum;               // [nbd] block sums of the pair emission
    int32_t* chunk_start;         // [N + 1]
    uint32_t* tkeyA;              // [cap] tile id of every (tile, rank) pair
    uint32_t* tkeyB;
    uint32_t* entA;               // [cap] rank of every pair
    uint32_t* entB;
    int2* seg;                    // [supers * N] (start, end) of every (super-tile, chunk) list
    float* g2d;                   // [n][12] per-rank gradient accumulators of the backward pass
    int4* r_items;                // [slots] parts of split lists: {list, part, parts, slot}
    float4* r_part;               // [slots][kSuper^2] partial (C, T) of every part
    int* r_arrive;                // [lists] parts of a split list finished
    long long r_nslots;           // partial-result slots
    size_t bytes;
    long long nb_sort, nb_dup;
};

size_t build_ws_layout(int64_t n, int32_t N, int32_t W, int32_t H, int64_t cap, void* base, BuildWs* out);
// tile-pair capacity that a workspace of ws_bytes holds (0 if too small)
int64_t ws_capacity(int64_t n, int32_t N, int32_t W, int32_t H, size_t ws_bytes);

// ---- per-launch parameters computed on the host -------------------------
struct ProjParams {
    double R[9];
    double t[3];
    double D_forward;
    double z_near;
    double rho;                    // |R20| + |R21| + |R22|
    double origin[3];              // voxels
    double base_size;              // voxels
    double cam_o[3];               // reference centre in world coordinates (FP64)
    float Rf[9];
    float t0f, t1f, t2rf;          // t2rf = (float)(t2 - D_forward)
    float fxf, fyf, cxf, cyf, fpf;
    float wmax, hmax;
    int W, H;
    long long n;
};

struct RasterParams {
    int W, H, N, tiles_x, tiles_y, supers_x, supers_y, dtype;
    // voxels: world-frame reference rays
    float Rt[9];                    // R^T row-major (camera -> world)
    float fx, fy, cx, cy;
};

struct BinParams {
    int N;
    int binning;
    double D_forward;
};

// ---- launchers ----------------------------------------------------------
void launch_init_header(const WsHeader& h, WsHeader* d, cudaStream_t s);
void launch_project_gaussians(const lf_gaussians& g, const ProjParams& p, const BuildWs& ws, int32_t* rect,
                              int32_t* chunk, cudaStream_t s);
void launch_project_voxels(const lf_voxels& v, const ProjParams& p, const BuildWs& ws, int32_t* rect,
                           int32_t* chunk, cudaStream_t s);

// Order of the culled-in primitives by (FP64 depth, index): valA[r] = the
// primitive of rank r (r < hdr->M). keyA keeps the primitives' depth keys
// (IEEE bits, by primitive index). Uses tkeyA/tkeyB, valB, keyB as scratch.
void sort_depth_keys(const BuildWs& ws, long long n, cudaStream_t s);

void launch_bin(const BuildWs& ws, const BinParams& p, long long n, int32_t* chunk, double* d, int32_t* count,
                const int32_t* rect, const float* rgb, const float* dens8, int kind, cudaStream_t s);
// (super-tile, chunk) lists: (super-tile, rank) pairs emitted in rank order,
// stable sort by super-tile, [start, end) of every (super-tile, chunk) list.
// Returns the sorted ranks.
const uint32_t* launch_tile_lists(const BuildWs& ws, long long n, long long cap, int N, int supers_x, int n_supers,
                                  cudaStream_t s);
void sort_tile_keys(const BuildWs& ws, long long cap, int tile_bits, cudaStream_t s, uint32_t** keys_out,
                    uint32_t** vals_out);
int tile_sort_passes(int tile_bits);
int tile_bits_for(long long tiles);

// blend3dgs: the alpha < 1/255 skip and T < 1e-4 stop of the 3DGS rasteriser
void launch_raster_gaussians(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                             bool blend3dgs, cudaStream_t s);
void launch_raster_voxels(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, void* planes,
                          cudaStream_t s);

// batched (several scenes, one persistent launch): per-scene item table
struct RasterScene {
    BuildWs w;
    RasterParams p;
    const uint32_t* ranks;
    void* planes;
    long long pbase;        // its first split-part CTA in the batch grid (raster_part_ctas of them)
    long long lbase;        // its first list CTA in the batch grid
};
// CTAs a raster reserves for the parts of split lists
long long raster_part_ctas(const BuildWs& ws);
// the split parts of one Gaussian raster into ws.r_items; blend3dgs splits
// no list
void launch_raster_plan(const BuildWs& ws, const RasterParams& p, bool blend3dgs, cudaStream_t s);
// raster of several scenes (their plans made) in one grid of total CTAs: the
// split-part CTAs of every scene first (parts_total of them), then the list
// CTAs
void launch_raster_gauss_batched(const RasterScene* scenes_dev, int n_sc, int dtype, long long parts_total,
                                 long long total, cudaStream_t s);

// backward: raster adjoints accumulate into ws.g2d (zeroed by the caller),
// then the per-rank chain rule / scatter writes the parameter gradients
// planes: the forward's plane texels (p.dtype), read for K with FP32 planes
void launch_raster_gaussians_bwd(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks,
                                 const void* planes, const float* dplanes, cudaStream_t s);
void launch_raster_voxels_bwd(const BuildWs& ws, const RasterParams& p, const uint32_t* ranks, const void* planes,
                              const float* dplanes, cudaStream_t s);
void launch_gauss_chain(const lf_gaussians& g, const ProjParams& p, const BuildWs& ws, const lf_gaussians_grad& out,
                        cudaStream_t s);
void launch_voxel_scatter(const BuildWs& ws, long long n, const lf_voxels_grad& out, cudaStream_t s);

// ---- helpers exported by lf_api.cu to the batch module -------------------
// the build of one Gaussian scene up to its tile lists (no raster)
lf_status build_gaussians_prefix(const lf_gaussians* g, const lf_ref_camera* ref, int32_t N, int32_t binning,
                                 void* ws, size_t ws_bytes, lf_planes* out, cudaStream_t stream, BuildWs* w,
                                 const uint32_t** ranks);
void raster_params(const lf_ref_camera* ref, int32_t N, int32_t dtype, RasterParams* p);

// ---- V2LF low-pass plane filter ------------------------------------------
constexpr int kFilterMaxRadius = 16;
struct FilterParams {
    int radius;
    float w[2 * kFilterMaxRadius + 1];   // normalised weights of offsets -radius..radius
};
void launch_filter_planes(void* planes, int dtype, int N, int W, int H, const FilterParams& f, cudaStream_t s);

// ---- composite ----------------------------------------------------------
struct CompWs {
    float* cx;      // [Vx][N][3] (gm, hn, hb) along x
    float* cy;      // [Vy][N][3] along y
    int* err;       // [1] set to 1 if a bounded device wait gave up
    int* wide;      // [N] 1 if some view's index range of plane k needs clamping
    size_t bytes;
};
size_t comp_ws_layout(int32_t N, int32_t Vx, int32_t Vy, void* base, CompWs* out);

struct CompParams {
    int N, W, H, Nx, Ny, Vx, Vy, P_s, bilinear, dtype;
    int atlas_cols;     // 0: separate views; c: quilt atlas of c view tiles per row
    float bg[3];
    // FP64 set-up for the per-(view, plane) coefficients
    double D_focal, D_forward, tth_x, tth_y, tthp_x, tthp_y, tphi_x, tphi_y;
};

// staged composite layout (see lf_composite.cu)
// Consumer threads of a staged-composite CTA (plus one producer warp): 256
// for the forward kernels (two CTAs per SM at up to 15 views per thread,
// four at 9 or fewer: an SM keeps working on one CTA's planes while the
// other's warps wait at its ring), 512 for the adjoint (two CTAs per SM).
constexpr int kStagedThreads = 256;
constexpr int kBwdStagedThreads = 512;
constexpr int kStages = 6;            // depth of its plane-row ring
constexpr size_t kTwoCtaSmem = 112 * 1024;   // dynamic shared memory that still lets two CTAs share an SM
constexpr int kTwoCtaViews = 9;               // widest view group run at the higher CTA count per SM
struct StagedGeom {
    int TX, BY, VG, rows_per_y;    // rows_per_y: 1 nearest, 2 bilinear
    int padl;                      // zero texels left of every staged row (16 bytes)
    int row_texels;                // padl + W + right pad, a multiple of 16 bytes
    size_t row_bytes, stage_bytes, smem_bytes;
    int groups_x;                  // view groups per view row
    int stages;                    // ring depth of the single-scene kernel (<= kStages)
    size_t blend_bytes;            // bilinear: two FP32 row buffers per output row (single-scene kernel)
};
StagedGeom staged_geom(const CompParams& p, int texel_bytes, bool bilinear, int VG, int tx_max,
                       int threads = kStagedThreads);

// batched (several scenes, one persistent launch): per-scene item table;
// item li of a scene: chunk group li % groups, then view group, then column
// tile, then row band
struct CompScene {
    CompParams p;
    StagedGeom G;
    const char* planes;
    const int32_t* count;
    CompWs w;
    float* out;
    long long base;     // first global item of this scene
    int nby, nbz;       // row bands, column tiles
    int groups;         // chunk groups: contiguous shares of the non-empty planes
    float4* part;       // groups > 1: [groups - 1][V][Ny][Nx] partial (Q, T) of groups 1.. (group 0 in out)
};
constexpr int kMaxChunkGroups = 4;
// groups > 1: composes the partials (group 0 in out, the others in part)
// front to back into out's final views
void launch_merge_chunk_groups(const CompParams& p, int groups, const float4* part, float* out, cudaStream_t s);
void launch_comp_coeffs(const CompParams& p, const double* d, const int32_t* count, const CompWs& ws,
                        cudaStream_t s);
// smem_bytes: the largest staged layout of the batch (its stage size, N)
bool launch_composite_batched(const CompScene* scenes_dev, int n_sc, long long total, int dtype, bool bilinear,
                              int VG, size_t max_stage_bytes, int maxN, unsigned long long* counter, int n_ctas,
                              cudaStream_t s);
size_t composite_batched_smem(size_t max_stage_bytes, int maxN, int VG);
// argument checks and parameters of one composite (lf_api.cu)
lf_status composite_args(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                         const float* out, void* ws, size_t ws_bytes, CompWs* cw, CompParams* p);
// state != null: the saving form, which also writes the adjoint's starting
// state ([V][Ny][Nx] float4, separate views order)
void launch_composite(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                      float* out, cudaStream_t s, float4* state = nullptr);
void launch_wait_selftest(unsigned long long limit_ns, int* result, cudaStream_t s);
// state != null: start from the saving forward's state (one plane walk)
void launch_composite_bwd(const CompParams& p, const void* planes, const int32_t* count, const CompWs& ws,
                          const float* dviews, float* dplanes, cudaStream_t s, const float4* state = nullptr);

}  // namespace lf
