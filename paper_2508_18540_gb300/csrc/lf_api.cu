// lf_api.cu -- C ABI entry points of liblf (declared in include/lf.h):
// argument checks, host-side FP64 set-up, workspace carving and the launch
// sequence of each stage. All arithmetic of the path runs in the kernels of
// the other translation units.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lf_internal.cuh"

#include <nvtx3/nvToolsExt.h>   // header-only; ranges are no-ops unless a profiler is attached

namespace lf {

static thread_local std::string g_last_error;

// ---- launch counting / stage tracing ------------------------------------
static std::atomic<long long> g_launches{0};
static thread_local bool g_trace_on = false;
struct TraceRec {
    std::string stage;
    cudaEvent_t a, b;
};
static thread_local std::vector<TraceRec> g_trace;
static thread_local std::vector<cudaEvent_t> g_event_pool;
static thread_local int g_trace_open = -1;

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// one NVTX range per stage on the calling thread (named like the stage), so
// a timeline profiler shows the pipeline's steps; a range left open by an
// early error return is closed by the next stage
static thread_local int g_nvtx_open = 0;

void trace_begin(const char* stage, cudaStream_t s)
{
    if (g_nvtx_open) nvtxRangePop();
    nvtxRangePushA(stage);
    g_nvtx_open = 1;
    if (!g_trace_on) return;
    TraceRec r{stage, pool_event(), pool_event()};
    cudaEventRecord(r.a, s);
    g_trace.push_back(r);
    g_trace_open = (int)g_trace.size() - 1;
}

void trace_end(cudaStream_t s)
{
    if (g_nvtx_open) {
        nvtxRangePop();
        g_nvtx_open = 0;
    }
    if (!g_trace_on || g_trace_open < 0) return;
    cudaEventRecord(g_trace[g_trace_open].b, s);
    g_trace_open = -1;
}

bool trace_swap(bool on)
{
    const bool old = g_trace_on;
    g_trace_on = on;
    return old;
}

void set_error(const std::string& msg) { g_last_error = msg; }

lf_status fail(lf_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

lf_status check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LF_OK;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename T>
static T* carve(char* base, size_t& off, size_t count)
{
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * count;
    return p;
}

size_t build_ws_layout(int64_t n, int32_t N, int32_t W, int32_t H, int64_t cap, void* basev, BuildWs* o)
{
    char* base = static_cast<char*>(basev);
    const long long supers = (long long)((W + kSuper - 1) / kSuper) * ((H + kSuper - 1) / kSuper);
    const long long S = supers * N;                                 // (super-tile, chunk) lists
    const long long nmax = n > cap ? n : cap;
    const long long nb = (nmax + kRadixBlockKeys - 1) / kRadixBlockKeys + 1;
    const long long nbd = (n + kDupBlock - 1) / kDupBlock + 1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t cc = (size_t)(cap > 0 ? cap : 1);
    size_t off = 0;
    BuildWs w;
    w.hdr = carve<WsHeader>(base, off, 1);
    w.keyA = carve<unsigned long long>(base, off, nn);
    w.keyB = carve<unsigned long long>(base, off, nn);
    w.valA = carve<uint32_t>(base, off, nn);
    w.valB = carve<uint32_t>(base, off, nn);
    w.mean2d = carve<float2>(base, off, nn);
    w.conic_o = carve<float4>(base, off, nn);
    w.r_geo = carve<float4>(base, off, nn);
    w.r_con = carve<float4>(base, off, nn);
    w.r_rect = carve<int4>(base, off, nn);
    w.r_rgb = carve<float4>(base, off, nn);
    w.r_den = carve<float4>(base, off, 2 * nn);
    w.r_chunk = carve<int32_t>(base, off, nn);
    w.hist = carve<uint32_t>(base, off, (size_t)kSortDigits * nb);
    w.dtot = carve<uint32_t>(base, off, (size_t)kSortDigits);
    w.bsum = carve<uint32_t>(base, off, (size_t)nbd);
    w.chunk_start = carve<int32_t>(base, off, (size_t)N + 1);
    w.tkeyA = carve<uint32_t>(base, off, cc);
    w.tkeyB = carve<uint32_t>(base, off, cc);
    w.entA = carve<uint32_t>(base, off, cc);
    w.entB = carve<uint32_t>(base, off, cc);
    w.seg = carve<int2>(base, off, (size_t)S);
    w.g2d = carve<float>(base, off, 12 * nn);
    // partial-result slots of split raster lists: enough that a frame of cap
    // pairs needs no more than kRasterSegMin entries per part, up to a cap
    long long slots = 2 * (long long)cc / kRasterSegMin + 2;
    slots = slots < 16 ? 16 : slots > kRasterSlotsMax ? kRasterSlotsMax : slots;
    w.r_nslots = slots;
    w.r_items = carve<int4>(base, off, (size_t)slots);
    w.r_arrive = carve<int>(base, off, (size_t)S);
    w.r_part = carve<float4>(base, off, (size_t)slots * kSuper * kSuper);
    w.bytes = align_up(off, 256);
    w.nb_sort = nb;
    w.nb_dup = nbd;
    if (o) *o = w;
    return w.bytes;
}

size_t comp_ws_layout(int32_t N, int32_t Vx, int32_t Vy, void* basev, CompWs* o)
{
    char* base = static_cast<char*>(basev);
    size_t off = 0;
    CompWs w;
    w.cx = carve<float>(base, off, (size_t)Vx * N * 3);
    w.cy = carve<float>(base, off, (size_t)Vy * N * 3);
    w.err = carve<int>(base, off, 1 + (size_t)N);
    w.wide = w.err + 1;
    w.bytes = align_up(off, 256);
    if (o) *o = w;
    return w.bytes;
}

// stream each build workspace was last used on (for lf_mpi_status)
static std::mutex g_ws_mu;
static std::map<const void*, cudaStream_t> g_ws_stream;

static int64_t default_cap(int64_t n) { return 8 * n + (1ll << 20); }

// pair capacity of a build workspace: the largest one ws_bytes holds (the
// layout size grows monotonically with it); 0 if none
int64_t ws_capacity(int64_t n, int32_t N, int32_t W, int32_t H, size_t ws_bytes)
{
    int64_t lo = 0, hi = (1ll << 31) - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (build_ws_layout(n, N, W, H, mid, nullptr, nullptr) <= ws_bytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

static lf_status check_ref(const lf_ref_camera* r)
{
    if (!r) return fail(LF_ERR_INVALID_ARG, "ref camera is NULL");
    if (r->W <= 0 || r->H <= 0 || r->W > 32768 || r->H > 32768)
        return fail(LF_ERR_INVALID_ARG, "reference plane size out of range (1..32768)");
    if (!(r->fx > 0) || !(r->fy > 0)) return fail(LF_ERR_INVALID_ARG, "ref camera not initialised");
    return LF_OK;
}

static lf_status check_planes(const lf_planes* p, const lf_ref_camera* r, int32_t N)
{
    if (!p) return fail(LF_ERR_INVALID_ARG, "planes is NULL");
    if (N < 1 || N > 65535) return fail(LF_ERR_INVALID_ARG, "N_chunk must be in 1..65535");
    if (p->N != N || p->W != r->W || p->H != r->H)
        return fail(LF_ERR_INVALID_ARG, "plane array shape does not match N / reference camera");
    if (p->dtype < LF_F32 || p->dtype > LF_U8) return fail(LF_ERR_INVALID_ARG, "unknown plane dtype");
    if (!p->rgba || !p->d || !p->count || !p->chunk || !p->rect)
        return fail(LF_ERR_INVALID_ARG, "a plane output pointer is NULL");
    return LF_OK;
}

static void fill_proj_params(const lf_ref_camera* r, int64_t n, ProjParams* p)
{
    std::memset(p, 0, sizeof(*p));
    for (int i = 0; i < 9; ++i) {
        p->R[i] = r->base.R[i];
        p->Rf[i] = (float)r->base.R[i];
    }
    for (int i = 0; i < 3; ++i) p->t[i] = r->base.t[i];
    p->D_forward = r->D_forward;
    p->z_near = r->disp.z_near;
    p->rho = std::fabs(r->base.R[6]) + std::fabs(r->base.R[7]) + std::fabs(r->base.R[8]);
    p->t0f = (float)r->base.t[0];
    p->t1f = (float)r->base.t[1];
    p->t2rf = (float)(r->base.t[2] - r->D_forward);
    p->fxf = (float)r->fx;
    p->fyf = (float)r->fy;
    p->cxf = (float)r->cx;
    p->cyf = (float)r->cy;
    p->fpf = (float)r->f_prime;
    p->wmax = (float)(r->W - 1);
    p->hmax = (float)(r->H - 1);
    p->W = r->W;
    p->H = r->H;
    p->n = n;
    // reference centre in world coordinates: R o + t - D_forward e_z = 0
    const double b[3] = {-r->base.t[0], -r->base.t[1], r->D_forward - r->base.t[2]};
    for (int i = 0; i < 3; ++i)
        p->cam_o[i] = r->base.R[i] * b[0] + r->base.R[3 + i] * b[1] + r->base.R[6 + i] * b[2];
}

static void fill_raster_params(const lf_ref_camera* r, int32_t N, int32_t dtype, RasterParams* p)
{
    std::memset(p, 0, sizeof(*p));
    p->W = r->W;
    p->H = r->H;
    p->N = N;
    p->tiles_x = (r->W + kTile - 1) / kTile;
    p->tiles_y = (r->H + kTile - 1) / kTile;
    p->supers_x = (r->W + kSuper - 1) / kSuper;
    p->supers_y = (r->H + kSuper - 1) / kSuper;
    p->dtype = dtype;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) p->Rt[3 * i + j] = (float)r->base.R[3 * j + i];
    p->fx = (float)r->fx;
    p->fy = (float)r->fy;
    p->cx = (float)r->cx;
    p->cy = (float)r->cy;
}

static void fill_comp_params(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                             CompParams* pp)
{
    CompParams& p = *pp;
    std::memset(&p, 0, sizeof(p));
    p.N = planes->N;
    p.W = ref->W;
    p.H = ref->H;
    p.Nx = ref->base.Nx;
    p.Ny = ref->base.Ny;
    p.Vx = views->Vx;
    p.Vy = views->Vy;
    p.P_s = ref->disp.P_s;
    p.bilinear = views->bilinear ? 1 : 0;
    p.atlas_cols = views->atlas_cols > 0 ? views->atlas_cols : 0;
    p.dtype = planes->dtype;
    for (int c = 0; c < 3; ++c) p.bg[c] = views->bg[c];
    p.D_focal = ref->disp.D_focal;
    p.D_forward = ref->D_forward;
    p.tth_x = ref->tth_x;
    p.tth_y = ref->tth_y;
    p.tthp_x = ref->tthp_x;
    p.tthp_y = ref->tthp_y;
    p.tphi_x = ref->tphi_x;
    p.tphi_y = ref->tphi_y;
}

// argument checks shared by lf_composite and its adjoint; views_buf is the
// output views (forward) or their gradient (backward)
static lf_status check_composite_args(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                                      const float* views_buf, void* ws, size_t ws_bytes, CompWs* cw)
{
    lf_status st = check_ref(ref);
    if (st != LF_OK) return st;
    if (!planes || !views || !views_buf) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (planes->N < 1 || planes->W != ref->W || planes->H != ref->H)
        return fail(LF_ERR_INVALID_ARG, "plane array shape does not match the reference camera");
    if (planes->dtype < LF_F32 || planes->dtype > LF_U8) return fail(LF_ERR_INVALID_ARG, "unknown plane dtype");
    if (!planes->rgba || !planes->d || !planes->count) return fail(LF_ERR_INVALID_ARG, "plane pointer is NULL");
    // texels are read whole (16, 8 or 4 bytes)
    const uintptr_t texel = planes->dtype == LF_F32 ? 16 : (planes->dtype == LF_U8 ? 4 : 8);
    if (((uintptr_t)planes->rgba) % texel) return fail(LF_ERR_INVALID_ARG, "planes->rgba is not texel-aligned");
    if (views->Vx < 1 || views->Vy < 1 || views->Vx > 65535 || views->Vy > 65535)
        return fail(LF_ERR_INVALID_ARG, "view counts must be in 1..65535");
    if (views->atlas_cols < 0) return fail(LF_ERR_INVALID_ARG, "atlas_cols must be >= 0");
    if (!ws) return fail(LF_ERR_WORKSPACE, "workspace is NULL");
    if (((uintptr_t)ws) % 256) return fail(LF_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    if (comp_ws_layout(planes->N, views->Vx, views->Vy, ws, cw) > ws_bytes)
        return fail(LF_ERR_WORKSPACE, "composite workspace too small");
    return LF_OK;
}

// The build pipeline. With prefix_only the raster is left to the caller
// (the batched persistent raster), which gets the carved workspace and the
// sorted tile-list ranks back.
template <typename Launch>
static lf_status build_common(int64_t n, const lf_ref_camera* ref, int32_t N, int32_t binning, void* ws,
                              size_t ws_bytes, lf_planes* out, cudaStream_t stream, int kind, Launch project,
                              const void* raster_arg, bool prefix_only = false, BuildWs* w_out = nullptr,
                              const uint32_t** ranks_out = nullptr)
{
    lf_status st = check_ref(ref);
    if (st != LF_OK) return st;
    st = check_planes(out, ref, N);
    if (st != LF_OK) return st;
    const bool blend3dgs = (binning & LF_BLEND_3DGS) != 0;
    binning &= ~(int32_t)LF_BLEND_3DGS;
    if (binning != LF_BIN_QUANTILE && binning != LF_BIN_DISPARITY)
        return fail(LF_ERR_INVALID_ARG, "unknown binning mode or flag");
    if (blend3dgs && (kind != 0 || prefix_only))
        return fail(LF_ERR_UNSUPPORTED, "3DGS blending is implemented for the single-scene Gaussian build only");
    if (n < 0 || n > (int64_t)0x7fffffff) return fail(LF_ERR_INVALID_ARG, "primitive count out of range");
    if (!ws) return fail(LF_ERR_WORKSPACE, "workspace is NULL");
    if (((uintptr_t)ws) % 256) return fail(LF_ERR_WORKSPACE, "workspace must be 256-byte aligned");

    const int64_t cap = ws_capacity(n, N, ref->W, ref->H, ws_bytes);
    if (cap < 1) {
        const size_t need = build_ws_layout(n, N, ref->W, ref->H, default_cap(n), nullptr, nullptr);
        return fail(LF_ERR_WORKSPACE, "workspace too small (default capacity needs " + std::to_string(need) +
                                          " bytes)");
    }
    BuildWs w;
    build_ws_layout(n, N, ref->W, ref->H, cap, ws, &w);

    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        g_ws_stream[ws] = stream;
    }

    WsHeader h;
    std::memset(&h, 0, sizeof(h));
    h.kmin = ~0ull;
    h.kmax = 0;
    h.kind = kind;
    h.n = n;
    h.dup_capacity = cap;
    h.N = N;
    h.W = ref->W;
    h.H = ref->H;
    h.tiles_x = (ref->W + kTile - 1) / kTile;
    h.tiles_y = (ref->H + kTile - 1) / kTile;
    h.supers_x = (ref->W + kSuper - 1) / kSuper;
    h.supers_y = (ref->H + kSuper - 1) / kSuper;
    h.binning = binning;
    // the header is written by a kernel so the whole build stays on the stream
    launch_init_header(h, w.hdr, stream);
    if ((st = check_launch("header init")) != LF_OK) return st;
    const long long n_supers = (long long)h.supers_x * h.supers_y;

    ProjParams pp;
    fill_proj_params(ref, n, &pp);
    trace_begin("project", stream);
    project(pp, w, stream);
    trace_end(stream);
    if ((st = check_launch("project")) != LF_OK) return st;

    trace_begin("depth_sort", stream);
    sort_depth_keys(w, n, stream);
    trace_end(stream);
    if ((st = check_launch("depth sort")) != LF_OK) return st;

    BinParams bp;
    bp.N = N;
    bp.binning = binning;
    bp.D_forward = ref->D_forward;
    const float* rgb = kind == 0 ? static_cast<const lf_gaussians*>(raster_arg)->rgb
                                 : static_cast<const lf_voxels*>(raster_arg)->rgb;
    const float* dens8 = kind == 0 ? nullptr : static_cast<const lf_voxels*>(raster_arg)->density8;
    trace_begin("bin", stream);
    launch_bin(w, bp, n, out->chunk, out->d, out->count, out->rect, rgb, dens8, kind, stream);
    trace_end(stream);
    if ((st = check_launch("bin")) != LF_OK) return st;

    trace_begin("tile_lists", stream);
    const uint32_t* ranks = launch_tile_lists(w, n, cap, N, h.supers_x, (int)n_supers, stream);
    trace_end(stream);
    if ((st = check_launch("tile lists")) != LF_OK) return st;

    if (prefix_only) {
        if (w_out) *w_out = w;
        if (ranks_out) *ranks_out = ranks;
        return LF_OK;
    }
    RasterParams rp;
    fill_raster_params(ref, N, out->dtype, &rp);
    trace_begin(kind == 0 ? "raster_gaussians" : "raster_voxels", stream);
    if (kind == 0)
        launch_raster_gaussians(w, rp, ranks, out->rgba, blend3dgs, stream);
    else
        launch_raster_voxels(w, rp, ranks, out->rgba, stream);
    trace_end(stream);
    return check_launch("rasterise");
}

lf_status build_gaussians_prefix(const lf_gaussians* g, const lf_ref_camera* ref, int32_t N, int32_t binning,
                                 void* ws, size_t ws_bytes, lf_planes* out, cudaStream_t stream, BuildWs* w,
                                 const uint32_t** ranks)
{
    if (!g) return fail(LF_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity || !g->rgb))
        return fail(LF_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
    const lf_gaussians gc = *g;
    auto project = [&](const ProjParams& pp, const BuildWs& ww, cudaStream_t s) {
        launch_project_gaussians(gc, pp, ww, out->rect, out->chunk, s);
    };
    return build_common(g->n, ref, N, binning, ws, ws_bytes, out, stream, 0, project, &gc, true, w, ranks);
}

lf_status composite_args(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                         const float* out, void* ws, size_t ws_bytes, CompWs* cw, CompParams* p)
{
    const lf_status st = check_composite_args(planes, ref, views, out, ws, ws_bytes, cw);
    if (st != LF_OK) return st;
    fill_comp_params(planes, ref, views, p);
    return LF_OK;
}

void raster_params(const lf_ref_camera* ref, int32_t N, int32_t dtype, RasterParams* p)
{
    fill_raster_params(ref, N, dtype, p);
}

}  // namespace lf

using namespace lf;

extern "C" {

const char* lf_last_error(void) { return lf::g_last_error.c_str(); }

const char* lf_version(void) { return "liblf 0.1 (sm_103a)"; }

}  // extern "C"

// result word of lf_selftest_bounded_wait (a static device variable: the
// self-test allocates nothing)
static __device__ int g_selftest_result;

extern "C" {

lf_status lf_composite_status(int32_t N, const lf_view_set* views, const void* cws, cudaStream_t stream)
{
    if (!views || !cws || N < 1 || views->Vx < 1 || views->Vy < 1) return fail(LF_ERR_INVALID_ARG, "bad argument");
    CompWs cw;
    comp_ws_layout(N, views->Vx, views->Vy, const_cast<void*>(cws), &cw);
    int err = 0;
    if (cudaStreamSynchronize(stream) != cudaSuccess ||
        cudaMemcpy(&err, cw.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_launch("composite status");
    if (err) return fail(LF_ERR_TIMEOUT, "a bounded wait of the composite gave up");
    return LF_OK;
}

lf_status lf_selftest_bounded_wait(int32_t limit_ms, cudaStream_t stream)
{
    if (limit_ms < 1 || limit_ms > 10000) return fail(LF_ERR_INVALID_ARG, "self-test limit must be 1..10000 ms");
    int* d = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&d), g_selftest_result) != cudaSuccess)
        return check_launch("self-test result word");
    if (cudaMemsetAsync(d, 0, sizeof(int), stream) != cudaSuccess) return check_launch("self-test reset");
    launch_wait_selftest((unsigned long long)limit_ms * 1000000ull, d, stream);
    int r = 0;
    if (cudaMemcpyAsync(&r, d, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return check_launch("self-test");
    if (r == 1) return fail(LF_ERR_TIMEOUT, "self-test: the bounded wait gave up as designed");
    return fail(LF_ERR_CUDA, "self-test: unexpected result " + std::to_string(r));
}

int64_t lf_launch_count(void) { return (int64_t)g_launches.load(); }

lf_status lf_trace_enable(int32_t on)
{
    g_trace_on = on != 0;
    return LF_OK;
}

int32_t lf_trace_collect(char* names, double* total_ms, int64_t* launches, int32_t max_stages)
{
    std::vector<std::string> order;
    std::map<std::string, std::pair<double, int64_t>> acc;
    for (auto& r : g_trace) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        if (!acc.count(r.stage)) order.push_back(r.stage);
        acc[r.stage].first += ms;
        acc[r.stage].second += 1;
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_trace.clear();
    int32_t k = 0;
    for (auto& nm : order) {
        if (k >= max_stages) break;
        if (names) {
            std::strncpy(names + 32 * k, nm.c_str(), 31);
            names[32 * k + 31] = 0;
        }
        if (total_ms) total_ms[k] = acc[nm].first;
        if (launches) launches[k] = acc[nm].second;
        ++k;
    }
    return k;
}

lf_status lf_make_ref_camera(const lf_camera* cam, const lf_display* disp, lf_ref_camera* r)
{
    if (!cam || !disp || !r) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    std::memset(r, 0, sizeof(*r));
    r->base = *cam;
    r->disp = *disp;
    if (cam->Nx <= 0 || cam->Ny <= 0 || disp->P_s <= 0) return fail(LF_ERR_INVALID_ARG, "sizes must be positive");
    if (!(disp->D_focal > 0.0) || !(disp->z_near > 0.0))
        return fail(LF_ERR_INVALID_ARG, "D_focal and z_near must be positive");
    if (!(cam->theta_x > 0.0 && cam->theta_x < M_PI) || !(cam->theta_y > 0.0 && cam->theta_y < M_PI))
        return fail(LF_ERR_INVALID_ARG, "field of view must be in (0, pi)");
    if (disp->phi_x < 0.0 || disp->phi_y < 0.0) return fail(LF_ERR_INVALID_ARG, "viewing angle must be >= 0");
    if ((int64_t)cam->Nx * disp->P_s > 32768 || (int64_t)cam->Ny * disp->P_s > 32768)
        return fail(LF_ERR_INVALID_ARG, "plane resolution too large");

    const double Df = disp->D_focal;
    r->tth_x = std::tan(0.5 * cam->theta_x);
    r->tth_y = std::tan(0.5 * cam->theta_y);
    r->tphi_x = std::tan(0.5 * disp->phi_x);
    r->tphi_y = std::tan(0.5 * disp->phi_y);
    // Eq. (1), maximum over the axes that have a viewing angle
    double fwd_x = 0.0, fwd_y = 0.0;
    if (r->tphi_x > 0.0) fwd_x = Df * r->tphi_x / (r->tphi_x + r->tth_x);
    if (r->tphi_y > 0.0) fwd_y = Df * r->tphi_y / (r->tphi_y + r->tth_y);
    r->D_forward0 = fwd_x > fwd_y ? fwd_x : fwd_y;
    // Eq. (2) with the unshifted forward distance
    r->tthp_x = Df * r->tth_x / (Df - r->D_forward0);
    r->tthp_y = Df * r->tth_y / (Df - r->D_forward0);
    r->theta_px = 2.0 * std::atan(r->tthp_x);
    r->theta_py = 2.0 * std::atan(r->tthp_y);
    // near-field shift
    r->D_forward = r->D_forward0 - disp->D_shift;
    if (!(r->D_forward < Df)) return fail(LF_ERR_INVALID_ARG, "D_shift leaves D_forward >= D_focal");
    r->W = cam->Nx * disp->P_s;
    r->H = cam->Ny * disp->P_s;
    r->fx = (double)r->W / (2.0 * r->tthp_x);
    r->fy = (double)r->H / (2.0 * r->tthp_y);
    r->cx = 0.5 * (double)(r->W - 1);
    r->cy = 0.5 * (double)(r->H - 1);
    // Eq. (gs_prefilter_fix) with the shifted forward distance
    const double ratio = Df * r->tth_x / ((Df - r->D_forward) * r->tthp_x) * (double)disp->P_s;
    r->f_prime = disp->f_aa * ratio * ratio;
    return LF_OK;
}

size_t lf_build_mpi_workspace_size(const lf_ref_camera* ref, int64_t n, int32_t N, int64_t dup_capacity)
{
    if (!ref || n < 0 || N < 1) return 0;
    if (dup_capacity <= 0) dup_capacity = default_cap(n);
    return build_ws_layout(n, N, ref->W, ref->H, dup_capacity, nullptr, nullptr);
}

lf_status lf_build_mpi_gaussians(const lf_gaussians* g, const lf_ref_camera* ref, int32_t N, int32_t binning,
                                 void* ws, size_t ws_bytes, lf_planes* out, cudaStream_t stream)
{
    if (!g) return fail(LF_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity || !g->rgb))
        return fail(LF_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
    const lf_gaussians gc = *g;
    auto project = [&](const ProjParams& pp, const BuildWs& w, cudaStream_t s) {
        launch_project_gaussians(gc, pp, w, out->rect, out->chunk, s);
    };
    return build_common(g->n, ref, N, binning, ws, ws_bytes, out, stream, 0, project, &gc);
}

lf_status lf_build_mpi_voxels(const lf_voxels* v, const lf_ref_camera* ref, int32_t N, int32_t binning, void* ws,
                              size_t ws_bytes, lf_planes* out, cudaStream_t stream)
{
    if (!v) return fail(LF_ERR_INVALID_ARG, "voxels is NULL");
    if (v->n > 0 && (!v->ijk || !v->level || !v->density8 || !v->rgb))
        return fail(LF_ERR_INVALID_ARG, "a voxel attribute pointer is NULL");
    if (!(v->base_size > 0.0)) return fail(LF_ERR_INVALID_ARG, "voxel base_size must be positive");
    const lf_voxels vc = *v;
    auto project = [&](const ProjParams& pp0, const BuildWs& w, cudaStream_t s) {
        ProjParams pp = pp0;
        for (int i = 0; i < 3; ++i) pp.origin[i] = vc.origin[i];
        pp.base_size = vc.base_size;
        launch_project_voxels(vc, pp, w, out->rect, out->chunk, s);
    };
    return build_common(v->n, ref, N, binning, ws, ws_bytes, out, stream, 1, project, &vc);
}

lf_status lf_mpi_status(const void* ws, int64_t* needed, int64_t* culled_in)
{
    if (!ws) return fail(LF_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t s = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws_stream.find(ws);
        if (it == g_ws_stream.end()) return fail(LF_ERR_INVALID_ARG, "no build was run on this workspace");
        s = it->second;
    }
    WsHeader h;
    if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("stream synchronise");
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return check_launch("header read");
    if (needed) *needed = (int64_t)h.total_dups;
    if (culled_in) *culled_in = (int64_t)h.M;
    if (h.overflow)
        return fail(LF_ERR_OVERFLOW, "tile list needs " + std::to_string(h.total_dups) + " pairs, capacity " +
                                         std::to_string(h.dup_capacity));
    return LF_OK;
}

lf_status lf_mpi_tile_lists(const void* ws, int32_t* order, int64_t n, int32_t* tile_prims, int64_t cap,
                            int32_t* seg, int64_t* n_pairs)
{
    int64_t needed = 0, M = 0;
    lf_status st = lf_mpi_status(ws, &needed, &M);
    if (st != LF_OK) return st;
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return check_launch("header read");
    BuildWs w;
    build_ws_layout(h.n, h.N, h.W, h.H, h.dup_capacity, const_cast<void*>(ws), &w);
    std::vector<uint32_t> rank_prim((size_t)(M > 0 ? M : 1));
    if (M > 0 && cudaMemcpy(rank_prim.data(), w.valA, sizeof(uint32_t) * (size_t)M, cudaMemcpyDeviceToHost) !=
                     cudaSuccess)
        return check_launch("order read");
    if (order) {
        if (n < M) return fail(LF_ERR_INVALID_ARG, "order buffer too small");
        std::memcpy(order, rank_prim.data(), sizeof(uint32_t) * (size_t)M);
    }
    if (!tile_prims && !seg && !n_pairs) return LF_OK;
    // device lists are per (super-tile, chunk); filter them per 16x16 tile on
    // the host with the footprint rectangles, keeping their (depth) order
    const int n_supers = h.supers_x * h.supers_y;
    std::vector<int2> sseg((size_t)n_supers * h.N);
    std::vector<uint32_t> sranks((size_t)(needed > 0 ? needed : 1));
    std::vector<int4> rrect((size_t)(M > 0 ? M : 1));
    const uint32_t* dranks = tile_sort_passes(tile_bits_for(n_supers)) % 2 ? w.entB : w.entA;
    if (cudaMemcpy(sseg.data(), w.seg, sizeof(int2) * sseg.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (needed > 0 &&
         cudaMemcpy(sranks.data(), dranks, sizeof(uint32_t) * (size_t)needed, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (M > 0 && cudaMemcpy(rrect.data(), w.r_rect, sizeof(int4) * (size_t)M, cudaMemcpyDeviceToHost) != cudaSuccess))
        return check_launch("tile list read");
    int64_t total = 0;
    for (int ty = 0; ty < h.tiles_y; ++ty)
        for (int tx = 0; tx < h.tiles_x; ++tx) {
            const int s = (ty / kTilesPerSuper) * h.supers_x + tx / kTilesPerSuper;
            const int x0 = tx * kTile, x1 = x0 + kTile - 1, y0 = ty * kTile, y1 = y0 + kTile - 1;
            for (int c = 0; c < h.N; ++c) {
                const int2 r = sseg[(size_t)s * h.N + c];
                const int64_t start = total;
                for (int i = r.x; i < r.y; ++i) {
                    const uint32_t rk = sranks[(size_t)i];
                    if (rk >= (uint64_t)M) return fail(LF_ERR_CUDA, "corrupt tile list entry");
                    const int4 q = rrect[rk];
                    if (q.x > x1 || q.z < x0 || q.y > y1 || q.w < y0) continue;
                    if (tile_prims) {
                        if (total >= cap) return fail(LF_ERR_INVALID_ARG, "tile list buffer too small");
                        tile_prims[total] = (int32_t)rank_prim[rk];
                    }
                    ++total;
                }
                if (seg) {
                    const size_t t = ((size_t)ty * h.tiles_x + tx) * h.N + c;
                    seg[2 * t] = (int32_t)start;
                    seg[2 * t + 1] = (int32_t)total;
                }
            }
        }
    if (n_pairs) *n_pairs = total;
    return LF_OK;
}

lf_status lf_filter_planes(const lf_planes* planes, double sigma, int32_t radius, cudaStream_t stream)
{
    if (!planes || !planes->rgba) return fail(LF_ERR_INVALID_ARG, "planes is NULL");
    if (planes->N < 1 || planes->W < 1 || planes->H < 1) return fail(LF_ERR_INVALID_ARG, "empty plane array");
    if (planes->dtype < LF_F32 || planes->dtype > LF_U8) return fail(LF_ERR_INVALID_ARG, "unknown plane dtype");
    if (!(sigma > 0.0)) return fail(LF_ERR_INVALID_ARG, "filter sigma must be positive");
    if (radius <= 0) radius = (int32_t)std::ceil(3.0 * sigma);
    if (radius > kFilterMaxRadius) return fail(LF_ERR_INVALID_ARG, "filter radius above 16");
    FilterParams f;
    std::memset(&f, 0, sizeof(f));
    f.radius = radius;
    // normalised FP64 Gaussian weights, rounded once to FP32
    double w[2 * kFilterMaxRadius + 1], sum = 0.0;
    for (int i = -radius; i <= radius; ++i) {
        w[i + radius] = std::exp(-0.5 * (double)i * (double)i / (sigma * sigma));
        sum += w[i + radius];
    }
    for (int i = 0; i <= 2 * radius; ++i) f.w[i] = (float)(w[i] / sum);
    trace_begin("plane_filter", stream);
    launch_filter_planes(planes->rgba, planes->dtype, planes->N, planes->W, planes->H, f, stream);
    trace_end(stream);
    return check_launch("plane filter");
}

size_t lf_composite_workspace_size(int32_t N, const lf_view_set* views)
{
    if (!views || N < 1 || views->Vx < 1 || views->Vy < 1) return 0;
    return comp_ws_layout(N, views->Vx, views->Vy, nullptr, nullptr);
}

lf_status lf_composite(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views, float* out,
                       void* ws, size_t ws_bytes, cudaStream_t stream)
{
    CompWs cw;
    lf_status st = check_composite_args(planes, ref, views, out, ws, ws_bytes, &cw);
    if (st != LF_OK) return st;
    CompParams p;
    fill_comp_params(planes, ref, views, &p);
    if (cudaMemsetAsync(cw.err, 0, sizeof(int) * (1 + (size_t)planes->N), stream) != cudaSuccess)
        return check_launch("composite reset");
    trace_begin("comp_coeffs", stream);
    launch_comp_coeffs(p, planes->d, planes->count, cw, stream);
    trace_end(stream);
    if ((st = check_launch("composite coefficients")) != LF_OK) return st;
    trace_begin("composite", stream);
    launch_composite(p, planes->rgba, planes->count, cw, out, stream);
    trace_end(stream);
    return check_launch("composite");
}

size_t lf_composite_state_size(const lf_ref_camera* ref, const lf_view_set* views)
{
    if (!ref || !views || views->Vx < 1 || views->Vy < 1 || ref->base.Nx < 1 || ref->base.Ny < 1) return 0;
    return (size_t)16 * views->Vx * views->Vy * ref->base.Nx * ref->base.Ny;
}

// after check_composite_args (ref and views valid)
static lf_status check_state(const lf_ref_camera* ref, const lf_view_set* views, const void* state,
                             size_t state_bytes)
{
    if (!state) return fail(LF_ERR_INVALID_ARG, "state is NULL");
    if (((uintptr_t)state) % 16) return fail(LF_ERR_INVALID_ARG, "state must be 16-byte aligned");
    if (state_bytes < lf_composite_state_size(ref, views))
        return fail(LF_ERR_INVALID_ARG, "state is smaller than lf_composite_state_size(ref, views)");
    return LF_OK;
}

lf_status lf_composite_save(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views, float* out,
                            float* state, size_t state_bytes, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    CompWs cw;
    lf_status st = check_composite_args(planes, ref, views, out, ws, ws_bytes, &cw);
    if (st != LF_OK) return st;
    if ((st = check_state(ref, views, state, state_bytes)) != LF_OK) return st;
    CompParams p;
    fill_comp_params(planes, ref, views, &p);
    if (cudaMemsetAsync(cw.err, 0, sizeof(int) * (1 + (size_t)planes->N), stream) != cudaSuccess)
        return check_launch("composite reset");
    trace_begin("comp_coeffs", stream);
    launch_comp_coeffs(p, planes->d, planes->count, cw, stream);
    trace_end(stream);
    if ((st = check_launch("composite coefficients")) != LF_OK) return st;
    trace_begin("composite_save", stream);
    launch_composite(p, planes->rgba, planes->count, cw, out, stream, reinterpret_cast<float4*>(state));
    trace_end(stream);
    return check_launch("composite (saving form)");
}

// state: NULL (two walks) or the saving forward's state
static lf_status composite_backward_impl(const lf_planes* planes, const lf_ref_camera* ref,
                                         const lf_view_set* views, const float* dviews, const float* state,
                                         size_t state_bytes, float* dplanes, void* ws, size_t ws_bytes,
                                         cudaStream_t stream)
{
    CompWs cw;
    lf_status st = check_composite_args(planes, ref, views, dviews, ws, ws_bytes, &cw);
    if (st != LF_OK) return st;
    if (state && (st = check_state(ref, views, state, state_bytes)) != LF_OK) return st;
    if (!dplanes) return fail(LF_ERR_INVALID_ARG, "dplanes is NULL");
    if (views->atlas_cols > 0) return fail(LF_ERR_UNSUPPORTED, "the composite adjoint takes separate views only");
    if (((uintptr_t)dviews) % 16 || ((uintptr_t)dplanes) % 16)
        return fail(LF_ERR_INVALID_ARG, "dviews and dplanes must be 16-byte aligned");
    CompParams p;
    fill_comp_params(planes, ref, views, &p);
    const size_t dbytes = sizeof(float) * 4 * (size_t)planes->N * planes->W * planes->H;
    if (cudaMemsetAsync(dplanes, 0, dbytes, stream) != cudaSuccess ||
        cudaMemsetAsync(cw.err, 0, sizeof(int) * (1 + (size_t)planes->N), stream) != cudaSuccess)
        return check_launch("composite backward reset");
    trace_begin("comp_coeffs", stream);
    launch_comp_coeffs(p, planes->d, planes->count, cw, stream);
    trace_end(stream);
    if ((st = check_launch("composite coefficients")) != LF_OK) return st;
    trace_begin(state ? "composite_bwd_saved" : "composite_bwd", stream);
    launch_composite_bwd(p, planes->rgba, planes->count, cw, dviews, dplanes, stream,
                         reinterpret_cast<const float4*>(state));
    trace_end(stream);
    return check_launch("composite backward");
}

lf_status lf_composite_backward(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                                const float* dviews, float* dplanes, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    return composite_backward_impl(planes, ref, views, dviews, nullptr, 0, dplanes, ws, ws_bytes, stream);
}

lf_status lf_composite_backward_saved(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                                      const float* dviews, const float* state, size_t state_bytes, float* dplanes,
                                      void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!state) return fail(LF_ERR_INVALID_ARG, "state is NULL");
    return composite_backward_impl(planes, ref, views, dviews, state, state_bytes, dplanes, ws, ws_bytes, stream);
}

// Common part of the two splat adjoints: argument checks, the forward's
// workspace layout, zeroing of the gradient accumulators and the raster
// adjoint. Returns the layout in *w.
static lf_status splat_backward_common(int64_t n, const lf_ref_camera* ref, const lf_planes* planes,
                                       const float* dplanes, void* ws, size_t ws_bytes, int kind, BuildWs* w,
                                       cudaStream_t stream)
{
    lf_status st = check_ref(ref);
    if (st != LF_OK) return st;
    if (!planes || !dplanes) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (planes->N < 1 || planes->N > 65535 || planes->W != ref->W || planes->H != ref->H)
        return fail(LF_ERR_INVALID_ARG, "plane array shape does not match the reference camera");
    if (((uintptr_t)dplanes) % 16) return fail(LF_ERR_INVALID_ARG, "dplanes must be 16-byte aligned");
    if (planes->dtype < LF_F32 || planes->dtype > LF_U8) return fail(LF_ERR_INVALID_ARG, "unknown plane dtype");
    // the adjoints read FP32 texels (C_end, 1 - T_end) of the forward
    if (planes->dtype == LF_F32 && (!planes->rgba || ((uintptr_t)planes->rgba) % 16))
        return fail(LF_ERR_INVALID_ARG, "FP32 planes->rgba must be non-NULL and 16-byte aligned");
    if (n < 0 || n > (int64_t)0x7fffffff) return fail(LF_ERR_INVALID_ARG, "primitive count out of range");
    if (!ws) return fail(LF_ERR_WORKSPACE, "workspace is NULL");
    if (((uintptr_t)ws) % 256) return fail(LF_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    const int64_t cap = ws_capacity(n, planes->N, ref->W, ref->H, ws_bytes);
    if (cap < 1) return fail(LF_ERR_WORKSPACE, "workspace too small for these primitives and planes");
    build_ws_layout(n, planes->N, ref->W, ref->H, cap, ws, w);
    if (n > 0 && cudaMemsetAsync(w->g2d, 0, sizeof(float) * 12 * (size_t)n, stream) != cudaSuccess)
        return check_launch("gradient accumulator reset");
    RasterParams rp;
    fill_raster_params(ref, planes->N, planes->dtype, &rp);
    const int n_supers = ((ref->W + kSuper - 1) / kSuper) * ((ref->H + kSuper - 1) / kSuper);
    const uint32_t* ranks = tile_sort_passes(tile_bits_for(n_supers)) % 2 ? w->entB : w->entA;
    trace_begin(kind == 0 ? "raster_gaussians_bwd" : "raster_voxels_bwd", stream);
    if (kind == 0)
        launch_raster_gaussians_bwd(*w, rp, ranks, planes->rgba, dplanes, stream);
    else
        launch_raster_voxels_bwd(*w, rp, ranks, planes->rgba, dplanes, stream);
    trace_end(stream);
    return check_launch("raster backward");
}

lf_status lf_build_mpi_backward_gaussians(const lf_gaussians* g, const lf_ref_camera* ref, const lf_planes* planes,
                                          const float* dplanes, lf_gaussians_grad* grad, void* ws, size_t ws_bytes,
                                          cudaStream_t stream)
{
    if (!g || !grad) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacity || !g->rgb))
        return fail(LF_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
    if (g->n > 0 && (!grad->dmeans || !grad->dscales || !grad->dquats || !grad->dopacity || !grad->drgb))
        return fail(LF_ERR_INVALID_ARG, "a gradient pointer is NULL");
    BuildWs w;
    lf_status st = splat_backward_common(g->n, ref, planes, dplanes, ws, ws_bytes, 0, &w, stream);
    if (st != LF_OK) return st;
    const size_t n = (size_t)g->n;
    if (n > 0) {
        const float* bufs[5] = {grad->dmeans, grad->dscales, grad->dquats, grad->dopacity, grad->drgb};
        const size_t widths[5] = {3, 3, 4, 1, 3};
        for (int b = 0; b < 5; ++b)
            if (cudaMemsetAsync(const_cast<float*>(bufs[b]), 0, sizeof(float) * widths[b] * n, stream) != cudaSuccess)
                return check_launch("gradient reset");
    }
    ProjParams pp;
    fill_proj_params(ref, g->n, &pp);
    trace_begin("project_bwd", stream);
    launch_gauss_chain(*g, pp, w, *grad, stream);
    trace_end(stream);
    return check_launch("projection backward");
}

lf_status lf_build_mpi_backward_voxels(const lf_voxels* v, const lf_ref_camera* ref, const lf_planes* planes,
                                       const float* dplanes, lf_voxels_grad* grad, void* ws, size_t ws_bytes,
                                       cudaStream_t stream)
{
    if (!v || !grad) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (v->n > 0 && (!grad->ddensity8 || !grad->drgb)) return fail(LF_ERR_INVALID_ARG, "a gradient pointer is NULL");
    BuildWs w;
    lf_status st = splat_backward_common(v->n, ref, planes, dplanes, ws, ws_bytes, 1, &w, stream);
    if (st != LF_OK) return st;
    const size_t n = (size_t)v->n;
    if (n > 0 && (cudaMemsetAsync(grad->ddensity8, 0, sizeof(float) * 8 * n, stream) != cudaSuccess ||
                  cudaMemsetAsync(grad->drgb, 0, sizeof(float) * 3 * n, stream) != cudaSuccess))
        return check_launch("gradient reset");
    trace_begin("scatter_bwd", stream);
    launch_voxel_scatter(w, v->n, *grad, stream);
    trace_end(stream);
    return check_launch("voxel gradient scatter");
}

// ---------------------------------------------------------------------------
// Allocation-free composite. The paper has no counterpart; this is a
// deployment form of lf_composite for callers that cannot hand the library a
// device buffer: e.g. a display runtime's per-frame present callback, which
// must not call into a device allocator (allocation can synchronise the
// device and stall the frame) and owns no workspace of its own. Its scratch
// (the per-(view, plane) coefficient tables, the error word and the
// wide-shift flags) lives in the file-scope device array below instead of a
// caller workspace. The error word and the flags must be zero before the
// composite kernel reads them; every call zeroes them on its stream first.
// Calls that overlap in time (two streams, or two host threads) share this
// one array and race; the caller serialises them.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace lf {
constexpr size_t kStaticCompBytes = 1u << 20;   // 1 MiB: e.g. N = 512 planes x 128 views
static __device__ __align__(256) unsigned char g_comp_scratch[kStaticCompBytes];

// Device address of g_comp_scratch on the calling thread's current device.
// In host code the array's name is only a host-side stand-in, so every call
// asks the runtime for the address (no allocation, and no address cached
// across a device reset that could move the module).
static lf_status static_scratch(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_comp_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(LF_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                     cudaGetErrorString(e));
    }
    *out = p;
    return LF_OK;
}
}  // namespace lf

extern "C" {

size_t lf_composite_noalloc_max_bytes(void) { return lf::kStaticCompBytes; }

lf_status lf_composite_noalloc(const lf_planes* planes, const lf_ref_camera* ref, const lf_view_set* views,
                               float* out, cudaStream_t stream)
{
    if (!planes || !views) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (planes->N < 1 || views->Vx < 1 || views->Vy < 1 || views->Vx > 65535 || views->Vy > 65535)
        return fail(LF_ERR_INVALID_ARG, "N and view counts must be positive");
    const size_t need = comp_ws_layout(planes->N, views->Vx, views->Vy, nullptr, nullptr);
    if (need > lf::kStaticCompBytes)
        return fail(LF_ERR_WORKSPACE, "lf_composite_noalloc: N = " + std::to_string(planes->N) + " planes and " +
                                          std::to_string(views->Vx) + " x " + std::to_string(views->Vy) +
                                          " views need " + std::to_string(need) + " scratch bytes, above its " +
                                          std::to_string(lf::kStaticCompBytes) + "-byte static limit; use lf_composite");
    void* scratch = nullptr;
    lf_status st = lf::static_scratch(&scratch);
    if (st != LF_OK) return st;
    CompWs cw;
    st = check_composite_args(planes, ref, views, out, scratch, lf::kStaticCompBytes, &cw);
    if (st != LF_OK) return st;
    CompParams p;
    fill_comp_params(planes, ref, views, &p);
    if (cudaMemsetAsync(cw.err, 0, sizeof(int) * (1 + (size_t)planes->N), stream) != cudaSuccess)
        return check_launch("composite reset");
    trace_begin("comp_coeffs", stream);
    launch_comp_coeffs(p, planes->d, planes->count, cw, stream);
    trace_end(stream);
    if ((st = check_launch("composite coefficients")) != LF_OK) return st;
    trace_begin("composite", stream);
    launch_composite(p, planes->rgba, planes->count, cw, out, stream);
    trace_end(stream);
    return check_launch("composite");
}

lf_status lf_composite_noalloc_status(int32_t N, const lf_view_set* views, cudaStream_t stream)
{
    if (!views || N < 1 || views->Vx < 1 || views->Vy < 1) return fail(LF_ERR_INVALID_ARG, "bad argument");
    if (comp_ws_layout(N, views->Vx, views->Vy, nullptr, nullptr) > lf::kStaticCompBytes)
        return fail(LF_ERR_INVALID_ARG, "N and views exceed what lf_composite_noalloc accepts");
    void* scratch = nullptr;
    const lf_status st = lf::static_scratch(&scratch);
    if (st != LF_OK) return st;
    return lf_composite_status(N, views, scratch, stream);
}

}  // extern "C"
