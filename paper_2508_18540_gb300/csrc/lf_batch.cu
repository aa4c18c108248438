// lf_batch.cu -- several G2LF scenes in one frame: per-scene builds up to the
// tile lists, then one persistent raster launch and one persistent staged
// composite launch over the work items of every scene (schedules 0 and 1),
// or every scene's own pipeline on a stream of its own, forked from and
// joined back into the caller's stream (schedule 2); CUDA-graph capture of
// the whole frame, and an autotuner over the launch plan.
//
// The method itself (Algorithm 1 per scene) is unchanged: a plan only
// changes how items are grouped and scheduled, never what is computed, so
// every plan gives identical planes and views.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "lf_internal.cuh"

using namespace lf;

struct lf_batch {
    std::vector<lf_batch_scene> sc;
    lf_batch_plan plan{9, 512, 1, 1};
    int dtype = LF_F32;
    int bilinear = 0;
    bool prepared = false;
    // device tables in the caller's batch workspace
    unsigned long long* counters = nullptr;   // [2]: raster, composite item counters
    RasterScene* rtab = nullptr;
    CompScene* ctab = nullptr;
    // host copies (kept alive: the uploads read them)
    std::vector<RasterScene> rhost;
    std::vector<CompScene> chost;
    long long r_heavy = 0, r_total = 0, c_total = 0;   // raster grid: split-part CTAs, all CTAs
    size_t max_stage = 0;
    int maxN = 0;
    int c_ctas = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;              // kernels in one launch of the graph
    // schedule 2: one stream per scene, a fork event and a join event per scene
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

size_t batch_tables_bytes(int n)
{
    return align256(16) + align256(sizeof(RasterScene) * n) + align256(sizeof(CompScene) * n);
}

// bytes of one scene's chunk-group partials (groups 1 .. groups - 1)
size_t scene_part_bytes(const lf_batch_scene& s, int groups)
{
    if (groups <= 1) return 0;
    return align256((size_t)(groups - 1) * s.views.Vx * s.views.Vy * s.ref.base.Nx * s.ref.base.Ny * sizeof(float4));
}

size_t batch_ws_bytes(const lf_batch* b, int groups)
{
    size_t t = batch_tables_bytes((int)b->sc.size());
    for (const lf_batch_scene& s : b->sc) t += scene_part_bytes(s, groups);
    return t;
}

bool plan_valid(const lf_batch_plan& pl)
{
    return (pl.views_per_thread == 3 || pl.views_per_thread == 5 || pl.views_per_thread == 9 ||
            pl.views_per_thread == 15) &&
           (pl.tile_x == 128 || pl.tile_x == 256 || pl.tile_x == 512) &&
           (pl.chunk_groups == 1 || pl.chunk_groups == 2 || pl.chunk_groups == kMaxChunkGroups) &&
           pl.schedule >= 0 && pl.schedule <= 2;
}

lf_status check_scene(const lf_batch_scene& s, int i)
{
    const std::string at = "batch scene " + std::to_string(i) + ": ";
    if (s.g.n < 0 || (s.g.n > 0 && (!s.g.means || !s.g.scales || !s.g.quats || !s.g.opacity || !s.g.rgb)))
        return fail(LF_ERR_INVALID_ARG, at + "bad Gaussian arrays");
    if (s.N < 1 || s.N > 65535) return fail(LF_ERR_INVALID_ARG, at + "N must be in 1..65535");
    if (s.planes.N != s.N || s.planes.W != s.ref.W || s.planes.H != s.ref.H)
        return fail(LF_ERR_INVALID_ARG, at + "plane array shape does not match N / reference camera");
    if (!s.planes.rgba || !s.planes.d || !s.planes.count || !s.planes.chunk || !s.planes.rect || !s.out)
        return fail(LF_ERR_INVALID_ARG, at + "NULL plane or view pointer");
    if (!s.ws || !s.cws || ((uintptr_t)s.ws) % 256 || ((uintptr_t)s.cws) % 256)
        return fail(LF_ERR_WORKSPACE, at + "workspaces must be non-NULL and 256-byte aligned");
    const int tb = texel_bytes(s.planes.dtype);
    if (((size_t)s.ref.W * tb) % 16 || ((uintptr_t)s.planes.rgba) % 16)
        return fail(LF_ERR_UNSUPPORTED, at + "plane rows must be 16-byte multiples on a 16-byte aligned base");
    return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_batch_create(const lf_batch_scene* scenes, int32_t n_scenes, lf_batch** out)
{
    if (!scenes || !out || n_scenes < 1 || n_scenes > 4096)
        return fail(LF_ERR_INVALID_ARG, "lf_batch_create: need 1..4096 scenes and an output pointer");
    for (int i = 0; i < n_scenes; ++i) {
        const lf_status st = check_scene(scenes[i], i);
        if (st != LF_OK) return st;
        if (scenes[i].binning & LF_BLEND_3DGS)
            return fail(LF_ERR_UNSUPPORTED, "lf_batch_create: batches blend in exact mode only");
        if (scenes[i].planes.dtype != scenes[0].planes.dtype || (scenes[i].views.bilinear != 0) !=
                                                                    (scenes[0].views.bilinear != 0))
            return fail(LF_ERR_INVALID_ARG, "lf_batch_create: scenes must share plane dtype and sampling");
    }
    lf_batch* b = new lf_batch;
    b->sc.assign(scenes, scenes + n_scenes);
    b->dtype = scenes[0].planes.dtype;
    b->bilinear = scenes[0].views.bilinear ? 1 : 0;
    *out = b;
    return LF_OK;
}

size_t lf_batch_workspace_size(const lf_batch* b) { return b ? batch_ws_bytes(b, 1) : 0; }

size_t lf_batch_plan_workspace_size(const lf_batch* b, const lf_batch_plan* plan)
{
    if (!b) return 0;
    const lf_batch_plan pl = plan ? *plan : lf_batch_plan{9, 512, 1, 1};
    if (!plan_valid(pl)) return 0;
    return batch_ws_bytes(b, pl.schedule == 2 ? 1 : pl.chunk_groups);
}

lf_status lf_batch_prepare(lf_batch* b, const lf_batch_plan* plan, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!b) return fail(LF_ERR_INVALID_ARG, "batch is NULL");
    const lf_batch_plan pl = plan ? *plan : lf_batch_plan{9, 512, 1, 1};
    if (!plan_valid(pl)) return fail(LF_ERR_INVALID_ARG, "lf_batch_prepare: plan out of range");
    const int groups = pl.schedule == 2 ? 1 : pl.chunk_groups;
    if (pl.schedule == 2 && b->side.empty()) {
        b->side.resize(b->sc.size(), nullptr);
        b->done.resize(b->sc.size(), nullptr);
        if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
            return check_launch("batch fork event");
        for (size_t i = 0; i < b->sc.size(); ++i)
            if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess)
                return check_launch("batch scene streams");
    }
    const int n = (int)b->sc.size();
    if (!ws || ((uintptr_t)ws) % 256) return fail(LF_ERR_WORKSPACE, "batch workspace NULL or not 256-byte aligned");
    if (ws_bytes < batch_ws_bytes(b, groups))
        return fail(LF_ERR_WORKSPACE, "batch workspace too small for this plan (lf_batch_plan_workspace_size)");
    char* base = static_cast<char*>(ws);
    b->counters = reinterpret_cast<unsigned long long*>(base);
    b->rtab = reinterpret_cast<RasterScene*>(base + align256(16));
    b->ctab = reinterpret_cast<CompScene*>(base + align256(16) + align256(sizeof(RasterScene) * n));

    const int tb = texel_bytes(b->dtype);
    std::vector<RasterScene> r(n);
    std::vector<CompScene> c(n);
    std::vector<double> rwork(n), cwork(n);
    size_t max_stage = 0;
    int maxN = 0;
    for (int i = 0; i < n; ++i) {
        lf_batch_scene& s = b->sc[i];
        const int64_t cap = ws_capacity(s.g.n, s.N, s.ref.W, s.ref.H, s.ws_bytes);
        if (cap < 1) return fail(LF_ERR_WORKSPACE, "batch scene " + std::to_string(i) + ": build workspace too small");
        build_ws_layout(s.g.n, s.N, s.ref.W, s.ref.H, cap, s.ws, &r[i].w);
        raster_params(&s.ref, s.N, s.planes.dtype, &r[i].p);
        const int n_supers = ((s.ref.W + kSuper - 1) / kSuper) * ((s.ref.H + kSuper - 1) / kSuper);
        r[i].ranks = tile_sort_passes(tile_bits_for(n_supers)) % 2 ? r[i].w.entB : r[i].w.entA;
        r[i].planes = s.planes.rgba;
        rwork[i] = (double)s.g.n;

        CompWs cw;
        CompParams cp;
        const lf_status st = composite_args(&s.planes, &s.ref, &s.views, s.out, s.cws, s.cws_bytes, &cw, &cp);
        if (st != LF_OK) return st;
        c[i].p = cp;
        c[i].G = staged_geom(cp, tb, b->bilinear != 0, pl.views_per_thread, pl.tile_x);
        c[i].planes = static_cast<const char*>(s.planes.rgba);
        c[i].count = s.planes.count;
        c[i].w = cw;
        c[i].out = s.out;
        c[i].nby = (cp.Ny + c[i].G.BY - 1) / c[i].G.BY;
        c[i].nbz = (cp.Nx + c[i].G.TX - 1) / c[i].G.TX;
        c[i].groups = groups;
        c[i].part = nullptr;
        cwork[i] = (double)cp.Vx * cp.Vy * cp.Nx * cp.Ny * cp.N;
        max_stage = std::max(max_stage, c[i].G.stage_bytes);
        maxN = std::max(maxN, s.N);
    }
    if (pl.schedule != 2 && composite_batched_smem(max_stage, maxN, pl.views_per_thread) > 200 * 1024)
        return fail(LF_ERR_UNSUPPORTED, "lf_batch_prepare: the batch's largest plane row and N need more than "
                                        "200 KB of shared memory for the staged composite");
    // schedule: order of the scenes in the item tables
    std::vector<int> ro(n), co(n);
    for (int i = 0; i < n; ++i) ro[i] = co[i] = i;
    if (pl.schedule == 1) {
        std::stable_sort(ro.begin(), ro.end(), [&](int a, int bb) { return rwork[a] > rwork[bb]; });
        std::stable_sort(co.begin(), co.end(), [&](int a, int bb) { return cwork[a] > cwork[bb]; });
    }
    b->rhost.resize(n);
    b->chost.resize(n);
    long long ct = 0, hb = 0, lb = 0;
    for (int q = 0; q < n; ++q) {
        RasterScene R = r[ro[q]];
        R.pbase = hb;
        hb += raster_part_ctas(R.w);
        b->rhost[q] = R;
        CompScene C = c[co[q]];
        C.base = ct;
        ct += (long long)C.G.groups_x * C.p.Vy * C.nby * C.nbz * C.groups;
        b->chost[q] = C;
    }
    for (int q = 0; q < n; ++q) {
        b->rhost[q].lbase = hb + lb;
        lb += (long long)b->rhost[q].p.supers_x * b->rhost[q].p.supers_y * b->rhost[q].p.N;
    }
    b->r_heavy = hb;
    b->r_total = hb + lb;
    b->c_total = ct;
    {
        char* part = base + batch_tables_bytes(n);
        for (int q = 0; q < n; ++q) {
            if (groups > 1) {
                const lf_batch_scene& sc = b->sc[co[q]];
                b->chost[q].part = reinterpret_cast<float4*>(part);
                part += scene_part_bytes(sc, groups);
            }
        }
    }
    b->max_stage = max_stage;
    b->maxN = maxN;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return check_launch("device query");
    const size_t smem = composite_batched_smem(max_stage, maxN, pl.views_per_thread);
    // CTAs per SM: the composite's launch bounds aim at four (views per
    // thread up to kTwoCtaViews) or two, as shared memory allows
    int per_sm = pl.views_per_thread <= kTwoCtaViews ? 4 : 2;
    while (per_sm > 1 && (size_t)per_sm * (smem + 1024) > (size_t)228 * 1024) --per_sm;
    b->c_ctas = sms * per_sm;
    if (cudaMemcpyAsync(b->rtab, b->rhost.data(), sizeof(RasterScene) * n, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->ctab, b->chost.data(), sizeof(CompScene) * n, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
        return check_launch("batch table upload");
    // the uploads read host memory that later prepares overwrite
    if (cudaStreamSynchronize(stream) != cudaSuccess) return check_launch("batch table upload");
    b->plan = pl;
    b->prepared = true;
    return LF_OK;
}

lf_status lf_batch_render(lf_batch* b, cudaStream_t stream)
{
    if (!b || !b->prepared) return fail(LF_ERR_INVALID_ARG, "batch not prepared");
    lf_status st;
    if (b->plan.schedule == 2) {
        // every scene's single-scene pipeline on its own stream, all forked
        // from and joined back into stream (captured as parallel branches)
        if (cudaEventRecord(b->fork, stream) != cudaSuccess) return check_launch("batch fork");
        for (size_t i = 0; i < b->sc.size(); ++i) {
            lf_batch_scene& s = b->sc[i];
            if (cudaStreamWaitEvent(b->side[i], b->fork, 0) != cudaSuccess) return check_launch("batch fork");
            if ((st = lf_build_mpi_gaussians(&s.g, &s.ref, s.N, s.binning, s.ws, s.ws_bytes, &s.planes,
                                             b->side[i])) != LF_OK)
                return st;
            if ((st = lf_composite(&s.planes, &s.ref, &s.views, s.out, s.cws, s.cws_bytes, b->side[i])) != LF_OK)
                return st;
            if (cudaEventRecord(b->done[i], b->side[i]) != cudaSuccess ||
                cudaStreamWaitEvent(stream, b->done[i], 0) != cudaSuccess)
                return check_launch("batch join");
        }
        return LF_OK;
    }
    if (cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), stream) != cudaSuccess)
        return check_launch("batch counter reset");
    for (size_t i = 0; i < b->sc.size(); ++i) {
        lf_batch_scene& s = b->sc[i];
        BuildWs w;
        const uint32_t* ranks = nullptr;
        st = build_gaussians_prefix(&s.g, &s.ref, s.N, s.binning, s.ws, s.ws_bytes, &s.planes, stream, &w, &ranks);
        if (st != LF_OK) return st;
        RasterParams rp;
        raster_params(&s.ref, s.N, s.planes.dtype, &rp);
        launch_raster_plan(w, rp, false, stream);
    }
    trace_begin("raster_batched", stream);
    launch_raster_gauss_batched(b->rtab, (int)b->sc.size(), b->dtype, b->r_heavy, b->r_total, stream);
    trace_end(stream);
    if ((st = check_launch("batched raster")) != LF_OK) return st;
    trace_begin("comp_coeffs", stream);
    for (size_t i = 0; i < b->sc.size(); ++i) {
        lf_batch_scene& s = b->sc[i];
        CompWs cw;
        CompParams cp;
        if ((st = composite_args(&s.planes, &s.ref, &s.views, s.out, s.cws, s.cws_bytes, &cw, &cp)) != LF_OK)
            return st;
        if (cudaMemsetAsync(cw.err, 0, sizeof(int) * (1 + (size_t)cp.N), stream) != cudaSuccess)
            return check_launch("composite reset");
        launch_comp_coeffs(cp, s.planes.d, s.planes.count, cw, stream);
    }
    trace_end(stream);
    if ((st = check_launch("batched coefficients")) != LF_OK) return st;
    trace_begin("composite_batched", stream);
    const bool ok = launch_composite_batched(b->ctab, (int)b->sc.size(), b->c_total, b->dtype, b->bilinear != 0,
                                             b->plan.views_per_thread, b->max_stage, b->maxN, b->counters + 1,
                                             b->c_ctas, stream);
    trace_end(stream);
    if (!ok) return fail(LF_ERR_UNSUPPORTED, "batched composite layout does not fit shared memory");
    if ((st = check_launch("batched composite")) != LF_OK) return st;
    if (b->plan.chunk_groups > 1) {
        trace_begin("merge_chunk_groups", stream);
        for (const CompScene& C : b->chost) launch_merge_chunk_groups(C.p, C.groups, C.part, C.out, stream);
        trace_end(stream);
        return check_launch("chunk-group merge");
    }
    return LF_OK;
}

lf_status lf_batch_capture(lf_batch* b, cudaStream_t stream)
{
    if (!b || !b->prepared) return fail(LF_ERR_INVALID_ARG, "batch not prepared");
    if (stream == nullptr) return fail(LF_ERR_INVALID_ARG, "capture needs a non-default stream");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return check_launch("begin capture");
    const bool tr = trace_swap(false);
    const long long k0 = lf_launch_count();
    const lf_status st = lf_batch_render(b, stream);
    // captured kernels are not launched yet: count them per graph launch
    b->graph_kernels = lf_launch_count() - k0;
    note_launches((int)-b->graph_kernels);
    trace_swap(tr);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (st != LF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || !g) return check_launch("end capture");
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return check_launch("graph instantiate");
    }
    b->graph = g;
    return LF_OK;
}

lf_status lf_batch_launch(lf_batch* b, cudaStream_t stream)
{
    if (!b || !b->exec) return fail(LF_ERR_INVALID_ARG, "no captured batch graph");
    if (cudaGraphLaunch(b->exec, stream) != cudaSuccess) return check_launch("graph launch");
    note_launches((int)b->graph_kernels);
    return LF_OK;
}

lf_status lf_batch_autotune(lf_batch* b, void* ws, size_t ws_bytes, int32_t reps, cudaStream_t stream,
                            lf_batch_plan* best, float* best_ms)
{
    if (!b || !best) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    if (reps < 1) reps = 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return check_launch("events");
    auto time_plan = [&](const lf_batch_plan& pl, float* ms) -> lf_status {
        lf_status st = lf_batch_prepare(b, &pl, ws, ws_bytes, stream);
        if (st != LF_OK) return st;
        if ((st = lf_batch_render(b, stream)) != LF_OK) return st;   // warm-up
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps; ++r)
            if ((st = lf_batch_render(b, stream)) != LF_OK) return st;
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return check_launch("autotune timing");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        return LF_OK;
    };
    lf_batch_plan cur{9, 512, 1, 1};
    float cur_ms = 3.4e38f;
    lf_status st = LF_OK;
    const int vgs[4] = {3, 5, 9, 15}, txs[3] = {128, 256, 512};
    for (int a = 0; a < 4 && st == LF_OK; ++a)
        for (int c = 0; c < 3 && st == LF_OK; ++c) {
            lf_batch_plan pl{vgs[a], txs[c], cur.chunk_groups, cur.schedule};
            float ms = 0.f;
            st = time_plan(pl, &ms);
            if (st == LF_ERR_UNSUPPORTED) {   // layout too large for this plan: skip it
                st = LF_OK;
                continue;
            }
            if (st == LF_OK && ms < cur_ms) cur_ms = ms, cur = pl;
        }
    // chunk groups x scene order, for the composite layout found above; only
    // the group counts whose partial buffers fit the workspace
    lf_batch_plan comp = cur;
    const int gs[3] = {1, 2, kMaxChunkGroups};
    for (int gi = 0; gi < 3 && st == LF_OK; ++gi)
        for (int sch = 0; sch <= 1 && st == LF_OK; ++sch) {
            lf_batch_plan pl{comp.views_per_thread, comp.tile_x, gs[gi], sch};
            if (pl.chunk_groups == comp.chunk_groups && pl.schedule == comp.schedule) continue;
            if (batch_ws_bytes(b, pl.chunk_groups) > ws_bytes) continue;
            float ms = 0.f;
            st = time_plan(pl, &ms);
            if (st == LF_ERR_UNSUPPORTED) {
                st = LF_OK;
                continue;
            }
            if (st == LF_OK && ms < cur_ms) cur_ms = ms, cur = pl;
        }
    if (st == LF_OK) {   // concurrent single-scene pipelines
        lf_batch_plan pl{cur.views_per_thread, cur.tile_x, 1, 2};
        float ms = 0.f;
        st = time_plan(pl, &ms);
        if (st == LF_OK && ms < cur_ms) cur_ms = ms, cur = pl;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LF_OK) return st;
    if (cur_ms > 3.0e38f) return fail(LF_ERR_UNSUPPORTED, "no plan fits this batch");
    if ((st = lf_batch_prepare(b, &cur, ws, ws_bytes, stream)) != LF_OK) return st;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return LF_OK;
}

lf_status lf_batch_status(lf_batch* b, cudaStream_t stream)
{
    if (!b || !b->prepared) return fail(LF_ERR_INVALID_ARG, "batch not prepared");
    if (cudaStreamSynchronize(stream) != cudaSuccess) return check_launch("stream synchronise");
    for (size_t i = 0; i < b->sc.size(); ++i) {
        WsHeader h;
        int err = 0;
        if (cudaMemcpy(&h, b->sc[i].ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
            return check_launch("header read");
        if (h.overflow)
            return fail(LF_ERR_OVERFLOW, "batch scene " + std::to_string(i) + ": tile list needs " +
                                             std::to_string(h.total_dups) + " pairs, capacity " +
                                             std::to_string(h.dup_capacity));
        CompWs cw;
        comp_ws_layout(b->sc[i].N, b->sc[i].views.Vx, b->sc[i].views.Vy, b->sc[i].cws, &cw);
        if (cudaMemcpy(&err, cw.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return check_launch("error word read");
        if (err) return fail(LF_ERR_TIMEOUT, "batch scene " + std::to_string(i) + ": a composite wait gave up");
    }
    return LF_OK;
}

lf_status lf_batch_destroy(lf_batch* b)
{
    if (!b) return LF_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->side)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return LF_OK;
}

}  // extern "C"
