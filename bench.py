"""Benchmark: light-field frames/s of the G2LF hot path on the display-scale
workload (1M anisotropic Gaussians in 200 blobs, 512x512 reference planes,
N_chunk = 64 quantile planes, 45 views over +-0.15), one step = one LF frame:
lf_build_mpi_gaussians (project, depth sort, bin, tile lists, rasterise)
+ lf_composite (45 views), all inputs resident in HBM.

Prints one JSON line (rank 0). FP32 planes are the primary number; FP16,
BF16 and RGBA8 planes are reported beside it, each with the roofline of its
two dominant kernels (composite against the measured HBM copy bandwidth,
raster against the FP32 issue rate at the sampled SM clock).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=1_000_000, res=512, N=64, V=45, seed=2)
METRIC = "LF frames/s (45 views, 512p, 1M Gaussians) FP16 vs FP32 planes; % HBM roofline"
UNIT = "LF frames/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FIT_TARGET_SEED = 6                 # perturbation of the fit's target scene


_VOXEL_WL = []


def _voxel_workload():
    """The 2M-voxel V2LF workload, generated once per process (both the GPU
    section and the oracle baseline use it)."""
    from paper_2508_18540_gb300 import synth as S
    if not _VOXEL_WL:
        _VOXEL_WL.append(S.workload_voxels())
    return _VOXEL_WL[0]


def _env_rank():
    from paper_2508_18540_gb300 import replicas
    return replicas.env_rank()


def _config(extra=None):
    c = {"workload": "g2lf_display_1M_512px_N64_45v",
         "gaussians": WORKLOAD["n"], "plane_res": [WORKLOAD["res"], WORKLOAD["res"]],
         "view_res": [WORKLOAD["res"], WORKLOAD["res"]], "N_chunk": WORKLOAD["N"], "views": WORKLOAD["V"],
         "binning": "quantile", "sampling": "nearest", "P_s": 1,
         "l2": "flushed between timed steps (512 MB write)"}
    if extra:
        c.update(extra)
    return c


# DRAM bytes (read + write) per launch from one ncu capture of the f32 frame
# (profiles/k_*_g2lf_display_1M_512px_N64_45v.md), valid only while the
# kernel's sources (their code, comments aside) hash to the value recorded
# with them.
NCU_TRAFFIC = {
    # the raster stage's two kernels: the parts of split lists and the lists
    "raster_gaussians": (11_979_008 + 0 + 71_470_848 + 204_340_480, ("lf_raster.cu", "lf_internal.cuh"),
                         "3e0cef0f8f9d1f2b"),
    "composite": (252_981_760 + 156_500_736, ("lf_composite.cu", "lf_internal.cuh"), "d93198e445d327bc"),
}


def _code_only(src):
    """C/CUDA source without its comments and with whitespace runs collapsed
    (string and character literals kept verbatim): what the compiler sees."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _source_hash(files):
    import hashlib
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2508_18540_gb300", "csrc", f)) as fh:
            m.update(_code_only(fh.read()).encode())
    return m.hexdigest()[:16]


def _traffic(kernel):
    ent = NCU_TRAFFIC.get(kernel)
    if ent is None:
        return None
    return ent[0] if _source_hash(ent[1]) == ent[2] else None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import replicas as R
    from paper_2508_18540_gb300 import synth as S

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # replicas: every rank renders its own frame stream of the same-sized workload
    wl = S.workload_display(seed=R.replica_seed(WORKLOAD["seed"], rank), n=WORKLOAD["n"], res=WORKLOAD["res"], N=WORKLOAD["N"],
                            V=WORKLOAD["V"])
    g = api.DeviceGaussians.from_scene(wl.scene, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        R.barrier(world, dev)

    def timed(renderer, steps, warmup, trace=False):
        for _ in range(warmup):
            renderer.render(g)
        st, needed, M = renderer.status()
        if st != 0:
            raise RuntimeError("build failed with status %d (pairs needed %d)" % (st, needed))
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if trace:
            api.lf_trace_collect()
            api.lf_trace_enable(True)
        l0 = api.lf_launch_count()
        for a, b in ev:
            flush.zero_()                  # L2 flush, outside the timed events
            a.record(stream)
            renderer.render(g)
            b.record(stream)
        launches = api.lf_launch_count() - l0
        barrier()
        if renderer.composite_status() != 0:
            raise RuntimeError("a bounded composite wait gave up during the timed frames")
        stages = {}
        if trace:
            api.lf_trace_enable(False)
            stages = api.lf_trace_collect()
        ms = R.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
        return ms / steps, launches // steps, stages

    res = {}
    clocks = ClockSampler(local)
    for dtype in ("f32", "f16", "bf16", "u8"):
        r = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, dtype, device=dev)
        ms, launches, stages = timed(r, args.steps, args.warmup, trace=True)
        res[dtype] = dict(ms=ms, launches=launches, stages=stages, renderer=r)
        if rank == 0 and world == 1:
            res[dtype]["views_host"] = r.out.cpu().numpy()

    # the same frames captured once into a CUDA graph and replayed (no launch
    # gaps between the frame's kernels); same timing rules
    def timed_graph(rr, steps, warmup):
        for _ in range(warmup):
            rr.replay()
        barrier()
        evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evg:
            flush.zero_()
            a.record(stream)
            rr.replay()
            b.record(stream)
        barrier()
        return R.max_over_ranks(sum(a.elapsed_time(b) for a, b in evg) / steps, world, dev)

    # a render loop with two frames in flight: two renderers (workspace,
    # planes, views each), one graph and one stream each, frames alternating;
    # K frames timed from the first frame's start to the last one's end (each
    # frame streams > 0.7 GB through the 129 MB L2, so no flush)
    pair_streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]

    def timed_in_flight(rr, steps, warmup):
        for i in range(2 * warmup):
            with torch.cuda.stream(pair_streams[i & 1]):
                rr[i & 1].replay()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(pair_streams[0])
        pair_streams[1].wait_event(e0)
        for i in range(steps):
            with torch.cuda.stream(pair_streams[i & 1]):
                rr[i & 1].replay()
        pair_streams[0].wait_stream(pair_streams[1])
        e1.record(pair_streams[0])
        e1.synchronize()
        barrier()
        return R.max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)

    r32 = res["f32"]["renderer"]
    graph_kernels = r32.capture(g)
    for d in res:
        r2 = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, d, device=dev)
        if d != "f32":
            res[d]["renderer"].capture(g)
        r2.capture(g)
        res[d]["pair"] = [res[d]["renderer"], r2]
    # the sampler runs from half a second of back-to-back replays (the GPU at
    # its working clock) through the end of the timed replays
    clocks.start()
    t_end = time.perf_counter() + 0.5
    while time.perf_counter() < t_end:
        for _ in range(50):
            r32.replay()
        torch.cuda.synchronize()
    g_ms = timed_graph(r32, args.steps, args.warmup)
    f_ms = timed_in_flight(res["f32"]["pair"], args.steps, args.warmup)
    clk = clocks.stop()
    clk["window"] = "0.5 s of back-to-back graph replays, then the timed replays"
    for d in ("f16", "bf16", "u8"):
        res[d]["graph_ms"] = timed_graph(res[d]["renderer"], args.steps, args.warmup)
        res[d]["flight_ms"] = timed_in_flight(res[d]["pair"], args.steps, args.warmup)
    for d in res:
        res[d]["pair"] = None

    # end to end through the public API with host buffers (pinned), f32 planes
    host_in = api.DeviceGaussians.from_scene(wl.scene, pin=True)
    host_out = torch.empty(r32.out.shape, dtype=torch.float32, pin_memory=True)
    h2d = sum(t.numel() * t.element_size() for t in (host_in.means, host_in.scales, host_in.quats,
                                                     host_in.opacity, host_in.rgb))
    d2h = host_out.numel() * host_out.element_size()

    # api.HostPipeline: each frame's host-to-device copy of the Gaussians and
    # device-to-host copy of its views overlap the compute of the frames
    # beside it (two slots, one copy stream each way)
    pipe = api.HostPipeline(r32, wl.scene.n, device=dev)
    for _ in range(args.warmup):
        pipe.submit(host_in, host_out)
    barrier()
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.s_in)
    last = None
    for _ in range(args.steps):
        last = pipe.submit(host_in, host_out)
    pipe.s_out.wait_event(last)
    e1.record(pipe.s_out)
    barrier()
    e_ms = R.max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)

    # per-kernel roofline of the dominant stage (live event times above)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    rect = r32.planes.rect[: wl.scene.n].to(torch.int64)
    area = ((rect[:, 2] - rect[:, 0] + 1).clamp(min=0) * (rect[:, 3] - rect[:, 1] + 1).clamp(min=0))
    pairs = int(area.sum().item())
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)

    def roof(dtype):
        st = res[dtype]["stages"]
        bp = {"f32": 4, "f16": 2, "bf16": 2, "u8": 1}[dtype]
        out = {}
        if "composite" in st:
            ms_c = st["composite"][0] / st["composite"][1]
            byt = WORKLOAD["N"] * WORKLOAD["res"] ** 2 * 4 * bp + WORKLOAD["V"] * WORKLOAD["res"] ** 2 * 16
            ach = byt / (ms_c * 1e-3) / 1e9
            out["composite"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                                "frac": round(ach / hbm, 4), "traffic": _traffic("composite") if dtype == "f32" else None,
                                "ms": round(ms_c, 4),
                                "algorithmic_bytes": byt, "peak_source": "measured"}
        if "raster_gaussians" in st:
            ms_r = st["raster_gaussians"][0] / st["raster_gaussians"][1]
            flops = pairs * 15
            peak = sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
            ach = flops / (ms_r * 1e-3) / 1e12
            out["raster_gaussians"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2),
                                       "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                                       "traffic": _traffic("raster_gaussians") if dtype == "f32" else None,
                                       "ms": round(ms_r, 4), "pairs": pairs, "flops_per_pair": 15,
                                       "peak_source": "SMs x 128 FP32 lanes x 2 x sampled median SM clock"}
        return out

    roofs = {d: roof(d) for d in res}
    dom = max(res["f32"]["stages"].items(), key=lambda kv: kv[1][0])[0] if res["f32"]["stages"] else None
    primary = roofs["f32"].get(dom) or roofs["f32"].get("composite")

    line = None
    if rank == 0:
        # the frame as a render loop runs it: one CUDA-graph replay per frame,
        # two frames in flight; the one-frame-at-a-time figure beside it
        fps = R.job_rate(f_ms, world)
        line = {
            "metric": METRIC, "value": round(fps, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(f_ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config({"planes": "f32", "parallelism": "replicas" if world > 1 else "single",
                               "launch": "one CUDA-graph replay per frame (%d kernels), two frames in flight "
                                         "(two renderers, two streams)" % graph_kernels,
                               "l2": "not flushed: each frame streams > 0.7 GB (planes, views, workspace) "
                                     "through the 129 MB L2"}),
            "views_per_s": round(fps * WORKLOAD["V"], 1),
            "one_frame_at_a_time": {"value": round(R.job_rate(g_ms, world), 2), "ms_per_step": round(g_ms, 4),
                                    "l2": "flushed between frames (512 MB write)",
                                    "note": "frame latency: one graph replay, the next frame starting after it"},
            "plain_launches": {"value": round(R.job_rate(res["f32"]["ms"], world), 2),
                               "ms_per_step": round(res["f32"]["ms"], 4)},
            "variants": {d: {"planes": d, "value": round(R.job_rate(res[d]["flight_ms"], world), 2),
                             "ms_per_step": round(res[d]["flight_ms"], 4),
                             "one_frame_at_a_time_value": round(R.job_rate(res[d]["graph_ms"], world), 2),
                             "plain_launches_value": round(R.job_rate(res[d]["ms"], world), 2), "roofline": roofs[d]}
                         for d in ("f16", "bf16", "u8")},
            "stages_ms": {d: {k: round(v[0] / v[1], 4) for k, v in res[d]["stages"].items()} for d in res},
            "e2e": {"value": round(R.job_rate(e_ms, world), 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(e_ms, 4),
                    "api": "HostPipeline.submit (pinned host Gaussians in, pinned host views out, two "
                           "frames in flight: a renderer and compute stream per slot, copies overlapped with "
                           "the neighbouring frames, one CUDA-graph replay per frame)",
                    "l2": "not flushed between steps: each step streams > 0.7 GB (planes, views, workspace) "
                          "through the 129 MB L2"},
            "gpu_launches": graph_kernels * args.steps,
            "roofline": dict(primary, kernel=dom if dom in roofs["f32"] else "composite") if primary else None,
            "roofline_by_kernel": roofs["f32"],
            "clocks": clk,
        }
    if rank == 0 and world == 1:
        line["_views_host"] = {d: res[d].pop("views_host", None) for d in res}
    if rank == 0 and world == 1 and not args.no_extras:
        for d in res:
            res[d]["renderer"] = None
        del r32, host_in, host_out, g, flush, pipe
        torch.cuda.empty_cache()
        line["v2lf"] = run_v2lf(args, dev)
        torch.cuda.empty_cache()
        line["differentiable"] = run_differentiable(args, dev, getattr(args, "fit_target", None))
        torch.cuda.empty_cache()
        line["batched"] = run_batched(args, dev)
        torch.cuda.empty_cache()
        line["sweeps"] = run_sweeps(args, dev)
        torch.cuda.empty_cache()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


def _event_ms(fn, steps, warmup, stream, flush=None):
    """Mean CUDA-event time of fn over steps calls after warmup calls (L2
    flushed before each timed call when a flush buffer is given)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def run_v2lf(args, dev):
    """V2LF at display scale: 2M sparse voxels (3-level grid), 512^2, N 64,
    45 views, FP32 planes; same timing rules as the primary number."""
    import torch
    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import synth as S
    wl = _voxel_workload()
    v = api.DeviceVoxels.from_scene(wl.scene, device=dev)
    r = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, "f32", device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    ms = _event_ms(lambda: r.render(v), args.steps, args.warmup, st, flush)
    status, needed, M = r.status()
    api.lf_trace_collect()
    api.lf_trace_enable(True)
    for _ in range(3):
        r.render(v)
    torch.cuda.synchronize()
    api.lf_trace_enable(False)
    stages = {k: round(t / c, 4) for k, (t, c) in api.lf_trace_collect().items()}
    # with the low-pass plane filter that replaces SVR's supersampling (Sec. 4.5)
    rf = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, "f32", device=dev,
                                plane_filter=0.7)
    ms_f = _event_ms(lambda: rf.render(v), args.steps, args.warmup, st, flush)
    api.lf_trace_collect()
    api.lf_trace_enable(True)
    for _ in range(3):
        rf.render(v)
    torch.cuda.synchronize()
    api.lf_trace_enable(False)
    f_ms = {k: round(t / c, 4) for k, (t, c) in api.lf_trace_collect().items()}.get("plane_filter")
    return {"workload": wl.name, "voxels": wl.scene.n, "culled_in": M, "status": status, "planes": "f32",
            "value": round(1000.0 / ms, 2), "unit": UNIT, "ms_per_step": round(ms, 4),
            "views_per_s": round(1000.0 / ms * wl.views.Vx, 1), "stages_ms": stages,
            "with_plane_filter": {"sigma_px": 0.7, "radius": 3, "value": round(1000.0 / ms_f, 2),
                                  "ms_per_step": round(ms_f, 4), "plane_filter_ms": f_ms}}


def run_differentiable(args, dev, fit_target=None):
    """Differentiable G2LF: 300k Gaussians, 512^2, N 64, 45 views: forward
    (build + composite) and backward (composite adjoint, splat adjoint,
    projection chain rule) per step, FP32; then a fit of all five parameter
    groups (means, scales, quaternions, opacities, colours) by Adam against
    target views of a perturbed copy of the scene (means + N(0, 0.01),
    opacities + N(0, 0.05)) rendered by the FP64 oracle, with its loss curve;
    then forward and backward of the 2M-voxel V2LF workload (FP32 planes)."""
    import torch
    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import autograd as AG
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_fit()
    g = api.DeviceGaussians.from_scene(wl.scene, device=dev)
    # the saving composite keeps 16 bytes of transmittance state per view
    # pixel, so the composite adjoint walks the planes once
    r = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, "f32", device=dev,
                               save_state=True)
    dv = torch.randn((wl.views.Vx, wl.camera.Ny, wl.camera.Nx, 4), device=dev)
    st = torch.cuda.current_stream()
    # beside it: the plain forward and the adjoint's own two walks
    r.save_state = False
    fwd_plain = _event_ms(lambda: r.render(g), args.steps, args.warmup, st)
    bwd_two = _event_ms(lambda: r.backward(g, dv), args.steps, args.warmup, st)
    r.save_state = True
    fwd = _event_ms(lambda: r.render(g), args.steps, args.warmup, st)
    bwd = _event_ms(lambda: r.backward(g, dv), args.steps, args.warmup, st)
    api.lf_trace_collect()
    api.lf_trace_enable(True)
    for _ in range(3):
        r.render(g)
        r.backward(g, dv)
    torch.cuda.synchronize()
    api.lf_trace_enable(False)
    stages = {k: round(t / c, 4) for k, (t, c) in api.lf_trace_collect().items()}
    out = {"workload": wl.name, "gaussians": wl.scene.n, "forward_ms": round(fwd, 4), "backward_ms": round(bwd, 4),
           "steps_per_s": round(1000.0 / (fwd + bwd), 2), "stages_ms": stages,
           "composite_state": "saved by the forward (16 B per view pixel); the adjoint walks the planes once",
           "without_saved_state": {"forward_ms": round(fwd_plain, 4), "backward_ms": round(bwd_two, 4)},
           "gradient_check": "tests/test_gpu_grad.py (finite differences of the FP64 oracle)"}
    # the fit: target views from the oracle (the CPU-baseline leg renders
    # them) or, without that leg, from this renderer on the perturbed scene
    if fit_target is None:
        tgt = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, "f32", device=dev)
        target = tgt.render(api.DeviceGaussians.from_scene(S.perturbed(wl.scene, FIT_TARGET_SEED), device=dev)).clone()
        source = "GPU render of the perturbed scene (oracle leg not run)"
        del tgt
    else:
        target = torch.as_tensor(fit_target, dtype=torch.float32).to(dev)
        source = "FP64 oracle render of the perturbed scene"
    lrs = [1e-3, 1e-4, 1e-3, 1e-2, 1e-2]

    def fit(n_steps):
        params = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.quats, g.opacity, g.rgb)]
        opt = torch.optim.Adam([{"params": [p], "lr": lr} for p, lr in zip(params, lrs)])
        losses = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n_steps):
            opt.zero_grad(set_to_none=True)
            v = AG.render_gaussians(r, *params)
            loss = ((v - target) ** 2).sum()
            loss.backward()
            opt.step()
            with torch.no_grad():
                params[1].clamp_(min=1e-6)
                params[3].clamp_(0.01, 0.99)
            losses.append(loss.detach())
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / n_steps, losses

    # warm-up steps from the same start, not kept: the first optimizer step
    # and the first backward pass through torch.autograd load their Python
    # modules and start autograd's device thread (seconds on a cold host)
    fit(max(3, args.warmup))
    n_steps = 40
    fit_ms, losses = fit(n_steps)
    curve = [float(x) for x in torch.stack(losses).cpu()]
    out["fit"] = {"target": source, "parameters": ["means", "scales", "quats", "opacity", "rgb"],
                  "optimizer": "Adam (torch), lr %s" % lrs, "loss": "sum of squared view differences",
                  "steps": n_steps, "ms_per_step": round(fit_ms, 3), "steps_per_s": round(1000.0 / fit_ms, 2),
                  "loss_first": curve[0], "loss_last": curve[-1], "loss_curve": [round(x, 3) for x in curve]}
    del r
    # the voxel model's adjoint: the V2LF workload (2M voxels), FP32 planes
    vw = _voxel_workload()
    vv = api.DeviceVoxels.from_scene(vw.scene, device=dev)
    rv = api.LightFieldRenderer(vw.camera, vw.display, vw.views, vw.N, vw.binning, "f32", device=dev,
                                save_state=True)
    dvv = torch.randn((vw.views.Vx, vw.camera.Ny, vw.camera.Nx, 4), device=dev)
    n_v = max(3, args.steps // 4)
    vf = _event_ms(lambda: rv.render(vv), n_v, 2, st)
    vb = _event_ms(lambda: rv.backward(vv, dvv), n_v, 2, st)
    api.lf_trace_collect()
    api.lf_trace_enable(True)
    rv.render(vv)
    rv.backward(vv, dvv)
    torch.cuda.synchronize()
    api.lf_trace_enable(False)
    out["voxels"] = {"workload": vw.name, "voxels": vw.scene.n, "forward_ms": round(vf, 4),
                     "backward_ms": round(vb, 4),
                     "stages_ms": {k: round(t / c, 4) for k, (t, c) in api.lf_trace_collect().items()},
                     "gradient_check": "tests/test_gpu_grad.py (finite differences of the FP64 oracle)"}
    return out


def oracle_fit_target():
    """Target views of the differentiable fit: the FP64 oracle's render of the
    perturbed copy of the 300k-Gaussian scene (part of the oracle leg)."""
    import oracle
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_fit()
    o = oracle.render(scene=S.perturbed(wl.scene, FIT_TARGET_SEED), camera=wl.camera, display=wl.display,
                      views=wl.views, N=wl.N, binning=wl.binning)
    return o["views"].astype(np.float32)


def run_batched(args, dev):
    """Six uneven G2LF scenes (50k..3M Gaussians, 9..128 views, 256^2..1024^2,
    N 64..512, FP16 planes): autotuned plan (views per thread, composite
    tile, chunk groups, scene schedule), one CUDA-graph launch per frame,
    against the same scenes rendered one by one; beside it the frame time of
    1, 2 and 4 chunk groups with the tuned composite layout."""
    import torch
    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import synth as S
    wls = S.workloads_batched()
    b = api.BatchRenderer(wls, "f16", device=dev, max_chunk_groups=4)
    plan, tune_ms = b.autotune(reps=1)
    s = b.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    by_groups = {}
    for gr in (1, 2, 4):
        pl = dict(plan, chunk_groups=gr, schedule=plan["schedule"] if plan["schedule"] != 2 else 1)
        b.prepare(pl)
        by_groups[str(gr)] = round(_event_ms(b.render, max(3, args.steps // 4), 2, s, flush), 3)
    b.prepare(plan)
    b.capture()
    k0 = api.lf_launch_count()
    g_ms = _event_ms(b.launch, args.steps, args.warmup, s, flush)
    launches = (api.lf_launch_count() - k0) // max(1, args.steps + args.warmup)
    status = b.status()
    rs = []
    for w in wls:
        r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f16", device=dev)
        rs.append((r, api.DeviceGaussians.from_scene(w.scene, device=dev)))

    def seq():
        for r, g in rs:
            r.render(g, s)
    with torch.cuda.stream(s):
        s_ms = _event_ms(seq, args.steps, args.warmup, s, flush)
    views = sum(w.views.Vx * w.views.Vy for w in wls)
    b.close()
    return {"scenes": [{"gaussians": w.scene.n, "views": w.views.Vx, "res": w.camera.Nx, "N": w.N} for w in wls],
            "planes": "f16", "status": status, "plan": plan, "autotune_ms": round(tune_ms, 3),
            "graph_ms_per_frame": round(g_ms, 3), "batch_frames_per_s": round(1000.0 / g_ms, 2),
            "views_per_s": round(views * 1000.0 / g_ms, 1), "kernels_per_frame": int(launches),
            "one_by_one_ms_per_frame": round(s_ms, 3),
            "chunk_groups_ms_per_frame": by_groups,
            "chunk_groups_note": "persistent schedule (tuned composite layout), plain launches, L2 flushed"}


def run_sweeps(args, dev):
    """Speed sweeps on the 1M-Gaussian display scene (the paper's scenes and
    trained models are not available): LF frames/s and views/s against the
    number of views (the paper's real-time-beyond-90-views claim), and over
    N_chunk x P_s x sampling (its Table 1 axes), FP32 and FP16 planes, one
    CUDA-graph replay per frame, L2 flushed between frames."""
    import torch
    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_display(seed=WORKLOAD["seed"])
    g = api.DeviceGaussians.from_scene(wl.scene, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    steps, warm = max(5, args.steps // 2), 3

    def fps(display, views, N, dtype, blend="exact"):
        r = api.LightFieldRenderer(wl.camera, display, views, N, wl.binning, dtype, device=dev, blend=blend)
        r.capture(g)
        ms = _event_ms(r.replay, steps, warm, st, flush)
        out = {"value": round(1000.0 / ms, 2), "views_per_s": round(1000.0 / ms * views.Vx * views.Vy, 1),
               "ms_per_step": round(ms, 4)}
        del r
        return out

    res = {"unit": UNIT, "views": {}, "table1": {}, "blend_3dgs": {}}
    # the 3DGS rasteriser's cut-offs (alpha < 1/255 skipped, stop before
    # T < 1e-4) against exact blending, same frame
    for dtype in ("f32", "f16"):
        res["blend_3dgs"][dtype] = fps(wl.display, wl.views, 64, dtype, blend="3dgs")
    for V in (9, 45, 90, 180):
        for dtype in ("f32", "f16"):
            res["views"]["V%d_%s" % (V, dtype)] = fps(wl.display, S.ViewSet(V), 64, dtype)
    for N in (16, 64, 256):
        for Ps in (1, 2):
            disp = S.display_for(wl.display.D_focal, 0.15, P_s=Ps)
            for bil in (False, True):
                for dtype in ("f32", "f16"):
                    key = "N%d_Ps%d_%s_%s" % (N, Ps, "bilinear" if bil else "nearest", dtype)
                    res["table1"][key] = fps(disp, S.ViewSet(45, 1, bil), N, dtype)
    torch.cuda.empty_cache()
    return res


def view_errors(gpu_views, oracle_views):
    """Per-view max-abs error and PSNR of GPU views against the FP64 oracle."""
    out = []
    for v in range(gpu_views.shape[0]):
        d = gpu_views[v].astype(np.float64) - oracle_views[v]
        mse = float(np.mean(d * d))
        out.append((float(np.abs(d).max()), float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)))
    return {"max_abs": round(max(e[0] for e in out), 6), "min_psnr_db": round(min(e[1] for e in out), 2),
            "per_view_max_abs": [round(e[0], 6) for e in out], "per_view_psnr_db": [round(e[1], 2) for e in out]}


def run_profile(args):
    """Short run for profilers: W warm-up frames then one frame per plane
    dtype (f32, f16), no timing, no e2e, no CPU baseline."""
    import torch

    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_display(seed=WORKLOAD["seed"], n=WORKLOAD["n"], res=WORKLOAD["res"], N=WORKLOAD["N"],
                            V=WORKLOAD["V"])
    g = api.DeviceGaussians.from_scene(wl.scene)
    for dtype in args.profile_dtypes.split(","):
        r = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, dtype)
        for _ in range(args.warmup + 1):
            r.render(g)
        torch.cuda.synchronize()
        st, needed, M = r.status()
        print("profile %s: status %d, M %d, pairs %d" % (dtype, st, M, needed), flush=True)


def run_profile_grad(args):
    """Short run for profilers of the differentiable workloads (300k Gaussians,
    then 2M voxels; 512^2, N 64, 45 views, FP32, saved composite state): W + 1
    forward + backward steps of each, no timing."""
    import torch

    from paper_2508_18540_gb300 import api
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_fit()
    g = api.DeviceGaussians.from_scene(wl.scene)
    r = api.LightFieldRenderer(wl.camera, wl.display, wl.views, wl.N, wl.binning, "f32", save_state=True)
    gen = torch.Generator(device="cuda").manual_seed(11)
    dv = torch.randn((wl.views.Vx, wl.camera.Ny, wl.camera.Nx, 4), device="cuda", generator=gen)
    for _ in range(args.warmup + 1):
        r.render(g)
        r.backward(g, dv)
    torch.cuda.synchronize()
    print("profile grad: composite status %d" % r.composite_status(), flush=True)
    del r
    # then the 2M-voxel V2LF workload, FP32 planes
    vw = _voxel_workload()
    v = api.DeviceVoxels.from_scene(vw.scene)
    rv = api.LightFieldRenderer(vw.camera, vw.display, vw.views, vw.N, vw.binning, "f32", save_state=True)
    dvv = torch.randn((vw.views.Vx, vw.camera.Ny, vw.camera.Nx, 4), device="cuda", generator=gen)
    for _ in range(args.warmup + 1):
        rv.render(v)
        rv.backward(v, dvv)
    torch.cuda.synchronize()
    print("profile grad voxels: composite status %d" % rv.composite_status(), flush=True)


def _oracle_rate(wl, min_seconds, max_frames):
    """Full LF frames of the oracle on wl, repeated until about min_seconds
    (at least one frame); returns (frames/s, frames, seconds, last result)."""
    import oracle
    t0 = time.perf_counter()
    n_frames, last = 0, None
    while n_frames < max_frames:
        last = oracle.render(wl)
        n_frames += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return n_frames / dt, n_frames, dt, last


def cpu_baseline(min_seconds=10.0, max_frames=40):
    """The FP64 oracle, as it stands, on the host cores: full LF frames of
    the same workload (all 1M Gaussians splatted into 64 planes, 45 views
    composited), repeated until about min_seconds of CPU work, with every
    core; beside it one frame on one thread, the 10k-Gaussian workload in
    full on one thread and on every core, and the 2M-voxel V2LF workload in
    full on every core."""
    import oracle
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_display(seed=WORKLOAD["seed"], n=WORKLOAD["n"], res=WORKLOAD["res"], N=WORKLOAD["N"],
                            V=WORKLOAD["V"])
    oracle.lib()
    oracle.set_num_threads(0)
    cores = oracle.num_threads()
    rate, n_frames, dt, last = _oracle_rate(wl, min_seconds, max_frames)
    by_config = {}
    oracle.set_num_threads(1)
    r1, n1, t1, _ = _oracle_rate(wl, 0.0, 1)
    by_config["g2lf_display_1M_512px_N64_45v"] = {
        "all_cores": {"value": round(rate, 4), "threads": cores, "frames": n_frames, "seconds": round(dt, 2)},
        "one_thread": {"value": round(r1, 4), "threads": 1, "frames": n1, "seconds": round(t1, 2)}}
    tiny = S.workload_tiny()
    r1, n1, t1, _ = _oracle_rate(tiny, 1.0, 200)
    oracle.set_num_threads(0)
    ra, na, ta, _ = _oracle_rate(tiny, 1.0, 200)
    by_config[tiny.name] = {"all_cores": {"value": round(ra, 3), "threads": cores, "frames": na, "seconds": round(ta, 2)},
                            "one_thread": {"value": round(r1, 3), "threads": 1, "frames": n1, "seconds": round(t1, 2)}}
    vw = _voxel_workload()
    rv, nv, tv, _ = _oracle_rate(vw, 0.0, 1)
    by_config[vw.name] = {"all_cores": {"value": round(rv, 4), "threads": cores, "frames": nv, "seconds": round(tv, 2)}}
    return {"value": round(rate, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d full LF frame(s) of the 1M-Gaussian 512px N64 45-view workload, FP64, OpenMP" % n_frames,
            "seconds": round(dt, 2), "host": _host(), "by_config": by_config,
            "by_config_unit": "LF frames/s (full frames: splat + composite)"}, last["views"]


def _host():
    """CPU of the machine the oracle ran on (architecture, model, logical CPUs)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import subprocess
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines()
                          if ln.lower().startswith("model name")), "")
        except (OSError, subprocess.SubprocessError):
            pass
    return {"arch": platform.machine(), "model": model or None, "logical_cpus": os.cpu_count()}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return None
    import oracle
    from paper_2508_18540_gb300 import synth as S
    wl = S.workload_display(seed=WORKLOAD["seed"], n=WORKLOAD["n"], res=WORKLOAD["res"], N=WORKLOAD["N"],
                            V=WORKLOAD["V"])
    oracle.lib()
    for _ in range(args.warmup):
        oracle.render(wl, with_views=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.render(wl)
    dt = (time.perf_counter() - t0) / args.steps
    cores = oracle.num_threads()
    v = round(1.0 / dt, 4)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config({"planes": "f64", "parallelism": "host cores"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full LF frame per step (warm-up steps splat only)", "host": _host()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the V2LF, differentiable and batched sections")
    ap.add_argument("--profile", action="store_true", help="short untimed run for ncu")
    ap.add_argument("--profile-dtypes", default="f32,f16")
    ap.add_argument("--profile-grad", action="store_true", help="short untimed forward + backward run for ncu")
    args = ap.parse_args()
    if args.profile_grad:
        import __graft_entry__
        __graft_entry__.build()
        run_profile_grad(args)
        return
    if args.profile:
        import __graft_entry__
        __graft_entry__.build()
        run_profile(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # the oracle arm builds and loads the oracle only (no CUDA library)
        from oracle import build as obuild
        obuild.build()
        line = run_reference(args)
    else:
        import __graft_entry__
        __graft_entry__.build()
        rank, world, _ = _env_rank()
        if world == 1 and not args.no_cpu_baseline and not args.no_extras:
            from oracle import build as obuild
            obuild.build()
            args.fit_target = oracle_fit_target()
        line = run_ours(args)
        rank, world, _ = _env_rank()
        views_host = line.pop("_views_host", None) if line is not None else None
        if line is not None and world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], oviews = cpu_baseline()
            if views_host:
                line["accuracy_vs_fp64_oracle"] = {d: view_errors(v, oviews) for d, v in views_host.items()
                                                   if v is not None}
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
