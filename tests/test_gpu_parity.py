"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer work is compared bit for bit (culling, footprint rectangles, depth
order, chunk membership, plane distances, chunk counts, tile lists); colour
within the tolerances stated below:
  FP32 planes: max-abs <= 1e-4 per channel (planes and views);
  FP16 planes: max-abs <= 4e-3 and PSNR >= 60 dB against the FP64 oracle;
  BF16 planes: max-abs <= 3e-2 and PSNR >= 45 dB.
"""
import numpy as np
import pytest
import torch

from paper_2508_18540_gb300 import synth as S
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = {"f32": (1e-4, 80.0), "f16": (4e-3, 60.0), "bf16": (3e-2, 45.0)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_18540_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _compare(gpu, o, W, H, N, dtype, check_lists=True):
    assert gpu["status"] == 0
    valid = o["valid"].astype(bool)
    n = valid.shape[0]
    # culling and footprints: bit-exact
    assert np.array_equal(gpu["rect"], o["rect"])
    # depth order and chunk membership: bit-exact
    assert gpu["M"] == o["M"]
    assert np.array_equal(gpu["order"], o["order"])
    assert np.array_equal(gpu["chunk"], o["chunk"])
    assert np.array_equal(gpu["count"], o["count"])
    assert np.array_equal(gpu["d"], o["d"])          # FP64 bits
    if check_lists:
        G.check_tile_lists(gpu, o, W, H, N)
    tol, min_psnr = TOL[dtype]
    err_p = np.abs(gpu["planes"] - o["planes"]).max()
    err_v = np.abs(gpu["views"] - o["views"]).max()
    assert err_p <= tol, err_p
    assert err_v <= tol, err_v
    for v in range(gpu["views"].shape[0]):
        assert G.psnr(gpu["views"][v], o["views"][v]) >= min_psnr
    return err_p, err_v


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_tiny_workload(orc, dtype):
    w = S.workload_tiny()
    o = orc.render(w)
    gpu = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning, dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, w.N, dtype, check_lists=(dtype == "f32"))


@pytest.mark.parametrize("bilinear", [False, True])
@pytest.mark.parametrize("binning", ["quantile", "disparity"])
def test_ragged_rotated_scaled(orc, bilinear, binning):
    # 100x70 views, P_s = 2 (200x140 planes: ragged 16x16 tiles), rotated and
    # translated camera, D_shift, 1037 anisotropic Gaussians, N = 5, 7 views
    cam = G.small_rotated_camera()
    disp = S.display_for(3.0, 0.12, P_s=2, D_shift=0.03)
    sc = S.blob_gaussians(1037, 21, n_blobs=12, z=(1.5, 6.0))
    views = S.ViewSet(7, 1, bilinear, (0.1, 0.2, 0.3))
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=5, binning=binning)
    gpu = G.run_gpu(sc, cam, disp, views, 5, binning, "f32")
    _compare(gpu, o, o["ref"].W, o["ref"].H, 5, "f32")


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_bilinear_nine_views_per_thread(orc, dtype):
    # bilinear with 9 views per thread: 11 x 2 views (a ragged view group and
    # two view rows), so every CTA pre-blends the rows of its own view row
    cam = S.Camera(np.eye(3), np.zeros(3), np.radians(50.0), np.radians(40.0), 96, 40)
    disp = S.Display(D_focal=3.0, phi_x=0.12, phi_y=0.05)
    sc = S.uniform_gaussians(4000, 17)
    views = S.ViewSet(11, 2, True, (0.3, 0.1, 0.2))
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=12, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 12, "quantile", dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, 12, dtype)


@pytest.mark.parametrize("dtype,bilinear", [("f32", False), ("f16", False), ("f32", True), ("u8", True)])
def test_fifteen_views_per_thread(orc, dtype, bilinear):
    # 30 x 2 views: the staged composite runs view groups of 15 (one CTA per
    # SM, its own launch bounds and shared-memory budget)
    cam = S.Camera(np.eye(3), np.zeros(3), np.radians(50.0), np.radians(40.0), 80, 48)
    disp = S.Display(D_focal=3.0, phi_x=0.12, phi_y=0.05)
    sc = S.uniform_gaussians(3000, 23)
    views = S.ViewSet(30, 2, bilinear, (0.2, 0.3, 0.1))
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=10, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 10, "quantile", dtype)
    if dtype == "u8":
        # RGBA8 planes: the composite of the GPU's own planes against FP64
        pl = gpu["renderer"].planes.rgba.cpu().numpy().astype(np.float64) / 255.0
        want = orc.composite(o["ref"], pl, o["d"], o["count"], 30, 2, bilinear, views.bg)
        assert np.abs(gpu["views"] - want).max() <= 1e-4
    else:
        _compare(gpu, o, o["ref"].W, o["ref"].H, 10, dtype)


def test_two_view_rows(orc):
    # vertical parallax too (Vy = 3), non-square views
    cam = S.Camera(np.eye(3), np.zeros(3), np.radians(50.0), np.radians(40.0), 64, 48)
    disp = S.Display(D_focal=3.0, phi_x=0.1, phi_y=0.06)
    sc = S.uniform_gaussians(3000, 5)
    views = S.ViewSet(5, 3, False)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=8, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 8, "quantile")
    _compare(gpu, o, o["ref"].W, o["ref"].H, 8, "f32")


@pytest.mark.parametrize("N", [1, 3, 64])
def test_chunk_counts_and_few_primitives(orc, N):
    # N = 1 (plain alpha blending), and M < N (empty chunks, zero planes)
    sc = S.uniform_gaussians(40, 9)
    w = S.workload_tiny()
    o = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=N, binning="quantile")
    gpu = G.run_gpu(sc, w.camera, w.display, w.views, N, "quantile")
    _compare(gpu, o, o["ref"].W, o["ref"].H, N, "f32")


@pytest.mark.parametrize("N,dtype", [(1, "f32"), (2, "f32"), (2, "f16"), (3, "bf16")])
def test_long_lists_are_split_and_merged(orc, N, dtype):
    # 30,000 Gaussians in a 128^2 frame with few chunks: (super-tile, chunk)
    # lists of thousands of entries, which the raster cuts into parts of
    # 1,024 entries (the smallest part), blends separately and composes in
    # part order; planes and views stay within the tolerance of the oracle
    sc = S.uniform_gaussians(30_000, 21)
    w = S.workload_tiny()
    o = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=N, binning="quantile")
    assert G.longest_super_tile_list(o, N) > 2 * 1024   # at least three parts
    gpu = G.run_gpu(sc, w.camera, w.display, w.views, N, "quantile", dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, N, dtype, check_lists=False)


def test_non_finite_inputs_are_culled(orc):
    # host-side fault injection: Gaussians with a NaN position, scale or
    # rotation, or an infinite scale, are culled by the same comparisons as
    # in the oracle (every comparison with NaN is false) before any of their
    # values is used as an index; the rest of the scene renders as usual
    w = S.workload_tiny(seed=3)
    sc = w.scene.subset(np.arange(2000))
    sc.means[0, 0] = np.nan
    sc.means[1, 2] = np.nan
    sc.scales[2, 1] = np.nan
    sc.quats[3, :] = np.nan
    sc.scales[4] = np.inf
    o = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=w.N, binning=w.binning)
    assert o["valid"][:5].tolist() == [0] * 5
    gpu = G.run_gpu(sc, w.camera, w.display, w.views, w.N, w.binning, "f32")
    _compare(gpu, o, o["ref"].W, o["ref"].H, w.N, "f32")
    assert np.isfinite(gpu["planes"]).all() and np.isfinite(gpu["views"]).all()


def test_everything_culled(orc):
    w = S.workload_tiny()
    sc = S.uniform_gaussians(500, 3)
    sc.means[:, 2] = -3.0
    views = S.ViewSet(3, 1, False, (0.5, 0.25, 0.125))
    o = orc.render(scene=sc, camera=w.camera, display=w.display, views=views, N=4, binning="quantile")
    gpu = G.run_gpu(sc, w.camera, w.display, views, 4, "quantile")
    assert gpu["M"] == 0
    _compare(gpu, o, o["ref"].W, o["ref"].H, 4, "f32")
    assert np.all(gpu["planes"] == 0.0)


def test_empty_scene(orc):
    w = S.workload_tiny()
    sc = S.uniform_gaussians(0, 3)
    gpu = G.run_gpu(sc, w.camera, w.display, w.views, 4, "quantile")
    assert gpu["status"] == 0 and gpu["M"] == 0
    assert np.all(gpu["planes"] == 0.0) and np.all(gpu["views"][..., 3] == 0.0)


def test_tile_list_overflow_is_reported(orc):
    from paper_2508_18540_gb300 import _lib
    w = S.workload_tiny()
    gpu = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning, dup_capacity=1000)
    assert gpu["status"] == _lib.LF_ERR_OVERFLOW
    assert gpu["needed"] > 1000


def test_deterministic(orc):
    w = S.workload_tiny(seed=4)
    a = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning)
    b = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning)
    assert np.array_equal(a["planes"], b["planes"]) and np.array_equal(a["views"], b["views"])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_voxels(orc, dtype):
    # small V2LF scene: 3-level sparse grid at 64^3 base, 96x96 views
    sc = S.sparse_voxels(20_000, 3, base_res=64)
    cam = S.identity_camera(96, t=(0.0, 0.0, 6.0))
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15)
    views = S.ViewSet(9)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=16, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 16, "quantile", dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, 16, dtype, check_lists=(dtype == "f32"))


def test_voxels_large_footprints(orc):
    # a dense block of coarse voxels (side 0.5 at depth 3 to 8, 64^2 views):
    # footprints of about 10x10 pixels, so one batch of staged voxels holds
    # more (voxel, pixel) pairs than a shared-memory pass (up to ~3200
    # against 2048) and is processed in several passes
    rng = np.random.default_rng(11)
    n1 = 10
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1).astype(np.int32)
    n = ijk.shape[0]
    base = 0.5
    sc = S.VoxelScene(ijk, np.zeros(n, np.uint8), np.array([-n1 * base / 2, -n1 * base / 2, 3.0]), base,
                      rng.uniform(0.05, 1.5, (n, 8)).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32))
    cam = S.identity_camera(64)
    disp = S.display_for(5.0, 0.15)
    views = S.ViewSet(3)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=1, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 1, "quantile", "f32")
    _compare(gpu, o, o["ref"].W, o["ref"].H, 1, "f32")


def test_voxels_rotated(orc):
    sc = S.sparse_voxels(5_000, 4, base_res=32)
    cam = G.small_rotated_camera(64, 48)
    cam.t = np.array([0.1, -0.05, 6.0])
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15, P_s=2)
    views = S.ViewSet(5, 1, True)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=6, binning="disparity")
    gpu = G.run_gpu(sc, cam, disp, views, 6, "disparity")
    _compare(gpu, o, o["ref"].W, o["ref"].H, 6, "f32")


@pytest.mark.parametrize("graphs,depth", [(True, 3), (False, 3), (True, 2), (True, 1)])
def test_host_pipeline_frames_match_synchronous_renders(graphs, depth):
    # api.HostPipeline overlaps copies with compute across frames; every
    # frame's host views must equal a plain synchronous render of its input
    # (five frames: every slot is reused at least once)
    from paper_2508_18540_gb300 import api
    w = S.workload_tiny()
    scenes = [w.scene] + [S.perturbed(w.scene, s) for s in (3, 4, 5, 6)]
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    pipe = api.HostPipeline(r, w.scene.n, graphs=graphs, depth=depth)
    outs, evs = [], []
    hosts = [api.DeviceGaussians.from_scene(sc, pin=True) for sc in scenes]
    for h in hosts:
        o = torch.empty(r.out.shape, dtype=torch.float32, pin_memory=True)
        evs.append(pipe.submit(h, o))
        outs.append(o)
    for ev in evs:
        ev.synchronize()
    torch.cuda.synchronize()
    ref = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    for sc, o in zip(scenes, outs):
        want = ref.render(api.DeviceGaussians.from_scene(sc)).cpu()
        assert torch.equal(o, want)


def test_depth_order_with_near_equal_depths(orc):
    # A camera turned by 1e-9 rad about y gives depth = z - 1e-9 x (FP64), so
    # Gaussians sharing z but not x differ in depth by ~1e-13: far below the
    # 24 bits the depth sort keeps of the key range. Clusters of 5000, 40 and
    # 10 such Gaussians (shuffled) exercise all three run fix-ups (global
    # memory network, shared memory network, insertion); the order must
    # still equal the oracle's (FP64 depth, index) order exactly.
    rng = np.random.default_rng(77)
    th = 1e-9
    R = np.array([[np.cos(th), 0.0, np.sin(th)], [0.0, 1.0, 0.0], [-np.sin(th), 0.0, np.cos(th)]])
    cam = S.Camera(R, np.zeros(3), np.radians(50.0), np.radians(50.0), 96, 96)
    bg = S.uniform_gaussians(3000, 78)
    parts = [bg]
    for cnt, z in ((5000, 4.0), (40, 3.0), (10, 5.0)):
        m = np.zeros((cnt, 3), np.float32)
        m[:, 0] = rng.permutation(np.linspace(-0.5, 0.5, cnt)).astype(np.float32)
        m[:, 1] = rng.uniform(-0.3, 0.3, cnt).astype(np.float32)
        m[:, 2] = z
        q = rng.normal(size=(cnt, 4)).astype(np.float32)
        parts.append(S.GaussianScene(m, np.full((cnt, 3), 0.01, np.float32), q,
                                     rng.uniform(0.1, 0.9, cnt).astype(np.float32),
                                     rng.uniform(0, 1, (cnt, 3)).astype(np.float32)))
    sc = S.GaussianScene(*(np.ascontiguousarray(np.concatenate([getattr(p, f) for p in parts]))
                           for f in ("means", "scales", "quats", "opacity", "rgb")))
    disp = S.display_for(3.0, 0.1)
    views = S.ViewSet(5)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=8, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 8, "quantile", "f32")
    _compare(gpu, o, o["ref"].W, o["ref"].H, 8, "f32")


@pytest.mark.parametrize("bilinear", [False, True])
def test_u8_planes(orc, bilinear):
    # RGBA8 planes (the paper's default format): every texel within half a
    # code (plus FP32 rounding) of the FP64 plane; the views equal the FP64
    # composite of the GPU's own dequantised planes within the FP32 bar; and
    # the quantisation error of the views against the FP64 oracle stays
    # above 40 dB PSNR per view.
    w = S.workload_tiny()
    views = S.ViewSet(w.views.Vx, 1, bilinear)
    o = orc.render(scene=w.scene, camera=w.camera, display=w.display, views=views, N=w.N, binning=w.binning)
    gpu = G.run_gpu(w.scene, w.camera, w.display, views, w.N, w.binning, "u8")
    assert gpu["status"] == 0
    pl = gpu["renderer"].planes.rgba.cpu().numpy().astype(np.float64) / 255.0
    assert np.abs(pl - o["planes"]).max() <= 0.5 / 255.0 + 2e-4
    ref = o["ref"]
    v_own = orc.composite(ref, pl, o["d"], o["count"], views.Vx, views.Vy, bilinear, views.bg)
    assert np.abs(gpu["views"] - v_own).max() <= 1e-4
    for k in range(gpu["views"].shape[0]):
        assert G.psnr(gpu["views"][k], o["views"][k]) >= 40.0


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("f16", 2e-3)])
def test_plane_filter_against_oracle(orc, dtype, tol):
    # the V2LF low-pass filter in place on the GPU planes against the FP64
    # filter of the same unfiltered planes; ragged width (not a multiple of
    # the row segment or the column block), several radii
    from paper_2508_18540_gb300 import api
    cam = S.identity_camera(72, t=(0.0, 0.0, 6.0))
    cam.Nx = 1100     # a row longer than one 1024-texel segment
    vs = S.sparse_voxels(3000, 9, base_res=32)
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15)
    r = api.LightFieldRenderer(cam, disp, S.ViewSet(3), 5, "quantile", dtype)
    v = api.DeviceVoxels.from_scene(vs)
    for sigma, radius in ((0.8, 0), (1.7, 5), (3.0, 16)):
        pl = r.build(v)
        torch.cuda.synchronize()
        before = pl.rgba.float().cpu().numpy().astype(np.float64)
        api.lf_filter_planes(pl, sigma, radius)
        torch.cuda.synchronize()
        after = pl.rgba.float().cpu().numpy().astype(np.float64)
        rad = radius if radius > 0 else int(np.ceil(3 * sigma))
        want = orc.filter_planes(before, sigma, rad)
        assert np.abs(after - want).max() <= tol, (sigma, radius)


def test_v2lf_with_plane_filter_end_to_end(orc):
    from paper_2508_18540_gb300 import api
    cam = S.identity_camera(64, t=(0.0, 0.0, 6.0))
    vs = S.sparse_voxels(2500, 10, base_res=32)
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15)
    views = S.ViewSet(5)
    r = api.LightFieldRenderer(cam, disp, views, 6, "quantile", "f32", plane_filter=0.7)
    out = r.render(api.DeviceVoxels.from_scene(vs)).cpu().numpy().astype(np.float64)
    o = orc.render(scene=vs, camera=cam, display=disp, views=views, N=6, binning="quantile")
    planes = orc.filter_planes(o["planes"], 0.7, 3)
    want = orc.composite(o["ref"], planes, o["d"], o["count"], 5, 1, False)
    assert np.abs(out - want).max() <= 1e-4


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_display_scale_workload(orc, dtype):
    # the benchmark's own workload and launch configuration (1M Gaussians,
    # 512^2, N = 64, 45 views): culling, rectangles, depth order, chunks and
    # plane depths bit-exact; planes and all views within the tolerance
    # (the 16x16 tile lists are checked at the smaller sizes above)
    w = S.workload_display()
    o = orc.render(w)
    gpu = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning, dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, w.N, dtype, check_lists=False)


def test_v2lf_display_scale_workload(orc):
    # the bench's V2LF workload and launch configuration (2M sparse voxels,
    # 512^2, N = 64, 45 views, FP32 planes): culling, rectangles, depth
    # order, chunks and plane depths bit-exact; planes and all views within
    # the FP32 tolerance
    w = S.workload_voxels()
    o = orc.render(w)
    gpu = G.run_gpu(w.scene, w.camera, w.display, w.views, w.N, w.binning, "f32")
    _compare(gpu, o, o["ref"].W, o["ref"].H, w.N, "f32", check_lists=False)


def test_renderer_graph_replay():
    # one CUDA graph per frame: replays equal a plain render, and read the
    # scene buffers in place (new colours show up in the next replay)
    from paper_2508_18540_gb300 import api
    w = S.workload_tiny()
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    g = api.DeviceGaussians.from_scene(w.scene)
    want = r.render(g).clone()
    kernels = r.capture(g)
    assert kernels > 10
    r.out.fill_(float("nan"))
    got = r.replay().clone()
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    with torch.no_grad():
        g.rgb.mul_(0.5)
    got2 = r.replay().clone()
    ref = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    want2 = ref.render(g).clone()
    torch.cuda.synchronize()
    assert torch.equal(got2, want2)


@pytest.mark.parametrize("dtype,Nx,Ny,bilinear", [("f16", 99, 37, False), ("f16", 99, 37, True),
                                                  ("f32", 2560, 24, False), ("bf16", 2561, 20, True)])
def test_unstaged_composite_fallback(orc, dtype, Nx, Ny, bilinear):
    # plane rows the staged kernel cannot take (an FP16 row that is not a
    # multiple of 16 bytes; rows too wide for the shared-memory ring) go
    # through the L1-cached kernel; same bar as the other parity tests
    cam = S.Camera(np.eye(3), np.zeros(3), np.radians(50.0), np.radians(20.0), Nx, Ny)
    sc = S.uniform_gaussians(4000, 31, xy=(-1.5, 1.5), z=(2.0, 6.0))
    views = S.ViewSet(7, 1, bilinear, (0.1, 0.2, 0.3))
    disp = S.display_for(3.0, 0.1)
    o = orc.render(scene=sc, camera=cam, display=disp, views=views, N=6, binning="quantile")
    gpu = G.run_gpu(sc, cam, disp, views, 6, "quantile", dtype)
    _compare(gpu, o, o["ref"].W, o["ref"].H, 6, dtype, check_lists=False)


@pytest.mark.parametrize("bilinear", [False, True])
def test_quilt_atlas_layout(bilinear):
    # the atlas output is the separate views laid out in tiles (row-major
    # from the top); tiles past the last view stay untouched; the adjoint
    # refuses the atlas layout
    from paper_2508_18540_gb300 import api
    w = S.workload_tiny()
    g = api.DeviceGaussians.from_scene(w.scene)
    r1 = api.LightFieldRenderer(w.camera, w.display, S.ViewSet(9, 1, bilinear), w.N, w.binning, "f32")
    r2 = api.LightFieldRenderer(w.camera, w.display, S.ViewSet(9, 1, bilinear, atlas_cols=4), w.N, w.binning, "f32")
    sep = r1.render(g).clone()
    r2.out.fill_(float("nan"))
    atlas = r2.render(g).clone()
    torch.cuda.synchronize()
    Ny, Nx = w.camera.Ny, w.camera.Nx
    assert tuple(atlas.shape) == (3 * Ny, 4 * Nx, 4)
    for v in range(9):
        tile = atlas[(v // 4) * Ny:(v // 4 + 1) * Ny, (v % 4) * Nx:(v % 4 + 1) * Nx]
        assert torch.equal(tile, sep[v]), v
    assert torch.isnan(atlas[2 * Ny:, Nx:]).all()
    with pytest.raises(api.L.LFError):
        r2.backward(g, torch.zeros_like(sep))


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_3dgs_blending_against_oracle(orc, dtype):
    # 3DGS-compatible blending (alpha < 1/255 skipped, stop before
    # T < 1e-4) on a dense scene where both cut-offs fire: structure
    # bit-exact as in exact mode; planes within the dtype's bar at every
    # texel except those the FP64 oracle marks as within 1e-6 of a threshold
    # (a decision FP32 may take the other way; their share is reported and
    # bounded); views equal to the FP64 composite of the GPU's own planes.
    # The exact-mode GPU planes differ where the oracle says the cut-offs
    # matter, so the flag is in effect.
    from paper_2508_18540_gb300 import api
    w = S.workload_tiny(seed=5)
    s0 = w.scene
    sc = S.GaussianScene(s0.means, s0.scales, s0.quats, (0.5 + 0.49 * s0.opacity).astype(np.float32), s0.rgb)
    N = 2
    o = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=N, binning=w.binning,
                   blend="3dgs")
    ex = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=N, binning=w.binning,
                    with_views=False)
    g = api.DeviceGaussians.from_scene(sc)
    r3 = api.LightFieldRenderer(w.camera, w.display, w.views, N, w.binning, dtype, blend="3dgs")
    v3 = r3.render(g).cpu().numpy().astype(np.float64)
    rx = api.LightFieldRenderer(w.camera, w.display, w.views, N, w.binning, dtype)
    rx.render(g)
    torch.cuda.synchronize()
    assert r3.status()[0] == 0 and rx.status()[0] == 0
    n = sc.n
    assert np.array_equal(r3.planes.rect[:n].cpu().numpy(), o["rect"])
    assert np.array_equal(r3.planes.chunk[:n].cpu().numpy(), o["chunk"])
    assert np.array_equal(r3.planes.d.cpu().numpy(), o["d"])
    p3 = r3.planes.rgba.float().cpu().numpy().astype(np.float64)
    px = rx.planes.rgba.float().cpu().numpy().astype(np.float64)
    keep = o["near"] == 0
    share = 1.0 - keep.mean()
    print("3dgs %s: %.3f %% of texels near a threshold" % (dtype, 100 * share))
    assert share < 0.01
    tol = TOL[dtype][0]
    err = np.abs(p3 - o["planes"]).max(-1)
    assert err[keep].max() <= tol, err[keep].max()
    matters = (np.abs(o["planes"] - ex["planes"]).max(-1) > 5e-3) & keep
    assert matters.sum() > 100
    assert (np.abs(p3 - px).max(-1)[matters] > 1e-3).all()
    want = orc.composite(o["ref"], p3, o["d"], o["count"], w.views.Vx, w.views.Vy, w.views.bilinear, w.views.bg)
    assert np.abs(v3 - want).max() <= 1e-4


def test_3dgs_blending_is_refused_where_not_implemented():
    # voxels, the adjoint and the batch blend in exact mode only
    from paper_2508_18540_gb300 import api
    w = S.workload_tiny()
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32", blend="3dgs")
    vw = S.workload_voxels(n=2000, res=64, N=4, V=3, base_res=32)
    with pytest.raises(ValueError):
        r.build(api.DeviceVoxels.from_scene(vw.scene))
    g = api.DeviceGaussians.from_scene(w.scene)
    r.render(g)
    with pytest.raises(ValueError):
        r.backward(g, torch.zeros_like(r.out))
    with pytest.raises(ValueError):
        api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32", blend="bogus")
