"""GPU adjoints (lf_composite_backward, lf_build_mpi_backward_*) against
central finite differences of the FP64 oracle.

The integer structure (culling, chunks, plane depths d_k, footprints, depth
order) is frozen at the unperturbed point: the oracle's own decisions, which
the parity tests show to be bit-identical to the GPU's. The loss is the
linear functional L = sum(W * views) with seeded Gaussian weights W, so
dL/dviews = W. Step h = 1e-6 max(1, |x|) per element (FP64). Opacities are
kept below 0.95 so the alpha = 0.99 clamp never binds (a kink the finite
difference would straddle). Bar: relative L2 error <= 1e-3 per parameter
group over the sampled elements, and the same for random directional
derivatives over whole groups.
"""
import numpy as np
import pytest
import torch

from paper_2508_18540_gb300 import api
from paper_2508_18540_gb300 import autograd as AG
from paper_2508_18540_gb300 import synth as S

pytestmark = pytest.mark.gpu

REL_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_18540_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _fd_scene(seed=5, n=2000, res=64, N=8, V=5):
    # the differentiable workload's distributions at the finite-difference size
    # plus 20 culled copies: 10 behind the camera, 10 far outside the frustum
    w = S.workload_display(seed=seed, n=n, res=res, N=N, V=V)
    sc = w.scene
    out = sc.subset(np.arange(20))
    out.means = out.means.copy()
    out.means[:10, 2] = -2.0
    out.means[10:, 0] = 50.0
    sc = S.GaussianScene(*(np.concatenate([a, b]) for a, b in
                           zip((sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb),
                               (out.means, out.scales, out.quats, out.opacity, out.rgb))))
    sc.opacity = np.minimum(sc.opacity, 0.95).astype(np.float32)
    return S.Workload(w.name + "_fd", sc, w.camera, w.display, w.views, w.N, w.binning)


class _OracleLoss:
    """L(params) = sum(W * views) through the FP64 oracle with frozen structure."""

    def __init__(self, orc, w, W):
        self.orc, self.w, self.W = orc, w, W
        self.ref = orc.make_ref(w.camera, w.display)
        z, valid, self.rect = orc.gauss_decide(self.ref, w.scene)
        self.order, self.chunk, self.d, self.count, self.M = orc.bin_primitives(self.ref, z, valid, w.N, w.binning)
        sc = w.scene
        self.p = {k: np.array(getattr(sc, k), np.float64) for k in ("means", "scales", "quats", "opacity", "rgb")}

    def __call__(self, p):
        o = self.orc
        sc = S.GaussianScene(p["means"], p["scales"], p["quats"], p["opacity"], p["rgb"])
        mean2d, conic, _ = o.gauss_values(self.ref, sc)
        planes = o.splat_gaussians(self.ref, self.order, self.chunk, self.rect, mean2d, conic, p["opacity"],
                                   p["rgb"], self.w.N)
        v = self.w.views
        views = o.composite(self.ref, planes, self.d, self.count, v.Vx, v.Vy, v.bilinear, v.bg)
        return float(np.sum(self.W * views))

    def fd_element(self, key, idx):
        p = {k: a.copy() for k, a in self.p.items()}
        x = p[key][idx]
        h = 1e-6 * max(1.0, abs(x))
        p[key][idx] = x + h
        lp = self(p)
        p[key][idx] = x - h
        lm = self(p)
        return (lp - lm) / (2 * h)

    def fd_direction(self, key, u, scale):
        p = {k: a.copy() for k, a in self.p.items()}
        h = 1e-6 * max(1.0, scale)
        base = p[key].copy()
        p[key] = base + h * u
        lp = self(p)
        p[key] = base - h * u
        lm = self(p)
        return (lp - lm) / (2 * h)


def _gpu_grads(w, W, dtype="f32", save_state=False):
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, dtype, save_state=save_state)
    g = api.DeviceGaussians.from_scene(w.scene)
    r.render(g)
    grads, dplanes = r.backward(g, torch.from_numpy(W.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    st, _, _ = r.status()
    assert st == 0
    return {"means": grads.dmeans.cpu().numpy().astype(np.float64),
            "scales": grads.dscales.cpu().numpy().astype(np.float64),
            "quats": grads.dquats.cpu().numpy().astype(np.float64),
            "opacity": grads.dopacity.cpu().numpy().astype(np.float64),
            "rgb": grads.drgb.cpu().numpy().astype(np.float64)}, dplanes, r


@pytest.fixture(scope="module")
def fd_case(orc):
    w = _fd_scene()
    rng = np.random.default_rng(11)
    W = rng.normal(size=(w.views.Vx * w.views.Vy, w.camera.Ny, w.camera.Nx, 4))
    loss = _OracleLoss(orc, w, W)
    g, _, _ = _gpu_grads(w, W)
    return w, W, loss, g


def test_gaussian_gradients_elementwise(fd_case):
    w, W, loss, g = fd_case
    rng = np.random.default_rng(12)
    culled_in = np.flatnonzero(loss.chunk >= 0)
    assert culled_in.size > 1000
    pick = rng.choice(culled_in, 30, replace=False)
    for key, width in (("means", 3), ("scales", 3), ("quats", 4), ("opacity", 1), ("rgb", 3)):
        fd, gp = [], []
        for i in pick:
            for c in range(width):
                idx = (i,) if width == 1 else (i, c)
                fd.append(loss.fd_element(key, idx))
                gp.append(g[key][idx])
        fd, gp = np.array(fd), np.array(gp)
        assert np.linalg.norm(fd) > 0, key
        assert _rel(gp, fd) <= REL_TOL, (key, _rel(gp, fd))


def test_gaussian_gradients_directional(fd_case):
    w, W, loss, g = fd_case
    rng = np.random.default_rng(13)
    for key in ("means", "scales", "quats", "opacity", "rgb"):
        for _ in range(3):
            u = rng.normal(size=loss.p[key].shape)
            u /= np.linalg.norm(u)
            fd = loss.fd_direction(key, u, float(np.abs(loss.p[key]).max()))
            an = float(np.sum(g[key] * u))
            assert abs(an - fd) <= REL_TOL * max(abs(fd), 1e-12) + 1e-9, (key, an, fd)


def test_gaussian_gradients_with_split_lists(orc):
    # 20,000 faint Gaussians in a 128^2 frame, one chunk: (super-tile,
    # chunk) lists of thousands of entries, which the raster cuts into parts;
    # the adjoint walks every part from the composition of the partials in
    # front of it. FP32 planes against finite differences of the FP64
    # oracle; FP16 planes track FP32
    from tests import gpu_util as G
    sc = S.uniform_gaussians(20_000, 23, opacity=(0.02, 0.3))
    t = S.workload_tiny()
    w = S.Workload("split_fd", sc, t.camera, t.display, S.ViewSet(3), 1, "quantile")
    o = orc.render(w)
    assert G.longest_super_tile_list(o, 1) > 2 * 1024   # three parts or more
    rng = np.random.default_rng(17)
    W = rng.normal(size=(3, w.camera.Ny, w.camera.Nx, 4))
    loss = _OracleLoss(orc, w, W)
    g, _, _ = _gpu_grads(w, W)
    for key in ("means", "scales", "opacity", "rgb"):
        for _ in range(2):
            u = rng.normal(size=loss.p[key].shape)
            u /= np.linalg.norm(u)
            fd = loss.fd_direction(key, u, float(np.abs(loss.p[key]).max()))
            an = float(np.sum(g[key] * u))
            assert abs(an - fd) <= REL_TOL * max(abs(fd), 1e-12) + 1e-9, (key, an, fd)
    # isotropic Gaussians: a rotation changes nothing, the quaternion
    # gradient is zero up to rounding
    assert np.linalg.norm(g["quats"]) <= 1e-5 * np.linalg.norm(g["means"])
    g16, _, _ = _gpu_grads(w, W, "f16")
    for key in ("means", "scales", "opacity", "rgb"):
        assert _rel(g16[key], g[key]) <= 2e-2, key


def test_culled_gaussians_get_zero_gradient(fd_case):
    w, W, loss, g = fd_case
    out = loss.chunk < 0
    assert out.any()
    for key in g:
        assert np.all(g[key][out] == 0.0), key


@pytest.mark.parametrize("save_state", [False, True])
def test_composite_adjoint_against_fd(orc, save_state):
    # dplanes of the composite alone, on random texels, nearest and bilinear;
    # the adjoint's own two walks, or one walk from the saving forward's state
    for bilinear in (False, True):
        w = _fd_scene(seed=6, n=1500)
        w = S.Workload(w.name, w.scene, w.camera, w.display, S.ViewSet(5, 1, bilinear, (0.2, 0.1, 0.3)), w.N,
                       w.binning)
        rng = np.random.default_rng(14)
        W = rng.normal(size=(5, w.camera.Ny, w.camera.Nx, 4))
        _, dplanes, r = _gpu_grads(w, W, save_state=save_state)
        dp = dplanes.cpu().numpy().astype(np.float64)
        o = orc.render(w)
        planes = o["planes"].copy()
        ref, d, count = o["ref"], o["d"], o["count"]

        def L(pl):
            return float(np.sum(W * orc.composite(ref, pl, d, count, 5, 1, bilinear, (0.2, 0.1, 0.3))))

        nz = np.argwhere(np.abs(dp).sum(axis=-1) > 0)
        assert nz.shape[0] > 100
        sel = nz[rng.choice(nz.shape[0], 40, replace=False)]
        fd, an = [], []
        for (k, y, x) in sel:
            for c in range(4):
                p = planes.copy()
                x0 = p[k, y, x, c]
                h = 1e-6 * max(1.0, abs(x0))
                p[k, y, x, c] = x0 + h
                lp = L(p)
                p[k, y, x, c] = x0 - h
                lm = L(p)
                fd.append((lp - lm) / (2 * h))
                an.append(dp[k, y, x, c])
        assert _rel(np.array(an), np.array(fd)) <= REL_TOL


def test_fp16_plane_gradients_track_fp32(fd_case):
    w, W, loss, g32 = fd_case
    g16, _, _ = _gpu_grads(w, W, "f16")
    for key in g32:
        assert _rel(g16[key], g32[key]) <= 2e-2, key


def test_voxel_gradients_against_fd(orc):
    cam = S.identity_camera(48, t=(0.0, 0.0, 6.0))
    vs = S.sparse_voxels(1500, 7, base_res=32)
    sc = S.VoxelScene(vs.ijk, vs.level, vs.origin, vs.base_size,
                      (0.5 * vs.density8).astype(np.float32), vs.rgb)
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15)
    views = S.ViewSet(5, 1, False)
    N = 6
    rng = np.random.default_rng(15)
    W = rng.normal(size=(5, 48, 48, 4))
    r = api.LightFieldRenderer(cam, disp, views, N, "quantile", "f32")
    v = api.DeviceVoxels.from_scene(sc)
    r.render(v)
    grads, _ = r.backward(v, torch.from_numpy(W.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    gd = grads.ddensity8.cpu().numpy().astype(np.float64)
    gc = grads.drgb.cpu().numpy().astype(np.float64)

    ref = orc.make_ref(cam, disp)
    z, valid, rect = orc.voxel_decide(ref, sc)
    order, chunk, d, count, M = orc.bin_primitives(ref, z, valid, N, "quantile")
    base = {"density8": np.array(sc.density8, np.float64), "rgb": np.array(sc.rgb, np.float64)}

    def L(p):
        s2 = S.VoxelScene(sc.ijk, sc.level, sc.origin, sc.base_size, p["density8"], p["rgb"])
        planes = orc.splat_voxels(ref, order, chunk, rect, s2, N)
        return float(np.sum(W * orc.composite(ref, planes, d, count, 5, 1, False)))

    vis = np.flatnonzero(np.abs(gc).sum(axis=1) > 0)
    assert vis.size > 50
    pick = rng.choice(vis, 20, replace=False)
    for key, g, width in (("density8", gd, 8), ("rgb", gc, 3)):
        fd, an = [], []
        for i in pick:
            for c in range(width):
                p = {k: a.copy() for k, a in base.items()}
                x0 = p[key][i, c]
                h = 1e-6 * max(1.0, abs(x0))
                p[key][i, c] = x0 + h
                lp = L(p)
                p[key][i, c] = x0 - h
                lm = L(p)
                fd.append((lp - lm) / (2 * h))
                an.append(g[i, c])
        assert _rel(np.array(an), np.array(fd)) <= REL_TOL, key


def test_voxel_fp16_gradients_track_fp32():
    # FP16 planes: the voxel adjoint first walks each list for (C_end,
    # T_end) instead of reading them from the texel
    cam = S.identity_camera(48, t=(0.0, 0.0, 6.0))
    vs = S.sparse_voxels(1500, 7, base_res=32)
    sc = S.VoxelScene(vs.ijk, vs.level, vs.origin, vs.base_size,
                      (0.5 * vs.density8).astype(np.float32), vs.rgb)
    disp = S.display_for(S.harmonic_focal(4.0, 8.0), 0.15)
    views = S.ViewSet(5, 1, False)
    rng = np.random.default_rng(16)
    W = torch.from_numpy(rng.normal(size=(5, 48, 48, 4)).astype(np.float32)).cuda()
    out = {}
    for dtype in ("f32", "f16"):
        r = api.LightFieldRenderer(cam, disp, views, 6, "quantile", dtype)
        v = api.DeviceVoxels.from_scene(sc)
        r.render(v)
        grads, _ = r.backward(v, W)
        torch.cuda.synchronize()
        out[dtype] = (grads.ddensity8.cpu().numpy().astype(np.float64), grads.drgb.cpu().numpy().astype(np.float64))
    for a, b in zip(out["f16"], out["f32"]):
        assert np.linalg.norm(b) > 0
        assert _rel(a, b) <= 2e-2


@pytest.mark.parametrize("save_state", [False, True])
def test_autograd_function_and_fit_step(save_state):
    # torch.autograd path: gradients equal the direct adjoint call, and a few
    # gradient steps on opacities reduce the L2 loss against target views
    w = _fd_scene(seed=8, n=3000)
    tgt_scene = S.perturbed(w.scene, 9, mean_std=0.0)
    r_t = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    target = r_t.render(api.DeviceGaussians.from_scene(tgt_scene)).clone()
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32", save_state=save_state)
    g = api.DeviceGaussians.from_scene(w.scene)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.quats, g.opacity, g.rgb)]
    views = AG.render_gaussians(r, *params)
    loss = ((views - target) ** 2).sum()
    loss.backward()
    grads, _ = r.backward(g, (2.0 * (views.detach() - target)).contiguous())
    # the adjoints sum with float atomics (dplanes over views, the per-primitive
    # sums over pixels), so two calls agree up to the order of those sums: an
    # element that cancels can move by more than 1e-4 of itself, the tensor by
    # a few FP32 rounding steps of its norm
    for p, ref_g in zip(params, (grads.dmeans, grads.dscales, grads.dquats, grads.dopacity, grads.drgb)):
        a, b = p.grad.double().cpu().numpy(), ref_g.double().cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-9, _rel(a, b)
    opa = params[3].detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([opa], lr=0.01)
    losses = []
    for _ in range(15):
        opt.zero_grad()
        v = AG.render_gaussians(r, params[0].detach(), params[1].detach(), params[2].detach(), opa,
                                params[4].detach())
        l2 = ((v - target) ** 2).sum()
        l2.backward()
        opt.step()
        with torch.no_grad():
            opa.clamp_(0.01, 0.99)
        losses.append(float(l2.detach()))
    assert losses[-1] < 0.8 * losses[0], losses


@pytest.mark.parametrize("dtype", ["f16", "u8"])
@pytest.mark.parametrize("bilinear", [False, True])
def test_staged_and_unstaged_composite_adjoints_agree(dtype, bilinear):
    # The staged adjoint (plane rows streamed through shared memory) runs when
    # plane rows start on 16-byte boundaries; a copy of the same planes one
    # texel off that boundary takes the unstaged adjoint. Both must give the
    # same dplanes up to FP32 rounding (T recovery, atomic summation order).
    w = _fd_scene(seed=7, n=3000, res=64, N=8)
    views = S.ViewSet(7, 1, bilinear, (0.2, 0.1, 0.3))
    r = api.LightFieldRenderer(w.camera, w.display, views, w.N, w.binning, dtype)
    r.render(api.DeviceGaussians.from_scene(w.scene))
    pl = r.planes
    gen = torch.Generator(device="cuda").manual_seed(3)
    dv = torch.randn((7, w.camera.Ny, w.camera.Nx, 4), device="cuda", generator=gen)
    shape = tuple(pl.rgba.shape)
    dp_staged = torch.empty(shape, dtype=torch.float32, device="cuda")
    api.lf_composite_backward(pl, r.ref, views, dv, dp_staged, r.cws)
    n_tex = shape[0] * shape[1] * shape[2]
    flat = torch.empty((n_tex + 1, 4), dtype=pl.rgba.dtype, device="cuda")
    moved = flat[1:].view(shape)
    moved.copy_(pl.rgba)
    assert moved.data_ptr() % 16 != 0
    pl2 = api.Planes(moved, pl.d, pl.count, pl.chunk, pl.rect, pl.dtype_code)
    dp_unstaged = torch.empty(shape, dtype=torch.float32, device="cuda")
    api.lf_composite_backward(pl2, r.ref, views, dv, dp_unstaged, r.cws)
    torch.cuda.synchronize()
    scale = float(dp_staged.abs().max())
    assert scale > 0.0
    assert float((dp_staged - dp_unstaged).abs().max()) <= 2e-5 * scale


def _opaque_planes(dtype, seed=21):
    # rendered planes with the alpha of 4 x 4 texel blocks (3 % of them) set
    # to 1 exactly (A = 1: T is 0 behind such a texel, as dense FP16 / U8
    # planes reach by rounding); bilinear samples inside a block get A = 1 or
    # 1 - a few ulp
    w = _fd_scene(seed=seed, n=3000, res=64, N=8)
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, dtype)
    r.render(api.DeviceGaussians.from_scene(w.scene))
    rgba = r.planes.rgba
    N, H, W = rgba.shape[:3]
    gen = torch.Generator(device="cuda").manual_seed(seed)
    blocks = torch.rand((N, (H + 3) // 4, (W + 3) // 4), device="cuda", generator=gen) < 0.03
    hit = blocks.repeat_interleave(4, 1).repeat_interleave(4, 2)[:, :H, :W]
    rgba[..., 3][hit] = 255 if dtype == "u8" else 1.0
    assert int(hit.sum()) > 50
    return w, r


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16", "u8"])
@pytest.mark.parametrize("bilinear", [False, True])
def test_saved_state_adjoint_matches_two_walks(dtype, bilinear):
    # lf_composite_save gives the views of lf_composite up to the colour
    # behind the plane where T falls below 2^-64, and
    # lf_composite_backward_saved the dplanes of lf_composite_backward up to
    # FP32 rounding (atomic order), with opaque texels (A = 1) in the planes;
    # the state names the stop plane of every pixel that has one. Staged
    # kernels, and the unstaged ones on a copy of the planes one texel off
    # the 16-byte boundary.
    w, r = _opaque_planes(dtype)
    views = S.ViewSet(7, 1, bilinear, (0.2, 0.1, 0.3))
    pl = r.planes
    V, Ny, Nx = 7, w.camera.Ny, w.camera.Nx
    cws = api.alloc_workspace(api.lf_composite_workspace_size(w.N, views), "cuda")
    gen = torch.Generator(device="cuda").manual_seed(5)
    dv = torch.randn((V, Ny, Nx, 4), device="cuda", generator=gen)
    shape = tuple(pl.rgba.shape)
    cases = [pl]
    if dtype != "f32":
        # one texel off: rows no longer start on 16-byte boundaries (FP32
        # texels are 16 bytes, so FP32 planes always stage)
        flat = torch.empty((shape[0] * shape[1] * shape[2] + 1, 4), dtype=pl.rgba.dtype, device="cuda")
        moved = flat[1:].view(shape)
        moved.copy_(pl.rgba)
        assert moved.data_ptr() % 16 != 0
        cases.append(api.Planes(moved, pl.d, pl.count, pl.chunk, pl.rect, pl.dtype_code))
    results = []
    for P in cases:
        plain = torch.empty((V, Ny, Nx, 4), device="cuda")
        saved = torch.full((V, Ny, Nx, 4), float("nan"), device="cuda")
        state = torch.full(api.composite_state_shape(r.ref, views), float("nan"), device="cuda")
        api.lf_composite(P, r.ref, views, plain, cws)
        api.lf_composite_save(P, r.ref, views, saved, state, cws)
        d2 = torch.empty(shape, dtype=torch.float32, device="cuda")
        d1 = torch.empty(shape, dtype=torch.float32, device="cuda")
        api.lf_composite_backward(P, r.ref, views, dv, d2, cws)
        api.lf_composite_backward_saved(P, r.ref, views, dv, state, d1, cws)
        assert api.lf_composite_status(w.N, views, cws) == 0
        assert float((saved - plain).abs().max()) <= 2e-6
        scale = float(d2.abs().max())
        assert scale > 0.0
        assert float((d1 - d2).abs().max()) <= 2e-5 * scale
        results.append((saved, state, d1))
    # the state's plane index: N where T never falls below 2^-64, else the
    # stop plane; staged and unstaged agree on it exactly
    # (bilinear: staged and unstaged round A differently, so a sample may be
    # exactly opaque in one and 1 - ulp in the other)
    k_st = results[0][1][..., 1].view(torch.int32)
    opq = k_st < w.N
    assert int((~opq).sum()) > 0 and bool((k_st >= 0).all())
    if not bilinear:
        assert int(opq.sum()) > 0
    if int(opq.sum()) > 0:
        alpha_opaque = results[0][0][..., 3][opq]
        assert float((alpha_opaque - 1.0).abs().max()) == 0.0      # T = 0 behind an opaque plane
    if len(results) == 2 and not bilinear:
        assert torch.equal(k_st, results[1][1][..., 1].view(torch.int32))
        assert float((results[0][0] - results[1][0]).abs().max()) <= 2e-6
        scale = float(results[0][2].abs().max())
        assert float((results[0][2] - results[1][2]).abs().max()) <= 2e-5 * scale


def test_saved_state_renderer_matches_oracle(orc):
    # the saving forward's views against the FP64 oracle (the display parity
    # bar), and the renderer falls back to the two-walk adjoint once it has
    # rebuilt without compositing
    w = _fd_scene(seed=12, n=3000, res=64, N=8)
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32", save_state=True)
    g = api.DeviceGaussians.from_scene(w.scene)
    v = r.render(g).cpu().numpy().astype(np.float64)
    o = orc.render(w)
    assert np.abs(v - o["views"]).max() <= 1e-4
    assert r.state_generation == r.generation
    r.build(g)
    assert r.state_generation != r.generation
    gen = torch.Generator(device="cuda").manual_seed(2)
    dv = torch.randn((w.views.Vx, w.camera.Ny, w.camera.Nx, 4), device="cuda", generator=gen)
    _, dp_two = r.backward(g, dv)
    r.composite()
    _, dp_one = r.backward(g, dv)
    torch.cuda.synchronize()
    scale = float(dp_two.abs().max())
    assert float((dp_one - dp_two).abs().max()) <= 2e-5 * scale
