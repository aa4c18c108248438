"""Pins for the oracle's sparse-voxel path (Sec. 4.5: voxels chunked like
Gaussians; per-voxel volume rendering of a trilinear density along the
reference ray, as in SVR [sun2024sparse])."""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from paper_2508_18540_gb300 import synth as S


def _trilinear_field(dens8):
    grid = np.zeros((2, 2, 2))
    for c in range(8):
        grid[c & 1, (c >> 1) & 1, (c >> 2) & 1] = dens8[c]
    return RegularGridInterpolator(([0.0, 1.0], [0.0, 1.0], [0.0, 1.0]), grid, method="linear")


def test_simpson_is_exact_for_trilinear_density(orc):
    rng = np.random.default_rng(0)
    for _ in range(30):
        lo = rng.uniform(-1, 1, 3)
        side = rng.uniform(0.01, 0.5)
        dens = rng.uniform(0, 5, 8).astype(np.float32)
        target = lo + side * rng.uniform(0.2, 0.8, 3)
        o = target - rng.normal(size=3) * 3.0
        d = target - o
        d /= np.linalg.norm(d)
        alpha, seg = orc.voxel_alpha(lo, side, dens, o, d)
        assert seg > 0
        # midpoint quadrature, 1e4 steps, of the library trilinear interpolant
        f = _trilinear_field(dens.astype(np.float64))
        # entry / exit by dense search along the ray
        ts = np.linspace(0, 10, 200001)
        pts = o[None] + ts[:, None] * d[None]
        inside = np.all((pts >= lo) & (pts <= lo + side), axis=1)
        t0, t1 = ts[inside][0], ts[inside][-1]
        assert seg == pytest.approx(t1 - t0, abs=2e-4)
        # refine the bracket with the exact segment from the oracle's length
        n = 10000
        tm = np.linspace(0, 1, n, endpoint=False) + 0.5 / n
        # exact entry point: bisection on the inside test
        a, b = t0 - 1e-4, t0
        for _ in range(80):
            m = 0.5 * (a + b)
            p = o + m * d
            if np.all((p >= lo) & (p <= lo + side)):
                b = m
            else:
                a = m
        te = b
        q = o[None] + (te + tm[:, None] * seg) * d[None]
        loc = np.clip((q - lo) / side, 0, 1)
        integral = f(loc).sum() * seg / n
        assert -math.log1p(-alpha) == pytest.approx(integral, rel=1e-7, abs=1e-12)


def test_constant_density_chord(orc):
    lo = np.array([0.0, 0.0, 5.0])
    side = 0.25
    dens = np.full(8, 2.0, np.float32)
    o = np.array([0.1, 0.2, 0.0])
    alpha, seg = orc.voxel_alpha(lo, side, dens, o, np.array([0.0, 0.0, 1.0]))
    assert seg == pytest.approx(side, rel=1e-15)
    assert alpha == pytest.approx(1 - math.exp(-2.0 * side), rel=1e-14)
    miss, seg = orc.voxel_alpha(lo, side, dens, np.array([1.0, 0.2, 0.0]), np.array([0.0, 0.0, 1.0]))
    assert miss == 0.0 and seg == 0.0


def _voxel_scene(n, seed, base=0.05):
    rng = np.random.default_rng(seed)
    ijk = rng.integers(-20, 20, (n, 3)).astype(np.int32)
    level = rng.integers(0, 3, n).astype(np.uint8)
    return S.VoxelScene(ijk, level, np.array([0.0, 0.0, 3.0]), base,
                        rng.uniform(0, 6, (n, 8)).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32))


def _cameras():
    a = 0.25
    R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    c2 = S.identity_camera(32, 50.0, t=(0.1, 0.0, 0.4))
    c2.R = R
    # non-square: different focal lengths along x and y
    c3 = S.Camera(np.eye(3), np.zeros(3), math.radians(50.0), math.radians(34.0), 40, 24)
    return [S.identity_camera(32, 50.0), c2, c3]


def _ref_ray_world(r, cam, x, y):
    """Reference-camera ray through plane pixel (x, y), in world coordinates."""
    u = (2 * x + 1) / r.W - 1
    v = (2 * y + 1) / r.H - 1
    dc = np.array([u * r.tthp_x, v * r.tthp_y, 1.0])
    R = np.asarray(cam.R)
    centre_cam = np.array([0.0, 0.0, 0.0])  # reference centre in its own frame
    o = R.T @ (centre_cam + np.array([0.0, 0.0, r.D_forward]) - np.asarray(cam.t))
    d = R.T @ dc
    return o, d / np.linalg.norm(d)


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_voxel_footprint_contains_every_hitting_ray(orc, ci):
    cam = _cameras()[ci]
    disp = S.display_for(3.0, 0.1)
    r = orc.make_ref(cam, disp)
    sc = _voxel_scene(30, 1 + ci, base=0.2)
    sc.ijk[:] = sc.ijk // 4
    z, valid, rect = orc.voxel_decide(r, sc)
    n_hit = 0
    for v in range(sc.n):
        s = sc.base_size * 2.0 ** -int(sc.level[v])
        lo = sc.origin + sc.ijk[v] * s
        x0, y0, x1, y1 = rect[v]
        for y in range(r.H):
            for x in range(r.W):
                o, d = _ref_ray_world(r, cam, x, y)
                _, seg = orc.voxel_alpha(lo, s, sc.density8[v], o, d)
                if seg > 0:
                    n_hit += 1
                    assert valid[v] and x0 <= x <= x1 and y0 <= y <= y1
    assert n_hit > 40


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_single_voxel_plane_is_its_opacity(orc, ci):
    cam = _cameras()[ci]
    disp = S.display_for(3.0, 0.1)
    sc = _voxel_scene(1, 5 + ci, base=0.4)
    sc.ijk[0] = [-1, 0, 0]
    sc.level[0] = 0
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile",
                     with_views=False)
    r = out["ref"]
    assert out["valid"][0] == 1
    s = sc.base_size
    lo = sc.origin + sc.ijk[0] * s
    P = out["planes"][0]
    for y in range(r.H):
        for x in range(r.W):
            o, d = _ref_ray_world(r, cam, x, y)
            a, _ = orc.voxel_alpha(lo, s, sc.density8[0], o, d)
            assert P[y, x, 3] == pytest.approx(a, abs=1e-12)
            assert np.allclose(P[y, x, :3], a * sc.rgb[0], atol=1e-12)


def test_two_voxels_compose_front_to_back(orc):
    # two overlapping voxels in one chunk blend with the "over" operator:
    # colour C_front + (1 - A_front) C_back, opacity 1 - (1 - A_front)(1 - A_back),
    # where each single-voxel plane is rendered alone
    cam = S.identity_camera(32, 50.0)
    disp = S.display_for(3.0, 0.1)
    rng = np.random.default_rng(21)
    ijk = np.array([[-1, -1, 0], [-1, -1, 1]], np.int32)
    sc = S.VoxelScene(ijk, np.zeros(2, np.uint8), np.array([0.1, 0.05, 3.0]), 0.4,
                      rng.uniform(0.5, 3.0, (2, 8)).astype(np.float32), rng.uniform(0, 1, (2, 3)).astype(np.float32))
    args = dict(camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile", with_views=False)
    both = orc.render(scene=sc, **args)["planes"][0]
    front = orc.render(scene=sc.subset([0]), **args)["planes"][0]
    back = orc.render(scene=sc.subset([1]), **args)["planes"][0]
    assert ((front[..., 3] > 0.05) & (back[..., 3] > 0.05)).sum() >= 10
    assert np.allclose(both[..., :3], front[..., :3] + (1 - front[..., 3:]) * back[..., :3], atol=1e-12)
    assert np.allclose(1 - both[..., 3], (1 - front[..., 3]) * (1 - back[..., 3]), atol=1e-12)


def test_voxel_depth_is_centre_depth(orc):
    cam = S.identity_camera(32)
    disp = S.display_for(3.0, 0.1)
    r = orc.make_ref(cam, disp)
    sc = _voxel_scene(10, 9)
    z, valid, rect = orc.voxel_decide(r, sc)
    for v in range(sc.n):
        s = sc.base_size * 2.0 ** -int(sc.level[v])
        c = sc.origin + (sc.ijk[v] + 0.5) * s
        assert z[v] == pytest.approx(c[2] - r.D_forward, rel=1e-15)


def test_voxel_near_plane_culling(orc):
    # a voxel is kept only if its whole cube lies past z_near (0.2) on
    # reference depth: a cube straddling z_near, or one between the
    # reference camera and z_near, is culled; one just beyond is kept
    cam = S.identity_camera(32)
    disp = S.display_for(3.0, 0.1)
    r = orc.make_ref(cam, disp)
    side = 0.05
    lows = [r.D_forward + 0.18, r.D_forward + 0.05, r.D_forward + 0.21, 1.0]   # cube low z (base frame)
    ijk = np.array([[-1, -1, 0]] * len(lows), np.int32)
    rng = np.random.default_rng(3)
    dens = rng.uniform(0, 6, (len(lows), 8)).astype(np.float32)
    rgb = rng.uniform(0, 1, (len(lows), 3)).astype(np.float32)
    valid = []
    for zlo, d8, c in zip(lows, dens, rgb):
        sc = S.VoxelScene(ijk[:1], np.zeros(1, np.uint8), np.array([0.0, 0.0, zlo]), side, d8[None], c[None])
        valid.append(int(orc.voxel_decide(r, sc)[1][0]))
    assert valid == [0, 0, 1, 1]


def test_generated_sparse_grid(orc):
    # small version of the 3-level sparse grid workload
    sc = S.sparse_voxels(20_000, 0, base_res=64)
    assert sc.n == 20_000
    assert set(np.unique(sc.level).tolist()) <= {0, 1, 2}
    assert np.all(sc.density8 >= 0)
    # leaves do not overlap: map each to its level-2 cell range
    scale = 4 >> sc.level.astype(np.int64)
    lo = sc.ijk.astype(np.int64) * scale[:, None]
    cells = set()
    for v in range(sc.n):
        for dz in range(scale[v]):
            for dy in range(scale[v]):
                for dx in range(scale[v]):
                    key = (lo[v, 0] + dx, lo[v, 1] + dy, lo[v, 2] + dz)
                    assert key not in cells
                    cells.add(key)
