"""The seeded synthetic inputs match the recipe they stand for (shapes,
ranges and distribution moments of the tiny, display, voxel, batched and
fitting workloads), and the same seed gives the same scene."""
import math

import numpy as np
import pytest

from paper_2508_18540_gb300 import synth as S


def test_tiny_workload_recipe():
    w = S.workload_tiny()
    g = w.scene
    assert g.n == 10_000
    assert g.means[:, :2].min() >= -1 and g.means[:, :2].max() <= 1
    assert g.means[:, 2].min() >= 2 and g.means[:, 2].max() <= 6
    assert np.array_equal(g.scales[:, 0], g.scales[:, 1]) and np.array_equal(g.scales[:, 0], g.scales[:, 2])
    ls = np.log(g.scales[:, 0].astype(np.float64))
    assert ls.mean() == pytest.approx(math.log(0.02), abs=0.02) and ls.std() == pytest.approx(0.3, abs=0.02)
    assert np.all(g.quats == np.array([1, 0, 0, 0], np.float32))
    assert g.opacity.min() >= 0.1 and g.opacity.max() <= 0.9
    assert (w.camera.Nx, w.camera.Ny) == (128, 128) and w.camera.theta_x == pytest.approx(math.radians(50))
    assert (w.N, w.binning, w.views.Vx, w.views.Vy) == (16, "disparity", 9, 1)
    assert w.display.D_focal == 3.0
    assert 3.0 * math.tan(w.display.phi_x / 2) == pytest.approx(0.1, rel=1e-12)   # outermost offset = baseline


def test_display_workload_recipe():
    g = S.blob_gaussians(200_000, 2)
    z = g.means[:, 2].astype(np.float64)
    # 200 blobs: members of blob b are b, b + 200, ...; blob spread 0.05 z around centres in [1.5, 10]
    cz = np.array([z[b::200].mean() for b in range(200)])
    assert cz.min() > 1.4 and cz.max() < 10.1
    sd = np.array([z[b::200].std() for b in range(200)])
    assert np.allclose(sd / cz, 0.05, rtol=0.1)
    assert np.allclose(np.linalg.norm(g.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    ls = np.log(g.scales.astype(np.float64))
    assert np.allclose(ls.mean(axis=0), math.log(0.01), atol=0.01) and np.allclose(ls.std(axis=0), 0.5, atol=0.01)
    o = g.opacity.astype(np.float64)
    assert o.mean() == pytest.approx(0.5, abs=0.005) and o.var() == pytest.approx(0.05, abs=0.002)   # Beta(2, 2)
    assert g.rgb.min() >= 0 and g.rgb.max() <= 1
    w = S.workload_display(n=1000)
    assert (w.camera.Nx, w.N, w.binning, w.views.Vx) == (512, 64, "quantile", 45)
    assert w.display.D_focal == pytest.approx(2.0 / (1 / 1.5 + 1 / 10.0), rel=1e-12)
    assert w.display.D_focal * math.tan(w.display.phi_x / 2) == pytest.approx(0.15, rel=1e-12)


def test_voxel_workload_recipe():
    v = S.sparse_voxels(20_000, 0, base_res=64)
    assert v.n == 20_000
    assert set(np.unique(v.level).tolist()) <= {0, 1, 2}
    assert v.base_size == pytest.approx(4.0 / 64)
    side = v.base_size * 2.0 ** -v.level.astype(np.float64)
    lo = v.origin + v.ijk * side[:, None]
    assert lo.min() >= -2 - 1e-9 and (lo + side[:, None]).max() <= 2 + 1e-9      # inside [-2, 2]^3
    assert v.density8.min() >= 0                                                  # softplus
    assert v.rgb.min() >= 0 and v.rgb.max() <= 1
    w = S.workload_voxels(n=2000, res=64, N=4, V=3, base_res=32)
    assert np.allclose(w.camera.t, [0, 0, 6])                                     # volume at depth [4, 8]
    assert w.display.D_focal == pytest.approx(2.0 / (1 / 4.0 + 1 / 8.0), rel=1e-12)


def test_batched_and_fit_recipes():
    ws = S.workloads_batched(scale=0.001)
    spec = [(9, 256, 64), (45, 384, 64), (45, 512, 128), (96, 512, 128), (96, 768, 256), (128, 1024, 512)]
    assert [(w.views.Vx, w.camera.Nx, w.N) for w in ws] == spec
    sizes = [w.scene.n for w in ws]
    assert sizes == sorted(sizes)
    f = S.workload_fit(n=5000)
    p = S.perturbed(f.scene, 1)
    dm = (p.means - f.scene.means).astype(np.float64)
    assert dm.std() == pytest.approx(0.01, rel=0.05)
    assert p.opacity.min() >= 0.01 and p.opacity.max() <= 0.99
    assert np.array_equal(p.scales, f.scene.scales) and np.array_equal(p.rgb, f.scene.rgb)


def test_seeds_are_reproducible():
    a, b, c = S.blob_gaussians(5000, 7), S.blob_gaussians(5000, 7), S.blob_gaussians(5000, 8)
    assert all(np.array_equal(x, y) for x, y in zip((a.means, a.scales, a.quats, a.opacity, a.rgb),
                                                     (b.means, b.scales, b.quats, b.opacity, b.rgb)))
    assert not np.array_equal(a.means, c.means)
    v1, v2 = S.sparse_voxels(3000, 1, base_res=32), S.sparse_voxels(3000, 1, base_res=32)
    assert np.array_equal(v1.ijk, v2.ijk) and np.array_equal(v1.density8, v2.density8)
