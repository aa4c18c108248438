"""Batched rendering (lf_batch_*): several uneven scenes through one
persistent raster launch and one persistent composite launch, graph capture
and the autotuner. The batch must give exactly the planes and views that the
same scenes give one by one (same arithmetic), for every plan, and the
one-by-one path is itself checked against the FP64 oracle here for one scene
(FP16 tolerance of the parity tests)."""
import numpy as np
import pytest
import torch

from paper_2508_18540_gb300 import api
from paper_2508_18540_gb300 import synth as S
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_18540_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _scenes():
    # uneven primitive counts, resolutions, N and view counts (the batched
    # workload's shape at test size)
    spec = [(2000, 9, 64, 8), (6000, 13, 96, 16), (4000, 5, 128, 12), (1200, 21, 80, 6)]
    return [S.workload_display(seed=30 + i, n=n, res=res, N=N, V=V) for i, (n, V, res, N) in enumerate(spec)]


def _single(w, dtype):
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, dtype)
    g = api.DeviceGaussians.from_scene(w.scene)
    out = r.render(g).clone()
    pl = r.planes.rgba.clone()
    torch.cuda.synchronize()
    return out, pl


def _check_equal(batch, wls, dtype):
    batch.synchronize()
    assert batch.status() == 0
    for i, w in enumerate(wls):
        want, want_pl = _single(w, dtype)
        assert torch.equal(batch.planes[i].rgba, want_pl), i
        assert torch.equal(batch.outputs[i], want), i


@pytest.mark.parametrize("dtype", ["f16", "f32", "u8"])
def test_batch_equals_one_by_one(dtype):
    wls = _scenes()
    b = api.BatchRenderer(wls, dtype)
    b.render()
    _check_equal(b, wls, dtype)
    b.close()


def test_every_plan_gives_the_same_result():
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")
    b.render()
    b.synchronize()
    ref = [o.clone() for o in b.outputs]
    for vg in (3, 5, 9):
        for tx in (128, 256, 512):
            for ppt, sch in ((4, 0), (8, 1), (4, 2)):
                b.prepare({"views_per_thread": vg, "tile_x": tx, "raster_ppt": ppt, "schedule": sch})
                for o in b.outputs:
                    o.fill_(float("nan"))
                b.render()
                b.synchronize()
                for i, o in enumerate(b.outputs):
                    assert torch.equal(o, ref[i]), (vg, tx, ppt, sch, i)
    b.close()


@pytest.mark.parametrize("schedule", [1, 2])
def test_graph_capture_replays_and_sees_new_inputs(schedule):
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")
    b.prepare({"views_per_thread": 9, "tile_x": 512, "raster_ppt": 4, "schedule": schedule})
    b.capture()
    for _ in range(2):
        for o in b.outputs:
            o.fill_(float("nan"))
        b.launch()
        b.synchronize()
        assert b.status() == 0
        for i, w in enumerate(wls):
            want, _ = _single(w, "f16")
            assert torch.equal(b.outputs[i], want), i
    # the graph reads the scene buffers in place: new colours show up
    with torch.no_grad():
        b.prims[1].rgb.mul_(0.5)
    b.launch()
    b.synchronize()
    w = wls[1]
    sc = S.GaussianScene(w.scene.means, w.scene.scales, w.scene.quats, w.scene.opacity,
                         (w.scene.rgb * np.float32(0.5)).astype(np.float32))
    w2 = S.Workload(w.name, sc, w.camera, w.display, w.views, w.N, w.binning)
    want, _ = _single(w2, "f16")
    assert torch.equal(b.outputs[1], want)
    b.close()


def test_autotune_picks_a_valid_plan():
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")
    plan, ms = b.autotune(reps=1)
    assert plan["views_per_thread"] in (3, 5, 9) and plan["tile_x"] in (128, 256, 512)
    assert plan["raster_ppt"] in (4, 8) and plan["schedule"] in (0, 1, 2)
    assert ms > 0
    b.render()
    _check_equal(b, wls, "f16")
    b.close()


def test_one_batched_scene_against_oracle(orc):
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")
    b.render()
    b.synchronize()
    o = orc.render(wls[2])
    v = b.outputs[2].cpu().numpy().astype(np.float64)
    assert np.abs(v - o["views"]).max() <= 4e-3
    for k in range(v.shape[0]):
        assert G.psnr(v[k], o["views"][k]) >= 60.0
    b.close()
