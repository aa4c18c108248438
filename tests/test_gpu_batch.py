"""Batched rendering (lf_batch_*): several uneven scenes through one
persistent raster launch and one persistent composite launch, graph capture
and the autotuner. With one chunk group the batch must give exactly the
planes and views that the same scenes give one by one (same arithmetic), for
every plan; with 2 or 4 chunk groups (planes composited in shares and
composed in order) the planes are the same and the views change only in
rounding, and every scene's views stay within the FP16 tolerance of the
parity tests against the FP64 oracle."""
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
    for vg in (3, 5, 9, 15):
        for tx in (128, 256, 512):
            for sch in (0, 1, 2):
                b.prepare({"views_per_thread": vg, "tile_x": tx, "chunk_groups": 1, "schedule": sch})
                for o in b.outputs:
                    o.fill_(float("nan"))
                b.render()
                b.synchronize()
                for i, o in enumerate(b.outputs):
                    assert torch.equal(o, ref[i]), (vg, tx, sch, i)
    b.close()


@pytest.mark.parametrize("groups", [1, 2, 4])
@pytest.mark.parametrize("schedule", [0, 1])
def test_chunk_groups_against_oracle(orc, groups, schedule):
    # the planes are cut into 1, 2 or 4 shares composited separately and
    # composed front to back: planes bit-identical to one-by-one, views equal
    # to the one-by-one views up to FP32 rounding of the composition, and
    # within the FP16 tolerance of the FP64 oracle
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16", max_chunk_groups=4)
    b.prepare({"views_per_thread": 5, "tile_x": 256, "chunk_groups": groups, "schedule": schedule})
    for o in b.outputs:
        o.fill_(float("nan"))
    b.render()
    b.synchronize()
    assert b.status() == 0
    for i, w in enumerate(wls):
        want, want_pl = _single(w, "f16")
        assert torch.equal(b.planes[i].rgba, want_pl), i
        assert float((b.outputs[i] - want).abs().max()) <= 1e-5, (groups, i)
        o = orc.render(w)
        v = b.outputs[i].cpu().numpy().astype(np.float64)
        assert np.abs(v - o["views"]).max() <= 4e-3, (groups, i)
        for k in range(v.shape[0]):
            assert G.psnr(v[k], o["views"][k]) >= 60.0, (groups, i, k)
    b.close()


@pytest.mark.parametrize("schedule", [1, 2])
def test_graph_capture_replays_and_sees_new_inputs(schedule):
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")
    b.prepare({"views_per_thread": 9, "tile_x": 512, "chunk_groups": 1, "schedule": schedule})
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
    b = api.BatchRenderer(wls, "f16", max_chunk_groups=4)
    plan, ms = b.autotune(reps=1)
    assert plan["views_per_thread"] in (3, 5, 9, 15) and plan["tile_x"] in (128, 256, 512)
    assert plan["chunk_groups"] in (1, 2, 4) and plan["schedule"] in (0, 1, 2)
    assert ms > 0
    b.render()
    if plan["chunk_groups"] == 1:
        _check_equal(b, wls, "f16")
    else:
        b.synchronize()
        assert b.status() == 0
        for i, w in enumerate(wls):
            want, want_pl = _single(w, "f16")
            assert torch.equal(b.planes[i].rgba, want_pl), i
            assert float((b.outputs[i] - want).abs().max()) <= 1e-5, i
    b.close()


def test_chunk_group_workspace_is_checked():
    wls = _scenes()
    b = api.BatchRenderer(wls, "f16")           # workspace for one chunk group
    with pytest.raises(api.L.LFError) as e:
        b.prepare({"views_per_thread": 9, "tile_x": 512, "chunk_groups": 2, "schedule": 0})
    assert e.value.status == api.L.LF_ERR_WORKSPACE
    with pytest.raises(api.L.LFError) as e:
        b.prepare({"views_per_thread": 9, "tile_x": 512, "chunk_groups": 3, "schedule": 0})
    assert e.value.status == api.L.LF_ERR_INVALID_ARG
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
