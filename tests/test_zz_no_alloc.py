"""lf_composite_noalloc, the form of lf_composite for callers that cannot
give the library device memory (a present callback of a display runtime may
not call a device allocator), against lf_composite on the same planes: two
calls in a row. Both run the same coefficient and composite kernels on the
same planes, so the views must agree bit for bit, and the static scratch's
error word must read LF_OK after each call. Named to be collected last; it
also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2508_18540_gb300 import api
from paper_2508_18540_gb300 import synth as S

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_18540_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("bilinear", [False, True])
def test_noalloc_matches_workspace_composite(bilinear):
    w = S.workload_tiny()
    views = S.ViewSet(w.views.Vx, 1, bilinear, (0.1, 0.0, 0.2))
    r = api.LightFieldRenderer(w.camera, w.display, views, w.N, w.binning, "f32")
    g = api.DeviceGaussians.from_scene(w.scene)
    want = r.render(g).clone()
    for _ in range(2):
        out = torch.full_like(want, float("nan"))
        api.lf_composite_noalloc(r.planes, r.ref, views, out)
        assert api.lf_composite_noalloc_status(w.N, views) == api.L.LF_OK
        torch.cuda.synchronize()
        assert torch.equal(out, want)


def test_noalloc_rejects_oversized_request():
    w = S.workload_tiny()
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    # 4096 planes x 32 views: 1.5 MiB of coefficient tables; rejected on the
    # host before any device work (the plane tensor is a placeholder)
    big = S.ViewSet(32, 1)
    ref = r.ref
    pl = api.Planes(torch.empty((4096, 1, 1, 4), dtype=torch.float32, device="cuda"),
                    torch.zeros(4096, dtype=torch.float64, device="cuda"),
                    torch.zeros(4096, dtype=torch.int32, device="cuda"),
                    torch.zeros(1, dtype=torch.int32, device="cuda"),
                    torch.zeros((1, 4), dtype=torch.int32, device="cuda"), api.L.LF_F32)
    out = torch.empty((32, ref.base.Ny, ref.base.Nx, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(api.L.LFError) as e:
        api.lf_composite_noalloc(pl, ref, big, out)
    assert e.value.status == api.L.LF_ERR_WORKSPACE
    assert "static limit" in str(e.value)
    assert api.lf_composite_noalloc_max_bytes() == 1 << 20
