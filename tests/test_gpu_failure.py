"""Failure detection without a GPU fault: every device-side wait of the
library is bounded in wall time; when it gives up, the kernel records it and
returns, the host reads LF_ERR_TIMEOUT, and the CUDA context stays usable.
The self-test waits on a shared-memory mbarrier that nothing arrives on."""
import time

import numpy as np
import pytest
import torch

from paper_2508_18540_gb300 import api
from paper_2508_18540_gb300 import synth as S
from paper_2508_18540_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_18540_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def test_bounded_wait_gives_up_and_context_survives(orc):
    s = torch.cuda.Stream()
    for limit_ms in (20, 200):
        t0 = time.perf_counter()
        st = api.lf_selftest_bounded_wait(limit_ms, s)
        dt = time.perf_counter() - t0
        assert st == L.LF_ERR_TIMEOUT, (st, L.load().lf_last_error())
        assert b"gave up" in L.load().lf_last_error()
        assert dt >= limit_ms / 1000.0 * 0.9
        assert dt < limit_ms / 1000.0 + 5.0
    # a limit out of range is rejected on the host, nothing launched
    assert api.lf_selftest_bounded_wait(0, s) == L.LF_ERR_INVALID_ARG
    # the context still renders correctly afterwards
    w = S.workload_tiny()
    r = api.LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, "f32")
    v = r.render(api.DeviceGaussians.from_scene(w.scene)).cpu().numpy().astype(np.float64)
    assert r.composite_status() == L.LF_OK
    o = orc.render(w)
    assert np.abs(v - o["views"]).max() <= 1e-4
