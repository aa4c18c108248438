"""The C-ABI library loads, exports every symbol include/lf.h declares, and
its host-side set-up and argument checks behave (no GPU work here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2508_18540_gb300 import build as B
from paper_2508_18540_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2508_18540_gb300 import _lib
    return _lib


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    lib = L.load()
    names = _declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the binding wraps every declared entry point under the same name
    assert {s[0] for s in L.SIGNATURES} == names


def test_ref_camera_matches_oracle_bitwise(L, orc):
    from paper_2508_18540_gb300 import api
    cams = [S.identity_camera(128), S.identity_camera(512, 50.0, t=(0.1, 0.2, 6.0))]
    a = 0.3
    c3 = S.identity_camera(96, 40.0, t=(0.2, -0.1, 0.5))
    c3.R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    cams.append(c3)
    disps = [S.display_for(3.0, 0.1), S.display_for(2.6087, 0.15, P_s=2, D_shift=0.05),
             S.Display(D_focal=4.0, phi_x=0.3, phi_y=0.1, P_s=3, f_aa=0.25, z_near=0.3)]
    fields = ["tth_x", "tth_y", "tphi_x", "tphi_y", "D_forward0", "D_forward", "tthp_x", "tthp_y", "theta_px",
              "theta_py", "fx", "fy", "cx", "cy", "f_prime", "W", "H"]
    for cam in cams:
        for disp in disps:
            r1 = api.lf_make_ref_camera(cam, disp)
            r2 = orc.make_ref(cam, disp)
            for f in fields:
                assert getattr(r1, f) == getattr(r2, f), f


def test_invalid_arguments_are_rejected(L):
    from paper_2508_18540_gb300 import api
    with pytest.raises(L.LFError) as e:
        api.lf_make_ref_camera(S.identity_camera(0), S.display_for(3.0, 0.1))
    assert e.value.status == L.LF_ERR_INVALID_ARG
    with pytest.raises(L.LFError):
        api.lf_make_ref_camera(S.identity_camera(64), S.display_for(3.0, 0.1, D_shift=-10.0))
    lib = L.load()
    ref = api.lf_make_ref_camera(S.identity_camera(64), S.display_for(3.0, 0.1))
    # NULL inputs fail on the host before any CUDA call
    st = lib.lf_build_mpi_gaussians(None, ctypes.byref(ref), 4, 0, None, 0, None, None)
    assert st == L.LF_ERR_INVALID_ARG and b"NULL" in lib.lf_last_error()
    g = L.LfGaussians(10, 0, 0, 0, 0, 0)
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 0, None, 0, None, None)
    assert st == L.LF_ERR_INVALID_ARG
    planes = L.LfPlanes(4, ref.H, ref.W, 0, 1, 1, 1, 1, 1)
    g = L.LfGaussians(10, 16, 16, 16, 16, 16)
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 7, ctypes.c_void_p(256), 1 << 20,
                                    ctypes.byref(planes), None)
    assert st == L.LF_ERR_INVALID_ARG                      # unknown binning
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 0x200, ctypes.c_void_p(256), 1 << 20,
                                    ctypes.byref(planes), None)
    assert st == L.LF_ERR_INVALID_ARG                      # unknown flag bit
    vox = L.LfVoxels(10, 16, 16, (ctypes.c_double * 3)(0.0, 0.0, 0.0), 1.0, 16, 16)
    st = lib.lf_build_mpi_voxels(ctypes.byref(vox), ctypes.byref(ref), 4, L.LF_BLEND_3DGS, ctypes.c_void_p(256),
                                 1 << 20, ctypes.byref(planes), None)
    assert st == L.LF_ERR_UNSUPPORTED                      # 3DGS blending is for Gaussians
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 0, None, 0, ctypes.byref(planes), None)
    assert st == L.LF_ERR_WORKSPACE
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 0, ctypes.c_void_p(256), 100,
                                    ctypes.byref(planes), None)
    assert st == L.LF_ERR_WORKSPACE                        # too small
    bad = L.LfPlanes(4, ref.H + 1, ref.W, 0, 1, 1, 1, 1, 1)
    st = lib.lf_build_mpi_gaussians(ctypes.byref(g), ctypes.byref(ref), 4, 0, ctypes.c_void_p(256), 1 << 30,
                                    ctypes.byref(bad), None)
    assert st == L.LF_ERR_INVALID_ARG
    vs = L.LfViewSet(0, 1, 0)
    st = lib.lf_composite(ctypes.byref(planes), ctypes.byref(ref), ctypes.byref(vs), ctypes.c_void_p(16),
                          ctypes.c_void_p(256), 1 << 20, None)
    assert st == L.LF_ERR_INVALID_ARG
    # status and self-test entry points reject bad arguments on the host
    vs = L.LfViewSet(5, 1, 0)
    assert lib.lf_composite_status(0, ctypes.byref(vs), ctypes.c_void_p(256), None) == L.LF_ERR_INVALID_ARG
    assert lib.lf_composite_status(4, ctypes.byref(vs), None, None) == L.LF_ERR_INVALID_ARG
    assert lib.lf_composite_noalloc_status(0, ctypes.byref(vs), None) == L.LF_ERR_INVALID_ARG
    assert lib.lf_composite_noalloc_status(1 << 20, ctypes.byref(vs), None) == L.LF_ERR_INVALID_ARG
    assert lib.lf_selftest_bounded_wait(0, None) == L.LF_ERR_INVALID_ARG
    assert lib.lf_selftest_bounded_wait(20000, None) == L.LF_ERR_INVALID_ARG
    # the saving composite and its adjoint check the state buffer on the host
    sb = lib.lf_composite_state_size(ctypes.byref(ref), ctypes.byref(vs))
    assert sb == 16 * 5 * ref.base.Nx * ref.base.Ny
    assert lib.lf_composite_state_size(None, ctypes.byref(vs)) == 0
    pl16 = L.LfPlanes(4, ref.H, ref.W, 0, 256, 1, 1, 1, 1)   # FP32 texels: rgba 16-byte aligned
    for state, nbytes, what in ((None, sb, b"NULL"), (8, sb, b"aligned"), (16, sb - 16, b"smaller")):
        st = lib.lf_composite_save(ctypes.byref(pl16), ctypes.byref(ref), ctypes.byref(vs), ctypes.c_void_p(16),
                                   ctypes.c_void_p(state), nbytes, ctypes.c_void_p(256), 1 << 20, None)
        assert st == L.LF_ERR_INVALID_ARG and what in lib.lf_last_error(), what
        st = lib.lf_composite_backward_saved(ctypes.byref(pl16), ctypes.byref(ref), ctypes.byref(vs),
                                             ctypes.c_void_p(16), ctypes.c_void_p(state), nbytes,
                                             ctypes.c_void_p(16), ctypes.c_void_p(256), 1 << 20, None)
        assert st == L.LF_ERR_INVALID_ARG and what in lib.lf_last_error(), what
    # texels are read whole: an FP32 plane array off a 16-byte boundary is refused
    st = lib.lf_composite(ctypes.byref(planes), ctypes.byref(ref), ctypes.byref(vs), ctypes.c_void_p(16),
                          ctypes.c_void_p(256), 1 << 20, None)
    assert st == L.LF_ERR_INVALID_ARG and b"texel-aligned" in lib.lf_last_error()


def test_workspace_sizes(L):
    from paper_2508_18540_gb300 import api
    ref = api.lf_make_ref_camera(S.identity_camera(512), S.display_for(2.6, 0.15))
    a = api.lf_build_mpi_workspace_size(ref, 1_000_000, 64, 0)
    b = api.lf_build_mpi_workspace_size(ref, 1_000_000, 64, 20_000_000)
    assert 0 < a < b
    assert api.lf_composite_workspace_size(64, S.ViewSet(45)) > 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # there is no CPU fallback: without liblf.so the binding raises
    from paper_2508_18540_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="liblf.so not found"):
        _lib.load(str(tmp_path / "liblf.so"))


def test_host_pipeline_rejects_no_slots():
    # the frame count in flight is checked before any device work
    from paper_2508_18540_gb300 import api
    with pytest.raises(ValueError, match="depth"):
        api.HostPipeline(None, 1, depth=0)
