"""ctypes mirror of include/lf.h and the loader of liblf.so.

Argument marshalling only: every step of the G2LF / V2LF path runs in the
library's CUDA kernels. There is no CPU fallback: if liblf.so is missing the
loader raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblf.so")

LF_OK = 0
LF_ERR_INVALID_ARG = 1
LF_ERR_WORKSPACE = 2
LF_ERR_CUDA = 3
LF_ERR_OVERFLOW = 4
LF_ERR_UNSUPPORTED = 5
LF_ERR_TIMEOUT = 6
STATUS_NAMES = {0: "LF_OK", 1: "LF_ERR_INVALID_ARG", 2: "LF_ERR_WORKSPACE", 3: "LF_ERR_CUDA",
                4: "LF_ERR_OVERFLOW", 5: "LF_ERR_UNSUPPORTED", 6: "LF_ERR_TIMEOUT"}

LF_F32, LF_F16, LF_BF16, LF_U8 = 0, 1, 2, 3
LF_BIN_QUANTILE, LF_BIN_DISPARITY = 0, 1
LF_BLEND_3DGS = 0x100          # OR into the binning argument: 3DGS alpha / transmittance cut-offs

_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


class LfCamera(ctypes.Structure):
    _fields_ = [("R", _D * 9), ("t", _D * 3), ("theta_x", _D), ("theta_y", _D), ("Nx", _I32), ("Ny", _I32)]


class LfDisplay(ctypes.Structure):
    _fields_ = [("D_focal", _D), ("phi_x", _D), ("phi_y", _D), ("D_shift", _D), ("P_s", _I32), ("f_aa", _D),
                ("z_near", _D)]


class LfRefCamera(ctypes.Structure):
    _fields_ = [("base", LfCamera), ("disp", LfDisplay),
                ("tth_x", _D), ("tth_y", _D), ("tphi_x", _D), ("tphi_y", _D),
                ("D_forward0", _D), ("D_forward", _D),
                ("tthp_x", _D), ("tthp_y", _D), ("theta_px", _D), ("theta_py", _D),
                ("fx", _D), ("fy", _D), ("cx", _D), ("cy", _D), ("f_prime", _D), ("W", _I32), ("H", _I32)]


class LfGaussians(ctypes.Structure):
    _fields_ = [("n", _I64), ("means", _P), ("scales", _P), ("quats", _P), ("opacity", _P), ("rgb", _P)]


class LfVoxels(ctypes.Structure):
    _fields_ = [("n", _I64), ("ijk", _P), ("level", _P), ("origin", _D * 3), ("base_size", _D),
                ("density8", _P), ("rgb", _P)]


class LfGaussiansGrad(ctypes.Structure):
    _fields_ = [("dmeans", _P), ("dscales", _P), ("dquats", _P), ("dopacity", _P), ("drgb", _P)]


class LfVoxelsGrad(ctypes.Structure):
    _fields_ = [("ddensity8", _P), ("drgb", _P)]


class LfPlanes(ctypes.Structure):
    _fields_ = [("N", _I32), ("H", _I32), ("W", _I32), ("dtype", _I32), ("rgba", _P), ("d", _P), ("count", _P),
                ("chunk", _P), ("rect", _P)]


class LfViewSet(ctypes.Structure):
    _fields_ = [("Vx", _I32), ("Vy", _I32), ("bilinear", _I32), ("bg", ctypes.c_float * 3), ("atlas_cols", _I32)]


class LfBatchScene(ctypes.Structure):
    _fields_ = [("g", LfGaussians), ("ref", LfRefCamera), ("N", _I32), ("binning", _I32), ("planes", LfPlanes),
                ("views", LfViewSet), ("out", _P), ("ws", _P), ("ws_bytes", ctypes.c_size_t), ("cws", _P),
                ("cws_bytes", ctypes.c_size_t)]


class LfBatchPlan(ctypes.Structure):
    _fields_ = [("views_per_thread", _I32), ("tile_x", _I32), ("chunk_groups", _I32), ("schedule", _I32)]


# (name, restype, argtypes) of every exported symbol declared in include/lf.h
SIGNATURES = [
    ("lf_make_ref_camera", ctypes.c_int, [ctypes.POINTER(LfCamera), ctypes.POINTER(LfDisplay),
                                          ctypes.POINTER(LfRefCamera)]),
    ("lf_build_mpi_workspace_size", ctypes.c_size_t, [ctypes.POINTER(LfRefCamera), _I64, _I32, _I64]),
    ("lf_build_mpi_gaussians", ctypes.c_int, [ctypes.POINTER(LfGaussians), ctypes.POINTER(LfRefCamera), _I32, _I32,
                                              _P, ctypes.c_size_t, ctypes.POINTER(LfPlanes), _P]),
    ("lf_build_mpi_voxels", ctypes.c_int, [ctypes.POINTER(LfVoxels), ctypes.POINTER(LfRefCamera), _I32, _I32,
                                           _P, ctypes.c_size_t, ctypes.POINTER(LfPlanes), _P]),
    ("lf_mpi_status", ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    ("lf_mpi_tile_lists", ctypes.c_int, [_P, _P, _I64, _P, _I64, _P, ctypes.POINTER(_I64)]),
    ("lf_filter_planes", ctypes.c_int, [ctypes.POINTER(LfPlanes), _D, _I32, _P]),
    ("lf_composite_workspace_size", ctypes.c_size_t, [_I32, ctypes.POINTER(LfViewSet)]),
    ("lf_composite", ctypes.c_int, [ctypes.POINTER(LfPlanes), ctypes.POINTER(LfRefCamera),
                                    ctypes.POINTER(LfViewSet), _P, _P, ctypes.c_size_t, _P]),
    ("lf_composite_noalloc", ctypes.c_int, [ctypes.POINTER(LfPlanes), ctypes.POINTER(LfRefCamera),
                                            ctypes.POINTER(LfViewSet), _P, _P]),
    ("lf_composite_noalloc_max_bytes", ctypes.c_size_t, []),
    ("lf_composite_noalloc_status", ctypes.c_int, [_I32, ctypes.POINTER(LfViewSet), _P]),
    ("lf_composite_backward", ctypes.c_int, [ctypes.POINTER(LfPlanes), ctypes.POINTER(LfRefCamera),
                                             ctypes.POINTER(LfViewSet), _P, _P, _P, ctypes.c_size_t, _P]),
    ("lf_composite_state_size", ctypes.c_size_t, [ctypes.POINTER(LfRefCamera), ctypes.POINTER(LfViewSet)]),
    ("lf_composite_save", ctypes.c_int, [ctypes.POINTER(LfPlanes), ctypes.POINTER(LfRefCamera),
                                         ctypes.POINTER(LfViewSet), _P, _P, ctypes.c_size_t, _P, ctypes.c_size_t,
                                         _P]),
    ("lf_composite_backward_saved", ctypes.c_int, [ctypes.POINTER(LfPlanes), ctypes.POINTER(LfRefCamera),
                                                   ctypes.POINTER(LfViewSet), _P, _P, ctypes.c_size_t, _P, _P,
                                                   ctypes.c_size_t, _P]),
    ("lf_build_mpi_backward_gaussians", ctypes.c_int, [ctypes.POINTER(LfGaussians), ctypes.POINTER(LfRefCamera),
                                                       ctypes.POINTER(LfPlanes), _P, ctypes.POINTER(LfGaussiansGrad),
                                                       _P, ctypes.c_size_t, _P]),
    ("lf_build_mpi_backward_voxels", ctypes.c_int, [ctypes.POINTER(LfVoxels), ctypes.POINTER(LfRefCamera),
                                                    ctypes.POINTER(LfPlanes), _P, ctypes.POINTER(LfVoxelsGrad),
                                                    _P, ctypes.c_size_t, _P]),
    ("lf_batch_create", ctypes.c_int, [ctypes.POINTER(LfBatchScene), _I32, ctypes.POINTER(_P)]),
    ("lf_batch_workspace_size", ctypes.c_size_t, [_P]),
    ("lf_batch_plan_workspace_size", ctypes.c_size_t, [_P, ctypes.POINTER(LfBatchPlan)]),
    ("lf_batch_prepare", ctypes.c_int, [_P, ctypes.POINTER(LfBatchPlan), _P, ctypes.c_size_t, _P]),
    ("lf_batch_render", ctypes.c_int, [_P, _P]),
    ("lf_batch_capture", ctypes.c_int, [_P, _P]),
    ("lf_batch_launch", ctypes.c_int, [_P, _P]),
    ("lf_batch_autotune", ctypes.c_int, [_P, _P, ctypes.c_size_t, _I32, _P, ctypes.POINTER(LfBatchPlan),
                                         ctypes.POINTER(ctypes.c_float)]),
    ("lf_batch_status", ctypes.c_int, [_P, _P]),
    ("lf_batch_destroy", ctypes.c_int, [_P]),
    ("lf_selftest_bounded_wait", ctypes.c_int, [_I32, _P]),
    ("lf_composite_status", ctypes.c_int, [_I32, ctypes.POINTER(LfViewSet), _P, _P]),
    ("lf_launch_count", _I64, []),
    ("lf_trace_enable", ctypes.c_int, [_I32]),
    ("lf_trace_collect", _I32, [_P, _P, _P, _I32]),
    ("lf_last_error", ctypes.c_char_p, []),
    ("lf_version", ctypes.c_char_p, []),
]

_lib = None


class LFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load liblf.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblf.so not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != LF_OK:
        raise LFError(status, load().lf_last_error().decode())
