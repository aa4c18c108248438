"""FP64 CPU oracle for the G2LF / V2LF hot path (ctypes binding of liborc.so).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm may import this package. It shares no code with
the CUDA library (paper_2508_18540_gb300); both consume the seeded inputs of
paper_2508_18540_gb300.synth, which holds no arithmetic of the method.

Every function follows a passage of arXiv 2508.18540 (cited in the C
sources). Parity is pinned by tests/test_oracle_*.py against closed forms,
invariants and brute-force renderings.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class OrcCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("theta_x", ctypes.c_double), ("theta_y", ctypes.c_double),
                ("Nx", ctypes.c_int32), ("Ny", ctypes.c_int32)]


class OrcDisplay(ctypes.Structure):
    _fields_ = [("D_focal", ctypes.c_double), ("phi_x", ctypes.c_double), ("phi_y", ctypes.c_double),
                ("D_shift", ctypes.c_double), ("P_s", ctypes.c_int32), ("f_aa", ctypes.c_double),
                ("z_near", ctypes.c_double)]


class OrcRef(ctypes.Structure):
    _fields_ = [("cam", OrcCamera), ("disp", OrcDisplay),
                ("tth_x", ctypes.c_double), ("tth_y", ctypes.c_double),
                ("tphi_x", ctypes.c_double), ("tphi_y", ctypes.c_double),
                ("D_forward0", ctypes.c_double), ("D_forward", ctypes.c_double),
                ("tthp_x", ctypes.c_double), ("tthp_y", ctypes.c_double),
                ("theta_px", ctypes.c_double), ("theta_py", ctypes.c_double),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("f_prime", ctypes.c_double), ("W", ctypes.c_int32), ("H", ctypes.c_int32)]


_P = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_make_ref.argtypes = [ctypes.POINTER(OrcCamera), ctypes.POINTER(OrcDisplay), ctypes.POINTER(OrcRef)]
        L.orc_make_ref.restype = ctypes.c_int
        L.orc_view_offsets.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int32, ctypes.c_int32, _P, _P]
        L.orc_plane_coord.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]
        L.orc_plane_coord.restype = ctypes.c_double
        L.orc_plane_pixel.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int32]
        L.orc_plane_pixel.restype = ctypes.c_double
        L.orc_axis_coeffs.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      _P, _P, _P]
        L.orc_nearest_index.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_float, ctypes.c_float, ctypes.c_int32]
        L.orc_nearest_index.restype = ctypes.c_int32
        L.orc_gauss_decide.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, _P, _P, _P]
        L.orc_gauss_values.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, _P, _P, _P]
        L.orc_voxel_decide.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, ctypes.c_double,
                                       _P, _P, _P]
        L.orc_bin.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_int32,
                              _P, _P, _P, _P]
        L.orc_bin.restype = ctypes.c_int64
        L.orc_splat_gaussians.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P,
                                          ctypes.c_int32, _P]
        L.orc_splat_gaussians_3dgs.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, _P, _P, _P,
                                               _P, ctypes.c_int32, _P, _P]
        L.orc_splat_voxels.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int64, _P, _P, _P, _P, _P, _P,
                                       ctypes.c_double, _P, _P, ctypes.c_int32, _P]
        L.orc_voxel_alpha.argtypes = [_P, ctypes.c_double, _P, _P, _P, _P]
        L.orc_voxel_alpha.restype = ctypes.c_double
        L.orc_filter_weights.argtypes = [ctypes.c_double, ctypes.c_int32, _P]
        L.orc_filter_planes.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_int32]
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_composite.argtypes = [ctypes.POINTER(OrcRef), ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, _P, _P]
        _lib = L
    return _lib


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Sets the threads of the oracle's OpenMP loops (n <= 0: one per processor)."""
    lib().orc_set_num_threads(int(n))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# Geometry (Sec. 4.2, 4.3)
# ---------------------------------------------------------------------------

def make_ref(camera, display) -> OrcRef:
    cam = OrcCamera()
    cam.R[:] = [float(v) for v in np.asarray(camera.R, np.float64).reshape(9)]
    cam.t[:] = [float(v) for v in np.asarray(camera.t, np.float64).reshape(3)]
    cam.theta_x, cam.theta_y = float(camera.theta_x), float(camera.theta_y)
    cam.Nx, cam.Ny = int(camera.Nx), int(camera.Ny)
    disp = OrcDisplay(float(display.D_focal), float(display.phi_x), float(display.phi_y), float(display.D_shift),
                      int(display.P_s), float(display.f_aa), float(display.z_near))
    ref = OrcRef()
    rc = lib().orc_make_ref(ctypes.byref(cam), ctypes.byref(disp), ctypes.byref(ref))
    if rc != 0:
        raise ValueError("oracle: invalid camera/display")
    return ref


def view_offsets(ref: OrcRef, Vx: int, Vy: int):
    dx = np.zeros(max(Vx, 1), np.float64)
    dy = np.zeros(max(Vy, 1), np.float64)
    lib().orc_view_offsets(ctypes.byref(ref), Vx, Vy, _ptr(dx), _ptr(dy))
    return dx[:Vx], dy[:Vy]


def plane_coord(ref: OrcRef, axis: int, delta: float, d_k: float, u: float) -> float:
    return lib().orc_plane_coord(ctypes.byref(ref), axis, delta, d_k, u)


def plane_pixel(ref: OrcRef, axis: int, delta: float, d_k: float, x: int) -> float:
    return lib().orc_plane_pixel(ctypes.byref(ref), axis, delta, d_k, x)


def axis_coeffs(ref: OrcRef, axis: int, delta: float, d_k: float):
    out = np.zeros(3, np.float32)
    p = out.ctypes.data
    lib().orc_axis_coeffs(ctypes.byref(ref), axis, delta, d_k, ctypes.c_void_p(p), ctypes.c_void_p(p + 4),
                          ctypes.c_void_p(p + 8))
    return out  # gm, hn, hb


def nearest_index(ref: OrcRef, gm: float, hn: float, x: int) -> int:
    return lib().orc_nearest_index(ctypes.byref(ref), gm, hn, x)


# ---------------------------------------------------------------------------
# Primitives (Sec. 4.4, 4.5)
# ---------------------------------------------------------------------------

def gauss_decide(ref: OrcRef, scene):
    n = scene.n
    means, scales, quats = (_c(a, np.float32) for a in (scene.means, scene.scales, scene.quats))
    z = np.zeros(n, np.float64)
    valid = np.zeros(n, np.uint8)
    rect = np.zeros((n, 4), np.int32)
    lib().orc_gauss_decide(ctypes.byref(ref), n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(z), _ptr(valid),
                           _ptr(rect))
    return z, valid, rect


def gauss_values(ref: OrcRef, scene):
    n = scene.n
    means, scales, quats = (_c(a, np.float64) for a in (scene.means, scene.scales, scene.quats))
    mean2d = np.zeros((n, 2), np.float64)
    conic = np.zeros((n, 3), np.float64)
    cov2d = np.zeros((n, 3), np.float64)
    lib().orc_gauss_values(ctypes.byref(ref), n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(mean2d),
                           _ptr(conic), _ptr(cov2d))
    return mean2d, conic, cov2d


def voxel_decide(ref: OrcRef, scene):
    n = scene.n
    ijk = _c(scene.ijk, np.int32)
    lvl = _c(scene.level, np.uint8)
    origin = _c(scene.origin, np.float64)
    z = np.zeros(n, np.float64)
    valid = np.zeros(n, np.uint8)
    rect = np.zeros((n, 4), np.int32)
    lib().orc_voxel_decide(ctypes.byref(ref), n, _ptr(ijk), _ptr(lvl), _ptr(origin), float(scene.base_size),
                           _ptr(z), _ptr(valid), _ptr(rect))
    return z, valid, rect


def bin_primitives(ref: OrcRef, z: np.ndarray, valid: np.ndarray, N: int, mode: str):
    n = z.shape[0]
    z = _c(z, np.float64)
    valid = _c(valid, np.uint8)
    order = np.zeros(max(n, 1), np.int64)
    chunk = np.zeros(max(n, 1), np.int32)
    d = np.zeros(N, np.float64)
    count = np.zeros(N, np.int64)
    M = lib().orc_bin(ctypes.byref(ref), n, _ptr(z), _ptr(valid), N, 0 if mode == "quantile" else 1,
                      _ptr(order), _ptr(chunk), _ptr(d), _ptr(count))
    return order[:M].copy(), chunk[:n].copy(), d, count, int(M)


def splat_gaussians(ref: OrcRef, order, chunk, rect, mean2d, conic, opacity, rgb, N: int) -> np.ndarray:
    order = _c(order, np.int64)
    planes = np.zeros((N, ref.H, ref.W, 4), np.float64)
    args = [_c(chunk, np.int32), _c(rect, np.int32), _c(mean2d, np.float64), _c(conic, np.float64),
            _c(opacity, np.float64), _c(rgb, np.float64)]
    lib().orc_splat_gaussians(ctypes.byref(ref), order.shape[0], _ptr(order), *[_ptr(a) for a in args], N,
                              _ptr(planes))
    return planes


def splat_gaussians_3dgs(ref: OrcRef, order, chunk, rect, mean2d, conic, opacity, rgb, N: int):
    """The splat with the 3DGS cut-offs (alpha < 1/255 skipped, stop before
    T < 1e-4); returns (planes, near), near[N][H][W] marking texels whose
    trace comes within 1e-6 of either threshold."""
    order = _c(order, np.int64)
    planes = np.zeros((N, ref.H, ref.W, 4), np.float64)
    near = np.zeros((N, ref.H, ref.W), np.uint8)
    args = [_c(chunk, np.int32), _c(rect, np.int32), _c(mean2d, np.float64), _c(conic, np.float64),
            _c(opacity, np.float64), _c(rgb, np.float64)]
    lib().orc_splat_gaussians_3dgs(ctypes.byref(ref), order.shape[0], _ptr(order), *[_ptr(a) for a in args], N,
                                   _ptr(planes), _ptr(near))
    return planes, near


def splat_voxels(ref: OrcRef, order, chunk, rect, scene, N: int) -> np.ndarray:
    order = _c(order, np.int64)
    planes = np.zeros((N, ref.H, ref.W, 4), np.float64)
    arrs = [_c(chunk, np.int32), _c(rect, np.int32), _c(scene.ijk, np.int32), _c(scene.level, np.uint8),
            _c(scene.origin, np.float64)]
    dens = _c(scene.density8, np.float64)
    rgb = _c(scene.rgb, np.float64)
    lib().orc_splat_voxels(ctypes.byref(ref), order.shape[0], _ptr(order), *[_ptr(a) for a in arrs],
                           float(scene.base_size), _ptr(dens), _ptr(rgb), N, _ptr(planes))
    return planes


def voxel_alpha(lo, side: float, density8, origin, direction):
    lo = _c(lo, np.float64)
    dens = _c(density8, np.float64)
    o = _c(origin, np.float64)
    d = _c(direction, np.float64)
    seg = ctypes.c_double(0.0)
    a = lib().orc_voxel_alpha(_ptr(lo), float(side), _ptr(dens), _ptr(o), _ptr(d), ctypes.byref(seg))
    return a, seg.value


def composite(ref: OrcRef, planes: np.ndarray, d, count, Vx: int, Vy: int, bilinear: bool,
              bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    N = planes.shape[0]
    planes = _c(planes, np.float64)
    d = _c(d, np.float64)
    count = _c(count, np.int64)
    bgv = _c(bg, np.float64)
    views = np.zeros((Vx * Vy, ref.cam.Ny, ref.cam.Nx, 4), np.float64)
    lib().orc_composite(ctypes.byref(ref), N, _ptr(planes), _ptr(d), _ptr(count), Vx, Vy, int(bool(bilinear)),
                        _ptr(bgv), _ptr(views))
    return views


def filter_weights(sigma: float, radius: int) -> np.ndarray:
    w = np.zeros(2 * radius + 1, np.float64)
    lib().orc_filter_weights(float(sigma), int(radius), _ptr(w))
    return w


def filter_planes(planes: np.ndarray, sigma: float, radius: int) -> np.ndarray:
    """Sec. 4.5 low-pass plane filter (separable Gaussian, zero padding); returns a filtered copy."""
    out = _c(planes, np.float64).copy()
    N, H, W, _ = out.shape
    lib().orc_filter_planes(_ptr(out), N, H, W, float(sigma), int(radius))
    return out


# ---------------------------------------------------------------------------
# Whole pipeline (Algorithm 1)
# ---------------------------------------------------------------------------

def render(workload=None, *, scene=None, camera=None, display=None, views=None, N=None, binning=None,
           kind: Optional[str] = None, with_views: bool = True, blend: str = "exact") -> dict:
    """Algorithm 1 end to end on the CPU: projection and culling, depth sort
    and chunking, per-chunk splatting, then swizzle blending. blend="3dgs"
    splats Gaussians with the 3DGS cut-offs and adds the near-threshold
    texel mask as out["near"]."""
    if blend not in ("exact", "3dgs"):
        raise ValueError("blend must be 'exact' or '3dgs'")
    if workload is not None:
        scene, camera, display = workload.scene, workload.camera, workload.display
        views, N, binning = workload.views, workload.N, workload.binning
    if kind is None:
        kind = "voxels" if hasattr(scene, "ijk") else "gaussians"
    ref = make_ref(camera, display)
    if kind == "gaussians":
        z, valid, rect = gauss_decide(ref, scene)
    else:
        z, valid, rect = voxel_decide(ref, scene)
    order, chunk, d, count, M = bin_primitives(ref, z, valid, N, binning)
    out = dict(ref=ref, z=z, valid=valid, rect=rect, order=order, chunk=chunk, d=d, count=count, M=M)
    if kind == "gaussians":
        mean2d, conic, cov2d = gauss_values(ref, scene)
        if blend == "3dgs":
            planes, out["near"] = splat_gaussians_3dgs(ref, order, chunk, rect, mean2d, conic, scene.opacity,
                                                       scene.rgb, N)
        else:
            planes = splat_gaussians(ref, order, chunk, rect, mean2d, conic, scene.opacity, scene.rgb, N)
        out.update(mean2d=mean2d, conic=conic, cov2d=cov2d)
    else:
        if blend != "exact":
            raise ValueError("3DGS blending applies to Gaussians only")
        planes = splat_voxels(ref, order, chunk, rect, scene, N)
    out["planes"] = planes
    if with_views:
        out["views"] = composite(ref, planes, d, count, views.Vx, views.Vy, views.bilinear, views.bg)
    return out
