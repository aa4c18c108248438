"""Thin PyTorch-facing binding of liblf (same names as the C ABI in include/lf.h).

PyTorch supplies device memory and streams; every computation of the path
runs in liblf's kernels. Tensors are passed by data pointer; shapes, dtypes,
devices and contiguity are checked here before the call.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from ._lib import check, load

DTYPES = {"f32": L.LF_F32, "f16": L.LF_F16, "bf16": L.LF_BF16, "u8": L.LF_U8}
TORCH_DTYPES = {L.LF_F32: torch.float32, L.LF_F16: torch.float16, L.LF_BF16: torch.bfloat16, L.LF_U8: torch.uint8}
BINNING = {"quantile": L.LF_BIN_QUANTILE, "disparity": L.LF_BIN_DISPARITY}
BLEND = {"exact": 0, "3dgs": L.LF_BLEND_3DGS}


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, shape, dtype, name):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


# ---------------------------------------------------------------------------
# set-up
# ---------------------------------------------------------------------------

def lf_make_ref_camera(camera, display) -> L.LfRefCamera:
    """Sec. 4.2: reference camera (Eqs. (1)-(2), D_shift, Eq. (gs_prefilter_fix))."""
    lib = load()
    cam = L.LfCamera()
    cam.R[:] = [float(v) for v in np.asarray(camera.R, np.float64).reshape(9)]
    cam.t[:] = [float(v) for v in np.asarray(camera.t, np.float64).reshape(3)]
    cam.theta_x, cam.theta_y = float(camera.theta_x), float(camera.theta_y)
    cam.Nx, cam.Ny = int(camera.Nx), int(camera.Ny)
    disp = L.LfDisplay(float(display.D_focal), float(display.phi_x), float(display.phi_y), float(display.D_shift),
                       int(display.P_s), float(display.f_aa), float(display.z_near))
    ref = L.LfRefCamera()
    check(lib.lf_make_ref_camera(ctypes.byref(cam), ctypes.byref(disp), ctypes.byref(ref)))
    return ref


# ---------------------------------------------------------------------------
# device-resident inputs and outputs
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class DeviceGaussians:
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacity: torch.Tensor
    rgb: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @classmethod
    def from_scene(cls, scene, device="cuda", pin: bool = False):
        def put(a):
            t = torch.from_numpy(np.ascontiguousarray(a, np.float32))
            return t.pin_memory() if pin else t.to(device)
        return cls(put(scene.means), put(scene.scales), put(scene.quats), put(scene.opacity), put(scene.rgb))

    def c_struct(self) -> L.LfGaussians:
        n = self.n
        for name, t, w in (("means", self.means, 3), ("scales", self.scales, 3), ("quats", self.quats, 4),
                           ("rgb", self.rgb, 3)):
            _need(t, (n, w), torch.float32, name)
        _need(self.opacity, (n,), torch.float32, "opacity")
        return L.LfGaussians(n, self.means.data_ptr(), self.scales.data_ptr(), self.quats.data_ptr(),
                             self.opacity.data_ptr(), self.rgb.data_ptr())


@dataclasses.dataclass
class DeviceVoxels:
    ijk: torch.Tensor
    level: torch.Tensor
    density8: torch.Tensor
    rgb: torch.Tensor
    origin: tuple
    base_size: float

    @property
    def n(self) -> int:
        return int(self.ijk.shape[0])

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        return cls(torch.from_numpy(np.ascontiguousarray(scene.ijk, np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(scene.level, np.uint8)).to(device),
                   torch.from_numpy(np.ascontiguousarray(scene.density8, np.float32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(scene.rgb, np.float32)).to(device),
                   tuple(float(v) for v in scene.origin), float(scene.base_size))

    def c_struct(self) -> L.LfVoxels:
        n = self.n
        _need(self.ijk, (n, 3), torch.int32, "ijk")
        _need(self.level, (n,), torch.uint8, "level")
        _need(self.density8, (n, 8), torch.float32, "density8")
        _need(self.rgb, (n, 3), torch.float32, "rgb")
        v = L.LfVoxels()
        v.n = n
        v.ijk, v.level = self.ijk.data_ptr(), self.level.data_ptr()
        v.origin[:] = list(self.origin)
        v.base_size = self.base_size
        v.density8, v.rgb = self.density8.data_ptr(), self.rgb.data_ptr()
        return v


@dataclasses.dataclass
class Planes:
    """Sweeping planes and the per-primitive build outputs (device)."""
    rgba: torch.Tensor       # [N][H][W][4] dtype
    d: torch.Tensor          # [N] float64
    count: torch.Tensor      # [N] int32
    chunk: torch.Tensor      # [n] int32
    rect: torch.Tensor       # [n][4] int32
    dtype_code: int

    @classmethod
    def empty(cls, ref: L.LfRefCamera, N: int, n: int, dtype: str = "f32", device="cuda"):
        code = DTYPES[dtype]
        return cls(torch.empty((N, ref.H, ref.W, 4), dtype=TORCH_DTYPES[code], device=device),
                   torch.empty(N, dtype=torch.float64, device=device),
                   torch.empty(N, dtype=torch.int32, device=device),
                   torch.empty(max(n, 1), dtype=torch.int32, device=device),
                   torch.empty((max(n, 1), 4), dtype=torch.int32, device=device), code)

    @property
    def N(self) -> int:
        return int(self.rgba.shape[0])

    def c_struct(self) -> L.LfPlanes:
        N, H, W = (int(v) for v in self.rgba.shape[:3])
        _need(self.rgba, (N, H, W, 4), TORCH_DTYPES[self.dtype_code], "planes.rgba")
        return L.LfPlanes(N, H, W, self.dtype_code, self.rgba.data_ptr(), self.d.data_ptr(),
                          self.count.data_ptr(), self.chunk.data_ptr(), self.rect.data_ptr())


def view_set(views) -> L.LfViewSet:
    vs = L.LfViewSet()
    vs.Vx, vs.Vy, vs.bilinear = int(views.Vx), int(views.Vy), int(bool(views.bilinear))
    vs.bg[:] = [float(c) for c in views.bg]
    vs.atlas_cols = int(getattr(views, "atlas_cols", 0) or 0)
    return vs


def views_shape(views, Nx: int, Ny: int):
    """Output shape: separate views [V][Ny][Nx][4], or the quilt atlas."""
    V = int(views.Vx) * int(views.Vy)
    c = int(getattr(views, "atlas_cols", 0) or 0)
    if c <= 0:
        return (V, Ny, Nx, 4)
    return ((V + c - 1) // c * Ny, c * Nx, 4)


def alloc_workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """Device workspace (caching-allocator blocks are 512-byte aligned)."""
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


# ---------------------------------------------------------------------------
# splat
# ---------------------------------------------------------------------------

def lf_build_mpi_workspace_size(ref: L.LfRefCamera, n: int, N: int, dup_capacity: int = 0) -> int:
    return int(load().lf_build_mpi_workspace_size(ctypes.byref(ref), int(n), int(N), int(dup_capacity)))


def lf_build_mpi_gaussians(g: DeviceGaussians, ref: L.LfRefCamera, N: int, binning: str, ws: torch.Tensor,
                           planes: Planes, stream=None, blend: str = "exact"):
    """Sec. 4.4 / the plane-building steps of Algorithm 1 for 3D Gaussians
    (asynchronous). blend="3dgs" adds the 3DGS rasteriser's cut-offs
    (alpha < 1/255 skipped, stop before T < 1e-4)."""
    gs = g.c_struct()
    ps = planes.c_struct()
    check(load().lf_build_mpi_gaussians(ctypes.byref(gs), ctypes.byref(ref), int(N),
                                        BINNING[binning] | BLEND[blend], _ptr(ws), ws.numel(), ctypes.byref(ps),
                                        _stream_ptr(stream)))


def lf_build_mpi_voxels(v: DeviceVoxels, ref: L.LfRefCamera, N: int, binning: str, ws: torch.Tensor,
                        planes: Planes, stream=None):
    """Sec. 4.5 / the plane-building steps of Algorithm 1 for sparse voxels (asynchronous)."""
    vs = v.c_struct()
    ps = planes.c_struct()
    check(load().lf_build_mpi_voxels(ctypes.byref(vs), ctypes.byref(ref), int(N), BINNING[binning],
                                     _ptr(ws), ws.numel(), ctypes.byref(ps), _stream_ptr(stream)))


def lf_mpi_status(ws: torch.Tensor):
    """(status, pairs needed, culled-in count) of the last build on ws (synchronising)."""
    needed = ctypes.c_int64(0)
    M = ctypes.c_int64(0)
    st = load().lf_mpi_status(_ptr(ws), ctypes.byref(needed), ctypes.byref(M))
    return st, needed.value, M.value


def lf_mpi_tile_lists(ws: torch.Tensor, n: int, n_tiles: int, N: int):
    """Depth order, 16x16 tile-list entries and (tile, chunk) segments (numpy)."""
    st, needed, M = lf_mpi_status(ws)
    check(st)
    total = ctypes.c_int64(0)
    check(load().lf_mpi_tile_lists(_ptr(ws), None, 0, None, 0, None, ctypes.byref(total)))
    order = np.zeros(max(n, 1), np.int32)
    prims = np.zeros(max(total.value, 1), np.int32)
    seg = np.zeros((n_tiles * N, 2), np.int32)
    check(load().lf_mpi_tile_lists(_ptr(ws), order.ctypes.data_as(ctypes.c_void_p), int(n),
                                   prims.ctypes.data_as(ctypes.c_void_p), int(prims.shape[0]),
                                   seg.ctypes.data_as(ctypes.c_void_p), ctypes.byref(total)))
    return order[:M], prims[:total.value], seg


def lf_filter_planes(planes: Planes, sigma: float, radius: int = 0, stream=None):
    """Sec. 4.5 low-pass plane filter (separable Gaussian, zero padding), in place."""
    ps = planes.c_struct()
    check(load().lf_filter_planes(ctypes.byref(ps), float(sigma), int(radius), _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# composite
# ---------------------------------------------------------------------------

def lf_composite_workspace_size(N: int, views) -> int:
    vs = view_set(views)
    return int(load().lf_composite_workspace_size(int(N), ctypes.byref(vs)))


def lf_composite(planes: Planes, ref: L.LfRefCamera, views, out: torch.Tensor, ws: torch.Tensor, stream=None):
    """Sec. 4.3 swizzle blending into out [Vy*Vx][Ny][Nx][4] float32 (asynchronous)."""
    vs = view_set(views)
    _need(out, views_shape(views, ref.base.Nx, ref.base.Ny), torch.float32, "views")
    ps = planes.c_struct()
    check(load().lf_composite(ctypes.byref(ps), ctypes.byref(ref), ctypes.byref(vs), _ptr(out), _ptr(ws),
                              ws.numel(), _stream_ptr(stream)))


def lf_composite_status(N: int, views, ws: torch.Tensor, stream=None) -> int:
    """Status of the last composite (or adjoint) on workspace ws:
    LF_ERR_TIMEOUT if a bounded device wait gave up, else LF_OK."""
    vs = view_set(views)
    return int(load().lf_composite_status(int(N), ctypes.byref(vs), _ptr(ws), _stream_ptr(stream)))


def lf_composite_noalloc(planes: Planes, ref: L.LfRefCamera, views, out: torch.Tensor, stream=None):
    """lf_composite with the library's static scratch instead of a workspace
    (calls must not overlap in time)."""
    vs = view_set(views)
    _need(out, views_shape(views, ref.base.Nx, ref.base.Ny), torch.float32, "views")
    ps = planes.c_struct()
    check(load().lf_composite_noalloc(ctypes.byref(ps), ctypes.byref(ref), ctypes.byref(vs), _ptr(out),
                                      _stream_ptr(stream)))


def lf_composite_noalloc_max_bytes() -> int:
    return int(load().lf_composite_noalloc_max_bytes())


def lf_composite_noalloc_status(N: int, views, stream=None) -> int:
    """Status of the last lf_composite_noalloc for N planes and these views:
    LF_ERR_TIMEOUT if a bounded device wait gave up, else LF_OK."""
    vs = view_set(views)
    return int(load().lf_composite_noalloc_status(int(N), ctypes.byref(vs), _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# differentiation
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class GaussianGrads:
    dmeans: torch.Tensor
    dscales: torch.Tensor
    dquats: torch.Tensor
    dopacity: torch.Tensor
    drgb: torch.Tensor

    @classmethod
    def empty(cls, n: int, device="cuda"):
        f = dict(dtype=torch.float32, device=device)
        return cls(torch.empty((n, 3), **f), torch.empty((n, 3), **f), torch.empty((n, 4), **f),
                   torch.empty((n,), **f), torch.empty((n, 3), **f))

    def c_struct(self, n: int) -> L.LfGaussiansGrad:
        for name, t, w in (("dmeans", self.dmeans, 3), ("dscales", self.dscales, 3), ("dquats", self.dquats, 4),
                           ("drgb", self.drgb, 3)):
            _need(t, (n, w), torch.float32, name)
        _need(self.dopacity, (n,), torch.float32, "dopacity")
        return L.LfGaussiansGrad(self.dmeans.data_ptr(), self.dscales.data_ptr(), self.dquats.data_ptr(),
                                 self.dopacity.data_ptr(), self.drgb.data_ptr())


@dataclasses.dataclass
class VoxelGrads:
    ddensity8: torch.Tensor
    drgb: torch.Tensor

    @classmethod
    def empty(cls, n: int, device="cuda"):
        return cls(torch.empty((n, 8), dtype=torch.float32, device=device),
                   torch.empty((n, 3), dtype=torch.float32, device=device))

    def c_struct(self, n: int) -> L.LfVoxelsGrad:
        _need(self.ddensity8, (n, 8), torch.float32, "ddensity8")
        _need(self.drgb, (n, 3), torch.float32, "drgb")
        return L.LfVoxelsGrad(self.ddensity8.data_ptr(), self.drgb.data_ptr())


def lf_composite_backward(planes: Planes, ref: L.LfRefCamera, views, dviews: torch.Tensor, dplanes: torch.Tensor,
                          ws: torch.Tensor, stream=None):
    """Adjoint of lf_composite: dplanes [N][H][W][4] float32 from dviews (asynchronous)."""
    vs = view_set(views)
    _need(dviews, (vs.Vx * vs.Vy, ref.base.Ny, ref.base.Nx, 4), torch.float32, "dviews")
    _need(dplanes, (planes.N, ref.H, ref.W, 4), torch.float32, "dplanes")
    ps = planes.c_struct()
    check(load().lf_composite_backward(ctypes.byref(ps), ctypes.byref(ref), ctypes.byref(vs), _ptr(dviews),
                                       _ptr(dplanes), _ptr(ws), ws.numel(), _stream_ptr(stream)))


def lf_composite_state_size(ref: L.LfRefCamera, views) -> int:
    vs = view_set(views)
    return int(load().lf_composite_state_size(ctypes.byref(ref), ctypes.byref(vs)))


def composite_state_shape(ref: L.LfRefCamera, views):
    """Shape of the saved composite state: [Vy*Vx][Ny][Nx][4] 32-bit words."""
    vs = view_set(views)
    return (vs.Vx * vs.Vy, ref.base.Ny, ref.base.Nx, 4)


def lf_composite_save(planes: Planes, ref: L.LfRefCamera, views, out: torch.Tensor, state: torch.Tensor,
                      ws: torch.Tensor, stream=None):
    """lf_composite that also writes the adjoint's starting state (16 bytes per
    view pixel) into state (asynchronous)."""
    vs = view_set(views)
    _need(out, views_shape(views, ref.base.Nx, ref.base.Ny), torch.float32, "views")
    _need(state, composite_state_shape(ref, views), torch.float32, "state")
    ps = planes.c_struct()
    check(load().lf_composite_save(ctypes.byref(ps), ctypes.byref(ref), ctypes.byref(vs), _ptr(out), _ptr(state),
                                   state.numel() * 4, _ptr(ws), ws.numel(), _stream_ptr(stream)))


def lf_composite_backward_saved(planes: Planes, ref: L.LfRefCamera, views, dviews: torch.Tensor,
                                state: torch.Tensor, dplanes: torch.Tensor, ws: torch.Tensor, stream=None):
    """Adjoint of lf_composite_save from its state: one back-to-front plane
    walk (asynchronous)."""
    vs = view_set(views)
    _need(dviews, (vs.Vx * vs.Vy, ref.base.Ny, ref.base.Nx, 4), torch.float32, "dviews")
    _need(state, composite_state_shape(ref, views), torch.float32, "state")
    _need(dplanes, (planes.N, ref.H, ref.W, 4), torch.float32, "dplanes")
    ps = planes.c_struct()
    check(load().lf_composite_backward_saved(ctypes.byref(ps), ctypes.byref(ref), ctypes.byref(vs), _ptr(dviews),
                                             _ptr(state), state.numel() * 4, _ptr(dplanes), _ptr(ws), ws.numel(),
                                             _stream_ptr(stream)))


def lf_build_mpi_backward_gaussians(g: DeviceGaussians, ref: L.LfRefCamera, planes: Planes, dplanes: torch.Tensor,
                                    grads: GaussianGrads, ws: torch.Tensor, stream=None):
    """Adjoint of lf_build_mpi_gaussians (ws: the forward's workspace, unchanged)."""
    _need(dplanes, (planes.N, ref.H, ref.W, 4), torch.float32, "dplanes")
    gs, ps, gr = g.c_struct(), planes.c_struct(), grads.c_struct(g.n)
    check(load().lf_build_mpi_backward_gaussians(ctypes.byref(gs), ctypes.byref(ref), ctypes.byref(ps),
                                                 _ptr(dplanes), ctypes.byref(gr), _ptr(ws), ws.numel(),
                                                 _stream_ptr(stream)))


def lf_build_mpi_backward_voxels(v: DeviceVoxels, ref: L.LfRefCamera, planes: Planes, dplanes: torch.Tensor,
                                 grads: VoxelGrads, ws: torch.Tensor, stream=None):
    """Adjoint of lf_build_mpi_voxels (ws: the forward's workspace, unchanged)."""
    _need(dplanes, (planes.N, ref.H, ref.W, 4), torch.float32, "dplanes")
    vs, ps, gr = v.c_struct(), planes.c_struct(), grads.c_struct(v.n)
    check(load().lf_build_mpi_backward_voxels(ctypes.byref(vs), ctypes.byref(ref), ctypes.byref(ps),
                                              _ptr(dplanes), ctypes.byref(gr), _ptr(ws), ws.numel(),
                                              _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# convenience: one object holding every buffer of a workload
# ---------------------------------------------------------------------------

class LightFieldRenderer:
    """Owns the device buffers for one (camera, display, views, N) set-up and
    runs splat + composite through the C ABI."""

    def __init__(self, camera, display, views, N: int, binning: str = "quantile", dtype: str = "f32",
                 n_capacity: int = 0, dup_capacity: int = 0, device="cuda", plane_filter: float = 0.0,
                 blend: str = "exact", save_state: bool = False):
        if blend not in BLEND:
            raise ValueError("blend must be one of %s" % sorted(BLEND))
        self.camera, self.display, self.views = camera, display, views
        self.N, self.binning, self.dtype = int(N), binning, dtype
        self.blend = blend                        # "3dgs": 3DGS cut-offs in the Gaussian splat
        self.ref = lf_make_ref_camera(camera, display)
        self.device = device
        self.n_capacity = int(n_capacity)
        self.dup_capacity = int(dup_capacity)
        self.plane_filter = float(plane_filter)   # V2LF low-pass sigma (plane pixels); 0 = off
        self.planes = None
        self.ws = None
        self.cws = alloc_workspace(lf_composite_workspace_size(self.N, views), device)
        self.out = torch.empty(views_shape(views, camera.Nx, camera.Ny), dtype=torch.float32, device=device)
        # save_state: composite() runs the saving form (lf_composite_save) and
        # backward() starts the composite adjoint from its state (one plane
        # walk instead of two); 16 bytes per view pixel
        self.save_state = bool(save_state)
        self.state = (torch.empty(composite_state_shape(self.ref, views), dtype=torch.float32, device=device)
                      if self.save_state else None)
        self.state_generation = -1
        self.generation = 0

    def _ensure(self, n: int):
        if self.planes is None or n > self.n_capacity:
            self.n_capacity = max(n, self.n_capacity)
            self.planes = Planes.empty(self.ref, self.N, self.n_capacity, self.dtype, self.device)
            cap = self.dup_capacity if self.dup_capacity > 0 else 8 * self.n_capacity + (1 << 20)
            self.ws = alloc_workspace(lf_build_mpi_workspace_size(self.ref, self.n_capacity, self.N, cap),
                                      self.device)

    def build(self, prims, stream=None):
        self._ensure(prims.n)
        self.generation += 1
        pl = self.planes
        view = Planes(pl.rgba, pl.d, pl.count, pl.chunk[: max(prims.n, 1)], pl.rect[: max(prims.n, 1)], pl.dtype_code)
        if isinstance(prims, DeviceGaussians):
            lf_build_mpi_gaussians(prims, self.ref, self.N, self.binning, self.ws, view, stream, self.blend)
        else:
            if self.blend != "exact":
                raise ValueError("3DGS blending applies to Gaussians only")
            lf_build_mpi_voxels(prims, self.ref, self.N, self.binning, self.ws, view, stream)
            if self.plane_filter > 0.0:
                lf_filter_planes(view, self.plane_filter, 0, stream)
        return view

    def composite(self, stream=None, out: Optional[torch.Tensor] = None):
        out = self.out if out is None else out
        if self.save_state:
            lf_composite_save(self.planes, self.ref, self.views, out, self.state, self.cws, stream)
            self.state_generation = self.generation
        else:
            lf_composite(self.planes, self.ref, self.views, out, self.cws, stream)
        return out

    def render(self, prims, stream=None):
        self.build(prims, stream)
        return self.composite(stream)

    def status(self):
        return lf_mpi_status(self.ws)

    def composite_status(self, stream=None) -> int:
        """Status code of the last composite (or its adjoint) on this renderer:
        LF_ERR_TIMEOUT if a bounded device wait gave up, else LF_OK."""
        vs = view_set(self.views)
        return int(load().lf_composite_status(int(self.N), ctypes.byref(vs), _ptr(self.cws), _stream_ptr(stream)))

    def capture(self, prims):
        """Captures one render of prims (build + composite, every kernel of the
        frame) into a CUDA graph; replay() then re-runs it on the current
        contents of the prims' and renderer's buffers. Stage tracing is turned
        off for this thread. Returns the number of kernels in the graph."""
        self._ensure(prims.n)
        self.render(prims)                      # warm: workspace and kernel attributes set up
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        lf_trace_enable(False)
        k0 = lf_launch_count()
        with torch.cuda.graph(g):
            self.render(prims, torch.cuda.current_stream())
        self.graph_kernels = lf_launch_count() - k0
        self.graph = g
        return self.graph_kernels

    def replay(self):
        self.graph.replay()
        return self.out

    def planes_view(self, n: int) -> Planes:
        pl = self.planes
        return Planes(pl.rgba, pl.d, pl.count, pl.chunk[: max(n, 1)], pl.rect[: max(n, 1)], pl.dtype_code)

    def backward(self, prims, dviews: torch.Tensor, stream=None):
        """Gradients of the last render of prims given dL/d(views): composite
        adjoint, then the splat adjoint on the same workspace."""
        if self.blend != "exact":
            raise ValueError("the adjoint differentiates exact blending; this renderer uses %r" % self.blend)
        dplanes = torch.empty((self.N, self.ref.H, self.ref.W, 4), dtype=torch.float32, device=self.device)
        if self.save_state and self.state_generation == self.generation:
            lf_composite_backward_saved(self.planes, self.ref, self.views, dviews, self.state, dplanes, self.cws,
                                        stream)
        else:
            lf_composite_backward(self.planes, self.ref, self.views, dviews, dplanes, self.cws, stream)
        view = self.planes_view(prims.n)
        if isinstance(prims, DeviceGaussians):
            grads = GaussianGrads.empty(prims.n, self.device)
            lf_build_mpi_backward_gaussians(prims, self.ref, view, dplanes, grads, self.ws, stream)
        else:
            grads = VoxelGrads.empty(prims.n, self.device)
            lf_build_mpi_backward_voxels(prims, self.ref, view, dplanes, grads, self.ws, stream)
        return grads, dplanes


# ---------------------------------------------------------------------------
# host-memory frames: copies overlapped with the compute of neighbouring frames
# ---------------------------------------------------------------------------

class HostPipeline:
    """Renders frames whose Gaussians live in (pinned) host memory and whose
    views go back to (pinned) host memory, `depth` frames in flight (2 by
    default). Each slot has its own device inputs, renderer (workspace,
    planes, views) and compute stream, so frames i and i-1 are computed side
    by side while frame i's host-to-device copy (copy stream) and earlier
    frames' device-to-host copies (second copy stream) run beside them,
    ordered by CUDA events. A slot is reused by frame i + depth once frame i's
    views have left it. (On the 1M-Gaussian display frame, FP32 views, two
    slots give 922 LF frames/s end to end and three 895: the frames computed
    side by side then slow each other more than the copies gain.) submit()
    returns the event that marks frame i's views in host memory."""

    def __init__(self, renderer: "LightFieldRenderer", n: int, device="cuda", graphs: bool = True, depth: int = 2):
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.r = renderer
        self.depth = depth
        self.renderers = [renderer] + [
            LightFieldRenderer(renderer.camera, renderer.display, renderer.views, renderer.N, renderer.binning,
                               renderer.dtype, n_capacity=max(n, renderer.n_capacity),
                               dup_capacity=renderer.dup_capacity, device=device,
                               plane_filter=renderer.plane_filter, blend=renderer.blend)
            for _ in range(depth - 1)]
        f = dict(dtype=torch.float32, device=device)
        # zero Gaussians sit at the world origin, in front of no reference camera
        # that sees them from z_near on, so warm-up and capture renders cull them
        self.slots = [DeviceGaussians(torch.zeros((n, 3), **f), torch.zeros((n, 3), **f), torch.zeros((n, 4), **f),
                                      torch.zeros((n,), **f), torch.zeros((n, 3), **f)) for _ in range(depth)]
        self.outs = [torch.empty_like(renderer.out) for _ in range(depth)]
        self.s_in, self.s_out = torch.cuda.Stream(device=device), torch.cuda.Stream(device=device)
        self.s_comp = [torch.cuda.Stream(device=device) for _ in range(depth)]
        E = torch.cuda.Event
        self.in_ready, self.in_free = [E() for _ in range(depth)], [E() for _ in range(depth)]
        self.out_ready, self.out_free = [E() for _ in range(depth)], [E() for _ in range(depth)]
        self.i = 0
        # one CUDA graph per slot: build from slot k, composite into view slot k
        self.graphs = None
        if graphs:
            self.graphs = []
            for k in range(depth):
                rk = self.renderers[k]
                rk.build(self.slots[k])
                rk.composite(out=self.outs[k])
                torch.cuda.synchronize()
                gk = torch.cuda.CUDAGraph()
                lf_trace_enable(False)
                with torch.cuda.graph(gk):
                    st = torch.cuda.current_stream()
                    rk.build(self.slots[k], st)
                    rk.composite(st, out=self.outs[k])
                self.graphs.append(gk)

    def submit(self, host: DeviceGaussians, host_out: torch.Tensor) -> torch.cuda.Event:
        k = self.i % self.depth
        dev, rk, sc = self.slots[k], self.renderers[k], self.s_comp[k]
        self.s_in.wait_event(self.in_free[k])          # frame i - depth no longer reads this slot
        with torch.cuda.stream(self.s_in):
            for dst, src in ((dev.means, host.means), (dev.scales, host.scales), (dev.quats, host.quats),
                             (dev.opacity, host.opacity), (dev.rgb, host.rgb)):
                dst.copy_(src, non_blocking=True)
        self.in_ready[k].record(self.s_in)
        sc.wait_event(self.in_ready[k])
        sc.wait_event(self.out_free[k])       # frame i - depth's views have left this slot
        if self.graphs is not None:
            with torch.cuda.stream(sc):
                self.graphs[k].replay()
        else:
            rk.build(dev, sc)
            rk.composite(sc, out=self.outs[k])
        self.in_free[k].record(sc)
        self.out_ready[k].record(sc)
        self.s_out.wait_event(self.out_ready[k])
        with torch.cuda.stream(self.s_out):
            host_out.copy_(self.outs[k], non_blocking=True)
        self.out_free[k].record(self.s_out)
        self.i += 1
        done = torch.cuda.Event()
        done.record(self.s_out)
        return done


# ---------------------------------------------------------------------------
# batching: several scenes, persistent launches, CUDA graph, autotuner
# ---------------------------------------------------------------------------

class BatchRenderer:
    """Several Gaussian scenes rendered as one batch (lf_batch_*): per-scene
    builds, one persistent raster and one persistent composite launch over
    every scene's work items; optionally captured once into a CUDA graph.
    workloads: objects with scene, camera, display, views, N, binning.
    Scene data is copied to the device once (update it in place through
    .prims[i] tensors; the captured graph reads the same buffers)."""

    def __init__(self, workloads, dtype: str = "f16", device="cuda", stream: Optional[torch.cuda.Stream] = None,
                 max_chunk_groups: int = 1):
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.parts = []
        scenes = (L.LfBatchScene * len(workloads))()
        for i, w in enumerate(workloads):
            r = LightFieldRenderer(w.camera, w.display, w.views, w.N, w.binning, dtype, device=device)
            g = DeviceGaussians.from_scene(w.scene, device=device)
            r._ensure(g.n)
            pv = r.planes_view(g.n)
            sc = scenes[i]
            sc.g = g.c_struct()
            sc.ref = r.ref
            sc.N, sc.binning = r.N, BINNING[w.binning]
            sc.planes = pv.c_struct()
            sc.views = view_set(w.views)
            sc.out = r.out.data_ptr()
            sc.ws, sc.ws_bytes = r.ws.data_ptr(), r.ws.numel()
            sc.cws, sc.cws_bytes = r.cws.data_ptr(), r.cws.numel()
            self.parts.append((r, g, pv))
        self._scenes = scenes
        h = ctypes.c_void_p()
        check(load().lf_batch_create(scenes, len(workloads), ctypes.byref(h)))
        self.handle = h
        # workspace for plans of up to max_chunk_groups chunk groups (1, 2 or 4)
        biggest = L.LfBatchPlan(9, 512, int(max_chunk_groups), 0)
        nbytes = int(load().lf_batch_plan_workspace_size(h, ctypes.byref(biggest)))
        if nbytes == 0:
            raise ValueError("max_chunk_groups must be 1, 2 or 4")
        self.ws = alloc_workspace(nbytes, device)
        self.plan = None
        self.prepare()

    @property
    def outputs(self):
        return [r.out for r, _, _ in self.parts]

    @property
    def prims(self):
        return [g for _, g, _ in self.parts]

    @property
    def planes(self):
        return [pv for _, _, pv in self.parts]

    def prepare(self, plan: Optional[dict] = None):
        p = None
        if plan is not None:
            p = L.LfBatchPlan(plan["views_per_thread"], plan["tile_x"], plan.get("chunk_groups", 1), plan["schedule"])
        check(load().lf_batch_prepare(self.handle, ctypes.byref(p) if p is not None else None, _ptr(self.ws),
                                      self.ws.numel(), ctypes.c_void_p(self.stream.cuda_stream)))
        self.plan = plan

    def render(self):
        check(load().lf_batch_render(self.handle, ctypes.c_void_p(self.stream.cuda_stream)))

    def capture(self):
        check(load().lf_batch_capture(self.handle, ctypes.c_void_p(self.stream.cuda_stream)))

    def launch(self):
        check(load().lf_batch_launch(self.handle, ctypes.c_void_p(self.stream.cuda_stream)))

    def autotune(self, reps: int = 2):
        best = L.LfBatchPlan()
        ms = ctypes.c_float(0.0)
        check(load().lf_batch_autotune(self.handle, _ptr(self.ws), self.ws.numel(), int(reps),
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(best), ctypes.byref(ms)))
        self.plan = {"views_per_thread": best.views_per_thread, "tile_x": best.tile_x,
                     "chunk_groups": best.chunk_groups, "schedule": best.schedule}
        return self.plan, float(ms.value)

    def status(self):
        return load().lf_batch_status(self.handle, ctypes.c_void_p(self.stream.cuda_stream))

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "handle", None) is not None:
            load().lf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# tracing
# ---------------------------------------------------------------------------

def lf_launch_count() -> int:
    return int(load().lf_launch_count())


def lf_selftest_bounded_wait(limit_ms: int = 50, stream=None) -> int:
    """Failure-detection self-test (bounded device wait that must give up):
    returns the status code, LF_ERR_TIMEOUT when the wait gave up as designed."""
    return int(load().lf_selftest_bounded_wait(int(limit_ms), _stream_ptr(stream)))


def lf_trace_enable(on: bool):
    check(load().lf_trace_enable(int(bool(on))))


def lf_trace_collect(max_stages: int = 64) -> dict:
    """{stage: (total_ms, calls)} of the traced stages since the last collect."""
    names = ctypes.create_string_buffer(32 * max_stages)
    ms = (ctypes.c_double * max_stages)()
    calls = (ctypes.c_int64 * max_stages)()
    k = load().lf_trace_collect(names, ms, calls, max_stages)
    out = {}
    for i in range(k):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(calls[i]))
    return out
