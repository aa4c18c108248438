"""Seeded synthetic inputs: scene, camera, display and view-set descriptions.

This module only draws random numbers and describes inputs; it holds none of
the method's arithmetic (no projection, binning or blending). Both the CUDA
library's tests/benchmarks and the CPU oracle consume these objects.

The paper evaluates on the Mip-NeRF360 scenes with trained 3DGS / SVR models
(Sec. 5.1), which are not available; these generators stand in for them with
scenes of the same kind and size: 3D Gaussians with non-directional (DC)
colour, or sparse voxels with per-corner densities, seen by a 45-view
horizontal-parallax quilt at 512x512 (Table 1 setting).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np


@dataclasses.dataclass
class Camera:
    """Base camera: world point p maps to R p + t (+x right, +y down, +z forward)."""
    R: np.ndarray            # (3, 3) float64, world -> camera rotation
    t: np.ndarray            # (3,) float64
    theta_x: float           # full horizontal field of view (radians)
    theta_y: float           # full vertical field of view (radians)
    Nx: int                  # per-view width
    Ny: int                  # per-view height


@dataclasses.dataclass
class Display:
    """Light-field display set-up (Sec. 4.2 / 4.3 notation)."""
    D_focal: float
    phi_x: float             # horizontal viewing angle (radians)
    phi_y: float = 0.0       # vertical viewing angle (radians)
    D_shift: float = 0.0
    P_s: int = 1
    f_aa: float = 0.3        # the 3DGS dilation f in pixels^2
    z_near: float = 0.2


@dataclasses.dataclass
class ViewSet:
    Vx: int
    Vy: int = 1
    bilinear: bool = False
    bg: tuple = (0.0, 0.0, 0.0)
    atlas_cols: int = 0      # 0: separate views; c: quilt atlas with c view tiles per row


@dataclasses.dataclass
class GaussianScene:
    """Activated 3D Gaussians, structure of arrays, float32."""
    means: np.ndarray        # (n, 3)
    scales: np.ndarray       # (n, 3) linear standard deviations
    quats: np.ndarray        # (n, 4) (w, x, y, z), need not be normalised
    opacity: np.ndarray      # (n,)
    rgb: np.ndarray          # (n, 3)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "GaussianScene":
        return GaussianScene(*(np.ascontiguousarray(a[idx]) for a in
                               (self.means, self.scales, self.quats, self.opacity, self.rgb)))


@dataclasses.dataclass
class VoxelScene:
    """Sparse voxels: cube v has low corner origin + ijk[v] * s_v and side
    s_v = base_size * 2^-level[v]; density8[v, c] is the density at corner
    c = i + 2 j + 4 k (offsets i, j, k along x, y, z)."""
    ijk: np.ndarray          # (n, 3) int32
    level: np.ndarray        # (n,) uint8
    origin: np.ndarray       # (3,) float64
    base_size: float
    density8: np.ndarray     # (n, 8) float32, already activated (>= 0)
    rgb: np.ndarray          # (n, 3) float32

    @property
    def n(self) -> int:
        return int(self.ijk.shape[0])

    def subset(self, idx) -> "VoxelScene":
        return VoxelScene(np.ascontiguousarray(self.ijk[idx]), np.ascontiguousarray(self.level[idx]),
                          self.origin.copy(), self.base_size,
                          np.ascontiguousarray(self.density8[idx]), np.ascontiguousarray(self.rgb[idx]))


@dataclasses.dataclass
class Workload:
    name: str
    scene: object
    camera: Camera
    display: Display
    views: ViewSet
    N: int                   # N_chunk
    binning: str             # "quantile" or "disparity"


def identity_camera(N: int, fov_deg: float = 50.0, t=(0.0, 0.0, 0.0)) -> Camera:
    th = math.radians(fov_deg)
    return Camera(np.eye(3), np.asarray(t, dtype=np.float64), th, th, N, N)


def display_for(D_focal: float, baseline: float, **kw) -> Display:
    """Reading: the configurations give a camera baseline (outermost lateral
    offset) instead of a viewing angle; tan(phi_x/2) = baseline / D_focal
    makes the outermost Delta x equal the baseline."""
    return Display(D_focal=D_focal, phi_x=2.0 * math.atan(baseline / D_focal), **kw)


def harmonic_focal(z_min: float, z_max: float) -> float:
    """Reading: D_focal at the disparity midpoint of the scene depth range."""
    return 2.0 / (1.0 / z_min + 1.0 / z_max)


# --------------------------------------------------------------------------
# Gaussian scenes
# --------------------------------------------------------------------------

def uniform_gaussians(n: int, seed: int, xy=(-1.0, 1.0), z=(2.0, 6.0),
                      log_scale=(math.log(0.02), 0.3), opacity=(0.1, 0.9)) -> GaussianScene:
    """Isotropic Gaussians, means uniform in a box, log-normal scale."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), np.float32)
    means[:, 0] = rng.uniform(xy[0], xy[1], n)
    means[:, 1] = rng.uniform(xy[0], xy[1], n)
    means[:, 2] = rng.uniform(z[0], z[1], n)
    s = np.exp(rng.normal(log_scale[0], log_scale[1], n)).astype(np.float32)
    scales = np.repeat(s[:, None], 3, axis=1).astype(np.float32)
    quats = np.zeros((n, 4), np.float32)
    quats[:, 0] = 1.0
    op = rng.uniform(opacity[0], opacity[1], n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    return GaussianScene(means, scales, quats, op, rgb)


def blob_gaussians(n: int, seed: int, n_blobs: int = 200, z=(1.5, 10.0), fov_deg: float = 50.0,
                   log_scale=(math.log(0.01), 0.5)) -> GaussianScene:
    """Anisotropic Gaussians clustered in blobs (reading of the 1M-Gaussian
    display-scale workload): blob centres z ~ U[z0, z1], (x, y) uniform in 0.8x
    the base frustum at that depth, blob std 0.05 z, random unit quaternions,
    per-axis log-scale ~ N(log 0.01, 0.5), opacity ~ Beta(2, 2), RGB ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    tth = math.tan(math.radians(fov_deg) / 2.0)
    cz = rng.uniform(z[0], z[1], n_blobs)
    cx = rng.uniform(-0.8, 0.8, n_blobs) * cz * tth
    cy = rng.uniform(-0.8, 0.8, n_blobs) * cz * tth
    blob = np.arange(n) % n_blobs
    std = 0.05 * cz[blob]
    means = np.stack([cx[blob], cy[blob], cz[blob]], axis=1) + rng.normal(size=(n, 3)) * std[:, None]
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3)))
    op = rng.beta(2.0, 2.0, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    f = np.float32
    return GaussianScene(means.astype(f), scales.astype(f), q.astype(f), op.astype(f), rgb.astype(f))


# --------------------------------------------------------------------------
# Sparse voxel scenes
# --------------------------------------------------------------------------

def _value_noise(rng, pts: np.ndarray, octaves=((8, 1.0), (24, 0.5), (64, 0.25))) -> np.ndarray:
    """Smooth seeded noise on [-2, 2]^3: random lattice values, trilinearly
    interpolated, summed over a few octaves (input texture only)."""
    out = np.zeros(pts.shape[0], np.float32)
    u = (pts.astype(np.float64) + 2.0) / 4.0
    for res, amp in octaves:
        lat = rng.standard_normal((res + 1, res + 1, res + 1)).astype(np.float32)
        g = np.clip(u * res, 0.0, res - 1e-6)
        i0 = np.floor(g).astype(np.int64)
        f = (g - i0).astype(np.float32)
        acc = np.zeros(pts.shape[0], np.float32)
        for c in range(8):
            ox, oy, oz = c & 1, (c >> 1) & 1, (c >> 2) & 1
            w = ((f[:, 0] if ox else 1 - f[:, 0]) * (f[:, 1] if oy else 1 - f[:, 1]) *
                 (f[:, 2] if oz else 1 - f[:, 2]))
            acc += w * lat[i0[:, 0] + ox, i0[:, 1] + oy, i0[:, 2] + oz]
        out += amp * acc
    return out


def sparse_voxels(n_keep: int, seed: int, base_res: int = 256, keep0: float = 0.035,
                  refine0: int = None, refine1: int = None) -> VoxelScene:
    """3-level sparse grid over [-2, 2]^3: base base_res^3 cells; the cells
    where a seeded noise field is highest are kept, the highest of those are
    split into 8 children (level 1) and the highest children split again
    (level 2); the n_keep leaves with the highest noise remain. Corner
    densities softplus(N(0, 2)), RGB ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    size0 = 4.0 / base_res
    if refine0 is None:
        refine0 = max(1, n_keep // 12)
    if refine1 is None:
        refine1 = max(1, n_keep // 20)
    # level 0: evaluate noise on all cell centres, slab by slab
    keep_n = max(int(keep0 * base_res ** 3), n_keep // 2)
    noise_rng = np.random.default_rng(seed + 7919)
    # one set of lattices reused for all evaluations of the field
    lat_seed = int(noise_rng.integers(1 << 31))

    def field(p):
        return _value_noise(np.random.default_rng(lat_seed), p)

    ax = (np.arange(base_res, dtype=np.float64) + 0.5) * size0 - 2.0
    vals = np.empty(base_res ** 3, np.float32)
    plane = np.stack(np.meshgrid(ax, ax, indexing="ij"), -1).reshape(-1, 2)
    for kz in range(base_res):
        pts = np.concatenate([plane, np.full((plane.shape[0], 1), ax[kz])], axis=1)
        vals[kz * base_res * base_res:(kz + 1) * base_res * base_res] = field(pts)
    top = np.argpartition(-vals, keep_n - 1)[:keep_n]
    top = top[np.argsort(-vals[top], kind="stable")]
    kz, rem = np.divmod(top, base_res * base_res)
    ki, kj = np.divmod(rem, base_res)
    ijk0 = np.stack([ki, kj, kz], 1).astype(np.int64)
    v0 = vals[top]

    def children(ijk):
        ch = []
        for c in range(8):
            ch.append(ijk * 2 + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]))
        return np.concatenate(ch, 0)

    def centres(ijk, level):
        s = size0 / (1 << level)
        return (ijk.astype(np.float64) + 0.5) * s - 2.0

    # refine the highest-noise level-0 cells
    r0 = min(refine0, ijk0.shape[0])
    ijk1 = children(ijk0[:r0])
    v1 = field(centres(ijk1, 1))
    o1 = np.argsort(-v1, kind="stable")
    ijk1, v1 = ijk1[o1], v1[o1]
    r1 = min(refine1, ijk1.shape[0])
    ijk2 = children(ijk1[:r1])
    v2 = field(centres(ijk2, 2))

    leaves_ijk = np.concatenate([ijk0[r0:], ijk1[r1:], ijk2], 0)
    leaves_lvl = np.concatenate([np.zeros(ijk0.shape[0] - r0, np.uint8), np.ones(ijk1.shape[0] - r1, np.uint8),
                                 np.full(ijk2.shape[0], 2, np.uint8)])
    leaves_v = np.concatenate([v0[r0:], v1[r1:], v2])
    n = min(n_keep, leaves_v.shape[0])
    sel = np.argsort(-leaves_v, kind="stable")[:n]
    sel.sort()
    ijk = leaves_ijk[sel].astype(np.int32)
    lvl = leaves_lvl[sel]
    dens = np.logaddexp(0.0, rng.normal(0.0, 2.0, (n, 8))).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    return VoxelScene(ijk, lvl, np.array([-2.0, -2.0, -2.0]), size0, dens, rgb)


# --------------------------------------------------------------------------
# Named workloads (sizes of the paper's Table 1 setting)
# --------------------------------------------------------------------------

def workload_tiny(seed: int = 1) -> Workload:
    """10k isotropic Gaussians, 128x128, N=16 uniform-in-disparity, 9 views
    over +-0.1."""
    scene = uniform_gaussians(10_000, seed)
    cam = identity_camera(128)
    disp = display_for(3.0, 0.1)
    return Workload("g2lf_tiny_10k_128px_N16_9v", scene, cam, disp, ViewSet(9), 16, "disparity")


def workload_display(seed: int = 2, n: int = 1_000_000, res: int = 512, N: int = 64, V: int = 45) -> Workload:
    """1M anisotropic Gaussians in 200 blobs over depth [1.5, 10], 512x512,
    N=64 quantile planes, 45 views over +-0.15."""
    scene = blob_gaussians(n, seed)
    cam = identity_camera(res)
    disp = display_for(harmonic_focal(1.5, 10.0), 0.15)
    return Workload(f"g2lf_{n // 1000}k_{res}px_N{N}_{V}v", scene, cam, disp, ViewSet(V), N, "quantile")


def workload_voxels(seed: int = 3, n: int = 2_000_000, res: int = 512, N: int = 64, V: int = 45,
                    base_res: int = 256) -> Workload:
    """2M sparse voxels from a 3-level grid, 512x512, N=64, 45 views. The
    volume [-2, 2]^3 sits 6 units in front of the camera (depth [4, 8])."""
    scene = sparse_voxels(n, seed, base_res=base_res)
    cam = identity_camera(res, t=(0.0, 0.0, 6.0))
    disp = display_for(harmonic_focal(4.0, 8.0), 0.15)
    return Workload(f"v2lf_{n // 1000}k_{res}px_N{N}_{V}v", scene, cam, disp, ViewSet(V), N, "quantile")


def workloads_batched(seed: int = 4, scale: float = 1.0) -> List[Workload]:
    """Six scenes of uneven size for the batched launch (reading of the
    batched configuration: pairing of resolution and N with scene size)."""
    spec = [(50_000, 9, 256, 64), (200_000, 45, 384, 64), (500_000, 45, 512, 128),
            (1_000_000, 96, 512, 128), (2_000_000, 96, 768, 256), (3_000_000, 128, 1024, 512)]
    out = []
    for s, (n, V, res, N) in enumerate(spec):
        n = max(1000, int(n * scale))
        out.append(workload_display(seed + 101 * s, n=n, res=res, N=N, V=V))
    return out


def workload_fit(seed: int = 5, n: int = 300_000, res: int = 512, N: int = 64, V: int = 45) -> Workload:
    """Differentiable workload: 300k Gaussians distributed as the display workload."""
    return workload_display(seed, n=n, res=res, N=N, V=V)


def perturbed(scene: GaussianScene, seed: int, mean_std: float = 0.01, op_std: float = 0.05) -> GaussianScene:
    """Copy of a scene with means + N(0, mean_std) and opacities + N(0, op_std),
    clipped to (0.01, 0.99)."""
    rng = np.random.default_rng(seed)
    m = (scene.means + rng.normal(0.0, mean_std, scene.means.shape)).astype(np.float32)
    o = np.clip(scene.opacity + rng.normal(0.0, op_std, scene.opacity.shape), 0.01, 0.99).astype(np.float32)
    return GaussianScene(m, scene.scales.copy(), scene.quats.copy(), o, scene.rgb.copy())
