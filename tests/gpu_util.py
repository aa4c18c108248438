"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and derive the expected tile lists from the oracle's outputs."""
import numpy as np
import torch

from paper_2508_18540_gb300 import api
from paper_2508_18540_gb300 import synth as S

TILE = 16


def run_gpu(scene, camera, display, views, N, binning, dtype="f32", dup_capacity=0, stream=None):
    r = api.LightFieldRenderer(camera, display, views, N, binning, dtype, dup_capacity=dup_capacity)
    prims = api.DeviceVoxels.from_scene(scene) if hasattr(scene, "ijk") else api.DeviceGaussians.from_scene(scene)
    pl = r.build(prims, stream)
    st, needed, M = r.status()
    out = dict(status=st, needed=needed, M=M, renderer=r, prims=prims)
    if st != 0:
        return out
    v = r.composite(stream)
    torch.cuda.synchronize()
    n = scene.n
    out.update(planes=pl.rgba.float().cpu().numpy().astype(np.float64), d=pl.d.cpu().numpy(),
               count=pl.count.cpu().numpy(), chunk=pl.chunk[:n].cpu().numpy(), rect=pl.rect[:n].cpu().numpy(),
               views=v.cpu().numpy().astype(np.float64))
    tiles_x = (r.ref.W + TILE - 1) // TILE
    tiles_y = (r.ref.H + TILE - 1) // TILE
    order, prims_l, seg = api.lf_mpi_tile_lists(r.ws, n, tiles_x * tiles_y, N)
    out.update(order=order, tile_prims=prims_l, seg=seg, tiles_x=tiles_x, tiles_y=tiles_y, n_pairs=len(prims_l))
    return out


def expected_tile_lists(orc_out, W, H, N):
    """Definition of the 3D tile lists: tile t, chunk c holds, in (depth,
    index) order, every primitive of chunk c whose footprint rectangle
    intersects tile t."""
    tx_n = (W + TILE - 1) // TILE
    ty_n = (H + TILE - 1) // TILE
    lists = {}
    for g in orc_out["order"]:
        x0, y0, x1, y1 = orc_out["rect"][g]
        c = int(orc_out["chunk"][g])
        for ty in range(y0 // TILE, y1 // TILE + 1):
            for tx in range(x0 // TILE, x1 // TILE + 1):
                lists.setdefault((ty * tx_n + tx, c), []).append(int(g))
    return lists, tx_n * ty_n


def check_tile_lists(gpu, orc_out, W, H, N):
    lists, n_tiles = expected_tile_lists(orc_out, W, H, N)
    seg = gpu["seg"]
    total = 0
    for t in range(n_tiles):
        for c in range(N):
            s, e = seg[t * N + c]
            want = lists.get((t, c), [])
            got = gpu["tile_prims"][s:e].tolist() if e > s else []
            assert got == want, (t, c)
            total += len(want)
    assert total == gpu["n_pairs"]


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def small_rotated_camera(Nx=100, Ny=70):
    a, b = 0.2, -0.1
    Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    cam = S.Camera(Rx @ Ry, np.array([0.1, -0.05, 0.3]), np.radians(50.0), np.radians(38.0), Nx, Ny)
    return cam


def longest_super_tile_list(o, N):
    """Longest (32 x 32 super-tile, chunk) list of an oracle render: the
    culled-in primitives whose rectangle meets the super-tile, per chunk."""
    v = o["valid"].astype(bool)
    r = o["rect"][v].astype(np.int64)
    ch = o["chunk"][v].astype(np.int64)
    W, H = o["ref"].W, o["ref"].H
    sx_n, sy_n = (W + 31) // 32, (H + 31) // 32
    counts = np.zeros((sy_n, sx_n, N), np.int64)
    for i in range(r.shape[0]):
        x0, y0, x1, y1 = r[i]
        counts[y0 // 32:y1 // 32 + 1, x0 // 32:x1 // 32 + 1, ch[i]] += 1
    return int(counts.max())
