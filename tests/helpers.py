"""Independent numpy geometry for pinning the oracle (tests only).

Nothing here reuses the oracle's formulas: rays are built from camera
positions and intersected with planes, rotations use quaternion products,
Jacobians are taken by finite differences.
"""
import math

import numpy as np

from paper_2508_18540_gb300 import synth as S


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def quat_rotate(q, v):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return qmul(qmul(q, np.concatenate([[0.0], v])), qc)[1:]


def sigma3_from_quat(q, s):
    """Sigma_3 = sum_l s_l^2 (q e_l q*)(q e_l q*)^T."""
    S3 = np.zeros((3, 3))
    for l in range(3):
        e = np.zeros(3)
        e[l] = 1.0
        a = quat_rotate(q, e)
        S3 += float(s[l]) ** 2 * np.outer(a, a)
    return S3


def base_view_ray(disp, cam, dx, dy, u, v):
    """Ray of quilt view (Delta x, Delta y) through normalised pixel (u, v):
    the view camera sits at (dx, dy, 0) in the base frame, all views share
    the focal-plane window (principal rays converge at its centre)."""
    Df = disp.D_focal
    tx, ty = math.tan(cam.theta_x / 2), math.tan(cam.theta_y / 2)
    o = np.array([dx, dy, 0.0])
    F = np.array([Df * tx * u, Df * ty * v, Df])
    return o, F - o


def hit_plane_z(o, d, z):
    t = (z - o[2]) / d[2]
    return o + t * d


def ref_pixel_of_point(ref, P):
    """Plane-pixel coordinates of a base-frame point seen by the reference
    camera located at (0, 0, D_forward), looking +z, fov theta'."""
    zr = P[2] - ref.D_forward
    u = P[0] / (zr * ref.tthp_x)
    v = P[1] / (zr * ref.tthp_y)
    return ((u + 1) * ref.W - 1) / 2, ((v + 1) * ref.H - 1) / 2


def ref_pixel_ray(ref, x, y):
    """Base-frame ray of the reference camera through plane pixel (x, y)."""
    u = (2 * x + 1) / ref.W - 1
    v = (2 * y + 1) / ref.H - 1
    o = np.array([0.0, 0.0, ref.D_forward])
    return o, np.array([u * ref.tthp_x, v * ref.tthp_y, 1.0])


def flat_gauss_alpha(P, mean, R2, s2, opacity):
    """Opacity of a flat fronto-parallel Gaussian (world-plane density) at P."""
    Sxy = R2 @ np.diag(np.asarray(s2, np.float64) ** 2) @ R2.T
    d = P[:2] - mean[:2]
    q = d @ np.linalg.solve(Sxy, d)
    return min(0.99, opacity * math.exp(-0.5 * q))


def flat_scene(specs):
    """specs: list of (mean3, (sx, sy), angle, opacity, rgb3) fronto-parallel
    flat Gaussians (z-scale 0, rotation about the optical axis)."""
    n = len(specs)
    means = np.zeros((n, 3), np.float32)
    scales = np.zeros((n, 3), np.float32)
    quats = np.zeros((n, 4), np.float32)
    op = np.zeros(n, np.float32)
    rgb = np.zeros((n, 3), np.float32)
    for i, (m, s, ang, o, c) in enumerate(specs):
        means[i] = m
        scales[i, :2] = s
        quats[i] = [math.cos(ang / 2), 0.0, 0.0, math.sin(ang / 2)]
        op[i] = o
        rgb[i] = c
    return S.GaussianScene(means, scales, quats, op, rgb)


def rot2(ang):
    c, s = math.cos(ang), math.sin(ang)
    return np.array([[c, -s], [s, c]])


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * math.log10(peak * peak / mse)
