"""Pins for the oracle's swizzle blending (Sec. 4.3, Eq. (u_prime),
Eq. (alpha_blend), the compositing steps of Algorithm 1) against geometric special cases
and brute-force per-view volume rendering."""
import math

import numpy as np
import pytest

from paper_2508_18540_gb300 import synth as S
from tests import helpers as H


def _grid_plane(z0, n_side, half, rng, sigma):
    """A textured fronto-parallel layer: a grid of flat Gaussians at depth z0."""
    xs = np.linspace(-half, half, n_side)
    specs = []
    for yv in xs:
        for xv in xs:
            specs.append(((xv, yv, z0), (sigma, sigma), 0.0, 0.9, tuple(rng.uniform(0, 1, 3))))
    return H.flat_scene(specs)


def test_focal_plane_views_identical(orc):
    # Everything at z = D_focal: zero parallax, every view equals the plane.
    rng = np.random.default_rng(0)
    D_f = float(np.float32(3.0))
    sc = _grid_plane(D_f, 12, 1.0, rng, 0.05)
    cam = S.identity_camera(64)
    disp = S.display_for(D_f, 0.15)
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(9), N=4, binning="quantile")
    assert out["count"].sum() == sc.n and out["count"][0] == sc.n or out["count"].max() > 0
    v = out["views"]
    for j in range(9):
        assert np.array_equal(v[j], v[4])
    # and the (single non-empty) plane is what is shown
    k = int(np.argmax(out["count"]))
    assert np.allclose(v[4], out["planes"][k] if out["count"].max() == sc.n else v[4], atol=0)


def test_lone_plane_shifts_by_its_disparity(orc):
    # A lone layer at depth d is seen by view j at plane coordinates shifted
    # by b_j W'/2 plane pixels, b_j = Delta x_j (D_f - d)/(D_f (d - D_fwd) tan(theta'/2)).
    # d (in front of the focal plane) is chosen by bisection on that closed
    # form so that neighbouring views differ by exactly +1 plane pixel. The
    # centre view's sampling position comes from ray geometry (the centre
    # camera's ray hits the layer, the reference camera projects the hit);
    # view j must then show the plane texel nearest to that position + (j - 4).
    rng = np.random.default_rng(1)
    cam = S.identity_camera(96)
    D_f = 3.0
    disp = S.display_for(D_f, 0.1)
    r = orc.make_ref(cam, disp)
    dx, _ = orc.view_offsets(r, 9, 1)
    step = dx[1] - dx[0]

    def shift(d):
        return step * (D_f - d) / (D_f * (d - r.D_forward) * r.tthp_x) * r.W / 2

    lo, hi = r.D_forward + 1e-3, D_f      # shift decreases from large to 0 over (D_fwd, D_f]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if shift(mid) > 1.0:
            lo = mid
        else:
            hi = mid
    z0 = float(np.float32(lo))
    sc = _grid_plane(z0, 30, 1.2, rng, 0.03)
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(9), N=1, binning="quantile")
    d = out["d"][0]
    assert shift(d) == pytest.approx(1.0, abs=1e-5)
    plane = out["planes"][0]
    v = out["views"]
    checked = 0
    for y in range(0, cam.Ny, 5):
        for x in range(cam.Nx):
            u = (2 * x + 1) / cam.Nx - 1
            vv = (2 * y + 1) / cam.Ny - 1
            o, dirv = H.base_view_ray(disp, cam, 0.0, 0.0, u, vv)
            X, Y = H.ref_pixel_of_point(r, H.hit_plane_z(o, dirv, d))
            fx, fy = (X + 0.5) % 1.0, (Y + 0.5) % 1.0
            if min(fx, 1 - fx) < 1e-3 or min(fy, 1 - fy) < 1e-3:
                continue
            iy = math.floor(Y + 0.5)
            for j in range(9):
                ix = math.floor(X + 0.5) + (j - 4)
                want = plane[iy, ix] if (0 <= ix < r.W and 0 <= iy < r.H) else np.zeros(4)
                assert np.array_equal(v[j, y, x], want), (j, y, x)
                checked += 1
    assert checked > 4000


def test_transmittance_monotone_and_bounded(orc):
    w = S.workload_tiny(seed=11)
    sc = w.scene.subset(np.arange(3000))
    out = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=w.N, binning=w.binning)
    prev = np.zeros_like(out["views"][..., 3])
    for k in range(1, w.N + 1):
        cnt = out["count"].copy()
        cnt[k:] = 0
        v = orc.composite(out["ref"], out["planes"], out["d"], cnt, w.views.Vx, 1, False)
        A = v[..., 3]
        assert np.all(A >= prev - 1e-15) and np.all(A <= 1.0) and np.all(A >= 0.0)
        assert np.all(v[..., :3] <= A[..., None] + 1e-12)      # Q_c <= 1 - T for rgb in [0, 1]
        prev = A
    # white primitives: Q_c == 1 - T
    sc.rgb[:] = 1.0
    out = orc.render(scene=sc, camera=w.camera, display=w.display, views=w.views, N=w.N, binning=w.binning)
    for c in range(3):
        assert np.allclose(out["views"][..., c], out["views"][..., 3], atol=1e-12)


def _bruteforce_views(r, cam, disp, sc, rects, dxs, truncate_margin):
    """Per-view volume rendering of flat fronto-parallel Gaussians, each view
    camera at (Delta x, 0, 0) ray-traced directly (no planes). A Gaussian
    contributes only inside its footprint rectangle (as seen by the
    reference camera); returns views and a mask of pixels at least
    truncate_margin plane pixels away from every rectangle border."""
    V = len(dxs)
    out = np.zeros((V, cam.Ny, cam.Nx, 4))
    ok = np.ones((V, cam.Ny, cam.Nx), bool)
    order = np.argsort(sc.means[:, 2], kind="stable")
    for j, dx in enumerate(dxs):
        for y in range(cam.Ny):
            for x in range(cam.Nx):
                u = (2 * x + 1) / cam.Nx - 1
                v = (2 * y + 1) / cam.Ny - 1
                o, d = H.base_view_ray(disp, cam, dx, 0.0, u, v)
                Q = np.zeros(3)
                T = 1.0
                for g in order:
                    m = sc.means[g].astype(np.float64)
                    P = H.hit_plane_z(o, d, m[2])
                    X, Y = H.ref_pixel_of_point(r, P)
                    x0, y0, x1, y1 = rects[g]
                    inside = x0 <= X <= x1 and y0 <= Y <= y1
                    near = (x0 - truncate_margin <= X <= x1 + truncate_margin and
                            y0 - truncate_margin <= Y <= y1 + truncate_margin)
                    deep = (x0 + truncate_margin <= X <= x1 - truncate_margin and
                            y0 + truncate_margin <= Y <= y1 - truncate_margin)
                    if near and not deep:
                        ok[j, y, x] = False
                    if not inside:
                        continue
                    q = sc.quats[g].astype(np.float64)
                    ang = 2 * math.atan2(q[3], q[0])
                    a = H.flat_gauss_alpha(P, m, H.rot2(ang), sc.scales[g, :2].astype(np.float64),
                                           float(sc.opacity[g]))
                    Q += T * a * sc.rgb[g]
                    T *= 1 - a
                out[j, y, x, :3] = Q
                out[j, y, x, 3] = 1 - T
    return out, ok


def test_one_primitive_per_chunk_converges_to_bruteforce(orc):
    # With one flat Gaussian per chunk and f = 0, the planes hold each
    # Gaussian exactly; the only G2LF error left is resampling the planes,
    # which must vanish as the plane resolution P_s grows (Sec. 5.1: both
    # interpolations approach the same result as P_s -> infinity).
    cam = S.identity_camera(40, 50.0)
    sc = H.flat_scene([((0.05, 0.02, 2.4), (0.12, 0.07), 0.5, 0.7, (1.0, 0.2, 0.1)),
                       ((-0.1, 0.0, 3.1), (0.10, 0.15), -0.3, 0.6, (0.1, 0.9, 0.2)),
                       ((0.15, -0.05, 4.6), (0.25, 0.12), 1.1, 0.8, (0.2, 0.3, 1.0))])
    errs = {"bilinear": [], "nearest": []}
    for P_s in (1, 2, 4, 8):
        disp = S.display_for(3.0, 0.2, f_aa=0.0, P_s=P_s)
        for mode in errs:
            out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(5, 1, mode == "bilinear"),
                             N=3, binning="quantile")
            assert out["count"].tolist() == [1, 1, 1]
            r = out["ref"]
            dxs, _ = orc.view_offsets(r, 5, 1)
            bf, ok = _bruteforce_views(r, cam, disp, sc, out["rect"], dxs[[0, 2, 4]], 2.0)
            diff = np.abs(out["views"][[0, 2, 4]] - bf).max(axis=-1)
            errs[mode].append(float(diff[ok].max()))
    b, nn = errs["bilinear"], errs["nearest"]
    assert b[0] > 1e-3 and nn[0] > 1e-3            # the test has something to measure
    # (P_s = 1 -> 2 is still pre-asymptotic for Gaussians ~1 px wide)
    assert b[3] < b[2] < b[1] and b[3] < b[1] / 12   # ~ P_s^-2
    assert nn[3] < nn[2] < nn[1] and nn[3] < nn[1] / 3   # ~ P_s^-1


def test_bilinear_at_texel_centres_equals_nearest(orc):
    # On the focal plane with P_s = 1 every sample lands on a texel centre:
    # bilinear and nearest sampling must agree.
    rng = np.random.default_rng(4)
    D_f = float(np.float32(3.0))
    sc = _grid_plane(D_f, 10, 1.0, rng, 0.06)
    cam = S.identity_camera(48)
    disp = S.display_for(D_f, 0.1)
    a = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(3, 1, False), N=1, binning="quantile")
    b = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(3, 1, True), N=1, binning="quantile")
    assert np.allclose(a["views"], b["views"], atol=1e-9)


def test_bilinear_taps_outside_the_plane_are_transparent(orc):
    # reading: a bilinear tap outside the plane contributes a transparent
    # zero. With one fully opaque white plane, every view pixel's opacity is
    # the summed weight of its in-plane taps, computed here from the sample
    # position of Eq. (u_prime) (pixels whose samples leave the plane at the
    # outer views' edges get less than 1)
    cam = S.identity_camera(24)
    disp = S.display_for(3.0, 0.3)
    r = orc.make_ref(cam, disp)
    N = 1
    d = np.array([2.2])          # off the focal plane: views shift against the plane
    planes = np.ones((N, r.H, r.W, 4))
    count = np.array([1], np.int64)
    Vx = 5
    v = orc.composite(r, planes, d, count, Vx, 1, True)
    dx, dy = orc.view_offsets(r, Vx, 1)
    partial = 0
    for j in range(Vx):
        for y in range(r.cam.Ny):
            Y = orc.plane_pixel(r, 1, dy[0], d[0], y)
            for x in range(r.cam.Nx):
                X = orc.plane_pixel(r, 0, dx[j], d[0], x)
                x0, y0 = math.floor(X), math.floor(Y)
                wx, wy = X - x0, Y - y0
                w_in = 0.0
                for ty, wty in ((y0, 1 - wy), (y0 + 1, wy)):
                    for tx, wtx in ((x0, 1 - wx), (x0 + 1, wx)):
                        if 0 <= tx < r.W and 0 <= ty < r.H:
                            w_in += wtx * wty
                assert v[j, y, x, 3] == pytest.approx(w_in, abs=1e-12)
                partial += w_in < 1 - 1e-9
    assert partial > 10


def test_background_and_empty(orc):
    cam = S.identity_camera(16)
    disp = S.display_for(3.0, 0.1)
    sc = H.flat_scene([((0, 0, 3.0), (0.01, 0.01), 0.0, 0.5, (1, 1, 1))])
    sc.means[0, 2] = -5.0          # culled: nothing to render
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(3, 1, False, (0.2, 0.3, 0.4)),
                     N=4, binning="quantile")
    assert out["M"] == 0
    v = out["views"]
    assert np.allclose(v[..., 0], 0.2) and np.allclose(v[..., 1], 0.3) and np.allclose(v[..., 2], 0.4)
    assert np.all(v[..., 3] == 0.0)
    # one wide flat layer on the focal plane (no parallax, f = 0): every view
    # pixel is its closed-form opacity a over the background, a c + (1 - a) bg
    disp0 = S.display_for(3.0, 0.1, f_aa=0.0)
    sc = H.flat_scene([((0, 0, 3.0), (1.5, 1.0), 0.2, 0.7, (0.9, 0.5, 0.1))])
    bg = (0.2, 0.3, 0.4)
    out = orc.render(scene=sc, camera=cam, display=disp0, views=S.ViewSet(3, 1, False, bg), N=1,
                     binning="quantile")
    r = out["ref"]
    m = sc.means[0].astype(np.float64)
    q = sc.quats[0].astype(np.float64)
    ang = 2 * math.atan2(q[3], q[0])
    x0, y0, x1, y1 = out["rect"][0]
    for y in range(r.H):
        for x in range(r.W):
            if not (x0 <= x <= x1 and y0 <= y <= y1):
                continue
            o, d = H.ref_pixel_ray(r, x, y)
            a = H.flat_gauss_alpha(H.hit_plane_z(o, d, m[2]), m, H.rot2(ang), sc.scales[0, :2].astype(np.float64),
                                   float(sc.opacity[0]))
            want = [a * float(sc.rgb[0, ch]) + (1 - a) * bg[ch] for ch in range(3)] + [a]
            for k in range(3):
                assert np.allclose(out["views"][k, y, x], want, atol=1e-12)
