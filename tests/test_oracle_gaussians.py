"""Pins for the oracle's Gaussian projection, footprint and rasterisation
(Sec. 4.4; EWA splatting of [kerbl20233d] with the dilation of
Eq. (gs_prefilter_fix))."""
import math

import numpy as np
import pytest

from paper_2508_18540_gb300 import synth as S
from tests import helpers as H


def _rand_scene(n, seed, rot=True):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1.5, 6, n)], 1)
    scales = np.exp(rng.normal(math.log(0.05), 0.6, (n, 3)))
    q = rng.normal(size=(n, 4)) if rot else np.tile([1.0, 0, 0, 0], (n, 1))
    f = np.float32
    return S.GaussianScene(means.astype(f), scales.astype(f), q.astype(f), rng.uniform(0.1, 0.9, n).astype(f),
                           rng.uniform(0, 1, (n, 3)).astype(f))


def _rotated_camera(N=96):
    # a camera rotated about y and x, translated
    a, b = 0.3, -0.2
    Ry = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    cam = S.identity_camera(N, 50.0, t=(0.2, -0.1, 0.5))
    cam.R = Rx @ Ry
    return cam


def test_ewa_covariance_matches_numeric_jacobian(orc):
    # Sigma_2 = J W Sigma_3 W^T J^T + f' I with J the Jacobian of the
    # perspective projection (taken here by central differences) and
    # Sigma_3 built from quaternion products.
    cam = _rotated_camera()
    disp = S.display_for(3.0, 0.1, D_shift=0.1)
    r = orc.make_ref(cam, disp)
    sc = _rand_scene(40, 3)
    mean2d, conic, cov2d = orc.gauss_values(r, sc)
    R = np.asarray(cam.R)
    t = np.asarray(cam.t)

    def proj(pc):
        return np.array([r.fx * pc[0] / pc[2] + r.cx, r.fy * pc[1] / pc[2] + r.cy])

    for g in range(sc.n):
        pc = R @ sc.means[g].astype(np.float64) + t - np.array([0, 0, r.D_forward])
        if pc[2] < 0.3:
            continue
        J = np.zeros((2, 3))
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            J[:, a] = (proj(pc + e) - proj(pc - e)) / (2 * h)
        S3 = H.sigma3_from_quat(sc.quats[g], sc.scales[g])
        S2 = J @ R @ S3 @ R.T @ J.T + r.f_prime * np.eye(2)
        got = np.array([[cov2d[g, 0], cov2d[g, 1]], [cov2d[g, 1], cov2d[g, 2]]])
        assert np.allclose(got, S2, rtol=1e-6, atol=1e-9)
        assert np.allclose(mean2d[g], proj(pc), rtol=1e-12, atol=1e-9)
        C = np.linalg.inv(got)
        assert np.allclose(conic[g], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-10)


def test_flat_gaussian_projection_is_exact(orc):
    # A flat fronto-parallel Gaussian maps affinely under perspective; with
    # f = 0 its plane texels are its world-plane density at the ray hit point.
    cam = S.identity_camera(64, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    r = orc.make_ref(cam, disp)
    sc = H.flat_scene([((0.1, -0.05, 3.5), (0.08, 0.03), 0.7, 0.8, (1, 1, 1))])
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile",
                     with_views=False)
    A = out["planes"][0, :, :, 3]
    x0, y0, x1, y1 = out["rect"][0]
    assert out["valid"][0] == 1
    m = sc.means[0].astype(np.float64)
    s = sc.scales[0, :2].astype(np.float64)               # the stored FP32 inputs
    q = sc.quats[0].astype(np.float64)
    ang = 2 * math.atan2(q[3], q[0])
    for y in range(r.H):
        for x in range(r.W):
            if x0 <= x <= x1 and y0 <= y <= y1:
                o, d = H.ref_pixel_ray(r, x, y)
                P = H.hit_plane_z(o, d, m[2])
                a = H.flat_gauss_alpha(P, m, H.rot2(ang), s, float(sc.opacity[0]))
                assert A[y, x] == pytest.approx(a, abs=1e-12)
            else:
                assert A[y, x] == 0.0


def test_opacity_is_clamped_at_099(orc):
    # alpha = min(0.99, o exp(-q/2)): a nearly opaque, wide flat Gaussian
    # (o = 0.9995, sigma 2 x 1.5 at depth 3) gives exactly 0.99 wherever
    # o exp(-q/2) exceeds it and the closed-form value elsewhere.
    cam = S.identity_camera(32, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    sc = H.flat_scene([((0.0, 0.0, 3.0), (2.0, 1.5), 0.3, 0.9995, (1, 1, 1))])
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile",
                     with_views=False)
    r = out["ref"]
    A = out["planes"][0, :, :, 3]
    x0, y0, x1, y1 = out["rect"][0]
    m = sc.means[0].astype(np.float64)
    s = sc.scales[0, :2].astype(np.float64)
    q = sc.quats[0].astype(np.float64)
    ang = 2 * math.atan2(q[3], q[0])
    o32 = float(sc.opacity[0])
    clamped = free = 0
    for y in range(y0, y1 + 1):
        for x in range(x0, x1 + 1):
            o, d = H.ref_pixel_ray(r, x, y)
            P = H.hit_plane_z(o, d, m[2])
            Sxy = H.rot2(ang) @ np.diag(s ** 2) @ H.rot2(ang).T
            dd = P[:2] - m[:2]
            raw = o32 * math.exp(-0.5 * dd @ np.linalg.solve(Sxy, dd))
            if raw > 0.99 + 1e-9:
                assert A[y, x] == 0.99
                clamped += 1
            elif raw < 0.99 - 1e-9:
                assert A[y, x] == pytest.approx(raw, abs=1e-12)
                free += 1
    assert clamped > 3 and free > 20


def test_footprint_contains_three_sigma_ellipse(orc):
    # Every plane pixel inside the 3-sigma ellipse of the projected Gaussian
    # (q <= 9) lies inside the FP32 footprint rectangle.
    cam = _rotated_camera(80)
    disp = S.display_for(3.0, 0.1)
    r = orc.make_ref(cam, disp)
    sc = _rand_scene(300, 5)
    z, valid, rect = orc.gauss_decide(r, sc)
    mean2d, conic, _ = orc.gauss_values(r, sc)
    ys, xs = np.mgrid[0:r.H, 0:r.W]
    checked = 0
    for g in range(sc.n):
        dx = xs - mean2d[g, 0]
        dy = ys - mean2d[g, 1]
        q = conic[g, 0] * dx * dx + 2 * conic[g, 1] * dx * dy + conic[g, 2] * dy * dy
        inside = q <= 9.0 * (1 - 1e-5)
        if not valid[g]:
            if z[g] > disp.z_near:
                assert not inside.any()
            continue
        x0, y0, x1, y1 = rect[g]
        inrect = (xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1)
        assert not (inside & ~inrect).any()
        checked += 1
    assert checked > 100


def test_fp32_footprint_agrees_with_fp64(orc):
    # The FP32 decision path equals the same rectangle computed in FP64
    # except for rare half-pixel ties, where it differs by one pixel.
    cam = S.identity_camera(256, 50.0)
    disp = S.display_for(2.6, 0.15)
    r = orc.make_ref(cam, disp)
    sc = _rand_scene(3000, 6)
    z, valid, rect = orc.gauss_decide(r, sc)
    mean2d, conic, cov2d = orc.gauss_values(r, sc)
    diffs = 0
    n_ok = 0
    for g in np.nonzero(valid)[0]:
        a, b, c = cov2d[g]
        det = a * c - b * b
        mid = 0.5 * (a + c)
        lam = mid + math.sqrt(max(mid * mid - det, 0.0))
        rad = math.ceil(3 * math.sqrt(lam))
        px, py = mean2d[g]
        ref = [max(0, math.ceil(px - rad)), max(0, math.ceil(py - rad)),
               min(r.W - 1, math.floor(px + rad)), min(r.H - 1, math.floor(py + rad))]
        d = np.abs(np.asarray(ref) - rect[g])
        assert d.max() <= 1
        diffs += int(d.max() > 0)
        n_ok += 1
    assert n_ok > 1000
    assert diffs <= 0.01 * n_ok


def test_culling(orc):
    cam = S.identity_camera(64, 50.0)
    disp = S.display_for(3.0, 0.1)
    r = orc.make_ref(cam, disp)
    sc = _rand_scene(6, 7)
    sc.means[0] = [0.0, 0.0, 0.1]       # behind the near plane (after D_forward)
    sc.means[1] = [50.0, 0.0, 3.0]      # far outside the frustum
    sc.means[2] = [0.0, 0.0, 3.0]       # centre
    sc.means[3] = [0.0, 0.0, -2.0]      # behind the camera
    # in front of the reference camera but nearer than z_near (0.2): culled;
    # just past z_near: kept
    sc.means[4] = [0.0, 0.0, r.D_forward + 0.15]
    sc.means[5] = [0.0, 0.0, r.D_forward + 0.25]
    sc.scales[4:6] = 0.001
    z, valid, rect = orc.gauss_decide(r, sc)
    assert valid.tolist() == [0, 0, 1, 0, 0, 1]
    assert z[2] == pytest.approx(3.0 - r.D_forward, rel=1e-15)
    assert 0.0 < z[4] < disp.z_near < z[5]


def test_degenerate_projection_is_culled(orc):
    # without the dilation (f = 0) a Gaussian whose projected covariance is
    # singular (all scales 0, or a flat Gaussian seen exactly edge-on) has
    # det(Sigma_2) = 0 and is culled; the same Gaussians with f > 0 are kept
    cam = S.identity_camera(32, 50.0)
    sc = _rand_scene(3, 12)
    sc.means[:] = [[0.0, 0.0, 3.0], [0.2, 0.1, 3.5], [-0.2, 0.0, 4.0]]
    sc.scales[0] = 0.0
    sc.scales[1] = [0.2, 0.0, 0.0]                    # a line segment: rank-1 covariance
    sc.quats[:] = [1.0, 0.0, 0.0, 0.0]
    sc.scales[2] = [0.1, 0.1, 0.05]                   # regular
    for f_aa, want in ((0.0, [0, 0, 1]), (0.3, [1, 1, 1])):
        r = orc.make_ref(cam, S.display_for(3.0, 0.1, f_aa=f_aa))
        z, valid, rect = orc.gauss_decide(r, sc)
        assert valid.tolist() == want, f_aa


def test_non_finite_geometry_is_culled(orc):
    # host-side fault injection: a Gaussian whose position, scale or
    # rotation is NaN, or whose scale is infinite, fails the culling tests
    # (every comparison with NaN is false) and never reaches a plane; the
    # rest of the scene renders as without it
    w = S.workload_tiny(seed=3)
    sc = w.scene.subset(np.arange(500))
    bad = sc.subset(np.arange(500))
    bad.means[0, 0] = np.nan
    bad.means[1, 2] = np.nan
    bad.scales[2, 1] = np.nan
    bad.quats[3, :] = np.nan
    bad.scales[4] = np.inf
    args = dict(camera=w.camera, display=w.display, views=w.views, N=w.N, binning=w.binning)
    out = orc.render(scene=bad, **args)
    assert out["valid"][:5].tolist() == [0] * 5
    assert np.isfinite(out["planes"]).all() and np.isfinite(out["views"]).all()
    ref = orc.render(scene=sc.subset(np.arange(5, 500)), **args)
    assert out["M"] == ref["M"]
    assert np.allclose(out["views"], ref["views"], atol=1e-12)


def test_depth_order_and_ties(orc):
    # Front-to-back within a chunk: the nearer opaque Gaussian dominates;
    # equal depths are ordered by index.
    cam = S.identity_camera(32, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    r = orc.make_ref(cam, disp)
    sc = H.flat_scene([((0, 0, 3.0), (0.3, 0.3), 0.0, 0.9, (1, 0, 0)),
                       ((0, 0, 3.0), (0.3, 0.3), 0.0, 0.9, (0, 1, 0)),
                       ((0, 0, 2.5), (0.3, 0.3), 0.0, 0.9, (0, 0, 1))])
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile",
                     with_views=False)
    assert out["order"].tolist() == [2, 0, 1]
    c = out["planes"][0, r.H // 2, r.W // 2]
    # blue (nearest) first, then red before green (equal depth, lower index)
    assert c[2] > 0.85 and c[2] > c[0] > c[1] > 0.0
    a_r = c[0] / (1 - c[2])
    assert c[1] == pytest.approx((1 - c[2]) * (1 - a_r) * a_r, rel=1e-9)


def test_chunk_invariance_is_plain_alpha_blending(orc):
    # No parallax between planes (phi = 0): compositing the chunked planes of
    # any N gives the plain depth-sorted alpha blending of all primitives,
    # i.e. the single-chunk plane (Eq. (alpha_blend) is associative).
    cam = S.identity_camera(48, 50.0)
    disp = S.Display(D_focal=3.0, phi_x=0.0)
    sc = _rand_scene(400, 8)
    one = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile")
    # independent front-to-back blend from the oracle's per-primitive values
    r = one["ref"]
    ys, xs = np.mgrid[0:r.H, 0:r.W]
    C = np.zeros((r.H, r.W, 3))
    T = np.ones((r.H, r.W))
    for g in one["order"]:
        x0, y0, x1, y1 = one["rect"][g]
        m = one["mean2d"][g]
        a, b, c = one["conic"][g]
        dx, dy = xs - m[0], ys - m[1]
        al = np.minimum(0.99, sc.opacity[g] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
        al = np.where((xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1), al, 0.0)
        C += (T * al)[..., None] * sc.rgb[g]
        T *= 1 - al
    assert np.allclose(one["planes"][0, ..., :3], C, atol=1e-12)
    assert np.allclose(one["planes"][0, ..., 3], 1 - T, atol=1e-12)
    assert np.allclose(one["views"][0], one["planes"][0], atol=1e-12)
    for N in (2, 7, 16, 64):
        for mode in ("quantile", "disparity"):
            many = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=N, binning=mode)
            assert np.allclose(many["views"], one["views"], atol=1e-12), (N, mode)


def test_chunk_invariance_with_shifted_reference(orc):
    # D_shift = D_forward0 puts the reference camera at the base camera:
    # every plane maps the centre view identically, so the centre view is
    # independent of N even with a viewing angle.
    cam = S.identity_camera(48, 50.0)
    d0 = orc.make_ref(cam, S.display_for(3.0, 0.1)).D_forward0
    disp = S.display_for(3.0, 0.1, D_shift=d0)
    sc = _rand_scene(400, 9)
    base = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile")
    for N in (3, 16):
        many = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=N, binning="quantile")
        assert np.allclose(many["views"], base["views"], atol=1e-12)


# ---- 3DGS-compatible blending (alpha < 1/255 skipped, stop before T < 1e-4)

def test_3dgs_blend_single_gaussian_alpha_cutoff(orc):
    # One flat Gaussian (f = 0, exact projection): the texel keeps the
    # closed-form opacity where it is at least 1/255 and is empty where it is
    # below; the near-threshold mask marks exactly the texels within 1e-6 of
    # the cut.
    cam = S.identity_camera(64, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    sc = H.flat_scene([((0.1, -0.05, 3.5), (0.08, 0.03), 0.7, 0.8, (1, 1, 1))])
    out = orc.render(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile",
                     with_views=False, blend="3dgs")
    r = out["ref"]
    A = out["planes"][0, :, :, 3]
    near = out["near"][0]
    x0, y0, x1, y1 = out["rect"][0]
    m = sc.means[0].astype(np.float64)
    s = sc.scales[0, :2].astype(np.float64)
    q = sc.quats[0].astype(np.float64)
    ang = 2 * math.atan2(q[3], q[0])
    kept = cut = 0
    for y in range(r.H):
        for x in range(r.W):
            if not (x0 <= x <= x1 and y0 <= y <= y1):
                assert A[y, x] == 0.0 and near[y, x] == 0
                continue
            o, d = H.ref_pixel_ray(r, x, y)
            a = H.flat_gauss_alpha(H.hit_plane_z(o, d, m[2]), m, H.rot2(ang), s, float(sc.opacity[0]))
            gap = abs(a - 1.0 / 255.0)
            if abs(gap - 1e-6) > 1e-9:
                assert near[y, x] == (1 if gap <= 1e-6 else 0)
            if near[y, x]:
                continue
            if a >= 1.0 / 255.0:
                assert A[y, x] == pytest.approx(a, abs=1e-12)
                kept += 1
            else:
                assert A[y, x] == 0.0
                cut += 1
    assert kept > 20 and cut > 20


def test_3dgs_near_mask_marks_both_threshold_events(orc):
    # The near-threshold mask flags a texel whose trace passes within 1e-6 of
    # a cut-off. Opacities are set from the closed form so that, at the
    # centre pixel, (a) a lone flat Gaussian's alpha is 1/255 + 5e-7, and (b)
    # two wide layers leave T (1 - alpha) = 1e-4 + 5e-7 (0.99, then the
    # second layer's exact complement): both texels are flagged, and both
    # are still blended (neither value crosses its cut-off).
    cam = S.identity_camera(16, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    args = dict(camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile", with_views=False)
    r = orc.make_ref(cam, disp)
    yc, xc = r.H // 2, r.W // 2
    o_, d_ = H.ref_pixel_ray(r, xc, yc)

    def unit_alpha(mean, sig):
        # exp(-q/2) of an axis-aligned flat Gaussian at the centre pixel's ray hit (no clamp)
        m = np.asarray(mean, np.float64)
        dd = H.hit_plane_z(o_, d_, m[2])[:2] - m[:2]
        return math.exp(-0.5 * float(np.sum((dd / np.asarray(sig, np.float64)) ** 2)))

    # (a) alpha event
    mean, sig = (0.05, 0.02, 3.0), (0.3, 0.25)
    o_a = (1.0 / 255.0 + 5e-7) / unit_alpha(mean, sig)
    sc = H.flat_scene([(mean, sig, 0.0, o_a, (1, 1, 1))])
    sc.opacity[0] = np.float32(o_a)
    out = orc.render(scene=sc, blend="3dgs", **args)
    a_pix = float(sc.opacity[0]) * unit_alpha(sc.means[0], sc.scales[0, :2])      # the stored FP32 inputs
    assert abs(a_pix - 1.0 / 255.0) < 1e-6 and a_pix >= 1.0 / 255.0
    assert out["near"][0, yc, xc] == 1
    assert out["planes"][0, yc, xc, 3] == pytest.approx(a_pix, abs=1e-12)
    # (b) transmittance event: the front layer is clamped to 0.99
    m1, m2, big = (0.0, 0.0, 2.5), (0.0, 0.0, 3.0), (3.0, 3.0)
    a2 = 1.0 - (1e-4 + 5e-7) / 0.01
    o_b = a2 / unit_alpha(m2, big)
    sc = H.flat_scene([(m1, big, 0.0, 0.9999, (1, 0, 0)), (m2, big, 0.0, o_b, (0, 1, 0))])
    out = orc.render(scene=sc, blend="3dgs", **args)
    a2_pix = float(sc.opacity[1]) * unit_alpha(sc.means[1], sc.scales[1, :2])
    t_after = 0.01 * (1.0 - a2_pix)
    assert abs(t_after - 1e-4) < 1e-6 and t_after >= 1e-4
    assert out["near"][0, yc, xc] == 1
    assert out["planes"][0, yc, xc, 3] == pytest.approx(1.0 - t_after, abs=1e-12)


def _layer_scene(n_layers, seed):
    # wide flat fronto-parallel layers on the optical axis, front to back at
    # z = 2, 2.25, ...; opacity 0.8 except a faint last layer (0.3), which a
    # pixel that has stopped must not blend even though its own factor
    # (1 - alpha) would keep T above 1e-4; distinct colours
    rng = np.random.default_rng(seed)
    return H.flat_scene([((0.0, 0.0, 2.0 + 0.25 * i), (2.0, 2.0), 0.0, 0.3 if i == n_layers - 1 else 0.8,
                          tuple(rng.uniform(0.1, 1.0, 3))) for i in range(n_layers)])


def test_3dgs_blend_stops_before_transmittance_cutoff(orc):
    # Six layers of opacity about 0.8 and a faint seventh: a pixel's
    # transmittance after m of them is the product of (1 - alpha_j), taken
    # here from each layer's closed-form opacity. In 3DGS mode a pixel blends
    # exactly the first m layers, m the count before the first layer that
    # would take the product below 1e-4 (5 near the centre: 3.2e-4, then
    # 6.4e-5), and nothing after it, i.e. it equals the exact render of a
    # scene holding only those m layers.
    cam = S.identity_camera(16, 50.0)
    disp = S.display_for(3.0, 0.1, f_aa=0.0)
    n_layers = 7
    sc = _layer_scene(n_layers, 1)
    args = dict(camera=cam, display=disp, views=S.ViewSet(1), N=1, binning="quantile", with_views=False)
    g3 = orc.render(scene=sc, blend="3dgs", **args)
    r = g3["ref"]
    prefix = {m: orc.render(scene=sc.subset(np.arange(m)), **args)["planes"][0] for m in range(1, n_layers + 1)}
    seen = set()
    for y in range(r.H):
        for x in range(r.W):
            o, d = H.ref_pixel_ray(r, x, y)
            T, m = 1.0, 0
            for j in range(n_layers):
                mj = sc.means[j].astype(np.float64)
                a = H.flat_gauss_alpha(H.hit_plane_z(o, d, mj[2]), mj, H.rot2(0.0),
                                       sc.scales[j, :2].astype(np.float64), float(sc.opacity[j]))
                assert a > 0.05                     # no alpha cut in this scene
                if T * (1 - a) < 1e-4:
                    break
                T *= 1 - a
                m += 1
            if g3["near"][0, y, x]:
                continue
            assert np.allclose(g3["planes"][0, y, x], prefix[m][y, x], atol=1e-12), (x, y, m)
            seen.add(m)
    assert {5, 6} <= seen                              # stops after five and after six layers


def test_3dgs_blend_stop_is_per_plane(orc):
    # The transmittance that decides the stop is the plane's own: split over
    # two chunks (4 + 3 layers) neither plane gets near 1e-4, so 3DGS mode
    # gives the exact planes bit for bit, and their composite differs from
    # the single-plane 3DGS render (which stopped).
    cam = S.identity_camera(16, 50.0)
    disp = S.Display(D_focal=3.0, phi_x=0.0)
    sc = _layer_scene(7, 2)
    args = dict(camera=cam, display=disp, views=S.ViewSet(1), binning="quantile")
    exact2 = orc.render(scene=sc, N=2, **args)
    g3_2 = orc.render(scene=sc, N=2, blend="3dgs", **args)
    assert np.array_equal(g3_2["planes"], exact2["planes"]) and not g3_2["near"].any()
    g3_1 = orc.render(scene=sc, N=1, blend="3dgs", **args)
    assert np.abs(g3_1["views"] - g3_2["views"]).max() > 1e-5


def test_3dgs_blend_only_removes_occlusion(orc):
    # Skipping a member or stopping early only drops factors (1 - alpha) from
    # a texel's transmittance: A in 3DGS mode never exceeds the exact A, and
    # the transmittance never goes below 1e-4.
    cam = S.identity_camera(64, 50.0)
    disp = S.display_for(3.0, 0.1)
    sc = _rand_scene(3000, 11)
    sc.opacity[:] = 0.5 + 0.49 * sc.opacity
    args = dict(scene=sc, camera=cam, display=disp, views=S.ViewSet(1), N=2, binning="quantile",
                with_views=False)
    ex = orc.render(**args)["planes"]
    g3 = orc.render(blend="3dgs", **args)["planes"]
    assert (g3[..., 3] <= ex[..., 3] + 1e-12).all()
    assert g3[..., 3].max() <= 1 - 1e-4 + 1e-15
    assert (np.abs(g3 - ex).max(axis=-1) > 1e-6).mean() > 0.01      # the cut-offs change many texels
    with pytest.raises(ValueError):
        orc.render(blend="bogus", **args)
