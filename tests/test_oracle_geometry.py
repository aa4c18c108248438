"""Pins for the oracle's display geometry (Sec. 4.2 Eqs. (1)-(2), Sec. 4.3
Eq. (u_prime), Eq. (gs_prefilter_fix)) against geometry and closed forms."""
import math

import numpy as np
import pytest

from paper_2508_18540_gb300 import synth as S
from tests import helpers as H


def _ref(orc, D_f=3.0, baseline=0.1, N=128, fov=50.0, **kw):
    return orc.make_ref(S.identity_camera(N, fov), S.display_for(D_f, baseline, **kw))


def test_forward_shift_is_where_outermost_edge_ray_crosses_axis(orc):
    # The right-most view's left frustum edge (through the focal-plane edge)
    # must cross the optical axis at D_forward: there the reference camera
    # exactly covers the display's visible volume (Sec. 4.2, Fig. 3 centre).
    for D_f, b, fov in [(3.0, 0.1, 50.0), (2.6087, 0.15, 50.0), (5.0, 0.6, 30.0)]:
        r = _ref(orc, D_f, b, fov=fov)
        th = math.radians(fov)
        o = np.array([b, 0.0])                      # camera at +baseline
        F = np.array([-D_f * math.tan(th / 2), D_f])  # left focal-plane edge
        t = -o[0] / (F[0] - o[0])
        z_cross = o[1] + t * (F[1] - o[1])
        assert r.D_forward0 == pytest.approx(z_cross, rel=1e-13)
        assert r.D_forward == r.D_forward0
        # the reference frustum's edge passes through the same focal-plane edge
        assert math.atan2(abs(F[0]), D_f - r.D_forward0) == pytest.approx(r.theta_px / 2, rel=1e-13)


def test_reference_fov_identity(orc):
    # With D_shift = 0: tan(theta'/2) = tan(phi/2) + tan(theta/2) (derived from Eqs. (1)-(2)).
    for D_f, b in [(3.0, 0.1), (1.0, 0.4), (7.0, 0.05)]:
        r = _ref(orc, D_f, b)
        assert r.tthp_x == pytest.approx(r.tphi_x + r.tth_x, rel=1e-13)


def test_backward_shift_widens_the_covered_region(orc):
    # Sec. 4.2: moving the reference camera back by D_shift widens the region
    # it covers. The reading that achieves this keeps theta' (from the
    # unshifted D_forward) and moves only the camera: then the frustum's
    # half-width (z - D_forward) tan(theta'/2) grows by D_shift tan(theta'/2)
    # at every depth, the focal plane included. Recomputing theta' from the
    # shifted camera would leave the focal-plane width unchanged instead.
    for D_f, b, shift in [(3.0, 0.1, 0.1), (2.6087, 0.15, 0.25), (5.0, 0.6, 1.0)]:
        r0 = _ref(orc, D_f, b)
        r1 = _ref(orc, D_f, b, D_shift=shift)
        assert r1.D_forward == pytest.approx(r0.D_forward - shift, rel=1e-14)
        assert r1.tthp_x == r0.tthp_x and r1.theta_px == r0.theta_px
        for z in (0.5 * D_f, D_f, 2.0 * D_f):
            w0 = (z - r0.D_forward) * r0.tthp_x
            w1 = (z - r1.D_forward) * r1.tthp_x
            assert w1 - w0 == pytest.approx(shift * r0.tthp_x, rel=1e-12)
        # unshifted, the reference frustum meets the base frustum at the focal plane
        assert (D_f - r0.D_forward) * r0.tthp_x == pytest.approx(D_f * r0.tth_x, rel=1e-12)


def test_adaptive_dilation(orc):
    # Eq. (gs_prefilter_fix): f' = f P_s^2 when D_shift = 0, and
    # f' = f (P_s (D_f - D_fwd0) / (D_f - D_fwd))^2 after a backward shift.
    for P_s in (1, 2, 3):
        r = _ref(orc, P_s=P_s)
        assert r.f_prime == pytest.approx(0.3 * P_s * P_s, rel=1e-13)
        r2 = _ref(orc, P_s=P_s, D_shift=0.4)
        expect = 0.3 * (P_s * (3.0 - r2.D_forward0) / (3.0 - r2.D_forward)) ** 2
        assert r2.f_prime == pytest.approx(expect, rel=1e-12)
        assert r2.f_prime < r.f_prime
        assert r2.W == 128 * P_s and r2.H == 128 * P_s


def test_view_offsets(orc):
    r = _ref(orc, 2.6087, 0.15)
    dx, dy = orc.view_offsets(r, 45, 1)
    assert dx[0] == pytest.approx(-0.15, rel=1e-13) and dx[-1] == pytest.approx(0.15, rel=1e-13)
    assert np.allclose(np.diff(dx), 0.3 / 44, rtol=1e-12)
    assert np.all(dy == 0.0)
    dx1, _ = orc.view_offsets(r, 1, 1)
    assert dx1[0] == 0.0
    # a vertical row of views with its own viewing angle: the outermost
    # vertical offsets equal the vertical baseline (tan(phi_y/2) = b_y / D_f)
    b_y = 0.05
    disp = S.display_for(2.6087, 0.15, phi_y=2.0 * math.atan(b_y / 2.6087))
    r2 = orc.make_ref(S.identity_camera(128, 50.0), disp)
    dx2, dy2 = orc.view_offsets(r2, 5, 3)
    assert dy2[0] == pytest.approx(-b_y, rel=1e-13) and dy2[-1] == pytest.approx(b_y, rel=1e-13)
    assert dy2[1] == 0.0
    assert dx2[0] == pytest.approx(-0.15, rel=1e-13)


def test_u_prime_matches_ray_geometry(orc):
    # Eq. (u_prime) against explicit ray construction: the view camera at
    # (Delta x, 0, 0) shoots a ray through the shared focal-plane window; it
    # meets the plane z = d, which the reference camera projects to u'.
    rng = np.random.default_rng(0)
    for D_shift in (0.0, 0.3):
        cam = S.identity_camera(64, 50.0)
        disp = S.display_for(3.0, 0.2, D_shift=D_shift)
        r = orc.make_ref(cam, disp)
        for _ in range(200):
            dx = rng.uniform(-0.2, 0.2)
            d = rng.uniform(r.D_forward + 0.3, 12.0)
            u = rng.uniform(-1, 1)
            o, dirv = H.base_view_ray(disp, cam, dx, 0.0, u, 0.0)
            P = H.hit_plane_z(o, dirv, d)
            u_geo = P[0] / ((d - r.D_forward) * r.tthp_x)
            assert orc.plane_coord(r, 0, dx, d, u) == pytest.approx(u_geo, rel=1e-11, abs=1e-12)
            v = rng.uniform(-1, 1)
            dy = rng.uniform(-0.1, 0.1)
            o, dirv = H.base_view_ray(disp, cam, 0.0, dy, 0.0, v)
            P = H.hit_plane_z(o, dirv, d)
            v_geo = P[1] / ((d - r.D_forward) * r.tthp_y)
            assert orc.plane_coord(r, 1, dy, d, v) == pytest.approx(v_geo, rel=1e-11, abs=1e-12)


def test_outermost_view_edges_map_to_plane_edges(orc):
    # s = +-1/2, u = -+1 -> u' = -+1 for every plane distance (the reference
    # camera covers the display volume exactly when D_shift = 0).
    r = _ref(orc, 2.6087, 0.15, N=512)
    dx, _ = orc.view_offsets(r, 45, 1)
    for d in np.linspace(r.D_forward + 0.05, 50.0, 37):
        assert orc.plane_coord(r, 0, dx[-1], d, -1.0) == pytest.approx(-1.0, abs=1e-12)
        assert orc.plane_coord(r, 0, dx[0], d, 1.0) == pytest.approx(1.0, abs=1e-12)


def test_focal_plane_has_no_parallax(orc):
    # At d = D_focal every view maps u' = u (zero parallax plane).
    r = _ref(orc, 2.6087, 0.15, N=512)
    dx, _ = orc.view_offsets(r, 45, 1)
    for j in (0, 7, 22, 44):
        for u in np.linspace(-1, 1, 9):
            assert orc.plane_coord(r, 0, dx[j], 2.6087, u) == pytest.approx(u, abs=1e-13)


def test_fp32_decision_form_tracks_fp64_map(orc):
    # The FP32 coefficients reproduce X = ((u'+1)W-1)/2 of Eq. (u_prime)
    # to well under 1e-4 plane pixels; nearest indices agree with
    # floor(X + 1/2) except at (FP-exact) ties.
    rng = np.random.default_rng(1)
    for P_s, D_shift in ((1, 0.0), (2, 0.0), (3, 0.2)):
        cam = S.identity_camera(512, 50.0)
        disp = S.display_for(2.6087, 0.15, P_s=P_s, D_shift=D_shift)
        r = orc.make_ref(cam, disp)
        dx, _ = orc.view_offsets(r, 45, 1)
        worst = 0.0
        for _ in range(60):
            j = int(rng.integers(45))
            d = float(rng.uniform(r.D_forward + 0.4, 11.0))
            gm, hn, hb = orc.axis_coeffs(r, 0, dx[j], d)
            for x in rng.integers(0, 512, 16):
                X = orc.plane_pixel(r, 0, dx[j], d, int(x))
                Xf = P_s * int(x) + float(np.float32(np.float32(gm) * np.float32(x) + np.float32(hb)))
                worst = max(worst, abs(Xf - X))
                frac = (X + 0.5) - math.floor(X + 0.5)
                if 1e-4 < frac < 1 - 1e-4:
                    assert orc.nearest_index(r, float(gm), float(hn), int(x)) == math.floor(X + 0.5)
        assert worst < 1e-4
