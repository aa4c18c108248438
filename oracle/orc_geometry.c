/*
 * orc_geometry.c -- oracle: display set-up and the quilt-to-plane map.
 * TEST INFRASTRUCTURE ONLY (see lf_oracle.h).
 *
 * Sec. 4.2 Eqs. (1)-(2), the D_shift update, Eq. (gs_prefilter_fix);
 * Sec. 4.3 s_j, Delta x_j, Eq. (u_prime).
 */
#include "lf_oracle.h"

#include <math.h>
#include <string.h>

int orc_make_ref(const orc_camera* cam, const orc_display* disp, orc_ref* r)
{
    memset(r, 0, sizeof(*r));
    r->cam = *cam;
    r->disp = *disp;
    if (cam->Nx <= 0 || cam->Ny <= 0 || disp->P_s <= 0) return -1;
    if (!(disp->D_focal > 0.0) || !(disp->z_near > 0.0)) return -1;
    if (!(cam->theta_x > 0.0 && cam->theta_x < M_PI)) return -1;
    if (!(cam->theta_y > 0.0 && cam->theta_y < M_PI)) return -1;
    if (disp->phi_x < 0.0 || disp->phi_y < 0.0) return -1;

    const double Df = disp->D_focal;
    r->tth_x = tan(0.5 * cam->theta_x);
    r->tth_y = tan(0.5 * cam->theta_y);
    r->tphi_x = tan(0.5 * disp->phi_x);
    r->tphi_y = tan(0.5 * disp->phi_y);

    /* Eq. (1): D_forward = max_k D_focal tan(phi_k/2) / (tan(phi_k/2) + tan(theta_k/2)).
     * An axis with no viewing angle needs no forward shift (term 0). */
    double fwd_x = 0.0, fwd_y = 0.0;
    if (r->tphi_x > 0.0) fwd_x = Df * r->tphi_x / (r->tphi_x + r->tth_x);
    if (r->tphi_y > 0.0) fwd_y = Df * r->tphi_y / (r->tphi_y + r->tth_y);
    r->D_forward0 = fwd_x > fwd_y ? fwd_x : fwd_y;

    /* Eq. (2): theta'_k = 2 atan(D_focal tan(theta_k/2) / (D_focal - D_forward)).
     * Reading: theta' uses D_forward before the near-field shift, so that the
     * shift widens the covered region (Sec. 4.2, last paragraph). */
    r->tthp_x = Df * r->tth_x / (Df - r->D_forward0);
    r->tthp_y = Df * r->tth_y / (Df - r->D_forward0);
    r->theta_px = 2.0 * atan(r->tthp_x);
    r->theta_py = 2.0 * atan(r->tthp_y);

    /* Near-field shift: D_forward <- D_forward - D_shift. */
    r->D_forward = r->D_forward0 - disp->D_shift;
    if (!(r->D_forward < Df)) return -1;

    /* Planes are P_s Ny x P_s Nx (Sec. 4.2). */
    r->W = cam->Nx * disp->P_s;
    r->H = cam->Ny * disp->P_s;
    r->fx = (double)r->W / (2.0 * r->tthp_x);
    r->fy = (double)r->H / (2.0 * r->tthp_y);
    r->cx = 0.5 * (double)(r->W - 1);
    r->cy = 0.5 * (double)(r->H - 1);

    /* Eq. (gs_prefilter_fix): f' = f (D_focal tan(theta_x/2) /
     * ((D_focal - D_forward) tan(theta'_x/2)) P_s)^2, with the shifted D_forward. */
    const double ratio = Df * r->tth_x / ((Df - r->D_forward) * r->tthp_x) * (double)disp->P_s;
    r->f_prime = disp->f_aa * ratio * ratio;
    return 0;
}

/* Sec. 4.3: s_j = (j-1)/(V-1) - 1/2 for 1-based j; Delta x_j = 2 D_focal s_j tan(phi_x/2).
 * Reading: s = 0 when V = 1 (the formula is 0/0 there). */
static double view_s(int32_t j, int32_t V)
{
    if (V <= 1) return 0.0;
    return (double)j / (double)(V - 1) - 0.5;
}

void orc_view_offsets(const orc_ref* r, int32_t Vx, int32_t Vy, double* dx, double* dy)
{
    const double Df = r->disp.D_focal;
    for (int32_t j = 0; j < Vx; ++j) dx[j] = 2.0 * Df * view_s(j, Vx) * r->tphi_x;
    for (int32_t i = 0; i < Vy; ++i) dy[i] = 2.0 * Df * view_s(i, Vy) * r->tphi_y;
}

/* Eq. (u_prime):
 *   u' = (Delta x_j (D_focal - d_k)/D_focal + d_k tan(theta_x/2) u)
 *        / ((d_k - D_forward) tan(theta'_x/2));
 * the vertical coordinate is the same with Delta y_i, theta_y, theta'_y. */
double orc_plane_coord(const orc_ref* r, int32_t axis, double delta, double d_k, double u)
{
    const double Df = r->disp.D_focal;
    const double tth = axis ? r->tth_y : r->tth_x;
    const double tthp = axis ? r->tthp_y : r->tthp_x;
    return (delta * (Df - d_k) / Df + d_k * tth * u) / ((d_k - r->D_forward) * tthp);
}

double orc_plane_pixel(const orc_ref* r, int32_t axis, double delta, double d_k, int32_t x)
{
    const int32_t n = axis ? r->cam.Ny : r->cam.Nx;
    const int32_t Wp = axis ? r->H : r->W;
    const double u = (2.0 * (double)x + 1.0) / (double)n - 1.0;
    const double up = orc_plane_coord(r, axis, delta, d_k, u);
    return ((up + 1.0) * (double)Wp - 1.0) / 2.0;
}

/* FP32 decision form of Eq. (u_prime). Substituting u = (2x+1)/n - 1 into
 * Eq. (u_prime) and X = ((u'+1) W - 1)/2 gives X = g x + h with
 *   den = (d_k - D_forward) tan(theta'/2),  a = d_k tan(theta/2),
 *   g   = W a / (n den),
 *   h   = (W/2) ((Delta (D_focal - d_k)/D_focal + a (1 - n)/n) / den + 1) - 1/2.
 * The integer part P_s x is split off so that the FP32 remainder stays small:
 *   gm = g - P_s,  hn = h + 1/2 (nearest),  hb = h (bilinear).
 * The operation order below is fixed; the CUDA library evaluates the same
 * sequence so both sides hold the same FP32 coefficients. */
void orc_axis_coeffs(const orc_ref* r, int32_t axis, double delta, double d_k,
                     float* gm, float* hn, float* hb)
{
    const double Df = r->disp.D_focal;
    const double tth = axis ? r->tth_y : r->tth_x;
    const double tthp = axis ? r->tthp_y : r->tthp_x;
    const int32_t n = axis ? r->cam.Ny : r->cam.Nx;
    const int32_t Wp = axis ? r->H : r->W;

    const double den = (d_k - r->D_forward) * tthp;
    const double a = d_k * tth;
    const double g = ((double)Wp * a) / ((double)n * den);
    const double A = delta * (Df - d_k) / Df;
    const double c0 = a * (double)(1 - n) / (double)n;
    const double hw = 0.5 * (double)Wp;
    const double h_near = hw * ((A + c0) / den + 1.0);
    *gm = (float)(g - (double)r->disp.P_s);
    *hn = (float)h_near;
    *hb = (float)(h_near - 0.5);
}

/* Returns -1 for a result that lies far outside any plane (the caller treats
 * every index outside [0, W) as a transparent sample). */
int32_t orc_nearest_index(const orc_ref* r, float gm, float hn, int32_t x)
{
    const float f = floorf(fmaf(gm, (float)x, hn));
    if (!(f >= -1.0e6f && f <= 1.0e6f)) return -1;
    return r->disp.P_s * x + (int32_t)f;
}
