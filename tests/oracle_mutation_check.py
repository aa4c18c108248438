"""Mutation check of the oracle's pins (a development tool, not collected by
pytest).

Each entry plants one plausible mistake in the oracle's C sources (a wrong
sign, a dropped factor, an off-by-half coordinate, a changed reading), rebuilds
the oracle, runs the CPU pin tests and records whether at least one of them
fails. The source file is restored and the oracle rebuilt after every entry,
whatever happens.

    python tests/oracle_mutation_check.py          # all entries
    python tests/oracle_mutation_check.py 3 7      # entries 3 and 7

Exit status 1 if any mistake goes unnoticed.
"""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["tests/test_oracle_geometry.py", "tests/test_oracle_gaussians.py", "tests/test_oracle_composite.py",
             "tests/test_oracle_voxels.py", "tests/test_oracle_binning.py", "tests/test_oracle_filter.py"]

# (file under oracle/, exact text, replacement, what the mistake is)
MUTATIONS = [
    ("orc_composite.c", "med = (keys[lo + c / 2 - 1].z + keys[lo + c / 2].z) * 0.5;", "med = keys[lo + c / 2 - 1].z;",
     "even-count median taken as the lower middle"),
    ("orc_composite.c", "const double f = floor((double)N * (izmin - 1.0 / keys[i].z) / span);",
     "const double f = floor((double)(N - 1) * (izmin - 1.0 / keys[i].z) / span);", "N - 1 disparity bins"),
    ("orc_composite.c", "const double disp = izmin - ((double)k + 0.5) / (double)N * span;",
     "const double disp = izmin - ((double)k + 0.0) / (double)N * span;", "disparity d_k at a bin edge"),
    ("orc_composite.c", "const int32_t k = (int32_t)((i * (int64_t)N) / M);",
     "const int32_t k = (int32_t)(((i + 1) * (int64_t)N - 1) / M);", "shifted quantile chunk formula"),
    ("orc_composite.c", "return (x->idx > y->idx) - (x->idx < y->idx);", "return (x->idx < y->idx) - (x->idx > y->idx);",
     "depth ties by descending index"),
    ("orc_composite.c", "const double w = (dx ? wx : 1.0 - wx) * (dy ? wy : 1.0 - wy);",
     "const double w = (dx ? 1.0 - wx : wx) * (dy ? wy : 1.0 - wy);", "bilinear x weights swapped"),
    ("orc_composite.c", "            const int64_t xx = x0 + dx, yy = y0 + dy;\n"
                        "            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;",
     "            int64_t xx = x0 + dx, yy = y0 + dy;\n"
     "            if (xx < 0) xx = 0; if (xx >= W) xx = W - 1; if (yy < 0) yy = 0; if (yy >= H) yy = H - 1;",
     "bilinear taps clamped instead of transparent"),
    ("orc_composite.c", "                        if (ix >= 0 && ix < W && iy >= 0 && iy < H) {\n"
                        "                            const double* t = P + 4 * ((int64_t)iy * W + ix);",
     "                        {\n"
     "                            const int32_t cx_ = ix < 0 ? 0 : (ix >= W ? W - 1 : ix), "
     "cy_ = iy < 0 ? 0 : (iy >= H ? H - 1 : iy);\n"
     "                            const double* t = P + 4 * ((int64_t)cy_ * W + cx_);",
     "nearest samples clamped instead of transparent"),
    ("orc_composite.c", "T *= 1.0 - c[3];", "T *= 1.0 - 0.999 * c[3];", "transmittance update off"),
    ("orc_composite.c", "                    Q[0] += T * c[0];", "                    Q[0] += T * c[0] * c[3];",
     "colour treated as straight alpha"),
    ("orc_composite.c", "o[0] = Q[0] + T * bg[0];", "o[0] = Q[0] + bg[0];", "background not attenuated"),
    ("orc_voxels.c", "4.0 * trilinear(density8, fm)", "2.0 * trilinear(density8, fm)", "Simpson weight"),
    ("orc_voxels.c", "0.5 * (t0 + t1), fm);", "0.45 * (t0 + t1), fm);", "Simpson midpoint"),
    ("orc_voxels.c", "if (!(zmin > r->disp.z_near)) continue;", "if (!(zmin > 0.0)) continue;",
     "voxel near-plane culling dropped"),
    ("orc_voxels.c", "const float fx0 = ceilf(mnx), fx1 = floorf(mxx);", "const float fx0 = ceilf(mnx) + 1.0f, fx1 = floorf(mxx);",
     "voxel rectangle shrunk"),
    ("orc_voxels.c", "for (int a = 0; a < 3; ++a) dw[a] /= nrm;", "for (int a = 0; a < 3; ++a) dw[a] /= 1.0;",
     "voxel ray not normalised"),
    ("orc_voxels.c", "                    px[0] += T * al * rgb[3 * v + 0];", "                    px[0] += al * rgb[3 * v + 0];",
     "voxel colour without the transmittance"),
    ("orc_voxels.c", "const double dc[3] = {((double)x - r->cx) / r->fx, ((double)y - r->cy) / r->fy, 1.0};",
     "const double dc[3] = {((double)x - r->cx) / r->fx, ((double)y - r->cy) / r->fx, 1.0};", "f_x used for the y ray"),
    ("orc_geometry.c", "r->tthp_x = Df * r->tth_x / (Df - r->D_forward0);",
     "r->tthp_x = Df * r->tth_x / (Df - (r->D_forward0 - disp->D_shift));", "theta' from the shifted camera"),
    ("orc_geometry.c", "const float f = floorf(fmaf(gm, (float)x, hn));", "const float f = floorf(fmaf(gm, (float)x, hn) - 0.5f);",
     "nearest index off by half"),
    ("orc_geometry.c", "return (double)j / (double)(V - 1) - 0.5;", "return 0.5 - (double)j / (double)(V - 1);",
     "view order reversed"),
    ("orc_geometry.c", "r->cx = 0.5 * (double)(r->W - 1);", "r->cx = 0.5 * (double)(r->W);", "principal point off by half"),
    ("orc_geometry.c", "for (int32_t i = 0; i < Vy; ++i) dy[i] = 2.0 * Df * view_s(i, Vy) * r->tphi_y;",
     "for (int32_t i = 0; i < Vy; ++i) dy[i] = 2.0 * Df * view_s(i, Vy) * r->tphi_x;", "vertical offsets from phi_x"),
    ("orc_geometry.c", "    const double u = (2.0 * (double)x + 1.0) / (double)n - 1.0;\n    const double up",
     "    const double u = (2.0 * (double)x) / (double)n - 1.0;\n    const double up", "view pixel centre off by half"),
    ("orc_geometry.c", "return (delta * (Df - d_k) / Df + d_k * tth * u) / ((d_k - r->D_forward) * tthp);",
     "return (-delta * (Df - d_k) / Df + d_k * tth * u) / ((d_k - r->D_forward) * tthp);", "parallax sign flipped"),
    ("orc_geometry.c", "return ((up + 1.0) * (double)Wp - 1.0) / 2.0;", "return ((up + 1.0) * (double)Wp) / 2.0;",
     "plane pixel centre off by half"),
    ("orc_gaussians.c", "const double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;\n"
                        "                    double al = o * exp(-0.5 * q);\n"
                        "                    if (al > 0.99) al = 0.99;\n"
                        "                    double* px = P + 4 * (y * W + x);",
     "const double q = a * dx * dx + b * dx * dy + c * dy * dy;\n"
     "                    double al = o * exp(-0.5 * q);\n"
     "                    if (al > 0.99) al = 0.99;\n"
     "                    double* px = P + 4 * (y * W + x);", "cross term without its factor 2"),
    ("orc_gaussians.c", "if (al > 0.99) al = 0.99;\n                    double* px = P + 4 * (y * W + x);",
     "if (al > 0.995) al = 0.995;\n                    double* px = P + 4 * (y * W + x);", "opacity clamp 0.995"),
    ("orc_gaussians.c", "const float rad = ceilf(3.0f * sqrtf(lam));", "const float rad = ceilf(2.5f * sqrtf(lam));",
     "2.5-sigma footprint"),
    ("orc_gaussians.c", "const float fx0 = ceilf(px - rad), fx1 = floorf(px + rad);",
     "const float fx0 = floorf(px - rad), fx1 = floorf(px + rad);", "floored left rectangle edge"),
    ("orc_gaussians.c", "const float lam = mid + sqrtf(fmaxf(fmaf(mid, mid, -det), 0.0f));", "const float lam = mid;",
     "lambda_max taken as the mean eigenvalue"),
    ("orc_gaussians.c", "const float py = fmaf(fyf, yn, cyf);", "const float py = fmaf(fyf, yn, cyf + 0.5f);",
     "FP32 2D mean off by half"),
    ("orc_gaussians.c", "if (!(det > 0.0f)) return 0;", "if (!(det > -1.0f)) return 0;", "singular covariance kept"),
    ("orc_gaussians.c", "if (!(zg > r->disp.z_near)) continue;", "if (!(zg > 0.0)) continue;",
     "Gaussian near-plane culling dropped"),
    ("orc_gaussians.c", "        S2[1][1] += r->f_prime;", "        S2[1][1] += 0.0 * r->f_prime;",
     "dilation dropped on one axis"),
    ("orc_gaussians.c", "double qn = sqrt(qf[0] * qf[0] + qf[1] * qf[1] + qf[2] * qf[2] + qf[3] * qf[3]);", "double qn = 1.0;",
     "quaternion not normalised"),
    ("orc_gaussians.c", "const double J[2][3] = {{r->fx / zz, 0.0, -r->fx * pc[0] / (zz * zz)},",
     "const double J[2][3] = {{r->fx / zz, 0.0, r->fx * pc[0] / (zz * zz)},", "EWA Jacobian sign"),
    ("orc_gaussians.c", "{2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},",
     "{2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},", "rotation matrix entry sign"),
    ("orc_gaussians.c", "for (int l = 0; l < 3; ++l) acc += tmp[i][l] * R[3 * j + l];",
     "for (int l = 0; l < 3; ++l) acc += tmp[i][l] * R[3 * l + j];", "W Sigma W^T transposed"),
    ("orc_gaussians.c", "                    if (Tn < t_min) {\n                        done[p] = 1;\n                        continue;\n",
     "                    if (Tn < t_min) {\n                        done[p] = 1;\n", "3DGS: the stopping member is blended"),
    ("orc_gaussians.c", "                    if (done[p]) continue;", "                    (void)done;",
     "3DGS: blending goes on after a stop"),
    ("orc_gaussians.c", "if (nr && fabs(Tn - t_min) <= window) nr[p] = 1;", "if (nr && fabs(Tn - t_min) <= 0.0) nr[p] = 1;",
     "3DGS near mask misses transmittance events"),
    ("orc_gaussians.c", "if (nr && fabs(al - a_min) <= window) nr[p] = 1;", "if (nr && fabs(al - a_min) <= 0.0) nr[p] = 1;",
     "3DGS near mask misses alpha events"),
    ("orc_filter.c", "w[i + radius] = exp(-0.5 * (double)i * (double)i / (sigma * sigma));",
     "w[i + radius] = exp(-(double)i * (double)i / (sigma * sigma));", "filter sigma off"),
    ("orc_filter.c", "for (int32_t i = 0; i <= 2 * radius; ++i) w[i] /= sum;",
     "for (int32_t i = 0; i <= 2 * radius; ++i) w[i] /= sum * 1.0001;", "filter weights not normalised"),
    ("orc_filter.c", "const int32_t xx = x + i;\n                        if (xx < 0 || xx >= W) continue;",
     "int32_t xx = x + i;\n                        if (xx < 0) xx = 0; if (xx >= W) xx = W - 1;", "filter rows clamp at the edge"),
    ("orc_filter.c", "                        const int32_t yy = y + i;\n                        if (yy < 0 || yy >= H) continue;",
     "                        int32_t yy = y + i;\n                        if (yy < 0) yy = 0; if (yy >= H) yy = H - 1;",
     "filter columns clamp at the edge"),
]


def _build():
    return subprocess.run([sys.executable, "-c", "from oracle import build; build.build(force=True)"], cwd=ROOT,
                          capture_output=True, text=True)


def run(indices):
    missed = []
    for n in indices:
        fname, old, new, what = MUTATIONS[n]
        path = os.path.join(ROOT, "oracle", fname)
        src = open(path).read()
        if src.count(old) != 1:
            print("%2d  STALE  %s (text found %d times)" % (n, what, src.count(old)))
            missed.append(n)
            continue
        backup = path + ".orig"
        shutil.copy(path, backup)
        try:
            with open(path, "w") as f:
                f.write(src.replace(old, new))
            if _build().returncode != 0:
                print("%2d  BUILD  %s" % (n, what))
                missed.append(n)
                continue
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu"] + PIN_TESTS, cwd=ROOT,
                               capture_output=True, text=True)
            failed = [ln[7:].split(" ")[0] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
            if r.returncode != 0 and failed:
                print("%2d  caught  %-45s by %s" % (n, what, failed[0]))
            else:
                print("%2d  MISSED  %s" % (n, what))
                missed.append(n)
        finally:
            shutil.move(backup, path)
    if _build().returncode != 0:
        raise SystemExit("could not rebuild the restored oracle")
    return missed


if __name__ == "__main__":
    sel = [int(a) for a in sys.argv[1:]] or list(range(len(MUTATIONS)))
    missed = run(sel)
    print("%d of %d planted mistakes caught" % (len(sel) - len(missed), len(sel)))
    sys.exit(1 if missed else 0)
