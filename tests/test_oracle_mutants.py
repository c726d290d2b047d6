"""Mutation tests of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle source (a
dropped term, a wrong sign or index, a transposed operand), builds it, and
runs the pin suite against that build in a subprocess.  The pins must fail
for every mutant: a mistake of that kind anywhere in the oracle would be
caught.  CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "smcrt_oracle.c")

# (name, exact text in the oracle, replacement)
MUTANTS = [
    ("philox_key_bump", "k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;", "k0 += 0x9E3779B9u; k1 += 0xBB67AE86u;"),
    ("log_series_term", "poly = poly * z + 1.0 / 5.0;", "poly = poly * z + 1.0 / 6.0;"),
    ("sincos_quadrant", "else if (qi == 1) { *sn = c;  *cs = -s; }", "else if (qi == 1) { *sn = c;  *cs = s; }"),
    ("sphere_radius_sign", "return sqrt(dx * dx + dy * dy + dz * dz) - q[3];", "return sqrt(dx * dx + dy * dy + dz * dz) + q[3];"),
    ("box_inside_term", "double inside = fmin(fmax(qx, fmax(qy, qz)), 0.0);", "double inside = fmin(fmax(qx, qy), 0.0);"),
    ("capsule_clamp", "t = fmin(fmax(t, 0.0), 1.0);", "t = fmin(fmax(t, 0.0), 0.5);"),
    ("subtract_sign", "if (op == 4) return fmax(a, -b);", "if (op == 4) return fmax(-a, b);"),
    ("smooth_operands", "double h = 0.5 + 0.5 * (b - a) / k;", "double h = 0.5 + 0.5 * (a - b) / k;"),
    ("hg_g_sign", "double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);", "double t = (1.0 - g * g) / (1.0 + g + 2.0 * g * xi);"),
    ("rotation_basis", "b2[0] = b; b2[1] = sg + n[1] * n[1] * a; b2[2] = -n[1];", "b2[0] = b; b2[1] = sg + n[0] * n[1] * a; b2[2] = -n[1];"),
    ("fresnel_p_term", "double rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);", "double rp = (n1 * ci - n2 * ct) / (n1 * ct + n2 * ci);"),
    ("snell_eta", "double eta = n1 / n2;\n        double k = sg * (eta * ci - ct);", "double eta = n2 / n1;\n        double k = sg * (eta * ci - ct);"),
    ("reflect_sign", "double c2 = 2.0 * c;", "double c2 = -2.0 * c;"),
    ("dda_plane_index", "tnext[a] = ((G->lo[a] + (double)(i + 1) * dl[a]) - p[a]) / u[a];", "tnext[a] = ((G->lo[a] + (double)(i + 2) * dl[a]) - p[a]) / u[a];"),
    ("tally_voxel_order", "size_t off = ((size_t)idx[2] * (size_t)G->n[1] + (size_t)idx[1]) * (size_t)G->n[0] + (size_t)idx[0];",
     "size_t off = ((size_t)idx[0] * (size_t)G->n[1] + (size_t)idx[1]) * (size_t)G->n[0] + (size_t)idx[2];"),
    ("free_path_mu", "double s = tau / mu_t;", "double s = tau / mu_s;"),
    ("tau_consumed", "tau = tau - mu_t * L;", "tau = tau - mu_a * L;"),
    ("absorbed_weight", "double wn = w * (mu_s / mu_t);", "double wn = w * (mu_a / mu_t);"),
    ("roulette_gain", "P.gain += fx(w * (OR_ROULETTE_M - 1.0));", "P.gain += fx(w * OR_ROULETTE_M);"),
    # survival chance not matched to the weight multiplier: the energy
    # identity still holds, only the roulette pin's expectation catches these
    ("roulette_survival_mismatch", "if (xi[2] <= 1.0 / OR_ROULETTE_M) {", "if (xi[2] <= 0.2) {"),
    ("roulette_survival_slight", "if (xi[2] <= 1.0 / OR_ROULETTE_M) {", "if (xi[2] <= 0.09) {"),
    ("roulette_survival_side", "if (xi[2] <= 1.0 / OR_ROULETTE_M) {", "if (xi[2] > 1.0 / OR_ROULETTE_M) {"),
    ("roulette_threshold", "if (w < OR_W_ROULETTE) {", "if (w < 10.0 * OR_W_ROULETTE) {"),
    ("escape_split", "if (u[0] * src->dir[0] + u[1] * src->dir[1] + u[2] * src->dir[2] < 0.0) P.R += fx(w);",
     "if (u[0] * src->dir[0] + u[1] * src->dir[1] + u[2] * src->dir[2] > 0.0) P.R += fx(w);"),
    ("region_priority", "if (d < 0.0) E.region = r;", "if (d < 0.0 && E.region < 0) E.region = r;"),
    ("disc_radius", "double rho = src->radius * sqrt(xi[0]);", "double rho = src->radius * xi[0];"),
    ("iso_cos_theta", "double ct = 2.0 * xi[0] - 1.0;\n        double st", "double ct = xi[0];\n        double st"),
    ("square_side", "c2 = src->radius * (2.0 * xi[1] - 1.0);", "c2 = src->radius * (2.0 * xi[0] - 1.0);"),
    ("segment_box_margin", "double e = d > 0.0 ? dh : -dh;", "double e = d > 0.0 ? 0.0 : -dh;"),
    ("segment_sphere_root", "t = cc / (sqrt(disc) - b);", "t = sqrt(disc) - b;"),
    ("segment_soft_bound", "if (region_soft(S, r) && ad < E.dsoft) E.dsoft = ad;", "if (0 && ad < E.dsoft) E.dsoft = ad;"),
    ("segment_step_rule", "if (S->stepping == 1) L = fmax(L, segment_bound(S, &E, p, u, T));",
     "if (S->stepping == 1) L = fmin(L, segment_bound(S, &E, p, u, T));"),
    ("torus_tube_radius", "return sqrt(ring * ring + dz * dz) - q[4];", "return sqrt(ring * ring + dz * dz) - q[3];"),
    ("cylinder_cap", "double b = fabs(dz) - q[4];", "double b = dz - q[4];"),
    ("frame_rotation_transposed", "double q[3];\n    q[0] = (X->rot[0] * vx + X->rot[3] * vy + X->rot[6] * vz) / X->s;",
     "double q[3];\n    q[0] = (X->rot[0] * vx + X->rot[1] * vy + X->rot[2] * vz) / X->s;"),
    ("frame_scale_dropped", "return X->s * sdf_base(pr->kind, pr->p, q) / L;", "return sdf_base(pr->kind, pr->p, q) / L;"),
    ("elongate_clamp", "q[a] = q[a] - fmin(fmax(q[a], -X->a[a]), X->a[a]);", "q[a] = q[a] - fmin(q[a], X->a[a]);"),
    ("repeat_rounding", "double k = floor(q[a] / c + 0.5);", "double k = floor(q[a] / c);"),
    ("twist_stretch_bound", "L = X->op == 2 ? 0.5 * (m + sqrt(m * m + 4.0)) : 1.0 + m;", "L = sqrt(1.0 + m * m);"),
    ("segment_capsule_margin", "double rr = d > 0.0 ? q[6] + dh : q[6] - dh;", "double rr = d > 0.0 ? q[6] : q[6] - dh;"),
    ("segment_capsule_far_ball", "ray_ball(ox - bax, oy - bay, oz - baz, rr, u, &t0[1], &t1[1]);",
     "ray_ball(ox + bax, oy + bay, oz + baz, rr, u, &t0[1], &t1[1]);"),
    ("segment_cylinder_cross_axis", "double vx = u[0] - k * bax, vy = u[1] - k * bay, vz = u[2] - k * baz;",
     "double vx = u[0], vy = u[1], vz = u[2];"),
    ("segment_capsule_exit", "if (t0[k] <= t1[k]) t = fmax(t, t1[k]);", "if (t0[k] <= t1[k]) t = fmax(t, t0[k]);"),
    ("segment_xprim_margin", "segment_base(pr->kind, pr->p, d / X->s, q, w, e / X->s);",
     "segment_base(pr->kind, pr->p, d / X->s, q, w, e);"),
    ("segment_xprim_scale", "return X->s * segment_base(", "return segment_base("),
    # smooth-union margin: one fold's k/4 instead of the sum over the folds
    ("segment_fold_margin", "m = m + 0.25 * S->nodes[R->begin + i].k;", "m = 0.25 * S->nodes[R->begin + i].k;"),
    ("segment_margin_unused", "double e = prim_margin(S, nd->prim) + dh;", "double e = dh;"),
    # passing over a primitive whose own distance (not less the margin)
    # reaches the bound so far
    ("segment_prune_margin", "if (fabs(d) - e >= t) continue;", "if (fabs(d) >= t) continue;"),
    ("segment_cylinder_cap", "double rr = q[3] + g, hh = q[4] + g;", "double rr = q[3] + g, hh = q[4];"),
    ("segment_cylinder_exit", "    return t1 > 0.0 ? t1 : 0.0;\n}\n\n/* Torus", "    return t0 > 0.0 ? t0 : 0.0;\n}\n\n/* Torus"),
    ("segment_torus_growth", "double R = q[3], rt = q[4] + e;", "double R = q[3], rt = q[4];"),
    ("segment_torus_hole", "if (b0 <= lo && lo < b1) lo = b1;", "if (0) lo = b1;"),
    ("segment_torus_inside_center", "double ball[4] = {q[0] + q[3] * dx / rho, q[1] + q[3] * dy / rho, q[2], q[4]};",
     "double ball[4] = {q[0] + q[3] * dx, q[1] + q[3] * dy, q[2], q[4]};"),
    ("segment_torus_inside_radius", "double ball[4] = {q[0] + q[3] * dx / rho, q[1] + q[3] * dy / rho, q[2], q[4]};",
     "double ball[4] = {q[0] + q[3] * dx / rho, q[1] + q[3] * dy / rho, q[2], q[3]};"),
    ("segment_xprim_direction", "w[0] = X->rot[0] * u[0] + X->rot[3] * u[1] + X->rot[6] * u[2];",
     "w[0] = X->rot[0] * u[0] + X->rot[1] * u[1] + X->rot[2] * u[2];"),
]


def _run_mutant(tmp, name, old, new):
    src = open(SRC).read()
    if src.count(old) != 1:
        return name, f"mutation site not unique/found"
    mpath = os.path.join(tmp, f"{name}.c")
    with open(mpath, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", mpath,
                           "-o", lib, "-lm"])
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return name, None if r.returncode != 0 else f"no pin caught it:\n{r.stdout[-1500:]}"


@pytest.mark.slow
def test_pins_catch_every_mutant(tmp_path):
    # the mutants run side by side, one pin-suite process each
    from concurrent.futures import ThreadPoolExecutor
    workers = max(2, min(len(MUTANTS), os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda m: _run_mutant(str(tmp_path), *m), MUTANTS))
    missed = [(n, why) for n, why in results if why]
    assert not missed, missed
