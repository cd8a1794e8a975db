"""Planted mistakes in the oracle must turn its pins red.

The oracle is trusted because tests pin it to something other than itself: closed forms,
invariants, brute force on tiny inputs, central differences. This file checks that those
pins would notice a plausible mistake. Each case copies oracle/oracle.c (or the oracle's
Python half, oracle/__init__.py) and plants one mistake: a dropped term, a flipped sign, a
transposed operand, a comparison made strict at equality, or a branch that lets a gradient
through. It then builds the copy and runs the oracle's pin suites against it in a child
process. For oracle.c, ORACLE_LIB points the oracle package at the compiled copy; for the
Python half, a pytest plugin loads the copy as the module `oracle`. The pins hold when every
planted copy fails at least one of them, and the unchanged copies pass them all.

The golden fixture is left out of the child runs. It is the oracle's own output, so it is a
regression check rather than a pin.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "oracle" / "oracle.c"
PIN_SUITES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint_fd.py", "tests/test_oracle_multi.py",
              "tests/test_oracle_prepack.py"]

# name -> (passage the mistake contradicts, [(text in oracle.c, replacement, occurrences)])
MUTATIONS = {
    "sh_condon_shortley_phase_dropped": (
        "section 3.2 colour: real SH with the Condon-Shortley phase",
        [("double sgn = (am % 2) ? -1.0 : 1.0;", "double sgn = 1.0;", 1)]),
    "dilation_on_one_axis": (
        "Eq. 1 with the low-pass dilation S + 0.3 I",
        [("double s00 = S2[0] + op->dilation, s01 = S2[1], s11 = S2[3] + op->dilation;",
          "double s00 = S2[0] + op->dilation, s01 = S2[1], s11 = S2[3];", 1)]),
    "conic_off_diagonal_sign": (
        "Eq. 2: the conic is the inverse of the 2D covariance",
        [("out->conic[3 * i + 1] = -s01 / det;", "out->conic[3 * i + 1] = s01 / det;", 1)]),
    "ewa_jacobian_sign": (
        "Eq. 1: J is the Jacobian of the perspective projection",
        [("double J[6] = {cam->fx / z, 0.0, -cam->fx * rx / z,", "double J[6] = {cam->fx / z, 0.0, cam->fx * rx / z,", 2)]),
    "quaternion_rotation_transposed": (
        "Algorithm 1, CovFromScaleRot: R from the unit quaternion",
        [("R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);",
          "R[1] = 2 * (x * y + w * z);     R[2] = 2 * (x * z - w * y);", 1),
         ("R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);",
          "R[3] = 2 * (x * y - w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z + w * x);", 1),
         ("R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);",
          "R[6] = 2 * (x * z + w * y);     R[7] = 2 * (y * z - w * x);", 1)]),
    "camera_centre_sign": (
        "section 3.2 colour: the view direction from the camera centre -R^T t",
        [("c[j] = -(cam->R[0 * 3 + j] * cam->t[0]", "c[j] = (cam->R[0 * 3 + j] * cam->t[0]", 1)]),
    "opacity_sigmoid_sign": (
        "section 3.2: opacity = sigmoid(logit)",
        [("return 1.0 / (1.0 + exp(-(double)sc->logits[i]));", "return 1.0 / (1.0 + exp((double)sc->logits[i]));", 1)]),
    "no_jacobian_guard": (
        "Eq. 1 with x/z, y/z clamped to 1.3 tan(half FOV)",
        [("double limx = 1.3 * (cam->W / (2.0 * cam->fx)), limy = 1.3 * (cam->H / (2.0 * cam->fy));",
          "double limx = 1e300, limy = 1e300;", 2)]),
    "no_opacity_cull": (
        "Algorithm 1 culling: opacity below 1/255",
        [("if (o < op->alpha_min) return;", "", 1)]),
    "opacity_cull_strict_at_equality": (
        "Algorithm 1 culling: opacity below 1/255 (equality kept)",
        [("if (o < op->alpha_min) return;", "if (o <= op->alpha_min) return;", 1)]),
    "extent_two_sigma": (
        "Algorithm 1: the 3-sigma screen extent",
        [("int rad = (int)ceil(3.0 * sqrt(lam));", "int rad = (int)ceil(2.0 * sqrt(lam));", 1)]),
    "no_alpha_clamp": (
        "Eq. 3 with alpha = min(0.99, o G)",
        [("if (alpha > op->alpha_max) alpha = op->alpha_max;", "", 1)]),
    "alpha_min_strict_at_equality": (
        "Eq. 3: splats with alpha below 1/255 are skipped (equality kept)",
        [("if (alpha < op->alpha_min) continue;", "if (alpha <= op->alpha_min) continue;", 1)]),
    "depth_test_strict_at_equality": (
        "section 3.4: the depth test against the opaque geometry (equal depth passes)",
        [("if (z > zlim) continue;", "if (z >= zlim) continue;", 1)]),
    "stopping_splat_composited": (
        "Eq. 3 with early termination before T would fall below 1e-4",
        [("if (Tn < op->t_stop) break;",
          "if (Tn < op->t_stop) { for (int ch = 0; ch < 3; ++ch) C[ch] += pp->rgb[3 * i + ch] * alpha * T; "
          "T = Tn; ++n_contrib; last_pos = (int)(j + 1); break; }", 1)]),
    "depth_tie_break_reversed": (
        "Algorithm 1's depth sort, equal depths in index order",
        [("return (x->idx < y->idx) ? -1 : (x->idx > y->idx);", "return (x->idx > y->idx) ? -1 : (x->idx < y->idx);", 1)]),
    "colour_clamp_dropped": (
        "section 3.2 colour: max(0, SH sum + 0.5)",
        [("out->rgb[3 * i + ch] = acc < 0 ? 0.0 : acc;", "out->rgb[3 * i + ch] = acc;", 1),
         ("if (acc < 0) continue;   /* clamped channel: no gradient */", "", 1)]),
    "colour_clamp_dropped_in_forward": (
        "section 3.2 colour: max(0, SH sum + 0.5)",
        [("out->rgb[3 * i + ch] = acc < 0 ? 0.0 : acc;", "out->rgb[3 * i + ch] = acc;", 1)]),
    "colour_clamp_dropped_in_adjoint": (
        "section 3.2 colour: a clamped channel passes no gradient",
        [("if (acc < 0) continue;   /* clamped channel: no gradient */", "", 1)]),
    "adjoint_alpha_clamp_passes_gradient": (
        "Eq. 3: a clamped alpha does not depend on the splat's parameters",
        [("if (cl[k].clamped) continue;", "", 1)]),
    "adjoint_jacobian_guard_passes_gradient": (
        "Eq. 1: a clamped x/z or y/z does not depend on the mean",
        [("if (!clx) {", "if (1) {", 1), ("if (!cly) {", "if (1) {", 1)]),
    "world_covariance_not_transposed": (
        "Algorithm 1, model transforms: Sigma_w = A Sigma A^T",
        [("Sw[r * 3 + c] = AS[r * 3 + 0] * sc->A[c * 3 + 0] + AS[r * 3 + 1] * sc->A[c * 3 + 1] +\n"
          "                            AS[r * 3 + 2] * sc->A[c * 3 + 2];",
          "Sw[r * 3 + c] = AS[r * 3 + 0] * sc->A[0 * 3 + c] + AS[r * 3 + 1] * sc->A[1 * 3 + c] +\n"
          "                            AS[r * 3 + 2] * sc->A[2 * 3 + c];", 1)]),
    "sh_ray_in_the_world_frame": (
        "Algorithm 1, model transforms: the colour is evaluated in the model's own frame",
        [("    if (!sc->has_model) { d[0] = w[0]; d[1] = w[1]; d[2] = w[2]; return; }",
          "    if (1) { d[0] = w[0]; d[1] = w[1]; d[2] = w[2]; return; }", 1)]),
    "conic_cross_term_factor_dropped": (
        "Eq. 2: q = d^T S^-1 d, whose cross term counts the off-diagonal twice",
        [("double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;",
          "double q = a * dx * dx + b * dx * dy + c * dy * dy;", 1)]),
    "extent_smaller_eigenvalue": (
        "Algorithm 1: the extent from the larger eigenvalue of the 2D covariance",
        [("double lam = m + sqrt(disc);", "double lam = m - sqrt(disc);", 1)]),
    "sh_coefficient_index_mirrored": (
        "section 3.2 colour: coefficient index l*l+l+m",
        [("int k = l * l + l + m;", "int k = l * l + l - m;", 1)]),
    "near_plane_strict_at_equality": (
        "Algorithm 1 culling: depth at or in front of the near plane",
        [("if (!(z > cam->near_z)) return;", "if (!(z >= cam->near_z)) return;", 1)]),
    "transmittance_not_updated": (
        "Eq. 3: T_i is the product of (1 - alpha_j) over the splats in front",
        [("        T = Tn;\n        ++n_contrib;", "        ++n_contrib;", 1)]),
    "background_weight_dropped": (
        "Eq. 3 over a background: C + T_final bg",
        [("out->rgb[ch] = C[ch] + T * bg[ch];", "out->rgb[ch] = C[ch] + bg[ch];", 1)]),
    "adjoint_sigmoid_derivative": (
        "section 3.2: d sigmoid / d logit = o (1 - o)",
        [("d_logits[i] = go * o * (1.0 - o);", "d_logits[i] = go * o;", 1)]),
    "duplicate_tile_id_transposed": (
        "Algorithm 1's key duplication: row-major tile id ty * tiles_x + tx",
        [("uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;",
          "uint64_t tile = (uint64_t)tx * (uint64_t)tiles_x + (uint64_t)ty;", 1)]),
    "duplicate_depth_bits_dropped": (
        "Algorithm 1's key: the tile id above the depth bits",
        [("keys[m] = (tile << 32) | (uint64_t)zb;", "keys[m] = (tile << 32);", 1)]),
    "stable_sort_ties_reversed": (
        "Algorithm 1's sort: equal keys keep their input order",
        [("return (x->pos < y->pos) ? -1 : (x->pos > y->pos);", "return (x->pos > y->pos) ? -1 : (x->pos < y->pos);", 1)]),
    "tile_range_end_inclusive": (
        "Algorithm 1: a tile's range [start, end) of the sorted keys",
        [("ranges[2 * t + 1] = (uint32_t)e;", "ranges[2 * t + 1] = (uint32_t)(e - 1);", 1)]),
    "ambiguity_flag_of_the_stop_dropped": (
        "Eq. 3's early stop: a T (1 - alpha) within rounding of 1e-4 is flagged",
        [("if (fabs(Tn - op->t_stop) <= AMB_T_REL * op->t_stop) amb = 1;", "", 1)]),
    "ambiguity_flag_of_alpha_min_dropped": (
        "Eq. 3's alpha_min skip: an alpha within rounding of 1/255 is flagged",
        [("if (fabs(alpha - op->alpha_min) <= AMB_ALPHA_REL * op->alpha_min) amb = 1;", "", 1)]),
    "ambiguity_flag_of_the_cut_dropped": (
        "the 3-sigma cut: a q within rounding of 9 is flagged",
        [("if (pp->opacity[i] * exp(-0.5 * q) >= op->alpha_min * (1.0 - AMB_ALPHA_REL)) amb = 1;", "", 1)]),
    "ambiguity_flag_of_the_depth_test_dropped": (
        "section 3.4's depth test: a depth within rounding of the buffer's is flagged",
        [("if (isfinite(zlim) && fabs(z - zlim) <= AMB_Z_REL * fabs(zlim)) amb = 1;", "", 1)]),
    "composite_colour_channel": (
        "Eq. 3: each channel composites its own colour",
        [("for (int ch = 0; ch < 3; ++ch) C[ch] += pp->rgb[3 * i + ch] * alpha * T;",
          "for (int ch = 0; ch < 3; ++ch) C[ch] += pp->rgb[3 * i] * alpha * T;", 1)]),
    "sh_normalisation_factorials_dropped": (
        "section 3.2 colour: orthonormal real SH, N = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)",
        [("double N = sqrt((2.0 * l + 1.0) / (4.0 * PI) * factorial(l - am) / factorial(l + am));",
          "double N = sqrt((2.0 * l + 1.0) / (4.0 * PI));", 1)]),
    "sh_sqrt2_dropped": (
        "section 3.2 colour: the real SH of m != 0 carry sqrt(2)",
        [("if (m != 0) N *= sqrt(2.0);", "", 1)]),
    "legendre_recursion": (
        "section 3.2 colour: Legendre polynomials by Bonnet's recursion",
        [("double b = (double)l * c[l - 1][k];", "double b = (double)(l + 1) * c[l - 1][k];", 1)]),
    "principal_point_dropped": (
        "Eq. 1: x_i = Pi(mu_i), the pinhole projection with its principal point",
        [("double u = cam->fx * p[0] / z + cam->cx;", "double u = cam->fx * p[0] / z;", 1)]),
    "view_translation_dropped": (
        "Eq. 1: the view transform p = R x_w + t",
        [("p[r] = cam->R[r * 3 + 0] * xw[0] + cam->R[r * 3 + 1] * xw[1] + cam->R[r * 3 + 2] * xw[2] + cam->t[r];\n"
          "    double z = p[2];",
          "p[r] = cam->R[r * 3 + 0] * xw[0] + cam->R[r * 3 + 1] * xw[1] + cam->R[r * 3 + 2] * xw[2];\n"
          "    double z = p[2];", 1)]),
    "scale_not_squared": (
        "Algorithm 1, CovFromScaleRot: Sigma = R diag(s)^2 R^T",
        [("for (int k = 0; k < 3; ++k) { double s = exp((double)log_s[k]); s2[k] = s * s; }",
          "for (int k = 0; k < 3; ++k) { double s = exp((double)log_s[k]); s2[k] = s; }", 1)]),
    "model_adjoint_left_factor_dropped": (
        "Algorithm 1, model transforms: dL/dSigma = A^T (dL/dSigma_w) A",
        [("acc += sc->A[r * 3 + a] * gSigw[r * 3 + c] * sc->A[c * 3 + b];",
          "acc += (double)(r == a) * gSigw[r * 3 + c] * sc->A[c * 3 + b];", 1)]),
}


# The same for the oracle's Python half (oracle/__init__.py: the fp16 pre-pack, the dynamic
# update, the thresholds as the library receives them). A pytest plugin in the child loads the
# planted copy as the module `oracle` before any test imports it.
PY_SRC = ROOT / "oracle" / "__init__.py"
PY_MUTATIONS = {
    "dynamic_mean_without_time": (
        "the dynamic workload: mu_t = mu_0 + t v",
        [("m = _f64(means0) + t * _f64(velocity)", "m = _f64(means0) + _f64(velocity)", 1)]),
    "dynamic_pulse_without_2pi": (
        "the dynamic workload: logit_t = logit_0 + A sin(2 pi f t + phi)",
        [("np.sin(2.0 * np.pi * _f64(freq) * t + _f64(phase))", "np.sin(np.pi * _f64(freq) * t + _f64(phase))", 1)]),
    "prepack_opacity_sign": (
        "Algorithm 1's pre-pack: opacity alpha = sigmoid(logit)",
        [('alpha = 1.0 / (1.0 + np.exp(-_f64(scene["opacity_logits"])))',
          'alpha = 1.0 / (1.0 + np.exp(_f64(scene["opacity_logits"])))', 1)]),
    "prepack_covariance_entry_order": (
        "section 3.4's pre-packed covariance (xx, xy, xz, yy, yz, zz)",
        [("cov6 = np.stack([sig[:, 0, 0], sig[:, 0, 1], sig[:, 0, 2], sig[:, 1, 1], sig[:, 1, 2], sig[:, 2, 2]], 1)",
          "cov6 = np.stack([sig[:, 0, 0], sig[:, 0, 2], sig[:, 0, 1], sig[:, 1, 1], sig[:, 1, 2], sig[:, 2, 2]], 1)",
          1)]),
    "prepack_means_not_half": (
        "section 3.4's pre-pack: the means are cast to fp16",
        [('mu_h = _f64(scene["means"]).astype(np.float16)', 'mu_h = _f64(scene["means"]).astype(np.float32)', 1)]),
    "thresholds_not_rounded_to_float32": (
        "the oracle compares against the float32 thresholds the library receives",
        [("return np.array([float(np.float32(v)) for v in vals], np.float64)",
          "return np.array([float(v) for v in vals], np.float64)", 1)]),
}

PY_CONTROL = "python_half_unchanged"   # the plugin route with nothing planted: must pass

PLUGIN = """import importlib.util, sys
_spec = importlib.util.spec_from_file_location("oracle", {path!r})
_mod = importlib.util.module_from_spec(_spec)
sys.modules["oracle"] = _mod
_spec.loader.exec_module(_mod)
"""


def _planted(name):
    """oracle.c (or, for a Python mistake, oracle/__init__.py) with the named mistake planted
    (None: oracle.c unchanged)."""
    table = PY_MUTATIONS if name in PY_MUTATIONS else MUTATIONS
    src = (PY_SRC if name in PY_MUTATIONS or name == PY_CONTROL else SRC).read_text()
    if name is None or name == PY_CONTROL:
        return src
    for old, new, count in table[name][1]:
        found = src.count(old)
        assert found == count, f"{name}: {old!r} occurs {found} times in the oracle, expected {count}"
        src = src.replace(old, new)
    return src


def _run_pins(name, workdir, lib_unchanged=None):
    """Build the planted copy and run the pin suites on it; returns (exit code, output tail)."""
    tag = name or "unchanged"
    env = dict(os.environ, OMP_NUM_THREADS="1")
    plugin = []
    if name in PY_MUTATIONS or name == PY_CONTROL:
        pkg = workdir / f"py_{tag}"
        pkg.mkdir()
        (pkg / "planted_oracle.py").write_text(_planted(name))
        (pkg / f"plant_{tag}.py").write_text(PLUGIN.format(path=str(pkg / "planted_oracle.py")))
        env["PYTHONPATH"] = os.pathsep.join([str(pkg)] + [p for p in [env.get("PYTHONPATH")] if p])
        env["ORACLE_LIB"] = str(lib_unchanged)
        plugin = ["-p", f"plant_{tag}"]
    else:
        c_file = workdir / f"{tag}.c"
        lib = workdir / f"lib{tag}.so"
        c_file.write_text(_planted(name))
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", str(lib), str(c_file),
                        "-lm"], check=True, capture_output=True)
        env["ORACLE_LIB"] = str(lib)
    r = subprocess.run([sys.executable, "-m", "pytest", *plugin, *PIN_SUITES, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-600:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    import oracle
    lib_unchanged = oracle.build()
    names = [None, PY_CONTROL] + list(MUTATIONS) + list(PY_MUTATIONS)
    for name in names[2:]:
        _planted(name)   # each planted text is found where expected before anything runs
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as pool:
        results = dict(zip(names, pool.map(lambda n: _run_pins(n, tmp_path, lib_unchanged), names)))
    for control in (None, PY_CONTROL):
        code, tail = results.pop(control)
        assert code == 0, f"the unchanged copy ({control or 'oracle.c'}) fails its pins:\n{tail}"
    survivors = {n: t for n, (c, t) in results.items() if c == 0}
    broken = {n: (c, t) for n, (c, t) in results.items() if c not in (0, 1)}
    assert not broken, "children that did not run their tests: " + "; ".join(
        f"{n} (exit {c}): {t[-200:]}" for n, (c, t) in broken.items())
    assert not survivors, "planted mistakes that no pin catches: " + ", ".join(
        f"{n} ({{**MUTATIONS, **PY_MUTATIONS}}[n][0])" for n in survivors)


@pytest.mark.parametrize("name", sorted(MUTATIONS) + sorted(PY_MUTATIONS))
def test_planted_text_is_in_the_oracle(name):
    _planted(name)
