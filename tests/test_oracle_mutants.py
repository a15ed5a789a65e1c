"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, index or bound,
a transposed operand) in a temporary copy of the oracle source, compiles it,
and runs the pin suite against it: at least one pin must fail.  Nothing here
touches a GPU or the CUDA library.
"""

import inspect
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

MUTANTS = {
    "no_dilation": ("#define DILATION 0.3", "#define DILATION 0.0"),
    "power_b_sign": ("- b * dx * dy;", "+ b * dx * dy;"),
    "rotation_transposed": ("2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},",
                            "2.0 * (x * y + w * z), 2.0 * (x * z - w * y)},"),
    "jacobian_sign": ("-cam.fx * txc", "cam.fx * txc"),
    "colour_offset": ("fmax(acc + 0.5, 0.0)", "fmax(acc, 0.0)"),
    "sh_index": ("Y[l * l + l + mm]", "Y[l * l + l - mm]"),
    "stop_not_permanent": ("if (stop) break;", "if (stop) continue;"),
    "invdepth_weight_without_T": ("D += alpha * T / depth[g];", "D += alpha / depth[g];"),
    "invdepth_depth_not_inverted": ("D += alpha * T / depth[g];", "D += alpha * T * depth[g];"),
    "n_contrib_blended_only": ("last = contrib;", "last = contrib - (contrib > 1);"),
    "rect_max_bound": ("floor((px + r + TILE - 1) / TILE)", "floor((px + r + TILE) / TILE)"),
    "range_end_off_by_one": ("ranges[2 * tile + 1] = (uint32_t)(i + 1);", "ranges[2 * tile + 1] = (uint32_t)i;"),
    "depth_order_reversed": ("return a->key < b->key ? -1 : 1;", "return a->key < b->key ? 1 : -1;"),
    "alpha_clamp": ("#define ALPHA_MAX 0.99", "#define ALPHA_MAX 0.999"),
    "alpha_skip": ("#define ALPHA_MIN (1.0 / 255.0)", "#define ALPHA_MIN (0.5 / 255.0)"),
    "t_stop": ("#define T_MIN 1e-4", "#define T_MIN 1e-3"),
    "near_plane": ("if (z32 <= NEAR_Z) continue;", "if (z32 <= 0.0f) continue;"),
    "eigen_floor": ("#define LAMBDA_FLOOR 0.1", "#define LAMBDA_FLOOR 0.0"),
    "radius_sigmas": ("double rr = 3.0 * sqrt", "double rr = 2.5 * sqrt"),
    "conic_b_sign": ("conic[3 * g + 1] = -s01 / det;", "conic[3 * g + 1] = s01 / det;"),
    "camera_centre_sign": ("campos[i] -= cam.V[j][i]", "campos[i] += cam.V[j][i]"),
    "sigmoid_sign": ("exp(-(double)opacity_logits[g])", "exp((double)opacity_logits[g])"),
    "frustum_slack": ("#define FRUSTUM_SLACK 1.3", "#define FRUSTUM_SLACK 1.0"),
    "background_unweighted": ("C[ch] + T * bg[ch]", "C[ch] + bg[ch]"),
    "quat_not_normalised": ("double w = qf[0] / qn, x = qf[1] / qn, y = qf[2] / qn, z = qf[3] / qn;",
                            "double w = qf[0], x = qf[1], y = qf[2], z = qf[3];"),
    "scale_not_squared": ("acc += R[i][k] * s[k] * s[k] * R[j][k];", "acc += R[i][k] * s[k] * R[j][k];"),
    "tile_id_transposed": ("(uint64_t)y * (uint64_t)tiles_x + (uint64_t)x", "(uint64_t)x * (uint64_t)tiles_x + (uint64_t)y"),
    "pixel_centre_offset": ("composite_pixel((double)px, (double)py, vals", "composite_pixel((double)px + 0.5, (double)py + 0.5, vals"),
    # near-decision bookkeeping (which pixels a parity test may excuse)
    "near_pos_err_dropped": ("double pos_err = pos_eps * (", "double pos_err = 0.0 * pos_eps * ("),
    "near_pos_err_no_offset": ("(fabs(xy[2 * g]) + 1.0)", "fabs(xy[2 * g])"),
    "alpha_margin_uses_tau_T": ("< tau_alpha + pos_err)", "< tau_T + pos_err)"),
    "stop_margin_uses_tau_alpha": ("< tau_T + pos_err * alpha", "< tau_alpha + pos_err * alpha"),
    "stop_margin_without_alpha_factor": ("pos_err * alpha / (1.0 - alpha))", "pos_err)"),
    "flip_of_stop_ignored": ("if (flip == 2 * i + DECIDE_STOP) stop = !stop;", ""),
    "flip_rewalk_never_stops": ("int stop = Tn < T_MIN;", "int stop = Tn < T_MIN && flip < 0;"),
    "flip_impact_first_near_only": ("for (int64_t k = 0; k < near.n; ++k) {",
                                    "for (int64_t k = 0; k < (near.n > 0 ? 1 : 0); ++k) {"),
    "flip_impact_first_channel_only": ("for (int ch = 0; ch < 3; ++ch) impact = fmax(",
                                       "for (int ch = 0; ch < 1; ++ch) impact = fmax("),
    "edge_dist_no_clamp": ("if (k < 1.0 || k > (double)hi) return 1e30;", "(void)hi;"),
    "edge_dist_drops_an_edge": ("e = fmin(e, rect_edge_dist(py - r, TILE, cam.tiles_y));", ""),
    "rad_dist_of_lambda": ("rad_dist[g] = dist_to_int(rr);", "rad_dist[g] = dist_to_int(sqrt(fmax(lam1, lam2)));"),
}


def _pin_functions():
    import test_oracle_exclusion as exclusion
    import test_oracle_pins as pins
    out = []
    for mod in (pins, exclusion):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_") or name == "test_unrestricted_bruteforce_difference_reported":
                continue
            if fn.__module__ != mod.__name__:
                continue  # imported helpers
            out.append((f"{mod.__name__}.{name}", fn))
    return out


def _run_pins(oracle_mod):
    failed = []
    for name, fn in _pin_functions():
        params = inspect.signature(fn).parameters
        marks = getattr(fn, "pytestmark", [])
        arg_sets = [{}]
        for mk in marks:
            if mk.name == "parametrize":
                names = [s.strip() for s in mk.args[0].split(",")]
                arg_sets = [dict(zip(names, v if isinstance(v, tuple) else (v,))) for v in mk.args[1]]
        for extra in arg_sets:
            kwargs = dict(extra)
            if "oracle" in params:
                kwargs["oracle"] = oracle_mod
            try:
                fn(**kwargs)
            except AssertionError:
                failed.append(name)
                break
            except Exception:  # a crash of the mutant also counts as caught
                failed.append(name)
                break
    return failed


def _child(lib_path):
    """Run in a subprocess: load the mutant, run the pins, print the failures."""
    sys.path.insert(0, HERE)
    sys.path.insert(0, os.path.dirname(HERE))
    from oracle import oracle as O
    with O.use_library(lib_path):
        failed = _run_pins(O)
    print("FAILED_PINS " + json.dumps(failed))


def test_harness_passes_clean_oracle(oracle, tmp_path):
    """The same harness, on an unmodified copy, reports no failing pin."""
    lib = oracle.compile_variant(oracle.source_text(), str(tmp_path / "clean.so"))
    code = f"import sys; sys.path.insert(0, {HERE!r}); import test_oracle_mutants as t; t._child({lib!r})"
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    line = [l for l in proc.stdout.splitlines() if l.startswith("FAILED_PINS ")][-1]
    assert json.loads(line[len("FAILED_PINS "):]) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_mutant(oracle, tmp_path, mutant):
    old, new = MUTANTS[mutant]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site not found: {old!r}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{mutant}.so"))
    code = f"import sys; sys.path.insert(0, {HERE!r}); import test_oracle_mutants as t; t._child({lib!r})"
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        return  # the mutant crashed the pin run: caught
    line = [l for l in proc.stdout.splitlines() if l.startswith("FAILED_PINS ")][-1]
    failed = json.loads(line[len("FAILED_PINS "):])
    assert failed, f"no pin caught mutant {mutant}"
