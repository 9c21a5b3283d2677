"""The pins are strong enough to catch plausible slips: each test plants one
mistake in a copy of the oracle's C source (on the CPU, in a temporary
directory), rebuilds it, and checks that the pin tests then fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "max_min_swapped_in_G_plus": ("const double ax = max0(dmx), bx = min0(dpx);",
                                  "const double ax = min0(dmx), bx = max0(dpx);"),
    "dropped_z_term": ("const double spz = az * az + bz * bz;", "const double spz = az * az;"),
    "F_sign_routed_wrong": ("max0(F) * gplus + min0(F) * gminus", "max0(F) * gminus + min0(F) * gplus"),
    "wrong_y_stride": ("one_sided(phi, i, (size_t)nx, y, ny", "one_sided(phi, i, (size_t)ny, y, ny"),
    "high_face_rule_missing": ("if (!has_p && has_m) p = m;", ""),
    "tube_not_strict": ("fabs(phi[idx3(nx, ny, x, y, z)]) < gamma", "fabs(phi[idx3(nx, ny, x, y, z)]) <= gamma"),
    "dilation_6_for_26": ("if (conn == 6 && manhattan > 1) continue;", "if (manhattan > 1) continue;"),
    "transposed_conv_weight": ("out[o] += in[c] * w[c * co + o];", "out[o] += in[c] * w[o * ci + c];"),
    "unflipped_conv_adjoint": ("const int X = xx - dx, Y = yy - dyy, Z = z - dz;",
                               "const int X = xx + dx, Y = yy + dyy, Z = z + dz;"),
    "cutoff_wrong_beta_factor": ("((2.0 * a + gamma) - 3.0 * beta)", "((2.0 * a + gamma) - 2.0 * beta)"),
    "cutoff_of_signed_phi": ("orc_cutoff(fabs(phi[i]), beta, gamma)", "orc_cutoff(phi[i], beta, gamma)"),
    "reinit_upwind_swapped": ("if (di > 0.0) {", "if (di < 0.0) {"),
    "reinit_S_without_dx": ("(g * g) * (h * h)", "(g * g)"),
    "reinit_source_sign": ("di - dtau * (S * (g - 1.0))", "di + dtau * (S * (g - 1.0))"),
    "region_n_missing_z_plus": ("if (!in && z < nz - 1) in = fabs(phi[idx3(nx, ny, x, y, z + 1)]) < gamma;", ""),
    "clamp_lower_side_missing": ("if (d[i] < -gamma) d[i] = -gamma;\n        else ", ""),
}

# slips in the corrector's numpy definitions (oracle/__init__.py)
PY_MUTATIONS = {
    "feature_step_channel_sign": ("(phit - phi) / h], axis=-1)", "(phi - phit) / h], axis=-1)"),
    "feature_clamp_missing": ("np.clip(phi / h, -FEATURE_CLAMP, FEATURE_CLAMP)", "phi / h"),
    "correction_without_h": ("float(h) * _f64(z)", "_f64(z)"),
    "check_not_strict": ("np.max(np.abs(c)) > float(dt) * float(M)", "np.max(np.abs(c)) >= float(dt) * float(M)"),
    "check_lets_nan_through": ("if not np.all(np.isfinite(c)):\n        return True\n", ""),
    "fallback_keeps_correction": ("(phit if rejected else phit + corr)", "(phit + corr)"),
    "mse_gradient_factor": ("2.0 * r / cnt", "r / cnt"),
    "mse_tube_not_strict": ("mask = np.abs(_f64(phi)) < gamma", "mask = np.abs(_f64(phi)) <= gamma"),
    "adam_no_bias_correction": ("mh = m / (1.0 - beta1 ** t)", "mh = m"),
    "adam_betas_swapped": ("m = beta1 * _f64(m) + (1.0 - beta1) * g", "m = beta1 * _f64(m) + (1.0 - beta2) * g"),
}


def _run_pins_with(tmp_path, fname, old, new):
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(old) >= 1, old
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (tmp_path / "oracle" / fname).write_text(src.replace(old, new, 1))
    shutil.copytree(os.path.join(ROOT, "paper_1612_04040_b300"), tmp_path / "paper_1612_04040_b300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "_build", "csrc"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           "tests/test_oracle_pins.py", "tests/test_oracle_learned_pins.py",
                           "tests/test_oracle_local_pins.py", "tests/test_oracle_learned_step_pins.py",
                           "tests/test_golden_cpu.py"],
                          cwd=tmp_path, capture_output=True, text=True, timeout=900)


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    r = _run_pins_with(tmp_path, "levelset_oracle.c", old, new)
    assert r.returncode != 0, "mutation %s was not caught:\n%s" % (name, r.stdout[-1500:])


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_corrector_mistake_is_caught(name, tmp_path):
    old, new = PY_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert src.count(old) == 1, name
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (tmp_path / "oracle" / "__init__.py").write_text(src.replace(old, new, 1))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_learned_step_pins.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutation %s was not caught:\n%s" % (name, r.stdout[-1500:])
