"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/resample_oracle.c (on the
CPU, in a temporary directory), builds it, and runs the pin suite against
that build: the suite has to fail. The Python-layer cases plant the mistake
in a copy of oracle/oracle.py instead (run against the real C library).
Every planted mistake keeps all memory accesses in bounds.
"""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "oracle" / "resample_oracle.c"

MUTANTS = {
    "keys_coefficient": ("return (a + 2.0) * x * x * x - (a + 3.0) * x * x + 1.0;",
                         "return (a + 2.0) * x * x * x - (a + 2.0) * x * x + 1.0;"),
    "dropped_cubic_tap": ("w[3] = keys(2.0 - t, a);", "w[3] = 0.0;"),
    "half_pixel_offset": ("num = (2 * j + 1) * n - m;", "num = (2 * j) * n - m;"),
    "wrong_low_clamp": ("if (i < 0) return 0;", "if (i < 0) return 1 % n;"),
    "swapped_axis_weights": ("acc += wy[p] * wx[q] * src[(iy[p] * W + ix[q]) * C + c];",
                             "acc += wx[p % nx] * wy[q % ny] * src[(iy[p] * W + ix[q]) * C + c];"),
    "adjoint_weight_index": ("gx[(iy[p] * W + ix[q]) * C + c] += wy[p] * wx[q] * g;",
                             "gx[(iy[p] * W + ix[q]) * C + c] += wy[q % ny] * wx[p % nx] * g;"),
    "bilinear_weights_swapped": ("w[0] = 1.0 - t;\n        w[1] = t;",
                                 "w[0] = t;\n        w[1] = 1.0 - t;"),
    "u8_round_half_up": ("out[k] = (uint8_t)nearbyint(x);", "out[k] = (uint8_t)floor(x + 0.5);"),
    "f16_round_half_away": ("double r = nearbyint(d / q) * q;", "double r = round(d / q) * q;"),
    "nearest_half_pixel": ("i = floor_div((2 * j + 1) * n, 2 * m);",
                           "i = floor_div((2 * j + 1) * n - m, 2 * m);"),
    "align_corners_denominator": ("        den = m - 1;\n", "        den = m;\n"),
    "align_corners_nearest_floor": ("i = floor_div(2 * num + den, 2 * den);", "i = floor_div(2 * num, 2 * den);"),
}


PY_SRC = ROOT / "oracle" / "oracle.py"
PY_MUTANTS = {
    "normalize_channel_order": ("out[n] = ((y - m) / s).transpose(2, 0, 1)",
                                "out[n] = ((y - m[::-1]) / s).transpose(2, 0, 1)"),
    "normalize_scale_not_divide": ("out[n] = ((y - m) / s).transpose(2, 0, 1)",
                                   "out[n] = ((y - m) * (1.0 / s[0])).transpose(2, 0, 1)"),
    "normalize_planar_axes": ("out[n] = ((y - m) / s).transpose(2, 0, 1)",
                              "out[n] = ((y - m) / s).transpose(2, 1, 0).reshape(C, Ho, Wo)"),
    "aa_adjoint_axes_swapped": ('return np.einsum("ih,ncij,jw->nchw", Ay, np.asarray(gy, np.float64), Ax, optimize=True)',
                                'return np.einsum("ih,ncij,jw->nchw", Ay, np.asarray(gy, np.float64), Ax[::-1], optimize=True)'),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_planted_python_mistake(name, tmp_path, oracle):
    old, new = PY_MUTANTS[name]
    text = PY_SRC.read_text()
    assert text.count(old) == 1, name
    src = tmp_path / "oracle_mutant.py"
    src.write_text(text.replace(old, new))
    env = dict(os.environ, RESAMPLE_ORACLE_PY=str(src), RESAMPLE_ORACLE_LIB=str(oracle.build()))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        str(ROOT / "tests" / "test_oracle_pins.py")],
                       env=env, cwd=str(ROOT), capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    text = SRC.read_text()
    assert text.count(old) == 1, name
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                    str(src), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, RESAMPLE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        str(ROOT / "tests" / "test_oracle_pins.py")],
                       env=env, cwd=str(ROOT), capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}"
