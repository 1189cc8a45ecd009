"""The pins must catch plausible mistakes: each case plants one mistake in a
copy of the oracle's C source (on the CPU), builds it, and checks that the
pin suite fails against it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qt_oracle.c")

MUTATIONS = {
    "transposed_matrix": ("a[i] = U[0] * x0 + U[1] * x1;\n        a[j] = U[2] * x0 + U[3] * x1;",
                          "a[i] = U[0] * x0 + U[2] * x1;\n        a[j] = U[1] * x0 + U[3] * x1;"),
    "dropped_control": ("        if (((uint64_t)i & cmask) != cmask) continue;\n        int64_t j",
                        "        int64_t j"),
    "ry_sign": ("U[0] = c; U[1] = -s; U[2] = s; U[3] = c;", "U[0] = c; U[1] = s; U[2] = -s; U[3] = c;"),
    "u3_phase": ("U[2] = cexp(I * p) * s;", "U[2] = cexp(I * l) * s;"),
    "t_angle": ("U[0] = 1; U[3] = cexp(I * M_PI / 4.0);", "U[0] = 1; U[3] = cexp(I * M_PI / 8.0);"),
    "swap_visits_twice": ("if ((uint64_t)i & (b0 | b1)) continue;", "if ((uint64_t)i & b0) continue;"),
    "rz_half_angle": ("U[0] = cexp(-I * t / 2.0); U[3] = cexp(I * t / 2.0);",
                      "U[0] = cexp(-I * t); U[3] = cexp(I * t);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "qt_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", str(mutated), "-o", str(so), "-lm"])
    env = dict(os.environ, QT_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
