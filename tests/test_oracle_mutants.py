"""The oracle's pins are not vacuous: each plausible mistake planted in a
copy of the oracle's C source (a flipped sign, a dropped term, a wrong index)
makes at least one pin test fail.  Mistakes are planted on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "glu_oracle.c")

MUTANTS = {
    "update_sign": ("x[ri[q]] = x[ri[q]] - prod;", "x[ri[q]] = x[ri[q]] + prod;"),
    "drop_division": ("lu_val[p] = x[ri[p]] / piv;", "lu_val[p] = x[ri[p]];"),
    "wrong_multiplier": ("double xk = x[k];", "double xk = x[j];"),
    "skip_first_update": ("for (int64_t p = cp[j]; p < dpos[j]; p++) {\n            int32_t k = ri[p];",
                          "for (int64_t p = cp[j] + 1; p < dpos[j]; p++) {\n            int32_t k = ri[p];"),
    "reach_through_u": ("spos[top] = (w < j) ? lbeg[w] : 0;", "spos[top] = (w < j) ? cp[w] : 0;"),
    "no_look_left": ("if (mark[i] != k) { mark[i] = k; tmp[m++] = i; }\n        }\n        qsort",
                     "if (0) { mark[i] = k; tmp[m++] = i; }\n        }\n        qsort"),
    "no_empty_l_test": ("if (i < k && has_l[i] && mark[i] != k)", "if (i < k && mark[i] != k)"),
    "level_no_increment": ("if (level_of[di[p]] + 1 > lv) lv = level_of[di[p]] + 1;",
                           "if (level_of[di[p]] > lv) lv = level_of[di[p]];"),
    "solve_no_pivot_divide": ("z[j] = z[j] / lu_val[dpos[j]];", "z[j] = z[j];"),
    "solve_forward_sign": ("z[ri[p]] = z[ri[p]] - lu_val[p] * zj;\n        }\n        for (int32_t j = n - 1",
                           "z[ri[p]] = z[ri[p]] + lu_val[p] * zj;\n        }\n        for (int32_t j = n - 1"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                           "-o", str(so), str(mpath), "-lm"])
    env = dict(os.environ, GLU_ORACLE_LIB=str(so), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
