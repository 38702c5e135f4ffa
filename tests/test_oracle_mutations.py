"""The pins must catch plausible mistakes.  Each case below plants one mistake
in a temporary copy of the oracle's C source, builds it, and runs the pin
suite against it in a child process: the suite has to fail."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "grbk_oracle.c")

MUTANTS = {
    "x_update_sign": ("X[row * q + j] += c * A[ik * p + row] * w[j];",
                      "X[row * q + j] -= c * A[ik * p + row] * w[j];"),
    "sample_by_weighted_residual": ("                run += s[i];\n                last = i;\n                double d = fabs(run - target) / SJ;",
                                    "                run += r[i] * (SJ / SJ);\n                last = i;\n                double d = fabs(run - target) / SJ;"),
    "threshold_weights_swapped": ("t = theta * rmax + (1.0 - theta) * (S / F);",
                                  "t = (1.0 - theta) * rmax + theta * (S / F);"),
    "threshold_mean_over_m": ("t = theta * rmax + (1.0 - theta) * (S / F);",
                              "t = theta * rmax + (1.0 - theta) * (S / (double)m);"),
    "residual_update_drops_step": ("R[i * n + l] -= c * g[i] * h[l];",
                                   "R[i * n + l] -= alpha * g[i] * h[l];"),
    "gram_offdiagonal_halved": ("acc += A[i * p + c] * A[j * p + c];\n                GA[i * m + j] = acc;",
                                "acc += A[i * p + c] * A[j * p + c] * (i == j ? 1.0 : 0.5);\n                GA[i * m + j] = acc;"),
    "philox_swapped_words": ("uint64_t y0 = hi1 ^ x1 ^ k0;", "uint64_t y0 = hi0 ^ x1 ^ k0;"),
    "uniform_low_bits": ("(double)(out[0] >> 11) * 0x1.0p-53;\n}\n\n/* The extended",
                         "(double)(out[1] >> 11) * 0x1.0p-53;\n}\n\n/* The extended"),
    "extended_residual_sign": ("R[i * n + l] += A[i * p + j] * zz[l];", "R[i * n + l] -= A[i * p + j] * zz[l];"),
    "extended_column_step_sign": ("Y[i * n + l] -= A[i * p + j] * zz[l];", "Y[i * n + l] += A[i * p + j] * zz[l];"),
    "extended_column_stream": ("uint64_t ctr[4] = {k, sys, 1, 0}", "uint64_t ctr[4] = {k, sys, 0, 0}"),
    "pick_first_not_exceeding": ("if (ik < 0 && run > target) ik = i;\n            }\n            if (ik < 0) ik = last;\n        } else if (variant == OR_MWRBK)",
                                 "if (ik < 0 && run >= 0.5 * target) ik = i;\n            }\n            if (ik < 0) ik = last;\n        } else if (variant == OR_MWRBK)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = oracle.compile_c(str(mut), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, GRBK_ORACLE_SO=so)
    proc = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                           "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)
    assert proc.returncode != 0, f"pins did not catch mutant {name}:\n{proc.stdout[-2000:]}"
