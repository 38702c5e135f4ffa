"""Writes oracle_rows_small.json: the FP64 oracle's selected rows and ||R^k||_F^2
for the first 200 iterations of every variant on the 200x100 / 80x150 system of
workloads.config_small(), with the step alpha stored as used (so the fixture
depends on no library routine).  Calls only oracle/ and workloads/.

    python tests/golden/make_oracle_rows.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

def x0_bk():
    """X^0 of the ME-BK case (the cyclic method from a nonzero start)."""
    return workloads.rng(77).standard_normal((100, 80))


CASES = [("grbk", 0.5), ("rgrbk", 0.3), ("rgrbk", 0.8), ("mwrbk", 1.0), ("rbk", 0.5), ("bk", 0.5)]
MAXIT, SEED = 200, 7


def main():
    A, B, C, _ = workloads.config_small()
    alpha = 1.0 / oracle.spectral_norm_sq(B)
    out = {"system": "workloads.config_small(): A 200x100, B 80x150, C = A X* B", "alpha": alpha.hex(),
           "seed": SEED, "maxit": MAXIT, "mode": "FACTORED", "cases": []}
    for variant, theta in CASES:
        X0 = x0_bk() if variant == "bk" else None
        r = oracle.solve(A, B, C, variant, theta=theta, alpha=alpha, X0=X0, seed=SEED, maxit=MAXIT,
                         mode=oracle.MODE_FACTORED)
        out["cases"].append({"variant": variant, "theta": theta, "x0": "workloads.rng(77) N(0,1)" if X0 is not None else "0",
                             "rows": [int(i) for i in r["rows"]], "S": [float(v).hex() for v in r["S"]]})
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_rows_small.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
