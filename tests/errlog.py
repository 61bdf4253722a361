"""Measured parity errors of the GPU path against the FP64 oracle, collected
while the parity tests run and written out at the end of the session (to the
JSON file named by the environment variable PTG_ERROR_REPORT, when set).

Each entry is keyed by (configuration, method, output dtype, launch
configuration) and holds the largest |gpu - oracle| over the compared samples,
that error divided by the total amplitude A_tot = sum_i p^i (the unit of the
FP32 bar, 2e-6 x A_tot), the number of samples compared, and for FP16 output
the largest ratio of the error to its bound (FP32 bar + half an FP16 ulp)."""
from __future__ import annotations

import json
import os

REPORT = {}


def record(config: str, method: str, dtype: str, err: float, a_tot: float, n: int, launch: str = "",
           bound_ratio: float | None = None) -> None:
    key = "|".join([config, method, dtype] + ([launch] if launch else []))
    e = {"max_abs_err": float(err), "err_over_atot": float(err) / a_tot, "samples": int(n)}
    if bound_ratio is not None:
        e["max_err_over_bound"] = float(bound_ratio)
    old = REPORT.get(key)
    if old is None or e["max_abs_err"] > old["max_abs_err"]:
        REPORT[key] = e


def write(path: str | None = None) -> None:
    path = path or os.environ.get("PTG_ERROR_REPORT")
    if not path or not REPORT:
        return
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(dict(sorted(REPORT.items())), f, indent=1)
