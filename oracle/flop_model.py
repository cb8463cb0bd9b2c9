"""Algorithmic-work model of the likelihood hot path: the oracle's own operations per active
(sample, mode, bin) unit and per active (sample, detector, bin), counted with its
operation-counting scalar (or_op_count) on the benchmark workload. TEST/MEASUREMENT
INFRASTRUCTURE: it calls only oracle/ (and the seeded input generators).

    python oracle/flop_model.py        # prints the model as one JSON line

The counts are those of the oracle's plain formulation: every unit evaluates its mode's waveform
and t_f (by a dual number), the orbit, six independent link responses (each with its own unit
vector, 3x3 contraction and exponential), the mode's -2Y_lm by the Wigner-d sum and the TDI
polynomial; each active bin adds the A/E/T combination and the three channels' likelihood terms.
Elementary flops are add/sub/mul/div (an FMA of the library counts two); math-library calls are
reported separately and, for a single figure, weighted 20 flops each (a degree-9 polynomial by
Horner's rule plus its reduction) -- a stated convention, not a measurement.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402
from paper_2602_12011_gb300 import workloads as W  # noqa: E402

MATH_CALL_FLOPS = 20.0
ELEMENTARY = ("add", "mul", "div", "sqrt")
MATH = ("sincos", "exp", "log", "cbrt", "pow")


def model(n_samples: int = 16) -> dict:
    wl = W.batch_hm(1024)
    det, T, k0, nb = wl["dets"][0]
    f = (k0 + np.arange(nb)) / T
    th = wl["theta"]
    order = np.argsort(th[:, 0])
    pick = order[np.linspace(0, th.shape[0] - 1, n_samples).astype(int)]
    units = bins = 0.0
    acc_u = {k: 0.0 for k in O.OP_NAMES}
    acc_b = {k: 0.0 for k in O.OP_NAMES}
    for s in pick:
        r = O.op_count(det, th[s], wl["mode_mask"], f, T=T)
        units += r["units"]
        bins += r["bins"]
        for k in O.OP_NAMES:
            acc_u[k] += r["per_unit"][k] * r["units"]
            acc_b[k] += r["per_bin"][k] * r["bins"]
    per_unit = {k: acc_u[k] / units for k in O.OP_NAMES}
    per_bin = {k: acc_b[k] / bins for k in O.OP_NAMES}
    elem_u = sum(per_unit[k] for k in ELEMENTARY)
    math_u = sum(per_unit[k] for k in MATH)
    elem_b = sum(per_bin[k] for k in ELEMENTARY)
    return {"workload": wl["name"], "samples": int(n_samples), "units": units, "bins": bins,
            "flops_per_unit": elem_u, "math_calls_per_unit": math_u,
            "flops_per_unit_with_math": elem_u + MATH_CALL_FLOPS * math_u,
            "flops_per_bin": elem_b, "bins_per_unit": bins / units,
            "per_unit": per_unit, "per_bin": per_bin, "math_call_flops": MATH_CALL_FLOPS}


if __name__ == "__main__":
    print(json.dumps(model()))
