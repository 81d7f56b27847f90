"""Longer runs on the GPU that report the paper's quantities over time.

preform_run: reactive infiltration of the synthetic carbon preform (the
paper's closing remark, Sec. IV, names the porosity of the preform as the
next question): per-component mass balance (fluid + what growth moved to the
ledger) and the growth of the solid fraction, in FP32 or FP16 storage.
"""
from __future__ import annotations

import json
import time

from . import inputs as I
from . import lbm


def preform_run(steps: int = 20000, every: int = 2000,
                precision: str = "fp16", n: int = 2048,
                k_r: float = 1e-3) -> dict:
    geom = I.preform(n=n)
    mp = I.ModelParams(g_ads=I.G_ADS_30, k_r=k_r, inlet=1)
    s = lbm.Solver(geom, mp, precision)
    solid0 = int(geom.solid.sum())
    rows = []
    o0 = s.observables()[0]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        s.step(k)
        done += k
        o = s.observables(allow_nan=True)[0]
        solid = int(s.solid_mask().sum())
        rows.append({
            "step": done,
            "mass_a_total": o["mass_a"] + o["ledger_a"],
            "mass_b_total": o["mass_b"] + o["ledger_b"],
            "precip_mass": o["precip_mass"],
            "solid_fraction": solid / geom.solid.size,
            "new_solid_nodes": solid - solid0,
            "nonfinite": o["nonfinite"],
        })
    wall = time.perf_counter() - t0
    ma0 = o0["mass_a"] + o0["ledger_a"]
    mb0 = o0["mass_b"] + o0["ledger_b"]
    return {
        "precision": precision, "n": n, "steps": steps, "k_r": k_r,
        "solid_fraction_region": geom.extra["solid_fraction"],
        "mass_a_rel_drift": (rows[-1]["mass_a_total"] - ma0) / ma0,
        "mass_b_rel_drift": (rows[-1]["mass_b_total"] - mb0) / mb0,
        "wall_s": wall, "series": rows,
    }


if __name__ == "__main__":
    import sys
    prec = sys.argv[1] if len(sys.argv) > 1 else "fp16"
    steps = int(sys.argv[2]) if len(sys.argv) > 2 else 20000
    r = preform_run(steps=steps, precision=prec)
    print(json.dumps({k: v for k, v in r.items() if k != "series"}))
    for row in r["series"]:
        print(json.dumps(row))
