"""Longer runs on the GPU that report the paper's quantities over time.

capillary_runs: the paper-scale single capillary (4096 x 128: H = 126,
L = 3712) at several reaction rates in one batch, the front position and
the radii of Sec. III (Eq. 1, Figs. 2 and 4) every `every` steps until
every lattice has closed or the step budget is spent.

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


def capillary_runs(steps: int = 200_000, every: int = 500,
                   k_values=(0.0, 1e-4, 1e-3),
                   precision: str = "fp32") -> dict:
    """One batch of paper-scale capillaries, one per reaction rate; returns
    the time series of the observables of each (front z, r_min, r_h,
    r_ave, Delta e, precipitated mass, closure step, masses)."""
    pairs = [I.config_paper_scale(k_r=k)[:2] for k in k_values]
    geoms = [g for g, _ in pairs]
    params = [p for _, p in pairs]
    s = lbm.Solver(geoms, params, precision)
    keys = ("front", "r_min", "r_h", "r_ave", "delta_e", "precip_mass",
            "closed", "mass_a", "mass_b", "ledger_a", "ledger_b")
    series = [{k: [] for k in ("step",) + keys} for _ in k_values]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(every, steps - done)
        s.step(n)
        done += n
        obs = s.observables(allow_nan=True)
        for j, o in enumerate(obs):
            series[j]["step"].append(done)
            for k in keys:
                series[j][k].append(float(o[k]))
        if all(o["closure_step"] >= 0 for o in obs):
            break
    wall = time.perf_counter() - t0
    obs = s.observables(allow_nan=True)
    s.close()
    g = geoms[0]
    return {"precision": precision, "nx": g.nx, "ny": g.ny,
            "H": g.ny - 2, "L": g.cap_x1 - g.cap_x0, "every": every,
            "steps": done, "wall_s": wall,
            "runs": [{"k_r": k, "closure_step": int(o["closure_step"]),
                      "nonfinite": int(o["nonfinite"]), "series": ser}
                     for k, o, ser in zip(k_values, obs, series)]}


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
    what = sys.argv[1] if len(sys.argv) > 1 else "preform"
    prec = sys.argv[2] if len(sys.argv) > 2 else "fp16"
    steps = int(sys.argv[3]) if len(sys.argv) > 3 else 20000
    if what == "capillary":
        print(json.dumps(capillary_runs(steps=steps, precision=prec)))
    else:
        r = preform_run(steps=steps, precision=prec)
        print(json.dumps({k: v for k, v in r.items() if k != "series"}))
        for row in r["series"]:
            print(json.dumps(row))
