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
import math
import time

import numpy as np

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


#: surface tension of the A/B interface (G_c = 2.5, densities 1 / 0.006):
#: the slope of the Laplace law Delta p = gamma / R measured on settled
#: drops of three radii
GAMMA = 0.144


def _fit_window(t, z, t_lo, z_hi):
    """Indices of the samples in the linear Washburn regime: after t_lo,
    before the front passes z_hi and up to its farthest advance (a front
    that stalls, the section narrowing, and then recedes has left the
    regime), finite."""
    t = np.asarray(t, float)
    z = np.asarray(z, float)
    ok = np.isfinite(z) & (t >= t_lo)
    past = np.flatnonzero(np.isfinite(z) & (z >= z_hi))
    if past.size:
        ok &= np.arange(z.size) < past[0]
    if ok.any():
        top = np.flatnonzero(ok)[np.argmax(z[ok])]
        ok &= np.arange(z.size) <= top
    return np.flatnonzero(ok)


def capillary_report(res: dict, t_lo: int = 16000,
                     margin: float = 30.0) -> dict:
    """Eq. 1 analysis of capillary_runs' series (paper Sec. III, Figs. 2 and
    4): the least-squares front speed v over the linear regime (from t_lo,
    about twice the viscous time rho H^2 / (12 mu), until the front comes
    within `margin` of the advance the A reservoir can feed, X_r (H + 2) /
    H); the k_r = 0 run calibrates gamma cos(theta_0) / mu through Eq. 1
    with r_eff = H / 2 (reading c16), and every run's r_eff follows from
    its own v (lbm_fit_reff).  Also: Eq. 1's speed with the Laplace-law
    gamma and the 30-degree contact angle, against the k_r = 0 speed."""
    H, L = res["H"], res["L"]
    x_res = 256  # the paper-scale capillary's reservoir
    z_cap = x_res * (H + 2) / H
    mu = 1.0 * (1.0 - 0.5) / 3.0  # rho nu, tau = 1
    runs = {r["k_r"]: r for r in res["runs"]}
    out = {"H": H, "L": L, "fit_t_from": t_lo, "fit_z_below": z_cap - margin,
           "reservoir_advance": z_cap, "runs": []}
    speeds = {}
    for k, r in sorted(runs.items()):
        ser = r["series"]
        idx = _fit_window(ser["step"], ser["front"], t_lo, z_cap - margin)
        t = np.asarray(ser["step"], float)[idx]
        z = np.asarray(ser["front"], float)[idx]
        speeds[k] = float(np.polyfit(t, z, 1)[0]) if idx.size >= 2 else float("nan")
    v0 = speeds.get(0.0, float("nan"))
    gamma_cos = 6.0 * mu * L * v0 / H  # Eq. 1 with r_eff = H / 2 at k_r = 0
    v_eq1 = GAMMA * H * math.cos(math.radians(30.0)) / (6.0 * mu * L)
    out["v_k0"] = v0
    out["v_eq1_laplace_30deg"] = v_eq1
    out["v_k0_over_eq1"] = v0 / v_eq1
    for k, r in sorted(runs.items()):
        ser = r["series"]
        zs = np.asarray(ser["front"], float)
        fin = np.flatnonzero(np.isfinite(np.asarray(ser["mass_a"], float)))
        last = int(fin[-1]) if fin.size else 0
        idx = _fit_window(ser["step"], ser["front"], t_lo, z_cap - margin)
        reff = float("nan")
        if idx.size >= 2:
            reff = lbm.fit_reff(np.asarray(ser["step"], float)[idx],
                                zs[idx], gamma_cos, mu, L, 1.0)
        bad = np.flatnonzero(~np.isfinite(np.asarray(ser["mass_a"], float)))
        row = {"k_r": k, "v": speeds[k], "r_eff": reff,
               "fit_samples": int(idx.size),
               "fit_until_step": int(ser["step"][idx[-1]]) if idx.size else None,
               "closure_step": r["closure_step"],
               "first_nonfinite_step": int(ser["step"][bad[0]]) if bad.size else None,
               "last_finite_step": int(ser["step"][last])}
        for key in ("r_min", "r_h", "r_ave", "delta_e", "precip_mass"):
            row[key + "_at_fit_end"] = float(ser[key][idx[-1]]) if idx.size else None
            row[key + "_last"] = float(ser[key][last])
        row["front"] = {int(ser["step"][i]): float(zs[i])
                        for i in range(len(zs)) if int(ser["step"][i]) % 20000 == 0}
        out["runs"].append(row)
    return out


def compare_storages(a: dict, b: dict) -> dict:
    """FP16 against FP32 (or any two capillary_runs results): per reaction
    rate, the largest front difference over the samples where both are
    finite, and the closure steps."""
    out = []
    for ra, rb in zip(a["runs"], b["runs"]):
        za = np.asarray(ra["series"]["front"], float)
        zb = np.asarray(rb["series"]["front"], float)
        n = min(za.size, zb.size)
        ok = np.isfinite(za[:n]) & np.isfinite(zb[:n])
        d = np.abs(za[:n] - zb[:n])[ok]
        out.append({"k_r": ra["k_r"], "front_max_abs_diff": float(d.max()) if d.size else None,
                    "samples": int(ok.sum()),
                    "closure_step": [ra["closure_step"], rb["closure_step"]]})
    return {"runs": out}


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
    steps = int(sys.argv[3]) if len(sys.argv) > 3 and what != "capillary-report" else 20000
    if what == "capillary":
        print(json.dumps(capillary_runs(steps=steps, precision=prec)))
    elif what == "capillary-report":
        # experiments capillary-report FP32.json FP16.json
        a, b = (json.load(open(f)) for f in sys.argv[2:4])
        print(json.dumps({"fp32": capillary_report(a), "fp16": capillary_report(b),
                          "fp16_vs_fp32": compare_storages(a, b)}, indent=1))
    else:
        r = preform_run(steps=steps, precision=prec)
        print(json.dumps({k: v for k, v in r.items() if k != "series"}))
        for row in r["series"]:
            print(json.dumps(row))
