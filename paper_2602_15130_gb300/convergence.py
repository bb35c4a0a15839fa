"""Refinement studies of Sec. 5 on the GPU: observed convergence rates of the
MMS error norms next to the rates the error analysis of Sec. 4 predicts.

Every run goes through the C ABI (``Pic``); this module only chooses the
configurations, collects the norms at t = T and fits the rates
p = log(eps_l / eps_{l+1}) / log(h_l / h_{l+1}) between consecutive levels
and by least squares over all levels.

Studies:
  table1-collisional    Table 1, s = 7, r = 5: isolated collisions (with and
                        without the injected Errors 1 and 2), uncoupled,
                        both one-way couplings and the coupled case, with
                        the manufactured anisotropic scattering of Sec. 5.1.
  table1-collisionless  Table 1, s = 5: both one-way couplings, coupled.
  paper-collisional     the paper's own problem of Sec. 5.2 (non-Maxwellian
                        f_v with vh(t), per-axis f_x, odd-power sigma with
                        its exact source) on the Table 1 schedule, s = 7,
                        r = 5, FP64: uncoupled, one-way and coupled.
  paper-collisionless   the same problem without collisions, s = 5.
  refine                the fixed-32-particles-per-cell sweep (n = 8..128,
                        dt = 0.02 / 2^l, T = 0.5): s = 3 and r = 0, so the
                        coupled collisionless rate is 1 and the collisional
                        error is not expected to converge.

Usage: python -m paper_2602_15130_gb300.convergence --study table1-collisional
       [--levels 0 1 2 3 4] [--precision fp64|mixed] [--out results.json]
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import Pic, _lib, workloads

QUANTITIES = ["x", "y", "z", "u", "v", "w", "phi"]

ISO, E1, E2, ANG, ANI = (_lib.PIC_VERIFY_ISOLATE, _lib.PIC_VERIFY_ERROR1, _lib.PIC_VERIFY_ERROR2,
                         _lib.PIC_VERIFY_ANGLES, _lib.PIC_VERIFY_ANISO)

# variant name -> (config overrides, predicted rates {group: rate or None})
# groups: "x" = positions, "v" = velocities, "phi" = potential; None = no
# convergence predicted. eps_2 and eps_inf share the prediction unless a
# "<group>2" key gives the eps_2 one.
TABLE1_COLLISIONAL = {
    "isolated": (dict(verify=ISO | ANG | ANI, couple_qm_zero=1), {"x": 2, "v": 2, "x2": 2.5, "v2": 2.5}),
    "isolated_error1": (dict(verify=ISO | ANG | ANI | E1, couple_qm_zero=1), {"x": None, "v": None}),
    "isolated_error2": (dict(verify=ISO | ANG | ANI | E2, couple_qm_zero=1), {"x": 2, "v": 2, "x2": 2.5, "v2": 2.5}),
    "uncoupled": (dict(verify=ANI, couple_qm_zero=1, couple_q_zero=1), {"x": 2, "v": 2, "phi": 2}),
    "oneway_qm0": (dict(verify=ANI, couple_qm_zero=1), {"phi": 2}),
    "oneway_q0": (dict(verify=ANI, couple_q_zero=1), {"x": 2, "v": 2}),
    "coupled": (dict(verify=ANI), {"x": 2, "v": 2, "phi": 2}),
}
TABLE1_COLLISIONLESS = {
    "oneway_qm0": (dict(couple_qm_zero=1), {"phi": 2}),
    "oneway_q0": (dict(couple_q_zero=1), {"x": 2, "v": 2}),
    "coupled": (dict(), {"x": 2, "v": 2, "phi": 2}),
}
PAPER_COLLISIONAL = {
    "uncoupled": (dict(couple_qm_zero=1, couple_q_zero=1), {"x": 2, "v": 2, "phi": 2}),
    "oneway_q0": (dict(couple_q_zero=1), {"x": 2, "v": 2}),
    "coupled": (dict(), {"x": 2, "v": 2, "phi": 2}),
}
PAPER_COLLISIONLESS = {
    "oneway_qm0": (dict(couple_qm_zero=1), {"phi": 2}),
    "coupled": (dict(), {"x": 2, "v": 2, "phi": 2}),
}
REFINE = {
    "collisionless_uncoupled": (dict(K=0, couple_qm_zero=1, couple_q_zero=1), {"x": 2, "phi": 2}),
    "collisionless_coupled": (dict(K=0), {"x": 1, "v": 1, "phi": 1}),
    "collisional_coupled": (dict(), {"x": None, "v": None}),
}


def levels_params(study: str, level: int, overrides: dict) -> dict:
    if study == "table1-collisional":
        p = workloads.table1_level(level, collisions=True)
    elif study == "table1-collisionless":
        p = workloads.table1_level(level, collisions=False)
    elif study == "paper-collisional":
        p = workloads.paper_table1_level(level, collisions=True)
    elif study == "paper-collisionless":
        p = workloads.paper_table1_level(level, collisions=False)
    elif study == "refine":
        p = workloads.refinement_level(level)
    else:
        raise ValueError(study)
    p.update(overrides)
    return p


def run_one(p: dict, precision: str) -> dict:
    if precision == "mixed":
        p = workloads.mixed(p)
    t0 = time.perf_counter()
    # a cell that outgrows max_ppc has its collisions skipped and the steps
    # return PIC_ECAPACITY: the level runs again from the start with twice
    # the capacity (which changes no result, only which cells fit)
    for attempt in range(4):
        sim = Pic(p)
        sim.sample_mms(0.0)
        sim.set_profiling(True)
        try:
            # a diverging run (velocities past g_max run away; see the refine
            # study) ends in a non-finite field: record it instead of
            # stopping the study
            status = sim.step(int(p["steps"]), allow=(_lib.PIC_ENOCONV,))
            break
        except _lib.PicError as e:
            if e.status != _lib.PIC_ECAPACITY or attempt == 3:
                raise
            sim.close()
            p = dict(p, max_ppc=2 * int(p["max_ppc"]))
    kt = sim.kernel_times()
    err = sim.mms_error()
    st = sim.stats()
    out = {"n": p["n"], "h": 1.0 / p["n"], "n_particles": p["n_particles"], "K": p["K"], "dt": p["dt"],
           "steps": p["steps"], "eps2": err["eps2"], "epsinf": err["epsinf"], "n_coll": st["n_coll"],
           "n_cand": st["n_cand"], "cg_iters_max": st["cg_iters_max"],
           "step_kernel_ms": {k: round(v["ms"], 3) for k, v in kt.items() if v["launches"]},
           "n_gmax_exceed": st["n_gmax_exceed"], "status": _lib.STATUS[status], "max_ppc": int(p["max_ppc"])}
    if p.get("verify", 0) & ANG:
        out["angles"] = sim.angle_stats()
    out["seconds"] = time.perf_counter() - t0
    sim.close()
    return out


def observed_rates(h: list[float], e: list[float]) -> dict:
    """Pairwise orders and the least-squares slope of log e against log h."""
    pair = [math.log(e[i] / e[i + 1]) / math.log(h[i] / h[i + 1]) if e[i] > 0 and e[i + 1] > 0 else float("nan")
            for i in range(len(h) - 1)]
    ok = [i for i in range(len(h)) if e[i] > 0]
    fit = float(np.polyfit(np.log([h[i] for i in ok]), np.log([e[i] for i in ok]), 1)[0]) if len(ok) >= 2 else None
    return {"pairwise": pair, "fit": fit}


def group_error(rec: dict, norm: str, group: str) -> float:
    e = rec[norm]
    if group == "x":
        return max(e["x"], e["y"], e["z"]) if norm == "epsinf" else math.sqrt((e["x"] ** 2 + e["y"] ** 2 + e["z"] ** 2) / 3)
    if group == "v":
        return max(e["u"], e["v"], e["w"]) if norm == "epsinf" else math.sqrt((e["u"] ** 2 + e["v"] ** 2 + e["w"] ** 2) / 3)
    return e["phi"]


def run_study(study: str, levels: list[int], precision: str, variants: list[str] | None = None, log=print,
              save=None) -> dict:
    table = {"table1-collisional": TABLE1_COLLISIONAL, "table1-collisionless": TABLE1_COLLISIONLESS,
             "paper-collisional": PAPER_COLLISIONAL, "paper-collisionless": PAPER_COLLISIONLESS,
             "refine": REFINE}[study]
    result = {"study": study, "precision": precision, "levels": levels, "variants": {}}
    for name, (over, pred) in table.items():
        if variants and name not in variants:
            continue
        recs = []
        for l in levels:
            rec = run_one(levels_params(study, l, over), precision)
            recs.append(rec)
            result["variants"][name] = {"records": recs, "rates": {}}
            if save:
                save(result)
            log(f"[{study}/{name}] n={rec['n']} Np={rec['n_particles']} K={rec['K']} steps={rec['steps']} "
                f"eps_inf(x,v,phi)=({group_error(rec, 'epsinf', 'x'):.3e}, {group_error(rec, 'epsinf', 'v'):.3e}, "
                f"{rec['epsinf']['phi']:.3e}) {rec['seconds']:.1f}s "
                f"(dsmc {rec['step_kernel_ms'].get('dsmc', 0.0) / 1e3:.1f}s)")
        h = [r["h"] for r in recs]
        rates = {}
        for group in ("x", "v", "phi"):
            for norm in ("eps2", "epsinf"):
                e = [group_error(r, norm, group) for r in recs]
                key = group + ("2" if norm == "eps2" else "")
                rates[f"{group}_{norm}"] = {"errors": e, **observed_rates(h, e),
                                            "predicted": pred.get(key, pred.get(group, "n/a"))}
        if recs and "angles" in recs[0]:
            ncoll = [r["angles"]["n_coll"] for r in recs]
            for k in ("eps2_chi", "epsinf_chi", "eps2_eps", "epsinf_eps"):
                e = [r["angles"][k] for r in recs]
                slope = float(np.polyfit(np.log(ncoll), np.log(e), 1)[0]) if all(x > 0 for x in e) else None
                rates[f"angle_{k}"] = {"errors": e, "n_coll": ncoll, "slope_vs_ncoll": slope, "predicted": -0.5}
        result["variants"][name] = {"records": recs, "rates": rates}
        if save:
            save(result)
    return result


def format_report(res: dict) -> str:
    lines = [f"## {res['study']} ({res['precision']})"]
    for name, v in res["variants"].items():
        lines.append(f"### {name}")
        for key, r in v["rates"].items():
            if key.startswith("angle_"):
                lines.append(f"  {key:16s} slope vs N_coll {r['slope_vs_ncoll']}, predicted -0.5; "
                             f"values {', '.join(f'{x:.2e}' for x in r['errors'])}")
                continue
            pw = ", ".join(f"{x:.2f}" for x in r["pairwise"])
            fit = f"{r['fit']:.2f}" if r["fit"] is not None else "-"
            lines.append(f"  {key:12s} errors {', '.join(f'{x:.3e}' for x in r['errors'])} | "
                         f"rates {pw} | fit {fit} | predicted {r['predicted']}")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--study", required=True, choices=["table1-collisional", "table1-collisionless",
                                                          "paper-collisional", "paper-collisionless", "refine"])
    ap.add_argument("--levels", type=int, nargs="+", default=[0, 1, 2, 3, 4])
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--variants", nargs="*", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    def save(res):
        if a.out:
            with open(a.out, "w") as f:
                json.dump(res, f, indent=1)

    res = run_study(a.study, a.levels, a.precision, a.variants, log=lambda s: print(s, flush=True), save=save)
    print(format_report(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
