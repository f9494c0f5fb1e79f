"""Stability of the collision operators at low resolution: the classical SRT operator with the
second-order equilibrium, TRT, and the paper's CHM-MRT on seeded synthetic aneurysms.

    python -m paper_2101_11107_gb300.stability_study --out stability.json
    python -m paper_2101_11107_gb300.stability_study --small --out small.json

The paper (Sec. 2.1.2, 3.1, 3.4) reports that the SRT operator with the second-order
equilibrium becomes unstable at the small relaxation times of under-resolved hemodynamics
(tau 0.503 on its coarse patient grid), while CHM-MRT keeps running.  Here each operator runs
the same case -- the synthetic aneurysm at a given box edge and Reynolds number, with its
pulsatile inlet, Bouzidi walls and outlet absorbing layer -- for a number of inflow periods;
every `check` steps the FP64 diagnostics report whether any population is non-finite, and
max |u| (a run whose max |u| exceeds 0.35, i.e. Mach ~0.6, is counted as blown up too).
Reported per operator and case: the step at which the run failed (or None), max |u| over the
run, and the time per step.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

MODELS = ("srt2", "trt2", "chm")
U_BLOWUP = 0.35


def run_case(g, collision, steps, check, storage="fp32"):
    import torch

    from . import lbm

    dom = lbm.Domain.from_geometry(g, storage=storage, collision=collision)
    umax, failed_at = 0.0, None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    done = 0
    while done < steps:
        n = min(check, steps - done)
        e0.record(dom.stream)
        dom.step(n)
        e1.record(dom.stream)
        d = dom.diagnostics(raise_unstable=False)
        ms += e0.elapsed_time(e1)
        done += n
        if d["n_nonfinite"] > 0 or not np.isfinite(d["max_u"]) or d["max_u"] > U_BLOWUP:
            failed_at = done
            break
        umax = max(umax, float(d["max_u"]))
    dom.close()
    return {"failed_at_step": failed_at, "steps_run": done, "max_u": umax,
            "ms_per_step": ms / max(done, 1)}


def run(edges, reynolds, seeds, periods, period_at_256=4000.0, check=100, log=print):
    from . import inputs as I

    out = {"reynolds": reynolds, "periods": periods, "check_every": check, "cases": []}
    for edge in edges:
        period = period_at_256 * edge / 256.0  # acoustic scaling: half the period at half the edge
        for seed in seeds:
            g = I.aneurysm(seed, edge=edge, period=period, reynolds=reynolds, wave_seed=seed)
            case = {"edge": edge, "seed": seed, "tau": g.tau, "fluid_cells": g.nfluid, "steps": int(periods * period)}
            for m in MODELS:
                case[m] = run_case(g, m, case["steps"], check)
                log(f"edge {edge} seed {seed} tau {g.tau:.5f} {m}: {case[m]}")
            out["cases"].append(case)
    for m in MODELS:
        out[f"{m}_failed"] = sum(c[m]["failed_at_step"] is not None for c in out["cases"])
    out["n_cases"] = len(out["cases"])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out", default=None)
    ap.add_argument("--small", action="store_true", help="the 64^3 / 128^3 quick version")
    ap.add_argument("--reynolds", type=float, default=300.0)
    ap.add_argument("--periods", type=float, default=2.0)
    a = ap.parse_args(argv)
    from . import build as lib_build

    lib_build.build()
    edges = (64, 128) if a.small else (128, 256)
    seeds = (200, 201) if a.small else (200, 201, 202, 203)
    res = run(edges, a.reynolds, seeds, a.periods)
    s = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(json.dumps({k: v for k, v in res.items() if k != "cases"}))


if __name__ == "__main__":
    main()
