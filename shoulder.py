#!/usr/bin/env python
"""Shoulder-plot diagnostic of CCMC population dynamics (Sec. IV.A).

A shoulder plot follows a run grown from a small reference population at a
constant shift (the shift never starts to vary here): it plots the ratio of
the total to the reference population, N_total / N_0, against N_total.  At the
shoulder the ratio reaches a maximum, after which both populations grow at a
stable rate; the population there measures how hard the calculation is, and
a run whose reference population is too small never shows one and simply
blows up (Sec. IV.A).  Sec. IV.B-C compare the original sampler, full
non-composite sampling and full non-composite sampling with multi-spawn by
their shoulder heights (Fig. fnc).

This script runs the three samplers on one workload through the CUDA library
and reports, per sampler, the (N_total, N_0) series and the shoulder: the
largest ratio of a running median of N_total / N_0 over a window of steps,
and the population where it occurs.  A run that reaches the population cap
without the ratio falling below `drop` of its maximum afterwards is reported
as having no shoulder below the cap.

    python shoulder.py --workload ueg14_m114_ccsdt_fnc_ms --tau 0.0005 --d0 20 --cap 2e6
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SAMPLERS = {"original": (False, False), "fnc": (True, False), "fnc+multispawn": (True, True)}


def running_median(x, w: int):
    """Median of x over the trailing window of w points (shorter at the start)."""
    import numpy as np

    x = np.asarray(x, dtype=np.float64)
    return np.array([np.median(x[max(0, i - w + 1): i + 1]) for i in range(len(x))])


def shoulder_of(ntot, n0, window: int = 20, drop: float = 0.9) -> dict:
    """The shoulder of one run from its per-step N_total and N_0: the maximum
    of the running median of N_total / N_0 (window steps), the step and
    N_total where it occurs, and whether the ratio fell below drop x that
    maximum later in the run (a shoulder, rather than a run cut off while the
    ratio was still rising)."""
    import numpy as np

    ntot = np.asarray(ntot, dtype=np.float64)
    n0 = np.abs(np.asarray(n0, dtype=np.float64))
    ratio = np.where(n0 > 0, ntot / np.maximum(n0, 1e-300), np.inf)
    sm = running_median(ratio, window)
    finite = np.isfinite(sm)
    if not finite.any():
        return {"found": False, "step": None, "n_total": None, "ratio": None}
    k = int(np.argmax(np.where(finite, sm, -np.inf)))
    found = bool(np.any(sm[k + 1:] < drop * sm[k]))
    return {"found": found, "step": k, "n_total": float(ntot[k]), "ratio": float(sm[k])}


def run_sampler(ccmc, w: dict, fnc: bool, ms: bool, tau: float, d0: float, cap: float, max_steps: int,
                stream=None, chunk: int = 10, seed: int = 0):
    """Grows one run at a constant shift from d0 particles on the reference
    until N_total exceeds cap (or max_steps); returns per-step (N_total, N_0)
    after each step and how the run ended."""
    # the shift would start to vary only past 2 x cap; the run stops at cap
    over = dict(tau=tau, d0_init=d0, target_pop=2.0 * cap, fnc=fnc, multispawn=ms)
    if seed:
        over["seed"] = seed
    w = {k: v for k, v in w.items() if k != "list_capacity"}   # capacities follow the target
    ctx = ccmc.from_workload(w, stream=stream, **over)
    ntot, n0 = [], []
    try:
        while len(ntot) < max_steps:
            ctx.step(chunk)
            for r in ctx.records():
                ntot.append(r["ntot_after"] / 65536.0)
                n0.append(r["n0"] / 65536.0)
            if ntot and ntot[-1] > cap:
                break
        status = "ok"
    except ccmc.CCMCError as e:   # a blow-up past the buffers ends the run
        status = str(e)
    ctx.close()
    return ntot, n0, status


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="ueg14_m114_ccsdt_fnc_ms")
    ap.add_argument("--tau", type=float, default=0.0005)
    ap.add_argument("--d0", type=float, default=20.0)
    ap.add_argument("--cap", type=float, default=2e6, help="stop once N_total exceeds this")
    ap.add_argument("--max-steps", type=int, default=20000)
    ap.add_argument("--window", type=int, default=20)
    ap.add_argument("--samplers", default=",".join(SAMPLERS))
    ap.add_argument("--eri-scale", type=float, default=0.0, help="molecule only: scale of the two-electron integrals")
    ap.add_argument("--series", action="store_true", help="include the per-step series in the output")
    ap.add_argument("--seeds", default="", help="comma-separated Philox seeds: one run per seed and sampler, "
                                                "with the mean and spread of the shoulder heights")
    args = ap.parse_args()
    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    w = workload(args.workload)
    if args.eri_scale:
        w["eri_scale"] = args.eri_scale
    out = {"workload": args.workload, "tau": args.tau, "d0": args.d0, "cap": args.cap,
           "eri_scale": w.get("eri_scale", 1.0), "runs": {}}
    seeds = [int(x) for x in args.seeds.split(",")] if args.seeds else [0]
    for name in args.samplers.split(","):
        fnc, ms = SAMPLERS[name]
        per_seed = []
        for seed in seeds:
            ntot, n0, status = run_sampler(ccmc, w, fnc, ms, args.tau, args.d0, args.cap, args.max_steps, seed=seed)
            res = dict(shoulder_of(ntot, n0, args.window), steps=len(ntot), status=status, seed=seed,
                       n_total_last=ntot[-1] if ntot else None, n0_last=n0[-1] if n0 else None)
            if args.series:
                res["n_total"], res["n0"] = ntot, n0
            per_seed.append(res)
            print(json.dumps({name: {k: v for k, v in res.items() if k not in ("n_total", "n0")}}), flush=True)
        out["runs"][name] = per_seed if len(seeds) > 1 else per_seed[0]
        found = [r["ratio"] for r in per_seed if r["found"]]
        if len(seeds) > 1 and found:
            import numpy as np

            out.setdefault("summary", {})[name] = {
                "found": len(found), "of": len(seeds), "ratio_mean": float(np.mean(found)),
                "ratio_sd": float(np.std(found, ddof=1)) if len(found) > 1 else None}
            print(json.dumps({name: out["summary"][name]}), flush=True)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
