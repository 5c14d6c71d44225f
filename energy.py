#!/usr/bin/env python
"""Projected correlation energy of a CCMC run on the GPU (Sec. II, Eq. E_proj).

Grows the wavefunction of a workload from the reference until the shift has
varied for --equilibrate steps, then runs --steps steps and reports

  E_proj = <E_num> / <N_0>    (ratio of the means over the window)
  E_shift = <S>               (both estimate the correlation energy)

with standard errors from a Flyvbjerg-Petersen blocking analysis (the
published method the paper uses for its error bars, Computational Methods):
the series is averaged pairwise repeatedly, and the error is read where the
blocked estimate stops growing.  For the ratio, the blocked series is
E_num - E_proj N_0 (its mean is zero at the estimate; the error of E_proj is
its error divided by <N_0>).

    python energy.py --workload ueg14_m358_ccsdtq --target-pop 3e7 --steps 20000
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def blocking(x):
    """Flyvbjerg-Petersen blocking of a correlated series: the standard error
    of the mean at every blocking level, and the error read off the first
    level from which it stays within its own uncertainty of the larger ones
    (the plateau); with no plateau the largest estimate."""
    import numpy as np

    x = np.asarray(x, dtype=np.float64)
    levels = []
    while len(x) >= 16:
        n = len(x)
        se = x.std(ddof=1) / math.sqrt(n)
        levels.append((n, se, se / math.sqrt(2.0 * (n - 1))))
        x = 0.5 * (x[: n - n % 2][0::2] + x[: n - n % 2][1::2])
    if not levels:
        return float("nan"), []
    for k, (n, se, dse) in enumerate(levels):
        rest = [s for _, s, _ in levels[k + 1:]]
        if rest and all(abs(s - se) <= 2.0 * dse + 1e-300 for s in rest[:3]) and n >= 64:
            return float(se), levels
    return float(max(s for _, s, _ in levels)), levels


def projected_energy(recs):
    """(E_proj, its standard error, E_shift, its standard error) over records."""
    import numpy as np

    en = np.array([r["e_num"] for r in recs])
    n0 = np.array([r["n0"] / 65536.0 for r in recs])
    e = float(en.mean() / n0.mean())
    se, _ = blocking(en - e * n0)
    sh = np.array([r["shift"] for r in recs])
    ss, _ = blocking(sh)
    return e, se / float(n0.mean()), float(sh.mean()), ss


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="ueg14_m358_ccsdtq")
    ap.add_argument("--target-pop", type=float, default=0.0)
    ap.add_argument("--tau", type=float, default=0.0)
    ap.add_argument("--d0", type=float, default=0.0)
    ap.add_argument("--equilibrate", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--max-seconds", type=float, default=1800.0, help="stop the window early after this")
    ap.add_argument("--grow-max", type=int, default=200000)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    import torch

    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    over = {}
    if args.target_pop:
        over["target_pop"] = args.target_pop
    if args.tau:
        over["tau"] = args.tau
    if args.d0:
        over["d0_init"] = args.d0
    if args.seed:
        over["seed"] = args.seed
    w = workload(args.workload, **over)
    stream = torch.cuda.Stream()
    ctx = ccmc.from_workload(w, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    grown, reached = 0, None
    while grown < args.grow_max:
        ctx.step(w["shift_a"])
        grown += w["shift_a"]
        if reached is None and ctx.get_state()[2]:
            reached = grown
        if reached is not None and grown >= reached + args.equilibrate:
            break
    ctx.records()
    t1 = time.perf_counter()
    recs = []
    chunk = 100
    while len(recs) < args.steps and time.perf_counter() - t1 < args.max_seconds:
        ctx.step(chunk)
        recs += ctx.records()
    t2 = time.perf_counter()
    e, se, es, ses = projected_energy(recs)
    e_hf = ctx.reference_energy()
    out = {"workload": w["name"], "electrons": w["nel"], "spin_orbitals": w.get("nso"), "truncation": w["lmax"],
           "tau": w["tau"], "target_pop": w["target_pop"], "sampling": "fnc+multispawn" if w["fnc"] else "original",
           "seed": w["seed"], "growth_steps": grown, "shift_from_step": reached, "window_steps": len(recs),
           "e_hf": e_hf, "e_proj": e, "e_proj_err": se, "e_shift": es, "e_shift_err": ses,
           "n_total_mean": sum(r["ntot_after"] for r in recs) / len(recs) / 65536.0,
           "n0_mean": sum(r["n0"] for r in recs) / len(recs) / 65536.0,
           "n_occ_last": recs[-1]["nocc_after"], "growth_seconds": t1 - t0, "window_seconds": t2 - t1}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
