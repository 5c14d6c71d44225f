#!/usr/bin/env python
"""The paper's distribution of excitors over processors, simulated on one GPU
(Sec. III, Eq. ccmc_dist; Fig. excitdistrib and Fig. bias).

colocation: for the determinants of the 14-electron gas in 186 spin-orbitals
at CCSD (3,813 of them, taken from the list of a CCSD run that occupies the
whole space), the probability that two excitors share a processor, averaged
over the first T iterations: its mean over pairs (times N_p, unbiased = 1)
and its standard deviation over pairs, rescaled as in Fig. excitdistrib by
N_p sqrt(T / (N_p - 1)) (fixed nu_move) and N_p sqrt(T / 2^nu_move) (fixed
N_p).  The binomial argument of Sec. III predicts the first rescaled spread
to be sqrt(2^nu_move) and the second sqrt(N_p - 1), independent of T.

bias: the CCSDT projected energy of the 14-electron, 66 spin-orbital gas at
r_s = 0.5 and 5 bohr (full non-composite sampling, Sec. III.B) when
composite clusters are formed only from excitors on one simulated processor,
for several N_p, against N_p = 1 (no bias).

    python distribution.py colocation
    python distribution.py bias --ranks 1,8,32,96,240 --steps 100000
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def space_determinants(ccmc, nel=14, nso=186, lmax=2, target=2e6, steps=3000):
    """The determinants a CCMC run occupies once its population is large
    (for a small truncated space: all of them), as rows of words."""
    import torch

    from ccmc_inputs import workload

    w = dict(workload("ueg14_m38_ccsd"), nso=nso, nel=nel, lmax=lmax, target_pop=target, d0_init=1e4, tau=0.01)
    stream = torch.cuda.Stream()
    ctx = ccmc.from_workload(w, stream=stream.cuda_stream)
    ctx.step(steps)
    bits, _, _ = ctx.get_list()
    ctx.close()
    return bits


def run_colocation(args):
    import numpy as np

    import paper_1807_03749_gb300 as ccmc

    dets = space_determinants(ccmc)
    n = len(dets)
    pairs = n * (n - 1) / 2
    ck = [1 << k for k in range(0, int(math.log2(args.t_max)) + 1)]
    out = {"determinants": n, "checkpoints": ck, "runs": []}
    grid = [(r, args.nu_fixed) for r in (8, 16, 32, 64, 128, 256)] + [(args.ranks_fixed, nu) for nu in range(0, 7)]
    for np_, nu in grid:
        s1, s2 = ccmc.colocation(dets, np_, nu, ck)
        rows = []
        for T, a, b in zip(ck, s1, s2):
            mean = float(a) / (pairs * T)
            var = max(float(b) / (pairs * T * T) - mean * mean, 0.0)
            sd = math.sqrt(var)
            rows.append({"T": T, "mean_x_np": mean * np_, "sd_scaled_by_ranks": sd * np_ * math.sqrt(T / (np_ - 1)),
                         "sd_scaled_by_moves": sd * np_ * math.sqrt(T / 2 ** nu)})
        out["runs"].append({"n_ranks": np_, "nu_move": nu, "rows": rows})
        last = rows[-1]
        print(json.dumps({"n_ranks": np_, "nu_move": nu, "T": last["T"], "mean_x_np": round(last["mean_x_np"], 5),
                          "sd_scaled_by_ranks": round(last["sd_scaled_by_ranks"], 4),
                          "expect_by_ranks": round(math.sqrt(2 ** nu), 4),
                          "sd_scaled_by_moves": round(last["sd_scaled_by_moves"], 4),
                          "expect_by_moves": round(math.sqrt(np_ - 1), 4)}), flush=True)
    if args.series:
        print(json.dumps(out), flush=True)


def run_bias(args):
    import time

    import torch

    import energy
    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    results = []
    for rs_name in args.systems.split(","):
        base = None
        for np_ in [int(x) for x in args.ranks.split(",")]:
            w = workload(rs_name, n_ranks=np_, nu_move=args.nu_move, tau=args.tau, target_pop=args.target_pop)
            stream = torch.cuda.Stream()
            ctx = ccmc.from_workload(w, stream=stream.cuda_stream)
            t0 = time.perf_counter()
            grown, reached, recs, status = 0, None, [], "ok"
            try:
                while grown < args.grow_max:
                    ctx.step(w["shift_a"])
                    grown += w["shift_a"]
                    if reached is None and ctx.get_state()[2]:
                        reached = grown
                    if reached is not None and grown >= reached + args.equilibrate:
                        break
                ctx.records()
                while reached is not None and len(recs) < args.steps:
                    ctx.step(100)
                    recs += ctx.records()
            except ccmc.CCMCError as e:   # a runaway population ends the run
                status = str(e).split(":")[0]
            ctx.close()
            row = {"system": rs_name, "n_ranks": np_, "nu_move": args.nu_move, "tau": args.tau, "status": status,
                   "steps": len(recs), "seconds": time.perf_counter() - t0}
            if status != "ok" or len(recs) < 1000:
                row["status"] = status if status != "ok" else "shift never started to vary"
                results.append(row)
                print(json.dumps(row), flush=True)
                continue
            e, se, es, ses = energy.projected_energy(recs)
            n0 = sum(r["n0"] for r in recs) / len(recs) / 65536.0
            nt = sum(r["ntot_after"] for r in recs) / len(recs) / 65536.0
            row.update(e_proj=e, e_proj_err=se, reference_fraction=n0 / nt, n_occ=recs[-1]["nocc_after"],
                       excitors_per_rank=recs[-1]["nocc_after"] / np_)
            if base is None:
                base = (e, se)
            row["bias"] = e - base[0]
            row["bias_err"] = math.sqrt(se ** 2 + base[1] ** 2)
            results.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"bias": results}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("mode", choices=["colocation", "bias"])
    ap.add_argument("--t-max", type=int, default=4096)
    ap.add_argument("--nu-fixed", type=int, default=4)
    ap.add_argument("--ranks-fixed", type=int, default=32)
    ap.add_argument("--series", action="store_true")
    ap.add_argument("--systems", default="ueg14_m66_ccsdt_rs0.5,ueg14_m66_ccsdt_rs5")
    ap.add_argument("--ranks", default="1,8,32,96,240")
    ap.add_argument("--nu-move", type=int, default=5)
    ap.add_argument("--tau", type=float, default=0.001)
    ap.add_argument("--target-pop", type=float, default=2e5)
    ap.add_argument("--equilibrate", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--grow-max", type=int, default=20000, help="growth steps before giving up on the shift")
    args = ap.parse_args()
    if args.mode == "colocation":
        run_colocation(args)
    else:
        run_bias(args)


if __name__ == "__main__":
    main()
