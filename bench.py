#!/usr/bin/env python
"""Benchmark of the CCMC time step (cluster samples/s and annihilated keys/s).

A "step" is one full CCMC time step (Spencer et al., Sec. II and IV.B-C):
a1 scans, a2-a5 cluster selection / collapse / spawning / death, a6 the full
non-composite sweep with multi-spawn where enabled, a7 radix sort, a8 key
reduction, a9 merge, a10 estimators.  value = (cluster samples + full
non-composite visits) per second over the timed steps; keys_per_s counts the
spawned records entering the sort.

Default run (no --workload): the headline line is the synthetic molecule,
20 electrons in 82 spin-orbitals, CCSDTQ, FP64, target 10^7, grown from the
reference on the GPU to a stationary population (untimed), then W warm-up
and K timed steps, each timed with CUDA events on the library's stream with
L2 flushed between steps.  The same line carries, under "configs", the
114 spin-orbital gas (CCSDT, FNC + multi-spawn, 10^6), the 64-replica batched
form and the 162 spin-orbital FP32 gas (10^8), each measured the same way.
--workload NAME measures one of them alone.

--impl reference times the CPU oracle on every host core, on bounded slices
of one full step of the headline workload (without a GPU it cannot grow the
state, so it steps the synthetic full-size list of the same system).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CCMC cluster samples/sec/GPU + annihilated keys/sec; % of HBM roofline"
L2_FLUSH_BYTES = 256 << 20
HEADLINE = "mol20_m82_ccsdtq"
EXTRA = ["ueg14_m114_ccsdt_fnc_ms", "batched64_ueg14", "ueg54_m162_ccsd_fp32"]
SMS, SMSP_PER_SM, LANES = 152, 4, 32


def peaks():
    """(HBM GB/s, SM clock MHz, source) from the measured peaks file."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def lane_issue_peak(sm_mhz: float) -> float:
    """Thread instructions per second the SMs can issue at most (G/s): every
    SM sub-partition issues one warp instruction of 32 lanes per cycle."""
    return SMS * SMSP_PER_SM * LANES * sm_mhz * 1e6 / 1e9


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per phase (what the method itself must move)
# ---------------------------------------------------------------------------

def mean_cluster_size(lmax: int, fnc: bool) -> float:
    """Mean drawn cluster size: p(s) = 2^-(s+1) for s < l + 2 and the
    remainder 2^-(l+2) at s = l + 2 (Sec. II); with full non-composite
    sampling the composite draw s >= 2 has p'(s) = 2^-(s-1), last 2^-l."""
    smax = lmax + 2
    if fnc:
        return sum(s * (2.0 ** -(s - 1) if s < smax else 2.0 ** -lmax) for s in range(2, smax + 1))
    return sum(s * (2.0 ** -(s + 1) if s < smax else 2.0 ** -(lmax + 2)) for s in range(0, smax + 1))


def phase_units(phase: str, r: dict) -> float:
    """The unit count a phase's per-unit profile figures scale with."""
    sorted_ = r["n_spawned"] - r.get("n_direct", 0)
    return {"scan": r["nocc_after"], "sample": r["n_sel"], "attempts": r["n_attempts"], "sort": sorted_,
            "reduce": sorted_, "merge": r["nocc_after"], "finalize": 1}.get(phase, 0)


def algorithmic_bytes(phase: str, recs: list, nw: int, lmax: int = 2, fnc: bool = False,
                      multispawn: bool = False) -> float:
    """Per-step algorithmic bytes of a phase, averaged over the records.
    A list entry is B_e = 8K (bits) + 8 (key) + 8 (population); a spawned
    record 16 B (key + population); a buffered multi-spawn cluster 8K + 24
    (bits, attempt coefficient, sample index, attempt prefix).
      scan:     8 B read + 8 B written per entry
      sample:   s_mean * B_e gathered per sample, plus what the sampler writes:
                16 B per record (inline attempts) or one buffered cluster
      attempts: each owner read once (list entries of the full
                non-composite sweep, buffered clusters), 16 B per record
      sort:     one read and one write of each record entering it (16 + 16 B);
                records added directly to listed determinants do not
      reduce:   16 B read per sorted record, 16 B written per distinct key
      merge:    the list read and written (B_e each way), 16 B per key."""
    be = 8 * nw + 16
    bc = 8 * nw + 24
    sbar = mean_cluster_size(lmax, fnc)
    out = []
    for r in recs:
        n = r["n_visit"] if r["n_visit"] else r["nocc_after"]
        sp = r["n_spawned"]
        ncl = r.get("n_clusters", 0)
        if phase == "scan":
            b = n * 16
        elif phase == "sample":
            # buffered clusters (multi-spawn, or the original sampler on a
            # generic Hamiltonian): their records are the attempt kernel's
            b = r["n_sel"] * sbar * be + (ncl * bc if ncl else sp * 16)
        elif phase == "attempts":
            b = r["n_visit"] * be + ncl * bc + (sp * 16 if (ncl or r["n_visit"]) else 0)
        elif phase == "sort":
            b = (sp - r.get("n_direct", 0)) * 32
        elif phase == "reduce":
            b = (sp - r.get("n_direct", 0)) * 16 + r["n_keys"] * 16
        elif phase == "merge":
            b = n * be + r["n_keys"] * 16 + r["nocc_after"] * be
        else:
            b = 0
        out.append(b)
    return sum(out) / max(1, len(out))


def read_profile(workload: str) -> dict:
    """Per-unit ncu figures of a workload's kernels from the committed summary
    profiles/traffic_<workload>.txt: {phase: {kernel, unit, dram_per_unit,
    inst_per_unit, issue_pct, lanes}} (missing file: {})."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    out = {}
    try:
        for line in open(path):
            f = line.split()
            if len(f) < 7 or line.startswith("#"):
                continue
            num = [None if x == "-" else float(x) for x in f[3:7]]
            out[f[0]] = {"kernel": f[1], "unit": f[2], "dram_per_unit": num[0], "inst_per_unit": num[1],
                         "issue_pct": num[2], "lanes": num[3]}
    except OSError:
        pass
    return out


PHASE_OF_KERNEL = [("k_scan", "scan"), ("k_local", "scan"), ("k_sample", "sample"), ("k_attempts", "attempts"), ("k_sort", "sort"),
                   ("k_seg", "reduce"), ("k_part_scan", "reduce"), ("k_merge", "merge"), ("k_keep", "merge"),
                   ("k_scatter", "merge"), ("k_finalize", "finalize")]
UNIT_OF_PHASE = {"scan": "entry", "sample": "sample", "attempts": "attempt", "sort": "record", "reduce": "record",
                 "merge": "entry", "finalize": "step"}


def summarize_ncu(csv_path: str, records_path: str, out_path: str, command: str):
    """Writes profiles/traffic_<workload>.txt from an ncu --csv capture of one
    step's kernels (metrics gpu__time_duration.sum, dram__bytes_read.sum,
    dram__bytes_write.sum, smsp__inst_executed.sum, smsp__thread_inst_executed.sum,
    smsp__issue_active.avg.pct_of_peak_sustained_active) and the records of
    the captured step (bench.py --records-out): per phase the DRAM bytes and
    thread instructions per unit (sample, attempt, record, list entry), the
    time-weighted issue activity and the lanes per warp instruction."""
    import csv

    rows = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        key = (r["ID"], r["Kernel Name"])
        try:
            v = float(r["Metric Value"].replace(",", ""))
        except ValueError:
            continue
        unit = r.get("Metric Unit", "")
        scale = {"Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "byte": 1.0, "KB": 1e3, "MB": 1e6, "GB": 1e9, "B": 1.0,
                 "usecond": 1e-6, "msecond": 1e-3, "nsecond": 1e-9, "second": 1.0, "us": 1e-6, "ms": 1e-3,
                 "ns": 1e-9, "s": 1.0}.get(unit, 1.0)
        rows.setdefault(key, {})[r["Metric Name"]] = v * scale
    recs = json.load(open(records_path))
    rec = recs[0] if isinstance(recs, list) else recs
    per = {}
    for (kid, name), m in rows.items():
        short = name.split("(")[0].split("<")[0].replace("ccmc::", "").replace("void ", "").strip()
        ph = next((p for pre, p in PHASE_OF_KERNEL if short.startswith(pre)), None)
        if ph is None:
            continue
        a = per.setdefault(ph, {"dram": 0.0, "tinst": 0.0, "inst": 0.0, "t": 0.0, "issue_t": 0.0, "top": (0.0, short)})
        t = m.get("gpu__time_duration.sum", 0.0)
        a["dram"] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        a["tinst"] += m.get("smsp__thread_inst_executed.sum", 0.0)
        a["inst"] += m.get("smsp__inst_executed.sum", 0.0)
        a["t"] += t
        a["issue_t"] += t * m.get("smsp__issue_active.avg.pct_of_peak_sustained_active", 0.0)
        if t > a["top"][0]:
            a["top"] = (t, short)
    with open(out_path, "w") as f:
        f.write("# Per-unit ncu figures of one CCMC step's kernels, by phase (bench.py --summarize-ncu).\n")
        f.write(f"# command: {command}\n")
        f.write("# step units: " + json.dumps({k: rec[k] for k in ("n_sel", "n_visit", "n_attempts", "n_spawned",
                                                                    "n_direct", "n_keys", "nocc_after")}) + "\n")
        f.write("# phase kernel(longest) unit dram_bytes_per_unit thread_inst_per_unit issue_active_pct "
                "lanes_per_inst\n")
        for ph in ("scan", "sample", "attempts", "sort", "reduce", "merge", "finalize"):
            if ph not in per:
                continue
            a = per[ph]
            u = max(1.0, float(phase_units(ph, rec)))
            issue = a["issue_t"] / a["t"] if a["t"] else 0.0
            lanes = a["tinst"] / a["inst"] if a["inst"] else 0.0
            f.write(f"{ph:9s} {a['top'][1]:18s} {UNIT_OF_PHASE[ph]:8s} {a['dram'] / u:14.3f} {a['tinst'] / u:14.3f} "
                    f"{issue:6.1f} {lanes:6.2f}\n")
        # the launch list of the captured step: per kernel its launches, total
        # time (serialised and cold-cache under ncu: compare shares), share,
        # DRAM bytes per launch
        kern = {}
        for (kid, name), m in rows.items():
            short = name.split("(")[0].replace("ccmc::", "").replace("void ", "").strip()
            k = kern.setdefault(short, [0, 0.0, 0.0])
            k[0] += 1
            k[1] += m.get("gpu__time_duration.sum", 0.0)
            k[2] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        tot = sum(v[1] for v in kern.values()) or 1.0
        f.write("# launch list of the captured step (kernel, launches, total us, share, DRAM MB per launch):\n")
        for name, (nl, t, b) in sorted(kern.items(), key=lambda kv: -kv[1][1]):
            f.write(f"#   {name:34s} {nl:4d} {t * 1e6:12.1f} {100.0 * t / tot:6.1f}% {b / nl / 1e6:10.2f}\n")


def roofline_objects(name: str, pms: dict, nprof: int, precs_by_ctx: list, nw_by_ctx: list, lmax_by_ctx: list,
                     fnc: bool, multispawn: bool):
    """(roofline of the dominant kernel, HBM roofline of the annihilation and
    list phases) from the per-phase CUDA-event times of the profile pass and
    the committed ncu per-unit figures."""
    hbm, sm_mhz, src = peaks()
    prof = read_profile(name)
    per = {k: v / max(1, nprof) for k, v in pms.items()}

    def alg(phase):
        return sum(algorithmic_bytes(phase, pr, nw, lm, fnc, multispawn)
                   for pr, nw, lm in zip(precs_by_ctx, nw_by_ctx, lmax_by_ctx))

    def units(phase):
        return sum(sum(phase_units(phase, r) for r in pr) / max(1, len(pr)) for pr in precs_by_ctx)

    def traffic(phase):
        p = prof.get(phase)
        return p["dram_per_unit"] * units(phase) if p and p["dram_per_unit"] is not None else None

    dom = max(per, key=lambda q: per[q])
    t = per[dom] * 1e-3
    hbm_part = {"achieved": alg(dom) / t / 1e9, "peak": hbm, "unit": "GB/s", "frac": alg(dom) / t / 1e9 / hbm,
                "algorithmic_bytes_per_launch": alg(dom), "traffic": traffic(dom)}
    p = prof.get(dom)
    if dom in ("sample", "attempts") and p and p["inst_per_unit"]:
        inst = p["inst_per_unit"] * units(dom)
        peak = lane_issue_peak(sm_mhz)
        roof = {"bound": "alu", "kernel": dom, "achieved": inst / t / 1e9, "peak": peak, "unit": "Ginst/s",
                "frac": inst / t / 1e9 / peak, "traffic": traffic(dom),
                "peak_source": f"{SMS} SMs x {SMSP_PER_SM} x {LANES} lanes x {sm_mhz:.0f} MHz ({src} clock)",
                "thread_inst_per_launch": inst, "issue_active_pct_ncu": p["issue_pct"],
                "lanes_per_inst_ncu": p["lanes"], "hbm": hbm_part}
    else:
        roof = dict({"bound": "hbm", "kernel": dom, "peak_source": src}, **hbm_part)
    roof["phase_ms_per_step"] = per
    ph = ["scan", "sort", "reduce", "merge"]
    ta = sum(per.get(q, 0.0) for q in ph) * 1e-3
    ba = sum(alg(q) for q in ph)
    tr = [traffic(q) for q in ph]
    ann = {"bound": "hbm", "phases": ph, "achieved": ba / ta / 1e9 if ta else None, "peak": hbm, "unit": "GB/s",
           "frac": ba / ta / 1e9 / hbm if ta else None, "algorithmic_bytes_per_step": ba,
           "traffic": sum(tr) if all(x is not None for x in tr) else None, "peak_source": src}
    return roof, ann


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

STATE_ITER, STATE_SHIFT = 1500, -0.35   # iteration and shift of the synthetic full-size states


def state_name(w):
    return "oracle-made full-space state" if w["kind"] == "ueg" else "synthetic full-size molecule state"


def oracle_system(w):
    import oracle
    from ccmc_inputs import molecule_integrals

    if w["kind"] == "ueg":
        return oracle.System.ueg(w["nel"], w["nso"], w["rs"], w["lmax"])
    h1, eri = molecule_integrals(norb=w["norb"], nocc=w["nel"] // 2, seed=w.get("molecule_seed", 7),
                                 scale=w.get("eri_scale", 1.0))
    return oracle.System.generic(w["nel"], h1, eri, w["lmax"])


def oracle_sim(w, so):
    import oracle

    return oracle.Sim(so, tau=w["tau"], target_pop=w["target_pop"], d0_init=w["d0_init"], shift_a=w["shift_a"],
                      zeta=w["zeta"], spawn_cutoff=w["spawn_cutoff"], fnc=w["fnc"], multispawn=w["multispawn"],
                      a_thresh=w["a_thresh"], seed=w["seed"], replica=w.get("replica", 0))


def oracle_state(w, state_file=None):
    """The oracle at the workload's full size.  With state_file (a list the
    GPU grew, saved by save_state) the same list and shift state; otherwise a
    synthetic full-size list: for the gas every excitor of the truncated space
    with seeded populations summing to the target (the oracle enumerates the
    space with its excitation generator), for the molecule molecule_state."""
    import numpy as np

    from ccmc_inputs import molecule_state, synthetic_populations

    so = oracle_system(w)
    sim = oracle_sim(w, so)
    if state_file:
        d = np.load(state_file)
        sim.set_list_words(d["bits"], d["pop"])
        sim.set_state(int(d["iter"]), float(d["shift"]), bool(d["vary"]), float(d["nprev"]))
        return sim, len(d["pop"])
    if w["kind"] == "ueg":
        keys = so.space_keys(w["lmax"], expand_top=False)
        dets = [so.unrank(int(k)) for k in keys]
        levels = [so.level(d) for d in dets]
        bits = np.stack([so.to_words(d) for d in dets])
        pops = synthetic_populations(levels, w["target_pop"], seed=21)
        ntot = w["target_pop"]
    else:
        bits, pops, _ = molecule_state(norb=w["norb"], nocc=w["nel"] // 2, n_total=w["target_pop"],
                                       seed=w.get("state_seed", 31))
        ntot = float(np.abs(pops).sum()) / 65536.0
    sim.set_list_words(bits, pops)
    sim.set_state(STATE_ITER, STATE_SHIFT, True, ntot)
    return sim, len(pops)


def save_state(ctx, path):
    """Saves a context's list and shift state for the oracle processes."""
    import numpy as np

    bits, _, pop = ctx.get_list()
    it, shift, vary, nprev = ctx.get_state()
    np.savez(path, bits=bits, pop=pop, iter=it, shift=shift, vary=int(vary), nprev=nprev)


def slices_for(sim, per_slice=200_000):
    """Number of slices of a full step holding about per_slice samples each."""
    r0 = sim.sample_range(0, 0, 0, 0)
    return max(1, (r0.n_sel + r0.n_visit + per_slice - 1) // per_slice)


def oracle_slices(sim, n_occ, nslices, count, first=0):
    """Times `count` slices (numbers first, first+1, ...), each 1/nslices of
    one full step's visits and cluster samples (propagation only), all from
    the sim's current state.  Returns (samples, seconds, spawned)."""
    samples, secs, spawned = 0, 0.0, 0
    it0, shift, vary, nprev = sim.get_state()
    r0 = sim.sample_range(0, 0, 0, 0)
    n_sel = r0.n_sel
    for k in range(first, first + count):
        q = k % nslices
        sim.set_state(it0 + k // nslices, shift, vary, nprev)
        i_lo, i_hi = q * n_occ // nslices, (q + 1) * n_occ // nslices
        g_lo, g_hi = q * n_sel // nslices, (q + 1) * n_sel // nslices
        t = time.perf_counter()
        r = sim.sample_range(i_lo if r0.n_visit else 0, i_hi if r0.n_visit else 0, g_lo, g_hi)
        secs += time.perf_counter() - t
        samples += ((i_hi - i_lo) if r0.n_visit else 0) + (g_hi - g_lo)
        spawned += r.n_spawned
    sim.set_state(it0, shift, vary, nprev)
    return samples, secs, spawned


# one oracle per host core (processes started with spawn, apart from any
# CUDA use); each builds its own full-size state, waits at a barrier, then
# times its own slices for about `seconds`
_POOL_BARRIER = None


def _pool_init(barrier):
    global _POOL_BARRIER
    _POOL_BARRIER = barrier


def _pool_slices(job):
    w, state_file, seconds, first, per_slice = job
    sim, n_occ = oracle_state(w, state_file)
    nslices = slices_for(sim, per_slice)
    _, t1, _ = oracle_slices(sim, n_occ, nslices, 1, first=first)        # calibration (untimed)
    count = max(1, int(seconds / max(t1, 1e-4)))
    _POOL_BARRIER.wait()
    samples, secs, spawned = oracle_slices(sim, n_occ, nslices, count, first=first + 1)
    return samples, secs, spawned, nslices, count


def oracle_all_cores(w, seconds: float, cores: int = 0, per_slice: int = 200_000, state_file=None):
    """Every host core runs the oracle on slices of one full step for about
    `seconds`; returns (samples/s, keys/s, cores, seconds, per-process rates,
    slices of a step, slices per process).  The job's rate is the summed
    samples over the slowest process's time."""
    import multiprocessing as mp

    cores = cores or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_pool_init, initargs=(barrier,)) as pool:
        res = pool.map(_pool_slices, [(w, state_file, seconds, c * 100_000, per_slice) for c in range(cores)])
    secs = max(r[1] for r in res)
    samples = sum(r[0] for r in res)
    spawned = sum(r[2] for r in res)
    rates = [r[0] / r[1] for r in res if r[1] > 0]
    return samples / secs, spawned / secs, cores, secs, rates, res[0][3], res[0][4]


def cpu_baseline(w, state_file=None, seconds: float = 6.0, state_note: str = ""):
    """The oracle as it stands, one process per host core, on slices of one
    full step of the same state the GPU timed (or a synthetic full-size one)."""
    try:
        v, _, cores, secs, rates, nslices, count = oracle_all_cores(w, seconds, state_file=state_file)
    except Exception as e:  # the oracle is a reported baseline only
        return {"value": None, "unit": "samples/s", "cores": 0, "kind": "oracle", "sample": f"unavailable: {e}"}
    where = state_note or state_name(w)
    return {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {count} slice(s) of 1/{nslices} of one full step (visits + cluster "
                      f"samples, propagation only) on {where}, {secs:.1f} s",
            "per_core_median": statistics.median(rates) if rates else None}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a reference "step" is one slice of a full step per process; the run
    # lasts about a minute of oracle time
    seconds = max(5.0, 60.0 * args.steps / max(1, args.steps + args.warmup))
    v, kps, cores, secs, rates, nslices, count = oracle_all_cores(w, seconds)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs * nslices / max(1, count * cores),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "keys_per_s": kps, "config": workload_config(w, "synthetic full-size list (the oracle cannot grow it)"),
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} processes x {count} slices of 1/{nslices} of a full step (visits + "
                                   f"cluster samples, propagation only) on the {state_name(w)}; ms_per_step is "
                                   f"the job's time per full step"},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, state_note):
    return {"workload": w["name"], "electrons": w["nel"], "spin_orbitals": w.get("nso", 2 * w.get("norb", 0)),
            "truncation": w["lmax"], "target_pop": w["target_pop"], "tau": w["tau"],
            "precision": w.get("precision", "fp64"),
            "sampling": "fnc+multispawn" if w["fnc"] else "original", "state": state_note}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def grow(ccmc, ctx, w, args, rank, stream):
    """Grows the wavefunction from the reference until the shift has varied
    for `equilibrate` steps (untimed).  Large workloads grow at a fraction f
    of the target, then every population (reference included) is scaled by
    1/f: t_HF exp(T/t_HF) scales as a whole, so this is the same wavefunction
    at the target population.  Returns a description of the state."""
    frac = float(w.get("grow_fraction", 1.0))
    eq = int(w.get("equilibrate", args.equilibrate))
    gctx = ctx if frac == 1.0 else ccmc.from_workload(w, replica=rank, stream=stream.cuda_stream,
                                                      target_pop=w["target_pop"] * frac)
    t0 = time.perf_counter()
    grown, reached = 0, None
    while grown < args.grow_max:
        gctx.step(w["shift_a"])
        grown += w["shift_a"]
        _, _, vary, _ = gctx.get_state()
        en = gctx.energy()
        if en["n_total"] > 64.0 * w["target_pop"] * frac or time.perf_counter() - t0 > args.grow_seconds:
            raise RuntimeError(f"{w['name']}: growth did not settle: N_total={en['n_total']:.3e}, "
                               f"t_HF={en['n0']:.3e} after {grown} steps")
        if vary and reached is None:
            reached = grown
        if reached is not None and grown >= reached + eq:
            break
    gctx.sync()
    note = f"grown from the reference for {grown} steps (shift varying for the last {grown - (reached or grown)})"
    if gctx is not ctx:
        bits, _, pop = gctx.get_list()
        it, shift, vary, nprev = gctx.get_state()
        n_now = float(abs(pop).sum()) / 65536.0
        scale = max(1, int(round(w["target_pop"] / n_now)))
        ctx.set_list(bits, pop * scale)
        ctx.set_state(it, shift, vary, nprev * scale)
        gctx.close()
        note += f" at {frac:g} of the target, populations then scaled x{scale}"
    return note + f", {time.perf_counter() - t0:.1f} s"


def timed_steps(torch, stream, flush, step, nsteps):
    """Per-step CUDA-event times (ms) of nsteps calls of step() on stream,
    with a 256 MiB write between steps to flush L2."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    with torch.cuda.stream(stream):
        for k in range(nsteps):
            flush.fill_(k)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
    stream.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def pinned_list_buffers(cap: int, nw: int):
    """Page-locked host arrays for a list of up to cap entries:
    (bits[cap, nw] uint64, keys[cap] uint64, pop[cap] int64)."""
    import torch

    bits = torch.empty((cap, nw), dtype=torch.int64, pin_memory=True).numpy().view("uint64")
    keys = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view("uint64")
    pop = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy()
    return bits, keys, pop


def stationarity(recs):
    """Smallest and largest one-step ratio of N_total over the timed steps."""
    nt = [r["ntot"] for r in recs] + [recs[-1]["ntot_after"]]
    q = [b / a for a, b in zip(nt, nt[1:]) if a > 0]
    return {"n_total_step_ratio_min": min(q) if q else None, "n_total_step_ratio_max": max(q) if q else None,
            "n_total_first": nt[0] / 65536.0, "n_total_last": nt[-1] / 65536.0}


def run_gpu(args, w, dist, rank, world, local):
    """One single-system workload; returns the result dict (rank 0) or None."""
    import torch

    import paper_1807_03749_gb300 as ccmc

    stream = torch.cuda.Stream()
    # independent replica per rank (replicas only: the path is single-GPU)
    ctx = ccmc.from_workload(w, replica=rank, stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    note = grow(ccmc, ctx, w, args, rank, stream)
    ctx.records()
    timed_steps(torch, stream, flush, lambda: ctx.step(1), args.warmup)
    ctx.records()
    fp32 = w.get("precision") == "fp32"
    if fp32:   # the timed window's start state, for the FP64 comparison
        start_list = ctx.get_list()
        start_state = ctx.get_state()
    _, _, launches0 = ctx.phase_times()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.start()
    times = timed_steps(torch, stream, flush, lambda: ctx.step(1), args.steps)
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    recs = ctx.records()[-args.steps:]
    if args.records_out and rank == 0:
        with open(args.records_out, "w") as f:
            json.dump(recs, f)
    _, _, launches1 = ctx.phase_times()
    ms_total = sum(times)
    samples = sum(r["n_sel"] + r["n_visit"] for r in recs)
    keys = sum(r["n_spawned"] for r in recs)
    ms_max, samples_all, keys_all = aggregate(dist, ms_total, samples, keys, "cuda")
    stat = stationarity(recs)

    # the oracle runs on this very state (saved before the profile pass)
    state_file = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        state_file = os.path.join(tempfile.mkdtemp(prefix="ccmc_bench_"), "state.npz")
        save_state(ctx, state_file)

    # per-phase timing pass (events between phases, one step at a time)
    ctx.profile(True)
    with torch.cuda.stream(stream):
        for k in range(args.profile_steps):
            flush.fill_(k)
            ctx.step(1)
    stream.synchronize()
    pms, _, _ = ctx.phase_times()
    ctx.profile(False)
    precs = ctx.records()[-max(1, args.profile_steps):]
    roof, ann = roofline_objects(w["name"], pms, args.profile_steps, [precs], [ctx.nw], [w["lmax"]],
                                 bool(w["fnc"]), bool(w["multispawn"]))

    # end to end through the public API with host buffers: upload the excip
    # list from pinned memory, one step, download the list and the estimators
    n_now = ctx.list_size()
    cap = 2 * n_now + 65536
    bufs = [pinned_list_buffers(cap, ctx.nw) for _ in range(2)]
    bits, _, pop = ctx.get_list(out=bufs[0])
    # one untimed round first: the step's graph is captured again after the
    # per-phase pass, and the upload's copy stream is created on first use
    ctx.set_list(bits, pop)
    ctx.step(1)
    bits, _, pop = ctx.get_list(out=bufs[1], with_keys=False)
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        ctx.set_list(bits, pop)
        h2d += bits.nbytes + pop.nbytes
        ctx.step(1)
        # the list and the estimators come back; its keys are recomputed on upload
        bits, _, pop = ctx.get_list(out=bufs[(k + 1) % 2], with_keys=False)
        ctx.energy()
        d2h += bits.nbytes + pop.nbytes + 40
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    e2e_samples = sum(r["n_sel"] + r["n_visit"] for r in ctx.records()[-args.e2e_steps:])

    fp32_energy = None
    if fp32:
        fp32_energy = fp32_vs_fp64(ccmc, w, ctx, stream, start_list, start_state, min(args.steps, 200), rank)
    ctx.close()

    cpu = None
    if state_file:
        cpu = cpu_baseline(w, state_file, state_note="the state the GPU timed (saved after the timed steps)")
        os.remove(state_file)
        os.rmdir(os.path.dirname(state_file))
    if rank != 0:
        return None
    out = {
        "value": samples_all / (ms_max * 1e-3), "unit": "samples/s", "ms_per_step": ms_max / args.steps,
        "keys_per_s": keys_all / (ms_max * 1e-3), "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32" if fp32 else "f64",
        "config": dict(workload_config(w, note), n_occ=recs[-1]["nocc_after"], stationarity=stat,
                       l2="flushed between timed steps (256 MiB write)", parallelism=f"replicas{world}"),
        "roofline": roof, "annihilation_roofline": ann, "clocks": clk,
        "e2e": {"value": e2e_samples / e2e_secs, "unit": "samples/s", "h2d_bytes_per_step": h2d // max(1, args.e2e_steps),
                "d2h_bytes_per_step": d2h // max(1, args.e2e_steps)},
        "gpu_launches": int(launches1 - launches0),
        "cpu_baseline": cpu,
    }
    if fp32_energy is not None:
        out["fp32_energy"] = fp32_energy
    return out


def blocked_error(x):
    """Standard error of the mean of a correlated series: the largest
    blocked estimate over block sizes that leave at least 8 blocks."""
    import numpy as np

    x = np.asarray(x, dtype=np.float64)
    best, b = 0.0, 1
    while len(x) // b >= 8:
        m = len(x) // b
        y = x[: m * b].reshape(m, b).mean(axis=1)
        best = max(best, float(y.std(ddof=1) / np.sqrt(m)))
        b *= 2
    return best


def fp32_vs_fp64(ccmc, w, ctx32, stream, start_list, start_state, nwin, rank):
    """Energy error of the FP32 form against the FP64 path from the timed
    window's start state: (1) the projected energy of single steps from the
    identical state (same samples, so the difference is the arithmetic),
    (2) the mean projected energy over nwin steps of each path, with blocked
    standard errors."""
    ctx64 = ccmc.from_workload(w, replica=rank, stream=stream.cuda_stream, precision="fp64")
    bits, _, pop = start_list
    it0, shift0, vary0, nprev0 = start_state

    def e_proj(r):
        return r["e_num"] / (r["n0"] / 65536.0) if r["n0"] else 0.0

    one = []
    for k in range(4):
        e = []
        for c in (ctx32, ctx64):
            c.records()
            c.set_list(bits, pop)
            c.set_state(it0 + k, shift0, vary0, nprev0)
            c.step(1)
            e.append(e_proj(c.records()[-1]))
        one.append(abs(e[0] - e[1]) / max(abs(e[1]), 1e-300))
    means = []
    for c in (ctx32, ctx64):
        c.records()
        c.set_list(bits, pop)
        c.set_state(it0, shift0, vary0, nprev0)
        c.step(nwin)
        ser = [e_proj(r) for r in c.records()[-nwin:]]
        means.append((sum(ser) / len(ser), blocked_error(ser)))
    ctx64.close()
    diff = means[0][0] - means[1][0]
    comb = (means[0][1] ** 2 + means[1][1] ** 2) ** 0.5
    return {"one_step_rel_diff_max": max(one), "one_step_steps": len(one), "window_steps": nwin,
            "e_proj_fp32": means[0][0], "err_fp32": means[0][1], "e_proj_fp64": means[1][0],
            "err_fp64": means[1][1], "diff": diff, "diff_over_combined_error": diff / comb if comb else None,
            "one_step_bound": 1e-6, "one_step_within_bound": max(one) <= 1e-6}


def aggregate(dist, ms_total: float, samples: float, keys: float, device: str):
    """Whole-job figures over the ranks: the slowest rank's time and the sum
    of every rank's samples and keys (each rank steps its own replica)."""
    if dist is None:
        return ms_total, float(samples), float(keys)
    import torch

    t = torch.tensor([ms_total], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(samples), float(keys)], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), float(c[0].item()), float(c[1].item())


def run_gpu_batched(args, local):
    """64 independent UEG problems (14 electrons, M in {38,54,66,114} x r_s in
    {0.5,1,2,5}, CCSD/CCSDT, targets 1e4-1e6) stepped as one batch: one launch
    per phase over all replicas of a word count, replayed from a CUDA graph.
    The same states are then stepped one context after another for
    comparison; the two must give bit-identical lists."""
    import numpy as np
    import torch

    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import batched_replicas

    reps = batched_replicas(64)
    stream = torch.cuda.Stream()
    ctxs = [ccmc.from_workload(w, stream=stream.cuda_stream) for w in reps]
    batch = ccmc.Batch(ctxs, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    t_grow = time.perf_counter()
    grown, reached = 0, None
    while grown < args.grow_max:
        batch.step(10)
        grown += 10
        states = [c.get_state() for c in ctxs]
        if time.perf_counter() - t_grow > args.grow_seconds:
            raise RuntimeError(f"batched growth did not settle within {args.grow_seconds} s ({grown} steps)")
        if grown % 100 == 0:
            for c, w in zip(ctxs, reps):
                en = c.energy()
                if en["n_total"] > 100.0 * w["target_pop"]:
                    raise RuntimeError(f"{w['name']}: population {en['n_total']:.3e} far above its target "
                                       f"{w['target_pop']:.0e} after {grown} steps")
        if reached is None and all(st[2] for st in states):
            reached = grown
        if reached is not None and grown >= reached + args.equilibrate:
            break
    t_grow = time.perf_counter() - t_grow
    for c in ctxs:
        c.records()

    timed_steps(torch, stream, flush, lambda: batch.step(1), args.warmup)
    for c in ctxs:
        c.records()
    with tempfile.TemporaryDirectory() as tmp:
        paths = [os.path.join(tmp, f"r{i}.ck") for i in range(len(ctxs))]
        for c, pth in zip(ctxs, paths):
            c.save(pth)
        _, _, launches0 = batch.phase_times()
        clocks = ClockSampler(local)
        clocks.start()
        torch.cuda.synchronize()
        if args.profile_window:
            torch.cuda.profiler.start()
        ms_batched = sum(timed_steps(torch, stream, flush, lambda: batch.step(1), args.steps))
        torch.cuda.synchronize()
        if args.profile_window:
            torch.cuda.profiler.stop()
        clk = clocks.stop()
        _, _, launches1 = batch.phase_times()
        recs = [c.records()[-args.steps:] for c in ctxs]
        if args.records_out:
            # the batch's units: every replica's records summed per step
            tot = [{k: sum(rr[i][k] for rr in recs) for k in recs[0][0] if k not in ("shift", "e_num")}
                   for i in range(len(recs[0]))]
            with open(args.records_out, "w") as f:
                json.dump(tot, f)
        samples = sum(r["n_sel"] + r["n_visit"] for rr in recs for r in rr)
        keys = sum(r["n_spawned"] for rr in recs for r in rr)
        final = [c.get_list() for c in ctxs]
        big = max(range(len(ctxs)), key=lambda i: recs[i][-1]["ntot_after"])
        state_file = None
        if not args.no_cpu_baseline:
            state_file = os.path.join(tmp, "state.npz")
            save_state(ctxs[big], state_file)

        # the same steps from the same states, one context after another
        seq_stream = torch.cuda.Stream()
        seq = [ccmc.from_workload(w, stream=seq_stream.cuda_stream) for w in reps]
        for c, pth in zip(seq, paths):
            c.load(pth)

        def seq_step():
            for c in seq:
                c.step(1)

        seq_step()  # graph capture of every context, then back to the saved states
        for c, pth in zip(seq, paths):
            c.load(pth)
        torch.cuda.synchronize()
        ms_seq = sum(timed_steps(torch, seq_stream, flush, seq_step, args.steps))
        identical = all(all(np.array_equal(x, y) for x, y in zip(f, c.get_list())) for f, c in zip(final, seq))
        for c in seq:
            c.close()
        del seq

        # per-phase timers (events between phases of every word-count group)
        batch.profile(True)
        nprof = max(1, args.profile_steps)
        timed_steps(torch, stream, flush, lambda: batch.step(1), nprof)
        pms, _, _ = batch.phase_times()
        batch.profile(False)
        precs = [c.records()[-nprof:] for c in ctxs]
        roof, ann = roofline_objects("batched64_ueg14", pms, nprof, precs, [c.nw for c in ctxs],
                                     [w["lmax"] for w in reps], False, False)

        # end to end: every replica's list from host memory, one batched step,
        # every list and estimator back to the host
        bufs = [[pinned_list_buffers(2 * c.list_size() + 65536, c.nw) for c in ctxs] for _ in range(2)]
        lists = [c.get_list(out=b) for c, b in zip(ctxs, bufs[0])]
        # one untimed round first (copy streams created, graphs captured)
        for c, (bits, _, pop) in zip(ctxs, lists):
            c.set_list(bits, pop)
        batch.step(1)
        lists = [c.get_list(out=b, with_keys=False) for c, b in zip(ctxs, bufs[1])]
        h2d = d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            for c, (bits, _, pop) in zip(ctxs, lists):
                c.set_list(bits, pop)
                h2d += bits.nbytes + pop.nbytes
            batch.step(1)
            lists = [c.get_list(out=b, with_keys=False) for c, b in zip(ctxs, bufs[(k + 1) % 2])]
            for c, (bits, _, pop) in zip(ctxs, lists):
                c.energy()
                d2h += bits.nbytes + pop.nbytes + 40
        torch.cuda.synchronize()
        e2e_secs = time.perf_counter() - t0
        e2e_samples = sum(r["n_sel"] + r["n_visit"] for c in ctxs for r in c.records()[-args.e2e_steps:])
        info = batch.info()
        batch.close()
        for c in ctxs:
            c.close()
        cpu = None
        if state_file:
            cpu = cpu_baseline(reps[big], state_file,
                               state_note=f"replica {big} (the largest) as the GPU timed it")
    return {
        "value": samples / (ms_batched * 1e-3), "unit": "samples/s", "ms_per_step": ms_batched / args.steps,
        "keys_per_s": keys / (ms_batched * 1e-3), "steps": args.steps, "warmup": args.warmup, "dtype": "f64",
        "config": {"workload": "batched64_ueg14", "replicas": len(ctxs),
                   "systems": "14 e, M in {38,54,66,114} x r_s in {0.5,1,2,5}, CCSD (r<16, 32<=r<48) else CCSDT, "
                              "target 10^(4 + r mod 3), dtau 0.01, original sampler",
                   "state": f"grown from the reference for {grown} steps ({t_grow:.1f} s), every shift varying",
                   "n_total": sum(rr[-1]["ntot_after"] for rr in recs) / 65536.0,
                   "sequential_samples_per_s": samples / (ms_seq * 1e-3),
                   "batched_speedup_over_sequential": ms_seq / ms_batched,
                   "bit_identical_to_sequential": identical, "tuned_shapes": info,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas64"},
        "roofline": roof, "annihilation_roofline": ann, "clocks": clk,
        "e2e": {"value": e2e_samples / e2e_secs, "unit": "samples/s",
                "h2d_bytes_per_step": h2d // max(1, args.e2e_steps),
                "d2h_bytes_per_step": d2h // max(1, args.e2e_steps)},
        "gpu_launches": int(launches1 - launches0),
        "cpu_baseline": cpu,
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="", help="measure one workload alone (default: the headline line "
                                                   "with the other configurations under 'configs')")
    ap.add_argument("--grow-max", type=int, default=8000)
    ap.add_argument("--equilibrate", type=int, default=100)
    ap.add_argument("--grow-seconds", type=float, default=180.0)
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--target-pop", type=float, default=0.0, help="override the workload's target population")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--records-out", default="", help="write the timed steps' records (JSON) to this file")
    ap.add_argument("--summarize-ncu", nargs=3, metavar=("CSV", "RECORDS", "OUT"),
                    help="write a per-phase traffic summary from an ncu CSV and the captured step's records")
    ap.add_argument("--ncu-command", default="", help="the capture command, quoted in the summary")
    args = ap.parse_args()
    if args.summarize_ncu:
        summarize_ncu(*args.summarize_ncu, command=args.ncu_command)
        return
    from ccmc_inputs import batched_replicas, workload

    over = {}
    if args.target_pop:
        over["target_pop"] = args.target_pop   # smaller cases of a workload for profiling
    name = args.workload or HEADLINE
    if args.impl == "reference":
        if name == "batched64_ueg14":
            # one replica (r = 63: M = 114, r_s = 5, CCSDT, target 1e4) as the oracle's sample
            run_reference(args, dict(batched_replicas(64)[-1], name="batched64_ueg14"))
        else:
            run_reference(args, workload(name, **over))
        return

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def one(nm):
        if nm == "batched64_ueg14":
            return run_gpu_batched(args, local) if rank == 0 else None
        w = workload(nm, **over)
        if args.target_pop and "list_capacity" in w:   # a smaller case keeps the same room per target
            w["list_capacity"] = int(w["list_capacity"] * args.target_pop / workload(nm)["target_pop"]) + 65536
        return run_gpu(args, w, dist, rank, world, local)

    head = one(name)
    extra = []
    if not args.workload and world == 1:   # the other configurations ride on the 1-GPU line
        for nm in EXTRA:
            extra.append(one(nm))
            torch.cuda.empty_cache()
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "samples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"],
                "data": "synthetic"}
        line.update({k: v for k, v in head.items() if k not in line and k not in ("steps", "warmup")})
        if extra:
            line["configs"] = extra
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
