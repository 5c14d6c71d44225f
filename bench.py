#!/usr/bin/env python
"""Benchmark of the CCMC time step (samples/s and annihilated keys/s).

Default workload: 14-electron uniform electron gas in 114 spin-orbitals,
CCSDT, full non-composite + multi-spawn sampling, 10^6 target population,
dtau = 0.005, FP64 (the paper's improved samplers, Sec. IV.B-C).  The
wavefunction is grown from the reference to the target population (untimed),
then W warm-up steps and K timed steps follow, each timed with CUDA events on
the library's stream and with L2 flushed between steps.

A "step" is one full CCMC time step: a1 scans, a2-a5 sampling/collapse/
spawn/death, a6 non-composite sweep with multi-spawn, a7 radix sort, a8 key
reduction, a9 merge, a10 estimators.  value = (cluster samples + non-composite
visits) per second over the timed steps; annihilated keys/s counts the
spawned records entering the sort.

--impl reference times the CPU oracle (single host core) on bounded slices of
the same workload at its target size.
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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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

def algorithmic_bytes(phase: str, recs: list, nw: int) -> float:
    """Per-step algorithmic bytes of a phase, averaged over the records.
    List entry B_e = 8K (bits) + 8 (key) + 8 (population); a spawned record is
    16 B (key + population).  The sort moves each record once in and once out;
    passes beyond that are implementation overhead."""
    be = 8 * nw + 16
    out = []
    for r in recs:
        n = r["n_visit"] if r["n_visit"] else r["nocc_after"]
        sp = r["n_spawned"]
        if phase == "scan":
            b = n * 8 + n * 8
        elif phase == "sample":
            b = r["n_sel"] * 0.97 * be + sp * 16
        elif phase == "attempts":
            b = r["n_attempts"] * be + sp * 16
        elif phase == "sort":
            b = sp * 32
        elif phase == "reduce":
            b = sp * 16 + r["n_keys"] * 16
        elif phase == "merge":
            b = n * be + r["n_keys"] * 16 + r["nocc_after"] * be
        else:
            b = 0
        out.append(b)
    return sum(out) / max(1, len(out))


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

STATE_ITER, STATE_SHIFT = 1500, -0.35   # iteration and shift of the synthetic full-size states


def synthetic_state(w):
    """The molecule workload's full-size start state: (words, pops, N_total)."""
    from ccmc_inputs import molecule_state

    words, pops, _ = molecule_state(norb=w["norb"], nocc=w["nel"] // 2, n_total=w["target_pop"],
                                    seed=w.get("state_seed", 31))
    return words, pops, float(abs(pops).sum()) / 65536.0


def state_name(w):
    return "oracle-made full-space state" if w["kind"] == "ueg" else "synthetic full-size molecule state"


def oracle_state(w):
    """The workload at its target size for the oracle: for the gas every
    excitor of the truncated space occupied with seeded populations summing to
    the target (the oracle enumerates the space with its excitation
    generator); for the molecule the synthetic full-size state."""
    import numpy as np

    import oracle
    from ccmc_inputs import molecule_integrals, synthetic_populations

    if w["kind"] == "ueg":
        so = oracle.System.ueg(w["nel"], w["nso"], w["rs"], w["lmax"])
        keys = so.space_keys(w["lmax"], expand_top=False)
        dets = [so.unrank(int(k)) for k in keys]
        levels = [so.level(d) for d in dets]
        bits = np.stack([so.to_words(d) for d in dets])
        pops = synthetic_populations(levels, w["target_pop"], seed=21)
        ntot = w["target_pop"]
    else:
        h1, eri = molecule_integrals(norb=w["norb"], nocc=w["nel"] // 2, seed=w.get("molecule_seed", 7),
                                     scale=w.get("eri_scale", 1.0))
        so = oracle.System.generic(w["nel"], h1, eri, w["lmax"])
        bits, pops, ntot = synthetic_state(w)
    sim = oracle.Sim(so, tau=w["tau"], target_pop=w["target_pop"], d0_init=w["d0_init"], shift_a=w["shift_a"],
                     zeta=w["zeta"], spawn_cutoff=w["spawn_cutoff"], fnc=w["fnc"], multispawn=w["multispawn"],
                     a_thresh=w["a_thresh"], seed=w["seed"])
    sim.set_list_words(bits, pops)
    sim.set_state(STATE_ITER, STATE_SHIFT, True, ntot)
    return sim, len(pops)


def slices_for(sim, per_slice=200_000):
    """Number of slices of a full step holding about per_slice samples each."""
    r0 = sim.sample_range(0, 0, 0, 0)
    return max(1, (r0.n_sel + r0.n_visit + per_slice - 1) // per_slice)


def oracle_slices(sim, n_occ, nslices, count, it0=STATE_ITER, first=0):
    """Times `count` slices (numbers first, first+1, ...), each 1/nslices of
    one full step's visits and cluster samples (propagation only).  Returns
    (samples, seconds, spawned)."""
    samples, secs, spawned = 0, 0.0, 0
    n_sel = None
    for k in range(first, first + count):
        q = k % nslices
        sim.set_state(it0 + k // nslices, STATE_SHIFT, True, 1.0)
        if n_sel is None:
            r0 = sim.sample_range(0, 0, 0, 0)
            n_sel = r0.n_sel
        i_lo, i_hi = q * n_occ // nslices, (q + 1) * n_occ // nslices
        g_lo, g_hi = q * n_sel // nslices, (q + 1) * n_sel // nslices
        t = time.perf_counter()
        r = sim.sample_range(i_lo, i_hi, g_lo, g_hi)
        secs += time.perf_counter() - t
        samples += (i_hi - i_lo) + (g_hi - g_lo)
        spawned += r.n_spawned
    return samples, secs, spawned


# one oracle per host core (processes started with spawn, after or apart
# from any CUDA use); each builds its own full-size state, waits at a
# barrier, then times its own slices
_POOL_BARRIER = None


def _pool_init(barrier):
    global _POOL_BARRIER
    _POOL_BARRIER = barrier


def _pool_slices(job):
    w, warm, count, first, per_slice = job
    sim, n_occ = oracle_state(w)
    nslices = slices_for(sim, per_slice)
    if warm:
        oracle_slices(sim, n_occ, nslices, warm, first=first)
    _POOL_BARRIER.wait()
    samples, secs, spawned = oracle_slices(sim, n_occ, nslices, count, first=first + warm)
    return samples, secs, spawned, nslices


def oracle_all_cores(w, warm: int, count: int, cores: int = 0, per_slice: int = 200_000):
    """Every host core runs the oracle on `count` slices of its own (about
    per_slice samples each); returns (samples/s, keys/s, cores, seconds,
    slices of a step).  The job's rate is the summed samples over the slowest
    process's time."""
    import multiprocessing as mp

    cores = cores or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_pool_init, initargs=(barrier,)) as pool:
        res = pool.map(_pool_slices, [(w, warm, count, c * (warm + count), per_slice) for c in range(cores)])
    secs = max(r[1] for r in res)
    samples = sum(r[0] for r in res)
    spawned = sum(r[2] for r in res)
    return samples / secs, spawned / secs, cores, secs, res[0][3]


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a reference "step" is one slice per process, sized so that the whole
    # run takes about a minute of oracle time
    sim, n_occ = oracle_state(w)
    n1 = slices_for(sim)
    _, t1, _ = oracle_slices(sim, n_occ, n1, 1)
    rate = (sim.sample_range(0, 0, 0, 0).n_sel + n_occ) / n1 / max(t1, 1e-6)
    per_slice = max(2000, int(rate * 60.0 / max(1, args.steps + args.warmup)))
    del sim
    v, kps, cores, secs, nslices = oracle_all_cores(w, args.warmup, args.steps, per_slice=per_slice)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs * nslices / (args.steps * cores),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "keys_per_s": kps,
        "config": {"workload": w["name"], "electrons": w["nel"], "spin_orbitals": w.get("nso", 2 * w.get("norb", 0)),
                   "truncation": w["lmax"], "target_pop": w["target_pop"], "tau": w["tau"],
                   "sampling": "fnc+multispawn" if w["fnc"] else "original"},
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} processes x {args.steps} slices of 1/{nslices} of a full step (visits + "
                                   f"cluster samples, propagation only) on the {state_name(w)}, N_total = target; "
                                   f"ms_per_step is the job's time per full step"},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, w):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_1807_03749_gb300 as ccmc

    stream = torch.cuda.Stream()
    # independent replica per rank (replicas only: the path is single-GPU)
    ctx = ccmc.from_workload(w, replica=rank, stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    restore = None
    if w.get("from_state"):
        # every timed step starts from the same synthetic full-size state,
        # restored (outside the timed region) before the step
        words, pops0, ntot0 = synthetic_state(w)

        def restore():
            ctx.set_list(words, pops0)
            ctx.set_state(STATE_ITER, STATE_SHIFT, 1, ntot0)
    # growth to the target population (untimed).  Large workloads grow at a
    # fraction f of the target, then every population (reference included)
    # is scaled by 1/f: t_HF exp(T/t_HF) scales as a whole, so this is the
    # same wavefunction at the target population.
    frac = float(w.get("grow_fraction", 1.0))
    gctx = ctx if frac == 1.0 else ccmc.from_workload(w, replica=rank, stream=stream.cuda_stream,
                                                      target_pop=w["target_pop"] * frac)
    t_grow = time.perf_counter()
    grown = 0
    reached = None
    while restore is None and grown < args.grow_max:
        gctx.step(w["shift_a"])
        grown += w["shift_a"]
        it, shift, vary, nprev = gctx.get_state()
        en = gctx.energy()
        if en["n_total"] > 1e3 * max(en["n0"], 1.0) or time.perf_counter() - t_grow > args.grow_seconds:
            raise RuntimeError(f"growth did not settle: N_total={en['n_total']:.3e}, t_HF={en['n0']:.3e} "
                               f"after {grown} steps")
        if vary and reached is None:
            reached = grown
        if reached is not None and grown >= reached + args.equilibrate:
            break
    gctx.sync()
    state_note = f"grown from HF for {grown} steps"
    if restore is not None:
        restore()
        state_note = (f"synthetic full-size state ({len(pops0)} excitors of levels 0-4, N_total = {ntot0:.4g}), "
                      f"restored before every timed step")
    if gctx is not ctx:
        bits, _, pop = gctx.get_list()
        it, shift, vary, nprev = gctx.get_state()
        n_now = float(abs(pop).sum()) / 65536.0
        scale = max(1, int(round(w["target_pop"] / n_now)))
        ctx.set_list(bits, pop * scale)
        ctx.set_state(it, shift, vary, nprev * scale)
        del gctx
        state_note += f" at {frac:g} of the target, populations then scaled x{scale}"
    t_grow = time.perf_counter() - t_grow
    ctx.records()

    def timed(nsteps):
        """Times nsteps steps; returns (per-step ms, their records).  With a
        restored start state each step's record is read before the next
        restore (restoring rewinds the iteration count)."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        recs_ = []
        with torch.cuda.stream(stream):
            for k in range(nsteps):
                if restore is not None:
                    recs_ += ctx.records()
                    restore()
                flush.fill_(k)
                starts[k].record(stream)
                ctx.step(1)
                ends[k].record(stream)
        stream.synchronize()
        recs_ += ctx.records()
        if restore is not None:
            recs_ = recs_[-nsteps:]
        return [s.elapsed_time(e) for s, e in zip(starts, ends)], recs_

    timed(args.warmup)
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
    times, recs = timed(args.steps)
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    _, _, launches1 = ctx.phase_times()
    ms_total = sum(times)
    samples = sum(r["n_sel"] + r["n_visit"] for r in recs)
    keys = sum(r["n_spawned"] for r in recs)
    ms_max, samples_all, keys_all = aggregate(dist, ms_total, samples, keys, "cuda")

    # per-phase timing pass (events between phases, one step at a time)
    ctx.profile(True)
    with torch.cuda.stream(stream):
        for k in range(args.profile_steps):
            if restore is not None:
                restore()
            flush.fill_(k)
            ctx.step(1)
    stream.synchronize()
    pms, plaunch, _ = ctx.phase_times()
    ctx.profile(False)
    precs = ctx.records()
    dom = max(pms, key=lambda p: pms[p])
    dom_ms = pms[dom] / max(1, args.profile_steps)
    alg = algorithmic_bytes(dom, precs, ctx.nw)
    hbm, src = peaks()
    achieved = alg / (dom_ms * 1e-3) / 1e9
    traffic, issue = read_traffic(w["name"], dom)

    # end-to-end through the public API with host buffers: upload the excip
    # list, one step, download the list and the estimators
    if restore is not None:
        restore()
    n_now = ctx.list_size()
    cap = 4 * n_now + 65536
    bufs = [pinned_list_buffers(cap, ctx.nw) for _ in range(2)]
    bits, _, pop = ctx.get_list(out=bufs[0])
    e2e_steps = args.e2e_steps
    h2d = d2h = 0
    e2e_samples = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.set_list(bits, pop)
        if restore is not None:
            ctx.set_state(STATE_ITER, STATE_SHIFT, 1, ntot0)
        h2d += bits.nbytes + pop.nbytes
        ctx.step(1)
        # outputs alternate between the two buffers; with a restored start
        # state the input stays in the first and every output goes to the second
        out_bits, keys_h, out_pop = ctx.get_list(out=bufs[1] if restore is not None else bufs[(k + 1) % 2])
        en = ctx.energy()
        d2h += out_bits.nbytes + keys_h.nbytes + out_pop.nbytes + 40
        if restore is None:
            bits, pop = out_bits, out_pop
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    erecs = ctx.records()
    if restore is not None:   # every e2e step ran from the same state
        e2e_samples = e2e_steps * (erecs[-1]["n_sel"] + erecs[-1]["n_visit"])
    else:
        e2e_samples = sum(r["n_sel"] + r["n_visit"] for r in erecs[-e2e_steps:])

    fp32_energy = None
    if fp32:
        fp32_energy = fp32_vs_fp64(ccmc, w, ctx, stream, start_list, start_state, min(args.steps, 200), rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle baseline is a 1-GPU figure
        cpu = cpu_baseline(w)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = samples_all / (ms_max * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if w.get("precision") == "fp32" else "f64", "data": "synthetic",
        "keys_per_s": keys_all / (ms_max * 1e-3),
        "config": {"workload": w["name"], "electrons": w["nel"], "spin_orbitals": w.get("nso", 2 * w.get("norb", 0)),
                   "truncation": w["lmax"], "target_pop": w["target_pop"], "tau": w["tau"],
                   "sampling": "fnc+multispawn" if w["fnc"] else "original",
                   "state": f"{state_note} ({t_grow:.1f} s), shift varying",
                   "n_occ": recs[-1]["nocc_after"], "n_total": recs[-1]["ntot_after"] / 65536.0,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": src,
                     "sm_issue_active_pct_ncu": issue,
                     "note": "the sampling and attempt kernels gather from L2-resident lists and are bound by integer "
                             "issue rate; their HBM fraction is low by construction",
                     "phase_ms_per_step": {k: v / max(1, args.profile_steps) for k, v in pms.items()},
                     "algorithmic_bytes_per_launch": alg},
        "clocks": clk,
        "e2e": {"value": e2e_samples / e2e_secs, "unit": "samples/s", "h2d_bytes_per_step": h2d // max(1, e2e_steps),
                "d2h_bytes_per_step": d2h // max(1, e2e_steps)},
        "gpu_launches": int(launches1 - launches0),
        "cpu_baseline": cpu,
    }
    if fp32_energy is not None:
        line["fp32_energy"] = fp32_energy
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def pinned_list_buffers(cap: int, nw: int):
    """Page-locked host arrays for a list of up to cap entries:
    (bits[cap, nw] uint64, keys[cap] uint64, pop[cap] int64)."""
    import torch

    bits = torch.empty((cap, nw), dtype=torch.int64, pin_memory=True).numpy().view("uint64")
    keys = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view("uint64")
    pop = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy()
    return bits, keys, pop


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
    return {"one_step_rel_diff_max": max(one), "one_step_steps": len(one), "window_steps": nwin,
            "e_proj_fp32": means[0][0], "err_fp32": means[0][1], "e_proj_fp64": means[1][0],
            "err_fp64": means[1][1], "diff": means[0][0] - means[1][0]}


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


def read_traffic(workload: str, phase: str):
    """(DRAM bytes per launch, SM issue-active %) of a phase's kernel from the
    committed ncu summary (profiles/traffic_<workload>.txt), or (None, None)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    try:
        for line in open(path):
            f = line.split()
            if len(f) >= 3 and not line.startswith("#") and f[0] == phase:
                return float(f[2]), (float(f[3]) if len(f) > 3 else None)
    except OSError:
        pass
    return None, None


def run_gpu_batched(args):
    """64 independent UEG problems (14 electrons, M in {38,54,66,114} x r_s in
    {0.5,1,2,5}, CCSD/CCSDT, targets 1e4-1e6) stepped as one batch: one launch
    per phase over all replicas of a word count, replayed from a CUDA graph.
    The same states are then stepped one context after another for
    comparison; the two must give bit-identical lists."""
    import numpy as np
    import torch

    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import batched_replicas

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
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

    def timed(step_fn, strm, nsteps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
        with torch.cuda.stream(strm):
            for k in range(nsteps):
                flush.fill_(k)
                starts[k].record(strm)
                step_fn()
                ends[k].record(strm)
        strm.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends))

    timed(lambda: batch.step(1), stream, args.warmup)
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
        ms_batched = timed(lambda: batch.step(1), stream, args.steps)
        torch.cuda.synchronize()
        if args.profile_window:
            torch.cuda.profiler.stop()
        clk = clocks.stop()
        _, _, launches1 = batch.phase_times()
        recs = [c.records() for c in ctxs]
        samples = sum(r["n_sel"] + r["n_visit"] for rr in recs for r in rr)
        keys = sum(r["n_spawned"] for rr in recs for r in rr)
        final = [c.get_list() for c in ctxs]

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
        ms_seq = timed(seq_step, seq_stream, args.steps)
        identical = all(all(np.array_equal(x, y) for x, y in zip(f, c.get_list())) for f, c in zip(final, seq))
        for c in seq:
            c.close()
        del seq

    # per-phase timers (events between phases of every word-count group)
    batch.profile(True)
    timed(lambda: batch.step(1), stream, args.profile_steps)
    pms, _, _ = batch.phase_times()
    batch.profile(False)
    nprof = max(1, args.profile_steps)
    precs = [c.records()[-nprof:] for c in ctxs]
    dom = max(pms, key=lambda q: pms[q])
    dom_ms = pms[dom] / nprof
    alg = sum(algorithmic_bytes(dom, rr, c.nw) for rr, c in zip(precs, ctxs))
    hbm, src = peaks()
    achieved = alg / (dom_ms * 1e-3) / 1e9

    # end to end: every replica's list from host memory, one batched step,
    # every list and estimator back to the host
    bufs = [[pinned_list_buffers(4 * c.list_size() + 65536, c.nw) for c in ctxs] for _ in range(2)]
    lists = [c.get_list(out=b) for c, b in zip(ctxs, bufs[0])]
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        for c, (bits, _, pop) in zip(ctxs, lists):
            c.set_list(bits, pop)
            h2d += bits.nbytes + pop.nbytes
        batch.step(1)
        lists = [c.get_list(out=b) for c, b in zip(ctxs, bufs[(k + 1) % 2])]
        for c, (bits, kk, pop) in zip(ctxs, lists):
            c.energy()
            d2h += bits.nbytes + kk.nbytes + pop.nbytes + 40
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    e2e_samples = sum(r["n_sel"] + r["n_visit"] for c in ctxs for r in c.records()[-args.e2e_steps:])
    info = batch.info()
    cpu = None if args.no_cpu_baseline else cpu_baseline(reps[-1])
    value = samples / (ms_batched * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batched / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "keys_per_s": keys / (ms_batched * 1e-3),
        "config": {"workload": "batched64_ueg14", "replicas": len(ctxs),
                   "systems": "14 e, M in {38,54,66,114} x r_s in {0.5,1,2,5}, CCSD (r<16, 32<=r<48) else CCSDT, "
                              "target 10^(4 + r mod 3), dtau 0.01, original sampler",
                   "state": f"grown from HF for {grown} steps ({t_grow:.1f} s), every shift varying",
                   "n_total": sum(rr[-1]["ntot_after"] for rr in recs) / 65536.0,
                   "sequential_samples_per_s": samples / (ms_seq * 1e-3),
                   "batched_speedup_over_sequential": ms_seq / ms_batched,
                   "bit_identical_to_sequential": identical, "tuned_shapes": info,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas64"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_source": src,
                     "phase_ms_per_step": {k: v / nprof for k, v in pms.items()},
                     "algorithmic_bytes_per_launch": alg},
        "clocks": clk,
        "e2e": {"value": e2e_samples / e2e_secs, "unit": "samples/s",
                "h2d_bytes_per_step": h2d // max(1, args.e2e_steps),
                "d2h_bytes_per_step": d2h // max(1, args.e2e_steps)},
        "gpu_launches": int(launches1 - launches0),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w):
    """The oracle on slices of one full step at the target size: one core
    (about 8 s of CPU work), then every host core with the same slice count
    each."""
    try:
        sim, n_occ = oracle_state(w)
    except Exception as e:  # the oracle is a reported baseline only
        return {"value": None, "unit": "samples/s", "cores": 1, "kind": "oracle", "sample": f"unavailable: {e}"}
    nslices = slices_for(sim)
    s1, t1, _ = oracle_slices(sim, n_occ, nslices, 1)          # calibration slice
    done = max(1, min(4 * nslices, int(8.0 / max(t1, 1e-3))))
    samples, secs, _ = oracle_slices(sim, n_occ, nslices, done)
    one = samples / secs
    del sim
    try:
        v, _, cores, psecs, _ = oracle_all_cores(w, 0, done)
    except Exception as e:
        return {"value": one, "unit": "samples/s", "cores": 1, "kind": "oracle",
                "sample": f"{done} slice(s) of 1/{nslices} of a full step on the {state_name(w)}, {secs:.1f} s "
                          f"(all-core run unavailable: {e})"}
    return {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {done} slice(s) of 1/{nslices} of a full step (visits + cluster samples, "
                      f"propagation only) on the {state_name(w)} at N_total = target, {psecs:.1f} s",
            "single_core": {"value": one, "cores": 1, "seconds": secs}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ueg14_m114_ccsdt_fnc_ms")
    ap.add_argument("--grow-max", type=int, default=8000)
    ap.add_argument("--equilibrate", type=int, default=100)
    ap.add_argument("--grow-seconds", type=float, default=180.0)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--target-pop", type=float, default=0.0, help="override the workload's target population")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    from ccmc_inputs import workload

    over = {}
    if args.target_pop:
        over["target_pop"] = args.target_pop   # smaller cases of a workload for profiling
    if args.workload == "batched64_ueg14":
        if args.impl == "reference":
            from ccmc_inputs import batched_replicas

            # one replica (r = 63: M = 114, r_s = 5, CCSDT, target 1e4) as the oracle's sample
            run_reference(args, dict(batched_replicas(64)[-1], name="batched64_ueg14"))
        else:
            run_gpu_batched(args)
        return
    w = workload(args.workload, **over)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
