"""Parity of the CUDA step with the CPU oracle, through the C ABI.

Both sides start from the same oracle-made state and draw the same Philox
numbers, so lists, populations, spawned records and counters must agree bit
for bit; the projected-energy numerator (a compensated FP64 sum in a
different order) must agree to 1e-12 relative.
"""
import os
import tempfile
import time

import numpy as np
import pytest

import oracle
from ccmc_inputs import molecule_integrals, synthetic_populations, workload

pytestmark = pytest.mark.gpu

INT_FIELDS = ["iter", "n0", "ntot", "n_sel", "n_visit", "n_attempts", "n_spawned", "ntot_after", "nocc_after",
              "n_keys"]


@pytest.fixture(scope="module")
def ccmc():
    import paper_1807_03749_gb300 as p

    p.load()
    return p


def _oracle_system(w):
    if w["kind"] == "ueg":
        s = oracle.System.ueg(w["nel"], w["nso"], w["rs"], w["lmax"])
    else:
        s = oracle.System.generic(w["nel"], w["h1"], w["eri"], w["lmax"])
    if w.get("precision") == "fp32":
        s.set_fp32()
    return s


def _pair(ccmc, w, **over):
    """The oracle and a GPU context for one workload.  The GPU context sends
    every spawned record through the sort (sort_all) unless the caller asks
    for the default direct accumulation, so that its spawned multiset can be
    compared with the oracle's."""
    w = dict(w)
    w.setdefault("sort_all", True)
    w.update(over)
    so = _oracle_system(w)
    keys = ("tau", "target_pop", "d0_init", "shift_a", "zeta", "spawn_cutoff", "fnc", "multispawn", "a_thresh",
            "seed", "replica", "n_ranks", "nu_move")
    sim = oracle.Sim(so, **{k: w[k] for k in keys if k in w})
    ctx = ccmc.from_workload(w)
    return so, sim, ctx


def _same_list(sim, ctx):
    ob, ok, op = sim.get_list()
    gb, gk, gp = ctx.get_list()
    assert len(ok) == len(gk)
    assert np.array_equal(ok, gk)
    assert np.array_equal(op, gp)
    assert np.array_equal(ob, gb)


def _same_record(orec, grec):
    o = orec.as_dict() if hasattr(orec, "as_dict") else orec
    for f in INT_FIELDS:
        assert o[f] == grec[f], (f, o[f], grec[f])
    assert o["shift"] == grec["shift"]
    assert abs(o["e_num"] - grec["e_num"]) <= 1e-12 * max(abs(o["e_num"]), 1e-300)


def _same_spawned(sim, ctx):
    ok_, op_ = sim.spawned()
    gk, gp = ctx.get_spawned()
    a = np.lexsort((op_, ok_))
    b = np.lexsort((gp, gk))
    assert np.array_equal(ok_[a], gk[b])
    assert np.array_equal(op_[a], gp[b])
    assert np.array_equal(sim.death(), ctx.get_death())


def _run_lockstep(sim, ctx, nsteps, check_spawned_every=10):
    """Steps both sides together; records and lists must agree after every
    step, spawned multisets every check_spawned_every steps (0: never).
    Returns the GPU's records."""
    grecs = []
    for k in range(nsteps):
        # death deltas belong to the list at the step start: take the oracle's before stepping
        rec = sim.step()
        ctx.step(1)
        grec = ctx.records()[-1]
        grecs.append(grec)
        _same_record(rec, grec)
        if check_spawned_every and k % check_spawned_every == 0:
            gk, gp = ctx.get_spawned()
            ok_, op_ = sim.spawned()
            a = np.lexsort((op_, ok_))
            b = np.lexsort((gp, gk))
            assert np.array_equal(ok_[a], gk[b]) and np.array_equal(op_[a], gp[b])
        _same_list(sim, ctx)
    return grecs


def test_ueg38_ccsd_full_run_bitexact(ccmc):
    """14 e / 38 spin-orbitals, CCSD, original sampling: the whole 200-step run."""
    w = workload("ueg14_m38_ccsd")
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, w["nsteps"])
    st = sim.get_state()
    assert ctx.get_state() == st


def test_ueg38_ccsd_shift_phase_bitexact(ccmc):
    """A low target so that the shift varies: host shift updates match bit for bit."""
    w = workload("ueg14_m38_ccsd", target_pop=800.0)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 300, check_spawned_every=50)
    assert ctx.get_state()[2] is True


def test_ueg114_fnc_multispawn_growth_bitexact(ccmc):
    """14 e / 114 spin-orbitals, CCSDT, full non-composite + multi-spawn: the
    first 60 steps of the run (two 64-bit words per determinant)."""
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 60)


def test_ueg114_long_lockstep_and_determinism(ccmc):
    """600 consecutive steps of the 114 spin-orbital FNC + multi-spawn run in
    lockstep with the oracle (records every step, lists every 50 steps), and
    a second context with the same seed reproducing the run exactly."""
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, ctx = _pair(ccmc, w)
    twin = ccmc.from_workload(w, sort_all=True)
    for k in range(600):
        rec = sim.step()
        ctx.step(1)
        twin.step(1)
        g = ctx.records()
        assert g == twin.records()
        _same_record(rec, g[-1])
        if k % 50 == 49:
            _same_list(sim, ctx)


def test_ueg114_lockstep_from_gpu_checkpoints(ccmc):
    """The 114 spin-orbital FNC + multi-spawn run in the production launch
    configuration (captured CUDA graph on a stream): the GPU state at steps
    1000 and 1980 (list, iteration, shift) is handed to the oracle, and the
    next 20 steps of both agree bit for bit."""
    torch = pytest.importorskip("torch")
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, _ = _pair(ccmc, w)
    stream = torch.cuda.Stream()
    ctx = ccmc.from_workload(w, stream=stream.cuda_stream)
    done = 0
    for start in (1000, 1980):
        ctx.step(start - done)
        bits, _, pop = ctx.get_list()
        it, shift, vary, nprev = ctx.get_state()
        sim.set_list_words(bits, pop)
        sim.set_state(it, shift, bool(vary), nprev)
        ctx.records()
        for _ in range(20):
            rec = sim.step()
            ctx.step(1)
            _same_record(rec, ctx.records()[-1])
        _same_list(sim, ctx)
        done = start + 20


def _full_space_state(so, lmax, n_total, seed):
    keys = so.space_keys(lmax, expand_top=False)
    dets = [so.unrank(int(k)) for k in keys]
    levels = [so.level(d) for d in dets]
    pops = synthetic_populations(levels, n_total, seed)
    bits = np.stack([so.to_words(d) for d in dets])
    return bits, pops


def test_ueg114_full_size_step_bitexact(ccmc):
    """The 114 spin-orbital CCSDT workload at full size: every excitor of the
    108,753-determinant space occupied, N_total = 10^6 (the target), two steps
    in the library's production launch configuration."""
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, ctx = _pair(ccmc, w)
    bits, pops = _full_space_state(so, 3, 1.0e6, seed=21)
    sim.set_list_words(bits, pops)
    ctx.set_list(bits, pops)
    for it in (1500, 1501):
        sim.set_state(it, -0.35, True, 1.0e6)
        ctx.set_state(it, -0.35, True, 1.0e6)
        rec = sim.step()
        ctx.step(1)
        _same_record(rec, ctx.records()[-1])
        assert rec.n_sel > 900_000
        _same_list(sim, ctx)


@pytest.mark.parametrize("multispawn", [False, True])
def test_molecule_full_size_step_bitexact(ccmc, multispawn):
    """The synthetic molecule (20 electrons, 82 spin-orbitals, CCSDTQ, two-word
    determinants) at full size: about 4e6 occupied excitors of levels 0-4 and
    N_total of about 1.2e7, one step in the production launch configuration.
    The step size 0.005 (larger than the benchmark's) makes the annihilation
    heavy: about 7.7e6 spawned records.  Spawned records, death deltas, the
    merged list and the record must match."""
    from ccmc_inputs import molecule_state

    w = workload("mol20_m82_ccsdtq", tau=0.005, multispawn=multispawn)
    h1, eri = molecule_integrals(norb=41, nocc=10, seed=7)
    w.update(h1=h1, eri=eri, nso=82)
    so, sim, ctx = _pair(ccmc, w)
    words, pops, _ = molecule_state()
    ntot = float(np.abs(pops).sum()) / 65536.0
    sim.set_list_words(words, pops)
    ctx.set_list(words, pops)
    sim.set_state(1500, -0.35, True, ntot)
    ctx.set_state(1500, -0.35, True, ntot)
    rec = sim.step()
    ctx.step(1)
    _same_record(rec, ctx.records()[-1])
    assert rec.n_sel > 10_000_000 and rec.n_spawned > 1_000_000
    _same_spawned(sim, ctx)
    _same_list(sim, ctx)


def test_molecule_grown_state_step_bitexact(ccmc):
    """The benchmark's own molecule state: grown on the GPU from the reference
    (tau = 2e-6, target 10^7) until the shift has varied for 400 steps, about
    1.8e7 occupied excitors and N_total = 2.3e7; the next step of GPU and
    oracle from that state agree bit for bit (records and list)."""
    w = workload("mol20_m82_ccsdtq")
    h1, eri = molecule_integrals(norb=41, nocc=10, seed=7)
    w.update(h1=h1, eri=eri, nso=82)
    so, sim, ctx = _pair(ccmc, w, sort_all=False)
    for _ in range(200):
        ctx.step(10)
        if ctx.get_state()[2]:
            break
    ctx.step(400)
    bits, _, pop = ctx.get_list()
    it, shift, vary, nprev = ctx.get_state()
    assert vary and len(pop) > 10_000_000
    sim.set_list_words(bits, pop)
    sim.set_state(it, shift, bool(vary), nprev)
    ctx.records()
    rec = sim.step()
    ctx.step(1)
    _same_record(rec, ctx.records()[-1])
    _same_list(sim, ctx)


@pytest.mark.parametrize("sort_all", [True, False])
def test_molecule_all_samplers_bitexact(ccmc, sort_all):
    """A small molecule-like Hamiltonian (singles exist, so composite clusters
    collapse onto the truncated space and composite death is exercised), with
    every record sorted and with direct accumulation onto listed determinants."""
    h1, eri = molecule_integrals(norb=8, nocc=3, seed=5, scale=0.1)
    base = dict(kind="generic", nel=6, norb=8, nso=16, lmax=3, h1=h1, eri=eri, tau=0.01, target_pop=3000.0,
                d0_init=400.0, shift_a=10, zeta=0.05, spawn_cutoff=2.0 ** -7, a_thresh=1.0, seed=3, replica=0)
    for fnc, ms in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        w = dict(base, fnc=fnc, multispawn=ms)
        so, sim, ctx = _pair(ccmc, w, sort_all=sort_all)
        grecs = _run_lockstep(sim, ctx, 80, check_spawned_every=20 if sort_all else 0)
        if not sort_all:
            assert sum(r["n_direct"] for r in grecs) > 0
        ctx.close()


def test_direct_accumulation_lockstep_ueg114(ccmc):
    """The annihilation fast path (records onto listed determinants added with
    integer atomics, only new keys sorted) on the 114 spin-orbital FNC +
    multi-spawn run at its working population: the GPU grows the run from the
    reference to 10^6 (the path switches itself on once a step spawns more
    than a tenth of the list's size in records), then 40 steps in lockstep
    with the oracle from the GPU's state, records and lists bit for bit, most
    records on the fast path."""
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, _ = _pair(ccmc, w)
    ctx = ccmc.from_workload(w)
    ctx.step(1500)
    bits, _, pop = ctx.get_list()
    it, shift, vary, nprev = ctx.get_state()
    sim.set_list_words(bits, pop)
    sim.set_state(it, shift, bool(vary), nprev)
    ctx.records()
    direct = total = 0
    for k in range(40):
        rec = sim.step()
        ctx.step(1)
        g = ctx.records()[-1]
        _same_record(rec, g)
        direct += g["n_direct"]
        total += g["n_spawned"]
    _same_list(sim, ctx)
    assert direct > total // 2


def test_direct_accumulation_fp32_gas_at_scale(ccmc):
    """The 162 spin-orbital FP32 gas (15,769 determinants, all of them
    occupied at scale) grown on the GPU to a population of 10^6, then two
    steps on both sides from the GPU's state: records and lists bit for bit,
    nearly every record added directly."""
    w = workload("ueg54_m162_ccsd_fp32", target_pop=1e6, d0_init=1e4)
    so, sim, _ = _pair(ccmc, w)
    ctx = ccmc.from_workload(w)
    for _ in range(40):
        ctx.step(10)
        if ctx.get_state()[2]:
            break
    ctx.step(20)
    bits, _, pop = ctx.get_list()
    it, shift, vary, nprev = ctx.get_state()
    sim.set_list_words(bits, pop)
    sim.set_state(it, shift, bool(vary), nprev)
    ctx.records()
    for _ in range(2):
        rec = sim.step()
        ctx.step(1)
        g = ctx.records()[-1]
        _same_record(rec, g)
        assert g["n_spawned"] > 100_000 and g["n_direct"] > 0.9 * g["n_spawned"]
    _same_list(sim, ctx)


def test_three_word_determinants_bitexact(ccmc):
    """54 e / 162 spin-orbitals (three words per determinant), CCSD."""
    w = workload("ueg54_m162_ccsd_fp32", precision="fp64", target_pop=1e5, d0_init=200.0)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 25, check_spawned_every=5)


def test_six_word_determinants_bitexact(ccmc):
    """14 e / 358 spin-orbitals (six words per determinant), CCSDTQ, full
    non-composite sampling with multi-spawn, grown from the reference."""
    w = workload("ueg14_m358_ccsdtq", target_pop=3e4, d0_init=200.0)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 30, check_spawned_every=5)
    assert len(ctx.get_list()[1]) > 1000


def test_distributed_sampling_bitexact(ccmc):
    """The simulated distribution over processors (Sec. III, Eq. ccmc_dist):
    8 processors, owners moving every 4 iterations, on the 66 spin-orbital
    CCSDT gas with full non-composite sampling and multi-spawn, in lockstep
    with the oracle."""
    w = workload("ueg14_m66_ccsdt_rs5", target_pop=2e4, d0_init=300.0, multispawn=True, n_ranks=8, nu_move=2)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 120, check_spawned_every=20)
    # the restriction is active: the same run on one processor differs
    so1, sim1, ctx1 = _pair(ccmc, dict(w, n_ranks=1))
    for _ in range(120):
        ctx1.step(1)
    assert not np.array_equal(ctx1.get_list()[2], ctx.get_list()[2])


def test_distributed_sampling_original_and_many_ranks(ccmc):
    """The restricted composite picks with the original sampler on a small
    molecule (buffered single attempts, singles present), and with 30,000
    processors, where the position table needs chunks of up to 128 entries
    and most processors hold at most one excitor."""
    h1, eri = molecule_integrals(norb=8, nocc=3, seed=5, scale=0.1)
    wm = dict(kind="generic", nel=6, norb=8, nso=16, lmax=3, h1=h1, eri=eri, tau=0.01, target_pop=3000.0,
              d0_init=400.0, shift_a=10, zeta=0.05, spawn_cutoff=2.0 ** -7, a_thresh=1.0, seed=3, replica=0,
              fnc=0, multispawn=0, n_ranks=5, nu_move=0)
    so, sim, ctx = _pair(ccmc, wm)
    _run_lockstep(sim, ctx, 80, check_spawned_every=20)
    w = workload("ueg14_m66_ccsdt_rs5", target_pop=2e5, d0_init=2e4, tau=0.01, multispawn=True, n_ranks=30000,
                 nu_move=3)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 80, check_spawned_every=20)
    assert ctx.get_list()[0].shape[0] > 8000   # 30,000 x ceil(n / 64) > 2^22: 128-entry chunks


def test_colocation_matches_oracle(ccmc):
    """Pair co-location sums of Fig. excitdistrib on the 3,813 excitors of the
    14-electron, 186 spin-orbital CCSD space: GPU and oracle agree exactly."""
    so = oracle.System.ueg(14, 186, 1.0, 2)
    keys = so.space_keys(2, expand_top=False)
    dets = np.stack([so.to_words(so.unrank(int(k))) for k in keys])
    assert len(dets) == 3813     # the paper's 3,813 (the reference included)
    ck = [1, 5, 16, 48]
    for np_, nu in ((32, 4), (7, 0)):
        g1, g2 = ccmc.colocation(dets, np_, nu, ck)
        o1, o2 = oracle.colocation(dets, np_, nu, ck)
        assert np.array_equal(g1, o1) and np.array_equal(g2, o2)


def test_fp32_form_ueg38_bitexact(ccmc):
    """FP32 matrix elements (original sampling): the 200-step run in lockstep
    with the oracle's FP32 form."""
    w = workload("ueg14_m38_ccsd", precision="fp32")
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 200, check_spawned_every=25)


def test_fp32_form_three_words_and_molecule_bitexact(ccmc):
    w = workload("ueg54_m162_ccsd_fp32", target_pop=1e5, d0_init=200.0)
    so, sim, ctx = _pair(ccmc, w)
    _run_lockstep(sim, ctx, 25, check_spawned_every=5)
    h1, eri = molecule_integrals(norb=8, nocc=3, seed=5, scale=0.1)
    wm = dict(kind="generic", nel=6, norb=8, nso=16, lmax=3, h1=h1, eri=eri, tau=0.01, target_pop=3000.0,
              d0_init=400.0, shift_a=10, zeta=0.05, spawn_cutoff=2.0 ** -7, a_thresh=1.0, seed=3, replica=0,
              fnc=1, multispawn=1, precision="fp32")
    so, sim, ctx = _pair(ccmc, wm)
    _run_lockstep(sim, ctx, 60, check_spawned_every=20)


def test_fp32_estimator_accuracy_on_one_state(ccmc):
    """From the same state both precisions draw the same clusters, so the
    projected-energy numerators differ only by the FP32 matrix elements."""
    w = workload("ueg14_m38_ccsd")
    so, sim, ctx = _pair(ccmc, w)
    sim.run(150)
    bits, keys, pops = sim.get_list()
    st = sim.get_state()
    c64 = ccmc.from_workload(w)
    c32 = ccmc.from_workload(w, precision="fp32")
    e = []
    for c in (c64, c32):
        c.set_list(bits, pops)
        c.set_state(*st)
        c.step(1)
        e.append(c.records()[-1]["e_num"])
    rel = abs(e[1] - e[0]) / abs(e[0])
    assert 0.0 < rel < 1e-5


def test_graph_replay_equals_kernel_launches(ccmc):
    """On a stream the step is replayed from a captured CUDA graph; it must
    give the same trajectory as launching the kernels one by one."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    g = ccmc.from_workload(w, stream=s1.cuda_stream)
    e = ccmc.from_workload(w, stream=s2.cuda_stream, use_graph=False)
    for _ in range(8):
        g.step(25)
        e.step(25)
        assert g.records() == e.records()
    for x, y in zip(g.get_list(), e.get_list()):
        assert np.array_equal(x, y)
    _, _, total = g.phase_times()
    assert total > 0


def test_negative_reference_weight(ccmc):
    """A wavefunction with a negative reference weight evolves identically."""
    w = workload("ueg14_m38_ccsd")
    so, sim, ctx = _pair(ccmc, w)
    sim.run(30)
    bits, keys, pops = sim.get_list()
    pops = -pops
    sim.set_list_words(bits, pops)
    ctx.set_list(bits, pops)
    ctx.set_state(*sim.get_state())
    _run_lockstep(sim, ctx, 20, check_spawned_every=5)


def test_death_and_spawned_multisets(ccmc):
    w = workload("ueg14_m114_ccsdt_fnc_ms")
    so, sim, ctx = _pair(ccmc, w)
    for _ in range(15):
        sim.step()
        ctx.step(1)
    _same_spawned(sim, ctx)


def test_checkpoint_resume_is_bitexact(ccmc):
    w = workload("ueg14_m38_ccsd", target_pop=800.0)
    ctx = ccmc.from_workload(w)
    ctx.step(40)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        ctx.save(path)
        ctx.step(30)
        a = ctx.get_list()
        sa = ctx.get_state()
        ctx2 = ccmc.from_workload(w)
        ctx2.load(path)
        ctx2.step(30)
        b = ctx2.get_list()
        assert ctx2.get_state() == sa
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_spawn_overflow_is_reported(ccmc):
    """A spawn buffer that is too small yields CCMC_ERR_SPAWN_OVERFLOW, not a fault."""
    w = workload("ueg14_m38_ccsd", spawn_capacity=4)
    ctx = ccmc.from_workload(w)
    with pytest.raises(ccmc.CCMCError) as e:
        ctx.step(30)
        ctx.sync()
    assert e.value.status == 4


def test_list_overflow_is_reported(ccmc):
    w = workload("ueg14_m38_ccsd", list_capacity=16)
    ctx = ccmc.from_workload(w)
    with pytest.raises(ccmc.CCMCError) as e:
        ctx.step(30)
        ctx.sync()
    assert e.value.status == 7


def test_runaway_population_is_reported(ccmc):
    """A population far above the target (more samples in one step than
    max(64 x target, 2^24)) abandons the step at once with CCMC_ERR_RUNAWAY."""
    w = workload("ueg14_m38_ccsd", target_pop=100.0)
    ctx = ccmc.from_workload(w)
    hf = np.array([[(1 << 14) - 1]], dtype=np.uint64)
    ctx.set_list(hf, np.array([((1 << 24) + 1000) * 65536], dtype=np.int64))
    t = time.perf_counter()
    with pytest.raises(ccmc.CCMCError) as e:
        ctx.step(1)
        ctx.sync()
    assert e.value.status == 9
    assert time.perf_counter() - t < 10.0


def test_runaway_cluster_attempts_are_not_run(ccmc):
    """Multi-spawn with a unit reference weight under 9e6 excitor particles:
    every composite cluster carries ~1e7 or more attempts.  The attempts are
    not run; the step ends quickly with CCMC_ERR_RUNAWAY."""
    w = workload("ueg14_m114_ccsdt_fnc_ms", target_pop=100.0)
    so = oracle.System.ueg(w["nel"], w["nso"], w["rs"], 2)
    keys = so.space_keys(2, expand_top=False)            # reference + doubles, in key order
    bits = np.stack([so.to_words(so.unrank(int(k))) for k in keys])
    pops = np.full(len(keys), 5000 * 65536, dtype=np.int64)
    pops[0] = 65536
    ctx = ccmc.from_workload(w)
    ctx.set_list(bits, pops)
    t = time.perf_counter()
    with pytest.raises(ccmc.CCMCError) as e:
        ctx.step(1)
        ctx.sync()
    assert e.value.status == 9
    assert time.perf_counter() - t < 10.0


def test_rejects_bad_lists(ccmc):
    w = workload("ueg14_m38_ccsd")
    ctx = ccmc.from_workload(w)
    hf = np.array([[(1 << 14) - 1]], dtype=np.uint64)
    with pytest.raises(ccmc.CCMCError):
        ctx.set_list(np.array([[(1 << 13) - 1]], dtype=np.uint64), np.array([65536]))   # 13 electrons
    d = ((1 << 14) - 1) ^ 0b11 ^ (0b11 << 14)
    with pytest.raises(ccmc.CCMCError):
        ctx.set_list(np.array([[d], [(1 << 14) - 1]], dtype=np.uint64), np.array([65536, 65536]))  # HF not first
    single = ((1 << 14) - 1) ^ (1 << 12) ^ (1 << 14)   # alpha 6 -> alpha 7: momentum changes
    with pytest.raises(ccmc.CCMCError):
        ctx.set_list(np.array([[(1 << 14) - 1], [single]], dtype=np.uint64), np.array([65536, 65536]))
    flip = ((1 << 14) - 1) ^ (1 << 13) ^ (1 << 14)      # beta hole, alpha particle: S_z changes
    with pytest.raises(ccmc.CCMCError):
        ctx.set_list(np.array([[(1 << 14) - 1], [flip]], dtype=np.uint64), np.array([65536, 65536]))
    ctx.set_list(hf, np.array([100 * 65536]))


def test_torch_allocator_and_stream(ccmc):
    """Device memory from PyTorch's caching allocator and a torch stream."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    w = workload("ueg14_m38_ccsd")
    s = torch.cuda.Stream()
    so, sim, ctx = _pair(ccmc, w, use_torch_allocator=True, stream=s.cuda_stream)
    _run_lockstep(sim, ctx, 30, check_spawned_every=10)


def test_get_list_without_keys(ccmc):
    """The list download can skip the keys (a NULL buffer at the ABI): the
    bit strings and populations are the same as with them."""
    w = workload("ueg14_m38_ccsd")
    ctx = ccmc.from_workload(w)
    ctx.step(50)
    bits, keys, pop = ctx.get_list()
    b2, k2, p2 = ctx.get_list(with_keys=False)
    assert k2 is None and np.array_equal(bits, b2) and np.array_equal(pop, p2) and len(keys) == len(pop)
    ctx.close()
