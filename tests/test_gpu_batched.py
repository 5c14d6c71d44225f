"""Batched form: replicas of different systems stepped in one launch per
phase must be bit-identical to the same contexts stepped alone."""
import numpy as np
import pytest

from ccmc_inputs import batched_replicas, molecule_integrals, workload

pytestmark = pytest.mark.gpu


def _replica_specs():
    h1, eri = molecule_integrals(norb=8, nocc=3, seed=5, scale=0.1)
    reps = batched_replicas(16)
    chosen = [reps[0], reps[5], reps[10], reps[15]]            # M = 38, 54, 66, 114 (one and two words)
    chosen += [dict(r, lmax=3, replica=100 + i) for i, r in enumerate(batched_replicas(16)[1:3])]   # CCSDT
    chosen.append(workload("ueg14_m114_ccsdt_fnc_ms", target_pop=2e4, replica=7))          # FNC + multi-spawn
    chosen.append(workload("ueg14_m38_ccsd", precision="fp32", replica=8))                  # FP32 group
    chosen.append(dict(kind="generic", nel=6, norb=8, nso=16, lmax=3, h1=h1, eri=eri, tau=0.01, target_pop=3000.0,
                       d0_init=400.0, shift_a=10, zeta=0.05, spawn_cutoff=2.0 ** -7, a_thresh=1.0, seed=3,
                       replica=9, fnc=0, multispawn=0))
    return chosen


def test_batched_equals_plain(ccmc_lib=None):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    import paper_1807_03749_gb300 as ccmc

    specs = _replica_specs()
    stream = torch.cuda.Stream()
    batch_ctx = [ccmc.from_workload(w) for w in specs]
    plain_ctx = [ccmc.from_workload(w) for w in specs]
    b = ccmc.Batch(batch_ctx, stream.cuda_stream)
    for chunk in (13, 27, 40):          # the first call tunes on its first steps
        b.step(chunk)
        for c in plain_ctx:
            c.step(chunk)
        for cb, cp in zip(batch_ctx, plain_ctx):
            rb, rp = cb.records(), cp.records()
            assert rb == rp
            for x, y in zip(cb.get_list(), cp.get_list()):
                assert np.array_equal(x, y)
            assert cb.get_state() == cp.get_state()
    info = b.info()
    assert info["groups"] == 3 and info["work_blocks"] in (32, 64, 128, 256) and info["digit_bits"] in (6, 8)
    assert info["sample_tile"] in (256, 512, 1024, 2048, 4096) and info["tunings"] >= 1


def test_batch_members_are_not_stepped_alone():
    """While a context belongs to a batch, stepping it alone is refused (the
    batch owns its step sequence) and it cannot join a second batch; after
    the batch is released it steps normally."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    import paper_1807_03749_gb300 as ccmc

    stream = torch.cuda.Stream()
    w = workload("ueg14_m38_ccsd")
    a, c = ccmc.from_workload(w), ccmc.from_workload(w, replica=1)
    b = ccmc.Batch([a, c], stream.cuda_stream)
    b.step(3)
    with pytest.raises(ccmc.CCMCError) as e:
        a.step(1)
    assert e.value.status == 8
    with pytest.raises(ccmc.CCMCError):
        ccmc.Batch([a], stream.cuda_stream)
    b.close()
    a.step(2)
    assert a.get_state()[0] == 5


def test_batch_member_freed_before_the_batch():
    """Freeing a member context first detaches it: the batch then refuses to
    step (its graph still points at the freed memory) and can be freed; the
    other member stays usable."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    import paper_1807_03749_gb300 as ccmc

    stream = torch.cuda.Stream()
    w = workload("ueg14_m38_ccsd")
    a, c = ccmc.from_workload(w), ccmc.from_workload(w, replica=1)
    b = ccmc.Batch([a, c], stream.cuda_stream)
    b.step(3)
    a.close()
    with pytest.raises(ccmc.CCMCError) as e:
        b.step(1)
    assert e.value.status == 8
    b.close()
    c.step(2)
    assert c.get_state()[0] == 5


def test_member_reads_wait_for_the_batch_stream():
    """Reads of a member right after ccmc_step_batched (work still pending on
    the batch's stream, no shift boundary reached) see the state after the
    issued steps: the same list as after an explicit synchronisation and as
    the same context stepped alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    import paper_1807_03749_gb300 as ccmc

    stream = torch.cuda.Stream()
    w = workload("ueg14_m114_ccsdt_fnc_ms", target_pop=2e4)
    a = ccmc.from_workload(w)
    ref = ccmc.from_workload(w)
    b = ccmc.Batch([a], stream.cuda_stream)
    b.step(40)      # tuning and growth, ends on a shift boundary
    ref.step(40)
    b.step(3)       # no boundary: returns with the steps in flight
    ref.step(3)
    early = a.get_list()
    torch.cuda.synchronize()
    late = a.get_list()
    want = ref.get_list()
    for x, y, z in zip(early, late, want):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    assert a.records()[-1] == ref.records()[-1]
    b.close()


def test_sixty_four_replicas_equal_plain():
    """The full 64-replica recipe (every M x r_s x truncation combination) at
    small targets: the batched step gives every replica the lists and records
    it gets stepped alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA")
    import paper_1807_03749_gb300 as ccmc

    reps = [dict(w, target_pop=w["target_pop"] / 100.0, d0_init=20.0, list_capacity=0) for w in batched_replicas(64)]
    stream = torch.cuda.Stream()
    bctx = [ccmc.from_workload(w) for w in reps]
    pctx = [ccmc.from_workload(w) for w in reps]
    b = ccmc.Batch(bctx, stream.cuda_stream)
    b.step(80)
    for c in pctx:
        c.step(80)
    for cb, cp in zip(bctx, pctx):
        assert cb.records() == cp.records()
        for x, y in zip(cb.get_list(), cp.get_list()):
            assert np.array_equal(x, y)
    b.close()
