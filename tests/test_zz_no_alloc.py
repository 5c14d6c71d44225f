"""The allocation-free sort-and-reduce entry point (ccmc_reduce_records_noalloc).

It serves callers that cannot allocate device memory; its result must equal
the annihilation's own records taken through the existing entry points
(ccmc_step + ccmc_get_spawned), summed per key.  Two calls in a row check
that the shared scratch is reset between calls.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_reduce_matches_step_records():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    lib = ccmc.load()
    ctx = ccmc.from_workload(workload("ueg14_m114_ccsdt_fnc_ms"))
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream()
    for call in range(2):
        ctx.step(30 + 20 * call)
        keys, pops = ctx.get_spawned()          # records that entered the annihilation
        assert 0 < len(keys) <= 65536
        want_k, inv = np.unique(keys, return_inverse=True)
        want_p = np.zeros(len(want_k), dtype=np.int64)
        np.add.at(want_p, inv, pops)
        perm = rng.permutation(len(keys))       # any input order
        dk = torch.from_numpy(keys[perm].view(np.int64).copy()).cuda()
        dp = torch.from_numpy(pops[perm].copy()).cuda()
        ok = torch.full_like(dk, -1)
        op = torch.full_like(dp, 123)
        n_out = ctypes.c_size_t(0)
        bits = max(1, int(keys.max()).bit_length())
        st = lib.ccmc_reduce_records_noalloc(_ptr(dk), _ptr(dp), len(keys), bits, _ptr(ok), _ptr(op),
                                             ctypes.byref(n_out), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        m = n_out.value
        assert m == len(want_k)
        got_k = ok[:m].cpu().numpy().view(np.uint64)
        got_p = op[:m].cpu().numpy()
        assert np.array_equal(got_k, want_k)
        assert np.array_equal(got_p, want_p)


def test_noalloc_rejects_oversized_input():
    import paper_1807_03749_gb300 as ccmc

    lib = ccmc.load()
    n_out = ctypes.c_size_t(7)
    st = lib.ccmc_reduce_records_noalloc(None, None, 65537, 20, None, None, ctypes.byref(n_out), None)
    assert st == 1 and n_out.value == 0
