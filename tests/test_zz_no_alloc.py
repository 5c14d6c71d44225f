"""The allocation-free sort-and-reduce entry point (ccmc_reduce_records_noalloc).

It serves callers that may not allocate device memory (a host application
that owns the device allocator, a loop with a fixed device-memory
footprint).  Its result must equal the annihilation's own records taken
through the existing entry points (ccmc_step + ccmc_get_spawned), summed per
key, and the sum per key of any record set (np.unique + np.add.at).  Every
case runs two calls in a row, which checks that the shared scratch (which
keeps the previous call's contents) is reset between calls.  This file is
collected last.
"""
import ctypes
import zlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NOALLOC_MAX = 65536


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _reduce(lib, torch, keys, pops, key_bits, stream):
    """One call through the C ABI; returns (distinct keys, summed weights)."""
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dp = torch.from_numpy(pops.copy()).cuda()
    ok = torch.full_like(dk, -1)
    op = torch.full_like(dp, 123)          # stale values that must be overwritten
    n_out = ctypes.c_size_t(0)
    handle = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    torch.cuda.synchronize()
    st = lib.ccmc_reduce_records_noalloc(_ptr(dk), _ptr(dp), len(keys), key_bits, _ptr(ok), _ptr(op),
                                         ctypes.byref(n_out), handle)
    assert st == 0
    m = n_out.value
    return ok[:m].cpu().numpy().view(np.uint64), op[:m].cpu().numpy()


def _expected(keys, pops):
    want_k, inv = np.unique(keys, return_inverse=True)
    want_p = np.zeros(len(want_k), dtype=np.int64)
    np.add.at(want_p, inv, pops)
    return want_k, want_p


def test_noalloc_reduce_matches_step_records():
    torch = _torch()
    import paper_1807_03749_gb300 as ccmc
    from ccmc_inputs import workload

    lib = ccmc.load()
    ctx = ccmc.from_workload(workload("ueg14_m114_ccsdt_fnc_ms"), sort_all=True)
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream()
    for call in range(2):
        ctx.step(30 + 20 * call)
        keys, pops = ctx.get_spawned()          # records that entered the annihilation
        assert 0 < len(keys) <= NOALLOC_MAX
        want_k, want_p = _expected(keys, pops)
        perm = rng.permutation(len(keys))       # any input order
        bits = max(1, int(keys.max()).bit_length())
        got_k, got_p = _reduce(lib, torch, keys[perm], pops[perm], bits, stream)
        assert np.array_equal(got_k, want_k)
        assert np.array_equal(got_p, want_p)


# (records, key bits, distinct-key range, stream): one radix pass (<= 8
# bits), an even pass count (16 bits: the result is read from the second
# scratch buffer), the full 64-bit range (8 passes), the maximum record
# count, all keys equal, a single record, and the legacy NULL stream.
CASES = [
    ("one_pass", 5000, 8, 1 << 8, "torch"),
    ("two_passes", 20000, 16, 3000, "torch"),
    ("three_passes_null_stream", 30000, 20, 1 << 20, None),
    ("full_64_bit_keys", 40000, 64, None, "torch"),
    ("maximum_count", NOALLOC_MAX, 27, 1 << 27, "torch"),
    ("all_keys_equal", NOALLOC_MAX, 33, 1, "torch"),
    ("single_record", 1, 12, 1 << 12, None),
]


@pytest.mark.parametrize("name,n,key_bits,span,stream_kind", CASES, ids=[c[0] for c in CASES])
def test_noalloc_reduce_edges(name, n, key_bits, span, stream_kind):
    torch = _torch()
    import paper_1807_03749_gb300 as ccmc

    lib = ccmc.load()
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    stream = torch.cuda.Stream() if stream_kind == "torch" else None
    for call in range(2):
        if span is None:       # keys over the whole 64-bit range, with repeats
            base = rng.integers(0, 1 << 63, size=max(1, n // 4), dtype=np.uint64) * np.uint64(2)
            base |= rng.integers(0, 2, size=len(base), dtype=np.uint64)
            keys = base[rng.integers(0, len(base), size=n)]
        elif span == 1:
            keys = np.full(n, (1 << key_bits) - 1 - call, dtype=np.uint64)
        else:
            keys = rng.integers(0, span, size=n, dtype=np.uint64)
        keys = keys & np.uint64((1 << key_bits) - 1 if key_bits < 64 else 0xFFFFFFFFFFFFFFFF)
        pops = rng.integers(-(1 << 40), 1 << 40, size=n, dtype=np.int64)
        if call == 1 and n > 1:
            pops[1] = -pops[0]                  # a run may sum to zero; it is kept
            keys[1] = keys[0]
        want_k, want_p = _expected(keys, pops)
        got_k, got_p = _reduce(lib, torch, keys, pops, key_bits, stream)
        assert np.array_equal(got_k, want_k), name
        assert np.array_equal(got_p, want_p), name


def test_noalloc_rejects_oversized_input():
    import paper_1807_03749_gb300 as ccmc

    lib = ccmc.load()
    n_out = ctypes.c_size_t(7)
    st = lib.ccmc_reduce_records_noalloc(None, None, NOALLOC_MAX + 1, 20, None, None, ctypes.byref(n_out), None)
    assert st == 1 and n_out.value == 0
