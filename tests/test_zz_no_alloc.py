"""The allocation-free sort entry point, vis_sort_pairs_noalloc.

Callers that cannot allocate device memory where they sort (a real-time loop with a
fixed budget, a plug-in whose host owns every allocation) use the library's static
device scratch instead of a workspace. Its output must equal the oracle's stable sort
bit for bit (the sort's parity bar) and the workspace sort's, on calls in a row through
the C ABI: each later call, smaller than the one before, checks that what the shared
scratch keeps from the previous call does not leak into the result. Key widths cover one
to eight radix passes, odd pass counts (whose first pass writes the caller's output
rather than the scratch) included, and sizes up to the scratch's limit of 2^20 keys.
This file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(keys, vals, key_bits):
    import torch
    L = vis.lib()
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    st = L.vis_sort_pairs_noalloc(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
                                  C.c_void_p(ko.data_ptr()), C.c_void_p(vo.data_ptr()),
                                  C.c_int64(keys.numel()), C.c_int(key_bits),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vis.VIS_OK, vis.vis_last_error()
    st = L.vis_sort_noalloc_check(C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == vis.VIS_OK, vis.vis_last_error()
    return ko, vo


def _inputs(m, bits, seed):
    rng = np.random.default_rng(seed)
    if bits == 45:
        keys, _ = synth.random_keys(m, seed, "random")
    else:
        hi = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        keys = rng.integers(0, np.iinfo(np.uint64).max, m, dtype=np.uint64, endpoint=True) & hi
        if bits <= 13:   # many equal keys: stability decides the order
            keys = keys & np.uint64(0xFF0 if bits > 8 else 0x3C)
    vals = rng.permutation(m).astype(np.uint32)
    return np.ascontiguousarray(keys, np.uint64), vals


# (m, key_bits) in call order: every call smaller than the one before, so leftovers of a
# larger sort sit in the shared scratch when the next one runs
CALLS = ((1 << 20, 64), ((1 << 20) - 1, 37), (900_000, 45), (70_001, 17), (65_537, 13), (4097, 8), (2, 45), (1, 64))


def test_noalloc_sort_equals_stable_sort_on_calls_in_a_row():
    import torch
    for i, (m, bits) in enumerate(CALLS):
        keys, vals = _inputs(m, bits, 11 + i)
        k = torch.from_numpy(keys.view(np.int64)).cuda()
        v = torch.from_numpy(vals.view(np.int32)).cuda()
        got_k, got_v = _noalloc(k, v, bits)
        ref_k, ref_v = vis.sort_pairs(k, v, bits)
        torch.cuda.synchronize()
        ek, ev = oracle.stable_sort_pairs(keys, vals)
        gk, gv = got_k.cpu().numpy().view(np.uint64), got_v.cpu().numpy().view(np.uint32)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev), (m, bits)
        assert torch.equal(got_k, ref_k) and torch.equal(got_v, ref_v), (m, bits)


def test_noalloc_sort_rejects_more_keys_than_its_scratch():
    import torch
    L = vis.lib()
    buf = torch.empty(16, dtype=torch.int64, device="cuda")
    too_many = (1 << 20) + 1
    st = L.vis_sort_pairs_noalloc(C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr() + 64),
                                  C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr() + 64),
                                  C.c_int64(too_many), C.c_int(45), C.c_void_p(0))
    assert st == vis.VIS_ERR_INVALID_ARG
    assert "limit" in vis.vis_last_error()
