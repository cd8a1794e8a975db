"""The allocation-free sort entry point, vis_sort_pairs_noalloc, against vis_sort_pairs.

Callers that cannot allocate device memory where they sort (a real-time loop with a
fixed budget, a plug-in whose host owns every allocation) use the library's static
device scratch instead of a workspace. Its output must equal the workspace sort's
bit for bit (the sort's parity bar), on two calls in a row through the C ABI: the
second call, smaller than the first, checks that what the shared scratch keeps from
the previous call does not leak into the result. This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

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
    return ko, vo


def test_noalloc_sort_equals_workspace_sort_on_two_calls():
    import torch
    for m, seed, bits in ((900_000, 1, 45), (70_001, 2, 45)):
        keys, _ = synth.random_keys(m, seed, "random")
        vals = np.random.default_rng(seed).permutation(m).astype(np.uint32)
        k = torch.from_numpy(keys.view(np.int64)).cuda()
        v = torch.from_numpy(vals.view(np.int32)).cuda()
        ref_k, ref_v = vis.sort_pairs(k, v, bits)
        got_k, got_v = _noalloc(k, v, bits)
        torch.cuda.synchronize()
        assert torch.equal(got_k, ref_k)
        assert torch.equal(got_v, ref_v)


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
