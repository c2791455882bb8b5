"""Allocation-free top-k (gsp_topk_mask_static) against the workspace version
and the oracle.

Some callers cannot allocate device memory at the moment they call the
library: real-time loops that forbid allocation once they run, and host
applications whose device memory is owned by their own allocator, where a
plug-in may not take memory behind its back.  gsp_topk_mask_static serves
them with its scratch in a static device array.  This test calls it through
the C ABI twice in a row (the second call sees the array as the first left
it) and requires the same masks and counts as gsp_topk_mask on the same
scores and as the oracle's top-k (selection is integer work: exact
equality).  It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import densify as od

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_topk_matches_workspace_topk_on_two_calls(gsp_lib):
    import torch
    L = gsp_lib._lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(7)
    for n, k in ((300_000, 30_000), (5_000, 4_999)):
        s = (rng.integers(0, 200, n) * 0.5).astype(np.float32)  # many ties at the threshold
        scores = torch.from_numpy(s).cuda()
        count = torch.tensor([n], dtype=torch.int32, device="cuda")
        ref_mask, ref_sel, ref_st = gsp_lib.topk_mask(scores, count, k)
        mask = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        sel = torch.zeros(1, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = L.gsp_topk_mask_static(_p(scores), _p(count), n, k, _p(mask), _p(sel), _p(status), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0 and int(ref_st.item()) == 0
        assert torch.equal(mask, ref_mask)
        assert int(sel.item()) == int(ref_sel.item()) == k
        assert np.array_equal(mask.cpu().numpy().astype(bool), od.topk_mask(s, k))


def test_static_topk_rejects_capacity_beyond_its_maximum(gsp_lib):
    import torch
    L = gsp_lib._lib.load()
    scores = torch.zeros(4, device="cuda")
    count = torch.tensor([4], dtype=torch.int32, device="cuda")
    mask = torch.zeros(4, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    too_big = gsp_lib._lib.GSP_TOPK_STATIC_MAX_CAPACITY + 1
    rc = L.gsp_topk_mask_static(_p(scores), _p(count), too_big, 1, _p(mask), None, _p(status), None)
    assert rc == gsp_lib._lib.GSP_ERR_INVALID_ARG
