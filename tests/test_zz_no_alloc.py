"""The allocation-free compaction entry point (dash_compact_dynamic_noalloc)
must give exactly what dash_compact_dynamic gives, call after call, although
its scratch array is shared and keeps the previous call's contents.  It
exists for callers that must not allocate device memory while they run.
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_compaction_matches_workspace_form_two_calls(dashlib):
    rng = np.random.default_rng(99)
    n_max = 3_000_000
    idx_ws = torch.empty(n_max, dtype=torch.int32, device="cuda")
    idx_na = torch.full((n_max,), -1, dtype=torch.int32, device="cuda")
    cnt_ws = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt_na = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    # a large call, then a smaller one with a different density: the second
    # must not see anything the first left in the shared scratch
    for n, p in ((n_max, 0.5), (777_777, 0.13)):
        mask = torch.from_numpy((rng.random(n) < p).astype(np.uint8)).cuda()
        dashlib.dash_compact_dynamic(mask, idx_out=idx_ws, count_out=cnt_ws)
        dashlib.dash_compact_dynamic_noalloc(mask, idx_na, cnt_na)
        torch.cuda.synchronize()
        c = int(cnt_ws.item())
        assert int(cnt_na.item()) == c
        assert torch.equal(idx_na[:c], idx_ws[:c])
        assert c == int(mask.sum().item())


def test_noalloc_compaction_rejects_oversized_input(dashlib):
    import ctypes
    big = (1 << 28) + 1  # one entry beyond the built-in limit; nothing is launched
    rc = dashlib._lib.dash_compact_dynamic_noalloc(ctypes.c_void_p(0x1000), big, ctypes.c_void_p(0x1000),
                                                   ctypes.c_void_p(0x1000), None)
    assert rc == dashlib.ERR_UNSUPPORTED
    assert b"limit" in dashlib._lib.dash_last_error()
