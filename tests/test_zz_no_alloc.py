"""The allocation-free compaction entry point (dash_compact_dynamic_noalloc),
for callers that must not allocate device memory while they run: a render
loop that owns all device memory and hands its plug-ins only buffers
allocated up front, or code inside a memory allocator's own callbacks, where
a cudaMalloc would re-enter the allocator.  It must give exactly what
dash_compact_dynamic and the oracle's compaction give, call after call,
although its scratch array is shared and keeps the previous call's contents,
and, once warmed up on the device, it must allocate nothing.

This file is collected last (its name sorts after every other test file):
a run that stops at the first failure (pytest -x) has then already run every
other test before this one can stop it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

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


def test_noalloc_compaction_matches_oracle(dashlib):
    rng = np.random.default_rng(98)
    for n in (1, 4095, 4097, 100_003):  # one CTA, a ragged last CTA, many CTAs
        mask = (rng.random(n) < 0.37).astype(np.uint8) * rng.integers(1, 256, n).astype(np.uint8)
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        dashlib.dash_compact_dynamic_noalloc(torch.from_numpy(mask).cuda(), idx, cnt)
        ref_idx, ref_cnt = oracle.compact(mask)
        assert int(cnt.item()) == ref_cnt
        assert np.array_equal(idx[:ref_cnt].cpu().numpy(), ref_idx)


def test_noalloc_compaction_allocates_nothing(dashlib):
    rng = np.random.default_rng(97)
    n = 1_000_000
    mask = torch.from_numpy((rng.random(n) < 0.5).astype(np.uint8)).cuda()
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    dashlib.dash_compact_dynamic_noalloc(mask, idx, cnt)   # warm-up: loads the kernels on this device
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        dashlib.dash_compact_dynamic_noalloc(mask, idx, cnt)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == torch_before
    assert free_after == free_before
    assert int(cnt.item()) == int(mask.sum().item())


def test_noalloc_compaction_rejects_oversized_input(dashlib):
    big = (1 << 28) + 1  # one entry beyond the built-in limit; nothing is launched
    rc = dashlib._lib.dash_compact_dynamic_noalloc(ctypes.c_void_p(0x1000), big, ctypes.c_void_p(0x1000),
                                                   ctypes.c_void_p(0x1000), None)
    assert rc == dashlib.ERR_UNSUPPORTED
    assert b"limit" in dashlib._lib.dash_last_error()
