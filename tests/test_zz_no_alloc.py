"""The allocation-free entry point (pfac_match_noalloc) against the regular
one (pfac_match).

pfac_match_noalloc serves callers that cannot allocate device memory when
they match (allocator callbacks, latency-critical loops, fixed memory
budgets); it takes its scratch from an array built into the library.  This
file is named so that pytest collects it last.  Each call goes through the
C ABI and must give exactly the keys pfac_match gives (integer output, so the
tolerance is zero), on calls in a row that reuse the shared scratch array.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


def noalloc_keys(table, text, seg, cap):
    dev = text.device
    out = torch.full((cap,), -1, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    st = torch.full((1,), 99, dtype=torch.int32, device=dev)
    pfac.match_noalloc(table, text, seg, out, cnt, st)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert int(st.item()) == 0
    assert n <= cap
    return out[:n]


def test_noalloc_matches_regular_entry_point_on_calls_in_a_row():
    cases = [
        workloads.config3(n_bytes=24 << 20, n_patterns=20000),   # packets, many segments
        workloads.config2(n_bytes=48 << 20, n_patterns=10000),   # one segment, DNA
        workloads.config3(n_bytes=24 << 20, n_patterns=20000),   # the first one again
    ]
    tables = {}
    for i, w in enumerate(cases):
        key = (w.sigma, len(w.patterns), w.name)
        if key not in tables:
            tables[key] = pfac.Table(w.patterns, w.sigma)
        t = tables[key]
        text, seg = to_device(w)
        ref = pfac.match(t, text, seg)
        torch.cuda.synchronize()
        got = noalloc_keys(t, text, seg, ref.numel() + 64)
        assert got.numel() == ref.numel() > 0, f"call {i}"
        assert torch.equal(got, ref), f"call {i}: keys differ"
    for t in tables.values():
        t.close()


def device_memory_state():
    """What an allocation would change: the driver's free device memory, the
    device's stream-ordered pool (used and reserved bytes) and torch's
    caching allocator.  Read through the driver library, which every GPU
    machine has."""
    cu = ctypes.CDLL("libcuda.so.1")
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0      # USED_MEM_CURRENT
    assert cu.cuMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0  # RESERVED_MEM_CURRENT
    return {"free": free.value, "pool_used": used.value, "pool_reserved": reserved.value,
            "torch_allocated": torch.cuda.memory_allocated(),
            "torch_reserved": torch.cuda.memory_reserved()}


def test_noalloc_allocates_nothing_and_matches_the_oracle():
    # the entry point's defining property: once the library's kernels are
    # loaded (a first call), a call changes no allocation anywhere
    w = workloads.config3(n_bytes=8 << 20, n_patterns=5000)
    with pfac.Table(w.patterns, w.sigma) as t:
        text, seg = to_device(w)
        cap = 1 << 16
        out = torch.full((cap,), -1, dtype=torch.int64, device=text.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=text.device)
        st = torch.full((1,), 99, dtype=torch.int32, device=text.device)
        pfac.match_noalloc(t, text, seg, out, cnt, st)  # loads kernels, looks up the array
        torch.cuda.synchronize()
        out.fill_(-1)
        cnt.zero_()
        torch.cuda.synchronize()
        before = device_memory_state()
        pfac.match_noalloc(t, text, seg, out, cnt, st)
        torch.cuda.synchronize()
        after = device_memory_state()
        assert after == before, f"memory changed during the call: {before} -> {after}"
        n = int(cnt.item())
        assert int(st.item()) == 0 and 0 < n <= cap
        # this call's keys, element by element, against the oracle
        assert_same(keys_np(out[:n]), oracle_keys(w), "noalloc vs oracle")


def test_noalloc_rejects_inputs_beyond_its_scratch():
    w = workloads.tiny_case(5, 4, 50, 2, 8, 1000)
    with pfac.Table(w.patterns, 4) as t:
        n = 80 << 20
        text = torch.zeros(n, dtype=torch.uint8, device="cuda")
        seg = torch.tensor([0, n], dtype=torch.int64, device="cuda")
        out = torch.empty(16, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match_noalloc(t, text, seg, out, cnt, st)
        assert ei.value.status == -1 and "scratch" in str(ei.value)
