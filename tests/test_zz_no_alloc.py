"""The allocation-free entry point (pfac_match_noalloc) against the regular
one (pfac_match).

pfac_match_noalloc serves callers that cannot allocate device memory when
they match (allocator callbacks, latency-critical loops, fixed memory
budgets); it takes its scratch from an array built into the library.  This
file is named so that pytest collects it last.  Each call goes through the
C ABI and must give exactly the keys pfac_match gives (integer output, so the
tolerance is zero), on calls in a row that reuse the shared scratch array.
"""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import to_device

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
