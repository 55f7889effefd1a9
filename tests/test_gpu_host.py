"""pfac_match_host: host text in, host keys out, the copies pipelined
against the matching chunk by chunk.  The keys must equal the device-buffer
call's (and the oracle's) for chunk sizes that cut segments and patterns at
every kind of place, with pinned and pageable buffers; a chunk with more
keys than a device slot holds is matched again on its own; a short output
buffer gives the two-call convention."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


def host_args(w, pinned=True):
    text = torch.from_numpy(w.text.copy())
    seg = torch.from_numpy(w.seg_offsets.astype(np.int64))
    if pinned:
        text, seg = text.pin_memory(), seg.pin_memory()
    return text, seg


def host_keys(t, w, chunk, pinned=True, cap=None, **opt):
    text, seg = host_args(w, pinned)
    out = torch.empty(cap if cap is not None else 1 << 22, dtype=torch.int64)
    if pinned:
        out = out.pin_memory()
    n = pfac.match_host(t, text, seg, out, chunk_bytes=chunk, **opt)
    return out[:n].numpy().view(np.uint64).copy(), n


CASES = {
    "dna": lambda: workloads.config2(n_bytes=5 << 20, n_patterns=3000),
    "packets": lambda: workloads.config3(n_bytes=6 << 20, n_patterns=4000),
    "tiny-segs": lambda: workloads.tiny_case(5, 4, 200, 1, 9, 300_001, n_segments=7000,
                                             n_plants=500),
    "sigma256": lambda: workloads.tiny_case(6, 256, 2000, 2, 60, 2_000_000, n_plants=3000),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("chunk", [256, 4096, 1 << 20, 0])
def test_host_path_equals_device_path(case, chunk):
    w = CASES[case]()
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma) as t:
        want = keys_np(pfac.match(t, text, seg))
        got, n = host_keys(t, w, chunk)
    assert n == want.size
    assert_same(got, want, f"{case} chunk {chunk}")
    if chunk == 4096:
        assert_same(got, oracle_keys(w), f"{case} vs oracle")


def test_host_path_pageable_and_options():
    w = CASES["packets"]()
    with pfac.Table(w.patterns, w.sigma) as t:
        a, _ = host_keys(t, w, 1 << 20)
        b, _ = host_keys(t, w, 1 << 20, pinned=False)
        c, _ = host_keys(t, w, 1 << 20, gram_filter=2)
    assert_same(b, a, "pageable")
    assert_same(c, a, "gram filter")


def test_host_path_chunk_overflow_and_enospc():
    # all-zero text, alphabet 1: every position matches every pattern that
    # fits, far more keys per chunk than a device slot holds
    pats = [bytes(k) for k in (1, 2, 3, 5, 8)]
    text = np.zeros(600_000, np.uint8)
    w = workloads.Workload("zeros", 1, pats, text, workloads.single_segment(text.size))
    want = sum(text.size - len(p) + 1 for p in pats)
    with pfac.Table(w.patterns, w.sigma) as t:
        got, n = host_keys(t, w, 512 << 10, cap=want + 10)
        assert n == want
        assert_same(got, oracle_keys(w), "overflowed chunks")
        with pytest.raises(pfac.PfacError) as ei:
            host_keys(t, w, 512 << 10, cap=1000)
        assert ei.value.status == -5  # PFAC_ENOSPC
