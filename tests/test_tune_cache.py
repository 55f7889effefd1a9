"""The autotuner's cache on CPU (a cache hit touches no device): a cached
choice is applied to the table, and a cached line that makes no plan (an
edited or foreign cache) is ignored rather than left to break every later
match."""
import math

import numpy as np
import pytest
import torch

import workloads

pfac = pytest.importorskip("paper_1704_02272_gb300")

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="the cache key names the GPU; this test keys it for none")


def cache_key(t, n_bytes, n_segments):
    i = t.info()
    # record format: 0 packed, 1 / 2 / 8 bitmap words, 3 dense rows
    fmt = {4: 0, 8: 1, 16: 2, 48: 8, 0: 3}[i["record_bytes"]]
    merged = "m" if i["merged_trie_nodes"] else ""
    return (f"sigma={i['alphabet_size']},n={i['n_patterns']},maxlen={i['max_len']},"
            f"rec={fmt}{merged},segs={'many' if n_segments > 1 else 'one'},"
            f"bytes=2^{int(math.log2(n_bytes))},gpu=unknown")


def sample():
    text = torch.zeros(1 << 16, dtype=torch.uint8)
    seg = torch.tensor([0, 1 << 16], dtype=torch.int64)
    return text, seg


def test_cached_choice_is_applied(tmp_path):
    w = workloads.config4(256, 1000, n_bytes=1 << 12)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as t:
        text, seg = sample()
        path = tmp_path / "tune.txt"
        # variant, depth, copies, masks, gram, bytes, warps, ms
        path.write_text(f"{cache_key(t, text.numel(), 1)} 1 2 1 1 2 1 24 0.5\n")
        r = pfac.autotune(t, text, seg, cache_path=str(path), stream=0)
        assert r["from_cache"] == 1 and r["warps_per_cta"] == 24 and r["gram_filter"] == 2
        p = pfac.plan(t)
        assert (p["variant"], p["prefix_depth"], p["warps_per_cta"], p["gram_filter"]) == (1, 2, 24, 2)


@pytest.mark.parametrize("line", ["1 2 1 1 2 1 20 0.5",    # no such CTA width
                                  "1 2 3 1 1 1 16 0.5",    # copies not a power of two
                                  "7 2 1 1 1 1 16 0.5",    # no such variant
                                  "1 2 1 1 2 2 16 0.5"])   # gram filter and prefix bytes
def test_cached_line_without_a_plan_is_ignored(tmp_path, line):
    w = workloads.config4(256, 1000, n_bytes=1 << 12)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as t:
        text, seg = sample()
        default = pfac.plan(t)
        path = tmp_path / "tune.txt"
        path.write_text(f"{cache_key(t, text.numel(), 1)} {line}\n")
        # with the line ignored the tuner times candidates, which needs a GPU
        with pytest.raises(pfac.PfacError):
            pfac.autotune(t, text, seg, cache_path=str(path), stream=0)
        assert pfac.plan(t) == default


def test_cached_resolver_is_applied(tmp_path):
    # a line with the records per slice and the resolver (12 tokens)
    w = workloads.config4(256, 1000, n_bytes=1 << 12)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as t:
        text, seg = sample()
        path = tmp_path / "tune.txt"
        path.write_text(f"{cache_key(t, text.numel(), 1)} 1 2 1 1 2 1 16 1 32 1 0.5\n")
        r = pfac.autotune(t, text, seg, cache_path=str(path), stream=0)
        assert r["from_cache"] == 1 and r["resolver"] == 1 and r["records_per_slice"] == 32
        p = pfac.plan(t)
        assert (p["scan_kernel"], p["records_per_slice"], p["resolver"]) == (1, 32, 1)
