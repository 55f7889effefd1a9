"""GPU sharding: one job split into k shards with the shard plan, each shard
matched on the GPU with its start range and global offset (the library
starts no walk in the read halo and reports global positions), the lists
concatenated in shard order.  The merged list must equal the unsharded
match and the oracle.  One GPU runs the shards one after another."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")
from paper_1704_02272_gb300 import shard  # noqa: E402

CASES = {
    "dna": lambda: workloads.config2(n_bytes=6 << 20, n_patterns=3000),
    "packets": lambda: workloads.config3(n_bytes=8 << 20, n_patterns=4000),
    "tiny-segs": lambda: workloads.tiny_case(7, 4, 200, 1, 9, 200_000, n_segments=5000,
                                             n_plants=400),
    "sigma256": lambda: workloads.tiny_case(9, 256, 3000, 2, 40, 3_000_003, n_plants=3000),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("world", [2, 3, 7])
@pytest.mark.parametrize("layout", ["compressed", "dense"])
def test_shards_merge_to_unsharded(case, world, layout):
    w = CASES[case]()
    lay = pfac.LAYOUT_COMPRESSED if layout == "compressed" else pfac.LAYOUT_DENSE
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma, layout=lay) as t:
        whole = pfac.match(t, text, seg)
        parts = [shard.match_shard_gpu(t, text, s)
                 for s in shard.plan(w.n_bytes, w.seg_offsets, world, w.max_len)]
        torch.cuda.synchronize()
    merged = torch.cat(parts)
    assert merged.numel() == whole.numel() and torch.equal(merged, whole)
    if world == 3 and layout == "compressed":
        assert_same(keys_np(merged), oracle_keys(w), f"{case} sharded vs oracle")


def test_start_range_and_position_base():
    # starts_end keeps walks from starting at or past it while they still read
    # beyond; position_base shifts every reported position
    w = workloads.tiny_case(31, 4, 300, 1, 12, 100_000, n_plants=500)
    text, seg = to_device(w)
    for layout in (pfac.LAYOUT_COMPRESSED, pfac.LAYOUT_DENSE):
        with pfac.Table(w.patterns, w.sigma, layout=layout) as t:
            full = keys_np(pfac.match(t, text, seg))
            for se in (1, 15, 16, 17, 511, 512, 513, 4096, 8191, 8193, 99_999, 100_000):
                got = keys_np(pfac.match(t, text, seg, starts_end=se, position_base=1000))
                want = full[(full >> np.uint64(24)) < np.uint64(se)] + np.uint64(1000 << 24)
                assert_same(got, want, f"layout {layout} starts_end {se}")
            with pytest.raises(pfac.PfacError):
                pfac.match(t, text, seg, starts_end=100_001)
