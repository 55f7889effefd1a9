"""GPU parity of the merged trie (reduction step 2 of Section 3.2): tables
built with suffix_merge=True against the CPU oracle, element by element,
through the queued kernel's merged-trie instance and every plan that fits
(the register-staged kernel refuses merged tries), on pattern sets whose
walks end inside shared subtrees at every depth (prefix entries whose state
is a merged node, walks that stop one to three levels below their last
unshared node, patterns that are prefixes of others), and at the full size
of the DNA-shaped workload and of the alphabet-4 sweep cell with 10,000
patterns (512 MiB, about 3e8 matches)."""
import itertools

import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")

KERNELS = (pfac.binding.KERNEL_QUEUED, pfac.binding.KERNEL_REGISTER)


def run(t, text, seg, **kw):
    keys = pfac.match(t, text, seg, **kw)
    torch.cuda.synchronize()
    return keys_np(keys)


def all_plans(w, ref, what, depths, copies=(1, 4)):
    text, seg = to_device(w)
    ran = 0
    with pfac.Table(w.patterns, w.sigma, suffix_merge=True) as t:
        info = t.info()
        assert 0 < info["merged_trie_nodes"] <= info["trie_nodes"]
        assert_same(run(t, text, seg), ref, f"{what} default")
        for kern, k, var, masks, gram, cp in itertools.product(
                KERNELS, depths, (1, 2), (1, 2), (1, 2), copies):
            opt = dict(scan_kernel=kern, prefix_depth=k, variant=var, child_masks=masks,
                       gram_filter=gram, bitmap_copies=cp)
            try:
                pfac.plan(t, **opt)
            except pfac.PfacError as e:  # does not fit, or no such kernel here
                assert e.status == -1, str(e)
                continue
            assert_same(run(t, text, seg, **opt), ref, f"{what} {opt}")
            ran += 1
    return ran


CASES = [
    # seed, sigma, n_patterns, lo, hi, n_bytes, n_segments, n_plants, text_sigma
    (301, 4, 300, 3, 12, 300_000, 1, 900, None),
    (302, 4, 2000, 8, 30, 200_003, 7, 600, None),        # ragged tail, segments
    (303, 4, 80, 1, 6, 100_000, 1, 400, 6),              # short patterns, bytes outside
    (304, 256, 1500, 1, 10, 400_000, 1, 1200, None),
    (305, 256, 300, 2, 40, 150_001, 33, 500, None),
    (306, 40, 700, 1, 8, 250_000, 3, 900, 64),
    (307, 3, 120, 2, 9, 120_000, 5, 500, None),
]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_merged_trie_all_plans(case):
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    assert ref.size > 0
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        kdef = th.info()["prefix_depth"]
    ran = all_plans(w, ref, f"case {seed}", sorted({max(1, kdef - 2), kdef}))
    assert ran >= 8


@pytest.mark.parametrize("seed", range(4))
def test_merged_trie_prefix_heavy(seed):
    # chains of patterns that are prefixes of one another: outputs of several
    # patterns on one walk, finals inside the merged levels
    w = workloads.prefix_heavy_case(seed, 3, 200_000, n_segments=1 + seed)
    ref = oracle_keys(w)
    assert ref.size > 0
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        kdef = th.info()["prefix_depth"]
    assert all_plans(w, ref, f"prefix-heavy {seed}", sorted({max(1, kdef - 2), kdef})) >= 4


def test_merged_trie_same_matches_as_tree():
    # the merged and the plain table give the same keys, and the merged one
    # keeps fewer records
    w = workloads.tiny_case(311, 4, 3000, 8, 40, 1 << 20, n_plants=3000)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 4) as t0, pfac.Table(w.patterns, 4, suffix_merge=True) as t1:
        a, b = run(t0, text, seg), run(t1, text, seg)
        assert t1.info()["records"] < t0.info()["records"]
    assert_same(b, a, "merged vs tree")
    assert_same(b, oracle_keys(w), "merged vs oracle")


def test_merged_trie_edges():
    # empty input, inputs ending inside a merged subtree, one-symbol patterns
    # (a prefix entry that is a leaf), patterns of exactly the prefix depth
    pats = [b"\x01", b"\x01\x02", b"\x02\x02\x02", b"\x03\x00\x01\x02", b"\x00\x00\x00\x00\x00",
            b"\x02\x01\x00\x03\x03\x01"]
    rs = np.random.RandomState(9)
    with pfac.Table(pats, 4, suffix_merge=True) as t:
        for n in (0, 1, 2, 3, 5, 511, 512, 513, 4099):
            text = rs.randint(0, 4, size=n).astype(np.uint8)
            w = workloads.Workload(f"edge-{n}", 4, pats, text, workloads.single_segment(n))
            tt, sg = to_device(w)
            assert_same(run(t, tt, sg), oracle_keys(w), f"n={n}")
        with pytest.raises(pfac.PfacError) as ei:
            pfac.plan(t, scan_kernel=pfac.binding.KERNEL_REGISTER)
        assert ei.value.status == -1


def test_merged_trie_full_size_dna():
    # the DNA-shaped workload at its full 256 MiB, whole list against the
    # oracle in 32 MiB windows of start positions
    w = workloads.config2()
    text, seg = to_device(w)
    import oracle
    ac = oracle.ACOracle(w.patterns)
    try:
        step = 32 << 20
        ref = np.concatenate([oracle_keys(w, lo=a, hi=min(a + step, w.n_bytes), ac=ac)
                              for a in range(0, w.n_bytes, step)])
        with pfac.Table(w.patterns, 4, suffix_merge=True) as t:
            for opt in ({}, {"child_masks": 1}, {"prefix_depth": 8}):
                assert_same(run(t, text, seg, **opt), ref, f"dna merged {opt}")
    finally:
        ac.close()


def test_merged_trie_full_size_sigma4_10k():
    # the match-dense alphabet-4 cell (patterns from 4 symbols long) at its
    # full 512 MiB: every key against the oracle, 32 MiB of start positions at
    # a time
    from tests.gpu_util import window
    w = workloads.config4(4, 10000)
    text, seg = to_device(w)
    import oracle
    ac = oracle.ACOracle(w.patterns)
    try:
        with pfac.Table(w.patterns, 4, suffix_merge=True) as t:
            assert t.info()["merged_trie_nodes"] < t.info()["trie_nodes"]
            kc = pfac.match(t, text, seg)
            torch.cuda.synchronize()
        chunk, total = 32 << 20, 0
        for a in range(0, w.n_bytes, chunk):
            ref = oracle_keys(w, lo=a, hi=min(a + chunk, w.n_bytes), ac=ac)
            assert_same(window(kc, a, a + chunk), ref, f"merged sigma4x10k chunk at {a}")
            total += ref.shape[0]
        assert total == kc.numel()
    finally:
        ac.close()
