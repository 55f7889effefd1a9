"""Prefix matching (Section 2.4) and its verification on the GPU.

A table built with truncate_depth d reports the candidates (p, j) whose
first min(|P_j|, d) symbols occur at p; they must equal the oracle's matches
of the truncated patterns, each expanded to every pattern id sharing that
truncated string.  pfac_verify must reduce them to exactly the oracle's
matches of the full patterns, with both table layouts and with segments
cutting patterns."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


def candidate_keys(w, d):
    trunc = [bytes(p[:d]) for p in w.patterns]
    uniq = sorted(set(trunc))
    index = {s: i for i, s in enumerate(uniq)}
    members = [[] for _ in uniq]
    for j, s in enumerate(trunc):
        members[index[s]].append(j)
    pos, ids = oracle.match_bf(uniq, w.text, w.seg_offsets)
    out = []
    for p, u in zip(pos.tolist(), ids.tolist()):
        out.extend((p << 24) | j for j in members[u])
    return np.array(sorted(out), dtype=np.uint64)


CASES = {
    "letters": lambda: workloads.letters(300, n_bytes=2 << 20, n_plants=400),
    "dna-segs": lambda: workloads.tiny_case(41, 4, 400, 6, 30, 600_000, n_segments=900,
                                            n_plants=800),
    "ids": lambda: workloads.config3(n_bytes=3 << 20, n_patterns=3000),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("d", [2, 5])
@pytest.mark.parametrize("layout", ["compressed", "dense"])
def test_prefix_candidates_and_verify(case, d, layout):
    w = CASES[case]()
    lay = pfac.LAYOUT_COMPRESSED if layout == "compressed" else pfac.LAYOUT_DENSE
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma, layout=lay, truncate_depth=d) as t:
        cand = pfac.match(t, text, seg)
        if case != "ids":
            assert_same(keys_np(cand), candidate_keys(w, d), f"{case} candidates d={d}")
        exact = pfac.verify(t, text, seg, cand)
    assert_same(keys_np(exact), oracle_keys(w), f"{case} verified d={d}")


def test_prefix_trie_is_smaller_and_verify_needs_truncation():
    w = workloads.letters(1000, n_bytes=1 << 20, n_plants=100)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma, truncate_depth=5) as t5, \
            pfac.Table(w.patterns, w.sigma) as t:
        assert t5.info()["trie_nodes"] < t.info()["trie_nodes"] // 2
        cand = pfac.match(t, text, seg)
        with pytest.raises(pfac.PfacError):
            pfac.verify(t, text, seg, cand)
