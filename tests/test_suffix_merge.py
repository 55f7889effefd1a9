"""Section 3.2 step 2 (merging the last three levels of the trie) in the
storage model: pinned against Eq. 2, a brute-force count of distinct
subtrees, the language the merged DAG accepts, matching with the id side
channel, and the paper's trend (the merge gains more at small alphabets)."""
import numpy as np
import pytest

import workloads
from oracle import pyref, trie as T


def random_set(rs, sigma, n, lo, hi):
    return workloads.uniform_patterns(rs, n, sigma, lo, hi)


def prefix_heavy(seed, sigma):
    return workloads.prefix_heavy_case(seed, sigma, 0).patterns


CASES = ([(f"rand-{s}-{k}", lambda s=s, k=k: random_set(np.random.RandomState(s), k, 30, 1, 7))
          for s in range(6) for k in (2, 3, 4)] +
         [(f"prefix-{s}", lambda s=s: prefix_heavy(s, 3)) for s in range(6)])


def serial(t, v):
    """Canonical text of a subtree, built recursively (independent of the
    signature interning of suffix_merge)."""
    bm, o = t.bitmap[v], t.offset[v]
    syms = [c for c in range(t.sigma) if (bm >> c) & 1]
    inner = ",".join(f"{c}:{serial(t, o + i)}" for i, c in enumerate(syms))
    return ("F" if t.final_id[v] >= 0 else "N") + "(" + inner + ")"


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_merge_counts_and_language(name, make):
    pats = make()
    sigma = max(max(p) for p in pats) + 1
    t = T.build_paper_trie(pats, sigma)
    # levels = 1 merges the leaves only: Eq. 2
    assert T.suffix_merge(t, 1).n_nodes == T.leaf_merged_count(t.n_nodes, T.leaf_count(pats))
    # levels = 3: nodes taller than 2 (and the root) stay, the rest collapse
    # to their distinct subtrees
    h = T.heights(t)
    tall = sum(1 for v in range(t.n_nodes) if h[v] >= 3 or v == 0)
    short = {serial(t, v) for v in range(1, t.n_nodes) if h[v] < 3}
    dag = T.suffix_merge(t, 3)
    assert dag.n_nodes == tall + len(short)
    # the DAG accepts exactly the patterns
    assert T.dag_strings(dag) == set(pats)


@pytest.mark.parametrize("seed", range(8))
def test_dag_walk_with_side_channel_equals_definition(seed):
    rs = np.random.RandomState(100 + seed)
    pats = prefix_heavy(seed, 3) if seed % 2 else random_set(rs, 3, 25, 1, 6)
    text = rs.randint(0, 4, size=400).astype(np.uint8)  # symbol 3 lies outside when sigma = 3
    cuts = np.sort(rs.randint(0, 401, size=3))
    seg = [0] + cuts.tolist() + [400]
    sigma = max(max(p) for p in pats) + 1
    dag = T.suffix_merge(T.build_paper_trie(pats, sigma), 3)
    got = T.dag_walk_matches(dag, T.side_channel(pats), text, seg)
    assert got == pyref.matches(pats, text.tobytes(), seg)


def test_losing_internal_finals_is_caught():
    # a merge that forgets the finality of inner nodes accepts fewer strings
    pats = prefix_heavy(3, 3)
    t = T.build_paper_trie(pats, 3)
    h = T.heights(t)
    t.final_id = [f if h[v] == 0 else -1 for v, f in enumerate(t.final_id)]
    assert T.dag_strings(T.suffix_merge(t, 3)) != set(pats)


def test_gain_is_larger_at_small_alphabets():
    # Section 4: the reduction is more effective with smaller alphabets
    # (fewer distinct suffixes), 20-symbol patterns
    for n in (100, 1000):
        gain = {}
        for sigma in (4, 52):
            pats = workloads.uniform_patterns(np.random.RandomState(n + sigma), n, sigma, 20, 20)
            t = T.build_paper_trie(pats, sigma)
            gain[sigma] = 1.0 - T.suffix_merge(t, 3).n_nodes / t.n_nodes
        assert gain[4] > gain[52] > 0


def test_last_levels_collapse_to_at_most_1_plus_sigma_plus_sigma_squared():
    # random 20-symbol patterns over 4 symbols: below depth 17 every node is
    # on one pattern's chain, so the three last levels keep at most 1 + 4 + 16
    # distinct subtrees (the final node, one per last symbol, one per pair)
    pats = workloads.uniform_patterns(np.random.RandomState(7), 1000, 4, 20, 20)
    t = T.build_paper_trie(pats, 4)
    h = T.heights(t)
    tall = sum(1 for v in range(t.n_nodes) if h[v] >= 3 or v == 0)
    assert T.suffix_merge(t, 3).n_nodes - tall == 1 + 4 + 16


@pytest.mark.parametrize("sigma,n", [(4, 20), (4, 60), (52, 1000)])
def test_distinct_two_symbol_chains_follow_the_occupancy_law(sigma, n):
    # Section 3.2's expected-reduction model counts the r = sigma^2 chains of
    # two symbols before the final node (Eq. 3; Eq. 4 is garbled).  For
    # random patterns the merged height-2 subtrees are the distinct last two
    # symbols, whose expected count is the occupancy law r(1 - (1 - 1/r)^n).
    r = sigma * sigma
    expect = r * (1.0 - (1.0 - 1.0 / r) ** n)
    counts = []
    for seed in range(30):
        pats = workloads.uniform_patterns(np.random.RandomState(seed), n, sigma, 20, 20)
        t = T.build_paper_trie(pats, sigma)
        h = T.heights(t)
        counts.append(len({serial(t, v) for v in range(1, t.n_nodes) if h[v] == 2}))
        # every pattern's chain is single below depth 17, so the height-2
        # subtrees are exactly its last two symbols
        assert counts[-1] == len({p[-2:] for p in pats})
    mean, se = np.mean(counts), np.std(counts) / np.sqrt(len(counts))
    assert abs(mean - expect) < 4 * se + 0.01 * expect, (mean, expect, se)


def _library():
    return pytest.importorskip("paper_1704_02272_gb300")


LIB_CASES = CASES + [
    ("dna-like", lambda: workloads.uniform_patterns(np.random.RandomState(41), 800, 4, 8, 30)),
    ("sigma256", lambda: workloads.uniform_patterns(np.random.RandomState(42), 300, 256, 1, 12)),
    ("sigma40", lambda: workloads.uniform_patterns(np.random.RandomState(43), 500, 40, 2, 9)),
]


@pytest.mark.parametrize("name,make", LIB_CASES, ids=[c[0] for c in LIB_CASES])
def test_library_merged_node_count_equals_model(name, make):
    # the library's merged trie (built on the host) keeps as many nodes as the
    # storage model of step 2 counts
    pfac = _library()
    pats = make()
    sigma = max(max(p) for p in pats) + 1
    t = T.build_paper_trie(pats, sigma)
    want = T.suffix_merge(t, 3).n_nodes
    with pfac.Table(pats, sigma, host_only=True, suffix_merge=True) as lt:
        info = lt.info()
    assert info["trie_nodes"] == t.n_nodes
    assert info["merged_trie_nodes"] == want
    # one record per merged node: the unshared nodes and one per class
    assert info["records"] == want
    # the side table holds an output for each tail node on whose path a
    # pattern ends, at most every tail node
    h = T.heights(t)
    n_tail = sum(1 for v in range(1, t.n_nodes) if h[v] < 3)
    n_final_tail = sum(1 for v in range(1, t.n_nodes) if h[v] < 3 and t.final_id[v] >= 0)
    assert n_final_tail <= info["side_entries"] <= n_tail


def test_library_merge_flag_needs_compressed_layout():
    pfac = _library()
    with pytest.raises(pfac.PfacError):
        pfac.Table([b"\x01\x02"], 4, layout=pfac.binding.LAYOUT_DENSE, host_only=True,
                   suffix_merge=True)


def test_library_merge_with_wide_records_is_refused():
    pfac = _library()
    with pytest.raises(pfac.PfacError):
        pfac.Table([b"\x01\x02\x03"], 4, host_only=True, suffix_merge=True, wide_records=True)
