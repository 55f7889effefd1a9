"""Pins for the CPU oracle: each check compares it with something other than
itself (the paper's worked example and quoted sizes, closed forms, a library
search routine, NumPy window comparisons, an independent algorithm, and brute
force over every small case)."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import workloads
from oracle import pyref, trie

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            rows.setdefault(k, []).append(v)
    return rows


def as_pairs(pos, ids):
    return list(zip(pos.tolist(), ids.tolist()))


def all_matchers(patterns, text, seg, threads=1):
    """O1, O2, the pure-Python loop and the storage-model walker."""
    out = {
        "bf": as_pairs(*oracle.match_bf(patterns, text, seg, threads=threads)),
        "ac": as_pairs(*oracle.match_ac(patterns, text, seg, threads=threads)),
        "py": pyref.matches(patterns, text, seg),
    }
    return out


# ---------------------------------------------------------------- paper --

def test_fig1_worked_example():
    g = read_golden("fig1_bitmap_trie.txt")
    pats = [p.encode() for p in g["patterns"][0]]
    t = trie.build_paper_trie(pats, int(g["sigma"][0][0]))
    node_a = int(g["node_A"][0][0])
    assert t.depth[node_a] == 1 and (t.bitmap[0] >> ord("A")) & 1
    assert t.child(0, ord("A")) == node_a
    assert t.offset[node_a] == int(g["offset_A"][0][0])
    bits = [c for c in range(256) if (t.bitmap[node_a] >> c) & 1]
    assert bits == [int(x) for x in g["bits_A"][0]]
    rank = bin(t.bitmap[node_a] & ((1 << ord("D")) - 1)).count("1")
    assert rank == int(g["rank_D"][0][0])
    assert t.child(node_a, ord("D")) == int(g["child_D"][0][0])
    assert t.child(node_a, ord("B")) == t.offset[node_a]


def test_quoted_table_sizes():
    g = read_golden("table_sizes_sec3_1.txt")
    for sigma, b in g["bytes_per_node"]:
        assert trie.paper_bytes_per_node(int(sigma)) == int(b)
    q = int(g["gravity_nodes"][0][0])
    mib = 2.0 ** 20
    ours = trie.paper_layout_bytes(q, 256) / mib
    dense = trie.dense_stt_bytes(q, 256) / mib
    assert round(ours, 1) == float(g["gravity_ours_mb"][0][0])
    assert round(dense) == int(g["gravity_dense_mb"][0][0])
    # the text rounds the quoted ratio; the sizes give 28.4
    assert abs(dense / ours - float(g["gravity_ratio"][0][0])) / 28.5 < 0.01
    q32 = int(g["sigma32_nodes"][0][0])
    s32 = trie.paper_layout_bytes(q32, 32) / mib
    assert abs(s32 - float(g["sigma32_ours_mb"][0][0])) < 0.1


# ------------------------------------------------------- closed forms ----

@pytest.mark.parametrize("seed,sigma,n,lo,hi", [(1, 2, 12, 1, 6), (2, 4, 60, 1, 9),
                                                (3, 256, 200, 2, 12), (4, 3, 40, 1, 5)])
def test_trie_size_closed_form(seed, sigma, n, lo, hi):
    w = workloads.tiny_case(seed, sigma, n, lo, hi, 0)
    t = trie.build_paper_trie(w.patterns, sigma)
    assert t.n_nodes == trie.prefix_set_count(w.patterns)
    assert t.n_leaves == trie.leaf_count(w.patterns)
    # breadth-first numbering = prefixes sorted by (length, bytes)
    prefixes = sorted({p[:k] for p in w.patterns for k in range(1, len(p) + 1)},
                      key=lambda s: (len(s), s))
    labels = {}
    for i, s in enumerate(prefixes, start=1):
        labels[s] = i
    for s, i in labels.items():
        node = 0
        for c in s:
            node = t.child(node, c)
        assert node == i
    # the AC oracle's goto trie has the same node count
    ac = oracle.ACOracle(w.patterns)
    assert ac.n_nodes == t.n_nodes


def test_eq2_prefix_free():
    rs = np.random.RandomState(7)
    # fixed-length patterns are prefix free: every pattern ends in a leaf
    pats = workloads.dedup([rs.randint(0, 4, 6).astype(np.uint8).tobytes() for _ in range(300)])
    t = trie.build_paper_trie(pats, 4)
    assert t.n_leaves == len(pats)
    q = t.n_nodes
    assert trie.leaf_merged_count(q, t.n_leaves) == q - (len(pats) - 1)


def test_all_zero_closed_form():
    N, m = 50, 6
    text = np.zeros(N, np.uint8)
    pats = [bytes(k) for k in range(1, m + 1)]
    seg = [0, N]
    expect = sorted((p, k - 1) for k in range(1, m + 1) for p in range(N - k + 1))
    assert len(expect) == sum(N - k + 1 for k in range(1, m + 1))
    for name, got in all_matchers(pats, text, seg).items():
        assert got == expect, name
    # a segment cut at c forbids exactly the occurrences that straddle it
    c = 23
    expect2 = sorted((p, k - 1) for k in range(1, m + 1) for p in range(N - k + 1)
                     if p + k <= c or p >= c)
    for name, got in all_matchers(pats, text, [0, c, N]).items():
        assert got == expect2, name


# --------------------------------------------------------- library pins --

@pytest.mark.parametrize("seed", [11, 12, 13])
def test_single_pattern_matches_regex_search(seed):
    rs = np.random.RandomState(seed)
    text = rs.randint(0, 3, 5000).astype(np.uint8)
    cuts = np.sort(rs.randint(0, 5001, 7))
    seg = np.concatenate([[0], cuts, [5000]]).astype(np.uint64)
    for L in (1, 2, 3, 5):
        pat = rs.randint(0, 3, L).astype(np.uint8).tobytes()
        expect = []
        tb = text.tobytes()
        for k in range(len(seg) - 1):
            a, b = int(seg[k]), int(seg[k + 1])
            # zero-width lookahead finds overlapping occurrences
            for m in re.finditer(b"(?=" + re.escape(pat) + b")", tb[a:b]):
                expect.append((a + m.start(), 0))
        for name, got in all_matchers([pat], text, seg).items():
            assert got == expect, (name, L)


@pytest.mark.parametrize("seed,sigma,n,lo,hi,N", [(21, 4, 80, 2, 9, 200_000),
                                                  (22, 256, 300, 2, 6, 300_000),
                                                  (23, 20, 150, 1, 4, 100_000)])
def test_per_pattern_counts_match_numpy_windows(seed, sigma, n, lo, hi, N):
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_plants=0)
    pos, ids = oracle.match_bf(w.patterns, w.text, w.seg_offsets)
    pos2, ids2 = oracle.match_ac(w.patterns, w.text, w.seg_offsets)
    assert np.array_equal(pos, pos2) and np.array_equal(ids, ids2)
    counts = np.bincount(ids.astype(np.int64), minlength=len(w.patterns))
    for j, p in enumerate(w.patterns):
        L = len(p)
        win = np.lib.stride_tricks.sliding_window_view(w.text, L)
        ref = int(np.all(win == np.frombuffer(p, np.uint8), axis=1).sum())
        assert counts[j] == ref, j
    # sorted by (position, id), no duplicates
    key = pos.astype(np.float64) * 2 ** 20 + ids
    assert np.all(np.diff(key) > 0)


# --------------------------------------------- exhaustive small cases ----

def _all_strings(sigma, max_len):
    out = []
    for L in range(1, max_len + 1):
        out += [bytes(t) for t in itertools.product(range(sigma), repeat=L)]
    return out


def _all_texts_as_segments(sigma, max_len):
    texts = [bytes(t) for L in range(0, max_len + 1) for t in itertools.product(range(sigma), repeat=L)]
    text = np.frombuffer(b"".join(texts), np.uint8)
    seg = np.zeros(len(texts) + 1, np.uint64)
    np.cumsum([len(t) for t in texts], out=seg[1:])
    return text, seg


@pytest.mark.parametrize("sigma,max_pat,max_set,max_text", [(2, 3, 3, 8), (3, 3, 2, 5)])
def test_exhaustive_small(sigma, max_pat, max_set, max_text):
    """Every pattern set of up to ``max_set`` strings of length <= ``max_pat``
    against every text of length <= ``max_text`` (each text one segment)."""
    strings = _all_strings(sigma, max_pat)
    text, seg = _all_texts_as_segments(sigma, max_text)
    n_sets = 0
    for r in range(1, max_set + 1):
        for pats in itertools.combinations(strings, r):
            pats = list(pats)
            res = all_matchers(pats, text, seg)
            t = trie.build_paper_trie(pats, sigma)
            res["paper-walk"] = trie.walk_matches(t, text, seg)
            ref = res["py"]
            for name, got in res.items():
                assert got == ref, (name, pats)
            n_sets += 1
    assert n_sets > 100


@pytest.mark.parametrize("seed", range(6))
def test_prefix_heavy_random(seed):
    w = workloads.prefix_heavy_case(seed, 3 + seed % 3, 3000, n_segments=1 + 7 * (seed % 2))
    res = all_matchers(w.patterns, w.text, w.seg_offsets)
    t = trie.build_paper_trie(w.patterns, w.sigma)
    res["paper-walk"] = trie.walk_matches(t, w.text, w.seg_offsets)
    ref = res["py"]
    assert len(ref) > 100
    for name, got in res.items():
        assert got == ref, name


def test_out_of_alphabet_text_symbols():
    # symbols outside the alphabet never match and never break a walk early
    # for the C oracles (they compare bytes)
    w = workloads.tiny_case(31, 4, 30, 1, 5, 4000, n_segments=5, n_plants=40, text_sigma=6)
    res = all_matchers(w.patterns, w.text, w.seg_offsets)
    t = trie.build_paper_trie(w.patterns, 4)
    res["paper-walk"] = trie.walk_matches(t, w.text, w.seg_offsets)
    ref = res["py"]
    for name, got in res.items():
        assert got == ref, name


# ------------------------------------------------------- invariants ------

def test_config1_full_bf_equals_ac_and_plants_present():
    w = workloads.config1()
    assert len(w.patterns) == 1000 and w.n_bytes == 1 << 20
    pos, ids = oracle.match_bf(w.patterns, w.text, w.seg_offsets)
    pos2, ids2 = oracle.match_ac(w.patterns, w.text, w.seg_offsets)
    assert np.array_equal(pos, pos2) and np.array_equal(ids, ids2)
    got = set(zip(pos.tolist(), ids.tolist()))
    intact = 0
    for p, j in w.plants.tolist():
        pat = w.patterns[j]
        if w.text[p:p + len(pat)].tobytes() == pat:
            intact += 1
            assert (p, j) in got
    assert intact >= 1900  # later plants overwrite ~3% of earlier ones


def test_segment_split_invariance():
    w = workloads.tiny_case(41, 4, 200, 2, 10, 60_000, n_segments=40, n_plants=100)
    ac = oracle.ACOracle(w.patterns)
    pos, ids = ac.match(w.text, w.seg_offsets)
    parts_p, parts_i = [], []
    for k in range(len(w.seg_offsets) - 1):
        a, b = int(w.seg_offsets[k]), int(w.seg_offsets[k + 1])
        p, i = ac.match(w.text[a:b], [0, b - a])
        parts_p.append(p + np.uint64(a))
        parts_i.append(i)
    assert np.array_equal(pos, np.concatenate(parts_p))
    assert np.array_equal(ids, np.concatenate(parts_i))


def test_windows_partition_the_result():
    w = workloads.tiny_case(42, 4, 300, 2, 12, 3_000_000, n_segments=3)
    ac = oracle.ACOracle(w.patterns)
    pos, ids = ac.match(w.text, w.seg_offsets, threads=4)
    cuts = [0, 123_457, 1_500_000, 1_500_001, 2_999_990, 3_000_000]
    pp, ii = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        p, i = ac.match(w.text, w.seg_offsets, lo=a, hi=b, threads=3)
        assert p.size == 0 or (p.min() >= a and p.max() < b)
        pp.append(p)
        ii.append(i)
    assert np.array_equal(pos, np.concatenate(pp)) and np.array_equal(ids, np.concatenate(ii))


def test_match_density_near_expectation():
    """Uniform text over 4 symbols: each pattern of length L matches at a
    position with probability 4^-L (sanity only, 6 sigma)."""
    w = workloads.tiny_case(43, 4, 400, 3, 7, 1_000_000)
    pos, ids = oracle.match_ac(w.patterns, w.text, w.seg_offsets)
    exp = sum((w.n_bytes - len(p) + 1) * 4.0 ** -len(p) for p in w.patterns)
    assert abs(len(pos) - exp) < 6 * np.sqrt(exp)


def test_rejects_invalid():
    with pytest.raises(ValueError):
        oracle.ACOracle([b"ab", b"ab"])
    with pytest.raises(ValueError):
        oracle.ACOracle([b"ab", b""])
    with pytest.raises(ValueError):
        oracle.match_bf([b"a"], np.zeros(4, np.uint8), [0, 5])
    with pytest.raises(ValueError):
        oracle.match_bf([b"a"], np.zeros(4, np.uint8), [0, 3, 2, 4])
    # empty text and empty segments are valid
    assert oracle.match_ac([b"a"], np.zeros(0, np.uint8), [0])[0].size == 0
    p, i = oracle.match_ac([b"\0"], np.zeros(3, np.uint8), [0, 0, 2, 2, 3])
    assert p.tolist() == [0, 1, 2]


# ------------------------------------------- the pins catch mistakes -----

def _mutants():
    """Plausible mistakes planted in copies of the pure-Python oracle."""
    def off_by_one_segment(patterns, text, seg):
        text = bytes(text)
        out = []
        for k in range(len(seg) - 1):
            a, b = int(seg[k]), int(seg[k + 1])
            for p in range(a, b):
                for j, pat in enumerate(patterns):
                    if p + len(pat) < b and text[p:p + len(pat)] == pat:
                        out.append((p, j))
        return sorted(out)

    def end_position(patterns, text, seg):
        return sorted((p + len(patterns[j]) - 1, j) for p, j in pyref.matches(patterns, text, seg))

    def ignores_segments(patterns, text, seg):
        return pyref.matches(patterns, text, [0, len(text)])

    def id_major_order(patterns, text, seg):
        return sorted(pyref.matches(patterns, text, seg), key=lambda x: (x[1], x[0]))

    def drops_longest(patterns, text, seg):
        m = pyref.matches(patterns, text, seg)
        keep = []
        for p, j in m:
            if len(patterns[j]) == max(len(x) for x in patterns) and len(patterns) > 1:
                continue
            keep.append((p, j))
        return keep

    return [off_by_one_segment, end_position, ignores_segments, id_major_order, drops_longest]


@pytest.mark.parametrize("mutant", _mutants(), ids=lambda f: f.__name__)
def test_pins_catch_planted_mistakes(mutant):
    """Each planted mistake fails at least one of: the all-zero closed form,
    the regex pin, or agreement with the independent Aho-Corasick program."""
    failures = 0
    N = 40
    pats = [bytes(k) for k in range(1, 5)]
    exp = sorted((p, k - 1) for k in range(1, 5) for p in range(N - k + 1)
                 if p + k <= 17 or p >= 17)
    if mutant(pats, np.zeros(N, np.uint8), [0, 17, N]) != exp:
        failures += 1
    rs = np.random.RandomState(5)
    text = rs.randint(0, 2, 300).astype(np.uint8)
    seg = [0, 100, 300]
    pat = b"\x01\x00\x01"
    expect = []
    for a, b in zip(seg[:-1], seg[1:]):
        for m in re.finditer(b"(?=" + re.escape(pat) + b")", text.tobytes()[a:b]):
            expect.append((a + m.start(), 0))
    if mutant([pat], text, seg) != expect:
        failures += 1
    w = workloads.prefix_heavy_case(3, 3, 800, n_segments=4)
    ac = as_pairs(*oracle.match_ac(w.patterns, w.text, w.seg_offsets))
    if mutant(w.patterns, w.text, w.seg_offsets) != ac:
        failures += 1
    assert failures >= 1
