"""CPU checks of the library boundary: the shared library loads without a
GPU, exports every function include/pfac.h declares, and its host-side trie
builder (run host-only, no device memory) reports the statistics the oracle's
storage model gives: trie size, leaves, the leaf merge of Eq. 2 and the
Section 3.1 byte counts."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from oracle import trie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfac.h")

pfac = pytest.importorskip("paper_1704_02272_gb300")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(pfac_\w+)\s*\(", src, re.M)))


def test_header_symbols_exported():
    names = declared_functions()
    assert "pfac_build" in names and "pfac_match" in names and len(names) >= 9
    lib = ctypes.CDLL(pfac.binding.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/pfac.h but not exported"


def test_status_strings():
    lib = pfac.binding.LIB
    for code in range(0, -9, -1):
        s = lib.pfac_status_str(code).decode()
        assert s and s != "unknown status"
    assert pfac.version() >= 100


def host_table(patterns, sigma, **kw):
    return pfac.Table(patterns, sigma, host_only=True, **kw)


@pytest.mark.parametrize("seed,sigma,n,lo,hi", [(1, 4, 500, 1, 12), (2, 256, 3000, 2, 20),
                                                (3, 20, 800, 1, 8), (4, 64, 900, 1, 9),
                                                (5, 2, 60, 1, 10), (6, 3, 200, 1, 7)])
def test_table_statistics_match_storage_model(seed, sigma, n, lo, hi):
    w = workloads.tiny_case(seed, sigma, n, lo, hi, 0)
    with host_table(w.patterns, sigma) as t:
        info = t.info()
    q = trie.prefix_set_count(w.patterns)
    leaves = trie.leaf_count(w.patterns)
    pt = trie.build_paper_trie(w.patterns, sigma)
    assert info["trie_nodes"] == q == pt.n_nodes
    assert info["trie_leaves"] == leaves == pt.n_leaves
    assert info["n_patterns"] == len(w.patterns)
    assert info["max_len"] == max(len(p) for p in w.patterns)
    # every merged leaf removes one record; the root always keeps one
    assert info["records"] + info["merged_leaves"] == q
    assert info["merged_leaves"] <= leaves
    assert info["paper_bytes"] == trie.paper_layout_bytes(q, sigma)
    assert info["dense_bytes"] == trie.dense_stt_bytes(q, sigma)
    assert info["output_lists"] == len(w.patterns)


def test_eq2_leaf_merge_on_prefix_free_sets():
    rs = np.random.RandomState(3)
    # equal-length patterns: prefix free, and every parent of a leaf has only
    # leaf children, so every leaf merges: records = Q - |P| (Eq. 2 counts the
    # one shared final node on top: Q - (|P| - 1))
    pats = workloads.dedup([rs.randint(0, 4, 7).astype(np.uint8).tobytes() for _ in range(2000)])
    with host_table(pats, 4) as t:
        info = t.info()
    q = trie.prefix_set_count(pats)
    assert info["merged_leaves"] == len(pats)
    assert info["records"] + 1 == trie.leaf_merged_count(q, len(pats))


def test_fig1_example_counts():
    # Section 3.1 worked example: patterns AB, AD and a third first symbol
    with host_table([b"AB", b"AD", b"E"], 256) as t:
        info = t.info()
    assert info["trie_nodes"] == 5 and info["trie_leaves"] == 3
    # 'AB' and 'AD' are the only children of 'A': both merge; 'E' has an
    # internal sibling ('A') and keeps its record
    assert info["merged_leaves"] == 2 and info["records"] == 3


@pytest.mark.parametrize("pats,sigma,status", [
    ([b"ab", b"ab"], 256, -2),
    ([b"ab", b""], 256, -1),
    ([b"\x05"], 4, -3),
    ([b"a"], 0, -1),
    ([b"a"], 257, -1),
])
def test_build_errors(pats, sigma, status):
    with pytest.raises(pfac.PfacError) as ei:
        host_table(pats, sigma)
    assert ei.value.status == status


def test_empty_pattern_set_builds():
    with host_table([], 256) as t:
        info = t.info()
    assert info["trie_nodes"] == 1 and info["records"] == 1 and info["n_patterns"] == 0


def test_host_only_table_cannot_match():
    # straight through the C ABI: a host-only table is rejected before any
    # pointer is used or any CUDA call is made
    import ctypes
    lib = pfac.binding.LIB
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced
    with host_table([b"ab"], 256) as t:
        o = pfac.binding.MatchOpts()
        rc = lib.pfac_match_async(t.handle, fake, 16, fake, 1, fake, 4, fake, fake, fake,
                                  1 << 16, ctypes.byref(o), None)
        assert rc == -1
        rc = lib.pfac_match_noalloc(t.handle, fake, 16, fake, 1, fake, 4, fake, fake,
                                    ctypes.byref(o), None)
        assert rc == -1
        n = ctypes.c_uint64()
        rc = lib.pfac_match(t.handle, fake, 16, fake, 1, fake, 4, ctypes.byref(n),
                            ctypes.byref(o), None)
        assert rc == -1


def gram_strings_brute(patterns, g, bps):
    """Strings x of g symbols (values 0 .. 2^bps - 1) whose walk from the root
    reaches depth g (x is a prefix of a pattern) or stops before depth g at a
    state with output (a pattern is a prefix of x)."""
    import itertools
    pats = [bytes(p) for p in patterns]
    prefixes = {p[:i] for p in pats for i in range(1, len(p) + 1)}
    pset = set(pats)
    n = 0
    for x in itertools.product(range(1 << bps), repeat=g):
        s = bytes(x)
        if s in prefixes or any(s[:i] in pset for i in range(1, g + 1)):
            n += 1
    return n


@pytest.mark.parametrize("seed,sigma,n,lo,hi,k,bps", [(11, 4, 40, 1, 6, 3, 2),
                                                       (12, 3, 30, 2, 9, 4, 2),
                                                       (13, 20, 60, 1, 4, 1, 5),
                                                       (14, 5, 25, 1, 7, 2, 3),
                                                       (15, 2, 20, 1, 12, 8, 1)])
def test_gram_filter_string_count(seed, sigma, n, lo, hi, k, bps):
    # the gram filter covers g = k + 1 symbols; its count of strings that
    # start a match is the brute-force count over all g-symbol strings
    w = workloads.tiny_case(seed, sigma, n, lo, hi, 0)
    with host_table(w.patterns, sigma, prefix_depth=k) as t:
        info = t.info()
    assert info["gram_len"] == k + 1
    assert info["gram_strings"] == gram_strings_brute(w.patterns, k + 1, bps)
    assert 10 <= info["gram_bits"] <= 20


def test_prefix_depth_too_small_rejected():
    # a prefix index must span at least 5 bits
    with pytest.raises(pfac.PfacError) as ei:
        host_table([b"\x01\x02"], 4, prefix_depth=2)
    assert ei.value.status == -1


@pytest.mark.parametrize("seed,sigma,n,lo,hi,d", [(21, 52, 300, 20, 20, 5), (22, 4, 500, 3, 16, 6),
                                                  (23, 256, 800, 1, 12, 2)])
def test_truncated_trie_counts(seed, sigma, n, lo, hi, d):
    # prefix matching (Section 2.4): the truncated trie is the trie of the
    # patterns cut to d symbols; its lists hold each distinct cut string
    w = workloads.tiny_case(seed, sigma, n, lo, hi, 0)
    cut = [bytes(p[:d]) for p in w.patterns]
    with host_table(w.patterns, sigma, truncate_depth=d) as t:
        info = t.info()
    assert info["trie_nodes"] == trie.prefix_set_count(cut)
    assert info["output_lists"] == len(set(cut))
    assert info["n_patterns"] == len(w.patterns)


def test_match_checks_its_tensors_before_the_library():
    import torch
    with host_table([b"ab"], 256) as t:
        z = torch.zeros(16, dtype=torch.uint8)
        s = torch.tensor([0, 16], dtype=torch.int64)
        with pytest.raises(ValueError):
            pfac.match(t, z, s)  # host text: the device path needs device memory
        with pytest.raises(ValueError):
            pfac.match_into(t, z, s.to(torch.int32), torch.zeros(4, dtype=torch.int64))


@pytest.mark.parametrize("fn", ["match_async", "match_noalloc"])
def test_async_entry_points_check_their_tensors(fn):
    # a wrongly typed or strided tensor would make the kernels read or write
    # past a smaller buffer: the binding refuses it before the library
    import torch
    with host_table([b"ab"], 256) as t:
        z = torch.zeros(16, dtype=torch.uint8)
        s = torch.tensor([0, 16], dtype=torch.int64)
        out = torch.zeros(4, dtype=torch.int64)
        cnt = torch.zeros(1, dtype=torch.int64)
        st = torch.zeros(1, dtype=torch.int32)
        ws = [torch.zeros(1 << 16, dtype=torch.uint8)] if fn == "match_async" else []
        call = getattr(pfac, fn)
        bad = [
            (z, s.to(torch.int32), out, cnt, st),          # 4-byte offsets
            (z, s, out.to(torch.int32), cnt, st),          # 4-byte keys
            (z, s, out, cnt.to(torch.int32), st),          # 4-byte count
            (z, s, out, cnt, st.to(torch.int64)),          # 8-byte status
            (z, s, torch.zeros(8, dtype=torch.int64)[::2], cnt, st),  # strided output
            (z.to(torch.int16), s, out, cnt, st),          # wide text
        ]
        for args in bad:
            with pytest.raises(ValueError, match="contiguous"):
                call(t, *args, *ws)
        if fn == "match_async":
            with pytest.raises(ValueError, match="contiguous"):
                call(t, z, s, out, cnt, st, ws[0].to(torch.int32))
        # well-formed host tensors: refused because the path needs device memory
        with pytest.raises(ValueError, match="CUDA device"):
            call(t, z, s, out, cnt, st, *ws)


@pytest.mark.parametrize("sigma,n", [(2, 50), (4, 800), (7, 600), (8, 300), (20, 500),
                                     (64, 400), (256, 300)])
def test_record_formats_and_table_parts(sigma, n):
    # alphabets of up to 8 symbols pack a node into one word (4 bytes); the
    # 32-symbol format takes 8, the 64- and 256-symbol ones 16 and 48; the
    # parts add up to the device bytes up to the 16-byte section alignment
    pats = workloads.uniform_patterns(np.random.RandomState(sigma * 7 + n), n, sigma, 2, 14)
    pats = list(dict.fromkeys(pats))
    with host_table(pats, sigma) as t:
        i = t.info()
    want = 4 if sigma <= 8 else (8 if sigma <= 32 else (16 if sigma <= 64 else 48))
    assert i["record_bytes"] == want
    parts = i["trie_bytes"] + i["index_bytes"] + i["other_bytes"]
    assert parts <= i["device_bytes"] <= parts + 16 * 64
    if sigma <= 8:
        with host_table(pats, sigma, wide_records=True) as tw:
            iw = tw.info()
        assert iw["record_bytes"] == 8 and iw["records"] == i["records"]
        # the packed records take half the bytes; the outputs move to the
        # ranked list of the records that have one
        assert i["trie_bytes"] < iw["trie_bytes"]


@pytest.mark.parametrize("sigma,n,lo,hi", [(4, 1000, 4, 64), (4, 10000, 4, 64),
                                           (4, 10000, 8, 64), (52, 1, 20, 20), (52, 10, 20, 20),
                                           (20, 1000, 4, 64), (256, 1000, 4, 64)])
def test_compressed_table_smaller_than_dense(sigma, n, lo, hi):
    # the compressed device table, with its prefix nodes and filter, takes
    # fewer bytes than the uncompressed transition table of the same trie
    pats = workloads.uniform_patterns(np.random.RandomState(sigma + n), n, sigma, lo, hi)
    pats = list(dict.fromkeys(pats))
    with host_table(pats, sigma) as t, host_table(pats, sigma, layout=pfac.LAYOUT_DENSE) as d:
        assert t.info()["device_bytes"] < d.info()["device_bytes"]
