"""GPU parity on small and edge-case inputs: the CUDA path through the C ABI
against the CPU oracle, element by element (sorted packed keys), for every
kernel variant, several prefix depths and both table layouts."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


def run(w, **kw):
    layout = kw.pop("layout", pfac.LAYOUT_COMPRESSED)
    prefix = kw.pop("build_prefix", 0)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma, layout=layout, prefix_depth=prefix) as t:
        keys = pfac.match(t, text, seg, **kw)
        torch.cuda.synchronize()
        return keys_np(keys)


def check_all_variants(w, what, depths=None):
    ref = oracle_keys(w)
    assert_same(run(w), ref, f"{what} default")
    # the dense layout: its transition table in the library's kernels, and
    # the thread-serial kernel
    assert_same(run(w, layout=pfac.LAYOUT_DENSE), ref, f"{what} dense")
    assert_same(run(w, layout=pfac.LAYOUT_DENSE, scan_kernel=pfac.binding.KERNEL_SERIAL), ref,
                f"{what} dense, thread-serial kernel")
    ran = 0
    for layout in (pfac.LAYOUT_COMPRESSED, pfac.LAYOUT_DENSE):
        for var in (pfac.VARIANT_FILTER, pfac.VARIANT_DSMEM):
            for k in depths or [0]:
                try:
                    kk = 0 if k is None else k
                    if k == "min":
                        with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
                            kk = max(1, th.info()["prefix_depth"] - 2)
                    got = run(w, layout=layout, variant=var, prefix_depth=kk)
                except pfac.PfacError as e:  # a prefix node too large for shared memory
                    assert e.status == -1, str(e)
                    continue
                assert_same(got, ref, f"{what} layout {layout} variant {var} depth {k}")
                ran += 1
    assert ran >= 2
    return ref


CASES = [
    # seed, sigma, n_patterns, lo, hi, n_bytes, n_segments, n_plants, text_sigma
    (101, 4, 60, 1, 9, 100_000, 1, 300, None),
    (102, 4, 400, 2, 14, 200_000, 300, 500, None),
    (103, 256, 2000, 2, 12, 1 << 20, 1, 2000, None),
    (104, 20, 500, 1, 6, 300_000, 50, 400, None),
    (105, 64, 800, 1, 7, 300_000, 7, 400, None),
    (106, 3, 100, 1, 8, 150_000, 20, 200, None),
    (107, 2, 40, 1, 10, 150_000, 3, 100, None),
    (108, 4, 200, 1, 8, 120_000, 40, 300, 7),      # out-of-alphabet bytes in the text
    (109, 100, 700, 1, 5, 250_000, 11, 300, None),
    (110, 256, 500, 1, 40, 100_003, 1, 300, None),  # ragged tail
    # few patterns, so that the child masks fit: out-of-alphabet bytes right
    # after outputs (byte >= 2^bits-per-symbol, and sigma <= byte < 2^bps)
    (111, 4, 30, 3, 12, 200_000, 5, 600, 7),
    (112, 5, 40, 2, 10, 200_000, 3, 600, 8),
    (113, 20, 60, 2, 9, 200_000, 9, 600, 40),
    # dense survivors (more than 32 per slice) that the child masks mostly drop
    (114, 4, 5000, 9, 14, 300_000, 3, 600, None),
]
MASK_CASES = CASES[-4:]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_random_cases(case):
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = check_all_variants(w, f"case {seed}", depths=[None, "min"])
    assert ref.size > 0


@pytest.mark.parametrize("case", MASK_CASES, ids=[f"s{c[0]}" for c in MASK_CASES])
def test_child_masks_forced(case):
    # the second on-chip stage on and off must give the oracle's keys
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        k = max(1, th.info()["prefix_depth"] - 2)  # the shallowest depth held fits with masks
    assert_same(run(w, prefix_depth=k, child_masks=2), ref, "child masks on")
    assert_same(run(w, prefix_depth=k, child_masks=1), ref, "child masks off")


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_gram_filter_forced(case):
    # the gram filter as the first stage (then the exact prefix-bitmap test)
    # at both ends of the depths held and with 1 and 32 copies
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        info = th.info()
    assert info["gram_len"] == info["prefix_depth"] + 1
    ran = 0
    for k in (info["prefix_depth"], max(1, info["prefix_depth"] - 2)):
        for copies in (0, 1, 32):
            try:
                got = run(w, prefix_depth=k, gram_filter=2, bitmap_copies=copies)
            except pfac.PfacError as e:  # does not fit in shared memory
                assert e.status == -1, str(e)
                continue
            assert_same(got, ref, f"gram filter depth {k} copies {copies}")
            ran += 1
    assert ran >= 2


def bits_per_symbol(sigma):
    b = 1
    while (1 << b) < sigma:
        b += 1
    return b


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_prefix_bytes_forced(case):
    # prefix bytes as the first stage (bucket test second) at every depth of
    # at most 16 index bits the table holds, child masks on and off
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        kdef = th.info()["prefix_depth"]
    b = bits_per_symbol(w.sigma)
    ran = 0
    for k in range(max(1, kdef - 2), kdef + 1):
        if k * b > 16 or k * b < 5:
            continue
        for masks in (1, 2):
            try:
                got = run(w, prefix_depth=k, prefix_bytes=2, child_masks=masks)
            except pfac.PfacError as e:  # does not fit, or no masks kept
                assert e.status == -1, str(e)
                continue
            assert_same(got, ref, f"prefix bytes depth {k} masks {masks}")
            ran += 1
    if sigma >= 8:
        assert ran >= 1


@pytest.mark.parametrize("seed", range(4))
def test_prefix_heavy(seed):
    w = workloads.prefix_heavy_case(seed, 3 + seed, 200_000, n_segments=1 + 30 * (seed % 2))
    check_all_variants(w, f"prefix-heavy {seed}")


@pytest.mark.parametrize("N", [0, 1, 15, 16, 17, 8191, 8192, 8193, 8208, 8209, 16400])
def test_sizes_around_tiles(N):
    w = workloads.tiny_case(200 + N, 4, 80, 1, 6, N, n_plants=min(N // 10, 50))
    check_all_variants(w, f"N={N}")


def test_sigma_one():
    pats = [bytes(k) for k in (1, 2, 5, 31, 40)]
    text = np.zeros(70_000, np.uint8)
    text[12345] = 0  # all zeros: every pattern matches nearly everywhere
    w = workloads.Workload("zeros", 1, pats, text, workloads.single_segment(text.size))
    ref = check_all_variants(w, "sigma 1")
    assert ref.size == sum(text.size - len(p) + 1 for p in pats)


def test_many_tiny_segments():
    # more segment ends per tile than the per-tile list holds, empty segments
    rs = np.random.RandomState(5)
    N = 60_000
    lens = rs.randint(0, 4, size=25_000)
    lens = lens[np.cumsum(lens) <= N]
    cuts = np.concatenate([[0], np.cumsum(lens), [N]]).astype(np.uint64)
    pats = workloads.uniform_patterns(rs, 50, 4, 1, 4)
    text = workloads.uniform_symbols(rs, N, 4)
    w = workloads.Workload("tiny-segs", 4, pats, text, cuts)
    check_all_variants(w, "tiny segments")


def test_long_patterns_across_tiles():
    # patterns far longer than the staged halo, planted across tile borders
    rs = np.random.RandomState(9)
    pats = workloads.uniform_patterns(rs, 40, 256, 100, 9000)
    N = 200_000
    text = workloads.uniform_symbols(rs, N, 256)
    for i, b in enumerate(range(8192, N - 9000, 8192)):
        p = pats[i % len(pats)]
        off = b - len(p) // 2
        text[off:off + len(p)] = np.frombuffer(p, np.uint8)
    w = workloads.Workload("long", 256, pats, text, workloads.single_segment(N))
    ref = check_all_variants(w, "long patterns")
    assert ref.size >= 15


def test_capacity_two_call():
    w = workloads.tiny_case(301, 4, 300, 2, 6, 200_000)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 4) as t:
        out = torch.empty(max(ref.size // 3, 1), dtype=torch.int64, device=text.device)
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match_into(t, text, seg, out)
        assert ei.value.status == -5 and ei.value.count == ref.size
        assert_same(keys_np(out), ref[:out.numel()], "truncated prefix")
        out2 = torch.empty(ref.size, dtype=torch.int64, device=text.device)
        assert pfac.match_into(t, text, seg, out2) == ref.size
        assert_same(keys_np(out2), ref, "second call")


def test_bad_offsets_reported():
    w = workloads.tiny_case(302, 4, 30, 2, 5, 10_000, n_segments=5)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 4) as t:
        o2, o3 = int(seg[2].item()), int(seg[3].item())
        bad = seg.clone()
        bad[2] = o3 + 1  # o_2 > o_3: not non-decreasing
        bad[3] = o2
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match_into(t, text, bad, torch.empty(10_000, dtype=torch.int64,
                                                      device=text.device))
        assert ei.value.status == -1
        bad2 = seg.clone()
        bad2[-1] -= 1
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match_into(t, text, bad2, torch.empty(10_000, dtype=torch.int64,
                                                       device=text.device))
        assert ei.value.status == -1


def test_unaligned_input_rejected():
    w = workloads.tiny_case(303, 4, 30, 2, 5, 10_000)
    text, seg = to_device(w)
    big = torch.zeros(text.numel() + 16, dtype=torch.uint8, device=text.device)
    with pfac.Table(w.patterns, 4) as t:
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match_into(t, big[1:1 + text.numel()], seg,
                            torch.empty(10, dtype=torch.int64, device=text.device))
        assert ei.value.status == -1


def test_async_and_graph_replay():
    w = workloads.tiny_case(304, 256, 1500, 2, 10, 3 << 20, n_segments=200, n_plants=3000)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    dev = text.device
    with pfac.Table(w.patterns, 256) as t:
        ws = torch.empty(pfac.workspace_bytes(t, text.numel(), seg.numel() - 1),
                         dtype=torch.uint8, device=dev)
        out = torch.empty(ref.size + 10, dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            pfac.match_async(t, text, seg, out, cnt, st, ws)
        s.synchronize()
        assert int(cnt.item()) == ref.size and int(st.item()) == 0
        assert_same(keys_np(out[:ref.size]), ref, "async")
        g = torch.cuda.CUDAGraph()
        out.zero_()
        with torch.cuda.graph(g, stream=s):
            pfac.match_async(t, text, seg, out, cnt, st, ws, stream=s)
        for _ in range(3):
            out.zero_()
            cnt.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert int(cnt.item()) == ref.size and int(st.item()) == 0
            assert_same(keys_np(out[:ref.size]), ref, "graph replay")


@pytest.mark.parametrize("sigma,n,lo,hi", [(256, 3000, 2, 12), (4, 2000, 4, 20)])
def test_autotune_keeps_results(tmp_path, sigma, n, lo, hi):
    w = workloads.tiny_case(401 + sigma, sigma, n, lo, hi, 4 << 20, n_plants=2000)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    cache = str(tmp_path / "tune.txt")
    with pfac.Table(w.patterns, sigma) as t:
        r = pfac.autotune(t, text, seg, cache_path=cache)
        assert r["n_tried"] >= 2 and r["from_cache"] == 0
        assert r["variant"] in (0, 1, 2)
        assert_same(run_table(t, text, seg), ref, "tuned default")
        r2 = pfac.autotune(t, text, seg, cache_path=cache)
        if r["variant"]:
            assert r2["from_cache"] == 1
            assert (r2["variant"], r2["prefix_depth"], r2["bitmap_copies"]) == \
                (r["variant"], r["prefix_depth"], r["bitmap_copies"])
        assert_same(run_table(t, text, seg), ref, "cached choice")


def run_table(t, text, seg):
    keys = pfac.match(t, text, seg)
    torch.cuda.synchronize()
    return keys_np(keys)


@pytest.mark.parametrize("copies", [1, 4, 16])
def test_bitmap_copies_option(copies):
    w = workloads.tiny_case(410, 256, 1000, 2, 10, 1 << 20, n_plants=1000)
    ref = oracle_keys(w)
    assert_same(run(w, variant=pfac.VARIANT_FILTER, bitmap_copies=copies), ref, f"copies {copies}")


@pytest.mark.parametrize("sigma,pattern", [(256, b"\x07"), (256, bytes(range(100))),
                                           (4, b"\x01\x02\x03\x00\x01"), (2, b"\x01" * 33)])
def test_single_pattern(sigma, pattern):
    # one pattern: its occurrences are the positions where it is planted (and
    # where the random text happens to hold it)
    rs = np.random.RandomState(len(pattern) * 7 + sigma)
    text = rs.randint(0, sigma, size=300_000).astype(np.uint8)
    for p in rs.randint(0, text.size - len(pattern), size=200):
        text[p:p + len(pattern)] = np.frombuffer(pattern, np.uint8)
    w = workloads.Workload("single", sigma, [pattern], text, workloads.single_segment(text.size))
    ref = check_all_variants(w, f"single pattern sigma {sigma}")
    assert ref.size >= 150


def test_patterns_longer_than_the_input():
    # no walk can complete; short inputs and segments shorter than every pattern
    pats = [bytes([1, 2, 3] * 20), bytes([2] * 70)]
    text = np.tile(np.array([1, 2, 3], np.uint8), 15)
    w = workloads.Workload("long-pats", 4, pats, text, workloads.single_segment(text.size))
    ref = check_all_variants(w, "patterns longer than the input")
    assert ref.size == 0


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_wide_cta(case):
    # 24 warps per CTA (80 registers a thread) wherever the tables leave room
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        kdef = th.info()["prefix_depth"]
    ran = 0
    for k in (kdef, max(1, kdef - 2)):
        for extra in ({}, {"gram_filter": 2}, {"child_masks": 2}):
            try:
                got = run(w, prefix_depth=k, warps_per_cta=24, **extra)
            except pfac.PfacError as e:  # does not fit
                assert e.status == -1, str(e)
                continue
            assert_same(got, ref, f"24 warps depth {k} {extra}")
            ran += 1
    assert ran >= 1


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_records_per_slice_both_ways(case):
    # 32 records per slice (slices with more matched positions are re-scanned
    # by the emit pass) and 512 (one record per position: one pass) give the
    # oracle's keys on both scan kernels where they apply
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma) as t:
        kernels = (1, 2) if bits_per_symbol(sigma) == 8 else (1,)
        for kern in kernels:
            for recs in (32, 512):
                p = pfac.plan(t, scan_kernel=kern, records_per_slice=recs)
                assert p["records_per_slice"] == recs and p["scan_kernel"] == kern
                keys = pfac.match(t, text, seg, scan_kernel=kern, records_per_slice=recs)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"kernel {kern} records {recs}")


def test_dense_matches_one_pass():
    # every position matches several patterns: with 512 records per slice the
    # scan pass keeps them all (no emit pass) and the warp-wide expansion
    # writes the keys; with 32 the emit pass does
    import itertools
    pats = [bytes(p) for L in range(1, 6) for p in itertools.product(range(3), repeat=L)]
    rs = np.random.RandomState(3)
    text = rs.randint(0, 3, size=300_001).astype(np.uint8)
    for sigma in (3, 4):
        w = workloads.Workload("dense", sigma, pats, text, workloads.single_segment(text.size))
        ref = oracle_keys(w)
        assert ref.size > 4 * text.size
        tt, sg = to_device(w)
        with pfac.Table(pats, sigma) as t:
            assert pfac.plan(t)["records_per_slice"] == 512  # the library's choice here
            for recs in (32, 512):
                keys = pfac.match(t, tt, sg, records_per_slice=recs)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"dense sigma {sigma} records {recs}")


@pytest.mark.parametrize("seed,sigma,n,lo,hi,N,S,plants", [
    (601, 4, 3000, 8, 40, 1 << 20, 1, 3000),     # DNA-like: queues of whole slices
    (602, 4, 400, 2, 6, 600_000, 9, 500),        # short patterns: buffer full, partly in place
    (603, 256, 2000, 2, 10, 1 << 20, 40, 2000),
    (604, 20, 800, 1, 6, 400_003, 3, 800),
])
def test_resolver_kernel_same_keys(seed, sigma, n, lo, hi, N, S, plants):
    # the scan kernel's own resolution (resolver=1) and the resolver kernel
    # (resolver=2, with the in-place fallback when its buffer is full) give
    # the oracle's keys through both scan kernels
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    ran = 0
    with pfac.Table(w.patterns, w.sigma) as t:
        for kern in (pfac.binding.KERNEL_QUEUED, pfac.binding.KERNEL_REGISTER):
            for res in (1, 2):
                for recs in (32, 512):
                    opt = dict(scan_kernel=kern, resolver=res, records_per_slice=recs)
                    try:
                        pfac.plan(t, **opt)
                    except pfac.PfacError as e:  # no register-staged kernel for this alphabet
                        assert e.status == -1, str(e)
                        continue
                    keys = pfac.match(t, text, seg, **opt)
                    torch.cuda.synchronize()
                    assert_same(keys_np(keys), ref, f"{opt}")
                    ran += 1
    assert ran >= 4
