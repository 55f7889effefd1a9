"""GPU parity of the register-staged scan kernel (alphabets of 129 to 256
symbols, and of up to 4): the C ABI with scan_kernel = 2 against the CPU
oracle, element by
element, for every first stage (prefix bitmap, gram filter), bitmap copies,
prefix depth, child masks on and off and entries in or out of shared memory,
on single- and multi-segment inputs with ragged ends, and on inputs dense
enough that slices overflow the queue and their record space."""
import itertools

import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")

REG = pfac.binding.KERNEL_REGISTER


def match_keys(t, text, seg, **kw):
    keys = pfac.match(t, text, seg, scan_kernel=REG, **kw)
    torch.cuda.synchronize()
    return keys_np(keys)


def every_plan(w, ref, what, depths):
    """Runs every register-staged plan that fits and checks each against the
    oracle; returns how many ran."""
    text, seg = to_device(w)
    ran = 0
    with pfac.Table(w.patterns, w.sigma) as t:
        # the library's own choice first
        assert_same(match_keys(t, text, seg), ref, f"{what} default")
        assert pfac.plan(t, scan_kernel=REG)["scan_kernel"] == REG
        for k, var, masks, gram, copies in itertools.product(
                depths, (1, 2), (1, 2), (1, 2), (1, 2, 4, 8, 16)):
            opt = dict(prefix_depth=k, variant=var, child_masks=masks, gram_filter=gram,
                       bitmap_copies=copies)
            try:
                p = pfac.plan(t, scan_kernel=REG, **opt)
            except pfac.PfacError as e:  # does not fit, or no masks / gram at this depth
                assert e.status == -1, str(e)
                continue
            assert p["scan_kernel"] == REG and p["warps_per_cta"] == 16
            assert_same(match_keys(t, text, seg, **opt), ref, f"{what} {opt}")
            ran += 1
    return ran


CASES = [
    # seed, sigma, n_patterns, lo, hi, n_bytes, n_segments, n_plants, text_sigma
    (201, 256, 2000, 2, 12, 1 << 20, 1, 2000, None),
    (202, 256, 500, 1, 40, 100_003, 1, 300, None),        # ragged tail, 1-byte patterns
    (203, 256, 3000, 2, 9, 600_000, 400, 1500, None),     # many segments
    (204, 200, 800, 1, 6, 300_000, 17, 800, 256),         # bytes >= sigma in the text
    (205, 256, 50, 3, 20, 33_000, 3, 200, None),          # few slices, tiny segments
    (206, 130, 4000, 1, 4, 500_000, 1, 1000, None),       # short patterns, dense prefixes
    # 2-bit symbols (one per byte)
    (221, 4, 400, 4, 14, 400_000, 1, 800, None),
    (222, 4, 2000, 8, 30, 300_003, 1, 500, None),          # ragged tail, long patterns
    (223, 4, 300, 2, 12, 350_000, 300, 700, None),         # many segments
    (224, 4, 200, 1, 9, 250_000, 9, 600, 8),               # bytes 4..7 in the text
    (225, 3, 150, 1, 8, 200_000, 5, 500, 4),               # symbol 3 outside the alphabet
    (226, 3, 60, 1, 12, 150_000, 3, 300, 200),            # bytes far outside the alphabet
]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_register_kernel_all_plans(case):
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    assert ref.size > 0
    with pfac.Table(w.patterns, w.sigma, host_only=True) as th:
        kdef = th.info()["prefix_depth"]
    ran = every_plan(w, ref, f"case {seed}", sorted({max(1, kdef - 2), kdef}))
    assert ran >= 8


def dense_case(seed, n_bytes, n_segments):
    """Every string of 1 to 6 symbols over {0, 1} as a pattern of a 256-symbol
    table, and a text over {0, 1}: every position matches up to six patterns,
    so every slice has 512 survivors (four queues' worth) and far more
    matched positions than its record space."""
    pats = [bytes(p) for L in range(1, 7) for p in itertools.product((0, 1), repeat=L)]
    rs = np.random.RandomState(seed)
    text = rs.randint(0, 2, size=n_bytes).astype(np.uint8)
    if n_segments <= 1:
        off = workloads.single_segment(n_bytes)
    else:
        cuts = np.sort(rs.randint(0, n_bytes + 1, size=n_segments - 1))
        off = np.concatenate([[0], cuts, [n_bytes]]).astype(np.uint64)
    return workloads.Workload(f"dense-{seed}", 256, pats, text, off)


@pytest.mark.parametrize("n_bytes,n_segments", [(200_000, 1), (150_001, 60)])
def test_register_kernel_dense_slices(n_bytes, n_segments):
    w = dense_case(7 + n_segments, n_bytes, n_segments)
    ref = oracle_keys(w)
    assert ref.size > 5 * n_bytes  # about six matches per position
    text, seg = to_device(w)
    with pfac.Table(w.patterns, w.sigma) as t:
        for copies in (1, 16):
            for masks in (1, 2):
                opt = dict(bitmap_copies=copies, child_masks=masks, gram_filter=1)
                try:
                    got = match_keys(t, text, seg, **opt)
                except pfac.PfacError as e:
                    assert e.status == -1, str(e)
                    continue
                assert_same(got, ref, f"dense {opt}")
        assert_same(match_keys(t, text, seg, gram_filter=2), ref, "dense, gram filter")


def test_register_kernel_edges():
    # empty input, inputs shorter than a slice, a pair, ragged lengths around
    # the 16-byte chunks and the 4-byte halo
    pats = [b"\x07", b"\x07\x08", b"\x08\x09\x0a", b"\xff\x00", b"\x00\x00\x00\x00\x00"]
    rs = np.random.RandomState(5)
    with pfac.Table(pats, 256) as t:
        for n in (0, 1, 2, 15, 16, 17, 511, 512, 513, 515, 516, 517, 527, 528, 1023, 1024,
                  1025, 1028, 1040, 4099):
            text = rs.choice(np.array([0, 7, 8, 9, 10, 255], np.uint8), size=n)
            w = workloads.Workload(f"edge-{n}", 256, pats, text, workloads.single_segment(n))
            ref = oracle_keys(w)
            tt, sg = to_device(w)
            for copies in (1, 16):
                got = match_keys(t, tt, sg, bitmap_copies=copies, gram_filter=1)
                assert_same(got, ref, f"n={n} copies {copies}")


def test_register_kernel_starts_end_and_base():
    # a shard: walks start below starts_end only, positions offset by
    # position_base, the max_len - 1 bytes after starts_end read as the halo
    w = workloads.tiny_case(211, 256, 1500, 2, 10, 300_000, n_plants=800)
    text, _ = to_device(w)
    ref = oracle_keys(w)
    base, hi = 70_000, 200_000  # base 16-byte aligned, like every input
    sub = text[base:min(hi + w.max_len - 1, w.n_bytes)]
    seg_sub = torch.tensor([0, sub.numel()], dtype=torch.int64, device=text.device)
    with pfac.Table(w.patterns, 256) as t:
        keys = pfac.match(t, sub, seg_sub, scan_kernel=REG, starts_end=hi - base,
                          position_base=base)
        torch.cuda.synchronize()
    pos = ref >> np.uint64(24)
    want = ref[(pos >= np.uint64(base)) & (pos < np.uint64(hi))]
    assert_same(keys_np(keys), want, "shard")


def test_register_kernel_full_size_dna():
    # the DNA-shaped workload at its full 256 MiB: whole list against the
    # oracle in 32 MiB windows of start positions
    w = workloads.config2()
    text, seg = to_device(w)
    import oracle
    ac = oracle.ACOracle(w.patterns)
    try:
        step = 32 << 20
        ref = np.concatenate([oracle_keys(w, lo=a, hi=min(a + step, w.n_bytes), ac=ac)
                              for a in range(0, w.n_bytes, step)])
        with pfac.Table(w.patterns, 4) as t:
            for opt in ({}, {"gram_filter": 2}, {"prefix_depth": 9, "bitmap_copies": 4}):
                keys = pfac.match(t, text, seg, scan_kernel=REG, **opt)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"dna {opt}")
    finally:
        ac.close()


def test_register_kernel_full_size_sweep_cell():
    # the alphabet-256 cell with 1,000 patterns at its full 512 MiB, through
    # the plan the library picks and the one with the most copies, whole list
    # against the oracle in 32 MiB windows of start positions
    w = workloads.config4(256, 1000)
    text, seg = to_device(w)
    import oracle
    ac = oracle.ACOracle(w.patterns)
    try:
        step = 32 << 20
        ref = np.concatenate([oracle_keys(w, lo=a, hi=min(a + step, w.n_bytes), ac=ac)
                              for a in range(0, w.n_bytes, step)])
        with pfac.Table(w.patterns, 256) as t:
            for opt in ({}, {"bitmap_copies": 16, "gram_filter": 1}):
                keys = pfac.match(t, text, seg, scan_kernel=REG, **opt)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"sweep 256x1000 {opt}")
    finally:
        ac.close()
