"""GPU parity of the two record formats for alphabets of up to 8 symbols:
one packed word per node (the default) and the two-word records of the
32-symbol format (wide_records=True), each against the CPU oracle through
the plans that fit, on plain, multi-segment and prefix-heavy sets."""
import itertools

import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")

CASES = [
    # seed, sigma, n_patterns, lo, hi, n_bytes, n_segments, n_plants, text_sigma
    (401, 4, 1500, 6, 30, 400_000, 1, 1500, None),
    (402, 2, 60, 1, 12, 200_001, 9, 400, 3),       # sigma 2, a byte outside
    (403, 8, 900, 2, 10, 300_000, 20, 900, 12),    # 8 symbols (8-bit bitmaps)
    (404, 6, 400, 1, 7, 250_000, 1, 600, None),
    (405, 3, 300, 3, 9, 150_003, 4, 500, None),
]


@pytest.mark.parametrize("case", CASES, ids=[f"s{c[0]}-sig{c[1]}" for c in CASES])
def test_packed_and_wide_records(case):
    seed, sigma, n, lo, hi, N, S, plants, ts = case
    w = workloads.tiny_case(seed, sigma, n, lo, hi, N, n_segments=S, n_plants=plants,
                            text_sigma=ts)
    ref = oracle_keys(w)
    assert ref.size > 0
    text, seg = to_device(w)
    for wide in (False, True):
        with pfac.Table(w.patterns, sigma, wide_records=wide) as t:
            info = t.info()
            assert info["record_bytes"] == (8 if wide else 4)
            keys = pfac.match(t, text, seg)
            torch.cuda.synchronize()
            assert_same(keys_np(keys), ref, f"wide={wide} default")
            kdef = info["prefix_depth"]
            ran = 0
            for k, var, masks in itertools.product(sorted({max(1, kdef - 2), kdef}), (1, 2),
                                                   (1, 2)):
                opt = dict(prefix_depth=k, variant=var, child_masks=masks)
                try:
                    pfac.plan(t, **opt)
                except pfac.PfacError as e:
                    assert e.status == -1, str(e)
                    continue
                keys = pfac.match(t, text, seg, **opt)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"wide={wide} {opt}")
                ran += 1
            assert ran >= 2


def test_prefix_heavy_packed_outputs():
    # many records with outputs (patterns that are prefixes of others): the
    # packed format's output ranks across many 32-record words
    for seed in range(3):
        w = workloads.prefix_heavy_case(20 + seed, 4, 300_000, n_segments=3)
        ref = oracle_keys(w)
        text, seg = to_device(w)
        for wide in (False, True):
            with pfac.Table(w.patterns, 4, wide_records=wide) as t:
                keys = pfac.match(t, text, seg)
                torch.cuda.synchronize()
                assert_same(keys_np(keys), ref, f"seed {seed} wide={wide}")
