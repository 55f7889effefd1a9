"""GPU parity at the full sizes of the five evaluation workloads, in the
launch configuration the benchmark times.

* plain (1 MiB), DNA (256 MiB) and IDS packets (1 GiB): the whole sorted key
  list against the oracle, element by element, for the compressed table and
  the uncompressed table.
* sweep cells (512 MiB each, up to 1.2e9 matches): the compressed and
  uncompressed kernels agree on the whole list, and both agree with the
  oracle on sampled 1 MiB windows (start, end and random offsets), which the
  oracle computes one window at a time.  Every cell is also compared with the
  oracle over the whole input, 32 MiB of start positions at a time.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device, window

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


def device_keys(w, text, seg, layout):
    with pfac.Table(w.patterns, w.sigma, layout=layout) as t:
        k = pfac.match(t, text, seg)
        torch.cuda.synchronize()
        return k


def full_check(w):
    text, seg = to_device(w)
    ac = oracle.ACOracle(w.patterns)
    ref = oracle_keys(w, ac=ac)
    ac.close()
    kc = device_keys(w, text, seg, pfac.LAYOUT_COMPRESSED)
    assert_same(keys_np(kc), ref, f"{w.name} compressed")
    del kc
    kd = device_keys(w, text, seg, pfac.LAYOUT_DENSE)
    assert_same(keys_np(kd), ref, f"{w.name} dense")
    return ref


def plants_present(w, ref):
    got = set(ref.tolist())
    n = 0
    for p, j in w.plants.tolist():
        pat = w.patterns[j]
        if w.text[p:p + len(pat)].tobytes() == pat:
            assert ((p << 24) | j) in got
            n += 1
    return n


def test_plain_config():
    w = workloads.config1()
    ref = full_check(w)
    assert plants_present(w, ref) >= 1900


def test_dna_config():
    w = workloads.config2()
    ref = full_check(w)
    assert plants_present(w, ref) > 200_000
    assert ref.size > 1_000_000


def test_ids_packets_config():
    w = workloads.config3()
    assert len(w.seg_offsets) > 1_300_000
    ref = full_check(w)
    assert plants_present(w, ref) > 6000


@pytest.mark.parametrize("n", [1, 10, 100, 1000])
def test_letters_shape(n):
    # the paper's throughput-experiment shape (52 letters, 20-symbol
    # patterns), at 8 MiB: the whole list against the oracle
    w = workloads.letters(n, n_bytes=8 << 20, n_plants=200)
    ref = full_check(w)
    assert plants_present(w, ref) >= 150


SWEEP = [(s, n) for s in workloads.CONFIG4_SIGMAS for n in workloads.CONFIG4_COUNTS]


@pytest.mark.parametrize("sigma,n", SWEEP, ids=[f"sig{s}-n{n}" for s, n in SWEEP])
def test_sweep_cell(sigma, n):
    w = workloads.config4(sigma, n)
    text, seg = to_device(w)
    kc = device_keys(w, text, seg, pfac.LAYOUT_COMPRESSED)
    kd = device_keys(w, text, seg, pfac.LAYOUT_DENSE)
    assert kc.numel() == kd.numel() and torch.equal(kc, kd), "compressed != dense"
    del kd
    # the dense layout's thread-serial kernel: another walk over the same trie
    with pfac.Table(w.patterns, w.sigma, layout=pfac.LAYOUT_DENSE) as t:
        ks = pfac.match(t, text, seg, scan_kernel=pfac.binding.KERNEL_SERIAL)
        torch.cuda.synchronize()
    assert ks.numel() == kc.numel() and torch.equal(ks, kc), "compressed != thread-serial dense"
    del ks
    # sorted, unique, in range
    if kc.numel() > 1:
        assert bool((kc[1:] > kc[:-1]).all())
        assert int((kc[-1] >> 24).item()) < w.n_bytes
        assert int((kc & 0xFFFFFF).max().item()) < len(w.patterns)
    ac = oracle.ACOracle(w.patterns)
    rs = np.random.RandomState(sigma * 7 + n)
    win = 1 << 20
    starts = [0, w.n_bytes - win] + [int(x) for x in rs.randint(0, w.n_bytes - win, 4)]
    for a in starts:
        ref = oracle_keys(w, lo=a, hi=a + win, ac=ac)
        assert_same(window(kc, a, a + win), ref, f"{w.name} window {a}")
    ac.close()


@pytest.mark.parametrize("sigma,n", SWEEP, ids=[f"sig{s}-n{n}" for s, n in SWEEP])
def test_sweep_cell_whole_list(sigma, n):
    # every key of the cell against the oracle, chunk by chunk (the oracle's
    # keys of one chunk at a time fit in host memory)
    w = workloads.config4(sigma, n)
    text, seg = to_device(w)
    kc = device_keys(w, text, seg, pfac.LAYOUT_COMPRESSED)
    ac = oracle.ACOracle(w.patterns)
    chunk, total = 32 << 20, 0
    for a in range(0, w.n_bytes, chunk):
        ref = oracle_keys(w, lo=a, hi=min(a + chunk, w.n_bytes), ac=ac)
        assert_same(window(kc, a, a + chunk), ref, f"{w.name} chunk at {a}")
        total += ref.shape[0]
    ac.close()
    assert total == kc.numel()


GRAM_CELLS = [("ids", 0, 0), ("sweep", 256, 10000), ("sweep", 256, 100000), ("sweep", 20, 100000),
              ("sweep", 4, 1000)]


@pytest.mark.parametrize("kind,sigma,n", GRAM_CELLS, ids=[f"{k}-{s}-{n}" for k, s, n in GRAM_CELLS])
def test_gram_filter_full_size(kind, sigma, n):
    # the gram filter as the first stage, forced on and off, gives the same
    # keys as the uncompressed kernel on full-size workloads
    w = workloads.config3() if kind == "ids" else workloads.config4(sigma, n)
    text, seg = to_device(w)
    kd = device_keys(w, text, seg, pfac.LAYOUT_DENSE)
    with pfac.Table(w.patterns, w.sigma) as t:
        assert t.info()["gram_len"] > 0
        for gram in (2, 1):
            kg = pfac.match(t, text, seg, gram_filter=gram)
            torch.cuda.synchronize()
            assert kg.numel() == kd.numel() and torch.equal(kg, kd), f"gram_filter={gram}"
            del kg
        # prefix bytes at the deepest depth of at most 16 index bits
        b = 1
        while (1 << b) < w.sigma:
            b += 1
        k = min(t.info()["prefix_depth"], 16 // b)
        if k >= max(1, t.info()["prefix_depth"] - 2):
            kb = pfac.match(t, text, seg, prefix_bytes=2, prefix_depth=k)
            torch.cuda.synchronize()
            assert kb.numel() == kd.numel() and torch.equal(kb, kd), "prefix_bytes=2"
            del kb
