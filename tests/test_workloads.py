"""The seeded inputs follow the stated recipe: alphabets, pattern-length
ranges and distributions, de-duplication, segment (packet) size mixes, plant
counts and placement, Poisson arrivals, and determinism per seed.  Sizes are
reduced where the recipe allows it (the generators take the size as an
argument), so the suite stays quick."""
import numpy as np
import pytest

import workloads


def lengths(pats):
    return np.array([len(p) for p in pats])


def symbols(pats):
    return np.frombuffer(b"".join(pats), dtype=np.uint8)


def intact_share(w):
    """Share of the plants still intact in the text (a later plant may
    overwrite part of an earlier one); the last plant is always intact."""
    ok = [bytes(w.text[p:p + len(w.patterns[j])]) == w.patterns[j] for p, j in w.plants.tolist()]
    assert ok[-1]
    return float(np.mean(ok))


def test_seeds_are_deterministic_and_distinct():
    a = workloads.config1(n_bytes=1 << 16)
    b = workloads.config1(n_bytes=1 << 16)
    assert a.patterns == b.patterns and np.array_equal(a.text, b.text)
    assert np.array_equal(a.plants, b.plants)
    c = workloads.config1(seed=workloads.seed_for(1) + 1, n_bytes=1 << 16)
    assert not np.array_equal(a.text, c.text)
    assert len({workloads.seed_for(4, s, n) for s in workloads.CONFIG4_SIGMAS
                for n in workloads.CONFIG4_COUNTS}) == 12


def test_dedup_keeps_first_occurrence_in_order():
    assert workloads.dedup([b"ab", b"c", b"ab", b"d", b"c"]) == [b"ab", b"c", b"d"]


def test_plain_config_shape():
    w = workloads.config1()
    L = lengths(w.patterns)
    assert w.sigma == 256 and w.n_bytes == 1 << 20
    assert 990 <= len(w.patterns) <= 1000 and L.min() >= 4 and L.max() <= 32
    assert len(set(w.patterns)) == len(w.patterns)
    assert w.seg_offsets.tolist() == [0, 1 << 20]
    assert w.plants.shape == (2000, 2) and intact_share(w) > 0.95
    assert int((w.plants[:, 0] + lengths(w.patterns)[w.plants[:, 1]]).max()) <= w.n_bytes


def test_dna_config_shape():
    w = workloads.config2(n_bytes=4 << 20)
    L = lengths(w.patterns)
    assert w.sigma == 4 and int(w.text.max()) <= 3 and int(symbols(w.patterns).max()) <= 3
    assert 9990 <= len(w.patterns) <= 10000 and L.min() >= 8 and L.max() <= 64
    assert abs(L.mean() - 36) < 1.0  # U[8,64]
    assert w.plants.shape[0] == round(0.001 * w.n_bytes) and intact_share(w) > 0.9
    assert int(np.bincount(w.text, minlength=4).min()) > 0.24 * w.n_bytes


def test_ids_config_shape():
    w = workloads.config3(n_bytes=64 << 20)
    L = lengths(w.patterns)
    assert w.sigma == 256 and len(w.patterns) > 19000
    assert L.min() >= 2 and L.max() <= 256
    assert 11 <= np.median(L) <= 13  # log-normal, median 12
    printable = [bool(((np.frombuffer(p, np.uint8) >= 0x20) & (np.frombuffer(p, np.uint8) <= 0x7E)).all())
                 for p in w.patterns if len(p) >= 8]
    assert 0.57 < np.mean(printable) < 0.63  # 60% printable (long ones rarely printable by chance)
    off = w.seg_offsets.astype(np.int64)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == w.n_bytes and (sizes > 0).all()
    body = sizes[:-1]  # the last packet is cut to the total
    small = (body >= 64) & (body <= 128)
    large = (body >= 1000) & (body <= 1500)
    assert (small | large).all()
    assert 0.38 < small.mean() < 0.42
    assert w.meta["n_packets"] == sizes.shape[0]
    # about 0.5% of packets carry one plant, fully inside the packet
    assert 0.004 < w.plants.shape[0] / sizes.shape[0] < 0.006
    seg_of = np.searchsorted(off, w.plants[:, 0], side="right") - 1
    ends = w.plants[:, 0] + L[w.plants[:, 1]]
    assert (ends <= off[seg_of + 1]).all()


@pytest.mark.parametrize("sigma", workloads.CONFIG4_SIGMAS)
def test_sweep_cell_shape(sigma):
    w = workloads.config4(sigma, 1000, n_bytes=1 << 20)
    L = lengths(w.patterns)
    assert L.min() >= 4 and L.max() <= 64
    assert int(symbols(w.patterns).max()) < sigma and int(w.text.max()) < sigma
    assert w.seg_offsets.tolist() == [0, 1 << 20]


def test_letters_shape():
    w = workloads.letters(100, n_bytes=1 << 20, n_plants=50)
    assert w.sigma == 52 and set(lengths(w.patterns).tolist()) == {20}
    assert int(w.text.max()) < 52 and int(symbols(w.patterns).max()) < 52
    assert w.plants.shape[0] == 50 and intact_share(w) > 0.9


def test_serving_batches_and_arrivals():
    rs = np.random.RandomState(5)
    pats = workloads.config5_patterns(n_patterns=2000)
    for _ in range(20):
        text, off = workloads.serving_batch(rs, pats)
        sizes = np.diff(off.astype(np.int64))
        assert 1 <= sizes.shape[0] <= 4096
        assert sizes.min() >= 64 and sizes.max() <= 9000 and int(off[-1]) == text.shape[0]
    t = workloads.poisson_arrivals(np.random.RandomState(1), 1000.0, 20000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all() and abs(gaps.mean() - 1e-3) < 3e-5
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential gaps
