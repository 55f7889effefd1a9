"""Seeded synthetic workloads for the PFAC matcher and its oracle.

This module only draws random data: pattern sets, input texts, segment
(packet) offsets and planted occurrences.  It holds none of the matching
arithmetic, so both the CPU oracle and the GPU path may take their inputs from
it without sharing any of the method.

Every generator uses NumPy's MT19937 (``RandomState``), the Mersenne Twister
that the paper's evaluation draws its synthetic files from (Section 4).  The
five workload shapes follow the evaluation plan of this project:

* ``config1``  alphabet 256, 1,000 patterns of length U[4,32], 1 MiB input,
  2,000 planted occurrences, one segment.
* ``config2``  DNA-shaped: alphabet 4 (codes 0..3), 10,000 patterns of length
  U[8,64], 256 MiB input, 0.1% of positions planted, one segment.
* ``config3``  IDS-shaped: 20,000 patterns with log-normal lengths (median 12,
  ln-sigma 0.75, rounded, clipped to [2,256]), 60% printable ASCII and 40%
  uniform bytes; 1 GiB of packets (40% U[64,128], 60% U[1000,1500] bytes),
  0.5% of packets carrying one planted pattern.
* ``config4``  sweep cell: alphabet in {4,20,64,256}, pattern count in
  {1k,10k,100k}, lengths U[4,64], 512 MiB uniform input, one segment.
* ``config5``  serving: 50,000 patterns drawn like config 3; batches of
  U[1,4096] packets of U[64,9000] bytes arriving as a Poisson process.

Duplicate patterns are dropped keeping the first occurrence, and the survivors
are re-indexed consecutively (pattern ids are positions in the returned list).
Planted occurrences are written in generation order, so a later plant may
overwrite part of an earlier one; the oracle always runs on the final buffer.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 170402272
PRINTABLE_LO, PRINTABLE_HI = 0x20, 0x7E


@dataclass
class Workload:
    name: str
    sigma: int
    patterns: list            # list[bytes]; pattern id = list index
    text: np.ndarray          # uint8[N]
    seg_offsets: np.ndarray   # uint64[S+1], 0 = o_0 <= ... <= o_S = N
    plants: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int64))  # (pos, id)
    meta: dict = field(default_factory=dict)

    @property
    def n_bytes(self) -> int:
        return int(self.text.shape[0])

    @property
    def max_len(self) -> int:
        return max((len(p) for p in self.patterns), default=0)


def seed_for(config: int, *cell) -> int:
    """Default seed of a workload: the base seed plus the config number,
    with sweep cells adding their (alphabet, pattern count) coordinates."""
    s = SEED_BASE + config
    if cell:
        sigma, n = cell
        s += (sigma << 20) + n
    return s


def dedup(patterns) -> list:
    seen = set()
    out = []
    for p in patterns:
        if p not in seen:
            seen.add(p)
            out.append(p)
    return out


def uniform_symbols(rs: np.random.RandomState, n: int, sigma: int) -> np.ndarray:
    if sigma == 256:
        return np.frombuffer(rs.bytes(n), dtype=np.uint8).copy()
    return rs.randint(0, sigma, size=n, dtype=np.uint8)


def uniform_patterns(rs, n, sigma, lo, hi) -> list:
    lens = rs.randint(lo, hi + 1, size=n)
    flat = uniform_symbols(rs, int(lens.sum()), sigma)
    out, o = [], 0
    for L in lens:
        out.append(flat[o:o + L].tobytes())
        o += L
    return dedup(out)


def lognormal_lengths(rs, n, median=12.0, ln_sigma=0.75, lo=2, hi=256) -> np.ndarray:
    raw = rs.lognormal(mean=np.log(median), sigma=ln_sigma, size=n)
    return np.clip(np.rint(raw), lo, hi).astype(np.int64)


def ids_patterns(rs, n, printable_frac=0.6) -> list:
    """Byte patterns shaped like IDS signatures: log-normal lengths, each
    pattern either printable ASCII (0x20..0x7E) or uniform bytes."""
    lens = lognormal_lengths(rs, n)
    printable = rs.random_sample(n) < printable_frac
    out = []
    for L, pr in zip(lens, printable):
        if pr:
            b = rs.randint(PRINTABLE_LO, PRINTABLE_HI + 1, size=L, dtype=np.uint8)
        else:
            b = np.frombuffer(rs.bytes(int(L)), dtype=np.uint8)
        out.append(b.tobytes())
    return dedup(out)


def plant_into(rs, text, patterns, seg_offsets, segs, tries=16) -> np.ndarray:
    """Write one occurrence of a uniformly chosen pattern into each listed
    segment, fully inside it.  A pattern longer than the segment is redrawn up
    to ``tries`` times; if none fits the segment gets no plant."""
    plants = []
    n = len(patterns)
    for s in segs:
        a, b = int(seg_offsets[s]), int(seg_offsets[s + 1])
        for _ in range(tries):
            j = int(rs.randint(0, n))
            L = len(patterns[j])
            if L <= b - a:
                p = int(rs.randint(a, b - L + 1))
                text[p:p + L] = np.frombuffer(patterns[j], dtype=np.uint8)
                plants.append((p, j))
                break
    return np.asarray(plants, dtype=np.int64).reshape(-1, 2)


def plant_positions(rs, text, patterns, n_plants) -> np.ndarray:
    """Plant ``n_plants`` occurrences at uniform offsets of a single-segment
    text (pattern index uniform, occurrence fully inside the text)."""
    N = text.shape[0]
    n = len(patterns)
    ids = rs.randint(0, n, size=n_plants)
    lens = np.array([len(p) for p in patterns], dtype=np.int64)[ids]
    keep = lens <= N
    ids, lens = ids[keep], lens[keep]
    pos = (rs.random_sample(ids.shape[0]) * (N - lens + 1)).astype(np.int64)
    for p, j in zip(pos.tolist(), ids.tolist()):
        pat = patterns[j]
        text[p:p + len(pat)] = np.frombuffer(pat, dtype=np.uint8)
    return np.stack([pos, ids.astype(np.int64)], axis=1) if ids.size else np.zeros((0, 2), np.int64)


def single_segment(n_bytes: int) -> np.ndarray:
    return np.array([0, n_bytes], dtype=np.uint64)


def packet_lengths(rs, total, mix=((0.4, 64, 128), (0.6, 1000, 1500))) -> np.ndarray:
    """Packet sizes drawn from a mixture of uniform ranges until ``total``
    bytes are covered; the last packet is cut so the sizes sum to ``total``."""
    mean = sum(w * (lo + hi) / 2 for w, lo, hi in mix)
    out = []
    covered = 0
    while covered < total:
        m = int((total - covered) / mean) + 1024
        u = rs.random_sample(m)
        lens = np.empty(m, dtype=np.int64)
        acc = 0.0
        for w, lo, hi in mix:
            sel = (u >= acc) & (u < acc + w)
            lens[sel] = rs.randint(lo, hi + 1, size=int(sel.sum()))
            acc += w
        lens[u >= acc] = rs.randint(mix[-1][1], mix[-1][2] + 1, size=int((u >= acc).sum()))
        cs = np.cumsum(lens) + covered
        cut = int(np.searchsorted(cs, total))
        if cut < m:
            lens = lens[:cut + 1]
            lens[-1] -= int(cs[cut] - total)
            out.append(lens)
            covered = total
        else:
            out.append(lens)
            covered = int(cs[-1])
    lens = np.concatenate(out)
    return lens[lens > 0] if total > 0 else lens[:0]


def offsets_from_lengths(lens) -> np.ndarray:
    off = np.zeros(len(lens) + 1, dtype=np.uint64)
    np.cumsum(np.asarray(lens, dtype=np.uint64), out=off[1:])
    return off


# --------------------------------------------------------------------------
# The five evaluation workloads
# --------------------------------------------------------------------------

def config1(seed=None, n_bytes=1 << 20, n_plants=2000, n_patterns=1000) -> Workload:
    rs = np.random.RandomState(seed_for(1) if seed is None else seed)
    pats = uniform_patterns(rs, n_patterns, 256, 4, 32)
    text = uniform_symbols(rs, n_bytes, 256)
    plants = plant_positions(rs, text, pats, n_plants)
    return Workload("plain-256x1k-1MiB", 256, pats, text, single_segment(n_bytes), plants)


def config2(seed=None, n_bytes=256 << 20, plant_frac=0.001, n_patterns=10000) -> Workload:
    rs = np.random.RandomState(seed_for(2) if seed is None else seed)
    pats = uniform_patterns(rs, n_patterns, 4, 8, 64)
    text = uniform_symbols(rs, n_bytes, 4)
    plants = plant_positions(rs, text, pats, int(round(plant_frac * n_bytes)))
    return Workload("dna-4x10k-256MiB", 4, pats, text, single_segment(n_bytes), plants)


def config3(seed=None, n_bytes=1 << 30, plant_frac=0.005, n_patterns=20000) -> Workload:
    rs = np.random.RandomState(seed_for(3) if seed is None else seed)
    pats = ids_patterns(rs, n_patterns)
    lens = packet_lengths(rs, n_bytes)
    off = offsets_from_lengths(lens)
    text = uniform_symbols(rs, n_bytes, 256)
    S = len(lens)
    segs = np.flatnonzero(rs.random_sample(S) < plant_frac)
    plants = plant_into(rs, text, pats, off, segs)
    return Workload("ids-256x20k-1GiB-packets", 256, pats, text, off, plants,
                    meta={"n_packets": S})


CONFIG4_SIGMAS = (4, 20, 64, 256)
CONFIG4_COUNTS = (1000, 10000, 100000)


def config4(sigma, n_patterns, seed=None, n_bytes=512 << 20) -> Workload:
    rs = np.random.RandomState(seed_for(4, sigma, n_patterns) if seed is None else seed)
    pats = uniform_patterns(rs, n_patterns, sigma, 4, 64)
    text = uniform_symbols(rs, n_bytes, sigma)
    return Workload(f"sweep-{sigma}x{n_patterns}-{n_bytes >> 20}MiB", sigma, pats, text,
                    single_segment(n_bytes))


def letters(n_patterns, seed=None, n_bytes=100 << 20, n_plants=1000) -> Workload:
    """The throughput experiments' shape (Section 4, Fig. 7-9): an alphabet of
    52 letters (codes 0..51), patterns of 20 symbols, uniform random 100 MiB
    text as one segment; a few plants so matches exist."""
    rs = np.random.RandomState(seed_for(6, 52, n_patterns) if seed is None else seed)
    pats = uniform_patterns(rs, n_patterns, 52, 20, 20)
    text = uniform_symbols(rs, n_bytes, 52)
    off = single_segment(n_bytes)
    plants = plant_into(rs, text, pats, off, np.zeros(n_plants, np.int64)) if pats else None
    return Workload(f"letters-52x{n_patterns}-{n_bytes >> 20}MiB", 52, pats, text, off, plants)


def config5_patterns(seed=None, n_patterns=50000) -> list:
    rs = np.random.RandomState(seed_for(5) if seed is None else seed)
    return ids_patterns(rs, n_patterns)


def serving_batch(rs, patterns, max_packets=4096, lo=64, hi=9000, plant_frac=0.005):
    """One request of the serving workload: U[1,max_packets] packets of
    U[lo,hi] uniform-random bytes, 0.5% of them carrying one planted pattern.
    Returns (text uint8[N], seg_offsets uint64[S+1])."""
    S = int(rs.randint(1, max_packets + 1))
    lens = rs.randint(lo, hi + 1, size=S)
    off = offsets_from_lengths(lens)
    text = uniform_symbols(rs, int(off[-1]), 256)
    segs = np.flatnonzero(rs.random_sample(S) < plant_frac)
    plant_into(rs, text, patterns, off, segs)
    return text, off


def poisson_arrivals(rs, rate_per_s, n) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process."""
    return np.cumsum(rs.exponential(1.0 / rate_per_s, size=n))


# --------------------------------------------------------------------------
# Small cases for tests
# --------------------------------------------------------------------------

def tiny_case(seed, sigma, n_patterns, lo, hi, n_bytes, n_segments=1, n_plants=0,
              text_sigma=None) -> Workload:
    """Random small case: uniform patterns over ``sigma`` symbols, uniform
    text over ``text_sigma`` symbols (default ``sigma``; a larger value puts
    out-of-alphabet bytes into the text), random segment cuts, plants."""
    rs = np.random.RandomState(seed)
    pats = uniform_patterns(rs, n_patterns, sigma, lo, hi) if n_patterns else []
    text = uniform_symbols(rs, n_bytes, text_sigma or sigma)
    if n_segments <= 1 or n_bytes == 0:
        off = single_segment(n_bytes)
    else:
        cuts = np.sort(rs.randint(0, n_bytes + 1, size=n_segments - 1))
        off = np.concatenate([[0], cuts, [n_bytes]]).astype(np.uint64)
    plants = np.zeros((0, 2), np.int64)
    if n_plants and pats:
        segs = rs.randint(0, len(off) - 1, size=n_plants)
        plants = plant_into(rs, text, pats, off, segs)
    return Workload(f"tiny-{seed}", sigma, pats, text, off, plants)


def prefix_heavy_case(seed, sigma, n_bytes, n_segments=1) -> Workload:
    """Patterns that are prefixes of one another (chains like a, ab, abc ...)
    plus their random extensions, over a small alphabet so they match often."""
    rs = np.random.RandomState(seed)
    pats = []
    for _ in range(6):
        L = int(rs.randint(3, 9))
        base = uniform_symbols(rs, L, sigma).tobytes()
        for k in range(1, L + 1):
            pats.append(base[:k])
        for _ in range(3):
            pats.append(base + uniform_symbols(rs, int(rs.randint(1, 4)), sigma).tobytes())
    pats = dedup(pats)
    rs.shuffle(pats)
    text = uniform_symbols(rs, n_bytes, sigma)
    if n_segments <= 1 or n_bytes == 0:
        off = single_segment(n_bytes)
    else:
        cuts = np.sort(rs.randint(0, n_bytes + 1, size=n_segments - 1))
        off = np.concatenate([[0], cuts, [n_bytes]]).astype(np.uint64)
    return Workload(f"prefix-heavy-{seed}", sigma, pats, text, off)


def flatten_patterns(patterns):
    """Concatenated bytes and uint64 offsets (n+1) of a pattern list."""
    lens = np.array([len(p) for p in patterns], dtype=np.uint64)
    off = np.zeros(len(patterns) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    flat = np.frombuffer(b"".join(patterns), dtype=np.uint8) if patterns else np.zeros(0, np.uint8)
    return flat.copy(), off
