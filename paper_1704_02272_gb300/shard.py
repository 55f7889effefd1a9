"""Data-parallel sharding of one matching job over several GPUs.

The failure-less walk of a start position reads at most max_len bytes and
never crosses its segment end (Section 2.3), so the start positions split into
independent ranges.  Rank r scans the starts in [a_r, a_{r+1}) and reads the
text up to a_{r+1} + max_len - 1 (the overlap the chunked matcher of Section
2.2 needs, here only as a read halo: every start is owned by one rank).  The
ranks' sorted lists are already in global order, so the merge is a
concatenation in rank order; the only exchange is one gather of counts and
lists, outside the matching itself.

Shard starts are multiples of 256 bytes so every shard's text stays 16-byte
aligned for the device path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ALIGN = 256


@dataclass
class Shard:
    rank: int
    start: int        # first start position owned
    stop: int         # one past the last start position owned
    read_end: int     # end of the text slice read (halo included)
    seg: np.ndarray   # segment offsets of the slice, relative to start


def plan(n_bytes: int, seg_offsets, world: int, max_len: int) -> list:
    seg = np.asarray(seg_offsets, dtype=np.uint64)
    cuts = [0] + [((r * n_bytes) // world) & ~(ALIGN - 1) for r in range(1, world)] + [n_bytes]
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    out = []
    for r in range(world):
        a, b = cuts[r], cuts[r + 1]
        end = min(b + max(max_len, 1) - 1, n_bytes) if b < n_bytes else n_bytes
        inner = seg[(seg > a) & (seg < end)].astype(np.int64) - a
        local = np.concatenate([[0], inner, [end - a]]).astype(np.uint64)
        out.append(Shard(r, a, b, end, local))
    return out


def own(keys, shard: Shard, id_bits: int = 24):
    """Keeps the keys whose local start is owned by the shard and moves them
    to global positions (works on NumPy uint64 arrays and torch int64 tensors)."""
    lim = (shard.stop - shard.start) << id_bits
    import torch
    if isinstance(keys, torch.Tensor):
        n = int(torch.searchsorted(keys, torch.tensor([lim], dtype=keys.dtype,
                                                      device=keys.device)).item())
        return keys[:n] + (shard.start << id_bits)
    keys = np.asarray(keys, dtype=np.uint64)
    n = int(np.searchsorted(keys, np.uint64(lim)))
    return keys[:n] + np.uint64(shard.start << id_bits)


def match_shard_gpu(table, text_dev, shard: Shard, **opt):
    """This rank's share of the matches, with global positions (device): the
    library starts walks only below the shard's stop and adds its start to
    every reported position, so the keys need no filtering."""
    import torch

    if shard.stop <= shard.start:
        # an empty share (inputs shorter than the ranks' alignment): no call,
        # since starts_end = 0 would mean every position of the halo
        return torch.empty(0, dtype=torch.int64, device=text_dev.device)
    from . import binding
    seg = torch.from_numpy(shard.seg.astype(np.int64)).to(text_dev.device)
    return binding.match(table, text_dev[shard.start:shard.read_end], seg,
                         starts_end=shard.stop - shard.start, position_base=shard.start, **opt)


def gather(keys, group=None):
    """Concatenation of every rank's key tensor in rank order (on all ranks).
    One all_gather of the counts, one of the padded lists."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([keys.numel()], dtype=torch.int64, device=keys.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts) if counts else 0
    pad = torch.zeros(m, dtype=keys.dtype, device=keys.device)
    pad[:keys.numel()] = keys
    bufs = [torch.zeros(m, dtype=keys.dtype, device=keys.device) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[:c] for b, c in zip(bufs, counts)])
