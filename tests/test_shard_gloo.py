"""Multi-rank path on CPU: world-size 2 and 3 gloo process groups split one
job with the shard plan, match their shares (the oracle stands in for the
per-rank GPU matcher here) and merge in rank order; the merged list must
equal the unsharded result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from paper_1704_02272_gb300 import shard


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CASES = {
    "dna": lambda: workloads.config2(n_bytes=3 << 20, n_patterns=3000),
    "packets": lambda: workloads.config3(n_bytes=4 << 20, n_patterns=4000),
    "tiny-segs": lambda: workloads.tiny_case(7, 4, 200, 1, 9, 50_000, n_segments=2000),
}


def worker(rank, world, port, case, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = CASES[case]()
        plan = shard.plan(w.n_bytes, w.seg_offsets, world, w.max_len)
        sh = plan[rank]
        pos, ids = oracle.match_ac(w.patterns, w.text[sh.start:sh.read_end], sh.seg, threads=2)
        local = shard.own(oracle.pack_keys(pos, ids), sh)
        merged = shard.gather(torch.from_numpy(local.astype(np.int64)))
        if rank == 0:
            ref = oracle.pack_keys(*oracle.match_ac(w.patterns, w.text, w.seg_offsets))
            q.put((merged.numpy().view(np.uint64).tolist() == ref.tolist(), int(ref.size),
                   [(p.start, p.stop) for p in plan]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_equals_unsharded(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    ok, n, cuts = q.get(timeout=10)
    assert n > 0 and ok, cuts
    # shards tile the start positions and start on aligned offsets
    assert cuts[0][0] == 0 and all(a % shard.ALIGN == 0 for a, _ in cuts)
    assert all(cuts[i][1] == cuts[i + 1][0] for i in range(len(cuts) - 1))


def test_plan_halo_and_segments():
    seg = np.array([0, 10, 10, 700, 1000, 4000], dtype=np.uint64)
    plan = shard.plan(4000, seg, 3, 50)
    assert [(p.start, p.stop) for p in plan] == [(0, 1280), (1280, 2560), (2560, 4000)]
    assert plan[0].read_end == 1280 + 49 and plan[2].read_end == 4000
    assert plan[0].seg.tolist() == [0, 10, 10, 700, 1000, 1329]
    assert plan[1].seg.tolist() == [0, 2560 + 49 - 1280]


def test_tiny_input_leaves_empty_shares_that_start_no_walk():
    # 1000 bytes over 8 ranks: the 256-byte alignment leaves some shares
    # empty; the shares still tile the input and an empty one yields nothing
    seg = np.array([0, 1000], dtype=np.uint64)
    plan = shard.plan(1000, seg, 8, 50)
    assert plan[0].start == 0 and plan[-1].stop == 1000
    assert all(plan[i].stop == plan[i + 1].start for i in range(7))
    empty = [p for p in plan if p.stop == p.start]
    assert empty
    text = torch.zeros(1000, dtype=torch.uint8)
    for p in empty:
        assert shard.match_shard_gpu(None, text, p).numel() == 0
        assert shard.own(np.array([0, 5 << 24], dtype=np.uint64), p).size == 0
