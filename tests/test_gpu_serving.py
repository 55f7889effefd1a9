"""Serving loop (continuous batching): requests of the serving workload go
through pfac_server_* concurrently, admitted as slots and pool memory free
up; each result must equal the same request matched alone (and the oracle
for a sample of them)."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpu_util import assert_same, keys_np

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")


@pytest.fixture(scope="module")
def serving_setup():
    pats = workloads.config5_patterns(n_patterns=50000)
    rs = np.random.RandomState(55)
    reqs = [workloads.serving_batch(rs, pats, max_packets=300) for _ in range(36)]
    table = pfac.Table(pats, 256)
    yield pats, reqs, table
    table.close()


def alone(table, text, seg):
    t = torch.from_numpy(text).cuda()
    s = torch.from_numpy(seg.astype(np.int64)).cuda()
    k = pfac.match(table, t, s)
    torch.cuda.synchronize()
    return keys_np(k)


# result arenas: the default (every result's keys land in it) and one of
# 64 KiB (most results go through the slots' staging copy instead)
ARENAS = [0, 1 << 16]


@pytest.mark.parametrize("host_bytes", ARENAS, ids=["arena", "small-arena"])
def test_results_same_alone_and_in_the_mix(serving_setup, host_bytes):
    pats, reqs, table = serving_setup
    ref = [alone(table, t, s) for t, s in reqs]
    # a pool that holds only a few requests at a time forces admission waits
    biggest = max(t.size for t, _ in reqs)
    with pfac.Server(table, n_slots=4, device_bytes=6 * biggest + (64 << 20),
                     max_request_bytes=biggest, host_bytes=host_bytes) as srv:
        ids = [srv.submit(t, s) for t, s in reqs]
        got = [srv.wait(i, timeout=120) for i in ids]
        for i in ids:
            srv.release(i)
    for k, (g, r) in enumerate(zip(got, ref)):
        assert g["status"] == 0
        assert_same(g["keys"], r, f"request {k}")
        assert g["t_submit"] <= g["t_admit"] <= g["t_issued"] <= g["t_counted"] <= g["t_done"]
    # later requests waited for earlier ones to free memory or slots
    assert max(g["t_admit"] - g["t_submit"] for g in got) > 0
    for k in (0, 7, 35):
        t, s = reqs[k]
        pos, ids_ = oracle.match_ac(pats, t, s)
        assert_same(got[k]["keys"], oracle.pack_keys(pos, ids_), f"oracle request {k}")


def test_poisson_arrivals_and_poll(serving_setup):
    pats, reqs, table = serving_setup
    ref = [alone(table, t, s) for t, s in reqs[:20]]
    rs = np.random.RandomState(7)
    arrivals = workloads.poisson_arrivals(rs, 400.0, 20)
    done = {}
    with pfac.Server(table, n_slots=3, device_bytes=1 << 30) as srv:
        order = []

        def submitter():
            t0 = time.perf_counter()
            for (t, s), at in zip(reqs[:20], arrivals):
                dt = at - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                order.append(srv.submit(t, s))

        th = threading.Thread(target=submitter)
        th.start()
        deadline = time.time() + 120
        while len(done) < 20 and time.time() < deadline:
            r = srv.poll()
            if r is None:
                time.sleep(0.0005)
                continue
            done[r["id"]] = r
        th.join()
        assert len(done) == 20
        for k, rid in enumerate(order):
            assert done[rid]["status"] == 0
            assert_same(done[rid]["keys"], ref[k], f"poisson request {k}")
            srv.release(rid)


def test_request_larger_than_pool_rejected(serving_setup):
    pats, reqs, table = serving_setup
    with pfac.Server(table, n_slots=2, device_bytes=8 << 20, max_request_bytes=1 << 20) as srv:
        big = np.zeros(2 << 20, np.uint8)
        with pytest.raises(pfac.PfacError) as ei:
            srv.submit(big, np.array([0, big.size], np.uint64))
        assert ei.value.status == -4


@pytest.mark.parametrize("host_bytes", ARENAS, ids=["arena", "small-arena"])
def test_requests_with_more_keys_than_their_first_buffer(host_bytes):
    # requests whose matches outnumber the server's first key estimate (one
    # key per 8 input bytes) take the re-match path: a buffer of exactly
    # their count, matched again on their slot with its status checked; they
    # share the server with ordinary requests and both kinds must give the
    # oracle's keys
    import itertools
    pats = [bytes(p) for L in range(1, 6) for p in itertools.product((0, 1), repeat=L)]
    rs = np.random.RandomState(77)
    reqs = []
    for k in range(12):
        n = int(rs.randint(2000, 60000))
        if k % 3 == 0:
            text = rs.randint(0, 2, size=n).astype(np.uint8)        # about 5 keys a byte
        else:
            text = rs.randint(0, 256, size=n).astype(np.uint8)      # a few keys
        cuts = np.sort(rs.randint(0, n + 1, size=int(rs.randint(0, 20))))
        seg = np.concatenate([[0], cuts, [n]]).astype(np.uint64)
        reqs.append((text, seg))
    with pfac.Table(pats, 256) as table:
        with pfac.Server(table, n_slots=3, device_bytes=64 << 20,
                         max_request_bytes=1 << 20, host_bytes=host_bytes) as srv:
            ids = [srv.submit(t, s) for t, s in reqs]
            got = [srv.wait(i, timeout=120) for i in ids]
            for i in ids:
                srv.release(i)
    for k, (g, (t, s)) in enumerate(zip(got, reqs)):
        assert g["status"] == 0, k
        pos, ids_ = oracle.match_ac(pats, t, s)
        ref = oracle.pack_keys(pos, ids_)
        if k % 3 == 0:
            assert ref.size > t.size // 8  # really past the first estimate
        assert_same(g["keys"], ref, f"request {k}")
