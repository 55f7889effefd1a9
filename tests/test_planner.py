"""Host logic of the scan planner (pfac_match_plan, no GPU needed): over a
grid of tables and every combination of the tuning options, a plan either
fits the 232,448-byte shared-memory limit of an sm_103a CTA and honours every
option the caller fixed, or the call fails cleanly with PFAC_EINVAL."""
import itertools

import numpy as np

import pytest

import workloads

pfac = pytest.importorskip("paper_1704_02272_gb300")

SMEM_LIMIT = 232448
EINVAL = -1
GRID = [(s, n) for s in (4, 20, 64, 256) for n in (100, 1000, 10000)]


def host_table(sigma, n):
    w = workloads.config4(sigma, n, n_bytes=1 << 12)
    return pfac.Table(w.patterns, w.sigma, host_only=True)


def held_depths(t):
    ks = []
    for k in range(1, 21):
        try:
            pfac.plan(t, prefix_depth=k)
            ks.append(k)
        except pfac.PfacError as e:
            assert e.status == EINVAL
    return ks


@pytest.mark.parametrize("sigma,n", GRID, ids=[f"sig{s}-n{n}" for s, n in GRID])
def test_plans_fit_and_honour_options(sigma, n):
    with host_table(sigma, n) as t:
        info = t.info()
        ks = held_depths(t)
        assert ks and ks == list(range(ks[0], ks[-1] + 1)) and len(ks) <= 3
        assert info["prefix_depth"] in ks
        default = pfac.plan(t)
        assert default["smem_bytes"] <= SMEM_LIMIT
        n_ok = 0
        for k, var, masks, gram, pbytes, nw, copies in itertools.product(
                ks, (0, 1, 2), (0, 1, 2), (0, 1, 2), (0, 1, 2), (0, 16, 24), (0, 1, 2, 32)):
            opt = dict(prefix_depth=k, variant=var, child_masks=masks, gram_filter=gram,
                       prefix_bytes=pbytes, warps_per_cta=nw, bitmap_copies=copies)
            try:
                p = pfac.plan(t, **opt)
            except pfac.PfacError as e:
                assert e.status == EINVAL, opt
                continue
            n_ok += 1
            assert p["smem_bytes"] <= SMEM_LIMIT, (opt, p)
            assert p["prefix_depth"] == k
            if var:
                assert p["variant"] == var
            assert p["warps_per_cta"] == (nw or 16)  # an untuned table defaults to 16
            if masks:
                assert p["child_masks"] == masks, (opt, p)
            if gram:
                assert p["gram_filter"] == gram, (opt, p)
            if pbytes:
                assert p["prefix_bytes"] == pbytes, (opt, p)
            assert not (p["gram_filter"] == 2 and p["prefix_bytes"] == 2)
            if copies:
                assert p["bitmap_copies"] == copies, (opt, p)
            if p["gram_filter"] == 2:
                assert info["gram_len"] > 0 and 10 <= p["gram_bits"] <= info["gram_bits"]
        assert n_ok > 0


def test_invalid_options_rejected():
    with host_table(256, 1000) as t:
        for opt in (dict(warps_per_cta=20), dict(child_masks=3), dict(gram_filter=3),
                    dict(prefix_bytes=3), dict(bitmap_copies=3), dict(variant=7),
                    dict(prefix_bytes=2, gram_filter=2), dict(prefix_bytes=2, bitmap_copies=2),
                    dict(prefix_depth=21)):
            with pytest.raises(pfac.PfacError) as e:
                pfac.plan(t, **opt)
            assert e.value.status == EINVAL, opt


def test_workspace_grows_with_the_input_and_stops_at_2_40():
    with host_table(256, 1000) as t:
        sizes = [0, 1, 511, 512, 513, 1 << 20, 1 << 30, (1 << 40) - 1]
        for S in (1, 2, 1000):
            ws = [pfac.workspace_bytes(t, n, S) for n in sizes]
            assert all(a <= b for a, b in zip(ws, ws[1:])), (S, ws)
            assert all(w % 256 == 0 for w in ws)
        assert pfac.workspace_bytes(t, 1 << 20, 1000) >= pfac.workspace_bytes(t, 1 << 20, 1)
        for n in (1 << 40, 1 << 41):
            with pytest.raises(pfac.PfacError) as e:
                pfac.workspace_bytes(t, n, 1)
            assert e.value.status == EINVAL


@pytest.mark.parametrize("n", (100, 1000, 10000))
def test_register_staged_plans(n):
    # the register-staged kernel (8-bit symbols here): every option combination
    # either fits shared memory and honours the options, or fails cleanly;
    # its CTA width is fixed and it takes neither prefix bytes nor a width
    with host_table(256, n) as t:
        ks = held_depths(t)
        n_ok = 0
        for k, var, masks, gram, copies, nw in itertools.product(
                ks, (0, 1, 2), (0, 1, 2), (0, 1, 2), (0, 1, 2, 4, 8, 16, 32), (0, 24)):
            opt = dict(prefix_depth=k, variant=var, child_masks=masks, gram_filter=gram,
                       bitmap_copies=copies, scan_kernel=2, warps_per_cta=nw)
            try:
                p = pfac.plan(t, **opt)
            except pfac.PfacError as e:
                assert e.status == EINVAL, opt
                continue
            n_ok += 1
            assert p["scan_kernel"] == 2 and p["warps_per_cta"] == (nw or 16), (opt, p)
            assert p["smem_bytes"] <= SMEM_LIMIT and p["prefix_bytes"] == 1, (opt, p)
            assert p["prefix_depth"] == k
            for key, val in (("variant", var), ("child_masks", masks), ("gram_filter", gram),
                             ("bitmap_copies", copies)):
                if val:
                    assert p[key] == val, (opt, p)
            assert p["bitmap_copies"] <= 16
        assert n_ok > 0
        for opt in (dict(scan_kernel=2, prefix_bytes=2), dict(scan_kernel=2, warps_per_cta=20),
                    dict(scan_kernel=3)):
            with pytest.raises(pfac.PfacError) as e:
                pfac.plan(t, **opt)
            assert e.value.status == EINVAL, opt
        assert pfac.plan(t, scan_kernel=1)["scan_kernel"] == 1


def test_register_staged_kernel_needs_8_or_2_bit_symbols():
    for sigma in (20, 64):
        with host_table(sigma, 1000) as t:
            assert pfac.plan(t)["scan_kernel"] == 1
            with pytest.raises(pfac.PfacError) as e:
                pfac.plan(t, scan_kernel=2)
            assert e.value.status == EINVAL
    with host_table(4, 1000) as t:
        assert pfac.plan(t)["scan_kernel"] == 1  # on request only, for 2-bit symbols
        assert pfac.plan(t, scan_kernel=2)["scan_kernel"] == 2


@pytest.mark.parametrize("n", (100, 1000, 10000))
def test_register_staged_plans_2_bit(n):
    with host_table(4, n) as t:
        ks = held_depths(t)
        n_ok = 0
        for k, var, masks, gram, copies in itertools.product(
                ks, (0, 1, 2), (0, 1, 2), (0, 1, 2), (0, 1, 4, 16)):
            opt = dict(prefix_depth=k, variant=var, child_masks=masks, gram_filter=gram,
                       bitmap_copies=copies, scan_kernel=2)
            try:
                p = pfac.plan(t, **opt)
            except pfac.PfacError as e:
                assert e.status == EINVAL, opt
                continue
            n_ok += 1
            assert p["scan_kernel"] == 2 and p["smem_bytes"] <= SMEM_LIMIT, (opt, p)
            assert p["prefix_depth"] == k
        assert n_ok > 0


def _entries_by_enumeration(t, k, bps):
    """Prefix-node entries of depth k, counted over every k-symbol index: the
    walk from the root over the index's symbols (b bits each, first symbol
    lowest; values >= sigma have no child) reaches depth k, or stops earlier
    at a node on whose path some pattern ends."""
    import numpy as np
    n = t.n_nodes
    A = 1 << bps
    child = np.full((n, A), -1, dtype=np.int64)
    for v in range(n):
        for c in range(t.sigma):
            u = t.child(v, c)
            if u is not None:
                child[v, c] = u
    # a node "has output" when a pattern ends on its path from the root
    out = np.zeros(n, dtype=bool)
    for v in range(n):  # breadth-first: parents first
        if t.final_id[v] >= 0:
            out[v] = True
        for c in range(t.sigma):
            u = t.child(v, c)
            if u is not None and out[v]:
                out[u] = True
    x = np.arange(1 << (k * bps), dtype=np.int64)
    state = np.zeros(x.size, dtype=np.int64)
    alive = np.ones(x.size, dtype=bool)
    count = 0
    for i in range(k):
        sym = (x >> (bps * i)) & (A - 1)
        nxt = np.where(alive, child[state, sym], -1)
        stopped = alive & (nxt < 0)
        count += int(out[state[stopped]].sum())
        alive &= nxt >= 0
        state = np.where(alive, nxt, state)
    return count + int(alive.sum())


@pytest.mark.parametrize("seed,sigma,n,lo,hi", [(1, 200, 300, 1, 6), (2, 256, 2000, 2, 9),
                                                (3, 64, 150, 1, 5), (4, 60, 40, 2, 8),
                                                (5, 256, 30, 1, 3)])
def test_default_prefix_depth_rule(seed, sigma, n, lo, hi):
    # the builder's default depth: the shallowest depth whose entries are at
    # most 1/256 of its indices, among the depths whose entries take at most
    # a quarter of the records' bytes (64 KiB at least), else the deepest of
    # those; entries counted here by enumerating every index
    from oracle import trie as T
    pats = workloads.uniform_patterns(np.random.RandomState(seed), n, sigma, lo, hi)
    pats = list(dict.fromkeys(pats))
    t = T.build_paper_trie(pats, sigma)
    bps = max(1, (sigma - 1).bit_length())
    klim = min(max(1, 20 // bps), 16)
    kfloor = (5 + bps - 1) // bps
    with pfac.Table(pats, sigma, host_only=True) as lt:
        info = lt.info()
    budget = max(64 * 1024, info["records"] * info["record_bytes"] // 4)
    ents = {k: _entries_by_enumeration(t, k, bps) for k in range(kfloor, klim + 1)}
    kcap = max([k for k in ents if 4 * ents[k] <= budget] or [kfloor])
    want = next((k for k in range(kfloor, kcap + 1) if ents[k] * 256 <= (1 << (k * bps))), kcap)
    assert info["prefix_depth"] == want, (ents, budget)


def test_resolver_option_checked():
    pats = workloads.uniform_patterns(np.random.RandomState(3), 100, 4, 4, 12)
    with pfac.Table(pats, 4, host_only=True) as t:
        for res in (0, 1, 2):
            pfac.plan(t, resolver=res)
        with pytest.raises(pfac.PfacError):
            pfac.plan(t, resolver=3)
    with pfac.Table(pats, 4, host_only=True, suffix_merge=True) as t:
        pfac.plan(t, resolver=1)
        with pytest.raises(pfac.PfacError):
            pfac.plan(t, resolver=2)
