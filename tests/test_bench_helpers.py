"""Host logic of the benchmark script: which DRAM-traffic capture applies to
a run (the kernel sources must hash to the capture's digest and the tuned
plan must be one of the captured plans), and that the digest ignores
comments."""
import bench


def test_traffic_needs_digest_and_plan(monkeypatch):
    plan_a = {"variant": 1, "prefix_depth": 2, "bitmap_copies": 1}
    plan_b = dict(plan_a, bitmap_copies=2)
    monkeypatch.setattr(bench, "kernel_digest", lambda: "d1")
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC",
                        {"w": [(100, "d1", plan_a), (200, "d1", plan_b), (300, "d0", plan_a)]})
    assert bench.measured_traffic("w", dict(plan_a, smem_bytes=5)) == 100
    assert bench.measured_traffic("w", plan_b) == 200
    assert bench.measured_traffic("w", dict(plan_a, bitmap_copies=4)) is None
    assert bench.measured_traffic("other", plan_a) is None
    monkeypatch.setattr(bench, "kernel_digest", lambda: "d0")
    assert bench.measured_traffic("w", plan_a) == 300
    assert bench.measured_traffic("w", plan_b) is None


def test_digest_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1704_02272_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cuh"])
    (csrc / "k.cuh").write_text("int a = 1;\nint b = 2;\n")
    d0 = bench.kernel_digest()
    (csrc / "k.cuh").write_text("// note\nint a = 1;  // one\n\n/* block\n comment */int b = 2;\n")
    assert bench.kernel_digest() == d0
    (csrc / "k.cuh").write_text("int a = 1;\nint b = 3;\n")
    assert bench.kernel_digest() != d0


def test_committed_table_is_well_formed():
    for workload, entries in bench.MEASURED_TRAFFIC.items():
        assert isinstance(entries, list) and entries, workload
        for traffic, digest, plan in entries:
            assert traffic > 0 and len(digest) == 16 and plan


def test_strong_scaling_shards_cover_the_job_once():
    # the multi-GPU bench mode: every start position of the job belongs to
    # exactly one rank; each rank's text is its share plus the read halo, and
    # the oracle over the shards (positions moved by position_base, starts
    # below starts_end) concatenates to the oracle over the whole input
    import numpy as np
    import oracle
    import workloads
    full = workloads.config3(n_bytes=3 << 20, n_patterns=3000)
    ref_pos, ref_ids = oracle.match_ac(full.patterns, full.text, full.seg_offsets)
    ref = oracle.pack_keys(ref_pos, ref_ids)
    for world in (2, 3, 8):
        parts, covered = [], 0
        for rank in range(world):
            w, opt, sh = bench.shard_workload(full, world, rank)
            assert opt["position_base"] == sh.start == covered
            assert w.n_bytes - opt["starts_end"] <= full.max_len - 1
            assert w.text.ctypes.data % 16 == 0 or sh.start % 16 == 0
            covered += opt["starts_end"]
            pos, ids = oracle.match_ac(w.patterns, w.text, w.seg_offsets, hi=opt["starts_end"])
            parts.append(oracle.pack_keys(pos + np.uint64(sh.start), ids))
        assert covered == full.n_bytes
        assert np.array_equal(np.concatenate(parts), ref), world
