"""GPU parity of tables taken from a file (pfac_table_save / pfac_table_load):
a device table saved and loaded back, and a table built on the host only
and loaded onto the device, match exactly what the oracle finds; the record
formats, the dense layout and the merged trie come back whole; a tuned
table keeps its tuned plan."""
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")

KINDS = {
    "packed": {},
    "wide-records": dict(wide_records=True),
    "dense": dict(layout=pfac.LAYOUT_DENSE),
    "suffix-merge": dict(suffix_merge=True),
}


@pytest.mark.parametrize("kind", list(KINDS))
def test_saved_device_table_matches_oracle(tmp_path, kind):
    w = workloads.tiny_case(611, 4, 1200, 4, 24, 600_001, n_segments=7, n_plants=1500)
    ref = oracle_keys(w)
    assert ref.size > 0
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 4, **KINDS[kind]) as t:
        before = keys_np(pfac.match(t, text, seg))
        info = t.info()
        t.save(tmp_path / "t.pfac")
    assert_same(before, ref, f"{kind} built")
    with pfac.Table.load(tmp_path / "t.pfac") as u:
        assert u.info() == info
        assert_same(keys_np(pfac.match(u, text, seg)), ref, f"{kind} loaded")


@pytest.mark.parametrize("sigma", [4, 20, 256])
def test_host_built_table_on_device(tmp_path, sigma):
    """Built on the host only (as a machine without a GPU would), matched on
    the device after a load."""
    w = workloads.tiny_case(612 + sigma, sigma, 800, 2, 16, 500_000, n_segments=3, n_plants=1200)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, sigma, host_only=True) as t:
        t.save(tmp_path / "h.pfac")
        info = t.info()
    with pfac.Table.load(tmp_path / "h.pfac") as u:
        assert u.info() == info
        assert_same(keys_np(pfac.match(u, text, seg)), ref, f"sigma {sigma} host-built")


def test_tuned_plan_survives(tmp_path):
    w = workloads.tiny_case(613, 20, 1000, 3, 20, 4_000_000, n_plants=2000)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 20) as t:
        pfac.autotune(t, text, seg)
        tuned = pfac.plan(t)
        t.save(tmp_path / "t.pfac")
    with pfac.Table.load(tmp_path / "t.pfac") as u:
        assert pfac.plan(u) == tuned
        assert_same(keys_np(pfac.match(u, text, seg)), ref, "tuned, loaded")
    torch.cuda.synchronize()
