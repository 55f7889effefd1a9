"""Failure path of the bounded device waits, made to run without a GPU fault:
the queued scan kernel is told never to issue one slice's bulk copy, so its
wait on that stage's mbarrier runs out after a short bound (1 ms here).  The
kernel records PFAC_ETIMEOUT, waits (bounded) for its other copies and
returns; the call reports the status and the device stays usable: the next
call on the same table and stream gives the oracle's keys."""
import pytest
import torch

import workloads
from tests.gpu_util import assert_same, keys_np, oracle_keys, to_device

pytestmark = pytest.mark.gpu

pfac = pytest.importorskip("paper_1704_02272_gb300")

ETIMEOUT = -7


@pytest.mark.parametrize("sigma,slice_no", [(4, 1), (4, 3000), (256, 77)])
def test_bounded_wait_gives_up_and_device_stays_usable(sigma, slice_no):
    w = workloads.tiny_case(500 + sigma, sigma, 300, 3, 12, 4 << 20, n_plants=500)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, sigma) as t:
        with pytest.raises(pfac.PfacError) as ei:
            pfac.match(t, text, seg, scan_kernel=1, test_withhold_slice=slice_no,
                       test_wait_limit_us=1000)
        assert ei.value.status == ETIMEOUT, str(ei.value)
        keys = pfac.match(t, text, seg, scan_kernel=1)
        torch.cuda.synchronize()
        assert_same(keys_np(keys), ref, "after the timeout")


def test_testing_aids_off_change_nothing():
    w = workloads.tiny_case(520, 4, 300, 3, 12, 1 << 20, n_plants=300)
    ref = oracle_keys(w)
    text, seg = to_device(w)
    with pfac.Table(w.patterns, 4) as t:
        # a short bound alone, with every copy issued, still completes
        keys = pfac.match(t, text, seg, test_wait_limit_us=200_000)
        torch.cuda.synchronize()
        assert_same(keys_np(keys), ref, "short bound")
