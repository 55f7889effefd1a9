"""Shared helpers of the GPU parity tests: move a workload to the device, run
the library through its C ABI, and compute the oracle's keys."""
import numpy as np
import torch

import oracle


def device():
    return torch.device("cuda:0")


def to_device(w):
    dev = device()
    text = torch.from_numpy(np.ascontiguousarray(w.text)).to(dev)
    seg = torch.from_numpy(np.asarray(w.seg_offsets, dtype=np.uint64).astype(np.int64)).to(dev)
    return text, seg


def keys_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def oracle_keys(w, lo=0, hi=None, ac=None):
    if ac is None:
        pos, ids = oracle.match_ac(w.patterns, w.text, w.seg_offsets, lo=lo, hi=hi)
    else:
        pos, ids = ac.match(w.text, w.seg_offsets, lo=lo, hi=hi)
    return oracle.pack_keys(pos, ids)


def window(keys_dev: torch.Tensor, lo: int, hi: int, id_bits=24) -> np.ndarray:
    """Device keys whose position lies in [lo, hi) (keys are sorted)."""
    b = torch.tensor([lo << id_bits, hi << id_bits], dtype=torch.int64, device=keys_dev.device)
    a, z = torch.searchsorted(keys_dev, b).tolist()
    return keys_np(keys_dev[a:z])


def assert_same(got: np.ndarray, ref: np.ndarray, what=""):
    if got.shape == ref.shape and np.array_equal(got, ref):
        return
    n = min(got.shape[0], ref.shape[0])
    diff = np.flatnonzero(got[:n] != ref[:n])
    first = int(diff[0]) if diff.size else n
    ctx = lambda a: [(int(k) >> 24, int(k) & 0xFFFFFF) for k in a[max(0, first - 2):first + 3]]
    raise AssertionError(f"{what}: {got.shape[0]} keys vs oracle {ref.shape[0]}; first "
                         f"difference at {first}: got {ctx(got)} want {ctx(ref)}")
