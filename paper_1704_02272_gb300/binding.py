"""ctypes binding of libpfac (argument marshalling only).

Every call forwards to the C ABI declared in include/pfac.h; all matching work
runs in the library's CUDA kernels.  There is no CPU path: if libpfac.so is
missing the import of this module raises.  PyTorch supplies device memory and
streams: texts, offsets, outputs and workspaces are CUDA tensors, and the
stream is torch's current stream unless one is given.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# PFAC_LIB may name another build of the same library (for example one
# compiled with different options); the default is the in-tree build.
LIB_PATH = os.environ.get("PFAC_LIB") or os.path.join(HERE, "_build", "libpfac.so")

ID_BITS = 24
LAYOUT_COMPRESSED, LAYOUT_DENSE = 0, 1
VARIANT_DEFAULT, VARIANT_FILTER, VARIANT_DSMEM = 0, 1, 2  # DSMEM: entries in shared memory too

STATUS = {0: "PFAC_OK", -1: "PFAC_EINVAL", -2: "PFAC_EDUP", -3: "PFAC_ESYMBOL",
          -4: "PFAC_ENOMEM", -5: "PFAC_ENOSPC", -6: "PFAC_ECUDA", -7: "PFAC_ETIMEOUT",
          -8: "PFAC_EDEVICE", -9: "PFAC_EIO", -10: "PFAC_EFORMAT"}


class PfacError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_uint32), ("prefix_depth", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("truncate_depth", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 4)]


BUILD_HOST_ONLY = 1
BUILD_SUFFIX_MERGE = 2
BUILD_WIDE_RECORDS = 4


class MatchOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("prefix_depth", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("bitmap_copies", ctypes.c_uint32),
                ("ev_scan_begin", ctypes.c_void_p), ("ev_scan_end", ctypes.c_void_p),
                ("child_masks", ctypes.c_uint32), ("gram_filter", ctypes.c_uint32),
                ("prefix_bytes", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("starts_end", ctypes.c_uint64), ("position_base", ctypes.c_uint64),
                ("ev_emit_begin", ctypes.c_void_p), ("ev_emit_end", ctypes.c_void_p),
                ("scan_kernel", ctypes.c_uint32), ("reserved_scan", ctypes.c_uint32),
                ("test_wait_limit_us", ctypes.c_uint32), ("test_withhold_slice", ctypes.c_uint32),
                ("records_per_slice", ctypes.c_uint32), ("resolver", ctypes.c_uint32)]


class TableInfo(ctypes.Structure):
    _fields_ = [("alphabet_size", ctypes.c_uint32), ("n_patterns", ctypes.c_uint32),
                ("min_len", ctypes.c_uint32), ("max_len", ctypes.c_uint32),
                ("layout", ctypes.c_uint32), ("prefix_depth", ctypes.c_uint32),
                ("trie_nodes", ctypes.c_uint64), ("trie_leaves", ctypes.c_uint64),
                ("records", ctypes.c_uint64), ("merged_leaves", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("paper_bytes", ctypes.c_uint64),
                ("dense_bytes", ctypes.c_uint64), ("output_lists", ctypes.c_uint64),
                ("output_list_words", ctypes.c_uint64), ("gram_len", ctypes.c_uint32),
                ("gram_bits", ctypes.c_uint32), ("gram_strings", ctypes.c_uint64),
                ("merged_trie_nodes", ctypes.c_uint64), ("side_entries", ctypes.c_uint64),
                ("trie_bytes", ctypes.c_uint64), ("index_bytes", ctypes.c_uint64),
                ("other_bytes", ctypes.c_uint64), ("record_bytes", ctypes.c_uint32),
                ("reserved_info", ctypes.c_uint32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("prefix_depth", ctypes.c_uint32),
                ("bitmap_copies", ctypes.c_uint32), ("child_masks", ctypes.c_uint32),
                ("n_tried", ctypes.c_uint32),
                ("scan_ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("from_cache", ctypes.c_int), ("gram_filter", ctypes.c_uint32),
                ("prefix_bytes", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("scan_kernel", ctypes.c_uint32), ("records_per_slice", ctypes.c_uint32),
                ("resolver", ctypes.c_uint32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("prefix_depth", ctypes.c_uint32),
                ("bitmap_copies", ctypes.c_uint32), ("child_masks", ctypes.c_uint32),
                ("gram_filter", ctypes.c_uint32), ("gram_bits", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_uint32), ("prefix_bytes", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_uint32), ("scan_kernel", ctypes.c_uint32),
                ("records_per_slice", ctypes.c_uint32), ("resolver", ctypes.c_uint32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("max_request_bytes", ctypes.c_uint64),
                ("host_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 3)]


class ResultC(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("in_arena", ctypes.c_int32), ("n_keys", ctypes.c_uint64),
                ("keys", ctypes.POINTER(ctypes.c_uint64)), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("t_issued", ctypes.c_double), ("t_counted", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpfac.so is not built ({LIB_PATH}); run "
                          "`python paper_1704_02272_gb300/build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u8p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8)
    u32, u64 = ctypes.c_uint32, ctypes.c_uint64
    lib.pfac_build.restype = ctypes.c_int
    lib.pfac_build.argtypes = [ctypes.POINTER(u8p), ctypes.POINTER(u32), u32, u32,
                               ctypes.POINTER(BuildOpts), vp, ctypes.POINTER(vp)]
    lib.pfac_workspace_bytes.restype = ctypes.c_int
    lib.pfac_workspace_bytes.argtypes = [vp, u64, u32, ctypes.POINTER(MatchOpts),
                                         ctypes.POINTER(u64)]
    lib.pfac_match_plan.restype = ctypes.c_int
    lib.pfac_match_plan.argtypes = [vp, ctypes.POINTER(MatchOpts), ctypes.POINTER(PlanInfo)]
    lib.pfac_match_host.restype = ctypes.c_int
    lib.pfac_match_host.argtypes = [vp, vp, u64, vp, u32, vp, u64, ctypes.POINTER(u64), u64,
                                    ctypes.POINTER(MatchOpts), vp]
    lib.pfac_verify.restype = ctypes.c_int
    lib.pfac_verify.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp, vp]
    lib.pfac_match_host_release.restype = None
    lib.pfac_match_host_release.argtypes = []
    lib.pfac_match_async.restype = ctypes.c_int
    lib.pfac_match_async.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp, vp, u64,
                                     ctypes.POINTER(MatchOpts), vp]
    lib.pfac_match.restype = ctypes.c_int
    lib.pfac_match.argtypes = [vp, vp, u64, vp, u32, vp, u64, ctypes.POINTER(u64),
                               ctypes.POINTER(MatchOpts), vp]
    lib.pfac_match_noalloc.restype = ctypes.c_int
    lib.pfac_match_noalloc.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp,
                                       ctypes.POINTER(MatchOpts), vp]
    lib.pfac_autotune.restype = ctypes.c_int
    lib.pfac_autotune.argtypes = [vp, vp, u64, vp, u32, ctypes.c_char_p, vp,
                                  ctypes.POINTER(TuneResult)]
    lib.pfac_server_create.restype = ctypes.c_int
    lib.pfac_server_create.argtypes = [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.pfac_server_submit.restype = ctypes.c_int
    lib.pfac_server_submit.argtypes = [vp, vp, u64, vp, u32, ctypes.POINTER(u64)]
    lib.pfac_server_wait.restype = ctypes.c_int
    lib.pfac_server_wait.argtypes = [vp, u64, ctypes.c_double, ctypes.POINTER(ResultC)]
    lib.pfac_server_poll.restype = ctypes.c_int
    lib.pfac_server_poll.argtypes = [vp, ctypes.POINTER(ResultC)]
    lib.pfac_server_release.restype = ctypes.c_int
    lib.pfac_server_release.argtypes = [vp, u64]
    lib.pfac_server_destroy.restype = None
    lib.pfac_server_destroy.argtypes = [vp]
    lib.pfac_table_info.restype = ctypes.c_int
    lib.pfac_table_info.argtypes = [vp, ctypes.POINTER(TableInfo)]
    lib.pfac_table_save.restype = ctypes.c_int
    lib.pfac_table_save.argtypes = [vp, ctypes.c_char_p]
    lib.pfac_table_load.restype = ctypes.c_int
    lib.pfac_table_load.argtypes = [ctypes.c_char_p, u32, vp, ctypes.POINTER(vp)]
    lib.pfac_table_free.restype = None
    lib.pfac_table_free.argtypes = [vp]
    lib.pfac_status_str.restype = ctypes.c_char_p
    lib.pfac_status_str.argtypes = [ctypes.c_int]
    lib.pfac_last_error.restype = ctypes.c_int
    lib.pfac_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.pfac_version.restype = ctypes.c_int
    lib.pfac_version.argtypes = []
    return lib


LIB = _load()


def _check(rc: int):
    if rc != 0:
        buf = ctypes.create_string_buffer(512)
        LIB.pfac_last_error(buf, 512)
        raise PfacError(rc, buf.value.decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


KERNEL_QUEUED, KERNEL_REGISTER, KERNEL_SERIAL = 1, 2, 3


def _opts(variant=0, prefix_depth=0, ctas_per_sm=0, bitmap_copies=0, child_masks=0,
          gram_filter=0, prefix_bytes=0, starts_end=0, position_base=0, warps_per_cta=0,
          scan_kernel=0, scan_events=None, emit_events=None, test_wait_limit_us=0,
          test_withhold_slice=0, records_per_slice=0, resolver=0):
    o = MatchOpts()
    o.variant, o.prefix_depth, o.ctas_per_sm = variant, prefix_depth, ctas_per_sm
    o.bitmap_copies, o.child_masks, o.gram_filter = bitmap_copies, child_masks, gram_filter
    o.prefix_bytes, o.starts_end, o.position_base = prefix_bytes, starts_end, position_base
    o.warps_per_cta, o.scan_kernel = warps_per_cta, scan_kernel
    o.test_wait_limit_us, o.test_withhold_slice = test_wait_limit_us, test_withhold_slice
    o.records_per_slice = records_per_slice
    o.resolver = resolver
    if scan_events is not None:  # (begin, end) torch.cuda.Event pair
        o.ev_scan_begin = scan_events[0].cuda_event
        o.ev_scan_end = scan_events[1].cuda_event
    if emit_events is not None:  # around the scan kernel's emit launch
        o.ev_emit_begin = emit_events[0].cuda_event
        o.ev_emit_end = emit_events[1].cuda_event
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


class Table:
    """A built matching table (pfac_build); device memory owned by libpfac."""

    def __init__(self, patterns, alphabet_size: int, layout: int = LAYOUT_COMPRESSED,
                 prefix_depth: int = 0, stream=None, host_only: bool = False,
                 truncate_depth: int = 0, suffix_merge: bool = False,
                 wide_records: bool = False):
        n = len(patterns)
        bufs = [ctypes.create_string_buffer(bytes(p), len(p)) for p in patterns]
        arr = (ctypes.POINTER(ctypes.c_uint8) * max(n, 1))()
        lens = (ctypes.c_uint32 * max(n, 1))()
        for i, (b, p) in enumerate(zip(bufs, patterns)):
            arr[i] = ctypes.cast(b, ctypes.POINTER(ctypes.c_uint8))
            lens[i] = len(p)
        o = BuildOpts()
        o.layout, o.prefix_depth = layout, prefix_depth
        o.flags = ((BUILD_HOST_ONLY if host_only else 0) | (BUILD_SUFFIX_MERGE if suffix_merge else 0)
                   | (BUILD_WIDE_RECORDS if wide_records else 0))
        o.truncate_depth = truncate_depth
        h = ctypes.c_void_p()
        st = 0 if host_only else _stream(stream)
        _check(LIB.pfac_build(arr, lens, n, alphabet_size, ctypes.byref(o),
                              ctypes.c_void_p(st), ctypes.byref(h)))
        self._h = h
        self.alphabet_size = alphabet_size
        self.layout = layout

    @classmethod
    def load(cls, path, stream=None, host_only: bool = False) -> "Table":
        """pfac_table_load: the table a pfac_table_save wrote to path, uploaded
        to the current device (or kept on the host with host_only)."""
        h = ctypes.c_void_p()
        st = 0 if host_only else _stream(stream)
        _check(LIB.pfac_table_load(os.fsencode(path), BUILD_HOST_ONLY if host_only else 0,
                                   ctypes.c_void_p(st), ctypes.byref(h)))
        t = cls.__new__(cls)
        t._h = h
        i = t.info()
        t.alphabet_size, t.layout = i["alphabet_size"], i["layout"]
        return t

    def save(self, path) -> None:
        """pfac_table_save: writes the table (and its tuned defaults) to path."""
        _check(LIB.pfac_table_save(self.handle, os.fsencode(path)))

    @property
    def handle(self):
        if not self._h:
            raise ValueError("table is closed")
        return self._h

    def info(self) -> dict:
        i = TableInfo()
        _check(LIB.pfac_table_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in TableInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            LIB.pfac_table_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def autotune(table: Table, text: torch.Tensor, seg: torch.Tensor, cache_path=None,
             stream=None) -> dict:
    """pfac_autotune on a device-resident sample; returns the choice."""
    r = TuneResult()
    n_seg = max(seg.numel() - 1, 0)
    cp = cache_path.encode() if cache_path else None
    _check(LIB.pfac_autotune(table.handle, _ptr(text), text.numel(), _ptr(seg), n_seg, cp,
                             ctypes.c_void_p(_stream(stream)), ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def workspace_bytes(table: Table, n_bytes: int, n_segments: int, **opt) -> int:
    b = ctypes.c_uint64()
    o = _opts(**opt)
    _check(LIB.pfac_workspace_bytes(table.handle, n_bytes, n_segments, ctypes.byref(o),
                                    ctypes.byref(b)))
    return b.value


def plan(table: Table, **opt) -> dict:
    """pfac_match_plan: the scan configuration a match with these options uses."""
    o = _opts(**opt)
    r = PlanInfo()
    _check(LIB.pfac_match_plan(table.handle, ctypes.byref(o), ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in PlanInfo._fields_ if f != "reserved"}


def match_host(table: Table, text: torch.Tensor, seg: torch.Tensor, out: torch.Tensor,
               chunk_bytes: int = 0, stream=None, **opt) -> int:
    """pfac_match_host: text (uint8), segment offsets (int64) and the key
    buffer (int64) in host memory (pinned for overlapped copies); returns the
    total count (raises PfacError with status PFAC_ENOSPC when it exceeds
    out.numel(), as pfac_match)."""
    for x in (text, seg, out):
        if x.device.type != "cpu" or not x.is_contiguous():
            raise ValueError("match_host takes contiguous host tensors")
    n = ctypes.c_uint64(0)
    o = _opts(**opt)
    rc = LIB.pfac_match_host(table.handle, _ptr(text), text.numel(), _ptr(seg),
                             max(seg.numel() - 1, 0), _ptr(out), out.numel(), ctypes.byref(n),
                             chunk_bytes, ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    _check(rc)
    return n.value


def verify_into(table: Table, text: torch.Tensor, seg: torch.Tensor, cand: torch.Tensor,
                out: torch.Tensor, cnt: torch.Tensor, stream=None) -> None:
    """pfac_verify, stream-ordered: the exact matches among the candidates go
    to out (room for cand.numel() keys), their number to cnt (device int64)."""
    _check(LIB.pfac_verify(table.handle, _ptr(text), text.numel(), _ptr(seg),
                           max(seg.numel() - 1, 0), _ptr(cand), cand.numel(), _ptr(out), _ptr(cnt),
                           ctypes.c_void_p(_stream(stream))))


def verify(table: Table, text: torch.Tensor, seg: torch.Tensor, cand: torch.Tensor,
           stream=None) -> torch.Tensor:
    """pfac_verify: the exact matches among prefix-matching candidates of a
    table built with truncate_depth (all on the device)."""
    out = torch.empty(max(cand.numel(), 1), dtype=torch.int64, device=cand.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=cand.device)
    verify_into(table, text, seg, cand, out, cnt, stream=stream)
    if stream is not None:
        stream.synchronize()
    else:
        torch.cuda.synchronize(cand.device)
    return out[:int(cnt.item())]


def _check_device_args(who: str, text: torch.Tensor, args) -> None:
    """Every tensor handed to the library as a raw pointer must have the dtype
    and layout the C ABI reads it with, on the text's CUDA device; otherwise
    the kernels would read or write past a smaller buffer."""
    for x, name, dt, optional in args:
        if x is None and optional:
            continue
        if x is None or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"{who}: {name} must be a contiguous {dt} tensor")
    if text.device.type != "cuda":
        raise ValueError(f"{who} takes the text on a CUDA device")
    for x, name, _, _ in args:
        if x is not None and x.device != text.device:
            raise ValueError(f"{who}: {name} must be on {text.device}, like the text")


def match_async(table: Table, text: torch.Tensor, seg: torch.Tensor, out: torch.Tensor,
                count: torch.Tensor, status: torch.Tensor, workspace: torch.Tensor,
                stream=None, **opt):
    """pfac_match_async: everything stays on the device (graph-capturable)."""
    _check_device_args("match_async", text, (
        (text, "text", torch.uint8, False), (seg, "segment offsets", torch.int64, False),
        (out, "output", torch.int64, True), (count, "count", torch.int64, False),
        (status, "status", torch.int32, True), (workspace, "workspace", torch.uint8, False)))
    o = _opts(**opt)
    n_seg = max(seg.numel() - 1, 0)
    with torch.cuda.device(text.device):
        _check(LIB.pfac_match_async(table.handle, _ptr(text), text.numel(), _ptr(seg), n_seg,
                                    _ptr(out), out.numel() if out is not None else 0,
                                    _ptr(count), _ptr(status), _ptr(workspace),
                                    workspace.numel(), ctypes.byref(o),
                                    ctypes.c_void_p(_stream(stream))))


def match_noalloc(table: Table, text: torch.Tensor, seg: torch.Tensor, out: torch.Tensor,
                  count: torch.Tensor, status: torch.Tensor, stream=None, **opt):
    """pfac_match_noalloc: like match_async, but the library uses its built-in
    scratch array instead of a workspace, so nothing is allocated."""
    _check_device_args("match_noalloc", text, (
        (text, "text", torch.uint8, False), (seg, "segment offsets", torch.int64, False),
        (out, "output", torch.int64, True), (count, "count", torch.int64, False),
        (status, "status", torch.int32, True)))
    o = _opts(**opt)
    n_seg = max(seg.numel() - 1, 0)
    with torch.cuda.device(text.device):
        _check(LIB.pfac_match_noalloc(table.handle, _ptr(text), text.numel(), _ptr(seg), n_seg,
                                      _ptr(out), out.numel() if out is not None else 0,
                                      _ptr(count), _ptr(status), ctypes.byref(o),
                                      ctypes.c_void_p(_stream(stream))))


def match_into(table: Table, text: torch.Tensor, seg: torch.Tensor, out: torch.Tensor,
               stream=None, **opt) -> int:
    """pfac_match: writes min(count, capacity) sorted keys into ``out`` and
    returns the total count (PfacError PFAC_ENOSPC when it does not fit)."""
    if text.device.type != "cuda":
        raise ValueError("match takes the text on a CUDA device (match_host takes host buffers)")
    for x, name, dt in ((text, "text", torch.uint8), (seg, "segment offsets", torch.int64),
                        (out, "output", torch.int64)):
        if x is None and name == "output":
            continue
        if x.dtype != dt or not x.is_contiguous() or x.device != text.device:
            raise ValueError(f"match: {name} must be a contiguous {dt} tensor on {text.device}")
    o = _opts(**opt)
    n = ctypes.c_uint64()
    n_seg = max(seg.numel() - 1, 0)
    with torch.cuda.device(text.device):
        rc = LIB.pfac_match(table.handle, _ptr(text), text.numel(), _ptr(seg), n_seg, _ptr(out),
                            out.numel() if out is not None else 0, ctypes.byref(n),
                            ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    if rc == -5:
        err = PfacError(rc, f"{n.value} matches exceed capacity {out.numel()}")
        err.count = n.value
        raise err
    _check(rc)
    return n.value


def match(table: Table, text: torch.Tensor, seg: torch.Tensor, capacity: int = None,
          stream=None, **opt) -> torch.Tensor:
    """Sorted match keys (int64 tensor on the text's device); grows the output
    buffer once if the first capacity was too small."""
    dev = text.device
    cap = capacity if capacity is not None else max(1024, text.numel() // 64)
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    try:
        n = match_into(table, text, seg, out, stream=stream, **opt)
    except PfacError as e:
        if e.status != -5:
            raise
        out = torch.empty(e.count, dtype=torch.int64, device=dev)
        n = match_into(table, text, seg, out, stream=stream, **opt)
    return out[:n]


def unpack(keys: torch.Tensor):
    """(positions, pattern ids) of packed keys."""
    return keys >> ID_BITS, keys & ((1 << ID_BITS) - 1)


def single_segment(n_bytes: int, device) -> torch.Tensor:
    return torch.tensor([0, n_bytes], dtype=torch.int64, device=device)


def version() -> int:
    return LIB.pfac_version()


class Server:
    """pfac_server_*: continuous batching over a resident table.  Host buffers
    passed to submit() are kept alive here until release()."""

    def __init__(self, table: Table, n_slots: int = 4, device_bytes: int = 1 << 30,
                 max_request_bytes: int = 0, host_bytes: int = 0):
        o = ServerOpts()
        o.n_slots, o.device_bytes, o.max_request_bytes = n_slots, device_bytes, max_request_bytes
        o.host_bytes = host_bytes
        h = ctypes.c_void_p()
        _check(LIB.pfac_server_create(table.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._table = table
        self._bufs = {}

    def submit(self, text, seg) -> int:
        """text: host uint8 array/tensor; seg: host uint64/int64 offsets."""
        import numpy as np
        if isinstance(text, torch.Tensor):
            t_ptr, n = text.data_ptr(), text.numel()
        else:
            text = np.ascontiguousarray(text, dtype=np.uint8)
            t_ptr, n = text.ctypes.data, text.size
        if isinstance(seg, torch.Tensor):
            s_ptr, ns = seg.data_ptr(), seg.numel()
        else:
            seg = np.ascontiguousarray(seg, dtype=np.uint64)
            s_ptr, ns = seg.ctypes.data, seg.size
        rid = ctypes.c_uint64()
        _check(LIB.pfac_server_submit(self._h, ctypes.c_void_p(t_ptr if n else 0), n,
                                      ctypes.c_void_p(s_ptr), max(ns - 1, 0), ctypes.byref(rid)))
        self._bufs[rid.value] = (text, seg)
        return rid.value

    @staticmethod
    def _result(r: ResultC, copy: bool = True) -> dict:
        """The result as a dict; keys copied out, or with copy=False a view of
        the server's memory that is valid until release()."""
        import numpy as np
        if r.n_keys:
            keys = np.ctypeslib.as_array(r.keys, shape=(r.n_keys,))
            if copy:
                keys = keys.copy()
        else:
            keys = np.zeros(0, np.uint64)
        return {"id": r.id, "status": r.status, "keys": keys, "in_arena": bool(r.in_arena),
                "t_submit": r.t_submit,
                "t_admit": r.t_admit, "t_done": r.t_done, "t_issued": r.t_issued,
                "t_counted": r.t_counted}

    def wait(self, rid: int, timeout: float = 0.0, copy: bool = True) -> dict:
        r = ResultC()
        _check(LIB.pfac_server_wait(self._h, rid, timeout, ctypes.byref(r)))
        return self._result(r, copy)

    def poll(self, copy: bool = True):
        r = ResultC()
        rc = LIB.pfac_server_poll(self._h, ctypes.byref(r))
        if rc == 1:
            return None
        _check(rc)
        return self._result(r, copy)

    def release(self, rid: int):
        _check(LIB.pfac_server_release(self._h, rid))
        self._bufs.pop(rid, None)

    def close(self):
        if getattr(self, "_h", None):
            LIB.pfac_server_destroy(self._h)
            self._h = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
